"""CPU oracle for the structured LQ solver over 2D grids (Zafar & Manchester,
"Structured linear quadratic control computations over 2D grids").

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, double-precision
definition that the CUDA path is checked against.  Only the test suite, the
smoke check and the benchmark's CPU-baseline leg may import it; the library
never does, and nothing here is shared with the CUDA sources.

Everything is written as explicit sparse/dense matrices following the paper's
stacked formulation, so that each function can be checked against the paper
by eye:

  * Section II-A, eq. (t_stacked_LQ_problem): A~, B~, Q~, R~, omega~
  * Section II-B, eq. (kkt_conditions) and the reduction below it:
        Delta delta = r_delta,  Delta = A~ Q~^-1 A~' + B~ R~^-1 B~',
        x = Q~^-1 A~' delta,    u = R~^-1 B~' delta
  * Section IV, eqs. (splitting_Delta), (splitting_Psi): the temporal split
        Delta = Psi~ - Xi~ and the column-pair split Psi~ = Phi~ - Omega~
  * Algorithm 2 (NBJM) with a fixed number S x L of sweeps
  * Theorem (posdef_preconditioner): the closed form D_S of Algorithm 2
  * Algorithm 1 (PCGM)
  * Section IV-B, eq. (decomposed_problem): one Cholesky factor per
    (column pair v, time t) block of Phi~

Unknown ordering.  A vector over time and grid is indexed
    idx = ((t * K + i) * N + j) * n + k
(time, then row i, then column j, then state component k; 0-based).  The
paper stacks columns first (x_bar_j = col over i); the two orders differ by a
fixed permutation, under which Delta, the masks that define Psi~/Phi~ and the
block solves are all covariant, so every quantity here equals the paper's up
to that relabelling.

Readings of the paper taken where it is silent, garbled or inconsistent
(each is also listed in the design notes):
  A1  omega~ = col(gamma, omega_0, ..., omega_{T-1}); row 0 of A~ is -I, so
      A~ x~ + B~ u~ + omega~ = 0 gives x_0 = gamma.
  A2  the factor 1/2 applies to every cost term, the terminal one included.
  A3  the returned multipliers are the delta of Delta delta = r_delta with
      r_delta = -omega~, x = Q~^-1 A~' delta, u = R~^-1 B~' delta.
  A7  Omega~ := Phi~ - Psi~ and Xi~ := Psi~ - Delta (signs inside).
  A8  inside PCG the NBJM runs exactly S x L sweeps (no epsilon exit).
  A9  PCG stops on the relative 2-norm ||r||_2 <= tol ||r_delta||_2 (mode
      "rel2"), or on the paper's absolute ||r||_inf < tol (mode "absinf").
  A10 r^(0) = r_delta - Delta delta^(0); zero iterations if it already passes.
  A16 column pairs are v = floor(j / 2) (0-based), the last pair holding one
      column when N is odd.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


# --------------------------------------------------------------------------
# Problem data and stacked matrices (Section II-A)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    K: int
    N: int
    T: int
    n: int
    m: int
    A_self: np.ndarray   # [K*N, n, n]
    A_nbr: np.ndarray    # [K*N, 4, n, n]  E (j-1), F (j+1), G (i-1), H (i+1)
    B: np.ndarray        # [K*N, n, m]
    Q: np.ndarray        # [K*N, n, n]
    R: np.ndarray        # [K*N, m, m]
    Q_T: np.ndarray      # [K*N, n, n]
    x0: np.ndarray       # [K*N, n]
    w: Optional[np.ndarray] = None   # [T, K*N, n] boundary/affine terms omega_t

    @staticmethod
    def from_arrays(K, N, T, n, m, A_self, A_nbr, B, Q, R, Q_T, x0, w=None):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        return Problem(K, N, T, n, m, f(A_self).reshape(K * N, n, n),
                       f(A_nbr).reshape(K * N, 4, n, n), f(B).reshape(K * N, n, m),
                       f(Q).reshape(K * N, n, n), f(R).reshape(K * N, m, m),
                       f(Q_T).reshape(K * N, n, n), f(x0).reshape(K * N, n),
                       None if w is None else f(w).reshape(T, K * N, n))

    @property
    def nodes(self):
        return self.K * self.N

    @property
    def dim_x(self):
        return (self.T + 1) * self.nodes * self.n

    @property
    def dim_u(self):
        return self.T * self.nodes * self.m


def grid_dynamics_matrix(P: Problem) -> sp.csr_matrix:
    """A_hat of eq. (h_stacked_LQ_problem): row block of node (i,j) holds
    A_{i,j} on the diagonal and E, F, G, H on the blocks of the neighbours
    (i,j-1), (i,j+1), (i-1,j), (i+1,j) (eq. 2d_graph_dynamics).  Neighbours
    outside the grid are the boundary states, zero here (they enter only
    through omega, Section II-A)."""
    K, N, n = P.K, P.N, P.n
    rows, cols, vals = [], [], []

    def put(p, q, blk):
        r, c = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        rows.append((p * n + r).ravel())
        cols.append((q * n + c).ravel())
        vals.append(blk.ravel())

    for i in range(K):
        for j in range(N):
            p = i * N + j
            put(p, p, P.A_self[p])
            if j - 1 >= 0:
                put(p, i * N + (j - 1), P.A_nbr[p, 0])
            if j + 1 < N:
                put(p, i * N + (j + 1), P.A_nbr[p, 1])
            if i - 1 >= 0:
                put(p, (i - 1) * N + j, P.A_nbr[p, 2])
            if i + 1 < K:
                put(p, (i + 1) * N + j, P.A_nbr[p, 3])
    size = P.nodes * n
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(size, size))


def block_diag_sparse(blocks: np.ndarray) -> sp.csr_matrix:
    """blkdiag(blocks[0], blocks[1], ...) for a stack of equal-shape blocks:
    entry (r, c) of block b sits at (b*rows + r, b*cols + c)."""
    nb, r, c = blocks.shape
    rows = np.broadcast_to(np.arange(nb)[:, None, None] * r + np.arange(r)[None, :, None], blocks.shape)
    cols = np.broadcast_to(np.arange(nb)[:, None, None] * c + np.arange(c)[None, None, :], blocks.shape)
    M = sp.csr_matrix((blocks.ravel(), (rows.ravel(), cols.ravel())), shape=(nb * r, nb * c))
    M.eliminate_zeros()
    return M


def blockwise_inverse(blocks: np.ndarray) -> np.ndarray:
    return np.linalg.inv(blocks)


@dataclasses.dataclass
class Stacked:
    """The temporally stacked QP of eq. (t_stacked_LQ_problem)."""
    At: sp.csr_matrix      # A~   [(T+1)Kn, (T+1)Kn]
    Bt: sp.csr_matrix      # B~   [(T+1)Kn, T Km]
    Qt: sp.csr_matrix      # Q~
    Rt: sp.csr_matrix      # R~
    Qt_inv: sp.csr_matrix
    Rt_inv: sp.csr_matrix
    omega: np.ndarray      # omega~ (reading A1)
    Ahat: sp.csr_matrix
    Bhat: sp.csr_matrix


def stack(P: Problem) -> Stacked:
    T, n, m, nodes = P.T, P.n, P.m, P.nodes
    Ahat = grid_dynamics_matrix(P)
    Bhat = block_diag_sparse(P.B) if m > 0 else sp.csr_matrix((nodes * n, 0))
    # A~: -I on the diagonal, A_hat on the first sub-diagonal.
    sub = sp.diags([np.ones(T)], [-1], shape=(T + 1, T + 1), format="csr")
    At = (sp.kron(sub, Ahat) - sp.identity((T + 1) * nodes * n)).tocsr()
    # B~: zero first block row, B_hat_{t} in block (t+1, t).
    sel = sp.csr_matrix((np.ones(T), (np.arange(1, T + 1), np.arange(T))), shape=(T + 1, T))
    Bt = sp.kron(sel, Bhat).tocsr()
    Qblocks = np.concatenate([np.tile(P.Q, (T, 1, 1)), P.Q_T], axis=0)
    Rblocks = np.tile(P.R, (T, 1, 1))
    Qt = block_diag_sparse(Qblocks)
    Rt = block_diag_sparse(Rblocks)
    Qt_inv = block_diag_sparse(blockwise_inverse(Qblocks))
    Rt_inv = block_diag_sparse(blockwise_inverse(Rblocks))
    omega = np.zeros((T + 1) * nodes * n)
    omega[: nodes * n] = P.x0.ravel()                 # reading A1
    if P.w is not None:
        omega[nodes * n:] = P.w.ravel()
    return Stacked(At, Bt, Qt, Rt, Qt_inv, Rt_inv, omega, Ahat, Bhat)


# --------------------------------------------------------------------------
# KKT reduction (Section II-B)
# --------------------------------------------------------------------------

def schur_matrix(S: Stacked) -> sp.csr_matrix:
    """Delta = A~ Q~^-1 A~' + B~ R~^-1 B~' (below eq. kkt_conditions)."""
    D = S.At @ S.Qt_inv @ S.At.T + S.Bt @ S.Rt_inv @ S.Bt.T
    D = D.tocsr()
    D.sum_duplicates()
    D.eliminate_zeros()
    return D


def rhs(S: Stacked) -> np.ndarray:
    """r_delta = -omega~ (eq. kkt_conditions)."""
    return -S.omega


def recover(S: Stacked, delta: np.ndarray):
    """x = Q~^-1 A~' delta and u = R~^-1 B~' delta (Section II-B)."""
    x = S.Qt_inv @ (S.At.T @ delta)
    u = S.Rt_inv @ (S.Bt.T @ delta)
    return x, u


def kkt_residual(S: Stacked, x: np.ndarray, u: np.ndarray, delta: np.ndarray) -> float:
    """Relative 2-norm of the full KKT residual (eq. kkt_conditions, with the
    multiplier sign of reading A3), normalised by ||r_delta||."""
    r1 = S.Qt @ x - S.At.T @ delta
    r2 = S.Rt @ u - S.Bt.T @ delta
    r3 = S.At @ x + S.Bt @ u + S.omega
    num = math.sqrt(r1 @ r1 + r2 @ r2 + r3 @ r3)
    den = np.linalg.norm(S.omega)
    return num / den if den > 0 else num


def cost(S: Stacked, x: np.ndarray, u: np.ndarray) -> float:
    """J = 1/2 (x~' Q~ x~ + u~' R~ u~) (eq. t_stacked_cost_function, reading A2)."""
    return 0.5 * (x @ (S.Qt @ x) + u @ (S.Rt @ u))


# --------------------------------------------------------------------------
# Splittings (Section IV, eqs. splitting_Delta and splitting_Psi)
# --------------------------------------------------------------------------

def labels(P: Problem):
    """Time t, row i, column j and column pair v of every unknown."""
    idx = np.arange(P.dim_x)
    k_rest = idx // P.n
    j = k_rest % P.N
    i = (k_rest // P.N) % P.K
    t = k_rest // (P.N * P.K)
    v = j // 2                                          # reading A16
    return t, i, j, v


def mask(M: sp.spmatrix, keep: Callable[[np.ndarray, np.ndarray], np.ndarray]) -> sp.csr_matrix:
    C = M.tocoo()
    sel = keep(C.row, C.col)
    return sp.csr_matrix((C.data[sel], (C.row[sel], C.col[sel])), shape=M.shape)


@dataclasses.dataclass
class Splitting:
    Delta: sp.csr_matrix
    Psi: sp.csr_matrix     # blkdiag_t(Psi_hat_t)
    Xi: sp.csr_matrix      # Psi~ - Delta
    Phi: sp.csr_matrix     # blkdiag_{t,v}(Phi_bar_{v,t})
    Omega: sp.csr_matrix   # Phi~ - Psi~
    groups: list           # index sets of the (v, t) diagonal blocks of Phi~


def split(P: Problem, Delta: sp.csr_matrix) -> Splitting:
    t, _, _, v = labels(P)
    Psi = mask(Delta, lambda r, c: t[r] == t[c])
    Xi = (Psi - Delta).tocsr()
    Phi = mask(Psi, lambda r, c: v[r] == v[c])
    Omega = (Phi - Psi).tocsr()
    V = (P.N + 1) // 2
    order = np.lexsort((np.arange(P.dim_x), v, t))      # group by (t, v), keep natural order inside
    key = t[order] * V + v[order]
    cuts = np.flatnonzero(np.diff(key)) + 1
    groups = np.split(order, cuts)
    return Splitting(Delta, Psi, Xi, Phi, Omega, groups)


# --------------------------------------------------------------------------
# Block solves with Phi~ (Section IV-B, eq. decomposed_problem)
# --------------------------------------------------------------------------

class PhiSolver:
    """Phi~ theta = tau as V x (T+1) independent SPD solves, one Cholesky
    factor per (v, t) block, computed once (Section IV-B).

    Inside a block the unknowns stay in their natural order (row i, then the
    pair's two columns, then component k), in which the block is banded; the
    factor is LAPACK's banded Cholesky of that band.
    """

    def __init__(self, Sp: Splitting):
        self.groups = Sp.groups
        self.factors = []
        self.flops_per_solve = 0
        # Gather the blocks once: with the unknowns listed group by group,
        # Phi~ is block diagonal with contiguous diagonal blocks.
        order = np.concatenate(Sp.groups)
        Phi_g = Sp.Phi[order][:, order].tocsr()
        start = 0
        for g in Sp.groups:
            stop = start + len(g)
            blk = Phi_g[start:stop, start:stop].toarray()
            start = stop
            bw = self._bandwidth(blk)
            band = np.zeros((bw + 1, len(g)))
            for d in range(bw + 1):
                band[d, : len(g) - d] = np.diagonal(blk, -d)
            cf = sla.cholesky_banded(band, lower=True)
            self.factors.append(cf)
            nnz_L = (bw + 1) * len(g) - bw * (bw + 1) // 2
            self.flops_per_solve += 4 * nnz_L

    @staticmethod
    def _bandwidth(blk: np.ndarray) -> int:
        r, c = np.nonzero(blk)
        return int(np.max(np.abs(r - c))) if r.size else 0

    def solve(self, tau: np.ndarray) -> np.ndarray:
        out = np.empty_like(tau)
        for g, cf in zip(self.groups, self.factors):
            out[g] = sla.cho_solve_banded((cf, True), tau[g])
        return out


# --------------------------------------------------------------------------
# Algorithm 2 (NBJM) with fixed S x L sweeps, and its closed form
# --------------------------------------------------------------------------

class Preconditioner:
    """Fixed S outer x L inner NBJM sweeps from zero starts (Algorithm 2,
    readings A8 and A21): the linear map r -> D_S r of the Theorem."""

    def __init__(self, Sp: Splitting, S: int, L: int, phi: Optional[PhiSolver] = None):
        self.Sp, self.S, self.L = Sp, S, L
        self.phi = phi if phi is not None else PhiSolver(Sp)

    def apply(self, r: np.ndarray) -> np.ndarray:
        Sp = self.Sp
        delta = np.zeros_like(r)                          # delta^(0) = 0
        for _s in range(self.S):
            r_theta = r + Sp.Xi @ delta                   # r_theta^(s) = r + Xi~ delta^(s)
            theta = np.zeros_like(r)                      # theta^(0) = 0
            for _l in range(self.L):
                theta = self.phi.solve(r_theta + Sp.Omega @ theta)   # Phi~ theta^(l+1) = r_theta + Omega~ theta^(l)
            delta = theta                                 # delta^(s+1) = theta^(L)
        return delta

    def flops(self) -> int:
        """Arithmetic of one application: every sparse product counted as
        2 nnz, every block solve as 4 nnz of its band factor, plus the vector
        additions."""
        Sp, dim = self.Sp, self.Sp.Delta.shape[0]
        per_sweep = 2 * Sp.Omega.nnz + self.phi.flops_per_solve + 2 * dim
        per_outer = 2 * Sp.Xi.nnz + dim + self.L * per_sweep
        return self.S * per_outer


def upsilon_dense(Sp: Splitting, L: int) -> np.ndarray:
    """Upsilon_L = sum_{l<L} (Phi~^-1 Omega~)^l Phi~^-1 (Lemma inverse_of_Psi)."""
    Phi = Sp.Phi.toarray()
    Om = Sp.Omega.toarray()
    Phi_inv = np.linalg.inv(Phi)
    G = Phi_inv @ Om
    U = np.zeros_like(Phi)
    term = Phi_inv.copy()
    for _ in range(L):
        U += term
        term = G @ term
    return U


def nbjm_closed_form(Sp: Splitting, S: int, L: int) -> np.ndarray:
    """D_S = sum_{s<S} (Upsilon_L Xi~)^s Upsilon_L (Theorem posdef_preconditioner)."""
    U = upsilon_dense(Sp, L)
    X = Sp.Xi.toarray()
    M = U @ X
    D = np.zeros_like(U)
    term = U.copy()
    for _ in range(S):
        D += term
        term = M @ term
    return D


@dataclasses.dataclass
class NBJMResult:
    delta: np.ndarray
    outer_iterations: int
    converged: bool


def nbjm_solve(Sp: Splitting, r_delta: np.ndarray, L: int, eps: float, max_outer: int,
               phi: Optional["PhiSolver"] = None, inner_start: str = "outer") -> NBJMResult:
    """Algorithm 2 as a solver (the paper's "standard nested block Jacobi",
    Section V): outer iterations with L inner sweeps each, until
    ||delta^(s+1) - delta^(s)||_inf < eps (its exit test; reading A8 keeps
    this exit out of the preconditioner).

    inner_start="outer" (reading A22) starts every inner iteration from the
    current outer iterate, theta^(0) = delta^(s), as the two-stage methods
    the paper cites do; its fixed point solves Delta delta = r_delta.
    inner_start="zero" is Algorithm 2 exactly as printed (theta^(0) = 0),
    whose fixed point solves (Upsilon_L^-1 - Xi~) delta = r_delta instead."""
    phi = phi if phi is not None else PhiSolver(Sp)
    delta = np.zeros_like(r_delta)
    for s in range(max_outer):
        r_theta = r_delta + Sp.Xi @ delta
        theta = delta.copy() if inner_start == "outer" else np.zeros_like(r_delta)
        for _l in range(L):
            theta = phi.solve(r_theta + Sp.Omega @ theta)
        change = np.max(np.abs(theta - delta))
        delta = theta
        if change < eps:
            return NBJMResult(delta, s + 1, True)
    return NBJMResult(delta, max_outer, False)


def lanczos_extremes(alphas, betas):
    """Extreme eigenvalues of the Lanczos tridiagonal matrix built from the
    CG coefficients (Saad, Iterative Methods, Section 6.7.3): diagonal
    1/a_0, 1/a_j + b_{j-1}/a_{j-1}; off-diagonal sqrt(b_j)/a_j."""
    a = np.asarray(alphas, dtype=np.float64)
    b = np.asarray(betas, dtype=np.float64)
    m = len(a)
    diag = 1.0 / a
    diag[1:] += b[: m - 1] / a[: m - 1]
    off = np.sqrt(b[: m - 1]) / a[: m - 1]
    ev = sla.eigvalsh_tridiagonal(diag, off)
    return ev[0], ev[-1]


# --------------------------------------------------------------------------
# Algorithm 1 (PCGM)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class PCGResult:
    delta: np.ndarray
    iterations: int
    converged: bool
    residual_history: list
    restarts: int
    alphas: list = dataclasses.field(default_factory=list)
    betas: list = dataclasses.field(default_factory=list)


def pcg(Delta: sp.csr_matrix, r_delta: np.ndarray, precond: Callable[[np.ndarray], np.ndarray],
        tol: float, max_iter: int, delta0: Optional[np.ndarray] = None,
        stop: str = "rel2", confirm_true_residual: bool = True,
        step_clock: Optional[list] = None) -> PCGResult:
    """Algorithm 1.  `stop` selects reading A9: "rel2" stops when
    ||r||_2 <= tol ||r_delta||_2, "absinf" when ||r||_inf < tol (the paper's
    test).  With confirm_true_residual the exit is re-checked on
    r_delta - Delta delta and the iteration restarts from the current delta
    if that check fails (reading A9).  A list passed as step_clock receives
    time.perf_counter() before the first pass of the loop and after every
    pass (a timing aid; it changes no arithmetic)."""
    import time
    bnorm = np.linalg.norm(r_delta)

    def passed(r):
        if stop == "absinf":
            return np.max(np.abs(r)) < tol
        return np.linalg.norm(r) <= tol * bnorm

    delta = np.zeros_like(r_delta) if delta0 is None else np.array(delta0, dtype=np.float64)
    hist = []
    alphas, betas = [], []
    it = 0
    restarts = 0
    while True:
        r = r_delta - Delta @ delta                       # initial residual
        hist.append(np.linalg.norm(r))
        if passed(r):                                     # reading A10
            return PCGResult(delta, it, True, hist, restarts, alphas, betas)
        if it >= max_iter:
            return PCGResult(delta, it, False, hist, restarts, alphas, betas)
        d = precond(r)                                    # first direction
        mu = d @ r
        converged = False
        if step_clock is not None:
            step_clock.append(time.perf_counter())
        while it < max_iter:
            y = Delta @ d                                 # operator product
            theta = mu / (y @ d)                          # step length
            alphas.append(theta)
            delta = delta + theta * d                     # iterate
            r = r - theta * y                             # residual
            it += 1
            hist.append(np.linalg.norm(r))
            if passed(r):                                 # stop test
                converged = True
                break
            q = precond(r)                                # preconditioner
            mu_new = q @ r
            betas.append(mu_new / mu)
            d = q + (mu_new / mu) * d                     # next direction
            mu = mu_new
            if step_clock is not None:
                step_clock.append(time.perf_counter())
        if not converged:
            return PCGResult(delta, it, False, hist, restarts, alphas, betas)
        if not confirm_true_residual or passed(r_delta - Delta @ delta):
            return PCGResult(delta, it, True, hist, restarts, alphas, betas)
        restarts += 1


def cg_iteration_bound(kappa: float, reduction: float) -> int:
    """Smallest k with 2((sqrt k - 1)/(sqrt k + 1))^k <= reduction: the
    standard CG energy-norm bound (Section III, eq. convergence_rate_CG_method,
    reading A13)."""
    s = math.sqrt(kappa)
    rate = (s - 1.0) / (s + 1.0)
    if rate <= 0.0:
        return 1
    return max(1, int(math.ceil(math.log(reduction / 2.0) / math.log(rate))))


# --------------------------------------------------------------------------
# One-call drivers
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Solution:
    x: np.ndarray          # [(T+1), K*N, n]
    u: np.ndarray          # [T, K*N, m]
    delta: np.ndarray      # [(T+1), K*N, n]
    iterations: int
    converged: bool
    rel_kkt: float
    cost: float
    history: list


class Oracle:
    """Builds every matrix of the method once for one problem."""

    def __init__(self, P: Problem):
        self.P = P
        self.S = stack(P)
        self.Delta = schur_matrix(self.S)
        self.r_delta = rhs(self.S)
        self._split = None
        self._phi = None

    @property
    def splitting(self) -> Splitting:
        if self._split is None:
            self._split = split(self.P, self.Delta)
        return self._split

    @property
    def phi(self) -> PhiSolver:
        if self._phi is None:
            self._phi = PhiSolver(self.splitting)
        return self._phi

    def preconditioner(self, S: int, L: int) -> Preconditioner:
        return Preconditioner(self.splitting, S, L, self.phi)

    def solve(self, tol: float, S: int = 2, L: int = 2, max_iter: int = 10000,
              delta0: Optional[np.ndarray] = None, stop: str = "rel2") -> Solution:
        pre = self.preconditioner(S, L)
        res = pcg(self.Delta, self.r_delta, pre.apply, tol, max_iter,
                  None if delta0 is None else np.ravel(delta0), stop=stop)
        return self.package(res)

    def package(self, res: PCGResult) -> Solution:
        P = self.P
        x, u = recover(self.S, res.delta)
        return Solution(x.reshape(P.T + 1, P.nodes, P.n), u.reshape(P.T, P.nodes, P.m),
                        res.delta.reshape(P.T + 1, P.nodes, P.n), res.iterations, res.converged,
                        kkt_residual(self.S, x, u, res.delta), cost(self.S, x, u),
                        res.residual_history)

    def solve_direct(self) -> Solution:
        """Brute force: the full KKT system of eq. (kkt_conditions), solved
        densely (tiny grids only)."""
        S = self.S
        nx, nu = S.At.shape[1], S.Bt.shape[1]
        Z = np.zeros
        Kkt = np.block([
            [S.Qt.toarray(), Z((nx, nu)), -S.At.T.toarray()],
            [Z((nu, nx)), S.Rt.toarray(), -S.Bt.T.toarray()],
            [S.At.toarray(), S.Bt.toarray(), Z((nx, nx))],
        ])
        b = np.concatenate([Z(nx), Z(nu), -S.omega])
        sol = np.linalg.solve(Kkt, b)
        x, u, delta = sol[:nx], sol[nx:nx + nu], sol[nx + nu:]
        P = self.P
        return Solution(x.reshape(P.T + 1, P.nodes, P.n), u.reshape(P.T, P.nodes, P.m),
                        delta.reshape(P.T + 1, P.nodes, P.n), 0, True,
                        kkt_residual(S, x, u, delta), cost(S, x, u), [])

    def step_flops(self, S: int, L: int) -> int:
        """Arithmetic of one PCG step (Algorithm 1, one pass of its loop):
        the Delta product, the preconditioner, three dot products and three
        vector updates (Table PCG_complexity_analysis)."""
        dim = self.Delta.shape[0]
        return 2 * self.Delta.nnz + self.preconditioner(S, L).flops() + 3 * 2 * dim + 3 * 2 * dim

    # Single-row evaluations for sampled checks at sizes where Delta itself
    # is too large to assemble: the row of Delta at one unknown, from the
    # product definition restricted to that row.
    def delta_row_apply(self, rows: np.ndarray, vec: np.ndarray) -> np.ndarray:
        return self.Delta[rows] @ vec


def delta_rows_matrix_free(P: Problem, rows: np.ndarray, vec: np.ndarray) -> np.ndarray:
    """(Delta vec)[rows] for large grids without assembling Delta: builds the
    stacked matrices restricted to the rows of A~ and B~ that the requested
    rows touch, then applies Delta = A~ Q~^-1 A~' + B~ R~^-1 B~' to vec on that
    support.  Same definition as schur_matrix, evaluated row by row."""
    n, nodes = P.n, P.nodes
    Ahat = grid_dynamics_matrix(P)
    Qinv = blockwise_inverse(P.Q)
    QTinv = blockwise_inverse(P.Q_T)
    Rinv = blockwise_inverse(P.R)
    Sblk = np.einsum("pab,pbc,pdc->pad", P.B, Rinv, P.B)
    V = vec.reshape(P.T + 1, nodes * n)
    out = np.empty(len(rows))
    AhT = Ahat.T.tocsr()
    for o, row in enumerate(rows):
        t, rem = divmod(int(row), nodes * n)
        # z_s = Q_s^-1 (A~' vec)_s for s in {t-1, t}; (A~' vec)_s = -vec_s + A_hat' vec_{s+1}
        def z(s):
            w = -V[s].copy()
            if s < P.T:
                w += AhT @ V[s + 1]
            blocks = QTinv if s == P.T else Qinv
            return np.einsum("pab,pb->pa", blocks, w.reshape(nodes, n)).ravel()
        zt = z(t)
        val = -zt[rem]
        if t >= 1:
            val += float((Ahat[rem] @ z(t - 1))[0])
            p, k = divmod(rem, n)
            val += Sblk[p, k] @ V[t, p * n:(p + 1) * n]
        out[o] = val
    return out


# --------------------------------------------------------------------------
# Slab-by-slab evaluation for grids too large to assemble (Section II)
# --------------------------------------------------------------------------
#
# The stacked matrices of eq. (t_stacked_LQ_problem) have a fixed pattern of
# per-slab blocks: A~ holds -I on its diagonal and A_hat in block (t, t-1);
# B~ holds B_hat in block (t, t-1) for t = 1..T and nothing in block row 0;
# Q~ = blkdiag(Q, ..., Q, Q_T) and R~ = blkdiag(R, ..., R).  The functions
# below apply the definitions of Section II-B one time slab at a time with
# these blocks, so the memory they need is a few slabs, not the assembled
# (T+1)KNn-square Delta.  They evaluate the same products as schur_matrix
# and recover, in the same order of factors.

@dataclasses.dataclass
class SlabBlocks:
    Ahat: sp.csr_matrix     # A_hat (eq. h_stacked_LQ_problem)
    AhatT: sp.csr_matrix    # A_hat'
    Bhat: sp.csr_matrix     # B_hat = blkdiag(B_{i,j})
    BhatT: sp.csr_matrix
    Qinv: sp.csr_matrix     # Q^-1 (slabs t < T)
    QTinv: sp.csr_matrix    # Q_T^-1 (slab T)
    Rinv: sp.csr_matrix     # R^-1


def slab_blocks(P: Problem) -> SlabBlocks:
    Ahat = grid_dynamics_matrix(P)
    Bhat = block_diag_sparse(P.B)
    return SlabBlocks(Ahat, Ahat.T.tocsr(), Bhat, Bhat.T.tocsr(),
                      block_diag_sparse(blockwise_inverse(P.Q)), block_diag_sparse(blockwise_inverse(P.Q_T)),
                      block_diag_sparse(blockwise_inverse(P.R)))


def rhs_slabs(P: Problem) -> np.ndarray:
    """r_delta = -omega~ as [(T+1), K*N*n] (reading A1: omega~ = col(gamma,
    omega_0, ..., omega_{T-1}))."""
    r = np.zeros((P.T + 1, P.nodes * P.n))
    r[0] = -P.x0.ravel()
    if P.w is not None:
        r[1:] = -P.w.reshape(P.T, -1)
    return r


def delta_apply_slabs(P: Problem, vec: np.ndarray, blocks: Optional[SlabBlocks] = None) -> np.ndarray:
    """Delta vec = A~ (Q~^-1 (A~' vec)) + B~ (R~^-1 (B~' vec)) (below eq.
    kkt_conditions), one time slab at a time:
        (A~' vec)_t = -vec_t + A_hat' vec_{t+1}  (t < T),   -vec_T  (t = T)
        z_t = Q_t^-1 (A~' vec)_t                 (Q_T^-1 at t = T)
        (A~ z)_0 = -z_0,   (A~ z)_t = A_hat z_{t-1} - z_t
        (B~' vec)_{t-1} = B_hat' vec_t,   (B~ R~^-1 B~' vec)_t = B_hat R^-1 B_hat' vec_t  (t >= 1).
    vec and the result are [(T+1), K*N*n] (any shape of that size in)."""
    b = blocks if blocks is not None else slab_blocks(P)
    T = P.T
    V = np.asarray(vec, dtype=np.float64).reshape(T + 1, P.nodes * P.n)
    out = np.empty_like(V)
    z_prev = None
    for t in range(T + 1):
        w = -V[t]
        if t < T:
            w = w + b.AhatT @ V[t + 1]
        z = (b.QTinv if t == T else b.Qinv) @ w
        y = -z
        if t >= 1:
            y = y + b.Ahat @ z_prev
            y = y + b.Bhat @ (b.Rinv @ (b.BhatT @ V[t]))
        out[t] = y
        z_prev = z
    return out


def recover_slabs(P: Problem, delta: np.ndarray, blocks: Optional[SlabBlocks] = None):
    """x = Q~^-1 A~' delta and u = R~^-1 B~' delta (Section II-B), slab by
    slab: x_t = Q_t^-1 (-delta_t + A_hat' delta_{t+1}) (no second term at
    t = T), u_t = R^-1 B_hat' delta_{t+1}.  Returns x [(T+1), K*N*n] and
    u [T, K*N*m]."""
    b = blocks if blocks is not None else slab_blocks(P)
    T = P.T
    D = np.asarray(delta, dtype=np.float64).reshape(T + 1, P.nodes * P.n)
    x = np.empty_like(D)
    u = np.empty((T, P.nodes * P.m))
    for t in range(T + 1):
        w = -D[t]
        if t < T:
            w = w + b.AhatT @ D[t + 1]
            u[t] = b.Rinv @ (b.BhatT @ D[t + 1])
        x[t] = (b.QTinv if t == T else b.Qinv) @ w
    return x, u


def true_residual_slabs(P: Problem, delta: np.ndarray, blocks: Optional[SlabBlocks] = None) -> float:
    """||r_delta - Delta delta||_2 / ||r_delta||_2, the relative true residual
    of the reduced system (reading A9), evaluated slab by slab."""
    b = blocks if blocks is not None else slab_blocks(P)
    r = rhs_slabs(P)
    res = r - delta_apply_slabs(P, delta, b)
    return float(np.linalg.norm(res) / np.linalg.norm(r))
