"""Algorithms 1 and 2 evaluated one time slab at a time, for grids whose
assembled Delta does not fit in memory (K = N = 256, T = 200: 52.7 M
multipliers, about 4.8 G nonzeros of Delta).

TEST INFRASTRUCTURE ONLY.  Like lq2d_oracle, this module is a plain,
double-precision CPU definition of the method that the CUDA path is checked
against and timed beside; only the tests, the smoke check and the
benchmark's CPU legs may use it, and nothing here is shared with the CUDA
sources.

It computes what lq2d_oracle computes from the explicit Delta and its masks,
from the per-slab blocks of the stacked matrices instead (Section II-B,
eq. structure_of_Delta), with Q_t = Q for t < T and Q_T at t = T:
    Delta_{t,t}   = Psi_hat_t = Q_t^-1 + [t >= 1] (A_hat Q^-1 A_hat' + B_hat R^-1 B_hat')
    Delta_{t,t-1} = -A_hat Q^-1,     Delta_{t-1,t} = -Q^-1 A_hat'
so Xi~ = Psi~ - Delta holds A_hat Q^-1 in block (t, t-1) and Q^-1 A_hat' in
block (t-1, t) (eq. splitting_Delta, reading A7).  Phi_hat_t keeps the
entries of Psi_hat_t whose row and column lie in one column pair
v = floor(j/2) (reading A16), and Omega_hat_t = Phi_hat_t - Psi_hat_t
(eq. splitting_Psi).  The blocks depend on t only through Q_t, so three
time classes exist (t = 0; 1 <= t <= T-1; t = T) and each class is formed
and factored once (reading A17); the factor of a class is applied to all of
its slabs at once.  Inside a column pair the unknowns keep their natural
order (row, column, component), in which the block is banded, and the
factor is LAPACK's banded Cholesky (Section IV-B, eq. decomposed_problem).

Algorithm 2 runs exactly S x L sweeps from zero starts (readings A8, A21),
in the same steps as lq2d_oracle.Preconditioner.apply, and Algorithm 1 is
lq2d_oracle.pcg itself, given the slab-wise product.

With workers > 1 each operator is split into contiguous ranges of time
slabs, one per worker process (spawned; the vectors live in shared memory),
so the per-(v, t) block solves and the node loops use all host cores.  The
arithmetic of every slab is the same as with workers = 1.
"""
from __future__ import annotations

import dataclasses
import multiprocessing as mp
import os
from multiprocessing import shared_memory
from typing import Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import lq2d_oracle as O


def time_class(t: int, T: int) -> int:
    """0 for t = 0, 1 for 1 <= t <= T-1, 2 for t = T (reading A17)."""
    return 0 if t == 0 else (2 if t == T else 1)


@dataclasses.dataclass
class ClassBlocks:
    Psi: sp.csr_matrix
    Phi: sp.csr_matrix
    Omega: sp.csr_matrix


class SlabSplitting:
    """The per-slab blocks of Delta, Psi~, Xi~, Phi~ and Omega~, one set per
    time class, and the banded Cholesky factors of Phi_hat per (class, v)."""

    def __init__(self, P: O.Problem, blocks: Optional[O.SlabBlocks] = None):
        self.P = P
        b = blocks if blocks is not None else O.slab_blocks(P)
        self.b = b
        AQA = (b.Ahat @ b.Qinv @ b.AhatT).tocsr()
        BRB = (b.Bhat @ b.Rinv @ b.BhatT).tocsr()
        psi = {0: b.Qinv, 1: b.Qinv + AQA + BRB, 2: b.QTinv + AQA + BRB}
        # column pair of every unknown of a slab: index (i*N + j)*n + k
        j = (np.arange(P.nodes * P.n) // P.n) % P.N
        v = j // 2
        self.v = v
        self.cls = {}
        for c, Psi in psi.items():
            Psi = Psi.tocsr()
            Psi.sum_duplicates()
            Phi = O.mask(Psi, lambda r, col: v[r] == v[col])
            Omega = (Phi - Psi).tocsr()
            self.cls[c] = ClassBlocks(Psi, Phi, Omega)
        # Xi~ blocks (t, t-1) and (t-1, t)
        self.XiL = (b.Ahat @ b.Qinv).tocsr()
        self.XiU = (b.Qinv @ b.AhatT).tocsr()
        # banded Cholesky factor of every (class, v) block of Phi_hat
        V = (P.N + 1) // 2
        self.groups = [np.flatnonzero(v == vv) for vv in range(V)]
        # the slab's unknowns listed pair by pair: block g of Phi_hat is the
        # contiguous run bounds[g] .. bounds[g+1] of this order
        self.perm = np.concatenate(self.groups)
        self.bounds = np.cumsum([0] + [len(g) for g in self.groups])
        self.factors = {}
        for c, cb in self.cls.items():
            fs = []
            for g in self.groups:
                blk = cb.Phi[g][:, g].toarray()
                r, col = np.nonzero(blk)
                bw = int(np.max(np.abs(r - col))) if r.size else 0
                band = np.zeros((bw + 1, len(g)))
                for d in range(bw + 1):
                    band[d, : len(g) - d] = np.diagonal(blk, -d)
                fs.append(sla.cholesky_banded(band, lower=True))
            self.factors[c] = fs

    def slab_classes(self, t0: int, t1: int):
        """The slabs t0 <= t < t1 grouped by time class: {class: [t, ...]}."""
        out = {}
        for t in range(t0, t1):
            out.setdefault(time_class(t, self.P.T), []).append(t)
        return out

    def phi_solve(self, tau: np.ndarray, t0: int, t1: int) -> np.ndarray:
        """theta_t = Phi_hat_t^-1 tau_t for the slabs t0..t1-1; tau is
        [t1 - t0, KNn]."""
        out = np.empty_like(tau)
        for c, ts in self.slab_classes(t0, t1).items():
            rows = np.asarray(ts) - t0
            X = np.ascontiguousarray(tau[rows][:, self.perm].T)   # [pair-ordered unknown, slab]
            Y = np.empty_like(X)
            for a, b, cf in zip(self.bounds[:-1], self.bounds[1:], self.factors[c]):
                Y[a:b] = sla.cho_solve_banded((cf, True), X[a:b], check_finite=False)
            res = np.empty((len(rows), X.shape[0]))
            res[:, self.perm] = Y.T
            out[rows] = res
        return out

    def omega_apply(self, theta: np.ndarray, t0: int, t1: int) -> np.ndarray:
        """(Omega~ theta)_t = Omega_hat_t theta_t for the slabs t0..t1-1."""
        out = np.empty_like(theta)
        for c, ts in self.slab_classes(t0, t1).items():
            rows = np.asarray(ts) - t0
            out[rows] = (self.cls[c].Omega @ theta[rows].T).T
        return out

    def xi_apply(self, delta: np.ndarray, t0: int, t1: int) -> np.ndarray:
        """(Xi~ delta)_t = A_hat Q^-1 delta_{t-1} + Q^-1 A_hat' delta_{t+1} for
        the slabs t0..t1-1; delta is the whole [(T+1), KNn] vector."""
        T = self.P.T
        out = np.zeros((t1 - t0, delta.shape[1]))
        lo = max(t0, 1)
        if lo < t1:
            out[lo - t0:] += (self.XiL @ delta[lo - 1:t1 - 1].T).T
        hi = min(t1, T)
        if t0 < hi:
            out[: hi - t0] += (self.XiU @ delta[t0 + 1:hi + 1].T).T
        return out

    def delta_apply(self, vec: np.ndarray, t0: int, t1: int) -> np.ndarray:
        """(Delta vec)_t for the slabs t0..t1-1, by the definition
        A~ Q~^-1 A~' + B~ R~^-1 B~' (as lq2d_oracle.delta_apply_slabs)."""
        b, T = self.b, self.P.T

        def z(t):
            w = -vec[t]
            if t < T:
                w = w + b.AhatT @ vec[t + 1]
            return (b.QTinv if t == T else b.Qinv) @ w

        out = np.empty((t1 - t0, vec.shape[1]))
        z_prev = z(t0 - 1) if t0 >= 1 else None
        for t in range(t0, t1):
            zt = z(t)
            y = -zt
            if t >= 1:
                y = y + b.Ahat @ z_prev
                y = y + b.Bhat @ (b.Rinv @ (b.BhatT @ vec[t]))
            out[t - t0] = y
            z_prev = zt
        return out


# --------------------------------------------------------------------------
# serial and process-parallel evaluation over ranges of slabs
# --------------------------------------------------------------------------

_W = {}   # worker state: the splitting and the attached shared arrays


def _worker_init(P: O.Problem, names, shape):
    """names: {array name: shared-memory block name}."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    _W["sp"] = SlabSplitting(P)
    _W["shm"] = {nm: shared_memory.SharedMemory(name=blk) for nm, blk in names.items()}
    _W["arr"] = {nm: np.ndarray(shape, dtype=np.float64, buffer=_W["shm"][nm].buf) for nm in names}


def _apply(S: SlabSplitting, A, task):
    """One operator on one range of slabs, arrays by name in A."""
    op, t0, t1, src, src2, dst = task
    if op == "noop":
        return
    if op == "delta":
        A[dst][t0:t1] = S.delta_apply(A[src], t0, t1)
    elif op == "xi":            # dst = src2 + Xi~ src
        A[dst][t0:t1] = A[src2][t0:t1] + S.xi_apply(A[src], t0, t1)
    elif op == "sweep0":        # dst = Phi~^-1 src
        A[dst][t0:t1] = S.phi_solve(A[src][t0:t1], t0, t1)
    elif op == "sweep":         # dst = Phi~^-1 (src2 + Omega~ src)
        A[dst][t0:t1] = S.phi_solve(A[src2][t0:t1] + S.omega_apply(A[src][t0:t1], t0, t1), t0, t1)


def _worker_task(task):
    _apply(_W["sp"], _W["arr"], task)


class SlabOracle:
    """Algorithm 1 with Algorithm 2 as preconditioner on one problem,
    evaluated slab by slab; `workers` processes share the slab ranges."""

    NAMES = ("vec_in", "vec_out", "r_theta", "theta_a", "theta_b", "delta_s")

    def __init__(self, P: O.Problem, workers: int = 1):
        self.P = P
        self.shape = (P.T + 1, P.nodes * P.n)
        self.workers = max(1, int(workers))
        self.r_delta = O.rhs_slabs(P).ravel()
        if self.workers == 1:
            self.sp = SlabSplitting(P)
            self.arr = {nm: np.zeros(self.shape) for nm in self.NAMES}
            self.pool = None
        else:
            nbytes = int(np.prod(self.shape)) * 8
            self.shm = {nm: shared_memory.SharedMemory(create=True, size=nbytes) for nm in self.NAMES}
            self.arr = {nm: np.ndarray(self.shape, dtype=np.float64, buffer=self.shm[nm].buf)
                        for nm in self.NAMES}
            ctx = mp.get_context("spawn")
            self.pool = ctx.Pool(self.workers, initializer=_worker_init,
                                 initargs=(P, {nm: self.shm[nm].name for nm in self.NAMES}, self.shape))
            self.pool.map(_worker_task, [("noop", 0, 0, None, None, None)] * self.workers)
        T1 = P.T + 1
        cuts = np.linspace(0, T1, self.workers + 1).round().astype(int)
        self.ranges = [(int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]

    def _run(self, op, src, src2, dst):
        tasks = [(op, t0, t1, src, src2, dst) for t0, t1 in self.ranges]
        if self.pool is None:
            for task in tasks:
                _apply(self.sp, self.arr, task)
        else:
            self.pool.map(_worker_task, tasks)

    # -- the two operators of Algorithm 1 ----------------------------------
    def delta_apply(self, vec: np.ndarray) -> np.ndarray:
        self.arr["vec_in"][...] = np.reshape(vec, self.shape)
        self._run("delta", "vec_in", None, "vec_out")
        return self.arr["vec_out"].ravel().copy()

    def precondition(self, r: np.ndarray, S: int, L: int) -> np.ndarray:
        """Algorithm 2 with exactly S x L sweeps from zero starts, the same
        steps as lq2d_oracle.Preconditioner.apply:
            delta^(0) = 0;  r_theta = r + Xi~ delta^(s);  theta^(0) = 0;
            theta^(l+1) = Phi~^-1 (r_theta + Omega~ theta^(l));  delta^(s+1) = theta^(L)."""
        A = self.arr
        A["vec_in"][...] = np.reshape(r, self.shape)
        A["delta_s"][...] = 0.0                                # delta^(0) = 0
        for _s in range(S):
            self._run("xi", "delta_s", "vec_in", "r_theta")   # r_theta = r + Xi~ delta^(s)
            A["theta_a"][...] = 0.0                            # theta^(0) = 0
            cur, nxt = "theta_a", "theta_b"
            for _l in range(L):
                self._run("sweep", cur, "r_theta", nxt)        # theta^(l+1) = Phi~^-1 (r_theta + Omega~ theta^(l))
                cur, nxt = nxt, cur
            A["delta_s"][...] = A[cur]                         # delta^(s+1) = theta^(L)
        return A["delta_s"].ravel().copy()

    def operator(self):
        """Delta as an object with `@`, for lq2d_oracle.pcg."""
        oracle = self

        class _Delta:
            def __matmul__(self, v):
                return oracle.delta_apply(v)

        return _Delta()

    def solve(self, tol: float, S: int = 2, L: int = 2, max_iter: int = 10000,
              confirm_true_residual: bool = True, step_clock: Optional[list] = None) -> O.PCGResult:
        return O.pcg(self.operator(), self.r_delta, lambda r: self.precondition(r, S, L), tol, max_iter,
                     confirm_true_residual=confirm_true_residual, step_clock=step_clock)

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None
            self.arr = {}
            for s in self.shm.values():
                s.close()
                s.unlink()
            self.shm = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
