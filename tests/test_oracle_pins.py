"""Pins for the CPU oracle: checks against facts fixed by the paper and by
mathematics, independent of the oracle's own assembly code.

* A per-node simulator written from the grid dynamics (Section II,
  eq. 2d_graph_dynamics) checks that the oracle's optimal (x, u) is feasible:
  this pins the stacked A~, B~, omega~ and the recovery x, u from delta.
* A finite-horizon Riccati recursion on the whole grid (a different method:
  dynamic programming, not the KKT system) pins the cost with its 1/2
  factors, the terminal weight and the sign convention of the multipliers.
* A dense solve of the full KKT system (brute force) pins the PCG result.
* The Theorem's closed form D_S pins Algorithm 2's loop structure.
* Spectral facts of Section IV pin the splittings.
* Table PCG_complexity_analysis pins the O(KNT) step count.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import lq2d_oracle as O
from paper_2304_04980_gb300 import synth


def as_problem(g, w=None):
    return O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays(), w=w)


# --------------------------------------------------------------------------
# independent per-node simulator (eq. 2d_graph_dynamics)
# --------------------------------------------------------------------------

def step_grid(P, x_t, u_t, w_t=None):
    """x_{t+1} from x_t [K*N, n] and u_t [K*N, m], node by node."""
    K, N = P.K, P.N
    out = np.zeros_like(x_t)
    for i in range(K):
        for j in range(N):
            p = i * N + j
            acc = P.A_self[p] @ x_t[p] + P.B[p] @ u_t[p]
            if j >= 1:
                acc += P.A_nbr[p, 0] @ x_t[i * N + j - 1]      # E x_{i,j-1}
            if j + 1 < N:
                acc += P.A_nbr[p, 1] @ x_t[i * N + j + 1]      # F x_{i,j+1}
            if i >= 1:
                acc += P.A_nbr[p, 2] @ x_t[(i - 1) * N + j]    # G x_{i-1,j}
            if i + 1 < K:
                acc += P.A_nbr[p, 3] @ x_t[(i + 1) * N + j]    # H x_{i+1,j}
            if w_t is not None:
                acc += w_t[p]
            out[p] = acc
    return out


def simulate(P, u, w=None):
    x = np.zeros((P.T + 1, P.nodes, P.n))
    x[0] = P.x0
    for t in range(P.T):
        x[t + 1] = step_grid(P, x[t], u[t], None if w is None else w[t])
    return x


def dense_maps(P):
    """Whole-grid A_hat, B_hat as dense matrices, read off the simulator's
    responses to unit states and unit inputs."""
    nx, nu = P.nodes * P.n, P.nodes * P.m
    zero_u = np.zeros((P.nodes, P.m))
    zero_x = np.zeros((P.nodes, P.n))
    A = np.zeros((nx, nx))
    B = np.zeros((nx, nu))
    for c in range(nx):
        e = np.zeros(nx)
        e[c] = 1.0
        A[:, c] = step_grid(P, e.reshape(P.nodes, P.n), zero_u).ravel()
    for c in range(nu):
        e = np.zeros(nu)
        e[c] = 1.0
        B[:, c] = step_grid(P, zero_x, e.reshape(P.nodes, P.m)).ravel()
    return A, B


def blkdiag(blocks):
    return sla.block_diag(*blocks)


def riccati(P):
    """Backward Riccati recursion for the whole grid as one system."""
    A, B = dense_maps(P)
    Qh, Rh, QTh = blkdiag(P.Q), blkdiag(P.R), blkdiag(P.Q_T)
    Ps = [None] * (P.T + 1)
    Ks = [None] * P.T
    Ps[P.T] = QTh
    for t in range(P.T - 1, -1, -1):
        Pn = Ps[t + 1]
        G = Rh + B.T @ Pn @ B
        Ks[t] = np.linalg.solve(G, B.T @ Pn @ A)
        Ps[t] = Qh + A.T @ Pn @ A - A.T @ Pn @ B @ Ks[t]
        Ps[t] = 0.5 * (Ps[t] + Ps[t].T)
    x = np.zeros((P.T + 1, P.nodes * P.n))
    u = np.zeros((P.T, P.nodes * P.m))
    x[0] = P.x0.ravel()
    for t in range(P.T):
        u[t] = -Ks[t] @ x[t]
        x[t + 1] = A @ x[t] + B @ u[t]
    J = 0.5 * x[0] @ Ps[0] @ x[0]
    return Ps, x, u, J


SHAPES = [  # (K, N, T, n, m): square, odd N (one-column last pair), single node, tall, wide
    (4, 4, 20, 2, 1),
    (3, 5, 6, 2, 1),
    (1, 1, 8, 3, 2),
    (5, 2, 4, 2, 2),
    (2, 3, 5, 1, 1),
]


@pytest.fixture(scope="module", params=SHAPES, ids=lambda s: "K%dN%dT%dn%dm%d" % s)
def case(request):
    K, N, T, n, m = request.param
    g = synth.random_grid(K, N, T, n, m, seed=11 + K + 3 * N + T)
    P = as_problem(g)
    orc = O.Oracle(P)
    sol = orc.solve(1e-12, 2, 2)
    return P, orc, sol


def test_solution_is_feasible_under_simulation(case):
    P, orc, sol = case
    assert sol.converged
    x_sim = simulate(P, sol.u)
    assert np.allclose(x_sim, sol.x, rtol=0, atol=1e-9 * max(1.0, np.abs(sol.x).max()))


def test_riccati_cost_controls_and_costates(case):
    P, orc, sol = case
    Ps, x_r, u_r, J_r = riccati(P)
    scale = max(1.0, abs(J_r))
    assert abs(sol.cost - J_r) <= 1e-9 * scale
    assert np.allclose(sol.u.reshape(P.T, -1), u_r, atol=1e-8 * max(1.0, np.abs(u_r).max()))
    assert np.allclose(sol.x.reshape(P.T + 1, -1), x_r, atol=1e-8 * max(1.0, np.abs(x_r).max()))
    # costate sign (reading A3): delta_t = -P_t x_t
    for t in range(P.T + 1):
        lhs = sol.delta[t].ravel()
        rhs = -Ps[t] @ x_r[t]
        assert np.allclose(lhs, rhs, atol=1e-8 * max(1.0, np.abs(rhs).max()))
    # optimal cost from the multipliers: J* = 1/2 delta' r_delta
    assert abs(0.5 * sol.delta.ravel() @ orc.r_delta - J_r) <= 1e-9 * scale


def test_pcg_matches_dense_kkt(case):
    P, orc, sol = case
    d = orc.solve_direct()
    for a, b in ((sol.delta, d.delta), (sol.x, d.x), (sol.u, d.u)):
        assert np.linalg.norm(a - b) <= 1e-9 * max(1e-300, np.linalg.norm(b))
    assert sol.rel_kkt <= 1e-11


def test_cost_is_minimal_among_feasible_perturbations(case):
    P, orc, sol = case
    rng = np.random.default_rng(5)
    Qt, Rt = blkdiag(list(np.tile(P.Q, (P.T, 1, 1))) + list(P.Q_T)), blkdiag(list(np.tile(P.R, (P.T, 1, 1))))

    def J(u):
        x = simulate(P, u)
        return 0.5 * (x.ravel() @ Qt @ x.ravel() + u.ravel() @ Rt @ u.ravel())

    J0 = J(sol.u)
    assert abs(J0 - sol.cost) <= 1e-9 * max(1.0, J0)
    for _ in range(3):
        v = rng.standard_normal(sol.u.shape)
        eps = 1e-3
        jp, jm = J(sol.u + eps * v), J(sol.u - eps * v)
        assert jp > J0 and jm > J0
        # first-order term vanishes at the optimum
        assert abs(jp - jm) / (2 * eps) <= 1e-6 * max(1.0, (jp + jm - 2 * J0) / eps ** 2)


def test_affine_terms_enter_as_omega():
    g = synth.random_grid(3, 3, 5, 2, 1, seed=3)
    w = synth.random_vector((g.T, g.nodes, g.n), seed=4)
    P = as_problem(g, w=w)
    sol = O.Oracle(P).solve(1e-12)
    x_sim = simulate(P, sol.u, w)
    assert np.allclose(x_sim, sol.x, atol=1e-9 * np.abs(sol.x).max())


def test_delta_block_structure(case):
    """eq. structure_of_Delta: Psi_0 = Q^-1, Psi_t = Q_t^-1 + A Q^-1 A' + B R^-1 B',
    Xi_t = -A Q^-1 (below the diagonal), zero beyond the first off-diagonal."""
    P, orc, sol = case
    A, B = dense_maps(P)
    Qi = np.linalg.inv(blkdiag(P.Q))
    QTi = np.linalg.inv(blkdiag(P.Q_T))
    Ri = np.linalg.inv(blkdiag(P.R))
    D = orc.Delta.toarray()
    s = P.nodes * P.n
    blk = lambda a, b: D[a * s:(a + 1) * s, b * s:(b + 1) * s]
    assert np.allclose(blk(0, 0), Qi, atol=1e-12)
    for t in range(1, P.T + 1):
        Qt_i = QTi if t == P.T else Qi
        assert np.allclose(blk(t, t), Qt_i + A @ Qi @ A.T + B @ Ri @ B.T, atol=1e-11)
    for t in range(P.T):
        assert np.allclose(blk(t + 1, t), -A @ Qi, atol=1e-12)
        assert np.allclose(blk(t, t + 1), (-A @ Qi).T, atol=1e-12)
    for t in range(P.T + 1):
        for t2 in range(P.T + 1):
            if abs(t - t2) > 1:
                assert not np.any(blk(t, t2))


def test_column_pair_blocks(case):
    """Phi~ is block diagonal with one block per (v, t), V = N/2 or (N+1)/2
    (Section II-B); each block spans its pair's columns over all rows; at t = 0
    Psi_0 = Q^-1 is node-diagonal, so Omega_0 = 0."""
    P, orc, sol = case
    Sp = orc.splitting
    V = P.N // 2 if P.N % 2 == 0 else (P.N + 1) // 2
    assert len(Sp.groups) == V * (P.T + 1)
    t_of, i_of, j_of, _ = O.labels(P)
    sizes = sorted({len(g) for g in Sp.groups})
    expect = {2 * P.K * P.n} if P.N % 2 == 0 else ({2 * P.K * P.n, P.K * P.n} if P.N > 1 else {P.K * P.n})
    assert set(sizes) == expect
    for g in Sp.groups:
        cols = sorted(set(j_of[g]))
        assert len(set(t_of[g])) == 1
        assert cols[0] % 2 == 0 and cols == list(range(cols[0], cols[0] + len(cols)))
        assert len(set(i_of[g])) == P.K
    Om = Sp.Omega.toarray()
    first = P.nodes * P.n
    assert not np.any(Om[:first, :first])
    Phi = Sp.Phi.toarray()[:first, :first]
    assert np.allclose(Phi, np.linalg.inv(blkdiag(P.Q)), atol=1e-12)


@pytest.mark.parametrize("S,L", [(1, 2), (2, 2), (3, 4), (2, 6)])
def test_nbjm_equals_theorem_closed_form_and_is_spd(S, L):
    g = synth.random_grid(3, 4, 6, 2, 1, seed=21)
    orc = O.Oracle(as_problem(g))
    D = O.nbjm_closed_form(orc.splitting, S, L)
    pre = orc.preconditioner(S, L)
    rng = np.random.default_rng(S * 10 + L)
    for _ in range(3):
        r = rng.standard_normal(D.shape[0])
        assert np.allclose(pre.apply(r), D @ r, rtol=0, atol=1e-11 * np.abs(D @ r).max())
    assert np.allclose(D, D.T, atol=1e-12 * np.abs(D).max())
    np.linalg.cholesky(0.5 * (D + D.T))          # Theorem: D_S is positive definite


def test_splittings_are_convergent_and_lemma_holds():
    g = synth.random_grid(3, 4, 5, 2, 1, seed=31)
    orc = O.Oracle(as_problem(g))
    Sp = orc.splitting
    Phi, Om, Psi, Xi = (M.toarray() for M in (Sp.Phi, Sp.Omega, Sp.Psi, Sp.Xi))
    rho = lambda M: np.max(np.abs(np.linalg.eigvals(M)))
    assert rho(np.linalg.solve(Phi, Om)) < 1.0
    assert rho(np.linalg.solve(Psi, Xi)) < 1.0
    for M in (Phi + Om, Phi - Om, Psi + Xi, Psi - Xi):      # sign-flip argument (reading A11)
        np.linalg.cholesky(M)
    # Lemma: Psi^-1 - Upsilon_L = Pi_L is positive semidefinite for even L
    for L in (2, 4):
        U = O.upsilon_dense(Sp, L)
        Pi = np.linalg.inv(Psi) - U
        assert np.linalg.eigvalsh(0.5 * (Pi + Pi.T)).min() >= -1e-10
        # Remark: Upsilon_L^-1 + Xi~ is positive definite
        np.linalg.cholesky(np.linalg.inv(U) + Xi)


def test_many_sweeps_approach_the_exact_inverse():
    """With S, L large enough for both Jacobi iterations to converge (their
    rates are the spectral radii of Section IV), D_S tends to Delta^-1 and PCG
    needs one or two steps."""
    g = synth.random_grid(3, 3, 4, 2, 1, seed=41)
    orc = O.Oracle(as_problem(g))
    Sp = orc.splitting
    rho = lambda M: np.max(np.abs(np.linalg.eigvals(M)))
    r_in = rho(np.linalg.solve(Sp.Phi.toarray(), Sp.Omega.toarray()))
    r_out = rho(np.linalg.solve(Sp.Psi.toarray(), Sp.Xi.toarray()))
    L = 2 * int(math.ceil(math.log(1e-15) / math.log(r_in) / 2.0))
    S = int(math.ceil(math.log(1e-13) / math.log(r_out)))
    D = O.nbjm_closed_form(Sp, S, L)
    Dinv = np.linalg.inv(orc.Delta.toarray())
    assert np.linalg.norm(D - Dinv) <= 1e-8 * np.linalg.norm(Dinv)
    sol = orc.solve(1e-10, S, L)
    assert sol.iterations <= 2


def test_step_arithmetic_scales_as_KNT():
    def flops(K, N, T):
        g = synth.random_grid(K, N, T, 2, 1, seed=51)
        return O.Oracle(as_problem(g)).step_flops(2, 2)

    base = flops(16, 16, 16)
    for ratio in (flops(32, 16, 16) / base, flops(16, 32, 16) / base,
                  flops(16, 16, 33) / base):
        assert 1.9 <= ratio <= 2.1, ratio


def test_conditioning_and_cg_bound_on_small_workload():
    g = synth.workload("grid4_T20")
    orc = O.Oracle(as_problem(g))
    D = orc.Delta.toarray()
    ev = np.linalg.eigvalsh(D)
    kappa = ev[-1] / ev[0]
    DS = O.nbjm_closed_form(orc.splitting, 2, 2)
    evp = sla.eigh(D, np.linalg.inv(DS), eigvals_only=True)
    kappa_p = evp[-1] / evp[0]
    # the preconditioner improves conditioning by more than an order (Section V)
    assert kappa_p < kappa / 10.0
    tol = 1e-10
    sol = orc.solve(tol, 2, 2)
    bound = O.cg_iteration_bound(kappa_p, tol / math.sqrt(kappa))
    assert sol.iterations <= bound
    assert sol.iterations <= D.shape[0]
    cg = O.pcg(orc.Delta, orc.r_delta, lambda r: r, tol, 100000)
    assert cg.iterations <= O.cg_iteration_bound(kappa, tol / math.sqrt(kappa))
    assert sol.iterations < cg.iterations


def test_zero_initial_state_and_warm_start_need_no_iterations():
    g = synth.random_grid(3, 3, 4, 2, 1, seed=61)
    orc = O.Oracle(as_problem(g.with_x0(np.zeros_like(g.x0))))
    sol = orc.solve(1e-10)
    assert sol.iterations == 0 and not np.any(sol.delta)
    orc2 = O.Oracle(as_problem(g))
    ref = orc2.solve(1e-12)
    again = orc2.solve(1e-10, delta0=ref.delta)
    assert again.iterations == 0


def test_absolute_infinity_norm_stop():
    g = synth.random_grid(3, 3, 6, 2, 1, seed=71)
    orc = O.Oracle(as_problem(g))
    sol = orc.solve(1e-9, stop="absinf")
    r = orc.r_delta - orc.Delta @ sol.delta.ravel()
    assert np.max(np.abs(r)) < 1e-9 * 1.01


def test_row_evaluation_matches_assembled_delta():
    """The row-by-row evaluation used for sampled checks at large sizes
    equals the rows of the assembled Delta (below eq. kkt_conditions)."""
    g = synth.random_grid(4, 5, 6, 3, 2, seed=81)
    P = as_problem(g)
    orc = O.Oracle(P)
    v = synth.random_vector(P.dim_x, seed=3)
    rows = np.arange(P.dim_x)
    got = O.delta_rows_matrix_free(P, rows, v)
    ref = orc.Delta @ v
    assert np.allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_standalone_nbjm_converges_to_the_kkt_solution():
    """Algorithm 2 run to its exit test converges (Section IV: the splittings
    are convergent) to the solution of Delta delta = r_delta, and needs far
    more iterations than PCGM (Section V)."""
    g = synth.random_grid(3, 4, 5, 2, 1, seed=91)
    orc = O.Oracle(as_problem(g))
    res = O.nbjm_solve(orc.splitting, orc.r_delta, 2, 1e-13, 200000, orc.phi)
    assert res.converged
    ref = orc.solve_direct().delta.ravel()
    assert np.linalg.norm(res.delta - ref) <= 1e-8 * np.linalg.norm(ref)
    assert res.outer_iterations > orc.solve(1e-10).iterations


def test_algorithm2_with_zero_inner_start_has_a_shifted_fixed_point():
    """Reading A22: with theta^(0) = 0 at every outer step (Algorithm 2 as
    printed), the outer iteration is delta <- Upsilon_L (r + Xi~ delta), whose
    fixed point is (Upsilon_L^-1 - Xi~)^-1 r, not Delta^-1 r."""
    g = synth.random_grid(3, 4, 5, 2, 1, seed=91)
    orc = O.Oracle(as_problem(g))
    Sp = orc.splitting
    res = O.nbjm_solve(Sp, orc.r_delta, 2, 1e-13, 200000, orc.phi, inner_start="zero")
    assert res.converged
    U = O.upsilon_dense(Sp, 2)
    fixed = np.linalg.solve(np.linalg.inv(U) - Sp.Xi.toarray(), orc.r_delta)
    assert np.linalg.norm(res.delta - fixed) <= 1e-8 * np.linalg.norm(fixed)
    exact = orc.solve_direct().delta.ravel()
    assert np.linalg.norm(fixed - exact) > 1e-3 * np.linalg.norm(exact)


def test_lanczos_estimates_match_dense_condition_numbers():
    """The extreme Ritz values of the Lanczos matrix built from the PCG
    coefficients bracket, and after enough steps match, the spectrum of the
    preconditioned operator (Saad 6.7.3)."""
    g = synth.workload("grid4_T20")
    orc = O.Oracle(as_problem(g))
    D = orc.Delta.toarray()
    ev = np.linalg.eigvalsh(D)
    cg = O.pcg(orc.Delta, orc.r_delta, lambda r: r, 1e-13, 100000)
    lo, hi = O.lanczos_extremes(cg.alphas, cg.betas)
    assert abs(hi / lo - ev[-1] / ev[0]) <= 0.02 * ev[-1] / ev[0]
    assert lo >= ev[0] * (1 - 1e-8) and hi <= ev[-1] * (1 + 1e-8)
    DS = O.nbjm_closed_form(orc.splitting, 2, 2)
    evp = sla.eigh(D, np.linalg.inv(DS), eigvals_only=True)
    pc = O.pcg(orc.Delta, orc.r_delta, orc.preconditioner(2, 2).apply, 1e-13, 10000)
    lo, hi = O.lanczos_extremes(pc.alphas, pc.betas)
    assert abs(hi / lo - evp[-1] / evp[0]) <= 0.02 * evp[-1] / evp[0]


def test_pcgm_steps_grow_at_most_linearly_with_the_grid():
    """Section V reports PCGM step counts that grow about linearly with K on
    its second case study; on the diffusion grids (K = N, T = 10, n = 4) the
    counts grow with K and no faster than K."""
    its = []
    for K in (4, 8, 16):
        g = synth.diffusion_grid(K, K, 10, 4, 2, seed=1)
        its.append(O.Oracle(as_problem(g)).solve(1e-10).iterations)
    assert its[0] <= its[1] <= its[2]
    assert its[1] <= 2 * its[0] and its[2] <= 2 * its[1]


# --------------------------------------------------------------------------
# slab-by-slab Delta product, recovery and residual (Section II-B)
# --------------------------------------------------------------------------

SLAB_CASES = [(3, 4, 5, 2, 1), (4, 5, 6, 3, 2), (1, 3, 4, 2, 2), (2, 1, 3, 1, 1), (5, 7, 2, 4, 2)]


@pytest.mark.parametrize("shape", SLAB_CASES)
def test_slab_delta_product_matches_assembled_delta(shape):
    """The slab-by-slab product against scipy's assembled
    A~ Q~^-1 A~' + B~ R~^-1 B~' (odd and even N, K = 1, N = 1), with and
    without boundary terms in omega~."""
    K, N, T, n, m = shape
    g = synth.random_grid(K, N, T, n, m, seed=sum(shape))
    rng = np.random.default_rng(7)
    for w in (None, rng.standard_normal((T, K * N, n))):
        P = as_problem(g, w)
        orc = O.Oracle(P)
        b = O.slab_blocks(P)
        for trial in range(2):
            vec = rng.standard_normal(P.dim_x)
            want = orc.Delta @ vec
            got = O.delta_apply_slabs(P, vec, b).ravel()
            assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()
        assert np.array_equal(O.rhs_slabs(P).ravel(), orc.r_delta)


@pytest.mark.parametrize("shape", SLAB_CASES[:3])
def test_slab_recovery_and_residual_match_the_assembled_forms(shape):
    K, N, T, n, m = shape
    g = synth.random_grid(K, N, T, n, m, seed=10 + sum(shape))
    P = as_problem(g)
    orc = O.Oracle(P)
    sol = orc.solve(1e-12)
    x, u = O.recover(orc.S, sol.delta.ravel())
    xs, us = O.recover_slabs(P, sol.delta)
    assert np.abs(xs.ravel() - x).max() <= 1e-13 * np.abs(x).max()
    assert np.abs(us.ravel() - u).max() <= 1e-13 * np.abs(u).max()
    # the true residual of the converged solve and of a perturbed iterate
    res = O.true_residual_slabs(P, sol.delta)
    want = np.linalg.norm(orc.r_delta - orc.Delta @ sol.delta.ravel()) / np.linalg.norm(orc.r_delta)
    assert res <= 1e-11 and abs(res - want) <= 1e-13
    bad = sol.delta.copy()
    bad[T // 2, 0, 0] += 1.0
    assert O.true_residual_slabs(P, bad) > 1e-3


def test_slab_recovery_is_feasible_under_simulation():
    """x and u from the slab recovery satisfy the grid dynamics node by node
    (the simulator of eq. 2d_graph_dynamics), independent of the stacked
    assembly."""
    g = synth.random_grid(4, 3, 6, 2, 1, seed=77)
    P = as_problem(g)
    sol = O.Oracle(P).solve_direct()
    x, u = O.recover_slabs(P, sol.delta)
    sim = simulate(P, u.reshape(P.T, P.nodes, P.m))
    assert np.abs(sim - x.reshape(sim.shape)).max() <= 1e-10 * max(1.0, np.abs(sim).max())


def test_cg_iteration_bound_golden_values():
    """The smallest k with 2((sqrt kappa - 1)/(sqrt kappa + 1))^k <= reduction
    (Section III's CG bound, reading A13), worked by hand:
      kappa = 100, 1e-6: rate 9/11, k >= ln(5e-7)/ln(9/11) = 72.30 -> 73
      kappa = 4,   1e-6: rate 1/3,  k >= ln(5e-7)/ln(1/3)  = 13.21 -> 14
      kappa = 100, 1e-3: k >= ln(5e-4)/ln(9/11) = 37.88 -> 38
      kappa = 1e4, 1e-8: rate 99/101, k >= ln(5e-9)/ln(99/101) = 955.7 -> 956
    and each value is checked to be the smallest that satisfies the bound."""
    for kappa, red, k in ((100.0, 1e-6, 73), (4.0, 1e-6, 14), (100.0, 1e-3, 38), (1e4, 1e-8, 956)):
        assert O.cg_iteration_bound(kappa, red) == k
        rate = (math.sqrt(kappa) - 1.0) / (math.sqrt(kappa) + 1.0)
        assert 2.0 * rate ** k <= red < 2.0 * rate ** (k - 1)
    assert O.cg_iteration_bound(1.0, 1e-6) == 1
