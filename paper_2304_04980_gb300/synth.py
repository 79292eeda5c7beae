"""Seeded synthetic LQ problems on a K x N grid of coupled subsystems.

This module only draws inputs: per-node dynamics blocks, cost blocks and the
initial state.  It holds none of the solver's arithmetic, so both the CUDA
path and the CPU oracle can be fed from it.

Every array is in the library's host layout, with node index p = i*N + j
(i: 0..K-1 vertical, j: 0..N-1 horizontal):

    A_self [K*N, n, n]      A_{i,j}
    A_nbr  [K*N, 4, n, n]   E (j-1), F (j+1), G (i-1), H (i+1)
    B      [K*N, n, m]
    Q      [K*N, n, n]      stage state weight (t < T)
    R      [K*N, m, m]      stage input weight
    Q_T    [K*N, n, n]      terminal state weight
    x0     [K*N, n]         gamma, the initial state

The dynamics these blocks define are those of the paper's grid model
(Section II, eq. 2d_graph_dynamics); the workload shapes follow the paper's
experiments (Section V: n = 4, m = 1..2, Q = I, R of order one).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class GridLQ:
    K: int
    N: int
    T: int
    n: int
    m: int
    A_self: np.ndarray
    A_nbr: np.ndarray
    B: np.ndarray
    Q: np.ndarray
    R: np.ndarray
    Q_T: np.ndarray
    x0: np.ndarray
    name: str = ""

    @property
    def nodes(self) -> int:
        return self.K * self.N

    def arrays(self):
        """The seven input arrays in argument order of lq2d_create."""
        return (self.A_self, self.A_nbr, self.B, self.Q, self.R, self.Q_T, self.x0)

    def with_x0(self, x0: np.ndarray) -> "GridLQ":
        return dataclasses.replace(self, x0=np.ascontiguousarray(x0, dtype=np.float64))


def _eye_blocks(count: int, size: int, scale: float) -> np.ndarray:
    return np.broadcast_to(np.eye(size) * scale, (count, size, size)).copy()


def random_grid(K: int, N: int, T: int, n: int, m: int, seed: int, *,
                rho: float = 0.95, coupling: float = 0.1, r_weight: float = 0.1,
                qT_weight: float = 10.0, name: str = "") -> GridLQ:
    """Random heterogeneous grid (the K=N=4, T=20 workload's recipe).

    Draw order from numpy's PCG64 stream: A_self for every node (node-major),
    then A_nbr, then B, then x0.  A_self is a standard-normal n x n matrix
    scaled so that its largest eigenvalue modulus is `rho`; each neighbour
    block is standard normal times `coupling`; B is standard normal; Q = I,
    R = r_weight * I, Q_T = qT_weight * I; x0 is standard normal.
    """
    rng = np.random.default_rng(seed)
    nodes = K * N
    A_self = rng.standard_normal((nodes, n, n))
    rad = np.max(np.abs(np.linalg.eigvals(A_self)), axis=1)
    A_self *= (rho / rad)[:, None, None]
    A_nbr = rng.standard_normal((nodes, 4, n, n)) * coupling
    B = rng.standard_normal((nodes, n, m))
    x0 = rng.standard_normal((nodes, n))
    return GridLQ(K, N, T, n, m, A_self, A_nbr, B,
                  _eye_blocks(nodes, n, 1.0), _eye_blocks(nodes, m, r_weight),
                  _eye_blocks(nodes, n, qT_weight), x0, name=name)


def diffusion_grid(K: int, N: int, T: int, n: int = 4, m: int = 2, seed: int = 1,
                   name: str = "") -> GridLQ:
    """Smooth diffusion-like grid (the K=N=64, T=100 workload's recipe).

    A_self = I + 0.05 * tridiag(1, -2, 1) at every node; each neighbour block
    is 0.05 * I plus entrywise normal noise of standard deviation 0.01;
    B ~ N(0, 1/m) entrywise; Q = I, R = 0.01 * I, Q_T = I; x0 is a Gaussian
    bump exp(-((i-c)^2 + (j-c)^2) / (2 sigma^2)) in every state component,
    with 1-based i, j, c = (K+1)/2 and sigma = K/8.
    Draw order: A_nbr noise, then B.
    """
    rng = np.random.default_rng(seed)
    nodes = K * N
    lap = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    A_self = np.broadcast_to(np.eye(n) + 0.05 * lap, (nodes, n, n)).copy()
    A_nbr = 0.05 * np.eye(n)[None, None] + 0.01 * rng.standard_normal((nodes, 4, n, n))
    B = rng.standard_normal((nodes, n, m)) / np.sqrt(m)
    ii, jj = np.meshgrid(np.arange(1, K + 1), np.arange(1, N + 1), indexing="ij")
    c_i, c_j = (K + 1) / 2.0, (N + 1) / 2.0
    sigma = K / 8.0
    bump = np.exp(-((ii - c_i) ** 2 + (jj - c_j) ** 2) / (2.0 * sigma ** 2)).reshape(nodes)
    x0 = np.repeat(bump[:, None], n, axis=1)
    return GridLQ(K, N, T, n, m, A_self, A_nbr, B,
                  _eye_blocks(nodes, n, 1.0), _eye_blocks(nodes, m, 0.01),
                  _eye_blocks(nodes, n, 1.0), x0, name=name)


# The named workloads.  S = L = 2 everywhere (the paper's setting, Section V).
WORKLOADS = {
    "grid4_T20": dict(kind="random", K=4, N=4, T=20, n=2, m=1, seed=0, tol=1e-10),
    "grid64_T100": dict(kind="diffusion", K=64, N=64, T=100, n=4, m=2, seed=1, tol=1e-8),
    "grid256_T200": dict(kind="random", K=256, N=256, T=200, n=4, m=2, seed=2, tol=1e-8),
    # profiling size: vectors of 52 MB, so one sweep's traffic exceeds the L2
    "grid128_T100": dict(kind="random", K=128, N=128, T=100, n=4, m=2, seed=3, tol=1e-8),
    # profiling size with the K = N = 256 grid's parallelism, half its horizon
    "grid256_T100": dict(kind="random", K=256, N=256, T=100, n=4, m=2, seed=2, tol=1e-8),
}


def workload(name: str) -> GridLQ:
    w = WORKLOADS[name]
    if w["kind"] == "random":
        return random_grid(w["K"], w["N"], w["T"], w["n"], w["m"], w["seed"], name=name)
    return diffusion_grid(w["K"], w["N"], w["T"], w["n"], w["m"], w["seed"], name=name)


def batch_grids(count: int = 512, seed: int = 3, n: int = 4, m: int = 2,
                K_range=(8, 64), N_range=(8, 64), T_range=(50, 200),
                coupling_range=(0.02, 0.2)) -> list:
    """Uneven instances for the batched solve: K, N and T uniform integers in
    their ranges and a coupling scale uniform in its range, drawn in that
    order per instance from a master stream (PCG64, `seed`); instance idx
    then uses the random_grid recipe with seed 10000 + idx."""
    rng = np.random.default_rng(seed)
    grids = []
    for idx in range(count):
        K = int(rng.integers(K_range[0], K_range[1] + 1))
        N = int(rng.integers(N_range[0], N_range[1] + 1))
        T = int(rng.integers(T_range[0], T_range[1] + 1))
        c = float(rng.uniform(coupling_range[0], coupling_range[1]))
        grids.append(random_grid(K, N, T, n, m, seed=10000 + idx, coupling=c, name="batch%d" % idx))
    return grids


def random_vector(shape, seed: int) -> np.ndarray:
    """A seeded standard-normal test vector (operator and preconditioner probes)."""
    return np.random.default_rng(seed).standard_normal(shape)


@dataclasses.dataclass
class WarmStartFamily:
    """A spatially uniform grid family for the learned warm start: every node
    shares one A_self, one neighbour block per direction and one B, drawn
    once; an instance picks the coupling scale c that multiplies the
    neighbour blocks and its own initial state x0."""
    K: int
    N: int
    T: int
    n: int
    m: int
    A_self: np.ndarray   # [n, n]
    E_dir: np.ndarray    # [4, n, n] neighbour blocks before scaling (west, east, north, south)
    B: np.ndarray        # [n, m]
    r_weight: float
    qT_weight: float
    coupling_range: tuple

    def instance_params(self, seed: int):
        """(c, x0) of instance `seed`: c uniform in coupling_range, then x0
        standard normal [K*N, n], from PCG64(seed)."""
        rng = np.random.default_rng(seed)
        c = float(rng.uniform(self.coupling_range[0], self.coupling_range[1]))
        x0 = rng.standard_normal((self.K * self.N, self.n))
        return c, x0

    def grid(self, c: float, x0: np.ndarray) -> GridLQ:
        nodes = self.K * self.N
        A_nbr = np.broadcast_to(self.E_dir * c, (nodes, 4, self.n, self.n)).copy()
        return GridLQ(self.K, self.N, self.T, self.n, self.m,
                      np.broadcast_to(self.A_self, (nodes, self.n, self.n)).copy(), A_nbr,
                      np.broadcast_to(self.B, (nodes, self.n, self.m)).copy(),
                      _eye_blocks(nodes, self.n, 1.0), _eye_blocks(nodes, self.m, self.r_weight),
                      _eye_blocks(nodes, self.n, self.qT_weight), np.ascontiguousarray(x0, dtype=np.float64),
                      name="warm_c%.4f" % c)

    def instance(self, seed: int) -> GridLQ:
        return self.grid(*self.instance_params(seed))


def warmstart_family(K: int = 128, N: int = 128, T: int = 100, n: int = 4, m: int = 2, seed: int = 5, *,
                     rho: float = 0.95, r_weight: float = 0.1, qT_weight: float = 10.0,
                     coupling_range=(0.02, 0.2)) -> WarmStartFamily:
    """The learned-warm-start workload (K = N = 128, n = 4, m = 2, T = 100 by
    default), with the random_grid recipe's distributions drawn once for the
    whole grid: A_self standard normal scaled to spectral radius rho, the
    four neighbour blocks standard normal, B standard normal (PCG64(seed), in
    that order); Q = I, R = r_weight I, Q_T = qT_weight I."""
    rng = np.random.default_rng(seed)
    A_self = rng.standard_normal((n, n))
    A_self *= rho / np.max(np.abs(np.linalg.eigvals(A_self)))
    E_dir = rng.standard_normal((4, n, n))
    B = rng.standard_normal((n, m))
    return WarmStartFamily(K, N, T, n, m, A_self, E_dir, B, r_weight, qT_weight, tuple(coupling_range))


def warmstart_init(layer_sizes, seed: int = 0, out_scale: float = 0.1) -> np.ndarray:
    """Initial FP32 parameter vector of the warm-start network (layout of
    include/lq2d_warmstart.h): He-normal weights, standard deviation
    sqrt(2 / (9 C_in)), the last layer's times out_scale; zero biases.
    Drawn layer by layer from PCG64(seed)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(layer_sizes) - 1):
        ci, co = layer_sizes[l], layer_sizes[l + 1]
        std = np.sqrt(2.0 / (9.0 * ci)) * (out_scale if l + 2 == len(layer_sizes) else 1.0)
        parts.append((rng.standard_normal(co * ci * 9) * std).astype(np.float32))
        parts.append(np.zeros(co, dtype=np.float32))
    return np.concatenate(parts)
