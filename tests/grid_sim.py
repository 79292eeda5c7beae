"""Vectorised forward simulation of the grid dynamics (Section II,
eq. 2d_graph_dynamics) for property checks at sizes where the oracle's
matrices are too large.  Independent of both the oracle and the library."""
import numpy as np


def step(K, N, A_self, A_nbr, B, x_t, u_t, w_t=None):
    """x_{t+1} for all nodes; x_t [K*N, n], u_t [K*N, m]."""
    n = x_t.shape[1]
    X = x_t.reshape(K, N, n)
    out = np.einsum("pab,pb->pa", A_self, x_t) + np.einsum("pab,pb->pa", B, u_t)
    shifted = np.zeros((4, K, N, n))
    shifted[0][:, 1:] = X[:, :-1]    # x_{i,j-1}  (E)
    shifted[1][:, :-1] = X[:, 1:]    # x_{i,j+1}  (F)
    shifted[2][1:, :] = X[:-1, :]    # x_{i-1,j}  (G)
    shifted[3][:-1, :] = X[1:, :]    # x_{i+1,j}  (H)
    for s in range(4):
        out += np.einsum("pab,pb->pa", A_nbr[:, s], shifted[s].reshape(K * N, n))
    if w_t is not None:
        out += w_t
    return out


def simulate(K, N, T, A_self, A_nbr, B, x0, u, w=None):
    x = np.zeros((T + 1,) + x0.shape)
    x[0] = x0
    for t in range(T):
        x[t + 1] = step(K, N, A_self, A_nbr, B, x[t], u[t], None if w is None else w[t])
    return x


def cost(Q, R, Q_T, x, u):
    J = 0.5 * np.einsum("tpa,pab,tpb->", x[:-1], Q, x[:-1])
    J += 0.5 * np.einsum("pa,pab,pb->", x[-1], Q_T, x[-1])
    J += 0.5 * np.einsum("tpa,pab,tpb->", u, R, u)
    return float(J)
