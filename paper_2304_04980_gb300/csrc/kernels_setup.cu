// Setup kernels (run once per problem): per-node inverses, the node blocks of
// Delta's splittings, and the banded block-Cholesky factors of Phi_bar.
//
// Paper: Section II-B (structure of Delta: Psi_t = Q_t^-1 + A Q^-1 A' +
// B R^-1 B', Xi_t = -A Q^-1), Section IV (splittings Delta = Psi~ - Xi~,
// Psi~ = Phi~ - Omega~ over column pairs v), Section IV-B (one Cholesky
// factorisation of each Phi_bar_{v,t}, done once before Algorithm 1).
// With time-invariant blocks Phi_bar_{v,t} takes only two values for t >= 1:
// one for 1 <= t <= T-1 (class 0) and one for t = T (class 1, Q_T^-1 on the
// diagonal).  At t = 0, Psi_0 = Q^-1 is node-diagonal, so no factor is needed.
#include "setup.h"

namespace lq2d {

namespace {

// Lower Cholesky of the leading d x d block of a (row stride d); returns
// false on a non-positive or non-finite pivot.
__device__ bool chol_small(double* a, int d) {
  for (int j = 0; j < d; ++j) {
    double s = a[j * d + j];
    for (int k = 0; k < j; ++k) s -= a[j * d + k] * a[j * d + k];
    if (!(s > 0.0) || !isfinite(s)) return false;
    const double ljj = sqrt(s);
    a[j * d + j] = ljj;
    for (int i = j + 1; i < d; ++i) {
      double t = a[i * d + j];
      for (int k = 0; k < j; ++k) t -= a[i * d + k] * a[j * d + k];
      a[i * d + j] = t / ljj;
    }
  }
  return true;
}

// inv = (L L')^-1 from the lower Cholesky factor L (d x d).
__device__ void spd_inverse_from_chol(const double* L, double* inv, int d) {
  double Li[kMaxN * kMaxN];
  for (int c = 0; c < d; ++c) {
    for (int r = 0; r < d; ++r) {
      if (r < c) { Li[r * d + c] = 0.0; continue; }
      double s = (r == c) ? 1.0 : 0.0;
      for (int k = c; k < r; ++k) s -= L[r * d + k] * Li[k * d + c];
      Li[r * d + c] = s / L[r * d + r];
    }
  }
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) {
      double s = 0.0;
      for (int k = (r > c ? r : c); k < d; ++k) s += Li[k * d + r] * Li[k * d + c];
      inv[r * d + c] = s;
    }
}

__device__ bool spd_inverse(const double* a, double* inv, int d) {
  double L[kMaxN * kMaxN];
  for (int e = 0; e < d * d; ++e) L[e] = a[e];
  if (!chol_small(L, d)) return false;
  spd_inverse_from_chol(L, inv, d);
  return true;
}

// A_hat block in row p, column r (r = neighbour of p in direction dir).
__device__ inline const double* ahat_row_block(const double* Aself, const double* Anb, int p, int dir, int n) {
  return dir == kSelf ? Aself + (size_t)p * n * n : Anb + ((size_t)p * 4 + (dir - 1)) * n * n;
}

// A_hat block in row r, column p, for r = neighbour of p in direction dir:
// the west neighbour reaches p through its F (east) block, the east one
// through E, the north one through H, the south one through G.
__device__ inline const double* ahat_col_block(const double* Aself, const double* Anb, int r, int dir, int n) {
  int slot;
  switch (dir) {
    case kSelf: return Aself + (size_t)r * n * n;
    case kWest: slot = 1; break;   // F_r
    case kEast: slot = 0; break;   // E_r
    case kNorth: slot = 3; break;  // H_r
    default: slot = 2; break;      // G_r
  }
  return Anb + ((size_t)r * 4 + slot) * n * n;
}

}  // namespace

// The 13 node offsets (di, dj) with |di| + |dj| <= 2.
__host__ __device__ int off13_index(int di, int dj) {
  const int ad = (di < 0 ? -di : di) + (dj < 0 ? -dj : dj);
  if (ad > 2) return -1;
  // order: (0,0) (0,-1) (0,1) (-1,0) (1,0) (-1,-1) (-1,1) (1,-1) (1,1) (0,-2) (0,2) (-2,0) (2,0)
  if (di == 0 && dj == 0) return 0;
  if (di == 0 && dj == -1) return 1;
  if (di == 0 && dj == 1) return 2;
  if (di == -1 && dj == 0) return 3;
  if (di == 1 && dj == 0) return 4;
  if (di == -1 && dj == -1) return 5;
  if (di == -1 && dj == 1) return 6;
  if (di == 1 && dj == -1) return 7;
  if (di == 1 && dj == 1) return 8;
  if (di == 0 && dj == -2) return 9;
  if (di == 0 && dj == 2) return 10;
  if (di == -2 && dj == 0) return 11;
  return 12;  // (2, 0)
}

__device__ static const int kOff13Di[13] = {0, 0, 0, -1, 1, -1, -1, 1, 1, 0, 0, -2, 2};
__device__ static const int kOff13Dj[13] = {0, -1, 1, 0, 0, -1, 1, -1, 1, -2, 2, 0, 0};

// Per node: zero the coupling blocks that point off the grid, invert Q, Q_T
// and R, and form S = B R^-1 B' and R^-1 B'.  Also checks every input entry
// of the node for finiteness.
__global__ void setup_nodes_kernel(SetupBuffers sb, int K, int N, int n, int m, int* status) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= K * N) return;
  const int i = p / N, j = p % N;
  const int nn = n * n;
  int bad = 0;
  // finiteness of the node's inputs
  for (int e = 0; e < nn; ++e) {
    bad |= !isfinite(sb.Aself[(size_t)p * nn + e]);
    bad |= !isfinite(sb.Qm[(size_t)p * nn + e]);
    bad |= !isfinite(sb.QTm[(size_t)p * nn + e]);
  }
  for (int e = 0; e < 4 * nn; ++e) bad |= !isfinite(sb.Anb[(size_t)p * 4 * nn + e]);
  for (int e = 0; e < n * m; ++e) bad |= !isfinite(sb.Bm[(size_t)p * n * m + e]);
  for (int e = 0; e < m * m; ++e) bad |= !isfinite(sb.Rm[(size_t)p * m * m + e]);
  for (int e = 0; e < n; ++e) bad |= !isfinite(sb.x0[(size_t)p * n + e]);
  if (bad) atomicOr(status, kSetupNonFinite);
  // coupling blocks towards boundary states are not part of the unknowns
  const bool edge[4] = {j == 0, j == N - 1, i == 0, i == K - 1};
  for (int s = 0; s < 4; ++s)
    if (edge[s])
      for (int e = 0; e < nn; ++e) sb.Anb[((size_t)p * 4 + s) * nn + e] = 0.0;
  double a[kMaxN * kMaxN];
  // symmetrised copies: the cost weights are symmetric by assumption
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c)
      a[r * n + c] = 0.5 * (sb.Qm[(size_t)p * nn + r * n + c] + sb.Qm[(size_t)p * nn + c * n + r]);
  if (!spd_inverse(a, sb.Qi + (size_t)p * nn, n)) atomicOr(status, kSetupNotPD);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c)
      a[r * n + c] = 0.5 * (sb.QTm[(size_t)p * nn + r * n + c] + sb.QTm[(size_t)p * nn + c * n + r]);
  if (!spd_inverse(a, sb.QTi + (size_t)p * nn, n)) atomicOr(status, kSetupNotPD);
  double Ri[kMaxM * kMaxM];
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < m; ++c)
      a[r * m + c] = 0.5 * (sb.Rm[(size_t)p * m * m + r * m + c] + sb.Rm[(size_t)p * m * m + c * m + r]);
  if (!spd_inverse(a, Ri, m)) atomicOr(status, kSetupNotPD);
  const double* B = sb.Bm + (size_t)p * n * m;
  // R^-1 B'  (m x n)
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += Ri[r * m + k] * B[c * m + k];
      sb.RiBt[(size_t)p * m * n + r * n + c] = s;
    }
  // B R^-1 B'  (n x n)
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += B[r * m + k] * sb.RiBt[(size_t)p * m * n + k * n + c];
      sb.Sb[(size_t)p * nn + r * n + c] = s;
    }
}

// Per (node, direction): AQ = A_hat_{p,r} Q_r^-1 and QAt = Q_p^-1 A_hat_{r,p}'.
// These are the node blocks of Xi~ (Section IV: Xi~ = Psi~ - Delta, whose
// blocks next to the diagonal are A Q^-1 and Q^-1 A').
__global__ void setup_aq_kernel(SetupBuffers sb, int K, int N, int n) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= K * N * 5) return;
  const int p = id / 5, dir = id % 5;
  const int i = p / N, j = p % N;
  const int nn = n * n;
  double* aq = sb.AQ + ((size_t)p * 5 + dir) * nn;
  double* qat = sb.QAt + ((size_t)p * 5 + dir) * nn;
  const int r = nbr_node(i, j, dir, K, N);
  if (r < 0) {
    for (int e = 0; e < nn; ++e) { aq[e] = 0.0; qat[e] = 0.0; }
    return;
  }
  const double* Apr = ahat_row_block(sb.Aself, sb.Anb, p, dir, n);
  const double* Arp = ahat_col_block(sb.Aself, sb.Anb, r, dir, n);
  const double* Qr = sb.Qi + (size_t)r * nn;
  const double* Qp = sb.Qi + (size_t)p * nn;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double s = 0.0, t = 0.0;
      for (int c = 0; c < n; ++c) {
        s += Apr[a * n + c] * Qr[c * n + b];
        t += Qp[a * n + c] * Arp[b * n + c];
      }
      aq[a * n + b] = s;
      qat[a * n + b] = t;
    }
}

// Per (node p, offset o of the 13-point stencil): M_{p,q} =
// sum_r A_hat_{p,r} Q_r^-1 A_hat_{q,r}' over the common neighbours r of p and
// q: the spatial blocks of A_hat Q^-1 A_hat' in Psi_t (Section II-B).
__global__ void setup_m13_kernel(SetupBuffers sb, int K, int N, int n) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= K * N * 13) return;
  const int p = id / 13, o = id % 13;
  const int i = p / N, j = p % N;
  const int nn = n * n;
  double* M = sb.M13 + ((size_t)p * 13 + o) * nn;
  for (int e = 0; e < nn; ++e) M[e] = 0.0;
  const int qi = i + kOff13Di[o], qj = j + kOff13Dj[o];
  if (qi < 0 || qi >= K || qj < 0 || qj >= N) return;
  const int q = qi * N + qj;
  for (int dp = 0; dp < 5; ++dp) {
    const int r = nbr_node(i, j, dp, K, N);
    if (r < 0) continue;
    const int ri = r / N, rj = r % N;
    const int di = ri - qi, dj = rj - qj;
    int dq;
    if (di == 0 && dj == 0) dq = kSelf;
    else if (di == 0 && dj == -1) dq = kWest;
    else if (di == 0 && dj == 1) dq = kEast;
    else if (di == -1 && dj == 0) dq = kNorth;
    else if (di == 1 && dj == 0) dq = kSouth;
    else continue;
    const double* aq = sb.AQ + ((size_t)p * 5 + dp) * nn;           // A_hat_{p,r} Q_r^-1
    const double* Aqr = ahat_row_block(sb.Aself, sb.Anb, q, dq, n);  // A_hat_{q,r}
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        double s = 0.0;
        for (int c = 0; c < n; ++c) s += aq[a * n + c] * Aqr[b * n + c];
        M[a * n + b] += s;
      }
  }
}

// Omega~ blocks: Omega~ = Phi~ - Psi~ holds minus the couplings of Psi~
// between a node and the five nodes of the neighbouring column pairs.
__global__ void setup_omega_kernel(SetupBuffers sb, int K, int N, int n) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= K * N * 5) return;
  const int p = id / 5, o = id % 5;
  const int i = p / N, j = p % N;
  const int nn = n * n;
  double* Om = sb.Om + ((size_t)p * 5 + o) * nn;
  const int q = offpair_node(i, j, o, K, N);
  if (q < 0) {
    for (int e = 0; e < nn; ++e) Om[e] = 0.0;
    return;
  }
  const int idx = off13_index(q / N - i, q % N - j);
  const double* M = sb.M13 + ((size_t)p * 13 + idx) * nn;
  for (int e = 0; e < nn; ++e) Om[e] = -M[e];
}

// Banded block-Cholesky factorisation of Phi_bar_{v,class} (Section IV-B),
// one warp per (column pair v, class).  Unknowns are ordered by pair-row i
// (the two nodes (i, 2v) and (i, 2v+1)) and, inside a pair-row, by node then
// component, so Phi_bar is block-pentadiagonal in 2n x 2n pair-row blocks and
// its Cholesky factor keeps that band:
//   L2_i = A_{i,i-2} L0_{i-2}^-T
//   L1_i = (A_{i,i-1} - L2_i L1_{i-1}') L0_{i-1}^-T
//   L0_i L0_i' = A_{i,i} - L1_i L1_i' - L2_i L2_i'
// A missing second column (odd N) is carried as a decoupled identity block,
// whose solution is zero.  The sweeps use the same factorisation with the
// pivots taken out, Phi_bar = F D F' with F unit block lower triangular:
//   F1_i = L1_i L0_{i-1}^-1,  F2_i = L2_i L0_{i-2}^-1,  D_i^-1 = L0_i^-T L0_i^-1
//   forward  (F y = tau):        y_i = tau_i - F2_i y_{i-2} - F1_i y_{i-1}
//   backward (F' x = D^-1 y):    x_i = D_i^-1 y_i - N2_i x_{i+2} - N1_i x_{i+1},
//                                N1_i = F1_{i+1}',  N2_i = F2_{i+2}'
// (N1, N2 are zero past the last pair-row).  Against the pre-multiplied
// Cholesky form (y_i = L0_i^-1 tau_i - ...) the forward step loses its
// product with the pivot, one of six 2n x 2n products per pair-row.
// Record of pair-row i (G2 = 2n, blocks G2 x G2 row-major, so a lane's row
// is contiguous):
//   [N2_i][N1_i][D_i^-1][E_i]  (backward step i; E_i = A_{i,i+2}, the block of
//                               Phi_bar coupling the pair-row to the one two
//                               rows on, so that N2_i = D_i^-1 E_i: the tiled
//                               sweeps form x_i = D_i^-1 (y_i - E_i x_{i+2})
//                               - N1_i x_{i+1}, E_i being block diagonal)
//   [F2_i][F1_i][L0_i^-1]      (forward step i; the sweeps read F2 and F1, the
//                               multi-right-hand-side path applies D_i^-1 as
//                               L0_i^-T L0_i^-1 in TF32)
//
// rev = 1 runs the same recurrences over the pair-rows in reverse order
// (step i factors physical pair-row K-1-i, whose "previous" rows are the ones
// below it), storing its records in step order in `out`: the factor of the
// two-ended (twisted) solve's bottom half.  With iface != NULL the pass keeps
// the blocks the interface rows k, k+1 (k = kI) need for their Schur
// complement, [V][2][9] blocks of (2n)^2 (slot: 0 C_k, 1 tmp_{k+1},
// 2 R_{k+1}, 3 A_kk, 4 A_{k+1,k+1}, 5 A_{k+1,k} from the forward pass;
// 6 C, 7 tmp, 8 R of the reversed pass at physical rows k+1, k, k), where
// C is the pivot block before its Cholesky, tmp = A_{i,prev} - L2 L1_prev'
// and R = A_ii - L2 L2'.
__global__ void setup_factor_kernel(SetupBuffers sb, int K, int N, int n, int V, long long fac_rec,
                                    long long fac_vc, int* status, int rev, double* out, double* iface,
                                    int kI) {
  extern __shared__ double smem[];
  const int vc = blockIdx.x;
  const int v = vc >> 1, cls = vc & 1;
  const int lane = threadIdx.x;
  const int G2 = 2 * n, BS = G2 * G2;
  double* Aii = smem;
  double* Aim1 = Aii + BS;
  double* Aim2 = Aim1 + BS;
  double* L2 = Aim2 + BS;
  double* L1 = L2 + BS;
  double* C = L1 + BS;
  double* tmp = C + BS;
  double* prevL0 = tmp + BS;       // [2][BS]: L0^-1 of pair-rows i-1, i-2
  double* prevL1 = prevL0 + 2 * BS;  // L1 of pair-row i-1
  __shared__ int bad;
  if (lane == 0) bad = 0;
  const int nn = n * n;
  const double* Qd = cls == 0 ? sb.Qi : sb.QTi;
  const bool two_cols = (2 * v + 1) < N;
  int cur = 0;  // index of the L0^-1 of pair-row i-1 inside prevL0
  __syncwarp();
  for (int i = 0; i < K; ++i) {
    const int ip = rev ? K - 1 - i : i;  // physical pair-row of step i
    // --- assemble the three blocks of row ip of Phi_bar (towards the rows
    //     of steps i-1 and i-2)
    for (int e = lane; e < 3 * BS; e += 32) {
      const int blk = e / BS, rc = e % BS;
      const int a = rc / G2, b = rc % G2;
      const int ja = a / n, ka = a % n, jb = b / n, kb = b % n;
      const int di = rev ? blk : -blk;  // column node lives in pair-row ip + di
      double val = 0.0;
      const bool colA = (ja == 0) || two_cols;
      const bool colB = (jb == 0) || two_cols;
      if (ip + di >= 0 && ip + di < K) {
        if (colA && colB) {
          const int p = ip * N + 2 * v + ja;
          const int o = off13_index(di, jb - ja);
          if (o >= 0) val = sb.M13[((size_t)p * 13 + o) * nn + ka * n + kb];
          if (blk == 0 && ja == jb) val += Qd[(size_t)p * nn + ka * n + kb] + sb.Sb[(size_t)p * nn + ka * n + kb];
        } else if (blk == 0 && ja == jb) {
          val = (ka == kb) ? 1.0 : 0.0;  // decoupled stand-in for the missing column
        }
      }
      (blk == 0 ? Aii : blk == 1 ? Aim1 : Aim2)[rc] = val;
    }
    __syncwarp();
    const double* L0m1 = prevL0 + cur * BS;        // pair-row i-1
    const double* L0m2 = prevL0 + (cur ^ 1) * BS;  // pair-row i-2
    // --- L2 = A_{i,i-2} L0_{i-2}^-T
    for (int e = lane; e < BS; e += 32) {
      const int a = e / G2, b = e % G2;
      double s = 0.0;
      if (i >= 2)
        for (int c = 0; c < G2; ++c) s += Aim2[a * G2 + c] * L0m2[b * G2 + c];
      L2[e] = s;
    }
    __syncwarp();
    // --- tmp = A_{i,i-1} - L2 L1_{i-1}'
    for (int e = lane; e < BS; e += 32) {
      const int a = e / G2, b = e % G2;
      double s = Aim1[e];
      if (i >= 2)
        for (int c = 0; c < G2; ++c) s -= L2[a * G2 + c] * prevL1[b * G2 + c];
      tmp[e] = s;
    }
    __syncwarp();
    // --- E of the record two pair-rows back: A_{i-2,i} = A_{i,i-2}'
    if (i >= 2) {
      double* rp = out + (size_t)vc * fac_vc + (size_t)(i - 2) * fac_rec;
      for (int e = lane; e < BS; e += 32) rp[3 * BS + e] = Aim2[(e % G2) * G2 + e / G2];
    }
    // --- L1 = tmp L0_{i-1}^-T
    for (int e = lane; e < BS; e += 32) {
      const int a = e / G2, b = e % G2;
      double s = 0.0;
      if (i >= 1)
        for (int c = 0; c < G2; ++c) s += tmp[a * G2 + c] * L0m1[b * G2 + c];
      L1[e] = s;
    }
    __syncwarp();
    // --- C = A_{i,i} - L1 L1' - L2 L2'
    for (int e = lane; e < BS; e += 32) {
      const int a = e / G2, b = e % G2;
      double s = Aii[e];
      for (int c = 0; c < G2; ++c) s -= L1[a * G2 + c] * L1[b * G2 + c] + L2[a * G2 + c] * L2[b * G2 + c];
      C[e] = s;
    }
    __syncwarp();
    // --- interface blocks of the two-ended solve (see above)
    if (iface != nullptr) {
      double* ib = iface + (size_t)vc * 9 * BS;
      const int at_k = rev ? K - kI - 1 : kI;      // step of physical row k
      const int at_k1 = rev ? K - kI - 2 : kI + 1; // step of physical row k+1
      const bool cap_c = rev ? (i == at_k1) : (i == at_k);
      const bool cap_t = rev ? (i == at_k) : (i == at_k1);
      for (int e = lane; e < BS; e += 32) {
        if (cap_c) {
          ib[(rev ? 6 : 0) * BS + e] = C[e];
          if (!rev) ib[3 * BS + e] = Aii[e];
        }
        if (cap_t) {
          const int a = e / G2, b = e % G2;
          double r2 = Aii[e];
          for (int c = 0; c < G2; ++c) r2 -= L2[a * G2 + c] * L2[b * G2 + c];
          ib[(rev ? 7 : 1) * BS + e] = tmp[e];
          ib[(rev ? 8 : 2) * BS + e] = r2;
          if (!rev) {
            ib[4 * BS + e] = Aii[e];
            ib[5 * BS + e] = Aim1[e];
          }
        }
      }
      __syncwarp();
    }
    // --- C = L0 L0' (right-looking, in place, lower triangle)
    for (int jc = 0; jc < G2; ++jc) {
      if (lane == 0) {
        const double d = C[jc * G2 + jc];
        if (!(d > 0.0) || !isfinite(d)) bad = 1;
        C[jc * G2 + jc] = sqrt(d > 0.0 ? d : 1.0);
      }
      __syncwarp();
      const double piv = C[jc * G2 + jc];
      for (int r = jc + 1 + lane; r < G2; r += 32) C[r * G2 + jc] /= piv;
      __syncwarp();
      for (int e = lane; e < BS; e += 32) {
        const int r = e / G2, c = e % G2;
        if (c > jc && r >= c) C[e] -= C[r * G2 + jc] * C[c * G2 + jc];
      }
      __syncwarp();
    }
    // --- F1_i = L1_i L0_{i-1}^-1 and F2_i = L2_i L0_{i-2}^-1, into the
    //     slots of A_{i,i-1} and A_{i,i-2} (no longer needed)
    double* F1 = Aim1;
    double* F2 = Aim2;
    for (int e = lane; e < BS; e += 32) {
      const int a = e / G2, b = e % G2;
      double s1 = 0.0, s2 = 0.0;
      for (int c = 0; c < G2; ++c) {
        if (i >= 1) s1 += L1[a * G2 + c] * L0m1[c * G2 + b];
        if (i >= 2) s2 += L2[a * G2 + c] * L0m2[c * G2 + b];
      }
      F1[e] = s1;
      F2[e] = s2;
    }
    __syncwarp();
    // --- backward blocks of the two previous records, now that F1_i and
    //     F2_i exist: N1_{i-1} = F1_i', N2_{i-2} = F2_i'
    double* rec_base = out + (size_t)vc * fac_vc;
    if (i >= 1) {
      double* rp = rec_base + (size_t)(i - 1) * fac_rec;
      for (int e = lane; e < BS; e += 32) rp[1 * BS + e] = F1[(e % G2) * G2 + e / G2];
    }
    if (i >= 2) {
      double* rp = rec_base + (size_t)(i - 2) * fac_rec;
      for (int e = lane; e < BS; e += 32) rp[0 * BS + e] = F2[(e % G2) * G2 + e / G2];
    }
    __syncwarp();
    // --- L0^-1 into the slot of pair-row i-2 (no longer needed); lane c
    //     solves column c of L0 X = I by forward substitution
    double* L0i = prevL0 + (cur ^ 1) * BS;
    if (lane < G2) {
      const int c = lane;
      for (int r = 0; r < G2; ++r) {
        if (r < c) { L0i[r * G2 + c] = 0.0; continue; }
        double s = (r == c) ? 1.0 : 0.0;
        for (int k = c; k < r; ++k) s -= C[r * G2 + k] * L0i[k * G2 + c];
        L0i[r * G2 + c] = s / C[r * G2 + r];
      }
    }
    __syncwarp();
    // --- record of pair-row i: the backward blocks N2_i, N1_i, E_i start
    //     at zero and are filled by the next two pair-rows
    double* rec = rec_base + (size_t)i * fac_rec;
    for (int e = lane; e < BS; e += 32) {
      const int a = e / G2, b = e % G2;
      // D_i^-1 = L0_i^-T L0_i^-1 (L0^-1 is lower triangular)
      double dinv = 0.0;
      for (int c = (a > b ? a : b); c < G2; ++c) dinv += L0i[c * G2 + a] * L0i[c * G2 + b];
      rec[0 * BS + e] = 0.0;
      rec[1 * BS + e] = 0.0;
      rec[2 * BS + e] = dinv;
      rec[3 * BS + e] = 0.0;
      rec[4 * BS + e] = F2[e];
      rec[5 * BS + e] = F1[e];
      rec[6 * BS + e] = L0i[e];
      prevL1[e] = L1[e];
    }
    __syncwarp();
    cur ^= 1;  // the slot just written becomes "pair-row i-1"
  }
  if (lane == 0 && bad) atomicOr(status, kSetupPhiNotPD);
  (void)V;
}

// Interface of the two-ended solve of Phi_bar_{v,class}: rows k, k+1 after
// eliminating rows 0..k-1 from the top and K-1..k+2 from the bottom,
//   S = A_II - A_IT A_TT^-1 A_TI - A_IB A_BB^-1 A_BI   (4n x 4n, SPD),
// from the blocks the two factor passes kept:
//   S_kk = C_k + R'_k - A_kk,  S_{k+1,k+1} = R_{k+1} + C'_{k+1} - A_{k+1,k+1},
//   S_{k+1,k} = tmp_{k+1} + tmp'_k' - A_{k+1,k}
// (unprimed: forward pass, primed: reversed pass); stored inverted,
// [V][2][(4n)^2].  One warp per (v, class), Gauss-Jordan without pivoting.
__global__ void setup_interface_kernel(const double* iface, double* sinv, int n, int* status) {
  extern __shared__ double smem[];
  const int vc = blockIdx.x, lane = threadIdx.x;
  const int G2 = 2 * n, BS = G2 * G2, W = 2 * G2, W2 = 2 * W;
  const double* ib = iface + (size_t)vc * 9 * BS;
  double* a = smem;  // [W][2W]: S | I
  for (int e = lane; e < W * W2; e += 32) {
    const int r = e / W2, c = e % W2;
    double val;
    if (c >= W) {
      val = (c - W == r) ? 1.0 : 0.0;
    } else {
      const int hr = r / G2, hc = c / G2, rr = r % G2, cc = c % G2;
      if (hr == 0 && hc == 0) val = ib[0 * BS + rr * G2 + cc] + ib[8 * BS + rr * G2 + cc] - ib[3 * BS + rr * G2 + cc];
      else if (hr == 1 && hc == 1)
        val = ib[2 * BS + rr * G2 + cc] + ib[6 * BS + rr * G2 + cc] - ib[4 * BS + rr * G2 + cc];
      else if (hr == 1)  // (k+1, k)
        val = ib[1 * BS + rr * G2 + cc] + ib[7 * BS + cc * G2 + rr] - ib[5 * BS + rr * G2 + cc];
      else  // (k, k+1): the transpose of (k+1, k)
        val = ib[1 * BS + cc * G2 + rr] + ib[7 * BS + rr * G2 + cc] - ib[5 * BS + cc * G2 + rr];
    }
    a[e] = val;
  }
  __syncwarp();
  __shared__ int bad;
  if (lane == 0) bad = 0;
  __syncwarp();
  for (int p = 0; p < W; ++p) {
    const double piv = a[p * W2 + p];
    if (lane == 0 && (!(piv > 0.0) || !isfinite(piv))) bad = 1;
    const double ip = 1.0 / (piv > 0.0 ? piv : 1.0);
    __syncwarp();
    for (int c = lane; c < W2; c += 32) a[p * W2 + c] *= ip;
    __syncwarp();
    for (int e = lane; e < W * W2; e += 32) {
      const int r = e / W2, c = e % W2;
      if (r == p || c == p) continue;
      a[e] -= a[r * W2 + p] * a[p * W2 + c];
    }
    __syncwarp();
    for (int r = lane; r < W; r += 32)
      if (r != p) a[r * W2 + p] = 0.0;
    __syncwarp();
  }
  double* out = sinv + (size_t)vc * W * W;
  for (int e = lane; e < W * W; e += 32) out[e] = a[(e / W) * W2 + W + e % W];
  if (lane == 0 && bad) atomicOr(status, kSetupPhiNotPD);
}

void launch_setup(const SetupBuffers& sb, int K, int N, int n, int m, int V, long long fac_rec,
                  long long fac_vc, int* d_status, cudaStream_t s) {
  const int NN = K * N;
  setup_nodes_kernel<<<(NN + 127) / 128, 128, 0, s>>>(sb, K, N, n, m, d_status);
  setup_aq_kernel<<<(NN * 5 + 127) / 128, 128, 0, s>>>(sb, K, N, n);
  setup_m13_kernel<<<(NN * 13 + 127) / 128, 128, 0, s>>>(sb, K, N, n);
  setup_omega_kernel<<<(NN * 5 + 127) / 128, 128, 0, s>>>(sb, K, N, n);
  const size_t shm = (size_t)11 * (2 * n) * (2 * n) * sizeof(double);
  const bool twisted = sb.fac_rev != nullptr && sb.iface != nullptr && sb.sinv != nullptr && K >= kTwistedMinK;
  const int kI = (K - 2) / 2;
  setup_factor_kernel<<<V * 2, 32, shm, s>>>(sb, K, N, n, V, fac_rec, fac_vc, d_status, 0, sb.fac,
                                             twisted ? sb.iface : nullptr, kI);
  if (twisted) {
    setup_factor_kernel<<<V * 2, 32, shm, s>>>(sb, K, N, n, V, fac_rec, fac_vc, d_status, 1, sb.fac_rev,
                                               sb.iface, kI);
    const size_t shi = (size_t)(4 * n) * (8 * n) * sizeof(double);
    setup_interface_kernel<<<V * 2, 32, shi, s>>>(sb.iface, sb.sinv, n, d_status);
  }
}

}  // namespace lq2d
