// Shared device-side definitions of the lq2d CUDA path.
//
// Vector layout in device memory ("internal layout"): component planes.
// A state-sized vector over the horizon holds n planes; plane k stores
//     v[k][p][t],  p = i*N + j (grid node),  t = 0..T,
// at offset k*Ps + p*(T+1) + t.  Consecutive threads take consecutive t of
// one node, so every load of a neighbour's value is a coalesced run, and the
// time-invariant per-node blocks are the same for a whole run of threads.
// Input-sized vectors (u) hold m planes of length K*N*T.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lq2d {

constexpr int kMaxN = 8;   // largest state dimension with compiled kernels
constexpr int kMaxM = 8;   // largest input dimension

// Device-resident scalars of one PCG solve (Algorithm 1).
struct SolverState {
  double mu;          // mu^(i) = q' r
  double beta;        // mu^(i+1) / mu^(i), used by the next direction update
  double ydot;        // y' d
  double theta;       // vartheta = mu / (y' d)
  double rnorm2;      // ||r||_2^2 after the last residual update
  double rnorm_inf;   // ||r||_inf after the last residual update
  double bnorm2;      // ||r_delta||_2^2
  double stop_bound;  // mode 0: (tol ||r_delta||)^2 against ||r||_2^2; mode 1: tol against ||r||_inf
  int iter;           // completed PCG steps
  int max_iter;
  int done;           // 0 running, 1 converged, 2 max_iter, 3 breakdown, 4 loop cap
  int stop_mode;      // 0 relative 2-norm, 1 absolute infinity norm
  int have_mu;        // 0 before the first preconditioner application
  int body_count;     // executions of the device-loop body
  int body_cap;       // hard cap on body executions
  int hist_cap;       // entries (pairs) available in hist
  unsigned int counters[8];  // arrival counters of the last-block reductions
  double* hist;       // optional: vartheta_j at [2j], beta_j at [2j+1] (Lanczos estimate), or NULL
  double tol_bound;   // the tolerance itself, in the units of stop_bound
  double phase_rho2;  // > 0 (precision mode 2): replace the recurrence residual by the true one once
                      // ||r||^2 <= phase_rho2 ||r_ref||^2
  double rref2;       // ||r||^2 at the start or at the last replacement
  int replace;        // set by the step whose residual met the replacement test; cleared by the replacement
  int replacements;   // residual replacements in this solve
};

// Records the PCG coefficients of step j (called by the last block of the
// reductions that produce them).
__device__ inline void record_theta(SolverState* st, int j) {
  if (st->hist != nullptr && j >= 0 && j < st->hist_cap) st->hist[2 * j] = st->theta;
}
__device__ inline void record_beta(SolverState* st, int j) {
  if (st->hist != nullptr && j >= 0 && j < st->hist_cap) st->hist[2 * j + 1] = st->beta;
}

enum StateDone { kRunning = 0, kConverged = 1, kMaxIter = 2, kBreakdown = 3, kLoopCap = 4 };
enum CounterSlot { kCntDot = 0, kCntNorm = 1, kCntMu = 2, kCntInit = 3, kCntKkt = 4, kCntAux = 5, kCntRepl = 6 };

struct Grid {
  int K, N, T, n, m, V, NN;
  int pad;
  long long P;    // NN*(T+1), length of one state plane
  long long Ps;   // stride between state planes
  long long Pu;   // NN*T, length of one input plane
  long long Pus;  // stride between input planes
};

// Per-node blocks, all row-major, all time-invariant.
struct NodeData {
  const double* Aself;  // [NN][n][n] A_{i,j}
  const double* Anb;    // [NN][4][n][n] E (j-1), F (j+1), G (i-1), H (i+1); blocks pointing off the grid are zero
  const double* Bm;     // [NN][n][m]
  const double* Qm;     // [NN][n][n] Q
  const double* QTm;    // [NN][n][n] Q_T
  const double* Rm;     // [NN][m][m] R
  const double* Qi;     // Q^-1
  const double* QTi;    // Q_T^-1
  const double* Sb;     // [NN][n][n] B R^-1 B'
  const double* RiBt;   // [NN][m][n] R^-1 B'
  const double* Om;     // [NN][5][n][n] Omega~ blocks towards the five off-pair neighbours
  const double* AQ;     // [NN][5][n][n] A_hat_{p,r} Q_r^-1,   r = self, west, east, north, south
  const double* QAt;    // [NN][5][n][n] Q_p^-1 A_hat_{r,p}',  same r
  const double* fac;    // banded block-Cholesky factors of Phi_bar_{v,class}
  long long fac_rec;    // doubles per pair-row record (24 n^2)
  long long fac_vc;     // doubles per (v, class) factor
};

// Neighbour directions of the 5-point stencil.
enum Dir { kSelf = 0, kWest = 1, kEast = 2, kNorth = 3, kSouth = 4 };

__host__ __device__ inline int nbr_node(int i, int j, int dir, int K, int N) {
  switch (dir) {
    case kSelf: return i * N + j;
    case kWest: return j >= 1 ? i * N + j - 1 : -1;
    case kEast: return j + 1 < N ? i * N + j + 1 : -1;
    case kNorth: return i >= 1 ? (i - 1) * N + j : -1;
    default: return i + 1 < K ? (i + 1) * N + j : -1;
  }
}

// Off-pair neighbours of node (i, j) that couple to it through
// A_hat Q^-1 A_hat' (Manhattan distance <= 2, column pair v = floor(j/2)):
// with s = -1 for the pair's left column and +1 for its right column,
//   o0 (i, j+s), o1 (i-1, j+s), o2 (i+1, j+s), o3 (i, j+2s), o4 (i, j-2s).
__host__ __device__ inline int offpair_node(int i, int j, int o, int K, int N) {
  const int s = (j & 1) ? 1 : -1;
  int ii = i, jj = j;
  switch (o) {
    case 0: jj = j + s; break;
    case 1: ii = i - 1; jj = j + s; break;
    case 2: ii = i + 1; jj = j + s; break;
    case 3: jj = j + 2 * s; break;
    default: jj = j - 2 * s; break;
  }
  if (ii < 0 || ii >= K || jj < 0 || jj >= N) return -1;
  return ii * N + jj;
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block reduction of two values (sum, and sum or max), then a deterministic
// last-block reduction over the per-block partials.  Every thread of the
// block must call it.  Returns true in thread 0 of the last block to arrive,
// with the grid totals in *out0 / *out1 (partials summed in block order).
// bid / nblocks: this block's index among the blocks that share `counter`
// and `partials` (the launch's blocks, or one problem's work units inside a
// batched launch).
template <bool SECOND_IS_MAX>
__device__ inline bool grid_reduce2_at(double v0, double v1, double* partials, unsigned int* counter,
                                       double* out0, double* out1, unsigned bid, unsigned nblocks) {
  __shared__ double s0[32];
  __shared__ double s1[32];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v0 = warp_sum(v0);
  v1 = SECOND_IS_MAX ? warp_max(v1) : warp_sum(v1);
  if (lane == 0) { s0[wid] = v0; s1[wid] = v1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < nw; ++w) { a += s0[w]; b = SECOND_IS_MAX ? fmax(b, s1[w]) : b + s1[w]; }
    partials[2 * bid] = a;
    partials[2 * bid + 1] = b;
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == nblocks - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  // The last block sums the partials with a fixed assignment and a fixed
  // tree, so the result does not depend on the order of arrival.
  double a = 0.0, b = 0.0;
  for (unsigned int blk = threadIdx.x; blk < nblocks; blk += blockDim.x) {
    const volatile double* vp = partials;
    a += vp[2 * blk];
    b = SECOND_IS_MAX ? fmax(b, vp[2 * blk + 1]) : b + vp[2 * blk + 1];
  }
  a = warp_sum(a);
  b = SECOND_IS_MAX ? warp_max(b) : warp_sum(b);
  __syncthreads();
  if (lane == 0) { s0[wid] = a; s1[wid] = b; }
  __syncthreads();
  if (threadIdx.x != 0) return false;
  double ta = 0.0, tb = 0.0;
  for (int w = 0; w < nw; ++w) { ta += s0[w]; tb = SECOND_IS_MAX ? fmax(tb, s1[w]) : tb + s1[w]; }
  *out0 = ta;
  *out1 = tb;
  *counter = 0u;
  return true;
}

template <bool SECOND_IS_MAX>
__device__ inline bool grid_reduce2(double v0, double v1, double* partials, unsigned int* counter,
                                    double* out0, double* out1) {
  return grid_reduce2_at<SECOND_IS_MAX>(v0, v1, partials, counter, out0, out1, blockIdx.x, gridDim.x);
}

}  // namespace lq2d
