// Dimension-generic kernels: solver-state initialisation, the initial
// residual, norms, the right-hand side, layout conversion, input recovery and
// the device-loop control of Algorithm 1.
#include "kernels.h"

namespace lq2d {

const KernelTable* kernel_table_n1();
const KernelTable* kernel_table_n2();
const KernelTable* kernel_table_n3();
const KernelTable* kernel_table_n4();
const KernelTable* kernel_table_n5();
const KernelTable* kernel_table_n6();
const KernelTable* kernel_table_n7();
const KernelTable* kernel_table_n8();

const KernelTable* kernel_table(int n) {
  switch (n) {
    case 1: return kernel_table_n1();
    case 2: return kernel_table_n2();
    case 3: return kernel_table_n3();
    case 4: return kernel_table_n4();
    case 5: return kernel_table_n5();
    case 6: return kernel_table_n6();
    case 7: return kernel_table_n7();
    case 8: return kernel_table_n8();
    default: return nullptr;
  }
}

namespace {

__global__ void init_state_kernel(SolverState* st, double tol, int max_iter, int stop_mode, const double* bnorm2,
                                  int keep_iter, double* hist, int hist_cap, double phase_rho2) {
  st->mu = 0.0;
  st->beta = 0.0;
  st->ydot = 0.0;
  st->theta = 0.0;
  st->bnorm2 = *bnorm2;
  st->stop_mode = stop_mode;
  st->stop_bound = stop_mode == 0 ? tol * tol * st->bnorm2 : tol;
  st->tol_bound = st->stop_bound;
  st->phase_rho2 = stop_mode == 0 ? phase_rho2 : 0.0;
  st->replace = 0;
  if (!keep_iter) {
    st->iter = 0;
    st->replacements = 0;
  }
  st->max_iter = max_iter;
  st->done = 0;
  st->have_mu = 0;
  st->body_count = 0;
  st->body_cap = max_iter + 2;
  st->hist = hist;
  st->hist_cap = hist_cap;
  for (int c = 0; c < 8; ++c) st->counters[c] = 0u;
}

// Identity preconditioner (plain CG, used to estimate kappa(Delta)): q = r
// and mu = r'r.  With UPDATE, the update and stop test of Algorithm 1 come first (delta +=
// vartheta d, r -= vartheta y, stop test), and mu is the new ||r||^2.
template <bool UPDATE>
__global__ void ident_kernel(Grid g, double* __restrict__ r, double* __restrict__ delta,
                             const double* __restrict__ y, const double* __restrict__ d, double* __restrict__ q,
                             double* partials, SolverState* st) {
  if (st->done) return;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double vth = UPDATE ? st->theta : 0.0;
  double s2 = 0.0, mx = 0.0;
  if (idx < g.P) {
    for (int k = 0; k < g.n; ++k) {
      const long long e = k * g.Ps + idx;
      double rv = r[e];
      if (UPDATE) {
        rv -= vth * y[e];
        r[e] = rv;
        delta[e] += vth * d[e];
      }
      q[e] = rv;
      s2 += rv * rv;
      mx = fmax(mx, fabs(rv));
    }
  }
  double t0, t1;
  if (grid_reduce2<true>(s2, mx, partials, &st->counters[UPDATE ? kCntNorm : kCntMu], &t0, &t1)) {
    if (UPDATE) {
      st->rnorm2 = t0;
      st->rnorm_inf = t1;
      const int it = st->iter + 1;
      st->iter = it;
      record_theta(st, it - 1);
      const bool pass = st->stop_mode == 0 ? (t0 <= st->stop_bound) : (t1 < st->stop_bound);
      if (!isfinite(t0)) { st->done = kBreakdown; return; }
      if (pass) { st->done = kConverged; return; }
      if (it >= st->max_iter) { st->done = kMaxIter; return; }
    }
    if (!(t0 > 0.0)) { st->done = kBreakdown; return; }
    if (!st->have_mu) {
      st->beta = 0.0;
    } else {
      st->beta = t0 / st->mu;
      record_beta(st, st->iter - 1);
    }
    st->mu = t0;
    st->have_mu = 1;
  }
}

// Exit test of the standalone NBJM solver (Algorithm 2's exit test):
// ||a - b||_inf < eps, b = NULL meaning zero; counts the outer step.
template <typename VT>
__global__ void nbjm_diff_kernel(Grid g, const VT* __restrict__ a, const VT* __restrict__ b, double* partials,
                                 SolverState* st) {
  if (st->done) return;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double mx = 0.0;
  if (idx < g.P)
    for (int k = 0; k < g.n; ++k) {
      const long long e = sizeof(VT) == 4 ? iter_f32_index(g.n, k, idx) : k * g.Ps + idx;
      const double dv = (double)a[e] - (b != nullptr ? (double)b[e] : 0.0);
      mx = fmax(mx, fabs(dv));
    }
  double t0, t1;
  if (grid_reduce2<true>(0.0, mx, partials, &st->counters[kCntNorm], &t0, &t1)) {
    const int it = st->iter + 1;
    st->iter = it;
    st->rnorm_inf = t1;
    if (!isfinite(t1)) st->done = kBreakdown;
    else if (t1 < st->stop_bound) st->done = kConverged;
    else if (it >= st->max_iter) st->done = kMaxIter;
  }
}

// r^(0) = r_delta - Delta delta^(0) (Algorithm 1, initial residual) with y = Delta delta^(0)
// given (or zero), delta = delta^(0); then the initial stop test (reading:
// no iterations when r^(0) already passes).
__global__ void init_residual_kernel(Grid g, const double* __restrict__ rhs, const double* __restrict__ y,
                                     double* __restrict__ r, double* __restrict__ delta,
                                     const double* __restrict__ delta0, double* partials, SolverState* st) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s2 = 0.0, mx = 0.0;
  if (idx < g.P) {
    for (int k = 0; k < g.n; ++k) {
      const long long e = k * g.Ps + idx;
      double rv = rhs[e];
      if (y != nullptr) rv -= y[e];
      r[e] = rv;
      if (delta0 != delta) delta[e] = delta0 != nullptr ? delta0[e] : 0.0;
      s2 += rv * rv;
      mx = fmax(mx, fabs(rv));
    }
  }
  double t0, t1;
  if (grid_reduce2<true>(s2, mx, partials, &st->counters[kCntInit], &t0, &t1)) {
    st->rnorm2 = t0;
    st->rnorm_inf = t1;
    const bool pass = st->stop_mode == 0 ? (t0 <= st->tol_bound) : (t1 < st->tol_bound);
    st->rref2 = t0;
    if (!isfinite(t0)) st->done = kBreakdown;
    else if (pass) st->done = kConverged;
    else if (st->iter >= st->max_iter) st->done = kMaxIter;
  }
}

// Reliable update of precision mode 2 (Krylov products in FP32): when the
// step just taken set the replacement flag, r = r_delta - Delta delta with
// Delta delta computed in FP64 (y, by the two gated Delta kernels before
// this one) replaces the recurrence residual; the search direction d is
// kept, so the iteration continues instead of restarting.
__global__ void replace_residual_kernel(Grid g, const double* __restrict__ rhs, const double* __restrict__ y,
                                        double* __restrict__ r, double* partials, SolverState* st) {
  if (st->done || !st->replace) return;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s2 = 0.0, mx = 0.0;
  if (idx < g.P) {
    for (int k = 0; k < g.n; ++k) {
      const long long e = k * g.Ps + idx;
      const double rv = rhs[e] - y[e];
      r[e] = rv;
      s2 += rv * rv;
      mx = fmax(mx, fabs(rv));
    }
  }
  double t0, t1;
  if (grid_reduce2<true>(s2, mx, partials, &st->counters[kCntRepl], &t0, &t1)) {
    st->rnorm2 = t0;
    st->rnorm_inf = t1;
    st->rref2 = t0;
    st->replace = 0;
    st->replacements += 1;
    if (!isfinite(t0)) st->done = kBreakdown;
  }
}

__global__ void norms_kernel(Grid g, const double* __restrict__ v, int comps, double* partials, unsigned* counter,
                             double* out2) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s2 = 0.0, mx = 0.0;
  if (idx < g.P)
    for (int k = 0; k < comps; ++k) {
      const double x = v[k * g.Ps + idx];
      s2 += x * x;
      mx = fmax(mx, fabs(x));
    }
  double t0, t1;
  if (grid_reduce2<true>(s2, mx, partials, counter, &t0, &t1)) {
    out2[0] = t0;
    out2[1] = t1;
  }
}

// r_delta = -omega~ with omega~ = col(gamma, omega_0, ..., omega_{T-1})
// (Section II-A, reading A1 for the first block).
__global__ void build_rhs_kernel(Grid g, const double* __restrict__ x0, const double* __restrict__ w_api,
                                 double* __restrict__ rhs) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.P) return;
  const int Tp = g.T + 1;
  const int p = (int)(idx / Tp), t = (int)(idx % Tp);
  for (int k = 0; k < g.n; ++k) {
    double val;
    if (t == 0) val = -x0[(size_t)p * g.n + k];
    else val = w_api != nullptr ? -w_api[((size_t)(t - 1) * g.NN + p) * g.n + k] : 0.0;
    rhs[k * g.Ps + idx] = val;
  }
}

// host layout [slice][node][comp]  <->  internal layout [comp][node][slice]
__global__ void to_internal_kernel(const double* __restrict__ api, double* __restrict__ intl, int NN, int slices,
                                   int comps, long long stride) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)NN * slices;
  if (idx >= per * comps) return;
  const int k = (int)(idx / per);
  const long long rem = idx % per;
  const int p = (int)(rem / slices), t = (int)(rem % slices);
  intl[k * stride + rem] = api[((long long)t * NN + p) * comps + k];
}

__global__ void to_api_kernel(const double* __restrict__ intl, double* __restrict__ api, int NN, int slices,
                              int comps, long long stride) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)NN * slices;
  if (idx >= per * comps) return;
  const int k = (int)(idx % comps);
  const long long tp = idx / comps;
  const int p = (int)(tp % NN), t = (int)(tp / NN);
  api[idx] = intl[k * stride + (long long)p * slices + t];
}

// u = R~^-1 B~' delta: u_{p,t} = R_p^-1 B_p' delta_{p,t+1} (Section II-B).
__global__ void recover_u_kernel(Grid g, NodeData nd, const double* __restrict__ delta, double* __restrict__ u) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)g.NN * g.T) return;
  const int p = (int)(idx / g.T), t = (int)(idx % g.T);
  const int n = g.n, m = g.m;
  const double* RB = nd.RiBt + (size_t)p * m * n;
  const long long base = (long long)p * (g.T + 1) + t + 1;
  for (int mm = 0; mm < m; ++mm) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += RB[mm * n + k] * delta[k * g.Ps + base];
    u[mm * g.Pus + idx] = s;
  }
}

// Device-side loop control of Algorithm 1: keep iterating while no stop
// condition is set and the body has run fewer than body_cap times.
__global__ void loop_ctrl_kernel(SolverState* st, cudaGraphConditionalHandle h) {
  const int c = st->body_count + 1;
  st->body_count = c;
  int keep = (st->done == kRunning) && (c < st->body_cap);
  if (st->done == kRunning && !keep) st->done = kLoopCap;
  cudaGraphSetConditional(h, keep ? 1u : 0u);
}

__global__ void to_f32_kernel(const double* __restrict__ src, float* __restrict__ dst, long long count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = (float)src[i];
}

__global__ void to_f64_kernel(const float* __restrict__ src, double* __restrict__ dst, long long count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = (double)src[i];
}

// FP32 iterate (node-major) -> FP64 component planes, one thread per (node, t)
__global__ void iter_f32_to_f64_kernel(Grid g, const float* __restrict__ src, double* __restrict__ dst) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.P) return;
  for (int k = 0; k < g.n; ++k) dst[k * g.Ps + idx] = (double)src[iter_f32_index(g.n, k, idx)];
}

// Records of Phi_bar_{v,0} = blkdiag(Q^-1) for the n = 4 FP32 sweeps, in the
// record layout of the banded factors ([N2][N1][D^-1][F2][F1][L0^-1] blocks
// of (2n)^2): the unit factor is the identity (F = N = 0) and D^-1 =
// blkdiag(Q of node (i, 2v), Q of node (i, 2v+1)); a missing second column
// (odd N) gets zero rows.  One thread per record entry.
__global__ void t0_records_kernel(Grid g, const float* __restrict__ Q, float* __restrict__ rec, long long fac_rec) {
  const int n = g.n, G2 = 2 * n, BS = G2 * G2;
  const long long total = (long long)g.V * g.K * fac_rec;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const long long vr = e / fac_rec;  // (v, i) record
  const int within = (int)(e % fac_rec);
  const int v = (int)(vr / g.K), i = (int)(vr % g.K);
  float val = 0.f;
  if (within >= 2 * BS && within < 3 * BS) {
    const int rc = within - 2 * BS, a = rc / G2, b = rc % G2;
    const int ja = a / n, jb = b / n;
    const int j = 2 * v + ja;
    if (ja == jb && j < g.N) val = Q[((size_t)i * g.N + j) * n * n + (a % n) * n + (b % n)];
  }
  rec[e] = val;
}

inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

void launch_init_state(SolverState* st, double tol, int max_iter, int stop_mode, const double* bnorm2,
                       int keep_iter, double* hist, int hist_cap, double phase_rho2, cudaStream_t s) {
  init_state_kernel<<<1, 1, 0, s>>>(st, tol, max_iter, stop_mode, bnorm2, keep_iter, hist, hist_cap, phase_rho2);
}

void launch_ident(const Grid& g, bool update, double* r, double* delta, const double* y, const double* d,
                  double* q, double* partials, SolverState* st, cudaStream_t s) {
  if (update)
    ident_kernel<true><<<blocks_for(g.P, kOpThreads), kOpThreads, 0, s>>>(g, r, delta, y, d, q, partials, st);
  else
    ident_kernel<false><<<blocks_for(g.P, kOpThreads), kOpThreads, 0, s>>>(g, r, delta, y, d, q, partials, st);
}

void launch_nbjm_diff(const Grid& g, const void* a, const void* b, int fp32, double* partials, SolverState* st,
                      cudaStream_t s) {
  if (fp32)
    nbjm_diff_kernel<float><<<blocks_for(g.P, kOpThreads), kOpThreads, 0, s>>>(
        g, static_cast<const float*>(a), static_cast<const float*>(b), partials, st);
  else
    nbjm_diff_kernel<double><<<blocks_for(g.P, kOpThreads), kOpThreads, 0, s>>>(
        g, static_cast<const double*>(a), static_cast<const double*>(b), partials, st);
}

void launch_init_residual(const Grid& g, const double* rhs, const double* y, double* r, double* delta,
                          const double* delta0, double* partials, SolverState* st, cudaStream_t s) {
  init_residual_kernel<<<blocks_for(g.P, kOpThreads), kOpThreads, 0, s>>>(g, rhs, y, r, delta, delta0, partials, st);
}

void launch_replace_residual(const Grid& g, const double* rhs, const double* y, double* r, double* partials,
                             SolverState* st, cudaStream_t s) {
  replace_residual_kernel<<<blocks_for(g.P, kOpThreads), kOpThreads, 0, s>>>(g, rhs, y, r, partials, st);
}

void launch_norms(const Grid& g, const double* v, int comps, double* partials, unsigned int* counter,
                  double* out2, cudaStream_t s) {
  norms_kernel<<<blocks_for(g.P, kOpThreads), kOpThreads, 0, s>>>(g, v, comps, partials, counter, out2);
}

void launch_build_rhs(const Grid& g, const double* x0, const double* w_api, double* rhs, cudaStream_t s) {
  build_rhs_kernel<<<blocks_for(g.P, kOpThreads), kOpThreads, 0, s>>>(g, x0, w_api, rhs);
}

void launch_to_internal(const double* api, double* intl, int NN, int slices, int comps, long long stride,
                        cudaStream_t s) {
  const long long total = (long long)NN * slices * comps;
  to_internal_kernel<<<blocks_for(total, 256), 256, 0, s>>>(api, intl, NN, slices, comps, stride);
}

void launch_to_api(const double* intl, double* api, int NN, int slices, int comps, long long stride,
                   cudaStream_t s) {
  const long long total = (long long)NN * slices * comps;
  to_api_kernel<<<blocks_for(total, 256), 256, 0, s>>>(intl, api, NN, slices, comps, stride);
}

void launch_recover_u(const Grid& g, const NodeData& nd, const double* delta, double* u, cudaStream_t s) {
  recover_u_kernel<<<blocks_for((long long)g.NN * g.T, 256), 256, 0, s>>>(g, nd, delta, u);
}

void launch_loop_ctrl(SolverState* st, cudaGraphConditionalHandle h, cudaStream_t s) {
  loop_ctrl_kernel<<<1, 1, 0, s>>>(st, h);
}

void launch_to_f32(const double* src, float* dst, long long count, cudaStream_t s) {
  to_f32_kernel<<<blocks_for(count, 256), 256, 0, s>>>(src, dst, count);
}

void launch_to_f64(const float* src, double* dst, long long count, cudaStream_t s) {
  to_f64_kernel<<<blocks_for(count, 256), 256, 0, s>>>(src, dst, count);
}

// d = q + beta d (Algorithm 1's direction update, beta from the state; d = q
// when beta = 0), in FP64, once per node-time ahead of the Delta product,
// which then reads d instead of forming it for each stencil neighbour.  q is
// the preconditioner output: FP64 component planes, or FP32 node-major.
__global__ void direction_update_kernel(Grid g, const void* __restrict__ q, int q_f32, double* __restrict__ d,
                                        const SolverState* __restrict__ st) {
  if (st->done) return;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.P) return;
  const double beta = st->beta;
  for (int k = 0; k < g.n; ++k) {
    const double qv = q_f32 ? (double)static_cast<const float*>(q)[iter_f32_index(g.n, k, idx)]
                            : static_cast<const double*>(q)[k * g.Ps + idx];
    double* dp = d + k * g.Ps + idx;
    double v = qv;
    if (beta != 0.0) v += beta * *dp;
    *dp = v;
  }
}

void launch_direction_update(const Grid& g, const void* q, bool q_f32, double* d, const SolverState* st,
                             cudaStream_t s) {
  direction_update_kernel<<<(unsigned)((g.P + 255) / 256), 256, 0, s>>>(g, q, q_f32 ? 1 : 0, d, st);
}

void launch_iter_f32_to_f64(const Grid& g, const float* src, double* dst, cudaStream_t s) {
  iter_f32_to_f64_kernel<<<blocks_for(g.P, 256), 256, 0, s>>>(g, src, dst);
}

void launch_t0_records(const Grid& g, const float* Q32, float* rec, long long fac_rec, cudaStream_t s) {
  const long long total = (long long)g.V * g.K * fac_rec;
  t0_records_kernel<<<blocks_for(total, 256), 256, 0, s>>>(g, Q32, rec, fac_rec);
}

}  // namespace lq2d
