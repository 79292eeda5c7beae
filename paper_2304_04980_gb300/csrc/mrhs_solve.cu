// Multi-right-hand-side PCG (Algorithm 1 run for up to 32 right-hand sides
// of one problem side by side, with the tensor-core NBJM preconditioner of
// mrhs.cu).  Vectors are [n][K*N][T+1][32]: a warp takes one (node, t) and
// its lane is the right-hand side, so every access is 32 consecutive words
// and the per-right-hand-side scalars (alpha, beta, mu) live in one
// register per lane.  Reductions are per lane: warp partial sums are added
// across the CTA through shared memory, one slot per CTA and lane is
// written, and the last CTA adds the slots in a fixed order (deterministic).
//
// Precision follows precision mode 2 of the single-right-hand-side solver:
// r, delta and d are FP64; the product Delta d runs in FP32 from an FP32
// copy of d; once a right-hand side's recurrence residual has dropped by
// sqrt(rho2) since its last replacement, r = r_delta - Delta delta (FP64)
// replaces it, keeping the direction; the preconditioner is not exactly
// symmetric (TF32), so beta is the flexible ratio q_new'(r_new - r_old) /
// mu_old = -alpha q_new'y / mu_old.  A right-hand side whose residual meets
// the tolerance is frozen (alpha = beta = 0) while the others go on.
#include "kernels_hot.cuh"
#include "mrhs.h"

namespace lq2d {
namespace mrhs {

namespace {

constexpr int kWarps = 8;  // warps per CTA of the element-wise kernels
constexpr int kMaxBlocks = 1216;  // 8 per SM of a 152-SM GPU

// Sums NV values per lane over the grid; true in the last CTA's warp 0,
// whose lane r then holds the totals of right-hand side r in out[].  The
// last CTA adds the per-CTA slots with all its warps (warp w takes every
// kWarps-th CTA, then warp 0 adds the kWarps sums in order), so the result
// does not depend on the order in which CTAs finish.
template <int NV>
__device__ bool rhs_reduce(const double (&v)[NV], double* partials, unsigned int* counter, double (&out)[NV]) {
  __shared__ double red[NV][kWarps][32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) red[j][wid][lane] = v[j];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s += red[j][w][lane];
      partials[((size_t)blockIdx.x * NV + j) * 32 + lane] = s;
    }
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(counter, 1u);
    last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double s = 0.0;
#pragma unroll 8
    for (unsigned int b = wid; b < gridDim.x; b += kWarps) s += __ldcg(&partials[((size_t)b * NV + j) * 32 + lane]);
    red[j][wid][lane] = s;
  }
  __syncthreads();
  if (wid != 0) return false;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += red[j][w][lane];
    out[j] = s;
  }
  if (lane == 0) *counter = 0u;
  return true;
}

__device__ __forceinline__ long long vidx(const Grid& g, long long plane, int k, long long pt) {
  return k * plane + pt * kRhs;
}

__global__ void init_kernel(Grid g, int nrhs, const double* __restrict__ x0s, const double* __restrict__ rhs1,
                            long long rhs1_stride, SolveVecs v, double* partials, State* ms, SolverState* st,
                            double tol, double rho2, int max_iter) {
  const int lane = threadIdx.x & 31;
  const int Tp = g.T + 1;
  const long long P = (long long)g.NN * Tp, plane = P * kRhs;
  double acc = 0.0;
  for (long long it = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); it < P; it += (long long)gridDim.x * kWarps) {
    const int p = (int)(it / Tp), t = (int)(it % Tp);
#pragma unroll
    for (int k = 0; k < kN; ++k) {
      double val = 0.0;
      if (lane < nrhs) {
        if (t == 0) val = -x0s[((size_t)lane * g.NN + p) * kN + k];
        else if (rhs1 != nullptr) val = rhs1[k * rhs1_stride + (long long)p * Tp + t];
      }
      const long long e = vidx(g, plane, k, it) + lane;
      v.rhs[e] = val;
      v.r[e] = val;
      v.delta[e] = 0.0;
      v.d[e] = 0.0;
      v.d32[e] = 0.f;
      v.r32[e] = (float)val;
      acc += val * val;
    }
  }
  const double in[1] = {acc};
  double out[1];
  if (rhs_reduce<1>(in, partials, &ms->counter, out)) {
    const double b2 = out[0];
    ms->bnorm2[lane] = b2;
    ms->rnorm2[lane] = b2;
    ms->rref2[lane] = b2;
    ms->mu[lane] = ms->beta[lane] = ms->alpha[lane] = 0.0;
    const int conv = b2 <= tol * tol * b2;  // a zero right-hand side needs no step
    ms->conv[lane] = conv;
    ms->repl[lane] = 0;
    ms->iters[lane] = 0;
    const bool all = __all_sync(0xffffffffu, conv != 0);
    const bool bad = __any_sync(0xffffffffu, !isfinite(b2));
    if (lane == 0) {
      ms->nrhs = nrhs;
      ms->any_repl = 0;
      ms->have_mu = 0;
      ms->breakdown = bad ? 1 : 0;
      ms->tol2 = tol * tol;
      ms->rho2 = rho2;
      st->iter = 0;
      st->max_iter = max_iter;
      st->body_count = 0;
      st->body_cap = max_iter + 2;
      st->done = bad ? kBreakdown : (all ? kConverged : kRunning);
    }
  }
}

// z = Q~^-1 A~' dn (see delta_z_kernel): FP32 in the loop with dn = q + beta
// d32, FP64 for a replacement with dn = delta.
template <typename CT, bool LOOP>
__global__ void __launch_bounds__(kWarps * 32, 3) z_kernel(Grid g, OpData<CT> op, const float* __restrict__ q, const float* __restrict__ d32,
                         const double* __restrict__ delta, CT* __restrict__ z, const State* ms,
                         const SolverState* st, int force) {
  if (LOOP && st->done) return;
  if (!LOOP && !force && (st->done || !ms->any_repl)) return;
  const int lane = threadIdx.x & 31;
  const int Tp = g.T + 1;
  const long long P = (long long)g.NN * Tp, plane = P * kRhs;
  const CT beta = LOOP ? (CT)ms->beta[lane] : CT(0);
  auto dn_at = [&](int k, long long pt) -> CT {
    const long long e = vidx(g, plane, k, pt) + lane;
    if constexpr (LOOP) return (CT)q[e] + beta * (CT)d32[e];
    else return (CT)delta[e];
  };
  for (long long it = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); it < P; it += (long long)gridDim.x * kWarps) {
    const int p = (int)(it / Tp), t = (int)(it % Tp);
    const int i = p / g.N, j = p % g.N;
    CT w[kN];
#pragma unroll
    for (int k = 0; k < kN; ++k) w[k] = -dn_at(k, it);
    if (t < g.T) {
      // every neighbour's values are loaded before any is used, so that the
      // loads of the five directions are in flight together (an absent
      // neighbour reads the node's own row and is skipped below)
      int rn[5];
      CT dv[5][kN];
#pragma unroll
      for (int dir = 0; dir < 5; ++dir) {
        rn[dir] = nbr_node(i, j, dir, g.K, g.N);
        const long long rpt = (long long)(rn[dir] >= 0 ? rn[dir] : p) * Tp + t + 1;
#pragma unroll
        for (int c = 0; c < kN; ++c) dv[dir][c] = dn_at(c, rpt);
      }
#pragma unroll
      for (int dir = 0; dir < 5; ++dir) {
        if (rn[dir] < 0) continue;
        const CT* blk = hot::ahat_col<kN>(op, rn[dir], dir);
#pragma unroll
        for (int c = 0; c < kN; ++c)
#pragma unroll
          for (int k = 0; k < kN; ++k) w[k] += blk[c * kN + k] * dv[dir][c];
      }
    }
    const CT* Qb = (t == g.T ? op.QTi : op.Qi) + (size_t)p * kN * kN;
#pragma unroll
    for (int k = 0; k < kN; ++k) {
      CT s = CT(0);
#pragma unroll
      for (int c = 0; c < kN; ++c) s += Qb[k * kN + c] * w[c];
      z[vidx(g, plane, k, it) + lane] = s;
    }
  }
}

// y = A~ z + B~ R~^-1 B~' dn (see delta_y_kernel).  Loop: dn = q + beta d in
// FP64 is written back to d and d32, y' dn is reduced per right-hand side
// and alpha = mu / (y' dn) set (0 for frozen right-hand sides).
// Replacement: dn = delta, y in FP64.
template <typename CT, bool LOOP>
__global__ void __launch_bounds__(kWarps * 32, 3) y_kernel(Grid g, OpData<CT> op, const CT* __restrict__ z, const float* __restrict__ q, SolveVecs v,
                         double* partials, State* ms, SolverState* st, int force) {
  if (LOOP && st->done) return;
  if (!LOOP && !force && (st->done || !ms->any_repl)) return;
  const int lane = threadIdx.x & 31;
  const int Tp = g.T + 1;
  const long long P = (long long)g.NN * Tp, plane = P * kRhs;
  const double beta = LOOP ? ms->beta[lane] : 0.0;
  double acc = 0.0;
  for (long long it = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); it < P; it += (long long)gridDim.x * kWarps) {
    const int p = (int)(it / Tp), t = (int)(it % Tp);
    const int i = p / g.N, j = p % g.N;
    double dn[kN];
    CT yk[kN];
#pragma unroll
    for (int k = 0; k < kN; ++k) {
      const long long e = vidx(g, plane, k, it) + lane;
      dn[k] = LOOP ? (double)q[e] + beta * v.d[e] : v.delta[e];
      yk[k] = -z[e];
    }
    if (t >= 1) {
      // neighbour loads first (see z_kernel)
      int rn[5];
      CT zv[5][kN];
#pragma unroll
      for (int dir = 0; dir < 5; ++dir) {
        rn[dir] = nbr_node(i, j, dir, g.K, g.N);
        const long long rpt = (long long)(rn[dir] >= 0 ? rn[dir] : p) * Tp + t - 1;
#pragma unroll
        for (int c = 0; c < kN; ++c) zv[dir][c] = z[vidx(g, plane, c, rpt) + lane];
      }
#pragma unroll
      for (int dir = 0; dir < 5; ++dir) {
        if (rn[dir] < 0) continue;
        const CT* blk = hot::ahat_row<kN>(op, p, dir);
#pragma unroll
        for (int k = 0; k < kN; ++k)
#pragma unroll
          for (int c = 0; c < kN; ++c) yk[k] += blk[k * kN + c] * zv[dir][c];
      }
      const CT* S = op.Sb + (size_t)p * kN * kN;
#pragma unroll
      for (int k = 0; k < kN; ++k)
#pragma unroll
        for (int c = 0; c < kN; ++c) yk[k] += S[k * kN + c] * (CT)dn[c];
    }
#pragma unroll
    for (int k = 0; k < kN; ++k) {
      const long long e = vidx(g, plane, k, it) + lane;
      if constexpr (LOOP) {
        v.y32[e] = (float)yk[k];
        v.d[e] = dn[k];
        v.d32[e] = (float)dn[k];
        acc += (double)yk[k] * dn[k];
      } else {
        v.y64[e] = (double)yk[k];
      }
    }
  }
  if constexpr (LOOP) {
    const double in[1] = {acc};
    double out[1];
    if (rhs_reduce<1>(in, partials, &ms->counter, out)) {
      const int frozen = ms->conv[lane];
      const double yd = out[0];
      const bool bad = !frozen && (!(yd > 0.0) || !isfinite(yd));
      ms->alpha[lane] = (frozen || bad) ? 0.0 : ms->mu[lane] / yd;
      if (__any_sync(0xffffffffu, bad) && lane == 0) {
        ms->breakdown = 1;
        st->done = kBreakdown;
      }
    }
  }
}

__global__ void update_kernel(Grid g, SolveVecs v, double* partials, State* ms, SolverState* st) {
  if (st->done) return;
  const int lane = threadIdx.x & 31;
  const int Tp = g.T + 1;
  const long long P = (long long)g.NN * Tp, plane = P * kRhs;
  const double alpha = ms->alpha[lane];
  double acc = 0.0;
  for (long long it = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); it < P; it += (long long)gridDim.x * kWarps) {
#pragma unroll
    for (int k = 0; k < kN; ++k) {
      const long long e = vidx(g, plane, k, it) + lane;
      double rv = v.r[e];
      if (alpha != 0.0) {
        rv -= alpha * (double)v.y32[e];
        v.r[e] = rv;
        v.r32[e] = (float)rv;
        v.delta[e] += alpha * v.d[e];
      }
      acc += rv * rv;
    }
  }
  const double in[1] = {acc};
  double out[1];
  if (rhs_reduce<1>(in, partials, &ms->counter, out)) {
    const double r2 = out[0];
    ms->rnorm2[lane] = r2;
    int conv = ms->conv[lane];
    if (!conv) {
      ms->iters[lane] += 1;
      if (r2 <= ms->tol2 * ms->bnorm2[lane]) conv = 1;
      else if (ms->rho2 > 0.0 && r2 <= ms->rho2 * ms->rref2[lane]) ms->repl[lane] = 1;
      ms->conv[lane] = conv;
    }
    const bool all = __all_sync(0xffffffffu, conv != 0);
    const bool repl = __any_sync(0xffffffffu, ms->repl[lane] != 0);
    const bool bad = __any_sync(0xffffffffu, !isfinite(r2));
    if (lane == 0) {
      const int step = st->iter + 1;
      st->iter = step;
      ms->any_repl = repl ? 1 : 0;
      if (bad) st->done = kBreakdown;
      else if (all) st->done = kConverged;
      else if (step >= st->max_iter) st->done = kMaxIter;
    }
  }
}

__global__ void mu_kernel(Grid g, const float* __restrict__ q, SolveVecs v, double* partials, State* ms,
                          SolverState* st) {
  if (st->done) return;
  const int lane = threadIdx.x & 31;
  const int Tp = g.T + 1;
  const long long P = (long long)g.NN * Tp, plane = P * kRhs;
  double accm = 0.0, accy = 0.0;
  for (long long it = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); it < P; it += (long long)gridDim.x * kWarps) {
#pragma unroll
    for (int k = 0; k < kN; ++k) {
      const long long e = vidx(g, plane, k, it) + lane;
      const double qv = (double)q[e];
      accm += qv * v.r[e];
      accy += qv * (double)v.y32[e];
    }
  }
  const double in[2] = {accm, accy};
  double out[2];
  if (rhs_reduce<2>(in, partials, &ms->counter, out)) {
    const int frozen = ms->conv[lane];
    const double mu_new = out[0];
    bool bad = false;
    if (frozen) {
      ms->beta[lane] = 0.0;
    } else {
      bad = !(mu_new > 0.0) || !isfinite(mu_new) || !isfinite(out[1]);
      ms->beta[lane] = (ms->have_mu && !bad) ? -ms->alpha[lane] * out[1] / ms->mu[lane] : 0.0;
      ms->mu[lane] = mu_new;
    }
    const bool anybad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      ms->have_mu = 1;
      if (anybad) {
        ms->breakdown = 1;
        st->done = kBreakdown;
      }
    }
  }
}

__global__ void replace_kernel(Grid g, SolveVecs v, double* partials, State* ms, SolverState* st, int force) {
  if (!force && (st->done || !ms->any_repl)) return;
  const int lane = threadIdx.x & 31;
  const int Tp = g.T + 1;
  const long long P = (long long)g.NN * Tp, plane = P * kRhs;
  const bool mine = force || ms->repl[lane];
  double acc = 0.0;
  for (long long it = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); it < P; it += (long long)gridDim.x * kWarps) {
#pragma unroll
    for (int k = 0; k < kN; ++k) {
      const long long e = vidx(g, plane, k, it) + lane;
      if (mine) {
        const double rv = v.rhs[e] - v.y64[e];
        v.r[e] = rv;
        v.r32[e] = (float)rv;
        acc += rv * rv;
      }
    }
  }
  const double in[1] = {acc};
  double out[1];
  if (rhs_reduce<1>(in, partials, &ms->counter, out)) {
    if (mine) {
      ms->rnorm2[lane] = out[0];
      ms->rref2[lane] = out[0];
      ms->repl[lane] = 0;
    }
    if (force) {
      // the true residual decides convergence
      const int conv = out[0] <= ms->tol2 * ms->bnorm2[lane];
      ms->conv[lane] = conv;
      const bool all = __all_sync(0xffffffffu, conv != 0);
      if (lane == 0 && st->done != kBreakdown) st->done = all ? kConverged : kRunning;
    }
    if (lane == 0) ms->any_repl = 0;
  }
}

__global__ void gather_kernel(Grid g, const double* __restrict__ vec, int r, double* __restrict__ single) {
  const long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int Tp = g.T + 1;
  const long long P = (long long)g.NN * Tp, plane = P * kRhs;
  if (it >= P) return;
#pragma unroll
  for (int k = 0; k < kN; ++k) single[k * g.Ps + it] = vec[k * plane + it * kRhs + r];
}

}  // namespace

int solve_blocks(const Grid& g) {
  const long long P = (long long)g.NN * (g.T + 1);
  const long long b = (P + kWarps - 1) / kWarps;
  return (int)(b < kMaxBlocks ? b : kMaxBlocks);
}

void launch_init(const Grid& g, int nrhs, const double* x0s, const double* rhs1, long long rhs1_stride,
                 const SolveVecs& v, double* partials, State* ms, SolverState* st, double tol, double rho2,
                 int max_iter, cudaStream_t s) {
  init_kernel<<<solve_blocks(g), kWarps * 32, 0, s>>>(g, nrhs, x0s, rhs1, rhs1_stride, v, partials, ms, st, tol, rho2,
                                                       max_iter);
}

void launch_delta_loop(const Grid& g, const OpData<float>& op, const float* q, const SolveVecs& v,
                       double* partials, State* ms, SolverState* st, cudaStream_t s) {
  const int nb = solve_blocks(g);
  z_kernel<float, true><<<nb, kWarps * 32, 0, s>>>(g, op, q, v.d32, nullptr, v.z32, ms, st, 0);
  y_kernel<float, true><<<nb, kWarps * 32, 0, s>>>(g, op, v.z32, q, v, partials, ms, st, 0);
}

void launch_update(const Grid& g, const SolveVecs& v, double* partials, State* ms, SolverState* st, cudaStream_t s) {
  update_kernel<<<solve_blocks(g), kWarps * 32, 0, s>>>(g, v, partials, ms, st);
}

void launch_mu(const Grid& g, const float* q, const SolveVecs& v, double* partials, State* ms, SolverState* st,
               cudaStream_t s) {
  mu_kernel<<<solve_blocks(g), kWarps * 32, 0, s>>>(g, q, v, partials, ms, st);
}

void launch_replace(const Grid& g, const OpData<double>& op, const SolveVecs& v, double* partials, State* ms,
                    SolverState* st, bool force, cudaStream_t s) {
  const int nb = solve_blocks(g);
  z_kernel<double, false><<<nb, kWarps * 32, 0, s>>>(g, op, nullptr, nullptr, v.delta, v.z64, ms, st, force ? 1 : 0);
  y_kernel<double, false><<<nb, kWarps * 32, 0, s>>>(g, op, v.z64, nullptr, v, partials, ms, st, force ? 1 : 0);
  replace_kernel<<<nb, kWarps * 32, 0, s>>>(g, v, partials, ms, st, force ? 1 : 0);
}

void launch_gather(const Grid& g, const double* vec, int r, double* single, cudaStream_t s) {
  const long long P = (long long)g.NN * (g.T + 1);
  gather_kernel<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(g, vec, r, single);
}

}  // namespace mrhs
}  // namespace lq2d
