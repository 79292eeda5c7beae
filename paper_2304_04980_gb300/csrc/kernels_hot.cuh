// Hot kernels of one PCG step, templated on the state dimension NS.
// Included once per NS by inst_n*.cu.
//
// Paper: Algorithm 1 (PCGM) and Algorithm 2 (NBJM with fixed S x L sweeps);
// Section II-B (Delta = A~ Q~^-1 A~' + B~ R~^-1 B~', applied matrix-free);
// Section IV-B (the Phi~ solve splits into V x (T+1) banded block solves).
#pragma once

#include "kernels.h"

namespace lq2d {
namespace hot {

// A_hat block in row p, column "p's neighbour in direction dir".
template <int NS, typename D>
__device__ __forceinline__ auto ahat_row(const D& nd, int p, int dir) {
  return dir == kSelf ? nd.Aself + (size_t)p * NS * NS : nd.Anb + ((size_t)p * 4 + (dir - 1)) * NS * NS;
}

// A_hat block in row r, column p, for r = neighbour of p in direction dir.
template <int NS, typename D>
__device__ __forceinline__ auto ahat_col(const D& nd, int r, int dir) {
  const int slot = dir == kWest ? 1 : dir == kEast ? 0 : dir == kNorth ? 3 : 2;  // F, E, H, G of r
  return dir == kSelf ? nd.Aself + (size_t)r * NS * NS : nd.Anb + ((size_t)r * 4 + slot) * NS * NS;
}

// Element of the preconditioner output q at component k of (node, t) with
// pt = node*(T+1) + t: component planes in FP64, node-major in FP32 (the
// layout of the FP32 sweeps' iterates, iter_f32_index).
template <int NS, typename QT>
__device__ __forceinline__ long long q_index(const Grid& g, int k, long long pt) {
  if constexpr (sizeof(QT) == 4) return iter_f32_index(NS, k, pt);
  else return k * g.Ps + pt;
}

// The NS components of a node-time pt of a vector in that layout (FP32
// node-major, one 16-byte access at NS = 4; FP64 component planes).  The
// Delta product's FP32 temporaries (z, the FP32 copy of d) use it too.
template <int NS, typename T>
__device__ __forceinline__ void load_iter(const Grid& g, const T* __restrict__ v, long long pt, T (&out)[NS]) {
  if constexpr (sizeof(T) == 4 && NS == 4) {
    const float4 x = *reinterpret_cast<const float4*>(v + pt * 4);
    out[0] = x.x; out[1] = x.y; out[2] = x.z; out[3] = x.w;
  } else {
#pragma unroll
    for (int k = 0; k < NS; ++k) out[k] = v[q_index<NS, T>(g, k, pt)];
  }
}
template <int NS, typename T>
__device__ __forceinline__ void store_iter(const Grid& g, T* __restrict__ v, long long pt, const T (&in)[NS]) {
  if constexpr (sizeof(T) == 4 && NS == 4) {
    *reinterpret_cast<float4*>(v + pt * 4) = make_float4(in[0], in[1], in[2], in[3]);
  } else {
#pragma unroll
    for (int k = 0; k < NS; ++k) v[q_index<NS, T>(g, k, pt)] = in[k];
  }
}

// An NS x NS node block (row-major) into registers, in 16-byte loads at
// NS = 4 (every block starts at a multiple of 64 bytes).
template <int NS, typename T>
__device__ __forceinline__ void load_block(const T* __restrict__ b, T (&out)[NS * NS]) {
  if constexpr (NS == 4 && sizeof(T) == 4) {
    const float4* v = reinterpret_cast<const float4*>(b);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float4 x = v[e];
      out[4 * e] = x.x; out[4 * e + 1] = x.y; out[4 * e + 2] = x.z; out[4 * e + 3] = x.w;
    }
  } else if constexpr (NS == 4 && sizeof(T) == 8) {
    const double2* v = reinterpret_cast<const double2*>(b);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const double2 x = v[e];
      out[2 * e] = x.x; out[2 * e + 1] = x.y;
    }
  } else {
#pragma unroll
    for (int e = 0; e < NS * NS; ++e) out[e] = b[e];
  }
}

// ---------------------------------------------------------------------------
// Delta apply, part 1: z = Q~^-1 A~' dn, one thread per (node, t).
//   (A~' dn)_t = -dn_t + A_hat' dn_{t+1}   (t < T),   (A~' dn)_T = -dn_T
//   z_t = Q_t^-1 (A~' dn)_t                 (Q_T at t = T)
// dn = q + beta d_old is formed on the fly (the direction update of
// Algorithm 1 fused into its operator product); beta comes from the device
// state.  use_beta: 0 plain, 1 with the direction update (skipped once the
// loop has stopped), 2 plain but only when the state asks for a residual
// replacement (the reliable update of precision mode 2).
// ---------------------------------------------------------------------------
template <int NS, typename QT, typename CT, typename DT>
__device__ __forceinline__ void delta_z_body(const Grid& g, const OpData<CT>& nd, const QT* __restrict__ q,
                                             const DT* __restrict__ dold, CT* __restrict__ z,
                                             const SolverState* __restrict__ st, int use_beta, long long bid) {
  if (use_beta == 1 && st->done) return;
  if (use_beta == 2 && (st->done || !st->replace)) return;
  const long long idx = bid * kOpThreads + threadIdx.x;
  if (idx >= g.P) return;
  const int Tp = g.T + 1;
  const int p = (int)(idx / Tp), t = (int)(idx % Tp);
  const int i = p / g.N, j = p % g.N;
  // dn = q + beta d_old is formed in the precision of d_old (FP64, or FP32
  // when the FP32 copy of d is read)
  const DT beta = use_beta == 1 ? (DT)st->beta : DT(0);
  const bool mix = beta != DT(0) && dold != nullptr;  // no d_old: q already holds the new direction
  // d_old: FP64 component planes, or the FP32 copy (node-major)
  auto dn_at = [&](long long pt, CT (&out)[NS], bool negate) {
    QT qv[NS];
    load_iter<NS, QT>(g, q, pt, qv);
    DT dv[NS];
    if (mix) load_iter<NS, DT>(g, dold, pt, dv);
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      DT d = (DT)qv[k];
      if (mix) d += beta * dv[k];
      out[k] = negate ? (CT)(-d) : (CT)d;
    }
  };
  CT w[NS];
  dn_at(idx, w, true);
  if (t < g.T) {
#pragma unroll
    for (int dir = 0; dir < 5; ++dir) {
      const int r = nbr_node(i, j, dir, g.K, g.N);
      if (r < 0) continue;
      CT blk[NS * NS];
      load_block<NS, CT>(ahat_col<NS>(nd, r, dir), blk);
      CT dv[NS];
      dn_at((long long)r * Tp + t + 1, dv, false);
#pragma unroll
      for (int c = 0; c < NS; ++c)
#pragma unroll
        for (int k = 0; k < NS; ++k) w[k] += blk[c * NS + k] * dv[c];
    }
  }
  CT Qb[NS * NS];
  load_block<NS, CT>((t == g.T ? nd.QTi : nd.Qi) + (size_t)p * NS * NS, Qb);
  CT zv[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    CT s = CT(0);
#pragma unroll
    for (int c = 0; c < NS; ++c) s += Qb[k * NS + c] * w[c];
    zv[k] = s;
  }
  store_iter<NS, CT>(g, z, idx, zv);  // FP32 z: node-major, read only by delta_y
}

template <int NS, typename QT, typename CT, typename DT>
__global__ void __launch_bounds__(kOpThreads) delta_z_kernel(Grid g, OpData<CT> nd, const QT* __restrict__ q,
                                                             const DT* __restrict__ dold,
                                                             CT* __restrict__ z,
                                                             const SolverState* __restrict__ st, int use_beta) {
  delta_z_body<NS, QT, CT, DT>(g, nd, q, dold, z, st, use_beta, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Delta apply, part 2: y = A~ z + B~ R~^-1 B~' dn, one thread per (node, t).
//   y_0 = -z_0,   y_t = A_hat z_{t-1} - z_t + S dn_t   (t >= 1, S = B R^-1 B')
// Loop mode (Algorithm 1: operator product, step length, direction update): dn = q + beta d_old is written back
// to d (each thread owns its entry), y' dn is reduced and vartheta set.
// Plain mode with a state: runs only when the state asks for a residual
// replacement (the reliable update of precision mode 2).
// ---------------------------------------------------------------------------
template <int NS, bool LOOP, typename QT, typename CT>
__device__ __forceinline__ void delta_y_body(const Grid& g, const OpData<CT>& nd, const CT* __restrict__ z,
                                             const QT* __restrict__ q, const double* __restrict__ dold,
                                             double* __restrict__ dout, float* __restrict__ dout32,
                                             double* __restrict__ y, double* __restrict__ partials,
                                             SolverState* st, long long bid, long long nblocks) {
  if (LOOP && st->done) return;
  if (!LOOP && st != nullptr && (st->done || !st->replace)) return;
  const long long idx = bid * kOpThreads + threadIdx.x;
  double acc = 0.0;
  if (idx < g.P) {
    const int Tp = g.T + 1;
    const int p = (int)(idx / Tp), t = (int)(idx % Tp);
    const int i = p / g.N, j = p % g.N;
    const double beta = LOOP ? st->beta : 0.0;
    double dn[NS];
    CT dnc[NS], yk[NS];
    {
      QT qv[NS];
      load_iter<NS, QT>(g, q, idx, qv);
      double dv[NS];
      const bool mix = LOOP && beta != 0.0 && dold != nullptr;  // no d_old: q is the new direction
      if (mix) load_iter<NS, double>(g, dold, idx, dv);
      CT zs[NS];
      load_iter<NS, CT>(g, z, idx, zs);
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        double d = (double)qv[k];
        if (mix) d += beta * dv[k];
        dn[k] = d;
        dnc[k] = (CT)d;
        yk[k] = -zs[k];
      }
    }
    if (t >= 1) {
#pragma unroll
      for (int dir = 0; dir < 5; ++dir) {
        const int r = nbr_node(i, j, dir, g.K, g.N);
        if (r < 0) continue;
        CT blk[NS * NS];
        load_block<NS, CT>(ahat_row<NS>(nd, p, dir), blk);
        CT zv[NS];
        load_iter<NS, CT>(g, z, (long long)r * Tp + t - 1, zv);
#pragma unroll
        for (int k = 0; k < NS; ++k)
#pragma unroll
          for (int c = 0; c < NS; ++c) yk[k] += blk[k * NS + c] * zv[c];
      }
      CT S[NS * NS];
      load_block<NS, CT>(nd.Sb + (size_t)p * NS * NS, S);
#pragma unroll
      for (int k = 0; k < NS; ++k)
#pragma unroll
        for (int c = 0; c < NS; ++c) yk[k] += S[k * NS + c] * dnc[c];
    }
    CT part = CT(0);  // FP32 product: y'dn of the node-time in FP32, summed in FP64 below
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      y[k * g.Ps + idx] = (double)yk[k];
      if (LOOP) {
        if (dout != nullptr) dout[k * g.Ps + idx] = dn[k];
        if constexpr (sizeof(CT) == 4) part += yk[k] * dnc[k];
        else acc += (double)yk[k] * dn[k];
      }
    }
    if (LOOP && sizeof(CT) == 4) {
      acc = (double)part;
      if (dout32 != nullptr) {
        float d32[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) d32[k] = (float)dnc[k];
        store_iter<NS, float>(g, dout32, idx, d32);  // node-major, read by the next delta_z
      }
    }
  }
  if (LOOP) {
    double tot0, tot1;
    if (grid_reduce2_at<false>(acc, 0.0, partials, &st->counters[kCntDot], &tot0, &tot1, (unsigned)bid,
                               (unsigned)nblocks)) {
      st->ydot = tot0;
      if (!(tot0 > 0.0) || !isfinite(tot0)) st->done = kBreakdown;
      else st->theta = st->mu / tot0;
    }
  }
}

template <int NS, bool LOOP, typename QT, typename CT>
__global__ void __launch_bounds__(kOpThreads) delta_y_kernel(Grid g, OpData<CT> nd, const CT* __restrict__ z,
                                                             const QT* __restrict__ q,
                                                             const double* __restrict__ dold,
                                                             double* __restrict__ dout, float* __restrict__ dout32,
                                                             double* __restrict__ y, double* __restrict__ partials,
                                                             SolverState* st) {
  delta_y_body<NS, LOOP, QT, CT>(g, nd, z, q, dold, dout, dout32, y, partials, st, blockIdx.x, gridDim.x);
}

}  // namespace hot
}  // namespace lq2d

#include "sweep_tiled.cuh"

namespace lq2d {
namespace hot {

// ---------------------------------------------------------------------------
// Recovery check (Section II-B): the full KKT residual of (x, u, delta) and
// the cost, one thread per (node, t).
//   r1 = Q_t x_t - (A~' delta)_t,  r2 = R u_t - B' delta_{t+1},
//   r3 = (A~ x + B~ u + omega~)_t
// ---------------------------------------------------------------------------
template <int NS>
__global__ void __launch_bounds__(kOpThreads) kkt_kernel(Grid g, NodeData nd, const double* __restrict__ x,
                                                         const double* __restrict__ u,
                                                         const double* __restrict__ delta,
                                                         const double* __restrict__ rhs,
                                                         double* __restrict__ partials, SolverState* st,
                                                         double* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double res2 = 0.0, cost2 = 0.0, rmax = 0.0;
  if (idx < g.P) {
    const int Tp = g.T + 1, m = g.m;
    const int p = (int)(idx / Tp), t = (int)(idx % Tp);
    const int i = p / g.N, j = p % g.N;
    double xv[NS], r3[NS], atd[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      xv[k] = x[k * g.Ps + idx];
      r3[k] = -xv[k] - rhs[k * g.Ps + idx];  // omega~ = -r_delta
      atd[k] = -delta[k * g.Ps + idx];
    }
    if (t >= 1) {
#pragma unroll
      for (int dir = 0; dir < 5; ++dir) {
        const int r = nbr_node(i, j, dir, g.K, g.N);
        if (r < 0) continue;
        const double* blk = ahat_row<NS>(nd, p, dir);
        const long long ridx = (long long)r * Tp + t - 1;
#pragma unroll
        for (int k = 0; k < NS; ++k)
#pragma unroll
          for (int c = 0; c < NS; ++c) r3[k] += blk[k * NS + c] * x[c * g.Ps + ridx];
      }
      const double* B = nd.Bm + (size_t)p * NS * m;
      for (int mm = 0; mm < m; ++mm) {
        const double uv = u[mm * g.Pus + (long long)p * g.T + t - 1];
#pragma unroll
        for (int k = 0; k < NS; ++k) r3[k] += B[k * m + mm] * uv;
      }
    }
    if (t < g.T) {
#pragma unroll
      for (int dir = 0; dir < 5; ++dir) {
        const int r = nbr_node(i, j, dir, g.K, g.N);
        if (r < 0) continue;
        const double* blk = ahat_col<NS>(nd, r, dir);
        const long long ridx = (long long)r * Tp + t + 1;
#pragma unroll
        for (int c = 0; c < NS; ++c) {
          const double dv = delta[c * g.Ps + ridx];
#pragma unroll
          for (int k = 0; k < NS; ++k) atd[k] += blk[c * NS + k] * dv;
        }
      }
      // r2 and the input cost
      const double* B = nd.Bm + (size_t)p * NS * m;
      const double* R = nd.Rm + (size_t)p * m * m;
      for (int mm = 0; mm < m; ++mm) {
        double ru = 0.0, btd = 0.0;
        const double um = u[mm * g.Pus + (long long)p * g.T + t];
        for (int c = 0; c < m; ++c) ru += R[mm * m + c] * u[c * g.Pus + (long long)p * g.T + t];
#pragma unroll
        for (int k = 0; k < NS; ++k) btd += B[k * m + mm] * delta[k * g.Ps + idx + 1];
        res2 += (ru - btd) * (ru - btd);
        cost2 += um * ru;
      }
    }
    const double* Qw = (t == g.T ? nd.QTm : nd.Qm) + (size_t)p * NS * NS;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      double qx = 0.0;
#pragma unroll
      for (int c = 0; c < NS; ++c) qx += Qw[k * NS + c] * xv[c];
      const double r1 = qx - atd[k];
      res2 += r1 * r1 + r3[k] * r3[k];
      cost2 += xv[k] * qx;
      rmax = fmax(rmax, fabs(r3[k]));
    }
  }
  double tot0, tot1;
  if (grid_reduce2<false>(res2, cost2, partials, &st->counters[kCntKkt], &tot0, &tot1)) {
    out[0] = tot0;
    out[1] = tot1;
  }
  if (grid_reduce2<true>(0.0, rmax, partials + 2 * (size_t)gridDim.x, &st->counters[kCntAux], &tot0, &tot1)) {
    out[2] = tot1;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int NS, typename QT, typename CT, typename DT>
void launch_delta_z(const Grid& g, const OpData<CT>& op, const QT* q, const DT* dold, CT* z,
                    const SolverState* st, int use_beta, cudaStream_t s) {
  const long long blocks = (g.P + kOpThreads - 1) / kOpThreads;
  delta_z_kernel<NS, QT, CT, DT><<<(unsigned)blocks, kOpThreads, 0, s>>>(g, op, q, dold, z, st, use_beta);
}

template <int NS, typename QT, typename CT>
void launch_delta_y_impl(const Grid& g, const OpData<CT>& op, const CT* z, const QT* q, const double* dold,
                         double* dout, float* dout32, double* y, double* partials, SolverState* st, int loop_mode,
                         cudaStream_t s) {
  const long long blocks = (g.P + kOpThreads - 1) / kOpThreads;
  if (loop_mode)
    delta_y_kernel<NS, true, QT, CT>
        <<<(unsigned)blocks, kOpThreads, 0, s>>>(g, op, z, q, dold, dout, dout32, y, partials, st);
  else
    delta_y_kernel<NS, false, QT, CT>
        <<<(unsigned)blocks, kOpThreads, 0, s>>>(g, op, z, q, dold, dout, dout32, y, partials, st);
}

template <int NS, typename QT, typename CT>
void launch_delta_y(const Grid& g, const OpData<CT>& op, const CT* z, const QT* q, const double* dold,
                    double* dout, double* y, double* partials, SolverState* st, int loop_mode, cudaStream_t s) {
  launch_delta_y_impl<NS, QT, CT>(g, op, z, q, dold, dout, nullptr, y, partials, st, loop_mode, s);
}

template <int NS, typename VT, int THR>
void launch_sweep_t(int variant, const Grid& g, const PrecData<VT>& pd, const SweepArgsT<VT>& a, SolverState* st,
                    cudaStream_t s) {
  const unsigned blocks = sweep_blocks<NS, THR>(g);
  const size_t shm = sweep_smem_bytes<NS, VT, THR>();
  switch (variant) {
    case kSweepPlain: nbjm_sweep_kernel<NS, kSweepPlain, VT, THR><<<blocks, THR, shm, s>>>(g, pd, a, st); break;
    case kSweepUpdate: nbjm_sweep_kernel<NS, kSweepUpdate, VT, THR><<<blocks, THR, shm, s>>>(g, pd, a, st); break;
    case kSweepOmega: nbjm_sweep_kernel<NS, kSweepOmega, VT, THR><<<blocks, THR, shm, s>>>(g, pd, a, st); break;
    case kSweepOmegaMu: nbjm_sweep_kernel<NS, kSweepOmegaMu, VT, THR><<<blocks, THR, shm, s>>>(g, pd, a, st); break;
    case kSweepXiOmega: nbjm_sweep_kernel<NS, kSweepXiOmega, VT, THR><<<blocks, THR, shm, s>>>(g, pd, a, st); break;
    default: nbjm_sweep_kernel<NS, kSweepXi, VT, THR><<<blocks, THR, shm, s>>>(g, pd, a, st); break;
  }
}

// The two-ended (twisted) sweep: CTAs of 2 THR threads, same tiles.
template <int NS, typename VT, int THR>
void launch_sweep_twisted_t(int variant, const Grid& g, const PrecData<VT>& pd, const SweepArgsT<VT>& a,
                            SolverState* st, cudaStream_t s) {
  const unsigned blocks = sweep_blocks<NS, THR>(g);
  const size_t shm = sweep_twisted_smem_bytes<NS, VT, THR>();
  switch (variant) {
    case kSweepPlain: nbjm_sweep_twisted_kernel<NS, kSweepPlain, VT, THR><<<blocks, 2 * THR, shm, s>>>(g, pd, a, st); break;
    case kSweepUpdate: nbjm_sweep_twisted_kernel<NS, kSweepUpdate, VT, THR><<<blocks, 2 * THR, shm, s>>>(g, pd, a, st); break;
    case kSweepOmega: nbjm_sweep_twisted_kernel<NS, kSweepOmega, VT, THR><<<blocks, 2 * THR, shm, s>>>(g, pd, a, st); break;
    case kSweepOmegaMu: nbjm_sweep_twisted_kernel<NS, kSweepOmegaMu, VT, THR><<<blocks, 2 * THR, shm, s>>>(g, pd, a, st); break;
    default: nbjm_sweep_twisted_kernel<NS, kSweepXi, VT, THR><<<blocks, 2 * THR, shm, s>>>(g, pd, a, st); break;
  }
}

template <int NS, typename VT, int THR>
cudaError_t prepare_twisted_t() {
  const int shm = (int)sweep_twisted_smem_bytes<NS, VT, THR>();
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
    if (r != cudaSuccess) e = r;
  };
  set((const void*)nbjm_sweep_twisted_kernel<NS, kSweepPlain, VT, THR>);
  set((const void*)nbjm_sweep_twisted_kernel<NS, kSweepUpdate, VT, THR>);
  set((const void*)nbjm_sweep_twisted_kernel<NS, kSweepOmega, VT, THR>);
  set((const void*)nbjm_sweep_twisted_kernel<NS, kSweepOmegaMu, VT, THR>);
  set((const void*)nbjm_sweep_twisted_kernel<NS, kSweepXi, VT, THR>);
  return e;
}

// Sweep launch with the CTA width (threads) chosen for the problem: 32, 64,
// 128 or 256 threads, i.e. a tile of threads/GS time steps per CTA.  The
// two-ended solve (pd.sinv set, n = 4, widths 32 and 64, every variant but
// the standalone solver's first sweep) runs CTAs of twice that width.
template <int NS, typename VT>
void launch_sweep(int variant, int threads, const Grid& g, const PrecData<VT>& pd, const SweepArgsT<VT>& a,
                  SolverState* st, cudaStream_t s) {
  if constexpr (NS == 4) {
    if (pd.sinv != nullptr && variant != kSweepXiOmega && (threads == 32 || threads == 64)) {
      if (threads == 32) launch_sweep_twisted_t<NS, VT, 32>(variant, g, pd, a, st, s);
      else launch_sweep_twisted_t<NS, VT, 64>(variant, g, pd, a, st, s);
      return;
    }
  }
  switch (threads) {
    case 32: launch_sweep_t<NS, VT, 32>(variant, g, pd, a, st, s); break;
    case 64: launch_sweep_t<NS, VT, 64>(variant, g, pd, a, st, s); break;
    case 256: launch_sweep_t<NS, VT, 256>(variant, g, pd, a, st, s); break;
    default: launch_sweep_t<NS, VT, 128>(variant, g, pd, a, st, s); break;
  }
}

// Allows every sweep instantiation its shared-memory footprint (above the
// 48 KB default for n >= 8 in FP64); called once per device before use.
template <int NS, typename VT, int THR>
cudaError_t prepare_sweeps_t() {
  const int shm = (int)sweep_smem_bytes<NS, VT, THR>();
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
    if (r != cudaSuccess) e = r;
  };
  set((const void*)nbjm_sweep_kernel<NS, kSweepPlain, VT, THR>);
  set((const void*)nbjm_sweep_kernel<NS, kSweepUpdate, VT, THR>);
  set((const void*)nbjm_sweep_kernel<NS, kSweepOmega, VT, THR>);
  set((const void*)nbjm_sweep_kernel<NS, kSweepOmegaMu, VT, THR>);
  set((const void*)nbjm_sweep_kernel<NS, kSweepXi, VT, THR>);
  set((const void*)nbjm_sweep_kernel<NS, kSweepXiOmega, VT, THR>);
  return e;
}

template <int NS>
cudaError_t prepare_sweeps() {
  cudaError_t e[4] = {prepare_sweeps_t<NS, double, 32>(), prepare_sweeps_t<NS, double, 64>(),
                      prepare_sweeps_t<NS, double, 128>(), prepare_sweeps_t<NS, double, 256>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  cudaError_t f[4] = {prepare_sweeps_t<NS, float, 32>(), prepare_sweeps_t<NS, float, 64>(),
                      prepare_sweeps_t<NS, float, 128>(), prepare_sweeps_t<NS, float, 256>()};
  for (cudaError_t x : f)
    if (x != cudaSuccess) return x;
  if constexpr (NS == 4) {
    // n = 4 also has two-ended sweeps and FP32 sweeps with bulk-copy staging
    cudaError_t t[4] = {prepare_twisted_t<NS, double, 32>(), prepare_twisted_t<NS, double, 64>(),
                        prepare_twisted_t<NS, float, 32>(), prepare_twisted_t<NS, float, 64>()};
    for (cudaError_t x : t)
      if (x != cudaSuccess) return x;
    return prepare_sweep4_f32();
  }
  return cudaSuccess;
}

// FP32 sweep: for n = 4 with steps >= 1 the bulk-copy kernels (a lane
// carries `steps` time steps), else the tiled kernel.
template <int NS>
void launch_sweep_f32(int variant, int threads, int steps, const Grid& g, const PrecData<float>& pd,
                      const SweepArgsT<float>& a, SolverState* st, cudaStream_t s) {
  if constexpr (NS == 4) {
    if (steps >= 1) {
      launch_sweep4_f32(variant, threads, steps, g, pd, a, st, s);
      return;
    }
  }
  launch_sweep<NS, float>(variant, threads, g, pd, a, st, s);
}

template <int NS>
void launch_kkt(const Grid& g, const NodeData& nd, const double* x, const double* u, const double* delta,
                const double* rhs, double* partials, SolverState* st, double* out, cudaStream_t s) {
  const long long blocks = (g.P + kOpThreads - 1) / kOpThreads;
  kkt_kernel<NS><<<(unsigned)blocks, kOpThreads, 0, s>>>(g, nd, x, u, delta, rhs, partials, st, out);
}

template <int NS>
const KernelTable* make_table() {
  static const KernelTable t = {&launch_delta_z<NS, double, double, double>,
                                &launch_delta_z<NS, float, double, double>,
                                &launch_delta_z<NS, float, float, float>,
                                &launch_delta_y<NS, double, double>, &launch_delta_y<NS, float, double>,
                                &launch_delta_y_impl<NS, float, float>,
                                &launch_sweep<NS, double>,   &launch_sweep_f32<NS>,
                                &launch_kkt<NS>, &prepare_sweeps<NS>};
  return &t;
}

}  // namespace hot
}  // namespace lq2d
