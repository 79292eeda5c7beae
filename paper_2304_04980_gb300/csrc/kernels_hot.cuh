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
template <int NS>
__device__ __forceinline__ const double* ahat_row(const NodeData& nd, int p, int dir) {
  return dir == kSelf ? nd.Aself + (size_t)p * NS * NS : nd.Anb + ((size_t)p * 4 + (dir - 1)) * NS * NS;
}

// A_hat block in row r, column p, for r = neighbour of p in direction dir.
template <int NS>
__device__ __forceinline__ const double* ahat_col(const NodeData& nd, int r, int dir) {
  const int slot = dir == kWest ? 1 : dir == kEast ? 0 : dir == kNorth ? 3 : 2;  // F, E, H, G of r
  return dir == kSelf ? nd.Aself + (size_t)r * NS * NS : nd.Anb + ((size_t)r * 4 + slot) * NS * NS;
}

// ---------------------------------------------------------------------------
// Delta apply, part 1: z = Q~^-1 A~' dn, one thread per (node, t).
//   (A~' dn)_t = -dn_t + A_hat' dn_{t+1}   (t < T),   (A~' dn)_T = -dn_T
//   z_t = Q_t^-1 (A~' dn)_t                 (Q_T at t = T)
// dn = q + beta d_old is formed on the fly (Algorithm 1 line 14 fused into
// line 7); beta comes from the device state.
// ---------------------------------------------------------------------------
template <int NS, typename QT>
__global__ void __launch_bounds__(kOpThreads) delta_z_kernel(Grid g, NodeData nd, const QT* __restrict__ q,
                                                             const double* __restrict__ dold,
                                                             double* __restrict__ z,
                                                             const SolverState* __restrict__ st, int use_beta) {
  if (use_beta && st->done) return;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.P) return;
  const int Tp = g.T + 1;
  const int p = (int)(idx / Tp), t = (int)(idx % Tp);
  const int i = p / g.N, j = p % g.N;
  const double beta = use_beta ? st->beta : 0.0;
  const bool mix = beta != 0.0;
  double w[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    double dv = (double)q[k * g.Ps + idx];
    if (mix) dv += beta * dold[k * g.Ps + idx];
    w[k] = -dv;
  }
  if (t < g.T) {
#pragma unroll
    for (int dir = 0; dir < 5; ++dir) {
      const int r = nbr_node(i, j, dir, g.K, g.N);
      if (r < 0) continue;
      const double* blk = ahat_col<NS>(nd, r, dir);
      const long long ridx = (long long)r * Tp + t + 1;
      double dv[NS];
#pragma unroll
      for (int c = 0; c < NS; ++c) {
        dv[c] = (double)q[c * g.Ps + ridx];
        if (mix) dv[c] += beta * dold[c * g.Ps + ridx];
      }
#pragma unroll
      for (int c = 0; c < NS; ++c)
#pragma unroll
        for (int k = 0; k < NS; ++k) w[k] += blk[c * NS + k] * dv[c];
    }
  }
  const double* Qb = (t == g.T ? nd.QTi : nd.Qi) + (size_t)p * NS * NS;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NS; ++c) s += Qb[k * NS + c] * w[c];
    z[k * g.Ps + idx] = s;
  }
}

// ---------------------------------------------------------------------------
// Delta apply, part 2: y = A~ z + B~ R~^-1 B~' dn, one thread per (node, t).
//   y_0 = -z_0,   y_t = A_hat z_{t-1} - z_t + S dn_t   (t >= 1, S = B R^-1 B')
// Loop mode (Algorithm 1 lines 7-8, 14): dn = q + beta d_old is written back
// to d (each thread owns its entry), y' dn is reduced and vartheta set.
// ---------------------------------------------------------------------------
template <int NS, bool LOOP, typename QT>
__global__ void __launch_bounds__(kOpThreads) delta_y_kernel(Grid g, NodeData nd, const double* __restrict__ z,
                                                             const QT* __restrict__ q,
                                                             const double* __restrict__ dold,
                                                             double* __restrict__ dout, double* __restrict__ y,
                                                             double* __restrict__ partials, SolverState* st) {
  if (LOOP && st->done) return;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (idx < g.P) {
    const int Tp = g.T + 1;
    const int p = (int)(idx / Tp), t = (int)(idx % Tp);
    const int i = p / g.N, j = p % g.N;
    const double beta = LOOP ? st->beta : 0.0;
    double dn[NS], yk[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      double dv = (double)q[k * g.Ps + idx];
      if (LOOP && beta != 0.0) dv += beta * dold[k * g.Ps + idx];
      dn[k] = dv;
      yk[k] = -z[k * g.Ps + idx];
    }
    if (t >= 1) {
#pragma unroll
      for (int dir = 0; dir < 5; ++dir) {
        const int r = nbr_node(i, j, dir, g.K, g.N);
        if (r < 0) continue;
        const double* blk = ahat_row<NS>(nd, p, dir);
        const long long ridx = (long long)r * Tp + t - 1;
        double zv[NS];
#pragma unroll
        for (int c = 0; c < NS; ++c) zv[c] = z[c * g.Ps + ridx];
#pragma unroll
        for (int k = 0; k < NS; ++k)
#pragma unroll
          for (int c = 0; c < NS; ++c) yk[k] += blk[k * NS + c] * zv[c];
      }
      const double* S = nd.Sb + (size_t)p * NS * NS;
#pragma unroll
      for (int k = 0; k < NS; ++k)
#pragma unroll
        for (int c = 0; c < NS; ++c) yk[k] += S[k * NS + c] * dn[c];
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      y[k * g.Ps + idx] = yk[k];
      if (LOOP) {
        dout[k * g.Ps + idx] = dn[k];
        acc += yk[k] * dn[k];
      }
    }
  }
  if (LOOP) {
    double tot0, tot1;
    if (grid_reduce2<false>(acc, 0.0, partials, &st->counters[kCntDot], &tot0, &tot1)) {
      st->ydot = tot0;
      if (!(tot0 > 0.0) || !isfinite(tot0)) st->done = kBreakdown;
      else st->theta = st->mu / tot0;
    }
  }
}

// ---------------------------------------------------------------------------
// One NBJM sweep (Algorithm 2 inner step): theta_out = Phi~^-1 tau.
//
// Phi~ is block diagonal with one block Phi_bar_{v,t} per (column pair v,
// time t) (Section IV-B).  A group of GS lanes solves one block; lane a owns
// unknown a = jj*NS + k of each pair-row (node (i, 2v+jj), component k).  The
// groups of a block run over consecutive t, which share the factor of their
// time class.  Per pair-row i:
//   forward:  y_i = L0_i^-1 (tau_i - L1_i y_{i-1} - L2_i y_{i-2})
//   backward: x_i = L0_i^-T (y_i - L1_{i+1}' x_{i+1} - L2_{i+2}' x_{i+2})
// y is kept in theta_out between the two passes.  At t = 0, Phi_bar = Q^-1
// node by node, so theta = Q tau.
// ---------------------------------------------------------------------------
template <int NS>
struct SweepGeom {
  static constexpr int G2 = 2 * NS;
  static constexpr int GS = G2 <= 2 ? 2 : G2 <= 4 ? 4 : G2 <= 8 ? 8 : G2 <= 16 ? 16 : 32;
  static constexpr int BS = G2 * G2;
};

template <int NS, int VAR, typename VT>
__global__ void __launch_bounds__(kSweepThreads) nbjm_sweep_kernel(Grid g, PrecData<VT> pd, SweepArgsT<VT> a,
                                                                   SolverState* st) {
  // VT = float is the mixed mode: FP32 factors, blocks and iterates, with
  // the flexible (Polak-Ribiere) ratio for the next direction
  constexpr bool FLEX = sizeof(VT) == 4;
  constexpr bool UPDATE = VAR == kSweepUpdate;
  constexpr bool XI = VAR == kSweepXi;
  constexpr bool OMEGA = VAR == kSweepOmega || VAR == kSweepOmegaMu;
  constexpr bool MU = VAR == kSweepOmegaMu;
  constexpr int G2 = SweepGeom<NS>::G2, GS = SweepGeom<NS>::GS, BS = SweepGeom<NS>::BS;
  if (st != nullptr && st->done) return;
  const int lane32 = threadIdx.x & 31;
  const int al = threadIdx.x & (GS - 1);
  const unsigned gmask = GS == 32 ? 0xffffffffu : (((1u << GS) - 1u) << (lane32 & ~(GS - 1)));
  const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / GS;
  const int Tp = g.T + 1;
  const bool active = gid < (long long)g.V * Tp;
  const int v = active ? (int)(gid / Tp) : 0;
  const int t = active ? (int)(gid % Tp) : 0;
  const int ac = al < G2 ? al : 0;
  const int jj = ac / NS, k = ac % NS;
  const int j = 2 * v + jj;
  const bool node_ok = active && al < G2 && j < g.N;
  const long long kP = (long long)k * g.Ps;
  const double vth = UPDATE ? st->theta : 0.0;
  const bool flex_dot = FLEX && MU && st->have_mu;  // q'y is needed only after the first step
  double acc0 = 0.0, acc1 = 0.0;

  if (active) {
    const int cls = (t == g.T) ? 1 : 0;
    const VT* fac = pd.fac + (size_t)(2 * v + cls) * pd.fac_vc;
    VT ym1[G2], ym2[G2];
#pragma unroll
    for (int b = 0; b < G2; ++b) { ym1[b] = VT(0); ym2[b] = VT(0); }
    for (int i = 0; i < g.K; ++i) {
      const int p = i * g.N + j;
      const long long off = node_ok ? (long long)p * Tp + t : 0;
      VT tau = VT(0);
      if (node_ok) {
        if (UPDATE) {
          const double rr = a.r[kP + off] - vth * a.y[kP + off];
          a.r[kP + off] = rr;
          a.delta[kP + off] += vth * a.d[kP + off];
          tau = (VT)rr;
          acc0 += rr * rr;
          acc1 = fmax(acc1, fabs(rr));
        } else {
          tau = (VT)a.src[kP + off];
        }
        if (XI) {
          // (Xi~ delta)_t = A_hat Q^-1 delta_{t-1} + Q^-1 A_hat' delta_{t+1}
#pragma unroll
          for (int dir = 0; dir < 5; ++dir) {
            const int r = nbr_node(i, j, dir, g.K, g.N);
            if (r < 0) continue;
            const long long rb = (long long)r * Tp + t;
            if (t >= 1) {
              const VT* blk = pd.AQ + (((size_t)p * 5 + dir) * NS + k) * NS;
#pragma unroll
              for (int c = 0; c < NS; ++c) tau += blk[c] * a.delta_s[c * g.Ps + rb - 1];
            }
            if (t < g.T) {
              const VT* blk = pd.QAt + (((size_t)p * 5 + dir) * NS + k) * NS;
#pragma unroll
              for (int c = 0; c < NS; ++c) tau += blk[c] * a.delta_s[c * g.Ps + rb + 1];
            }
          }
          a.rtheta_out[kP + off] = (double)tau;
        }
        if (OMEGA && t >= 1) {
#pragma unroll
          for (int o = 0; o < 5; ++o) {
            const int qn = offpair_node(i, j, o, g.K, g.N);
            if (qn < 0) continue;
            const VT* blk = pd.Om + (((size_t)p * 5 + o) * NS + k) * NS;
            const long long qb = (long long)qn * Tp + t;
#pragma unroll
            for (int c = 0; c < NS; ++c) tau += blk[c] * a.theta_in[c * g.Ps + qb];
          }
        }
      }
      if (t == 0) {
        // Phi_bar_{v,0} = blkdiag(Q^-1): theta = Q tau, node by node
        VT out = VT(0);
        const VT* Qrow = pd.Qm + ((size_t)p * NS + k) * NS;
#pragma unroll
        for (int c = 0; c < NS; ++c) {
          const VT tc = __shfl_sync(gmask, tau, jj * NS + c, GS);
          if (node_ok) out += Qrow[c] * tc;
        }
        if (node_ok) {
          a.theta_out[kP + off] = out;
          if (MU) acc0 += (double)out * a.r[kP + off];
          if (flex_dot) acc1 += (double)out * a.y[kP + off];
        }
        continue;
      }
      // forward substitution over pair-row i
      const VT* rec = fac + (size_t)i * pd.fac_rec;
      VT w = tau;
      if (i >= 1) {
#pragma unroll
        for (int b = 0; b < G2; ++b) w -= rec[BS + b * G2 + ac] * ym1[b];
      }
      if (i >= 2) {
#pragma unroll
        for (int b = 0; b < G2; ++b) w -= rec[b * G2 + ac] * ym2[b];
      }
      VT yv = VT(0);
#pragma unroll
      for (int b = 0; b < G2; ++b) yv += rec[2 * BS + b * G2 + ac] * __shfl_sync(gmask, w, b, GS);
      if (node_ok) a.theta_out[kP + off] = yv;
#pragma unroll
      for (int b = 0; b < G2; ++b) {
        ym2[b] = ym1[b];
        ym1[b] = __shfl_sync(gmask, yv, b, GS);
      }
    }
    if (t >= 1) {
      VT xp1[G2], xp2[G2];
#pragma unroll
      for (int b = 0; b < G2; ++b) { xp1[b] = VT(0); xp2[b] = VT(0); }
      for (int i = g.K - 1; i >= 0; --i) {
        const int p = i * g.N + j;
        const long long off = node_ok ? (long long)p * Tp + t : 0;
        const VT* rec = fac + (size_t)i * pd.fac_rec;
        VT w = node_ok ? a.theta_out[kP + off] : VT(0);
        if (i + 1 < g.K) {
          const VT* r1 = rec + pd.fac_rec;
#pragma unroll
          for (int b = 0; b < G2; ++b) w -= r1[4 * BS + b * G2 + ac] * xp1[b];
        }
        if (i + 2 < g.K) {
          const VT* r2 = rec + 2 * pd.fac_rec;
#pragma unroll
          for (int b = 0; b < G2; ++b) w -= r2[3 * BS + b * G2 + ac] * xp2[b];
        }
        VT xv = VT(0);
#pragma unroll
        for (int b = 0; b < G2; ++b) xv += rec[5 * BS + b * G2 + ac] * __shfl_sync(gmask, w, b, GS);
        if (node_ok) {
          a.theta_out[kP + off] = xv;
          if (MU) acc0 += (double)xv * a.r[kP + off];
          if (flex_dot) acc1 += (double)xv * a.y[kP + off];
        }
#pragma unroll
        for (int b = 0; b < G2; ++b) {
          xp2[b] = xp1[b];
          xp1[b] = __shfl_sync(gmask, xv, b, GS);
        }
      }
    }
  }
  if (UPDATE) {
    double tot0, tot1;
    if (grid_reduce2<true>(acc0, acc1, a.partials, &st->counters[kCntNorm], &tot0, &tot1)) {
      // Algorithm 1 line 11, with the stop rule selected by stop_mode
      st->rnorm2 = tot0;
      st->rnorm_inf = tot1;
      const int it = st->iter + 1;
      st->iter = it;
      const bool pass = st->stop_mode == 0 ? (tot0 <= st->stop_bound) : (tot1 < st->stop_bound);
      if (!isfinite(tot0)) st->done = kBreakdown;
      else if (pass) st->done = kConverged;
      else if (it >= st->max_iter) st->done = kMaxIter;
    }
  }
  if (MU) {
    double tot0, tot1;
    if (grid_reduce2<false>(acc0, acc1, a.partials, &st->counters[kCntMu], &tot0, &tot1)) {
      // Algorithm 1 lines 13-14: mu^(i+1) and the ratio used for d^(i+1);
      // the mixed mode takes q^(i+1)'(r^(i+1) - r^(i)) / mu^(i), which equals
      // mu^(i+1) / mu^(i) for an exactly symmetric preconditioner
      if (!(tot0 > 0.0) || !isfinite(tot0) || !isfinite(tot1)) {
        st->done = kBreakdown;
      } else {
        if (!st->have_mu) st->beta = 0.0;
        else st->beta = FLEX ? (-st->theta * tot1) / st->mu : tot0 / st->mu;
        st->mu = tot0;
        st->have_mu = 1;
      }
    }
  }
}

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
template <int NS, typename QT>
void launch_delta_z(const Grid& g, const NodeData& nd, const QT* q, const double* dold, double* z,
                    const SolverState* st, int use_beta, cudaStream_t s) {
  const long long blocks = (g.P + kOpThreads - 1) / kOpThreads;
  delta_z_kernel<NS, QT><<<(unsigned)blocks, kOpThreads, 0, s>>>(g, nd, q, dold, z, st, use_beta);
}

template <int NS, typename QT>
void launch_delta_y(const Grid& g, const NodeData& nd, const double* z, const QT* q, const double* dold,
                    double* dout, double* y, double* partials, SolverState* st, int loop_mode, cudaStream_t s) {
  const long long blocks = (g.P + kOpThreads - 1) / kOpThreads;
  if (loop_mode)
    delta_y_kernel<NS, true, QT><<<(unsigned)blocks, kOpThreads, 0, s>>>(g, nd, z, q, dold, dout, y, partials, st);
  else
    delta_y_kernel<NS, false, QT><<<(unsigned)blocks, kOpThreads, 0, s>>>(g, nd, z, q, dold, dout, y, partials, st);
}

template <int NS, typename VT>
void launch_sweep(int variant, const Grid& g, const PrecData<VT>& pd, const SweepArgsT<VT>& a, SolverState* st,
                  cudaStream_t s) {
  constexpr int GS = SweepGeom<NS>::GS;
  const long long threads = (long long)g.V * (g.T + 1) * GS;
  const unsigned blocks = (unsigned)((threads + kSweepThreads - 1) / kSweepThreads);
  switch (variant) {
    case kSweepPlain: nbjm_sweep_kernel<NS, kSweepPlain, VT><<<blocks, kSweepThreads, 0, s>>>(g, pd, a, st); break;
    case kSweepUpdate: nbjm_sweep_kernel<NS, kSweepUpdate, VT><<<blocks, kSweepThreads, 0, s>>>(g, pd, a, st); break;
    case kSweepOmega: nbjm_sweep_kernel<NS, kSweepOmega, VT><<<blocks, kSweepThreads, 0, s>>>(g, pd, a, st); break;
    case kSweepOmegaMu:
      nbjm_sweep_kernel<NS, kSweepOmegaMu, VT><<<blocks, kSweepThreads, 0, s>>>(g, pd, a, st);
      break;
    default: nbjm_sweep_kernel<NS, kSweepXi, VT><<<blocks, kSweepThreads, 0, s>>>(g, pd, a, st); break;
  }
}

template <int NS>
void launch_kkt(const Grid& g, const NodeData& nd, const double* x, const double* u, const double* delta,
                const double* rhs, double* partials, SolverState* st, double* out, cudaStream_t s) {
  const long long blocks = (g.P + kOpThreads - 1) / kOpThreads;
  kkt_kernel<NS><<<(unsigned)blocks, kOpThreads, 0, s>>>(g, nd, x, u, delta, rhs, partials, st, out);
}

template <int NS>
const KernelTable* make_table() {
  static const KernelTable t = {&launch_delta_z<NS, double>, &launch_delta_z<NS, float>,
                                &launch_delta_y<NS, double>, &launch_delta_y<NS, float>,
                                &launch_sweep<NS, double>,   &launch_sweep<NS, float>,
                                &launch_kkt<NS>};
  return &t;
}

}  // namespace hot
}  // namespace lq2d
