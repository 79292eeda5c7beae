// One NBJM sweep (Algorithm 2 inner step), theta_out = Phi~^-1 tau, with the
// per-pair-row operands staged in shared memory.
//
// Phi~ is block diagonal with one block Phi_bar_{v,t} per (column pair v,
// time t) (Section IV-B).  A CTA takes one column pair v and a tile of TT
// consecutive time steps; a group of GS lanes solves one (v, t) block, lane
// a owning unknown a = jj*NS + k of every pair-row (node (i, 2v+jj),
// component k).  All groups of a CTA walk the K pair-rows together.  For
// pair-row i+1 the CTA copies into shared memory, with cp.async while
// pair-row i is computed:
//   * the factor blocks of pair-row i+1 (both time classes when the tile
//     holds t = T), read by every group of the tile;
//   * the right-hand side of the pair-row's two nodes for the TT steps;
//   * the eight neighbouring nodes' theta (Omega~ term, same t) or
//     delta^(s) (Xi~ term, t-1 and t+1) for the TT steps: contiguous runs
//     in the component-plane layout;
//   * the Omega~ / Xi~ node blocks of the pair-row's two nodes.
// Per pair-row i:
//   forward:  y_i = L0_i^-1 (tau_i - L1_i y_{i-1} - L2_i y_{i-2})
//   backward: x_i = L0_i^-T (y_i - L1_{i+1}' x_{i+1} - L2_{i+2}' x_{i+2})
// y is kept in theta_out between the two passes.  At t = 0, Phi_bar = Q^-1
// node by node, so theta = Q tau.
#pragma once

#include "kernels.h"

namespace lq2d {
namespace hot {

template <int NS>
struct SweepGeom {
  static constexpr int G2 = 2 * NS;
  static constexpr int GS = G2 <= 2 ? 2 : G2 <= 4 ? 4 : G2 <= 8 ? 8 : G2 <= 16 ? 16 : 32;
  static constexpr int BS = G2 * G2;
  static constexpr int TT = kSweepThreads / GS;  // time steps per CTA
  static constexpr int NH = 8;                   // staged neighbour nodes per pair-row
  static constexpr int HW = TT + 2;              // staged time window (t0-1 .. t0+TT)
};

__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  if constexpr (sizeof(T) == 8) cp_async_8(smem, gmem);
  else cp_async_4(smem, gmem);
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The eight staged neighbours of pair-row i of column pair v (j0 = 2v).
// Omega~ (off-pair, same t):  (i,j0-1) (i-1,j0-1) (i+1,j0-1) (i,j0-2)
//                             (i,j0+2) (i-1,j0+2) (i+1,j0+2) (i,j0+3)
// Xi~ (5-point, t -/+ 1):     (i,j0) (i,j0+1) (i-1,j0) (i+1,j0)
//                             (i-1,j0+1) (i+1,j0+1) (i,j0-1) (i,j0+2)
__device__ __forceinline__ int staged_node(bool xi, int h, int i, int j0, int K, int N) {
  int di = 0, dj = 0;
  if (!xi) {
    switch (h) {
      case 0: dj = -1; break;
      case 1: di = -1; dj = -1; break;
      case 2: di = 1; dj = -1; break;
      case 3: dj = -2; break;
      case 4: dj = 2; break;
      case 5: di = -1; dj = 2; break;
      case 6: di = 1; dj = 2; break;
      default: dj = 3; break;
    }
  } else {
    switch (h) {
      case 0: break;
      case 1: dj = 1; break;
      case 2: di = -1; break;
      case 3: di = 1; break;
      case 4: di = -1; dj = 1; break;
      case 5: di = 1; dj = 1; break;
      case 6: dj = -1; break;
      default: dj = 2; break;
    }
  }
  const int ii = i + di, jj = j0 + dj;
  if (ii < 0 || ii >= K || jj < 0 || jj >= N) return -1;
  return ii * N + jj;
}

// Index of the staged node for off-pair neighbour o of column jj (order o0..o4
// of offpair_node), and for direction dir (self, west, east, north, south)
// of the 5-point stencil.
__device__ __forceinline__ int h_of_offpair(int jj, int o) {
  return jj == 0 ? o : (o == 4 ? 0 : o + 4);
}
__device__ __forceinline__ int h_of_dir(int jj, int dir) {
  if (jj == 0) return dir == 0 ? 0 : dir == 1 ? 6 : dir == 2 ? 1 : dir == 3 ? 2 : 3;
  return dir == 0 ? 1 : dir == 1 ? 0 : dir == 2 ? 7 : dir == 3 ? 4 : 5;
}

template <int NS, typename VT>
struct SweepSmem {
  using Geo = SweepGeom<NS>;
  VT fac[2][2][3 * Geo::BS];                  // [buffer][class][3 blocks]
  double src[2][2][NS][Geo::TT];              // [buffer][jj][k][t]
  VT halo[2][Geo::NH][NS][Geo::HW];           // [buffer][h][k][t window]
  VT blk[2][2][10][NS * NS];                  // [buffer][jj][block][n x n]
};

template <int NS, int VAR, typename VT>
__global__ void __launch_bounds__(kSweepThreads) nbjm_sweep_kernel(Grid g, PrecData<VT> pd, SweepArgsT<VT> a,
                                                                   SolverState* st) {
  // VT = float is the mixed mode: FP32 factors, blocks and iterates, with
  // the flexible (Polak-Ribiere) ratio for the next direction
  constexpr bool FLEX = sizeof(VT) == 4;
  constexpr bool UPDATE = VAR == kSweepUpdate;
  constexpr bool XI = VAR == kSweepXi || VAR == kSweepXiOmega;
  constexpr bool OMEGA = VAR == kSweepOmega || VAR == kSweepOmegaMu || VAR == kSweepXiOmega;
  constexpr bool MU = VAR == kSweepOmegaMu;
  constexpr bool HALO = XI || OMEGA;
  using Geo = SweepGeom<NS>;
  constexpr int G2 = Geo::G2, GS = Geo::GS, BS = Geo::BS, TT = Geo::TT, HW = Geo::HW;
  extern __shared__ __align__(16) unsigned char sweep_smem[];
  SweepSmem<NS, VT>& sm = *reinterpret_cast<SweepSmem<NS, VT>*>(sweep_smem);

  if (st != nullptr && st->done) return;
  const int Tp = g.T + 1;
  const int tiles = (Tp + TT - 1) / TT;
  const int v = blockIdx.x / tiles;
  const int t0 = (blockIdx.x % tiles) * TT;
  const int j0 = 2 * v;
  const bool two_cols = j0 + 1 < g.N;
  const bool has_last = t0 + TT > g.T;  // the tile holds t = T (class 1)
  const int tid = threadIdx.x;
  const int lane32 = tid & 31;
  const int al = tid & (GS - 1);
  const int grp = tid / GS;
  const unsigned gmask = GS == 32 ? 0xffffffffu : (((1u << GS) - 1u) << (lane32 & ~(GS - 1)));
  const int t = t0 + grp;
  const bool active = t <= g.T;
  const int ac = al < G2 ? al : 0;
  const int jj = ac / NS, k = ac % NS;
  const int j = j0 + jj;
  const bool node_ok = active && al < G2 && j < g.N;
  const long long kP = (long long)k * g.Ps;
  const int cls = (t == g.T) ? 1 : 0;
  const double vth = UPDATE ? st->theta : 0.0;
  const bool flex_dot = FLEX && MU && st->have_mu;
  const VT* fac_pair = pd.fac + (size_t)(2 * v) * pd.fac_vc;  // class c at fac_pair + c * fac_vc
  double acc0 = 0.0, acc1 = 0.0;

  // ---- staging of the forward step for pair-row i into buffer b
  auto stage_forward = [&](int i, int b) {
    // factor blocks L2', L1', L0^-1' of pair-row i, per class in the tile
    const int ncls = has_last ? 2 : 1;
    constexpr int CH = 16 / sizeof(VT);  // elements per 16-byte copy
    for (int e = tid * CH; e < ncls * 3 * BS; e += kSweepThreads * CH) {
      const int c = e / (3 * BS), off = e % (3 * BS);  // slot c holds class c
      cp_async_16(&sm.fac[b][c][off], fac_pair + (size_t)c * pd.fac_vc + (size_t)i * pd.fac_rec + off);
    }
    // right-hand side of the pair-row's nodes
    if (!UPDATE) {
      for (int e = tid; e < 2 * NS * TT; e += kSweepThreads) {
        const int cjj = e / (NS * TT), kk = (e / TT) % NS, gg = e % TT;
        const int tt = t0 + gg;
        if (tt <= g.T && (cjj == 0 || two_cols)) {
          const int p = i * g.N + j0 + cjj;
          cp_async_8(&sm.src[b][cjj][kk][gg], a.src + kk * g.Ps + (long long)p * Tp + tt);
        }
      }
    }
    if (HALO) {
      const VT* vec = XI ? a.delta_s : a.theta_in;
      for (int e = tid; e < Geo::NH * NS * HW; e += kSweepThreads) {
        const int h = e / (NS * HW), kk = (e / HW) % NS, w = e % HW;
        const int tt = t0 - 1 + w;
        if (tt < 0 || tt > g.T) continue;
        const int q = staged_node(XI, h, i, j0, g.K, g.N);
        if (q < 0) continue;
        cp_async_elem(&sm.halo[b][h][kk][w], vec + kk * g.Ps + (long long)q * Tp + tt);
      }
      // node blocks: Omega~ (5 per node) or AQ, QAt (5 + 5 per node)
      constexpr int nb = XI ? 10 : 5;
      for (int e = tid; e < 2 * nb * NS * NS; e += kSweepThreads) {
        const int cjj = e / (nb * NS * NS), bb = (e / (NS * NS)) % nb, rc = e % (NS * NS);
        if (cjj == 1 && !two_cols) continue;
        const int p = i * g.N + j0 + cjj;
        const VT* srcb;
        if (XI) srcb = (bb < 5 ? pd.AQ : pd.QAt) + ((size_t)p * 5 + (bb % 5)) * NS * NS + rc;
        else srcb = pd.Om + ((size_t)p * 5 + bb) * NS * NS + rc;
        cp_async_elem(&sm.blk[b][cjj][bb][rc], srcb);
      }
    }
  };

  // ---- staging of the backward step for pair-row i: L0^-1 of i, L1 of i+1,
  // L2 of i+2 (blocks 5, 4, 3 of their records)
  auto stage_backward = [&](int i, int b) {
    const int ncls = has_last ? 2 : 1;
    constexpr int CH = 16 / sizeof(VT);
    for (int e = tid * CH; e < ncls * 3 * BS; e += kSweepThreads * CH) {
      const int c = e / (3 * BS), off = e % (3 * BS);
      const int part = off / BS, in = off % BS;  // 0: L0^-1 of i, 1: L1 of i+1, 2: L2 of i+2
      const int row = i + part;
      if (row >= g.K) continue;
      cp_async_16(&sm.fac[b][c][off], fac_pair + (size_t)c * pd.fac_vc + (size_t)row * pd.fac_rec + (5 - part) * BS + in);
    }
  };

  VT ym1[G2], ym2[G2];
#pragma unroll
  for (int b = 0; b < G2; ++b) { ym1[b] = VT(0); ym2[b] = VT(0); }
  // in a tile without t = T only class 0 is staged, at slot 0
  const int my_slot = has_last ? cls : 0;

  // the update sweep's own entries of r, y, d, delta, loaded one pair-row ahead
  double nr = 0.0, ny = 0.0, nd_ = 0.0, ndl = 0.0;
  if (UPDATE && node_ok) {
    const long long o0 = kP + (long long)j * Tp + t;
    nr = a.r[o0];
    ny = a.y[o0];
    nd_ = a.d[o0];
    ndl = a.delta[o0];
  }
  stage_forward(0, 0);
  cp_async_commit();
  for (int i = 0; i < g.K; ++i) {
    const int b = i & 1;
    if (i + 1 < g.K) stage_forward(i + 1, b ^ 1);
    cp_async_commit();
    const int p = i * g.N + j;
    const long long off = node_ok ? (long long)p * Tp + t : 0;
    const double cr = nr, cy = ny, cd = nd_, cdl = ndl;
    if (UPDATE && node_ok && i + 1 < g.K) {
      const long long o1 = off + (long long)g.N * Tp;
      nr = a.r[kP + o1];
      ny = a.y[kP + o1];
      nd_ = a.d[kP + o1];
      ndl = a.delta[kP + o1];
    }
    cp_async_wait<1>();
    __syncthreads();
    VT tau = VT(0);
    if (node_ok) {
      if (UPDATE) {
        const double rr = cr - vth * cy;
        a.r[kP + off] = rr;
        a.delta[kP + off] = cdl + vth * cd;
        tau = (VT)rr;
        acc0 += rr * rr;
        acc1 = fmax(acc1, fabs(rr));
      } else {
        tau = (VT)sm.src[b][jj][k][grp];
      }
      if (XI) {
        // (Xi~ delta)_t = A_hat Q^-1 delta_{t-1} + Q^-1 A_hat' delta_{t+1}
#pragma unroll
        for (int dir = 0; dir < 5; ++dir) {
          if (nbr_node(i, j, dir, g.K, g.N) < 0) continue;
          const int h = h_of_dir(jj, dir);
          if (t >= 1) {
            const VT* blk = &sm.blk[b][jj][dir][k * NS];
#pragma unroll
            for (int c = 0; c < NS; ++c) tau += blk[c] * sm.halo[b][h][c][grp];
          }
          if (t < g.T) {
            const VT* blk = &sm.blk[b][jj][5 + dir][k * NS];
#pragma unroll
            for (int c = 0; c < NS; ++c) tau += blk[c] * sm.halo[b][h][c][grp + 2];
          }
        }
        a.rtheta_out[kP + off] = (double)tau;
      }
      if (OMEGA && t >= 1) {
        if (XI) {
          // inner start from the outer iterate (standalone solver only):
          // Omega~ delta^(s) at the same t, read directly
#pragma unroll
          for (int o = 0; o < 5; ++o) {
            const int qn = offpair_node(i, j, o, g.K, g.N);
            if (qn < 0) continue;
            const VT* blk = pd.Om + (((size_t)p * 5 + o) * NS + k) * NS;
            const long long qb = (long long)qn * Tp + t;
#pragma unroll
            for (int c = 0; c < NS; ++c) tau += blk[c] * a.theta_in[c * g.Ps + qb];
          }
        } else {
#pragma unroll
          for (int o = 0; o < 5; ++o) {
            if (offpair_node(i, j, o, g.K, g.N) < 0) continue;
            const int h = h_of_offpair(jj, o);
            const VT* blk = &sm.blk[b][jj][o][k * NS];
#pragma unroll
            for (int c = 0; c < NS; ++c) tau += blk[c] * sm.halo[b][h][c][grp + 1];
          }
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
    } else {
      const VT* rec = sm.fac[b][my_slot];
      VT w = tau;
      if (i >= 1) {
#pragma unroll
        for (int bb = 0; bb < G2; ++bb) w -= rec[BS + bb * G2 + ac] * ym1[bb];
      }
      if (i >= 2) {
#pragma unroll
        for (int bb = 0; bb < G2; ++bb) w -= rec[bb * G2 + ac] * ym2[bb];
      }
      VT yv = VT(0);
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) yv += rec[2 * BS + bb * G2 + ac] * __shfl_sync(gmask, w, bb, GS);
      if (node_ok) a.theta_out[kP + off] = yv;
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) {
        ym2[bb] = ym1[bb];
        ym1[bb] = __shfl_sync(gmask, yv, bb, GS);
      }
    }
    __syncthreads();  // buffer b is refilled two steps later
  }
  cp_async_wait<0>();
  __syncthreads();

  // ---- backward substitution
  VT xp1[G2], xp2[G2];
#pragma unroll
  for (int bb = 0; bb < G2; ++bb) { xp1[bb] = VT(0); xp2[bb] = VT(0); }
  stage_backward(g.K - 1, 0);
  cp_async_commit();
  for (int i = g.K - 1; i >= 0; --i) {
    const int b = (g.K - 1 - i) & 1;
    if (i >= 1) stage_backward(i - 1, b ^ 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    if (t >= 1) {
      const int p = i * g.N + j;
      const long long off = node_ok ? (long long)p * Tp + t : 0;
      const VT* rec = sm.fac[b][my_slot];
      VT w = node_ok ? a.theta_out[kP + off] : VT(0);
      if (i + 1 < g.K) {
#pragma unroll
        for (int bb = 0; bb < G2; ++bb) w -= rec[BS + bb * G2 + ac] * xp1[bb];
      }
      if (i + 2 < g.K) {
#pragma unroll
        for (int bb = 0; bb < G2; ++bb) w -= rec[2 * BS + bb * G2 + ac] * xp2[bb];
      }
      VT xv = VT(0);
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) xv += rec[bb * G2 + ac] * __shfl_sync(gmask, w, bb, GS);
      if (node_ok) {
        a.theta_out[kP + off] = xv;
        if (MU) acc0 += (double)xv * a.r[kP + off];
        if (flex_dot) acc1 += (double)xv * a.y[kP + off];
      }
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) {
        xp2[bb] = xp1[bb];
        xp1[bb] = __shfl_sync(gmask, xv, bb, GS);
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();

  if (UPDATE) {
    double tot0, tot1;
    if (grid_reduce2<true>(acc0, acc1, a.partials, &st->counters[kCntNorm], &tot0, &tot1)) {
      // Algorithm 1 line 11, with the stop rule selected by stop_mode
      st->rnorm2 = tot0;
      st->rnorm_inf = tot1;
      const int it = st->iter + 1;
      st->iter = it;
      const bool pass = st->stop_mode == 0 ? (tot0 <= st->stop_bound) : (tot1 < st->stop_bound);
      record_theta(st, it - 1);
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
        if (!st->have_mu) {
          st->beta = 0.0;
        } else {
          st->beta = FLEX ? (-st->theta * tot1) / st->mu : tot0 / st->mu;
          record_beta(st, st->iter - 1);
        }
        st->mu = tot0;
        st->have_mu = 1;
      }
    }
  }
}

template <int NS, typename VT>
constexpr size_t sweep_smem_bytes() { return sizeof(SweepSmem<NS, VT>); }

template <int NS>
inline unsigned sweep_blocks(const Grid& g) {
  constexpr int TT = SweepGeom<NS>::TT;
  const int tiles = (g.T + 1 + TT - 1) / TT;
  return (unsigned)((long long)g.V * tiles);
}

}  // namespace hot
}  // namespace lq2d
