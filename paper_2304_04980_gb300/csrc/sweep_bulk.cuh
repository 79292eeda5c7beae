// One NBJM sweep (Algorithm 2 inner step) for state dimension n = 4 in FP32,
// the preconditioner of the mixed-precision modes: theta_out = Phi~^-1 tau.
//
// Same arithmetic as nbjm_sweep_kernel (unit block factor F, pivots D,
// Phi_bar = F D F'; forward y_i = tau_i - F2_i y_{i-2} - F1_i y_{i-1},
// backward x_i = D_i^-1 y_i - N2_i x_{i+2} - N1_i x_{i+1}), organised for
// fewer instructions per unknown:
//
//  * Each lane owns one row a = jj*4 + k of a pair-row (node (i, 2v+jj),
//    component k) for R consecutive time steps of its group, so every factor
//    row it loads from shared memory serves R right-hand sides (the
//    multi-right-hand-side view of time-invariant blocks), and it runs R
//    independent multiply-add chains.
//  * Groups are class-uniform: group 0 of the first tile holds t = 0 alone,
//    the last group holds t = T alone, the others hold R steps of
//    1 <= t <= T-1.  t = 0 is a third factor class whose record has
//    F = N = 0 and D^-1 = blkdiag(Q, Q) (Phi_bar_{v,0} = blkdiag(Q^-1)), so
//    the code has no special case for it.
//  * The FP32 iterates (theta, delta^(s), q, r_theta) are node-major,
//    [p][t][k]: one (node, t) is an aligned 16-byte run and a node's time
//    window is one contiguous run.  Every operand of a pair-row step (factor
//    records, node blocks, neighbour windows, the FP64 residual runs as
//    aligned supersets) is staged by one cp.async.bulk copy per contiguous
//    run, completing on the step buffer's mbarrier, instead of one cp.async
//    per element.
//  * Three staging buffers keep two pair-rows in flight (two buffers, one
//    pair-row, for the update and mu sweeps when a lane carries four time
//    steps).  Every wait on an
//    mbarrier is bounded; a wait that runs out sets the solver state to the
//    loop-cap status and a fault word, lets the copies in flight land
//    (again bounded) and ends the CTA.
#pragma once

#include <stdint.h>

#include "kernels.h"

namespace lq2d {
namespace hot {
namespace bulk {

constexpr int NS = 4, G2 = 8, BS = 64, REC = 7 * BS;  // record: [N2][N1][D^-1][E][F2][F1][L0^-1]
// Staging buffers: three (two pair-rows in flight), except two for the
// sweeps that stage FP64 runs of several vectors (the PCG update, the mu
// sweep) at four time steps per lane: their steps are long enough to cover a
// copy's latency with one pair-row in flight, and a third buffer would cost
// them CTAs per SM (a second wave on the 256 x 256 x 200 grid).
template <int VAR, int R>
constexpr int stages() { return R >= 4 && (VAR == kSweepUpdate || VAR == kSweepOmegaMu) ? 2 : 3; }
// A wait gives up after kWaitCap rounds of try_wait, each suspending for at
// most about kWaitHintNs: about a second in all.
constexpr unsigned kWaitCap = 1u << 20;
constexpr unsigned kWaitHintNs = 1000u;

__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  unsigned long long state;
  asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];\n" : "=l"(state) : "r"(saddr(bar)) : "memory");
  (void)state;
}
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, unsigned bytes) {
  unsigned long long state;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;\n"
               : "=l"(state)
               : "r"(saddr(bar)), "r"(bytes)
               : "memory");
  (void)state;
}
// One bounded wait for the phase with the given parity; true once complete.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (unsigned it = 0; it < kWaitCap; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(saddr(bar)), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    if (done) return true;
  }
  return false;
}
// Global -> shared bulk copy (both addresses 16-byte aligned, bytes a
// multiple of 16), counted on the mbarrier's transaction count.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// Time steps of group G (counted over the whole column pair): t = 0 alone
// (class 2), then R steps of 1..T-1 per group (class 0), then t = T alone
// (class 1).
struct GroupSpan {
  int t0, count, cls;
};
template <int R>
__host__ __device__ __forceinline__ int class0_groups(int T) { return T >= 2 ? (T - 1 + R - 1) / R : 0; }
template <int R>
__host__ __device__ __forceinline__ GroupSpan group_span(int G, int T) {
  const int nc = class0_groups<R>(T);
  if (G == 0) return {0, 1, 2};
  if (G <= nc) {
    const int t0 = 1 + (G - 1) * R;
    const int cnt = (T - 1) - t0 + 1;
    return {t0, cnt < R ? cnt : R, 0};
  }
  if (G == nc + 1) return {T, 1, 1};
  return {0, 0, 0};
}
template <int R, int THR>
__host__ __device__ __forceinline__ int tiles_per_pair(int T) {
  constexpr int NG = THR / 8;
  return (class0_groups<R>(T) + 2 + NG - 1) / NG;
}

template <int VAR, int R, int THR>
struct Geo {
  static constexpr int NG = THR / 8;  // groups of 8 lanes
  static constexpr int TT = NG * R;   // time steps a tile can hold
  static constexpr int HW = TT + 2;   // staged window t_lo-1 .. t_hi+1
  static constexpr bool UPDATE = VAR == kSweepUpdate;
  static constexpr bool XI = VAR == kSweepXi || VAR == kSweepXiOmega;
  static constexpr bool OMEGA = VAR == kSweepOmega || VAR == kSweepOmegaMu || VAR == kSweepXiOmega;
  static constexpr bool MU = VAR == kSweepOmegaMu;
  static constexpr int NV = UPDATE ? 4 : (MU ? 2 : 1);  // FP64 runs per (jj, k) in one buffer
  static constexpr int RUN64 = TT + 2;                   // doubles per FP64 run slot (aligned superset)
  // copies of a step, at most: 3 factor classes, then node blocks, 8
  // neighbour windows and the pair-row's own runs (forward), or y_i and the
  // mu runs (backward)
  static constexpr int NFWD = UPDATE ? 3 + 4 * 8 : 3 + 2 + 8 + 8;
  static constexpr int NBWD = MU ? 3 + 2 + 16 : 3 + 2;
};

constexpr int kMaxCopies = 48;  // bulk copies of one step, at most

// One bulk copy of a pair-row step: a fixed run whose source advances by a
// fixed stride per pair-row.
struct CopyDesc {
  const char* base;     // source at pair-row 0 (flagged windows: outside the array there)
  unsigned stride8;     // 8-byte words per pair-row
  unsigned short dst;   // byte offset inside a staging buffer
  unsigned short info;  // bytes (bits 0..11) and the flags below
};
constexpr unsigned short kNeedAbove = 1u << 12;  // window of the row above: pair-rows 1..K-1
constexpr unsigned short kNeedBelow = 1u << 13;  // window of the row below: pair-rows 0..K-2
constexpr unsigned short kRun64 = 1u << 14;      // FP64 run, copied as its aligned 16-byte superset
constexpr unsigned short kBytesMask = 0xfffu;

template <int VAR, int R, int THR>
struct Smem {
  using G = Geo<VAR, R, THR>;
  struct Buf {
    float fac[3][3 * BS];                 // per class slot: forward F2 F1, backward N2 N1 D^-1
    float blk[320];                       // Omega~: [jj][5][16]; Xi~: AQ [jj][5][16], QAt at 160 + ...
    float halo[8][G::HW][NS];             // neighbour windows, node-major (t, k)
    float src32[2][G::HW][NS];            // forward: r_theta (FP32); backward: the forward result y_i
    double src64[G::NV][2][NS][G::RUN64]; // FP64 runs: r, y, d, delta (update); r (source); r, y (mu)
  };
  Buf buf[stages<VAR, R>()];
  float xy[G::NG][R][G2];                 // per group: the step's result, exchanged inside the group
  uint64_t bar[stages<VAR, R>()];
  CopyDesc desc_f[G::NFWD];               // the CTA's copies per step: forward pass
  CopyDesc desc_b[G::NBWD];               // backward pass
  int ndesc[2];
};

// CTAs per SM to budget registers for: as many as shared memory allows.
template <int VAR, int R, int THR>
constexpr int min_blocks() {
  constexpr int by_smem = 232448 / ((int)sizeof(Smem<VAR, R, THR>) + 1024);
  constexpr int by_threads = 2048 / THR;
  constexpr int b = by_smem < by_threads ? by_smem : by_threads;
  return b < 1 ? 1 : (b > 8 ? 8 : b);
}

}  // namespace bulk

template <int VAR, int R, int THR>
__global__ void __launch_bounds__(THR, (bulk::min_blocks<VAR, R, THR>()))
    nbjm_sweep_bulk_kernel(Grid g, PrecData<float> pd, SweepArgsT<float> a, SolverState* st) {
  using namespace bulk;
  using Gm = Geo<VAR, R, THR>;
  using Sm = Smem<VAR, R, THR>;
  constexpr int NG = Gm::NG;
  constexpr bool UPDATE = Gm::UPDATE, XI = Gm::XI, OMEGA = Gm::OMEGA, MU = Gm::MU;
  constexpr bool HALO = XI || OMEGA;
  constexpr bool XIOM = VAR == kSweepXiOmega;
  constexpr int NB = stages<VAR, R>();
  constexpr int PD = NB - 1;
  constexpr int CPT = (kMaxCopies + THR - 1) / THR;
  extern __shared__ __align__(128) unsigned char bulk_smem[];
  Sm& sm = *reinterpret_cast<Sm*>(bulk_smem);

  if (st != nullptr && st->done) return;
  const int T = g.T, Tp = T + 1, K = g.K, N = g.N;
  const int tiles = tiles_per_pair<R, THR>(T);
  const int v = blockIdx.x / tiles, tile = blockIdx.x % tiles;
  const int j0 = 2 * v;
  const bool two_cols = j0 + 1 < N;
  const int tid = threadIdx.x, grp = tid >> 3, al = tid & 7, jj = al >> 2, k = al & 3;
  const int j = j0 + jj;
  const bool node_ok = jj == 0 || two_cols;
  // the tile's groups, its time range and the factor classes it needs
  const int nc = class0_groups<R>(T);
  const int G0 = tile * NG;
  const int Glast = (G0 + NG < nc + 2 ? G0 + NG : nc + 2) - 1;
  const GroupSpan sp = group_span<R>(G0 + grp, T);
  // time step of each slot; slots past the group's count alias a live one,
  // so that every staged index they form stays inside the tile's window
  int tr[R];
  const GroupSpan s_last = group_span<R>(Glast, T);
  const int tl = group_span<R>(G0, T).t0, th = s_last.t0 + s_last.count - 1;
  const unsigned cls_mask = (G0 == 0 ? 4u : 0u) | (Glast == nc + 1 ? 2u : 0u) |
                            ((G0 > 1 ? G0 : 1) <= (Glast < nc ? Glast : nc) ? 1u : 0u);
  const int ntl = th - tl + 1;
#pragma unroll
  for (int r = 0; r < R; ++r) tr[r] = sp.count > 0 ? sp.t0 + (r < sp.count ? r : 0) : tl;
  const long long Ps = g.Ps;
  const double vth = UPDATE ? st->theta : 0.0;
  const bool flex_dot = MU && st->have_mu;
  const float* src32g = a.src_rtheta ? reinterpret_cast<const float*>(a.src) : nullptr;
  const float* hvec = XI ? a.delta_s : a.theta_in;
  double acc0 = 0.0, acc1 = 0.0;

  // staged neighbours inside the grid, by pair-row
  const unsigned long long packed = XI ? kXiPacked : kOmPacked;
  unsigned col_ok = 0u, above = 0u, below = 0u;
#pragma unroll
  for (int h = 0; h < 8; ++h) {
    const unsigned code = (unsigned)((packed >> (5 * h)) & 31ull);
    const int di = (int)(code & 3u) - 1, jn = j0 + (int)(code >> 2) - 2;
    if (jn >= 0 && jn < N) col_ok |= 1u << h;
    if (di < 0) above |= 1u << h;
    if (di > 0) below |= 1u << h;
  }
  auto row_valid = [&](int i) -> unsigned {
    unsigned m = col_ok;
    if (i < 1) m &= ~above;
    if (i + 1 >= K) m &= ~below;
    return m;
  };

  if (tid == 0) {
    for (int b = 0; b < NB; ++b) mbar_init(&sm.bar[b], THR);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (!two_cols) {
    // the missing column's entries of y are never staged: keep them zero
    for (int e = tid; e < NB * Gm::HW * NS; e += THR) {
      const int b = e / (Gm::HW * NS), w = e % (Gm::HW * NS);
      (&sm.buf[b].src32[1][0][0])[w] = 0.f;
    }
  }
  __syncthreads();

  // ---- the copies of a step, described once per CTA (thread 0): candidate
  // copy c of a pass -> (source at pair-row 0, stride, place, bytes, flags),
  // false when the copy does not exist for this tile
  auto buf_off = [&](const void* q) -> unsigned short {
    return (unsigned short)(reinterpret_cast<const char*>(q) - reinterpret_cast<const char*>(&sm.buf[0]));
  };
  const unsigned row_iter8 = (unsigned)((long long)N * Tp * 2);  // 8-byte words per grid row of an FP32 iterate
  auto run64 = [&](const double* vec, int cjj, int kk, CopyDesc& d) {
    d.base = reinterpret_cast<const char*>(vec + kk * Ps + (long long)(j0 + cjj) * Tp + tl);
    d.stride8 = (unsigned)((long long)N * Tp);
    d.info = kRun64;
  };
  auto describe = [&](int c, bool fwd, CopyDesc& d) -> bool {
    typename Sm::Buf& B = sm.buf[0];
    if (c < 3) {
      if (!((cls_mask >> c) & 1u)) return false;
      const float* f = c == 2 ? pd.fac_t0 + (size_t)v * pd.fac_vc : pd.fac + (size_t)(2 * v + c) * pd.fac_vc;
      d.base = reinterpret_cast<const char*>(f + (fwd ? 4 * BS : 0));  // [F2][F1] or [N2][N1][D^-1]
      d.stride8 = (unsigned)(pd.fac_rec / 2);
      d.dst = buf_off(&B.fac[c][0]);
      d.info = (unsigned short)(fwd ? 2 * BS * 4 : 3 * BS * 4);
      return true;
    }
    c -= 3;
    if (fwd) {
      constexpr int NBLK = HALO ? (XI ? 2 : 1) : 0;
      if (c < NBLK) {
        const float* arr = XI ? (c == 0 ? pd.AQ : pd.QAt) : pd.Om;
        d.base = reinterpret_cast<const char*>(arr + (size_t)j0 * 80);
        d.stride8 = (unsigned)(N * 40);
        d.dst = buf_off(&B.blk[c * 160]);
        d.info = (unsigned short)((two_cols ? 2u : 1u) * 320u);
        return true;
      }
      c -= NBLK;
      if (HALO) {
        if (c < 8) {
          if (!((col_ok >> c) & 1u)) return false;
          const unsigned code = (unsigned)((packed >> (5 * c)) & 31ull);
          const int di = (int)(code & 3u) - 1, jn = j0 + (int)(code >> 2) - 2;
          const int ta = XI ? (tl - 1 > 0 ? tl - 1 : 0) : tl;
          const int tb = XI ? (th + 1 < T ? th + 1 : T) : th;
          d.base = reinterpret_cast<const char*>(hvec) + ((long long)(di * N + jn) * Tp + ta) * NS * 4;
          d.stride8 = row_iter8;
          d.dst = buf_off(&B.halo[c][ta - (tl - 1)][0]);
          d.info = (unsigned short)((tb - ta + 1) * 16) | (di < 0 ? kNeedAbove : 0) | (di > 0 ? kNeedBelow : 0);
          return true;
        }
        c -= 8;
      }
      if (src32g != nullptr) {
        if (c >= 2 || (c == 1 && !two_cols)) return false;
        d.base = reinterpret_cast<const char*>(src32g + ((long long)(j0 + c) * Tp + tl) * NS);
        d.stride8 = row_iter8;
        d.dst = buf_off(&B.src32[c][0][0]);
        d.info = (unsigned short)(ntl * 16);
        return true;
      }
      constexpr int NVF = UPDATE ? 4 : 1;
      if (c >= NVF * 8) return false;
      const int vv = c >> 3, cjj = (c >> 2) & 1, kk = c & 3;
      if (cjj == 1 && !two_cols) return false;
      run64(UPDATE ? (vv == 0 ? a.r : vv == 1 ? a.y : vv == 2 ? a.d : a.delta) : a.src, cjj, kk, d);
      d.dst = buf_off(&B.src64[vv][cjj][kk][0]);
      return true;
    }
    // backward: the forward result y_i of the tile, then r (and y) for mu
    if (c < 2) {
      if (c == 1 && !two_cols) return false;
      d.base = reinterpret_cast<const char*>(a.theta_out + ((long long)(j0 + c) * Tp + tl) * NS);
      d.stride8 = row_iter8;
      d.dst = buf_off(&B.src32[c][0][0]);
      d.info = (unsigned short)(ntl * 16);
      return true;
    }
    c -= 2;
    if (!MU || c >= (flex_dot ? 16 : 8)) return false;
    const int vv = c >> 3, cjj = (c >> 2) & 1, kk = c & 3;
    if (cjj == 1 && !two_cols) return false;
    run64(vv == 0 ? a.r : a.y, cjj, kk, d);
    d.dst = buf_off(&B.src64[vv][cjj][kk][0]);
    return true;
  };
  if (tid == 0) {
    for (int pass = 0; pass < 2; ++pass) {
      CopyDesc* out = pass == 0 ? sm.desc_f : sm.desc_b;
      const int cap = pass == 0 ? Gm::NFWD : Gm::NBWD;
      int nd = 0;
      for (int c = 0; c < kMaxCopies; ++c) {
        CopyDesc d;  // cap: the most copies a pass of this variant has (never reached past)
        if (describe(c, pass == 0, d) && nd < cap) out[nd++] = d;
      }
      sm.ndesc[pass] = nd;
    }
  }
  __syncthreads();
  // the thread of copy c: spread over the warps (c = lane * warps + warp),
  // so that every warp issues about as many copies
  auto copy_index = [&](int q) -> int {
    if constexpr (THR >= 64) return (tid & 31) * (THR / 32) + (tid >> 5) + q * THR;
    else return tid + q * THR;
  };
  // every thread arrives once per staged step, announcing the bytes of its copies
  auto stage = [&](int s) {
    const bool fwd = s < K;
    const int i = fwd ? s : 2 * K - 1 - s;
    const int b = s % NB;
    const int pass = fwd ? 0 : 1;
    const int nd = sm.ndesc[pass];
    unsigned char* dbuf = reinterpret_cast<unsigned char*>(&sm.buf[b]);
    const char* srcs[CPT];
    unsigned dsts[CPT];
    unsigned by[CPT];
    unsigned total = 0u;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      by[q] = 0u;
      const int c = copy_index(q);
      if (c < nd) {
        const CopyDesc d = fwd ? sm.desc_f[c] : sm.desc_b[c];
        const bool ok = !((d.info & kNeedAbove) && i < 1) && !((d.info & kNeedBelow) && i + 1 >= K);
        if (ok) {
          const char* src = d.base + (long long)i * d.stride8 * 8;
          unsigned bytes = d.info & kBytesMask;
          if (d.info & kRun64) {
            // the run's first element may sit at an odd double: copy from the
            // 16-byte boundary below it (the reader offsets by that parity)
            const unsigned par = (unsigned)(reinterpret_cast<uintptr_t>(src) >> 3) & 1u;
            src -= par * 8;
            bytes = ((par + (unsigned)ntl + 1u) & ~1u) * 8u;
          }
          srcs[q] = src;
          dsts[q] = d.dst;
          by[q] = bytes;
          total += bytes;
        }
      }
    }
    if (total) mbar_arrive_expect(&sm.bar[b], total);
    else mbar_arrive(&sm.bar[b]);
#pragma unroll
    for (int q = 0; q < CPT; ++q)
      if (by[q]) bulk_load(dbuf + dsts[q], srcs[q], by[q], &sm.bar[b]);
  };
  // a wait that ran out: record it, let the staged copies land, end the CTA
  int staged = 0;
  auto give_up = [&](int waited) {
    if (tid == 0) {
      if (st != nullptr) st->done = kLoopCap;
      if (a.fault != nullptr) atomicOr(a.fault, 1);
    }
    for (int s = waited; s < staged; ++s) mbar_wait(&sm.bar[s % NB], (unsigned)(s / NB) & 1u);
  };

  float ym1[G2][R], ym2[G2][R];
#pragma unroll
  for (int bb = 0; bb < G2; ++bb)
#pragma unroll
    for (int r = 0; r < R; ++r) { ym1[bb][r] = 0.f; ym2[bb][r] = 0.f; }

  // ------------------------------------------------------------ forward pass
  for (; staged < PD && staged < K; ++staged) stage(staged);
  for (int i = 0; i < K; ++i) {
    const int s = i, b = s % NB;
    const bool ok = mbar_wait(&sm.bar[b], (unsigned)(s / NB) & 1u);
    if (__syncthreads_or(!ok)) { give_up(s); return; }
    if (staged < K) stage(staged++);
    typename Sm::Buf& B = sm.buf[b];
    const long long prow = (long long)(i * N + j) * Tp;
    const int o64 = (int)(((long long)(i * N + j) * Tp + tl) & 1);
    float tau[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int w = tr[r] - tl;
      const bool live = node_ok && r < sp.count;
      float tv = 0.f;
      if (UPDATE) {
        const double rr = B.src64[0][jj][k][o64 + w] - vth * B.src64[1][jj][k][o64 + w];
        const double dd = B.src64[3][jj][k][o64 + w] + vth * B.src64[2][jj][k][o64 + w];
        if (live) {
          const long long e = k * Ps + prow + tr[r];
          a.r[e] = rr;
          a.delta[e] = dd;
          acc0 += rr * rr;
          acc1 = fmax(acc1, fabs(rr));
          tv = (float)rr;
        }
      } else if (src32g != nullptr) {
        tv = live ? B.src32[jj][w][k] : 0.f;
      } else {
        tv = live ? (float)B.src64[0][jj][k][o64 + w] : 0.f;
      }
      tau[r] = tv;
    }
    const unsigned valid = HALO ? row_valid(i) : 0u;
    if (XI && node_ok) {
      // (Xi~ delta)_t = A_hat Q^-1 delta_{t-1} + Q^-1 A_hat' delta_{t+1}
#pragma unroll
      for (int dir = 0; dir < 5; ++dir) {
        const int h = h_of_dir(jj, dir);
        if (!((valid >> h) & 1u)) continue;
        const float4 lo = lds4(&B.blk[jj * 80 + dir * 16 + k * 4]);
        const float4 up = lds4(&B.blk[160 + jj * 80 + dir * 16 + k * 4]);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int t = tr[r], w = t - tl;
          if (t >= 1) {
            const float4 hv = lds4(&B.halo[h][w][0]);
            tau[r] = fmaf(lo.x, hv.x, fmaf(lo.y, hv.y, fmaf(lo.z, hv.z, fmaf(lo.w, hv.w, tau[r]))));
          }
          if (t < T) {
            const float4 hv = lds4(&B.halo[h][w + 2][0]);
            tau[r] = fmaf(up.x, hv.x, fmaf(up.y, hv.y, fmaf(up.z, hv.z, fmaf(up.w, hv.w, tau[r]))));
          }
        }
      }
      float* rt = reinterpret_cast<float*>(a.rtheta_out);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (r < sp.count) rt[(prow + tr[r]) * NS + k] = tau[r];
    }
    if (OMEGA && !XIOM && node_ok) {
#pragma unroll
      for (int o = 0; o < 5; ++o) {
        const int h = h_of_offpair(jj, o);
        if (!((valid >> h) & 1u)) continue;
        const float4 row = lds4(&B.blk[jj * 80 + o * 16 + k * 4]);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int t = tr[r];
          if (t >= 1) {
            const float4 hv = lds4(&B.halo[h][t - tl + 1][0]);
            tau[r] = fmaf(row.x, hv.x, fmaf(row.y, hv.y, fmaf(row.z, hv.z, fmaf(row.w, hv.w, tau[r]))));
          }
        }
      }
    }
    if (XIOM && node_ok) {
      // inner start from the outer iterate (standalone solver): Omega~
      // delta^(s) at the same t, read directly
      const int p = i * N + j;
#pragma unroll
      for (int o = 0; o < 5; ++o) {
        const int qn = offpair_node(i, j, o, K, N);
        if (qn < 0) continue;
        const float4 row = *reinterpret_cast<const float4*>(pd.Om + (((size_t)p * 5 + o) * NS + k) * NS);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int t = tr[r];
          if (t >= 1 && r < sp.count) {
            const float4 hv = *reinterpret_cast<const float4*>(a.theta_in + ((long long)qn * Tp + t) * NS);
            tau[r] = fmaf(row.x, hv.x, fmaf(row.y, hv.y, fmaf(row.z, hv.z, fmaf(row.w, hv.w, tau[r]))));
          }
        }
      }
    }
    // y_i = tau_i - F2 y_{i-2} - F1 y_{i-1}
    const float* rec = B.fac[sp.cls];
    const float4 f2a = lds4(rec + al * 8), f2b = lds4(rec + al * 8 + 4);
    const float4 f1a = lds4(rec + BS + al * 8), f1b = lds4(rec + BS + al * 8 + 4);
    const float f2[8] = {f2a.x, f2a.y, f2a.z, f2a.w, f2b.x, f2b.y, f2b.z, f2b.w};
    const float f1[8] = {f1a.x, f1a.y, f1a.z, f1a.w, f1b.x, f1b.y, f1b.z, f1b.w};
#pragma unroll
    for (int r = 0; r < R; ++r) {
      // two independent sums (F2 y_{i-2} onto tau, F1 y_{i-1} from zero)
      // halve the dependent chain of the step
      float yv = tau[r], y1 = 0.f;
      if (i >= 2) {
#pragma unroll
        for (int bb = 0; bb < G2; ++bb) yv = fmaf(-f2[bb], ym2[bb][r], yv);
      }
      if (i >= 1) {
#pragma unroll
        for (int bb = 0; bb < G2; ++bb) y1 = fmaf(f1[bb], ym1[bb][r], y1);
      }
      yv -= y1;
      if (node_ok && r < sp.count) a.theta_out[(prow + tr[r]) * NS + k] = yv;
      sm.xy[grp][r][al] = yv;
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 lo = lds4(&sm.xy[grp][r][0]), hi = lds4(&sm.xy[grp][r][4]);
      const float nv[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) {
        ym2[bb][r] = ym1[bb][r];
        ym1[bb][r] = nv[bb];
      }
    }
  }
  // the forward results in theta_out are read back by bulk copies (the
  // async proxy): order this thread's generic writes before them
  asm volatile("fence.proxy.async.global;\n" ::: "memory");
  __syncthreads();

  // ----------------------------------------------------------- backward pass
  float xp1[G2][R], xp2[G2][R];
#pragma unroll
  for (int bb = 0; bb < G2; ++bb)
#pragma unroll
    for (int r = 0; r < R; ++r) { xp1[bb][r] = 0.f; xp2[bb][r] = 0.f; }
  for (; staged < K + PD && staged < 2 * K; ++staged) stage(staged);
  for (int i = K - 1; i >= 0; --i) {
    const int s = 2 * K - 1 - i, b = s % NB;
    const bool ok = mbar_wait(&sm.bar[b], (unsigned)(s / NB) & 1u);
    if (__syncthreads_or(!ok)) { give_up(s); return; }
    if (staged < 2 * K) stage(staged++);
    typename Sm::Buf& B = sm.buf[b];
    const long long prow = (long long)(i * N + j) * Tp;
    const int o64 = (int)(((long long)(i * N + j) * Tp + tl) & 1);
    const float* rec = B.fac[sp.cls];  // [N2][N1][D^-1]
    const float4 n2a = lds4(rec + al * 8), n2b = lds4(rec + al * 8 + 4);
    const float4 n1a = lds4(rec + BS + al * 8), n1b = lds4(rec + BS + al * 8 + 4);
    const float4 da = lds4(rec + 2 * BS + al * 8), db = lds4(rec + 2 * BS + al * 8 + 4);
    const float n2[8] = {n2a.x, n2a.y, n2a.z, n2a.w, n2b.x, n2b.y, n2b.z, n2b.w};
    const float n1[8] = {n1a.x, n1a.y, n1a.z, n1a.w, n1b.x, n1b.y, n1b.z, n1b.w};
    const float dv[8] = {da.x, da.y, da.z, da.w, db.x, db.y, db.z, db.w};
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int w = tr[r] - tl;
      const float4 y0 = lds4(&B.src32[0][w][0]), y1 = lds4(&B.src32[1][w][0]);
      const float yall[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
      // three independent sums, so the step's dependent chain is 2n long
      float xv = 0.f, x2 = 0.f, x1 = 0.f;
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) xv = fmaf(dv[bb], yall[bb], xv);
      if (i + 2 < K) {
#pragma unroll
        for (int bb = 0; bb < G2; ++bb) x2 = fmaf(n2[bb], xp2[bb][r], x2);
      }
      if (i + 1 < K) {
#pragma unroll
        for (int bb = 0; bb < G2; ++bb) x1 = fmaf(n1[bb], xp1[bb][r], x1);
      }
      xv = xv - x2 - x1;
      if (node_ok && r < sp.count) {
        a.theta_out[(prow + tr[r]) * NS + k] = xv;
        if (MU) {
          acc0 += (double)xv * B.src64[0][jj][k][o64 + w];
          if (flex_dot) acc1 += (double)xv * B.src64[1][jj][k][o64 + w];
        }
      }
      sm.xy[grp][r][al] = xv;
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 lo = lds4(&sm.xy[grp][r][0]), hi = lds4(&sm.xy[grp][r][4]);
      const float nv[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) {
        xp2[bb][r] = xp1[bb][r];
        xp1[bb][r] = nv[bb];
      }
    }
  }

  if (UPDATE) {
    double tot0, tot1;
    if (grid_reduce2<true>(acc0, acc1, a.partials, &st->counters[kCntNorm], &tot0, &tot1)) {
      // the stop test of Algorithm 1, with the rule selected by stop_mode
      st->rnorm2 = tot0;
      st->rnorm_inf = tot1;
      const int it = st->iter + 1;
      st->iter = it;
      const bool pass = st->stop_mode == 0 ? (tot0 <= st->stop_bound) : (tot1 < st->stop_bound);
      record_theta(st, it - 1);
      if (!isfinite(tot0)) st->done = kBreakdown;
      else if (pass) st->done = kConverged;
      else if (it >= st->max_iter) st->done = kMaxIter;
      if (!st->done && st->phase_rho2 > 0.0 && tot0 <= st->phase_rho2 * st->rref2) st->replace = 1;
    }
  }
  if (MU) {
    double tot0, tot1;
    if (grid_reduce2<false>(acc0, acc1, a.partials, &st->counters[kCntMu], &tot0, &tot1)) {
      // mu^(i+1) and the flexible ratio q^(i+1)'(r^(i+1) - r^(i)) / mu^(i)
      // = -vartheta q^(i+1)'y / mu^(i) of the mixed mode
      if (!(tot0 > 0.0) || !isfinite(tot0) || !isfinite(tot1)) {
        st->done = kBreakdown;
      } else {
        if (!st->have_mu) {
          st->beta = 0.0;
        } else {
          st->beta = (-st->theta * tot1) / st->mu;
          record_beta(st, st->iter - 1);
        }
        st->mu = tot0;
        st->have_mu = 1;
      }
    }
  }
}

template <int VAR, int R, int THR>
constexpr size_t sweep_bulk_smem() { return sizeof(bulk::Smem<VAR, R, THR>); }

template <int R, int THR>
inline unsigned sweep_bulk_blocks(const Grid& g) {
  return (unsigned)((long long)g.V * bulk::tiles_per_pair<R, THR>(g.T));
}

}  // namespace hot
}  // namespace lq2d
