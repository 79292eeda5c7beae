// One NBJM sweep (Algorithm 2 inner step), theta_out = Phi~^-1 tau, with the
// per-pair-row operands staged in shared memory.
//
// Phi~ is block diagonal with one block Phi_bar_{v,t} per (column pair v,
// time t) (Section IV-B).  A CTA takes one column pair v and a tile of TT
// consecutive time steps; a group of GS lanes solves one (v, t) block, lane
// a owning unknown a = jj*NS + k of every pair-row (node (i, 2v+jj),
// component k).  All groups of a CTA walk the K pair-rows together.  For
// pair-row i+PD the CTA copies into shared memory, with cp.async while
// pair-row i is computed (PD + 1 buffers, PD = 2):
//   * the factor blocks of pair-row i+PD (both time classes when the tile
//     holds t = T), read by every group of the tile;
//   * the pair-row's own entries for the TT steps (the right-hand side, or
//     r, y, d, delta in the sweep that performs the PCG update);
//   * the eight neighbouring nodes' theta (Omega~ term, same t) or
//     delta^(s) (Xi~ term, t-1 and t+1) for the TT steps: contiguous runs
//     in the component-plane layout;
//   * the Omega~ / Xi~ node blocks of the pair-row's two nodes.
// Per pair-row i, with the block Cholesky factor split at setup into a unit
// block factor F and the pivots D (Phi_bar = F D F'; N1_i = F1_{i+1}',
// N2_i = F2_{i+2}' = D_i^-1 E_i with E_i = A_{i,i+2}, the block of Phi_bar
// coupling pair-row i to pair-row i+2, which is block diagonal):
//   forward:  y_i = tau_i - F2_i y_{i-2} - F1_i y_{i-1}
//   backward: x_i = D_i^-1 (y_i - E_i x_{i+2}) - N1_i x_{i+1}
// Each lane computes one row of every block product, from row-major blocks,
// so a lane's operands are contiguous in shared memory.  Only the last
// product of a step waits for the previous pair-row's result, which keeps
// the dependent chain of a step at 2n multiply-adds.  The forward step
// starts from the lane's own entry of tau; the backward step needs all 2n
// values of y - E x_{i+2}, and the group exchanges them, and each step's
// result, through shared memory.  y is kept in theta_out between the two passes.
// At t = 0, Phi_bar = Q^-1 node by node, so theta = Q tau.
#pragma once

#include <string.h>

#include "kernels.h"

namespace lq2d {
namespace hot {

template <int NS, int THR>
struct SweepGeom {
  static constexpr int G2 = 2 * NS;
  static constexpr int GS = G2 <= 2 ? 2 : G2 <= 4 ? 4 : G2 <= 8 ? 8 : G2 <= 16 ? 16 : 32;
  static constexpr int BS = G2 * G2;
  static constexpr int TT = THR / GS;            // time steps per CTA
  static constexpr int NH = 8;                   // staged neighbour nodes per pair-row
  static constexpr int HW = TT + 2;              // staged time window (t0-1 .. t0+TT)
};

// Pipeline depth (staging buffers; pair-rows in flight = NB - 1).  Two
// pair-rows in flight cover the load latency in both precisions: six
// buffers timed no faster in FP32 on the 64 x 64 x 100 grid and slower on
// the 256 x 256 x 200 grid (fewer CTAs per SM).
template <typename VT>
__host__ __device__ constexpr int sweep_stages() { return 3; }

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

// CNT consecutive elements from shared memory, with 16-byte loads when a run
// of CNT elements is a multiple of 16 bytes (callers keep runs 16-byte
// aligned in that case).
template <typename VT, int CNT>
__device__ __forceinline__ void lds_run(const VT* p, VT (&out)[CNT]) {
  constexpr int bytes = CNT * (int)sizeof(VT);
  if constexpr (bytes % 16 == 0) {
    const int4* q = reinterpret_cast<const int4*>(p);
#pragma unroll
    for (int e = 0; e < bytes / 16; ++e) {
      const int4 v = q[e];
      memcpy(&out[e * (16 / (int)sizeof(VT))], &v, 16);
    }
  } else {
#pragma unroll
    for (int e = 0; e < CNT; ++e) out[e] = p[e];
  }
}

// Offsets (di, dj) of the eight staged neighbours of pair-row i of column
// pair v (j0 = 2v), packed as two bits of di + 1 and three bits of dj + 2.
// Omega~ (off-pair, same t):  (i,j0-1) (i-1,j0-1) (i+1,j0-1) (i,j0-2)
//                             (i,j0+2) (i-1,j0+2) (i+1,j0+2) (i,j0+3)
// Xi~ (5-point, t -/+ 1):     (i,j0) (i,j0+1) (i-1,j0) (i+1,j0)
//                             (i-1,j0+1) (i+1,j0+1) (i,j0-1) (i,j0+2)
constexpr unsigned long long pack_offsets(const int (&di)[8], const int (&dj)[8]) {
  unsigned long long r = 0;
  for (int h = 0; h < 8; ++h)
    r |= (unsigned long long)(((di[h] + 1) & 3) | (((dj[h] + 2) & 7) << 2)) << (5 * h);
  return r;
}
constexpr int kOmDi[8] = {0, -1, 1, 0, 0, -1, 1, 0};
constexpr int kOmDj[8] = {-1, -1, -1, -2, 2, 2, 2, 3};
constexpr int kXiDi[8] = {0, 0, -1, 1, -1, 1, 0, 0};
constexpr int kXiDj[8] = {0, 1, 0, 0, 1, 1, -1, 2};
constexpr unsigned long long kOmPacked = pack_offsets(kOmDi, kOmDj);
constexpr unsigned long long kXiPacked = pack_offsets(kXiDi, kXiDj);

__device__ __forceinline__ int staged_node(bool xi, int h, int i, int j0, int K, int N) {
  const unsigned long long code = ((xi ? kXiPacked : kOmPacked) >> (5 * h)) & 31ull;
  const int di = (int)(code & 3) - 1, dj = (int)(code >> 2) - 2;
  const int ii = i + di, jj = j0 + dj;
  if (ii < 0 || ii >= K || jj < 0 || jj >= N) return -1;
  return ii * N + jj;
}

// Index of the staged node for off-pair neighbour o of column jj (order o0..o4
// of offpair_node), and for direction dir (self, west, east, north, south)
// of the 5-point stencil.
__device__ __forceinline__ int h_of_offpair(int jj, int o) { return jj == 0 ? o : (o == 4 ? 0 : o + 4); }
__device__ __forceinline__ int h_of_dir(int jj, int dir) {
  if (jj == 0) return dir == 0 ? 0 : dir == 1 ? 6 : dir == 2 ? 1 : dir == 3 ? 2 : 3;
  return dir == 0 ? 1 : dir == 1 ? 0 : dir == 2 ? 7 : dir == 3 ? 4 : 5;
}

template <int NS, typename VT, int THR, int NBUF = sweep_stages<VT>()>
struct SweepSmem {
  using Geo = SweepGeom<NS, THR>;
  static constexpr int NB = NBUF;
  VT fac[NB][2][3 * Geo::BS];         // [buffer][class][3 blocks]
  VT halo[NB][Geo::NH][Geo::HW][NS];  // [buffer][h][t window][k]
  VT blk[NB][2][10][NS * NS];         // [buffer][jj][block][n x n]
  VT xw[Geo::TT][Geo::G2];            // per group: y of the current backward step
  VT xy[Geo::TT][Geo::G2];            // per group: result (y or x) of the current step
  double src[NB][4][2][NS][Geo::TT];  // [buffer][r, y, d, delta or src][jj][k][t]; backward: r, y
  VT ys[NB][2][NS][Geo::TT];          // backward: forward result y of the pair-row
  alignas(16) VT qb[NB][2][NS * NS];  // Q of the pair-row's nodes (tiles holding t = 0)
};

// Staging buffers of the two-ended (twisted) solve.  Its CTAs hold two
// halves' staging areas; in FP64 three buffers each would leave room for
// half as many CTAs per SM, which on grids of few (column pair, time) blocks
// costs a second wave, and one pair-row in flight covers the load latency
// of its long FP64 steps.  The shorter FP32 steps keep two in flight.
template <typename VT>
__host__ __device__ constexpr int twisted_stages() { return sizeof(VT) == 8 ? 2 : 3; }

// Shared memory of the interface step of the two-ended solve, after the two
// halves' staging areas: the exchanges between the halves.  (The interface
// couplings and S^-1 are read once per lane, straight from global memory.)
template <int NS, typename VT, int THR>
struct TwistSmem {
  using Geo = SweepGeom<NS, THR>;
  VT xch[2][Geo::TT][Geo::G2];     // each half's y two rows before the interface
  VT rhs[Geo::TT][2 * Geo::G2];    // right-hand side of the interface solve
  VT xs[Geo::TT][2 * Geo::G2];     // x_k, x_{k+1}
};

// Register budget of the sweeps: one CTA per SM fewer than the shared-memory
// footprint allows (233 KB per SM, 1 KB reserved per CTA), which leaves the
// staging descriptors and the block rows in registers without spills.
template <int NS, typename VT, int THR>
constexpr int sweep_min_blocks() {
  constexpr int by_smem = 232448 / ((int)sizeof(SweepSmem<NS, VT, THR>) + 1024) - 1;
  constexpr int by_threads = 2048 / THR;
  constexpr int b = by_smem < by_threads ? by_smem : by_threads;
  return b < 1 ? 1 : (b > 8 ? 8 : b);
}

// The sweep for work unit `bid` of `nblocks` (one CTA's tile: column pair
// bid / tiles, time steps from (bid % tiles) * TT); the kernel below runs one
// unit per CTA, the batched persistent kernel many per CTA.
//
// TW: the two-ended (twisted) solve of each Phi_bar_{v,t}.  The CTA holds
// two halves of THR threads: the top half eliminates pair-rows 0..k with the
// forward factor, the bottom half pair-rows K-1..k+1 with the factor of the
// reversed order (k = (K-2)/2), each with the staging and step of the
// one-sided sweep; then both halves solve the interface rows k, k+1 with
// S^-1 and run their backward substitutions away from it (rows k-1..0 and
// k+2..K-1).  Half the dependent chain, twice the warps per (v, t).
template <int NS, int VAR, typename VT, int THR, bool TW = false>
__device__ __forceinline__ void nbjm_sweep_body(const Grid& g, const PrecData<VT>& pd, const SweepArgsT<VT>& a,
                                                SolverState* st, int bid, int nblocks) {
  // VT = float is the mixed mode: FP32 factors, blocks and iterates, with
  // the flexible (Polak-Ribiere) ratio for the next direction
  constexpr bool FLEX = sizeof(VT) == 4;
  constexpr bool UPDATE = VAR == kSweepUpdate;
  constexpr bool XI = VAR == kSweepXi || VAR == kSweepXiOmega;
  constexpr bool OMEGA = VAR == kSweepOmega || VAR == kSweepOmegaMu || VAR == kSweepXiOmega;
  constexpr bool MU = VAR == kSweepOmegaMu;
  constexpr bool HALO = XI || OMEGA;
  using Geo = SweepGeom<NS, THR>;
  constexpr int G2 = Geo::G2, GS = Geo::GS, BS = Geo::BS, TT = Geo::TT, HW = Geo::HW;
  extern __shared__ __align__(16) unsigned char sweep_smem[];
  constexpr int NB = TW ? twisted_stages<VT>() : sweep_stages<VT>();
  constexpr int PD = NB - 1;  // prefetch distance in pair-rows
  using Smem = SweepSmem<NS, VT, THR, NB>;
  const int half = TW ? (int)(threadIdx.x / THR) : 0;  // 0: top (or one-sided), 1: bottom
  Smem& sm = reinterpret_cast<Smem*>(sweep_smem)[half];
  TwistSmem<NS, VT, THR>& tw = *reinterpret_cast<TwistSmem<NS, VT, THR>*>(sweep_smem + 2 * sizeof(Smem));
  const int K = g.K;
  const int kI = TW ? (K - 2) / 2 : 0;                                // interface rows kI, kI + 1
  const int nf = TW ? (half ? K - kI - 1 : kI + 1) : K;               // forward steps of this half
  const int nb = TW ? (half ? K - kI - 2 : kI) : K;                   // backward steps of this half
  const int nf_all = TW ? (kI + 1 > K - kI - 1 ? kI + 1 : K - kI - 1) : K;
  const int nb_all = TW ? (kI > K - kI - 2 ? kI : K - kI - 2) : K;
  // physical pair-row of forward step s and of backward step s, and the
  // record of the half's factor that backward step s reads
  auto row_f = [&](int s) { return half ? K - 1 - s : s; };
  auto row_b = [&](int s) { return TW ? (half ? kI + 2 + s : kI - 1 - s) : K - 1 - s; };
  auto rec_b = [&](int s) { return half ? K - 1 - row_b(s) : row_b(s); };

  if (st != nullptr && st->done) return;
  const int Tp = g.T + 1;
  const int tiles = (Tp + TT - 1) / TT;
  const int v = bid / tiles;
  const int t0 = (bid % tiles) * TT;
  const int j0 = 2 * v;
  const bool two_cols = j0 + 1 < g.N;
  const bool has_last = t0 + TT > g.T;  // the tile holds t = T (class 1)
  const int tid = TW ? (int)(threadIdx.x % THR) : (int)threadIdx.x;
  const int lane32 = tid & 31;
  const int al = tid & (GS - 1);
  const int grp = tid / GS;
  const unsigned gmask = GS == 32 ? 0xffffffffu : (((1u << GS) - 1u) << (lane32 & ~(GS - 1)));
  const int t = t0 + grp;
  const bool active = t <= g.T;
  const bool lane_ok = al < G2;
  const int ac = lane_ok ? al : 0;
  const int jj = ac / NS, k = ac % NS;
  const int j = j0 + jj;
  const bool node_ok = active && lane_ok && j < g.N;
  const long long kP = (long long)k * g.Ps;
  // element index of an iterate (theta, delta^(s)) at component kk of
  // pt = node*(T+1) + t: component planes in FP64, node-major in FP32
  auto it_idx = [&](int kk, long long pt) -> long long { return FLEX ? pt * NS + kk : kk * g.Ps + pt; };
  constexpr int VS = FLEX ? NS : 1;  // iterate elements per (node, t) step along a row
  const int cls = (t == g.T) ? 1 : 0;
  const int my_slot = has_last ? cls : 0;  // tiles without t = T stage class 0 only, at slot 0
  const double vth = UPDATE ? st->theta : 0.0;
  const bool flex_dot = FLEX && MU && st->have_mu;
  const VT* fac_pair = (half ? pd.fac_rev : pd.fac) + (size_t)(2 * v) * pd.fac_vc;  // class c at + c * fac_vc
  const int ncls = has_last ? 2 : 1;
  constexpr int CH = 16 / sizeof(VT);  // elements per 16-byte copy
  double acc0 = 0.0, acc1 = 0.0;

  // ---- staging descriptors.  Every staged array is a fixed set of
  // elements per thread ("slots"): slot sl of thread tid is element
  // e = tid + sl * THR (16-byte chunk e for the factor and node-block runs).
  // An element's shared-memory place is fixed and its global address
  // advances by one grid row (N nodes) per pair-row, so each thread keeps
  // one pointer per slot, set for pair-row 0, and a step adds the row
  // offset.  In-range flags are bit masks over the slots; for the halo the
  // row above / below exists or not with the pair-row, which two more masks
  // (slots with di < 0, di > 0) select.
  const long long row_stride = (long long)g.N * Tp;
  const unsigned long long packed = XI ? kXiPacked : kOmPacked;
  // FP32 node-major iterates at n = 4: one (node, t) is a 16-byte run, staged
  // by one copy; otherwise one copy per element
  constexpr bool H16 = FLEX && NS == 4;
  constexpr int HU = H16 ? NS : 1;  // elements per halo copy
  constexpr int HALO_N = HALO ? Geo::NH * NS * HW / HU : 0;
  constexpr int HSL = (HALO_N + THR - 1) / THR > 0 ? (HALO_N + THR - 1) / THR : 1;
  const VT* h_ptr[HSL];
  unsigned h_ok = 0u, h_up = 0u, h_dn = 0u;
  if constexpr (HALO) {
    const VT* vec = XI ? a.delta_s : a.theta_in;
#pragma unroll
    for (int sl = 0; sl < HSL; ++sl) {
      // component fastest, so that consecutive threads fill consecutive
      // words of the [h][w][k] staging array
      const int e = (tid + sl * THR) * HU;
      const int h = e / (NS * HW), w = (e / NS) % HW, kk = e % NS;
      const int tt = t0 - 1 + w;
      const unsigned code = (unsigned)((packed >> (5 * (h & 7))) & 31ull);
      const int di = (int)(code & 3u) - 1, jn = j0 + (int)(code >> 2) - 2;
      const bool ok = tid + sl * THR < HALO_N && tt >= 0 && tt <= g.T && jn >= 0 && jn < g.N;
      // pair-row 0's address; at di = -1 it lies one grid row below the
      // plane's start and is used only from pair-row 1 on
      h_ptr[sl] = vec + (ok ? it_idx(kk, (long long)(di * g.N + jn) * Tp + tt) : 0);
      if (ok) h_ok |= 1u << sl;
      if (di < 0) h_up |= 1u << sl;
      if (di > 0) h_dn |= 1u << sl;
    }
  } else {
    h_ptr[0] = nullptr;
  }
  // node blocks: runs of 5 n x n blocks per node (Omega~: Om of both nodes;
  // Xi~: AQ and QAt of both nodes), 16-byte chunks where a run is a multiple
  // of 16 bytes
  constexpr int RUN = 5 * NS * NS;
  constexpr int CB = (RUN * (int)sizeof(VT)) % 16 == 0 ? 16 / (int)sizeof(VT) : 1;
  constexpr int NRUN = XI ? 4 : 2;
  constexpr int BLK_N = HALO ? NRUN * (RUN / CB) : 0;
  constexpr int BSL = (BLK_N + THR - 1) / THR > 0 ? (BLK_N + THR - 1) / THR : 1;
  const VT* b_ptr[BSL];
  int b_sm[BSL];
  unsigned b_ok = 0u;
#pragma unroll
  for (int sl = 0; sl < BSL; ++sl) {
    const int c = tid + sl * THR;
    const int run = c / (RUN / CB), within = (c % (RUN / CB)) * CB;
    const int cjj = run & 1;
    const bool ok = HALO && c < BLK_N && (cjj == 0 || two_cols);
    const VT* arr = XI ? (run >= 2 ? pd.QAt : pd.AQ) : pd.Om;
    b_ptr[sl] = ok ? arr + (size_t)(j0 + cjj) * RUN + within : nullptr;
    b_sm[sl] = (cjj * 10 + (run >= 2 ? 5 : 0)) * NS * NS + within;
    if (ok) b_ok |= 1u << sl;
  }
  // the pair-row's own entries for the tile (double): r, y, d, delta in the
  // update sweep, else the source; element e = ((vv * 2 + jj) * NS + k) * TT + t
  constexpr int NV = UPDATE ? 4 : 1;
  constexpr int SRC_N = NV * 2 * NS * TT;
  constexpr int SSL = (SRC_N + THR - 1) / THR;
  const double* s_ptr[SSL];
  unsigned s_ok = 0u;
#pragma unroll
  for (int sl = 0; sl < SSL; ++sl) {
    const int e = tid + sl * THR;
    const int vv = e / (2 * NS * TT), cjj = (e / (NS * TT)) % 2, kk = (e / TT) % NS, gg = e % TT;
    const int tt = t0 + gg;
    const bool ok = e < SRC_N && tt <= g.T && (cjj == 0 || two_cols);
    const double* base = UPDATE ? (vv == 0 ? a.r : vv == 1 ? a.y : vv == 2 ? a.d : a.delta) : a.src;
    s_ptr[sl] = ok ? base + kk * g.Ps + (long long)(j0 + cjj) * Tp + tt : nullptr;
    if (ok) s_ok |= 1u << sl;
  }
  // factor blocks, 16-byte chunks: forward F2, F1 (record blocks 4..5),
  // backward N1, D^-1, E (blocks 1..3), per class present in the tile
  constexpr int FSL = (2 * 2 * BS + THR * CH - 1) / (THR * CH);
  constexpr int FSLB = (2 * 3 * BS + THR * CH - 1) / (THR * CH);
  const VT* f_ptr[FSL];
  int f_sm[FSL];
  unsigned f_ok = 0u;
#pragma unroll
  for (int sl = 0; sl < FSL; ++sl) {
    const int e = (tid + sl * THR) * CH;
    const int c = e / (2 * BS), off = e % (2 * BS);
    f_ptr[sl] = fac_pair + (size_t)c * pd.fac_vc + 4 * BS + off;
    f_sm[sl] = c * 3 * BS + off;
    if (e < ncls * 2 * BS) f_ok |= 1u << sl;
  }
  const VT* fb_ptr[FSLB];
  unsigned fb_ok = 0u;
#pragma unroll
  for (int sl = 0; sl < FSLB; ++sl) {
    const int e = (tid + sl * THR) * CH;  // also the shared-memory place
    fb_ptr[sl] = fac_pair + (size_t)(e / (3 * BS)) * pd.fac_vc + BS + e % (3 * BS);
    if (e < ncls * 3 * BS) fb_ok |= 1u << sl;
  }
  // backward pass: the forward result y_i of the tile (kept in theta_out
  // between the passes; written by this CTA before the barrier that ends the
  // forward pass), and in the mu sweep r (and y of Algorithm 1 for the
  // flexible ratio); element e = ((vv * 2 + jj) * NS + k) * TT + t, vv = 0
  // for y_i (VT), 1.. for r, y (double)
  constexpr int NVB = MU ? (FLEX ? 3 : 2) : 1;
  constexpr int BN = NVB * 2 * NS * TT;
  constexpr int BSLB = (BN + THR - 1) / THR;
  const char* bs_ptr[BSLB];
  int bs_sm[BSLB];
  unsigned bs_ok = 0u, bs_y = 0u;
#pragma unroll
  for (int sl = 0; sl < BSLB; ++sl) {
    const int e = tid + sl * THR;
    const int vv = e / (2 * NS * TT), w = e % (2 * NS * TT), cjj = w / (NS * TT), gg = e % TT;
    const int tt = t0 + gg;
    const bool ok = e < BN && tt <= g.T && (cjj == 0 || two_cols);
    const long long go = ((e / TT) % NS) * g.Ps + (long long)(j0 + cjj) * Tp + tt;
    if (vv == 0) {
      const long long gi = it_idx((e / TT) % NS, (long long)(j0 + cjj) * Tp + tt);
      bs_ptr[sl] = ok ? reinterpret_cast<const char*>(a.theta_out + gi) : nullptr;
      bs_sm[sl] = w;
      bs_y |= 1u << sl;
    } else {
      bs_ptr[sl] = ok ? reinterpret_cast<const char*>((vv == 1 ? a.r : a.y) + go) : nullptr;
      bs_sm[sl] = (vv - 1) * 2 * NS * TT + w;
    }
    if (ok) bs_ok |= 1u << sl;
  }
  // staged neighbours inside the grid, by pair-row: the column test is fixed
  // for the CTA, the row test depends on whether the row above / below exists
  unsigned col_ok = 0u, above = 0u, below = 0u;
#pragma unroll
  for (int h = 0; h < Geo::NH; ++h) {
    const unsigned code = (unsigned)((packed >> (5 * h)) & 31ull);
    const int di = (int)(code & 3u) - 1, jn = j0 + (int)(code >> 2) - 2;
    if (jn >= 0 && jn < g.N) col_ok |= 1u << h;
    if (di < 0) above |= 1u << h;
    if (di > 0) below |= 1u << h;
  }
  auto row_valid = [&](int i) -> unsigned {
    unsigned m = col_ok;
    if (i < 1) m &= ~above;
    if (i + 1 >= g.K) m &= ~below;
    return m;
  };

  // ---- staging of the forward step for pair-row i into buffer b: F2, F1
  // of pair-row i per class, Q of its nodes (tiles holding t = 0), its own
  // entries, the neighbours' halo and the node blocks
  auto stage_forward = [&](int step, int b) {
    const int i = row_f(step);  // physical pair-row; the record is the half's step
    const long long rb = (long long)i * row_stride;
    const long long fo = (long long)step * pd.fac_rec;
#pragma unroll
    for (int sl = 0; sl < FSL; ++sl)
      if ((f_ok >> sl) & 1u) cp_async_16(&sm.fac[b][0][0] + f_sm[sl], f_ptr[sl] + fo);
    if (t0 == 0) {
      // Q of the pair-row's nodes, for theta = Q tau at t = 0
      for (int e = tid; e < 2 * NS * NS; e += THR) {
        const int cjj = e / (NS * NS), w = e % (NS * NS);
        if (cjj == 1 && !two_cols) continue;
        cp_async_elem(&sm.qb[b][cjj][w], pd.Qm + (size_t)(i * g.N + j0 + cjj) * NS * NS + w);
      }
    }
#pragma unroll
    for (int sl = 0; sl < SSL; ++sl)
      if ((s_ok >> sl) & 1u) cp_async_8(&sm.src[b][0][0][0][0] + tid + sl * THR, s_ptr[sl] + rb);
    if constexpr (HALO) {
      const unsigned hv = h_ok & (i == 0 ? ~h_up : ~0u) & (i + 1 >= g.K ? ~h_dn : ~0u);
#pragma unroll
      for (int sl = 0; sl < HSL; ++sl)
        if ((hv >> sl) & 1u) {
          VT* dst = &sm.halo[b][0][0][0] + (tid + sl * THR) * HU;
          if constexpr (H16) cp_async_16(dst, h_ptr[sl] + rb * VS);
          else cp_async_elem(dst, h_ptr[sl] + rb * VS);
        }
      const long long bb = (long long)i * g.N * RUN;
#pragma unroll
      for (int sl = 0; sl < BSL; ++sl) {
        if (!((b_ok >> sl) & 1u)) continue;
        if constexpr (CB > 1) cp_async_16(&sm.blk[b][0][0][0] + b_sm[sl], b_ptr[sl] + bb);
        else cp_async_elem(&sm.blk[b][0][0][0] + b_sm[sl], b_ptr[sl] + bb);
      }
    }
  };

  // ---- staging of the backward step for pair-row i: N1, D^-1 and E of
  // pair-row i, y_i of the tile and, in the mu sweep, r (and y)
  auto stage_backward = [&](int step, int b) {
    const int i = row_b(step);
    const long long fo = (long long)rec_b(step) * pd.fac_rec;
#pragma unroll
    for (int sl = 0; sl < FSLB; ++sl)
      if ((fb_ok >> sl) & 1u) cp_async_16(&sm.fac[b][0][0] + (tid + sl * THR) * CH, fb_ptr[sl] + fo);
    const long long rb = (long long)i * row_stride;
#pragma unroll
    for (int sl = 0; sl < BSLB; ++sl) {
      if (!((bs_ok >> sl) & 1u)) continue;
      if ((bs_y >> sl) & 1u)
        cp_async_elem(&sm.ys[b][0][0][0] + bs_sm[sl], reinterpret_cast<const VT*>(bs_ptr[sl]) + rb * VS);
      else
        cp_async_8(&sm.src[b][0][0][0][0] + bs_sm[sl], reinterpret_cast<const double*>(bs_ptr[sl]) + rb);
    }
  };

  VT ym1[G2], ym2[G2];
#pragma unroll
  for (int bb = 0; bb < G2; ++bb) { ym1[bb] = VT(0); ym2[bb] = VT(0); }
  VT y_last = VT(0);  // the lane's own result of the half's last forward step

  // one commit group per pair-row (empty past the last one), so that the
  // wait below counts pair-rows
#pragma unroll
  for (int s0 = 0; s0 < PD; ++s0) {
    if (s0 < nf) stage_forward(s0, s0);
    cp_async_commit();
  }
  for (int fs = 0; fs < nf_all; ++fs) {
    const int b = fs % NB;
    const int i = row_f(fs);
    const int p = i * g.N + j;
    const long long off = node_ok ? (long long)p * Tp + t : 0;
    // step fs has landed (steps fs+1 .. fs+PD-1 may be in flight); after the
    // barrier every thread is done with step fs-1, whose buffer takes step
    // fs+PD.  A half with fewer steps (two-ended solve, K odd) idles through
    // the last one.
    cp_async_wait<PD - 1>();
    __syncthreads();
    if (fs + PD < nf) stage_forward(fs + PD, (fs + PD) % NB);
    cp_async_commit();
    if (fs >= nf) continue;
    const unsigned valid = HALO ? row_valid(i) : 0u;
    VT tau = VT(0);
    if (node_ok) {
      if (UPDATE) {
        const double rr = sm.src[b][0][jj][k][grp] - vth * sm.src[b][1][jj][k][grp];
        a.r[kP + off] = rr;
        a.delta[kP + off] = sm.src[b][3][jj][k][grp] + vth * sm.src[b][2][jj][k][grp];
        tau = (VT)rr;
        acc0 += rr * rr;
        acc1 = fmax(acc1, fabs(rr));
      } else {
        tau = (VT)sm.src[b][0][jj][k][grp];
      }
      if (XI) {
        // (Xi~ delta)_t = A_hat Q^-1 delta_{t-1} + Q^-1 A_hat' delta_{t+1}
#pragma unroll
        for (int dir = 0; dir < 5; ++dir) {
          const int h = h_of_dir(jj, dir);
          if (!((valid >> h) & 1u)) continue;
          if (t >= 1) {
            VT row[NS], hv[NS];
            lds_run<VT, NS>(&sm.blk[b][jj][dir][k * NS], row);
            lds_run<VT, NS>(&sm.halo[b][h][grp][0], hv);
#pragma unroll
            for (int c = 0; c < NS; ++c) tau += row[c] * hv[c];
          }
          if (t < g.T) {
            VT row[NS], hv[NS];
            lds_run<VT, NS>(&sm.blk[b][jj][5 + dir][k * NS], row);
            lds_run<VT, NS>(&sm.halo[b][h][grp + 2][0], hv);
#pragma unroll
            for (int c = 0; c < NS; ++c) tau += row[c] * hv[c];
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
            for (int c = 0; c < NS; ++c) tau += blk[c] * a.theta_in[it_idx(c, qb)];
          }
        } else {
#pragma unroll
          for (int o = 0; o < 5; ++o) {
            const int h = h_of_offpair(jj, o);
            if (!((valid >> h) & 1u)) continue;
            VT row[NS], hv[NS];
            lds_run<VT, NS>(&sm.blk[b][jj][o][k * NS], row);
            lds_run<VT, NS>(&sm.halo[b][h][grp + 1][0], hv);
#pragma unroll
            for (int c = 0; c < NS; ++c) tau += row[c] * hv[c];
          }
        }
      }
    }
    if (t == 0) {
      // Phi_bar_{v,0} = blkdiag(Q^-1): theta = Q tau, node by node (Q rows
      // staged with the pair-row; the mu terms of t = 0 are added in the
      // backward pass, where r and y of the tile are staged)
      VT out = VT(0);
      VT Qrow[NS];
      lds_run<VT, NS>(&sm.qb[b][jj][k * NS], Qrow);
#pragma unroll
      for (int c = 0; c < NS; ++c) {
        const VT tc = __shfl_sync(gmask, tau, jj * NS + c, GS);
        out += Qrow[c] * tc;
      }
      if (node_ok) a.theta_out[it_idx(k, off)] = out;
      y_last = out;
    } else {
      // y_i = tau_i - F2 y_{i-2} - F1 y_{i-1}, one chain of multiply-adds
      // (the FP64 pipe's issue rate, not its latency, bounds the sweep, so
      // no partial sums are split off)
      const VT* rec = sm.fac[b][my_slot];  // [F2][F1], row-major
      VT yv = tau;
      if (fs >= 2) {
        VT row[G2];
        lds_run<VT, G2>(rec + ac * G2, row);
#pragma unroll
        for (int bb = 0; bb < G2; ++bb) yv -= row[bb] * ym2[bb];
      }
      if (fs >= 1) {
        VT row[G2];
        lds_run<VT, G2>(rec + BS + ac * G2, row);
#pragma unroll
        for (int bb = 0; bb < G2; ++bb) yv -= row[bb] * ym1[bb];
      }
      if (node_ok) a.theta_out[it_idx(k, off)] = yv;
      y_last = yv;
      if (lane_ok) sm.xy[grp][al] = yv;
      __syncwarp(gmask);
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) ym2[bb] = ym1[bb];
      lds_run<VT, G2>(&sm.xy[grp][0], ym1);
    }
  }
  cp_async_wait<0>();
  __syncthreads();

  VT xp1[G2], xp2[G2];
#pragma unroll
  for (int bb = 0; bb < G2; ++bb) { xp1[bb] = VT(0); xp2[bb] = VT(0); }

  // ---- interface of the two-ended solve, rows k and k+1:
  //   [x_k; x_{k+1}] = S^-1 [y_k - J w_{k+2}; w_{k+1} - H y_{k-1}]
  // (y: top half's forward results, w: bottom half's), which seeds both
  // backward substitutions
  if constexpr (TW) {
    // the lane's rows of the coupling (top: J, the reversed factor's F2 of
    // row k; bottom: H, the forward factor's F2 of row k+1) and of S^-1
    const VT* Cm = half ? pd.fac + (size_t)(2 * v + cls) * pd.fac_vc + (size_t)(kI + 1) * pd.fac_rec
                        : pd.fac_rev + (size_t)(2 * v + cls) * pd.fac_vc + (size_t)(K - kI - 1) * pd.fac_rec;
    Cm += 4 * BS + ac * G2;
    const VT* Srow = pd.sinv + (size_t)(2 * v + cls) * 4 * BS + (half * G2 + ac) * 2 * G2;
    if (active && al == 0) {
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) tw.xch[half][grp][bb] = ym2[bb];
    }
    __syncthreads();
    if (active && lane_ok && t >= 1) {
      VT rr = y_last;
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) rr -= Cm[bb] * tw.xch[half ^ 1][grp][bb];
      tw.rhs[grp][half * G2 + al] = rr;
    }
    __syncthreads();
    if (active && lane_ok) {
      const long long offI = ((long long)(kI + half) * g.N + j) * Tp + t;
      VT xv = y_last;  // t = 0: theta_0 = Q tau_0 is final after the forward pass
      if (t >= 1) {
        xv = VT(0);
#pragma unroll
        for (int c = 0; c < 2 * G2; ++c) xv += Srow[c] * tw.rhs[grp][c];
        if (node_ok) a.theta_out[it_idx(k, offI)] = xv;
      }
      if (node_ok) {
        if (MU) acc0 += (double)xv * a.r[kP + offI];
        if (flex_dot) acc1 += (double)xv * a.y[kP + offI];
      }
      tw.xs[grp][half * G2 + al] = xv;
    }
    __syncthreads();
    if (active) {
      // top: x_{i+1} = x_k, x_{i+2} = x_{k+1}; bottom: x_{i-1} = x_{k+1}, x_{i-2} = x_k
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) {
        xp1[bb] = tw.xs[grp][half * G2 + bb];
        xp2[bb] = tw.xs[grp][(half ^ 1) * G2 + bb];
      }
    }
  }

  // ---- backward substitution (one-sided: pair-rows K-1..0; two-ended: each
  // half from the interface outwards)
#pragma unroll
  for (int s0 = 0; s0 < PD; ++s0) {
    if (s0 < nb) stage_backward(s0, s0);
    cp_async_commit();
  }
  for (int bstep = 0; bstep < nb_all; ++bstep) {
    const int i = row_b(bstep);
    const int b = bstep % NB;
    const int p = i * g.N + j;
    const long long off = node_ok ? (long long)p * Tp + t : 0;
    cp_async_wait<PD - 1>();
    __syncthreads();
    if (bstep + PD < nb) stage_backward(bstep + PD, (bstep + PD) % NB);
    cp_async_commit();
    if (bstep >= nb) continue;
    VT yown = VT(0);
    double r_own = 0.0, y_own = 0.0;
    if (node_ok) {
      yown = sm.ys[b][jj][k][grp];
      if (MU) r_own = sm.src[b][0][jj][k][grp];
      if (flex_dot) y_own = sm.src[b][1][jj][k][grp];
      if (t == 0) {
        // theta_0 = Q tau_0 is final after the forward pass
        if (MU) acc0 += (double)yown * r_own;
        if (flex_dot) acc1 += (double)yown * y_own;
      }
    }
    if (t >= 1) {
      // x_i = D^-1 (y_i - E x_{i+2}) - N1 x_{i+1}  (= D^-1 y_i - N2 x_{i+2} -
      // N1 x_{i+1} with N2 = D^-1 E; E is block diagonal, so the lane's row
      // of it meets only its own node's n components of x_{i+2})
      const VT* rec = sm.fac[b][my_slot];  // [N1][D^-1][E], row-major
      VT vown = yown;
      if (TW || i + 2 < g.K) {
        VT erow[NS];
        lds_run<VT, NS>(rec + 2 * BS + ac * G2 + jj * NS, erow);
#pragma unroll
        for (int c = 0; c < NS; ++c) vown -= erow[c] * (jj ? xp2[NS + c] : xp2[c]);
      }
      if (lane_ok) sm.xw[grp][al] = vown;
      __syncwarp(gmask);
      VT vall[G2], row0[G2];
      lds_run<VT, G2>(&sm.xw[grp][0], vall);
      lds_run<VT, G2>(rec + BS + ac * G2, row0);
      VT xv = VT(0);
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) xv += row0[bb] * vall[bb];
      if (TW || i + 1 < g.K) {
        VT row[G2];
        lds_run<VT, G2>(rec + ac * G2, row);
#pragma unroll
        for (int bb = 0; bb < G2; ++bb) xv -= row[bb] * xp1[bb];
      }
      if (node_ok) {
        a.theta_out[it_idx(k, off)] = xv;
        if (MU) acc0 += (double)xv * r_own;
        if (flex_dot) acc1 += (double)xv * y_own;
      }
      if (lane_ok) sm.xy[grp][al] = xv;
      __syncwarp(gmask);
#pragma unroll
      for (int bb = 0; bb < G2; ++bb) xp2[bb] = xp1[bb];
      lds_run<VT, G2>(&sm.xy[grp][0], xp1);
    }
  }
  cp_async_wait<0>();

  if (UPDATE) {
    double tot0, tot1;
    if (grid_reduce2_at<true>(acc0, acc1, a.partials, &st->counters[kCntNorm], &tot0, &tot1, bid, nblocks)) {
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
      // precision mode 2: the residual is due for replacement by the true one
      if (!st->done && st->phase_rho2 > 0.0 && tot0 <= st->phase_rho2 * st->rref2) st->replace = 1;
    }
  }
  if (MU) {
    double tot0, tot1;
    if (grid_reduce2_at<false>(acc0, acc1, a.partials, &st->counters[kCntMu], &tot0, &tot1, bid, nblocks)) {
      // Algorithm 1: mu^(i+1) and the ratio used for d^(i+1);
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

template <int NS, int VAR, typename VT, int THR>
__global__ void __launch_bounds__(THR, (sweep_min_blocks<NS, VT, THR>()))
    nbjm_sweep_kernel(Grid g, PrecData<VT> pd, SweepArgsT<VT> a, SolverState* st) {
  nbjm_sweep_body<NS, VAR, VT, THR>(g, pd, a, st, blockIdx.x, gridDim.x);
}

// The two-ended solve: CTAs of 2 THR threads (two halves).
template <int NS, typename VT, int THR>
constexpr size_t sweep_twisted_smem_bytes() {
  return 2 * sizeof(SweepSmem<NS, VT, THR, twisted_stages<VT>()>) + sizeof(TwistSmem<NS, VT, THR>);
}

// CTAs per SM the two-ended sweep's shared memory allows (at most 8)
template <int NS, typename VT, int THR>
constexpr int sweep_twisted_min_blocks() {
  constexpr int by_smem = 232448 / ((int)sweep_twisted_smem_bytes<NS, VT, THR>() + 1024);
  constexpr int by_threads = 2048 / (2 * THR);
  constexpr int b = by_smem < by_threads ? by_smem : by_threads;
  return b < 1 ? 1 : (b > 8 ? 8 : b);
}

template <int NS, int VAR, typename VT, int THR>
__global__ void __launch_bounds__(2 * THR, (sweep_twisted_min_blocks<NS, VT, THR>()))
    nbjm_sweep_twisted_kernel(Grid g, PrecData<VT> pd, SweepArgsT<VT> a, SolverState* st) {
  nbjm_sweep_body<NS, VAR, VT, THR, true>(g, pd, a, st, blockIdx.x, gridDim.x);
}

template <int NS, typename VT, int THR>
constexpr size_t sweep_smem_bytes() { return sizeof(SweepSmem<NS, VT, THR>); }


template <int NS, int THR>
inline unsigned sweep_blocks(const Grid& g) {
  constexpr int TT = SweepGeom<NS, THR>::TT;
  const int tiles = (g.T + 1 + TT - 1) / TT;
  return (unsigned)((long long)g.V * tiles);
}

}  // namespace hot
}  // namespace lq2d
