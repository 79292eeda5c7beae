// Multi-right-hand-side NBJM sweeps on the tensor cores.
//
// Many initial states x0 of one problem give right-hand sides r_delta that
// share Delta, its splittings and the banded factors of Phi_bar (Section
// IV-B).  Solving Phi~ theta = tau for 32 of them at once turns every block
// product of a sweep step into a small matrix product: for the pair-row
// blocks (2n = 8 unknowns) an 8 x 8 block times an 8 x 32 panel of
// right-hand sides, for the Omega~ / Xi~ coupling an 8 x 32 matrix (the
// pair-row against its eight staged neighbour nodes) times a 32 x 32 panel.
// These run as mma.sync.m16n8k8 with TF32 operands and FP32 accumulation:
//
//   D (16 rhs x 8 rows) += A (16 rhs x 8 cols) * B (8 cols x 8 rows),
//   A[m][c] = panel[c][m],  B[c][a] = block[a][c],
//
// so the right-hand sides are the M dimension (two tiles of 16) and the
// block rows the N dimension.  A warp owns one (column pair v, time t):
// fragments (PTX ISA, m16n8k8 .tf32; g = lane / 4, q = lane % 4):
//   A: a0 (g, q) a1 (g+8, q) a2 (g, q+4) a3 (g+8, q+4)
//   B: b0 (q, g) b1 (q+4, g)
//   D: d0 (g, 2q) d1 (g, 2q+1) d2 (g+8, 2q) d3 (g+8, 2q+1)
// Results leave the D layout through a shared-memory panel [8 rows][32 rhs],
// from which the next product reads its A fragment.
//
// The factor record of a pair-row holds six blocks (the unit block factor F
// of Phi_bar = F D F', as in the single-RHS sweep, with the pivot inverse
// D^-1 = L0^-T L0^-1 kept as its two triangular factors):
//   0: -N2  1: -N1  2: L0^-T   (backward: x_i = L0^-T z_i - N2 x_{i+2} - N1 x_{i+1})
//   3: -F2  4: -F1  5: L0^-1   (forward:  y_i = tau_i - F2 y_{i-2} - F1 y_{i-1},
//                                         z_i = L0^-1 y_i)
// each stored as B fragments, lane-major: element 2*lane + k of a block is
// b_k of that lane.  In TF32 the two triangular products keep the rounding
// error at the condition number of L0, where one product with D^-1 would
// take that of D, its square.  The forward step starts from tau's
// accumulator.  Class 2 is t = 0, where Phi_bar = Q^-1 node by node: there
// block 5 is blkdiag(Q, Q) of the pair's two nodes, y = Q tau is final and
// the other forward blocks are zero (the backward pass is skipped at t = 0).
#include "mrhs.h"
#include "sweep_tiled.cuh"

namespace lq2d {
namespace mrhs {

namespace {

constexpr int kWpc = 4;                  // warps (time steps) per CTA
constexpr int kNb = 2;                   // staging buffers
constexpr int kPs = 32;                  // row stride (floats) of the [rows][32 rhs] panels
constexpr int kRec = 384;                // floats per pair-row record
constexpr int kW = 256;                  // floats per coupling matrix (4 k-steps of 64)

__device__ __forceinline__ unsigned tf32_bits(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 16-byte copy to shared memory; a false `valid` writes zeros instead.
__device__ __forceinline__ void cp16z(float* smem, const float* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int bytes = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes) : "memory");
}

// Panels P[row][rhs] are stored with a swizzle: element (row, col) sits at
// row * kPs + (col ^ swz(row)).  It moves whole 8-float groups, so 16-byte
// chunks stay contiguous, and it spreads the four rows an A fragment reads
// at once (rows c0 + q, q = 0..3) over all 32 banks.
__device__ __forceinline__ int swz(int row) { return (row & 3) << 3; }
__device__ __forceinline__ int pidx(int row, int col) { return row * kPs + (col ^ swz(row)); }

// A fragment (16 rhs x 8 columns) of right-hand-side tile `tile` from a
// panel P[col][rhs], with columns c0 .. c0+7 (c0 a multiple of 8).
__device__ __forceinline__ void a_frag(const float* P, int c0, int tile, int g, int q, unsigned (&a)[4]) {
  const int m = g + 16 * tile;
  a[0] = tf32_bits(P[pidx(c0 + q, m)]);
  a[1] = tf32_bits(P[pidx(c0 + q, m + 8)]);
  a[2] = tf32_bits(P[pidx(c0 + q + 4, m)]);
  a[3] = tf32_bits(P[pidx(c0 + q + 4, m + 8)]);
}

// D fragment of tile `tile` to / from a panel P[row][rhs].
__device__ __forceinline__ void d_store(float* P, int tile, int g, int q, const float (&d)[4]) {
  const int m = g + 16 * tile;
  P[pidx(2 * q, m)] = d[0];
  P[pidx(2 * q + 1, m)] = d[1];
  P[pidx(2 * q, m + 8)] = d[2];
  P[pidx(2 * q + 1, m + 8)] = d[3];
}
__device__ __forceinline__ void d_load(const float* P, int tile, int g, int q, float (&d)[4]) {
  const int m = g + 16 * tile;
  d[0] = P[pidx(2 * q, m)];
  d[1] = P[pidx(2 * q + 1, m)];
  d[2] = P[pidx(2 * q, m + 8)];
  d[3] = P[pidx(2 * q + 1, m + 8)];
}

// Writes an 8 x 32 panel P[a][rhs] (pair-row unknown a = jj*4 + k) to a
// vector as 16-byte chunks: lane (k = lane / 8, chunk = lane % 8) writes
// row a = 4 jj + k for jj = 0, 1.  pt0 is the (node, time) offset of the
// pair's first node, times 32; the second node follows at + (T+1)*32.
__device__ __forceinline__ void panel_to_global(float* vec, const float* P, long long plane, long long pt0,
                                                long long node_step, bool two, int lane) {
  const int k = lane >> 3, ch = lane & 7;
#pragma unroll
  for (int jj = 0; jj < 2; ++jj) {
    if (jj == 1 && !two) continue;
    const float4 val = *reinterpret_cast<const float4*>(P + pidx(4 * jj + k, ch * 4));
    *reinterpret_cast<float4*>(vec + k * plane + pt0 + jj * node_step + ch * 4) = val;
  }
}

// Shared-memory layout of variant VAR.  The neighbour panels are time
// slices shared by the CTA's warps: slice s holds time t0 - 1 + s for the
// Xi~ sweep (kWpc + 2 slices; warp w reads slices w and w + 2, i.e. t - 1
// and t + 1) and t0 + s for the Omega~ sweep (kWpc slices).
template <int VAR>
struct Layout {
  static constexpr int NW = VAR == 0 ? 0 : (VAR == 1 ? 1 : 2);   // coupling matrices
  static constexpr int NSL = VAR == 0 ? 0 : (VAR == 1 ? kWpc : kWpc + 2);  // neighbour slices
  // offsets in floats of the dynamic shared memory
  static constexpr int rec = 0;                                   // [kNb][3][kRec]
  static constexpr int w = rec + kNb * 3 * kRec;                  // [kNb][NW][kW]
  static constexpr int src = w + kNb * NW * kW;                   // [kNb][kWpc][8][kPs]
  static constexpr int halo = src + kNb * kWpc * 8 * kPs;         // [kNb][NSL][32][kPs]
  static constexpr int ring = halo + kNb * NSL * 32 * kPs;        // [kWpc][3][8][kPs]
  static constexpr int xch = ring + kWpc * 3 * 8 * kPs;           // [kWpc][8][kPs]
  static constexpr int total = xch + kWpc * 8 * kPs;
};

// One sweep for 32 right-hand sides (see launch_sweep).  A CTA takes column
// pair v and kWpc consecutive time steps, one per warp; all warps walk the K
// pair-rows together, and for pair-row i+1 the CTA stages with cp.async
// (two buffers) the record (all three classes), the coupling matrices, and
// per warp its 8 x 32 panel of tau's source (forward) or of y_i (backward)
// and its neighbours' 32 x 32 panels (coupling term).  Every staged row is
// 32 right-hand sides = 8 chunks of 16 bytes, and a lane always copies the
// same chunk of the same component, so its global offsets are fixed up to a
// shift of one grid row (N (T+1) 32 floats) per pair-row and are computed
// once.
template <int VAR>
__global__ void __launch_bounds__(kWpc * 32) mrhs_sweep_kernel(Grid g, Buffers bf, const float* __restrict__ src,
                                                               const float* __restrict__ th_in,
                                                               float* __restrict__ th_out,
                                                               float* __restrict__ rth_out,
                                                               const SolverState* __restrict__ st) {
  if (st != nullptr && st->done) return;
  using Ly = Layout<VAR>;
  constexpr int NW = Ly::NW, NSL = Ly::NSL;
  extern __shared__ __align__(16) float smf[];
  const int Tp = g.T + 1;
  const int tiles = (Tp + kWpc - 1) / kWpc;
  const int v = blockIdx.x / tiles;
  const int t0 = (blockIdx.x % tiles) * kWpc;
  const int j0 = 2 * v;
  const bool two = j0 + 1 < g.N;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int gq = lane >> 2, q = lane & 3;
  const int t = t0 + w;
  const bool active = t <= g.T;
  const int cls = t == 0 ? 2 : (t == g.T ? 1 : 0);
  const long long plane = (long long)g.NN * Tp * kRhs;
  const long long row_step = (long long)g.N * Tp * kRhs;  // one grid row
  const long long node_step = (long long)Tp * kRhs;        // one node
  // this lane's component and chunk in every staged or written row
  const int lk = lane >> 3, lch = lane & 7;
  const long long own0 = (long long)lk * plane + ((long long)j0 * Tp + t) * kRhs + lch * 4;  // pair-row 0, jj = 0

  // neighbour rows staged by this thread: rows hr[x] = tid / 8 + 16 x of
  // every slice (row = 4 h + c for staged node h, component c), chunk
  // tid % 8; node offset from the pair's first node of pair-row 0, and
  // whether the node exists
  const int hch = tid & 7;
  int hr[2];
  long long hoff[2];
  bool hcol[2], hup[2], hdn[2];
  if (NW > 0) {
    const unsigned long long packed = VAR == 2 ? hot::kXiPacked : hot::kOmPacked;
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      hr[x] = (tid >> 3) + 16 * x;
      const int h = hr[x] >> 2, c = hr[x] & 3;
      const unsigned code = (unsigned)((packed >> (5 * h)) & 31ull);
      const int di = (int)(code & 3u) - 1, jn = j0 + (int)(code >> 2) - 2;
      hcol[x] = jn >= 0 && jn < g.N;
      hup[x] = di < 0;
      hdn[x] = di > 0;
      hoff[x] = (long long)c * plane + ((long long)(di * g.N + jn) * Tp) * kRhs + hch * 4;
    }
  }
  // whether this warp's coupling terms exist (warp-uniform): Omega~ is zero
  // at t = 0; Xi~ takes t - 1 for t >= 1 and t + 1 for t < T
  bool tok[2] = {false, false};
  if (VAR == 1) tok[0] = active && t >= 1;
  if (VAR == 2) {
    tok[0] = active && t >= 1;
    tok[1] = active && t < g.T;
  }

  // ---- staging of pair-row i into buffer b (fwd: forward pass)
  auto stage = [&](int i, int b, bool fwd) {
    // records of the three classes, then the coupling matrices
    for (int e = tid; e < 3 * kRec / 4; e += kWpc * 32) {
      const int c = e / (kRec / 4), off = (e % (kRec / 4)) * 4;
      cp16z(smf + Ly::rec + (b * 3 + c) * kRec + off, bf.rec + (((size_t)v * 3 + c) * g.K + i) * kRec + off, true);
    }
    if (fwd && NW > 0) {
      for (int e = tid; e < NW * kW / 4; e += kWpc * 32) {
        const int which = e / (kW / 4), off = (e % (kW / 4)) * 4;
        const float* arr = VAR == 1 ? bf.wom : (which == 0 ? bf.wxa : bf.wxq);
        cp16z(smf + Ly::w + (b * NW + which) * kW + off, arr + ((size_t)v * g.K + i) * kW + off, true);
      }
    }
    // this warp's 8 x 32 panel: tau's source (forward) or y_i (backward)
    const float* pv = fwd ? src : th_out;
    const long long rb = (long long)i * row_step;
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const bool ok = active && (jj == 0 || two);
      cp16z(smf + Ly::src + (b * kWpc + w) * 8 * kPs + pidx(4 * jj + lk, lch * 4),
            pv + (ok ? own0 + rb + jj * node_step : 0), ok);
    }
    if (fwd && NW > 0) {
#pragma unroll
      for (int sl = 0; sl < NSL; ++sl) {
        const int tn = t0 + sl - (VAR == 2 ? 1 : 0);
        const bool t_ok = tn >= 0 && tn <= g.T;
        const long long tb = rb + (long long)tn * kRhs;
#pragma unroll
        for (int x = 0; x < 2; ++x) {
          const bool ok = t_ok && hcol[x] && !(hup[x] && i < 1) && !(hdn[x] && i + 1 >= g.K);
          cp16z(smf + Ly::halo + (b * NSL + sl) * 32 * kPs + pidx(hr[x], hch * 4), th_in + (ok ? hoff[x] + tb : 0),
                ok);
        }
      }
    }
  };

  float* ring = smf + Ly::ring + w * 3 * 8 * kPs;
  float* xch = smf + Ly::xch + w * 8 * kPs;

  // ---- forward substitution
  stage(0, 0, true);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int i = 0; i < g.K; ++i) {
    const int b = i & 1;
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    if (i + 1 < g.K) stage(i + 1, b ^ 1, true);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    if (!active) continue;
    const long long pt0 = ((long long)(i * g.N + j0) * Tp + t) * kRhs;
    const float* P = smf + Ly::src + ((b * kWpc + w) * 8) * kPs;
    float d[2][4];
    d_load(P, 0, gq, q, d[0]);
    d_load(P, 1, gq, q, d[1]);
    if (NW > 0) {
#pragma unroll
      for (int qq = 0; qq < NW; ++qq) {
        if (!tok[qq]) continue;
        const float* H = smf + Ly::halo + (b * NSL + w + 2 * qq) * 32 * kPs;
        const float* W = smf + Ly::w + (b * NW + qq) * kW;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const float2 bw = *reinterpret_cast<const float2*>(W + s * 64 + 2 * lane);
#pragma unroll
          for (int tile = 0; tile < 2; ++tile) {
            unsigned a[4];
            a_frag(H, 8 * s, tile, gq, q, a);
            mma_tf32(d[tile], a, __float_as_uint(bw.x), __float_as_uint(bw.y));
          }
        }
      }
    }
    // tau to the exchange panel, then y = tau - F2 y_{i-2} - F1 y_{i-1}
    // (at t = 0, y = Q tau), z = L0^-1 y
    d_store(xch, 0, gq, q, d[0]);
    d_store(xch, 1, gq, q, d[1]);
    __syncwarp();
    if (VAR == 2) panel_to_global(rth_out, xch, plane, pt0, node_step, two, lane);
    const float* R = smf + Ly::rec + (b * 3 + cls) * kRec;
    float y[2][4];
    if (cls == 2) {
      const float2 bw = *reinterpret_cast<const float2*>(R + 5 * 64 + 2 * lane);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) y[tile][e] = 0.f;
        a_frag(xch, 0, tile, gq, q, a);
        mma_tf32(y[tile], a, __float_as_uint(bw.x), __float_as_uint(bw.y));
      }
    } else {
#pragma unroll
      for (int tile = 0; tile < 2; ++tile)
#pragma unroll
        for (int e = 0; e < 4; ++e) y[tile][e] = d[tile][e];
    }
    if (i >= 2 && cls != 2) {
      const float* Y2 = ring + ((i - 2) % 3) * 8 * kPs;
      const float2 bw = *reinterpret_cast<const float2*>(R + 3 * 64 + 2 * lane);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
        a_frag(Y2, 0, tile, gq, q, a);
        mma_tf32(y[tile], a, __float_as_uint(bw.x), __float_as_uint(bw.y));
      }
    }
    if (i >= 1 && cls != 2) {
      const float* Y1 = ring + ((i - 1) % 3) * 8 * kPs;
      const float2 bw = *reinterpret_cast<const float2*>(R + 4 * 64 + 2 * lane);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
        a_frag(Y1, 0, tile, gq, q, a);
        mma_tf32(y[tile], a, __float_as_uint(bw.x), __float_as_uint(bw.y));
      }
    }
    float* Y0 = ring + (i % 3) * 8 * kPs;
    d_store(Y0, 0, gq, q, y[0]);
    d_store(Y0, 1, gq, q, y[1]);
    __syncwarp();
    if (cls == 2) {
      panel_to_global(th_out, Y0, plane, pt0, node_step, two, lane);
    } else {
      // z = L0^-1 y, the first half of D^-1 = L0^-T L0^-1, is what the
      // backward step reads
      float z[2][4];
      const float2 bw = *reinterpret_cast<const float2*>(R + 5 * 64 + 2 * lane);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) z[tile][e] = 0.f;
        a_frag(Y0, 0, tile, gq, q, a);
        mma_tf32(z[tile], a, __float_as_uint(bw.x), __float_as_uint(bw.y));
      }
      d_store(xch, 0, gq, q, z[0]);
      d_store(xch, 1, gq, q, z[1]);
      __syncwarp();
      panel_to_global(th_out, xch, plane, pt0, node_step, two, lane);
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();

  // ---- backward substitution (t = 0 is final after the forward pass)
  stage(g.K - 1, 0, false);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int i = g.K - 1; i >= 0; --i) {
    const int b = (g.K - 1 - i) & 1;
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    if (i >= 1) stage(i - 1, b ^ 1, false);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    if (!active || cls == 2) continue;
    const long long pt0 = ((long long)(i * g.N + j0) * Tp + t) * kRhs;
    const float* P = smf + Ly::src + ((b * kWpc + w) * 8) * kPs;
    const float* R = smf + Ly::rec + (b * 3 + cls) * kRec;
    float x[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    {
      const float2 bw = *reinterpret_cast<const float2*>(R + 2 * 64 + 2 * lane);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
        a_frag(P, 0, tile, gq, q, a);
        mma_tf32(x[tile], a, __float_as_uint(bw.x), __float_as_uint(bw.y));
      }
    }
    if (i + 2 < g.K) {
      const float* X2 = ring + ((i + 2) % 3) * 8 * kPs;
      const float2 bw = *reinterpret_cast<const float2*>(R + 0 * 64 + 2 * lane);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
        a_frag(X2, 0, tile, gq, q, a);
        mma_tf32(x[tile], a, __float_as_uint(bw.x), __float_as_uint(bw.y));
      }
    }
    if (i + 1 < g.K) {
      const float* X1 = ring + ((i + 1) % 3) * 8 * kPs;
      const float2 bw = *reinterpret_cast<const float2*>(R + 1 * 64 + 2 * lane);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
        a_frag(X1, 0, tile, gq, q, a);
        mma_tf32(x[tile], a, __float_as_uint(bw.x), __float_as_uint(bw.y));
      }
    }
    float* X0 = ring + (i % 3) * 8 * kPs;
    d_store(X0, 0, gq, q, x[0]);
    d_store(X0, 1, gq, q, x[1]);
    __syncwarp();
    panel_to_global(th_out, X0, plane, pt0, node_step, two, lane);
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Records: one CTA of 32 lanes per (v, class, pair-row).  Lane (g, q) stores
// b0 = block[g][q] and b1 = block[g][q+4] of each of the six blocks.
__global__ void mrhs_records_kernel(Grid g, NodeData nd, float* rec) {
  const int idx = blockIdx.x;  // (v * 3 + cls) * K + i
  const int i = idx % g.K, cls = (idx / g.K) % 3, v = idx / (3 * g.K);
  const int lane = threadIdx.x, gq = lane >> 2, q = lane & 3;
  const int j0 = 2 * v;
  const bool two = j0 + 1 < g.N;
  float* out = rec + (size_t)idx * kRec;
  for (int bk = 0; bk < 6; ++bk) {
#pragma unroll
    for (int k2 = 0; k2 < 2; ++k2) {
      const int row = gq, col = q + 4 * k2;
      double val = 0.0;
      if (cls < 2) {
        // source slots of the FP64 record [N2][N1][D^-1][E][F2][F1][L0^-1]:
        // block 2 is L0^-T, the transpose of L0^-1 (the record's D^-1
        // serves the single-RHS sweeps)
        const int slot = bk == 0 ? 0 : bk == 1 ? 1 : bk == 3 ? 4 : bk == 4 ? 5 : 6;
        const double* blk = nd.fac + (size_t)(2 * v + cls) * nd.fac_vc + (size_t)i * nd.fac_rec + slot * 64;
        val = bk == 2 ? blk[col * 8 + row] : blk[row * 8 + col];
        if (bk == 0 || bk == 1 || bk == 3 || bk == 4) val = -val;
      } else if (bk == 2) {
        val = row == col ? 1.0 : 0.0;
      } else if (bk == 5) {
        const int jj = row >> 2;
        if (jj == (col >> 2) && (jj == 0 || two))
          val = nd.Qm[((size_t)(i * g.N + j0 + jj) * kN + (row & 3)) * kN + (col & 3)];
      }
      out[bk * 64 + 2 * lane + k2] = __uint_as_float(tf32_bits((float)val));
    }
  }
}

// Coupling matrices: one CTA of 32 lanes per (v, pair-row).  W[a][(h, c)]
// couples unknown a = jj*4 + k of the pair-row to component c of staged
// neighbour h; lane (g, q) stores, for k-step s, W[g][8s + q] and
// W[g][8s + q + 4].
__global__ void mrhs_coupling_kernel(Grid g, NodeData nd, float* wom, float* wxa, float* wxq) {
  const int idx = blockIdx.x;  // v * K + i
  const int i = idx % g.K, v = idx / g.K;
  const int lane = threadIdx.x, gq = lane >> 2, q = lane & 3;
  const int j0 = 2 * v;
  for (int s = 0; s < 4; ++s) {
#pragma unroll
    for (int k2 = 0; k2 < 2; ++k2) {
      const int row = gq, col = 8 * s + q + 4 * k2;
      const int jj = row >> 2, k = row & 3, h = col >> 2, c = col & 3;
      const int j = j0 + jj;
      double om = 0.0, xa = 0.0, xq = 0.0;
      if (j < g.N) {
        const size_t p = (size_t)i * g.N + j;
        for (int o = 0; o < 5; ++o)
          if (hot::h_of_offpair(jj, o) == h && offpair_node(i, j, o, g.K, g.N) >= 0)
            om = nd.Om[((p * 5 + o) * kN + k) * kN + c];
        for (int dir = 0; dir < 5; ++dir)
          if (hot::h_of_dir(jj, dir) == h && nbr_node(i, j, dir, g.K, g.N) >= 0) {
            xa = nd.AQ[((p * 5 + dir) * kN + k) * kN + c];
            xq = nd.QAt[((p * 5 + dir) * kN + k) * kN + c];
          }
      }
      const size_t o = (size_t)idx * kW + s * 64 + 2 * lane + k2;
      wom[o] = __uint_as_float(tf32_bits((float)om));
      wxa[o] = __uint_as_float(tf32_bits((float)xa));
      wxq[o] = __uint_as_float(tf32_bits((float)xq));
    }
  }
}

// api [nrhs][T+1][NN][n] <-> vector [n][NN][T+1][32] by 32 x 32 tiles
// through shared memory: for one time t, the api slice is a matrix
// [rhs][c] with c = node*n + k, and the vector holds its transpose in rows
// of 32 right-hand sides.  A CTA of 32 x 8 threads moves the tile of
// columns c0 .. c0+31 at time t = blockIdx.y, reading and writing 32
// consecutive elements per warp access on both sides.
template <typename FT, typename TT, bool TO_VEC>
__global__ void transpose_kernel(Grid g, int nrhs, const FT* __restrict__ in, TT* __restrict__ out) {
  __shared__ float tile[32][33];
  const int Tp = g.T + 1;
  const long long C = (long long)g.NN * kN;
  const long long c0 = (long long)blockIdx.x * 32;
  const int t = blockIdx.y;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const long long plane = (long long)g.NN * Tp * kRhs;
  if (TO_VEC) {
    for (int r = ty; r < 32; r += 8) {
      const long long c = c0 + tx;
      float val = 0.f;
      if (r < nrhs && c < C) val = (float)in[((long long)r * Tp + t) * C + c];
      tile[r][tx] = val;
    }
    __syncthreads();
    for (int cc = ty; cc < 32; cc += 8) {
      const long long c = c0 + cc;
      if (c >= C) continue;
      const long long p = c / kN, k = c % kN;
      out[k * plane + (p * Tp + t) * kRhs + tx] = (TT)tile[tx][cc];
    }
  } else {
    for (int cc = ty; cc < 32; cc += 8) {
      const long long c = c0 + cc;
      if (c >= C) continue;
      const long long p = c / kN, k = c % kN;
      tile[tx][cc] = (float)in[k * plane + (p * Tp + t) * kRhs + tx];
    }
    __syncthreads();
    for (int r = ty; r < nrhs; r += 8) {
      const long long c = c0 + tx;
      if (c < C) out[((long long)r * Tp + t) * C + c] = (TT)tile[r][tx];
    }
  }
}

template <int VAR>
size_t smem_bytes() {
  return (size_t)Layout<VAR>::total * sizeof(float);
}

}  // namespace

long long rec_floats(const Grid& g) { return (long long)g.V * 3 * g.K * kRec; }
long long w_floats(const Grid& g) { return (long long)g.V * g.K * kW; }
long long vec_floats(const Grid& g) { return (long long)kN * g.NN * (g.T + 1) * kRhs; }

void launch_build(const Grid& g, const NodeData& nd, const Buffers& b, cudaStream_t s) {
  mrhs_records_kernel<<<g.V * 3 * g.K, 32, 0, s>>>(g, nd, b.rec);
  mrhs_coupling_kernel<<<g.V * g.K, 32, 0, s>>>(g, nd, b.wom, b.wxa, b.wxq);
}

void launch_from_api(const Grid& g, int nrhs, const double* api, float* vec, cudaStream_t s) {
  const dim3 grid((unsigned)(((long long)g.NN * kN + 31) / 32), (unsigned)(g.T + 1));
  transpose_kernel<double, float, true><<<grid, dim3(32, 8), 0, s>>>(g, nrhs, api, vec);
}

void launch_to_api(const Grid& g, int nrhs, const float* vec, double* api, cudaStream_t s) {
  const dim3 grid((unsigned)(((long long)g.NN * kN + 31) / 32), (unsigned)(g.T + 1));
  transpose_kernel<float, double, false><<<grid, dim3(32, 8), 0, s>>>(g, nrhs, vec, api);
}

void launch_sweep(int variant, const Grid& g, const Buffers& b, const float* src, const float* theta_in,
                  float* theta_out, float* rth_out, const SolverState* st, cudaStream_t s) {
  const unsigned blocks = (unsigned)((long long)g.V * ((g.T + 1 + kWpc - 1) / kWpc));
  switch (variant) {
    case 0:
      mrhs_sweep_kernel<0><<<blocks, kWpc * 32, smem_bytes<0>(), s>>>(g, b, src, theta_in, theta_out, rth_out, st);
      break;
    case 1:
      mrhs_sweep_kernel<1><<<blocks, kWpc * 32, smem_bytes<1>(), s>>>(g, b, src, theta_in, theta_out, rth_out, st);
      break;
    default:
      mrhs_sweep_kernel<2><<<blocks, kWpc * 32, smem_bytes<2>(), s>>>(g, b, src, theta_in, theta_out, rth_out, st);
      break;
  }
}

cudaError_t prepare() {
  cudaError_t e = cudaFuncSetAttribute((const void*)mrhs_sweep_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes<0>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)mrhs_sweep_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<1>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)mrhs_sweep_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<2>());
  return e;
}

}  // namespace mrhs
}  // namespace lq2d
