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
// The factor record of a pair-row holds six blocks (forward and backward
// substitution with the pivots pre-multiplied, as in the single-RHS sweep):
//   0: -N2  1: -N1  2: L0^-T  (backward: x_i = L0^-T y_i - N2 x_{i+2} - N1 x_{i+1})
//   3: -M2  4: -M1  5: L0^-1  (forward:  y_i = L0^-1 tau_i - M2 y_{i-2} - M1 y_{i-1})
// each stored as B fragments, lane-major: element 2*lane + k of a block is
// b_k of that lane.  Class 2 is t = 0, where Phi_bar = Q^-1 node by node:
// its forward block 5 is blkdiag(Q, Q) of the pair's two nodes and the
// other forward blocks are zero (the backward pass is skipped at t = 0).
#include "mrhs.h"
#include "sweep_tiled.cuh"

namespace lq2d {
namespace mrhs {

namespace {

constexpr int kWpc = 4;                  // warps (time steps) per CTA
constexpr int kNb = 2;                   // staging buffers
constexpr int kPs = 40;                  // row stride (floats) of the [rows][32 rhs] panels
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

// A fragment (16 rhs x 8 columns) of right-hand-side tile `tile` from a
// panel P[col][rhs] (row stride kPs), with columns c0 .. c0+7.
__device__ __forceinline__ void a_frag(const float* P, int c0, int tile, int g, int q, unsigned (&a)[4]) {
  const int m = g + 16 * tile;
  a[0] = tf32_bits(P[(c0 + q) * kPs + m]);
  a[1] = tf32_bits(P[(c0 + q) * kPs + m + 8]);
  a[2] = tf32_bits(P[(c0 + q + 4) * kPs + m]);
  a[3] = tf32_bits(P[(c0 + q + 4) * kPs + m + 8]);
}

// D fragment of tile `tile` to / from a panel P[row][rhs].
__device__ __forceinline__ void d_store(float* P, int tile, int g, int q, const float (&d)[4]) {
  const int m = g + 16 * tile;
  P[(2 * q) * kPs + m] = d[0];
  P[(2 * q + 1) * kPs + m] = d[1];
  P[(2 * q) * kPs + m + 8] = d[2];
  P[(2 * q + 1) * kPs + m + 8] = d[3];
}
__device__ __forceinline__ void d_load(const float* P, int tile, int g, int q, float (&d)[4]) {
  const int m = g + 16 * tile;
  d[0] = P[(2 * q) * kPs + m];
  d[1] = P[(2 * q + 1) * kPs + m];
  d[2] = P[(2 * q) * kPs + m + 8];
  d[3] = P[(2 * q + 1) * kPs + m + 8];
}

// Writes a D fragment of tile `tile` (rows = pair-row unknowns a = jj*4 + k,
// columns = right-hand sides) to a vector at pair-row i, time t.
__device__ __forceinline__ void d_to_global(float* vec, const Grid& g, long long plane, int i, int j0, bool two,
                                            int t, int tile, int gq, int q, const float (&d)[4]) {
  const int Tp = g.T + 1;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int row = 2 * q + (e & 1);
    const int m = gq + 8 * (e >> 1) + 16 * tile;
    const int jj = row >> 2, k = row & 3;
    if (jj == 1 && !two) continue;
    vec[k * plane + ((long long)(i * g.N + j0 + jj) * Tp + t) * kRhs + m] = d[e];
  }
}

template <int NW>
struct Layout {
  // offsets in floats of the dynamic shared memory
  static constexpr int rec = 0;                               // [kNb][3][kRec]
  static constexpr int w = rec + kNb * 3 * kRec;              // [kNb][NW][kW]
  static constexpr int src = w + kNb * NW * kW;               // [kNb][kWpc][8][kPs]
  static constexpr int halo = src + kNb * kWpc * 8 * kPs;     // [kNb][kWpc][NW][32][kPs]
  static constexpr int ring = halo + kNb * kWpc * NW * 32 * kPs;  // [kWpc][3][8][kPs]
  static constexpr int xch = ring + kWpc * 3 * 8 * kPs;       // [kWpc][8][kPs]
  static constexpr int total = xch + kWpc * 8 * kPs;
};

// One sweep for 32 right-hand sides (see launch_sweep).  A CTA takes column
// pair v and kWpc consecutive time steps, one per warp; all warps walk the K
// pair-rows together, and for pair-row i+1 the CTA stages with cp.async
// (two buffers) the record (all three classes), the coupling matrices, and
// per warp its 8 x 32 panel of tau's source (forward) or of y_i (backward)
// and its neighbours' 32 x 32 panels (coupling term).
template <int VAR>
__global__ void __launch_bounds__(kWpc * 32) mrhs_sweep_kernel(Grid g, Buffers bf, const float* __restrict__ src,
                                                               const float* __restrict__ th_in,
                                                               float* __restrict__ th_out,
                                                               float* __restrict__ rth_out) {
  constexpr int NW = VAR == 0 ? 0 : (VAR == 1 ? 1 : 2);
  using Ly = Layout<NW>;
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
  const bool xi = VAR == 2;

  // ---- staging of pair-row i into buffer b (fwd: forward pass)
  auto stage = [&](int i, int b, bool fwd) {
    // records of the three classes
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
    for (int e = lane; e < 64; e += 32) {
      const int a = e >> 3, ch = e & 7;
      const int jj = a >> 2, k = a & 3;
      const bool ok = active && (jj == 0 || two);
      const long long go = ok ? k * plane + ((long long)(i * g.N + j0 + jj) * Tp + t) * kRhs + ch * 4 : 0;
      cp16z(smf + Ly::src + ((b * kWpc + w) * 8 + a) * kPs + ch * 4, pv + go, ok);
    }
    if (fwd && NW > 0) {
      // neighbour panels: rows (h, c) of the eight staged nodes
#pragma unroll
      for (int qq = 0; qq < NW; ++qq) {
        const int tn = VAR == 1 ? t : (qq == 0 ? t - 1 : t + 1);
        const bool t_ok = active && tn >= 0 && tn <= g.T && (VAR != 1 || t >= 1);
        for (int e = lane; e < 256; e += 32) {
          const int row = e >> 3, ch = e & 7;
          const int h = row >> 2, c = row & 3;
          const int node = hot::staged_node(xi, h, i, j0, g.K, g.N);
          const bool ok = t_ok && node >= 0;
          const long long go = ok ? c * plane + ((long long)node * Tp + tn) * kRhs + ch * 4 : 0;
          cp16z(smf + Ly::halo + (((b * kWpc + w) * NW + qq) * 32 + row) * kPs + ch * 4, th_in + go, ok);
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
    const float* P = smf + Ly::src + ((b * kWpc + w) * 8) * kPs;
    float d[2][4];
    d_load(P, 0, gq, q, d[0]);
    d_load(P, 1, gq, q, d[1]);
    if (NW > 0) {
#pragma unroll
      for (int qq = 0; qq < NW; ++qq) {
        const bool use = VAR == 1 ? t >= 1 : (qq == 0 ? t >= 1 : t < g.T);
        if (!use) continue;
        const float* H = smf + Ly::halo + ((b * kWpc + w) * NW + qq) * 32 * kPs;
        const float* W = smf + Ly::w + (b * NW + qq) * kW;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const unsigned b0 = __float_as_uint(W[s * 64 + 2 * lane]);
          const unsigned b1 = __float_as_uint(W[s * 64 + 2 * lane + 1]);
#pragma unroll
          for (int tile = 0; tile < 2; ++tile) {
            unsigned a[4];
            a_frag(H, 8 * s, tile, gq, q, a);
            mma_tf32(d[tile], a, b0, b1);
          }
        }
      }
      if (VAR == 2) {
        d_to_global(rth_out, g, plane, i, j0, two, t, 0, gq, q, d[0]);
        d_to_global(rth_out, g, plane, i, j0, two, t, 1, gq, q, d[1]);
      }
    }
    // tau to the exchange panel, then y = L0^-1 tau - M2 y_{i-2} - M1 y_{i-1}
    d_store(xch, 0, gq, q, d[0]);
    d_store(xch, 1, gq, q, d[1]);
    __syncwarp();
    const float* R = smf + Ly::rec + (b * 3 + cls) * kRec;
    float y[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    {
      const unsigned b0 = __float_as_uint(R[5 * 64 + 2 * lane]), b1 = __float_as_uint(R[5 * 64 + 2 * lane + 1]);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
        a_frag(xch, 0, tile, gq, q, a);
        mma_tf32(y[tile], a, b0, b1);
      }
    }
    if (i >= 2 && cls != 2) {
      const float* Y2 = ring + ((i - 2) % 3) * 8 * kPs;
      const unsigned b0 = __float_as_uint(R[3 * 64 + 2 * lane]), b1 = __float_as_uint(R[3 * 64 + 2 * lane + 1]);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
        a_frag(Y2, 0, tile, gq, q, a);
        mma_tf32(y[tile], a, b0, b1);
      }
    }
    if (i >= 1 && cls != 2) {
      const float* Y1 = ring + ((i - 1) % 3) * 8 * kPs;
      const unsigned b0 = __float_as_uint(R[4 * 64 + 2 * lane]), b1 = __float_as_uint(R[4 * 64 + 2 * lane + 1]);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
        a_frag(Y1, 0, tile, gq, q, a);
        mma_tf32(y[tile], a, b0, b1);
      }
    }
    float* Y0 = ring + (i % 3) * 8 * kPs;
    d_store(Y0, 0, gq, q, y[0]);
    d_store(Y0, 1, gq, q, y[1]);
    d_to_global(th_out, g, plane, i, j0, two, t, 0, gq, q, y[0]);
    d_to_global(th_out, g, plane, i, j0, two, t, 1, gq, q, y[1]);
    __syncwarp();
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
    const float* P = smf + Ly::src + ((b * kWpc + w) * 8) * kPs;
    const float* R = smf + Ly::rec + (b * 3 + cls) * kRec;
    float x[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    {
      const unsigned b0 = __float_as_uint(R[2 * 64 + 2 * lane]), b1 = __float_as_uint(R[2 * 64 + 2 * lane + 1]);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
        a_frag(P, 0, tile, gq, q, a);
        mma_tf32(x[tile], a, b0, b1);
      }
    }
    if (i + 2 < g.K) {
      const float* X2 = ring + ((i + 2) % 3) * 8 * kPs;
      const unsigned b0 = __float_as_uint(R[0 * 64 + 2 * lane]), b1 = __float_as_uint(R[0 * 64 + 2 * lane + 1]);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
        a_frag(X2, 0, tile, gq, q, a);
        mma_tf32(x[tile], a, b0, b1);
      }
    }
    if (i + 1 < g.K) {
      const float* X1 = ring + ((i + 1) % 3) * 8 * kPs;
      const unsigned b0 = __float_as_uint(R[1 * 64 + 2 * lane]), b1 = __float_as_uint(R[1 * 64 + 2 * lane + 1]);
#pragma unroll
      for (int tile = 0; tile < 2; ++tile) {
        unsigned a[4];
        a_frag(X1, 0, tile, gq, q, a);
        mma_tf32(x[tile], a, b0, b1);
      }
    }
    float* X0 = ring + (i % 3) * 8 * kPs;
    d_store(X0, 0, gq, q, x[0]);
    d_store(X0, 1, gq, q, x[1]);
    d_to_global(th_out, g, plane, i, j0, two, t, 0, gq, q, x[0]);
    d_to_global(th_out, g, plane, i, j0, two, t, 1, gq, q, x[1]);
    __syncwarp();
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
        const double* blk = nd.fac + (size_t)(2 * v + cls) * nd.fac_vc + (size_t)i * nd.fac_rec + bk * 64;
        val = blk[row * 8 + col];
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

// api [nrhs][T+1][NN][n] <-> vector [n][NN][T+1][32], one thread per vector element.
__global__ void from_api_kernel(Grid g, int nrhs, const double* __restrict__ api, float* __restrict__ vec) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int Tp = g.T + 1;
  const long long total = (long long)kN * g.NN * Tp * kRhs;
  if (e >= total) return;
  const int r = (int)(e % kRhs);
  const long long pt = (e / kRhs) % ((long long)g.NN * Tp);
  const int k = (int)(e / ((long long)kRhs * g.NN * Tp));
  const int p = (int)(pt / Tp), t = (int)(pt % Tp);
  vec[e] = r < nrhs ? (float)api[(((long long)r * Tp + t) * g.NN + p) * kN + k] : 0.f;
}

__global__ void to_api_kernel(Grid g, int nrhs, const float* __restrict__ vec, double* __restrict__ api) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int Tp = g.T + 1;
  const long long total = (long long)kN * g.NN * Tp * kRhs;
  if (e >= total) return;
  const int r = (int)(e % kRhs);
  if (r >= nrhs) return;
  const long long pt = (e / kRhs) % ((long long)g.NN * Tp);
  const int k = (int)(e / ((long long)kRhs * g.NN * Tp));
  const int p = (int)(pt / Tp), t = (int)(pt % Tp);
  api[(((long long)r * Tp + t) * g.NN + p) * kN + k] = (double)vec[e];
}

template <int VAR>
size_t smem_bytes() {
  return (size_t)Layout<VAR == 0 ? 0 : (VAR == 1 ? 1 : 2)>::total * sizeof(float);
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
  const long long total = vec_floats(g);
  from_api_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g, nrhs, api, vec);
}

void launch_to_api(const Grid& g, int nrhs, const float* vec, double* api, cudaStream_t s) {
  const long long total = vec_floats(g);
  to_api_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(g, nrhs, vec, api);
}

void launch_sweep(int variant, const Grid& g, const Buffers& b, const float* src, const float* theta_in,
                  float* theta_out, float* rth_out, cudaStream_t s) {
  const unsigned blocks = (unsigned)((long long)g.V * ((g.T + 1 + kWpc - 1) / kWpc));
  switch (variant) {
    case 0: mrhs_sweep_kernel<0><<<blocks, kWpc * 32, smem_bytes<0>(), s>>>(g, b, src, theta_in, theta_out, rth_out); break;
    case 1: mrhs_sweep_kernel<1><<<blocks, kWpc * 32, smem_bytes<1>(), s>>>(g, b, src, theta_in, theta_out, rth_out); break;
    default: mrhs_sweep_kernel<2><<<blocks, kWpc * 32, smem_bytes<2>(), s>>>(g, b, src, theta_in, theta_out, rth_out); break;
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
