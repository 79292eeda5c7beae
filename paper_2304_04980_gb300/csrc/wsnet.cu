// Learned warm start: the convolutional network that proposes the initial
// PCG iterate delta^(0) (Algorithm 1 accepts any; the paper starts from
// zero), with its forward pass, backward pass and Adam update as CUDA
// kernels.
//
// Every 3x3 convolution (zero padding, stride 1) and its two gradients run
// as one implicit-GEMM kernel on FP32 CUDA cores, with the operands gathered
// from the NCHW activations while they are staged in shared memory:
//
//   forward       Y[o][q]      = sum_{(c,tap)} W[o][c][tap] X[c][q + tap]          M=Cout N=pixels K=Cin*9
//   input grad    GX[c][q]     = sum_{(o,tap)} W[o][c][tap] GY[o][q - tap]         M=Cin  N=pixels K=Cout*9
//   weight grad   GW[o][(c,tap)] = sum_q GY[o][q] X[c][q + tap]                    M=Cout N=Cin*9+1 K=pixels
//
// q runs over the pixels of all instances of the batch, tap = (di, dj) with
// offset (di-1, dj-1), and X is zero outside the grid.  The weight gradient
// gets one extra column of ones, whose result is the bias gradient, and is
// split over the pixels (partial sums per split, added in a fixed order by
// a second kernel, so that the result does not depend on scheduling).
// Weights are read as bfloat16 (the copy refreshed after every Adam step);
// products and sums are FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lq2d.h"
#include "../../include/lq2d_warmstart.h"
#include "common.cuh"

namespace lq2d {
void set_last_error(const std::string& msg);  // lq2d.cu: the message lq2d_last_error() returns

namespace wsnet {

enum ConvMode { kFwd = 0, kBwdData = 1, kBwdWeight = 2 };

constexpr int BM = 64, BN = 64, BK = 16, CT = 256;  // tile and threads of the GEMM kernel

struct ConvArgs {
  int B, H, W, Cin, Cout;
  const __nv_bfloat16* w;  // [Cout][Cin][9]
  const float* bias;       // [Cout] (forward)
  const float* x;          // layer input [B][Cin][H][W] (forward, weight grad)
  const float* gy;         // gradient of the layer output [B][Cout][H][W] (input grad, weight grad)
  const float* gate;       // input grad: the layer input, whose sign gates the previous ReLU (or null)
  float* out;              // forward [B][Cout][H][W]; input grad [B][Cin][H][W]; weight grad partials
  int relu;                // forward: ReLU on the output
  int k_split;             // weight grad: pixels per split (multiple of BK)
};

// Operand gathering.  Element e = tid + 256 r (r = 0..3) of a 64 x 16 A
// tile is (m = e / 16, k = e % 16) and of a 16 x 64 B tile is
// (k = e / 64, n = e % 64), except the weight grad's B tile, which runs
// along k: (k = e % 16, n = e / 16).  In every mode a thread's four
// elements share one pixel (forward and input grad: its column n; weight
// grad: its k), so the pixel is decoded once per K slice and the channel /
// tap indices advance by 16 per slice without divisions.

// (c, tap) of k + 16 from (c, tap) of k, tap in 0..8
__device__ __forceinline__ void advance16(int& c, int& tap) {
  tap += 7;
  c += 1;
  if (tap >= 9) { tap -= 9; c += 1; }
}
__device__ __forceinline__ int tap_row(int tap) { return (tap * 11) >> 5; }  // tap / 3 for 0 <= tap <= 8

// C[M][N] = A[M][K] B[K][N] on a BM x BN tile per CTA, 4 x 4 outputs per
// thread, the next K slice prefetched into registers while the current one
// is multiplied.  blockIdx.z is the split of K (weight grad only).
template <int MODE>
__global__ void __launch_bounds__(CT) conv_gemm_kernel(ConvArgs a, int M, int N, int K) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int HW = a.H * a.W;
  int k_begin = 0, k_end = K;
  if (MODE == kBwdWeight) {
    k_begin = blockIdx.z * a.k_split;
    k_end = min(K, k_begin + a.k_split);
  }
  const int tm = (tid / 16) * 4, tn = (tid % 16) * 4;
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;

  // per-thread gather state
  const int kl_a = tid % BK;              // k of the A elements (all modes)
  const int ml_a = tid / BK;              // + 16 r: m of the A elements
  int pb = 0, pi = 0, pj = 0;             // pixel (batch, row, column) of the thread's B column / k
  bool pix_ok = false;
  int cb[4], tb[4];                       // forward / input grad: (channel, tap) of the four B rows
  int ca = 0, ta = 0;                     // input grad: (output channel, tap) of the A column
  int wc[4], wt[4];                       // weight grad: (channel, tap) of the four B columns
  if (MODE != kBwdWeight) {
    const int n = n0 + tid % BN;
    pix_ok = n < N;
    pb = pix_ok ? n / HW : 0;
    const int pix = pix_ok ? n - pb * HW : 0;
    pi = pix / a.W;
    pj = pix - pi * a.W;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int k = k_begin + tid / BN + 4 * r;
      cb[r] = k / 9;
      tb[r] = k - 9 * cb[r];
    }
    if (MODE == kBwdData) {
      const int k = k_begin + kl_a;
      ca = k / 9;
      ta = k - 9 * ca;
    }
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int n = n0 + tid / BK + 16 * r;
      wc[r] = n / 9;
      wt[r] = n - 9 * wc[r];
    }
  }

  float ra[4], rb[4];
  auto fetch = [&](int k0) {
    if (MODE == kFwd) {
      const int k = k0 + kl_a;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + ml_a + 16 * r;
        ra[r] = (m < M && k < K) ? __bfloat162float(a.w[(size_t)m * K + k]) : 0.f;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float v = 0.f;
        const int k = k0 + tid / BN + 4 * r;
        if (pix_ok && k < K) {
          const int di = tap_row(tb[r]);
          const int ii = pi + di - 1, jj = pj + tb[r] - 3 * di - 1;
          if (ii >= 0 && ii < a.H && jj >= 0 && jj < a.W)
            v = a.x[((size_t)pb * a.Cin + cb[r]) * HW + ii * a.W + jj];
        }
        rb[r] = v;
      }
    } else if (MODE == kBwdData) {
      const int k = k0 + kl_a;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + ml_a + 16 * r;
        ra[r] = (m < M && k < K) ? __bfloat162float(a.w[((size_t)ca * a.Cin + m) * 9 + ta]) : 0.f;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float v = 0.f;
        const int k = k0 + tid / BN + 4 * r;
        if (pix_ok && k < K) {
          const int di = tap_row(tb[r]);
          const int ii = pi - di + 1, jj = pj - (tb[r] - 3 * di) + 1;
          if (ii >= 0 && ii < a.H && jj >= 0 && jj < a.W)
            v = a.gy[((size_t)pb * a.Cout + cb[r]) * HW + ii * a.W + jj];
        }
        rb[r] = v;
      }
    } else {
      // weight grad: the thread's pixel is k = k0 + kl_a, for A and B alike
      const int q = k0 + kl_a;
      const bool ok = q < k_end;
      const int b = ok ? q / HW : 0;
      const int pix = ok ? q - b * HW : 0;
      const int i = pix / a.W, j = pix - (pix / a.W) * a.W;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + ml_a + 16 * r;
        ra[r] = (ok && m < M) ? a.gy[((size_t)b * a.Cout + m) * HW + pix] : 0.f;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int n = n0 + tid / BK + 16 * r;
        float v = 0.f;
        if (ok && n < N) {
          if (n == a.Cin * 9) {
            v = 1.f;
          } else {
            const int di = tap_row(wt[r]);
            const int ii = i + di - 1, jj = j + wt[r] - 3 * di - 1;
            if (ii >= 0 && ii < a.H && jj >= 0 && jj < a.W)
              v = a.x[((size_t)b * a.Cin + wc[r]) * HW + ii * a.W + jj];
          }
        }
        rb[r] = v;
      }
    }
  };
  auto advance = [&]() {
    if (MODE != kBwdWeight) {
#pragma unroll
      for (int r = 0; r < 4; ++r) advance16(cb[r], tb[r]);
      if (MODE == kBwdData) advance16(ca, ta);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + CT * r;
      As[buf][e % BK][e / BK] = ra[r];
      if (MODE == kBwdWeight) Bs[buf][e % BK][e / BK] = rb[r];
      else Bs[buf][e / BN][e % BN] = rb[r];
    }
  };

  int buf = 0;
  fetch(k_begin);
  advance();
  store(0);
  __syncthreads();
  for (int k0 = k_begin; k0 < k_end; k0 += BK) {
    const bool more = k0 + BK < k_end;
    if (more) {
      fetch(k0 + BK);
      advance();
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 av = *reinterpret_cast<const float4*>(&As[buf][kk][tm]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[buf][kk][tn]);
      const float am[4] = {av.x, av.y, av.z, av.w};
      const float bn[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(am[r], bn[c], acc[r][c]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int m = m0 + tm + r;
    if (m >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int n = n0 + tn + c;
      if (n >= N) continue;
      if (MODE == kBwdWeight) {
        a.out[((size_t)blockIdx.z * M + m) * N + n] = acc[r][c];
      } else {
        const int b = n / HW, pix = n - b * HW;
        const size_t idx = ((size_t)b * M + m) * HW + pix;
        float v = acc[r][c];
        if (MODE == kFwd) {
          v += a.bias[m];
          if (a.relu) v = fmaxf(v, 0.f);
        } else if (a.gate != nullptr && !(a.gate[idx] > 0.f)) {
          v = 0.f;
        }
        a.out[idx] = v;
      }
    }
  }
}

// grads[off_w + o*Cin*9 + n] (n < Cin*9) and grads[off_b + o] (n = Cin*9):
// the sum over the splits of the weight-grad partials, in split order.
__global__ void reduce_wgrad_kernel(const float* part, int splits, int M, int N, float* gw, float* gb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += part[(size_t)z * M * N + e];
  const int o = e / N, nn = e - o * N;
  if (nn == N - 1) gb[o] = s;
  else gw[(size_t)o * (N - 1) + nn] = s;
}

// Network input: X[b][c][pix] = x0[b][pix][c] for c < n, coupling[b] for c = n.
__global__ void features_kernel(const double* x0, const double* coupling, int B, int HW, int n, float* X) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)B * (n + 1) * HW;
  if (e >= total) return;
  const int pix = (int)(e % HW);
  const int c = (int)((e / HW) % (n + 1));
  const int b = (int)(e / ((long long)HW * (n + 1)));
  X[e] = c < n ? (float)x0[((long long)b * HW + pix) * n + c] : (float)coupling[b];
}

// delta0[b][t][pix][k] = sigma * yhat[b][t*n + k][pix].
__global__ void output_kernel(const float* yhat, int B, int Tp, int HW, int n, double sigma, double* delta0) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)B * Tp * HW * n;
  if (e >= total) return;
  const int k = (int)(e % n);
  const int pix = (int)((e / n) % HW);
  const long long bt = e / ((long long)n * HW);  // b * Tp + t
  const int t = (int)(bt % Tp);
  const int b = (int)(bt / Tp);
  delta0[e] = sigma * (double)yhat[((long long)b * Tp * n + (long long)t * n + k) * HW + pix];
}

// Mean squared error against target/sigma and its gradient
// gy = 2 (yhat - target/sigma) / count, with the loss summed in FP64 by a
// deterministic two-stage reduction.
__global__ void loss_kernel(const float* yhat, const double* target, int B, int Tp, int HW, int n, double sigma,
                            float* gy, double* partials, unsigned int* counter, double* loss_out) {
  const long long total = (long long)B * Tp * n * HW;
  const double inv = 1.0 / sigma, scale = 2.0 / (double)total;
  double acc = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    // e indexes yhat [b][o][pix] with o = t*n + k
    const int pix = (int)(e % HW);
    const long long bo = e / HW;
    const int o = (int)(bo % ((long long)Tp * n));
    const int b = (int)(bo / ((long long)Tp * n));
    const int t = o / n, k = o - t * n;
    const double d = (double)yhat[e] - target[(((long long)b * Tp + t) * HW + pix) * n + k] * inv;
    gy[e] = (float)(scale * d);
    acc += d * d;
  }
  double tot0, tot1;
  if (grid_reduce2<false>(acc, 0.0, partials, counter, &tot0, &tot1)) *loss_out = tot0 / (double)total;
}

// Adam with bias corrections c1 = 1/(1 - beta1^t), c2 = 1/(1 - beta2^t);
// also refreshes the bfloat16 copy used by the passes.
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, __nv_bfloat16* pbf, long long count,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.f - b1) * gi;
  const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  const float pi = p[e] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  p[e] = pi;
  pbf[e] = __float2bfloat16_rn(pi);
}

__global__ void to_bf16_kernel(const float* p, __nv_bfloat16* pbf, long long count) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) pbf[e] = __float2bfloat16_rn(p[e]);
}

inline unsigned blocks_for(long long count, int threads) { return (unsigned)((count + threads - 1) / threads); }

template <int MODE>
void launch_conv(const ConvArgs& a, int M, int N, int K, int splits, cudaStream_t s) {
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)splits);
  conv_gemm_kernel<MODE><<<grid, CT, 0, s>>>(a, M, N, K);
}

}  // namespace wsnet
}  // namespace lq2d

using namespace lq2d::wsnet;

struct lq2d_wsnet {
  int K = 0, N = 0, T = 0, n = 0, C = 0, L = 0, maxB = 0;
  double sigma = 1.0;
  std::vector<int> cin, cout;
  std::vector<long long> off_w, off_b;
  long long P = 0;
  float* params = nullptr;
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* wbf = nullptr;
  std::vector<float*> act;  // act[0] network input, act[l + 1] output of layer l
  float* gbuf[2] = {nullptr, nullptr};
  float* wpart = nullptr;
  long long wpart_count = 0;
  double* partials = nullptr;
  unsigned int* counter = nullptr;
  double* loss_dev = nullptr;
  double* coupling_dev = nullptr;
  double* h_loss = nullptr;
  int step = 0;
  std::vector<void*> allocs;
};

namespace {

int ws_fail(int code, const std::string& msg) {
  lq2d::set_last_error(msg);
  return code;
}

#define WS_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return ws_fail(LQ2D_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int ws_alloc(lq2d_wsnet* net, T** p, size_t count) {
  void* ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, count * sizeof(T) + 256);
  if (e != cudaSuccess) return ws_fail(LQ2D_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  net->allocs.push_back(ptr);
  *p = static_cast<T*>(ptr);
  return LQ2D_OK;
}

constexpr int kPartialBlocks = 1024;  // blocks of the loss reduction

// Splits of the weight-grad reduction: enough CTAs for every SM a few times.
int wgrad_splits(int M, int N, int K, int* k_split) {
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  int splits = (4 * 152 + tiles - 1) / tiles;
  const int max_splits = (K + BK - 1) / BK;
  if (splits > max_splits) splits = max_splits;
  if (splits < 1) splits = 1;
  int ks = (K + splits - 1) / splits;
  ks = (ks + BK - 1) / BK * BK;
  *k_split = ks;
  return (K + ks - 1) / ks;
}

int check_batch(const lq2d_wsnet* net, int batch, const void* a, const void* b) {
  if (!net) return ws_fail(LQ2D_EINVAL, "network is NULL");
  if (batch < 1 || batch > net->maxB) return ws_fail(LQ2D_EINVAL, "batch must be in 1..max_batch");
  if (!a || !b) return ws_fail(LQ2D_EINVAL, "null argument");
  return LQ2D_OK;
}

// Forward pass of `batch` instances into net->act.
int run_forward(lq2d_wsnet* net, int batch, const double* d_x0, const double* coupling, cudaStream_t s) {
  const int HW = net->K * net->N;
  WS_CUDA(cudaMemcpyAsync(net->coupling_dev, coupling, batch * sizeof(double), cudaMemcpyHostToDevice, s));
  const long long fin = (long long)batch * (net->n + 1) * HW;
  features_kernel<<<blocks_for(fin, 256), 256, 0, s>>>(d_x0, net->coupling_dev, batch, HW, net->n, net->act[0]);
  for (int l = 0; l < net->L; ++l) {
    ConvArgs a{};
    a.B = batch; a.H = net->K; a.W = net->N; a.Cin = net->cin[l]; a.Cout = net->cout[l];
    a.w = net->wbf + net->off_w[l];
    a.bias = net->params + net->off_b[l];
    a.x = net->act[l];
    a.out = net->act[l + 1];
    a.relu = l + 1 < net->L;
    launch_conv<kFwd>(a, a.Cout, batch * HW, a.Cin * 9, 1, s);
  }
  WS_CUDA(cudaGetLastError());
  return LQ2D_OK;
}

// Loss and gradient into net->grads (device); the loss into *loss.
int run_loss_grad(lq2d_wsnet* net, int batch, const double* d_x0, const double* coupling, const double* d_target,
                  double* loss, cudaStream_t s) {
  int rc = run_forward(net, batch, d_x0, coupling, s);
  if (rc) return rc;
  const int HW = net->K * net->N, Tp = net->T + 1;
  float* gy = net->gbuf[0];
  float* gx = net->gbuf[1];
  loss_kernel<<<kPartialBlocks, 256, 0, s>>>(net->act[net->L], d_target, batch, Tp, HW, net->n, net->sigma, gy,
                                             net->partials, net->counter, net->loss_dev);
  for (int l = net->L - 1; l >= 0; --l) {
    ConvArgs a{};
    a.B = batch; a.H = net->K; a.W = net->N; a.Cin = net->cin[l]; a.Cout = net->cout[l];
    a.w = net->wbf + net->off_w[l];
    a.x = net->act[l];
    a.gy = gy;
    const int Mw = a.Cout, Nw = a.Cin * 9 + 1, Kw = batch * HW;
    int ks = 0;
    const int splits = wgrad_splits(Mw, Nw, Kw, &ks);
    a.k_split = ks;
    a.out = net->wpart;
    launch_conv<kBwdWeight>(a, Mw, Nw, Kw, splits, s);
    reduce_wgrad_kernel<<<blocks_for((long long)Mw * Nw, 256), 256, 0, s>>>(
        net->wpart, splits, Mw, Nw, net->grads + net->off_w[l], net->grads + net->off_b[l]);
    if (l > 0) {
      ConvArgs d = a;
      d.gate = net->act[l];  // input of layer l = relu output of layer l - 1
      d.out = gx;
      launch_conv<kBwdData>(d, a.Cin, batch * HW, a.Cout * 9, 1, s);
      float* t = gy;
      gy = gx;
      gx = t;
    }
  }
  WS_CUDA(cudaGetLastError());
  WS_CUDA(cudaMemcpyAsync(net->h_loss, net->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  WS_CUDA(cudaStreamSynchronize(s));
  if (loss) *loss = *net->h_loss;
  return LQ2D_OK;
}

}  // namespace

extern "C" {

int lq2d_wsnet_create(lq2d_wsnet** out, int K, int N, int T, int n, int channels, int layers, int max_batch,
                      double sigma) {
  if (!out) return ws_fail(LQ2D_EINVAL, "out is NULL");
  *out = nullptr;
  if (K < 1 || N < 1 || T < 1 || n < 1 || n > 8) return ws_fail(LQ2D_EINVAL, "K, N, T >= 1 and 1 <= n <= 8 required");
  if (channels < 1 || channels > 256 || layers < 1 || layers > 64)
    return ws_fail(LQ2D_EINVAL, "channels in 1..256 and layers in 1..64 required");
  if (max_batch < 1 || !(sigma > 0.0) || !std::isfinite(sigma))
    return ws_fail(LQ2D_EINVAL, "max_batch >= 1 and a positive finite sigma required");
  const long long HW = (long long)K * N;
  const long long outc = (long long)(T + 1) * n;
  if (outc * HW * max_batch > (1LL << 31) - 1 || outc > (1 << 20))
    return ws_fail(LQ2D_EINVAL, "network output too large for one batch");
  lq2d_wsnet* net = new lq2d_wsnet();
  net->K = K; net->N = N; net->T = T; net->n = n; net->C = channels; net->L = layers; net->maxB = max_batch;
  net->sigma = sigma;
  long long P = 0, max_act = 0, max_wpart = 0;
  for (int l = 0; l < layers; ++l) {
    const int ci = l == 0 ? n + 1 : channels;
    const int co = l + 1 == layers ? (int)outc : channels;
    net->cin.push_back(ci);
    net->cout.push_back(co);
    net->off_w.push_back(P);
    P += (long long)co * ci * 9;
    net->off_b.push_back(P);
    P += co;
    max_act = std::max(max_act, (long long)std::max(ci, co) * HW * max_batch);
    int ks = 0;
    const int splits = wgrad_splits(co, ci * 9 + 1, (int)(HW * max_batch), &ks);
    max_wpart = std::max(max_wpart, (long long)splits * co * (ci * 9 + 1));
  }
  net->P = P;
  net->wpart_count = max_wpart;
  int rc = LQ2D_OK;
  net->act.assign(layers + 1, nullptr);
  if (!rc) rc = ws_alloc(net, &net->params, P);
  if (!rc) rc = ws_alloc(net, &net->grads, P);
  if (!rc) rc = ws_alloc(net, &net->m, P);
  if (!rc) rc = ws_alloc(net, &net->v, P);
  if (!rc) rc = ws_alloc(net, &net->wbf, P);
  for (int l = 0; l <= layers && !rc; ++l) {
    const long long c = l == 0 ? n + 1 : net->cout[l - 1];
    rc = ws_alloc(net, &net->act[l], c * HW * max_batch);
  }
  if (!rc) rc = ws_alloc(net, &net->gbuf[0], max_act);
  if (!rc) rc = ws_alloc(net, &net->gbuf[1], max_act);
  if (!rc) rc = ws_alloc(net, &net->wpart, max_wpart);
  if (!rc) rc = ws_alloc(net, &net->partials, 2 * kPartialBlocks);
  if (!rc) rc = ws_alloc(net, &net->counter, 8);
  if (!rc) rc = ws_alloc(net, &net->loss_dev, 1);
  if (!rc) rc = ws_alloc(net, &net->coupling_dev, max_batch);
  if (!rc && cudaMallocHost(&net->h_loss, sizeof(double)) != cudaSuccess)
    rc = ws_fail(LQ2D_ENOMEM, "cudaMallocHost failed");
  if (!rc) {
    cudaError_t e = cudaMemset(net->counter, 0, 8 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(net->params, 0, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(net->m, 0, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(net->v, 0, P * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(net->wbf, 0, P * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) rc = ws_fail(LQ2D_ECUDA, cudaGetErrorString(e));
  }
  if (rc) {
    lq2d_wsnet_destroy(net);
    return rc;
  }
  *out = net;
  return LQ2D_OK;
}

int lq2d_wsnet_param_count(const lq2d_wsnet* net, long long* count) {
  if (!net || !count) return ws_fail(LQ2D_EINVAL, "null argument");
  *count = net->P;
  return LQ2D_OK;
}

int lq2d_wsnet_set_params(lq2d_wsnet* net, const float* params) {
  if (!net || !params) return ws_fail(LQ2D_EINVAL, "null argument");
  for (long long e = 0; e < net->P; ++e)
    if (!std::isfinite(params[e])) return ws_fail(LQ2D_EINVAL, "non-finite parameter");
  WS_CUDA(cudaMemcpy(net->params, params, net->P * sizeof(float), cudaMemcpyHostToDevice));
  WS_CUDA(cudaMemset(net->m, 0, net->P * sizeof(float)));
  WS_CUDA(cudaMemset(net->v, 0, net->P * sizeof(float)));
  to_bf16_kernel<<<blocks_for(net->P, 256), 256>>>(net->params, net->wbf, net->P);
  WS_CUDA(cudaDeviceSynchronize());
  net->step = 0;
  return LQ2D_OK;
}

int lq2d_wsnet_get_params(const lq2d_wsnet* net, float* params) {
  if (!net || !params) return ws_fail(LQ2D_EINVAL, "null argument");
  WS_CUDA(cudaMemcpy(params, net->params, net->P * sizeof(float), cudaMemcpyDeviceToHost));
  return LQ2D_OK;
}

int lq2d_wsnet_forward_device(lq2d_wsnet* net, int batch, const double* d_x0, const double* coupling,
                              double* d_delta0, void* stream) {
  int rc = check_batch(net, batch, d_x0, coupling);
  if (rc) return rc;
  if (!d_delta0) return ws_fail(LQ2D_EINVAL, "null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = run_forward(net, batch, d_x0, coupling, s);
  if (rc) return rc;
  const int HW = net->K * net->N, Tp = net->T + 1;
  const long long total = (long long)batch * Tp * HW * net->n;
  output_kernel<<<blocks_for(total, 256), 256, 0, s>>>(net->act[net->L], batch, Tp, HW, net->n, net->sigma, d_delta0);
  WS_CUDA(cudaGetLastError());
  WS_CUDA(cudaStreamSynchronize(s));
  return LQ2D_OK;
}

int lq2d_wsnet_loss_grad_device(lq2d_wsnet* net, int batch, const double* d_x0, const double* coupling,
                                const double* d_target, double* loss, float* grads, void* stream) {
  int rc = check_batch(net, batch, d_x0, coupling);
  if (rc) return rc;
  if (!d_target) return ws_fail(LQ2D_EINVAL, "null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = run_loss_grad(net, batch, d_x0, coupling, d_target, loss, s);
  if (rc) return rc;
  if (grads) WS_CUDA(cudaMemcpy(grads, net->grads, net->P * sizeof(float), cudaMemcpyDeviceToHost));
  return LQ2D_OK;
}

int lq2d_wsnet_train_step_device(lq2d_wsnet* net, int batch, const double* d_x0, const double* coupling,
                                 const double* d_target, double lr, double* loss, void* stream) {
  int rc = check_batch(net, batch, d_x0, coupling);
  if (rc) return rc;
  if (!d_target) return ws_fail(LQ2D_EINVAL, "null argument");
  if (!(lr > 0.0) || !std::isfinite(lr)) return ws_fail(LQ2D_EINVAL, "lr must be positive and finite");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = run_loss_grad(net, batch, d_x0, coupling, d_target, loss, s);
  if (rc) return rc;
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  net->step += 1;
  const double c1 = 1.0 / (1.0 - std::pow(b1, net->step));
  const double c2 = 1.0 / (1.0 - std::pow(b2, net->step));
  adam_kernel<<<blocks_for(net->P, 256), 256, 0, s>>>(net->params, net->grads, net->m, net->v, net->wbf, net->P,
                                                      (float)lr, (float)b1, (float)b2, (float)eps, (float)c1,
                                                      (float)c2);
  WS_CUDA(cudaGetLastError());
  WS_CUDA(cudaStreamSynchronize(s));
  return LQ2D_OK;
}

void lq2d_wsnet_destroy(lq2d_wsnet* net) {
  if (!net) return;
  cudaDeviceSynchronize();
  for (void* p : net->allocs) cudaFree(p);
  if (net->h_loss) cudaFreeHost(net->h_loss);
  delete net;
}

}  // extern "C"
