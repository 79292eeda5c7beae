// y = Delta d without any device allocation: the variant of the Delta apply
// (delta_z_kernel + delta_y_kernel) whose scratch lives in one file-scope
// device array instead of buffers owned by a problem handle.
//
// Some callers cannot allocate device memory once they are running: a
// controller that re-evaluates Delta d inside a fixed-period loop, where an
// allocator call adds latency it cannot bound, and host frameworks that own
// every device allocation of the process and hand libraries only the
// buffers they manage.  Such callers cannot create a problem handle (it
// allocates) and pass the raw problem blocks instead.
//
// The scratch array holds the per-node blocks Q^-1, Q_T^-1, B R^-1 B' and the
// intermediate z = Q~^-1 A~' d.  Every GPU that loads the library holds it
// until the process exits; with lazy module loading (the CUDA default) the
// module and its array are loaded on a device by the first call there, so
// that call belongs in a caller's set-up, before its fixed-period loop.
// All calls share the array and it keeps the last call's contents; both
// parts are rewritten in full by every call, so nothing in it has to start
// at zero.  Calls whose work overlaps on the GPU (different streams, or
// different host threads on one device) race on it.
#include <mutex>
#include <string>

#include "../../include/lq2d.h"
#include "common.cuh"

namespace lq2d {
void set_last_error(const std::string& msg);  // lq2d.cu: the message lq2d_last_error() returns
}

namespace {

// 2^21 doubles = 16 MiB.  A call needs (T+1)*K*N*n + 3*K*N*n*n + 1 of them;
// the K = N = 64, T = 100, n = 4 grid needs 1,851,393.
constexpr long long kStaticScratchDoubles = 1LL << 21;

__device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Inverse of a small SPD block by Gauss-Jordan elimination without pivoting
// (SPD matrices need none); false on a non-positive or non-finite pivot.
__device__ bool invert_spd(const double* a, double* inv, int d) {
  double w[lq2d::kMaxN * 2 * lq2d::kMaxN];
  const int W = 2 * d;
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < W; ++c) w[r * W + c] = c < d ? 0.5 * (a[r * d + c] + a[c * d + r]) : (c - d == r ? 1.0 : 0.0);
  for (int p = 0; p < d; ++p) {
    const double piv = w[p * W + p];
    if (!(piv > 0.0) || !isfinite(piv)) return false;
    const double inv_piv = 1.0 / piv;
    for (int c = 0; c < W; ++c) w[p * W + c] *= inv_piv;
    for (int r = 0; r < d; ++r) {
      if (r == p) continue;
      const double f = w[r * W + p];
      for (int c = 0; c < W; ++c) w[r * W + c] -= f * w[p * W + c];
    }
  }
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) inv[r * d + c] = w[r * W + d + c];
  return true;
}

// Per node: Q^-1, Q_T^-1 and S = B R^-1 B' into the scratch array.
__global__ void static_nodes_kernel(int NN, int n, int m, const double* __restrict__ Q, const double* __restrict__ R,
                                    const double* __restrict__ QT, const double* __restrict__ B, double* scratch,
                                    int* bad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NN) return;
  const int nn = n * n;
  double* Qi = scratch + (size_t)p * 3 * nn;
  double* QTi = Qi + nn;
  double* S = QTi + nn;
  double Ri[lq2d::kMaxM * lq2d::kMaxM];
  bool ok = invert_spd(Q + (size_t)p * nn, Qi, n);
  ok = invert_spd(QT + (size_t)p * nn, QTi, n) && ok;
  ok = invert_spd(R + (size_t)p * m * m, Ri, m) && ok;
  const double* Bp = B + (size_t)p * n * m;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) {
      double s = 0.0;
      for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) s += Bp[r * m + a] * Ri[a * m + b] * Bp[c * m + b];
      S[r * n + c] = s;
    }
  if (!ok) atomicOr(bad, 1);
}

// A_hat block in row p towards its neighbour in direction dir (E, F, G, H of p).
__device__ inline const double* row_block(const double* A, const double* Anb, int p, int dir, int nn) {
  return dir == lq2d::kSelf ? A + (size_t)p * nn : Anb + ((size_t)p * 4 + (dir - 1)) * nn;
}

// A_hat block in row r, column p, for r = neighbour of p in direction dir.
__device__ inline const double* col_block(const double* A, const double* Anb, int r, int dir, int nn) {
  const int slot = dir == lq2d::kWest ? 1 : dir == lq2d::kEast ? 0 : dir == lq2d::kNorth ? 3 : 2;
  return dir == lq2d::kSelf ? A + (size_t)r * nn : Anb + ((size_t)r * 4 + slot) * nn;
}

// z_t = Q_t^-1 (-d_t + A_hat' d_{t+1}) (the last term absent at t = T), host
// layout [t][node][k], one thread per (t, node).
__global__ void static_z_kernel(int K, int N, int T, int n, const double* __restrict__ A,
                                const double* __restrict__ Anb, const double* __restrict__ d,
                                const double* scratch, double* z) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int NN = K * N;
  if (idx >= (long long)NN * (T + 1)) return;
  const int t = (int)(idx / NN), p = (int)(idx % NN);
  const int i = p / N, j = p % N, nn = n * n;
  double w[lq2d::kMaxN];
  for (int k = 0; k < n; ++k) w[k] = -d[idx * n + k];
  if (t < T) {
    for (int dir = 0; dir < 5; ++dir) {
      const int r = lq2d::nbr_node(i, j, dir, K, N);
      if (r < 0) continue;
      const double* blk = col_block(A, Anb, r, dir, nn);
      const double* dr = d + ((long long)(t + 1) * NN + r) * n;
      for (int c = 0; c < n; ++c)
        for (int k = 0; k < n; ++k) w[k] += blk[c * n + k] * dr[c];
    }
  }
  const double* Qb = scratch + (size_t)p * 3 * nn + (t == T ? nn : 0);
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int c = 0; c < n; ++c) s += Qb[k * n + c] * w[c];
    z[idx * n + k] = s;
  }
}

// y_0 = -z_0, y_t = A_hat z_{t-1} - z_t + S d_t, host layout.
__global__ void static_y_kernel(int K, int N, int T, int n, const double* __restrict__ A,
                                const double* __restrict__ Anb, const double* __restrict__ d,
                                const double* scratch, const double* z, double* __restrict__ y) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int NN = K * N;
  if (idx >= (long long)NN * (T + 1)) return;
  const int t = (int)(idx / NN), p = (int)(idx % NN);
  const int i = p / N, j = p % N, nn = n * n;
  double acc[lq2d::kMaxN];
  for (int k = 0; k < n; ++k) acc[k] = -z[idx * n + k];
  if (t >= 1) {
    for (int dir = 0; dir < 5; ++dir) {
      const int r = lq2d::nbr_node(i, j, dir, K, N);
      if (r < 0) continue;
      const double* blk = row_block(A, Anb, p, dir, nn);
      const double* zr = z + ((long long)(t - 1) * NN + r) * n;
      for (int k = 0; k < n; ++k)
        for (int c = 0; c < n; ++c) acc[k] += blk[k * n + c] * zr[c];
    }
    const double* S = scratch + (size_t)p * 3 * nn + 2 * nn;
    for (int k = 0; k < n; ++k)
      for (int c = 0; c < n; ++c) acc[k] += S[k * n + c] * d[idx * n + c];
  }
  for (int k = 0; k < n; ++k) y[idx * n + k] = acc[k];
}

// Address of the scratch array on the current device, looked up once per
// device (cudaGetSymbolAddress with that device current) and cached.
int scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    lq2d::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return LQ2D_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    lq2d::set_last_error("lq2d_apply_delta_static: device index " + std::to_string(dev) +
                         " is beyond the " + std::to_string(kMaxDevices) + " devices the library tracks");
    return LQ2D_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    double* ptr = nullptr;
    e = cudaGetSymbolAddress((void**)&ptr, g_static_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      lq2d::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return LQ2D_ECUDA;
    }
    g_scratch_ptr[dev] = ptr;
  }
  *out = g_scratch_ptr[dev];
  return LQ2D_OK;
}

}  // namespace

extern "C" int lq2d_apply_delta_static(int K, int N, int T, int n, int m, const double* d_A_self,
                                       const double* d_A_nbr, const double* d_B, const double* d_Q,
                                       const double* d_R, const double* d_Q_T, const void* d_in, void* d_out,
                                       void* stream) {
  if (K < 1 || N < 1 || T < 1 || n < 1 || n > lq2d::kMaxN || m < 1 || m > lq2d::kMaxM) {
    lq2d::set_last_error("lq2d_apply_delta_static: K, N, T >= 1, 1 <= n <= 8, 1 <= m <= 8 required");
    return LQ2D_EINVAL;
  }
  if (!d_A_self || !d_A_nbr || !d_B || !d_Q || !d_R || !d_Q_T || !d_in || !d_out) {
    lq2d::set_last_error("lq2d_apply_delta_static: null pointer");
    return LQ2D_EINVAL;
  }
  const long long NN = (long long)K * N;
  const long long need = NN * (T + 1LL) * n + NN * 3LL * n * n + 1;  // z, node blocks, status word
  if (need > kStaticScratchDoubles) {
    lq2d::set_last_error("lq2d_apply_delta_static: problem needs " + std::to_string(need) +
                   " scratch doubles, more than the fixed " + std::to_string(kStaticScratchDoubles) +
                   " (require (T+1)*K*N*n + 3*K*N*n*n + 1 <= that)");
    return LQ2D_EINVAL;
  }
  // the product reads d while it writes y (y is declared restrict in the
  // kernels), so the two ranges must not overlap
  const long long bytes = NN * (T + 1LL) * n * (long long)sizeof(double);
  const char* in_b = static_cast<const char*>(d_in);
  const char* out_b = static_cast<const char*>(d_out);
  if (in_b < out_b + bytes && out_b < in_b + bytes) {
    lq2d::set_last_error("lq2d_apply_delta_static: d_in and d_out overlap");
    return LQ2D_EINVAL;
  }
  double* scratch = nullptr;
  int rc = scratch_on_current_device(&scratch);
  if (rc != LQ2D_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* blocks = scratch;
  double* z = scratch + NN * 3LL * n * n;
  int* bad = reinterpret_cast<int*>(scratch + kStaticScratchDoubles - 1);
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    static_nodes_kernel<<<(unsigned)((NN + 127) / 128), 128, 0, s>>>((int)NN, n, m, d_Q, d_R, d_Q_T, d_B, blocks, bad);
    const long long total = NN * (T + 1);
    const unsigned grid = (unsigned)((total + 255) / 256);
    static_z_kernel<<<grid, 256, 0, s>>>(K, N, T, n, d_A_self, d_A_nbr, static_cast<const double*>(d_in), blocks, z);
    static_y_kernel<<<grid, 256, 0, s>>>(K, N, T, n, d_A_self, d_A_nbr, static_cast<const double*>(d_in), blocks,
                                         z, static_cast<double*>(d_out));
    e = cudaGetLastError();
  }
  int h_bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    lq2d::set_last_error(std::string("lq2d_apply_delta_static: ") + cudaGetErrorString(e));
    return LQ2D_ECUDA;
  }
  if (h_bad) {
    lq2d::set_last_error("lq2d_apply_delta_static: Q, Q_T or R is not positive definite");
    return LQ2D_ENOTPD;
  }
  return LQ2D_OK;
}

