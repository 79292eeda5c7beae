// Kernels of the persistent batched solve (batch.h): the Delta product and
// the NBJM sweeps of every problem of a batch, one launch each, with CTAs
// pulling (problem, unit) work from a device queue; and the loop control.
#include "batch.h"
#include "kernels_hot.cuh"

namespace lq2d {
namespace {

using namespace hot;

// The problem owning unit u: the last p with off[p] <= u (off[0] = 0).
template <typename I>
__device__ __forceinline__ int owner(const I* __restrict__ off, int nprob, long long u) {
  int lo = 0, hi = nprob;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((long long)off[mid] <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Next unit of the queue for the whole CTA.
__device__ __forceinline__ long long next_unit(unsigned* head) {
  __shared__ long long s_unit;
  __syncthreads();  // every thread is done with the previous unit
  if (threadIdx.x == 0) s_unit = (long long)atomicAdd(head, 1u);
  __syncthreads();
  return s_unit;
}

__global__ void __launch_bounds__(kOpThreads) batch_delta_z_kernel(const BatchProblem* __restrict__ probs, int nprob,
                                                                   const long long* __restrict__ off,
                                                                   unsigned* head) {
  const long long total = off[nprob];
  for (;;) {
    const long long u = next_unit(head);
    if (u >= total) break;
    const int p = owner(off, nprob, u);
    const Grid g = probs[p].g;
    const OpData<double> op = probs[p].op;
    delta_z_body<4, double, double, double>(g, op, probs[p].q, probs[p].d, probs[p].z, probs[p].st, 1, u - off[p]);
  }
}

__global__ void __launch_bounds__(kOpThreads) batch_delta_y_kernel(const BatchProblem* __restrict__ probs, int nprob,
                                                                   const long long* __restrict__ off,
                                                                   unsigned* head) {
  const long long total = off[nprob];
  for (;;) {
    const long long u = next_unit(head);
    if (u >= total) break;
    const int p = owner(off, nprob, u);
    const Grid g = probs[p].g;
    const OpData<double> op = probs[p].op;
    const BatchProblem& P = probs[p];
    delta_y_body<4, true, double, double>(g, op, P.z, P.q, P.d, P.d, nullptr, P.y, P.partials, P.st, u - off[p],
                                          off[p + 1] - off[p]);
  }
}

template <int VAR, int THR>
__global__ void __launch_bounds__(THR, (sweep_min_blocks<4, double, THR>()))
    batch_sweep_kernel(const BatchProblem* __restrict__ probs, int nprob, const int* __restrict__ off,
                       const SweepArgsT<double>* __restrict__ args, unsigned* head) {
  const int total = off[nprob];
  for (;;) {
    const long long u = next_unit(head);
    if (u >= total) break;
    const int p = owner(off, nprob, u);
    const Grid g = probs[p].g;
    const PrecData<double> pd = probs[p].pd;
    const SweepArgsT<double> a = args[p];
    nbjm_sweep_body<4, VAR, double, THR>(g, pd, a, probs[p].st, (int)(u - off[p]), off[p + 1] - off[p]);
  }
}

__global__ void batch_loop_ctrl_kernel(const BatchProblem* __restrict__ probs, int nprob, unsigned* heads,
                                       cudaGraphConditionalHandle h) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int mine = 0;
  for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
    SolverState* st = probs[p].st;
    if (st->done == kRunning) {
      const int c = st->body_count + 1;
      st->body_count = c;
      if (c < st->body_cap) mine = 1;
      else st->done = kLoopCap;
    }
  }
  if (mine) atomicOr(&any, 1);
  if (threadIdx.x < kBatchHeads) heads[threadIdx.x] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    heads[kBatchHeads] += 1u;  // body passes of this solve
    cudaGraphSetConditional(h, any ? 1u : 0u);
  }
}

template <int VAR, int THR>
void sweep_launch(const BatchPlan& p, int row, int head, cudaStream_t s) {
  batch_sweep_kernel<VAR, THR><<<p.grid_sweep, THR, sweep_smem_bytes<4, double, THR>(), s>>>(
      p.probs, p.nprob, p.sweep_off, p.args + (size_t)row * p.nprob, p.heads + head);
}

template <int THR>
void sweep_by_variant(const BatchPlan& p, int variant, int row, int head, cudaStream_t s) {
  switch (variant) {
    case kSweepPlain: sweep_launch<kSweepPlain, THR>(p, row, head, s); break;
    case kSweepUpdate: sweep_launch<kSweepUpdate, THR>(p, row, head, s); break;
    case kSweepOmega: sweep_launch<kSweepOmega, THR>(p, row, head, s); break;
    case kSweepOmegaMu: sweep_launch<kSweepOmegaMu, THR>(p, row, head, s); break;
    default: sweep_launch<kSweepXi, THR>(p, row, head, s); break;
  }
}

template <int VAR, int THR>
cudaError_t allow_smem() {
  return cudaFuncSetAttribute((const void*)batch_sweep_kernel<VAR, THR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sweep_smem_bytes<4, double, THR>());
}

template <int THR>
cudaError_t prepare_width() {
  const cudaError_t e[5] = {allow_smem<kSweepPlain, THR>(), allow_smem<kSweepUpdate, THR>(),
                            allow_smem<kSweepOmega, THR>(), allow_smem<kSweepOmegaMu, THR>(),
                            allow_smem<kSweepXi, THR>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

template <int THR>
cudaError_t occupancy(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void*)batch_sweep_kernel<kSweepXi, THR>,
                                                       THR, sweep_smem_bytes<4, double, THR>());
}

}  // namespace

int batch_sweep_units(const Grid& g, int threads) {
  const int TT = threads / 8;  // time steps per CTA at n = 4 (groups of 8 lanes)
  return g.V * ((g.T + 1 + TT - 1) / TT);
}

cudaError_t batch_grid_sizes(BatchPlan& p) {
  int dev = 0, sms = 0, per_sm = 0, op_per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    switch (p.threads) {
      case 32: e = occupancy<32>(&per_sm); break;
      case 128: e = occupancy<128>(&per_sm); break;
      default: e = occupancy<64>(&per_sm); break;
    }
  }
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&op_per_sm, (const void*)batch_delta_y_kernel, kOpThreads, 0);
  if (e != cudaSuccess) return e;
  p.grid_sweep = sms * (per_sm > 0 ? per_sm : 1);
  p.grid_op = sms * (op_per_sm > 0 ? op_per_sm : 1);
  return cudaSuccess;
}

void batch_enqueue_delta(const BatchPlan& p, int head, cudaStream_t s) {
  batch_delta_z_kernel<<<p.grid_op, kOpThreads, 0, s>>>(p.probs, p.nprob, p.op_off, p.heads + head);
  batch_delta_y_kernel<<<p.grid_op, kOpThreads, 0, s>>>(p.probs, p.nprob, p.op_off, p.heads + head + 1);
}

void batch_enqueue_sweep(const BatchPlan& p, int variant, int row, int head, cudaStream_t s) {
  switch (p.threads) {
    case 32: sweep_by_variant<32>(p, variant, row, head, s); break;
    case 128: sweep_by_variant<128>(p, variant, row, head, s); break;
    default: sweep_by_variant<64>(p, variant, row, head, s); break;
  }
}

void batch_enqueue_loop_ctrl(const BatchPlan& p, cudaGraphConditionalHandle h, cudaStream_t s) {
  batch_loop_ctrl_kernel<<<1, 256, 0, s>>>(p.probs, p.nprob, p.heads, h);
}

cudaError_t batch_prepare() {
  const cudaError_t e[3] = {prepare_width<32>(), prepare_width<64>(), prepare_width<128>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

}  // namespace lq2d
