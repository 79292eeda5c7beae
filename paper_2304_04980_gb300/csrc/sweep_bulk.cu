// Launchers of the n = 4 FP32 NBJM sweep (sweep_bulk.cuh), the mixed
// precision preconditioner, for the supported schedules: CTA width
// (threads) and time steps per lane (steps).
#include "sweep_tiled.cuh"
#include "sweep_bulk.cuh"

namespace lq2d {
namespace {

using namespace hot;

template <int VAR, int R, int THR>
void go(const Grid& g, const PrecData<float>& pd, const SweepArgsT<float>& a, SolverState* st, cudaStream_t s) {
  nbjm_sweep_bulk_kernel<VAR, R, THR>
      <<<sweep_bulk_blocks<R, THR>(g), THR, sweep_bulk_smem<VAR, R, THR>(), s>>>(g, pd, a, st);
}

template <int R, int THR>
void by_variant(int variant, const Grid& g, const PrecData<float>& pd, const SweepArgsT<float>& a,
                SolverState* st, cudaStream_t s) {
  switch (variant) {
    case kSweepPlain: go<kSweepPlain, R, THR>(g, pd, a, st, s); break;
    case kSweepUpdate: go<kSweepUpdate, R, THR>(g, pd, a, st, s); break;
    case kSweepOmega: go<kSweepOmega, R, THR>(g, pd, a, st, s); break;
    case kSweepOmegaMu: go<kSweepOmegaMu, R, THR>(g, pd, a, st, s); break;
    case kSweepXiOmega: go<kSweepXiOmega, R, THR>(g, pd, a, st, s); break;
    default: go<kSweepXi, R, THR>(g, pd, a, st, s); break;
  }
}

template <int VAR, int R, int THR>
cudaError_t allow_smem() {
  return cudaFuncSetAttribute((const void*)nbjm_sweep_bulk_kernel<VAR, R, THR>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_bulk_smem<VAR, R, THR>());
}

template <int R, int THR>
cudaError_t prepare_config() {
  const cudaError_t e[6] = {allow_smem<kSweepPlain, R, THR>(),   allow_smem<kSweepUpdate, R, THR>(),
                            allow_smem<kSweepOmega, R, THR>(),   allow_smem<kSweepOmegaMu, R, THR>(),
                            allow_smem<kSweepXi, R, THR>(),      allow_smem<kSweepXiOmega, R, THR>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

}  // namespace

// Schedules of the n = 4 FP32 sweep: (threads per CTA, time steps per
// lane).  With steps >= 1 a CTA of the bulk-copy kernel holds threads/8
// groups of 8 lanes, each group `steps` consecutive time steps of one column
// pair; steps = 0 is the tiled kernel (one time step per group, per-element
// cp.async staging), whose finer tiles suit small grids.
constexpr int kBulkConfigs[][2] = {{32, 4}, {64, 4}, {64, 2}, {128, 2}, {32, 2}, {64, 1},
                                   {32, 0}, {64, 0}, {128, 0}};
constexpr int kNumBulkConfigs = 9;

bool sweep4_f32_config_ok(int threads, int steps) {
  for (int c = 0; c < kNumBulkConfigs; ++c)
    if (kBulkConfigs[c][0] == threads && kBulkConfigs[c][1] == steps) return true;
  return false;
}

int sweep4_f32_configs(int (*out)[2], int cap) {
  const int n = kNumBulkConfigs < cap ? kNumBulkConfigs : cap;
  for (int c = 0; c < n; ++c) {
    out[c][0] = kBulkConfigs[c][0];
    out[c][1] = kBulkConfigs[c][1];
  }
  return n;
}

void launch_sweep4_f32(int variant, int threads, int steps, const Grid& g, const PrecData<float>& pd,
                       const SweepArgsT<float>& a, SolverState* st, cudaStream_t s) {
  if (threads == 32 && steps == 4) by_variant<4, 32>(variant, g, pd, a, st, s);
  else if (threads == 64 && steps == 2) by_variant<2, 64>(variant, g, pd, a, st, s);
  else if (threads == 128 && steps == 2) by_variant<2, 128>(variant, g, pd, a, st, s);
  else if (threads == 32 && steps == 2) by_variant<2, 32>(variant, g, pd, a, st, s);
  else if (threads == 64 && steps == 1) by_variant<1, 64>(variant, g, pd, a, st, s);
  else by_variant<4, 64>(variant, g, pd, a, st, s);
}

cudaError_t prepare_sweep4_f32() {
  const cudaError_t e[6] = {prepare_config<4, 32>(),  prepare_config<4, 64>(), prepare_config<2, 64>(),
                            prepare_config<2, 128>(), prepare_config<2, 32>(), prepare_config<1, 64>()};
  for (cudaError_t x : e)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
}

}  // namespace lq2d
