// Persistent batched solve: many problems (uneven K, N, T) advanced by one
// set of kernel launches per PCG step.  Each launch is persistent (one wave of
// CTAs sized from the occupancy of the kernel) and its CTAs pull work units
// -- (problem, block of node-times) for the Delta product, (problem, column
// pair, time tile) for an NBJM sweep -- from a device work queue, so small
// and large problems share the SMs.  Per-problem reductions (y'd, norms, mu)
// and stop tests stay per problem: the last unit of a problem to finish
// completes them.  Problems whose state is done skip their units.
//
// FP64 path, state dimension n = 4 (the batched workloads), S x L sweeps.
#pragma once

#include "kernels.h"

namespace lq2d {

// Device-side descriptor of one problem of the batch.
struct BatchProblem {
  Grid g;
  OpData<double> op;
  PrecData<double> pd;
  SolverState* st;
  double* partials;
  const double* q;  // preconditioner output of the step (the last sweep's theta)
  double* d;        // direction: read as d_old, written as d_new
  double* y;        // Delta d
  double* z;        // scratch of the Delta product
};

constexpr int kBatchHeads = 16;  // queue heads: one per launch of a loop body

// Device arrays of a batch plan (owned by the batch).
struct BatchPlan {
  BatchProblem* probs = nullptr;
  int nprob = 0;
  int* sweep_off = nullptr;           // [nprob + 1] prefix sums of sweep units
  long long* op_off = nullptr;        // [nprob + 1] prefix sums of Delta units (blocks of kOpThreads)
  SweepArgsT<double>* args = nullptr; // [sweeps][nprob] arguments of each sweep of a step
  unsigned* heads = nullptr;          // [kBatchHeads] queue heads, zeroed by the loop control
  int threads = kSweepThreads;        // CTA width of the sweeps (32, 64 or 128)
  int grid_sweep = 0, grid_op = 0;    // persistent grid sizes
};

// Sweep units of one problem for a CTA width (column pairs x time tiles).
int batch_sweep_units(const Grid& g, int threads);
// Persistent grid sizes (one wave) for the plan's CTA width on this device.
cudaError_t batch_grid_sizes(BatchPlan& p);
// y = Delta d_new with d_new = q + beta d_old written back, y'd reduced and
// vartheta set, for every running problem (Algorithm 1's operator product).
void batch_enqueue_delta(const BatchPlan& p, int head, cudaStream_t s);
// One NBJM sweep of every running problem; args row `row` of the plan.
void batch_enqueue_sweep(const BatchPlan& p, int variant, int row, int head, cudaStream_t s);
// Loop control: counts the body pass of every running problem, stops a
// problem at its cap, keeps the loop while any problem runs, zeroes the heads.
void batch_enqueue_loop_ctrl(const BatchPlan& p, cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t batch_prepare();

}  // namespace lq2d
