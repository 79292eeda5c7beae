// Host-visible launch interface of the per-state-dimension hot kernels.
// Each state dimension n = 1..kMaxN is compiled in its own translation unit
// (inst_n*.cu) and exposes one KernelTable.
#pragma once

#include "common.cuh"

namespace lq2d {

constexpr int kOpThreads = 256;     // threads per block of the node-time kernels
// Default threads per block of the sweep kernels (32, 64, 128 or 256 are
// compiled).  Two warps per CTA spread the (column pair, time step) block
// solves over the SMs in fine units, each staging a factor row once for
// 64/g time steps (g = 2n rounded up to a power of two); this width timed
// fastest on the 64 x 64 x 100 and 256 x 256 x 200 grids in both precisions.
constexpr int kSweepThreads = 64;

// Operands of the Delta product in its compute precision CT (double, or
// float in precision mode 2): the grid blocks and the per-node Q^-1, Q_T^-1,
// B R^-1 B'.
template <typename CT>
struct OpData {
  const CT* Aself;  // [NN][n][n]
  const CT* Anb;    // [NN][4][n][n]
  const CT* Qi;     // [NN][n][n]
  const CT* QTi;    // [NN][n][n]
  const CT* Sb;     // [NN][n][n]
};

// Operands of the preconditioner in the precision VT of the sweeps (double,
// or float in the mixed mode): the banded block-Cholesky factors of
// Phi_bar, the Omega~ and Xi~ node blocks, and Q for the t = 0 blocks.
template <typename VT>
struct PrecData {
  const VT* fac;
  long long fac_rec;  // elements per pair-row record (24 n^2)
  long long fac_vc;   // elements per (v, class) factor
  const VT* Om;       // [NN][5][n][n]
  const VT* AQ;       // [NN][5][n][n]
  const VT* QAt;      // [NN][5][n][n]
  const VT* Qm;       // [NN][n][n]
  // FP32, n = 4: records of Phi_bar_{v,0} = blkdiag(Q^-1) in the layout of
  // fac ([V][K] records, F = N = 0, D^-1 = blkdiag(Q, Q)); NULL otherwise
  const VT* fac_t0;
  // two-ended solve (when enabled): the factor of the reversed pair-row
  // order (layout of fac, records in step order) and S^-1 of the interface
  // rows per (v, class), [V][2][(4n)^2]; NULL otherwise
  const VT* fac_rev;
  const VT* sinv;
};

// Layout of the preconditioner's FP32 iterates (theta, delta^(s) and its
// output q in the mixed modes): node-major, v[(p*(T+1) + t)*n + k], so that
// one (node, t) is n contiguous values and a node's time window is one
// contiguous run.  FP64 vectors use the component planes of common.cuh.
__host__ __device__ inline long long iter_f32_index(int n, int k, long long pt) { return pt * n + k; }

// Arguments of one NBJM sweep: theta_out = Phi~^-1 tau with
//   tau = src                           (first sweep of the first outer step)
//   tau = r + Xi~ delta_s               (first sweep of a later outer step; tau is kept in rtheta_out)
//   tau = src + Omega~ theta_in         (later sweeps)
// and, in the first sweep of a PCG step, the update of Algorithm 1 lines
// 9-10 fused in front (delta += vartheta d, r -= vartheta y; tau = r).
// The iterates theta and delta_s are in the sweep precision VT (FP32 ones
// node-major, iter_f32_index); the PCG vectors r, delta, y, d are double in
// component planes, and so is the stored r_theta except in the n = 4 FP32
// sweeps, which keep it as FP32 in the node-major layout.
template <typename VT>
struct SweepArgsT {
  // the source tau of the first sweep of a later inner step: FP64 r in
  // component planes, or (src_rtheta != 0, n = 4 FP32 sweeps) the stored
  // r_theta as FP32 in the iterates' node-major layout
  const double* src;
  double* rtheta_out;
  const VT* delta_s;
  const VT* theta_in;
  VT* theta_out;
  double* r;
  double* delta;
  const double* y;
  const double* d;
  double* partials;
  int src_rtheta;
  int* fault;  // set when a bounded wait of the sweep ran out (may be NULL)
};
using SweepArgs = SweepArgsT<double>;

enum SweepVariant {
  kSweepPlain = 0,      // tau = src
  kSweepUpdate = 1,     // PCG update fused, tau = updated r, norms reduced, stop test
  kSweepOmega = 2,      // tau = src + Omega~ theta_in
  kSweepOmegaMu = 3,    // as kSweepOmega, plus mu = theta_out' r reduced (last sweep)
  kSweepXi = 4,         // tau = r + Xi~ delta_s, written to rtheta_out
  kSweepXiOmega = 5,    // tau = r + Xi~ delta_s + Omega~ theta_in (theta_in = delta_s): the first inner
                        // sweep of the standalone NBJM solver, started from the outer iterate
};

struct KernelTable {
  // z = Q~^-1 A~' dn with dn = q + beta d_old (beta from the state when use_beta),
  // computed in CT; q is the preconditioner output (double, or float in the
  // mixed modes); z is stored in CT.
  void (*delta_z)(const Grid& g, const OpData<double>& op, const double* q, const double* dold, double* z,
                  const SolverState* st, int use_beta, cudaStream_t s);
  void (*delta_z_f32)(const Grid& g, const OpData<double>& op, const float* q, const double* dold, double* z,
                      const SolverState* st, int use_beta, cudaStream_t s);
  // precision mode 2: everything in FP32, d_old read from its FP32 copy
  void (*delta_z_f32op)(const Grid& g, const OpData<float>& op, const float* q, const float* dold32, float* z,
                        const SolverState* st, int use_beta, cudaStream_t s);
  // y = A~ z + B~ R~^-1 B~' dn; in loop mode also writes dn into dout, reduces
  // y' dn and sets vartheta = mu / (y' dn) (Algorithm 1: operator product and step length)
  void (*delta_y)(const Grid& g, const OpData<double>& op, const double* z, const double* q, const double* dold,
                  double* dout, double* y, double* partials, SolverState* st, int loop_mode, cudaStream_t s);
  void (*delta_y_f32)(const Grid& g, const OpData<double>& op, const double* z, const float* q, const double* dold,
                      double* dout, double* y, double* partials, SolverState* st, int loop_mode, cudaStream_t s);
  // precision mode 2: also writes the FP32 copy of the new direction
  void (*delta_y_f32op)(const Grid& g, const OpData<float>& op, const float* z, const float* q, const double* dold,
                        double* dout, float* dout32, double* y, double* partials, SolverState* st, int loop_mode,
                        cudaStream_t s);
  // FP64 sweep (Algorithm 2 step); the OmegaMu variant sets beta = mu_new / mu_old
  // threads: CTA width of the sweep, 32, 64, 128 or 256 (a tile of threads / 2n
  // time steps, 2n rounded up to a power of two)
  void (*sweep)(int variant, int threads, const Grid& g, const PrecData<double>& pd, const SweepArgsT<double>& a,
                SolverState* st, cudaStream_t s);
  // FP32 sweep of the mixed mode; the OmegaMu variant sets the flexible
  // beta = q_new'(r_new - r_old) / mu_old = -vartheta q_new'y / mu_old.
  // steps: time steps per lane of the n = 4 schedule (ignored for other n)
  void (*sweep_f32)(int variant, int threads, int steps, const Grid& g, const PrecData<float>& pd,
                    const SweepArgsT<float>& a, SolverState* st, cudaStream_t s);
  // KKT residual pieces and cost of (x, u, delta): out[0] = sum of squared
  // residual entries, out[1] = x'Q~x + u'R~u, out[2] = max |A~x + B~u + omega~|
  void (*kkt)(const Grid& g, const NodeData& nd, const double* x, const double* u, const double* delta,
              const double* rhs, double* partials, SolverState* st, double* out, cudaStream_t s);
  // sets the sweep kernels' shared-memory limits on the current device
  cudaError_t (*prepare)();
};

const KernelTable* kernel_table(int n);

// The n = 4 FP32 sweep with bulk-copy staging (sweep_bulk.cu): launch with a
// schedule (threads per CTA, time steps per lane), the schedules compiled,
// and the shared-memory limits of its kernels.
void launch_sweep4_f32(int variant, int threads, int steps, const Grid& g, const PrecData<float>& pd,
                       const SweepArgsT<float>& a, SolverState* st, cudaStream_t s);
bool sweep4_f32_config_ok(int threads, int steps);
int sweep4_f32_configs(int (*out)[2], int cap);
cudaError_t prepare_sweep4_f32();
constexpr int kSweepSteps = 4;  // time steps per lane of the n = 4 FP32 bulk-copy sweep by default
// (column pair, time) blocks from which the n = 4 FP32 sweeps default to the
// bulk-copy kernel (below: the tiled kernel, whose finer tiles fill the GPU)
constexpr long long kBulkMinBlocks = 16384;

// dimension-generic helpers (kernels_misc.cu)
void launch_init_state(SolverState* st, double tol, int max_iter, int stop_mode, const double* bnorm2,
                       int keep_iter, double* hist, int hist_cap, double phase_rho2, cudaStream_t s);
// identity preconditioner (plain CG): q = r, mu = r'r; with update, the PCG
// update and stop test of Algorithm 1 first
void launch_ident(const Grid& g, bool update, double* r, double* delta, const double* y, const double* d,
                  double* q, double* partials, SolverState* st, cudaStream_t s);
// standalone NBJM exit test: max |a - b| (b = NULL: max |a|) < eps, counts the outer step
void launch_nbjm_diff(const Grid& g, const void* a, const void* b, int fp32, double* partials, SolverState* st,
                      cudaStream_t s);
void launch_init_residual(const Grid& g, const double* rhs, const double* y, double* r, double* delta,
                          const double* delta0, double* partials, SolverState* st, cudaStream_t s);
// reliable update of precision mode 2: r = rhs - y when the state asks for a
// replacement (y = Delta delta from the gated Delta kernels), else nothing
void launch_replace_residual(const Grid& g, const double* rhs, const double* y, double* r, double* partials,
                             SolverState* st, cudaStream_t s);
void launch_norms(const Grid& g, const double* v, int comps, double* partials, unsigned int* counter,
                  double* out2, cudaStream_t s);
void launch_build_rhs(const Grid& g, const double* x0, const double* w_api, double* rhs, cudaStream_t s);
void launch_to_internal(const double* api, double* intl, int NN, int slices, int comps, long long stride,
                        cudaStream_t s);
void launch_to_api(const double* intl, double* api, int NN, int slices, int comps, long long stride,
                   cudaStream_t s);
void launch_recover_u(const Grid& g, const NodeData& nd, const double* delta, double* u, cudaStream_t s);
void launch_loop_ctrl(SolverState* st, cudaGraphConditionalHandle h, cudaStream_t s);
void launch_to_f32(const double* src, float* dst, long long count, cudaStream_t s);
void launch_to_f64(const float* src, double* dst, long long count, cudaStream_t s);
// an FP32 iterate of the preconditioner (node-major) into an FP64 vector in
// component planes
// d = q + beta d in FP64 (beta from the state), skipped once the state is
// done; q FP64 (component planes) or FP32 (node-major)
void launch_direction_update(const Grid& g, const void* q, bool q_f32, double* d, const SolverState* st,
                             cudaStream_t s);
void launch_iter_f32_to_f64(const Grid& g, const float* src, double* dst, cudaStream_t s);
// records of the t = 0 factor class for the n = 4 FP32 sweeps: F = N = 0,
// D^-1 = blkdiag(Q of the pair-row's nodes), from the FP32 copy of Q
void launch_t0_records(const Grid& g, const float* Q32, float* rec, long long fac_rec, cudaStream_t s);

}  // namespace lq2d
