// Host-visible interface of the multi-right-hand-side preconditioner: the
// NBJM sweeps (Algorithm 2) applied to up to 32 right-hand sides of one
// problem at once, with the block products on the tensor cores (TF32
// operands, FP32 accumulation).  State dimension n = 4 only.
#pragma once

#include "kernels.h"

namespace lq2d {
namespace mrhs {

constexpr int kRhs = 32;  // right-hand sides per vector (innermost index)
constexpr int kN = 4;     // state dimension served

// Library-owned buffers (float, TF32-rounded where they are tensor-core
// operands).
//   rec  [V][3][K][384]  per (column pair, class, pair-row): six 8 x 8 blocks
//                        in B-fragment order (see mrhs.cu); class 2 is t = 0
//   wom  [V][K][256]     Omega~ of the pair-row against its 8 staged
//                        neighbours (an 8 x 32 matrix), B-fragment order
//   wxa  [V][K][256]     A_hat Q^-1 (Xi~ term of delta_{t-1}), same form
//   wxq  [V][K][256]     Q^-1 A_hat' (Xi~ term of delta_{t+1}), same form
// Vectors are [n][K*N][T+1][32] floats (component plane, node, time, RHS).
struct Buffers {
  float* rec = nullptr;
  float* wom = nullptr;
  float* wxa = nullptr;
  float* wxq = nullptr;
};

// Element counts of the buffers above and of one vector.
long long rec_floats(const Grid& g);
long long w_floats(const Grid& g);
long long vec_floats(const Grid& g);

// Builds rec, wom, wxa, wxq from the FP64 setup (factors, node blocks).
void launch_build(const Grid& g, const NodeData& nd, const Buffers& b, cudaStream_t s);

// api [nrhs][T+1][K*N][n] (FP64)  <->  vector [n][K*N][T+1][32] (FP32);
// right-hand sides nrhs..31 are zero.
void launch_from_api(const Grid& g, int nrhs, const double* api, float* vec, cudaStream_t s);
void launch_to_api(const Grid& g, int nrhs, const float* vec, double* api, cudaStream_t s);

// One sweep theta_out = Phi~^-1 tau for all 32 right-hand sides:
//   variant 0: tau = src
//   variant 1: tau = src + Omega~ theta_in
//   variant 2: tau = src + Xi~ theta_in, also written to rth_out
// st (may be NULL): the sweep returns at once when st->done is set.
void launch_sweep(int variant, const Grid& g, const Buffers& b, const float* src, const float* theta_in,
                  float* theta_out, float* rth_out, const SolverState* st, cudaStream_t s);

// ---- multi-right-hand-side PCG (Algorithm 1 for each right-hand side)
//
// Per-right-hand-side scalars of the Krylov loop; the loop's own state
// (iteration count, stop flag, body counter) is a SolverState.
struct State {
  double mu[kRhs], beta[kRhs], alpha[kRhs];
  double rnorm2[kRhs], bnorm2[kRhs], rref2[kRhs];
  int conv[kRhs];   // the residual met the tolerance: this right-hand side is frozen
  int repl[kRhs];   // its residual is due for replacement by the true one
  int iters[kRhs];  // PCG steps taken by it
  int nrhs, any_repl, have_mu, breakdown;
  double tol2, rho2;
  unsigned int counter;
  int pad;
};

// Vectors of the loop, all [n][K*N][T+1][32]: FP64 rhs, r, delta, d and the
// FP64 product of a replacement; FP32 copies and products.
struct SolveVecs {
  double *rhs, *r, *delta, *d, *y64, *z64;
  float *d32, *z32, *y32, *r32;
};

// Blocks of the element-wise kernels (grid-stride over (node, t), one warp
// per (node, t), lane = right-hand side) and their partial-sum slots.
int solve_blocks(const Grid& g);

// r = r_delta (x0s [nrhs][K*N][n] at t = 0, rhs1 [n][..] of the problem's
// own right-hand side at t >= 1), delta = d = 0, norms and state.
void launch_init(const Grid& g, int nrhs, const double* x0s, const double* rhs1, long long rhs1_stride,
                 const SolveVecs& v, double* partials, State* ms, SolverState* st, double tol, double rho2,
                 int max_iter, cudaStream_t s);
// y32 = Delta d_new with d_new = q + beta d (FP32 product, FP64 d), y' d_new
// and alpha per right-hand side.
void launch_delta_loop(const Grid& g, const OpData<float>& op, const float* q, const SolveVecs& v,
                       double* partials, State* ms, SolverState* st, cudaStream_t s);
// delta += alpha d, r -= alpha y (right-hand sides not yet converged),
// norms, stop and replacement tests.
void launch_update(const Grid& g, const SolveVecs& v, double* partials, State* ms, SolverState* st, cudaStream_t s);
// mu = q' r and beta (flexible ratio) per right-hand side.
void launch_mu(const Grid& g, const float* q, const SolveVecs& v, double* partials, State* ms, SolverState* st,
               cudaStream_t s);
// r = r_delta - Delta delta in FP64 for the right-hand sides due for
// replacement (force: all of them, then the convergence flags follow the
// true residual); gated on the state unless forced.
void launch_replace(const Grid& g, const OpData<double>& op, const SolveVecs& v, double* partials, State* ms,
                    SolverState* st, bool force, cudaStream_t s);
// Right-hand side r of a vector into the single-right-hand-side internal
// layout [k][node][t] (plane stride Ps).
void launch_gather(const Grid& g, const double* vec, int r, double* single, cudaStream_t s);

// Shared-memory limits of the sweep kernels; once per device.
cudaError_t prepare();

}  // namespace mrhs
}  // namespace lq2d
