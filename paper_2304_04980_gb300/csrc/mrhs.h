// Host-visible interface of the multi-right-hand-side preconditioner: the
// NBJM sweeps (Algorithm 2) applied to up to 32 right-hand sides of one
// problem at once, with the block products on the tensor cores (TF32
// operands, FP32 accumulation).  State dimension n = 4 only.
#pragma once

#include "common.cuh"

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
void launch_sweep(int variant, const Grid& g, const Buffers& b, const float* src, const float* theta_in,
                  float* theta_out, float* rth_out, cudaStream_t s);

// Shared-memory limits of the sweep kernels; once per device.
cudaError_t prepare();

}  // namespace mrhs
}  // namespace lq2d
