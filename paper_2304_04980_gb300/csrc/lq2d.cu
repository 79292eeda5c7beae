// C-ABI library: problem handle, setup, and the PCG driver (Algorithm 1 with
// Algorithm 2 as preconditioner) over the CUDA kernels of this directory.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lq2d.h"
#include "batch.h"
#include "kernels.h"
#include "mrhs.h"
#include "setup.h"

using namespace lq2d;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define LQ_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(e_ == cudaErrorMemoryAllocation ? LQ2D_ENOMEM : LQ2D_ECUDA,                  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

struct GraphEntry {
  int S = 0, L = 0, precision = 0, precond = 0, threads = 0, steps = 0, twisted = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

constexpr int kMaxGraphs = 8;
constexpr int kHistCap = 1 << 16;  // PCG steps whose coefficients are kept for the Lanczos estimate
// Precision mode 2: once the recurrence residual of the FP32-product Krylov
// loop has dropped by kPhaseRho since the last replacement, the FP64 true
// residual replaces it and the iteration continues with the same direction.
constexpr double kPhaseRho = 1e-4;
constexpr int kStreamChunk = 4;  // steps enqueued between stop-flag reads (driver 1)

long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

}  // namespace

struct lq2d_problem {
  Grid g{};
  NodeData nd{};
  SetupBuffers sb{};
  const KernelTable* kt = nullptr;
  cudaStream_t priv = nullptr;  // private stream for graph capture
  std::vector<void*> allocs;
  // vectors, internal layout
  double *rhs = nullptr, *delta = nullptr, *r = nullptr, *d = nullptr, *y = nullptr, *z = nullptr;
  double *thA = nullptr, *thB = nullptr, *rth = nullptr, *u = nullptr;
  double *w_aff = nullptr;     // active affine terms, host layout [T][NN][n] (NULL: none)
  double *w_buf = nullptr;     // their device buffer, allocated on first use
  double* stage_x = nullptr;   // host-layout staging, [T+1][NN][n]
  double* stage_u = nullptr;   // [T][NN][m]
  double* partials = nullptr;
  double* bnorm = nullptr;     // [2]: ||r_delta||_2^2, ||r_delta||_inf
  double* kkt_out = nullptr;   // [4]
  int* setup_status = nullptr;
  SolverState* st = nullptr;
  // pinned host mirrors
  SolverState* h_st = nullptr;
  double* h_kkt = nullptr;
  int* h_done = nullptr;  // [2] stop-flag slots for driver 1
  // options
  int stop_mode = 0;
  int driver = 0;
  int timing = 0;
  int max_restarts = 3;
  GraphEntry graphs[kMaxGraphs];
  int ngraphs = 0;
  lq2d_stats stats{};
  std::vector<cudaEvent_t> ev_pool;
  long long launches = 0;  // kernels launched on behalf of this handle since creation
  // precision of the preconditioner: 0 = FP64, 1 = FP32 sweeps and factors
  int precision = 0;
  PrecData<double> pd64{};
  PrecData<float> pd32{};
  OpData<double> op64{};
  OpData<float> op32{};
  float* f32_buf = nullptr;  // FP32 copies of the factors and node blocks (mode 1, allocated on first use)
  float* d32 = nullptr;      // FP32 copy of the direction d (mode 2)
  int precond_kind = 0;      // 0: NBJM (Algorithm 2), 1: none (plain CG)
  int sweep_threads[2] = {kSweepThreads, kSweepThreads};  // CTA width of the FP64 / FP32 sweeps (32..256)
  int sweep_steps = kSweepSteps;  // time steps per lane of the n = 4 FP32 sweeps
  int twisted[2] = {0, 0};        // two-ended solve of Phi_bar in the FP64 / FP32 sweeps (option)
  bool twisted_ready = false;     // reversed factor and interface inverses allocated (n = 4, K >= 4)
  float* fac_rev32 = nullptr;     // FP32 copies of the reversed factor and the interface inverses
  float* sinv32 = nullptr;
  int* fault = nullptr;           // device word set when a bounded wait inside a sweep ran out
  int kappa = 0;             // record the PCG coefficients and estimate the condition number
  double* hist = nullptr;    // device: vartheta_j, beta_j pairs
  std::vector<double> h_hist;
  int graph_body_kernels = 0;  // kernels per device-loop body of the last graph launch (0: no graph)
  // multi-right-hand-side preconditioner (n = 4; allocated on first use,
  // rebuilt after every setup)
  mrhs::Buffers mb{};
  float *m_src = nullptr, *m_thA = nullptr, *m_thB = nullptr, *m_rth = nullptr;
  bool mrhs_built = false;
  // multi-right-hand-side PCG (allocated on its first solve)
  mrhs::SolveVecs mv{};
  mrhs::State* mstate = nullptr;
  mrhs::State* h_mstate = nullptr;  // pinned mirror
  double* m_partials = nullptr;
  cudaGraph_t m_graph = nullptr;
  cudaGraphExec_t m_exec = nullptr;
  int m_graph_S = 0, m_graph_L = 0;
};

// Many problems solved by one graph launch: one independent chain per
// problem (initial residual and preconditioner, the device loop of
// Algorithm 1 under a conditional while node, recovery), all in one graph.
struct lq2d_batch {
  std::vector<lq2d_problem*> probs;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double* results = nullptr;   // device: kBatchSlot doubles per problem
  double* h_results = nullptr; // pinned host mirror
  // what the graph was built for
  double tol = 0.0;
  int S = 0, L = 0, max_iter = -1;
  std::vector<int> built_modes;
  // persistent batched loop (problems with n = 4 in FP64 with the NBJM
  // preconditioner): one launch per kernel of a PCG step for all problems
  int persistent = 1;              // option: use it when the problems allow it
  int threads = kSweepThreads;     // CTA width of its sweeps (32, 64 or 128)
  bool built_persistent = false;   // the current graph is the persistent one
  BatchPlan plan{};                // device arrays, inside plan_mem
  void* plan_mem = nullptr;
  size_t plan_bytes = 0;
  std::vector<int> variants;       // [2 S L]: loop-step sweeps, then a plain D_S
  unsigned* h_heads = nullptr;     // pinned: the queue heads and the pass counter
};

namespace {

constexpr int kBatchSlot = 32;  // doubles per problem in the batch result array

// Failure injection for the allocation path, on the host: with the
// environment variable LQ2D_FAIL_ALLOC_AT=k (k >= 1), the k-th device
// allocation of every handle reports cudaErrorMemoryAllocation without
// calling cudaMalloc, so the LQ2D_ENOMEM path and the release of the
// allocations made before it can be tested without exhausting a GPU.
bool simulated_alloc_failure(const lq2d_problem* h) {
  const char* v = std::getenv("LQ2D_FAIL_ALLOC_AT");
  if (v == nullptr || *v == '\0') return false;
  const long k = std::strtol(v, nullptr, 10);
  return k >= 1 && (long)h->allocs.size() + 1 == k;
}

int dev_alloc(lq2d_problem* h, double** p, size_t count) {
  void* ptr = nullptr;
  cudaError_t e = simulated_alloc_failure(h) ? cudaErrorMemoryAllocation
                                             : cudaMalloc(&ptr, count * sizeof(double) + 256);
  if (e != cudaSuccess) return fail(LQ2D_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocs.push_back(ptr);
  *p = static_cast<double*>(ptr);
  return LQ2D_OK;
}

void free_all(lq2d_problem* h) {
  for (int i = 0; i < h->ngraphs; ++i) {
    if (h->graphs[i].exec) cudaGraphExecDestroy(h->graphs[i].exec);
    if (h->graphs[i].graph) cudaGraphDestroy(h->graphs[i].graph);
  }
  h->ngraphs = 0;
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear();
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->h_st) cudaFreeHost(h->h_st);
  if (h->h_kkt) cudaFreeHost(h->h_kkt);
  if (h->h_done) cudaFreeHost(h->h_done);
  if (h->h_mstate) cudaFreeHost(h->h_mstate);
  if (h->m_exec) cudaGraphExecDestroy(h->m_exec);
  if (h->m_graph) cudaGraphDestroy(h->m_graph);
  h->h_mstate = nullptr;
  h->m_exec = nullptr;
  h->m_graph = nullptr;
  if (h->priv) cudaStreamDestroy(h->priv);
  h->h_st = nullptr;
  h->h_kkt = nullptr;
  h->h_done = nullptr;
  h->priv = nullptr;
}

int check_dims(int K, int N, int T, int n, int m) {
  if (K < 1 || N < 1 || T < 1) return fail(LQ2D_EINVAL, "K, N and T must be >= 1");
  if (n < 1 || n > kMaxN) return fail(LQ2D_EINVAL, "n must be in 1..8");
  if (m < 1 || m > kMaxM) return fail(LQ2D_EINVAL, "m must be in 1..8");
  const long long NN = (long long)K * N;
  if (NN * (T + 1) * (long long)n > (1LL << 40) || NN > (1LL << 30))
    return fail(LQ2D_EINVAL, "problem too large");
  // the sweeps keep offsets within three grid rows of a plane in 32-bit ints
  if (3LL * (N + 3) * (T + 1) > (1LL << 31) - 1) return fail(LQ2D_EINVAL, "grid rows too long (N * (T + 1))");
  return LQ2D_OK;
}

int allocate(lq2d_problem* h, int K, int N, int T, int n, int m) {
  Grid& g = h->g;
  g.K = K; g.N = N; g.T = T; g.n = n; g.m = m;
  g.V = (N + 1) / 2;
  g.NN = K * N;
  g.P = (long long)g.NN * (T + 1);
  g.Ps = round_up(g.P, 64);
  g.Pu = (long long)g.NN * T;
  g.Pus = round_up(g.Pu, 64);
  h->kt = kernel_table(n);
  if (!h->kt) return fail(LQ2D_EINVAL, "no kernels for this n");
  // n = 4 FP32 sweeps: the bulk-copy kernel (four time steps per lane) once
  // the grid has enough (column pair, time) blocks to fill the GPU with its
  // coarse tiles, else the tiled kernel
  h->sweep_steps = (long long)g.V * (T + 1) >= kBulkMinBlocks ? kSweepSteps : 0;
  LQ_CUDA(h->kt->prepare());
  LQ_CUDA(cudaStreamCreateWithFlags(&h->priv, cudaStreamNonBlocking));
  const size_t NN = g.NN, nn = (size_t)n * n;
  int rc;
#define ALLOC(ptr, cnt) \
  if ((rc = dev_alloc(h, &(ptr), (cnt))) != LQ2D_OK) return rc
  SetupBuffers& sb = h->sb;
  ALLOC(sb.Aself, NN * nn);
  ALLOC(sb.Anb, NN * 4 * nn);
  ALLOC(sb.Bm, NN * n * m);
  ALLOC(sb.Qm, NN * nn);
  ALLOC(sb.QTm, NN * nn);
  ALLOC(sb.Rm, NN * m * m);
  ALLOC(sb.x0, NN * n);
  ALLOC(sb.Qi, NN * nn);
  ALLOC(sb.QTi, NN * nn);
  ALLOC(sb.Sb, NN * nn);
  ALLOC(sb.RiBt, NN * m * n);
  ALLOC(sb.AQ, NN * 5 * nn);
  ALLOC(sb.QAt, NN * 5 * nn);
  ALLOC(sb.M13, NN * 13 * nn);
  ALLOC(sb.Om, NN * 5 * nn);
  const long long fac_rec = 28LL * n * n;  // 7 blocks of (2n)^2: [N2][N1][D^-1][E][F2][F1][L0^-1]
  const long long fac_vc = fac_rec * K;
  ALLOC(sb.fac, (size_t)g.V * 2 * fac_vc);
  if (n == 4 && K >= kTwistedMinK) {
    // the tiled sweeps (FP64, and FP32 below the bulk-copy kernel's grid
    // size) solve Phi_bar from both ends by default: half the dependent
    // chain per (column pair, time) block, twice the warps
    ALLOC(sb.fac_rev, (size_t)g.V * 2 * fac_vc);
    ALLOC(sb.iface, (size_t)g.V * 2 * 9 * (size_t)(4 * nn));
    ALLOC(sb.sinv, (size_t)g.V * 2 * 4 * (size_t)(4 * nn));
    h->twisted[0] = h->twisted[1] = 1;
    h->twisted_ready = true;  // filled by the setup that follows allocation
  }
  const size_t vec = (size_t)g.Ps * n;
  ALLOC(h->rhs, vec);
  ALLOC(h->delta, vec);
  ALLOC(h->r, vec);
  ALLOC(h->d, vec);
  ALLOC(h->y, vec);
  ALLOC(h->z, vec);
  ALLOC(h->thA, vec);
  ALLOC(h->thB, vec);
  ALLOC(h->rth, vec);
  ALLOC(h->u, (size_t)g.Pus * m);
  ALLOC(h->stage_x, (size_t)g.P * n);
  ALLOC(h->stage_u, (size_t)g.Pu * m);
  // partials: two values per block, two reductions in the KKT kernel
  const long long op_blocks = (g.P + kOpThreads - 1) / kOpThreads;
  const long long sw_blocks = (long long)g.V * (T + 1);  // at least one time step per sweep CTA
  const long long pblocks = op_blocks > sw_blocks ? op_blocks : sw_blocks;
  ALLOC(h->partials, (size_t)pblocks * 4 + 64);
  double* misc = nullptr;
  ALLOC(misc, 64);
  h->bnorm = misc;
  h->kkt_out = misc + 8;
  h->setup_status = reinterpret_cast<int*>(misc + 16);
  h->fault = h->setup_status + 1;
  h->st = reinterpret_cast<SolverState*>(misc + 24);
  static_assert(sizeof(SolverState) <= 40 * sizeof(double), "state slot");
#undef ALLOC
  LQ_CUDA(cudaMemset(misc, 0, 64 * sizeof(double) + 256));
  LQ_CUDA(cudaMemset(h->d, 0, vec * sizeof(double)));
  LQ_CUDA(cudaMallocHost(&h->h_st, sizeof(SolverState)));
  LQ_CUDA(cudaMallocHost(&h->h_kkt, 8 * sizeof(double)));
  LQ_CUDA(cudaMallocHost(&h->h_done, 2 * sizeof(int)));
  NodeData& nd = h->nd;
  nd.Aself = sb.Aself; nd.Anb = sb.Anb; nd.Bm = sb.Bm; nd.Qm = sb.Qm; nd.QTm = sb.QTm; nd.Rm = sb.Rm;
  nd.Qi = sb.Qi; nd.QTi = sb.QTi; nd.Sb = sb.Sb; nd.RiBt = sb.RiBt; nd.Om = sb.Om; nd.AQ = sb.AQ;
  nd.QAt = sb.QAt; nd.fac = sb.fac; nd.fac_rec = fac_rec; nd.fac_vc = fac_vc;
  h->pd64 = PrecData<double>{sb.fac, fac_rec, fac_vc, sb.Om, sb.AQ, sb.QAt, sb.Qm};
  h->op64 = OpData<double>{sb.Aself, sb.Anb, sb.Qi, sb.QTi, sb.Sb};
  return LQ2D_OK;
}

// Element counts of the FP32 operand copies: the preconditioner's factors,
// Omega~, AQ, QAt, Q, then the Delta product's A, E/F/G/H, Q^-1, Q_T^-1,
// B R^-1 B', and (n = 4) the records of the t = 0 factor class.
constexpr int kF32Arrays = 11;
void prec_counts(const lq2d_problem* h, long long c[kF32Arrays]) {
  const Grid& g = h->g;
  const long long nn = (long long)g.n * g.n;
  c[0] = (long long)g.V * 2 * h->nd.fac_vc;
  c[1] = (long long)g.NN * 5 * nn;
  c[2] = c[1];
  c[3] = c[1];
  c[4] = (long long)g.NN * nn;
  c[5] = (long long)g.NN * nn;
  c[6] = (long long)g.NN * 4 * nn;
  c[7] = c[5];
  c[8] = c[5];
  c[9] = c[5];
  c[10] = g.n == 4 ? (long long)g.V * g.K * h->nd.fac_rec : 0;
}

// FP32 copies of the operands for the mixed modes.
void convert_prec_f32(lq2d_problem* h, cudaStream_t s) {
  long long c[kF32Arrays];
  prec_counts(h, c);
  const double* src[kF32Arrays - 1] = {h->sb.fac, h->sb.Om, h->sb.AQ, h->sb.QAt, h->sb.Qm,
                                       h->sb.Aself, h->sb.Anb, h->sb.Qi, h->sb.QTi, h->sb.Sb};
  float* dst = h->f32_buf;
  for (int a = 0; a < kF32Arrays - 1; ++a) {
    launch_to_f32(src[a], dst, c[a], s);
    dst += c[a];
  }
  h->launches += kF32Arrays - 1;
  if (c[kF32Arrays - 1] > 0) {
    launch_t0_records(h->g, h->pd32.Qm, const_cast<float*>(h->pd32.fac_t0), h->nd.fac_rec, s);
    h->launches += 1;
  }
  if (h->fac_rev32) {
    launch_to_f32(h->sb.fac_rev, h->fac_rev32, (long long)h->g.V * 2 * h->nd.fac_vc, s);
    launch_to_f32(h->sb.sinv, h->sinv32, (long long)h->g.V * 2 * 16LL * h->g.n * h->g.n, s);
    h->launches += 2;
  }
}

// Setup on `s`: inverses, splitting blocks, factors, right-hand side and its
// norm; then waits for `s` and checks the setup status.
int run_setup(lq2d_problem* h, cudaStream_t s) {
  const Grid& g = h->g;
  LQ_CUDA(cudaMemsetAsync(h->setup_status, 0, sizeof(int), s));
  launch_setup(h->sb, g.K, g.N, g.n, g.m, g.V, h->nd.fac_rec, h->nd.fac_vc, h->setup_status, s);
  if (h->f32_buf) convert_prec_f32(h, s);
  h->mrhs_built = false;
  launch_build_rhs(g, h->sb.x0, h->w_aff, h->rhs, s);
  launch_norms(g, h->rhs, g.n, h->partials, &h->st->counters[kCntAux], h->bnorm, s);
  h->launches += 7;
  LQ_CUDA(cudaMemcpyAsync(&h->h_done[0], h->setup_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  LQ_CUDA(cudaStreamSynchronize(s));
  LQ_CUDA(cudaGetLastError());
  const int status = h->h_done[0];
  if (status & kSetupNonFinite) return fail(LQ2D_EINVAL, "non-finite input entry");
  if (status & kSetupNotPD) return fail(LQ2D_ENOTPD, "Q, Q_T or R is not positive definite");
  if (status & kSetupPhiNotPD) return fail(LQ2D_ENOTPD, "a Phi_bar block is not positive definite");
  return LQ2D_OK;
}

int copy_inputs(lq2d_problem* h, const double* const src[7], cudaMemcpyKind kind, cudaStream_t s) {
  const Grid& g = h->g;
  const size_t NN = g.NN, n = g.n, m = g.m;
  double* dst[7] = {h->sb.Aself, h->sb.Anb, h->sb.Bm, h->sb.Qm, h->sb.Rm, h->sb.QTm, h->sb.x0};
  const size_t cnt[7] = {NN * n * n, NN * 4 * n * n, NN * n * m, NN * n * n, NN * m * m, NN * n * n, NN * n};
  for (int a = 0; a < 7; ++a) {
    if (!src[a]) return fail(LQ2D_EINVAL, "null input array");
    LQ_CUDA(cudaMemcpyAsync(dst[a], src[a], cnt[a] * sizeof(double), kind, s));
  }
  return LQ2D_OK;
}

int create_common(lq2d_problem** out, int K, int N, int T, int n, int m, const double* const src[7],
                  cudaMemcpyKind kind, cudaStream_t s) {
  if (!out) return fail(LQ2D_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_dims(K, N, T, n, m);
  if (rc) return rc;
  lq2d_problem* h = new lq2d_problem();
  rc = allocate(h, K, N, T, n, m);
  if (!rc) rc = copy_inputs(h, src, kind, s);
  if (!rc) rc = run_setup(h, s);
  if (rc) {
    std::string keep = g_err;
    free_all(h);
    delete h;
    g_err = keep;
    return rc;
  }
  *out = h;
  return LQ2D_OK;
}

// Preconditioner data of the FP64 / FP32 sweeps: with the two-ended solve
// enabled for that precision (and set up), the reversed factor and the
// interface inverses ride along, which selects the two-ended kernels; the
// n = 4 FP32 bulk-copy schedules (steps >= 1) are one-sided.
PrecData<double> prec64(const lq2d_problem* h) {
  PrecData<double> p = h->pd64;
  if (h->twisted[0] && h->twisted_ready) {
    p.fac_rev = h->sb.fac_rev;
    p.sinv = h->sb.sinv;
  }
  return p;
}
PrecData<float> prec32(const lq2d_problem* h) {
  PrecData<float> p = h->pd32;
  if (h->twisted[1] && h->twisted_ready && h->fac_rev32 && !(h->g.n == 4 && h->sweep_steps >= 1)) {
    p.fac_rev = h->fac_rev32;
    p.sinv = h->sinv32;
  }
  return p;
}

// The S x L sweeps of one preconditioner application q = D_S r_in
// (Algorithm 2 from zero starts): each sweep's variant and arguments, in
// launch order.  fuse_update: the first sweep also performs the update and
// stop test of Algorithm 1; mu: the last sweep reduces mu = q' r.  The
// iterates alternate between thA and thB, so q ends in thB (S*L is even);
// its elements are double in FP64 mode and float in the mixed modes.
template <typename VT>
struct SweepPlanEntry {
  int variant;
  SweepArgsT<VT> a;
};
template <typename VT>
std::vector<SweepPlanEntry<VT>> precond_plan(lq2d_problem* h, int S, int L, bool fuse_update, bool mu,
                                             const double* r_in) {
  std::vector<SweepPlanEntry<VT>> plan;
  VT* bufs[2] = {reinterpret_cast<VT*>(h->thA), reinterpret_cast<VT*>(h->thB)};
  int out_i = 0;
  const VT* prev = nullptr;
  for (int so = 0; so < S; ++so) {
    for (int l = 0; l < L; ++l) {
      SweepArgsT<VT> a{};
      a.partials = h->partials;
      a.theta_out = bufs[out_i];
      a.y = h->y;
      a.fault = h->fault;
      int variant;
      if (l == 0 && so == 0) {
        variant = fuse_update ? kSweepUpdate : kSweepPlain;
        a.src = r_in;
        a.r = const_cast<double*>(r_in);
        a.delta = h->delta;
        a.d = h->d;
      } else if (l == 0) {
        variant = kSweepXi;
        a.src = r_in;
        a.delta_s = prev;
        a.rtheta_out = h->rth;
      } else {
        variant = (mu && so == S - 1 && l == L - 1) ? kSweepOmegaMu : kSweepOmega;
        a.src = so == 0 ? r_in : h->rth;
        a.src_rtheta = so == 0 ? 0 : 1;
        a.theta_in = prev;
        a.r = const_cast<double*>(r_in);
      }
      plan.push_back({variant, a});
      prev = bufs[out_i];
      out_i ^= 1;
    }
  }
  return plan;
}

// One preconditioner application (the plan above, launched on `s`).
// Returns the buffer holding q.
template <typename VT>
const void* enqueue_precond_t(lq2d_problem* h, int S, int L, bool fuse_update, bool mu, SolverState* st,
                              const double* r_in, cudaStream_t s, bool timing) {
  const std::vector<SweepPlanEntry<VT>> plan = precond_plan<VT>(h, S, L, fuse_update, mu, r_in);
  for (const SweepPlanEntry<VT>& e : plan) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timing) {
      const size_t k = h->ev_pool.size();
      h->ev_pool.resize(k + 2);
      cudaEventCreate(&h->ev_pool[k]);
      cudaEventCreate(&h->ev_pool[k + 1]);
      e0 = h->ev_pool[k];
      e1 = h->ev_pool[k + 1];
      cudaEventRecord(e0, s);
    }
    if constexpr (sizeof(VT) == 4)
      h->kt->sweep_f32(e.variant, h->sweep_threads[1], h->sweep_steps, h->g, prec32(h), e.a, st, s);
    else
      h->kt->sweep(e.variant, h->sweep_threads[0], h->g, prec64(h), e.a, st, s);
    h->launches += 1;
    if (timing) cudaEventRecord(e1, s);
  }
  return plan.back().a.theta_out;
}

const void* enqueue_precond(lq2d_problem* h, int S, int L, bool fuse_update, bool mu, SolverState* st,
                            const double* r_in, cudaStream_t s, bool timing) {
  if (h->precision >= 1) return enqueue_precond_t<float>(h, S, L, fuse_update, mu, st, r_in, s, timing);
  return enqueue_precond_t<double>(h, S, L, fuse_update, mu, st, r_in, s, timing);
}

// The preconditioner output q is FP32 only for the NBJM preconditioner in
// the mixed mode; the identity preconditioner copies r in FP64.
bool q_is_f32(const lq2d_problem* h) { return h->precision >= 1 && h->precond_kind == 0; }

// y = Delta dn with dn = q + beta d_old; q is the preconditioner output in
// the preconditioner's precision.
void enqueue_delta(lq2d_problem* h, const void* q, const double* dold, double* dout, double* y,
                   SolverState* st, bool loop, cudaStream_t s, bool timing) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (timing) {
    // events of the Delta apply are kept after the sweep events, tagged by parity
    const size_t k = h->ev_pool.size();
    h->ev_pool.resize(k + 2);
    cudaEventCreate(&h->ev_pool[k]);
    cudaEventCreate(&h->ev_pool[k + 1]);
    e0 = h->ev_pool[k];
    e1 = h->ev_pool[k + 1];
    cudaEventRecord(e0, s);
  }
  if (q_is_f32(h) && h->precision == 2 && loop) {
    // precision mode 2: the product inside the Krylov loop in FP32; the
    // first kernel reads the FP32 copy of d, the second writes both copies
    const float* qf = static_cast<const float*>(q);
    float* zf = reinterpret_cast<float*>(h->z);
    h->kt->delta_z_f32op(h->g, h->op32, qf, h->d32, zf, st, 1, s);
    h->kt->delta_y_f32op(h->g, h->op32, zf, qf, dold, dout, h->d32, y, h->partials, st, 1, s);
  } else if (loop && dold == dout && q_is_f32(h)) {
    // FP64 product of an FP32 preconditioner output (precision mode 1): the
    // direction update first, once per node-time, then the product of the
    // new direction, which saves converting q for every stencil neighbour
    // (in plain FP64 the fused form is faster: measured 5.28 against 5.55 ms
    // per product on the 256 x 256 x 200 grid)
    launch_direction_update(h->g, q, q_is_f32(h), dout, st, s);
    h->kt->delta_z(h->g, h->op64, dout, nullptr, h->z, st, 1, s);
    h->kt->delta_y(h->g, h->op64, h->z, dout, nullptr, nullptr, y, h->partials, st, 1, s);
    h->launches += 1;
  } else if (q_is_f32(h)) {
    const float* qf = static_cast<const float*>(q);
    h->kt->delta_z_f32(h->g, h->op64, qf, dold, h->z, st, loop ? 1 : 0, s);
    h->kt->delta_y_f32(h->g, h->op64, h->z, qf, dold, dout, y, h->partials, st, loop ? 1 : 0, s);
  } else {
    const double* qd = static_cast<const double*>(q);
    h->kt->delta_z(h->g, h->op64, qd, dold, h->z, st, loop ? 1 : 0, s);
    h->kt->delta_y(h->g, h->op64, h->z, qd, dold, dout, y, h->partials, st, loop ? 1 : 0, s);
  }
  h->launches += 2;
  if (timing) cudaEventRecord(e1, s);
}

// One PCG step (Algorithm 1, operator product to next direction): y = Delta d with d = q + beta d
// fused in, then the preconditioner with the update fused into its first
// sweep and mu into its last.
void enqueue_step(lq2d_problem* h, int S, int L, cudaStream_t s, bool timing) {
  enqueue_delta(h, h->thB, h->d, h->d, h->y, h->st, true, s, timing);
  if (h->precond_kind == 1) {
    cudaEvent_t e1 = nullptr;
    if (timing) {
      const size_t k = h->ev_pool.size();
      h->ev_pool.resize(k + 2);
      cudaEventCreate(&h->ev_pool[k]);
      cudaEventCreate(&h->ev_pool[k + 1]);
      cudaEventRecord(h->ev_pool[k], s);
      e1 = h->ev_pool[k + 1];
    }
    launch_ident(h->g, true, h->r, h->delta, h->y, h->d, h->thB, h->partials, h->st, s);
    h->launches += 1;
    if (timing) cudaEventRecord(e1, s);
    return;
  }
  enqueue_precond(h, S, L, true, true, h->st, h->r, s, timing);
  if (h->precision == 2) {
    // reliable update: when this step's residual has dropped by kPhaseRho
    // since the last replacement, r = r_delta - Delta delta in FP64 replaces
    // the recurrence residual (the three kernels return at once otherwise);
    // d, q and mu of the step are kept
    h->kt->delta_z(h->g, h->op64, h->delta, nullptr, h->z, h->st, 2, s);
    h->kt->delta_y(h->g, h->op64, h->z, h->delta, nullptr, nullptr, h->y, h->partials, h->st, 0, s);
    launch_replace_residual(h->g, h->rhs, h->y, h->r, h->partials, h->st, s);
    h->launches += 3;
  }
}

// CTA width of the sweeps the current precision mode launches, and the rest
// of its schedule (time steps per lane of the n = 4 FP32 sweeps, two-ended
// solve), which captured graphs depend on.
int current_threads(const lq2d_problem* h) { return h->sweep_threads[h->precision >= 1 ? 1 : 0]; }
int current_steps(const lq2d_problem* h) { return h->precision >= 1 ? h->sweep_steps : 0; }
int current_twisted(const lq2d_problem* h) { return h->twisted[h->precision >= 1 ? 1 : 0] && h->twisted_ready; }

int sweeps_per_step(const lq2d_problem* h, int S, int L) { return h->precond_kind == 1 ? 1 : S * L; }

int get_graph(lq2d_problem* h, int S, int L, cudaGraphExec_t* exec) {
  for (int i = 0; i < h->ngraphs; ++i)
    if (h->graphs[i].S == S && h->graphs[i].L == L && h->graphs[i].precision == h->precision &&
        h->graphs[i].precond == h->precond_kind && h->graphs[i].threads == current_threads(h) &&
        h->graphs[i].steps == current_steps(h) && h->graphs[i].twisted == current_twisted(h)) {
      *exec = h->graphs[i].exec;
      return LQ2D_OK;
    }
  if (h->ngraphs == kMaxGraphs) {
    cudaGraphExecDestroy(h->graphs[0].exec);
    cudaGraphDestroy(h->graphs[0].graph);
    for (int i = 1; i < kMaxGraphs; ++i) h->graphs[i - 1] = h->graphs[i];
    h->ngraphs--;
  }
  GraphEntry ge;
  ge.S = S;
  ge.L = L;
  ge.precision = h->precision;
  ge.precond = h->precond_kind;
  ge.threads = current_threads(h);
  ge.steps = current_steps(h);
  ge.twisted = current_twisted(h);
  LQ_CUDA(cudaGraphCreate(&ge.graph, 0));
  cudaGraphConditionalHandle hc;
  LQ_CUDA(cudaGraphConditionalHandleCreate(&hc, ge.graph, 1u, cudaGraphCondAssignDefault));
  // zero-initialised storage: the struct's union has no default constructor
  alignas(cudaGraphNodeParams) unsigned char cp_storage[sizeof(cudaGraphNodeParams)];
  std::memset(cp_storage, 0, sizeof(cp_storage));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_storage);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  LQ_CUDA(cudaGraphAddNode(&node, ge.graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  LQ_CUDA(cudaStreamBeginCaptureToGraph(h->priv, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const long long before = h->launches;
  enqueue_step(h, S, L, h->priv, false);
  h->launches = before;  // captured, not launched: body executions are counted after each solve
  launch_loop_ctrl(h->st, hc, h->priv);
  cudaGraph_t captured = nullptr;
  cudaError_t ce = cudaStreamEndCapture(h->priv, &captured);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(ge.graph);
    return fail(LQ2D_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  }
  ce = cudaGraphInstantiate(&ge.exec, ge.graph, 0);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(ge.graph);
    return fail(LQ2D_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
  }
  h->graphs[h->ngraphs++] = ge;
  *exec = ge.exec;
  return LQ2D_OK;
}

// Driver 1: steps enqueued from the host in chunks; the stop flag of the
// previous chunk is read while the current one runs.  Kernels return at
// once when the flag is set, so the overshoot costs only empty launches.
template <typename Step>
int run_host_loop(lq2d_problem* h, int max_iter, cudaStream_t s, Step&& enqueue_one) {
  const int cap = max_iter + 2;
  int enq = 0;
  cudaEvent_t flag_ev[2];
  LQ_CUDA(cudaEventCreateWithFlags(&flag_ev[0], cudaEventDisableTiming));
  LQ_CUDA(cudaEventCreateWithFlags(&flag_ev[1], cudaEventDisableTiming));
  int slot = 0;
  bool pending[2] = {false, false};
  int rc = LQ2D_OK;
  while (enq < cap) {
    for (int c = 0; c < kStreamChunk && enq < cap; ++c, ++enq) enqueue_one();
    cudaMemcpyAsync(&h->h_done[slot], &h->st->done, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaEventRecord(flag_ev[slot], s);
    pending[slot] = true;
    slot ^= 1;
    if (pending[slot]) {
      cudaEventSynchronize(flag_ev[slot]);
      pending[slot] = false;
      if (h->h_done[slot] != 0) break;
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) rc = fail(LQ2D_ECUDA, std::string("stream loop: ") + cudaGetErrorString(e));
  cudaEventDestroy(flag_ev[0]);
  cudaEventDestroy(flag_ev[1]);
  return rc;
}

int run_loop(lq2d_problem* h, int S, int L, int max_iter, cudaStream_t s) {
  const bool use_stream = h->driver == 1 || h->timing;
  if (!use_stream) {
    cudaGraphExec_t exec;
    int rc = get_graph(h, S, L, &exec);
    if (rc) return rc;
    LQ_CUDA(cudaGraphLaunch(exec, s));
    h->graph_body_kernels = 2 + sweeps_per_step(h, S, L) + 1;
    return LQ2D_OK;
  }
  return run_host_loop(h, max_iter, s, [&]() { enqueue_step(h, S, L, s, h->timing != 0); });
}


// Sums the event pairs of the timed steps.  Pool order per step: one pair
// around the Delta apply, then S*L pairs around the sweeps.  Only launches
// that did work are counted: in the step that met the stop test the sweeps
// after the first return at once, and later steps are empty.
void collect_timing(lq2d_problem* h, int sweeps, int steps_done) {
  const size_t per = 2 + 2 * (size_t)sweeps;
  const size_t steps = h->ev_pool.size() / per;
  for (size_t k = 0; k < steps && (int)k < steps_done; ++k) {
    const size_t b = k * per;
    const bool last = (int)k == steps_done - 1;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[b], h->ev_pool[b + 1]) == cudaSuccess) {
      h->stats.delta_ms += ms;
      h->stats.delta_launches += 1;
    }
    const size_t nsw = last ? 1 : (size_t)sweeps;
    for (size_t w = 0; w < nsw; ++w) {
      if (cudaEventElapsedTime(&ms, h->ev_pool[b + 2 + 2 * w], h->ev_pool[b + 3 + 2 * w]) == cudaSuccess) {
        h->stats.sweep_ms += ms;
        h->stats.sweep_launches += 1;
      }
    }
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear();
}

// Number of eigenvalues of the symmetric tridiagonal (d, e2 = squared
// off-diagonal) below x (Sturm sequence).
int sturm_below(const std::vector<double>& d, const std::vector<double>& e2, double x) {
  int c = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    q = d[i] - x - (i ? e2[i - 1] / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++c;
  }
  return c;
}

// k-th smallest eigenvalue by bisection inside [lo, hi].
double tridiag_eig(const std::vector<double>& d, const std::vector<double>& e2, int k, double lo, double hi) {
  for (int it = 0; it < 200 && hi - lo > 1e-13 * std::max(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_below(d, e2, mid) > k) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Extreme Ritz values of the preconditioned operator from the recorded PCG
// coefficients: the Lanczos matrix has diagonal 1/a_0, 1/a_j + b_{j-1}/a_{j-1}
// and off-diagonal sqrt(b_j)/a_j (CG-Lanczos relation; the paper reports
// kappa(P_S^-1/2 Delta P_S^-1/2) in Section V).
void lanczos_estimate(lq2d_problem* h, int iterations, cudaStream_t s) {
  const int m = std::min(iterations, kHistCap);
  h->stats.kappa_estimate = 0.0;
  h->stats.lambda_min = 0.0;
  h->stats.lambda_max = 0.0;
  if (m < 1) return;
  h->h_hist.assign(2 * (size_t)m, 0.0);
  if (cudaMemcpyAsync(h->h_hist.data(), h->hist, 2 * (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return;
  std::vector<double> d(m), e2(m > 1 ? m - 1 : 0);
  for (int j = 0; j < m; ++j) {
    const double a = h->h_hist[2 * j];
    d[j] = 1.0 / a;
    if (j > 0) {
      const double ap = h->h_hist[2 * (j - 1)], bp = h->h_hist[2 * (j - 1) + 1];
      d[j] += bp / ap;
      e2[j - 1] = bp / (ap * ap);
    }
  }
  double lo = d[0], hi = d[0];
  for (int j = 0; j < m; ++j) {
    const double r = (j > 0 ? std::sqrt(e2[j - 1]) : 0.0) + (j + 1 < m ? std::sqrt(e2[j]) : 0.0);
    lo = std::min(lo, d[j] - r);
    hi = std::max(hi, d[j] + r);
  }
  const double lmin = tridiag_eig(d, e2, 0, lo, hi);
  const double lmax = tridiag_eig(d, e2, m - 1, lo, hi);
  h->stats.lambda_min = lmin;
  h->stats.lambda_max = lmax;
  h->stats.kappa_estimate = lmin > 0.0 ? lmax / lmin : 0.0;
}

// The full solve on device buffers (host layout), ordered on s.
int solve_impl(lq2d_problem* h, double tol, int S, int L, int max_iter, const double* d_delta0, double* d_x,
               double* d_u, double* d_costate, int* iterations, double* rel_kkt, cudaStream_t s) {
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(LQ2D_EINVAL, "tol must be positive and finite");
  if (S < 1) return fail(LQ2D_EINVAL, "outer_S must be >= 1");
  if (L < 2 || (L & 1)) return fail(LQ2D_EINVAL, "inner_L must be even and >= 2 (Theorem posdef_preconditioner)");
  if (max_iter < 0) return fail(LQ2D_EINVAL, "max_iter must be >= 0");
  const Grid& g = h->g;
  const KernelTable* kt = h->kt;
  std::memset(&h->stats, 0, sizeof(h->stats));
  h->ev_pool.clear();
  if (h->kappa && !h->hist) {
    int rc = dev_alloc(h, &h->hist, 2 * (size_t)kHistCap);
    if (rc) return rc;
  }
  const double phase_rho2 = h->precision == 2 ? kPhaseRho * kPhaseRho : 0.0;
  const int max_restarts = h->max_restarts;
  launch_init_state(h->st, tol, max_iter, h->stop_mode, h->bnorm, 0, h->kappa ? h->hist : nullptr, kHistCap,
                    phase_rho2, s);
  h->launches += 2;  // state and initial residual
  if (d_delta0) {
    h->launches += 3;
    launch_to_internal(d_delta0, h->thA, g.NN, g.T + 1, g.n, g.Ps, s);
    kt->delta_z(g, h->op64, h->thA, nullptr, h->z, nullptr, 0, s);
    kt->delta_y(g, h->op64, h->z, h->thA, nullptr, nullptr, h->y, h->partials, nullptr, 0, s);
    launch_init_residual(g, h->rhs, h->y, h->r, h->delta, h->thA, h->partials, h->st, s);
  } else {
    launch_init_residual(g, h->rhs, nullptr, h->r, h->delta, nullptr, h->partials, h->st, s);
  }
  int restarts = 0;
  int status = LQ2D_OK;
  double rel = 0.0;
  int iter_before = 0;
  for (;;) {
    if (h->precond_kind == 1) {
      launch_ident(g, false, h->r, h->delta, h->y, h->d, h->thB, h->partials, h->st, s);
      h->launches += 1;
    } else {
      enqueue_precond(h, S, L, false, true, h->st, h->r, s, false);
    }
    LQ_CUDA(cudaMemsetAsync(h->d, 0, (size_t)g.Ps * g.n * sizeof(double), s));
    h->graph_body_kernels = 0;
    int rc = run_loop(h, S, L, max_iter, s);
    if (rc) return rc;
    h->launches += 3;  // recovery
    // recovery (Section II-B): x = Q~^-1 A~' delta into z, u = R~^-1 B~' delta,
    // and the full KKT residual of (x, u, delta)
    kt->delta_z(g, h->op64, h->delta, nullptr, h->z, nullptr, 0, s);
    launch_recover_u(g, h->nd, h->delta, h->u, s);
    kt->kkt(g, h->nd, h->z, h->u, h->delta, h->rhs, h->partials, h->st, h->kkt_out, s);
    LQ_CUDA(cudaMemcpyAsync(h->h_st, h->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    LQ_CUDA(cudaMemcpyAsync(h->h_kkt, h->kkt_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    LQ_CUDA(cudaStreamSynchronize(s));
    LQ_CUDA(cudaGetLastError());
    const SolverState& hs = *h->h_st;
    h->launches += (long long)hs.body_count * h->graph_body_kernels;
    if (h->timing) collect_timing(h, sweeps_per_step(h, S, L), hs.iter - iter_before);
    iter_before = hs.iter;
    const double bn = std::sqrt(hs.bnorm2);
    rel = bn > 0 ? std::sqrt(h->h_kkt[0]) / bn : std::sqrt(h->h_kkt[0]);
    const bool true_pass = h->stop_mode == 0 ? (rel <= tol || h->h_kkt[0] == 0.0) : (h->h_kkt[2] < tol);
    if (hs.done == kConverged && !true_pass && restarts < max_restarts && hs.iter < max_iter) {
      // the recurrence residual passed but the true one did not: restart
      // from the current iterate with r = r_delta - Delta delta
      ++restarts;
      h->launches += 4;
      launch_init_state(h->st, tol, max_iter, h->stop_mode, h->bnorm, 1, nullptr, 0, phase_rho2, s);
      kt->delta_z(g, h->op64, h->delta, nullptr, h->z, nullptr, 0, s);
      kt->delta_y(g, h->op64, h->z, h->delta, nullptr, nullptr, h->y, h->partials, nullptr, 0, s);
      launch_init_residual(g, h->rhs, h->y, h->r, h->delta, h->delta, h->partials, h->st, s);
      continue;
    }
    switch (hs.done) {
      case kConverged: status = true_pass ? LQ2D_OK : LQ2D_ENOCONV; break;
      case kMaxIter: status = LQ2D_ENOCONV; break;
      case kBreakdown: status = LQ2D_EBREAKDOWN; break;
      case kLoopCap: status = LQ2D_ETIMEOUT; break;
      default: status = LQ2D_ECUDA; break;
    }
    h->stats.iterations = hs.iter;
    h->stats.restarts = restarts;
    h->stats.residual_replacements = hs.replacements;
    h->stats.rel_residual = bn > 0 ? std::sqrt(hs.rnorm2) / bn : std::sqrt(hs.rnorm2);
    h->stats.rel_kkt_residual = rel;
    h->stats.kkt_inf = h->h_kkt[2];
    h->stats.cost = 0.5 * h->h_kkt[1];
    h->stats.status = status;
    h->stats.body_executions = hs.body_count;
    if (h->kappa) lanczos_estimate(h, hs.iter, s);
    break;
  }
  if (d_x) launch_to_api(h->z, d_x, g.NN, g.T + 1, g.n, g.Ps, s);
  if (d_u) launch_to_api(h->u, d_u, g.NN, g.T, g.m, g.Pus, s);
  if (d_costate) launch_to_api(h->delta, d_costate, g.NN, g.T + 1, g.n, g.Ps, s);
  h->launches += (d_x != nullptr) + (d_u != nullptr) + (d_costate != nullptr);
  LQ_CUDA(cudaStreamSynchronize(s));
  LQ_CUDA(cudaGetLastError());
  if (iterations) *iterations = h->stats.iterations;
  if (rel_kkt) *rel_kkt = rel;
  if (status == LQ2D_ENOCONV) return fail(status, "max_iter reached before the tolerance");
  if (status == LQ2D_EBREAKDOWN) return fail(status, "breakdown: y'd <= 0 or a non-finite scalar");
  if (status == LQ2D_ETIMEOUT) return fail(status, "device loop cap reached");
  if (status != LQ2D_OK) return fail(status, "solver state not set");
  return LQ2D_OK;
}

// Buffer that holds delta^(s) after `steps` outer steps of the standalone
// NBJM solver (-1: none yet, delta^(0) = 0).  Buffers 0..2 rotate: each step
// writes its L sweeps alternately into the two buffers other than the
// current iterate, the last one into the second of them.
int nbjm_buffer_after(int steps, int L) {
  int cur = -1;
  for (int k = 0; k < steps; ++k) {
    int others[2];
    int c = 0;
    for (int b = 0; b < 3 && c < 2; ++b)
      if (b != cur) others[c++] = b;
    cur = others[(L - 1) & 1];
  }
  return cur;
}

// One outer step of Algorithm 2 as a solver: L sweeps, the first started
// from the outer iterate (tau = r_delta + Xi~ delta + Omega~ delta, reading
// A22), then the exit test on ||delta^(s+1) - delta^(s)||_inf.
template <typename VT>
void enqueue_nbjm_outer(lq2d_problem* h, int L, int step, cudaStream_t s) {
  VT* B[3] = {reinterpret_cast<VT*>(h->thA), reinterpret_cast<VT*>(h->thB), reinterpret_cast<VT*>(h->z)};
  const int cur = nbjm_buffer_after(step, L);
  int others[2];
  int c = 0;
  for (int b = 0; b < 3 && c < 2; ++b)
    if (b != cur) others[c++] = b;
  const VT* prev = nullptr;
  for (int l = 0; l < L; ++l) {
    SweepArgsT<VT> a{};
    a.partials = h->partials;
    a.theta_out = B[others[l & 1]];
    a.y = h->y;
    a.r = h->rhs;
    a.fault = h->fault;
    int variant;
    if (l == 0 && cur < 0) {
      variant = kSweepPlain;
      a.src = h->rhs;
    } else if (l == 0) {
      variant = kSweepXiOmega;
      a.src = h->rhs;
      a.delta_s = B[cur];
      a.theta_in = B[cur];
      a.rtheta_out = h->rth;
    } else {
      variant = kSweepOmega;
      a.src = cur < 0 ? h->rhs : h->rth;
      a.src_rtheta = cur < 0 ? 0 : 1;
      a.theta_in = prev;
    }
    if constexpr (sizeof(VT) == 4)
      h->kt->sweep_f32(variant, h->sweep_threads[1], h->sweep_steps, h->g, prec32(h), a, h->st, s);
    else
      h->kt->sweep(variant, h->sweep_threads[0], h->g, prec64(h), a, h->st, s);
    prev = B[others[l & 1]];
  }
  launch_nbjm_diff(h->g, prev, cur < 0 ? nullptr : B[cur], sizeof(VT) == 4, h->partials, h->st, s);
  h->launches += L + 1;
}

int solve_nbjm_impl(lq2d_problem* h, double eps, int L, int max_outer, double* d_x, double* d_u,
                    double* d_costate, int* outer, double* rel_kkt, cudaStream_t s) {
  if (!(eps > 0.0) || !std::isfinite(eps)) return fail(LQ2D_EINVAL, "eps must be positive and finite");
  if (L < 1) return fail(LQ2D_EINVAL, "inner_L must be >= 1");
  if (max_outer < 1) return fail(LQ2D_EINVAL, "max_outer must be >= 1");
  const Grid& g = h->g;
  const bool f32 = h->precision >= 1;
  std::memset(&h->stats, 0, sizeof(h->stats));
  launch_init_state(h->st, eps, max_outer, 1, h->bnorm, 0, nullptr, 0, 0.0, s);
  h->launches += 1;
  cudaEvent_t flag_ev[2];
  LQ_CUDA(cudaEventCreateWithFlags(&flag_ev[0], cudaEventDisableTiming));
  LQ_CUDA(cudaEventCreateWithFlags(&flag_ev[1], cudaEventDisableTiming));
  bool pending[2] = {false, false};
  int slot = 0, enq = 0;
  while (enq < max_outer) {
    for (int c = 0; c < kStreamChunk * 4 && enq < max_outer; ++c, ++enq) {
      if (f32) enqueue_nbjm_outer<float>(h, L, enq, s);
      else enqueue_nbjm_outer<double>(h, L, enq, s);
    }
    cudaMemcpyAsync(&h->h_done[slot], &h->st->done, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaEventRecord(flag_ev[slot], s);
    pending[slot] = true;
    slot ^= 1;
    if (pending[slot]) {
      cudaEventSynchronize(flag_ev[slot]);
      pending[slot] = false;
      if (h->h_done[slot] != 0) break;
    }
  }
  cudaEventDestroy(flag_ev[0]);
  cudaEventDestroy(flag_ev[1]);
  LQ_CUDA(cudaMemcpyAsync(h->h_st, h->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
  LQ_CUDA(cudaStreamSynchronize(s));
  LQ_CUDA(cudaGetLastError());
  const int steps = h->h_st->iter;
  const int done = h->h_st->done;
  const int buf = nbjm_buffer_after(steps, L);
  double* B64[3] = {h->thA, h->thB, h->z};
  if (buf >= 0) {
    if (f32) launch_iter_f32_to_f64(g, reinterpret_cast<const float*>(B64[buf]), h->delta, s);
    else LQ_CUDA(cudaMemcpyAsync(h->delta, B64[buf], (size_t)g.Ps * g.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    LQ_CUDA(cudaMemsetAsync(h->delta, 0, (size_t)g.Ps * g.n * sizeof(double), s));
  }
  // recovery (Section II-B) and the true KKT residual of the result
  h->kt->delta_z(g, h->op64, h->delta, nullptr, h->z, nullptr, 0, s);
  launch_recover_u(g, h->nd, h->delta, h->u, s);
  h->kt->kkt(g, h->nd, h->z, h->u, h->delta, h->rhs, h->partials, h->st, h->kkt_out, s);
  h->launches += 3 + (f32 ? 1 : 0);
  LQ_CUDA(cudaMemcpyAsync(h->h_kkt, h->kkt_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (d_x) launch_to_api(h->z, d_x, g.NN, g.T + 1, g.n, g.Ps, s);
  if (d_u) launch_to_api(h->u, d_u, g.NN, g.T, g.m, g.Pus, s);
  if (d_costate) launch_to_api(h->delta, d_costate, g.NN, g.T + 1, g.n, g.Ps, s);
  h->launches += (d_x != nullptr) + (d_u != nullptr) + (d_costate != nullptr);
  LQ_CUDA(cudaStreamSynchronize(s));
  LQ_CUDA(cudaGetLastError());
  const double bn = std::sqrt(h->h_st->bnorm2);
  const double rel = bn > 0 ? std::sqrt(h->h_kkt[0]) / bn : std::sqrt(h->h_kkt[0]);
  h->stats.outer_iterations = steps;
  h->stats.rel_kkt_residual = rel;
  h->stats.kkt_inf = h->h_kkt[2];
  h->stats.cost = 0.5 * h->h_kkt[1];
  h->stats.rel_residual = h->h_st->rnorm_inf;  // last change ||delta^(s+1) - delta^(s)||_inf
  if (outer) *outer = steps;
  if (rel_kkt) *rel_kkt = rel;
  int status = done == kConverged ? LQ2D_OK : done == kMaxIter ? LQ2D_ENOCONV : LQ2D_EBREAKDOWN;
  h->stats.status = status;
  if (status == LQ2D_ENOCONV) return fail(status, "max_outer reached before the exit test passed");
  if (status == LQ2D_EBREAKDOWN) return fail(status, "non-finite iterate");
  return LQ2D_OK;
}

// The part of a solve before the device loop: state, r^(0) = r_delta,
// q = P^-1 r^(0) with mu, d = 0 (the start of Algorithm 1).
void enqueue_solve_init(lq2d_problem* h, double tol, int S, int L, int max_iter, cudaStream_t s) {
  const Grid& g = h->g;
  const double phase_rho2 = h->precision == 2 ? kPhaseRho * kPhaseRho : 0.0;
  launch_init_state(h->st, tol, max_iter, h->stop_mode, h->bnorm, 0, nullptr, 0, phase_rho2, s);
  launch_init_residual(g, h->rhs, nullptr, h->r, h->delta, nullptr, h->partials, h->st, s);
  if (h->precond_kind == 1) launch_ident(g, false, h->r, h->delta, h->y, h->d, h->thB, h->partials, h->st, s);
  else enqueue_precond(h, S, L, false, true, h->st, h->r, s, false);
  cudaMemsetAsync(h->d, 0, (size_t)g.Ps * g.n * sizeof(double), s);
}

// Recovery (Section II-B) and the copy of the state and KKT figures into
// the batch result slot.
void enqueue_solve_finish(lq2d_problem* h, double* slot, cudaStream_t s) {
  const Grid& g = h->g;
  h->kt->delta_z(g, h->op64, h->delta, nullptr, h->z, nullptr, 0, s);
  launch_recover_u(g, h->nd, h->delta, h->u, s);
  h->kt->kkt(g, h->nd, h->z, h->u, h->delta, h->rhs, h->partials, h->st, h->kkt_out, s);
  cudaMemcpyAsync(slot, h->st, sizeof(SolverState), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(slot + 24, h->kkt_out, 4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

// The per-problem settings a captured batch graph depends on.
int batch_mode_key(const lq2d_problem* h) {
  const int sched = (current_threads(h) * 8 + current_steps(h)) * 2 + current_twisted(h);
  return ((sched * 4 + h->precision) * 4 + h->precond_kind) * 4 + h->stop_mode;
}

// The persistent batched loop serves FP64 NBJM problems with n = 4, S x L
// sweeps that fit the queue heads.
bool batch_persistent_ok(const lq2d_batch* b, int S, int L) {
  if (!b->persistent || S * L + 2 > kBatchHeads) return false;
  for (const lq2d_problem* h : b->probs)
    if (h->g.n != 4 || h->precision != 0 || h->precond_kind != 0) return false;
  return true;
}

// Uploads the batch plan (problem descriptors, unit offsets, the arguments
// of every sweep of a loop step and of a plain D_S application) for the
// batch's CTA width; sets the persistent grid sizes.
int batch_plan_upload(lq2d_batch* b, int S, int L, cudaStream_t s) {
  const int np = (int)b->probs.size();
  const int SL = S * L;
  std::vector<BatchProblem> probs(np);
  std::vector<int> soff(np + 1, 0);
  std::vector<long long> ooff(np + 1, 0);
  std::vector<SweepArgsT<double>> args((size_t)2 * SL * np);
  b->variants.assign(2 * SL, 0);
  for (int i = 0; i < np; ++i) {
    lq2d_problem* h = b->probs[i];
    BatchProblem& P = probs[i];
    P.g = h->g;
    P.op = h->op64;
    P.pd = h->pd64;
    P.st = h->st;
    P.partials = h->partials;
    P.q = h->thB;
    P.d = h->d;
    P.y = h->y;
    P.z = h->z;
    soff[i + 1] = soff[i] + batch_sweep_units(h->g, b->threads);
    ooff[i + 1] = ooff[i] + (h->g.P + kOpThreads - 1) / kOpThreads;
    const std::vector<SweepPlanEntry<double>> loop = precond_plan<double>(h, S, L, true, true, h->r);
    const std::vector<SweepPlanEntry<double>> plain = precond_plan<double>(h, S, L, false, false, h->rhs);
    for (int k = 0; k < SL; ++k) {
      args[(size_t)k * np + i] = loop[k].a;
      args[(size_t)(SL + k) * np + i] = plain[k].a;
      b->variants[k] = loop[k].variant;
      b->variants[SL + k] = plain[k].variant;
    }
  }
  auto up = [](size_t v) { return (v + 255) / 256 * 256; };
  const size_t o_probs = 0, o_soff = up(np * sizeof(BatchProblem)), o_ooff = o_soff + up((np + 1) * sizeof(int)),
               o_args = o_ooff + up((np + 1) * sizeof(long long)),
               o_heads = o_args + up(args.size() * sizeof(SweepArgsT<double>)),
               total = o_heads + up((kBatchHeads + 1) * sizeof(unsigned));
  if (total > b->plan_bytes) {
    if (b->plan_mem) cudaFree(b->plan_mem);
    b->plan_mem = nullptr;
    b->plan_bytes = 0;
    cudaError_t e = cudaMalloc(&b->plan_mem, total);
    if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? LQ2D_ENOMEM : LQ2D_ECUDA, cudaGetErrorString(e));
    b->plan_bytes = total;
  }
  char* base = static_cast<char*>(b->plan_mem);
  BatchPlan& pl = b->plan;
  pl.probs = reinterpret_cast<BatchProblem*>(base + o_probs);
  pl.sweep_off = reinterpret_cast<int*>(base + o_soff);
  pl.op_off = reinterpret_cast<long long*>(base + o_ooff);
  pl.args = reinterpret_cast<SweepArgsT<double>*>(base + o_args);
  pl.heads = reinterpret_cast<unsigned*>(base + o_heads);
  pl.nprob = np;
  pl.threads = b->threads;
  LQ_CUDA(cudaMemcpyAsync(pl.probs, probs.data(), np * sizeof(BatchProblem), cudaMemcpyHostToDevice, s));
  LQ_CUDA(cudaMemcpyAsync(pl.sweep_off, soff.data(), (np + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  LQ_CUDA(cudaMemcpyAsync(pl.op_off, ooff.data(), (np + 1) * sizeof(long long), cudaMemcpyHostToDevice, s));
  LQ_CUDA(cudaMemcpyAsync(pl.args, args.data(), args.size() * sizeof(SweepArgsT<double>), cudaMemcpyHostToDevice, s));
  LQ_CUDA(cudaMemsetAsync(pl.heads, 0, (kBatchHeads + 1) * sizeof(unsigned), s));
  LQ_CUDA(cudaStreamSynchronize(s));
  LQ_CUDA(batch_grid_sizes(pl));
  return LQ2D_OK;
}

// The persistent graph: every problem's initial part (independent), one
// conditional while node whose body is the batched step (Delta product, the
// S x L sweeps, loop control), then every problem's recovery.
int batch_build_persistent(lq2d_batch* b, double tol, int S, int L, int max_iter) {
  int rc = batch_plan_upload(b, S, L, b->cap);
  if (rc) return rc;
  cudaGraph_t root = b->graph;
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  std::vector<cudaGraphNode_t> tails;
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaGraph_t captured = nullptr;
  LQ_CUDA(cudaStreamBeginCaptureToGraph(b->cap, root, nullptr, nullptr, 0, mode));
  LQ_CUDA(cudaMemsetAsync(b->plan.heads, 0, (kBatchHeads + 1) * sizeof(unsigned), b->cap));
  LQ_CUDA(cudaStreamGetCaptureInfo(b->cap, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
  tails.insert(tails.end(), deps, deps + ndeps);
  LQ_CUDA(cudaStreamEndCapture(b->cap, &captured));
  for (lq2d_problem* h : b->probs) {
    LQ_CUDA(cudaStreamBeginCaptureToGraph(b->cap, root, nullptr, nullptr, 0, mode));
    const long long before = h->launches;
    enqueue_solve_init(h, tol, S, L, max_iter, b->cap);
    h->launches = before;
    LQ_CUDA(cudaStreamGetCaptureInfo(b->cap, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
    tails.insert(tails.end(), deps, deps + ndeps);
    LQ_CUDA(cudaStreamEndCapture(b->cap, &captured));
  }
  cudaGraphConditionalHandle hc;
  LQ_CUDA(cudaGraphConditionalHandleCreate(&hc, root, 1u, cudaGraphCondAssignDefault));
  alignas(cudaGraphNodeParams) unsigned char cp_storage[sizeof(cudaGraphNodeParams)];
  std::memset(cp_storage, 0, sizeof(cp_storage));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_storage);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  LQ_CUDA(cudaGraphAddNode(&cnode, root, tails.data(), nullptr, tails.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const int SL = S * L;
  LQ_CUDA(cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0, mode));
  batch_enqueue_delta(b->plan, 0, b->cap);
  for (int k = 0; k < SL; ++k) batch_enqueue_sweep(b->plan, b->variants[k], k, 2 + k, b->cap);
  batch_enqueue_loop_ctrl(b->plan, hc, b->cap);
  LQ_CUDA(cudaStreamEndCapture(b->cap, &captured));
  for (size_t i = 0; i < b->probs.size(); ++i) {
    LQ_CUDA(cudaStreamBeginCaptureToGraph(b->cap, root, &cnode, nullptr, 1, mode));
    enqueue_solve_finish(b->probs[i], b->results + i * kBatchSlot, b->cap);
    LQ_CUDA(cudaStreamEndCapture(b->cap, &captured));
  }
  b->built_persistent = true;
  return LQ2D_OK;
}

int batch_build(lq2d_batch* b, double tol, int S, int L, int max_iter) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  static_assert(sizeof(SolverState) <= 24 * sizeof(double), "batch slot");
  cudaGraph_t root;
  LQ_CUDA(cudaGraphCreate(&root, 0));
  b->graph = root;
  b->built_persistent = false;
  if (batch_persistent_ok(b, S, L)) {
    int rc = batch_build_persistent(b, tol, S, L, max_iter);
    if (rc) return rc;
  }
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  for (size_t i = 0; !b->built_persistent && i < b->probs.size(); ++i) {
    lq2d_problem* h = b->probs[i];
    // initial part, appended to the root graph with no dependency
    LQ_CUDA(cudaStreamBeginCaptureToGraph(b->cap, root, nullptr, nullptr, 0, mode));
    const long long before = h->launches;
    enqueue_solve_init(h, tol, S, L, max_iter, b->cap);
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    LQ_CUDA(cudaStreamGetCaptureInfo(b->cap, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
    std::vector<cudaGraphNode_t> tail(deps, deps + ndeps);
    cudaGraph_t captured = nullptr;
    LQ_CUDA(cudaStreamEndCapture(b->cap, &captured));
    // the device loop under a conditional while node
    cudaGraphConditionalHandle hc;
    LQ_CUDA(cudaGraphConditionalHandleCreate(&hc, root, 1u, cudaGraphCondAssignDefault));
    alignas(cudaGraphNodeParams) unsigned char cp_storage[sizeof(cudaGraphNodeParams)];
    std::memset(cp_storage, 0, sizeof(cp_storage));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_storage);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    LQ_CUDA(cudaGraphAddNode(&cnode, root, tail.data(), nullptr, tail.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    LQ_CUDA(cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0, mode));
    enqueue_step(h, S, L, b->cap, false);
    launch_loop_ctrl(h->st, hc, b->cap);
    LQ_CUDA(cudaStreamEndCapture(b->cap, &captured));
    // recovery after the loop
    LQ_CUDA(cudaStreamBeginCaptureToGraph(b->cap, root, &cnode, nullptr, 1, mode));
    enqueue_solve_finish(h, b->results + i * kBatchSlot, b->cap);
    LQ_CUDA(cudaStreamEndCapture(b->cap, &captured));
    h->launches = before;  // captured, not launched: counted per batch solve
  }
  cudaError_t e = cudaGraphInstantiate(&b->exec, root, 0);
  if (e != cudaSuccess) return fail(LQ2D_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
  b->tol = tol;
  b->S = S;
  b->L = L;
  b->max_iter = max_iter;
  b->built_modes.clear();
  for (lq2d_problem* h : b->probs) b->built_modes.push_back(batch_mode_key(h));
  return LQ2D_OK;
}

int ensure_twisted_f32(lq2d_problem* h, cudaStream_t s);

// FP32 copies of the preconditioner's operands and of the Delta product's
// blocks (precision modes 1 and 2, and the multi-right-hand-side solve),
// allocated on first use and refreshed at every setup.
int ensure_f32(lq2d_problem* h) {
  if (h->f32_buf) return LQ2D_OK;
  {
    long long c[kF32Arrays];
    prec_counts(h, c);
    long long total = 0;
    for (int a = 0; a < kF32Arrays; ++a) total += c[a];
    double* buf = nullptr;
    int rc = dev_alloc(h, &buf, (size_t)(total + 1) / 2 + 64);
    if (rc) return rc;
    h->f32_buf = reinterpret_cast<float*>(buf);
    float* p = h->f32_buf;
    h->pd32.fac = p;
    p += c[0];
    h->pd32.Om = p;
    p += c[1];
    h->pd32.AQ = p;
    p += c[2];
    h->pd32.QAt = p;
    p += c[3];
    h->pd32.Qm = p;
    p += c[4];
    h->op32.Aself = p;
    p += c[5];
    h->op32.Anb = p;
    p += c[6];
    h->op32.Qi = p;
    p += c[7];
    h->op32.QTi = p;
    p += c[8];
    h->op32.Sb = p;
    p += c[9];
    h->pd32.fac_t0 = c[10] > 0 ? p : nullptr;
    h->pd32.fac_rec = h->nd.fac_rec;
    h->pd32.fac_vc = h->nd.fac_vc;
    convert_prec_f32(h, nullptr);
    LQ_CUDA(cudaStreamSynchronize(nullptr));
    LQ_CUDA(cudaGetLastError());
  }
  return ensure_twisted_f32(h, nullptr);
}

// Float buffer of `count` elements from the handle's allocations.
int alloc_floats(lq2d_problem* h, float** p, size_t count) {
  double* d = nullptr;
  const int rc = dev_alloc(h, &d, (count + 1) / 2);
  *p = reinterpret_cast<float*>(d);
  return rc;
}

// FP32 copies of the two-ended solve's arrays (when both the FP32 operands
// and the two-ended setup exist); converted at every setup.
int ensure_twisted_f32(lq2d_problem* h, cudaStream_t s) {
  if (h->fac_rev32 || !h->twisted_ready || !h->f32_buf) return LQ2D_OK;
  const Grid& g = h->g;
  int rc;
  if ((rc = alloc_floats(h, &h->fac_rev32, (size_t)g.V * 2 * h->nd.fac_vc)) != LQ2D_OK) return rc;
  if ((rc = alloc_floats(h, &h->sinv32, (size_t)g.V * 2 * 16 * g.n * g.n)) != LQ2D_OK) return rc;
  launch_to_f32(h->sb.fac_rev, h->fac_rev32, (long long)g.V * 2 * h->nd.fac_vc, s);
  launch_to_f32(h->sb.sinv, h->sinv32, (long long)g.V * 2 * 16LL * g.n * g.n, s);
  h->launches += 2;
  LQ_CUDA(cudaStreamSynchronize(s));
  return LQ2D_OK;
}

// Multi-right-hand-side operands: allocated on first use, rebuilt from the
// FP64 setup after every setup.
int ensure_mrhs(lq2d_problem* h, cudaStream_t s) {
  const Grid& g = h->g;
  if (!h->mb.rec) {
    LQ_CUDA(mrhs::prepare());
    int rc;
    if ((rc = alloc_floats(h, &h->mb.rec, (size_t)mrhs::rec_floats(g))) != LQ2D_OK) return rc;
    if ((rc = alloc_floats(h, &h->mb.wom, (size_t)mrhs::w_floats(g))) != LQ2D_OK) return rc;
    if ((rc = alloc_floats(h, &h->mb.wxa, (size_t)mrhs::w_floats(g))) != LQ2D_OK) return rc;
    if ((rc = alloc_floats(h, &h->mb.wxq, (size_t)mrhs::w_floats(g))) != LQ2D_OK) return rc;
    const size_t vec = (size_t)mrhs::vec_floats(g);
    if ((rc = alloc_floats(h, &h->m_src, vec)) != LQ2D_OK) return rc;
    if ((rc = alloc_floats(h, &h->m_thA, vec)) != LQ2D_OK) return rc;
    if ((rc = alloc_floats(h, &h->m_thB, vec)) != LQ2D_OK) return rc;
    if ((rc = alloc_floats(h, &h->m_rth, vec)) != LQ2D_OK) return rc;
  }
  if (!h->mrhs_built) {
    mrhs::launch_build(g, h->nd, h->mb, s);
    h->launches += 2;
    h->mrhs_built = true;
  }
  return LQ2D_OK;
}

// q = D_S r for the 32 right-hand sides of m_src (Algorithm 2, S x L sweeps
// from zero starts); returns the buffer holding q.
const float* enqueue_precond_multi(lq2d_problem* h, int S, int L, const float* src0, const SolverState* st,
                                   cudaStream_t s) {
  float* bufs[2] = {h->m_thA, h->m_thB};
  int out_i = 0;
  const float* prev = nullptr;
  for (int so = 0; so < S; ++so) {
    for (int l = 0; l < L; ++l) {
      int variant;
      const float* src = src0;
      if (l == 0 && so == 0) variant = 0;
      else if (l == 0) variant = 2;
      else {
        variant = 1;
        if (so > 0) src = h->m_rth;
      }
      mrhs::launch_sweep(variant, h->g, h->mb, src, prev, bufs[out_i], h->m_rth, st, s);
      h->launches += 1;
      prev = bufs[out_i];
      out_i ^= 1;
    }
  }
  return prev;
}

// Buffers of the multi-right-hand-side PCG: allocated on its first solve.
int ensure_mrhs_solve(lq2d_problem* h) {
  int rc = ensure_f32(h);
  if (rc != LQ2D_OK) return rc;
  if (h->mstate) return LQ2D_OK;
  const Grid& g = h->g;
  const size_t vec = (size_t)mrhs::vec_floats(g);
  mrhs::SolveVecs& v = h->mv;
  if ((rc = dev_alloc(h, &v.rhs, vec)) != LQ2D_OK) return rc;
  if ((rc = dev_alloc(h, &v.r, vec)) != LQ2D_OK) return rc;
  if ((rc = dev_alloc(h, &v.delta, vec)) != LQ2D_OK) return rc;
  if ((rc = dev_alloc(h, &v.d, vec)) != LQ2D_OK) return rc;
  if ((rc = dev_alloc(h, &v.y64, vec)) != LQ2D_OK) return rc;
  if ((rc = dev_alloc(h, &v.z64, vec)) != LQ2D_OK) return rc;
  if ((rc = alloc_floats(h, &v.d32, vec)) != LQ2D_OK) return rc;
  if ((rc = alloc_floats(h, &v.z32, vec)) != LQ2D_OK) return rc;
  if ((rc = alloc_floats(h, &v.y32, vec)) != LQ2D_OK) return rc;
  v.r32 = h->m_src;  // the preconditioner's source
  if ((rc = dev_alloc(h, &h->m_partials, (size_t)mrhs::solve_blocks(g) * 2 * mrhs::kRhs + 64)) != LQ2D_OK)
    return rc;
  double* st = nullptr;
  if ((rc = dev_alloc(h, &st, (sizeof(mrhs::State) + 7) / 8)) != LQ2D_OK) return rc;
  LQ_CUDA(cudaMemset(st, 0, sizeof(mrhs::State)));
  LQ_CUDA(cudaMallocHost(&h->h_mstate, sizeof(mrhs::State)));
  h->mstate = reinterpret_cast<mrhs::State*>(st);
  return LQ2D_OK;
}

// The preconditioner's output buffer of the multi-right-hand-side loop
// (S*L sweeps alternate between two buffers; S*L is even).
float* multi_q(lq2d_problem* h) { return h->m_thB; }

constexpr int kMultiStepKernels = 7;  // besides the S*L sweeps

// One step of the multi-right-hand-side PCG: the product and alpha, the
// update and tests, the preconditioner, mu and beta, then the residual
// replacements that are due.
void enqueue_multi_step(lq2d_problem* h, int S, int L, cudaStream_t s) {
  const Grid& g = h->g;
  mrhs::launch_delta_loop(g, h->op32, multi_q(h), h->mv, h->m_partials, h->mstate, h->st, s);
  mrhs::launch_update(g, h->mv, h->m_partials, h->mstate, h->st, s);
  enqueue_precond_multi(h, S, L, h->mv.r32, h->st, s);
  mrhs::launch_mu(g, multi_q(h), h->mv, h->m_partials, h->mstate, h->st, s);
  mrhs::launch_replace(g, h->op64, h->mv, h->m_partials, h->mstate, h->st, false, s);
  h->launches += kMultiStepKernels;
}

int get_multi_graph(lq2d_problem* h, int S, int L, cudaGraphExec_t* exec) {
  if (h->m_exec && h->m_graph_S == S && h->m_graph_L == L) {
    *exec = h->m_exec;
    return LQ2D_OK;
  }
  if (h->m_exec) cudaGraphExecDestroy(h->m_exec);
  if (h->m_graph) cudaGraphDestroy(h->m_graph);
  h->m_exec = nullptr;
  h->m_graph = nullptr;
  cudaGraph_t graph;
  LQ_CUDA(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle hc;
  LQ_CUDA(cudaGraphConditionalHandleCreate(&hc, graph, 1u, cudaGraphCondAssignDefault));
  alignas(cudaGraphNodeParams) unsigned char cp_storage[sizeof(cudaGraphNodeParams)];
  std::memset(cp_storage, 0, sizeof(cp_storage));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_storage);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  LQ_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  LQ_CUDA(cudaStreamBeginCaptureToGraph(h->priv, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  const long long before = h->launches;
  enqueue_multi_step(h, S, L, h->priv);
  h->launches = before;
  launch_loop_ctrl(h->st, hc, h->priv);
  cudaGraph_t captured = nullptr;
  cudaError_t ce = cudaStreamEndCapture(h->priv, &captured);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(LQ2D_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  }
  ce = cudaGraphInstantiate(&h->m_exec, graph, 0);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(LQ2D_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
  }
  h->m_graph = graph;
  h->m_graph_S = S;
  h->m_graph_L = L;
  *exec = h->m_exec;
  return LQ2D_OK;
}

// The whole multi-right-hand-side solve on device buffers, ordered on s.
int solve_multi_impl(lq2d_problem* h, int nrhs, const double* d_x0s, double tol, int S, int L, int max_iter,
                     double* d_x, double* d_u, double* d_costate, int* iterations, double* rel_res,
                     cudaStream_t s) {
  int rc = ensure_mrhs(h, s);
  if (rc == LQ2D_OK) rc = ensure_mrhs_solve(h);
  if (rc != LQ2D_OK) return rc;
  const Grid& g = h->g;
  const double rho2 = kPhaseRho * kPhaseRho;
  mrhs::launch_init(g, nrhs, d_x0s, h->rhs, g.Ps, h->mv, h->m_partials, h->mstate, h->st, tol, rho2, max_iter, s);
  h->launches += 1;
  int restarts = 0;
  int status = LQ2D_OK;
  long long bodies = 0;
  for (;;) {
    // first direction: q = P^-1 r, mu (beta = 0)
    enqueue_precond_multi(h, S, L, h->mv.r32, h->st, s);
    mrhs::launch_mu(g, multi_q(h), h->mv, h->m_partials, h->mstate, h->st, s);
    LQ_CUDA(cudaMemsetAsync(h->mv.d, 0, (size_t)mrhs::vec_floats(g) * sizeof(double), s));
    LQ_CUDA(cudaMemsetAsync(h->mv.d32, 0, (size_t)mrhs::vec_floats(g) * sizeof(float), s));
    h->launches += S * L + 1;
    if (h->driver == 1 || h->timing) {
      // host-enqueued steps (driver 1): every kernel is a launch of its own
      rc = run_host_loop(h, max_iter, s, [&]() { enqueue_multi_step(h, S, L, s); });
      if (rc != LQ2D_OK) return rc;
    } else {
      cudaGraphExec_t exec;
      rc = get_multi_graph(h, S, L, &exec);
      if (rc != LQ2D_OK) return rc;
      LQ_CUDA(cudaGraphLaunch(exec, s));
    }
    // the true residual of every right-hand side decides convergence
    mrhs::launch_replace(g, h->op64, h->mv, h->m_partials, h->mstate, h->st, true, s);
    h->launches += 3;
    LQ_CUDA(cudaMemcpyAsync(h->h_st, h->st, sizeof(SolverState), cudaMemcpyDeviceToHost, s));
    LQ_CUDA(cudaMemcpyAsync(h->h_mstate, h->mstate, sizeof(mrhs::State), cudaMemcpyDeviceToHost, s));
    LQ_CUDA(cudaStreamSynchronize(s));
    LQ_CUDA(cudaGetLastError());
    const SolverState& hs = *h->h_st;
    const mrhs::State& ms = *h->h_mstate;
    h->launches += (long long)(hs.body_count - bodies) * (kMultiStepKernels + S * L + 1);
    bodies = hs.body_count;
    if (ms.breakdown || hs.done == kBreakdown) { status = LQ2D_EBREAKDOWN; break; }
    if (hs.done == kConverged) break;
    if (hs.body_count >= hs.body_cap) { status = LQ2D_ETIMEOUT; break; }
    if (hs.iter >= max_iter || restarts >= h->max_restarts) { status = LQ2D_ENOCONV; break; }
    // a recurrence residual passed while the true one did not: restart the
    // right-hand sides concerned from their current iterate
    ++restarts;
    const int zero = 0;
    LQ_CUDA(cudaMemcpyAsync(&h->mstate->have_mu, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    LQ_CUDA(cudaStreamSynchronize(s));
  }
  // outputs: recovery (Section II-B) per right-hand side through the
  // single-right-hand-side buffers
  const long long nx = (long long)(g.T + 1) * g.NN * g.n, nu = (long long)g.T * g.NN * g.m;
  for (int r = 0; r < nrhs; ++r) {
    mrhs::launch_gather(g, h->mv.delta, r, h->delta, s);
    h->kt->delta_z(g, h->op64, h->delta, nullptr, h->z, nullptr, 0, s);
    launch_recover_u(g, h->nd, h->delta, h->u, s);
    if (d_x) launch_to_api(h->z, d_x + r * nx, g.NN, g.T + 1, g.n, g.Ps, s);
    if (d_u) launch_to_api(h->u, d_u + r * nu, g.NN, g.T, g.m, g.Pus, s);
    if (d_costate) launch_to_api(h->delta, d_costate + r * nx, g.NN, g.T + 1, g.n, g.Ps, s);
    h->launches += 3 + (d_x != nullptr) + (d_u != nullptr) + (d_costate != nullptr);
  }
  LQ_CUDA(cudaStreamSynchronize(s));
  LQ_CUDA(cudaGetLastError());
  const mrhs::State& ms = *h->h_mstate;
  int iters_max = 0;
  for (int r = 0; r < nrhs; ++r) {
    if (iterations) iterations[r] = ms.iters[r];
    if (rel_res) rel_res[r] = ms.bnorm2[r] > 0 ? std::sqrt(ms.rnorm2[r] / ms.bnorm2[r]) : std::sqrt(ms.rnorm2[r]);
    iters_max = std::max(iters_max, ms.iters[r]);
  }
  h->stats.iterations = iters_max;
  h->stats.restarts = restarts;
  h->stats.status = status;
  if (status == LQ2D_ENOCONV) return fail(status, "max_iter reached before every right-hand side met the tolerance");
  if (status == LQ2D_EBREAKDOWN) return fail(status, "breakdown: y'd <= 0 or a non-finite scalar");
  if (status == LQ2D_ETIMEOUT) return fail(status, "device loop cap reached");
  return LQ2D_OK;
}

}  // namespace

namespace lq2d {
// Lets other translation units of the library report a message through
// lq2d_last_error().
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace lq2d

extern "C" {

int lq2d_create(lq2d_problem** out, int K, int N, int T, int n, int m, const double* A_self, const double* A_nbr,
                const double* B, const double* Q, const double* R, const double* Q_T, const double* x0) {
  const double* src[7] = {A_self, A_nbr, B, Q, R, Q_T, x0};
  int rc = check_dims(K, N, T, n, m);
  if (rc) return rc;
  // reject non-finite host input before touching the device
  const size_t NN = (size_t)K * N;
  const size_t cnt[7] = {NN * n * n, NN * 4 * n * n, NN * n * m, NN * n * n, NN * m * m, NN * n * n, NN * n};
  for (int a = 0; a < 7; ++a) {
    if (!src[a]) return fail(LQ2D_EINVAL, "null input array");
    for (size_t e = 0; e < cnt[a]; ++e)
      if (!std::isfinite(src[a][e])) return fail(LQ2D_EINVAL, "non-finite input entry");
  }
  return create_common(out, K, N, T, n, m, src, cudaMemcpyHostToDevice, nullptr);
}

int lq2d_create_device(lq2d_problem** out, int K, int N, int T, int n, int m, const double* d_A_self,
                       const double* d_A_nbr, const double* d_B, const double* d_Q, const double* d_R,
                       const double* d_Q_T, const double* d_x0, void* stream) {
  const double* src[7] = {d_A_self, d_A_nbr, d_B, d_Q, d_R, d_Q_T, d_x0};
  return create_common(out, K, N, T, n, m, src, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
}

int lq2d_update_device(lq2d_problem* h, const double* d_A_self, const double* d_A_nbr, const double* d_B,
                       const double* d_Q, const double* d_R, const double* d_Q_T, const double* d_x0,
                       void* stream) {
  if (!h) return fail(LQ2D_EINVAL, "handle is NULL");
  const double* src[7] = {d_A_self, d_A_nbr, d_B, d_Q, d_R, d_Q_T, d_x0};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = copy_inputs(h, src, cudaMemcpyDeviceToDevice, s);
  if (rc) return rc;
  return run_setup(h, s);
}

int lq2d_update(lq2d_problem* h, const double* A_self, const double* A_nbr, const double* B, const double* Q,
                const double* R, const double* Q_T, const double* x0) {
  if (!h) return fail(LQ2D_EINVAL, "handle is NULL");
  const double* src[7] = {A_self, A_nbr, B, Q, R, Q_T, x0};
  const Grid& g = h->g;
  const size_t NN = g.NN, n = g.n, m = g.m;
  const size_t cnt[7] = {NN * n * n, NN * 4 * n * n, NN * n * m, NN * n * n, NN * m * m, NN * n * n, NN * n};
  for (int a = 0; a < 7; ++a) {
    if (!src[a]) return fail(LQ2D_EINVAL, "null input array");
    for (size_t e = 0; e < cnt[a]; ++e)
      if (!std::isfinite(src[a][e])) return fail(LQ2D_EINVAL, "non-finite input entry");
  }
  int rc = copy_inputs(h, src, cudaMemcpyHostToDevice, nullptr);
  if (rc) return rc;
  return run_setup(h, nullptr);
}

int lq2d_set_affine(lq2d_problem* h, const double* w) {
  if (!h) return fail(LQ2D_EINVAL, "handle is NULL");
  const Grid& g = h->g;
  const size_t cnt = (size_t)g.T * g.NN * g.n;
  if (w) {
    for (size_t e = 0; e < cnt; ++e)
      if (!std::isfinite(w[e])) return fail(LQ2D_EINVAL, "non-finite affine entry");
    if (!h->w_buf) {
      int rc = dev_alloc(h, &h->w_buf, cnt);
      if (rc) return rc;
    }
    LQ_CUDA(cudaMemcpy(h->w_buf, w, cnt * sizeof(double), cudaMemcpyHostToDevice));
    h->w_aff = h->w_buf;
  } else {
    h->w_aff = nullptr;
  }
  launch_build_rhs(g, h->sb.x0, h->w_aff, h->rhs, nullptr);
  launch_norms(g, h->rhs, g.n, h->partials, &h->st->counters[kCntAux], h->bnorm, nullptr);
  h->launches += 2;
  LQ_CUDA(cudaStreamSynchronize(nullptr));
  LQ_CUDA(cudaGetLastError());
  return LQ2D_OK;
}

int lq2d_solve(lq2d_problem* h, double tol, int S, int L, int max_iter, const double* delta0, double* x,
               double* u, double* costate, int* iterations, double* rel_kkt) {
  if (!h) return fail(LQ2D_EINVAL, "handle is NULL");
  const Grid& g = h->g;
  const size_t nx = (size_t)g.P * g.n, nu = (size_t)g.Pu * g.m;
  const double* d_delta0 = nullptr;
  if (delta0) {
    LQ_CUDA(cudaMemcpy(h->stage_x, delta0, nx * sizeof(double), cudaMemcpyHostToDevice));
    d_delta0 = h->stage_x;
  }
  // x goes through stage_x after delta0 has been consumed; costate through
  // the same staging buffer after x has been copied out
  int rc = solve_impl(h, tol, S, L, max_iter, d_delta0, nullptr, h->stage_u, nullptr, iterations, rel_kkt, nullptr);
  if (rc != LQ2D_OK && rc != LQ2D_ENOCONV && rc != LQ2D_EBREAKDOWN) return rc;
  std::string keep = g_err;
  if (u) LQ_CUDA(cudaMemcpy(u, h->stage_u, nu * sizeof(double), cudaMemcpyDeviceToHost));
  if (x) {
    h->launches += 1;
    launch_to_api(h->z, h->stage_x, g.NN, g.T + 1, g.n, g.Ps, nullptr);
    LQ_CUDA(cudaMemcpy(x, h->stage_x, nx * sizeof(double), cudaMemcpyDeviceToHost));
  }
  if (costate) {
    h->launches += 1;
    launch_to_api(h->delta, h->stage_x, g.NN, g.T + 1, g.n, g.Ps, nullptr);
    LQ_CUDA(cudaMemcpy(costate, h->stage_x, nx * sizeof(double), cudaMemcpyDeviceToHost));
  }
  g_err = keep;
  return rc;
}

int lq2d_solve_device(lq2d_problem* h, double tol, int S, int L, int max_iter, const void* d_delta0, void* d_x,
                      void* d_u, void* d_costate, int* iterations, double* rel_kkt, void* stream) {
  if (!h) return fail(LQ2D_EINVAL, "handle is NULL");
  return solve_impl(h, tol, S, L, max_iter, static_cast<const double*>(d_delta0), static_cast<double*>(d_x),
                    static_cast<double*>(d_u), static_cast<double*>(d_costate), iterations, rel_kkt,
                    static_cast<cudaStream_t>(stream));
}

int lq2d_apply_delta_device(lq2d_problem* h, const void* d_in, void* d_out, void* stream) {
  if (!h || !d_in || !d_out) return fail(LQ2D_EINVAL, "null argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Grid& g = h->g;
  h->launches += 4;
  launch_to_internal(static_cast<const double*>(d_in), h->thA, g.NN, g.T + 1, g.n, g.Ps, s);
  h->kt->delta_z(g, h->op64, h->thA, nullptr, h->z, nullptr, 0, s);
  h->kt->delta_y(g, h->op64, h->z, h->thA, nullptr, nullptr, h->y, h->partials, nullptr, 0, s);
  launch_to_api(h->y, static_cast<double*>(d_out), g.NN, g.T + 1, g.n, g.Ps, s);
  LQ_CUDA(cudaStreamSynchronize(s));
  LQ_CUDA(cudaGetLastError());
  return LQ2D_OK;
}

int lq2d_apply_precond_device(lq2d_problem* h, int S, int L, const void* d_r, void* d_q, void* stream) {
  if (!h || !d_r || !d_q) return fail(LQ2D_EINVAL, "null argument");
  if (S < 1) return fail(LQ2D_EINVAL, "outer_S must be >= 1");
  if (L < 2 || (L & 1)) return fail(LQ2D_EINVAL, "inner_L must be even and >= 2");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Grid& g = h->g;
  h->launches += 2;
  launch_to_internal(static_cast<const double*>(d_r), h->y, g.NN, g.T + 1, g.n, g.Ps, s);
  const void* q = enqueue_precond(h, S, L, false, false, nullptr, h->y, s, false);
  const double* qd = static_cast<const double*>(q);
  if (h->precision >= 1) {
    // widen the FP32 result (node-major) into thA (free after the sweeps) in
    // component planes, before the layout change
    launch_iter_f32_to_f64(g, static_cast<const float*>(q), h->thA, s);
    h->launches += 1;
    qd = h->thA;
  }
  launch_to_api(qd, static_cast<double*>(d_q), g.NN, g.T + 1, g.n, g.Ps, s);
  int fault = 0;
  LQ_CUDA(cudaMemcpyAsync(&fault, h->fault, sizeof(int), cudaMemcpyDeviceToHost, s));
  LQ_CUDA(cudaStreamSynchronize(s));
  LQ_CUDA(cudaGetLastError());
  if (fault) {
    LQ_CUDA(cudaMemset(h->fault, 0, sizeof(int)));
    return fail(LQ2D_ETIMEOUT, "a bounded wait inside a preconditioner sweep ran out");
  }
  return LQ2D_OK;
}

int lq2d_apply_precond_multi_device(lq2d_problem* h, int nrhs, int S, int L, const void* d_r, void* d_q,
                                    void* stream) {
  if (!h || !d_r || !d_q) return fail(LQ2D_EINVAL, "null argument");
  if (h->g.n != mrhs::kN) return fail(LQ2D_EINVAL, "the multi-right-hand-side path needs n = 4");
  if (nrhs < 1 || nrhs > mrhs::kRhs) return fail(LQ2D_EINVAL, "nrhs must be in 1..32");
  if (S < 1) return fail(LQ2D_EINVAL, "outer_S must be >= 1");
  if (L < 2 || (L & 1)) return fail(LQ2D_EINVAL, "inner_L must be even and >= 2");
  if (h->g.T + 1 > 65535) return fail(LQ2D_EINVAL, "the layout transposes need T + 1 <= 65535");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = ensure_mrhs(h, s);
  if (rc != LQ2D_OK) return rc;
  mrhs::launch_from_api(h->g, nrhs, static_cast<const double*>(d_r), h->m_src, s);
  const float* q = enqueue_precond_multi(h, S, L, h->m_src, nullptr, s);
  mrhs::launch_to_api(h->g, nrhs, q, static_cast<double*>(d_q), s);
  h->launches += 2;
  LQ_CUDA(cudaStreamSynchronize(s));
  LQ_CUDA(cudaGetLastError());
  return LQ2D_OK;
}

int lq2d_solve_multi_device(lq2d_problem* h, int nrhs, const void* d_x0s, double tol, int S, int L, int max_iter,
                            void* d_x, void* d_u, void* d_costate, int* iterations, double* rel_residuals,
                            void* stream) {
  if (!h || !d_x0s) return fail(LQ2D_EINVAL, "null argument");
  if (h->g.n != mrhs::kN) return fail(LQ2D_EINVAL, "the multi-right-hand-side path needs n = 4");
  if (nrhs < 1 || nrhs > mrhs::kRhs) return fail(LQ2D_EINVAL, "nrhs must be in 1..32");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(LQ2D_EINVAL, "tol must be positive");
  if (S < 1) return fail(LQ2D_EINVAL, "outer_S must be >= 1");
  if (L < 2 || (L & 1)) return fail(LQ2D_EINVAL, "inner_L must be even and >= 2");
  if (max_iter < 0) return fail(LQ2D_EINVAL, "max_iter must be >= 0");
  return solve_multi_impl(h, nrhs, static_cast<const double*>(d_x0s), tol, S, L, max_iter, static_cast<double*>(d_x),
                          static_cast<double*>(d_u), static_cast<double*>(d_costate), iterations, rel_residuals,
                          static_cast<cudaStream_t>(stream));
}

int lq2d_autotune(lq2d_problem* h, int S, int L, int reps, int* threads, double* ms, void* stream) {
  if (!h) return fail(LQ2D_EINVAL, "handle is NULL");
  if (S < 1) return fail(LQ2D_EINVAL, "outer_S must be >= 1");
  if (L < 2 || (L & 1)) return fail(LQ2D_EINVAL, "inner_L must be even and >= 2");
  if (reps < 1) return fail(LQ2D_EINVAL, "reps must be >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Grid& g = h->g;
  const int slot = h->precision >= 1 ? 1 : 0;
  const int saved = h->sweep_threads[slot];
  // the right-hand side of the problem stands in for a residual
  LQ_CUDA(cudaMemcpyAsync(h->y, h->rhs, (size_t)g.Ps * g.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  cudaEvent_t e0, e1;
  LQ_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(LQ2D_ECUDA, "cudaEventCreate failed");
  }
  // candidates (width, time steps per lane, two-ended): the CTA widths, for
  // the n = 4 FP32 sweeps the compiled (width, steps) schedules, and the
  // two-ended solve where it applies (n = 4, K >= 4, tiled widths 32, 64)
  int sched[12][2] = {{32, 0}, {64, 0}, {128, 0}, {256, 0}};
  int nsched = 4;
  const bool bulk = slot == 1 && g.n == 4;
  if (bulk) nsched = sweep4_f32_configs(sched, 12);
  const bool tw_ok = h->twisted_ready;
  std::vector<std::array<int, 3>> cand;
  for (int c = 0; c < nsched; ++c) {
    cand.push_back({sched[c][0], sched[c][1], 0});
    if (tw_ok && sched[c][1] == 0 && (sched[c][0] == 32 || sched[c][0] == 64))
      cand.push_back({sched[c][0], sched[c][1], 1});
  }
  const int saved_steps = h->sweep_steps, saved_tw = h->twisted[slot];
  double best_ms = 0.0;
  int best = saved, best_steps = saved_steps, best_tw = saved_tw;
  cudaError_t err = cudaSuccess;
  for (size_t c = 0; c < cand.size() && err == cudaSuccess; ++c) {
    h->sweep_threads[slot] = cand[c][0];
    if (bulk) h->sweep_steps = cand[c][1];
    h->twisted[slot] = cand[c][2];
    enqueue_precond(h, S, L, false, false, nullptr, h->y, s, false);  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) enqueue_precond(h, S, L, false, false, nullptr, h->y, s, false);
    cudaEventRecord(e1, s);
    err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    const double per = (double)t / reps;
    if (err == cudaSuccess && (c == 0 || per < best_ms)) {
      best_ms = per;
      best = cand[c][0];
      best_steps = bulk ? cand[c][1] : saved_steps;
      best_tw = cand[c][2];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  if (err != cudaSuccess) {
    h->sweep_threads[slot] = saved;
    h->sweep_steps = saved_steps;
    h->twisted[slot] = saved_tw;
    return fail(LQ2D_ECUDA, cudaGetErrorString(err));
  }
  h->sweep_threads[slot] = best;
  h->sweep_steps = best_steps;
  h->twisted[slot] = best_tw;
  if (threads) *threads = best;
  if (ms) *ms = best_ms;
  return LQ2D_OK;
}

int lq2d_solve_nbjm_device(lq2d_problem* h, double eps, int inner_L, int max_outer, void* d_x, void* d_u,
                           void* d_costate, int* outer_iterations, double* rel_kkt_residual, void* stream) {
  if (!h) return fail(LQ2D_EINVAL, "handle is NULL");
  return solve_nbjm_impl(h, eps, inner_L, max_outer, static_cast<double*>(d_x), static_cast<double*>(d_u),
                         static_cast<double*>(d_costate), outer_iterations, rel_kkt_residual,
                         static_cast<cudaStream_t>(stream));
}

int lq2d_batch_create(lq2d_batch** out, int count, lq2d_problem* const* problems) {
  if (!out || count < 1 || !problems) return fail(LQ2D_EINVAL, "batch needs a positive count and a problem array");
  *out = nullptr;
  for (int i = 0; i < count; ++i)
    if (!problems[i]) return fail(LQ2D_EINVAL, "null problem in batch");
  lq2d_batch* b = new lq2d_batch();
  b->probs.assign(problems, problems + count);
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&b->results, (size_t)count * kBatchSlot * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_results, (size_t)count * kBatchSlot * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_heads, (kBatchHeads + 1) * sizeof(unsigned));
  if (e == cudaSuccess) e = batch_prepare();
  if (e != cudaSuccess) {
    lq2d_batch_destroy(b);
    return fail(e == cudaErrorMemoryAllocation ? LQ2D_ENOMEM : LQ2D_ECUDA, cudaGetErrorString(e));
  }
  *out = b;
  return LQ2D_OK;
}

int lq2d_batch_solve(lq2d_batch* b, double tol, int S, int L, int max_iter, int* iterations, double* rel_kkt,
                     int* statuses, void* stream) {
  if (!b) return fail(LQ2D_EINVAL, "batch is NULL");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(LQ2D_EINVAL, "tol must be positive and finite");
  if (S < 1 || L < 2 || (L & 1)) return fail(LQ2D_EINVAL, "outer_S >= 1 and even inner_L >= 2 required");
  if (max_iter < 0) return fail(LQ2D_EINVAL, "max_iter must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bool rebuild = !b->exec || b->tol != tol || b->S != S || b->L != L || b->max_iter != max_iter;
  for (size_t i = 0; !rebuild && i < b->probs.size(); ++i) {
    const lq2d_problem* h = b->probs[i];
    rebuild = b->built_modes[i] != batch_mode_key(h);
  }
  if (rebuild) {
    int rc = batch_build(b, tol, S, L, max_iter);
    if (rc) return rc;
  }
  const size_t count = b->probs.size();
  LQ_CUDA(cudaGraphLaunch(b->exec, s));
  LQ_CUDA(cudaMemcpyAsync(b->h_results, b->results, count * kBatchSlot * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (b->built_persistent)
    LQ_CUDA(cudaMemcpyAsync(b->h_heads, b->plan.heads, (kBatchHeads + 1) * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  LQ_CUDA(cudaStreamSynchronize(s));
  LQ_CUDA(cudaGetLastError());
  const long long passes = b->built_persistent ? (long long)b->h_heads[kBatchHeads] : 0;
  int worst = LQ2D_OK;
  for (size_t i = 0; i < count; ++i) {
    lq2d_problem* h = b->probs[i];
    const SolverState& hs = *reinterpret_cast<const SolverState*>(b->h_results + i * kBatchSlot);
    const double* kkt = b->h_results + i * kBatchSlot + 24;
    const double bn = std::sqrt(hs.bnorm2);
    const double rel = bn > 0 ? std::sqrt(kkt[0]) / bn : std::sqrt(kkt[0]);
    const bool true_pass = h->stop_mode == 0 ? (rel <= tol || kkt[0] == 0.0) : (kkt[2] < tol);
    int status;
    switch (hs.done) {
      case kConverged: status = true_pass ? LQ2D_OK : LQ2D_ENOCONV; break;
      case kMaxIter: status = LQ2D_ENOCONV; break;
      case kBreakdown: status = LQ2D_EBREAKDOWN; break;
      case kLoopCap: status = LQ2D_ETIMEOUT; break;
      default: status = LQ2D_ECUDA; break;
    }
    std::memset(&h->stats, 0, sizeof(h->stats));
    h->stats.iterations = hs.iter;
    h->stats.rel_residual = bn > 0 ? std::sqrt(hs.rnorm2) / bn : std::sqrt(hs.rnorm2);
    h->stats.rel_kkt_residual = rel;
    h->stats.kkt_inf = kkt[2];
    h->stats.cost = 0.5 * kkt[1];
    h->stats.status = status;
    h->stats.body_executions = hs.body_count;
    const int sweeps = sweeps_per_step(h, S, L);
    if (b->built_persistent) {
      // the loop's launches serve every problem; they are counted once, on the first
      h->launches += (2 + sweeps) + 3 + (i == 0 ? passes * (2 + sweeps + 1) : 0);
    } else {
      h->launches += (2 + sweeps) + 3 + (long long)hs.body_count * (2 + sweeps + 1);
    }
    if (iterations) iterations[i] = hs.iter;
    if (rel_kkt) rel_kkt[i] = rel;
    if (statuses) statuses[i] = status;
    if (status != LQ2D_OK && worst == LQ2D_OK) worst = status;
  }
  if (worst != LQ2D_OK) return fail(worst, "some problems of the batch did not converge; see statuses");
  return LQ2D_OK;
}

void lq2d_batch_destroy(lq2d_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->results) cudaFree(b->results);
  if (b->h_results) cudaFreeHost(b->h_results);
  if (b->h_heads) cudaFreeHost(b->h_heads);
  if (b->plan_mem) cudaFree(b->plan_mem);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

int lq2d_batch_set_option(lq2d_batch* b, int option, int value) {
  if (!b) return fail(LQ2D_EINVAL, "batch is NULL");
  switch (option) {
    case LQ2D_BATCH_PERSISTENT:
      if (value != 0 && value != 1) return fail(LQ2D_EINVAL, "persistent must be 0 or 1");
      b->persistent = value;
      break;
    case LQ2D_BATCH_THREADS:
      if (value != 32 && value != 64 && value != 128) return fail(LQ2D_EINVAL, "batch threads must be 32, 64 or 128");
      b->threads = value;
      break;
    default:
      return fail(LQ2D_EINVAL, "unknown batch option");
  }
  // the next solve rebuilds its graph
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  return LQ2D_OK;
}

int lq2d_batch_get_option(const lq2d_batch* b, int option, int* value) {
  if (!b || !value) return fail(LQ2D_EINVAL, "null argument");
  switch (option) {
    case LQ2D_BATCH_PERSISTENT: *value = b->persistent; return LQ2D_OK;
    case LQ2D_BATCH_THREADS: *value = b->threads; return LQ2D_OK;
    case LQ2D_BATCH_USES_PERSISTENT: *value = b->built_persistent ? 1 : 0; return LQ2D_OK;
    default: return fail(LQ2D_EINVAL, "unknown batch option");
  }
}

int lq2d_batch_autotune(lq2d_batch* b, int S, int L, int reps, int* threads, double* ms, void* stream) {
  if (!b) return fail(LQ2D_EINVAL, "batch is NULL");
  if (S < 1 || L < 2 || (L & 1)) return fail(LQ2D_EINVAL, "outer_S >= 1 and even inner_L >= 2 required");
  if (reps < 1) return fail(LQ2D_EINVAL, "reps must be >= 1");
  if (!batch_persistent_ok(b, S, L))
    return fail(LQ2D_EINVAL, "the batch does not run the persistent loop (n = 4, FP64, NBJM problems required)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int SL = S * L;
  // running states, so that no sweep skips its problem
  for (lq2d_problem* h : b->probs) {
    launch_init_state(h->st, 1.0, 1, h->stop_mode, h->bnorm, 0, nullptr, 0, 0.0, s);
    h->launches += 1;
  }
  const int saved = b->threads;
  const int cand[3] = {32, 64, 128};
  cudaEvent_t e0, e1;
  LQ_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(LQ2D_ECUDA, "cudaEventCreate failed");
  }
  double best_ms = 0.0;
  int best = saved, rc = LQ2D_OK;
  cudaError_t err = cudaSuccess;
  auto dsr = [&]() {  // one plain D_S application of every problem (r = the right-hand side)
    cudaMemsetAsync(b->plan.heads, 0, kBatchHeads * sizeof(unsigned), s);
    for (int k = 0; k < SL; ++k) batch_enqueue_sweep(b->plan, b->variants[SL + k], SL + k, 2 + k, s);
  };
  for (int c = 0; c < 3 && err == cudaSuccess && rc == LQ2D_OK; ++c) {
    b->threads = cand[c];
    rc = batch_plan_upload(b, S, L, s);
    if (rc) break;
    dsr();
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) dsr();
    cudaEventRecord(e1, s);
    err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    const double per = (double)t / reps;
    if (err == cudaSuccess && (c == 0 || per < best_ms)) {
      best_ms = per;
      best = cand[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  b->probs[0]->launches += (long long)3 * (reps + 1) * SL;
  if (rc == LQ2D_OK && err != cudaSuccess) rc = fail(LQ2D_ECUDA, cudaGetErrorString(err));
  if (rc != LQ2D_OK) best = saved;
  const int keep = lq2d_batch_set_option(b, LQ2D_BATCH_THREADS, best);
  if (rc != LQ2D_OK) return rc;
  if (keep != LQ2D_OK) return keep;
  if (threads) *threads = best;
  if (ms) *ms = best_ms;
  return LQ2D_OK;
}

int lq2d_get_solution_device(lq2d_problem* h, void* d_x, void* d_u, void* d_costate, void* stream) {
  if (!h) return fail(LQ2D_EINVAL, "handle is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Grid& g = h->g;
  if (d_x) launch_to_api(h->z, static_cast<double*>(d_x), g.NN, g.T + 1, g.n, g.Ps, s);
  if (d_u) launch_to_api(h->u, static_cast<double*>(d_u), g.NN, g.T, g.m, g.Pus, s);
  if (d_costate) launch_to_api(h->delta, static_cast<double*>(d_costate), g.NN, g.T + 1, g.n, g.Ps, s);
  h->launches += (d_x != nullptr) + (d_u != nullptr) + (d_costate != nullptr);
  LQ_CUDA(cudaStreamSynchronize(s));
  LQ_CUDA(cudaGetLastError());
  return LQ2D_OK;
}

int lq2d_set_option(lq2d_problem* h, int option, double value) {
  if (!h) return fail(LQ2D_EINVAL, "handle is NULL");
  const int v = (int)value;
  switch (option) {
    case LQ2D_OPT_STOP_MODE:
      if (v != 0 && v != 1) return fail(LQ2D_EINVAL, "stop mode must be 0 or 1");
      h->stop_mode = v;
      return LQ2D_OK;
    case LQ2D_OPT_DRIVER:
      if (v != 0 && v != 1) return fail(LQ2D_EINVAL, "driver must be 0 or 1");
      h->driver = v;
      return LQ2D_OK;
    case LQ2D_OPT_TIMING:
      h->timing = v ? 1 : 0;
      return LQ2D_OK;
    case LQ2D_OPT_PRECONDITIONER:
      if (v != 0 && v != 1) return fail(LQ2D_EINVAL, "preconditioner must be 0 (NBJM) or 1 (none)");
      h->precond_kind = v;
      return LQ2D_OK;
    case LQ2D_OPT_KAPPA:
      h->kappa = v ? 1 : 0;
      return LQ2D_OK;
    case LQ2D_OPT_MAX_RESTARTS:
      if (v < 0) return fail(LQ2D_EINVAL, "max restarts must be >= 0");
      h->max_restarts = v;
      return LQ2D_OK;
    case LQ2D_OPT_SWEEP_THREADS:
      if (v != 32 && v != 64 && v != 128 && v != 256)
        return fail(LQ2D_EINVAL, "sweep threads must be 32, 64, 128 or 256");
      h->sweep_threads[0] = h->sweep_threads[1] = v;
      return LQ2D_OK;
    case LQ2D_OPT_SWEEP_STEPS:
      if (v != 0 && v != 1 && v != 2 && v != 4) return fail(LQ2D_EINVAL, "sweep steps must be 0, 1, 2 or 4");
      h->sweep_steps = v;
      return LQ2D_OK;
    case LQ2D_OPT_TWISTED:
      if (v != 0 && v != 1) return fail(LQ2D_EINVAL, "twisted must be 0 or 1");
      h->twisted[0] = h->twisted[1] = v;
      return LQ2D_OK;
    default:
      return fail(LQ2D_EINVAL, "unknown option");
  }
}

int lq2d_get_option(const lq2d_problem* h, int option, double* value) {
  if (!h || !value) return fail(LQ2D_EINVAL, "null argument");
  const int slot = h->precision >= 1 ? 1 : 0;
  switch (option) {
    case LQ2D_OPT_STOP_MODE: *value = h->stop_mode; return LQ2D_OK;
    case LQ2D_OPT_DRIVER: *value = h->driver; return LQ2D_OK;
    case LQ2D_OPT_TIMING: *value = h->timing; return LQ2D_OK;
    case LQ2D_OPT_MAX_RESTARTS: *value = h->max_restarts; return LQ2D_OK;
    case LQ2D_OPT_PRECONDITIONER: *value = h->precond_kind; return LQ2D_OK;
    case LQ2D_OPT_KAPPA: *value = h->kappa; return LQ2D_OK;
    case LQ2D_OPT_SWEEP_THREADS: *value = h->sweep_threads[slot]; return LQ2D_OK;
    case LQ2D_OPT_SWEEP_STEPS: *value = h->sweep_steps; return LQ2D_OK;
    case LQ2D_OPT_TWISTED: {  // widths above 64 and the bulk-copy FP32 schedules solve one-ended
      const int thr = h->sweep_threads[slot];
      *value = (current_twisted(h) && (thr == 32 || thr == 64) &&
                !(slot == 1 && h->g.n == 4 && h->sweep_steps >= 1)) ? 1 : 0;
      return LQ2D_OK;
    }
    default: return fail(LQ2D_EINVAL, "unknown option");
  }
}

int lq2d_get_stats(const lq2d_problem* h, lq2d_stats* out) {
  if (!h || !out) return fail(LQ2D_EINVAL, "null argument");
  *out = h->stats;
  out->launches_total = h->launches;
  out->sweep_threads = h->sweep_threads[h->precision >= 1 ? 1 : 0];
  out->sweep_steps = (h->precision >= 1 && h->g.n == 4) ? h->sweep_steps : 1;
  return LQ2D_OK;
}

int lq2d_set_precision(lq2d_problem* h, int mode) {
  if (!h) return fail(LQ2D_EINVAL, "handle is NULL");
  if (mode < 0 || mode > 2)
    return fail(LQ2D_EINVAL, "precision mode must be 0 (FP64), 1 (FP32 preconditioner) or 2 (FP32 preconditioner and product)");
  if (mode == 2 && !h->d32) {
    double* buf = nullptr;
    int rc = dev_alloc(h, &buf, ((size_t)h->g.Ps * h->g.n + 1) / 2 + 64);
    if (rc) return rc;
    h->d32 = reinterpret_cast<float*>(buf);
    LQ_CUDA(cudaMemset(h->d32, 0, (size_t)h->g.Ps * h->g.n * sizeof(float)));
  }
  if (mode >= 1) {
    const int rc = ensure_f32(h);
    if (rc != LQ2D_OK) return rc;
  }
  h->precision = mode;
  return LQ2D_OK;
}

void lq2d_destroy(lq2d_problem* h) {
  if (!h) return;
  free_all(h);
  delete h;
}

const char* lq2d_last_error(void) { return g_err.c_str(); }

}  // extern "C"
