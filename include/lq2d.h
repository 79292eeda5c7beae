/*
 * lq2d — structured LQ optimal control over a K x N grid of coupled
 * subsystems, solved by preconditioned conjugate gradients with the nested
 * block-Jacobi preconditioner (Zafar & Manchester, "Structured linear
 * quadratic control computations over 2D grids").
 *
 * Problem (Section II, eqs. 2d_graph_dynamics and LQ_problem): node (i, j),
 * i = 0..K-1 (vertical), j = 0..N-1 (horizontal), state x in R^n, input u
 * in R^m, horizon t = 0..T:
 *   x_{i,j,t+1} = A x_{i,j,t} + B u_{i,j,t} + E x_{i,j-1,t} + F x_{i,j+1,t}
 *                 + G x_{i-1,j,t} + H x_{i+1,j,t} (+ omega_{t}, optional)
 *   x_{i,j,0} = gamma_{i,j};  states beyond the grid edge are zero
 *   minimise 1/2 sum_t sum_{i,j} (x'Q x + u'R u), with Q_T at t = T, no u_T.
 * All blocks are time-invariant; Q, R, Q_T must be symmetric positive
 * definite.
 *
 * The solve reduces the KKT system to Delta delta = r_delta (Section II-B),
 * Delta = A~ Q~^-1 A~' + B~ R~^-1 B~', r_delta = -omega~, and runs
 * Algorithm 1 (PCGM) with S outer x L inner sweeps of Algorithm 2 (NBJM) as
 * preconditioner (Theorem posdef_preconditioner: SPD for even L).  Then
 * x = Q~^-1 A~' delta and u = R~^-1 B~' delta.
 *
 * Conventions
 *   - Node index p = i*N + j.  All arrays are row-major FP64.
 *   - Host-layout vectors are time-major: x and costate [T+1][K*N][n],
 *     u [T][K*N][m].  Device entry points take device pointers in the same
 *     layout and run on the caller's CUDA stream (a cudaStream_t passed as
 *     void*, NULL = legacy default stream).
 *   - Inputs are copied; the caller keeps ownership of every pointer.
 *     Outputs are written only into caller buffers; any output pointer may
 *     be NULL to skip it.
 *   - Every call returns an lq2d status; on a non-OK status
 *     lq2d_last_error() describes it (thread-local, valid until the next
 *     call on the same thread).  A call that fails leaves the handle usable
 *     unless the status is LQ2D_ECUDA.
 *   - The library needs a CUDA GPU (sm_103a); there is no CPU fallback.
 */
#ifndef LQ2D_H
#define LQ2D_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lq2d_problem lq2d_problem; /* opaque, library-owned */

enum {
  LQ2D_OK = 0,
  LQ2D_EINVAL = 1,      /* bad dimensions or arguments, non-finite input, L odd or < 2 */
  LQ2D_ENOTPD = 2,      /* Cholesky of Q, Q_T, R or of a Phi_bar block failed */
  LQ2D_ENOCONV = 3,     /* max_iter reached; outputs hold the last iterate */
  LQ2D_EBREAKDOWN = 4,  /* y'd <= 0 or a non-finite scalar inside Algorithm 1 */
  LQ2D_ECUDA = 5,       /* a CUDA call failed */
  LQ2D_ENOMEM = 6,      /* device allocation failed (the environment variable
                           LQ2D_FAIL_ALLOC_AT=k makes a handle's k-th device
                           allocation fail on the host, for tests of this path) */
  LQ2D_ETIMEOUT = 7     /* the device loop hit its hard iteration cap */
};

/* Options for lq2d_set_option. */
enum {
  LQ2D_OPT_STOP_MODE = 1,    /* 0: stop when ||r||_2 <= tol ||r_delta||_2 (default);
                                1: stop when ||r||_inf < tol (the stop test of Algorithm 1 as printed) */
  LQ2D_OPT_DRIVER = 2,       /* 0: the PCG loop runs on the device as a CUDA graph with a
                                   conditional while node (default);
                                1: the host enqueues the steps, checking the stop flag every
                                   few steps */
  LQ2D_OPT_TIMING = 3,       /* 1: record CUDA events around every sweep and Delta-apply launch
                                   (forces driver 1); read the totals with lq2d_get_stats */
  LQ2D_OPT_MAX_RESTARTS = 4, /* restarts allowed when the recurrence residual passes but the
                                true residual does not (default 3) */
  LQ2D_OPT_PRECONDITIONER = 5, /* 0: NBJM, Algorithm 2 (default); 1: none (plain CG on Delta,
                                  used to estimate kappa(Delta)) */
  LQ2D_OPT_KAPPA = 6,         /* 1: record the PCG coefficients of each solve and estimate the
                                  extreme eigenvalues of the preconditioned operator (Lanczos
                                  matrix of CG; Section V reports kappa before and after
                                  preconditioning); read them with lq2d_get_stats */
  LQ2D_OPT_SWEEP_THREADS = 7, /* 32, 64, 128 or 256: threads per CTA of the NBJM sweeps, i.e. a
                                  tile of threads/g time steps per CTA (g = 2n rounded up to a
                                  power of two); sets the FP64 and FP32 sweeps alike.
                                  Default 64; lq2d_autotune picks it by timing.  Results may
                                  differ in the last bits between widths (partial sums are
                                  grouped per CTA) */
  LQ2D_OPT_SWEEP_STEPS = 8,   /* 0, 1, 2 or 4: time steps each lane carries in the n = 4 FP32
                                  sweeps with bulk-copy staging (a CTA then holds threads/8 * steps
                                  time steps); 0 selects the tiled FP32 kernel (LQ2D_OPT_SWEEP_THREADS
                                  as for FP64).  The bulk schedules compiled are (threads, steps) =
                                  (32, 4), (64, 4), (64, 2), (128, 2), (32, 2), (64, 1); another pair
                                  with steps >= 1 runs as (64, 4).  Default: 4 when the grid has at
                                  least 16384 (column pair, time) blocks, else 0; lq2d_autotune picks
                                  the pair by timing.  No effect on FP64 sweeps or other n */
  LQ2D_OPT_TWISTED = 9        /* 1 (default where it applies): solve each Phi_bar block from both
                                  ends at once (Section IV-B's banded solve with the pair-rows
                                  eliminated from the first and the last towards two interface
                                  rows, whose 2x2-block Schur complement is inverted at setup):
                                  half the dependent chain of a sweep and twice its warps.  It
                                  applies to the tiled sweeps of n = 4 with K >= 4 at widths 32
                                  and 64; other schedules, and other n or K, stay one-sided.  The
                                  handle keeps the reversed factor for it (one more factor's
                                  memory).  0: one-sided.  lq2d_autotune tries both */
};

/* Statistics of the last solve on a handle. */
typedef struct lq2d_stats {
  int iterations;          /* PCG steps (loop passes of Algorithm 1) over all restarts */
  int restarts;            /* restarts from the true residual (direction reset) */
  int status;              /* status returned by the solve */
  int sweep_launches;      /* timed sweep launches (timing option) */
  int delta_launches;      /* timed Delta-apply launches (timing option, 2 kernels each) */
  int sweep_steps;         /* time steps per lane of the current mode's sweeps (n = 4 FP32), else 1 */
  double rel_residual;     /* ||r||_2 / ||r_delta||_2 of the recurrence residual at exit */
  double rel_kkt_residual; /* ||KKT residual of (x, u, delta)||_2 / ||r_delta||_2 */
  double kkt_inf;          /* max |A~x + B~u + omega~| */
  double cost;             /* 1/2 (x'Q~x + u'R~u) */
  double sweep_ms;         /* summed device time of the timed sweep launches */
  double delta_ms;         /* summed device time of the timed Delta-apply launches */
  long long launches_total; /* kernels launched for this handle since creation (setup included) */
  int body_executions;     /* device-loop body executions in the last solve */
  int outer_iterations;    /* outer steps of the last standalone NBJM solve */
  double kappa_estimate;   /* lambda_max / lambda_min (LQ2D_OPT_KAPPA), else 0 */
  double lambda_min;       /* extreme Ritz values of the preconditioned operator */
  double lambda_max;
  int sweep_threads;       /* threads per CTA of the current precision mode's sweeps */
  int residual_replacements; /* precision mode 2: recurrence residuals replaced by the true one */
} lq2d_stats;

/* Creates a problem from host arrays, copies them to the current device and
 * factors the preconditioner (Section IV-B: one banded block-Cholesky
 * factorisation per column pair v and time class, done once).
 *   A_self [K*N][n][n]      A_{i,j}
 *   A_nbr  [K*N][4][n][n]   E (j-1), F (j+1), G (i-1), H (i+1); blocks that
 *                           point off the grid are ignored
 *   B      [K*N][n][m]
 *   Q, Q_T [K*N][n][n]      stage and terminal state weights (SPD)
 *   R      [K*N][m][m]      input weight (SPD)
 *   x0     [K*N][n]         gamma
 * Limits: 1 <= n <= 8, 1 <= m <= 8, K, N, T >= 1.
 * Returns LQ2D_EINVAL, LQ2D_ENOTPD, LQ2D_ENOMEM or LQ2D_ECUDA on failure
 * (then *out is NULL). */
int lq2d_create(lq2d_problem **out, int K, int N, int T, int n, int m,
                const double *A_self, const double *A_nbr, const double *B,
                const double *Q, const double *R, const double *Q_T,
                const double *x0);

/* As lq2d_create, with the seven arrays already in device memory (same
 * layouts).  Work is ordered on `stream`; the call returns after it. */
int lq2d_create_device(lq2d_problem **out, int K, int N, int T, int n, int m,
                       const double *d_A_self, const double *d_A_nbr, const double *d_B,
                       const double *d_Q, const double *d_R, const double *d_Q_T,
                       const double *d_x0, void *stream);

/* Replaces the problem data of an existing handle by new device arrays of
 * the same sizes and re-runs the setup (inverses, splitting blocks,
 * factorisation of Phi_bar).  Allocates nothing. */
int lq2d_update_device(lq2d_problem *h, const double *d_A_self, const double *d_A_nbr,
                       const double *d_B, const double *d_Q, const double *d_R,
                       const double *d_Q_T, const double *d_x0, void *stream);

/* As lq2d_update_device with host arrays (copied to the device, then the
 * setup is re-run).  Allocates no device memory. */
int lq2d_update(lq2d_problem *h, const double *A_self, const double *A_nbr, const double *B,
                const double *Q, const double *R, const double *Q_T, const double *x0);

/* Boundary/affine terms omega_t (Section II-A: M_hat alpha + N_hat beta),
 * host array [T][K*N][n] entering x_{t+1} = ... + omega_t; NULL clears them. */
int lq2d_set_affine(lq2d_problem *h, const double *w);

/* Solves with host buffers (Algorithm 1 with Algorithm 2 as preconditioner).
 *   tol        > 0; see LQ2D_OPT_STOP_MODE
 *   outer_S    >= 1 outer sweeps; inner_L >= 2 and even (the Theorem needs even L)
 *   max_iter   >= 0 PCG steps
 *   delta0     NULL for delta^(0) = 0, else a warm start [T+1][K*N][n]
 *   x [T+1][K*N][n], u [T][K*N][m], costate [T+1][K*N][n] = delta of
 *   Delta delta = r_delta (so delta_t = -P_t x_t for the Riccati matrices P_t)
 *   iterations, rel_kkt_residual: scalar outputs (see lq2d_stats)
 * LQ2D_ENOCONV and LQ2D_EBREAKDOWN still write the outputs. */
int lq2d_solve(lq2d_problem *h, double tol, int outer_S, int inner_L, int max_iter,
               const double *delta0, double *x, double *u, double *costate,
               int *iterations, double *rel_kkt_residual);

/* As lq2d_solve with device buffers, ordered on `stream`.  Returns after
 * the work on `stream` is complete; other streams are not synchronised. */
int lq2d_solve_device(lq2d_problem *h, double tol, int outer_S, int inner_L, int max_iter,
                      const void *d_delta0, void *d_x, void *d_u, void *d_costate,
                      int *iterations, double *rel_kkt_residual, void *stream);

/* Algorithm 2 run as a solver: the "standard nested block Jacobi method" the
 * paper compares PCGM against (Section V).  Each outer step runs inner_L
 * sweeps (L = 2 in the paper) and stops when
 * ||delta^(s+1) - delta^(s)||_inf < eps (the exit test of Algorithm 2).
 * Each inner iteration starts from the current outer iterate, theta^(0) =
 * delta^(s): with a zero inner start at every outer step, as printed, the
 * fixed point would be (Upsilon_L^-1 - Xi~)^-1 r_delta instead of the
 * solution.  Honours lq2d_set_precision.  Device buffers as in
 * lq2d_solve_device; outer_iterations and rel_kkt_residual are optional
 * outputs.  LQ2D_ENOCONV when max_outer steps do not pass the exit test
 * (outputs still written). */
int lq2d_solve_nbjm_device(lq2d_problem *h, double eps, int inner_L, int max_outer,
                           void *d_x, void *d_u, void *d_costate,
                           int *outer_iterations, double *rel_kkt_residual, void *stream);

/* y = Delta d (Section II-B, the operator product of Algorithm 1), device
 * buffers [T+1][K*N][n].  Returns after the work on `stream` is complete. */
int lq2d_apply_delta_device(lq2d_problem *h, const void *d_in, void *d_out, void *stream);

/* q = D_S r: S outer x L inner NBJM sweeps from zero starts (Algorithm 2;
 * Theorem posdef_preconditioner), device buffers [T+1][K*N][n]. */
int lq2d_apply_precond_device(lq2d_problem *h, int outer_S, int inner_L, const void *d_r,
                              void *d_q, void *stream);

/* q_r = D_S r_r for up to 32 right-hand sides r_r of one problem at once
 * (Algorithm 2, S outer x L inner sweeps from zero starts; Theorem
 * posdef_preconditioner), the right-hand sides sharing Delta, its splittings
 * and the banded factors of Phi_bar (Section IV-B).  Every sweep step
 * applies each 2n x 2n factor block and the pair-row's coupling to the
 * neighbouring nodes to all 32 right-hand sides as one matrix product on
 * the tensor cores: TF32 operands (10-bit mantissa) with FP32
 * accumulation, FP32 iterates.  The result is therefore D_S r only to about
 * 1e-3 relative, enough for a preconditioner.
 *   nrhs       1..32
 *   d_r, d_q   device buffers [nrhs][T+1][K*N][n] (FP64), right-hand side
 *              r of index i at d_r + i (T+1) K N n
 * Needs n = 4 and T + 1 <= 65535 (LQ2D_EINVAL otherwise).  The first call allocates the
 * operands of this path (about 16 (T+1) K N n bytes per vector, four
 * vectors, plus the rearranged factors) and every setup invalidates them;
 * they are rebuilt on the next call.  Returns after the work on `stream`
 * is complete. */
int lq2d_apply_precond_multi_device(lq2d_problem *h, int nrhs, int outer_S, int inner_L, const void *d_r,
                                    void *d_q, void *stream);

/* Solves the problem for up to 32 initial states at once (config: many x0
 * of one instance): Algorithm 1 runs for each right-hand side r_delta(x0_r)
 * side by side, sharing every product with Delta and every preconditioner
 * sweep, with the tensor-core preconditioner of
 * lq2d_apply_precond_multi_device.  Precision as in precision mode 2: r,
 * delta and d are FP64, the product Delta d is FP32 with the true residual
 * replacing the recurrence one after each drop of 1e4 (per right-hand
 * side), beta is the flexible ratio; a right-hand side that meets the
 * tolerance stops moving while the others go on.  At exit the true
 * residual of every right-hand side is checked; one that fails restarts
 * from its iterate (at most LQ2D_OPT_MAX_RESTARTS times).  The stop test is
 * the relative 2-norm, ||r_delta - Delta delta||_2 <= tol ||r_delta||_2,
 * whatever LQ2D_OPT_STOP_MODE says.  Boundary terms set by lq2d_set_affine
 * apply to every right-hand side.
 *   nrhs       1..32
 *   d_x0s      device [nrhs][K*N][n], the initial states gamma_r
 *   d_x, d_u, d_costate  device outputs [nrhs][T+1][K*N][n], [nrhs][T][K*N][m],
 *              [nrhs][T+1][K*N][n]; any may be NULL
 *   iterations, rel_residuals  host outputs [nrhs] (may be NULL): PCG steps
 *              and final true relative residual of each right-hand side
 * Needs n = 4 (LQ2D_EINVAL otherwise).  Uses the handle's solution
 * buffers as scratch: lq2d_get_solution_device afterwards returns the last
 * right-hand side's solution.  LQ2D_ENOCONV when max_iter is reached before
 * every right-hand side converged (outputs still written), LQ2D_EBREAKDOWN,
 * LQ2D_ETIMEOUT as for lq2d_solve.  Returns after the work on `stream` is
 * complete. */
int lq2d_solve_multi_device(lq2d_problem *h, int nrhs, const void *d_x0s, double tol, int outer_S, int inner_L,
                            int max_iter, void *d_x, void *d_u, void *d_costate, int *iterations,
                            double *rel_residuals, void *stream);

/* Chooses the sweep tile (LQ2D_OPT_SWEEP_THREADS, and for the n = 4 FP32
 * sweeps also LQ2D_OPT_SWEEP_STEPS) for this problem's shape and the
 * handle's current precision mode by timing: runs D_S (S outer x L
 * inner sweeps, Algorithm 2) once as warm-up and then `reps` times with each
 * candidate width (32, 64, 128, 256; for n = 4 in FP32 each compiled
 * (width, steps) schedule), with CUDA events on `stream`, and keeps
 * the fastest for later solves of this precision mode (FP64 and FP32 sweeps
 * keep separate choices).  The problem's right-hand side is the input; the
 * handle's solution buffers are not touched.
 *   threads (out, may be NULL): the chosen width
 *   ms      (out, may be NULL): its time per D_S application, milliseconds
 * Errors: LQ2D_EINVAL for bad S, L or reps < 1; LQ2D_ECUDA (the previous
 * width is kept).  Returns after the work on `stream` is complete. */
int lq2d_autotune(lq2d_problem *h, int outer_S, int inner_L, int reps, int *threads, double *ms,
                  void *stream);

/* y = Delta d as lq2d_apply_delta_device computes it, for callers that may
 * not allocate device memory: it takes the raw problem blocks (device
 * pointers, layouts as in lq2d_create) instead of a handle, and keeps its
 * scratch (Q^-1, Q_T^-1, B R^-1 B' per node, and the intermediate
 * Q~^-1 A~' d) in one fixed array compiled into the library.  The paper has
 * no counterpart; it is an allocation-free form of the Delta product.
 *   Callers: a controller that re-evaluates Delta d in a fixed-period loop,
 *   where an allocator call adds latency it cannot bound, and host
 *   frameworks that own every device allocation and pass libraries only
 *   the buffers they manage.
 *   Limit: (T+1)*K*N*n + 3*K*N*n*n + 1 <= 2^21 doubles (16 MiB, held on
 *   every GPU that loads the library until the process exits); larger
 *   problems return LQ2D_EINVAL with the required size in the message.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and caches it.  With
 *   lazy module loading (the CUDA default) that first call also loads the
 *   library's device code on the device, which reserves the array, so
 *   make it during set-up, before a fixed-period loop and before any
 *   stream capture.  All calls share the array and it keeps the last
 *   call's contents; calls whose work overlaps on the GPU race on it.
 *   Calls no cudaMalloc or cudaFree.  Every call is synchronous: it reads
 *   a status word back on `stream` and returns after the work on `stream`
 *   is complete.  d_in and d_out must not overlap (LQ2D_EINVAL).
 *   LQ2D_ENOTPD if Q, Q_T or R is not SPD. */
int lq2d_apply_delta_static(int K, int N, int T, int n, int m,
                            const double *d_A_self, const double *d_A_nbr, const double *d_B,
                            const double *d_Q, const double *d_R, const double *d_Q_T,
                            const void *d_in, void *d_out, void *stream);

/* Many problems (uneven K, N, T, each with its own data and x0) solved by
 * one launch: a CUDA graph with one independent chain per problem (the
 * initial residual and preconditioner, the device loop of Algorithm 1
 * under a conditional while node, the recovery of x, u and the KKT
 * residual), built on the first lq2d_batch_solve and rebuilt only when tol,
 * S, L, max_iter or a problem's precision/preconditioner/stop options
 * change.  The problems stay owned by the caller and must outlive the
 * batch; their data may be replaced with lq2d_update(_device) between
 * solves without a rebuild.  Results stay in each problem: read them with
 * lq2d_get_solution_device and lq2d_get_stats. */
typedef struct lq2d_batch lq2d_batch; /* opaque, library-owned */
int lq2d_batch_create(lq2d_batch **out, int count, lq2d_problem *const *problems);
/* iterations [count], rel_kkt_residuals [count] and statuses [count] are
 * optional outputs; the return value is LQ2D_OK when every problem
 * converged, else the first failing status.  Returns after the work on
 * `stream` is complete. */
int lq2d_batch_solve(lq2d_batch *b, double tol, int outer_S, int inner_L, int max_iter,
                     int *iterations, double *rel_kkt_residuals, int *statuses, void *stream);
void lq2d_batch_destroy(lq2d_batch *b);

/* Options of a batch (lq2d_batch_set_option / lq2d_batch_get_option).
 * When every problem has n = 4, precision mode 0 and the NBJM
 * preconditioner, and S*L <= 14, the loop of Algorithm 1 runs persistently
 * for the whole batch: one conditional loop whose body is one launch of the
 * Delta product (two kernels) and one launch per NBJM sweep for all
 * problems, each a single wave of CTAs sized by occupancy that pull
 * (problem, node-time block) or (problem, column pair, time tile) units from
 * a device work queue; problems that have stopped skip their units.  Its
 * sweeps are one-sided (the queue fills the GPU without the two-ended
 * solve's extra warps): each problem's arithmetic and reductions are those
 * of its single solve with the same sweep width and LQ2D_OPT_TWISTED = 0,
 * so those results are equal bit for bit.  Other batches keep one chain per
 * problem in the graph, with each problem's own options. */
enum {
  LQ2D_BATCH_PERSISTENT = 1,      /* 1 (default): use the persistent loop when the problems allow it; 0: never */
  LQ2D_BATCH_THREADS = 2,         /* CTA width of its sweeps: 32, 64 (default) or 128 */
  LQ2D_BATCH_USES_PERSISTENT = 3  /* read only: 1 if the last built graph runs the persistent loop */
};
/* Setting an option makes the next lq2d_batch_solve rebuild its graph.
 * Errors: LQ2D_EINVAL for an unknown option or value. */
int lq2d_batch_set_option(lq2d_batch *b, int option, int value);
int lq2d_batch_get_option(const lq2d_batch *b, int option, int *value);
/* Chooses LQ2D_BATCH_THREADS by timing: for each width (32, 64, 128) runs
 * one D_S application (S outer x L inner sweeps of Algorithm 2, right-hand
 * sides as input) of every problem through the persistent sweep launches,
 * once as warm-up and then `reps` times with CUDA events on `stream`, and
 * keeps the fastest.  threads and ms (per D_S of the whole batch) are
 * optional outputs.  Errors: LQ2D_EINVAL when the batch cannot run the
 * persistent loop or for bad S, L, reps; LQ2D_ECUDA.  Leaves every
 * problem's solver state reset; returns after the work on `stream` is
 * complete. */
int lq2d_batch_autotune(lq2d_batch *b, int outer_S, int inner_L, int reps, int *threads, double *ms,
                        void *stream);
/* Copies the solution of the problem's last solve (x, u, costate, layouts as
 * in lq2d_solve_device) into device buffers; any pointer may be NULL. */
int lq2d_get_solution_device(lq2d_problem *h, void *d_x, void *d_u, void *d_costate, void *stream);

int lq2d_set_option(lq2d_problem *h, int option, double value);
/* The current value of an option (LQ2D_OPT_SWEEP_THREADS and
 * LQ2D_OPT_TWISTED: as the current precision mode's sweeps use it, e.g.
 * after lq2d_autotune).  LQ2D_EINVAL for an unknown option or NULL. */
int lq2d_get_option(const lq2d_problem *h, int option, double *value);
int lq2d_get_stats(const lq2d_problem *h, lq2d_stats *out);

/* Precision of the preconditioner (Algorithm 2) and of the Delta product.
 *   0: FP64 everywhere (default).
 *   1: the sweeps, the banded factors of Phi_bar and the Omega~/Xi~ blocks in
 *      FP32; the residual, iterate, direction, Delta d, every dot product and
 *      the stop test stay FP64.  The FP32 preconditioner is not exactly
 *      symmetric, so the next direction uses the flexible ratio
 *      q_new'(r_new - r_old) / mu_old.  The tolerance still applies to the
 *      FP64 residual.
 *   2: as 1, and the product Delta d inside the Krylov loop in FP32 too.
 *      The recurrence residual then drifts from the true one at FP32 level,
 *      so whenever it has dropped by 1e4 since the last replacement, the
 *      residual is recomputed in FP64 from the iterate, r = r_delta -
 *      Delta delta, and replaces it on the device; the search direction is
 *      kept, so the iteration continues without a restart (a reliable
 *      update; lq2d_stats.residual_replacements counts them).  Residual
 *      recomputation, the direction update and every dot product stay FP64;
 *      the stop test is confirmed on the true residual at exit.
 * Modes 1 and 2 allocate FP32 copies of the operands on first use and
 * refresh them at every setup. */
int lq2d_set_precision(lq2d_problem *h, int mode);

/* Frees every device buffer of the handle; NULL is a no-op. */
void lq2d_destroy(lq2d_problem *h);

/* Message of the last non-OK status on this thread. */
const char *lq2d_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LQ2D_H */
