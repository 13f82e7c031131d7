/*
 * pdhg.h -- C ABI of the GB300 restarted-PDHG library (libpdhg.so).
 *
 * Problem (Section 2 of "Hybridizing PDHG and Interior-Point Methods"):
 *     primal  min c^T x   s.t.  A x = b,  x >= 0        (A is m x n)
 *     dual    max b^T y   s.t.  A^T y + z = c,  z >= 0
 * with residuals r_P = b - A x, r_D = c - A^T y - z and the relative
 * termination test of Section 2:
 *     ||r_P||_2 <= eps (1 + ||b||_2),  ||r_D||_2 <= eps (1 + ||c||_2),
 *     |c^T x - b^T y| <= eps (1 + |c^T x| + |b^T y|).
 * For a PDHG iterate the library takes z = max(0, c - A^T y).
 *
 * The iteration, scaling, step size and restart rule are a stated reading of
 * the paper's "PDHG following cuPDLP+" (Section 4.1); Algorithm 1 (Section
 * 3.1) is computed on device by pdhg_warmstart_point.
 *
 * Conventions for every entry point:
 *  - Return value: a pdhg_status.  Negative values mean the call failed and
 *    the context (if any) must only be destroyed; pdhg_last_error() then
 *    holds a message (thread-local, valid until the next call on the thread).
 *  - Array arguments are borrowed for the duration of the call and copied;
 *    the caller keeps ownership.  They are HOST pointers unless the context
 *    was created with options.io_on_device = 1, in which case they are
 *    device pointers on this GPU, read and written in order on
 *    options.stream.  A NULL output pointer is skipped.
 *  - Outputs are float64 in the original (unscaled) model unless stated.
 *  - No C++ exception or process exit crosses this boundary.
 *  - A context is not thread-safe; distinct contexts may be used from
 *    distinct threads on distinct streams.
 */
#ifndef PDHG_H
#define PDHG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdhg_ctx pdhg_ctx;

typedef enum pdhg_status {
  PDHG_OK = 0,
  PDHG_CONVERGED = 0,        /* termination test met                         */
  PDHG_MAX_ITER = 1,         /* iteration limit reached first                */
  PDHG_NUMERICAL_ERROR = 2,  /* NaN/Inf met in the iterate or the residuals  */
  PDHG_TIMEOUT = 3,          /* a bounded device wait gave up                */
  PDHG_INVALID_ARG = -1,
  PDHG_CUDA_ERROR = -2,
  PDHG_OOM = -3
} pdhg_status;

enum { PDHG_FP64 = 0, PDHG_FP32_MIXED = 1 };

typedef struct pdhg_options {
  int32_t precision;       /* PDHG_FP64 (default) or PDHG_FP32_MIXED: A~ and the
                              iterates in float32 with float32-accumulated SpMV;
                              norms, gap, restart rule and step/weight updates in
                              float64 */
  int32_t eval_freq;       /* F: iterations between evaluations (default 64)    */
  int32_t ruiz_iters;      /* Ruiz infinity-norm rounds (default 10)            */
  int32_t pock_chambolle;  /* 1: one Pock-Chambolle step after Ruiz (default 1) */
  double eta_safety;       /* eta = eta_safety / sigma_max(A~) (default 0.95)   */
  int32_t power_max_iter;  /* power-iteration limit (default 200)               */
  double power_rel_tol;    /* power-iteration stop on rel. change (1e-10)       */
  double beta_sufficient;  /* restart if KKT <= 0.2 KKT(last restart)           */
  double beta_necessary;   /* ... or <= 0.8 KKT(last) and no progress           */
  double beta_artificial;  /* ... or iterations since restart >= 0.36 k         */
  double theta;            /* primal-weight smoothing (0.5)                     */
  int32_t io_on_device;    /* 1: every array argument is a device pointer       */
  void* stream;            /* cudaStream_t to run on; NULL: a library stream    */
  int32_t use_graphs;      /* 1 (default): replay each F-iteration chunk as a
                              CUDA graph                                        */
  int32_t autotune;        /* 1 (default): time SpMV tile schedules at create   */
  int32_t tile_nnz;        /* 0: autotune; > 0: segmented SpMV tiles of at most
                              tile_nnz nonzeros, walked with 8 (tile_nnz <=
                              2044), 16 (<= 4092) or 32 nonzeros per thread;
                              -4 / -8: the vector SpMV with 4 / 8 lanes per row
                              (matrices whose rows all have <= 256 nonzeros;
                              others fall back to segmented)                   */
  int32_t kernel_timing;   /* 1: sample primal/dual kernel durations with CUDA
                              events during pdhg_solve                          */
  int32_t verbose;
  int32_t method;          /* 0 (default): restarted averaged PDHG; 1: reflected
                              Halpern iteration of cuPDLP+, the solver Section
                              4.1 says its PDHG follows: z <- lam((1 + rho) T(z)
                              - rho z) + (1 - lam) z0, lam = (t+1)/(t+2), z0 =
                              the last restart point, T = one PDHG step; the
                              evaluation's second candidate is T(z) (single-LP
                              contexts only)                                   */
  double reflection;       /* rho of method 1, in [0, 1] (default 1)           */
  int32_t spmv_layout;     /* FP32_MIXED single-LP half-steps (the products
                              A~^T y and A~ x+ of Section 2's iteration):
                              0 (default): the faster combination of CSR
                              tiles and column panels, timed at create when
                              autotune is on and nnz >= 2^20 (CSR tiles
                              otherwise);
                              1: CSR tiles only; 2: column panels wherever
                              they apply.  Column panels stage a slice of the
                              gathered vector in shared memory and apply when
                              (panels x rows) <= 2 nnz + rows and nnz <= 2^30;
                              float64 and batched contexts use CSR tiles.  */
  int32_t panel_width;     /* 0 (default): the widest panel shared memory holds
                              (about 49k columns); > 0: at most this many
                              columns per panel (rounded down to a multiple of
                              8, at least 8)                                   */
  double fp32_screen;      /* PDHG_FP32_MIXED: the Section 2 test evaluated on
                              the float32 caches is a screen that passes at
                              eps_rel * fp32_screen (default 1, at most 1e6);
                              the screened candidate is then re-evaluated with
                              every product recomputed in float64, and only
                              that test at eps_rel ends the solve (a rejected
                              candidate continues: the restart rule of that
                              evaluation is applied as usual)                  */
  int32_t omega_rule;      /* primal weight at a restart, with dx, dy the primal
                              and dual distances moved since the last restart
                              point (both > 1e-10, else omega is kept):
                              0 (default): exp(theta log(dy/dx) + (1 - theta)
                              log omega);
                              1: PID control of log omega, the reading of
                              cuPDLP+'s primal-weight control (Section 4.1
                              names cuPDLP+): e = log(dy/dx) - log omega,
                              I += e, log omega += pid_kp e + pid_ki I +
                              pid_kd (e - e_prev)                              */
  double pid_kp;           /* proportional gain (default 0.99)                  */
  double pid_ki;           /* integral gain (default 0.01)                      */
  double pid_kd;           /* derivative gain (default 0)                       */
  int32_t persistent;      /* batched contexts: 0 (default): each F-iteration
                              chunk is a CUDA graph of per-half-step launches;
                              1: the whole solve is one cooperative launch
                              (every block resident), the phases separated by
                              grid-wide barriers whose waits are bounded; it
                              runs the SpMV schedules of 8 nonzeros per thread
                              (full tiles) whatever the tuner picked           */
  int32_t wait_limit_ms;   /* bound of one device-side wait (default 1000): a
                              grid barrier of the persistent batched solve,
                              or the bulk copy of a column panel of the
                              gathered vector; a wait past it ends the solve
                              with PDHG_TIMEOUT                               */
  int32_t wait_test;       /* 1: every grid barrier waits for one arrival more
                              than the grid has, and every column-panel load
                              for 16 bytes more than its copies deliver, so
                              the bounded waits run out (tests the
                              PDHG_TIMEOUT path; default 0)                   */
  int32_t step_rule;       /* 0 (default): constant step eta = eta_safety /
                              sigma_max; 1: PDLP's adaptive step (Applegate et
                              al. 2021): each attempt's move (dx, dy) allows
                              eta_max = (w||dx||^2 + ||dy||^2/w) /
                              (2|dy^T A~ dx|), w the primal weight; accepted
                              when eta <= eta_max, else undone; next step
                              min((1-(j+1)^-0.3) eta_max, (1+(j+1)^-0.6) eta)
                              with j the attempts so far; averages weighted
                              by the accepted steps; attempts count as
                              iterations.  Single LPs, method 0, CSR tiles
                              (spmv_layout 2 and batches: PDHG_INVALID_ARG) */
} pdhg_options;

/* Fill *opt with the defaults listed above. */
void pdhg_default_options(pdhg_options* opt);

/* Create a solver context for one LP (Section 2 standard form).
 *  m, n       rows and columns of A (m >= 1, n >= 1)
 *  row_ptr    int32[m+1], row_ptr[0] = 0, non-decreasing, nnz = row_ptr[m]
 *             <= 2^31 - 2^16 (int32 tile indexing)
 *  col        int32[nnz], strictly increasing within each row, in [0, n)
 *  val        float64[nnz], finite
 *  b, c       float64[m], float64[n], finite
 *  opt        NULL for defaults
 * On device: builds A^T (stable by row), scales (Ruiz + Pock-Chambolle),
 * estimates sigma_max(A~) by power iteration, sets omega_0 = ||c~||/||b~||,
 * and starts from x = 0, y = 0.  Invalid CSR -> PDHG_INVALID_ARG.  */
pdhg_status pdhg_create(pdhg_ctx** out, int32_t m, int32_t n, const int32_t* row_ptr,
                        const int32_t* col, const double* val, const double* b,
                        const double* c, const pdhg_options* opt);

/* Run restarted PDHG from the context's current state until the Section 2
 * test holds with eps = eps_rel (evaluated every F iterations, on the current
 * iterate first, then the running average) or the cumulative iteration count
 * reaches max_iter.  Returns PDHG_CONVERGED, PDHG_MAX_ITER or an error.
 * PDHG_FP32_MIXED: the test on the float32 caches only screens; the solve
 * converges when the screened iterate passes the test in float64 (x~, y~
 * widened to float64, A~x~ and A~^T y~ recomputed from the float64 scaled
 * matrices), so a converged float32-mixed solve meets the test at eps_rel
 * exactly as pdhg_get reports it.  If a column-panel SpMV's bounded wait for
 * its bulk copy ran out (options.wait_limit_ms), the call returns
 * PDHG_TIMEOUT and pdhg_last_error says so; the iterate is then not
 * meaningful, the context stays usable.  */
pdhg_status pdhg_solve(pdhg_ctx* ctx, double eps_rel, int64_t max_iter);

/* The returned iterate (the one that passed the test, else the current one)
 * in the original model: x[n], y[m], z[n] = max(0, c - A^T y), and
 * ||r_P||_2, ||r_D||_2, |c^T x - b^T y|, all evaluated in float64.  */
pdhg_status pdhg_get(pdhg_ctx* ctx, double* x, double* y, double* z, double* r_P,
                     double* r_D, double* gap);

/* The PID primal-weight controller's state (options.omega_rule = 1): the
 * sum of its errors so far and its last error; part of a checkpoint beside
 * pdhg_get_state / pdhg_set_state.  Single-LP contexts.  */
pdhg_status pdhg_get_pid_state(pdhg_ctx* ctx, double* integral, double* prev_error);
pdhg_status pdhg_set_pid_state(pdhg_ctx* ctx, double integral, double prev_error);

/* The adaptive step's state (options.step_rule = 1): the next attempt's step
 * eta, the sum of the accepted steps since the last restart (the averages'
 * weight), and the rejected attempts so far (get only); part of a checkpoint
 * beside pdhg_get_state / pdhg_set_state.  Setting also resets tau, sigma and
 * the next averaging weight from them.  eta > 0, eta_sum >= 0, finite; else
 * PDHG_INVALID_ARG.  Single-LP contexts.  */
pdhg_status pdhg_get_step_state(pdhg_ctx* ctx, double* eta, double* eta_sum, int64_t* rejects);
pdhg_status pdhg_set_step_state(pdhg_ctx* ctx, double eta, double eta_sum);

/* Float64 checks of float32-mixed candidates in the last solve (single LP
 * or summed over a batch): how many screened candidates were re-evaluated
 * in float64 and how many of them failed the Section 2 test there and were
 * iterated on.  Float64 contexts report 0, 0.  */
pdhg_status pdhg_get_fp64_checks(pdhg_ctx* ctx, int64_t* checks, int64_t* rejects);

/* Iterations done, restarts taken, the Section 4.3 maximum violation
 * max(||r_P||_inf, ||r_D||_inf, x^T z / (1 + |c^T x|)) of the returned
 * iterate, whether it is the running average (1) or the current iterate (0),
 * and the status of the last pdhg_solve.  */
pdhg_status pdhg_get_info(pdhg_ctx* ctx, int64_t* iters, int64_t* restarts,
                          double* max_violation, int32_t* chosen_average,
                          int32_t* last_status);

/* Algorithm 1's centered start point (Section 3.1), computed on device on the scaled
 * returned iterate (x~, y~, z~ = max(0, c~ - A~^T y~)):
 *   mu = max(x~^T z~ / n, mu_min); per j lift to alpha_min, then move the
 *   smaller of the pair toward mu / (other) within +-delta_max, then the
 *   other toward mu / (updated first); a tie moves z' first.
 * Outputs x_ws[n], y_ws[m], z_ws[n] in the scaled model, or mapped back to
 * the original model (x = D_c x', y = D_r y~, z = z' / D_c) if unscaled = 1;
 * *mu_target receives mu.  The paper's values: mu_min = alpha_min = 1e-6,
 * delta_max = 1e-4.  */
pdhg_status pdhg_warmstart_point(pdhg_ctx* ctx, double mu_min, double delta_max,
                                 double alpha_min, int32_t unscaled, double* x_ws,
                                 double* y_ws, double* z_ws, double* mu_target);

/* Scaling and step data: D_r[m], D_c[n] (A~ = D_r A D_c), sigma_max(A~)
 * estimate, eta, omega_0 and the power iterations taken.  */
pdhg_status pdhg_get_scaling(pdhg_ctx* ctx, double* D_r, double* D_c, double* sigma_max,
                             double* eta, double* omega0, int32_t* power_iters);

/* The stored transpose with the ORIGINAL values: row_ptr_t[n+1],
 * col_t[nnz] (row indices of A, increasing within each row of A^T),
 * val_t[nnz].  */
pdhg_status pdhg_get_transpose(pdhg_ctx* ctx, int32_t* row_ptr_t, int32_t* col_t,
                               double* val_t);

/* Checkpoint: scaled iterate x[n], y[m], running averages, last restart point,
 * and scalars[8] = {omega, k, t, restarts, kkt_last, kkt_prev, eta, 0}.
 * pdhg_set_state restores the same fields and recomputes the A~x caches (of
 * x, of the running average and of the restart point) by one SpMV each, so a
 * resumed run matches an uninterrupted one up to the rounding of those caches
 * (the cached average of A~x is not A~ x_avg bit for bit) unless the caches
 * are restored too (pdhg_get_caches / pdhg_set_caches).  */
pdhg_status pdhg_get_state(pdhg_ctx* ctx, double* x, double* y, double* x_avg,
                           double* y_avg, double* x_last, double* y_last, double* scalars);
pdhg_status pdhg_set_state(pdhg_ctx* ctx, const double* x, const double* y,
                           const double* x_avg, const double* y_avg, const double* x_last,
                           const double* y_last, const double* scalars);

/* The A~x caches of a checkpoint, float64 [m] each (HOST or device as the
 * other arrays; NULL skips): A~x of the iterate, the running average of A~x
 * and A~x of the last restart point.  pdhg_set_caches after pdhg_set_state
 * makes a resumed run repeat the uninterrupted one bit for bit, for a
 * checkpoint taken at an iteration count that is not a multiple of
 * eval_freq (a solve that stops at max_iter = j * eval_freq does not apply
 * that evaluation's restart decision; the uninterrupted run does).  */
pdhg_status pdhg_get_caches(pdhg_ctx* ctx, double* Ax, double* Ax_avg, double* Ax_last);
pdhg_status pdhg_set_caches(pdhg_ctx* ctx, const double* Ax, const double* Ax_avg,
                            const double* Ax_last);

/* Evaluation log of the restart rule (one entry per evaluation with k % F == 0
 * that did not terminate; up to `cap` entries, oldest first):
 *   k[i]; flags[i] = restart | cand_is_average << 1 | r1 << 2 | r2 << 3 | r3 << 4;
 *   kkt[3 i + 0..2] = KKT(current), KKT(average), omega at evaluation.  */
pdhg_status pdhg_get_log(pdhg_ctx* ctx, int32_t cap, int32_t* count, int64_t* k,
                         int32_t* flags, double* kkt);

/* With options.kernel_timing = 1: mean duration (ms) of the sampled primal
 * (A^T y + projection) and dual (A x + dual step) half-steps of the last
 * pdhg_solve (one kernel on the CSR tiles, two on the column panels), and
 * the number of samples of each.  */
pdhg_status pdhg_get_kernel_timing(pdhg_ctx* ctx, double* primal_ms, double* dual_ms,
                                   int64_t* samples);

/* With options.kernel_timing = 1: the same samples split by kernel, ms[4]
 * (HOST) = {primal SpMV kernel, primal row pass, dual SpMV kernel, dual row
 * pass}.  A half-step on the CSR tiles is one fused kernel (its row pass
 * reads 0); on the column panels, the panel SpMV and the row pass that adds
 * the panel sums and applies the step.  */
pdhg_status pdhg_get_kernel_timing_parts(pdhg_ctx* ctx, double* ms, int64_t* samples);

/* Mean duration in ms of `reps` back-to-back launches (after 3 untimed) of,
 * ms[5] (HOST): {0: the primal half-step (A~^T y~ and the projected primal
 * step), 1: the dual half-step (A~ x~+ and the dual step), 2: one iteration
 * (both in turn), 3: the column-panel SpMV kernel of the primal half-step
 * alone, 4: that of the dual half-step (3, 4: 0 on the CSR tiles, where a
 * half-step is one fused kernel)}, timed with CUDA events on the context's
 * stream on its current iterate.  With options.step_rule = 1 the half-steps
 * are the adaptive step's own: the primal also saves the accepted state
 * and writes the attempt's x beside it, the dual also forms A~ times the
 * move and applies the acceptance test, followed by the kernel that undoes a
 * rejected attempt (timed with the dual).  Launches are back to back as in a solve
 * (programmatic dependent launch), with no event between them.  The solver
 * state is saved to a temporary device buffer first and restored after, so
 * a solve continues as if the call had not happened.  Single-LP contexts.  */
pdhg_status pdhg_time_kernels(pdhg_ctx* ctx, int32_t reps, double* ms);

/* Tile schedule picked for A (dual kernel) and A^T (primal kernel): nonzeros
 * per tile (at most), threads per block, tiles, and the SpMV variant (8, 16,
 * 32: segmented with that many nonzeros per thread; -4, -8: vector with that
 * many lanes per row).  Any pointer may be NULL.  */
pdhg_status pdhg_get_schedule(pdhg_ctx* ctx, int32_t* a_tile_nnz, int32_t* a_block,
                              int32_t* a_tiles, int32_t* at_tile_nnz, int32_t* at_block,
                              int32_t* at_tiles, int32_t* a_variant, int32_t* at_variant);

/* Column-panel layout of A (dual half-step) and A^T (primal half-step): the
 * number of panels (0: that half-step runs on the CSR tiles), the panel
 * width in columns, the pseudo-rows (a row's nonzeros inside one panel) and
 * the warp tiles.  Any pointer may be NULL; arrays are HOST int64[2] in the
 * order {A, A^T}.  */
pdhg_status pdhg_get_layout(pdhg_ctx* ctx, int64_t* panels, int64_t* panel_width,
                            int64_t* pseudo_rows, int64_t* tiles);

/* ---- batched solves -------------------------------------------------------
 * `count` independent LPs iterated together as one block-diagonal system: each
 * LP keeps its own scaling, step sizes, primal weight, restart state and
 * status (Section 2 test per LP); an LP that has passed its test is masked
 * while the others continue.  Sizes are given per LP; arrays are the
 * concatenation over LPs in order:
 *  m, n       HOST int32[count], each >= 1
 *  row_ptr    int32[sum(m) + count]: each LP's own row pointer (starting at 0)
 *  col        int32[sum nnz]: each LP's local column indices, strictly
 *             increasing within a row, in [0, n_l)
 *  val        float64[sum nnz];  b float64[sum m];  c float64[sum n]
 * Pointers are host or device as for pdhg_create (options.io_on_device).
 * Totals of rows, columns and nonzeros must fit in int32.  */
pdhg_status pdhg_batch_create(pdhg_ctx** out, int32_t count, const int32_t* m, const int32_t* n,
                              const int32_t* row_ptr, const int32_t* col, const double* val,
                              const double* b, const double* c, const pdhg_options* opt);

/* New right-hand sides for every LP of a batch with the same A: b[sum m],
 * c[sum n] (host or device as the context's other arrays), finite.  A's
 * scaling, its transpose, the power iteration and the tuned schedules are
 * kept (they depend on A only); b~ = D_r b, c~ = D_c c, the norms, the
 * initial primal weight and step sizes are recomputed, and every LP starts
 * again from x = 0, y = 0 with a fresh restart state, as a new context on
 * (A, b, c) with the same tile schedules would.  The active set of a previous
 * pdhg_batch_polish is dropped (polish again before pdhg_batch_adjoint).
 * Non-finite data -> PDHG_INVALID_ARG (the context stays usable).  */
pdhg_status pdhg_batch_set_rhs(pdhg_ctx* ctx, const double* b, const double* c);

/* Iterate every LP (in lockstep, F iterations per chunk) until each has
 * passed the Section 2 test with eps_rel or the iteration count reaches
 * max_iter.  lp_status (HOST int32[count] or NULL) receives each LP's
 * status; the return value is the largest of them (PDHG_CONVERGED only if
 * all converged).  With options.persistent = 1 the solve is one cooperative
 * launch; if one of its grid barriers waits past options.wait_limit_ms every
 * block returns and the call returns PDHG_TIMEOUT (every lp_status too): the
 * iterates are then not meaningful, the context stays usable (destroy it, or
 * restore a state before solving again).  */
pdhg_status pdhg_batch_solve(pdhg_ctx* ctx, double eps_rel, int64_t max_iter,
                             int32_t* lp_status);

/* Returned iterates in the original models, concatenated: x[sum n], y[sum m],
 * z[sum n]; per LP (HOST arrays [count], NULL skips): ||r_P||_2, ||r_D||_2,
 * |c^T x - b^T y|, the Section 4.3 maximum violation, iterations done.  */
pdhg_status pdhg_batch_get(pdhg_ctx* ctx, double* x, double* y, double* z, double* lp_r_P,
                           double* lp_r_D, double* lp_gap, double* lp_max_violation,
                           int64_t* lp_iters);

/* Algorithm 1 (Section 3.1) for every LP of the batch, as
 * pdhg_warmstart_point; lp_mu (HOST float64[count] or NULL) receives each
 * LP's mu_target.  */
pdhg_status pdhg_batch_warmstart_point(pdhg_ctx* ctx, double mu_min, double delta_max,
                                       double alpha_min, int32_t unscaled, double* x_ws,
                                       double* y_ws, double* z_ws, double* lp_mu);

/* ---- differentiation through the converged batch solution ---------------
 * At a PDHG fixed point x = max(0, x - tau (c - A^T y)) the positive set B
 * gives A_B x_B = b, x_j = 0 off B.  pdhg_batch_polish predicts B from each
 * LP's returned iterate by complementarity in the scaled model,
 * B = {j : x~_j > z~_j} with z~ = max(0, c~ - A~^T y~), and replaces x_B by the least-squares solution of A_B x_B = b (conjugate
 * gradients on the scaled normal equations, warm-started at the PDHG
 * iterate, stopping at relative residual cg_tol or cg_max_iter steps).
 *  x            float64[sum n] polished x in the original models (or NULL)
 *  lp_active    HOST int32[count]: |B| per LP (or NULL)
 *  lp_cg_iters  HOST int32[count]: CG steps per LP (or NULL)  */
pdhg_status pdhg_batch_polish(pdhg_ctx* ctx, double cg_tol, int32_t cg_max_iter, double* x,
                              int32_t* lp_active, int32_t* lp_cg_iters);

/* Vector-Jacobian product through x*(b, c) with B fixed by pdhg_batch_polish:
 * given grad_x = dL/dx (float64[sum n]) returns
 *   grad_b = A_B (A_B^T A_B)^{-1} grad_x_B   (float64[sum m], per LP)
 *   grad_c = 0                               (float64[sum n], or NULL)
 * (x_B does not move with c while B is fixed).  Requires a prior
 * pdhg_batch_polish; otherwise PDHG_INVALID_ARG.  */
pdhg_status pdhg_batch_adjoint(pdhg_ctx* ctx, const double* grad_x, double* grad_b,
                               double* grad_c, double cg_tol, int32_t cg_max_iter,
                               int32_t* lp_cg_iters);

/* The scaled start point of pdhg_warmstart_point, computed for caller-provided
 * DEVICE vectors with no device allocation by the library.  The paper has no
 * counterpart of this entry point.  It exists for callers that cannot call
 * cudaMalloc: an interior-point solver that owns a fixed device memory pool
 * and must not grow it, or a host thread that must not take the device
 * allocator's locks (for example a latency-bound solver loop).
 *  n              entries, 1 <= n <= 8,388,608 (larger n -> PDHG_INVALID_ARG;
 *                 the static scratch holds 4096 partial sums of 2048 entries)
 *  x, z           device float64[n]: the PDHG x and z of the scaled LP
 *  x_out, z_out   device float64[n]: x' and z' (may not alias x or z)
 *  mu_target      device float64[1] receiving mu, or NULL
 *  stream         cudaStream_t to run on (NULL: the legacy default stream)
 * The scratch is one file-scope device array per GPU that loads the library
 * (32 KB, held until the process exits), shared by every call: calls whose
 * work overlaps on the GPU race and must be serialised by the caller (for
 * example by using one stream).  Each call writes every scratch slot it
 * reads before reading it, so nothing needs clearing between calls.  The
 * first call on a device looks up the array's device address with that
 * device current and caches it for the process; make that first call
 * before any stream capture.  The cached address belongs to the device's
 * primary context: after cudaDeviceReset the library must not be used
 * again in the process.  The call is asynchronous: results are ready when
 * `stream` reaches it.  */
pdhg_status pdhg_centered_point_noalloc(int32_t n, const double* x, const double* z,
                                        double mu_min, double delta_max, double alpha_min,
                                        double* x_out, double* z_out, double* mu_target,
                                        void* stream);

/* Kernels this context has launched since pdhg_create (graph replays count
 * every kernel node).  */
pdhg_status pdhg_get_launch_count(pdhg_ctx* ctx, int64_t* launches);

/* Diagnostic (the paper has no counterpart): mean time in ms of `reps` launches
 * of a pass over the same nonzeros as the dual (on_a = 1: A~, gathering x) or
 * primal (on_a = 0: A~^T, gathering y) kernel that keeps only the memory work -
 * 128-bit loads of column indices and values with the same cache policy, the
 * random gathers and one multiply-add each - and no row logic, scan or
 * epilogue: the floor of gathering through L1/L2, which bounds the CSR-tile
 * kernels (the column-panel half-steps gather from shared memory and can go
 * below it).  Single-LP contexts; leaves the solver state unchanged.  */
pdhg_status pdhg_gather_floor(pdhg_ctx* ctx, int32_t on_a, int32_t reps, double* ms);

void pdhg_destroy(pdhg_ctx* ctx);

/* Message for the last failing call on this thread ("" if none). */
const char* pdhg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PDHG_H */
