/*
 * domdec.h -- C ABI of the GB300 (sm_103a) library for unbalanced entropic
 * domain decomposition (Medina, Nguyen, Schmitzer, "Domain decomposition for
 * entropic unbalanced optimal transport").
 *
 * Problem (Eq. unbalanced-problem with D_1 = D_2 = lam*KL, Section 5.1):
 *   min_pi <c,pi> + eps KL(pi | mu x nu) + lam KL(P_X pi | mu) + lam KL(P_Y pi | nu)
 * on X = Y = the N x N pixel grid {h (i, j)}, h = 1/N, c(x,y) = |x - y|^2.
 *
 * One call of domdec_iterate performs parallel DomDec iterations (Algorithm 4)
 * over partition A, then B, ... (Algorithm 2).  With the staggered strategies
 * each iteration is split into the 2^2 staggered sub-batches of Section 5.3
 * (otherwise one batch per partition) and, for each sub-batch:
 *   a1 nu_{-J}/nu on the cell's Y-box B_J            (Section 5.1, "Computing and handling nu_{-J}")
 *   a2-a4 the cell Sinkhorn with Newton Y-half and PD stopping
 *                                                     (Eqs. sinkhorn-X/Y-iteration, proxdiv-problem, PD-gap-KL)
 *   a5 the new basic-cell Y-marginals, C_i, H_i      (Eq. sinkhorn-primal, Definition 2.4)
 *   a6 GetWeights per domdec_params.strategy         (Proposition 4.3, Section 4.4 "staggered")
 *   a7 the convex combination, truncation, box refresh (Algorithm 4 last line; Section 5.3 truncation)
 * all on the GPU, enqueued on the stream given at domdec_init.
 *
 * Conventions for every entry point
 *  - Arrays of N*N doubles are row-major images (index i*N + j).
 *  - "host or device" pointers are accepted either way (copied with
 *    cudaMemcpyDefault); the caller keeps ownership of every pointer it passes.
 *  - Return value: DOMDEC_OK (0), a negative DOMDEC_E* error, or the
 *    positive warning DOMDEC_WNOTCONV.  Nothing aborts the process.  After an
 *    error the handle is "sticky": later calls return DOMDEC_ESTATE until
 *    domdec_free.
 *  - Calls marked "synchronises" wait for the handle's stream; the others
 *    only enqueue work.
 */
#ifndef DOMDEC_H
#define DOMDEC_H

#ifdef __cplusplus
extern "C" {
#endif

#define DOMDEC_OK        0
#define DOMDEC_WNOTCONV  1   /* warning: some cell solves hit maxit (Section 5.3, "Issues with non-convergence") */
#define DOMDEC_EINVAL   -1   /* bad argument: N % (2 s) != 0, mu/nu not finite and > 0, eps <= 0, lam not finite and > 0 ... */
#define DOMDEC_ENOMEM   -2   /* device allocation failed */
#define DOMDEC_ECUDA    -3   /* a CUDA runtime call failed */
#define DOMDEC_ETOOBIG  -4   /* a cell Y-box exceeds the kernel's shared-memory capacity (max_ny) */
#define DOMDEC_EARENA   -5   /* the box arena could not be grown after an overflow */
#define DOMDEC_ESTATE   -6   /* the handle is in an error state */
#define DOMDEC_ENOLIB   -7   /* reserved for bindings: library not loaded */
#define DOMDEC_EEMPTY   -8   /* a composite cell has no Y-support left: every member basic-cell marginal
                                fell below trunc_thr (Section 5.3 truncation); raise the masses or lower trunc_thr */
#define DOMDEC_ENONFINITE -9 /* a cell solve produced a non-finite value (NaN/Inf in the potentials or the
                                stopping gap) */

#define DOMDEC_STAGGERED 0   /* swift on each of the 4 staggered sub-batches (Section 4.4) */
#define DOMDEC_SWIFT     1   /* swift on the whole partition (Proposition 4.3, item 2) */
#define DOMDEC_SAFE      2   /* theta = 1/|J| (Proposition 4.3, item 1) */
#define DOMDEC_GREEDY    3   /* theta = 1 (Eq. GWFast); may diverge */
#define DOMDEC_LINE      4   /* GetWeights_line (Proposition 4.3): one zeta in [1/|b|, 1] for all cells of the
                                partition minimising the tracked score (convex in zeta; safeguarded Newton on
                                its derivative, at most 48 steps, on the device); not for batches */
#define DOMDEC_STAGGERED_LINE 5  /* the staggered sub-batches of DOMDEC_STAGGERED with GetWeights_line on each
                                    (zeta in [1/|b|, 1] per sub-batch); not for batches */

#define DOMDEC_FP32 0        /* cell Sinkhorn arithmetic in float (state, score, decision stay double) */
#define DOMDEC_FP64 1        /* cell Sinkhorn arithmetic in double */
#define DOMDEC_MIXED 2       /* domdec_full_sinkhorn only: float for coarse eps stages (eps >= 64 h^2); for the
                                fine ones double potentials and exponents with float exponentials of the kept
                                terms (relative error ~1e-7 per log-sum-exp, i.e. ~1e-7 eps in the potentials) */

typedef struct domdec_s* domdec_t;

typedef struct {
  double eps;          /* entropic strength eps > 0 */
  double lambda;       /* KL marginal penalty lam > 0, finite */
  int    basic_cell;   /* s: basic cells are s x s pixels, composite cells 2s x 2s; N % (2 s) == 0, s <= 16 */
  double err;          /* cell stopping tolerance: PD/lam <= err * |mu_J| (Section 5.3; paper: 2e-5);
                          err < 0 runs exactly maxit iterations per cell */
  double trunc_thr;    /* nu_i(y) < trunc_thr is dropped (Section 5.3; paper: 1e-15) */
  double tau;          /* greedy leniency: accept theta = 1 if E(1) <= (1 + tau) E (Section 5.3: 0.005); 0 = pure swift */
  int    strategy;     /* DOMDEC_STAGGERED | SWIFT | SAFE | GREEDY | LINE | STAGGERED_LINE */
  int    maxit;        /* cap on cell Sinkhorn iterations (status MAXIT when hit) */
  int    newton_maxit; /* cap on Newton steps per y in the Y-half */
  int    precision;    /* DOMDEC_FP32 | DOMDEC_FP64 */
  int    box_margin;   /* pixels added around B_J (0 in the paper) */
  int    max_ny;       /* capacity of a cell Y-box in the kernel (0: default 8192 for FP32, 4096 for FP64) */
  double arena_factor; /* box arena capacity in units of N*N doubles (0: default 48, and at least 8x the
                          initial plan).  When the new boxes of a sub-batch would not fit, the sweep kernels
                          stop changing the state from that sub-batch on; the next synchronising call grows
                          the arena (twice the capacity) and runs the skipped sub-batches, so the result is
                          the same as with a large arena (DOMDEC_EARENA only if growth fails repeatedly) */
  double eps_init;     /* eps of the warm-start duals passed to domdec_init (ignored without duals) */
  int    profile;      /* 1: time every kernel of a sweep with CUDA events on the handle's stream */
  int    spill_slots;  /* cells whose Y-box exceeds max_ny run from global memory slots (per sub-batch): 0 = default
                          (one per cell of the largest sub-batch, at most 1 GiB), > 0 = that many, < 0 = none
                          (such cells fail with DOMDEC_ETOOBIG) */
  int    cell_ctas;    /* CTAs per cell.  The cell kernel is a persistent grid over the resident CTAs that
                          takes the cells of a sub-batch in order of decreasing estimated work (the exp
                          terms of one iteration, from the box sizes).  A cell may be solved by a whole
                          thread-block cluster, its Y box split by rows over the CTAs (each CTA holds its
                          rows' Y-side arrays; the X-half log-sum-exp is combined from per-CTA parts).
                          0 = automatic: clusters of 4 CTAs (s <= 8) or 8 (s > 8) for the cells whose
                          work exceeds twice the mean work per CTA or whose box exceeds one CTA's
                          shared memory, one CTA for the others; 1 = one CTA per cell; 2, 4, 8 = every
                          cell whose box fits the cluster layout on a cluster of that many CTAs.  With
                          balance or cell_ti every cell runs on one CTA. */
  int    cell_ti;      /* 1: after each X-half of a cell solve, shift alpha by the t maximising the cell
                          dual along (alpha + t, beta - t) (closed form; not in the paper: it removes the
                          slow total-mass mode of the alternation when eps << lam, same fixed point);
                          0 (default): the paper's plain alternation */
  int    balance;      /* 1: balancing step after each cell solve (Section 5.3, Eq. balancing): targets
                          m_i = mu_bar(X_i) |nu_J| / mu_bar(X_J) from one more X-half; donors scale their
                          plan rows by m_i/|nu_i|, receivers share the donated mass at every y in
                          proportion to their deficits (nu_J preserved); C_i, H_i, P_X follow the
                          balanced plan.  Cells then run on one CTA each; not for batches.  0: off */
  double cell_split;   /* a cell goes to a cluster when its estimated work exceeds cell_split times the mean
                          work per resident CTA of its sub-batch (or when its box exceeds one CTA's shared
                          memory); 0: default 2.  domdec_autotune chooses it with the cluster size */
} domdec_params;

typedef struct {
  long long sweeps;          /* partition sweeps done */
  long long cell_solves;     /* cell subproblems solved */
  long long cell_iters;      /* cell Sinkhorn iterations (one X-half + one Y-half on one cell) */
  long long maxit_cells;     /* cell solves that stopped at maxit */
  long long greedy_steps;    /* sub-batches that accepted theta = 1 */
  long long safe_steps;      /* sub-batches that fell back to theta = 1/|b| */
  long long box_entries;     /* stored entries of all nu_i (memory diagnostic, Section 5.3 "Sparsity") */
  long long lse_terms;       /* exp terms of the cell log-sum-exp passes (algorithmic work of the cell kernel) */
  long long box_points;      /* sum over the cell solves of the Y-box size |B_J| (the points that the mixing
                                and box refresh of a7 read and write) */
  long long arena_regrows;   /* arena growths after a sub-batch's new boxes did not fit (see arena_factor) */
  int       max_cell_iters;  /* largest iteration count of one cell solve */
  int       max_ny;          /* largest cell Y-box seen */
  long long cluster_regroups;  /* sweeps rerun with the largest cluster size after a cell fit neither one CTA
                                  nor the cluster size in use (see domdec_autotune) */
} domdec_stats;

/* Fill *p with the defaults (eps = lambda = 1, s = 4, err = 2e-5,
 * trunc_thr = 1e-15, tau = 0, staggered, maxit = 2000, newton_maxit = 30,
 * FP32, margin 0).  Never fails. */
void domdec_default_params(domdec_params* p);

/* Create a solver for marginals mu, nu (N*N each, finite, > 0, host or
 * device) on the N x N grid (Assumption 4.2: full support).
 * Initial plan (Algorithm 2, pi_init):
 *   alpha0 == beta0 == NULL : pi0 = mu x nu (Section 4.4 toy set-up); every
 *                             nu_i lives on the full grid, so this needs
 *                             N*N <= max_ny.
 *   alpha0, beta0 != NULL    : pi0 = exp((alpha0 (+) beta0 - c)/eps_init) mu x nu,
 *                             e.g. the duals of a global Sinkhorn warm start
 *                             (Section 5.3, "Sinkhorn warm start"); N*N doubles each.
 *                             The box test of this plan keeps s*N doubles and
 *                             s*N floats per basic cell in shared memory
 *                             (about 12 s N bytes: N <= 1024 at s = 16 on GB300's
 *                             227 KB); larger s*N returns DOMDEC_ECUDA.
 * `stream` is a cudaStream_t (NULL = legacy default stream); all later work of
 * the handle is enqueued there.  Synchronises.  *out is NULL on failure. */
int domdec_init(domdec_t* out, const double* mu, const double* nu, int N,
                const domdec_params* p, const double* alpha0, const double* beta0,
                void* stream);

/* Start a new problem of the same size in an existing handle: copy mu, nu
 * (N*N, finite, > 0, host or device) and, if given, the warm-start duals
 * alpha0, beta0 at eps_init (as domdec_init), rebuild the initial plan, and
 * reset eps and err to the values given at domdec_init, the sweep count, the
 * counters, the decision log and the kernel timers.  The handle's device
 * allocations are reused (the box arenas are reallocated only if the new
 * initial plan does not fit them; the dual buffers are allocated on the first
 * call with duals), so a sequence of problems pays domdec_init's allocation
 * and set-up once.  A handle in an error state returns DOMDEC_ESTATE.
 * Synchronises. */
int domdec_reset(domdec_t h, const double* mu, const double* nu, const double* alpha0,
                 const double* beta0, double eps_init);

/* Autotuner of the cell kernel's launch: runs one sweep with each candidate --
 * one CTA per cell, and clusters of 2, 4 and 8 CTAs (as far as the handle's
 * cluster layout and the GPU allow) with the split thresholds 0.5, 1 and 2
 * (cell_split) -- times each with CUDA events on the handle's stream and keeps
 * the highest cell-iteration rate for later sweeps.  The timed sweeps are real
 * sweeps (they continue the alternation).  *cluster_ctas and *split_factor (if
 * not NULL) receive the choice.  Synchronises. */
int domdec_autotune(domdec_t h, int* cluster_ctas, double* split_factor);

/* Set the cell kernel's launch shape directly (for example the choice that
 * domdec_autotune made on another handle of the same workload):
 * cluster_ctas in {1, 2, 4, 8}, reduced to 1 when it exceeds the handle's
 * cluster layout or the clusters that fit the GPU; split_factor > 0 (the
 * cell_split threshold).  A sweep that meets a cell fitting neither one CTA
 * nor a cluster of this size halts before its cell solves, and the next
 * synchronisation reruns it with the layout's largest cluster size (counted
 * in domdec_stats.cluster_regroups); that size stays in use.  *effective_ctas
 * (if not NULL) receives the cluster size in use.  DOMDEC_EINVAL for other
 * values.  Enqueues nothing. */
int domdec_set_launch(domdec_t h, int cluster_ctas, double split_factor, int* effective_ctas);

/* Run n_sweeps partition sweeps (A, B, A, ... continuing the alternation of
 * earlier calls).  Enqueues only; errors found on the device are reported by
 * the next synchronising call. */
int domdec_iterate(domdec_t h, int n_sweeps);

/* Change eps between sweeps (eps-scaling stage).  The stored C_i and H_i make
 * the tracked score valid for the new eps without re-instantiating the plan. */
int domdec_set_eps(domdec_t h, double eps);

/* Change the cell stopping tolerance `err` of domdec_params between sweeps
 * (Section 5.3, "Stopping criterion"; the paper keeps it fixed at 2e-5, a
 * caller may tighten it as the global gap falls).  err < 0 runs maxit
 * iterations per cell. */
int domdec_set_tolerance(domdec_t h, double err);

/* Wait for the stream and report device-side errors / warnings: DOMDEC_WNOTCONV
 * if a cell solve stopped at maxit since the previous domdec_sync of this
 * handle (or since domdec_init), DOMDEC_EEMPTY / DOMDEC_ENONFINITE / ... for
 * errors (sticky).  Synchronises. */
int domdec_sync(domdec_t h);

/* out[0] tracked score E_hat = sum_i (C_i + eps H_i) + lam KL(P_X|mu) + lam KL(P_Y|nu)
 * (an upper bound of the plan's score, equal to it after greedy steps),
 * out[1] sum_i (C_i + eps H_i), out[2] lam KL(P_X|mu), out[3] lam KL(P_Y|nu),
 * out[4] |P_Y pi|, out[5] theta of the last sub-batch.  Synchronises. */
int domdec_score(domdec_t h, double out[6]);

/* P_X pi and P_Y pi of the current plan into PX, PY (N*N doubles each, host
 * or device; either may be NULL).  Synchronises. */
int domdec_plan_marginals(domdec_t h, double* PX, double* PY);

/* The stitched X-potential alpha (proof of Proposition 4.2) into alpha (N*N
 * doubles, host or device).  Synchronises. */
int domdec_duals(domdec_t h, double* alpha);

/* The tracked per-basic-cell terms of the score (reading R3 of the tracked
 * score, Section 4.4): C[i] = <c, pi_i> and H[i] = KL(pi_i | mu_i x nu) of the
 * plan part of basic cell i, mixed linearly by the step sizes, (N/s)^2 doubles
 * each in basic-cell order (row-major over the basic cells), host or device;
 * either may be NULL.  Synchronises. */
int domdec_basic_costs(domdec_t h, double* C, double* H);

/* Primal-dual certificate: out[0] = E_hat, out[1] = D(alpha, beta_star) with beta_star
 * from one global closed-form Y-half (Eq. sinkhorn-iters-ot), out[2] =
 * (E_hat - D)/|D| (Section 5.3, "Solution quality"), out[3] = L1 X-marginal
 * error |P_X - e^{-alpha/lam} mu|_1, out[4] = L1 Y-marginal error
 * |P_Y - e^{-beta_star/lam} nu|_1.  beta (N*N, host or device) receives beta_star
 * if not NULL.  Uses the separable FP64 log-sum-exp.  Synchronises. */
int domdec_pd_gap(domdec_t h, double out[5], double* beta);

/* Gradients of the unbalanced OT value S(mu, nu, x) = max D(alpha, beta)
 * (Eq. dual-problem, nu_- = 0, D_i = lam KL) with respect to the weights mu, nu
 * and the source positions x = (i, j)/N of the grid (row-major).  The paper
 * does not differentiate S; by the envelope theorem its derivatives at the
 * optimal potentials are those of D at fixed (alpha, beta):
 *   grad_mu(x) = eps |nu| - eps P_X(x)/mu(x) - lam (e^{-alpha(x)/lam} - 1)
 *   grad_nu(y) = eps |mu| - eps P_Y(y)/nu(y) - lam (e^{-beta(y)/lam} - 1)
 *   grad_x(x)  = 2 P_X(x) (x - T(x)),  T(x) = sum_y pi(x,y) y / P_X(x)
 * with pi = exp((alpha + beta - c)/eps) mu x nu never formed (separable
 * log-sum-exp passes over the grid; T carried as conditional means).
 * mu, nu (> 0), alpha, beta: N*N doubles, host or device.  precision:
 * DOMDEC_FP32 or DOMDEC_FP64 for the exponentials and sums of the summed
 * terms (either way their exponents are formed in double and terms below
 * 2^-32 (FP32) / 2^-64 (FP64) of the largest are skipped after a float test).  grad_mu, grad_nu (N*N), grad_x (2*N*N: d/dx_i,
 * d/dx_j per point) are host or device buffers, each may be NULL.
 * out[0] = D(alpha, beta), out[1] = |mu|, out[2] = |nu|, out[3] = |P_X pi|,
 * out[4] = |P_Y pi| (out may be NULL).  N <= 4096.  DOMDEC_EINVAL on a bad
 * argument or a non-positive weight / non-finite potential.  Allocates its
 * scratch with cudaMallocAsync on `stream`; synchronises. */
int domdec_uot_gradients(const double* mu, const double* nu, const double* alpha,
                         const double* beta, int N, double eps, double lambda,
                         int precision, double* grad_mu, double* grad_nu,
                         double* grad_x, double out[5], void* stream);

/* domdec_uot_gradients at the handle's state: alpha = the stitched X-potential
 * (as domdec_duals), beta = beta_star of one global closed-form Y-half of it
 * (as domdec_pd_gap; written to `beta` if not NULL).  On the handle's stream;
 * synchronises. */
int domdec_gradients(domdec_t h, int precision, double* grad_mu, double* grad_nu,
                     double* grad_x, double out[5], double* beta);

/* Basic-cell Y-marginals: box[4*i..4*i+3] = (k0, l0, H, W) of nu_i in Y pixel
 * coordinates (H*W == 0: empty), values of all boxes concatenated in basic-cell
 * order (row-major inside a box) into `values` (host, capacity `cap` doubles).
 * Returns the number of values (or a negative error; DOMDEC_EINVAL if cap is
 * too small).  box must hold 4 * (N/s)^2 ints.  Synchronises. */
long long domdec_basic_marginals(domdec_t h, int* box, double* values, long long cap);

/* Step-size decisions of the most recent sub-batches, oldest first: record k
 * is out[4k..4k+3] = (E_hat before the step, E(theta = 1), E(theta = 1/|b|),
 * chosen theta) -- the GetWeights_swift comparison of Proposition 4.3.
 * Writes at most max_records records (host buffer); returns how many, at most
 * the 4096 most recent.  Synchronises. */
int domdec_decision_log(domdec_t h, double* out, int max_records);

/* With params.profile = 1: accumulated device time (ms, CUDA events on the
 * handle's stream) and launch counts of the sweep kernels since the last reset,
 * per class: [0] cell solve (a1-a5), [1] step-size decision (a6),
 * [2] mix / truncate / box refresh (a7), [3] arena compaction.
 * reset != 0 clears the accumulators after reading.  Synchronises. */
int domdec_kernel_times(domdec_t h, double ms[4], long long launches[4], int reset);

/* Per-cell records of the most recent sub-batch (diagnostics): record j is
 * out[9j..9j+8] = (k0, l0, H, W of the cell's Y-box B_J, cell Sinkhorn
 * iterations, status (0 ok, 1 maxit, 2 empty, 3 too big, 4 non-finite), last
 * PD/lam, spill slot or -1, duration of the solve in microseconds on the GPU's
 * global timer).  Returns the number of records (<= max_records).
 * Synchronises. */
int domdec_cell_log(domdec_t h, double* out, int max_records);

/* Counters since domdec_init.  Synchronises. */
int domdec_get_stats(domdec_t h, domdec_stats* s);

/* Free all device memory of the handle (waits for its stream). */
void domdec_free(domdec_t h);

/* Static text for an error code. */
const char* domdec_error_string(int code);

/* Global unbalanced Sinkhorn (Eq. sinkhorn-iters-ot, nu_- = 0) on the N x N
 * grid: the comparator, and the warm start of Section 5.3.
 *   variant   DOMDEC_SINKHORN_DENSE     : the plain method, O(N^4) per half-step
 *             DOMDEC_SINKHORN_SEPARABLE : the same update evaluated as two 1-D
 *                                         log-sum-exp passes (|x-y|^2 separates
 *                                         over the axes), O(N^3) per half-step
 *   precision DOMDEC_FP32 | DOMDEC_FP64 | DOMDEC_MIXED (float stages while
 *             eps >= 64 h^2, double below)
 *   eps_start >= eps: geometric eps-scaling eps_start, eps_start/2, ... eps;
 *   at each stage iterate until PD/lam <= err*|mu| (Eq. PD-gap-KL, tested every
 *   check_every iterations) or maxit iterations.
 * mu, nu, alpha, beta: N*N doubles, host or device; beta (in) is the start
 * (NULL: 0), alpha/beta (out) the final duals if non-NULL.
 * out[0] total iterations, out[1] last PD/lam, out[2] primal E (= D + PD),
 * out[3] dual D.  Synchronises.  Returns DOMDEC_WNOTCONV if the last stage hit
 * maxit. */
#define DOMDEC_SINKHORN_DENSE     0
#define DOMDEC_SINKHORN_SEPARABLE 1
#define DOMDEC_SINKHORN_TI        4  /* or-ed into `variant`: translation step after each X-half (not in the
                                        paper): alpha += (lam/2) log(<e^{-alpha/lam},mu> / <e^{-beta/lam},nu>),
                                        the dual's maximiser along (alpha + t, beta - t); same fixed point.
                                        Not accepted by domdec_full_sinkhorn_noalloc. */
int domdec_full_sinkhorn(const double* mu, const double* nu, int N, double eps_start,
                         double eps, double lambda, int variant, int precision,
                         int maxit, double err, int check_every,
                         const double* beta_in, double* alpha, double* beta,
                         double out[4], void* stream);

/* Many independent problems swept together (many-instance batching): every
 * launch of a sweep covers the cells of one staggered sub-batch of all
 * instances, taken from a work queue by a persistent grid over the resident
 * CTAs in order of decreasing estimated work (from the current box sizes,
 * sorted on the device), the largest ones by thread-block clusters.  `handles` (n >= 1) must share precision and strategy and have done
 * the same number of sweeps; N, eps, lambda, s may differ.  The batch does not
 * own the handles; the handles stay usable (query them after
 * domdec_batch_sync) and must outlive the batch.  Work is enqueued on the
 * first handle's stream (give all handles the same stream). */
typedef struct domdec_batch_s* domdec_batch_t;
int domdec_batch_create(domdec_batch_t* out, domdec_t* handles, int n);
/* n_sweeps sweeps of every instance (A, B, ... as for domdec_iterate).  Enqueues only. */
int domdec_batch_iterate(domdec_batch_t b, int n_sweeps);
/* domdec_sync of every handle; returns the first error, else the largest warning.  Synchronises. */
int domdec_batch_sync(domdec_batch_t b);
/* Autotuner of the batch's cell kernel: runs one sweep with each candidate --
 * one CTA per cell, and clusters of 2 and 4 CTAs (as far as every instance's
 * cluster layout allows) for the cells whose estimated work exceeds 1, 2 or 4
 * times the mean work per CTA (plus the cells too large for one CTA) -- times
 * each with CUDA events, and keeps the highest cell-iteration rate for later
 * sweeps.  *cluster_ctas and *split_factor (if not NULL) receive the choice.
 * The timed sweeps are real sweeps of every instance.  Synchronises. */
int domdec_batch_autotune(domdec_batch_t b, int* cluster_ctas, double* split_factor);
void domdec_batch_free(domdec_batch_t b);

/* Allocation-free variant of domdec_full_sinkhorn (no counterpart in the
 * paper; it exists for callers that cannot allocate device memory while the
 * solver runs -- e.g. a process whose device memory is all handed to its own
 * pool at start-up, where cudaMalloc would fail or fragment it, or a loop that
 * must not pay the device-wide synchronisation of cudaMalloc/cudaFree).
 * Same arguments and results as domdec_full_sinkhorn, except:
 *  - mu, nu (N*N, > 0), alpha and beta (N*N outputs, also the iteration state)
 *    must be DEVICE pointers of the current device; beta_in may be NULL
 *    (start from 0), equal to beta, or another device pointer.  Each pointer
 *    is checked with cudaPointerGetAttributes before any work is enqueued:
 *    host memory (pinned or pageable) or memory of another device returns
 *    DOMDEC_EINVAL;
 *  - precision must be DOMDEC_FP32 or DOMDEC_FP64;
 *  - N*N must not exceed 65536 (N <= 256): larger grids return DOMDEC_ETOOBIG.
 * It calls no cudaMalloc, cudaFree or allocating library routine: all working
 * arrays live in one static device array of about 4.2 MB that every GPU which
 * loads the library keeps until the process exits.  Every call looks up that
 * array's address in the current context (cudaGetSymbolAddress, which
 * allocates nothing), so a cudaDeviceReset or another context of the same
 * device between calls is handled; the first call in a context loads the
 * module, so make it before any stream capture.  All calls share the one array, which keeps the last call's contents (the
 * status word it needs cleared is reset at the start of each call): calls that
 * overlap on the GPU -- from several streams or host threads -- race and
 * must be serialised by the caller.  Synchronises. */
int domdec_full_sinkhorn_noalloc(const double* mu, const double* nu, int N, double eps_start,
                                 double eps, double lambda, int variant, int precision,
                                 int maxit, double err, int check_every,
                                 const double* beta_in, double* alpha, double* beta,
                                 double out[4], void* stream);

/* Measurement helper (the paper has no counterpart): throughput probes that
 * give the roofline denominators of the cell kernel on the current device.
 * Runs, on all SMs, one kernel of 16 independent ex2.approx.ftz.f32 chains
 * per thread (x <- 2^{-x}: the exponential of every log-sum-exp term) and one
 * of 16 independent FP32 FFMA chains, `iters` loop passes of 16 operations per thread, each launched
 * twice with the second launch timed by CUDA events on `stream`.
 * out[0] ex2/s, out[1] ex2 per SM per clock, out[2] SM clock (MHz, from
 * clock64 against the global timer inside the ex2 kernel), out[3] FFMA/s,
 * out[4] FFMA per SM per clock, out[5] SM clock of the FFMA kernel,
 * out[6] SM count, out[7] blocks launched.  Allocates a few KB with
 * cudaMallocAsync; synchronises. */
int domdec_probe_peaks(int iters, double out[8], void* stream);

/* Diagnostics helper (the paper has no counterpart): y[i] = the library's
 * table-driven double logarithm of x[i] (the one the step-size decision
 * uses), for n DEVICE values x > 0 (finite, normal or subnormal); y is a device
 * buffer of n doubles.  Lets a test compare it with CUDA's log.
 * Synchronises `stream`. */
int domdec_probe_log(const double* x, double* y, int n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DOMDEC_H */
