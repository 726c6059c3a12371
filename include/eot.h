/*
 * eot.h -- C ABI of the GB300 entropic optimal transport solver (SK-NR).
 *
 * Problem (paper Sec. 2, Eq. primal_EOT / dual_EOT): two discrete probability
 * vectors a = alpha (n) and b = beta (m), a cost C (n x m) or two point clouds
 * X (n x d), Y (m x d) with C_ij = ||x_i - y_j||^2, and a regularisation eps > 0.
 * The solver returns Kantorovich potentials f (n), g (m); the coupling is
 * pi_ij = a_i b_j exp((f_i + g_j - C_ij) / eps)  (Eq. Optimal_P_epsilon).
 *
 * Methods: log-domain Sinkhorn (Eq. SK_iterations) and SK-NR(l) (Algorithm 4.1):
 * Sinkhorn sweeps followed by a Newton-Raphson step of the semi-dual objective
 * (Eq. def_Q_semi) restricted to l low-frequency modes V_l, accepted only if it
 * increases the semi-dual value; V_l comes from a partial eigendecomposition of
 * Op(pi) o Op(pi)^T (Eq. semidual_Hessian) at a larger eps' (Sec. 4), with eps
 * continuation (Sec. 5).
 *
 * Conventions shared by every entry point:
 *  - All arrays are dense and row-major.  Sizes are element counts.
 *  - Pointers are host or device memory as stated per call (eot_mem for the
 *    problem-level calls; "device" calls take device pointers only).
 *  - Inputs are borrowed for the duration of the call; outputs are caller
 *    allocated.  Nothing returned by the library needs freeing except an
 *    eot_server (eot_server_destroy).
 *  - Errors are return codes; no call throws or aborts.  eot_last_error()
 *    gives a thread-local message for the last non-OK status of this thread.
 *  - Device work runs on the CUDA device that is current on the calling thread.
 *    There is no CPU fallback: without a usable device every compute call
 *    returns EOT_ECUDA.
 */
#ifndef EOT_H
#define EOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EOT_OK = 0,             /* converged (or the call completed)                      */
    EOT_NOT_CONVERGED = 1,  /* max_iter reached; potentials are still returned        */
    EOT_PENDING = 2,        /* server: the request is not finished yet                */
    EOT_EINVAL = -1,        /* invalid argument (message in eot_last_error)           */
    EOT_ENOMEM = -2,        /* device allocation failed or admission budget exceeded  */
    EOT_ENUMERIC = -3,      /* non-finite values or potentials out of the safe range  */
    EOT_ETIMEDOUT = -4,     /* a bounded device wait gave up                          */
    EOT_ECUDA = -5,         /* CUDA runtime error or no usable device                 */
    EOT_ENOTFOUND = -6      /* server: unknown ticket                                 */
} eot_status;

typedef enum { EOT_MEM_HOST = 0, EOT_MEM_DEVICE = 1 } eot_mem;

/* Arithmetic of the O(nm) passes.
 *  FP64: float64 cost and float64 exponentials and sums in the Sinkhorn and SK-NR
 *        passes (small problems, tight tolerances); the modes are computed on a
 *        float32 copy of the cost.
 *  FP32: float32 stored cost; float32 exponentials and sums; potentials kept in
 *        float64 and the exponent f_i + g_j - C_ij formed without rounding error
 *        before the division by eps (so the marginal error can reach ~1e-7).
 *  SPLIT_TC: no stored cost: every pass forms C_ij = |x_i|^2 + |y_j|^2 - 2 x_i.y_j
 *        from X, Y (float32, 1 <= d <= 64) with the Gram products on the tensor
 *        cores (TF32 high + low parts, three products, float32 accumulation).
 *        The marginal test is met against this cost, which differs from the
 *        exact one by the float32 error of a dot product (|dC| ~ 1e-6 for unit
 *        scale points): potentials within ~1e-3 eps of the exact iterates.
 *        Plain Sinkhorn only (ell = 0: EOT_EINVAL otherwise). */
typedef enum { EOT_PREC_FP64 = 0, EOT_PREC_FP32 = 1, EOT_PREC_SPLIT_TC = 2 } eot_prec;

/* Semi-dual Hessian used by the Newton step (Eq. d2Q_semi):
 *  EOT_HESS_DIAG_ALPHA: -(1/eps) [V^T D_a V - W^T D_b^{-1} W], W = pi^T V
 *                       (D_r replaced by D_a; equal at the optimum; 3 passes per
 *                       iteration).  The device implements this form only.
 *  EOT_HESS_EXACT:      D_r with r = pi(f, f^{C,eps}) 1 (it would need one extra
 *                       row pass per iteration); rejected with EOT_EINVAL. */
typedef enum { EOT_HESS_DIAG_ALPHA = 0, EOT_HESS_EXACT = 1 } eot_hessian;

typedef struct {
    int32_t n, m;          /* numbers of source / target points, >= 1                 */
    int32_t d;             /* 0: C is given; > 0: X (n x d), Y (m x d) given          */
    const double *a;       /* (n) positive weights summing to 1 (renormalised)        */
    const double *b;       /* (m) positive weights summing to 1 (renormalised)        */
    const void *C;         /* (n x m) cost: double for FP64, float otherwise; or NULL */
    const void *X, *Y;     /* point clouds (float32 in every mode; the FP64 mode forms
                              the cost from them in float64); or NULL                 */
    eot_mem mem;           /* memory space of a, b, C, X, Y, f_init, g_init, V_init,
                              V_out and the outputs                                  */
    int32_t normalize_cost;/* 1: divide C by max_ij C_ij (after forming it from X, Y) */
    double eps;            /* target regularisation eps > 0                           */
    const double *f_init;  /* optional warm start f (n) (NULL: zeros; Alg. 4.1 line 1) */
    /* Warm-start state (the resume side of a checkpoint (f, g, V)):
     *  g_init (m): used when f_init is NULL; the solve starts from
     *      f = g_init^{C,eps_0} (one row half-step, Eq. foc_f, at the first
     *      level's eps).  NULL: not used.
     *  V_init (n x ell, row-major): modes for SK-NR (needs ell > 0).  The first
     *      level runs SK-NR on their span instead of plain Sinkhorn (the static
     *      modes of Sec. 5); the library scales each column to unit root mean
     *      square and makes them a-orthonormal and orthogonal to the constants
     *      (Cholesky-QR in L2(a), in column order: the span of the first k
     *      columns is kept for every k); a column whose part outside the
     *      constants and the earlier columns has an a-norm below about 3e-3 of
     *      the largest is dropped (zeroed).
     *      With sequential_modes they also start the next level's mode
     *      computation.  NULL: not used.
     *  V_out (n x ell, row-major, output; needs ell > 0): the ell leading modes
     *      (Sec. 3, descending rho_k^2) of the returned pair at eps,
     *      a-orthonormal and orthogonal to a, as computed for a continuation
     *      level (eig_tol, eig_max_iter, eig_degree); one more mode
     *      computation after the last level, counted in seconds, seconds_eig
     *      and eig_iters.  NULL: not computed.
     * Entries must be finite (EOT_EINVAL otherwise).  Ignored by the server,
     * which warm-starts from its own resident state (eot_server_submit). */
    const double *g_init;
    const double *V_init;
    double *V_out;
} eot_problem;

typedef struct {
    double tol;             /* omega: stop when ||pi1-a||_1 + ||pi^T1-b||_1 < tol     */
    int32_t max_iter;       /* per continuation level                                 */
    int32_t ell;            /* number of low-frequency modes l; 0 = plain Sinkhorn    */
    double eps_start;       /* continuation start; <= eps: a single level at eps      */
    double eps_factor;      /* geometric factor in (0, 1) between levels              */
    double level_tol;       /* tolerance of intermediate levels (<= 0: use tol)        */
    int32_t sequential_modes; /* 1: recompute V at every level; 0: once at eps_start  */
    int32_t oversample;     /* extra block columns of the subspace iteration           */
    double eig_tol;         /* Ritz residual ||M z - theta z||_a stopping threshold (below
                               2e-3 formed from the residual vectors; above, from the
                               Gram entries, whose float32 estimate floors near 6e-4) */
    int32_t eig_max_iter;   /* subspace iteration cap                                  */
    eot_prec prec;
    eot_hessian hessian;
    int32_t poll_every;     /* iterations between host convergence polls (0: auto)    */
    void *stream;           /* cudaStream_t to run on; NULL: the library's own stream */
    double wait_limit_s;    /* bound of every device-side wait of one CTA on others
                               (the grid barriers of the cooperative Sinkhorn loop, the
                               gang barriers of eot_solve_batch); a wait that exceeds it
                               gives up and the solve returns EOT_ETIMEDOUT (the device
                               stays usable).  <= 0 or not finite: 30 s               */
    int32_t stall_window;   /* iterations between stall checkpoints of a level: when the
                               L1 marginal error has not fallen below 0.99 times its
                               value at the previous checkpoint the level stops (the
                               error has reached the float32 rounding floor, or falls
                               so slowly that a decade would take > 200 windows); the
                               solve then returns EOT_OK if the returned pair meets
                               tol, else EOT_NOT_CONVERGED, with eot_result.stalled = 1.
                               0: no check.  Default 1000.                            */
    int32_t eig_degree;     /* mode computation (Sec. 3-4): 0 or 1, block subspace
                               iteration with a Rayleigh-Ritz step per application of
                               Op(pi) o Op(pi)^T; 2..8, Chebyshev-filtered subspace
                               iteration: between two Rayleigh-Ritz steps the Ritz
                               vectors are multiplied by the Chebyshev polynomial of
                               this degree that damps the spectrum below the block's
                               smallest Ritz value (eig_degree applications per step;
                               eig_max_iter counts Rayleigh-Ritz steps).  Default 0.  */
    int32_t newton_solver;  /* solve of the projected Newton system (eps H_V) Delta =
                               -eps grad_V of Algorithm 4.1 line 10: 0 (default), L D L^T
                               factorisation; 1, conjugate gradients (Sec. 4 design
                               remarks: the iterative solve, the form that parallelises
                               over many problems): float32, stops at a relative residual
                               of 1e-6 or after 10 l steps; a search direction of
                               non-positive curvature rejects the step, as a failed
                               factorisation does.  Other values: EOT_EINVAL.           */
} eot_options;

typedef struct {
    eot_status status;
    int32_t iters;          /* Algorithm 4.1 iterations at the final level            */
    int32_t total_iters;    /* over all continuation levels                           */
    int32_t nr_accepted, nr_rejected; /* Newton steps at the final level              */
    int32_t levels;         /* continuation levels run                                */
    int32_t eig_iters;      /* subspace iterations over all levels                    */
    double l1_marginal;     /* ||pi1-a||_1 + ||pi^T1-b||_1 of the returned (f, g)      */
    double row_l1, col_l1;
    double q_dual;          /* Q_eps(f, g), Eq. def_Q                                  */
    double q_semi;          /* Q_semi(f), Eq. def_Q_semi                               */
    double dual_gap;        /* <pi1-a,f> + <pi^T1-b,g> + eps (sum pi - 1)               */
    double seconds;         /* device time of the whole solve                          */
    double seconds_eig;     /* part of it spent computing modes                        */
    double seconds_last_level; /* device time of the final eps level incl. its modes   */
    int64_t kernel_launches; /* device kernels this solve launched (all levels)        */
    int64_t device_t_begin_ns, device_t_end_ns; /* the device clock (globaltimer, ns) at
                               the solve's first and last kernel: solves whose
                               intervals intersect ran on the device at once         */
    int32_t stalled;        /* 1: the final level stopped on the stall check           */
} eot_result;

/* Fill *opt with defaults: tol 1e-6, max_iter 100000, ell 0, single level,
 * eps_factor 0.5, sequential modes, oversample 10, eig_tol 1e-2, eig_max_iter 100,
 * FP32, Hessian with D_a, automatic polling, library stream, 30 s wait limit. */
void eot_default_options(eot_options *opt);

/* Solve one problem (Algorithm 4.1 with eps continuation).  f_out (n) and
 * g_out (m) receive float64 potentials in the memory space of prob->mem,
 * gauge-normalised so that <f,a> = <g,b> (Sec. 2: the dual is invariant under
 * (f, g) + c(1, -1)).  res (host, may be NULL) receives the statistics.
 * Returns EOT_OK, EOT_NOT_CONVERGED, or a negative error. */
eot_status eot_solve(const eot_problem *prob, const eot_options *opt,
                     double *f_out, double *g_out, eot_result *res);

/* One record of a solve's iteration trace: iteration `iter` (1-based within
 * its level; a final level continued after its verification restarts at 1)
 * of the level at `eps`: the stop test's L1 value at f_k (the column term
 * ||pi(f_k, g_k)^T 1 - b||_1; the row term is zero after the row half-step,
 * Alg. 4.1 line 5) and Q_semi(f_k) (Eq. def_Q_semi); for SK-NR the Newton
 * trial's dq = Q_semi(f') - Q_semi(f_k) and accepted = 1 (dq > 0), 0
 * (rejected, or -H_V not positive definite: dq NaN); accepted = -1 and dq NaN
 * for a plain Sinkhorn iteration or one whose test stopped the level. */
typedef struct {
    double eps, l1, q_semi, dq;
    int32_t iter, accepted;
} eot_trace_rec;

/* eot_solve with the per-iteration trace: the device appends one record per
 * iteration to a ring of trace_cap records (device memory of the call), copied
 * back at the end: trace (host, trace_cap records) receives the last
 * min(count, trace_cap) records, oldest first; *trace_count (may be NULL) the
 * number of iterations recorded over all levels (count).  The solve's
 * arithmetic and results are those of eot_solve.  EOT_EINVAL if trace is NULL
 * or trace_cap < 1. */
eot_status eot_solve_traced(const eot_problem *prob, const eot_options *opt, double *f_out,
                            double *g_out, eot_result *res, eot_trace_rec *trace,
                            int32_t trace_cap, int64_t *trace_count);

/* Solve count independent problems of uneven sizes.  Plain Sinkhorn on float32
 * costs (opt->ell == 0, FP32) runs every problem in one persistent launch;
 * SK-NR (ell > 0) and the other precisions run each problem as a whole solve
 * (eot_solve's path) on a pool of host worker threads, each with its own
 * stream, so that the solves overlap on the device, the problems with the
 * most predicted work first.  Arrays of count pointers; results[k]
 * (host) holds each problem's status; the call returns the worst status.  Each
 * problem's result does not depend on which others share the batch, nor on how
 * many CTAs the scheduler gives it (bit for bit).  A problem with n > m and no
 * f_init runs transposed internally (Sinkhorn is symmetric in the two sides),
 * and so does a plain-Sinkhorn problem given g_init and no f_init (its first
 * half-step is then the row transform of g_init): f_out, g_out, row_l1 and
 * col_l1 are returned in the caller's roles, and its q_semi is the semi-dual
 * in g. */
eot_status eot_solve_batch(int32_t count, const eot_problem *probs, const eot_options *opt,
                           double *const *f_out, double *const *g_out, eot_result *results);

/* ---------------------------------------------------------------- serving */
typedef struct eot_server eot_server;

/* Create a server with a background scheduler that batches incoming requests
 * continuously: a request is admitted as soon as a slot is free and its device
 * footprint fits in hbm_budget_bytes; admitted requests share the device.
 * Potentials of requests submitted with a cloud_id stay resident and
 * warm-start later requests on the same cloud (with ell > 0, so do the modes
 * of the last level, which become the next request's V_init).  Ownership:
 * *srv until destroy. */
eot_status eot_server_create(const eot_options *opt, size_t hbm_budget_bytes,
                             int32_t max_slots, eot_server **srv);
/* Deep-copies the problem (host memory only) and returns a ticket.  The
 * request runs with the server's options, except that a request whose stored
 * float32 cost would exceed 256 MB (4 n m bytes) and that gives points with
 * d <= 64 and plain Sinkhorn runs with the on-the-fly cost (EOT_PREC_SPLIT_TC).
 * Scheduling: a request is admitted when a slot is free and its device
 * footprint fits the free budget; among those that fit, the one with the
 * least predicted work (n m times the iterations of its eps schedule) goes
 * first; a request that has waited more than 1 s goes before all others, and
 * while it does not fit no other request is admitted (no starvation); one
 * that can never fit the budget fails with EOT_ENOMEM.  The problem's f_init,
 * g_init, V_init and V_out are ignored: a request with a cloud_id warm-starts
 * from the state the cloud's last completed request left resident, and with
 * cloud_id 0 starts cold. */
eot_status eot_server_submit(eot_server *srv, const eot_problem *prob, uint64_t cloud_id,
                             uint64_t *ticket);
/* eot_server_submit with the request's own options (eps schedule, ell,
 * tolerance, precision; its stream field is ignored); NULL: the server's. */
eot_status eot_server_submit_opts(eot_server *srv, const eot_problem *prob, uint64_t cloud_id,
                                  const eot_options *opt, uint64_t *ticket);
/* EOT_PENDING until done; then copies f (n), g (m) to host memory and fills res
 * (which may be NULL), returns the request's status and forgets the ticket.
 * Unknown tickets give EOT_ENOTFOUND. */
eot_status eot_server_poll(eot_server *srv, uint64_t ticket, double *f_out, double *g_out,
                           eot_result *res);
/* Latency percentiles (submit -> completion, seconds) and completed solves per
 * second since creation. */
eot_status eot_server_stats(eot_server *srv, double *p50_s, double *p99_s,
                            double *solves_per_s);
/* Current load (host outputs, each optional): requests waiting, requests
 * being solved, device bytes admitted (their footprints), completed solves. */
eot_status eot_server_status(eot_server *srv, int32_t *queued, int32_t *running,
                             uint64_t *hbm_in_use, uint64_t *completed);
void eot_server_destroy(eot_server *srv);

/* The server's scheduling policy replayed on the host (no device work): count
 * requests arriving at t_arrive[k] (seconds) with device footprints
 * footprint[k] (bytes), predicted work work[k] and service times service_s[k],
 * served by `slots` workers within `budget` bytes, a request that has waited
 * more than max_wait_s going first (the server uses 1 s).  t_start[k] and
 * t_done[k] receive the dispatch and completion times (-1 for a request that
 * can never fit).  Host arrays of count entries. */
eot_status eot_server_simulate(int32_t count, const double *t_arrive, const uint64_t *footprint,
                               const double *work, const double *service_s, uint64_t budget,
                               int32_t slots, double max_wait_s, double *t_start, double *t_done);

/* --------------------------------------------------- single hot-path steps
 * Device-pointer entry points for the individual passes.  They run on `stream`
 * (NULL: the legacy default stream) and return once the work is enqueued.
 * C is float32 (n x m, row-major, device). */

typedef enum { EOT_SIDE_COL = 0, EOT_SIDE_ROW = 1 } eot_side;

/* One (C,eps)-transform (Eq. foc_g for COL, Eq. foc_f for ROW):
 *   COL: out_j = -eps log sum_i a_i exp((f_i - C_ij)/eps)      (pot = f, w = a)
 *   ROW: out_i = -eps log sum_j b_j exp((g_j - C_ij)/eps)      (pot = g, w = b)
 * shift (the current potential on the output side, or NULL) is a reference
 * point: the sum is formed relative to it, and log_ratio (optional, same length
 * as out) receives (shift - out)/eps, the log of the marginal ratio of
 * pi(pot, shift) on the output side (0 at a fixed point).  With shift NULL the
 * call runs two passes (the first computes a reference).
 * All pointers are device pointers: pot, w, shift float64; out, log_ratio float64. */
eot_status eot_ctransform(eot_side side, int32_t n, int32_t m, const float *C,
                          const double *pot, const double *w, const double *shift,
                          double eps, double *out, double *log_ratio, void *stream);

/* Coupling products (Eq. def_Op_pi, def_Op_pi_T) at potentials (f, g):
 *   COL: out (m x k) = Op(pi)^T Z,  out_j = sum_i exp((f_i+g_j-C_ij)/eps) a_i Z_i
 *   ROW: out (n x k) = Op(pi) Z,    out_i = sum_j exp((f_i+g_j-C_ij)/eps) b_j Z_j
 * Z is float32 row-major ((n or m) x k), 1 <= k <= 64; out float32.  Device
 * pointers. */
eot_status eot_kapply(eot_side side, int32_t n, int32_t m, int32_t k, const float *C,
                      const double *f, const double *g, const double *a, const double *b,
                      double eps, const float *Z, float *out, void *stream);

/* Squared Euclidean cost C_ij = ||x_i - y_j||^2 (float64 arithmetic, one
 * rounding to float32), divided by max_ij C_ij when normalize != 0.  X (n x d),
 * Y (m x d) float32, C float32 (n x m); device pointers.  cmax_out (device,
 * optional) receives the float64 maximum before normalisation. */
eot_status eot_cost(int32_t n, int32_t m, int32_t d, const float *X, const float *Y,
                    int32_t normalize, float *C, double *cmax_out, void *stream);

/* Low-frequency modes V_l(eps) (Sec. 4; Eq. semidual_Hessian): the ell leading
 * non-trivial eigenvectors of Op(pi) o Op(pi)^T at potentials (f, g), by block
 * subspace iteration with Rayleigh-Ritz (block ell + oversample), orthonormal in
 * L2(a) and a-orthogonal to the constants.  V (n x ell, float64, device, row
 * major) is both the optional start block (if use_V_as_start) and the output;
 * rho2 (ell, float64, device, optional) receives the Ritz values rho_k^2.
 * iters_out / resid_out (host, optional): iterations and final max residual. */
eot_status eot_spectral_modes(int32_t n, int32_t m, const float *C, const double *f,
                              const double *g, const double *a, const double *b, double eps,
                              int32_t ell, int32_t oversample, double tol, int32_t max_iter,
                              int32_t use_V_as_start, double *V, double *rho2,
                              int32_t *iters_out, double *resid_out, void *stream);

/* The same modes by Chebyshev-filtered block subspace iteration (a faster
 * spectral step where the rho_k^2 cluster near 1, Sec. 3): after each
 * Rayleigh-Ritz step that misses tol, the Ritz vectors are multiplied by
 * T_degree((M - c)/e), [c - e, c + e] = [0, smallest Ritz value of the block]
 * (scaled three-term recurrence, every product deflated of the constants),
 * and the filtered block is orthonormalised in L2(a) by a Cholesky-QR of its
 * column-scaled Gram matrix.  degree 0 or 1: eot_spectral_modes; 2..8 otherwise
 * (EOT_EINVAL beyond).  iters_out counts Rayleigh-Ritz steps; each but the
 * last costs degree applications of Op(pi) o Op(pi)^T.  Other arguments as
 * eot_spectral_modes. */
eot_status eot_spectral_modes_filtered(int32_t n, int32_t m, const float *C, const double *f,
                                       const double *g, const double *a, const double *b,
                                       double eps, int32_t ell, int32_t oversample,
                                       int32_t degree, double tol, int32_t max_iter,
                                       int32_t use_V_as_start, double *V, double *rho2,
                                       int32_t *iters_out, double *resid_out, void *stream);

/* Scalars of one SK-NR iteration (eot_sknr_step). */
typedef struct {
    double col_l1;      /* sum_j b_j |exp((g_j - h_j)/eps) - 1|: the column term of the
                           L1 test of Algorithm 4.1 at (f_k, g_k)                      */
    double q_semi;      /* Q_semi(f_k) = <f_k, a> + <h, b>  (Eq. def_Q_semi)            */
    double dq;          /* Q_semi(f') - Q_semi(f_k), summed as <V Delta, a> + <h' - h, b> */
    int32_t newton_ok;  /* 0: -H_V not positive definite (or the products saw
                           exponentials out of range): no trial, the step is rejected */
    int32_t accepted;   /* 1: dq > 0, (f', h') is the next iterate; 0: (f_k, h) is     */
    int32_t products_in_range; /* 0: the S4 pass saw a column whose largest term lies
                           more than 2^60 from 1 (W would lose range): the step is
                           then skipped, newton_ok = 0                              */
    double stage_seconds[4]; /* device time (CUDA events on the call's stream) of the
                           row half-step that forms f_k, the S4 pass (h, W, test),
                           the Newton solve (W^T D_b^-1 W reduction, factorisation,
                           f'), and the trial column pass                          */
} eot_sknr_info;

/* One iteration of Algorithm 4.1 (lines 4-16) from g_k with the caller's modes
 * V, on a float32 cost, exposing every intermediate of the Newton step:
 *   f_k   = g_k^{C,eps}                                  (Eq. foc_f, line 4)
 *   h     = f_k^{C,eps}                                  (Eq. foc_g)
 *   W     = pi(f_k, h)^T V   (m x ell, float32)
 *   grad  = V^T (a - pi(f_k, h) 1), formed as -sum_j d_j W_j with
 *           d_j = 1 - exp((g_j - h_j)/eps)               (Eq. dQ_semi on V)
 *   GV    = V^T D_a V,  WtDW = W^T D_b^-1 W,  -H_V = (GV - WtDW)/eps
 *                                                        (Eq. d2Q_semi, D_r ~ D_a)
 *   delta = (-H_V)^-1 grad                               (lines 12-13)
 *   f'    = f_k + V delta,  h' = f'^{C,eps}               (lines 14-16)
 * and the scalars in *info.  The float32 passes, tensor-core products and
 * float32 factorisation are those of eot_solve's SK-NR iterations.
 * Arguments: n >= 3, m >= 1, 1 <= ell <= 47, ell < n.  C (n x m, float32),
 * a (n), b (m) (used as given), g (m), V (n x ell, float64 row-major; the
 * library rounds it to float32 as eot_solve stores its modes; it should be
 * a-orthonormal and a-orthogonal to the constants, Sec. 4): device pointers.
 * Outputs (device pointers, each optional): f_k (n), h (m), W (m x ell,
 * float32), grad (ell), GV (ell x ell), WtDW (ell x ell), delta (ell),
 * f_trial (n) and h_trial (m) (left untouched when newton_ok is 0); info
 * (host, optional).  newton_solver: the Newton system's solve, as
 * eot_options.newton_solver (0: L D L^T, 1: conjugate gradients).
 * Synchronises `stream` before it returns. */
eot_status eot_sknr_step(int32_t n, int32_t m, int32_t ell, const float *C, const double *a,
                         const double *b, double eps, const double *g, const double *V,
                         double *f_k, double *h, float *W, double *grad, double *GV,
                         double *WtDW, double *delta, double *f_trial, double *h_trial,
                         eot_sknr_info *info, int32_t newton_solver, void *stream);

/* The tuning of eot_solve_batch on the current device, run on first use (the
 * first batch call runs it too): the gang cost model (step_ns, fix_ns, bar_ns;
 * see eot_batch_plan) and the pass tiles picked by timing: tiles[c] for the
 * problems whose column count m (rows being the shorter side, as the kernel
 * runs them) is at most 64, 128, 256, 512, 1024, 2048 (c = 0..5) or larger
 * (c = 6); bit 0 of a tile: 64-column blocks of the column half-step (two
 * columns a lane) instead of 128; bit 1: eight rows a warp per chunk of the
 * row half-step instead of four.  tile_ms[4 c + t] receives the calibration
 * time of tile t on class c (a min(m, 256) x m problem, a copy on every
 * resident CTA); a tile other than 0 is picked only when at least 2% faster
 * than tile 0.  No tile
 * changes a result (the order of every sum depends on the problem's shape
 * alone); EOT_BATCH_TILE=t in the environment forces tile t.  Each output may
 * be NULL (tiles: 7 entries, tile_ms: 28). */
eot_status eot_batch_tuning(double *step_ns, double *fix_ns, double *bar_ns, int32_t *tiles,
                            float *tile_ms);

/* The schedule eot_solve_batch would use, computed on the host only (no
 * device work, no GPU needed): for count problems of sizes n[k] x m[k] at
 * eps[k] (has_f_init[k]: 0 no warm start, 2 a g_init and no f_init, any
 * other value an f_init; NULL: none has one), the options' eps schedule and max_iter, a grid of grid_ctas resident
 * CTAs and a cost model (step_ns: one load-and-reduce step of a CTA; fix_ns:
 * the fixed cost of an iteration; bar_ns: one gang barrier; the library
 * calibrates these on the device before its first batch), gang_out[k]
 * receives the number of CTAs of problem k (a power of two, at most 32 and an
 * eighth of the grid) and transposed_out[k] 1 if it runs as the transposed
 * problem (n > m without a warm start, or a g_init without f_init).  Host
 * arrays of count entries.
 * Returns EOT_EINVAL on a member with n, m < 1 or eps <= 0, or a model with
 * step_ns <= 0. */
eot_status eot_batch_plan(int32_t count, const int32_t *n, const int32_t *m, const double *eps,
                          const int32_t *has_f_init, const eot_options *opt, int32_t grid_ctas,
                          double step_ns, double fix_ns, double bar_ns, int32_t *gang_out,
                          int32_t *transposed_out);

/* Marginal errors of pi(f, g) computed on the device (float32 exponentials,
 * float64 sums): row_l1 = ||pi1 - a||_1, col_l1 = ||pi^T1 - b||_1 (host outputs). */
eot_status eot_marginal_error(int32_t n, int32_t m, const float *C, const double *f,
                              const double *g, const double *a, const double *b, double eps,
                              double *row_l1, double *col_l1, void *stream);

/* The (C,eps)-transform of eot_ctransform (same arguments, same result) for
 * callers that may not allocate device memory: code that runs inside a device
 * memory pool owned by another allocator (a framework's caching allocator, an
 * application that sized the device at start-up), where a foreign cudaMalloc
 * can fail or break the pool's budget, and latency-critical loops, where
 * cudaMalloc / cudaFree may synchronise the device.  The paper has no
 * counterpart; this is a deployment variant of the same pass.
 * It allocates nothing: its temporaries live in one static device array of
 * 4 MiB that every GPU loading the library holds until the process exits.
 * Limits: n, m <= 16384 (EOT_EINVAL beyond).  The first call on a device looks
 * up the array's address, so make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents: calls that
 * overlap on the GPU (other streams or threads without ordering) race.  Runs
 * on `stream` (NULL: the legacy default stream); every call synchronises that
 * stream before it returns, on success and on failure alike (it reads the
 * cost's range back to the host, and a failed call leaves no work of its own
 * running on the shared array). */
eot_status eot_ctransform_noalloc(eot_side side, int32_t n, int32_t m, const float *C,
                                  const double *pot, const double *w, const double *shift,
                                  double eps, double *out, double *log_ratio, void *stream);

/* The coupling of a pair of potentials (Eq. pi(f,g)) and its scalars:
 *   P_ij = a_i b_j exp((f_i + g_j - C_ij)/eps)        (n x m, float32, row major)
 *   cost_out   = <C, P>,  mass_out = sum_ij P_ij,
 *   primal_out = <C, P> + eps KL(P | a x b)            (Eq. primal_EOT), with
 *                KL(P | a x b) = sum P log(P/(a b)); primal_out minus the dual
 *                value Q_eps(f, g) is the duality gap <P1-a,f> + <P^T1-b,g> +
 *                eps (sum P - 1).
 * At a solution (f, g) of the dual, P is also the derivative of the optimal
 * value with respect to the cost (envelope theorem: dQ_eps/dC_ij = P_ij), and
 * the potentials are its derivatives with respect to a and b (up to a
 * constant).  The exponent is formed in float64 from the float64 potentials and
 * the float32 cost, the scalars summed in float64 in a fixed order.  C, f, g, a,
 * b are device pointers (a, b as given: the solves return potentials for the
 * weights normalised to sum 1); P (device, n*m floats) is optional, and so are
 * the host outputs.  Runs on `stream` (NULL: the library's stream of the
 * calling thread) and returns when the scalars are on the host.  Scratch of
 * 24 n + 24 bytes comes from the stream-ordered allocator. */
eot_status eot_plan(int32_t n, int32_t m, const float *C, const double *f, const double *g,
                    const double *a, const double *b, double eps, float *P, double *cost_out,
                    double *mass_out, double *primal_out, void *stream);

/* The two exponentials of the float32 passes, elementwise, so that callers can
 * check their accuracy (not a step of the method; Sec. 2 only needs exp):
 *   variant 0: out_i = 2^(p_i + q_i) as the evaluation passes that verify a
 *              result form it: p a float32 exponent, q a small correction
 *              (|q| < 1/4) carried beside it; range reduction and a degree-7
 *              Taylor series in float32, unbiased (mean relative error below
 *              1e-9 over a range of arguments).
 *   variant 1: out_i = the hardware approximation ex2.approx of the float32 sum
 *              p_i + q_i, as the iterations form their terms (biased by a few
 *              1e-8 relative, the same sign for every term).
 * count >= 0 elements; p, q, out float32 device pointers.  Runs on `stream`
 * (NULL: the legacy default stream) and returns once enqueued. */
eot_status eot_exp2(int32_t count, const float *p, const float *q, int32_t variant, float *out,
                    void *stream);

/* Thread-local description of the last non-OK status returned on this thread. */
const char *eot_last_error(void);

/* Library version string. */
const char *eot_version(void);

/* 1 in a library built with -DEOT_DEBUG, else 0.  In that build the kernels
 * check the indexes and launch shapes they rely on (shared-memory tables,
 * partial-state slots, mode widths, gang ranks); a failed check records its
 * site (100 x unit + k) in a device word and skips the access it guards, and
 * the call that launched the work fails with EOT_ECUDA naming the site
 * (eot_last_error).  The release build has no checks and the same results. */
int32_t eot_debug_build(void);

#ifdef __cplusplus
}
#endif
#endif /* EOT_H */
