/*
 * eot.h — C ABI of the GB300 library for entropic-regularised optimal transport
 * solved by the truncated Newton method of Kemertas, Farahmand and Jepson,
 * "A Truncated Newton Method for Optimal Transport" (ICLR 2025, arXiv 2504.02067).
 *
 * Problem (Sec. 2.1, Eq. sinkhorn-primal): given marginals r in the (n-1)-simplex,
 * c in the (m-1)-simplex and a cost C with entries in [0, 1], find
 *     P* = argmin_{P in U(r, c)} <P, C> - H(P) / gamma,
 * whose form is P(u, v; gamma) = exp(u 1^T + 1 v^T - gamma C) (Eq.
 * lagrangian-closed-form). gamma is the INVERSE temperature; the potentials u, v
 * are log-domain (u, not u / gamma). The plan is never stored: every O(n m)
 * operation re-forms it tile by tile inside a CUDA kernel.
 *
 * Conventions for every call below:
 *  - Pointers marked "device" must be device memory of the handle's GPU;
 *    pointers marked "host" are host memory. The caller owns every buffer it
 *    passes; the library never frees or keeps them after the call returns.
 *  - Dense costs are row-major with leading dimension ldc (elements); n x ldc
 *    elements must be readable. 16-byte alignment of C with ldc and m multiples
 *    of 16 bytes / element size enables the vectorised path; otherwise a scalar
 *    path is used.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are stream-ordered. Calls with host outputs synchronise the stream.
 *  - Return value: EOT_OK or an error code; the handle keeps a message that
 *    eot_last_error() returns. No call aborts the process. After
 *    EOT_ERR_CUDA the handle should be destroyed; after any other error it
 *    stays usable.
 *  - Results are bit-reproducible for a fixed handle, problem and stream (all
 *    reductions have a fixed order; no floating-point atomics).
 */
#ifndef EOT_H_
#define EOT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EOT_OK = 0,
  EOT_ERR_INVALID_ARG = 1,    /* bad pointer, size, kind, precision or parameter */
  EOT_ERR_NONFINITE = 2,      /* NaN/Inf met in potentials, marginals or CG scalars */
  EOT_ERR_CG_MAXITER = 3,     /* a linear CG solve hit max_cg iterations (Alg. 2) */
  EOT_ERR_LINESEARCH = 4,     /* backtracking hit max_ls halvings (Alg. 4's line search) */
  EOT_ERR_MAXSTAGES = 5,      /* Alg. 1 did not reach gamma_f within max_stages */
  EOT_ERR_MAXNEWTON = 6,      /* Alg. 4 did not reach its tolerance within max_newton */
  EOT_ERR_RANGE = 7,          /* |potential| >= 2^19: outside the mixed-precision split */
  EOT_ERR_CUDA = 8,           /* a CUDA runtime call failed; destroy the handle */
  EOT_ERR_UNSUPPORTED = 9,    /* combination of cost kind and precision not built */
  EOT_ERR_DEVICE_TIMEOUT = 10, /* a bounded device-side wait (an mbarrier of the tensor-core
                                 sweeps or a group barrier of eot_solve_batched) ran out:
                                 the kernel recorded it and returned, its outputs are not
                                 valid, and the handle stays usable */
  EOT_ERR_TIME_LIMIT = 11     /* eot_solve reached eot_params.max_seconds (checked before
                                 each Newton step and each stage) */
} eot_status;

typedef enum {
  EOT_COST_DENSE_F32 = 0,       /* C: float, n x m */
  EOT_COST_DENSE_F64 = 1,       /* C: double, n x m */
  EOT_COST_SQEUCLID_POINTS = 2  /* C_ij = s_C |x_i - y_j|^2 formed on the fly from X, Y */
} eot_cost_kind;

typedef enum {
  EOT_PREC_FP64 = 0,       /* every operation in FP64 (the paper's setting, Sec. 4) */
  EOT_PREC_MIXED = 1,      /* FP32 exp and sums on a double-float exponent; FP64
                              potentials, shifts, CG scalars and combines */
  EOT_PREC_PLAIN_FP32 = 2  /* potentials rounded to FP32 before the exponent; FP32
                              exponent and exp, no shift or split */
} eot_precision;

typedef struct {
  int32_t kind;        /* eot_cost_kind */
  int32_t precision;   /* eot_precision: how P is formed. DENSE_F64 needs FP64;
                          DENSE_F32 and points take MIXED or PLAIN_FP32. */
  int64_t n, m;        /* rows (len r) and columns (len c); n, m >= 1 */
  int64_t d;           /* point dimension (points only), 1 <= d <= 64 */
  int64_t ldc;         /* leading dimension of C in elements (dense only), >= m */
  const void* C;       /* device: dense cost (float or double per kind) */
  const float* X;      /* device: n x d row-major points (points only) */
  const float* Y;      /* device: m x d row-major points (points only) */
  double cost_scale;   /* points: s_C; <= 0 asks the library for 1 / max_ij |x_i - y_j|^2 */
  const double* r;     /* device: n target row marginal (solve / newton / backward) */
  const double* c;     /* device: m target column marginal */
} eot_problem;

typedef struct {
  double gamma_i;      /* initial gamma (Alg. 1); default 2^4 (Table 3 caption) */
  double gamma_f;      /* final gamma; default 2^12 */
  double p;            /* eps_d = min(H(r), H(c)) / gamma^p (Alg. 1); default 1.5 */
  double q1;           /* initial decay factor q^(1) (Sec. 3.3); default 2 */
  double w_r;          /* row smoothing weight, w_c = 1/2 - w_r (Sec. 3.4); default 0.45 */
  double tol_final;    /* target marginal L1 error at gamma_f; the last stage uses
                          eps_d = min(eps_d, 2 tol_final / 3); default 1e-6 */
  int32_t max_stages;  /* default 200 */
  int32_t max_newton;  /* Newton steps per stage; default 200 */
  int32_t max_cg;      /* CG iterations per linear solve; default min(4n, 2000) when 0 */
  int32_t max_ls;      /* Armijo halvings per step; default 30 */
  int32_t projector;   /* Bregman projection of each stage: EOT_PROJECT_NEWTON (Alg. 4,
                          default) or EOT_PROJECT_SINKHORN (alternating row/column fixes
                          until ||grad g||_1 <= eps: MDOT-Sinkhorn, Sec. 4) */
  int32_t max_sinkhorn; /* Sinkhorn iterations per projection; default 10^6 when 0 */
  int32_t newton_system; /* the linear system of each NewtonSolve (dense costs):
                            EOT_NEWTON_REDUCED (Alg. 2: CG on F_r(rho), default) or
                            EOT_NEWTON_FULL (CG on the (n + m) discounted Hessian of
                            Eq. discounted-hessian, one two-sided sweep per iteration;
                            the same outer loop and forcing test) */
  int32_t reserved;
  double max_seconds;  /* wall-clock budget of eot_solve (<= 0: none); checked on the
                          device before each Newton step and on the host before each
                          stage, so a call may overrun it by one Newton step */
} eot_params;

enum { EOT_PROJECT_NEWTON = 0, EOT_PROJECT_SINKHORN = 1 };
enum { EOT_NEWTON_REDUCED = 0, EOT_NEWTON_FULL = 1 };

/* One stage t of Alg. 1 in eot_solve: the temperature, the tolerance of its
 * Bregman projection, AdjustSchedule's input and output (Sec. 3.3, Eq. delta_k-
 * ratio: delta_min is the smallest ratio of actual to predicted reduction of
 * ||grad g||_1 over the stage's Newton steps, +inf with none) and its work. */
typedef struct {
  double gamma;             /* gamma^(t) */
  double eps;               /* tolerance of the projection, eps_d / 2 (Alg. 1) */
  double delta_min;         /* min_k delta_k of the stage */
  double q_next;            /* q^(t+1) chosen by AdjustSchedule */
  int32_t newton_steps, cg_iters, ls_trials, sinkhorn_iters;  /* of this stage */
  int64_t sweeps;           /* O(nm) sweeps of this stage */
} eot_stage_record;

typedef struct {       /* host-side counters of one eot_solve call */
  int64_t sweeps_cg;        /* O(nm) sweeps inside linear CG (2 per CG iteration) */
  int64_t sweeps_newton;    /* other NewtonSolve sweeps (setup, d_v) */
  int64_t sweeps_linesearch; /* Armijo trials of Alg. 4 (with the alpha = 0 reference) and its row LSE after each update */
  int64_t sweeps_sinkhorn;  /* LSE sweeps of ChiSinkhorn (Alg. 3) or of the Sinkhorn projector */
  int64_t sweeps_total;
  int32_t stages, newton_steps, cg_iters, cg_solves, ls_trials, sinkhorn_iters;
  int32_t curvature_stops;  /* CG solves stopped because <p, F_r p> <= 0 in finite precision */
  int32_t reserved;
  double final_gamma;
  double final_rho;
  double grad_l1;           /* ||r~ - r(P)||_1 at the end of the last projection */
  double marg_err_l1;       /* ||r(P) - r||_1 + ||c(P) - c||_1 of the output (unsmoothed r, c) */
  double seconds;           /* wall time of the call */
  int64_t sweeps_stage;     /* the column fix and row LSE that open each projection of Alg. 4 */
  eot_stage_record* stage_records; /* in: host array for one record per stage (nullable; eot_solve only) */
  int32_t stage_records_cap;       /* in: its capacity */
  int32_t stage_records_len;       /* out: records written, min(stages, capacity) */
} eot_stats;

typedef struct eot_handle_s* eot_handle;

/* Create a handle on `device` with workspace for problems up to max_n x max_m
 * and point dimension max_d (grown on demand by later calls, which then allocate
 * and synchronise the device). max_d = 0: no point workspace is reserved; max_d
 * in [1, 64]: the per-point buffers of the point sweeps (for d >= 17 on the
 * mixed path, the tensor-core digit slices) are reserved now for max_n, max_m
 * points. Allocates device memory; not stream-ordered. Errors: INVALID_ARG
 * (max_n, max_m < 1 or max_d outside [0, 64]), CUDA. */
eot_status eot_create(eot_handle* out, int device, int64_t max_n, int64_t max_m, int64_t max_d);
/* Free the handle and its workspace. Synchronises the handle's device. */
eot_status eot_destroy(eot_handle h);
/* Message of the last error on this handle (never NULL; valid until the next call). */
const char* eot_last_error(eot_handle h);
const char* eot_status_string(eot_status s);
/* Defaults of eot_params listed above. */
eot_params eot_params_default(void);

/* Marginals of P(u, v; gamma) (Sec. 2, r(P) = P 1, c(P) = P^T 1), by one row and one
 * column log-sum-exp sweep (stable for any finite u, v).
 * u: device [n], v: device [m] (FP64). Outputs (device FP64, each nullable):
 * r_out [n], c_out [m], log_r_out [n], log_c_out [m], total_out [1] = sum_ij P_ij.
 * Errors: INVALID_ARG, NONFINITE, RANGE, CUDA. */
eot_status eot_marginals(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                         double gamma, double* r_out, double* c_out, double* log_r_out,
                         double* log_c_out, double* total_out, void* stream);

/* Hessian-vector product of the dual g (Eq. hessian; with s = sqrt(rho) the
 * discounted Hessian of Eq. discounted-hessian):
 *   out_u = r(P) * du + s P dv,   out_v = s P^T du + c(P) * dv.
 * One row LSE sweep (row shifts) and one fused two-sided sweep.
 * u, du, out_u: device [n]; v, dv, out_v: device [m]; r_out, c_out nullable. */
eot_status eot_hvp(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                   double gamma, double s, const double* du, const double* dv, double* out_u,
                   double* out_v, double* r_out, double* c_out, void* stream);

/* NewtonSolve (Alg. 2) at (u, v): anneal rho from rho0, solving F_r(rho) d_u =
 * -grad_u g with Jacobi-preconditioned CG from 0 to ||res||_1 <= (eta/4)||grad g||_1,
 * until ||F_r(1) d_u + grad_u g||_1 <= eta ||grad g||_1; d_u is then taken
 * modulo the gauge (d_u - k 1 with <r(P), d_u - k 1> = 0: the same plans, since
 * F_r(1) 1 = 0 and P_c 1 = 1) and d_v = -P_c d_u (Eq. bellman2 with Alg. 4's d_v step). grad_u g = r(P) - r_target, ||grad g||_1 =
 * ||grad_u g||_1 (assumes c(P) = c, as Alg. 4 maintains).
 * r_target: device [n]. du_out: device [n]; dv_out: device [m] (nullable).
 * rho_out, cg_iters_out: host, nullable (rho of the last CG solve, Appx. B).
 * Errors: INVALID_ARG, NONFINITE, CG_MAXITER, RANGE, CUDA. Synchronises. */
eot_status eot_newton_solve(eot_handle h, const eot_problem* prob, const double* u,
                            const double* v, double gamma, const double* r_target, double eta,
                            double rho0, int32_t max_cg, double* du_out, double* dv_out,
                            double* rho_out, int32_t* cg_iters_out, void* stream);

/* NewtonSolve as eot_newton_solve, but each linear solve runs PCG on the full
 * discounted system (Sec. 3.1, Eq. discounted-hessian)
 *   [D(r(P)) d_u + sqrt(rho) P d_v ; sqrt(rho) P^T d_u + D(c(P)) d_v] = [-grad_u g ; 0]
 * from 0 with the diagonal preconditioner (r(P), c(P)), to an L1 residual of the
 * (n + m)-vector <= (eta/4) ||grad g||_1, keeping its u-block (in exact arithmetic
 * the solution of F_r(rho) d_u = -grad_u g, the Schur complement of Eq.
 * matrix-definitions). Each CG iteration is one fused two-sided sweep over C
 * (Alg. 2's CG makes two); the outer test ||F_r(1) d_u + grad_u g||_1 <= eta
 * ||grad g||_1 takes two more per linear solve. A different Krylov iteration,
 * offered for measurement against Alg. 2. Dense costs only (EOT_ERR_UNSUPPORTED
 * for points). Arguments and errors as eot_newton_solve; cg_iters_out counts
 * full-system iterations. Synchronises. */
eot_status eot_newton_solve_full(eot_handle h, const eot_problem* prob, const double* u,
                                 const double* v, double gamma, const double* r_target, double eta,
                                 double rho0, int32_t max_cg, double* du_out, double* dv_out,
                                 double* rho_out, int32_t* cg_iters_out, void* stream);

/* Round (Alg. 1's closing step; the paper cites Algorithm 2 of Altschuler, Weed and
 * Rigollet, 2017) of P = P(u, v; gamma) onto U(r, c), kept implicit:
 *   x = min(r / r(P), 1), y = min(c / c(D(x) P), 1), F = D(x) P D(y),
 *   a = r - r(F), b = c - c(F),  Round(P) = F + a b^T / ||a||_1,
 * where F = P(u + log x, v + log y; gamma). Evaluated in FP64 (three passes over C).
 * u, v: device [n], [m]. Outputs, each nullable: u_out [n] = u + log x (-inf where
 * r_i = 0), v_out [m] = v + log y, a_out [n], b_out [m] (device FP64);
 * cost_out = <Round(P), C> (host; C as the solver sees it, s_C |x - y|^2 for points),
 * corr_l1_out = ||a||_1 (host). prob->r and prob->c are required.
 * Errors: INVALID_ARG, CUDA. Synchronises. */
eot_status eot_round(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                     double gamma, double* u_out, double* v_out, double* a_out, double* b_out,
                     double* cost_out, double* corr_l1_out, void* stream);

/* Full solve: MDOT (Alg. 1) with adaptive q and asymmetric smoothing, each
 * stage projected by TruncatedNewtonProject (Alg. 4 with Alg. 2 and Alg. 3).
 * u: device [n], v: device [m]: outputs (the last projected potentials at gamma_f).
 * When a cap (CG_MAXITER, LINESEARCH, MAXNEWTON, MAXSTAGES), a non-finite value
 * or the split range stops the solve, u and v still receive the last iterate (of
 * the stage in progress), which does not meet the requested tolerance, and stats
 * (when given) the work done so far, with final_gamma = the temperature of that
 * stage, grad_l1 = its last ||r~ - r(P)||_1 and marg_err_l1 = NaN.
 * stats: host, nullable; with stats->stage_records set (and stats->stage_records_cap
 * > 0) one eot_stage_record per stage of Alg. 1 is written there. Errors: any.
 * Synchronises. */
eot_status eot_solve(eot_handle h, const eot_problem* prob, const eot_params* params, double* u,
                     double* v, eot_stats* stats, void* stream);

/* Many point-cloud problems in ONE persistent kernel launch (the batching
 * regime: problems of uneven size solved together). Each problem runs the same
 * method as eot_solve (Alg. 1 with Alg. 4, Alg. 3 and Alg. 2) on the device,
 * with no host round trip: a cooperative launch of all co-resident CTAs, formed
 * into groups of G CTAs that take problems from a queue, largest n m first.
 * G and the own elements per thread are chosen by an autotuner that times
 * probe sweeps of the actual batch (once per batch shape, cached in the
 * handle; EOT_BATCH_CFG="G,k" in the environment forces G in {1,2,4,8} and
 * k in {1,2,4}).
 * probs: host array [nprob]; every problem EOT_COST_SQEUCLID_POINTS with
 *   1 <= d <= 4, 1 <= n, m <= 32768, all MIXED or all FP64; r, c, X, Y device.
 *   cost_scale <= 0: s_C = 1 / max |x_i - y_j|^2 computed per problem.
 * u, v: host arrays [nprob] of device pointers to the outputs ([n_k], [m_k]).
 * status_out: host [nprob], nullable: each problem's eot_status.
 * stats: host [nprob], nullable (sweeps_total only among the sweep counters;
 *   seconds = the whole call; each struct is overwritten, stage_records included).
 * Returns EOT_OK when every problem succeeded, else the status of the first
 * failing problem (in input order). A group barrier whose bounded wait (2 s)
 * ran out returns EOT_ERR_DEVICE_TIMEOUT for the whole call (the kernel records
 * it and every CTA returns); a failed launch returns EOT_ERR_CUDA. Synchronises. */
eot_status eot_solve_batched(eot_handle h, int32_t nprob, const eot_problem* probs,
                             const eot_params* params, double* const* u, double* const* v,
                             int32_t* status_out, eot_stats* stats, void* stream);

/* The configuration of the last batched launch: out3[0] = G (CTAs per group),
 * out3[1] = own elements per thread and round, out3[2] = groups. Host pointer. */
eot_status eot_batch_last_config(eot_handle h, int32_t* out3);

/* The EOT value at the potentials (u, v), from the dual (Sec. 2.1, Eq. sinkhorn-dual):
 *   value = ( <r, u> + <c, v> - sum_ij P_ij + 1 ) / gamma,   P = P(u, v; gamma),
 * which equals the primal value F* = <P*, C> - H(P*) / gamma at the optimum and is
 * stationary in (u, v) there, so potentials solved to a marginal tolerance give it
 * to second order in that tolerance. prob->r and prob->c are required.
 * value_out: device FP64 scalar. One row log-sum-exp sweep and two O(n) dot
 * products; asynchronous on `stream` (no host readback).
 * Errors: INVALID_ARG, NONFINITE, RANGE, CUDA (NONFINITE / RANGE are detected at
 * the next call that synchronises; the value is then not finite). */
eot_status eot_value(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                     double gamma, double* value_out, void* stream);

/* Gradients of the EOT value F* = <P*, C> - H(P*) / gamma at the potentials (u, v)
 * (envelope theorem on the Lagrangian, Appx. A; not stated in the paper), with
 * s = grad_scale * (*grad_scale_dev when given):
 *   dC = s * P                          (dense; device n x m FP32, ld m)
 *   dX_i = s * 2 s_C sum_j P_ij (x_i - y_j)  (points; device n x d FP32)
 *   dY_j = s * 2 s_C sum_i P_ij (y_j - x_i)  (points; device m x d FP32)
 *   dr = s * u / gamma, dc = s * v / gamma (device FP64)
 * grad_scale_dev: device FP64 scalar, nullable (e.g. the incoming gradient of an
 * autograd graph, read on the device so that no host synchronisation is needed).
 * Each output nullable. s_C is the problem's cost scale, held constant. P is
 * formed with each side shifted by its own log-marginal, so (u + k, v - k) gives
 * the same outputs for any k. dC needs a dense problem, dX / dY a point problem
 * (EOT_ERR_UNSUPPORTED otherwise). Outputs below the FP32 range flush to zero.
 * Errors: INVALID_ARG, UNSUPPORTED, NONFINITE, CUDA. Synchronises. */
eot_status eot_backward(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                        double gamma, double grad_scale, const double* grad_scale_dev, float* dC,
                        float* dX, float* dY, double* dr, double* dc, void* stream);

/* Integer outputs of the plan P = P(u, v; gamma) (Sec. 2.1, Eq. lagrangian-closed-form),
 * bit-exact by construction: every decision is taken in FP64 on an exponent
 * formed in a fixed order of correctly rounded operations, with no fused
 * multiply-add, so any IEEE-754 implementation of the same order agrees:
 *   C_ij  = (double)C_ij for dense costs (exact); for points
 *           C_ij = s_C * D_ij, D_ij = (...((x_i0 - y_j0)^2 + (x_i1 - y_j1)^2) + ...),
 *           the coordinates promoted to FP64 and summed in coordinate order,
 *           each difference, square, sum and the product with s_C rounded;
 *   gC_ij = gamma * C_ij (rounded), gamma used as given (not rounded to FP32).
 *
 * Row argmax: idx_out[i] = the smallest j maximising P_ij, i.e. maximising
 * t_ij = v_j - gC_ij (u_i is constant along the row and exp is increasing);
 * ties go to the lowest index. v: device [m]; idx_out: device int64 [n].
 * Errors: INVALID_ARG, CUDA. Asynchronous on `stream`. */
eot_status eot_plan_argmax(eot_handle h, const eot_problem* prob, const double* v, double gamma,
                           int64_t* idx_out, void* stream);

/* Plan support: the entries with P_ij > tau, decided as
 *   (u_i + v_j) - gC_ij > log_tau      (log_tau = log(tau), given by the caller),
 * counted per row into row_counts_out (device int64 [n], nullable) and in total
 * into total_out (device int64 scalar, nullable). u: device [n], v: device [m].
 * Errors: INVALID_ARG, CUDA. Asynchronous on `stream`. */
eot_status eot_plan_support(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                            double gamma, double log_tau, int64_t* row_counts_out, int64_t* total_out,
                            void* stream);

/* Measurement aid: times `iters` launches of one sweep kernel at (u, v) with CUDA
 * events recorded on `stream` (after an untimed set-up at the same point):
 *   kind 0: the CG column half  w = P^T p            (Alg. 2 inner CG, F_r(rho) p; dense
 *           costs: P^T (rowfac z) + beta w_prev, with the stop test in its prologue)
 *   kind 1: the CG row half     y = P (w / c(P)), q = r(P) p - rho y, <p, q> (dense
 *           costs: also p = z + beta p_prev per row)
 *   kind 2: the fused two-sided HVP sweep of eot_hvp
 *   kind 3: the row log-sum-exp sweep (Alg. 3 / Alg. 4 row updates)
 * flush == NULL: the launches run back to back between two events (the cost stays
 * in L2 when it fits, as inside a solve). flush != NULL: a device buffer of
 * flush_bytes (caller's, larger than L2) is overwritten on `stream` before each
 * launch and each launch is timed alone, so every launch reads the cost from
 * HBM. ms_out: host, average milliseconds per launch. Synchronises. */
eot_status eot_sweep_bench(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                           double gamma, int32_t kind, int32_t iters, void* flush, size_t flush_bytes,
                           double* ms_out, void* stream);

/* The marginals of eot_marginals without a handle and without allocating any
 * device memory, for callers that cannot allocate (their allocator or memory
 * budget belongs to another component, or an allocation would synchronise the
 * device at the wrong moment). The paper has no counterpart; this is a library
 * facility. The scratch space is a fixed array of about 3 MB in the library,
 * held by every GPU that loads the library until the process exits.
 * n and m must be <= 16384 (EOT_ERR_INVALID_ARG otherwise). DENSE_F32 (MIXED or
 * PLAIN_FP32) and DENSE_F64 (FP64) costs; u, v, r_out [n], c_out [m] are device
 * FP64 buffers owned by the caller; status_out (device int, nullable) receives
 * the kernels' status bits (0 = fine; non-finite or out-of-range potentials set
 * bits and give non-finite outputs). Asynchronous on `stream`; no host readback.
 * The first call on a device looks up the scratch array's address, so make it
 * before any stream capture. All calls on a device share the array: calls that
 * overlap on the GPU race, and the caller must order them. */
eot_status eot_marginals_noalloc(const eot_problem* prob, const double* u, const double* v,
                                 double gamma, double* r_out, double* c_out, int32_t* status_out,
                                 void* stream);

/* Number of this library's kernel launches issued on the handle so far. The
 * kernels of a captured program count once per execution: the body of each of
 * its loops times the trip count the device recorded. For launch accounting in
 * benchmarks. */
int64_t eot_kernel_launches(eot_handle h);

#ifdef __cplusplus
}
#endif

#endif /* EOT_H_ */
