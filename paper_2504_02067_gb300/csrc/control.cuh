// Device-side control of one stage of Alg. 1: the decisions of Alg. 4
// (TruncatedNewtonProject), Alg. 3 (ChiSinkhorn) and Alg. 2 (NewtonSolve with
// Jacobi PCG and rho annealing), taken by single-thread kernels that read the
// FP64 device scalars the sweeps reduced and write the next scalars and loop
// flags. Inside a CUDA graph each flag also drives a conditional node
// (cudaGraphSetConditional), so a whole stage runs with no host round trip;
// without a graph the host reads the same flags and runs the same kernels in
// the same order.
//
// Termination: every loop flag is cleared by a counter cap (max_newton Newton
// steps, 2000 ChiSinkhorn iterations, 61 rho annealings, max_cg CG iterations,
// max_ls halvings), by convergence, or by an error, and no flag is set again
// once an error is recorded.
#pragma once
#include "kernels.cuh"

namespace eot {

// loop / branch flags of a stage (index into Ctl::hd and the FL_* slots)
enum Flag : int { F_NEWTON = 0, F_SK, F_GO, F_CGOUT, F_CG, F_DEC, F_LS, F_UPD, F_COUNT };

// device scalars of the stage control (continuing the Sc enum of kernels.cuh)
enum ScCtl : int {
  SC_EPS = SC_CTL_BEGIN,  // tolerance eps of the projection (Alg. 4)
  SC_EPSCHI,        // eps^(2/5), ChiSinkhorn's tolerance (Alg. 3)
  SC_ETA,           // forcing parameter of the Newton step
  SC_GL1K,          // ||grad g||_1 at the start of the Newton step
  SC_RHOLAST,       // rho of the last CG solve (Appx. B); persists across steps and stages
  SC_RHOSTEP,       // rho of the last CG solve of this Newton step
  SC_ALS,           // line-search step alpha
  SC_ZERO,          // constant 0 (the alpha of the Armijo reference)
  SC_LHS0,          // Armijo left side at alpha = 0
  SC_DEC,           // the Armijo test is decidable in this precision
  SC_TRIALS,        // halvings of this line search
  SC_STEPS,         // Newton steps of this stage
  SC_DMIN,          // min delta_k of this stage (AdjustSchedule's input)
  SC_SOLVES,        // rho annealings of this Newton step
  SC_RAN,           // a CG solve ran in this Newton step
  SC_ERR,           // error code (Err) of this stage, 0 = none
  SC_SKC,           // ChiSinkhorn iterations of this Newton step
  SC_DUSRC,         // Newton direction source: 0 = Alg. 2's initial d_u0, 1 = the CG iterate
  SC_MAXNEWTON,     // caps (eot_params)
  SC_MAXLS,
  // cumulative counters of the call (doubles, exact below 2^53)
  SC_N_CGIT, SC_N_CGSOLVE, SC_N_CURV, SC_N_NEWTON, SC_N_LSTRIAL, SC_N_LSDEC, SC_N_UPD, SC_N_SK,
  SC_N_CGPASS, SC_N_NLOOP, SC_N_GO,
  SC_DEADLINE,      // %globaltimer value (ns) after which no Newton step starts (0: none)
  SC_FL0,           // SC_FL0 + Flag: the flags as doubles (read by the host executor)
  SC_ACTIVE_COL = SC_FL0 + F_COUNT,  // dense CG: the column half's stop decision, committed to
                                     // SC_ACTIVE by the update kernel (SC_ACTIVE never changes
                                     // while a column half runs)
  SC_CTL_END
};
static_assert((int)SC_CTL_END <= (int)SC_TOTAL, "device scalar array too small for the stage control");

enum Err : int { E_NONE = 0, E_MAXNEWTON, E_CHISK, E_CGMAX, E_RHO, E_LS, E_TIME };

__device__ __forceinline__ double global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (double)t;
}

// SC_DEADLINE = now + seconds (the call's wall-clock budget; seconds <= 0: none).
static __global__ void set_deadline_kernel(double* sc, double seconds) {
  pdl_wait();
  sc[SC_DEADLINE] = seconds > 0.0 ? global_ns() + seconds * 1e9 : 0.0;
}

constexpr int kMaxChiSinkhorn = 2000;  // ChiSinkhorn iterations per Newton step
constexpr int kMaxAnneal = 60;         // rho annealings per NewtonSolve
constexpr int kCgBody = 8;             // CG iterations per pass of the CG loop body

struct Ctl {
  double* sc;
  int* status;
  cudaGraphConditionalHandle hd[F_COUNT];
  int graph;        // 1: set the conditional handles too
  unsigned mask;    // flags whose handle belongs to a node of this program
  int fp64;         // FP64 path: the Armijo test is always decided
  int fused_cg;     // dense-cost CG: the column half of iteration k + 1 decides the stop
  double floor32;   // FP32 paths: rounding floor of sum P(alpha) - 1 (reading R28)
};

__device__ __forceinline__ void set_flag(const Ctl& c, int f, bool v) {
  c.sc[SC_FL0 + f] = v ? 1.0 : 0.0;
  if (c.graph && ((c.mask >> f) & 1u)) cudaGraphSetConditional(c.hd[f], v ? 1u : 0u);
}
__device__ __forceinline__ void fail(const Ctl& c, int code) {
  if (c.sc[SC_ERR] == 0.0) c.sc[SC_ERR] = (double)code;
  set_flag(c, F_NEWTON, false);
}
__device__ __forceinline__ bool ok(const Ctl& c) { return c.sc[SC_ERR] == 0.0; }

#define EOT_CTL_KERNEL(name) static __global__ void __launch_bounds__(32) name(Ctl c)
#define EOT_CTL_BEGIN       \
  pdl_wait();               \
  if (threadIdx.x != 0) return; \
  double* sc = c.sc;

// After the opening column fix and row LSE of Alg. 4.
EOT_CTL_KERNEL(ctl_stage_init) {
  EOT_CTL_BEGIN
  sc[SC_STEPS] = 0.0;
  sc[SC_DMIN] = INFINITY;
  sc[SC_ERR] = 0.0;
  set_flag(c, F_NEWTON, sc[SC_GL1] > sc[SC_EPS]);
}

// Start of a Newton-loop pass: the max_newton cap and the wall-clock budget,
// then Alg. 3's test.
EOT_CTL_KERNEL(ctl_step_a) {
  EOT_CTL_BEGIN
  sc[SC_N_NLOOP] += 1.0;
  if (sc[SC_STEPS] >= sc[SC_MAXNEWTON]) fail(c, E_MAXNEWTON);
  if (sc[SC_DEADLINE] > 0.0 && global_ns() > sc[SC_DEADLINE]) fail(c, E_TIME);
  sc[SC_SKC] = 0.0;
  set_flag(c, F_SK, ok(c) && sc[SC_CHI2] > sc[SC_EPSCHI]);
}

// After one ChiSinkhorn iteration (u fix, column fix, row LSE).
EOT_CTL_KERNEL(ctl_sk) {
  EOT_CTL_BEGIN
  sc[SC_N_SK] += 1.0;
  sc[SC_SKC] += 1.0;
  if (sc[SC_SKC] > (double)kMaxChiSinkhorn) fail(c, E_CHISK);
  set_flag(c, F_SK, ok(c) && sc[SC_CHI2] > sc[SC_EPSCHI]);
}

// Alg. 4's projection test after ChiSinkhorn, the forcing parameter and the
// first rho of the Newton step (Appx. B: max(0, 1 - 4 (1 - rho_last))).
EOT_CTL_KERNEL(ctl_step_b) {
  EOT_CTL_BEGIN
  const double gl1 = sc[SC_GL1], eps = sc[SC_EPS];
  const bool go = ok(c) && gl1 > eps;
  if (!go) set_flag(c, F_NEWTON, false);
  if (go) {
    sc[SC_N_GO] += 1.0;
    sc[SC_ETA] = fmax(gl1, 0.8 * eps / gl1);
    sc[SC_RHO] = fmax(0.0, 1.0 - 4.0 * (1.0 - sc[SC_RHOLAST]));
    sc[SC_GL1K] = gl1;
    sc[SC_SOLVES] = 0.0;
    sc[SC_RAN] = 0.0;
  }
  set_flag(c, F_GO, go);
}

// Alg. 2's first test, at d_u0 = -D(r(P))^-1 grad_u g (SC_CHECK from the set-up
// sweeps): CG runs unless it already meets the forcing test.
EOT_CTL_KERNEL(ctl_cg_begin) {
  EOT_CTL_BEGIN
  const double lim = sc[SC_ETA] * sc[SC_GL1];
  sc[SC_TOL] = 0.25 * lim;
  sc[SC_DUSRC] = 0.0;
  sc[SC_RAN] = 0.0;
  sc[SC_SOLVES] = 0.0;
  set_flag(c, F_CGOUT, ok(c) && !(sc[SC_CHECK] <= lim));
}

// After a linear CG solve and its outer test (cg_check_kernel): the counters,
// the loss-of-curvature stop (reading R21), the max_cg error, Alg. 2's forcing
// test and the rho anneal rho <- 1 - (1 - rho) / 4.
EOT_CTL_KERNEL(ctl_cg_end) {
  EOT_CTL_BEGIN
  const double it = sc[SC_ITERS];
  const bool curv = (atomicAnd(c.status, ~kStatCurv) & kStatCurv) != 0;
  // iterations whose kernels ran: the loop body repeats kCgBody of them
  const double tried = c.fused_cg ? it + 1.0 : it + (curv ? 1.0 : 0.0);
  sc[SC_N_CGIT] += it;
  sc[SC_N_CGPASS] += ceil(tried / (double)kCgBody);
  sc[SC_N_CGSOLVE] += 1.0;
  sc[SC_RAN] = 1.0;
  sc[SC_RHOSTEP] = sc[SC_RHO];
  bool more = false;
  if (curv) {
    // <p, F_r p> <= 0 in finite precision: keep the iterate and stop annealing
    sc[SC_N_CURV] += 1.0;
    sc[SC_DUSRC] = it > 0.0 ? 1.0 : 0.0;
  } else if (sc[SC_RESL1] > sc[SC_TOL]) {
    fail(c, E_CGMAX);
  } else {
    sc[SC_DUSRC] = 1.0;
    if (!(sc[SC_CHK] <= sc[SC_ETA] * sc[SC_GL1])) {
      sc[SC_RHO] = 1.0 - (1.0 - sc[SC_RHO]) / 4.0;
      sc[SC_SOLVES] += 1.0;
      if (sc[SC_SOLVES] > (double)kMaxAnneal) fail(c, E_RHO);
      else more = true;
    }
  }
  set_flag(c, F_CGOUT, more && ok(c));
}

// After d_v (Alg. 4): rho_last for the next step, the decidability of the
// Armijo test (reading R28) and the line-search start alpha = 1.
EOT_CTL_KERNEL(ctl_ls_begin) {
  EOT_CTL_BEGIN
  if (sc[SC_RAN] != 0.0) sc[SC_RHOLAST] = sc[SC_RHOSTEP];
  sc[SC_N_NEWTON] += 1.0;
  const bool dec = c.fp64 || 0.99 * sc[SC_SLOPE] >= c.floor32;
  sc[SC_DEC] = dec ? 1.0 : 0.0;
  sc[SC_ALS] = 1.0;
  sc[SC_TRIALS] = 0.0;
  sc[SC_LHS0] = 0.0;
  set_flag(c, F_DEC, dec && ok(c));
  set_flag(c, F_LS, ok(c));
  set_flag(c, F_UPD, false);
}

// The Armijo reference: the left side at alpha = 0 (reading R27).
EOT_CTL_KERNEL(ctl_lhs0) {
  EOT_CTL_BEGIN
  sc[SC_LHS0] = sc[SC_LHS];
  sc[SC_N_LSDEC] += 1.0;
}

// One trial of the backtracking line search: the simplified Armijo test
// (sum P(alpha) - 1) - (sum P(0) - 1) <= 0.99 alpha <-grad_u g, d_u> (Alg. 4,
// Lemma sufficient-decrease); a trial outside the FP32 split range is rejected
// (reading R20); alpha halves up to max_ls times.
EOT_CTL_KERNEL(ctl_trial) {
  EOT_CTL_BEGIN
  sc[SC_N_LSTRIAL] += 1.0;
  const bool range = (atomicAnd(c.status, ~kStatRange) & kStatRange) != 0;
  const double a = sc[SC_ALS];
  const bool accept = !range && (sc[SC_DEC] == 0.0 || sc[SC_LHS] - sc[SC_LHS0] <= 0.99 * a * sc[SC_SLOPE]);
  bool more = false;
  if (accept) {
    set_flag(c, F_UPD, ok(c));
  } else {
    sc[SC_TRIALS] += 1.0;
    if (sc[SC_TRIALS] > sc[SC_MAXLS]) {
      fail(c, E_LS);
      set_flag(c, F_UPD, false);
    } else {
      sc[SC_ALS] = 0.5 * a;
      more = true;
    }
  }
  set_flag(c, F_LS, more && ok(c));
}

// After the update and its row LSE: delta_k of Sec. 3.3 (actual over predicted
// decrease of ||grad g||_1), the step count and Alg. 4's loop test.
EOT_CTL_KERNEL(ctl_step_end) {
  EOT_CTL_BEGIN
  sc[SC_N_UPD] += 1.0;
  const double g0 = sc[SC_GL1K], g1 = sc[SC_GL1];
  const double delta = (g0 - g1) / ((1.0 - sc[SC_ETA]) * g0);
  if (delta < sc[SC_DMIN]) sc[SC_DMIN] = delta;
  sc[SC_STEPS] += 1.0;
  set_flag(c, F_NEWTON, ok(c) && g1 > sc[SC_EPS]);
}

#undef EOT_CTL_BEGIN
#undef EOT_CTL_KERNEL

// d_u <- the CG iterate x, or Alg. 2's initial direction d_u0 when no CG
// iterate was kept (SC_DUSRC).
static __global__ void select_du_kernel(int64_t n, const double* x, const double* du0, double* du,
                                        const double* sc) {
  pdl_wait();
  const double* src = sc[SC_DUSRC] != 0.0 ? x : du0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    du[i] = src[i];
}

}  // namespace eot
