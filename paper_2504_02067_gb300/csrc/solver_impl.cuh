// Definitions of the entry points declared in solver.cuh, instantiated for the
// FP32 (mixed / plain) and FP64 element types in solver_f32.cu / solver_f64.cu.
#pragma once
#include <algorithm>

#include "round.cuh"
#include "solver.cuh"

namespace eot {

inline double wall_now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

template <class T>
double round_gamma(double g) {
  // Reading of the paper (Sec. 4 uses FP64 only): the FP32 paths run every
  // temperature rounded to FP32, so that gamma * C_ij is an exact product in
  // the FMA; the FP64 path uses gamma as given.
  return sizeof(T) == 4 ? (double)(float)g : g;
}

template <class T>
void run_marginals(eot_handle h, const eot_problem* P, const double* u, const double* v,
                   double gamma, double* r_out, double* c_out, double* lr_out, double* lc_out,
                   double* total_out, cudaStream_t st) {
  Solver<T> S(h, P, st);
  EOT_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), st));
  S.set_scalar(SC_GAMMA, round_gamma<T>(gamma));
  double* lr = lr_out ? lr_out : h->logrP;
  double* lc = lc_out ? lc_out : h->logcP;
  S.row_lse(u, v, nullptr, lr, nullptr, nullptr, SC_MASS, SC_AUX1);
  S.col_lse(u, nullptr, v, nullptr, 0.0, nullptr, lc, 0, SC_AUX0, 0.0);
  if (r_out) {
    launch_k(exp_kernel, dim3(S.vg_n), dim3(kOnThreads), st, P->n, lr, r_out);
    h->launches++;
  }
  if (c_out) {
    launch_k(exp_kernel, dim3(S.vg_m), dim3(kOnThreads), st, P->m, lc, c_out);
    h->launches++;
  }
  EOT_LAUNCH_CHECK();
  if (total_out)
    EOT_CUDA(cudaMemcpyAsync(total_out, h->sc + SC_MASS, sizeof(double), cudaMemcpyDeviceToDevice, st));
  S.read();
}

// The dual value (<r, u> + <c, v> - sum P + 1) / gamma (Eq. sinkhorn-dual) into a
// device scalar: one row LSE sweep for sum P, two dot products, no host readback.
template <class T>
void run_value(eot_handle h, const eot_problem* P, const double* u, const double* v, double gamma,
               double* value_out, cudaStream_t st) {
  Solver<T> S(h, P, st);
  const double g = round_gamma<T>(gamma);
  S.set_scalar(SC_GAMMA, g);
  S.row_lse(u, v, nullptr, nullptr, nullptr, nullptr, SC_MASS, SC_AUX1);
  launch_k(dot_kernel, dim3(S.vg_n), dim3(kOnThreads), st, P->n, P->r, u, h->sc, (int)SC_AUX0, h->dotpart,
           h->cnt_dot);
  launch_k(dot_kernel, dim3(S.vg_m), dim3(kOnThreads), st, P->m, P->c, v, h->sc, (int)SC_CHK, h->dotpart,
           h->cnt_dot);
  launch_k(dual_value_kernel, dim3(1), dim3(1), st, (const double*)h->sc, (int)SC_AUX0, (int)SC_CHK,
           (int)SC_MASS, g, value_out);
  EOT_LAUNCH_CHECK();
  h->launches += 3;
}

template <class T>
void run_hvp(eot_handle h, const eot_problem* P, const double* u, const double* v, double gamma,
             double s, const double* du, const double* dv, double* ou, double* ov, double* r_out,
             double* c_out, cudaStream_t st) {
  Solver<T> S(h, P, st);
  EOT_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), st));
  S.set_scalar(SC_GAMMA, round_gamma<T>(gamma));
  // row maxima for the factorisation P = rowfac * colfac * E
  S.row_lse(u, v, nullptr, h->logrP, h->rowmax, nullptr, SC_AUX0, SC_AUX1);
  S.split_rows(u, nullptr, 0.0, h->rowmax, h->Al, nullptr, h->rowfac, h->rowmax);
  S.split_cols(v, nullptr, 0.0, nullptr, h->Bl, nullptr, h->colfac, nullptr);
  launch_k(weight_kernel<T>, dim3(S.vg_n), dim3(kOnThreads), st, P->n, h->rowfac, nullptr, S.xw0());
  launch_k(weight_kernel<T>, dim3(S.vg_n), dim3(kOnThreads), st, P->n, h->rowfac, du, S.xw1());
  launch_k(weight_kernel<T>, dim3(S.vg_m), dim3(kOnThreads), st, P->m, h->colfac, nullptr, S.zf());
  launch_k(weight_kernel<T>, dim3(S.vg_m), dim3(kOnThreads), st, P->m, h->colfac, dv, S.wsq());
  EOT_LAUNCH_CHECK();
  h->launches += 4;
  if (S.points) {
    // point costs: a row sweep (r(P), P dv) and a column sweep (c(P), P^T du), then
    // out_u = r(P) du + s P dv, out_v = s P^T du + c(P) dv
    SweepArgs<T> a = S.args();
    a.wc[0] = S.zf();
    a.wc[1] = S.wsq();
    S.template row<2, false, 0>(a, RowSumEpi{h->rowfac, h->rP, h->y});
    SweepArgs<T> b = S.args();
    b.wr[0] = S.xw0();
    b.wr[1] = S.xw1();
    S.template col<2, false, 0>(b, ColSumEpi{h->colfac, h->cP, h->mt1});
    launch_k(hvp_assemble_kernel, dim3(S.vg_n), dim3(kOnThreads), st, P->n, (const double*)h->rP,
             (const double*)h->y, du, s, ou, r_out);
    launch_k(hvp_assemble_kernel, dim3(S.vg_m), dim3(kOnThreads), st, P->m, (const double*)h->cP,
             (const double*)h->mt1, dv, s, ov, c_out);
    h->launches += 2;
    S.read();
    return;
  }
  ensure_rowpart(h, P->n, S.geo.S);
  SweepArgs<T> a = S.args();
  a.wr[0] = S.xw0();
  a.wr[1] = S.xw1();
  a.wc[0] = S.zf();
  a.wc[1] = S.wsq();
  HvpEpi e{h->rowfac, h->colfac, du, dv, s, ou, ov, r_out, c_out};
  S.template col<2, false, 2>(a, e);
  S.read();
}

template <class T>
void run_newton(eot_handle h, const eot_problem* P, const double* u, const double* v,
                double gamma, const double* rtarget, double eta, double rho0, int max_cg,
                double* du_out, double* dv_out, double* rho_out, int* iters_out, bool full, cudaStream_t st) {
  Solver<T> S(h, P, st);
  S.set_full_system(full);
  EOT_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), st));
  if (max_cg <= 0) max_cg = (int)std::min<int64_t>(4 * (full ? P->n + P->m : P->n), 2000);
  S.init_control(1, 1, max_cg);
  S.set_scalar(SC_GAMMA, round_gamma<T>(gamma));
  // the program runs on the handle's buffers (a captured graph keeps their addresses)
  S.copy(h->U, u, P->n);
  S.copy(h->V, v, P->m);
  S.copy(h->rt, rtarget, P->n);
  S.row_lse(h->U, h->V, nullptr, h->logrP, h->rowmax, h->rt);
  S.set_scalar(SC_ETA, eta);
  S.set_scalar(SC_RHO, rho0);
  const typename Solver<T>::Counters c0(S.read());
  const ProgGraph* pg = S.run_program(Solver<T>::kProgNewton, Solver<T>::kNewtonFlags, false,
                                      [&] { S.emit_newton(h->U, h->V, h->rt); });
  const double* s = S.read();
  S.account(pg, c0, typename Solver<T>::Counters(s));
  S.check_err(s);
  const double rho = s[SC_RAN] != 0.0 ? s[SC_RHOSTEP] : rho0;
  S.copy(du_out, h->du, P->n);
  if (dv_out) S.copy(dv_out, h->dv, P->m);
  S.read();
  if (rho_out) *rho_out = rho;
  if (iters_out) *iters_out = (int)S.cnt.cg_iters;
}

template <class T>
void run_solve(eot_handle h, const eot_problem* P, const eot_params* prm_in, double* u, double* v,
               eot_stats* stats, cudaStream_t st) {
  const double t0 = wall_now();
  const eot_params prm = *prm_in;
  Solver<T> S(h, P, st);
  const int64_t n = P->n, m = P->m;
  S.set_full_system(prm.newton_system == EOT_NEWTON_FULL);
  const bool capped = prm.max_seconds > 0.0;
  const int max_cg = prm.max_cg > 0 ? prm.max_cg : (int)std::min<int64_t>(4 * (S.full_system ? n + m : n), 2000);
  EOT_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), st));
  S.init_control(prm.max_newton, prm.max_ls, max_cg);
  if (capped) {
    launch_k(set_deadline_kernel, dim3(1), dim3(1), st, h->sc, prm.max_seconds);
    EOT_LAUNCH_CHECK();
    h->launches++;
  }
  // Alg. 1 runs on the handle's working potentials (h->U, h->V); u, v receive them at the end
  double* const U = h->U;
  double* const V = h->V;
  S.retain_cost();
  struct Release {  // demote the cost's L2 lines on every exit path
    Solver<T>& s;
    ~Release() {
      try {
        s.release_cost();
      } catch (...) {
      }
    }
  } release_guard{S};

  // H(r), H(c) and the masses (Alg. 1's eps_d needs min(H(r), H(c)))
  launch_k(vec_stats_kernel, dim3(S.vg_n), dim3(kOnThreads), st, n, P->r, nullptr, 0, h->sc, SC_AUX0, SC_AUX1,
                                                 h->dotpart, h->cnt_dot, h->status);
  EOT_LAUNCH_CHECK();
  EOT_CUDA(cudaMemcpyAsync(h->h_sc + SC_TOTAL - 2, h->sc + SC_AUX0, 2 * sizeof(double),
                           cudaMemcpyDeviceToHost, st));
  EOT_CUDA(cudaStreamSynchronize(st));
  const double Hr = -h->h_sc[SC_TOTAL - 2], mr = h->h_sc[SC_TOTAL - 1];
  launch_k(vec_stats_kernel, dim3(S.vg_m), dim3(kOnThreads), st, m, P->c, nullptr, 0, h->sc, SC_AUX0, SC_AUX1,
                                                 h->dotpart, h->cnt_dot, h->status);
  EOT_LAUNCH_CHECK();
  h->launches += 2;
  EOT_CUDA(cudaMemcpyAsync(h->h_sc + SC_TOTAL - 2, h->sc + SC_AUX0, 2 * sizeof(double),
                           cudaMemcpyDeviceToHost, st));
  EOT_CUDA(cudaMemcpyAsync(h->h_status, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  EOT_CUDA(cudaStreamSynchronize(st));
  const double Hc = -h->h_sc[SC_TOTAL - 2], mc = h->h_sc[SC_TOTAL - 1];
  if (*h->h_status != 0 || std::fabs(mr - 1.0) > 1e-6 || std::fabs(mc - 1.0) > 1e-6)
    throw EotError{EOT_ERR_INVALID_ARG, "r and c must be finite, non-negative and sum to 1"};
  const double H = std::min(Hr, Hc);

  // Alg. 1
  const double gamma_f = round_gamma<T>(prm.gamma_f);
  double gamma = round_gamma<T>(std::min(prm.gamma_i, prm.gamma_f));
  double gamma_prev = 0.0, q = prm.q1, gl1 = 0.0;
  const double w_c = 0.5 - prm.w_r;
  int t = 1;
  if (n == 1 || m == 1) {
    // one row or one column: U(r, c) is the single plan r c^T and eps_d of Alg. 1
    // (min(H(r), H(c)) / gamma^p) is 0; return its potentials directly
    launch_k(closed_form_kernel<T>, dim3(std::max(S.vg_n, S.vg_m)), dim3(kOnThreads), st, n, m, P->r, P->c,
             gamma_f, S.points ? (const T*)nullptr : S.C, P->ldc, S.X, S.Y, (int)S.d, S.sC, U, V);
    EOT_LAUNCH_CHECK();
    h->launches++;
    gamma = gamma_f;
    t = 0;
  }
  // stats of the call; s == nullptr: stopped by an error (marg_err_l1 = NaN,
  // final_gamma = the stage in progress)
  auto fill_stats = [&](const double* s) {
    if (!stats) return;
    const SolveCounters& c = S.cnt;
    stats->sweeps_cg = c.sweeps_cg;
    stats->sweeps_newton = c.sweeps_newton;
    stats->sweeps_linesearch = c.sweeps_ls;
    stats->sweeps_sinkhorn = c.sweeps_sk;
    stats->sweeps_total = c.sweeps_cg + c.sweeps_newton + c.sweeps_ls + c.sweeps_sk + c.sweeps_stage + c.sweeps_other;
    stats->sweeps_stage = c.sweeps_stage;
    stats->stage_records_len = stats->stage_records ? std::min<int32_t>(s ? t : t - 1, stats->stage_records_cap) : 0;
    stats->stages = t;
    stats->newton_steps = (int32_t)c.newton_steps;
    stats->cg_iters = (int32_t)c.cg_iters;
    stats->cg_solves = (int32_t)c.cg_solves;
    stats->ls_trials = (int32_t)c.ls_trials;
    stats->sinkhorn_iters = (int32_t)c.sk_iters;
    stats->curvature_stops = (int32_t)c.curvature_stops;
    stats->final_gamma = gamma;
    stats->final_rho = s ? s[SC_RHOLAST] : h->h_sc[SC_RHOLAST];
    stats->grad_l1 = s ? gl1 : h->h_sc[SC_GL1];
    stats->marg_err_l1 = s ? s[SC_GL1] + s[SC_AUX1] : NAN;
    stats->seconds = wall_now() - t0;
  };
  try {
    for (; t > 0;) {
      if (capped && wall_now() - t0 > prm.max_seconds)
        throw EotError{EOT_ERR_TIME_LIMIT, "max_seconds reached before stage " + std::to_string(t)};
      const bool done = gamma == gamma_f;
      double eps_d = H / std::pow(gamma, prm.p);
      if (done) eps_d = std::min(eps_d, 2.0 * prm.tol_final / 3.0);
      launch_k(smooth_kernel, dim3(S.vg_n), dim3(kOnThreads), st, n, P->r, prm.w_r * eps_d, h->rt, h->logrt);
      launch_k(smooth_kernel, dim3(S.vg_m), dim3(kOnThreads), st, m, P->c, w_c * eps_d, h->ct, h->logct);
      EOT_LAUNCH_CHECK();
      h->launches += 2;
      if (t == 1) {
        S.copy(U, h->logrt, n);
        S.copy(V, h->logct, m);
        S.copy(h->nt0, h->logrt, n);
        S.copy(h->mt0, h->logct, m);
      }
      S.set_scalar(SC_GAMMA, gamma);
      double dmin = INFINITY;
      const SolveCounters c0 = S.cnt;
      if (prm.projector == EOT_PROJECT_SINKHORN) {
        if (!S.project_sinkhorn(eps_d / 2.0, prm, &gl1))
          throw EotError{EOT_ERR_MAXNEWTON, "Sinkhorn projection exceeded max_sinkhorn"};
      } else {
        S.project(eps_d / 2.0, &dmin, &gl1);
      }
      // AdjustSchedule (Sec. 3.3); a stage without Newton steps has delta_min = +inf
      if (dmin > 0.95) q = std::min(2.0, q * q);
      else if (dmin < 0.8) q = std::sqrt(q);
      if (stats && stats->stage_records && t - 1 < stats->stage_records_cap) {
        const SolveCounters& c1 = S.cnt;
        eot_stage_record& rec = stats->stage_records[t - 1];
        rec.gamma = gamma;
        rec.eps = eps_d / 2.0;
        rec.delta_min = dmin;
        rec.q_next = q;
        rec.newton_steps = (int32_t)(c1.newton_steps - c0.newton_steps);
        rec.cg_iters = (int32_t)(c1.cg_iters - c0.cg_iters);
        rec.ls_trials = (int32_t)(c1.ls_trials - c0.ls_trials);
        rec.sinkhorn_iters = (int32_t)(c1.sk_iters - c0.sk_iters);
        rec.sweeps = (c1.sweeps_cg + c1.sweeps_newton + c1.sweeps_ls + c1.sweeps_sk + c1.sweeps_stage +
                      c1.sweeps_other) -
                     (c0.sweeps_cg + c0.sweeps_newton + c0.sweeps_ls + c0.sweeps_sk + c0.sweeps_stage +
                      c0.sweeps_other);
      }
      const double gamma_next = round_gamma<T>(std::min(q * gamma, gamma_f));
      if (done) break;
      if (t >= prm.max_stages) throw EotError{EOT_ERR_MAXSTAGES, "gamma_f not reached within max_stages"};
      // Alg. 1's extrapolated warm start: z <- z + ratio (z - z_prev), z_prev <- z
      const double ratio = (gamma_next - gamma) / (gamma - gamma_prev);
      S.copy(h->nt1, U, n);
      S.axpy(n, U, 1.0 + ratio, h->nt0, -ratio);
      std::swap(h->nt0, h->nt1);
      S.copy(h->mt1, V, m);
      S.axpy(m, V, 1.0 + ratio, h->mt0, -ratio);
      std::swap(h->mt0, h->mt1);
      gamma_prev = gamma;
      gamma = gamma_next;
      ++t;
    }
  } catch (const EotError& e) {
    // a cap or a non-finite value stopped Alg. 1: the caller still gets the last
    // iterate (the stage in progress) and the work done so far, e.g. to measure
    // the error it reached at that stage's temperature
    if (e.st != EOT_ERR_CUDA && e.st != EOT_ERR_DEVICE_TIMEOUT) {
      S.copy(u, U, n);
      S.copy(v, V, m);
      cudaStreamSynchronize(st);
      fill_stats(nullptr);
    }
    throw;
  }

  // marginal L1 error of the output against the unsmoothed r, c, at gamma_f (set
  // here too: the one-row / one-column closed form runs no stage that sets it)
  S.set_scalar(SC_GAMMA, gamma);
  S.sweep_bucket = &S.cnt.sweeps_other;
  S.copy(u, U, n);
  S.copy(v, V, m);
  S.row_lse(u, v, nullptr, h->logrP, nullptr, P->r, SC_GL1, SC_CHI2);
  S.col_lse(u, nullptr, v, nullptr, 0.0, nullptr, h->logcP, 0, SC_AUX0, 0.0);
  launch_k(exp_kernel, dim3(S.vg_m), dim3(kOnThreads), st, m, h->logcP, h->mt1);
  launch_k(vec_stats_kernel, dim3(S.vg_m), dim3(kOnThreads), st, m, h->mt1, P->c, 1, h->sc, SC_AUX1, -1,
                                                 h->dotpart, h->cnt_dot, h->status);
  EOT_LAUNCH_CHECK();
  h->launches += 2;
  S.release_cost();
  fill_stats(S.read());
}

template <class T>
double run_sweep_bench(eot_handle h, const eot_problem* P, const double* u, const double* v,
                       double gamma, int kind, int iters, void* flush, size_t flush_bytes, cudaStream_t st) {
  Solver<T> S(h, P, st);
  EOT_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), st));
  S.retain_cost();
  S.set_scalar(SC_GAMMA, round_gamma<T>(gamma));
  // untimed set-up: the Newton-step factorisation and a CG start at rho = 1/2
  S.row_lse(u, v, nullptr, h->logrP, h->rowmax, nullptr, SC_AUX0, SC_AUX1);
  launch_k(exp_kernel, dim3(S.vg_n), dim3(kOnThreads), st, P->n, h->logrP, h->rt);  // r~ := r(P) (any finite target)
  EOT_LAUNCH_CHECK();
  // Newton-step set-up without CG (eta huge: Alg. 2's first test passes), run directly
  S.init_control(1, 1, 1);
  S.copy(h->U, u, P->n);
  S.copy(h->V, v, P->m);
  S.set_scalar(SC_GL1, 1.0);
  S.set_scalar(SC_ETA, 1e300);
  S.set_scalar(SC_RHO, 0.0);
  S.run_program(Solver<T>::kProgNewton, Solver<T>::kNewtonFlags, true, [&] { S.emit_newton(h->U, h->V, h->rt); });
  S.set_scalar(SC_RHO, 0.5);
  S.set_scalar(SC_TOL, -1.0);
  S.set_scalar(SC_MAXIT, 1e6);
  // a positive direction p = rowfac (so <p, F_r p> > 0) and its column-sweep weights
  launch_k(weight_kernel<double>, dim3(S.vg_n), dim3(kOnThreads), st, P->n, h->rowfac, nullptr, h->p);
  launch_k(weight_kernel<T>, dim3(S.vg_n), dim3(kOnThreads), st, P->n, h->rowfac, h->p, S.xw0());
  S.set_scalar(SC_RZ, 1.0);
  if (!S.points) {
    // the dense CG kernels read the update kernel's partials: start them as cg_init does
    launch_k(cg_init_fused_kernel<T>, dim3(S.vg_n), dim3(kOnThreads), st, P->n, (const double*)h->rP,
             (const double*)h->rPs, (const double*)h->rt, (const double*)h->diag, (const double*)h->rowfac, h->M,
             h->x, h->res, h->z, h->p, h->Yx, S.xw0(), h->sc, h->cgpart, (int)SC_ACTIVE_COL,
             (cudaGraphConditionalHandle)0);
    EOT_LAUNCH_CHECK();
  }
  EOT_LAUNCH_CHECK();
  if (kind == 2 && S.points) throw EotError{EOT_ERR_UNSUPPORTED, "kind 2 (fused HVP sweep) needs a dense cost"};
  if (kind == 2) {
    launch_k(weight_kernel<T>, dim3(S.vg_n), dim3(kOnThreads), st, P->n, h->rowfac, nullptr, S.xw1());
    launch_k(weight_kernel<T>, dim3(S.vg_m), dim3(kOnThreads), st, P->m, h->colfac, nullptr, S.wsq());
    ensure_rowpart(h, P->n, S.geo.S);
  }
  cudaEvent_t e0, e1;
  EOT_CUDA(cudaEventCreate(&e0));
  EOT_CUDA(cudaEventCreate(&e1));
  SweepArgs<T> a = S.args();
  float total_ms = 0.f;
  if (!flush) EOT_CUDA(cudaEventRecord(e0, st));
  for (int k = 0; k < iters; ++k) {
    if (flush) {
      // evict the cost from L2; the GPU stays busy up to e0, so the launch
      // below is queued behind it and no host latency enters the timing
      EOT_CUDA(cudaMemsetAsync(flush, (k + 1) & 0xff, flush_bytes, st));
      EOT_CUDA(cudaEventRecord(e0, st));
    }
    if (kind == 0) {
      a.wr[0] = S.xw0();
      if (S.points)
        S.template col<1, false, 0>(a, CgColEpi<T>{h->colfac, h->cP, S.zf()});
      else
        S.launch_cg_col(st, a, CgColFusedEpi<T>{h->colfac, h->cP, S.zf(), h->wprev, h->cgpart, S.vg_n, h->sc,
                                                h->status, (cudaGraphConditionalHandle)0, 0.0, false, 0,
                                                (int)SC_ACTIVE_COL});
    } else if (kind == 1) {
      a.wc[0] = S.zf();
      if (S.points)
        S.template row<1, false, 0>(a, CgRowEpi{h->rowfac, h->rPs, h->p, h->y, h->q, h->sc, h->status});
      else
        S.template launch_row_dense<1, false, 0>(st, a, CgRowFusedEpi{h->rowfac, h->rPs, h->z, h->p, h->y, h->q, h->sc});
    } else if (kind == 2) {
      a.wr[0] = S.xw0();
      a.wr[1] = S.xw1();
      a.wc[0] = S.zf();
      a.wc[1] = S.wsq();
      S.template col<2, false, 2>(a, HvpEpi{h->rowfac, h->colfac, h->x, h->dv, 1.0, h->y, h->mt1, nullptr, nullptr});
    } else {
      a.wc[0] = S.ewc();
      S.template row<1, true, 0>(a, RowLseEpi{nullptr, h->Al, h->y, nullptr, nullptr, h->sc, SC_AUX0, SC_AUX1});
    }
    if (flush) {
      EOT_CUDA(cudaEventRecord(e1, st));
      EOT_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      EOT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      total_ms += ms;
    }
  }
  if (!flush) {
    EOT_CUDA(cudaEventRecord(e1, st));
    EOT_CUDA(cudaEventSynchronize(e1));
    EOT_CUDA(cudaEventElapsedTime(&total_ms, e0, e1));
  }
  S.release_cost();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  S.read();
  return (double)total_ms / (iters > 0 ? iters : 1);
}

template <class T>
void run_backward_dense(eot_handle h, const eot_problem* P, const double* u, const double* v,
                        double gamma, double scale, const double* scale_dev, float* dC, cudaStream_t st) {
  Solver<T> S(h, P, st);
  EOT_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), st));
  S.set_scalar(SC_GAMMA, round_gamma<T>(gamma));
  S.row_lse(u, v, nullptr, h->logrP, h->rowmax, nullptr, SC_AUX0, SC_AUX1);
  S.split_rows(u, nullptr, 0.0, h->rowmax, h->Al, nullptr, h->rowfac, h->rowmax);
  S.split_cols(v, nullptr, 0.0, nullptr, h->Bl, nullptr, h->colfac, nullptr);
  if (scale_dev) {
    launch_k(scale_by_dev_kernel, dim3(S.vg_n), dim3(kOnThreads), st, P->n, h->rowfac, scale_dev);
    h->launches++;
  }
  int64_t blocks = (P->n * P->m + kThreads - 1) / kThreads;
  if (blocks > 16 * (int64_t)h->sms * 8) blocks = 16 * (int64_t)h->sms * 8;
  launch_k(plan_dense_kernel<T>, dim3((unsigned)blocks), dim3(kThreads), st, P->n, P->m, S.C, P->ldc, S.Ah(), S.Bh(),
                                                              h->sc + SC_GAMMA, h->rowfac, h->colfac,
                                                              scale, dC, P->m);
  EOT_LAUNCH_CHECK();
  h->launches++;
  S.read();
}

// dX_i = scale 2 s_C sum_j P_ij (x_i - y_j), dY_j = scale 2 s_C sum_i P_ij (y_j - x_i)
// at the potentials (u, v). Each side is swept with its own log-marginal as the
// shift (Ah = u - log r(P) for dX, Bh = v - log c(P) for dY), so the FP32
// exponents are <= 0 whatever the gauge of (u, v).
template <class T>
void run_backward_points(eot_handle h, const eot_problem* P, const double* u, const double* v,
                         double gamma, double scale, const double* scale_dev, float* dX, float* dY,
                         cudaStream_t st) {
  Solver<T> S(h, P, st);
  EOT_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), st));
  S.set_scalar(SC_GAMMA, round_gamma<T>(gamma));
  const double f = scale * 2.0 * S.sC;
  if (dX) {
    S.row_lse(u, v, nullptr, h->logrP, h->rowmax, nullptr, SC_AUX0, SC_AUX1);
    S.split_rows(u, nullptr, 0.0, h->logrP, h->Al, nullptr, h->rowfac, h->logrP);
    S.split_cols(v, nullptr, 0.0, nullptr, h->Bl, S.ewc(), nullptr, nullptr);
    if (scale_dev) {
      launch_k(scale_by_dev_kernel, dim3(S.vg_n), dim3(kOnThreads), st, P->n, h->rowfac, scale_dev);
      h->launches++;
    }
    S.template grad_pts<true>(f, h->rowfac, dX);
  }
  if (dY) {
    S.col_lse(u, nullptr, v, nullptr, 0.0, nullptr, h->logcP, 0, SC_AUX0, 0.0);
    S.split_rows(u, nullptr, 0.0, nullptr, h->Al, S.ewr(), nullptr, nullptr);
    S.split_cols(v, nullptr, 0.0, h->logcP, h->Bl, nullptr, h->colfac, h->logcP);
    if (scale_dev) {
      launch_k(scale_by_dev_kernel, dim3(S.vg_m), dim3(kOnThreads), st, P->m, h->colfac, scale_dev);
      h->launches++;
    }
    S.template grad_pts<false>(f, h->colfac, dY);
  }
  S.read();
}

}  // namespace eot

namespace eot {

// Round (see round.cuh) of P(u, v; gamma) onto U(r, c), implicit: outputs
// u + log x, v + log y, a, b (device, nullable) and <Round(P), C>, ||a||_1 (host,
// nullable). gamma is rounded as the solver rounds it for this precision.
template <class T>
void run_round(eot_handle h, const eot_problem* P, const double* u, const double* v, double gamma,
               double* u_out, double* v_out, double* a_out, double* b_out, double* cost_out, double* corr_out,
               cudaStream_t st) {
  Solver<T> S(h, P, st);
  const int64_t n = P->n, m = P->m;
  const double g = round_gamma<T>(gamma);
  const int64_t strips = (m + 31) / 32;
  int64_t nrb = std::min<int64_t>(64, std::max<int64_t>(1, (8 * (int64_t)h->sms + strips - 1) / strips));
  nrb = std::min<int64_t>(nrb, n);
  const int64_t rows_per = (n + nrb - 1) / nrb;
  nrb = (n + rows_per - 1) / rows_per;
  const size_t need = (size_t)(4 * n + 3 * m + nrb * m + 2) * sizeof(double);
  if (need > h->rd_bytes) {
    EOT_CUDA(cudaStreamSynchronize(st));
    if (h->rd_mem) cudaFree(h->rd_mem);
    h->rd_mem = nullptr;
    h->rd_bytes = 0;
    EOT_CUDA(cudaMalloc(&h->rd_mem, need));
    h->rd_bytes = need;
  }
  double* w = (double*)h->rd_mem;
  double* x = w;
  double* a = a_out ? a_out : w + n;
  double* rowc = w + 2 * n;
  double* rowcb = w + 3 * n;
  double* y = w + 4 * n;
  double* b = b_out ? b_out : w + 4 * n + m;
  double* part = w + 4 * n + 2 * m;
  double* tot = part + nrb * m;
  const int row_blocks = (int)std::min<int64_t>((n + 7) / 8, 32 * (int64_t)h->sms);
  const dim3 col_grid((unsigned)strips, (unsigned)nrb);
  const int fin_blocks = (int)std::min<int64_t>((m + rnd::kThreads - 1) / rnd::kThreads, 8 * (int64_t)h->sms);
  auto go = [&](auto cost) {
    rnd::round_row_kernel<<<row_blocks, rnd::kThreads, 0, st>>>(n, m, u, v, g, cost, P->r, nullptr, nullptr, nullptr,
                                                              x, u_out, nullptr, nullptr, nullptr);
    rnd::round_col_kernel<<<col_grid, rnd::kThreads, 0, st>>>(n, m, u, x, v, g, cost, rows_per, part);
    rnd::round_colfin_kernel<<<fin_blocks, rnd::kThreads, 0, st>>>(m, (int)nrb, part, P->c, v, y, v_out, b);
    rnd::round_row_kernel<<<row_blocks, rnd::kThreads, 0, st>>>(n, m, u, v, g, cost, P->r, x, y, b, nullptr,
                                                              nullptr, a, rowc, rowcb);
    rnd::round_total_kernel<<<1, 1024, 0, st>>>(n, a, rowc, rowcb, tot);
    EOT_LAUNCH_CHECK();
    h->launches += 5;
  };
  if (S.points) go(rnd::PointCost{S.X, S.Y, S.d, S.sC});
  else if (P->kind == EOT_COST_DENSE_F64) go(rnd::DenseCost<double>{(const double*)P->C, P->ldc});
  else go(rnd::DenseCost<float>{(const float*)P->C, P->ldc});
  EOT_CUDA(cudaMemcpyAsync(h->h_sc + SC_TOTAL - 2, tot, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  EOT_CUDA(cudaStreamSynchronize(st));
  if (cost_out) *cost_out = h->h_sc[SC_TOTAL - 2];
  if (corr_out) *corr_out = h->h_sc[SC_TOTAL - 1];
}

}  // namespace eot
