// C ABI of include/eot.h: handle lifecycle, argument checks, dispatch to the
// FP32 (mixed / plain) and FP64 solver instantiations, error capture.
#include <cmath>
#include <cstring>

#include "plan_int.cuh"
#include "solver.cuh"

using namespace eot;

namespace eot {

static void free_all(eot_handle h) {
  free_graphs(h);
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->h_sc) cudaFreeHost(h->h_sc);
  if (h->h_status) cudaFreeHost(h->h_status);
  h->h_sc = nullptr;
  h->h_status = nullptr;
  h->cap_n = h->cap_m = h->cap_rowpart = 0;
  h->rowpart = nullptr;
}

void free_graphs(eot_handle h) {
  for (auto& kv : h->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  h->graphs.clear();
}

void ensure_capacity(eot_handle h, int64_t n, int64_t m) {
  if (n <= h->cap_n && m <= h->cap_m) return;
  EOT_CUDA(cudaDeviceSynchronize());
  const int64_t N = std::max(n, h->cap_n), Mm = std::max(m, h->cap_m);
  free_all(h);
  const int64_t L = std::max(N, Mm);
  h->max_strips = (Mm + 31) / 32 + 1;
  h->dot_slots = std::max<int64_t>(std::max<int64_t>((N + kWarps - 1) / kWarps + 1, h->max_strips), kVecCtas);
  EOT_CUDA(cudaHostAlloc((void**)&h->h_sc, (SC_TOTAL + 1) * sizeof(double), cudaHostAllocDefault));
  EOT_CUDA(cudaHostAlloc((void**)&h->h_status, sizeof(int), cudaHostAllocDefault));
  h->sc = (double*)dev_alloc(h, SC_TOTAL * sizeof(double));
  h->status = (int*)dev_alloc(h, sizeof(int));
  h->cnt_strip = (int*)dev_alloc(h, h->max_strips * sizeof(int));
  h->rowblk_slots = std::max<int64_t>(h->max_rowblk, L / 128 + 2);  // 128-point blocks of the tensor-core sweeps
  h->cnt_rowblk = (int*)dev_alloc(h, h->rowblk_slots * sizeof(int));
  h->maxbuf_len = L / 256 + 8 * (int64_t)h->sms + 64;
  h->maxbuf = (double*)dev_alloc(h, h->maxbuf_len * sizeof(double));
  h->cnt_dot = (int*)dev_alloc(h, sizeof(int));
  EOT_CUDA(cudaMemset(h->sc, 0, SC_TOTAL * sizeof(double)));
  EOT_CUDA(cudaMemset(h->status, 0, sizeof(int)));
  EOT_CUDA(cudaMemset(h->cnt_strip, 0, h->max_strips * sizeof(int)));
  EOT_CUDA(cudaMemset(h->cnt_rowblk, 0, h->rowblk_slots * sizeof(int)));
  EOT_CUDA(cudaMemset(h->cnt_dot, 0, sizeof(int)));
  h->colpart = (double*)dev_alloc(h, 2 * h->max_rowblk * Mm * sizeof(double));
  h->dotpart = (double*)dev_alloc(h, 2 * h->dot_slots * sizeof(double));
  h->cgpart = (double*)dev_alloc(h, 2 * (4 * (int64_t)h->sms + 8) * sizeof(double));
  double** nv[] = {&h->Al, &h->rowfac, &h->rP, &h->logrP, &h->rowmax, &h->rt, &h->logrt,
                   &h->du, &h->x, &h->res, &h->z, &h->p, &h->q, &h->y, &h->Yx, &h->M,
                   &h->diag, &h->y0, &h->du0, &h->nt0, &h->nt1, &h->rPs, &h->U};
  for (double** p : nv) *p = (double*)dev_alloc(h, N * sizeof(double));
  double** mv[] = {&h->Bl, &h->colfac, &h->cP, &h->logcP, &h->ct, &h->logct, &h->dv, &h->mt0, &h->mt1, &h->V, &h->wprev,
                   &h->fxv, &h->frv, &h->fzv, &h->fpv, &h->fqv};
  for (double** p : mv) *p = (double*)dev_alloc(h, Mm * sizeof(double));
  void** ev[] = {&h->Ah, &h->Bh, &h->xw0, &h->xw1, &h->zf, &h->wsq, &h->ewr, &h->ewc};
  for (void** p : ev) *p = dev_alloc(h, L * sizeof(double));
  h->cap_n = N;
  h->cap_m = Mm;
}

void ensure_rowpart(eot_handle h, int64_t n, int64_t strips) {
  ensure_rowpart_elems(h, 2 * strips * std::max(n, h->cap_n));
}

void ensure_rowpart_elems(eot_handle h, int64_t need) {
  if (need <= h->cap_rowpart) return;
  if (h->rowpart) {
    EOT_CUDA(cudaStreamSynchronize(0));
    EOT_CUDA(cudaDeviceSynchronize());
    for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
      if (*it == h->rowpart) {
        cudaFree(*it);
        h->allocs.erase(it);
        break;
      }
    free_graphs(h);
  }
  h->rowpart = (double*)dev_alloc(h, need * sizeof(double));
  h->cap_rowpart = need;
}

}  // namespace eot

namespace {

template <class F>
eot_status guarded(eot_handle h, F&& f) {
  if (!h) return EOT_ERR_INVALID_ARG;
  try {
    EOT_CUDA(cudaSetDevice(h->device));
    cudaGetLastError();  // a failed earlier call must not surface in this call's launch checks
    f();
    h->err = "no error";
    return EOT_OK;
  } catch (const EotError& e) {
    h->err = e.msg;
    if (e.st == EOT_ERR_CUDA) return e.st;
    // reset the tickets so that the next call starts clean
    if (h->cnt_strip) {
      cudaDeviceSynchronize();
      cudaMemset(h->cnt_strip, 0, h->max_strips * sizeof(int));
      cudaMemset(h->cnt_rowblk, 0, h->rowblk_slots * sizeof(int));
      cudaMemset(h->cnt_dot, 0, sizeof(int));
    }
    return e.st;
  } catch (const std::exception& e) {
    h->err = e.what();
    return EOT_ERR_CUDA;
  }
}

void check_problem(eot_handle h, const eot_problem* P, bool need_marginals) {
  if (!P) throw EotError{EOT_ERR_INVALID_ARG, "problem is NULL"};
  if (P->n < 1 || P->m < 1) throw EotError{EOT_ERR_INVALID_ARG, "n and m must be >= 1"};
  if (P->n > ((int64_t)1 << 31) || P->m > ((int64_t)1 << 31))
    throw EotError{EOT_ERR_INVALID_ARG, "n and m must be <= 2^31"};
  if (need_marginals && (!P->r || !P->c)) throw EotError{EOT_ERR_INVALID_ARG, "r and c are required"};
  switch (P->kind) {
    case EOT_COST_DENSE_F32:
      if (P->precision != EOT_PREC_MIXED && P->precision != EOT_PREC_PLAIN_FP32)
        throw EotError{EOT_ERR_UNSUPPORTED, "DENSE_F32 takes MIXED or PLAIN_FP32 precision"};
      break;
    case EOT_COST_DENSE_F64:
      if (P->precision != EOT_PREC_FP64)
        throw EotError{EOT_ERR_UNSUPPORTED, "DENSE_F64 takes FP64 precision"};
      break;
    case EOT_COST_SQEUCLID_POINTS:
      if (!P->X || !P->Y) throw EotError{EOT_ERR_INVALID_ARG, "X and Y are required for point costs"};
      if (P->d < 1 || P->d > 64) throw EotError{EOT_ERR_INVALID_ARG, "point dimension d must be in [1, 64]"};
      if (P->precision < EOT_PREC_FP64 || P->precision > EOT_PREC_PLAIN_FP32)
        throw EotError{EOT_ERR_INVALID_ARG, "unknown precision"};
      if (!(P->cost_scale >= 0.0) || !std::isfinite(P->cost_scale))
        throw EotError{EOT_ERR_INVALID_ARG, "cost_scale must be finite (<= 0 asks for 1 / max cost)"};
      ensure_capacity(h, P->n, P->m);
      return;
    default:
      throw EotError{EOT_ERR_INVALID_ARG, "unknown cost kind"};
  }
  if (!P->C) throw EotError{EOT_ERR_INVALID_ARG, "C is NULL"};
  if (P->ldc < P->m) throw EotError{EOT_ERR_INVALID_ARG, "ldc < m"};
  ensure_capacity(h, P->n, P->m);
}

void check_gamma(double g) {
  if (!(g > 0.0) || !std::isfinite(g) || g >= kSplitLimit)
    throw EotError{EOT_ERR_INVALID_ARG, "gamma must be finite, > 0 and < 2^19"};
}

bool is_f64(const eot_problem* P) {
  return P->kind == EOT_COST_DENSE_F64 ||
         (P->kind == EOT_COST_SQEUCLID_POINTS && P->precision == EOT_PREC_FP64);
}

}  // namespace

namespace {
// Row argmax (MODE 0) or support counts (MODE 1) of the plan; see plan_int.cuh.
template <int MODE>
void run_plan_int(eot_handle h, const eot_problem* P, const double* u, const double* v, double gamma,
                  double log_tau, int64_t* idx_out, int64_t* counts, int64_t* total, cudaStream_t st) {
  unsigned long long* tot = reinterpret_cast<unsigned long long*>(total);
  if (tot) EOT_CUDA(cudaMemsetAsync(tot, 0, sizeof(unsigned long long), st));
  const dim3 grid((unsigned)((P->n + pint::kWarps - 1) / pint::kWarps));
  if (P->kind == EOT_COST_SQEUCLID_POINTS) {
    double sC = P->cost_scale;
    if (!(sC > 0.0)) {
      Solver<double> S(h, P, st);  // computes s_C = 1 / max |x_i - y_j|^2 as the solver does
      sC = S.sC;
    }
    launch_k(pint::plan_int_points_kernel<MODE>, grid, dim3(pint::kThreads), st, P->n, P->m, (int)P->d, P->X, P->Y,
             sC, u, v, gamma, log_tau, idx_out, counts, tot);
  } else if (P->kind == EOT_COST_DENSE_F64) {
    launch_k(pint::plan_int_dense_kernel<double, MODE>, grid, dim3(pint::kThreads), st, P->n, P->m,
             (const double*)P->C, P->ldc, u, v, gamma, log_tau, idx_out, counts, tot);
  } else {
    launch_k(pint::plan_int_dense_kernel<float, MODE>, grid, dim3(pint::kThreads), st, P->n, P->m,
             (const float*)P->C, P->ldc, u, v, gamma, log_tau, idx_out, counts, tot);
  }
  EOT_LAUNCH_CHECK();
  h->launches++;
}
}  // namespace

extern "C" {

eot_status eot_create(eot_handle* out, int device, int64_t max_n, int64_t max_m, int64_t max_d) {
  if (!out || max_n < 1 || max_m < 1 || max_d < 0 || max_d > 64) return EOT_ERR_INVALID_ARG;
  *out = nullptr;
  eot_handle h = new eot_handle_s();
  h->device = device;
  try {
    EOT_CUDA(cudaSetDevice(device));
    EOT_CUDA(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device));
    int l2 = 0;
    EOT_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device));
    h->l2_bytes = l2;
    ensure_capacity(h, max_n, max_m);
    if (max_d > 0) {
      reserve_points(h, max_n, max_m, (int)max_d, nullptr);
      EOT_CUDA(cudaDeviceSynchronize());
    }
  } catch (const EotError& e) {
    free_all(h);
    delete h;
    return e.st;
  }
  *out = h;
  return EOT_OK;
}

eot_status eot_destroy(eot_handle h) {
  if (!h) return EOT_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  free_all(h);
  if (h->bt_mem) cudaFree(h->bt_mem);
  if (h->tc_mem) cudaFree(h->tc_mem);
  if (h->rd_mem) cudaFree(h->rd_mem);
  for (cudaStream_t& s : h->cap_streams)
    if (s) cudaStreamDestroy(s);
  delete h;
  return EOT_OK;
}

const char* eot_last_error(eot_handle h) { return h ? h->err.c_str() : "NULL handle"; }

const char* eot_status_string(eot_status s) {
  switch (s) {
    case EOT_OK: return "EOT_OK";
    case EOT_ERR_INVALID_ARG: return "EOT_ERR_INVALID_ARG";
    case EOT_ERR_NONFINITE: return "EOT_ERR_NONFINITE";
    case EOT_ERR_CG_MAXITER: return "EOT_ERR_CG_MAXITER";
    case EOT_ERR_LINESEARCH: return "EOT_ERR_LINESEARCH";
    case EOT_ERR_MAXSTAGES: return "EOT_ERR_MAXSTAGES";
    case EOT_ERR_MAXNEWTON: return "EOT_ERR_MAXNEWTON";
    case EOT_ERR_RANGE: return "EOT_ERR_RANGE";
    case EOT_ERR_CUDA: return "EOT_ERR_CUDA";
    case EOT_ERR_UNSUPPORTED: return "EOT_ERR_UNSUPPORTED";
    case EOT_ERR_DEVICE_TIMEOUT: return "EOT_ERR_DEVICE_TIMEOUT";
    case EOT_ERR_TIME_LIMIT: return "EOT_ERR_TIME_LIMIT";
  }
  return "unknown status";
}

eot_params eot_params_default(void) {
  eot_params p;
  p.gamma_i = 16.0;
  p.gamma_f = 4096.0;
  p.p = 1.5;
  p.q1 = 2.0;
  p.w_r = 0.45;
  p.tol_final = 1e-6;
  p.max_stages = 200;
  p.max_newton = 200;
  p.max_cg = 0;
  p.max_ls = 30;
  p.projector = EOT_PROJECT_NEWTON;
  p.max_sinkhorn = 0;
  p.newton_system = EOT_NEWTON_REDUCED;
  p.reserved = 0;
  p.max_seconds = 0.0;
  return p;
}

eot_status eot_marginals(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                         double gamma, double* r_out, double* c_out, double* log_r_out,
                         double* log_c_out, double* total_out, void* stream) {
  return guarded(h, [&] {
    check_problem(h, prob, false);
    check_gamma(gamma);
    if (!u || !v) throw EotError{EOT_ERR_INVALID_ARG, "u and v are required"};
    cudaStream_t st = (cudaStream_t)stream;
    if (is_f64(prob)) run_marginals<double>(h, prob, u, v, gamma, r_out, c_out, log_r_out, log_c_out, total_out, st);
    else run_marginals<float>(h, prob, u, v, gamma, r_out, c_out, log_r_out, log_c_out, total_out, st);
  });
}

eot_status eot_round(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                     double gamma, double* u_out, double* v_out, double* a_out, double* b_out,
                     double* cost_out, double* corr_l1_out, void* stream) {
  return guarded(h, [&] {
    check_problem(h, prob, true);
    check_gamma(gamma);
    if (!u || !v) throw EotError{EOT_ERR_INVALID_ARG, "u and v are required"};
    cudaStream_t st = (cudaStream_t)stream;
    if (is_f64(prob)) run_round<double>(h, prob, u, v, gamma, u_out, v_out, a_out, b_out, cost_out, corr_l1_out, st);
    else run_round<float>(h, prob, u, v, gamma, u_out, v_out, a_out, b_out, cost_out, corr_l1_out, st);
  });
}

eot_status eot_hvp(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                   double gamma, double s, const double* du, const double* dv, double* out_u,
                   double* out_v, double* r_out, double* c_out, void* stream) {
  return guarded(h, [&] {
    check_problem(h, prob, false);
    check_gamma(gamma);
    if (!u || !v || !du || !dv || !out_u || !out_v)
      throw EotError{EOT_ERR_INVALID_ARG, "u, v, du, dv, out_u, out_v are required"};
    if (!std::isfinite(s)) throw EotError{EOT_ERR_INVALID_ARG, "s must be finite"};
    cudaStream_t st = (cudaStream_t)stream;
    if (is_f64(prob)) run_hvp<double>(h, prob, u, v, gamma, s, du, dv, out_u, out_v, r_out, c_out, st);
    else run_hvp<float>(h, prob, u, v, gamma, s, du, dv, out_u, out_v, r_out, c_out, st);
  });
}

eot_status eot_newton_solve(eot_handle h, const eot_problem* prob, const double* u,
                            const double* v, double gamma, const double* r_target, double eta,
                            double rho0, int32_t max_cg, double* du_out, double* dv_out,
                            double* rho_out, int32_t* cg_iters_out, void* stream) {
  return guarded(h, [&] {
    check_problem(h, prob, false);
    check_gamma(gamma);
    if (!u || !v || !r_target || !du_out) throw EotError{EOT_ERR_INVALID_ARG, "u, v, r_target, du_out are required"};
    if (!(eta > 0.0) || !(rho0 >= 0.0 && rho0 < 1.0))
      throw EotError{EOT_ERR_INVALID_ARG, "eta must be > 0 and rho0 in [0, 1)"};
    cudaStream_t st = (cudaStream_t)stream;
    int it = 0;
    if (is_f64(prob)) run_newton<double>(h, prob, u, v, gamma, r_target, eta, rho0, max_cg, du_out, dv_out, rho_out, &it, false, st);
    else run_newton<float>(h, prob, u, v, gamma, r_target, eta, rho0, max_cg, du_out, dv_out, rho_out, &it, false, st);
    if (cg_iters_out) *cg_iters_out = it;
  });
}

eot_status eot_newton_solve_full(eot_handle h, const eot_problem* prob, const double* u,
                                 const double* v, double gamma, const double* r_target, double eta,
                                 double rho0, int32_t max_cg, double* du_out, double* dv_out,
                                 double* rho_out, int32_t* cg_iters_out, void* stream) {
  return guarded(h, [&] {
    check_problem(h, prob, false);
    check_gamma(gamma);
    if (prob->kind == EOT_COST_SQEUCLID_POINTS)
      throw EotError{EOT_ERR_UNSUPPORTED, "the full-system NewtonSolve needs a dense cost"};
    if (!u || !v || !r_target || !du_out) throw EotError{EOT_ERR_INVALID_ARG, "u, v, r_target, du_out are required"};
    if (!(eta > 0.0) || !(rho0 >= 0.0 && rho0 < 1.0))
      throw EotError{EOT_ERR_INVALID_ARG, "eta must be > 0 and rho0 in [0, 1)"};
    cudaStream_t st = (cudaStream_t)stream;
    int it = 0;
    if (is_f64(prob)) run_newton<double>(h, prob, u, v, gamma, r_target, eta, rho0, max_cg, du_out, dv_out, rho_out, &it, true, st);
    else run_newton<float>(h, prob, u, v, gamma, r_target, eta, rho0, max_cg, du_out, dv_out, rho_out, &it, true, st);
    if (cg_iters_out) *cg_iters_out = it;
  });
}

eot_status eot_solve(eot_handle h, const eot_problem* prob, const eot_params* params, double* u,
                     double* v, eot_stats* stats, void* stream) {
  return guarded(h, [&] {
    check_problem(h, prob, true);
    if (!u || !v) throw EotError{EOT_ERR_INVALID_ARG, "u and v are required"};
    eot_params prm = params ? *params : eot_params_default();
    check_gamma(prm.gamma_f);
    check_gamma(prm.gamma_i);
    if (!(prm.p >= 1.0) || !(prm.q1 > 1.0) || !(prm.w_r > 0.25 && prm.w_r < 0.5) ||
        !(prm.tol_final > 0.0) || prm.max_stages < 1 || prm.max_newton < 1 || prm.max_ls < 1 ||
        (prm.projector != EOT_PROJECT_NEWTON && prm.projector != EOT_PROJECT_SINKHORN) || prm.max_sinkhorn < 0 ||
        (prm.newton_system != EOT_NEWTON_REDUCED && prm.newton_system != EOT_NEWTON_FULL) ||
        !std::isfinite(prm.max_seconds))
      throw EotError{EOT_ERR_INVALID_ARG, "invalid eot_params"};
    if (stats) {
      // outputs cleared; the caller's record array (an input) kept
      eot_stage_record* recs = stats->stage_records;
      const int32_t cap = stats->stage_records_cap;
      std::memset(stats, 0, sizeof(*stats));
      stats->stage_records = recs;
      stats->stage_records_cap = recs ? cap : 0;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (is_f64(prob)) run_solve<double>(h, prob, &prm, u, v, stats, st);
    else run_solve<float>(h, prob, &prm, u, v, stats, st);
  });
}

eot_status eot_backward(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                        double gamma, double grad_scale, const double* grad_scale_dev, float* dC,
                        float* dX, float* dY, double* dr, double* dc, void* stream) {
  return guarded(h, [&] {
    check_problem(h, prob, false);
    check_gamma(gamma);
    if (!u || !v) throw EotError{EOT_ERR_INVALID_ARG, "u and v are required"};
    const bool pts = prob->kind == EOT_COST_SQEUCLID_POINTS;
    if ((dX || dY) && !pts) throw EotError{EOT_ERR_UNSUPPORTED, "dX / dY need a point-cloud problem"};
    if (dC && pts) throw EotError{EOT_ERR_UNSUPPORTED, "dC needs a dense cost (points: use dX / dY)"};
    cudaStream_t st = (cudaStream_t)stream;
    if (dC) {
      if (is_f64(prob)) run_backward_dense<double>(h, prob, u, v, gamma, grad_scale, grad_scale_dev, dC, st);
      else run_backward_dense<float>(h, prob, u, v, gamma, grad_scale, grad_scale_dev, dC, st);
    }
    if (dX || dY) {
      if (is_f64(prob)) run_backward_points<double>(h, prob, u, v, gamma, grad_scale, grad_scale_dev, dX, dY, st);
      else run_backward_points<float>(h, prob, u, v, gamma, grad_scale, grad_scale_dev, dX, dY, st);
    }
    const double a = grad_scale / gamma;
    if (dr) {
      launch_k(axpy4_kernel, dim3(vec_grid(prob->n)), dim3(kThreads), st, prob->n, dr, 0.0, u, a, (const double*)nullptr, (const double*)nullptr, 0.0, (const double*)nullptr, 0.0);
      launch_k(scale_by_dev_kernel, dim3(vec_grid(prob->n)), dim3(kThreads), st, prob->n, dr, grad_scale_dev);
      h->launches += 2;
    }
    if (dc) {
      launch_k(axpy4_kernel, dim3(vec_grid(prob->m)), dim3(kThreads), st, prob->m, dc, 0.0, v, a, (const double*)nullptr, (const double*)nullptr, 0.0, (const double*)nullptr, 0.0);
      launch_k(scale_by_dev_kernel, dim3(vec_grid(prob->m)), dim3(kThreads), st, prob->m, dc, grad_scale_dev);
      h->launches += 2;
    }
    EOT_LAUNCH_CHECK();
  });
}

eot_status eot_value(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                     double gamma, double* value_out, void* stream) {
  return guarded(h, [&] {
    check_problem(h, prob, true);
    check_gamma(gamma);
    if (!u || !v || !value_out) throw EotError{EOT_ERR_INVALID_ARG, "u, v and value_out are required"};
    cudaStream_t st = (cudaStream_t)stream;
    if (is_f64(prob)) run_value<double>(h, prob, u, v, gamma, value_out, st);
    else run_value<float>(h, prob, u, v, gamma, value_out, st);
  });
}


eot_status eot_plan_argmax(eot_handle h, const eot_problem* prob, const double* v, double gamma,
                           int64_t* idx_out, void* stream) {
  return guarded(h, [&] {
    check_problem(h, prob, false);
    if (!(gamma >= 0.0) || !std::isfinite(gamma)) throw EotError{EOT_ERR_INVALID_ARG, "gamma must be finite and >= 0"};
    if (!v || !idx_out) throw EotError{EOT_ERR_INVALID_ARG, "v and idx_out are required"};
    run_plan_int<0>(h, prob, nullptr, v, gamma, 0.0, idx_out, nullptr, nullptr, (cudaStream_t)stream);
  });
}

eot_status eot_plan_support(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                            double gamma, double log_tau, int64_t* row_counts_out, int64_t* total_out,
                            void* stream) {
  return guarded(h, [&] {
    check_problem(h, prob, false);
    if (!(gamma >= 0.0) || !std::isfinite(gamma)) throw EotError{EOT_ERR_INVALID_ARG, "gamma must be finite and >= 0"};
    if (!u || !v) throw EotError{EOT_ERR_INVALID_ARG, "u and v are required"};
    if (std::isnan(log_tau)) throw EotError{EOT_ERR_INVALID_ARG, "log_tau is NaN"};
    run_plan_int<1>(h, prob, u, v, gamma, log_tau, nullptr, row_counts_out, total_out, (cudaStream_t)stream);
  });
}

eot_status eot_sweep_bench(eot_handle h, const eot_problem* prob, const double* u, const double* v,
                           double gamma, int32_t kind, int32_t iters, void* flush, size_t flush_bytes,
                           double* ms_out, void* stream) {
  return guarded(h, [&] {
    check_problem(h, prob, false);
    check_gamma(gamma);
    if (!u || !v || !ms_out || kind < 0 || kind > 3 || iters < 1 || (flush && flush_bytes == 0))
      throw EotError{EOT_ERR_INVALID_ARG, "u, v, ms_out required; kind in 0..3; iters >= 1; flush_bytes > 0"};
    cudaStream_t st = (cudaStream_t)stream;
    *ms_out = is_f64(prob) ? run_sweep_bench<double>(h, prob, u, v, gamma, kind, iters, flush, flush_bytes, st)
                           : run_sweep_bench<float>(h, prob, u, v, gamma, kind, iters, flush, flush_bytes, st);
  });
}

int64_t eot_kernel_launches(eot_handle h) { return h ? h->launches : 0; }

}  // extern "C"
