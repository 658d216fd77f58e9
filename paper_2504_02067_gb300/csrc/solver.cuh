// Host orchestration of the truncated-Newton EOT solver over the sweep kernels.
//   Alg. 1 (MDOT, adaptive q, smoothing)  -> run_solve
//   Alg. 4 (TruncatedNewtonProject)       -> Solver::project
//   Alg. 3 (ChiSinkhorn)                  -> inside Solver::project
//   Alg. 2 (NewtonSolve) + Jacobi PCG     -> Solver::newton
// Control flow stays on the host; every test reads a few FP64 scalars that the
// kernels reduced on the device. The CG iterations of one linear solve run as a
// captured CUDA graph of several iterations whose kernels turn into no-ops once
// the device-side stop flag is cleared (or, optionally, as a graph WHILE node).
#pragma once
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "handle.cuh"
#include "sweep_pts.cuh"
#include "sweep_tc.cuh"
#include "sweep_bulk.cuh"
#include "cg_persistent.cuh"

namespace eot {

struct SolveCounters {
  int64_t sweeps_cg = 0, sweeps_newton = 0, sweeps_ls = 0, sweeps_sk = 0, sweeps_stage = 0, sweeps_other = 0;
  int64_t cg_iters = 0, cg_solves = 0, newton_steps = 0, ls_trials = 0, sk_iters = 0;
  int64_t curvature_stops = 0;
  double rho_last = 0.0;
};

enum class CgMode { kHost, kBatch, kWhile };

// Default: one graph launch per linear CG solve, its WHILE node re-evaluated
// every kWhileBody iterations (no host round trip inside the solve); "batch":
// graph launches of six iterations with a host check of the stop flag after
// each (measured 4% slower on the 64 x 64 grid workload); "none": direct
// launches, four iterations per check.
constexpr int kWhileBody = 8;
inline CgMode cg_mode_from_env() {
  const char* e = std::getenv("EOT_CG_GRAPH");
  if (!e) return CgMode::kWhile;
  if (!std::strcmp(e, "batch")) return CgMode::kBatch;
  if (!std::strcmp(e, "none")) return CgMode::kHost;
  return CgMode::kWhile;
}

template <class T>
struct Solver {
  static constexpr int VEC = 16 / (int)sizeof(T);
  eot_handle h;
  cudaStream_t st;
  int64_t n, m, ldc;
  const T* C;
  int V;
  bool plain;
  int vg_n, vg_m, rg;
  ColGeo geo;
  SolveCounters cnt;
  int64_t* sweep_bucket;

  // point-cloud cost (C == nullptr): C_ij = sC |x_i - y_j|^2
  bool points = false;
  const float *X = nullptr, *Y = nullptr;
  int d = 0;
  double sC = 0.0;

  Solver(eot_handle h_, const eot_problem* P, cudaStream_t s)
      : h(h_), st(s), n(P->n), m(P->m), ldc(P->ldc), C((const T*)P->C) {
    plain = P->precision == EOT_PREC_PLAIN_FP32;
    points = P->kind == EOT_COST_SQEUCLID_POINTS;
    if (points) {
      C = nullptr;
      ldc = m;
      X = P->X;
      Y = P->Y;
      d = (int)P->d;
      V = 1;
      // partial buffers of both orientations, before any graph capture: up to
      // kPtsMaxPartials FP64 partials per owned element and chunk (the Newton
      // set-up row sweep reduces three sums)
      ensure_rowpart_elems(h, kPtsMaxPartials * pts_geo(true).S * n);
      ensure_rowpart_elems(h, kPtsMaxPartials * pts_geo(false).S * m);
      sC = P->cost_scale > 0.0 ? P->cost_scale : max_cost_scale();
      if constexpr (sizeof(T) == 4) {
        if (!plain && d >= tc::kMinD && tc_enabled()) setup_tc();
      }
    } else {
      const bool aligned = ((uintptr_t)C % 16) == 0;
      V = (aligned && (m % VEC) == 0 && (ldc % VEC) == 0) ? VEC : 1;
    }
    vg_n = vec_grid(n);
    vg_m = vec_grid(m);
    rg = row_grid(n);
    geo = col_geo(h, n, m, V);
    sweep_bucket = &cnt.sweeps_other;
    if constexpr (sizeof(T) == 4) {
      if (!points) setup_bulk();
    }
  }

  // ---- bulk-copy sweeps (dense FP32 cost, 16-byte rows, large enough) ----
  bool bulk_rows = false, bulk_cols = false;
  int bulk_rg = 0;                 // row sweep: CTAs
  int bulk_br = 0, bulk_R = 0;     // column sweep: rows per block, blocks
  int64_t bulk_S = 0;              // column sweep: strips of kColSW columns
  int bulk_stages = 0;             // column sweep: ring stages
  CUtensorMap bulk_map;            // column sweep: the cost as an m x n tensor of kColSW x kColRB boxes
  // Opt-in (EOT_BULK=1): on the 64 x 64 grid workload these sweeps measured
  // slower than the register-load kernels (CG halves 17.7 / 16.5 us against
  // 13.1 / 14.7 us back to back, solve 0.118 s against 0.091 s), so they are not
  // the default.
  static bool bulk_enabled() {
    const char* e = std::getenv("EOT_BULK");
    return e && e[0] == '1';
  }
  static void bulk_attr(const void* kernel) {
    EOT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  bulk::kSmemOptIn - bulk::kBarBytes));
  }
  // cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
  typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeTiled encode_tiled() {
    static EncodeTiled fn = [] {
      void* f = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
              cudaSuccess ||
          q != cudaDriverEntryPointSuccess)
        f = nullptr;
      return (EncodeTiled)f;
    }();
    return fn;
  }
  void setup_bulk() {
    if (!bulk_enabled() || V != VEC || n * m < bulk::kMinEntries || m < 128) return;
    bulk_rg = (int)std::min<int64_t>(std::min<int64_t>(h->sms, n), h->dot_slots);
    bulk_rows = true;
    // column strips of kColSW columns x row blocks (multiples of kColRB rows)
    // filling the SMs once
    const int64_t S = (m + bulk::kColSW - 1) / bulk::kColSW;
    int64_t R = std::min<int64_t>(std::min<int64_t>(h->sms / std::max<int64_t>(S, 1), (n + bulk::kColRB - 1) / bulk::kColRB),
                                  h->max_rowblk);
    EncodeTiled enc = encode_tiled();
    if (S <= h->sms && S <= h->max_strips && S <= h->dot_slots && R >= 1 && enc) {
      int64_t BR = (n + R - 1) / R;
      BR = (BR + bulk::kColRB - 1) / bulk::kColRB * bulk::kColRB;
      R = (n + BR - 1) / BR;
      const int64_t room = bulk::kSmemOptIn - 1024 - bulk::kBarBytes - 3 * BR * 4;
      const int stages = (int)std::min<int64_t>(bulk::kColMaxStages, room / bulk::kStageBytes);
      const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
      const cuuint64_t strides[1] = {(cuuint64_t)ldc * sizeof(float)};
      const cuuint32_t box[2] = {(cuuint32_t)bulk::kColSW, (cuuint32_t)bulk::kColRB};
      const cuuint32_t estr[2] = {1, 1};
      if (stages >= 4 &&
          enc(&bulk_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)C, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
        bulk_S = S;
        bulk_R = (int)R;
        bulk_br = (int)BR;
        bulk_stages = stages;
        bulk_cols = true;
      }
    }
    static bool attrs = false;
    if (!attrs) {
      // every instantiation, before any graph capture
      bulk_attr((const void*)bulk::row_bulk_kernel<12, 1, 1, true, 0, RowLseEpi>);
      bulk_attr((const void*)bulk::row_bulk_kernel<8, 1, 1, true, 0, RowLseEpi>);
      bulk_attr((const void*)bulk::row_bulk_kernel<12, 1, 3, false, 2, SetupRowEpi>);
      bulk_attr((const void*)bulk::row_bulk_kernel<8, 1, 3, false, 2, SetupRowEpi>);
      bulk_attr((const void*)bulk::row_bulk_kernel<12, 1, 1, false, 0, CgRowEpi>);
      bulk_attr((const void*)bulk::row_bulk_kernel<8, 1, 1, false, 0, CgRowEpi>);
      bulk_attr((const void*)bulk::col_bulk_kernel<1, true, ColLseEpi>);
      bulk_attr((const void*)bulk::col_bulk_kernel<2, false, SetupColEpi<float>>);
      bulk_attr((const void*)bulk::col_bulk_kernel<1, false, CgColEpi<float>>);
      bulk_attr((const void*)bulk::col_bulk_kernel<1, false, DvColEpi>);
      attrs = true;
    }
  }
  // Bulk row sweep when eligible: twelve one-stage consumer warps when the
  // column vectors fit beside their 192 KB ring, else eight; false: use the
  // register-load kernel.
  template <int NR, bool LSE, int SQM, class Epi>
  bool launch_row_bulk(cudaStream_t s, const SweepArgs<T>& a, const Epi& e) {
    if constexpr (sizeof(T) != 4) {
      return false;
    } else {
      if (!bulk_rows) return false;
      constexpr int NV = 1 + (LSE ? 1 : NR);
      const size_t s12 = bulk::row_smem_bytes(12, NV, m), s8 = bulk::row_smem_bytes(8, NV, m);
      if (s12 + 1024 <= (size_t)bulk::kSmemOptIn)
        launch_kd(bulk::row_bulk_kernel<12, 1, NR, LSE, SQM, Epi>, dim3(bulk_rg), dim3(13 * 32), s12, s, a, e);
      else if (s8 + 1024 <= (size_t)bulk::kSmemOptIn)
        launch_kd(bulk::row_bulk_kernel<8, 1, NR, LSE, SQM, Epi>, dim3(bulk_rg), dim3(9 * 32), s8, s, a, e);
      else
        return false;
      return true;
    }
  }
  template <int NC, bool LSE, class Epi>
  bool launch_col_bulk(cudaStream_t s, const SweepArgs<T>& a, const Epi& e) {
    if constexpr (sizeof(T) != 4) {
      return false;
    } else {
      if (!bulk_cols) return false;
      SweepArgs<T> b = a;
      b.rows_per_block = bulk_br;
      b.nrowblk = bulk_R;
      b.stages = bulk_stages;
      const size_t smem = (size_t)bulk::kBarBytes + (size_t)bulk_stages * bulk::kStageBytes + 3 * (size_t)bulk_br * 4;
      launch_kd(bulk::col_bulk_kernel<NC, LSE, Epi>, dim3((unsigned)bulk_S, (unsigned)bulk_R),
                dim3(bulk::kColThreads), smem, s, b, e, bulk_map);
      return true;
    }
  }

  // ---- point-cloud geometry: own blocks of 256 RO elements x S chunks ----
  struct PtsGeo {
    int64_t B, S, chunk;
  };
  static int pts_ro(int d) { return d <= 4 ? 4 : (d <= 16 ? 2 : 1); }
  PtsGeo pts_geo(bool rows) const {
    const int64_t n_own = rows ? n : m, n_oth = rows ? m : n;
    PtsGeo g;
    g.B = (n_own + (int64_t)kThreads * pts_ro(d) - 1) / ((int64_t)kThreads * pts_ro(d));
    int64_t S = (2 * (int64_t)h->sms + g.B - 1) / g.B;
    S = std::max<int64_t>(1, std::min<int64_t>(S, (n_oth + 31) / 32));
    g.chunk = ((n_oth + S - 1) / S + 31) / 32 * 32;
    g.S = (n_oth + g.chunk - 1) / g.chunk;
    return g;
  }
  // ---- tensor-core point path (mixed precision, d >= tc::kMinD) ----
  bool tc_on = false;
  tc::TcArgs targs{};
  static bool tc_enabled() {
    const char* e = std::getenv("EOT_TC");
    return !(e && e[0] == '0');
  }
  struct TcGeo {
    int64_t B, S, chunk;
  };
  // own blocks of 128 points x S chunks of the other side (multiples of 48),
  // S chosen so that B S fills whole waves of one-CTA-per-SM blocks
  TcGeo tc_geo(bool rows) const {
    const int64_t n_own = rows ? n : m, n_oth = rows ? m : n;
    TcGeo g;
    g.B = (n_own + tc::kM - 1) / tc::kM;
    double best = -1.0;
    g.S = 1;
    g.chunk = (n_oth + tc::kN - 1) / tc::kN * tc::kN;
    for (int64_t S = 1; S <= 128; ++S) {
      const int64_t chunk = ((n_oth + S - 1) / S + tc::kN - 1) / tc::kN * tc::kN;
      const int64_t Sr = (n_oth + chunk - 1) / chunk;
      if (Sr != S) continue;
      if (S > 1 && chunk < 2 * tc::kN) break;
      const int64_t ctas = g.B * S, waves = (ctas + h->sms - 1) / h->sms;
      const double eff = (double)ctas / (double)(waves * h->sms) - 0.002 * (double)S;  // prefer fewer chunks
      if (eff > best) {
        best = eff;
        g.S = S;
        g.chunk = chunk;
      }
    }
    return g;
  }
  template <int NR, bool LSE, int SQM, bool ROWS, class Epi>
  static void tc_attr() {
    static bool done = false;
    if (done) return;
    EOT_CUDA(cudaFuncSetAttribute(tc::tc_sweep_kernel<NR, LSE, SQM, ROWS, Epi>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::kSmemBytes));
    done = true;
  }
  void setup_tc() {
    const int64_t npX = tc::pad_rows(n), npY = tc::pad_rows(m);
    auto side_bytes = [](int64_t np) { return (size_t)np * (tc::kSlices * 64 * 2 + 3 * 4) + 1024; };
    const size_t need = side_bytes(npX) + side_bytes(npY);
    if (need > h->tc_bytes) {
      EOT_CUDA(cudaStreamSynchronize(st));
      if (h->tc_mem) cudaFree(h->tc_mem);
      h->tc_mem = nullptr;
      h->tc_bytes = 0;
      EOT_CUDA(cudaMalloc(&h->tc_mem, need));
      h->tc_bytes = need;
    }
    unsigned char* b = (unsigned char*)h->tc_mem;
    auto carve = [&](tc::Side& sd, int64_t np, const float* P, int64_t len) {
      __nv_bfloat16* sl = (__nv_bfloat16*)b;
      b += (size_t)np * tc::kSlices * 64 * 2;
      float* sc = (float*)b;
      b += (size_t)np * 4;
      float* nxh = (float*)b;
      b += (size_t)np * 4;
      float* nxl = (float*)b;
      b += (size_t)np * 4;
      b = (unsigned char*)(((uintptr_t)b + 255) & ~(uintptr_t)255);
      sd = tc::Side{sl, sc, nxh, nxl, np};
      const int64_t threads = np * 32;
      launch_k(tc::tc_prep_kernel, dim3((unsigned)((threads + kThreads - 1) / kThreads)), dim3(kThreads), st, P,
               len, d, np, X /* the first point of X is the common centre */, sl, sc, nxh, nxl);
      EOT_LAUNCH_CHECK();
      h->launches++;
    };
    carve(targs.X, npX, X, n);
    carve(targs.Y, npY, Y, m);
    targs.err = h->status;
    for (bool rows : {true, false}) {
      const TcGeo g = tc_geo(rows);
      ensure_rowpart_elems(h, kPtsMaxPartials * g.S * (rows ? n : m));
      if (g.B > h->rowblk_slots) throw EotError{EOT_ERR_INVALID_ARG, "ticket array too small"};
    }
    // shared-memory opt-in for every instantiation, before any graph capture
    tc_attr<1, true, 0, true, RowLseEpi>();
    tc_attr<1, true, 0, false, ColLseEpi>();
    tc_attr<2, false, 0, false, SetupColEpi<float>>();
    tc_attr<3, false, 2, true, SetupRowEpi>();
    tc_attr<1, false, 0, false, CgColEpi<float>>();
    tc_attr<1, false, 0, true, CgRowEpi>();
    tc_attr<1, false, 0, false, DvColEpi>();
    tc_attr<2, false, 0, true, RowSumEpi>();
    tc_attr<2, false, 0, false, ColSumEpi>();
    tc_on = true;
  }
  template <int NR, bool LSE, int SQM, bool ROWS, class Epi>
  void launch_tc(cudaStream_t s, SweepArgs<T> a, const Epi& e) {
    const TcGeo g = tc_geo(ROWS);
    a.chunk = g.chunk;
    constexpr int NP = LSE ? 2 : NR;
    static_assert(NP <= kPtsMaxPartials, "point partial buffer sized for kPtsMaxPartials");
    if ((int64_t)NP * g.S * (ROWS ? n : m) > h->cap_rowpart || g.B > h->rowblk_slots)
      throw EotError{EOT_ERR_INVALID_ARG, "tensor-core sweep scratch smaller than the launch needs"};
    tc_attr<NR, LSE, SQM, ROWS, Epi>();
    launch_kd(tc::tc_sweep_kernel<NR, LSE, SQM, ROWS, Epi>, dim3((unsigned)g.B, (unsigned)g.S),
              dim3(tc::kTcThreads), (size_t)tc::kSmemBytes, s, a, targs, e);
  }

  // s_C = 1 / max_ij |x_i - y_j|^2 (cost normalised to max 1, Sec. 4.1): FP32 scan,
  // FP64 re-evaluation of each thread's arg-max pair, maximum on the host.
  double max_cost_scale() {
    const int64_t B = (n + kThreads - 1) / kThreads;
    int64_t S = std::max<int64_t>(1, (2 * (int64_t)h->sms + B - 1) / B);
    S = std::min<int64_t>(S, (m + 255) / 256);
    const int64_t chunk = (m + S - 1) / S;
    S = (m + chunk - 1) / chunk;
    if (B * S > h->maxbuf_len) throw EotError{EOT_ERR_INVALID_ARG, "cost-max buffer too small"};
    const dim3 grid((unsigned)B, (unsigned)S);
    if (d <= 4) launch_k(pts_maxdist_kernel<4>, grid, dim3(kThreads), st, X, Y, n, m, d, chunk, h->maxbuf);
    else if (d <= 16) launch_k(pts_maxdist_kernel<16>, grid, dim3(kThreads), st, X, Y, n, m, d, chunk, h->maxbuf);
    else launch_k(pts_maxdist_kernel<64>, grid, dim3(kThreads), st, X, Y, n, m, d, chunk, h->maxbuf);
    h->launches++;
    std::vector<double> v((size_t)(B * S));
    EOT_CUDA(cudaMemcpyAsync(v.data(), h->maxbuf, v.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    EOT_CUDA(cudaStreamSynchronize(st));
    double mx = 0.0;
    for (double x : v) mx = std::max(mx, x);
    if (!(mx > 0.0) || !std::isfinite(mx))
      throw EotError{EOT_ERR_INVALID_ARG, "point costs: all points coincide or are not finite"};
    return 1.0 / mx;
  }

  // Keep the cost resident in L2 across the sweeps of one call when it fits in
  // 60% of L2 (evict-last loads); release() demotes it again.
  bool keep_l2 = false;
  void retain_cost() {
    keep_l2 = !points && (double)n * (double)ldc * sizeof(T) <= 0.6 * (double)h->l2_bytes;
  }
  void release_cost() {
    if (!keep_l2) return;
    const int64_t bytes = n * ldc * (int64_t)sizeof(T);
    launch_k(l2_demote_kernel, dim3(4 * h->sms), dim3(kThreads), st, (const char*)C, bytes);
    h->launches++;
    keep_l2 = false;
  }

  T* Ah() { return (T*)h->Ah; }
  T* Bh() { return (T*)h->Bh; }
  T* xw0() { return (T*)h->xw0; }
  T* xw1() { return (T*)h->xw1; }
  T* zf() { return (T*)h->zf; }
  T* wsq() { return (T*)h->wsq; }
  T* ewr() { return (T*)h->ewr; }
  T* ewc() { return (T*)h->ewc; }

  SweepArgs<T> args() const {
    SweepArgs<T> a{};
    a.C = C;
    a.n = n;
    a.m = m;
    a.ldc = ldc;
    a.Ah = (const T*)h->Ah;
    a.Bh = (const T*)h->Bh;
    a.gamma = T(0);
    a.colpart = h->colpart;
    a.rowpart = h->rowpart;
    a.cnt_strip = h->cnt_strip;
    a.cnt_rowblk = h->cnt_rowblk;
    a.dotpart = h->dotpart;
    a.cnt_dot = h->cnt_dot;
    a.rows_per_block = geo.BR;
    a.nrowblk = geo.R;
    a.gamma_dev = h->sc + SC_GAMMA;
    a.active = nullptr;
    a.keep_l2 = keep_l2 ? 1 : 0;
    a.X = X;
    a.Y = Y;
    a.d = d;
    a.sC = sC;
    a.chunk = 0;
    a.err = h->status;
    return a;
  }

  double gamma_host = 0.0;
  void set_scalar(int slot, double v) {
    if (slot == SC_GAMMA) gamma_host = v;
    launch_k(set_scalar_kernel, dim3(1), dim3(1), st, h->sc, slot, v);
    EOT_LAUNCH_CHECK();
    h->launches++;
  }

  std::string ctx;  // where the solver is, for error messages
  const bool trace = std::getenv("EOT_TRACE") != nullptr;

  // Read every device scalar and the status word (synchronises the stream).
  // Lost CG curvature (kStatCurv) is handled by the caller, not thrown.
  // Status bits in `tolerated` are left for the caller to inspect (status_bits()).
  const double* read(int tolerated = 0) {
    EOT_CUDA(cudaMemcpyAsync(h->h_sc, h->sc, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, st));
    EOT_CUDA(cudaMemcpyAsync(h->h_status, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    EOT_CUDA(cudaStreamSynchronize(st));
    const int s = *h->h_status & ~tolerated;
    if (s & kStatNonfinite) throw EotError{EOT_ERR_NONFINITE, "non-finite potential or marginal" + ctx};
    if (s & kStatCgNan) throw EotError{EOT_ERR_NONFINITE, "non-finite CG residual" + ctx};
    if (s & kStatRange) throw EotError{EOT_ERR_RANGE, "|potential| >= 2^19 (mixed-precision split)" + ctx};
    if (s & kStatTimeout) throw EotError{EOT_ERR_CUDA, "a bounded device wait ran out" + ctx};
    return h->h_sc;
  }
  int status_bits() const { return *h->h_status; }
  void clear_status() { EOT_CUDA(cudaMemsetAsync(h->status, 0, sizeof(int), st)); }

  // ---------------- O(n) helpers ----------------
  void split_rows(const double* x, const double* y, double alpha, const double* z, double* l,
                  T* ew, double* fac, const double* fshift) {
    launch_k(split_kernel<T>, dim3(vg_n), dim3(kThreads), st, n, x, y, alpha, z, plain ? 1 : 0, Ah(), l, ew, fac,
                                               fshift, h->status);
    EOT_LAUNCH_CHECK();
    h->launches++;
  }
  void split_cols(const double* x, const double* y, double alpha, const double* z, double* l,
                  T* ew, double* fac, const double* fshift) {
    launch_k(split_kernel<T>, dim3(vg_m), dim3(kThreads), st, m, x, y, alpha, z, plain ? 1 : 0, Bh(), l, ew, fac,
                                               fshift, h->status);
    EOT_LAUNCH_CHECK();
    h->launches++;
  }
  void axpy(int64_t len, double* y, double b, const double* x, double a, const double* z = nullptr,
            double c = 0.0, const double* w = nullptr, double d = 0.0) {
    launch_k(axpy4_kernel, dim3(vec_grid(len)), dim3(kThreads), st, len, y, b, x, a, z, c, w, d);
    EOT_LAUNCH_CHECK();
    h->launches++;
  }
  void copy(double* dst, const double* src, int64_t len) {
    EOT_CUDA(cudaMemcpyAsync(dst, src, len * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }

  // ---------------- sweep launchers ----------------
  // point sweep: own side = rows (ROWS) or columns, dispatched on d
  template <int NR, bool LSE, int SQM, bool ROWS, class Epi>
  void launch_pts(cudaStream_t s, SweepArgs<T> a, const Epi& e) {
    if constexpr (sizeof(T) == 4) {
      if (tc_on) {
        launch_tc<NR, LSE, SQM, ROWS>(s, a, e);
        return;
      }
    }
    const PtsGeo g = pts_geo(ROWS);
    a.chunk = g.chunk;
    const dim3 grid((unsigned)g.B, (unsigned)g.S);
    constexpr int NP = LSE ? 2 : NR;  // FP64 partials per owned element and chunk
    static_assert(NP <= kPtsMaxPartials, "point partial buffer sized for kPtsMaxPartials");
    if ((int64_t)NP * g.S * (ROWS ? n : m) > h->cap_rowpart || g.B > h->rowblk_slots)
      throw EotError{EOT_ERR_INVALID_ARG, "point sweep scratch smaller than the launch needs"};
    // the FP32 mixed path forms D compensated; plain FP32 and FP64 use the
    // direct sum of squares
    constexpr bool F32 = sizeof(T) == 4;
    const bool precise = F32 && !plain;
    if (d <= 4) {
      if (precise) launch_k(pts_sweep_kernel<T, 4, 4, NR, LSE, SQM, ROWS, F32, Epi>, grid, dim3(kThreads), s, a, e);
      else launch_k(pts_sweep_kernel<T, 4, 4, NR, LSE, SQM, ROWS, false, Epi>, grid, dim3(kThreads), s, a, e);
    } else if (d <= 16) {
      if (precise) launch_k(pts_sweep_kernel<T, 16, 2, NR, LSE, SQM, ROWS, F32, Epi>, grid, dim3(kThreads), s, a, e);
      else launch_k(pts_sweep_kernel<T, 16, 2, NR, LSE, SQM, ROWS, false, Epi>, grid, dim3(kThreads), s, a, e);
    } else {
      if (precise) launch_k(pts_sweep_kernel<T, 64, 1, NR, LSE, SQM, ROWS, F32, Epi>, grid, dim3(kThreads), s, a, e);
      else launch_k(pts_sweep_kernel<T, 64, 1, NR, LSE, SQM, ROWS, false, Epi>, grid, dim3(kThreads), s, a, e);
    }
  }
  template <int NR, bool LSE, int SQM, class Epi>
  void launch_row(cudaStream_t s, const SweepArgs<T>& a, const Epi& e) {
    if (points) launch_pts<NR, LSE, SQM, true>(s, a, e);
    else if (launch_row_bulk<NR, LSE, SQM>(s, a, e)) return;
    else if (V == VEC) launch_k(row_sweep_kernel<T, VEC, NR, LSE, SQM, Epi>, dim3(rg), dim3(kThreads), s, a, e);
    else launch_k(row_sweep_kernel<T, 1, NR, LSE, SQM, Epi>, dim3(rg), dim3(kThreads), s, a, e);
  }
  template <int NC, bool LSE, int NR, class Epi>
  void launch_col(cudaStream_t s, const SweepArgs<T>& a, const Epi& e) {
    if (points) {
      if constexpr (NR == 0) launch_pts<NC, LSE, 0, false>(s, a, e);
      else throw EotError{EOT_ERR_UNSUPPORTED, "fused two-sided sweep needs a dense cost"};
      return;
    }
    if constexpr (NR == 0) {
      if (launch_col_bulk<NC, LSE>(s, a, e)) return;
    }
    const dim3 grid((unsigned)geo.S, (unsigned)geo.R);
    if (V == VEC) launch_k(col_sweep_kernel<T, VEC, NC, LSE, NR, Epi>, grid, dim3(kThreads), s, a, e);
    else launch_k(col_sweep_kernel<T, 1, NC, LSE, NR, Epi>, grid, dim3(kThreads), s, a, e);
  }
  template <int NR, bool LSE, int SQM, class Epi>
  void row(const SweepArgs<T>& a, const Epi& e) {
    launch_row<NR, LSE, SQM>(st, a, e);
    EOT_LAUNCH_CHECK();
    h->launches++;
    (*sweep_bucket)++;
  }
  template <int NC, bool LSE, int NR, class Epi>
  void col(const SweepArgs<T>& a, const Epi& e) {
    launch_col<NC, LSE, NR>(st, a, e);
    EOT_LAUNCH_CHECK();
    h->launches++;
    (*sweep_bucket)++;
  }

  // log r(P) and the running row max at (u, v): A = u - rshift, B = v.
  // With a target rt, also ||rt - r(P)||_1 -> SC_GL1 and chi^2(rt | r(P)) -> SC_CHI2.
  // Point gradients: out = scale * ownfac * sum_o P-weights (x_own - x_other),
  // components in groups of DG (one launch per group); ROWS: own = rows.
  template <bool ROWS>
  void grad_pts(double scale, const double* ownfac, float* out) {
    const int64_t n_own = ROWS ? n : m, n_oth = ROWS ? m : n;
    const int64_t B = (n_own + kThreads - 1) / kThreads;
    int64_t S = (2 * (int64_t)h->sms + B - 1) / B;
    S = std::max<int64_t>(1, std::min<int64_t>(S, (n_oth + 31) / 32));
    const int64_t chunk = ((n_oth + S - 1) / S + 31) / 32 * 32;
    S = (n_oth + chunk - 1) / chunk;
    const int DG = d <= 4 ? 4 : 16;
    ensure_rowpart_elems(h, (int64_t)DG * S * n_own);
    if (B > h->rowblk_slots) throw EotError{EOT_ERR_INVALID_ARG, "ticket array too small"};
    SweepArgs<T> a = args();
    a.rowpart = h->rowpart;
    a.chunk = chunk;
    a.wc[0] = ewc();
    a.wr[0] = ewr();
    const dim3 grid((unsigned)B, (unsigned)S);
    constexpr bool F32 = sizeof(T) == 4;
    const bool precise = F32 && !plain;
    for (int k0 = 0; k0 < d; k0 += DG) {
      if (d <= 4) {
        if (precise) launch_k(pts_grad_kernel<T, 4, 4, ROWS, F32>, grid, dim3(kThreads), st, a, k0, scale, ownfac, out);
        else launch_k(pts_grad_kernel<T, 4, 4, ROWS, false>, grid, dim3(kThreads), st, a, k0, scale, ownfac, out);
      } else if (d <= 16) {
        if (precise) launch_k(pts_grad_kernel<T, 16, 16, ROWS, F32>, grid, dim3(kThreads), st, a, k0, scale, ownfac, out);
        else launch_k(pts_grad_kernel<T, 16, 16, ROWS, false>, grid, dim3(kThreads), st, a, k0, scale, ownfac, out);
      } else {
        if (precise) launch_k(pts_grad_kernel<T, 64, 16, ROWS, F32>, grid, dim3(kThreads), st, a, k0, scale, ownfac, out);
        else launch_k(pts_grad_kernel<T, 64, 16, ROWS, false>, grid, dim3(kThreads), st, a, k0, scale, ownfac, out);
      }
      EOT_LAUNCH_CHECK();
      h->launches++;
    }
  }

  void row_lse(const double* u, const double* v, const double* rshift, double* out_lse,
               double* out_max, const double* rt, int s0 = SC_GL1, int s1 = SC_CHI2) {
    split_rows(u, nullptr, 0.0, rshift, h->Al, nullptr, nullptr, nullptr);
    split_cols(v, nullptr, 0.0, nullptr, h->Bl, ewc(), nullptr, nullptr);
    SweepArgs<T> a = args();
    a.wc[0] = ewc();
    RowLseEpi e{rshift, h->Al, out_lse, out_max, rt, h->sc, s0, s1};
    row<1, true, 0>(a, e);
  }

  // Column LSE at (u + alpha du, v + alpha dv): B = v + alpha dv - cshift.
  // mode 0: out = cshift + LSE (log c(P)); mode 1: out -= LSE (column fix).
  void col_lse(const double* u, const double* du, const double* v, const double* dv, double alpha,
               const double* cshift, double* out, int mode, int slot, double minus) {
    split_rows(u, du, alpha, nullptr, h->Al, ewr(), nullptr, nullptr);
    split_cols(v, dv, alpha, cshift, h->Bl, nullptr, nullptr, nullptr);
    SweepArgs<T> a = args();
    a.wr[0] = ewr();
    ColLseEpi e{h->Bl, mode == 0 ? cshift : nullptr, out, mode, h->sc, slot, minus};
    col<1, true, 0>(a, e);
  }

  // ---------------- Alg. 2: NewtonSolve ----------------
  // At (u, v) with log r(P) and the row maxima from the last row LSE. Targets r~.
  // Leaves d_u in h->du and d_v = -P_c d_u in h->dv; returns the rho of the last CG
  // solve (or rho0 when no CG solve ran). Also leaves r(P), c(P) in h->rP, h->cP.
  double newton(const double* u, const double* v, const double* rt, double gl1, double eta,
                double rho0, int max_cg, CgMode mode, bool* ran_cg) {
    int64_t* saved = sweep_bucket;
    sweep_bucket = &cnt.sweeps_newton;
    // factorisation P = rowfac * colfac * E with row shift = running row max
    split_rows(u, nullptr, 0.0, h->rowmax, h->Al, nullptr, h->rowfac, h->rowmax);
    split_cols(v, nullptr, 0.0, nullptr, h->Bl, ewc(), h->colfac, nullptr);
    launch_k(prep_setup_kernel<T>, dim3(vg_n), dim3(kThreads), st, n, h->logrP, rt, h->rowfac, h->rP, h->du0,
                                                    xw0(), xw1());
    EOT_LAUNCH_CHECK();
    h->launches++;
    {
      SweepArgs<T> a = args();
      a.wr[0] = xw0();
      a.wr[1] = xw1();
      SetupColEpi<T> e{h->colfac, h->cP, zf(), wsq()};
      col<2, false, 0>(a, e);
    }
    {
      SweepArgs<T> a = args();
      a.wc[0] = zf();
      a.wc[1] = wsq();
      a.wc[2] = ewc();
      SetupRowEpi e{h->rowfac, h->rP, h->du0, h->y0, h->diag, h->rPs, h->sc};
      row<3, false, 2>(a, e);
    }
    const double check0 = read()[SC_CHECK];
    double rho = rho0, rho_last = rho0;
    *ran_cg = false;
    const double* du_final = h->du0;
    if (!(check0 <= eta * gl1)) {
      const double tol = 0.25 * eta * gl1;
      set_scalar(SC_TOL, tol);
      set_scalar(SC_MAXIT, (double)max_cg);
      for (int solve = 0;; ++solve) {
        set_scalar(SC_RHO, rho);
        run_cg(mode, max_cg, rt);
        launch_k(cg_check_kernel, dim3(vg_n), dim3(kThreads), st, n, h->res, h->Yx, h->sc, h->dotpart, h->cnt_dot);
        EOT_LAUNCH_CHECK();
        h->launches++;
        const double* s = read();
        const double it = s[SC_ITERS], rl1 = s[SC_RESL1], chk = s[SC_CHK];
        if (mode == CgMode::kWhile && pcg_geo().G == 0) {
          // passes of the WHILE body: the one whose update kernel stopped CG is the last
          const int64_t passes = std::max<int64_t>(1, ((int64_t)it + kWhileBody - 1) / kWhileBody);
          h->launches += 4 * kWhileBody * passes;
        }
        cnt.cg_iters += (int64_t)it;
        cnt.sweeps_cg += 2 * (int64_t)it + ((status_bits() & kStatCurv) ? 2 : 0);
        cnt.cg_solves++;
        *ran_cg = true;
        rho_last = rho;
        if (status_bits() & kStatCurv) {
          // <p, F_r(rho) p> <= 0 in finite precision: stop CG and keep the iterate,
          // the truncated-Newton convention; no larger rho can help, so return.
          cnt.curvature_stops++;
          clear_status();
          du_final = it > 0 ? h->x : h->du0;
          break;
        }
        if (rl1 > tol) throw EotError{EOT_ERR_CG_MAXITER, "linear CG reached max_cg" + ctx};
        du_final = h->x;
        if (chk <= eta * gl1) break;
        rho = 1.0 - (1.0 - rho) / 4.0;
        if (solve > 60) throw EotError{EOT_ERR_CG_MAXITER, "rho annealing did not meet the forcing test" + ctx};
      }
    }
    if (du_final != h->du) copy(h->du, du_final, n);
    // d_u modulo the gauge, d_v = -(P^T d_u) / c(P) and the Armijo slope <r~ - r(P), d_u>
    launch_k(gauge_kernel, dim3(vg_n), dim3(kThreads), st, n, (const double*)h->du, (const double*)h->rP,
             h->sc, h->dotpart, h->cnt_dot);
    EOT_LAUNCH_CHECK();
    h->launches++;
    launch_k(prep_dv_kernel<T>, dim3(vg_n), dim3(kThreads), st, n, h->du, h->rowfac, rt, h->rP, xw0(), h->sc,
                                                 h->dotpart, h->cnt_dot);
    EOT_LAUNCH_CHECK();
    h->launches++;
    {
      SweepArgs<T> a = args();
      a.wr[0] = xw0();
      DvColEpi e{h->colfac, h->cP, h->dv};
      col<1, false, 0>(a, e);
    }
    sweep_bucket = saved;
    return rho_last;
  }

  // One CG iteration's four kernels (column half, row half, update, p update).
  void cg_iteration(cudaStream_t s, cudaGraphConditionalHandle cond) {
    {
      SweepArgs<T> a = args();
      a.wr[0] = xw0();
      a.active = h->sc + SC_ACTIVE;
      CgColEpi<T> e{h->colfac, h->cP, zf()};
      launch_col<1, false, 0>(s, a, e);
    }
    {
      SweepArgs<T> a = args();
      a.wc[0] = zf();
      a.active = h->sc + SC_ACTIVE;
      CgRowEpi e{h->rowfac, h->rPs, h->p, h->y, h->q, h->sc, h->status};
      launch_row<1, false, 0>(s, a, e);
    }
    launch_k(cg_update_kernel<T>, dim3(vg_n), dim3(kThreads), s, n, h->p, h->q, h->y, h->M, h->x, h->res, h->Yx,
                                                  h->z, h->sc, h->dotpart, h->cnt_dot, h->status,
                                                  cond);
    launch_k(cg_pupdate_kernel<T>, dim3(vg_n), dim3(kThreads), s, n, h->z, h->rowfac, h->p, xw0(), h->sc);
  }

  CgGraph& get_graph(CgMode mode) {
    const int B = mode == CgMode::kWhile ? kWhileBody : 6;  // CG iterations per launch / per pass
    const CgKey key{(int)sizeof(T) + (points ? 100 * d : 0) + (bulk_rows ? 1000 : 0) + (bulk_cols ? 2000 : 0), V,
                    mode == CgMode::kWhile ? B : 0, n, m,
                    ldc, points ? (uintptr_t)X ^ ((uintptr_t)Y << 1) : (uintptr_t)C};
    auto it = h->graphs.find(key);
    if (it != h->graphs.end()) return it->second;
    if (h->graphs.size() >= 32) free_graphs(h);
    CgGraph g;
    if (!h->cap_stream) EOT_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    if (mode == CgMode::kWhile) {
      EOT_CUDA(cudaGraphCreate(&g.graph, 0));
      cudaGraphConditionalHandle cond;
      EOT_CUDA(cudaGraphConditionalHandleCreate(&cond, g.graph, 1, cudaGraphCondAssignDefault));
      cudaGraphNodeParams np{};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = cond;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      EOT_CUDA(cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &np));
      cudaGraph_t body = np.conditional.phGraph_out[0];
      EOT_CUDA(cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed));
      // B iterations per pass: the condition is re-evaluated every B iterations;
      // iterations past the stop are no-ops (device stop flag)
      for (int b = 0; b < B; ++b) cg_iteration(h->cap_stream, cond);
      cudaGraph_t out;
      EOT_CUDA(cudaStreamEndCapture(h->cap_stream, &out));
    } else {
      EOT_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
      for (int b = 0; b < B; ++b) cg_iteration(h->cap_stream, 0);
      EOT_CUDA(cudaStreamEndCapture(h->cap_stream, &g.graph));
    }
    EOT_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
    g.iters_per_launch = B;
    return h->graphs.emplace(key, g).first->second;
  }

  // ---- the persistent CG kernel (dense FP32 cost, mixed path) ----
  // Opt-in (EOT_CG_PERSIST=1): on the 64 x 64 grid workload its four grid
  // barriers per iteration at two CTAs per SM cost more (57 us per CG iteration)
  // than the kernel boundaries of the graph path (29 us), so it is not the default.
  static bool persist_env() {
    const char* e = std::getenv("EOT_CG_PERSIST");
    return e && e[0] == '1';
  }
  struct PcgGeo {
    int S = 0, R = 0, rpb = 0, G = 0;
  };
  PcgGeo pcg_geo() const {
    PcgGeo g;
    if constexpr (sizeof(T) != 4) return g;
    if (points || plain || V != 4 || m > pcg::kTWp || !persist_env()) return g;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pcg::cg_persistent_kernel, kThreads, 0) != cudaSuccess)
      return g;
    const int gmax = nb * h->sms;
    const int S = (int)((m + pcg::kSW - 1) / pcg::kSW);
    if (S > gmax) return g;
    int R = (int)std::min<int64_t>(gmax / S, (n + kWarps - 1) / kWarps);
    R = std::max(R, 1);
    const int rpb = (int)((n + R - 1) / R);
    R = (int)((n + rpb - 1) / rpb);
    if ((int64_t)R * m > 2 * h->max_rowblk * h->cap_m) return g;  // FP32-pair partials in colpart
    g.S = S;
    g.R = R;
    g.rpb = rpb;
    g.G = R * S;
    return g;
  }
  void run_cg_persistent(const PcgGeo& geo) {
    const size_t need = (size_t)4 * geo.G * sizeof(double) + 256;
    if (need > h->pcg_bytes) {
      EOT_CUDA(cudaStreamSynchronize(st));
      if (h->pcg_mem) cudaFree(h->pcg_mem);
      h->pcg_mem = nullptr;
      h->pcg_bytes = 0;
      EOT_CUDA(cudaMalloc(&h->pcg_mem, need));
      h->pcg_bytes = need;
    }
    unsigned char* b = (unsigned char*)h->pcg_mem;
    pcg::Args a{};
    a.C = (const float*)C;
    a.n = n;
    a.m = m;
    a.ldc = ldc;
    a.Ah = (const float*)h->Ah;
    a.Bh = (const float*)h->Bh;
    a.rowfac = h->rowfac;
    a.colfac = h->colfac;
    a.cP = h->cP;
    a.rPs = h->rPs;
    a.M = h->M;
    a.x = h->x;
    a.res = h->res;
    a.z = h->z;
    a.q = h->q;
    a.y = h->y;
    a.Yx = h->Yx;
    a.pbuf[0] = h->p;
    a.pbuf[1] = h->p2;
    a.xw = (float*)h->xw0;
    a.zf = (float*)h->zf;
    a.colpart = reinterpret_cast<float2*>(h->colpart);
    a.dots = (double*)(b + 256);
    a.sc = h->sc;
    a.bar = (unsigned*)b;
    a.abort = (int*)(b + 64);
    a.status = h->status;
    a.R = geo.R;
    a.S = geo.S;
    a.rows_per_block = geo.rpb;
    a.keep_l2 = keep_l2 ? 1 : 0;
    EOT_CUDA(cudaMemsetAsync(b, 0, 256, st));
    void* args[] = {&a};
    EOT_CUDA(cudaLaunchCooperativeKernel((const void*)pcg::cg_persistent_kernel, dim3(geo.G), dim3(kThreads), args,
                                         0, st));
    h->launches++;
  }

  // Runs PCG from x = 0 on F_r(rho) until the device stop flag clears.
  void run_cg(CgMode mode, int max_cg, const double* rt) {
    launch_k(cg_init_kernel<T>, dim3(vg_n), dim3(kThreads), st, n, h->rP, h->rPs, rt, h->diag, h->rowfac, h->M, h->x,
                                                 h->res, h->z, h->p, h->Yx, xw0(), h->sc,
                                                 h->dotpart, h->cnt_dot);
    EOT_LAUNCH_CHECK();
    h->launches++;
    {
      const PcgGeo geo = pcg_geo();
      if (geo.G > 0) {
        run_cg_persistent(geo);
        return;
      }
    }
    if (mode == CgMode::kHost) {
      for (int it = 0; it < max_cg; it += 4) {
        for (int b = 0; b < 4; ++b) cg_iteration(st, 0);
        EOT_LAUNCH_CHECK();
        h->launches += 16;
        if (read()[SC_ACTIVE] == 0.0) break;
      }
      return;
    }
    CgGraph& g = get_graph(mode);
    if (mode == CgMode::kWhile) {
      EOT_CUDA(cudaGraphLaunch(g.exec, st));  // its kernels are counted once the iterations are known
      return;
    }
    const int maxl = (max_cg + g.iters_per_launch - 1) / g.iters_per_launch + 1;
    for (int l = 0; l < maxl; ++l) {
      EOT_CUDA(cudaGraphLaunch(g.exec, st));
      h->launches += 4 * g.iters_per_launch;
      if (read()[SC_ACTIVE] == 0.0) break;
    }
  }

  // ---------------- MDOT-Sinkhorn projection (Sec. 4 comparison) ----------------
  // Column fix, then row and column fixes while ||r~ - r(P)||_1 > eps, then the
  // closing row step of Alg. 4. The host reads the gradient norm every kSkCheck
  // iterations; sk_step_kernel makes the iterations past the stopping point
  // no-ops, so the result and the count are those of a per-iteration test.
  static constexpr int kSkCheck = 8;
  bool project_sinkhorn(double* u, double* v, double eps, const eot_params& prm, double* gl1_out) {
    double* rt = h->rt;
    double* logrt = h->logrt;
    double* logct = h->logct;
    sweep_bucket = &cnt.sweeps_stage;
    col_lse(u, nullptr, v, nullptr, 0.0, logct, v, 1, SC_AUX0, 0.0);
    row_lse(u, v, logrt, h->logrP, h->rowmax, rt);
    sweep_bucket = &cnt.sweeps_sk;
    set_scalar(SC_AUX1, 0.0);
    const int64_t max_it = prm.max_sinkhorn > 0 ? prm.max_sinkhorn : 1000000;
    double gl1 = read()[SC_GL1];
    int64_t it = 0;
    bool ok = true;
    while (gl1 > eps) {
      if (it >= max_it) {
        ok = false;
        break;
      }
      const int64_t k = std::min<int64_t>(kSkCheck, max_it - it);
      for (int64_t j = 0; j < k; ++j) {
        launch_k(sk_step_kernel, dim3(vg_n), dim3(kThreads), st, n, u, (const double*)logrt,
                 (const double*)h->logrP, h->sc, eps);
        EOT_LAUNCH_CHECK();
        h->launches++;
        col_lse(u, nullptr, v, nullptr, 0.0, logct, v, 1, SC_AUX0, 0.0);
        row_lse(u, v, logrt, h->logrP, h->rowmax, rt);
      }
      const double* s = read();
      gl1 = s[SC_GL1];
      it = (int64_t)s[SC_AUX1];
    }
    cnt.sk_iters += it;
    if (trace)
      std::fprintf(stderr, "[eot] sinkhorn stage gamma %.6g iters %lld grad %.4e eps %.4e\n", gamma_host,
                   (long long)it, gl1, eps);
    axpy(n, u, 1.0, logrt, 1.0, h->logrP, -1.0);
    *gl1_out = gl1;
    return ok;
  }

  // ---------------- Alg. 4: TruncatedNewtonProject ----------------
  // (u, v) in/out; targets (rt, ct) = smoothed marginals with logs; tolerance eps.
  // Returns false if the Newton budget ran out. delta_min is reported.
  bool project(double* u, double* v, double eps, const eot_params& prm, int max_cg, CgMode mode,
               double* delta_min, double* gl1_out) {
    double* rt = h->rt;
    double* logrt = h->logrt;
    double* logct = h->logct;
    sweep_bucket = &cnt.sweeps_stage;
    // opening column fix: v <- log c~ - LSE_c(u 1^T - gamma C)
    col_lse(u, nullptr, v, nullptr, 0.0, logct, v, 1, SC_AUX0, 0.0);
    // then log r(P) <- u + LSE_r(1 v^T - gamma C)
    row_lse(u, v, logrt, h->logrP, h->rowmax, rt);
    const double* s = read();
    double gl1 = s[SC_GL1], chi2 = s[SC_CHI2];
    if (trace) std::fprintf(stderr, "[eot] stage start gamma %.6g grad %.4e chi2 %.4e eps %.4e\n", gamma_host, gl1, chi2, eps);
    *delta_min = INFINITY;
    int steps = 0;
    bool ok = true;
    const double eps_chi = std::pow(eps, 0.4);
    while (gl1 > eps) {
      ctx = " (gamma " + std::to_string(gamma_host) + ", Newton step " + std::to_string(steps) +
            ", ||grad g||_1 " + std::to_string(gl1) + ", eps " + std::to_string(eps) + ")";
      if (steps >= prm.max_newton) {
        ok = false;
        break;
      }
      // Alg. 3 (ChiSinkhorn): while chi^2(r~ | r(P)) > eps^(2/5)
      sweep_bucket = &cnt.sweeps_sk;
      int sk = 0;
      while (chi2 > eps_chi) {
        axpy(n, u, 1.0, logrt, 1.0, h->logrP, -1.0);  // u <- u + log r~ - log r(P)
        col_lse(u, nullptr, v, nullptr, 0.0, logct, v, 1, SC_AUX0, 0.0);
        row_lse(u, v, logrt, h->logrP, h->rowmax, rt);
        s = read();
        gl1 = s[SC_GL1];
        chi2 = s[SC_CHI2];
        cnt.sk_iters++;
        if (++sk > 2000) throw EotError{EOT_ERR_MAXNEWTON, "ChiSinkhorn did not converge"};
      }
      if (gl1 <= eps) break;
      // forcing parameter
      const double eta = std::fmax(gl1, 0.8 * eps / gl1);
      // NewtonSolve and d_v = -P_c d_u
      bool ran;
      const double rho0 = std::fmax(0.0, 1.0 - 4.0 * (1.0 - cnt.rho_last));
      const double rho = newton(u, v, rt, gl1, eta, rho0, max_cg, mode, &ran);
      if (ran) cnt.rho_last = rho;
      cnt.newton_steps++;
      // backtracking on the simplified Armijo test, whose left side
      // (sum P(alpha) - 1) is taken relative to its computed value at alpha = 0
      // (0 in exact arithmetic, since c(P) = c~): this removes the rounding
      // offset of the mass, which near the final tolerance can exceed the
      // sufficient decrease itself
      sweep_bucket = &cnt.sweeps_ls;
      // With FP32 plan entries sum P(alpha) carries a rounding floor (about
      // 2^-22 / sqrt(max(n, m))); when the whole decrease the test asks for at
      // alpha = 1 is below it
      // the test cannot decide, and the unit step (accepted near the solution,
      // Sec. 3) is taken. Trials outside the split range are still rejected.
      const bool decidable = sizeof(T) == 8 || 0.99 * read()[SC_SLOPE] >= armijo_floor32(n, m);
      double lhs0 = 0.0;
      if (decidable) {
        col_lse(u, h->du, v, h->dv, 0.0, logct, h->logcP, 0, SC_LHS, 1.0);
        lhs0 = read()[SC_LHS];
      }
      double alpha = 1.0;
      int trials = 0;
      for (;;) {
        col_lse(u, h->du, v, h->dv, alpha, logct, h->logcP, 0, SC_LHS, 1.0);
        // A trial point outside the split range (|u + a d_u| >= 2^19) has a plan
        // whose mass overflows, so it fails the Armijo test: reject it.
        s = read(kStatRange);
        const bool out_of_range = (status_bits() & kStatRange) != 0;
        if (out_of_range) clear_status();
        cnt.ls_trials++;
        if (trace)
          std::fprintf(stderr, "[eot]   trial alpha %.4g lhs %.6e lhs0 %.6e slope %.6e range %d\n", alpha,
                       s[SC_LHS], lhs0, s[SC_SLOPE], out_of_range ? 1 : 0);
        if (!out_of_range && (!decidable || s[SC_LHS] - lhs0 <= 0.99 * alpha * s[SC_SLOPE])) break;
        if (++trials > prm.max_ls) throw EotError{EOT_ERR_LINESEARCH, "Armijo backtracking exhausted"};
        alpha *= 0.5;
      }
      // update and column fix: u += a d_u; v += a d_v + log c~ - log c(P(a))
      axpy(n, u, 1.0, h->du, alpha);
      axpy(m, v, 1.0, h->dv, alpha, logct, 1.0, h->logcP, -1.0);
      // log r(P) at the new point
      sweep_bucket = &cnt.sweeps_ls;
      row_lse(u, v, logrt, h->logrP, h->rowmax, rt);
      s = read();
      const double new_gl1 = s[SC_GL1];
      chi2 = s[SC_CHI2];
      const double delta = (gl1 - new_gl1) / ((1.0 - eta) * gl1);
      if (trace)
        std::fprintf(stderr, "[eot] gamma %.6g step %d grad %.3e -> %.3e eta %.3e alpha %.4g rho %.9f cg %lld curv %lld sk %lld decidable %d\n",
                     gamma_host, steps, gl1, new_gl1, eta, alpha, cnt.rho_last, (long long)cnt.cg_iters,
                     (long long)cnt.curvature_stops, (long long)cnt.sk_iters, decidable ? 1 : 0);
      if (delta < *delta_min) *delta_min = delta;
      gl1 = new_gl1;
      steps++;
    }
    // closing row step: u <- u + log r~ - log r(P)
    axpy(n, u, 1.0, logrt, 1.0, h->logrP, -1.0);
    *gl1_out = gl1;
    return ok;
  }
};

// ---------------- entry points (instantiated for float and double) ----------------
template <class T>
void run_marginals(eot_handle h, const eot_problem* P, const double* u, const double* v,
                   double gamma, double* r_out, double* c_out, double* lr_out, double* lc_out,
                   double* total_out, cudaStream_t st);
template <class T>
void run_hvp(eot_handle h, const eot_problem* P, const double* u, const double* v, double gamma,
             double s, const double* du, const double* dv, double* ou, double* ov, double* r_out,
             double* c_out, cudaStream_t st);
template <class T>
void run_newton(eot_handle h, const eot_problem* P, const double* u, const double* v,
                double gamma, const double* rtarget, double eta, double rho0, int max_cg,
                double* du_out, double* dv_out, double* rho_out, int* iters_out, cudaStream_t st);
template <class T>
void run_solve(eot_handle h, const eot_problem* P, const eot_params* prm, double* u, double* v,
               eot_stats* stats, cudaStream_t st);
template <class T>
double run_sweep_bench(eot_handle h, const eot_problem* P, const double* u, const double* v,
                       double gamma, int kind, int iters, void* flush, size_t flush_bytes, cudaStream_t st);
template <class T>
void run_backward_dense(eot_handle h, const eot_problem* P, const double* u, const double* v,
                        double gamma, double scale, float* dC, cudaStream_t st);
template <class T>
void run_backward_points(eot_handle h, const eot_problem* P, const double* u, const double* v,
                         double gamma, double scale, float* dX, float* dY, cudaStream_t st);
template <class T>
void run_round(eot_handle h, const eot_problem* P, const double* u, const double* v, double gamma,
               double* u_out, double* v_out, double* a_out, double* b_out, double* cost_out, double* corr_out,
               cudaStream_t st);

}  // namespace eot
