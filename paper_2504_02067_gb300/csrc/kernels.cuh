// Epilogues of the sweeps and the O(n) kernels of the solver.
//
// Factorisation used throughout (see common.cuh):
//   P_ij = rowfac_i * colfac_j * E_ij,  E_ij = exp(Ah_i + Bh_j - gamma C_ij).
// Device scalars live in one FP64 array `sc` indexed by the Sc enum, so that
// captured CUDA graphs stay valid when rho, gamma or tolerances change.
#pragma once
#include <algorithm>

#include "sweep.cuh"

namespace eot {

enum Sc : int {
  SC_RZ = 0, SC_PQ, SC_ALPHA, SC_BETA, SC_RESL1, SC_TOL, SC_RHO, SC_ITERS, SC_ACTIVE, SC_MAXIT,
  SC_CHECK, SC_GL1, SC_CHI2, SC_LHS, SC_SLOPE, SC_MASS, SC_CHK, SC_GAMMA, SC_AUX0, SC_AUX1,
  SC_GRD, SC_GMASS,  // <r(P), d_u> and sum r(P): the gauge component of d_u
  SC_RZPREV,         // <res, z> of the previous CG iteration (dense CG: beta's denominator)
  SC_CTL_BEGIN,      // the stage control's slots follow (control.cuh)
  SC_COUNT = 32,     // the slots the sweeps and O(n) kernels use (eot_marginals_noalloc keeps these)
  SC_TOTAL = 64      // with the stage control's slots (control.cuh): the handle's array
};

// ----------------------------------------------------------------------------
// epilogues of row sweeps
// ----------------------------------------------------------------------------

// LSE of a row: lse_i = shift_i + Al_i + M + log S. Dots: with a target rt,
// ||rt - exp(lse)||_1 and sum rt^2 / exp(lse) (for ||grad g||_1 and chi^2,
// Alg. 3 / Alg. 4); without a target, sum exp(lse) (total mass).
struct RowLseEpi {
  static constexpr int kDot = 2;
  const double* shift;   // nullable
  const double* Al;      // nullable
  double* out_lse;       // nullable
  double* out_max;       // nullable: shift + Al + M (running max of the row)
  const double* rt;      // nullable
  double* sc;
  int i0, i1;            // scalar slots of the two totals
  __device__ void row_lse(int64_t i, double M, double S, double* d) {
    const double off = (shift ? shift[i] : 0.0) + (Al ? Al[i] : 0.0);
    const double lse = off + M + log(S);
    if (out_lse) out_lse[i] = lse;
    if (out_max) out_max[i] = off + M;
    const double e = exp(lse);
    if (rt) {
      d[0] = fabs(rt[i] - e);
      d[1] = rt[i] * rt[i] / e;
    } else {
      d[0] = e;
      d[1] = 0.0;
    }
  }
  __device__ void finish(const double* t) {
    sc[i0] = t[0];
    sc[i1] = rt ? t[1] - 1.0 : t[1];
  }
};

// CG row half: y = P (w / c(P)), q = r(P) * p - rho * y, pq = <p, q>, alpha = rz / pq.
struct CgRowEpi {
  static constexpr int kDot = 1;
  const double *rowfac, *rP, *p;
  double *y, *q, *sc;
  int* status;
  __device__ void row(int64_t i, const double* s, double* d) {
    const double yi = rowfac[i] * s[0];
    const double qi = rP[i] * p[i] - sc[SC_RHO] * yi;
    y[i] = yi;
    q[i] = qi;
    d[0] = p[i] * qi;
  }
  __device__ void finish(const double* t) {
    sc[SC_PQ] = t[0];
    if (!(t[0] > 0.0) || !isfinite(t[0])) {
      atomicOr(status, kStatCurv);
      sc[SC_ACTIVE] = 0.0;
      sc[SC_ALPHA] = 0.0;
    } else {
      sc[SC_ALPHA] = sc[SC_RZ] / t[0];
    }
  }
};

// Newton-step setup, row half: y0 = P (P^T d_u0 / c(P)) and the Jacobi sums
// sum_j P_ij^2 / c(P)_j (Lemma condition-number). check = ||y0||_1, which is
// ||F_r(1) d_u0 + grad_u g||_1 for d_u0 = -D(r(P))^-1 grad_u g (Alg. 2's outer test).
// The operator F_r uses the row sums rPs of this very factorised plan (so that
// F_r(1) 1 = 0 holds to summation rounding); grad_u g and d_u0 use r(P) from the
// row LSE, as Alg. 4 defines them.
struct SetupRowEpi {
  static constexpr int kDot = 1;
  const double *rowfac, *rP, *du0;
  double *y0, *diag, *rPs, *sc;
  __device__ void row(int64_t i, const double* s, double* d) {
    const double f = rowfac[i];
    const double yy = f * s[0];
    const double rs = f * s[2];
    y0[i] = yy;
    diag[i] = f * f * s[1];
    rPs[i] = rs;
    d[0] = fabs((rs - rP[i]) * du0[i] - yy);
  }
  __device__ void finish(const double* t) { sc[SC_CHECK] = t[0]; }
};

// Plain row sums: out_i = rowfac_i * s0 (and * s1).
struct RowSumEpi {
  static constexpr int kDot = 0;
  const double* rowfac;
  double *o0, *o1;
  __device__ void row(int64_t i, const double* s, double* d) {
    const double f = rowfac ? rowfac[i] : 1.0;
    if (o0) o0[i] = f * s[0];
    if (o1) o1[i] = f * s[1];
  }
  __device__ void finish(const double*) {}
};

// ----------------------------------------------------------------------------
// epilogues of column sweeps
// ----------------------------------------------------------------------------

// CG column half: zf_j = colfac_j * (P^T p)_j / c(P)_j, as the next row weight.
template <class T>
struct CgColEpi {
  static constexpr int kDot = 0;
  const double *colfac, *cP;
  T* zf;
  __device__ void col(int64_t j, const double* s, double* d) {
    const double f = colfac[j];
    zf[j] = (T)(f * f * s[0] / cP[j]);
  }
  __device__ void finish(const double*) {}
};

// ---- the CG iteration of dense costs: three kernels, one grid-wide ticket ----
// PCG on F_r(rho) (Alg. 2) with the search-direction update folded into the
// sweeps. By linearity, w = P^T (rowfac p) for p = z + beta p_prev is
// P^T (rowfac z) + beta w_prev, so the column half sweeps the row weights
// rowfac z that the update kernel wrote and adds beta w_prev per column; the
// row half forms p = z + beta p_prev per row. beta and the stop test come from
// the update kernel's per-CTA partials of <res, z> and ||res||_1, which every
// CTA of the column half sums itself in fixed order (no grid-wide ticket);
// likewise the update kernel sums the row half's partials of <p, q> for alpha.

// (<res, z>, ||res||_1) from `nparts` per-CTA partials, in fixed order; one warp.
__device__ __forceinline__ void sum_cg_partials(const double* part, int nparts, double& rz, double& r1) {
  const int lane = threadIdx.x & 31;
  double a = 0.0, b = 0.0;
  for (int k = lane; k < nparts; k += 32) {
    a += part[2 * k];
    b += part[2 * k + 1];
  }
  rz = warp_sum(a);
  r1 = warp_sum(b);
}

constexpr int kCgMaxParts = 1024;  // update-kernel partials a column half can stage
constexpr int kCgMaxStrip = 128;   // columns of one strip of the column sweep (32 V)
struct CgStage {
  double part[2 * kCgMaxParts];   // (<res, z>, ||res||_1) partials
  double wprev[kCgMaxStrip];      // w_prev of the CTA's strip
  double colfac[kCgMaxStrip];     // colfac and c(P) of the strip (read by the finisher)
  double cP[kCgMaxStrip];
  double iters, rzprev;           // SC_ITERS, SC_RZPREV
};
__device__ __forceinline__ CgStage& cg_stage_smem() {
  __shared__ __align__(16) CgStage st;
  return st;
}

// Column half: w_j = (P^T (rowfac z))_j + beta w_prev_j; zf_j = colfac_j^2 w_j / c(P)_j,
// with beta = <res, z> / <res, z>_prev (0 on the first iteration). begin(): warp 0
// starts asynchronous copies of what the strip's epilogue needs (the update
// kernel's partials, w_prev, colfac and c(P) of the strip's columns, two
// scalars) into shared
// memory, where they land while the CTA sweeps; drain(): warp 0 waits for them;
// prepare() (the CTAs that finish a strip): beta and the stop test ||res||_1 <=
// tol or the iteration cap, published by the finisher of strip 0. When the test
// stops CG this sweep's results are not used: the row half and the update see
// the cleared flag and return.
template <class T>
struct CgColFusedEpi {
  static constexpr int kDot = 0;
  static constexpr bool kPrefetch = true;
  const double *colfac, *cP;
  T* zf;
  double* wprev;       // [m] w of the previous iteration
  const double* part;  // [nparts][2] partials of the update kernel (or of cg_init)
  int nparts;          // <= kCgMaxParts
  double* sc;
  int* status;
  cudaGraphConditionalHandle cond;
  double beta;
  bool first;
  int64_t j0;          // first column of the strip
  int acol;            // slot of the stop decision: the row half reads it, the update kernel commits it
  __device__ void begin(int64_t strip0, int sw, int64_t m) {
    j0 = strip0;
    if (threadIdx.x < 32) {
      CgStage& s = cg_stage_smem();
      for (int k = threadIdx.x; k < nparts; k += 32) cp_async16(s.part + 2 * k, part + 2 * k);
      // w_prev of the strip (pairs of columns: the strip start is a multiple of 32 V >= 32)
      const int w = (int)min((int64_t)sw, m - strip0);
      for (int k = 2 * threadIdx.x; k < w; k += 64) {
        if (k + 1 < w) {
          cp_async16(s.wprev + k, wprev + strip0 + k);
          cp_async16(s.colfac + k, colfac + strip0 + k);
          cp_async16(s.cP + k, cP + strip0 + k);
        } else {
          cp_async8(s.wprev + k, wprev + strip0 + k);
          cp_async8(s.colfac + k, colfac + strip0 + k);
          cp_async8(s.cP + k, cP + strip0 + k);
        }
      }
      if (threadIdx.x == 0) {
        cp_async8(&s.iters, sc + SC_ITERS);
        cp_async8(&s.rzprev, sc + SC_RZPREV);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  }
  __device__ void drain() {
    if (threadIdx.x < 32) asm volatile("cp.async.wait_all;" ::: "memory");
  }
  __device__ void prepare(bool publish) {
    __shared__ double sbeta;
    __shared__ int sfirst;
    CgStage& st = cg_stage_smem();
    __syncthreads();  // the copies warp 0 waited for are visible to every thread
    if (threadIdx.x < 32) {
      double rz, r1;
      sum_cg_partials(st.part, nparts, rz, r1);
      if (threadIdx.x == 0) {
        const double it = st.iters;
        const bool f = it == 0.0;
        const double b = f ? 0.0 : rz / st.rzprev;
        sbeta = b;
        sfirst = f ? 1 : 0;
        if (publish) {
          const bool fin = isfinite(rz) && isfinite(r1) && isfinite(b);
          const bool go = fin && r1 > sc[SC_TOL] && it < sc[SC_MAXIT] && it < 1.0e6;
          sc[SC_RZ] = rz;
          sc[SC_RESL1] = r1;
          sc[SC_BETA] = b;
          if (!fin) atomicOr(status, kStatCgNan);
          if (!go) {
            sc[acol] = 0.0;  // not SC_ACTIVE: the other CTAs of this launch may still read it
            if (cond) cudaGraphSetConditional(cond, 0);
          }
        }
      }
    }
    __syncthreads();
    beta = sbeta;
    first = sfirst != 0;
  }
  __device__ void col(int64_t j, const double* s, double* d) {
    const CgStage& st = cg_stage_smem();
    const int64_t k = j - j0;
    const double w = first ? s[0] : s[0] + beta * st.wprev[k];
    wprev[j] = w;
    const double f = st.colfac[k];
    zf[j] = (T)(f * f * w / st.cP[k]);
  }
  __device__ void finish(const double*) {}
};

// Row half: p = z + beta p_prev (in place), y = P (w / c(P)), q = r(P) p - rho y;
// one partial of <p, q> per CTA.
// The row's operands (z, p, rowfac, r(P)) and beta, rho are copied into the
// warp's shared-memory slot by cp.async when the sweep starts (prefetch, lane 0),
// so the epilogue does not wait for a memory round trip at the end of the row.
struct CgRowStage {
  double z, p, rowfac, rP, beta, rho;
};
__device__ __forceinline__ CgRowStage* cg_row_stage() {
  __shared__ __align__(16) CgRowStage st[kWarps];
  return st;
}
struct CgRowFusedEpi {
  static constexpr int kDot = 1;
  static constexpr bool kNoTicket = true;
  static constexpr bool kRowPrefetch = true;
  const double *rowfac, *rP, *z;
  double *p, *y, *q, *sc;
  __device__ void prefetch(int64_t i) {
    CgRowStage& s = cg_row_stage()[threadIdx.x >> 5];
    cp_async8(&s.z, z + i);
    cp_async8(&s.p, p + i);
    cp_async8(&s.rowfac, rowfac + i);
    cp_async8(&s.rP, rP + i);
    cp_async8(&s.beta, sc + SC_BETA);
    cp_async8(&s.rho, sc + SC_RHO);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  // called by the lane that issued prefetch(i)
  __device__ void row(int64_t i, const double* s, double* d) {
    cp_async_wait_all();
    const CgRowStage& st = cg_row_stage()[threadIdx.x >> 5];
    const double pi = st.z + st.beta * st.p;
    p[i] = pi;
    const double yi = st.rowfac * s[0];
    const double qi = st.rP * pi - st.rho * yi;
    y[i] = yi;
    q[i] = qi;
    d[0] = pi * qi;
  }
  __device__ void finish(const double*) {}
};

// Newton-step setup, column half: c(P), and the weights of the setup row sweep.
template <class T>
struct SetupColEpi {
  static constexpr int kDot = 0;
  const double* colfac;
  double* cP;
  T *zf, *wsq;
  __device__ void col(int64_t j, const double* s, double* d) {
    const double f = colfac[j];
    const double c = f * s[0];
    cP[j] = c;
    zf[j] = (T)(f * f * s[1] / c);
    wsq[j] = (T)(f * f / c);
  }
  __device__ void finish(const double*) {}
};

// d_v = -P_c d_u = -(P^T d_u) / c(P)  (Alg. 4's d_v step).
struct DvColEpi {
  static constexpr int kDot = 0;
  const double *colfac, *cP;
  double* dv;
  __device__ void col(int64_t j, const double* s, double* d) { dv[j] = -colfac[j] * s[0] / cP[j]; }
  __device__ void finish(const double*) {}
};

// Column LSE: lse_j = Bl_j + M + log S.
//  mode 0: out_j = base_j + lse_j           (log c(P) given the column shift base)
//  mode 1: out_j = out_j - lse_j            (the column fixes of Alg. 4)
// Dot: sum_j exp(base_j + lse_j) (the total mass, for the Armijo test).
struct ColLseEpi {
  static constexpr int kDot = 1;
  const double* Bl;      // nullable
  const double* base;    // nullable
  double* out;
  int mode;
  double* sc;
  int slot;
  double minus;          // subtracted from the total (1 for the Armijo lhs)
  __device__ void col_lse(int64_t j, double M, double S, double* d) {
    const double lse = (Bl ? Bl[j] : 0.0) + M + log(S);
    const double b = base ? base[j] : 0.0;
    if (mode == 0) out[j] = b + lse;
    else out[j] = out[j] - lse;
    d[0] = exp(b + lse);
  }
  __device__ void finish(const double* t) { sc[slot] = t[0] - minus; }
};

// Column sums: out_j = colfac_j * s0 (and * s1).
struct ColSumEpi {
  static constexpr int kDot = 0;
  const double* colfac;
  double *o0, *o1;
  __device__ void col(int64_t j, const double* s, double* d) {
    const double f = colfac ? colfac[j] : 1.0;
    if (o0) o0[j] = f * s[0];
    if (o1) o1[j] = f * s[1];
  }
  __device__ void finish(const double*) {}
};

// Fused two-sided Hessian-vector product (Eq. hessian / discounted-hessian):
//   out_u = r(P) * du + s P dv,  out_v = s P^T du + c(P) * dv.
struct HvpEpi {
  static constexpr int kDot = 0;
  const double *rowfac, *colfac, *du, *dv;
  double s;
  double *out_u, *out_v, *r_out, *c_out;
  __device__ void col(int64_t j, const double* t, double* d) {
    const double f = colfac[j];
    const double c = f * t[0];
    if (c_out) c_out[j] = c;
    out_v[j] = s * f * t[1] + c * dv[j];
  }
  __device__ void row_part(int64_t i, const double* t) {
    const double f = rowfac[i];
    const double r = f * t[0];
    if (r_out) r_out[i] = r;
    out_u[i] = r * du[i] + s * f * t[1];
  }
  __device__ void finish(const double*) {}
};

// ----------------------------------------------------------------------------
// O(n) kernels
// ----------------------------------------------------------------------------

constexpr int kVecCtas = 64;  // fixed grid of the O(n) kernels of eot_marginals_noalloc

inline int vec_grid(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  return (int)(g < 1 ? 1 : (g > kVecCtas ? kVecCtas : g));
}

// The solver's O(n) kernels run one warp per CTA, spread over all SMs: their
// cost is FP64 instructions (the exponent splits, the CG vectors and dots), and
// this GPU's FP64 pipe retires about two lanes per SM and clock, so a CTA of
// eight warps on one SM would serialise eight warps' FP64 work. With the grid
// at most four CTAs per SM (and at most `slots` CTAs, the deterministic
// reduction's partial slots) each element is usually one thread's work.
constexpr int kOnThreads = 32;
constexpr int kOnWarps = kOnThreads / 32;
inline int on_grid(int64_t n, int sms, int64_t slots) {
  int64_t g = (n + kOnThreads - 1) / kOnThreads;
  const int64_t cap = std::min<int64_t>(4 * (int64_t)sms, slots);
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// Split A = x + alpha*y - z into a high part h (multiple of 1/8, exact in T)
// and a low FP64 part l; optional ew = (T)exp(l), fac = exp(fshift + l).
// plain != 0: round A to T directly and drop the remainder (plain FP32 path).
template <class T>
__device__ __forceinline__ void split_range(int64_t n, const double* x, const double* y, double alpha,
                                            const double* z, int plain, T* h, double* l, T* ew, double* fac,
                                            const double* fshift, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double A = x[i];
    if (y) A += alpha * y[i];
    if (z) A -= z[i];
    double hh, ll;
    if (!isfinite(A)) {
      atomicOr(status, kStatNonfinite);
      hh = A;
      ll = 0.0;
    } else if (sizeof(T) == 8) {
      hh = A;
      ll = 0.0;
    } else if (plain) {
      hh = (double)(float)A;
      ll = 0.0;
    } else {
      if (fabs(A) >= kSplitLimit) atomicOr(status, kStatRange);
      hh = rint(A * 8.0) * kGrid;
      ll = A - hh;
    }
    h[i] = (T)hh;
    if (l) l[i] = ll;
    if (ew) ew[i] = (T)exp(ll);
    if (fac) fac[i] = exp((fshift ? fshift[i] : 0.0) + ll);
  }
}
template <class T>
__global__ void split_kernel(int64_t n, const double* x, const double* y, double alpha,
                             const double* z, int plain, T* h, double* l, T* ew, double* fac,
                             const double* fshift, int* status) {
  pdl_wait();
  split_range<T>(n, x, y, alpha, z, plain, h, l, ew, fac, fshift, status);
}
// The same split with alpha read on the device (a line-search step decided there).
template <class T>
__global__ void split_dev_kernel(int64_t n, const double* x, const double* y, const double* alpha,
                                 const double* z, int plain, T* h, double* l, T* ew, double* fac,
                                 const double* fshift, int* status) {
  pdl_wait();
  split_range<T>(n, x, y, *alpha, z, plain, h, l, ew, fac, fshift, status);
}

// Deterministic grid reduction of up to two per-thread values: warp sums, then
// cta_dot_finish (fixed CTA order). Epi::finish receives the totals. Kernels that
// call it are launched with kOnThreads threads per CTA.
template <int ND, class Epi>
__device__ __forceinline__ void vec_finish(double (&v)[2], double* dotpart, int* cnt, Epi& epi) {
  double wd[ND > 0 ? ND : 1];
#pragma unroll
  for (int k = 0; k < ND; ++k) wd[k] = warp_sum(v[k]);
  cta_dot_finish<ND, Epi, kOnWarps>(wd, blockIdx.x, gridDim.x, dotpart, cnt, epi);
}

struct SlotFinish {
  static constexpr int kDot = 2;
  double* sc;
  int s0, s1;  // -1 = unused
  double add0, add1;
  __device__ void finish(const double* t) {
    if (s0 >= 0) sc[s0] = t[0] + add0;
    if (s1 >= 0) sc[s1] = t[1] + add1;
  }
};

struct CgInitFinish {
  static constexpr int kDot = 2;
  double* sc;
  cudaGraphConditionalHandle cond;  // the CG loop's conditional node (0: none)
  __device__ void finish(const double* t) {
    sc[SC_RZ] = t[0];
    sc[SC_RESL1] = t[1];
    sc[SC_ITERS] = 0.0;
    sc[SC_BETA] = 0.0;
    const bool go = t[1] > sc[SC_TOL] && isfinite(t[0]);
    sc[SC_ACTIVE] = go ? 1.0 : 0.0;
    if (cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
  }
};

struct CgUpdateFinish {
  static constexpr int kDot = 2;
  double* sc;
  int* status;
  cudaGraphConditionalHandle cond;
  __device__ void finish(const double* t) {
    const double rz_new = t[0];
    sc[SC_BETA] = rz_new / sc[SC_RZ];
    sc[SC_RZ] = rz_new;
    sc[SC_RESL1] = t[1];
    const double it = sc[SC_ITERS] + 1.0;
    sc[SC_ITERS] = it;
    bool go = t[1] > sc[SC_TOL] && it < sc[SC_MAXIT] && it < 1.0e6;
    if (!isfinite(t[0]) || !isfinite(t[1])) {
      atomicOr(status, kStatCgNan);
      go = false;
    }
    sc[SC_ACTIVE] = go ? 1.0 : 0.0;
    if (!go && cond) cudaGraphSetConditional(cond, 0);
  }
};

// Newton-step preparation: r(P) = exp(log r(P)), d_u0 = r~ / r(P) - 1 (Alg. 2's
// initial direction), row weights of the setup column sweep.
template <class T>
__global__ void prep_setup_kernel(int64_t n, const double* logrP, const double* rt,
                                  const double* rowfac, double* rP, double* du0, T* xw0, T* xw1) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double r = exp(logrP[i]);
    const double d = rt[i] / r - 1.0;
    rP[i] = r;
    du0[i] = d;
    xw0[i] = (T)rowfac[i];
    xw1[i] = (T)(rowfac[i] * d);
  }
}

// PCG start (x = 0): M = diag(F_r(rho)) = r(P) - rho * diag, res = b = r~ - r(P),
// z = res / M, p = z; rz = <res, z>, ||res||_1.
// M_ii = r(P)_i (1 - rho mu_i) >= (1 - rho) r(P)_i since mu_i = (P_rc)_ii <= 1
// (Lemma condition-number); the bound is applied to absorb FP32 summation
// rounding when mu_i is close to 1.
template <class T>
__global__ void cg_init_kernel(int64_t n, const double* rP, const double* rPs, const double* rt,
                               const double* diag, const double* rowfac, double* M, double* x,
                               double* res, double* z, double* p, double* Yx, T* xw, double* sc,
                               double* dotpart, int* cnt, cudaGraphConditionalHandle cond) {
  pdl_wait();
  const double rho = sc[SC_RHO];
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double Mi = fmax(rPs[i] - rho * diag[i], (1.0 - rho) * rPs[i]);
    const double b = rt[i] - rP[i];
    const double zi = b / Mi;
    M[i] = Mi;
    x[i] = 0.0;
    res[i] = b;
    z[i] = zi;
    p[i] = zi;
    Yx[i] = 0.0;
    xw[i] = (T)(rowfac[i] * zi);
    v[0] += b * zi;
    v[1] += fabs(b);
  }
  CgInitFinish f{sc, cond};
  vec_finish<2>(v, dotpart, cnt, f);
}

// PCG step, after q = F_r(rho) p and alpha = rz / <p, q> are known:
// x += alpha p, res -= alpha q, Yx += alpha y, z = res / M; then beta, the stop test.
template <class T>
__global__ void cg_update_kernel(int64_t n, const double* p, const double* q, const double* y,
                                 const double* M, double* x, double* res, double* Yx, double* z,
                                 double* sc, double* dotpart, int* cnt, int* status,
                                 cudaGraphConditionalHandle cond) {
  pdl_wait();
  if (sc[SC_ACTIVE] == 0.0) {
    if (cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
    return;
  }
  const double alpha = sc[SC_ALPHA];
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double r = res[i] - alpha * q[i];
    res[i] = r;
    Yx[i] += alpha * y[i];
    const double zi = r / M[i];
    z[i] = zi;
    v[0] += r * zi;
    v[1] += fabs(r);
  }
  CgUpdateFinish f{sc, status, cond};
  vec_finish<2>(v, dotpart, cnt, f);
}

// p = z + beta p, and the FP32 row weights of the next column sweep.
template <class T>
__global__ void cg_pupdate_kernel(int64_t n, const double* z, const double* rowfac, double* p,
                                  T* xw, const double* sc) {
  pdl_wait();
  if (sc[SC_ACTIVE] == 0.0) return;
  const double beta = sc[SC_BETA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = z[i] + beta * p[i];
    p[i] = pi;
    xw[i] = (T)(rowfac[i] * pi);
  }
}

// Dense-cost PCG start (x = 0): Minv = 1 / diag(F_r(rho)) (clamped as in
// cg_init_kernel) into M, res = r~ - r(P), z = Minv res, p_prev = 0, the column half's row weights
// rowfac z, and one (<res, z>, ||res||_1) partial per CTA; the CG loop starts
// (the first column half decides whether it runs).
template <class T>
__global__ void cg_init_fused_kernel(int64_t n, const double* rP, const double* rPs, const double* rt,
                                     const double* diag, const double* rowfac, double* M, double* x, double* res,
                                     double* z, double* p, double* Yx, T* xw, double* sc, double* part,
                                     int acol, cudaGraphConditionalHandle cond) {
  pdl_wait();
  const double rho = sc[SC_RHO];
  double a = 0.0, b1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double Mi = fmax(rPs[i] - rho * diag[i], (1.0 - rho) * rPs[i]);
    const double b = rt[i] - rP[i];
    const double mi = 1.0 / Mi;
    const double zi = b * mi;
    M[i] = mi;
    x[i] = 0.0;
    res[i] = b;
    z[i] = zi;
    p[i] = 0.0;
    Yx[i] = 0.0;
    xw[i] = (T)(rowfac[i] * zi);
    a += b * zi;
    b1 += fabs(b);
  }
  a = warp_sum(a);
  b1 = warp_sum(b1);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc[SC_ITERS] = 0.0;
    sc[SC_BETA] = 0.0;
    sc[SC_ACTIVE] = 1.0;
    sc[acol] = 1.0;
    if (cond) cudaGraphSetConditional(cond, 1);
  }
}

// Dense-cost PCG step: alpha = <res, z> / <p, q> from the row half's partials
// (summed by every CTA in fixed order; <p, F_r p> <= 0 stops CG, reading R21),
// x += alpha p, res -= alpha q, Yx += alpha y, z = Minv res, the next column
// half's row weights rowfac z, and one (<res, z>, ||res||_1) partial per CTA.
// A stop that this iteration's column half decided (slot acol) becomes the
// loop's stop flag SC_ACTIVE here, after every column CTA has read that flag.
template <class T>
__global__ void cg_update_fused_kernel(int64_t n, const double* p, const double* q, const double* y,
                                       const double* Minv, const double* rowfac, double* x, double* res,
                                       double* Yx, double* z, T* xw, double* sc, const double* rowpart,
                                       int nrow, double* part, int* status, int acol,
                                       cudaGraphConditionalHandle cond) {
  pdl_wait();
  if (sc[acol] == 0.0) {  // stopped by this iteration's column half (or earlier): commit it
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      sc[SC_ACTIVE] = 0.0;
      if (cond) cudaGraphSetConditional(cond, 0);
    }
    return;
  }
  // the operands of this thread's first element are loaded before the sum of
  // the partials (they do not depend on alpha): one memory round trip less
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double p0 = 0.0, q0 = 0.0, y0 = 0.0, m0 = 0.0, f0 = 0.0, x0 = 0.0, r0 = 0.0, u0 = 0.0;
  if (i0 < n) {
    p0 = p[i0];
    q0 = q[i0];
    y0 = y[i0];
    m0 = Minv[i0];
    f0 = rowfac[i0];
    x0 = x[i0];
    r0 = res[i0];
    u0 = Yx[i0];
  }
  // this lane's partials k = lane, lane + 32, ... in order, their loads in
  // batches of 16 (one L2 round trip at nrow <= 512)
  double pq = 0.0;
  if ((int)threadIdx.x < nrow)
    ordered_loads<16>(rowpart + 2 * threadIdx.x, 64, (nrow - (int)threadIdx.x + 31) / 32, [&](double v) { pq += v; });
  pq = warp_sum(pq);
  if (!(pq > 0.0) || !isfinite(pq)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicOr(status, kStatCurv);
      sc[SC_PQ] = pq;
      sc[SC_ALPHA] = 0.0;
      sc[SC_ACTIVE] = 0.0;
      sc[acol] = 0.0;
      if (cond) cudaGraphSetConditional(cond, 0);
    }
    return;
  }
  const double alpha = sc[SC_RZ] / pq;
  double a = 0.0, b1 = 0.0;
  for (int64_t i = i0; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const bool first = i == i0;
    const double pi = first ? p0 : p[i], qi = first ? q0 : q[i], yi = first ? y0 : y[i];
    const double mi = first ? m0 : Minv[i], fi = first ? f0 : rowfac[i];
    x[i] = (first ? x0 : x[i]) + alpha * pi;
    const double r = (first ? r0 : res[i]) - alpha * qi;
    res[i] = r;
    Yx[i] = (first ? u0 : Yx[i]) + alpha * yi;
    const double zi = r * mi;
    z[i] = zi;
    xw[i] = (T)(fi * zi);
    a += r * zi;
    b1 += fabs(r);
  }
  a = warp_sum(a);
  b1 = warp_sum(b1);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc[SC_ITERS] += 1.0;
    sc[SC_PQ] = pq;
    sc[SC_ALPHA] = alpha;
    sc[SC_RZPREV] = sc[SC_RZ];
  }
}

// ---- NewtonSolve on the full discounted system (Sec. 3.1, Eq. discounted-hessian) ----
// H(rho) (du, dv) = (r(P) du + s P dv, s P^T du + c(P) dv) with s = sqrt(rho): PCG on
// H(rho) x = (r~ - r(P), 0) from x = 0 with the diagonal preconditioner
// (r(P), c(P)), one two-sided sweep per iteration; d_u is the u-block of x.

// The fused two-sided sweep's epilogue: q = H(rho) p (column sums with row weights
// rowfac p_u, row sums with column weights colfac p_v).
struct FullHvpEpi {
  static constexpr int kDot = 0;
  const double *rowfac, *colfac, *rPs, *cP, *pu, *pv;
  double *qu, *qv;
  const double* sc;
  __device__ void col(int64_t j, const double* t, double* d) {
    qv[j] = cP[j] * pv[j] + sqrt(sc[SC_RHO]) * colfac[j] * t[0];
  }
  __device__ void row_part(int64_t i, const double* t) {
    qu[i] = rPs[i] * pu[i] + sqrt(sc[SC_RHO]) * rowfac[i] * t[0];
  }
  __device__ void finish(const double*) {}
};

// Alg. 2's outer test for the full-system direction: ||F_r(1) x_u + grad_u g||_1 =
// ||r(P) x_u - P D(c(P))^-1 P^T x_u - (r~ - r(P)_lse)||_1 into SC_CHK (row half of a
// two-sweep F_r(1) product whose column half wrote zf).
struct FullCheckRowEpi {
  static constexpr int kDot = 1;
  const double *rowfac, *rPs, *x, *rt, *rP;
  double* sc;
  __device__ void row(int64_t i, const double* s, double* d) {
    d[0] = fabs(rPs[i] * x[i] - rowfac[i] * s[0] - (rt[i] - rP[i]));
  }
  __device__ void finish(const double* t) { sc[SC_CHK] = t[0]; }
};

// One (n + m)-vector of the full system, stored as a u-part [n] and a v-part [m].
struct Split2 {
  double* u;
  double* v;
  __device__ __forceinline__ double& at(int64_t k, int64_t n) { return k < n ? u[k] : v[k - n]; }
};

// Full-system PCG start: x = 0, res = (r~ - r(P), 0), z = res / (r(P), c(P)), p = z,
// the sweep weights rowfac p_u and colfac p_v; <res, z> and ||res||_1 -> CgInitFinish.
template <class T>
__global__ void full_init_kernel(int64_t n, int64_t m, const double* rP, const double* rPs, const double* cP,
                                 const double* rt, const double* rowfac, const double* colfac, Split2 x, Split2 res,
                                 Split2 z, Split2 p, T* wu, T* wv, double* sc, double* dotpart, int* cnt,
                                 cudaGraphConditionalHandle cond) {
  pdl_wait();
  double v[2] = {0.0, 0.0};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n + m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const bool up = k < n;
    const int64_t i = up ? k : k - n;
    const double b = up ? rt[i] - rP[i] : 0.0;
    const double zi = b / (up ? rPs[i] : cP[i]);
    x.at(k, n) = 0.0;
    res.at(k, n) = b;
    z.at(k, n) = zi;
    p.at(k, n) = zi;
    if (up) wu[i] = (T)(rowfac[i] * zi);
    else wv[i] = (T)(colfac[i] * zi);
    v[0] += b * zi;
    v[1] += fabs(b);
  }
  CgInitFinish f{sc, cond};
  vec_finish<2>(v, dotpart, cnt, f);
}

// <p, q> of the full system and alpha = <res, z> / <p, q> (a non-positive or
// non-finite curvature stops CG, reading R21).
struct FullPqFinish {
  static constexpr int kDot = 1;
  double* sc;
  int* status;
  __device__ void finish(const double* t) {
    sc[SC_PQ] = t[0];
    if (!(t[0] > 0.0) || !isfinite(t[0])) {
      atomicOr(status, kStatCurv);
      sc[SC_ACTIVE] = 0.0;
      sc[SC_ALPHA] = 0.0;
    } else {
      sc[SC_ALPHA] = sc[SC_RZ] / t[0];
    }
  }
};
static __global__ void full_pq_kernel(int64_t n, int64_t m, Split2 p, Split2 q, double* sc, int* status,
                                      double* dotpart, int* cnt) {
  pdl_wait();
  if (sc[SC_ACTIVE] == 0.0) return;
  double v[2] = {0.0, 0.0};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n + m;
       k += (int64_t)gridDim.x * blockDim.x)
    v[0] += p.at(k, n) * q.at(k, n);
  FullPqFinish f{sc, status};
  vec_finish<1>(v, dotpart, cnt, f);
}

// x += alpha p, res -= alpha q, z = res / (r(P), c(P)); beta and the stop test
// (CgUpdateFinish: ||res||_1 <= tol or the iteration cap).
static __global__ void full_update_kernel(int64_t n, int64_t m, Split2 p, Split2 q, const double* rPs,
                                          const double* cP, Split2 x, Split2 res, Split2 z, double* sc,
                                          double* dotpart, int* cnt, int* status, cudaGraphConditionalHandle cond) {
  pdl_wait();
  if (sc[SC_ACTIVE] == 0.0) {
    if (cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0);
    return;
  }
  const double alpha = sc[SC_ALPHA];
  double v[2] = {0.0, 0.0};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n + m;
       k += (int64_t)gridDim.x * blockDim.x) {
    x.at(k, n) += alpha * p.at(k, n);
    const double r = res.at(k, n) - alpha * q.at(k, n);
    res.at(k, n) = r;
    const double zi = r / (k < n ? rPs[k] : cP[k - n]);
    z.at(k, n) = zi;
    v[0] += r * zi;
    v[1] += fabs(r);
  }
  CgUpdateFinish f{sc, status, cond};
  vec_finish<2>(v, dotpart, cnt, f);
}

// p = z + beta p and the next sweep's weights rowfac p_u, colfac p_v.
template <class T>
__global__ void full_pupdate_kernel(int64_t n, int64_t m, Split2 z, Split2 p, const double* rowfac,
                                    const double* colfac, T* wu, T* wv, const double* sc) {
  pdl_wait();
  if (sc[SC_ACTIVE] == 0.0) return;
  const double beta = sc[SC_BETA];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n + m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double pk = z.at(k, n) + beta * p.at(k, n);
    p.at(k, n) = pk;
    if (k < n) wu[k] = (T)(rowfac[k] * pk);
    else wv[k - n] = (T)(colfac[k - n] * pk);
  }
}

// Undiscounted Newton residual of the CG iterate: F_r(1) x + grad_u g
// = -(res + (1 - rho) Yx), with Yx = P D(c)^-1 P^T x accumulated along the CG
// steps. chk = ||.||_1 (Alg. 2's outer test).
static __global__ void cg_check_kernel(int64_t n, const double* res, const double* Yx, double* sc,
                                double* dotpart, int* cnt) {
  pdl_wait();
  const double om = 1.0 - sc[SC_RHO];
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[0] += fabs(res[i] + om * Yx[i]);
  SlotFinish f{sc, SC_CHK, -1, 0.0, 0.0};
  vec_finish<1>(v, dotpart, cnt, f);
}

// Gauge component of d_u: <r(P), d_u> and sum r(P) into SC_GRD, SC_GMASS.
static __global__ void gauge_kernel(int64_t n, const double* du, const double* rP, double* sc,
                                    double* dotpart, int* cnt) {
  pdl_wait();
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    v[0] += rP[i] * du[i];
    v[1] += rP[i];
  }
  SlotFinish f{sc, SC_GRD, SC_GMASS, 0.0, 0.0};
  vec_finish<2>(v, dotpart, cnt, f);
}

// d_u <- d_u - k 1 with k = <r(P), d_u> / sum r(P) (the direction modulo the gauge:
// (d_u - k 1, d_v + k 1) gives the same plans), then the row weights rowfac * d_u
// of the d_v sweep and the Armijo slope <-grad_u g, d_u> = <r~ - r(P), d_u>.
template <class T>
__global__ void prep_dv_kernel(int64_t n, double* du, const double* rowfac, const double* rt,
                               const double* rP, T* xw, double* sc, double* dotpart, int* cnt) {
  pdl_wait();
  const double kap = sc[SC_GRD] / sc[SC_GMASS];
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double d = du[i] - kap;
    du[i] = d;
    xw[i] = (T)(rowfac[i] * d);
    v[0] += (rt[i] - rP[i]) * d;
  }
  SlotFinish f{sc, SC_SLOPE, -1, 0.0, 0.0};
  vec_finish<1>(v, dotpart, cnt, f);
}

// y = a*x + b*y + c*z (+ d*w): small FP64 vector updates of the outer loops;
// a_dev (nullable) multiplies a by a device scalar (a line-search step).
static __global__ void axpy4_kernel(int64_t n, double* y, double b, const double* x, double a,
                                    const double* a_dev, const double* z, double c, const double* w, double d) {
  pdl_wait();
  if (a_dev) a *= *a_dev;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double t = b == 0.0 ? 0.0 : b * y[i];
    if (x) t += a * x[i];
    if (z) t += c * z[i];
    if (w) t += d * w[i];
    y[i] = t;
  }
}

// One Sinkhorn row fix of the MDOT-Sinkhorn projector, taken only while the
// last row sweep's ||r~ - r(P)||_1 (sc[SC_GL1]) is above eps: u <- u + log r~ -
// log r(P). Once the test passes, u stays fixed and the sweeps that follow
// recompute the same v and log r(P), so the host may check every few
// iterations. sc[SC_AUX1] counts the fixes taken.
static __global__ void sk_step_kernel(int64_t n, double* u, const double* logrt, const double* logrP, double* sc,
                                      double eps) {
  pdl_wait();
  if (!(sc[SC_GL1] > eps)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[SC_AUX1] += 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] = (u[i] + logrt[i]) - logrP[i];
}

// Asymmetric smoothing (Sec. 3.4): t = (1 - w eps) r + (w eps / n); log t.
static __global__ void smooth_kernel(int64_t n, const double* r, double w_eps, double* t, double* logt) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (1.0 - w_eps) * r[i] + w_eps / (double)n;
    t[i] = v;
    logt[i] = log(v);
  }
}

// Sums of up to two functions of one vector: kind 0: x log x (entropy terms,
// 0 log 0 = 0) and x; kind 1: |x - y| and x.
static __global__ void vec_stats_kernel(int64_t n, const double* x, const double* y, int kind, double* sc,
                                 int s0, int s1, double* dotpart, int* cnt, int* status) {
  pdl_wait();
  double v[2] = {0.0, 0.0};
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = x[i];
    if (!isfinite(a)) bad = true;
    if (kind == 0) {
      v[0] += a > 0.0 ? a * log(a) : 0.0;
      v[1] += a;
      if (a < 0.0) bad = true;
    } else {
      v[0] += fabs(a - y[i]);
      v[1] += a;
    }
  }
  if (bad) atomicOr(status, kStatNonfinite);
  SlotFinish f{sc, s0, s1, 0.0, 0.0};
  vec_finish<2>(v, dotpart, cnt, f);
}

// out[i] = (T)(f[i] * x[i]) (x nullable = 1): FP32 / FP64 sweep weights from FP64 factors.
template <class T>
__global__ void weight_kernel(int64_t n, const double* f, const double* x, T* out) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (T)(f[i] * (x ? x[i] : 1.0));
}

// One row or one column: U(r, c) = {r c^T}, whose potentials at gamma are
// u = log r, v_j = log c_j + gamma C_0j (n = 1), or v = log c,
// u_i = log r_i + gamma C_i0 (m = 1); zero masses are clamped to 1e-300.
// C from the dense cost (Cd, ld ldc) or from points (X, Y, d, s_C) in FP64.
template <class T>
__global__ void closed_form_kernel(int64_t n, int64_t m, const double* r, const double* c,
                                   double gamma, const T* Cd, int64_t ldc, const float* X,
                                   const float* Y, int d, double sC, double* u, double* v) {
  pdl_wait();
  const int64_t L = n == 1 ? m : n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = n == 1 ? 0 : k, j = n == 1 ? k : 0;
    double C;
    if (Cd) {
      C = (double)Cd[i * ldc + j];
    } else {
      double D = 0.0;
      for (int q = 0; q < d; ++q) {
        const double df = (double)X[i * d + q] - (double)Y[j * d + q];
        D += df * df;
      }
      C = sC * D;
    }
    if (n == 1) {
      v[j] = log(fmax(c[j], 1e-300)) + gamma * C;
      if (k == 0) u[0] = log(fmax(r[0], 1e-300));
    } else {
      u[i] = log(fmax(r[i], 1e-300)) + gamma * C;
      if (k == 0) v[0] = log(fmax(c[0], 1e-300));
    }
  }
}

// dC_ij = scale * P_ij written densely (ld ldo), P_ij = rowfac_i colfac_j exp(Ah_i + Bh_j - gamma C_ij).
template <class T>
__global__ void plan_dense_kernel(int64_t n, int64_t m, const T* C, int64_t ldc, const T* Ah,
                                  const T* Bh, const double* gamma_dev, const double* rowfac,
                                  const double* colfac, double scale, float* out, int64_t ldo) {
  pdl_wait();
  const T g = (T)*gamma_dev;
  const int64_t total = n * m;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / m, j = k - i * m;
    const T t = fmaT(-g, C[i * ldc + j], Ah[i] + Bh[j]);
    out[i * ldo + j] = (float)(scale * rowfac[i] * colfac[j] * (double)expT(t));
  }
}

// out = f * d + s * g for one side of the two-sweep Hessian-vector product;
// f (a marginal) is also copied to fout when given.
static __global__ void hvp_assemble_kernel(int64_t n, const double* f, const double* g,
                                           const double* d, double s, double* out, double* fout) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = f[i] * d[i] + s * g[i];
    if (fout) fout[i] = f[i];
  }
}

// Resets the L2 eviction priority of a cost marked evict-last by the sweeps
// (one applypriority per 128-byte line, all lines inside the cost's rows), so
// that later traffic evicts it normally.
static __global__ void l2_demote_kernel(const char* base, int64_t bytes) {
  pdl_wait();
  const uintptr_t b0 = (uintptr_t)base & ~(uintptr_t)127;
  const int64_t lines = ((int64_t)((uintptr_t)base - b0) + bytes + 127) / 128;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < lines;
       k += (int64_t)gridDim.x * blockDim.x)
    asm volatile("applypriority.global.L2::evict_normal [%0], 128;" ::"l"(b0 + 128 * k));
}

static __global__ void exp_kernel(int64_t n, const double* x, double* y) {
  pdl_wait();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = exp(x[i]);
}

// y *= *s (nullable s: no-op): applies a device-resident scale, e.g. the
// incoming gradient of an autograd graph, without a host round trip.
static __global__ void scale_by_dev_kernel(int64_t n, double* y, const double* s) {
  pdl_wait();
  if (!s) return;
  const double f = *s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] *= f;
}

// <a, b> into sc[slot] (deterministic grid reduction).
static __global__ void dot_kernel(int64_t n, const double* a, const double* b, double* sc, int slot,
                                  double* dotpart, int* cnt) {
  pdl_wait();
  double v[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[0] += a[i] * b[i];
  SlotFinish f{sc, slot, -1, 0.0, 0.0};
  vec_finish<1>(v, dotpart, cnt, f);
}

// The dual value (<r, u> + <c, v> - sum P + 1) / gamma from the device scalars
// of the two dot products and the plan's mass (Eq. sinkhorn-dual).
static __global__ void dual_value_kernel(const double* sc, int s_ru, int s_cv, int s_mass, double gamma,
                                         double* out) {
  pdl_wait();
  *out = (sc[s_ru] + sc[s_cv] - sc[s_mass] + 1.0) / gamma;
}

static __global__ void set_scalar_kernel(double* sc, int slot, double v) {
  pdl_wait(); sc[slot] = v; }

}  // namespace eot
