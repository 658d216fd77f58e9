// eot_solve_batched: many point-cloud problems of uneven size solved by ONE
// persistent kernel launch.
//
// All co-resident CTAs are launched cooperatively and formed into groups of G
// CTAs. Each group takes problems from a queue (largest n m first) and runs the
// whole method for that problem on the device: Alg. 1 (annealing with adaptive
// q, smoothing and extrapolation), each stage projected by Alg. 4 with Alg. 3
// (ChiSinkhorn) and Alg. 2 (NewtonSolve, Jacobi-preconditioned CG with rho
// annealing and the adaptive rho0 of Appx. B). The steps and their order are
// those of the single-problem solver (solver.cuh, solver_impl.cuh).
//
// A sweep here is a loop of the group's threads over their OWN rows (or
// columns), each thread reducing over the whole OTHER side staged through
// shared memory, so a sweep needs no cross-CTA partial sums. The group's CTAs
// meet at software barriers in global memory whose waits are bounded in time
// (a stuck barrier aborts the launch with an error instead of hanging). Every
// control decision uses scalars that all CTAs of a group compute identically
// (fixed-order reductions, status bits OR-ed across the group at each
// reduction), so the CTAs of a group always take the same path.
//
// G and the number of own elements per thread come from an autotuner that
// times probe sweeps of the actual batch once per batch shape (cached in the
// handle).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "handle.cuh"
#include "kernels.cuh"
#include "sweep_pts.cuh"

namespace eot {
namespace bt {

constexpr int kTO = 256;                              // other-side elements per shared tile
constexpr int kDmax = 4;                              // point dimension of the batched kernel
constexpr int kFlush = 16;                            // FP32 terms per compensated flush
constexpr unsigned long long kWaitNs = 2000000000ull;  // bound on one barrier wait (2 s)

struct Prob {  // one problem, device copy
  const float* X;
  const float* Y;
  const double* r;
  const double* c;
  double* u;
  double* v;
  int64_t n, m;
  int32_t d, pad;
  double sC;  // <= 0: computed on the device as 1 / max |x_i - y_j|^2
};

struct Out {  // per-problem result, written by the group that solved it
  int32_t status, stages, newton_steps, cg_iters, cg_solves, ls_trials, sinkhorn_iters, curvature_stops;
  int64_t sweeps;
  double final_gamma, final_rho, grad_l1, marg_err_l1, sC;
};

struct Params {
  double gamma_i, gamma_f, p, q1, w_r, tol_final;
  int32_t max_stages, max_newton, max_cg, max_ls;
  int32_t plain;  // plain FP32 exponent (no split)
  int32_t probe;  // > 0: autotuner probe, that many LSE sweep pairs per problem
};

struct Launch {
  const Prob* probs;
  Out* outs;
  const int32_t* order;  // problem indices, largest first
  int32_t nprob;
  int32_t G;             // CTAs per group
  int32_t ro;            // own elements per thread and round (1, 2 or 4)
  int32_t* queue;        // next position in `order`
  unsigned* bar;         // [groups] barrier counters
  double* part;          // [groups][2][G][4] reduction partials
  int32_t* ipart;        // [groups][2][G] status words
  int32_t* abort;        // set when a barrier wait runs out
  unsigned char* ws;     // [groups] workspaces
  int64_t ws_stride;     // bytes per group
  int64_t maxN, maxM;
  Params prm;
};

// ---------------------------------------------------------------------------
// group machinery: barrier, reductions
// ---------------------------------------------------------------------------

template <class T>
struct Smem {
  T sh[kTO];
  T sw[3][kTO];
  T sy[kDmax][kTO];
  double sc[SC_COUNT];
  double red[4][kWarps];
  double tot[4];
  int ired[kWarps];
  int status;
  int fail;
  int prob;
};

struct Grp {
  int g, rank, G, GT, gt;
  unsigned* bar;
  unsigned gen;
  double* part;
  int32_t* ipart;
  int rcount;
  int32_t* abort;
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Group barrier: every CTA adds 1 to the group's counter and waits until the
// counter reaches (barriers passed) x G. The wait gives up after kWaitNs or when
// another group has given up; the failure is sticky (s.fail) and every caller
// returns false from then on.
template <class T>
__device__ bool gbar(Grp& c, Smem<T>& s) {
  __syncthreads();
  c.gen++;
  if (threadIdx.x == 0 && !s.fail) {
    __threadfence();
    atomicAdd(c.bar, 1u);
    const unsigned target = c.gen * (unsigned)c.G;
    const unsigned long long t0 = gtimer();
    for (unsigned it = 0;; ++it) {
      if ((int)(ld_acquire_u32(c.bar) - target) >= 0) break;
      if (*(volatile int32_t*)c.abort) {
        s.fail = 1;
        break;
      }
      // the timer alone is not trusted (it can jump under a profiler): at least
      // 2^16 polls of >= 64 ns as well, and 2^26 polls always end the wait
      if ((it & 63u) == 63u && ((it >= (1u << 16) && gtimer() - t0 > kWaitNs) || it >= (1u << 26))) {
        atomicExch(c.abort, 1);
        s.fail = 1;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  return s.fail == 0;
}

// Group-wide sums of ND values (totals returned in v, identical in every thread
// of the group: warp order, then CTA rank order). The CTAs' status words are
// OR-ed into every CTA's s.status at the same time.
template <int ND, class T>
__device__ bool greduce(Grp& c, Smem<T>& s, double (&v)[ND]) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < ND; ++k) v[k] = warp_sum(v[k]);
  if (l == 0) {
#pragma unroll
    for (int k = 0; k < ND; ++k) s.red[k][w] = v[k];
  }
  __syncthreads();
  const int buf = c.rcount++ & 1;
  double* P = c.part + (size_t)buf * c.G * 4;
  int32_t* IP = c.ipart + (size_t)buf * c.G;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      double t = 0.0;
      for (int q = 0; q < kWarps; ++q) t += s.red[k][q];
      P[c.rank * 4 + k] = t;
    }
    IP[c.rank] = s.status;
  }
  if (!gbar(c, s)) return false;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      double t = 0.0;
      for (int q = 0; q < c.G; ++q) t += __ldcg(P + q * 4 + k);
      s.tot[k] = t;
    }
    int st = 0;
    for (int q = 0; q < c.G; ++q) st |= __ldcg(IP + q);
    s.status = st;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < ND; ++k) v[k] = s.tot[k];
  return true;
}

// Group-wide maximum of one value (same order rules as greduce).
template <class T>
__device__ bool gmax(Grp& c, Smem<T>& s, double& v) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (l == 0) s.red[0][w] = v;
  __syncthreads();
  const int buf = c.rcount++ & 1;
  double* P = c.part + (size_t)buf * c.G * 4;
  if (threadIdx.x == 0) {
    double t = s.red[0][0];
    for (int q = 1; q < kWarps; ++q) t = fmax(t, s.red[0][q]);
    P[c.rank * 4] = t;
  }
  if (!gbar(c, s)) return false;
  if (threadIdx.x == 0) {
    double t = __ldcg(P);
    for (int q = 1; q < c.G; ++q) t = fmax(t, __ldcg(P + q * 4));
    s.tot[0] = t;
  }
  __syncthreads();
  v = s.tot[0];
  return true;
}

// ---------------------------------------------------------------------------
// one problem, solved by one group
// ---------------------------------------------------------------------------

template <class T>
__device__ __forceinline__ T ldv(const T* p) { return __ldcg(p); }

template <class T>
struct Dev {
  Grp& gp;
  Smem<T>& s;
  const Params& prm;
  int ro;
  // problem
  int64_t n, m;
  int d;
  const float *X, *Y;
  double sC;
  const double *r0, *c0;
  double *u, *v;
  // workspace (layout: see ws_bytes)
  T *Ah, *Bh, *xw0, *xw1, *zf, *wsq, *ewr, *ewc;
  double *Al, *rowfac, *rP, *logrP, *rowmax, *rt, *logrt, *du, *x, *res, *z, *p, *q, *y, *Yx, *M, *diag,
      *y0, *du0, *nt0, *nt1, *rPs;
  double *Bl, *colfac, *cP, *logcP, *ct, *logct, *dv, *mt0, *mt1;
  // counters
  int64_t sweeps = 0;
  int newton_steps = 0, cg_iters = 0, cg_solves = 0, ls_trials = 0, sk_iters = 0, curv = 0;
  double rho_last = 0.0;
  int err = 0;  // eot_status of this problem

  __device__ Dev(Grp& g_, Smem<T>& s_, const Params& p_, int ro_, const Prob& P, unsigned char* ws,
                 int64_t maxN, int64_t maxM)
      : gp(g_), s(s_), prm(p_), ro(ro_) {
    n = P.n;
    m = P.m;
    d = P.d;
    X = P.X;
    Y = P.Y;
    sC = P.sC;
    r0 = P.r;
    c0 = P.c;
    u = P.u;
    v = P.v;
    double* b = (double*)ws;
    double** rv[] = {&Al, &rowfac, &rP, &logrP, &rowmax, &rt, &logrt, &du, &x, &res, &z,
                     &p, &q, &y, &Yx, &M, &diag, &y0, &du0, &nt0, &nt1, &rPs};
    for (double** a : rv) {
      *a = b;
      b += maxN;
    }
    double** cv[] = {&Bl, &colfac, &cP, &logcP, &ct, &logct, &dv, &mt0, &mt1};
    for (double** a : cv) {
      *a = b;
      b += maxM;
    }
    const int64_t L = maxN > maxM ? maxN : maxM;
    T** tv[] = {&Ah, &Bh, &xw0, &xw1, &zf, &wsq, &ewr, &ewc};
    for (T** a : tv) {
      *a = (T*)b;
      b += L;
    }
  }

  __device__ bool bar() { return gbar(gp, s); }
  template <int ND>
  __device__ bool reduce(double (&a)[ND]) { return greduce<ND>(gp, s, a); }
  __device__ void set_status(int bits) { atomicOr(&s.status, bits); }
  // the status bits that end a problem, as the single-problem solver's read()
  __device__ bool bad() {
    const int st = s.status;
    if (st & kStatNonfinite) err = EOT_ERR_NONFINITE;
    else if (st & kStatCgNan) err = EOT_ERR_NONFINITE;
    else if (st & kStatRange) err = EOT_ERR_RANGE;
    return err != 0;
  }
  __device__ void clear_status() {
    __syncthreads();
    if (threadIdx.x == 0) s.status = 0;
    __syncthreads();
  }
  __device__ void set_sc(int slot, double val) {
    __syncthreads();
    if (threadIdx.x == 0) s.sc[slot] = val;
    __syncthreads();
  }

  // A = x + alpha y - z split into h (1/8 grid, exact in T) + l (FP64), as split_kernel
  __device__ void split(int64_t len, const double* xa, const double* ya, double alpha, const double* za,
                        T* h, double* l, T* ew, double* fac, const double* fshift) {
    for (int64_t i = gp.gt; i < len; i += gp.GT) {
      double A = ldv(xa + i);
      if (ya) A += alpha * ldv(ya + i);
      if (za) A -= ldv(za + i);
      double hh, ll;
      if (!isfinite(A)) {
        set_status(kStatNonfinite);
        hh = A;
        ll = 0.0;
      } else if (sizeof(T) == 8) {
        hh = A;
        ll = 0.0;
      } else {
        if (fabs(A) >= kSplitLimit) set_status(kStatRange);
        hh = rint(A * 8.0) * kGrid;
        ll = A - hh;
      }
      h[i] = (T)hh;
      if (l) l[i] = ll;
      if (ew) ew[i] = (T)exp(ll);
      if (fac) fac[i] = exp((fshift ? ldv(fshift + i) : 0.0) + ll);
    }
  }

  // ---- the sweep: own elements of this thread against the whole other side ----
  template <int RO, int NR, bool LSE, int SQM, bool ROWS, class Epi>
  __device__ bool sweep_ro(const T* w0, const T* w1, const T* w2, Epi& epi) {
    constexpr bool PRECISE = sizeof(T) == 4;
    constexpr int NA = LSE ? 1 : NR;
    constexpr int NW = LSE ? 1 : NR;
    constexpr int ND = Epi::kDot;
    const int64_t n_own = ROWS ? n : m, n_oth = ROWS ? m : n;
    const float* xo = ROWS ? X : Y;
    const float* xt = ROWS ? Y : X;
    const T* ho = ROWS ? Ah : Bh;
    const T* ht = ROWS ? Bh : Ah;
    const T* wv[3] = {w0, w1, w2};
    const T g = (T)s.sc[SC_GAMMA];
    T Kh, Kl;
    split_k<T>((double)g * sC, Kh, Kl);
    double dots[ND > 0 ? ND : 1];
#pragma unroll
    for (int k = 0; k < (ND > 0 ? ND : 1); ++k) dots[k] = 0.0;
    const int64_t step = (int64_t)RO * gp.GT;
    for (int64_t base = 0; base < n_own; base += step) {
      if (base + (int64_t)gp.rank * kThreads >= n_own) continue;  // no element of this CTA
      int64_t e[RO];
      bool ev[RO];
      T xr[RO][kDmax], h[RO];
#pragma unroll
      for (int r = 0; r < RO; ++r) {
        e[r] = base + (int64_t)r * gp.GT + gp.gt;
        ev[r] = e[r] < n_own;
        h[r] = ev[r] ? ldv(ho + e[r]) : T(0);
#pragma unroll
        for (int k = 0; k < kDmax; ++k) xr[r][k] = (ev[r] && k < d) ? (T)xo[e[r] * d + k] : T(0);
      }
      T Sa[RO][NA], Ca[RO][NA], mx[RO], hm[RO];
      bool mx_set[RO];
#pragma unroll
      for (int r = 0; r < RO; ++r) {
        mx[r] = T(0);
        hm[r] = h[r];
        mx_set[r] = false;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
          Sa[r][k] = T(0);
          Ca[r][k] = T(0);
        }
      }
      for (int64_t jt = 0; jt < n_oth; jt += kTO) {
        const int tn = (int)min((int64_t)kTO, n_oth - jt);
        __syncthreads();
        for (int qq = threadIdx.x; qq < tn; qq += kThreads) {
          const int64_t j = jt + qq;
          s.sh[qq] = ldv(ht + j);
#pragma unroll
          for (int k = 0; k < NW; ++k) s.sw[k][qq] = ldv(wv[k] + j);
#pragma unroll
          for (int k = 0; k < kDmax; ++k) s.sy[k][qq] = k < d ? (T)xt[j * d + k] : T(0);
        }
        __syncthreads();
        for (int q0 = 0; q0 < tn; q0 += kFlush) {
        const int q1 = min(tn, q0 + kFlush);
        T acc[RO][NA];
#pragma unroll
        for (int r = 0; r < RO; ++r)
#pragma unroll
          for (int k = 0; k < NA; ++k) acc[r][k] = T(0);
#pragma unroll 2
        for (int qq = q0; qq < q1; ++qq) {
          T yq[kDmax];
#pragma unroll
          for (int k = 0; k < kDmax; ++k) yq[k] = s.sy[k][qq];
          const T hb = s.sh[qq];
          T wq[NW];
#pragma unroll
          for (int k = 0; k < NW; ++k) wq[k] = s.sw[k][qq];
#pragma unroll
          for (int r = 0; r < RO; ++r) {
            T Dh, Dl;
            dist2<PRECISE, T, kDmax>(xr[r], [&](int k) { return yq[k]; }, Dh, Dl);
            if constexpr (!LSE) {
              const T ex = expT(expo<PRECISE>(h[r] + hb, Kh, Kl, Dh, Dl));
#pragma unroll
              for (int k = 0; k < NR; ++k) {
                if ((SQM >> k) & 1) acc[r][k] = fmaT(ex * ex, wq[k], acc[r][k]);
                else acc[r][k] = fmaT(ex, wq[k], acc[r][k]);
              }
            } else {
              if (!mx_set[r]) {  // the running max starts at the first element
                mx[r] = ceil_grid(expo<PRECISE>(h[r] + hb, Kh, Kl, Dh, Dl));
                hm[r] = h[r] - mx[r];
                mx_set[r] = true;
              }
              T t = expo<PRECISE>(hm[r] + hb, Kh, Kl, Dh, Dl);
              for (int k = 0; k < 4 && t > T(kTheta); ++k) {  // raise the max, at most 4 steps
                const T dlt = ceil_grid(t);
                mx[r] += dlt;
                hm[r] = h[r] - mx[r];
                const T f = expT(-dlt);
                acc[r][0] *= f;
                Sa[r][0] *= f;
                Ca[r][0] *= f;
                t = expo<PRECISE>(hm[r] + hb, Kh, Kl, Dh, Dl);
              }
              acc[r][0] = fmaT(expT(t), wq[0], acc[r][0]);
            }
          }
        }
#pragma unroll
        for (int r = 0; r < RO; ++r)
#pragma unroll
          for (int k = 0; k < NA; ++k) kadd(Sa[r][k], Ca[r][k], acc[r][k]);
        }
      }
#pragma unroll
      for (int r = 0; r < RO; ++r) {
        if (!ev[r]) continue;
        DotArr<ND> dd;
        if constexpr (!LSE) {
          double tot[NR];
#pragma unroll
          for (int k = 0; k < NR; ++k) tot[k] = (double)Sa[r][k] + (double)Ca[r][k];
          if constexpr (ROWS) epi.row(e[r], tot, dd.v);
          else epi.col(e[r], tot, dd.v);
        } else {
          const double Ssum = (double)Sa[r][0] + (double)Ca[r][0];
          if constexpr (ROWS) epi.row_lse(e[r], (double)mx[r], Ssum, dd.v);
          else epi.col_lse(e[r], (double)mx[r], Ssum, dd.v);
        }
#pragma unroll
        for (int k = 0; k < ND; ++k) dots[k] += dd.v[k];
      }
    }
    if constexpr (ND > 0) {
      if (!reduce<ND>(dots)) return false;
      if (threadIdx.x == 0) epi.finish(dots);
      __syncthreads();
      return true;
    } else {
      return bar();
    }
  }

  template <int NR, bool LSE, int SQM, bool ROWS, class Epi>
  __device__ bool sweep(const T* w0, const T* w1, const T* w2, Epi epi) {
    sweeps++;
    if (ro == 1) return sweep_ro<1, NR, LSE, SQM, ROWS>(w0, w1, w2, epi);
    if (ro == 2) return sweep_ro<2, NR, LSE, SQM, ROWS>(w0, w1, w2, epi);
    return sweep_ro<4, NR, LSE, SQM, ROWS>(w0, w1, w2, epi);
  }

  // ---- log-sum-exp sweeps (as Solver::row_lse / Solver::col_lse) ----
  __device__ bool row_lse(const double* uu, const double* vv, const double* rshift, double* out_lse,
                          double* out_max, const double* rtg, int s0 = SC_GL1, int s1 = SC_CHI2) {
    split(n, uu, nullptr, 0.0, rshift, Ah, Al, nullptr, nullptr, nullptr);
    split(m, vv, nullptr, 0.0, nullptr, Bh, Bl, ewc, nullptr, nullptr);
    if (!bar()) return false;
    RowLseEpi e{rshift, Al, out_lse, out_max, rtg, s.sc, s0, s1};
    return sweep<1, true, 0, true>(ewc, nullptr, nullptr, e);
  }
  __device__ bool col_lse(const double* uu, const double* duu, const double* vv, const double* dvv,
                          double alpha, const double* cshift, double* out, int mode, int slot,
                          double minus) {
    split(n, uu, duu, alpha, nullptr, Ah, Al, ewr, nullptr, nullptr);
    split(m, vv, dvv, alpha, cshift, Bh, Bl, nullptr, nullptr, nullptr);
    if (!bar()) return false;
    ColLseEpi e{Bl, mode == 0 ? cshift : nullptr, out, mode, s.sc, slot, minus};
    return sweep<1, true, 0, false>(ewr, nullptr, nullptr, e);
  }

  // ---- Alg. 2: NewtonSolve (as Solver::newton); false on a failed barrier or error ----
  __device__ bool newton(double gl1, double eta, double rho0, int max_cg, double* rho_out, bool* ran) {
    split(n, u, nullptr, 0.0, rowmax, Ah, Al, nullptr, rowfac, rowmax);
    split(m, v, nullptr, 0.0, nullptr, Bh, Bl, ewc, colfac, nullptr);
    // prep_setup: r(P), d_u0 = r~ / r(P) - 1, row weights of the setup column sweep
    for (int64_t i = gp.gt; i < n; i += gp.GT) {
      const double rr = exp(ldv(logrP + i));
      const double dd = ldv(rt + i) / rr - 1.0;
      const double f = ldv(rowfac + i);
      rP[i] = rr;
      du0[i] = dd;
      xw0[i] = (T)f;
      xw1[i] = (T)(f * dd);
    }
    if (!bar()) return false;
    if (!sweep<2, false, 0, false>(xw0, xw1, nullptr, SetupColEpi<T>{colfac, cP, zf, wsq})) return false;
    if (!sweep<3, false, 2, true>(zf, wsq, ewc, SetupRowEpi{rowfac, rP, du0, y0, diag, rPs, s.sc}))
      return false;
    if (bad()) return false;
    const double check0 = s.sc[SC_CHECK];
    double rho = rho0, rl = rho0;
    *ran = false;
    const double* du_final = du0;
    if (!(check0 <= eta * gl1)) {
      const double tol = 0.25 * eta * gl1;
      set_sc(SC_TOL, tol);
      set_sc(SC_MAXIT, (double)max_cg);
      for (int solve = 0;; ++solve) {
        set_sc(SC_RHO, rho);
        if (!run_cg()) return false;
        // cg_check: ||F_r(1) x + grad_u g||_1 = ||res + (1 - rho) Yx||_1
        double a1[1] = {0.0};
        const double om = 1.0 - rho;
        for (int64_t i = gp.gt; i < n; i += gp.GT) a1[0] += fabs(ldv(res + i) + om * ldv(Yx + i));
        if (!reduce<1>(a1)) return false;
        const double it = s.sc[SC_ITERS], rl1 = s.sc[SC_RESL1], chk = a1[0];
        cg_iters += (int)it;
        cg_solves++;
        *ran = true;
        rl = rho;
        if (s.status & kStatCurv) {
          // <p, F_r(rho) p> <= 0 in finite precision: keep the iterate (truncated Newton)
          curv++;
          clear_status();
          du_final = it > 0 ? x : du0;
          break;
        }
        if (bad()) return false;
        if (rl1 > tol) {
          err = EOT_ERR_CG_MAXITER;
          return false;
        }
        du_final = x;
        if (chk <= eta * gl1) break;
        rho = 1.0 - (1.0 - rho) / 4.0;
        if (solve > 60) {
          err = EOT_ERR_CG_MAXITER;
          return false;
        }
      }
    }
    // d_u modulo the gauge (as gauge_kernel), then prep_dv: row weights rowfac d_u
    // and the Armijo slope <r~ - r(P), d_u>
    double g2[2] = {0.0, 0.0};
    for (int64_t i = gp.gt; i < n; i += gp.GT) {
      const double ri = ldv(rP + i);
      g2[0] += ri * ldv(du_final + i);
      g2[1] += ri;
    }
    if (!reduce<2>(g2)) return false;
    const double kap = g2[0] / g2[1];
    double a1[1] = {0.0};
    for (int64_t i = gp.gt; i < n; i += gp.GT) {
      const double di = ldv(du_final + i) - kap;
      du[i] = di;
      xw0[i] = (T)(ldv(rowfac + i) * di);
      a1[0] += (ldv(rt + i) - ldv(rP + i)) * di;
    }
    if (!reduce<1>(a1)) return false;
    set_sc(SC_SLOPE, a1[0]);
    if (!sweep<1, false, 0, false>(xw0, nullptr, nullptr, DvColEpi{colfac, cP, dv})) return false;
    *rho_out = rl;
    return true;
  }

  // PCG from x = 0 on F_r(rho) (cg_init, then CG iterations until inactive)
  __device__ bool run_cg() {
    const double rho = s.sc[SC_RHO];
    double a2[2] = {0.0, 0.0};
    for (int64_t i = gp.gt; i < n; i += gp.GT) {
      const double rs = ldv(rPs + i);
      const double Mi = fmax(rs - rho * ldv(diag + i), (1.0 - rho) * rs);
      const double b = ldv(rt + i) - ldv(rP + i);
      const double zi = b / Mi;
      M[i] = Mi;
      x[i] = 0.0;
      res[i] = b;
      z[i] = zi;
      p[i] = zi;
      Yx[i] = 0.0;
      xw0[i] = (T)(ldv(rowfac + i) * zi);
      a2[0] += b * zi;
      a2[1] += fabs(b);
    }
    if (!reduce<2>(a2)) return false;
    if (threadIdx.x == 0) CgInitFinish{s.sc}.finish(a2);
    __syncthreads();
    while (s.sc[SC_ACTIVE] != 0.0) {
      if (!sweep<1, false, 0, false>(xw0, nullptr, nullptr, CgColEpi<T>{colfac, cP, zf})) return false;
      if (!sweep<1, false, 0, true>(zf, nullptr, nullptr,
                                    CgRowEpi{rowfac, rPs, p, y, q, s.sc, &s.status}))
        return false;
      if (s.sc[SC_ACTIVE] == 0.0) break;  // curvature stop in the row half
      const double alpha = s.sc[SC_ALPHA];
      double b2[2] = {0.0, 0.0};
      for (int64_t i = gp.gt; i < n; i += gp.GT) {
        x[i] = ldv(x + i) + alpha * ldv(p + i);
        const double ri = ldv(res + i) - alpha * ldv(q + i);
        res[i] = ri;
        Yx[i] = ldv(Yx + i) + alpha * ldv(y + i);
        const double zi = ri / ldv(M + i);
        z[i] = zi;
        b2[0] += ri * zi;
        b2[1] += fabs(ri);
      }
      if (!reduce<2>(b2)) return false;
      if (threadIdx.x == 0) CgUpdateFinish{s.sc, &s.status, 0}.finish(b2);
      __syncthreads();
      if (s.sc[SC_ACTIVE] == 0.0) break;
      const double beta = s.sc[SC_BETA];
      for (int64_t i = gp.gt; i < n; i += gp.GT) {
        const double pi = ldv(z + i) + beta * ldv(p + i);
        p[i] = pi;
        xw0[i] = (T)(ldv(rowfac + i) * pi);
      }
      if (!bar()) return false;
    }
    return true;
  }

  // ---- Alg. 4: TruncatedNewtonProject (as Solver::project) ----
  // Returns false on error / failed barrier; *ok = false if the Newton budget ran out.
  __device__ bool project(double eps, int max_cg, double* delta_min, double* gl1_out, bool* ok) {
    if (!col_lse(u, nullptr, v, nullptr, 0.0, logct, v, 1, SC_AUX0, 0.0)) return false;
    if (!row_lse(u, v, logrt, logrP, rowmax, rt)) return false;
    if (bad()) return false;
    double gl1 = s.sc[SC_GL1], chi2 = s.sc[SC_CHI2];
    *delta_min = INFINITY;
    *ok = true;
    int steps = 0;
    const double eps_chi = pow(eps, 0.4);
    const double floor32 = (1.0 / 4194304.0) / sqrt((double)(n > m ? n : m));  // as armijo_floor32
    while (gl1 > eps) {
      if (steps >= prm.max_newton) {
        *ok = false;
        break;
      }
      int sk = 0;
      while (chi2 > eps_chi) {  // Alg. 3
        for (int64_t i = gp.gt; i < n; i += gp.GT) u[i] = ldv(u + i) + ldv(logrt + i) - ldv(logrP + i);
        if (!col_lse(u, nullptr, v, nullptr, 0.0, logct, v, 1, SC_AUX0, 0.0)) return false;
        if (!row_lse(u, v, logrt, logrP, rowmax, rt)) return false;
        if (bad()) return false;
        gl1 = s.sc[SC_GL1];
        chi2 = s.sc[SC_CHI2];
        sk_iters++;
        if (++sk > 2000) {
          err = EOT_ERR_MAXNEWTON;
          return false;
        }
      }
      if (gl1 <= eps) break;
      const double eta = fmax(gl1, 0.8 * eps / gl1);
      const double rho0 = fmax(0.0, 1.0 - 4.0 * (1.0 - rho_last));
      double rho = rho0;
      bool ran = false;
      if (!newton(gl1, eta, rho0, max_cg, &rho, &ran)) return false;
      if (ran) rho_last = rho;
      newton_steps++;
      // backtracking on the simplified Armijo test, left side relative to its
      // computed value at alpha = 0 (as Solver::project)
      // an undecidable FP32 test takes the unit step (as Solver::project)
      const bool decidable = sizeof(T) == 8 || 0.99 * s.sc[SC_SLOPE] >= floor32;
      double lhs0 = 0.0;
      if (decidable) {
        if (!col_lse(u, du, v, dv, 0.0, logct, logcP, 0, SC_LHS, 1.0)) return false;
        if (bad()) return false;
        lhs0 = s.sc[SC_LHS];
      }
      double alpha = 1.0;
      int trials = 0;
      for (;;) {
        if (!col_lse(u, du, v, dv, alpha, logct, logcP, 0, SC_LHS, 1.0)) return false;
        const bool out_of_range = (s.status & kStatRange) != 0;
        if (out_of_range) clear_status();  // a trial outside the split range is rejected
        if (bad()) return false;
        ls_trials++;
        if (!out_of_range && (!decidable || s.sc[SC_LHS] - lhs0 <= 0.99 * alpha * s.sc[SC_SLOPE])) break;
        if (++trials > prm.max_ls) {
          err = EOT_ERR_LINESEARCH;
          return false;
        }
        alpha *= 0.5;
      }
      for (int64_t i = gp.gt; i < n; i += gp.GT) u[i] = ldv(u + i) + alpha * ldv(du + i);
      for (int64_t j = gp.gt; j < m; j += gp.GT)
        v[j] = ldv(v + j) + alpha * ldv(dv + j) + ldv(logct + j) - ldv(logcP + j);
      if (!bar()) return false;
      if (!row_lse(u, v, logrt, logrP, rowmax, rt)) return false;
      if (bad()) return false;
      const double new_gl1 = s.sc[SC_GL1];
      chi2 = s.sc[SC_CHI2];
      const double delta = (gl1 - new_gl1) / ((1.0 - eta) * gl1);
      if (delta < *delta_min) *delta_min = delta;
      gl1 = new_gl1;
      steps++;
    }
    for (int64_t i = gp.gt; i < n; i += gp.GT) u[i] = ldv(u + i) + ldv(logrt + i) - ldv(logrP + i);
    *gl1_out = gl1;
    return bar();
  }

  static __device__ double rg(double g) { return sizeof(T) == 4 ? (double)(float)g : g; }

  // s_C = 1 / max |x_i - y_j|^2: FP32 scan per own row, FP64 re-evaluation of
  // each thread's arg-max pair, group maximum (as pts_maxdist_kernel)
  __device__ bool compute_sC() {
    double best = -1.0;
    for (int64_t i = gp.gt; i < n; i += gp.GT) {
      float xi[kDmax];
#pragma unroll
      for (int k = 0; k < kDmax; ++k) xi[k] = k < d ? X[i * d + k] : 0.f;
      float bD = -1.f;
      int64_t bj = 0;
      for (int64_t j = 0; j < m; ++j) {
        float D = 0.f;
#pragma unroll
        for (int k = 0; k < kDmax; ++k) {
          const float df = xi[k] - (k < d ? Y[j * d + k] : 0.f);
          D = fmaf(df, df, D);
        }
        if (D > bD) {
          bD = D;
          bj = j;
        }
      }
      double b64 = 0.0;
      for (int k = 0; k < d; ++k) {
        const double df = (double)X[i * d + k] - (double)Y[bj * d + k];
        b64 += df * df;
      }
      best = fmax(best, b64);
    }
    if (!gmax(gp, s, best)) return false;
    if (!(best > 0.0) || !isfinite(best)) {
      err = EOT_ERR_INVALID_ARG;  // all points coincide: no normalisation
      return false;
    }
    sC = 1.0 / best;
    return true;
  }

  // asymmetric smoothing (Sec. 3.4) of a marginal into (t, log t)
  __device__ void smooth(int64_t len, const double* a, double w_eps, double* t, double* logt) {
    for (int64_t i = gp.gt; i < len; i += gp.GT) {
      const double val = (1.0 - w_eps) * ldv(a + i) + w_eps / (double)len;
      t[i] = val;
      logt[i] = log(val);
    }
  }

  // ---- Alg. 1 (as run_solve) ----
  __device__ bool solve(double* gamma_out, double* gl1_out, int* stages_out, double* merr_out) {
    const int max_cg = prm.max_cg > 0 ? prm.max_cg : (int)(4 * n < 2000 ? 4 * n : 2000);
    double a[2] = {0.0, 0.0};
    for (int64_t i = gp.gt; i < n; i += gp.GT) {
      const double ri = ldv(r0 + i);
      if (!isfinite(ri) || ri < 0.0) set_status(kStatNonfinite);
      a[0] += ri > 0.0 ? ri * log(ri) : 0.0;
      a[1] += ri;
    }
    if (!reduce<2>(a)) return false;
    const double Hr = -a[0], mr = a[1];
    double b[2] = {0.0, 0.0};
    for (int64_t j = gp.gt; j < m; j += gp.GT) {
      const double cj = ldv(c0 + j);
      if (!isfinite(cj) || cj < 0.0) set_status(kStatNonfinite);
      b[0] += cj > 0.0 ? cj * log(cj) : 0.0;
      b[1] += cj;
    }
    if (!reduce<2>(b)) return false;
    const double Hc = -b[0], mc = b[1];
    if ((s.status & kStatNonfinite) || fabs(mr - 1.0) > 1e-6 || fabs(mc - 1.0) > 1e-6) {
      err = EOT_ERR_INVALID_ARG;
      return false;
    }
    const double H = fmin(Hr, Hc);
    const double gamma_f = rg(prm.gamma_f);
    double gamma = rg(fmin(prm.gamma_i, prm.gamma_f));
    double gamma_prev = 0.0, qf = prm.q1, gl1 = 0.0;
    const double w_c = 0.5 - prm.w_r;
    double *n0 = nt0, *n1 = nt1, *m0 = mt0, *m1 = mt1;
    int t = 1;
    if (n == 1 || m == 1) {
      // one row or one column: U(r, c) = {r c^T}; eps_d of Alg. 1 is 0 there
      const int64_t Lc = n == 1 ? m : n;
      for (int64_t k = gp.gt; k < Lc; k += gp.GT) {
        const int64_t i = n == 1 ? 0 : k, j = n == 1 ? k : 0;
        double D = 0.0;
        for (int qd = 0; qd < d; ++qd) {
          const double df = (double)X[i * d + qd] - (double)Y[j * d + qd];
          D += df * df;
        }
        if (n == 1) {
          v[j] = log(fmax(ldv(c0 + j), 1e-300)) + gamma_f * sC * D;
          if (k == 0) u[0] = log(fmax(ldv(r0), 1e-300));
        } else {
          u[i] = log(fmax(ldv(r0 + i), 1e-300)) + gamma_f * sC * D;
          if (k == 0) v[0] = log(fmax(ldv(c0), 1e-300));
        }
      }
      gamma = gamma_f;
      t = 0;
      set_sc(SC_GAMMA, gamma);
      if (!bar()) return false;
    }
    for (; t > 0;) {
      const bool done = gamma == gamma_f;
      double eps_d = H / pow(gamma, prm.p);
      if (done) eps_d = fmin(eps_d, 2.0 * prm.tol_final / 3.0);
      smooth(n, r0, prm.w_r * eps_d, rt, logrt);
      smooth(m, c0, w_c * eps_d, ct, logct);
      if (t == 1) {
        for (int64_t i = gp.gt; i < n; i += gp.GT) {
          u[i] = logrt[i];
          n0[i] = logrt[i];
        }
        for (int64_t j = gp.gt; j < m; j += gp.GT) {
          v[j] = logct[j];
          m0[j] = logct[j];
        }
      }
      set_sc(SC_GAMMA, gamma);
      if (!bar()) return false;
      double dmin = INFINITY;
      bool ok = true;
      if (!project(eps_d / 2.0, max_cg, &dmin, &gl1, &ok)) return false;
      if (!ok) {
        err = EOT_ERR_MAXNEWTON;
        return false;
      }
      if (dmin > 0.95) qf = fmin(2.0, qf * qf);  // AdjustSchedule (Sec. 3.3)
      else if (dmin < 0.8) qf = sqrt(qf);
      const double gamma_next = rg(fmin(qf * gamma, gamma_f));
      if (done) break;
      if (t >= prm.max_stages) {
        err = EOT_ERR_MAXSTAGES;
        return false;
      }
      // Alg. 1's extrapolated warm start: z <- z + ratio (z - z_prev), z_prev <- z
      const double ratio = (gamma_next - gamma) / (gamma - gamma_prev);
      for (int64_t i = gp.gt; i < n; i += gp.GT) {
        const double ui = ldv(u + i);
        n1[i] = ui;
        u[i] = (1.0 + ratio) * ui - ratio * ldv(n0 + i);
      }
      for (int64_t j = gp.gt; j < m; j += gp.GT) {
        const double vj = ldv(v + j);
        m1[j] = vj;
        v[j] = (1.0 + ratio) * vj - ratio * ldv(m0 + j);
      }
      double* tmp = n0;
      n0 = n1;
      n1 = tmp;
      tmp = m0;
      m0 = m1;
      m1 = tmp;
      if (!bar()) return false;
      gamma_prev = gamma;
      gamma = gamma_next;
      ++t;
    }
    // marginal L1 error of the output against the unsmoothed r, c
    if (!row_lse(u, v, nullptr, logrP, nullptr, r0, SC_GL1, SC_CHI2)) return false;
    if (!col_lse(u, nullptr, v, nullptr, 0.0, nullptr, logcP, 0, SC_AUX0, 0.0)) return false;
    double e1[1] = {0.0};
    for (int64_t j = gp.gt; j < m; j += gp.GT) e1[0] += fabs(exp(ldv(logcP + j)) - ldv(c0 + j));
    if (!reduce<1>(e1)) return false;
    if (bad()) return false;
    *gamma_out = gamma;
    *gl1_out = gl1;
    *stages_out = t;
    *merr_out = s.sc[SC_GL1] + e1[0];
    return true;
  }

  // autotuner probe: the start of a projection (column fix + row LSE), `reps` times
  __device__ bool probe(int reps) {
    smooth(n, r0, 0.01, rt, logrt);
    smooth(m, c0, 0.01, ct, logct);
    for (int64_t i = gp.gt; i < n; i += gp.GT) nt0[i] = logrt[i];
    for (int64_t j = gp.gt; j < m; j += gp.GT) mt0[j] = logct[j];
    set_sc(SC_GAMMA, rg(fmin(prm.gamma_i, prm.gamma_f)));
    if (!bar()) return false;
    for (int k = 0; k < reps; ++k) {
      if (!col_lse(nt0, nullptr, mt0, nullptr, 0.0, logct, mt0, 1, SC_AUX0, 0.0)) return false;
      if (!row_lse(nt0, mt0, logrt, logrP, rowmax, rt)) return false;
    }
    return true;
  }
};

template <class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 2 : 1) batch_kernel(Launch L) {
  __shared__ Smem<T> s;
  Grp gp;
  gp.G = L.G;
  gp.g = blockIdx.x / L.G;
  gp.rank = blockIdx.x % L.G;
  gp.GT = L.G * kThreads;
  gp.gt = gp.rank * kThreads + threadIdx.x;
  gp.bar = L.bar + gp.g;
  gp.gen = 0;
  gp.part = L.part + (size_t)gp.g * 2 * L.G * 4;
  gp.ipart = L.ipart + (size_t)gp.g * 2 * L.G;
  gp.rcount = 0;
  gp.abort = L.abort;
  if (threadIdx.x == 0) {
    s.fail = 0;
    s.status = 0;
  }
  __syncthreads();
  unsigned char* ws = L.ws + (size_t)gp.g * L.ws_stride;
  int32_t* slot = L.ipart + (size_t)(gridDim.x / L.G) * 2 * L.G + gp.g;  // after the status words
  for (;;) {
    // the group's first CTA takes the next problem; all CTAs read it after a barrier
    if (gp.rank == 0 && threadIdx.x == 0) *(volatile int32_t*)slot = atomicAdd(L.queue, 1);
    if (!gbar(gp, s)) return;
    if (threadIdx.x == 0) s.prob = *(volatile int32_t*)slot;
    __syncthreads();
    const int k = s.prob;
    if (k >= L.nprob) return;
    const int pi = L.order[k];
    const Prob P = L.probs[pi];
    if (threadIdx.x < SC_COUNT) s.sc[threadIdx.x] = 0.0;
    if (threadIdx.x == 0) s.status = 0;
    __syncthreads();
    Dev<T> D(gp, s, L.prm, L.ro, P, ws, L.maxN, L.maxM);
    double gamma = 0.0, gl1 = 0.0, merr = 0.0;
    int stages = 0;
    bool alive = true;
    if (P.sC <= 0.0) alive = D.compute_sC();
    if (alive) alive = L.prm.probe > 0 ? D.probe(L.prm.probe) : D.solve(&gamma, &gl1, &stages, &merr);
    if (s.fail) return;  // a barrier gave up: leave the launch (the host reports it)
    if (gp.rank == 0 && threadIdx.x == 0) {
      Out o;
      o.status = alive ? 0 : (D.err ? D.err : (int)EOT_ERR_CUDA);
      o.stages = stages;
      o.newton_steps = D.newton_steps;
      o.cg_iters = D.cg_iters;
      o.cg_solves = D.cg_solves;
      o.ls_trials = D.ls_trials;
      o.sinkhorn_iters = D.sk_iters;
      o.curvature_stops = D.curv;
      o.sweeps = D.sweeps;
      o.final_gamma = gamma;
      o.final_rho = D.rho_last;
      o.grad_l1 = gl1;
      o.marg_err_l1 = merr;
      o.sC = D.sC;
      L.outs[pi] = o;
    }
  }
}
}  // namespace bt
}  // namespace eot

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

using namespace eot;
using eot::bt::Launch;
using eot::bt::Out;
using eot::bt::Prob;

constexpr int64_t kBatchMaxSide = 32768;  // n, m per problem (bounds one sweep's time)

double wall_seconds() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

struct Layout {
  size_t probs, outs, order, queue, abort, bar, part, ipart, ws, total;
  int64_t ws_stride;
};

Layout layout(int nprob, int groups, int G, int64_t maxN, int64_t maxM) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.probs = take(sizeof(Prob) * nprob);
  L.outs = take(sizeof(Out) * nprob);
  L.order = take(sizeof(int32_t) * nprob);
  L.queue = take(sizeof(int32_t));
  L.abort = take(sizeof(int32_t));
  L.bar = take(sizeof(unsigned) * groups);
  L.part = take(sizeof(double) * groups * 2 * G * 4);
  L.ipart = take(sizeof(int32_t) * (groups * 2 * G + groups));  // status words, then slots
  const int64_t Lm = std::max(maxN, maxM);
  L.ws_stride = (int64_t)align256((size_t)(22 * maxN + 9 * maxM + 8 * Lm) * 8);
  L.ws = take((size_t)L.ws_stride * groups);
  L.total = o;
  return L;
}

template <class T>
int max_resident_ctas(eot_handle h) {
  int nb = 0;
  EOT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bt::batch_kernel<T>, kThreads, 0));
  return nb * h->sms;
}

// One cooperative launch over `nprob` problems with groups of G CTAs; returns ms.
template <class T>
double launch_batch(eot_handle h, const std::vector<Prob>& probs, const std::vector<int32_t>& order,
                    std::vector<Out>& outs, int G, int ro, const bt::Params& prm, int64_t maxN,
                    int64_t maxM, cudaStream_t st) {
  const int nprob = (int)probs.size();
  const int resident = max_resident_ctas<T>(h);
  const int groups = std::max(1, std::min(nprob, resident / G));
  if (groups * G > resident) throw EotError{EOT_ERR_INVALID_ARG, "batched kernel does not fit"};
  const Layout Lo = layout(nprob, groups, G, maxN, maxM);
  if (Lo.total > h->bt_bytes) {
    EOT_CUDA(cudaStreamSynchronize(st));
    if (h->bt_mem) cudaFree(h->bt_mem);
    h->bt_mem = nullptr;
    h->bt_bytes = 0;
    EOT_CUDA(cudaMalloc(&h->bt_mem, Lo.total));
    h->bt_bytes = Lo.total;
  }
  unsigned char* b = (unsigned char*)h->bt_mem;
  for (Out& o : outs) {
    std::memset(&o, 0, sizeof(Out));
    o.status = EOT_ERR_DEVICE_TIMEOUT;  // stays so if a barrier wait ran out before the problem ended
  }
  EOT_CUDA(cudaMemcpyAsync(b + Lo.probs, probs.data(), sizeof(Prob) * nprob, cudaMemcpyHostToDevice, st));
  EOT_CUDA(cudaMemcpyAsync(b + Lo.outs, outs.data(), sizeof(Out) * nprob, cudaMemcpyHostToDevice, st));
  EOT_CUDA(cudaMemcpyAsync(b + Lo.order, order.data(), sizeof(int32_t) * nprob, cudaMemcpyHostToDevice, st));
  EOT_CUDA(cudaMemsetAsync(b + Lo.queue, 0, Lo.bar + sizeof(unsigned) * groups - Lo.queue, st));
  Launch L{};
  L.probs = (const Prob*)(b + Lo.probs);
  L.outs = (Out*)(b + Lo.outs);
  L.order = (const int32_t*)(b + Lo.order);
  L.nprob = nprob;
  L.G = G;
  L.ro = ro;
  L.queue = (int32_t*)(b + Lo.queue);
  L.abort = (int32_t*)(b + Lo.abort);
  L.bar = (unsigned*)(b + Lo.bar);
  L.part = (double*)(b + Lo.part);
  L.ipart = (int32_t*)(b + Lo.ipart);
  L.ws = b + Lo.ws;
  L.ws_stride = Lo.ws_stride;
  L.maxN = maxN;
  L.maxM = maxM;
  L.prm = prm;
  cudaEvent_t e0, e1;
  EOT_CUDA(cudaEventCreate(&e0));
  EOT_CUDA(cudaEventCreate(&e1));
  EOT_CUDA(cudaEventRecord(e0, st));
  void* args[] = {&L};
  const cudaError_t le = cudaLaunchCooperativeKernel((const void*)bt::batch_kernel<T>, dim3(groups * G),
                                                     dim3(kThreads), args, 0, st);
  EOT_CUDA(cudaEventRecord(e1, st));
  int32_t abort_flag = 0;
  EOT_CUDA(cudaMemcpyAsync(outs.data(), b + Lo.outs, sizeof(Out) * nprob, cudaMemcpyDeviceToHost, st));
  EOT_CUDA(cudaMemcpyAsync(&abort_flag, b + Lo.abort, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  EOT_CUDA(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (le != cudaSuccess) throw EotError{EOT_ERR_CUDA, std::string("batched launch: ") + cudaGetErrorString(le)};
  h->launches++;
  h->bt_last[0] = G;
  h->bt_last[1] = ro;
  h->bt_last[2] = groups;
  if (abort_flag) throw EotError{EOT_ERR_DEVICE_TIMEOUT, "batched kernel: a group barrier wait ran out"};
  return ms;
}

// Autotuner: times the probe (two column-fix + row LSE pairs per problem) of the
// actual batch for each candidate (G, elements per thread) and keeps the fastest.
template <class T>
std::pair<int, int> tune(eot_handle h, const std::vector<Prob>& probs, const std::vector<int32_t>& order,
                         bt::Params prm, int64_t maxN, int64_t maxM, cudaStream_t st) {
  const char* env = std::getenv("EOT_BATCH_CFG");
  if (env) {
    int G = 0, ro = 0;
    if (std::sscanf(env, "%d,%d", &G, &ro) == 2 && (G == 1 || G == 2 || G == 4 || G == 8) &&
        (ro == 1 || ro == 2 || ro == 4))
      return {G, ro};
  }
  std::string key = std::to_string(sizeof(T)) + ":";
  for (const Prob& p : probs) key += std::to_string(p.n) + "x" + std::to_string(p.m) + "x" + std::to_string(p.d) + ",";
  auto it = h->bt_tune.find(key);
  if (it != h->bt_tune.end()) return it->second;
  prm.probe = 2;
  std::vector<Out> outs(probs.size());
  const int resident = max_resident_ctas<T>(h);
  std::pair<int, int> best{2, 2};
  double best_ms = INFINITY;
  for (int G : {1, 2, 4, 8}) {
    if (G > resident) continue;
    for (int ro : {1, 2, 4}) {
      const double ms = launch_batch<T>(h, probs, order, outs, G, ro, prm, maxN, maxM, st);
      if (ms < best_ms) {
        best_ms = ms;
        best = {G, ro};
      }
    }
  }
  h->bt_tune[key] = best;
  return best;
}

template <class T>
eot_status run_batched(eot_handle h, int nprob, const eot_problem* P, const eot_params& prm_in,
                       double* const* u, double* const* v, int32_t* status_out, eot_stats* stats,
                       cudaStream_t st) {
  const double t0 = wall_seconds();
  std::vector<Prob> probs((size_t)nprob);
  int64_t maxN = 1, maxM = 1;
  for (int k = 0; k < nprob; ++k) {
    const eot_problem& q = P[k];
    Prob& b = probs[k];
    b.X = q.X;
    b.Y = q.Y;
    b.r = q.r;
    b.c = q.c;
    b.u = u[k];
    b.v = v[k];
    b.n = q.n;
    b.m = q.m;
    b.d = (int32_t)q.d;
    b.pad = 0;
    b.sC = q.cost_scale;
    maxN = std::max(maxN, q.n);
    maxM = std::max(maxM, q.m);
  }
  std::vector<int32_t> order((size_t)nprob);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return probs[a].n * probs[a].m > probs[b].n * probs[b].m;
  });
  bt::Params prm{};
  prm.gamma_i = prm_in.gamma_i;
  prm.gamma_f = prm_in.gamma_f;
  prm.p = prm_in.p;
  prm.q1 = prm_in.q1;
  prm.w_r = prm_in.w_r;
  prm.tol_final = prm_in.tol_final;
  prm.max_stages = prm_in.max_stages;
  prm.max_newton = prm_in.max_newton;
  prm.max_cg = prm_in.max_cg;
  prm.max_ls = prm_in.max_ls;
  prm.plain = 0;
  prm.probe = 0;
  const std::pair<int, int> cfg = tune<T>(h, probs, order, prm, maxN, maxM, st);
  std::vector<Out> outs((size_t)nprob);
  launch_batch<T>(h, probs, order, outs, cfg.first, cfg.second, prm, maxN, maxM, st);
  const double secs = wall_seconds() - t0;
  eot_status first = EOT_OK;
  for (int k = 0; k < nprob; ++k) {
    const Out& o = outs[k];
    if (status_out) status_out[k] = o.status;
    if (o.status != EOT_OK && first == EOT_OK) first = (eot_status)o.status;
    if (stats) {
      eot_stats& S = stats[k];
      std::memset(&S, 0, sizeof(S));
      S.sweeps_total = o.sweeps;
      S.stages = o.stages;
      S.newton_steps = o.newton_steps;
      S.cg_iters = o.cg_iters;
      S.cg_solves = o.cg_solves;
      S.ls_trials = o.ls_trials;
      S.sinkhorn_iters = o.sinkhorn_iters;
      S.curvature_stops = o.curvature_stops;
      S.final_gamma = o.final_gamma;
      S.final_rho = o.final_rho;
      S.grad_l1 = o.grad_l1;
      S.marg_err_l1 = o.marg_err_l1;
      S.seconds = secs;
    }
  }
  if (first != EOT_OK) h->err = "a problem of the batch failed (see the per-problem status)";
  return first;
}

}  // namespace

extern "C" eot_status eot_solve_batched(eot_handle h, int32_t nprob, const eot_problem* probs,
                                        const eot_params* params, double* const* u, double* const* v,
                                        int32_t* status_out, eot_stats* stats, void* stream) {
  if (!h) return EOT_ERR_INVALID_ARG;
  try {
    cudaGetLastError();  // a failed earlier call must not surface in this call's checks
    EOT_CUDA(cudaSetDevice(h->device));
    if (nprob < 0 || (nprob > 0 && (!probs || !params || !u || !v)))
      throw EotError{EOT_ERR_INVALID_ARG, "nprob >= 0; probs, params, u, v required"};
    if (nprob == 0) return EOT_OK;
    const int prec = probs[0].precision;
    for (int k = 0; k < nprob; ++k) {
      const eot_problem& q = probs[k];
      if (q.kind != EOT_COST_SQEUCLID_POINTS)
        throw EotError{EOT_ERR_UNSUPPORTED, "eot_solve_batched takes point-cloud problems"};
      if (q.precision != prec) throw EotError{EOT_ERR_INVALID_ARG, "all problems need the same precision"};
      if (q.n < 1 || q.m < 1 || q.n > kBatchMaxSide || q.m > kBatchMaxSide || q.d < 1 || q.d > bt::kDmax)
        throw EotError{EOT_ERR_INVALID_ARG, "batched problems: 1 <= n, m <= 32768 and 1 <= d <= 4"};
      if (!q.X || !q.Y || !q.r || !q.c || !u[k] || !v[k])
        throw EotError{EOT_ERR_INVALID_ARG, "X, Y, r, c, u[k], v[k] required"};
      if (!std::isfinite(q.cost_scale)) throw EotError{EOT_ERR_INVALID_ARG, "cost_scale must be finite"};
    }
    const eot_params& prm = *params;
    if (!(prm.gamma_i > 0.0) || !(prm.gamma_f > 0.0) || prm.gamma_f >= kSplitLimit)
      throw EotError{EOT_ERR_INVALID_ARG, "0 < gamma_i, 0 < gamma_f < 2^19"};
    if (prm.projector != EOT_PROJECT_NEWTON)
      throw EotError{EOT_ERR_INVALID_ARG, "batched solves use the Newton projector (Alg. 4)"};
    const cudaStream_t st = (cudaStream_t)stream;
    if (prec == EOT_PREC_FP64) return run_batched<double>(h, nprob, probs, prm, u, v, status_out, stats, st);
    if (prec == EOT_PREC_MIXED) return run_batched<float>(h, nprob, probs, prm, u, v, status_out, stats, st);
    throw EotError{EOT_ERR_UNSUPPORTED, "eot_solve_batched: precision MIXED or FP64"};
  } catch (const EotError& e) {
    h->err = e.msg;
    return e.st;
  } catch (...) {
    h->err = "unknown error";
    return EOT_ERR_CUDA;
  }
}

extern "C" eot_status eot_batch_last_config(eot_handle h, int32_t* out3) {
  if (!h || !out3) return EOT_ERR_INVALID_ARG;
  for (int k = 0; k < 3; ++k) out3[k] = h->bt_last[k];
  return EOT_OK;
}
