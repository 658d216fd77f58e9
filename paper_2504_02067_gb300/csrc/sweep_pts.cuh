// Sweeps over the implicit plan of a point-cloud problem: the cost
// C_ij = s_C |x_i - y_j|^2 is formed on the fly from the points and never stored
// (the O(n)-memory variant of Sec. 4.2). The exponent is
//     t_ij = Ah_i + Bh_j - K D_ij,   D_ij = sum_k (x_ik - y_jk)^2,   K = gamma s_C,
// with D from direct coordinate differences (accurate for the near pairs that
// carry the plan's mass) and K split into an FP32 high part and an FP32 low
// correction, so that the FP32 exponent keeps a single rounding of K D.
//
// One kernel serves row sweeps (reductions over j for each row i) and column
// sweeps (over i for each column j): t is symmetric in the two sides, so each
// thread OWNS RO elements of the side being reduced (their coordinates in
// registers) and reads the OTHER side from shared-memory tiles (broadcasts).
// grid = (own blocks of 256 * RO elements, S chunks of the other side); each
// chunk writes FP64 partials [S][n_own], and the last CTA of each own block
// (atomic ticket) adds the S partials in fixed order and calls the epilogue.
#pragma once
#include "sweep.cuh"

namespace eot {

// FP32 terms summed plainly before each compensated (Neumaier) flush: a plain
// FP32 sum of k positive terms is off by up to ~k 2^-24 relative, which at k = 256
// is already the 1e-6 scale of the marginal tolerance.
constexpr int kPtsFlush = 16;
constexpr int kPtsMaxPartials = 3;  // widest point sweep: three sums per owned element

template <class T>
__device__ __forceinline__ void split_k(double K, T& hi, T& lo) {
  hi = (T)K;
  lo = (T)(K - (double)hi);
}

// Squared distance as an unevaluated sum Dh + Dl. With PRECISE (FP32 mixed path)
// the coordinate differences are exact (Knuth's TwoSum), the squares exact (FMA
// error term) and the accumulation compensated, so Dh + Dl carries D to about
// 2^-44 relative: the product K D can reach hundreds and the exponent needs it
// to ~1e-8. Without PRECISE (plain FP32, and FP64 where it is not needed) Dl = 0.
// Round-to-nearest add / multiply that the compiler never contracts into an
// FMA: the error-free transformations below need every rounding where written.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

template <bool PRECISE, class T, int DMAX, class YGet>
__device__ __forceinline__ void dist2(const T (&x)[DMAX], YGet yk, T& Dh, T& Dl) {
  Dh = T(0);
  Dl = T(0);
#pragma unroll
  for (int k = 0; k < DMAX; ++k) {
    const T y = yk(k);
    if constexpr (!PRECISE) {
      const T sd = x[k] - y;
      Dh = fmaT(sd, sd, Dh);
    } else {
      const T sd = sub_rn(x[k], y);                                  // TwoSum: x - y = sd + e
      const T bv = sub_rn(sd, x[k]);
      const T e = sub_rn(sub_rn(x[k], sub_rn(sd, bv)), add_rn(y, bv));
      const T p = mul_rn(sd, sd);                                    // TwoProduct: sd^2 = p + pe
      const T pe = fmaT(sd, sd, -p);
      const T t = add_rn(Dh, p);                                     // TwoSum: Dh + p = t + err
      const T z = sub_rn(t, Dh);
      const T err = add_rn(sub_rn(Dh, sub_rn(t, z)), sub_rn(p, z));
      Dh = t;
      Dl += err + fmaT(sd + sd, e, pe);                              // (sd + e)^2 - sd^2 to first order
    }
  }
}

// t = h - K (Dh + Dl) with K = Kh + Kl: the large product Kh Dh is exact inside the
// first FMA, so t is rounded about once relative to its own size.
template <bool PRECISE, class T>
__device__ __forceinline__ T expo(T h, T Kh, T Kl, T Dh, T Dl) {
  T t = fmaT(-Kh, Dh, h);
  if constexpr (PRECISE) t = fmaT(-Kh, Dl, t);
  return fmaT(-Kl, Dh, t);
}

template <class T, int DMAX, int RO, int NR, bool LSE, int SQM, bool ROWS, bool PRECISE, class Epi>
__global__ void __launch_bounds__(kThreads, 2) pts_sweep_kernel(SweepArgs<T> a, Epi epi) {
  // other-side elements per shared-memory tile (<= 16 KB of coordinates)
  constexpr int TO = (DMAX * (int)sizeof(T) * 256 <= 16384) ? 256 : 16384 / (DMAX * (int)sizeof(T));
  constexpr int NA = LSE ? 1 : NR;       // accumulators per owned element
  constexpr int NW = LSE ? 1 : NR;       // staged weight vectors
  constexpr int ND = Epi::kDot;
  __shared__ T sy[DMAX][TO];
  __shared__ T sh[TO];
  __shared__ T sw[NW][TO];
  __shared__ int last_blk;

  const int64_t n_own = ROWS ? a.n : a.m, n_oth = ROWS ? a.m : a.n;
  const float* xo = ROWS ? a.X : a.Y;
  const float* xt = ROWS ? a.Y : a.X;
  const int d = a.d;
  const int64_t blk = blockIdx.x, s = blockIdx.y, S = gridDim.y;
  const int64_t j0 = s * a.chunk, j1 = min(n_oth, j0 + a.chunk);
  pdl_wait();
  if (a.active && *a.active == 0.0) return;
  const T* ho = ROWS ? a.Ah : a.Bh;
  const T* ht = ROWS ? a.Bh : a.Ah;
  const T g = a.gamma_dev ? (T)*a.gamma_dev : a.gamma;
  T Kh, Kl;
  split_k<T>((double)g * a.sC, Kh, Kl);

  // owned elements, their coordinates and offsets
  int64_t e[RO];
  bool ev[RO];
  T x[RO][DMAX], h[RO];
#pragma unroll
  for (int r = 0; r < RO; ++r) {
    e[r] = blk * (int64_t)kThreads * RO + r * kThreads + threadIdx.x;
    ev[r] = e[r] < n_own;
    h[r] = ev[r] ? ho[e[r]] : T(0);
#pragma unroll
    for (int k = 0; k < DMAX; ++k) x[r][k] = (ev[r] && k < d) ? (T)xo[e[r] * d + k] : T(0);
  }
  T Sa[RO][NA], Ca[RO][NA];
  T mx[RO], hm[RO];  // LSE: running max (1/8 grid) and h - max
  bool mx_set[RO];
#pragma unroll
  for (int r = 0; r < RO; ++r) {
    mx[r] = T(0);
    hm[r] = h[r];
    mx_set[r] = false;
#pragma unroll
    for (int k = 0; k < NA; ++k) { Sa[r][k] = T(0); Ca[r][k] = T(0); }
  }

  for (int64_t jt = j0; jt < j1; jt += TO) {
    const int tn = (int)min((int64_t)TO, j1 - jt);
    __syncthreads();
    for (int q = threadIdx.x; q < tn; q += kThreads) {
      const int64_t j = jt + q;
      sh[q] = ht[j];
#pragma unroll
      for (int k = 0; k < NW; ++k) sw[k][q] = ROWS ? a.wc[k][j] : a.wr[k][j];
#pragma unroll
      for (int k = 0; k < DMAX; ++k) sy[k][q] = k < d ? (T)xt[j * d + k] : T(0);
    }
    __syncthreads();
    for (int q0 = 0; q0 < tn; q0 += kPtsFlush) {
    const int q1 = min(tn, q0 + kPtsFlush);
    T acc[RO][NA];
#pragma unroll
    for (int r = 0; r < RO; ++r)
#pragma unroll
      for (int k = 0; k < NA; ++k) acc[r][k] = T(0);
#pragma unroll 2
    for (int q = q0; q < q1; ++q) {
      constexpr bool YREG = DMAX <= 16;  // keep the other point in registers for small d
      T y[YREG ? DMAX : 1];
      if constexpr (YREG) {
#pragma unroll
        for (int k = 0; k < DMAX; ++k) y[k] = sy[k][q];
      }
      const T hb = sh[q];
      T w[NW];
#pragma unroll
      for (int k = 0; k < NW; ++k) w[k] = sw[k][q];
#pragma unroll
      for (int r = 0; r < RO; ++r) {
        T Dh, Dl;
        dist2<PRECISE, T, DMAX>(x[r], [&](int k) { if constexpr (YREG) return y[k]; else return sy[k][q]; },
                                Dh, Dl);
        if constexpr (!LSE) {
          const T ex = expT(expo<PRECISE>(h[r] + hb, Kh, Kl, Dh, Dl));
#pragma unroll
          for (int k = 0; k < NR; ++k) {
            if ((SQM >> k) & 1) acc[r][k] = fmaT(ex * ex, w[k], acc[r][k]);
            else acc[r][k] = fmaT(ex, w[k], acc[r][k]);
          }
        } else {
          if (!mx_set[r]) {
            // start the running max at the first element (see the dense row sweep)
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
          acc[r][0] = fmaT(expT(t), w[0], acc[r][0]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RO; ++r)
#pragma unroll
      for (int k = 0; k < NA; ++k) kadd(Sa[r][k], Ca[r][k], acc[r][k]);
    }
  }
  pdl_trigger();

  // ---- partials [NP][S][n_own], then the last CTA of this own block combines ----
  constexpr int NP = LSE ? 2 : NR;
#pragma unroll
  for (int r = 0; r < RO; ++r) {
    if (!ev[r]) continue;
    if constexpr (!LSE) {
#pragma unroll
      for (int k = 0; k < NR; ++k)
        a.rowpart[((int64_t)k * S + s) * n_own + e[r]] = (double)Sa[r][k] + (double)Ca[r][k];
    } else {
      a.rowpart[((int64_t)0 * S + s) * n_own + e[r]] = (double)mx[r];
      a.rowpart[((int64_t)1 * S + s) * n_own + e[r]] = (double)Sa[r][0] + (double)Ca[r][0];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last_blk = (atomicAdd(a.cnt_rowblk + blk, 1) == (int)S - 1);
  }
  __syncthreads();
  if (!last_blk) return;
  __threadfence();
  double wd[ND > 0 ? ND : 1];
#pragma unroll
  for (int k = 0; k < (ND > 0 ? ND : 1); ++k) wd[k] = 0.0;
#pragma unroll
  for (int r = 0; r < RO; ++r) {
    if (!ev[r]) continue;
    DotArr<ND> dd;
    if constexpr (!LSE) {
      double tot[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        double v = 0.0;
        ordered_loads(a.rowpart + (int64_t)k * S * n_own + e[r], n_own, S, [&](double q) { v += q; });
        tot[k] = v;
      }
      if constexpr (ROWS) epi.row(e[r], tot, dd.v);
      else epi.col(e[r], tot, dd.v);
    } else {
      LsePair p{0.0, 0.0};
      ordered_loads2(a.rowpart + e[r], a.rowpart + S * n_own + e[r], n_own, S,
                     [&](double qm, double qs) { p = lse_combine<T>(p, LsePair{qm, qs}); });
      if constexpr (ROWS) epi.row_lse(e[r], p.m, p.s, dd.v);
      else epi.col_lse(e[r], p.m, p.s, dd.v);
    }
#pragma unroll
    for (int k = 0; k < ND; ++k) wd[k] += dd.v[k];
  }
  if (threadIdx.x == 0) a.cnt_rowblk[blk] = 0;
  if constexpr (ND > 0) {
#pragma unroll
    for (int k = 0; k < ND; ++k) wd[k] = warp_sum(wd[k]);
    cta_dot_finish<ND>(wd, blk, gridDim.x, a.dotpart, a.cnt_dot, epi);
  }
}

// Gradient of the EOT value with respect to the owned points (envelope theorem
// on the Lagrangian of Appx. A, with s_C held constant):
//     out_e,k = scale * ownfac_e * sum_o exp(h_e + h_o - K D_eo) w_o (x_ek - x_ok)
// for the components k0 <= k < k0 + DG, where ownfac_e * exp(h_e + h_o - K D) w_o
// = P_eo with the owned side shifted by its own log-marginal (so every exponent
// is <= 0 up to the 1/8 grid). ROWS: own = rows (dX); else own = columns (dY).
// grid = (own blocks of 256, S chunks of the other side); FP64 partials
// [DG][S][n_own], last CTA of each own block adds them in fixed order.
template <class T, int DMAX, int DG, bool ROWS, bool PRECISE>
__global__ void __launch_bounds__(kThreads, DMAX > 16 ? 1 : 2)
    pts_grad_kernel(SweepArgs<T> a, int k0, double scale, const double* ownfac, float* out) {
  constexpr int TO = (DMAX * (int)sizeof(T) * 256 <= 16384) ? 256 : 16384 / (DMAX * (int)sizeof(T));
  __shared__ T sy[DMAX][TO];
  __shared__ T sh[TO];
  __shared__ T sw[TO];
  __shared__ int last_blk;

  const int64_t n_own = ROWS ? a.n : a.m, n_oth = ROWS ? a.m : a.n;
  const float* xo = ROWS ? a.X : a.Y;
  const float* xt = ROWS ? a.Y : a.X;
  const int d = a.d;
  const int64_t blk = blockIdx.x, s = blockIdx.y, S = gridDim.y;
  const int64_t j0 = s * a.chunk, j1 = min(n_oth, j0 + a.chunk);
  pdl_wait();
  const T* ho = ROWS ? a.Ah : a.Bh;
  const T* ht = ROWS ? a.Bh : a.Ah;
  const T* wt = ROWS ? a.wc[0] : a.wr[0];
  const T g = a.gamma_dev ? (T)*a.gamma_dev : a.gamma;
  T Kh, Kl;
  split_k<T>((double)g * a.sC, Kh, Kl);

  const int64_t e = blk * (int64_t)kThreads + threadIdx.x;
  const bool ev = e < n_own;
  const T h = ev ? ho[e] : T(0);
  T x[DMAX], xg[DG];
#pragma unroll
  for (int k = 0; k < DMAX; ++k) x[k] = (ev && k < d) ? (T)xo[e * d + k] : T(0);
#pragma unroll
  for (int k = 0; k < DG; ++k) xg[k] = (ev && k0 + k < d) ? (T)xo[e * d + k0 + k] : T(0);
  T Sa[DG], Ca[DG];
#pragma unroll
  for (int k = 0; k < DG; ++k) { Sa[k] = T(0); Ca[k] = T(0); }

  for (int64_t jt = j0; jt < j1; jt += TO) {
    const int tn = (int)min((int64_t)TO, j1 - jt);
    __syncthreads();
    for (int q = threadIdx.x; q < tn; q += kThreads) {
      const int64_t j = jt + q;
      sh[q] = ht[j];
      sw[q] = wt[j];
#pragma unroll
      for (int k = 0; k < DMAX; ++k) sy[k][q] = k < d ? (T)xt[j * d + k] : T(0);
    }
    __syncthreads();
    for (int q0 = 0; q0 < tn; q0 += kPtsFlush) {
      const int q1 = min(tn, q0 + kPtsFlush);
      T acc[DG];
#pragma unroll
      for (int k = 0; k < DG; ++k) acc[k] = T(0);
      for (int q = q0; q < q1; ++q) {
        T Dh, Dl;
        dist2<PRECISE, T, DMAX>(x, [&](int k) { return sy[k][q]; }, Dh, Dl);
        const T pw = expT(expo<PRECISE>(h + sh[q], Kh, Kl, Dh, Dl)) * sw[q];
#pragma unroll
        for (int k = 0; k < DG; ++k) acc[k] = fmaT(pw, xg[k] - sy[k0 + k][q], acc[k]);
      }
#pragma unroll
      for (int k = 0; k < DG; ++k) kadd(Sa[k], Ca[k], acc[k]);
    }
  }
  pdl_trigger();

  if (ev) {
#pragma unroll
    for (int k = 0; k < DG; ++k) a.rowpart[((int64_t)k * S + s) * n_own + e] = (double)Sa[k] + (double)Ca[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last_blk = (atomicAdd(a.cnt_rowblk + blk, 1) == (int)S - 1);
  }
  __syncthreads();
  if (!last_blk) return;
  __threadfence();
  if (ev) {
    const double f = scale * ownfac[e];
#pragma unroll
    for (int k = 0; k < DG; ++k) {
      if (k0 + k >= d) break;
      double v = 0.0;
      ordered_loads(a.rowpart + (int64_t)k * S * n_own + e, n_own, S, [&](double q) { v += q; });
      out[e * d + k0 + k] = (float)(f * v);
    }
  }
  if (threadIdx.x == 0) a.cnt_rowblk[blk] = 0;
}

// Largest squared distance max_ij |x_i - y_j|^2 (the cost normalisation of
// Sec. 4.1 for point costs): each thread scans its rows against a tile of
// columns in FP32, keeps its arg-max pair, re-evaluates that pair in FP64, and
// writes the CTA's FP64 maximum to out[blockIdx.y * gridDim.x + blockIdx.x].
template <int DMAX>
__global__ void __launch_bounds__(kThreads) pts_maxdist_kernel(const float* X, const float* Y,
                                                               int64_t n, int64_t m, int d,
                                                               int64_t chunk, double* out) {
  constexpr int TO = 256;
  __shared__ float sy[DMAX][TO];
  __shared__ double sbest[kThreads];
  pdl_wait();
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool iv = i < n;
  float x[DMAX];
#pragma unroll
  for (int k = 0; k < DMAX; ++k) x[k] = (iv && k < d) ? X[i * d + k] : 0.f;
  const int64_t j0 = (int64_t)blockIdx.y * chunk, j1 = min(m, j0 + chunk);
  float best = -1.f;
  int64_t bj = -1;
  for (int64_t jt = j0; jt < j1; jt += TO) {
    const int tn = (int)min((int64_t)TO, j1 - jt);
    __syncthreads();
    for (int q = threadIdx.x; q < tn; q += kThreads)
#pragma unroll
      for (int k = 0; k < DMAX; ++k) sy[k][q] = k < d ? Y[(jt + q) * d + k] : 0.f;
    __syncthreads();
    for (int q = 0; q < tn; ++q) {
      float D = 0.f;
#pragma unroll
      for (int k = 0; k < DMAX; ++k) {
        const float df = x[k] - sy[k][q];
        D = fmaf(df, df, D);
      }
      if (D > best) {
        best = D;
        bj = jt + q;
      }
    }
  }
  double b64 = -1.0;
  if (iv && bj >= 0) {
    b64 = 0.0;
    for (int k = 0; k < d; ++k) {
      const double df = (double)X[i * d + k] - (double)Y[bj * d + k];
      b64 += df * df;
    }
  }
  sbest[threadIdx.x] = b64;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mxv = -1.0;
    for (int t = 0; t < kThreads; ++t) mxv = fmax(mxv, sbest[t]);
    out[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = mxv;
  }
}

}  // namespace eot
