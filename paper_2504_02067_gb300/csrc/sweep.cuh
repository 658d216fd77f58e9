// Tile sweeps over the implicit plan (Sec. 2.1 Eq. lagrangian-closed-form and the
// "primitive operations" of Appx. D): one pass over the cost matrix, forming
// E_ij = exp(Ah_i + Bh_j - gamma C_ij) tile by tile in registers and reducing it
// along rows and/or columns. Every O(n^2) operation of the solver (HVP halves,
// marginals, the Jacobi diagonal, the LSE updates of Alg. 3 / Alg. 4) is one of
// these sweeps with a different reduction and epilogue.
//
// Row sweep   : each warp owns whole rows; lanes stride the row with 16-byte
//               loads; per-lane FP32 partials are flushed to FP64 every U*V
//               entries and combined with FP64 shuffles. No cross-CTA traffic.
// Column sweep: CTA (strip s, row block b) owns 32*V columns x BR rows; per-lane
//               FP32 column partials are combined across warps in FP64 and
//               written to a [R x m] partial array; the last CTA of each strip
//               (atomic ticket) adds the R partials in fixed order, so results
//               are bit-reproducible and no float atomics are used.
// Both kernels optionally compute an online (max, sum) log-sum-exp instead of a
// plain sum; the running max lives on the 1/8 grid so that (Ah - max) stays
// exact and t - max is rounded once, relative to its own (small) magnitude.
#pragma once
#include "common.cuh"

namespace eot {

template <class T>
struct SweepArgs {
  const T* C;           // n x m row-major cost, leading dimension ldc (elements)
  int64_t n, m, ldc;
  const T* Ah;          // [n] high part of the row offsets
  const T* Bh;          // [m] high part of the column offsets
  const T* wc[3];       // [m] column weights of row reductions
  const T* wr[2];       // [n] row weights of column reductions
  T gamma;
  double* colpart;      // [NC or 2][R][m] column partials
  double* rowpart;      // [NR][S][n] row partials (column sweep with row reductions)
  int* cnt_strip;       // [S] tickets of the column finalize
  int* cnt_rowblk;      // [R] tickets of the row finalize
  double* dotpart;      // [>= max(grid.x, S)][2] epilogue partial sums
  int* cnt_dot;         // [1] ticket of the epilogue finish
  int rows_per_block;   // BR (column sweep)
  int nrowblk;          // R  (column sweep)
  const double* gamma_dev;  // nullable: read gamma here (keeps captured graphs valid)
  const double* active;     // nullable: the kernel does nothing while *active == 0
};

template <int N>
struct DotArr {
  double v[N > 0 ? N : 1];
};

// ----------------------------------------------------------------------------
// CTA-level deterministic sum of per-warp epilogue contributions, then a ticket
// so that the last CTA calls epi.finish with the totals over all CTAs.
// ----------------------------------------------------------------------------
template <int ND, class Epi>
__device__ __forceinline__ void cta_dot_finish(double (&wd)[ND > 0 ? ND : 1], int64_t part_idx,
                                               int64_t nparts, double* dotpart, int* cnt,
                                               Epi& epi) {
  if constexpr (ND > 0) {
    __shared__ double sd[kWarps][ND];
    __shared__ int last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < ND; ++k) sd[warp][k] = wd[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < ND; ++k) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += sd[w][k];
        dotpart[part_idx * 2 + k] = t;
      }
      __threadfence();
      last = (atomicAdd(cnt, 1) == (int)nparts - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
      __threadfence();
      DotArr<ND> tot;
#pragma unroll
      for (int k = 0; k < ND; ++k) tot.v[k] = 0.0;
      for (int64_t p = 0; p < nparts; ++p) {
#pragma unroll
        for (int k = 0; k < ND; ++k) tot.v[k] += __ldcg(dotpart + p * 2 + k);
      }
      *cnt = 0;
      epi.finish(tot.v);
    }
  }
}

// ----------------------------------------------------------------------------
// Row sweep: out_i = reduce_j E_ij * wc_k[j] (NR = 1..3 reductions; bit k of SQM
// makes reduction k use E_ij^2), or the online LSE of (t_ij + log wc_0[j]).
// ----------------------------------------------------------------------------
template <class T, int V, int NR, bool LSE, int SQM, class Epi>
__global__ void __launch_bounds__(kThreads) row_sweep_kernel(SweepArgs<T> a, Epi epi) {
  constexpr int U = 4;  // chunks per lane in flight
  constexpr int ND = Epi::kDot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (a.active && *a.active == 0.0) return;
  double wd[ND > 0 ? ND : 1];
#pragma unroll
  for (int k = 0; k < (ND > 0 ? ND : 1); ++k) wd[k] = 0.0;
  const T g = a.gamma_dev ? (T)*a.gamma_dev : a.gamma;
  const int64_t wstride = (int64_t)gridDim.x * kWarps;
  for (int64_t i = (int64_t)blockIdx.x * kWarps + warp; i < a.n; i += wstride) {
    const T* crow = a.C + i * a.ldc;
    const T ah = a.Ah[i];
    if constexpr (!LSE) {
      double tot[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) tot[k] = 0.0;
      for (int64_t j0 = (int64_t)lane * V; j0 < a.m; j0 += 32 * V * U) {
        T c[U][V], b[U][V], w[NR][U][V];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t j = j0 + (int64_t)u * 32 * V;
          ok[u] = j < a.m;
          if (ok[u]) {
            ld_stream(crow + j, c[u]);
            ld_vec<V>(a.Bh + j, b[u]);
#pragma unroll
            for (int k = 0; k < NR; ++k) ld_vec<V>(a.wc[k] + j, w[k][u]);
          }
        }
        T acc[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) acc[k] = T(0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (!ok[u]) continue;
#pragma unroll
          for (int e = 0; e < V; ++e) {
            const T t = fmaT(-g, c[u][e], ah + b[u][e]);
            const T x = expT(t);
#pragma unroll
            for (int k = 0; k < NR; ++k) {
              if ((SQM >> k) & 1) acc[k] = fmaT(x * x, w[k][u][e], acc[k]);
              else acc[k] = fmaT(x, w[k][u][e], acc[k]);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < NR; ++k) tot[k] += (double)acc[k];
      }
#pragma unroll
      for (int k = 0; k < NR; ++k) tot[k] = warp_sum(tot[k]);
      if (lane == 0) {
        DotArr<ND> d;
        epi.row(i, tot, d.v);  // tot: [NR] sums
#pragma unroll
        for (int k = 0; k < ND; ++k) wd[k] += d.v[k];
      }
    } else {
      // online log-sum-exp of t_ij + log w_j with a lazily moved running max mx.
      // mx starts at 0 (so am = ah is exact) and stays on the 1/8 grid; it moves
      // up when t > theta, and onto the element while nothing is accumulated yet
      // (t < -kLow), so that no dominant term can underflow.
      T mx = T(0);
      T am = ah;
      T s = T(0);
      double S = 0.0;           // flushed part of s, relative to mx
      for (int64_t j0 = (int64_t)lane * V; j0 < a.m; j0 += 32 * V * U) {
        T c[U][V], b[U][V], w0[U][V];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t j = j0 + (int64_t)u * 32 * V;
          ok[u] = j < a.m;
          if (ok[u]) {
            ld_stream(crow + j, c[u]);
            ld_vec<V>(a.Bh + j, b[u]);
            ld_vec<V>(a.wc[0] + j, w0[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (!ok[u]) continue;
#pragma unroll
          for (int e = 0; e < V; ++e) {
            T t = fmaT(-g, c[u][e], am + b[u][e]);
            // move the running max; at most 4 steps (a non-finite or huge t
            // leaves the loop unchanged and shows up as a non-finite sum)
            for (int k = 0; k < 4 && (t > T(kTheta) || (t < T(-kLow) && s == T(0) && S == 0.0)); ++k) {
              const T dlt = ceil_grid(t);
              mx += dlt;
              am = ah - mx;
              if (dlt > T(0)) {
                const T f = expT(-dlt);
                s *= f;
                S *= (double)f;
              }
              t = fmaT(-g, c[u][e], am + b[u][e]);
            }
            s = fmaT(expT(t), w0[u][e], s);
          }
        }
        S += (double)s;
        s = T(0);
      }
      LsePair p{(double)mx, S};
      p = warp_lse(p);
      if (lane == 0) {
        DotArr<ND> d;
        epi.row_lse(i, p.m, p.s, d.v);
#pragma unroll
        for (int k = 0; k < ND; ++k) wd[k] += d.v[k];
      }
    }
  }
  cta_dot_finish<ND>(wd, blockIdx.x, gridDim.x, a.dotpart, a.cnt_dot, epi);
}

// ----------------------------------------------------------------------------
// Column sweep: out_j = reduce_i E_ij * wr_k[i] (NC = 1 or 2), or the online LSE
// of (t_ij + log wr_0[i]). Optional NR row reductions (with column weights wc_k)
// give the fused two-sided sweep of the Hessian-vector product.
// grid = (S strips of 32*V columns, R row blocks of BR rows).
// ----------------------------------------------------------------------------
template <class T, int V, int NC, bool LSE, int NR, class Epi>
__global__ void __launch_bounds__(kThreads) col_sweep_kernel(SweepArgs<T> a, Epi epi) {
  constexpr int U = 4;  // rows per warp in flight
  constexpr int SW = 32 * V;
  constexpr int ND = Epi::kDot;
  constexpr int NP = LSE ? 2 : NC;  // partial arrays
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t strip = blockIdx.x;
  const int rb = blockIdx.y;
  const int64_t S = gridDim.x;
  const int R = a.nrowblk;
  const int64_t j = strip * SW + (int64_t)lane * V;
  const bool jv = j < a.m;
  const int64_t r0 = (int64_t)rb * a.rows_per_block;
  const int64_t r1 = min(a.n, r0 + (int64_t)a.rows_per_block);
  if (a.active && *a.active == 0.0) return;
  const T g = a.gamma_dev ? (T)*a.gamma_dev : a.gamma;

  T b[V], wcv[2][V];
#pragma unroll
  for (int e = 0; e < V; ++e) { b[e] = T(0); wcv[0][e] = T(0); wcv[1][e] = T(0); }
  if (jv) {
    ld_vec<V>(a.Bh + j, b);
    if constexpr (NR > 0) ld_vec<V>(a.wc[0] + j, wcv[0]);
    if constexpr (NR > 1) ld_vec<V>(a.wc[1] + j, wcv[1]);
  }
  double tot[NP][V];
#pragma unroll
  for (int k = 0; k < NP; ++k)
#pragma unroll
    for (int e = 0; e < V; ++e) tot[k][e] = 0.0;
  // LSE state per column: running max mx (on the grid, starting at 0) and bm = Bh - mx
  T mx[V], bm[V];
  if constexpr (LSE) {
#pragma unroll
    for (int e = 0; e < V; ++e) { mx[e] = T(0); bm[e] = b[e]; }
  }

  for (int64_t i0 = r0 + warp; i0 < r1; i0 += (int64_t)kWarps * U) {
    T c[U][V], ah[U], x0[U], x1[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + (int64_t)u * kWarps;
      ok[u] = i < r1;
      if (ok[u]) {
        ah[u] = a.Ah[i];
        x0[u] = a.wr[0][i];
        if constexpr (NC > 1) x1[u] = a.wr[1][i];
        if (jv) ld_stream(a.C + i * a.ldc + j, c[u]);
        else {
#pragma unroll
          for (int e = 0; e < V; ++e) c[u][e] = T(0);
        }
      }
    }
    T acc[NP][V];
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
      for (int e = 0; e < V; ++e) acc[k][e] = T(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      T racc0 = T(0), racc1 = T(0);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        if constexpr (!LSE) {
          const T t = fmaT(-g, c[u][e], ah[u] + b[e]);
          const T x = jv ? expT(t) : T(0);
          acc[0][e] = fmaT(x, x0[u], acc[0][e]);
          if constexpr (NC > 1) acc[1][e] = fmaT(x, x1[u], acc[1][e]);
          if constexpr (NR > 0) racc0 = fmaT(x, wcv[0][e], racc0);
          if constexpr (NR > 1) racc1 = fmaT(x, wcv[1][e], racc1);
        } else {
          if (jv) {
            T t = fmaT(-g, c[u][e], ah[u] + bm[e]);
            // bounded, as in the row sweep
            for (int k = 0; k < 4 && (t > T(kTheta) ||
                                      (t < T(-kLow) && acc[1][e] == T(0) && tot[1][e] == 0.0)); ++k) {
              const T dlt = ceil_grid(t);
              mx[e] += dlt;
              bm[e] = b[e] - mx[e];
              if (dlt > T(0)) {
                const T f = expT(-dlt);
                acc[1][e] *= f;  // unflushed part
                tot[1][e] *= (double)f;
              }
              t = fmaT(-g, c[u][e], ah[u] + bm[e]);
            }
            acc[1][e] = fmaT(expT(t), x0[u], acc[1][e]);
          }
        }
      }
      if constexpr (NR > 0) {
        double rs0 = warp_sum((double)racc0);
        double rs1 = 0.0;
        if constexpr (NR > 1) rs1 = warp_sum((double)racc1);
        if (lane == 0) {
          const int64_t i = i0 + (int64_t)u * kWarps;
          a.rowpart[(0 * S + strip) * a.n + i] = rs0;
          if constexpr (NR > 1) a.rowpart[(1 * S + strip) * a.n + i] = rs1;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
      for (int e = 0; e < V; ++e) tot[k][e] += (double)acc[k][e];
  }

  // ---- combine the 8 warps of this CTA in FP64 and write the [R][m] partials ----
  __shared__ double sred[NP][kWarps][SW];
  __shared__ double smax[LSE ? kWarps : 1][LSE ? SW : 1];
#pragma unroll
  for (int k = 0; k < NP; ++k)
#pragma unroll
    for (int e = 0; e < V; ++e) sred[k][warp][lane * V + e] = tot[k][e];
  if constexpr (LSE) {
#pragma unroll
    for (int e = 0; e < V; ++e) smax[warp][lane * V + e] = (double)mx[e];
  }
  __syncthreads();
  for (int cc = threadIdx.x; cc < SW; cc += kThreads) {
    const int64_t jj = strip * SW + cc;
    if (jj >= a.m) continue;
    if constexpr (!LSE) {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += sred[k][w][cc];
        a.colpart[((int64_t)k * R + rb) * a.m + jj] = t;
      }
    } else {
      LsePair p{0.0, 0.0};
      for (int w = 0; w < kWarps; ++w) p = lse_combine(p, LsePair{smax[w][cc], sred[1][w][cc]});
      a.colpart[((int64_t)0 * R + rb) * a.m + jj] = p.m;
      a.colpart[((int64_t)1 * R + rb) * a.m + jj] = p.s;
    }
  }

  // ---- tickets: the last CTA of the strip combines the R partials ----
  __shared__ int last_strip, last_rows;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last_strip = (atomicAdd(a.cnt_strip + strip, 1) == R - 1);
    if constexpr (NR > 0) last_rows = (atomicAdd(a.cnt_rowblk + rb, 1) == (int)S - 1);
  }
  __syncthreads();
  if (last_strip) {
    __threadfence();
    double wd[ND > 0 ? ND : 1];
#pragma unroll
    for (int k = 0; k < (ND > 0 ? ND : 1); ++k) wd[k] = 0.0;
    for (int cc = threadIdx.x; cc < SW; cc += kThreads) {
      const int64_t jj = strip * SW + cc;
      if (jj >= a.m) continue;
      DotArr<ND> d;
      if constexpr (!LSE) {
        double s[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          double t = 0.0;
          for (int r = 0; r < R; ++r) t += __ldcg(a.colpart + ((int64_t)k * R + r) * a.m + jj);
          s[k] = t;
        }
        epi.col(jj, s, d.v);
      } else {
        LsePair p{0.0, 0.0};
        for (int r = 0; r < R; ++r)
          p = lse_combine(p, LsePair{__ldcg(a.colpart + (int64_t)r * a.m + jj),
                                     __ldcg(a.colpart + ((int64_t)R + r) * a.m + jj)});
        epi.col_lse(jj, p.m, p.s, d.v);
      }
#pragma unroll
      for (int k = 0; k < ND; ++k) wd[k] += d.v[k];
    }
    if (threadIdx.x == 0) a.cnt_strip[strip] = 0;
    if constexpr (ND > 0) {
      // per-warp sums, then the strip-level partial and the global ticket
#pragma unroll
      for (int k = 0; k < ND; ++k) wd[k] = warp_sum(wd[k]);
      cta_dot_finish<ND>(wd, strip, S, a.dotpart, a.cnt_dot, epi);
    }
  }
  if constexpr (NR > 0) {
    if (last_rows) {
      __threadfence();
      for (int64_t i = r0 + threadIdx.x; i < r1; i += kThreads) {
        double s[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          double t = 0.0;
          for (int64_t q = 0; q < S; ++q) t += __ldcg(a.rowpart + ((int64_t)k * S + q) * a.n + i);
          s[k] = t;
        }
        epi.row_part(i, s);
      }
      if (threadIdx.x == 0) a.cnt_rowblk[rb] = 0;
    }
  }
}

}  // namespace eot
