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
#include <type_traits>

#include "common.cuh"

namespace eot {

template <class T>
struct SweepArgs {
  const T* C;           // n x m row-major cost, leading dimension ldc (elements)
  int64_t n, m, ldc;
  const T* Ah;          // [n] high part of the row offsets
  const T* Bh;          // [m] high part of the column offsets
  const T* wc[3];       // [m] column weights of row reductions
  const T* wr[3];       // [n] row weights of column reductions
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
  int keep_l2;              // mark the cost's L2 lines evict-last (cost fits in L2)
  // point-cloud cost (C == nullptr): C_ij = sC |x_i - y_j|^2
  const float* X;           // [n][d]
  const float* Y;           // [m][d]
  int d;
  double sC;
  int64_t chunk;            // other-side elements per chunk (grid.y)
};

template <int N>
struct DotArr {
  double v[N > 0 ? N : 1];
};

// Epilogue traits. kNoTicket: the sweep only writes one partial per CTA of its
// epilogue sums (the next kernel reduces them itself, in fixed order, so no CTA
// waits on a grid-wide ticket). kPrefetch (column sweeps): every CTA calls
// epi.begin(first column, strip width, m) after the dependency wait and
// epi.drain() before its ticket, and a
// CTA that finishes a strip calls epi.prepare(publish) before its epilogue
// (publish: strip 0).
template <class E, class = void>
struct NoTicket : std::false_type {};
template <class E>
struct NoTicket<E, std::void_t<decltype(E::kNoTicket)>> : std::bool_constant<E::kNoTicket> {};
// row sweeps whose epilogue copies a row's operands ahead (Epi::prefetch(i), by
// the lane that later calls Epi::row(i))
template <class E, class = void>
struct HasRowPrefetch : std::false_type {};
template <class E>
struct HasRowPrefetch<E, std::void_t<decltype(E::kRowPrefetch)>> : std::bool_constant<E::kRowPrefetch> {};
template <class E, class = void>
struct HasPrefetch : std::false_type {};
template <class E>
struct HasPrefetch<E, std::void_t<decltype(E::kPrefetch)>> : std::bool_constant<E::kPrefetch> {};

// ----------------------------------------------------------------------------
// CTA-level deterministic sum of per-warp epilogue contributions, then a ticket
// so that the last CTA calls epi.finish with the totals over all CTAs.
// ----------------------------------------------------------------------------
template <int ND, class Epi, int NW = kWarps>
__device__ __forceinline__ void cta_dot_finish(double (&wd)[ND > 0 ? ND : 1], int64_t part_idx,
                                               int64_t nparts, double* dotpart, int* cnt,
                                               Epi& epi) {
  if constexpr (ND > 0) {
    __shared__ double sd[NW][ND];
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
        for (int w = 0; w < NW; ++w) t += sd[w][k];
        dotpart[part_idx * 2 + k] = t;
      }
      if constexpr (!NoTicket<Epi>::value) {
        __threadfence();
        last = (atomicAdd(cnt, 1) == (int)nparts - 1);
      }
    }
    if constexpr (NoTicket<Epi>::value) return;
    __syncthreads();
    if (last) {
      // all threads of the last CTA add the partials: fixed assignment and a
      // fixed reduction tree, so the totals are bit-reproducible
      __threadfence();
      double v[ND];
#pragma unroll
      for (int k = 0; k < ND; ++k) v[k] = 0.0;
      for (int64_t p = threadIdx.x; p < nparts; p += NW * 32) {
#pragma unroll
        for (int k = 0; k < ND; ++k) v[k] += __ldcg(dotpart + p * 2 + k);
      }
#pragma unroll
      for (int k = 0; k < ND; ++k) v[k] = warp_sum(v[k]);
      __syncthreads();
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < ND; ++k) sd[warp][k] = v[k];
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        DotArr<ND> tot;
#pragma unroll
        for (int k = 0; k < ND; ++k) {
          tot.v[k] = 0.0;
          for (int w = 0; w < NW; ++w) tot.v[k] += sd[w][k];
        }
        *cnt = 0;
        epi.finish(tot.v);
      }
    }
  }
}

// ----------------------------------------------------------------------------
// FP32 result of one row held by a warp: the lanes' compensated pairs are
// combined in FP32 (the FP64 pipe is narrow) and lane 0 hands the row's FP64
// result to the epilogue. LSE: common max of the lanes (1/8 grid: exact), one
// rescale per lane.
// ----------------------------------------------------------------------------
template <int NA, bool LSE, int ND, class Epi>
__device__ __forceinline__ void row_result_f32(int64_t i, int lane, const float (&S)[NA], const float (&Cc)[NA],
                                               float mx, bool mx_set, Epi& epi, double (&wd)[ND > 0 ? ND : 1]) {
  if constexpr (!LSE) {
    double tot[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) {
      float s0 = S[k], c0 = Cc[k];
      warp_sum_pair(s0, c0);
      tot[k] = (double)s0 + (double)c0;
    }
    if (lane == 0) {
      DotArr<ND> d;
      epi.row(i, tot, d.v);  // tot: [NA] sums
#pragma unroll
      for (int k = 0; k < ND; ++k) wd[k] += d.v[k];
    }
  } else {
    const float M = warp_max_f(mx_set ? mx : -INFINITY);
    const float f = mx_set ? expT(mx - M) : 0.f;
    float s0 = S[0] * f, c0 = Cc[0] * f;
    warp_sum_pair(s0, c0);
    if (lane == 0) {
      DotArr<ND> d;
      epi.row_lse(i, (double)M, (double)s0 + (double)c0, d.v);
#pragma unroll
      for (int k = 0; k < ND; ++k) wd[k] += d.v[k];
    }
  }
}

// FP32 column result: combine the R compensated partial pairs of column jj in
// fixed order (LSE: the (max, 0) pairs of slot 0 and the sums of slot 1) and
// hand the FP64 result to the epilogue.
template <int NC, bool LSE, class Epi>
__device__ __forceinline__ void col_combine_f32(const float2* cp2, int R, int64_t m, int64_t jj, Epi& epi,
                                                double* dv) {
  if constexpr (!LSE) {
    double s[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      float s0 = 0.f, c0 = 0.f;
      // up to 16 row blocks in one batch of loads: one L2 round trip at the
      // usual R = 9 (the finisher's latency is the column sweep's tail)
      ordered_loads<16>(cp2 + (int64_t)k * R * m + jj, m, R, [&](float2 q) {
        kadd(s0, c0, q.x);
        c0 += q.y;
      });
      s[k] = (double)s0 + (double)c0;
    }
    epi.col(jj, s, dv);
  } else {
    // slot 0 holds the (max, 0) pairs, slot 1 the compensated sums
    const float2* mx = cp2 + jj;
    const float2* sm = cp2 + (int64_t)R * m + jj;
    float M = -INFINITY;
    ordered_loads2(mx, sm, m, R, [&](float2 qm, float2 qs) {
      if (qs.x != 0.f || qs.y != 0.f) M = fmaxf(M, qm.x);
    });
    float s0 = 0.f, c0 = 0.f;
    ordered_loads2(mx, sm, m, R, [&](float2 qm, float2 qs) {
      if (qs.x == 0.f && qs.y == 0.f) return;
      const float f = expT(qm.x - M);
      kadd(s0, c0, qs.x * f);
      c0 += qs.y * f;
    });
    epi.col_lse(jj, (double)M, (double)s0 + (double)c0, dv);
  }
}

// ----------------------------------------------------------------------------
// Row sweep: out_i = reduce_j E_ij * wc_k[j] (NR = 1..3 reductions; bit k of SQM
// makes reduction k use E_ij^2), or the online LSE of (t_ij + log wc_0[j]).
// One row per warp, 8 rows per CTA. The column vectors (Bh and the weights) are
// staged in shared memory tile by tile and shared by the CTA's 8 rows. Each lane
// streams its part of the row in batches of U 16-byte loads, software-pipelined
// over two register buffers: the loads of batch k+1 are in flight while batch k
// is reduced.
// ----------------------------------------------------------------------------
template <class T, int V, int U>
__device__ __forceinline__ void row_load(const T* crow, int j0, int tw, T (&c)[U][V], uint64_t pol) {
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int jl = j0 + u * 32 * V;
    if (jl < tw) ld_stream(crow + jl, c[u], pol);
  }
}

template <class T, int V, int U, int NR, int SQM, int NV, int TW>
__device__ __forceinline__ void row_reduce_sum(const T (&c)[U][V], int j0, int tw, T ah, T g,
                                               const T (&sv)[NV][TW], T (&S)[NR], T (&Cc)[NR]) {
  T acc[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) acc[k] = T(0);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int jl = j0 + u * 32 * V;
    if (jl >= tw) continue;
    T b[V], w[NR][V];
    ld_vec_smem<V>(&sv[0][jl], b);
#pragma unroll
    for (int k = 0; k < NR; ++k) ld_vec_smem<V>(&sv[1 + k][jl], w[k]);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const T x = expT(fmaT(-g, c[u][e], ah + b[e]));
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        if ((SQM >> k) & 1) acc[k] = fmaT(x * x, w[k][e], acc[k]);
        else acc[k] = fmaT(x, w[k][e], acc[k]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < NR; ++k) kadd(S[k], Cc[k], acc[k]);
}

// Online LSE of t + log w over one batch. The running max mx lives on the 1/8
// grid so that am = ah - mx is exact. One max test per 16-byte chunk: if the
// chunk holds a t above theta, mx is raised once and the chunk's t are formed
// again against the new mx (at most 4 raises; a non-finite t leaves a
// non-finite sum).
template <class T, int V, int U, int NV, int TW>
__device__ __forceinline__ void row_reduce_lse(const T (&c)[U][V], int j0, int tw, T ah, T g,
                                               const T (&sv)[NV][TW], T& mx, T& am, T& S, T& Cc) {
  T acc = T(0);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int jl = j0 + u * 32 * V;
    if (jl >= tw) continue;
    T b[V], w[V], t[V];
    ld_vec_smem<V>(&sv[0][jl], b);
    ld_vec_smem<V>(&sv[1][jl], w);
    T tmax = T(-3.0e38);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      t[e] = fmaT(-g, c[u][e], am + b[e]);
      tmax = fmax(tmax, t[e]);
    }
    for (int k = 0; k < 4 && tmax > T(kTheta); ++k) {
      const T dlt = ceil_grid(tmax);
      mx += dlt;
      am = ah - mx;
      const T f = expT(-dlt);
      acc *= f;
      S *= f;
      Cc *= f;
      tmax = T(-3.0e38);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        t[e] = fmaT(-g, c[u][e], am + b[e]);
        tmax = fmax(tmax, t[e]);
      }
    }
#pragma unroll
    for (int e = 0; e < V; ++e) acc = fmaT(expT(t[e]), w[e], acc);
  }
  kadd(S, Cc, acc);
}

template <class T, int V, int NR, bool LSE, int SQM, class Epi>
__global__ void __launch_bounds__(kThreads, 4) row_sweep_kernel(SweepArgs<T> a, Epi epi) {
  constexpr int U = 4;                               // chunks per batch (two batches in flight)
  constexpr int NV = 1 + (LSE ? 1 : NR);             // staged column vectors
  // tile width (<= 32 KB smem), a multiple of 128 so that tiles and rows of sv stay 16-byte aligned
  constexpr int TW = ((sizeof(T) == 4 ? 8192 : 4096) / NV) / 128 * 128;
  constexpr int ND = Epi::kDot;
  constexpr int NA = LSE ? 1 : NR;
  constexpr int STEP = 32 * V * U;
  __shared__ __align__(16) T sv[NV][TW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kWarps + warp;
  const bool rv = i < a.n;
  const T* crow = a.C + (rv ? i : 0) * a.ldc;
  // the first batch of the (immutable) cost row is in flight before the wait
  const uint64_t pol = cost_policy(a.keep_l2);
  T cA[U][V], cB[U][V];
  const int tw0 = (int)min((int64_t)TW, a.m);
  if (rv && lane * V < tw0) row_load<T, V, U>(crow, lane * V, tw0, cA, pol);
  pdl_wait();
  if (a.active && *a.active == 0.0) return;
  const T g = a.gamma_dev ? (T)*a.gamma_dev : a.gamma;
  const T ah = rv ? a.Ah[i] : T(0);
  // 16-byte rows (V > 1): t0, tw and the workspace vectors are 16-byte aligned;
  // the tile is staged by asynchronous copies (through L1, which the CTAs of an
  // SM share), all of a thread's in flight at once
  auto stage = [&](int64_t t0, int tw) {
    for (int q = threadIdx.x * V; q < tw; q += kThreads * V) {
      cp_async16_ca(&sv[0][q], a.Bh + t0 + q);
#pragma unroll
      for (int k = 0; k < NV - 1; ++k) cp_async16_ca(&sv[1 + k][q], a.wc[k] + t0 + q);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if constexpr (V > 1) stage(0, tw0);
  if constexpr (HasRowPrefetch<Epi>::value) {
    if (rv && lane == 0) epi.prefetch(i);
  }
  double wd[ND > 0 ? ND : 1];
#pragma unroll
  for (int k = 0; k < (ND > 0 ? ND : 1); ++k) wd[k] = 0.0;
  T S[NA], Cc[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) { S[k] = T(0); Cc[k] = T(0); }
  T mx = T(0), am = ah;
  bool mx_set = false;

  for (int64_t t0 = 0; t0 < a.m; t0 += TW) {
    const int tw = (int)min((int64_t)TW, a.m - t0);
    if constexpr (V > 1) {
      if (t0 > 0) {
        __syncthreads();  // every warp is done with the previous tile
        stage(t0, tw);
      }
      cp_async_wait_all();
    } else {
      __syncthreads();
      for (int q = threadIdx.x; q < tw; q += kThreads) {
        sv[0][q] = a.Bh[t0 + q];
#pragma unroll
        for (int k = 0; k < NV - 1; ++k) sv[1 + k][q] = a.wc[k][t0 + q];
      }
    }
    __syncthreads();
    if (!rv) continue;
    const T* ct = crow + t0;
    int j0 = lane * V;
    if (j0 >= tw) continue;
    if (t0 > 0) row_load<T, V, U>(ct, j0, tw, cA, pol);  // tile 0 was prefetched
    if constexpr (LSE) {
      if (!mx_set) {
        // start the running max at the lane's first element, so that the
        // dominant terms cannot underflow against a far-away start value
        const T b0 = sv[0][j0];
        mx = ceil_grid(fmaT(-g, cA[0][0], ah + b0));
        am = ah - mx;
        mx_set = true;
      }
    }
    for (;;) {
      const int j1 = j0 + STEP;
      if (j1 < tw) row_load<T, V, U>(ct, j1, tw, cB, pol);
      if constexpr (!LSE) row_reduce_sum<T, V, U, NR, SQM, NV, TW>(cA, j0, tw, ah, g, sv, S, Cc);
      else row_reduce_lse<T, V, U, NV, TW>(cA, j0, tw, ah, g, sv, mx, am, S[0], Cc[0]);
      if (j1 >= tw) break;
      const int j2 = j1 + STEP;
      if (j2 < tw) row_load<T, V, U>(ct, j2, tw, cA, pol);
      if constexpr (!LSE) row_reduce_sum<T, V, U, NR, SQM, NV, TW>(cB, j1, tw, ah, g, sv, S, Cc);
      else row_reduce_lse<T, V, U, NV, TW>(cB, j1, tw, ah, g, sv, mx, am, S[0], Cc[0]);
      if (j2 >= tw) break;
      j0 = j2;
    }
  }
  pdl_trigger();
  if (rv) {
    if constexpr (sizeof(T) == 4) {
      row_result_f32<NA, LSE, ND>(i, lane, S, Cc, mx, mx_set, epi, wd);
    } else {
      if constexpr (!LSE) {
        double tot[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) tot[k] = warp_sum((double)S[k] + (double)Cc[k]);
        if (lane == 0) {
          DotArr<ND> d;
          epi.row(i, tot, d.v);  // tot: [NR] sums
#pragma unroll
          for (int k = 0; k < ND; ++k) wd[k] += d.v[k];
        }
      } else {
        LsePair p{mx_set ? (double)mx : 0.0, (double)S[0] + (double)Cc[0]};
        p = warp_lse<T>(p);
        if (lane == 0) {
          DotArr<ND> d;
          epi.row_lse(i, p.m, p.s, d.v);
#pragma unroll
          for (int k = 0; k < ND; ++k) wd[k] += d.v[k];
        }
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
// CL (FP32, NC = 1, no LSE, no row reductions): launched as clusters of the R
// CTAs of a strip (R <= 8). Instead of global partials and a ticket, the CTAs
// of a strip combine their column sums through distributed shared memory and
// each finishes a share of the strip's columns: no CTA waits for the last one
// of its strip, which was this sweep's tail. Every CTA of a cluster must take
// the same path through both cluster barriers, so *a.active must not change
// while the kernel runs (its epilogue publishes stops elsewhere).
// ----------------------------------------------------------------------------
template <class T, int V, int NC, bool LSE, int NR, class Epi, bool CL = false>
__global__ void __launch_bounds__(kThreads, kColCtasPerSm) col_sweep_kernel(SweepArgs<T> a, Epi epi) {
  static_assert(!CL || (sizeof(T) == 4 && NC == 1 && !LSE && NR == 0 && Epi::kDot == 0),
                "cluster finish: FP32 column sums without dots or row reductions");
  constexpr int U = 4;  // rows per batch (two batches in flight)
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
  // the first batch of (immutable) cost rows is in flight before the wait
  const uint64_t pol = cost_policy(a.keep_l2);
  T cA[U][V], cB[U][V];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t i = r0 + warp + (int64_t)u * kWarps;
    if (i < r1 && jv) ld_stream(a.C + i * a.ldc + j, cA[u], pol);
  }
  pdl_wait();
  if (a.active && *a.active == 0.0) return;
  if constexpr (HasPrefetch<Epi>::value) epi.begin(strip * SW, SW, a.m);
  const T g = a.gamma_dev ? (T)*a.gamma_dev : a.gamma;

  T b[V], wcv[2][V];
#pragma unroll
  for (int e = 0; e < V; ++e) { b[e] = T(0); wcv[0][e] = T(0); wcv[1][e] = T(0); }
  if (jv) {
    ld_vec<V>(a.Bh + j, b);
    if constexpr (NR > 0) ld_vec<V>(a.wc[0] + j, wcv[0]);
    if constexpr (NR > 1) ld_vec<V>(a.wc[1] + j, wcv[1]);
  }
  T tot[NP][V], cmp[NP][V];  // compensated running sums
#pragma unroll
  for (int k = 0; k < NP; ++k)
#pragma unroll
    for (int e = 0; e < V; ++e) { tot[k][e] = T(0); cmp[k][e] = T(0); }
  // LSE state per column: running max mx (on the grid) and bm = Bh - mx
  T mx[V], bm[V];
#pragma unroll
  for (int e = 0; e < V; ++e) { mx[e] = T(0); bm[e] = b[e]; }

  // rows of this warp in batches of U, software-pipelined over two buffers
  T hA[U], hB[U], xA[2][U], xB[2][U];
  auto load_vec = [&](int64_t i0, T (&hh)[U], T (&xx)[2][U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + (int64_t)u * kWarps;
      if (i < r1) {
        hh[u] = a.Ah[i];
        xx[0][u] = a.wr[0][i];
        if constexpr (NC > 1) xx[1][u] = a.wr[1][i];
      }
    }
  };
  auto load = [&](int64_t i0, T (&c)[U][V], T (&hh)[U], T (&xx)[2][U]) {
    load_vec(i0, hh, xx);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + (int64_t)u * kWarps;
      if (i < r1 && jv) ld_stream(a.C + i * a.ldc + j, c[u], pol);
    }
  };
  auto reduce = [&](int64_t i0, const T (&c)[U][V], const T (&hh)[U], const T (&xx)[2][U]) {
    T acc[NP][V];
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
      for (int e = 0; e < V; ++e) acc[k][e] = T(0);
    if constexpr (LSE) {
      // per column: form the batch's t, raise the running max once if a t
      // exceeds theta (then form them again; at most 4 raises), accumulate
      if (jv) {
#pragma unroll
        for (int e = 0; e < V; ++e) {
          T t[U];
          T tmax = T(-3.0e38);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            t[u] = fmaT(-g, c[u][e], hh[u] + bm[e]);
            if (i0 + (int64_t)u * kWarps < r1) tmax = fmax(tmax, t[u]);
          }
          for (int k = 0; k < 4 && tmax > T(kTheta); ++k) {
            const T dlt = ceil_grid(tmax);
            mx[e] += dlt;
            bm[e] = b[e] - mx[e];
            const T f = expT(-dlt);
            tot[1][e] *= f;
            cmp[1][e] *= f;
            tmax = T(-3.0e38);
#pragma unroll
            for (int u = 0; u < U; ++u) {
              t[u] = fmaT(-g, c[u][e], hh[u] + bm[e]);
              if (i0 + (int64_t)u * kWarps < r1) tmax = fmax(tmax, t[u]);
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (i0 + (int64_t)u * kWarps < r1) acc[1][e] = fmaT(expT(t[u]), xx[0][u], acc[1][e]);
        }
      }
    } else {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (i0 + (int64_t)u * kWarps >= r1) continue;
      T racc0 = T(0), racc1 = T(0);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        if constexpr (!LSE) {
          const T t = fmaT(-g, c[u][e], hh[u] + b[e]);
          const T x = jv ? expT(t) : T(0);
          acc[0][e] = fmaT(x, xx[0][u], acc[0][e]);
          if constexpr (NC > 1) acc[1][e] = fmaT(x, xx[1][u], acc[1][e]);
          if constexpr (NR > 0) racc0 = fmaT(x, wcv[0][e], racc0);
          if constexpr (NR > 1) racc1 = fmaT(x, wcv[1][e], racc1);
        }
      }
      if constexpr (NR > 0) {
        const double rs0 = warp_sum_t(racc0);
        double rs1 = 0.0;
        if constexpr (NR > 1) rs1 = warp_sum_t(racc1);
        if (lane == 0) {
          const int64_t i = i0 + (int64_t)u * kWarps;
          a.rowpart[(0 * S + strip) * a.n + i] = rs0;
          if constexpr (NR > 1) a.rowpart[(1 * S + strip) * a.n + i] = rs1;
        }
      }
    }
    }
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
      for (int e = 0; e < V; ++e) kadd(tot[k][e], cmp[k][e], acc[k][e]);
  };
  constexpr int64_t BSTEP = (int64_t)kWarps * U;
  int64_t i0 = r0 + warp;
  if (i0 < r1) {
    load_vec(i0, hA, xA);  // the cost rows of this batch were prefetched
    if constexpr (LSE) {
      // start each column's running max at its first element
      if (jv) {
#pragma unroll
        for (int e = 0; e < V; ++e) {
          mx[e] = ceil_grid(fmaT(-g, cA[0][e], hA[0] + b[e]));
          bm[e] = b[e] - mx[e];
        }
      }
    }
    for (;;) {
      const int64_t i1 = i0 + BSTEP;
      if (i1 < r1) load(i1, cB, hB, xB);
      reduce(i0, cA, hA, xA);
      if (i1 >= r1) break;
      const int64_t i2 = i1 + BSTEP;
      if (i2 < r1) load(i2, cA, hA, xA);
      reduce(i1, cB, hB, xB);
      if (i2 >= r1) break;
      i0 = i2;
    }
  }

  pdl_trigger();
  // ---- combine the 8 warps of this CTA and write the [R][m] partials ----
  __shared__ float2 ccol[CL ? SW : 1];  // CL: this CTA's column sums, read by its cluster
  // FP32 path: compensated FP32 pairs (the FP64 pipe is narrow), stored as a
  // float2 (sum, compensation) per partial slot; LSE: (max, 0) in slot 0 and the
  // pair in slot 1. FP64 path: FP64 partials.
  if constexpr (sizeof(T) == 4) {
    __shared__ float fsum[NP][kWarps][SW], fcmp[NP][kWarps][SW];
    __shared__ float fmx[LSE ? kWarps : 1][LSE ? SW : 1];
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
      for (int e = 0; e < V; ++e) {
        fsum[k][warp][lane * V + e] = (float)tot[k][e];
        fcmp[k][warp][lane * V + e] = (float)cmp[k][e];
      }
    if constexpr (LSE) {
#pragma unroll
      for (int e = 0; e < V; ++e) fmx[warp][lane * V + e] = (float)mx[e];
    }
    __syncthreads();
    float2* cp2 = reinterpret_cast<float2*>(a.colpart);
    for (int cc = threadIdx.x; cc < SW; cc += kThreads) {
      const int64_t jj = strip * SW + cc;
      if (jj >= a.m) continue;
      if constexpr (CL) {
        float s0 = 0.f, c0 = 0.f;
        for (int w = 0; w < kWarps; ++w) {
          kadd(s0, c0, fsum[0][w][cc]);
          c0 += fcmp[0][w][cc];
        }
        ccol[cc] = make_float2(s0, c0);
      } else if constexpr (!LSE) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          float s0 = 0.f, c0 = 0.f;
          for (int w = 0; w < kWarps; ++w) {
            kadd(s0, c0, fsum[k][w][cc]);
            c0 += fcmp[k][w][cc];
          }
          cp2[((int64_t)k * R + rb) * a.m + jj] = make_float2(s0, c0);
        }
      } else {
        float M = -INFINITY;
        for (int w = 0; w < kWarps; ++w)
          if (fsum[1][w][cc] != 0.f || fcmp[1][w][cc] != 0.f) M = fmaxf(M, fmx[w][cc]);
        float s0 = 0.f, c0 = 0.f;
        for (int w = 0; w < kWarps; ++w) {
          if (fsum[1][w][cc] == 0.f && fcmp[1][w][cc] == 0.f) continue;
          const float f = (float)expT((T)(fmx[w][cc] - M));
          kadd(s0, c0, fsum[1][w][cc] * f);
          c0 += fcmp[1][w][cc] * f;
        }
        cp2[((int64_t)0 * R + rb) * a.m + jj] = make_float2(M, 0.f);
        cp2[((int64_t)1 * R + rb) * a.m + jj] = make_float2(s0, c0);
      }
    }
  } else {
    __shared__ double sred[NP][kWarps][SW];
    __shared__ double smax[LSE ? kWarps : 1][LSE ? SW : 1];
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
      for (int e = 0; e < V; ++e) sred[k][warp][lane * V + e] = (double)tot[k][e] + (double)cmp[k][e];
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
        for (int w = 0; w < kWarps; ++w) p = lse_combine<T>(p, LsePair{smax[w][cc], sred[1][w][cc]});
        a.colpart[((int64_t)0 * R + rb) * a.m + jj] = p.m;
        a.colpart[((int64_t)1 * R + rb) * a.m + jj] = p.s;
      }
    }
  }

  if constexpr (CL) {
    // ---- the strip's CTAs combine through distributed shared memory ----
    const uint32_t rank = cluster_rank();
    if constexpr (HasPrefetch<Epi>::value) {  // (before the barrier: it needs no column sums)
      epi.drain();
      epi.prepare(strip == 0 && rank == 0);
    }
    cluster_sync();  // every CTA's column sums are visible to the cluster
    const int per = (SW + R - 1) / R;  // columns this CTA finishes
    const int lo = (int)rank * per, hi = min(SW, lo + per);
    for (int cc = lo + threadIdx.x; cc < hi; cc += kThreads) {
      const int64_t jj = strip * SW + cc;
      if (jj >= a.m) continue;
      float s0 = 0.f, c0 = 0.f;
      for (int r = 0; r < R; ++r) {  // in rank order, as the ticketed combine adds row blocks
        const float2 q = ld_cluster_f2(&ccol[cc], (uint32_t)r);
        kadd(s0, c0, q.x);
        c0 += q.y;
      }
      double s[1] = {(double)s0 + (double)c0};
      double d[1];
      epi.col(jj, s, d);
    }
    cluster_sync();  // no CTA leaves while another reads its shared memory
    return;
  }
  // ---- tickets: the last CTA of the strip combines the R partials ----
  __shared__ int last_strip, last_rows;
  if constexpr (HasPrefetch<Epi>::value) epi.drain();
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last_strip = (atomicAdd(a.cnt_strip + strip, 1) == R - 1);
    if constexpr (NR > 0) last_rows = (atomicAdd(a.cnt_rowblk + rb, 1) == (int)S - 1);
  }
  __syncthreads();
  if (last_strip) {
    __threadfence();
    if constexpr (HasPrefetch<Epi>::value) epi.prepare(strip == 0);
    double wd[ND > 0 ? ND : 1];
#pragma unroll
    for (int k = 0; k < (ND > 0 ? ND : 1); ++k) wd[k] = 0.0;
    for (int cc = threadIdx.x; cc < SW; cc += kThreads) {
      const int64_t jj = strip * SW + cc;
      if (jj >= a.m) continue;
      DotArr<ND> d;
      if constexpr (sizeof(T) == 4) {
        col_combine_f32<NC, LSE>(reinterpret_cast<const float2*>(a.colpart), R, a.m, jj, epi, d.v);
      } else if constexpr (!LSE) {
        double s[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          double t = 0.0;
          ordered_loads(a.colpart + (int64_t)k * R * a.m + jj, a.m, R, [&](double q) { t += q; });
          s[k] = t;
        }
        epi.col(jj, s, d.v);
      } else {
        LsePair p{0.0, 0.0};
        ordered_loads2(a.colpart + jj, a.colpart + (int64_t)R * a.m + jj, a.m, R,
                       [&](double qm, double qs) { p = lse_combine<T>(p, LsePair{qm, qs}); });
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
          ordered_loads(a.rowpart + (int64_t)k * S * a.n + i, a.n, S, [&](double q) { t += q; });
          s[k] = t;
        }
        epi.row_part(i, s);
      }
      if (threadIdx.x == 0) a.cnt_rowblk[rb] = 0;
    }
  }
}

}  // namespace eot
