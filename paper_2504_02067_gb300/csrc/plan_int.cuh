// Integer outputs of the implicit plan P_ij = exp(u_i + v_j - gamma C_ij) (Sec. 2.1,
// Eq. lagrangian-closed-form): the row argmax and the support {P_ij > tau}.
//
// Every decision is taken on an FP64 exponent formed by a fixed sequence of
// correctly rounded operations (__dmul_rn / __dadd_rn / __dsub_rn are never
// contracted into an FMA), so the results are bit-exact against any IEEE-754
// evaluation of the same sequence:
//   C_ij  = (double)C_ij                       dense cost (exact promotion)
//   C_ij  = s_C * D_ij, D_ij = ((x_i0 - y_j0)^2 + (x_i1 - y_j1)^2) + ...
//                                             points, summed in coordinate order
//   gC_ij = gamma * C_ij
//   argmax: t_ij = v_j - gC_ij        (u_i is constant along row i, exp increasing)
//   support: t_ij = (u_i + v_j) - gC_ij > log_tau
// One warp owns a row; ties of the argmax go to the lowest column index.
#pragma once
#include "common.cuh"

namespace eot {
namespace pint {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kTile = 128;  // other-side points staged per tile (point costs)
constexpr int kMaxD = 64;

// (value, index) pair of a running argmax: an index < 0 marks an empty pair.
// `b` wins over `a` if it is larger, or equal with a lower index.
__device__ __forceinline__ void argmax_merge(double& av, int64_t& ai, double bv, int64_t bi) {
  if (bi < 0) return;
  if (ai < 0 || bv > av || (bv == av && bi < ai)) {
    av = bv;
    ai = bi;
  }
}

template <int MODE>  // MODE 0: argmax of v_j - gC_ij; MODE 1: count of (u_i + v_j) - gC_ij > log_tau
struct Acc {
  double best = 0.0;
  int64_t idx = -1;
  long long cnt = 0;
  __device__ __forceinline__ void add(double ui, double vj, double gC, int64_t j, double log_tau) {
    if constexpr (MODE == 0) {
      const double t = __dsub_rn(vj, gC);
      // a lane visits its columns in increasing order: a later column replaces the
      // held one only if strictly larger
      if (idx < 0 || t > best) {
        best = t;
        idx = j;
      }
    } else {
      const double t = __dsub_rn(__dadd_rn(ui, vj), gC);
      cnt += (t > log_tau) ? 1 : 0;
    }
  }
  // warp-wide combine; lane 0 writes row i's result
  __device__ __forceinline__ void finish(int64_t i, int lane, int64_t* idx_out, int64_t* counts,
                                         unsigned long long* total) {
    if constexpr (MODE == 0) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double bv = __shfl_xor_sync(0xffffffffu, best, o);
        const long long bi = __shfl_xor_sync(0xffffffffu, (long long)idx, o);
        argmax_merge(best, idx, bv, (int64_t)bi);
      }
      if (lane == 0) idx_out[i] = idx < 0 ? 0 : idx;
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      if (lane == 0) {
        if (counts) counts[i] = (int64_t)cnt;
        if (total) atomicAdd(total, (unsigned long long)cnt);
      }
    }
  }
};

// Dense cost (float or double), row-major with leading dimension ldc.
template <class T, int MODE>
__global__ void __launch_bounds__(kThreads) plan_int_dense_kernel(int64_t n, int64_t m, const T* C, int64_t ldc,
                                                                  const double* u, const double* v, double gamma,
                                                                  double log_tau, int64_t* idx_out,
                                                                  int64_t* counts, unsigned long long* total) {
  pdl_wait();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kWarps + warp;
  if (i >= n) return;
  const T* crow = C + i * ldc;
  const double ui = MODE == 1 ? u[i] : 0.0;
  Acc<MODE> acc;
  for (int64_t j = lane; j < m; j += 32) {
    const double gC = __dmul_rn(gamma, (double)__ldg(crow + j));
    acc.add(ui, __ldg(v + j), gC, j, log_tau);
  }
  acc.finish(i, lane, idx_out, counts, total);
}

// Point costs: C_ij = s_C * sum_k (x_ik - y_jk)^2 in coordinate order. The CTA's
// 8 rows share tiles of kTile other-side points, staged coordinate-major in
// shared memory (lanes read consecutive points: no bank conflicts); each warp
// keeps its row's coordinates, promoted to FP64, in shared memory (broadcast reads).
template <int MODE>
__global__ void __launch_bounds__(kThreads) plan_int_points_kernel(int64_t n, int64_t m, int d, const float* X,
                                                                   const float* Y, double sC, const double* u,
                                                                   const double* v, double gamma, double log_tau,
                                                                   int64_t* idx_out, int64_t* counts,
                                                                   unsigned long long* total) {
  __shared__ float ys[kMaxD][kTile];
  __shared__ double xs[kWarps][kMaxD];
  pdl_wait();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kWarps + warp;
  const bool rv = i < n;
  for (int k = lane; k < d; k += 32) xs[warp][k] = rv ? (double)X[i * d + k] : 0.0;
  const double ui = (MODE == 1 && rv) ? u[i] : 0.0;
  Acc<MODE> acc;
  for (int64_t j0 = 0; j0 < m; j0 += kTile) {
    const int tw = (int)min((int64_t)kTile, m - j0);
    __syncthreads();
    // the tile's tw * d floats are contiguous in Y: coalesced loads, transposed store
    for (int q = threadIdx.x; q < tw * d; q += kThreads) {
      const int jj = q / d, k = q - jj * d;
      ys[k][jj] = Y[(j0 + jj) * d + k];
    }
    __syncthreads();
    if (!rv) continue;
    for (int jj = lane; jj < tw; jj += 32) {
      double D = 0.0;
      for (int k = 0; k < d; ++k) {
        const double df = __dsub_rn(xs[warp][k], (double)ys[k][jj]);
        D = __dadd_rn(D, __dmul_rn(df, df));
      }
      const double gC = __dmul_rn(gamma, __dmul_rn(sC, D));
      acc.add(ui, __ldg(v + j0 + jj), gC, j0 + jj, log_tau);
    }
  }
  if (rv) acc.finish(i, lane, idx_out, counts, total);
}

}  // namespace pint
}  // namespace eot
