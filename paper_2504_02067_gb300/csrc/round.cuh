// Round: the step after the last projection of Alg. 1, which the paper cites as
// Algorithm 2 of Altschuler, Weed and Rigollet (2017). It maps a near-feasible
// plan F onto the transport polytope U(r, c):
//   x = min(r / r(F), 1),  F' = D(x) F;   y = min(c / c(F'), 1),  F'' = F' D(y);
//   a = r - r(F''),  b = c - c(F''),  Round(F) = F'' + a b^T / ||a||_1.
// Here F = P(u, v; gamma) stays implicit: F'' = P(u + log x, v + log y) and the
// correction is the rank-one term a b^T / ||a||_1, so the rounded plan costs
// O(n + m) memory. The transport cost <Round(F), C> is
//   sum_ij C_ij F''_ij + (a^T C b) / ||a||_1.
//
// Everything is FP64 with plain exp: Round runs once per solve (three passes
// over the cost), so it favours a direct evaluation over the mixed-precision
// machinery of the sweeps; on this GPU it is bound by the FP64 pipe
// (an FP64 exp and a few FP64 operations per plan entry and pass).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace eot {
namespace rnd {

constexpr int kThreads = 256;
constexpr int kColWarps = kThreads / 32;

// C_ij of a dense cost stored as CT (float or double), row-major with stride ldc.
template <class CT>
struct DenseCost {
  const CT* C;
  int64_t ldc;
  __device__ __forceinline__ double operator()(int64_t i, int64_t j) const { return (double)C[i * ldc + j]; }
};

// C_ij = sC |x_i - y_j|^2 of FP32 point clouds in R^d, evaluated in FP64.
struct PointCost {
  const float *X, *Y;
  int d;
  double sC;
  __device__ __forceinline__ double operator()(int64_t i, int64_t j) const {
    const float* xi = X + i * d;
    const float* yj = Y + j * d;
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
      const double t = (double)xi[k] - (double)yj[k];
      s = fma(t, t, s);
    }
    return sC * s;
  }
};

__device__ __forceinline__ double warp_sum64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Row pass, one warp per row. With x == nullptr (first pass): the row sums s_i of
// F, x_i = min(r_i / s_i, 1) and u1_i = u_i + log x_i. With x, y (last pass): the
// row sums of F'' = D(x) F D(y), a_i = r_i - r_i(F''), rowc_i = sum_j C_ij F''_ij
// and rowcb_i = sum_j C_ij b_j.
template <class Cost>
__global__ void __launch_bounds__(kThreads) round_row_kernel(int64_t n, int64_t m, const double* u,
                                                             const double* v, double gamma, Cost cost,
                                                             const double* r, const double* x_in,
                                                             const double* y, const double* b, double* x_out,
                                                             double* u1, double* a, double* rowc, double* rowcb) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const double ui = u[i];
    double s = 0.0, sc = 0.0, sb = 0.0;
    if (x_in) {
      const double xi = x_in[i];
      for (int64_t j = lane; j < m; j += 32) {
        const double cij = cost(i, j);
        const double f = (xi * exp(ui + v[j] - gamma * cij)) * y[j];
        s += f;
        sc += cij * f;
        sb += cij * b[j];
      }
    } else {
      for (int64_t j = lane; j < m; j += 32) s += exp(ui + v[j] - gamma * cost(i, j));
    }
    s = warp_sum64(s);
    if (x_in) {
      sc = warp_sum64(sc);
      sb = warp_sum64(sb);
    }
    if (lane == 0) {
      if (x_in) {
        a[i] = r[i] - s;
        rowc[i] = sc;
        rowcb[i] = sb;
      } else {
        // min(r / s, 1) without 0 / 0: an empty row (s = 0) keeps x = 1
        const double xi = s <= r[i] ? 1.0 : r[i] / s;
        x_out[i] = xi;
        if (u1) u1[i] = ui + log(xi);
      }
    }
  }
}

// Column pass over F' = D(x) F: block (32 columns, kColWarps row lanes) of one
// row block; part[rb * m + j] = the row block's partial column sum.
template <class Cost>
__global__ void __launch_bounds__(kThreads) round_col_kernel(int64_t n, int64_t m, const double* u,
                                                             const double* x, const double* v, double gamma,
                                                             Cost cost, int64_t rows_per, double* part) {
  __shared__ double red[kColWarps][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  const int64_t i0 = (int64_t)blockIdx.y * rows_per;
  const int64_t i1 = i0 + rows_per < n ? i0 + rows_per : n;
  double s = 0.0;
  if (j < m) {
    const double vj = v[j];
    for (int64_t i = i0 + w; i < i1; i += kColWarps) s += x[i] * exp(u[i] + vj - gamma * cost(i, j));
  }
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && j < m) {
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < kColWarps; ++k) t += red[k][lane];
    part[(int64_t)blockIdx.y * m + j] = t;
  }
}

// Column totals c(F')_j (row blocks in order), y_j = min(c_j / c(F')_j, 1),
// v1_j = v_j + log y_j, b_j = c_j - y_j c(F')_j (= c_j - c(F'')_j).
static __global__ void round_colfin_kernel(int64_t m, int nrb, const double* part, const double* c, const double* v,
                                    double* y, double* v1, double* b) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    double cs = 0.0;
    for (int k = 0; k < nrb; ++k) cs += part[(int64_t)k * m + j];
    const double yj = cs <= c[j] ? 1.0 : c[j] / cs;
    y[j] = yj;
    if (v1) v1[j] = v[j] + log(yj);
    b[j] = c[j] - yj * cs;
  }
}

// One block: out[0] = sum_i rowc_i + (sum_i a_i rowcb_i) / ||a||_1 (the rank-one
// term only when ||a||_1 > 0), out[1] = ||a||_1. Fixed reduction order.
static __global__ void __launch_bounds__(1024) round_total_kernel(int64_t n, const double* a, const double* rowc,
                                                           const double* rowcb, double* out) {
  __shared__ double red[3][32];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    s0 += rowc[i];
    s1 += a[i] * rowcb[i];
    s2 += fabs(a[i]);
  }
  s0 = warp_sum64(s0);
  s1 = warp_sum64(s1);
  s2 = warp_sum64(s2);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][w] = s0;
    red[1][w] = s1;
    red[2][w] = s2;
  }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    s0 = lane < nw ? red[0][lane] : 0.0;
    s1 = lane < nw ? red[1][lane] : 0.0;
    s2 = lane < nw ? red[2][lane] : 0.0;
    s0 = warp_sum64(s0);
    s1 = warp_sum64(s1);
    s2 = warp_sum64(s2);
    if (lane == 0) {
      out[0] = s2 > 0.0 ? s0 + s1 / s2 : s0;
      out[1] = s2;
    }
  }
}

}  // namespace rnd
}  // namespace eot
