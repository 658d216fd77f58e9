// Device helpers shared by the sweep kernels and the O(n) kernels.
//
// The implicit plan of the paper, P_ij = exp(u_i + v_j - gamma C_ij) (Sec. 2.1,
// Eq. lagrangian-closed-form), is never stored. Every kernel forms
//     P_ij = rowfac_i * colfac_j * exp(t_ij),   t_ij = Ah_i + Bh_j - gamma C_ij,
// where (Ah, Bh) are the "high" parts of FP64 exponent offsets A_i, B_j rounded
// to a multiple of 1/8 (so that Ah_i + Bh_j is exact in FP32 for |A|,|B| < 2^19)
// and the FP64 factors carry the remaining low parts and any shifts exactly.
// gamma * C_ij is formed inside one FMA (exact product, one rounding), so the
// only FP32 error of t_ij is a single rounding relative to |t_ij|.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace eot {

constexpr int kWarps = 8;            // warps per CTA of every sweep kernel
constexpr int kThreads = kWarps * 32;
constexpr double kGrid = 0.125;      // split grid of the high parts
constexpr double kSplitLimit = 524288.0;  // |A|, |B| < 2^19 keeps Ah + Bh exact in FP32
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kTheta = 8.0f;       // lazy-rescale threshold of the online max
constexpr float kLow = 32.0f;        // an empty LSE accumulator re-centres below -kLow

// status bits written by kernels into the workspace status word
enum : int {
  kStatNonfinite = 1,   // non-finite potential or marginal entering a sweep
  kStatRange = 2,       // |potential| beyond the mixed-precision split range
  kStatTimeout = 4,     // a bounded device wait gave up
  kStatCurv = 8,        // CG: <p, F_r(rho) p> <= 0 or non-finite (loss of precision)
  kStatCgNan = 16       // CG: non-finite residual or preconditioned residual
};

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// exp in the element type: FP32 via the MUFU ex2 unit, FP64 via the libm exp.
__device__ __forceinline__ float expT(float t) { return ex2_approx(t * kLog2e); }
__device__ __forceinline__ double expT(double t) { return exp(t); }

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// round up to the 1/8 grid (exact for |x| < 2^20 in FP32)
__device__ __forceinline__ float ceil_grid(float x) { return ceilf(x * 8.0f) * 0.125f; }
__device__ __forceinline__ double ceil_grid(double x) { return ceil(x * 8.0) * 0.125; }

// streaming 16-byte loads of the cost matrix that do not allocate in L1
__device__ __forceinline__ void ld_stream(const float* p, float (&c)[4]) {
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(c[0]), "=f"(c[1]), "=f"(c[2]), "=f"(c[3]) : "l"(p));
}
__device__ __forceinline__ void ld_stream(const double* p, double (&c)[2]) {
  asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];"
               : "=d"(c[0]), "=d"(c[1]) : "l"(p));
}
__device__ __forceinline__ void ld_stream(const float* p, float (&c)[1]) { c[0] = __ldg(p); }
__device__ __forceinline__ void ld_stream(const double* p, double (&c)[1]) { c[0] = __ldg(p); }

// read-only vector loads of V consecutive elements (aligned when V > 1)
template <int V, class T>
__device__ __forceinline__ void ld_vec(const T* p, T (&c)[V]) {
  if constexpr (V == 4 && sizeof(T) == 4) {
    float4 x = __ldg(reinterpret_cast<const float4*>(p));
    c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w;
  } else if constexpr (V == 2 && sizeof(T) == 8) {
    double2 x = __ldg(reinterpret_cast<const double2*>(p));
    c[0] = x.x; c[1] = x.y;
  } else {
#pragma unroll
    for (int e = 0; e < V; ++e) c[e] = __ldg(p + e);
  }
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// (max, sum) pair of an online log-sum-exp; s == 0 marks an empty pair
struct LsePair {
  double m, s;
};
__device__ __forceinline__ LsePair lse_combine(LsePair a, LsePair b) {
  if (b.s == 0.0) return a;
  if (a.s == 0.0) return b;
  double M = fmax(a.m, b.m);
  return {M, a.s * exp(a.m - M) + b.s * exp(b.m - M)};
}
__device__ __forceinline__ LsePair warp_lse(LsePair p) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    LsePair q{__shfl_xor_sync(0xffffffffu, p.m, o), __shfl_xor_sync(0xffffffffu, p.s, o)};
    p = lse_combine(p, q);
  }
  return p;
}

}  // namespace eot
