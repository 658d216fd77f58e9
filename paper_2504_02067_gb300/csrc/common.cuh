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
#include <cmath>
#include <cuda_runtime.h>
#include <stdint.h>

namespace eot {

constexpr int kWarps = 8;            // warps per CTA of every sweep kernel
constexpr int kThreads = kWarps * 32;
constexpr int kColCtasPerSm = 2;     // resident column-sweep CTAs per SM (register bound)
constexpr int kColClusterMax = 8;    // row blocks of a strip in one cluster (the portable cluster size)
constexpr double kGrid = 0.125;      // split grid of the high parts
constexpr double kSplitLimit = 524288.0;  // |A|, |B| < 2^19 keeps Ah + Bh exact in FP32
constexpr float kLog2e = 1.4426950408889634f;
// Rounding floor of sum P - 1 evaluated with FP32 plan entries: each marginal
// entry errs by up to about 2^-22 relative (ex2.approx), and these errors add
// with random signs over the max(n, m) entries of the marginal.
inline double armijo_floor32(int64_t n, int64_t m) {
  return (1.0 / 4194304.0) / std::sqrt((double)(n > m ? n : m));
}
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

// Programmatic dependent launch (sm_90+): a kernel launched with programmatic
// stream serialisation may start while its predecessor drains. Everything that
// reads data written by earlier kernels, or writes anything, comes after
// pdl_wait(); only loads of the immutable cost matrix may precede it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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

// L2 policy for cost loads: with keep != 0 the cost's lines are marked
// evict-last, so that a cost that fits in L2 stays resident across the many
// sweeps of a solve (l2_demote_kernel resets the priority at the end).
__device__ __forceinline__ uint64_t cost_policy(int keep) {
  uint64_t pol;
  if (keep) asm volatile("createpolicy.fractional.L2::evict_last.L2::evict_unchanged.b64 %0, 1.0;" : "=l"(pol));
  else asm volatile("createpolicy.fractional.L2::evict_normal.L2::evict_unchanged.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// streaming 16-byte loads of the cost matrix: no L1 allocation, L2 policy `pol`
__device__ __forceinline__ void ld_stream(const float* p, float (&c)[4], uint64_t pol) {
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(c[0]), "=f"(c[1]), "=f"(c[2]), "=f"(c[3]) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld_stream(const double* p, double (&c)[2], uint64_t pol) {
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
               : "=d"(c[0]), "=d"(c[1]) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld_stream(const float* p, float (&c)[1], uint64_t pol) {
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(c[0]) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld_stream(const double* p, double (&c)[1], uint64_t pol) {
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(c[0]) : "l"(p), "l"(pol));
}

// Asynchronous global -> shared copies (cg: L2 only; ca: through L1), completed
// by cp.async.wait_all of the issuing thread.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16_ca(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Thread-block clusters: a barrier over the cluster's CTAs (every thread of
// every CTA arrives; writes before it are visible to reads after it), the CTA's
// rank in its cluster, and a read of another CTA's shared memory.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ float2 ld_cluster_f2(const float2* p, uint32_t rank) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(ra) : "memory");
  return v;
}

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

// Compensated (Neumaier) accumulation s + c += x. In FP32 it keeps the running
// sums of the sweeps accurate to about one rounding without FP64 instructions in
// the inner loops (the FP64 pipe of this GPU is narrow); in FP64 it is a plain add.
__device__ __forceinline__ void kadd(float& s, float& c, float x) {
  // __fadd_rn / __fsub_rn: never contracted with a product that formed x
  const float t = __fadd_rn(s, x);
  c += (fabsf(s) >= fabsf(x)) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s);
  s = t;
}
__device__ __forceinline__ void kadd(double& s, double& c, double x) { s += x; }

// Warp-wide sum of Neumaier pairs (s, c) in FP32 (compensated at every step).
// The xor butterfly gives every lane the same bits (the steps are symmetric).
__device__ __forceinline__ void warp_sum_pair(float& s, float& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    kadd(s, c, s2);
    c += c2;
  }
}
__device__ __forceinline__ float warp_max_f(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// V consecutive elements from shared memory (16-byte aligned when V > 1)
template <int V, class T>
__device__ __forceinline__ void ld_vec_smem(const T* p, T (&c)[V]) {
  if constexpr (V == 4 && sizeof(T) == 4) {
    const float4 x = *reinterpret_cast<const float4*>(p);
    c[0] = x.x; c[1] = x.y; c[2] = x.z; c[3] = x.w;
  } else if constexpr (V == 2 && sizeof(T) == 8) {
    const double2 x = *reinterpret_cast<const double2*>(p);
    c[0] = x.x; c[1] = x.y;
  } else {
#pragma unroll
    for (int e = 0; e < V; ++e) c[e] = p[e];
  }
}

// 16-byte vector type of an element type, and packing V = 16 / sizeof(T) elements
template <class T>
struct VecOf;
template <>
struct VecOf<float> {
  typedef float4 type;
};
template <>
struct VecOf<double> {
  typedef double2 type;
};
template <class T>
__device__ __forceinline__ typename VecOf<T>::type pack(const T (&x)[16 / sizeof(T)]) {
  if constexpr (sizeof(T) == 4) return make_float4(x[0], x[1], x[2], x[3]);
  else return make_double2(x[0], x[1]);
}

// In-order combine of a strided sequence base[k * stride], k < cnt, written by
// earlier CTAs: the loads go out in batches of B (independent L2 round trips
// overlap) and f(value) consumes them in index order, so the result is the same
// as a plain sequential loop.
template <int B = 8, class V, class F>
__device__ __forceinline__ void ordered_loads(const V* base, int64_t stride, int64_t cnt, F&& f) {
  for (int64_t k0 = 0; k0 < cnt; k0 += B) {
    V q[B];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (k0 + u < cnt) q[u] = __ldcg(base + (k0 + u) * stride);
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (k0 + u < cnt) f(q[u]);
  }
}
// The same for two sequences read in step: f(a_k, b_k).
template <int B = 8, class V, class W, class F>
__device__ __forceinline__ void ordered_loads2(const V* a, const W* b, int64_t stride, int64_t cnt, F&& f) {
  for (int64_t k0 = 0; k0 < cnt; k0 += B) {
    V qa[B];
    W qb[B];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (k0 + u < cnt) {
        qa[u] = __ldcg(a + (k0 + u) * stride);
        qb[u] = __ldcg(b + (k0 + u) * stride);
      }
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (k0 + u < cnt) f(qa[u], qb[u]);
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
// Combine two pairs. The scaling factor exp(m - M) is formed in the element type
// T: one FP32 rounding is far below the FP32 path's own error, and it keeps the
// FP64 pipe free; the FP64 path scales in FP64.
template <class T = double>
__device__ __forceinline__ LsePair lse_combine(LsePair a, LsePair b) {
  if (b.s == 0.0) return a;
  if (a.s == 0.0) return b;
  const double M = fmax(a.m, b.m);
  return {M, a.s * (double)expT((T)(a.m - M)) + b.s * (double)expT((T)(b.m - M))};
}
template <class T = double>
__device__ __forceinline__ LsePair warp_lse(LsePair p) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    LsePair q{__shfl_xor_sync(0xffffffffu, p.m, o), __shfl_xor_sync(0xffffffffu, p.s, o)};
    p = lse_combine<T>(p, q);
  }
  return p;
}

__device__ __forceinline__ float warp_sum_f(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
// warp sum in the element type (FP32 path: FP32 shuffles and adds)
__device__ __forceinline__ double warp_sum_t(float x) { return (double)warp_sum_f(x); }
__device__ __forceinline__ double warp_sum_t(double x) { return warp_sum(x); }

}  // namespace eot
