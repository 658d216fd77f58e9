// The whole linear CG solve of NewtonSolve (Alg. 2, inner PCG on F_r(rho)) as ONE
// persistent cooperative kernel, for dense FP32 costs on the mixed path.
//
// Every CG iteration is the same arithmetic as the per-kernel path (CgColEpi,
// CgRowEpi, cg_update_kernel, cg_pupdate_kernel), in four phases separated by
// grid barriers instead of kernel boundaries:
//   A  column half  w_j = sum_i E_ij xw_i, xw_i = rowfac_i p_i with
//      p = z + beta p formed on the fly (p double-buffered: read one array,
//      the strip-0 CTAs write the other); CTA partials as FP32 pairs [R][m];
//   C  column finalize, columns spread over the CTAs: zf_j = colfac_j^2 w_j / c_j;
//   E  row half  y_i = rowfac_i sum_j E_ij zf_j, q_i = rPs_i p_i - rho y_i,
//      CTA partials of <p, q>;
//   G  alpha = rz / <p, q> (every CTA, same order), x += alpha p,
//      res -= alpha q, Yx += alpha y, z = res / M; partials of <res, z>, |res|;
//   then beta, the stop test (every CTA decides alike) and the next iteration.
// The barriers count arrivals in global memory and wait with a bounded spin; a
// CTA that gives up sets kStatTimeout and an abort word, so all CTAs leave.
#pragma once
#include "kernels.cuh"

namespace eot {
namespace pcg {

struct Args {
  const float* C;
  int64_t n, m, ldc;
  const float *Ah, *Bh;
  const double *rowfac, *colfac, *cP, *rPs, *M;
  double *x, *res, *z, *q, *y, *Yx;
  double* pbuf[2];   // p, double-buffered by iteration parity
  float *xw, *zf;    // zf: row weights of phase E
  float2* colpart;   // [R][m]
  double* dots;      // [2][G][2] CTA partials
  double* sc;        // solver scalars (SC_*)
  unsigned* bar;     // grid barrier counter (zero at launch)
  int* abort;        // set by a CTA whose barrier wait ran out
  int* status;
  int R, S;          // row blocks and column strips of phase A (grid = R * S)
  int rows_per_block;
  int keep_l2;
};

constexpr int kSW = 128;  // columns per strip (32 lanes x float4)

__device__ __forceinline__ unsigned long long pnow() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acq(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier number `gen` (1, 2, ...); false if this CTA or another gave up.
__device__ __forceinline__ bool grid_bar(const Args& a, unsigned gen, int& fail) {
  __syncthreads();
  if (threadIdx.x == 0 && !fail) {
    __threadfence();
    atomicAdd(a.bar, 1u);
    const unsigned target = gen * gridDim.x;
    const unsigned long long t0 = pnow();
    for (unsigned it = 0;; ++it) {
      if ((int)(ld_acq(a.bar) - target) >= 0) break;
      if ((it & 63u) == 63u) {
        if (*(volatile int*)a.abort) {
          fail = 1;
          break;
        }
        // time alone is not trusted (it can jump under a profiler): also a poll count
        if ((it >= (1u << 16) && pnow() - t0 > 2000000000ull) || it >= (1u << 26)) {
          atomicExch(a.abort, 1);
          atomicOr(a.status, kStatTimeout);
          fail = 1;
          break;
        }
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  return true;  // the caller checks the shared fail flag
}

// Deterministic sum of G CTA partials (each CTA computes the same value).
__device__ __forceinline__ void sum_partials(const double* part, int G, double (&out)[2], double* sh) {
  double v0 = 0.0, v1 = 0.0;
  for (int g = threadIdx.x; g < G; g += kThreads) {
    v0 += __ldcg(part + 2 * g);
    v1 += __ldcg(part + 2 * g + 1);
  }
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sh[2 * warp] = v0;
    sh[2 * warp + 1] = v1;
  }
  __syncthreads();
  double t0 = 0.0, t1 = 0.0;
  for (int w = 0; w < kWarps; ++w) {
    t0 += sh[2 * w];
    t1 += sh[2 * w + 1];
  }
  out[0] = t0;
  out[1] = t1;
  __syncthreads();
}

// CTA-level deterministic sum of two per-thread values into part[2 * blockIdx.x + k].
__device__ __forceinline__ void cta_partial(double v0, double v1, double* part, double* sh) {
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sh[2 * warp] = v0;
    sh[2 * warp + 1] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      t0 += sh[2 * w];
      t1 += sh[2 * w + 1];
    }
    part[2 * blockIdx.x] = t0;
    part[2 * blockIdx.x + 1] = t1;
  }
  __syncthreads();
}


constexpr int kTWp = 4096;  // columns staged for phase E (the persistent path takes m <= kTWp)

static __global__ void __launch_bounds__(kThreads, 2) cg_persistent_kernel(Args a) {
  __shared__ int fail;
  __shared__ double sh[2 * kWarps];
  __shared__ float fsum[kWarps][kSW], fcmp[kWarps][kSW];
  __shared__ __align__(16) float svb[kTWp], svz[kTWp];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = gridDim.x;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  if (a.sc[SC_ACTIVE] == 0.0) return;  // nothing to iterate (uniform)
  const int strip = (int)(blockIdx.x % a.S), rb = (int)(blockIdx.x / a.S);
  const int64_t n = a.n, m = a.m;
  const int64_t r0 = (int64_t)rb * a.rows_per_block, r1 = min(n, r0 + (int64_t)a.rows_per_block);
  const int64_t jA = (int64_t)strip * kSW + lane * 4;
  const bool jv = jA < m;  // m % 4 == 0: a lane's four columns are all valid or all not
  const float g = (float)a.sc[SC_GAMMA];
  const double rho = a.sc[SC_RHO], tol = a.sc[SC_TOL], maxit = a.sc[SC_MAXIT];
  double rz = a.sc[SC_RZ], beta = 0.0, resl1 = a.sc[SC_RESL1], iters = 0.0, alpha = 0.0, pq = 0.0;
  const uint64_t pol = cost_policy(a.keep_l2);
  float bA[4] = {0.f, 0.f, 0.f, 0.f};
  if (jv) ld_vec<4>(a.Bh + jA, bA);
  const int64_t u0 = (int64_t)blockIdx.x * n / G, u1 = (int64_t)(blockIdx.x + 1) * n / G;
  const int64_t c0 = (int64_t)blockIdx.x * m / G, c1 = (int64_t)(blockIdx.x + 1) * m / G;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, Gw = (int64_t)G * kWarps;
  unsigned gen = 0;
  int par = 0;
  bool curv = false;
  for (;;) {
    const double* pold = a.pbuf[par];
    double* pnew = a.pbuf[par ^ 1];
    // ---------------- A: column half, p = z + beta p on the fly ----------------
    {
      float S[4] = {0.f, 0.f, 0.f, 0.f}, Cc[4] = {0.f, 0.f, 0.f, 0.f};
      constexpr int U = 4;
      constexpr int64_t STEP = (int64_t)kWarps * U;
      // batch of U rows of this warp: cost float4s and the row scalars
      auto load = [&](int64_t i0, float (&c)[U][4], float (&ah)[U], float (&xw)[U]) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t i = i0 + (int64_t)u * kWarps;
          if (i < r1) {
            if (jv) ld_stream(a.C + i * a.ldc + jA, c[u], pol);
            const double pn = __ldcg(a.z + i) + beta * __ldcg(pold + i);
            if (strip == 0 && lane == 0) pnew[i] = pn;
            ah[u] = a.Ah[i];
            xw[u] = (float)(a.rowfac[i] * pn);
          } else {
            ah[u] = 0.f;
            xw[u] = 0.f;
          }
        }
      };
      auto reduce = [&](int64_t i0, const float (&c)[U][4], const float (&ah)[U], const float (&xw)[U]) {
        if (!jv) return;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (i0 + (int64_t)u * kWarps >= r1) continue;
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[e] = fmaf(expT(fmaf(-g, c[u][e], ah[u] + bA[e])), xw[u], acc[e]);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) kadd(S[e], Cc[e], acc[e]);
      };
      float cA[U][4], cB[U][4], hA[U], hB[U], wA[U], wB[U];
      int64_t i0 = r0 + warp;
      if (i0 < r1) {
        load(i0, cA, hA, wA);
        for (;;) {
          const int64_t i1 = i0 + STEP;
          if (i1 < r1) load(i1, cB, hB, wB);
          reduce(i0, cA, hA, wA);
          if (i1 >= r1) break;
          const int64_t i2 = i1 + STEP;
          if (i2 < r1) load(i2, cA, hA, wA);
          reduce(i1, cB, hB, wB);
          if (i2 >= r1) break;
          i0 = i2;
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        fsum[warp][lane * 4 + e] = S[e];
        fcmp[warp][lane * 4 + e] = Cc[e];
      }
      __syncthreads();
      if (threadIdx.x < kSW) {
        const int64_t jc = (int64_t)strip * kSW + threadIdx.x;
        if (jc < m) {
          float s0 = 0.f, cc0 = 0.f;
          for (int w = 0; w < kWarps; ++w) {
            kadd(s0, cc0, fsum[w][threadIdx.x]);
            cc0 += fcmp[w][threadIdx.x];
          }
          a.colpart[(int64_t)rb * m + jc] = make_float2(s0, cc0);
        }
      }
    }
    grid_bar(a, ++gen, fail);
    if (fail) break;
    // ---------------- C: column finalize ----------------
    for (int64_t jc = c0 + threadIdx.x; jc < c1; jc += kThreads) {
      float s0 = 0.f, cc0 = 0.f;
      for (int r = 0; r < a.R; ++r) {
        const float2 qv = __ldcg(a.colpart + (int64_t)r * m + jc);
        kadd(s0, cc0, qv.x);
        cc0 += qv.y;
      }
      const double f = a.colfac[jc];
      a.zf[jc] = (float)(f * f * ((double)s0 + (double)cc0) / a.cP[jc]);
    }
    grid_bar(a, ++gen, fail);
    if (fail) break;
    // ---------------- E: row half ----------------
    {
      for (int qq = threadIdx.x; qq < m; qq += kThreads) {
        svb[qq] = a.Bh[qq];
        svz[qq] = __ldcg(a.zf + qq);
      }
      __syncthreads();
      double dpq = 0.0;
      constexpr int U = 4;
      constexpr int64_t STEP = 128 * U;
      for (int64_t i = gw; i < n; i += Gw) {
        const float* crow = a.C + i * a.ldc;
        const float ah = a.Ah[i];
        float s0 = 0.f, cc0 = 0.f;
        auto load = [&](int64_t j0, float (&c)[U][4]) {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int64_t jj = j0 + 128 * u;
            if (jj < m) ld_stream(crow + jj, c[u], pol);
          }
        };
        auto reduce = [&](int64_t j0, const float (&c)[U][4]) {
          float acc = 0.f;
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int64_t jj = j0 + 128 * u;
            if (jj >= m) continue;
            float bb[4], zz[4];
            ld_vec_smem<4>(&svb[jj], bb);
            ld_vec_smem<4>(&svz[jj], zz);
#pragma unroll
            for (int e = 0; e < 4; ++e) acc = fmaf(expT(fmaf(-g, c[u][e], ah + bb[e])), zz[e], acc);
          }
          kadd(s0, cc0, acc);
        };
        float cA[U][4], cB[U][4];
        int64_t j0 = (int64_t)lane * 4;
        if (j0 < m) {
          load(j0, cA);
          for (;;) {
            const int64_t j1 = j0 + STEP;
            if (j1 < m) load(j1, cB);
            reduce(j0, cA);
            if (j1 >= m) break;
            const int64_t j2 = j1 + STEP;
            if (j2 < m) load(j2, cA);
            reduce(j1, cB);
            if (j2 >= m) break;
            j0 = j2;
          }
        }
        warp_sum_pair(s0, cc0);
        if (lane == 0) {
          const double yi = a.rowfac[i] * ((double)s0 + (double)cc0);
          const double pi = __ldcg(pnew + i);
          const double qi = a.rPs[i] * pi - rho * yi;
          a.y[i] = yi;
          a.q[i] = qi;
          dpq += pi * qi;
        }
      }
      cta_partial(dpq, 0.0, a.dots, sh);
    }
    grid_bar(a, ++gen, fail);
    if (fail) break;
    // ---------------- G: alpha and the vector update ----------------
    {
      double t[2];
      sum_partials(a.dots, G, t, sh);
      pq = t[0];
      if (!(pq > 0.0) || !isfinite(pq)) {  // <p, F_r p> <= 0: keep the iterate (as CgRowEpi)
        curv = true;
        break;
      }
      alpha = rz / pq;
      double v0 = 0.0, v1 = 0.0;
      for (int64_t i = u0 + threadIdx.x; i < u1; i += kThreads) {
        const double pi = __ldcg(pnew + i);
        a.x[i] += alpha * pi;
        const double r = a.res[i] - alpha * __ldcg(a.q + i);
        a.res[i] = r;
        a.Yx[i] += alpha * __ldcg(a.y + i);
        const double zi = r / a.M[i];
        a.z[i] = zi;
        v0 += r * zi;
        v1 += fabs(r);
      }
      cta_partial(v0, v1, a.dots + 2 * G, sh);
    }
    grid_bar(a, ++gen, fail);
    if (fail) break;
    {
      double t[2];
      sum_partials(a.dots + 2 * G, G, t, sh);
      const double rz_new = t[0];
      resl1 = t[1];
      beta = rz_new / rz;
      rz = rz_new;
      iters += 1.0;
      bool go = resl1 > tol && iters < maxit && iters < 1.0e6;
      if (!isfinite(rz_new) || !isfinite(resl1)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.status, kStatCgNan);
        go = false;
      }
      if (!go) break;
    }
    par ^= 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (curv) atomicOr(a.status, kStatCurv);
    a.sc[SC_PQ] = pq;
    a.sc[SC_ALPHA] = curv ? 0.0 : alpha;
    a.sc[SC_RZ] = rz;
    a.sc[SC_BETA] = beta;
    a.sc[SC_RESL1] = resl1;
    a.sc[SC_ITERS] = iters;
    a.sc[SC_ACTIVE] = 0.0;
  }
}

}  // namespace pcg
}  // namespace eot
