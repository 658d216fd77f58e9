// Bulk-copy sweeps over a dense FP32 cost (the same reductions as sweep.cuh).
//
// One persistent CTA per SM streams its share of the cost through a ring of
// 16 KB shared-memory stages filled by 1-D bulk copies (the TMA engine): one
// producer thread issues the copies, each completing on the stage's "full"
// mbarrier, and the consumer warps release a stage through its "empty"
// mbarrier once they have reduced it. A handful of copies keeps the whole
// ring (up to 192 KB per SM) in flight, where the register-load sweeps need
// every thread to hold its own loads; this is what lets a sweep over a cost
// that stays resident in L2 across the sweeps of a solve run at L2 rather than
// load-issue speed.
//
// Row sweep   : consumer warp w owns the CTA's rows w, w + NW, ... and its own
//               two ring stages (a row of up to 4096 columns per stage, longer
//               rows in several stages); the column vectors (Bh and weights)
//               sit in shared memory for the whole sweep. Row results are
//               formed exactly as in row_sweep_kernel.
// Column sweep: CTA (strip s, row block b) owns SW columns x BR rows; a stage
//               holds 16 KB / (4 SW) rows of the strip (one copy per row) and
//               every consumer warp reduces every stage, each thread four
//               columns of a subset of the stage's rows. Partials, tickets and
//               the strip's fixed-order finish are those of col_sweep_kernel.
//
// Every wait is bounded (tc::mbar_wait): on expiry the kernel sets kStatTimeout
// in the status word, stops issuing copies, waits (again bounded) for the
// copies already in flight and leaves; the host reads the status and raises.
#pragma once
#include <cuda.h>

#include "sweep.cuh"
#include "tc.cuh"

namespace eot {
namespace bulk {

constexpr int kStageF = 4096;                   // floats per ring stage
constexpr int kStageBytes = kStageF * 4;        // 16 KB
constexpr int kBarBytes = 1024;                 // mbarriers at the start of shared memory
constexpr int kSmemOptIn = 232448;              // 227 KB of opt-in shared memory per CTA
constexpr int kColWarps = 8;                    // consumer warps of the column sweep
constexpr int kColThreads = (kColWarps + 1) * 32;
constexpr int kColMaxStages = 12;
constexpr int kColSW = 256;                     // column sweep: strip width = tensor box width
constexpr int kColRB = kStageF / kColSW;        // column sweep: rows per stage = tensor box height
constexpr int64_t kMinEntries = (int64_t)1 << 20;  // smaller sweeps keep the register-load kernels

// 1-D bulk copy global -> shared with an L2 cache policy, completing on an mbarrier
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                          uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
      "%4;" ::"r"(tc::smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(tc::smem_u32(bar)), "l"(pol)
      : "memory");
}

// 2-D tensor copy of a box (kColSW x kColRB elements at column x, row y) into
// shared memory, L2 policy `pol`; parts of the box outside the cost read as 0
__device__ __forceinline__ void tensor_load(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                            uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(tc::smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(tc::smem_u32(bar)), "l"(pol)
      : "memory");
}

// bounded wait with a fast path: the first poll before any timer read
__device__ __forceinline__ bool wait_fast(uint64_t* bar, uint32_t parity, int* err) {
  if (tc::mbar_try_wait(bar, parity)) return true;
  return tc::mbar_wait(bar, parity, err, kStatTimeout);
}

// barrier over the consumer warps only (the producer thread keeps issuing)
__device__ __forceinline__ void consumers_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Shared memory of a row sweep with `stages` ring stages and NV column vectors of length m.
inline size_t row_smem_bytes(int stages, int nv, int64_t m) {
  return (size_t)kBarBytes + (size_t)stages * kStageBytes + (size_t)nv * m * 4;
}

// ----------------------------------------------------------------------------
// Row sweep consumers: one stage (len columns from column c0 of the row), the
// lane-strided 16-byte layout of row_sweep_kernel, FP32 batches of 16 entries
// added into the compensated pairs.
// ----------------------------------------------------------------------------
template <int NR, int SQM>
__device__ __forceinline__ void stage_row_sum(const float* st, const float* vb, int64_t m, int len, int lane,
                                              float ah, float g, float (&S)[NR], float (&Cc)[NR]) {
  for (int q0 = lane * 4; q0 < len; q0 += 512) {
    float acc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc[k] = 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = q0 + u * 128;
      if (q >= len) break;
      const float4 c = *reinterpret_cast<const float4*>(st + q);
      const float4 b = *reinterpret_cast<const float4*>(vb + q);
      float4 w[NR];
#pragma unroll
      for (int k = 0; k < NR; ++k) w[k] = *reinterpret_cast<const float4*>(vb + (int64_t)(1 + k) * m + q);
      const float cc[4] = {c.x, c.y, c.z, c.w}, bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float x = expT(fmaf(-g, cc[e], ah + bb[e]));
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          const float we = e == 0 ? w[k].x : e == 1 ? w[k].y : e == 2 ? w[k].z : w[k].w;
          if ((SQM >> k) & 1) acc[k] = fmaf(x * x, we, acc[k]);
          else acc[k] = fmaf(x, we, acc[k]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) kadd(S[k], Cc[k], acc[k]);
  }
}

// Online LSE of t + log w over one stage (running max on the 1/8 grid, raised
// lazily as in row_reduce_lse; the first element of the lane starts it).
__device__ __forceinline__ void stage_row_lse(const float* st, const float* vb, int64_t m, int len, int lane,
                                              float ah, float g, float& mx, float& am, bool& mx_set, float& S,
                                              float& Cc) {
  if (!mx_set && lane * 4 < len) {
    mx = ceil_grid(fmaf(-g, st[lane * 4], ah + vb[lane * 4]));
    am = ah - mx;
    mx_set = true;
  }
  for (int q0 = lane * 4; q0 < len; q0 += 512) {
    float acc = 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = q0 + u * 128;
      if (q >= len) break;
      const float4 c = *reinterpret_cast<const float4*>(st + q);
      const float4 b = *reinterpret_cast<const float4*>(vb + q);
      const float4 w = *reinterpret_cast<const float4*>(vb + m + q);
      const float cc[4] = {c.x, c.y, c.z, c.w}, bb[4] = {b.x, b.y, b.z, b.w}, ww[4] = {w.x, w.y, w.z, w.w};
      float t[4];
      float tmax = -3.0e38f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        t[e] = fmaf(-g, cc[e], am + bb[e]);
        tmax = fmaxf(tmax, t[e]);
      }
      for (int k = 0; k < 4 && tmax > kTheta; ++k) {
        const float dlt = ceil_grid(tmax);
        mx += dlt;
        am = ah - mx;
        const float f = expT(-dlt);
        acc *= f;
        S *= f;
        Cc *= f;
        tmax = -3.0e38f;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          t[e] = fmaf(-g, cc[e], am + bb[e]);
          tmax = fmaxf(tmax, t[e]);
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) acc = fmaf(expT(t[e]), ww[e], acc);
    }
    kadd(S, Cc, acc);
  }
}

// ----------------------------------------------------------------------------
// Row sweep: grid = CTAs (<= SMs), CTA b owns rows [n b / G, n (b + 1) / G);
// (NW + 1) warps, warp NW is the producer; consumer warp w owns NS ring stages;
// dynamic shared memory row_smem_bytes(NW * NS, NV, m). Requires m % 4 == 0,
// ldc % 4 == 0 and a 16-byte aligned cost, Bh and weights.
// ----------------------------------------------------------------------------
template <int NW, int NS, int NR, bool LSE, int SQM, class Epi>
__global__ void __launch_bounds__((NW + 1) * 32, 1) row_bulk_kernel(SweepArgs<float> a, Epi epi) {
  constexpr int NV = 1 + (LSE ? 1 : NR);
  constexpr int NA = LSE ? 1 : NR;
  constexpr int ND = Epi::kDot;
  static_assert(2 * NW * NS + 1 <= kBarBytes / 8, "mbarriers exceed their area");
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + NW * NS;
  uint64_t* vbar = empty + NW * NS;  // the column vectors
  float* ring = reinterpret_cast<float*>(smem + kBarBytes);
  float* sv = ring + (size_t)NW * NS * kStageF;  // [NV][m]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m = a.m;
  const int tw = (int)min((int64_t)kStageF, m);
  const int64_t T = (m + tw - 1) / tw;  // stages per row
  const int64_t i0 = a.n * blockIdx.x / gridDim.x, i1 = a.n * (blockIdx.x + 1) / gridDim.x;
  const int64_t nrows = i1 - i0;
  const uint64_t pol = cost_policy(a.keep_l2);

  if (threadIdx.x == 0) {
    for (int k = 0; k < NW * NS; ++k) {
      tc::mbar_init(&full[k], 1);
      tc::mbar_init(&empty[k], 1);
    }
    tc::mbar_init(vbar, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();

  // stage p of warp w: local row w + (p / T) NW, columns [(p % T) tw, ...), slot w NS + p % NS
  const bool producer = warp == NW && lane == 0;
  int64_t nst[NW], iss[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    nst[w] = nrows > w ? ((nrows - 1 - w) / NW + 1) * T : 0;
    iss[w] = 0;
  }
  auto issue = [&](int w) {
    const int64_t p = iss[w]++;
    const int64_t i = i0 + w + (p / T) * NW;
    const int64_t c0 = (p % T) * tw;
    const uint32_t bytes = (uint32_t)min((int64_t)tw, m - c0) * 4u;
    const int slot = w * NS + (int)(p % NS);
    tc::mbar_arrive_expect_tx(&full[slot], bytes);
    bulk_load(ring + (size_t)slot * kStageF, a.C + i * a.ldc + c0, bytes, &full[slot], pol);
  };
  // The first stages of the (immutable) cost go out before the wait, unless the
  // predecessor has already cleared the active flag (a hint only: the flag is
  // read again after the wait).
  const bool hint = !(a.active && *(volatile const double*)a.active == 0.0);
  if (producer && hint) {
#pragma unroll
    for (int w = 0; w < NW; ++w)
      while (iss[w] < NS && iss[w] < nst[w]) issue(w);
  }
  pdl_wait();
  const bool active = !(a.active && *a.active == 0.0);
  double wd[ND > 0 ? ND : 1];
#pragma unroll
  for (int k = 0; k < (ND > 0 ? ND : 1); ++k) wd[k] = 0.0;

  if (warp == NW) {
    if (producer) {
      bool ok = active;
      if (active) {
        // the column vectors, written by earlier kernels
        tc::mbar_arrive_expect_tx(vbar, (uint32_t)(NV * m * 4));
        tc::bulk_g2s(sv, a.Bh, (uint32_t)(m * 4), vbar);
#pragma unroll
        for (int k = 0; k < NV - 1; ++k) tc::bulk_g2s(sv + (1 + k) * m, a.wc[k], (uint32_t)(m * 4), vbar);
      }
      // remaining stages: whichever warp has released its next slot gets it
      int64_t left = 0;
#pragma unroll
      for (int w = 0; w < NW; ++w) left += nst[w] - iss[w];
      uint32_t idle = 0;
      unsigned long long t_idle = 0;
      while (ok && left > 0) {
        bool any = false;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const int64_t p = iss[w];
          if (p >= nst[w]) continue;
          if (p >= NS && !tc::mbar_try_wait(&empty[w * NS + (int)(p % NS)], (uint32_t)(((p / NS) - 1) & 1)))
            continue;
          issue(w);
          --left;
          any = true;
        }
        if (any) {
          idle = 0;
        } else {
          if (idle == 0) t_idle = tc::now_ns();
          if ((++idle & 15u) == 0u) {
            if (*(volatile int*)a.err & kStatTimeout) {
              ok = false;
            } else if ((idle >= tc::kMinPolls && tc::now_ns() - t_idle > tc::kTcWaitNs) || idle >= tc::kMaxPolls) {
              atomicOr(a.err, kStatTimeout);
              ok = false;
            }
          }
        }
      }
      // every issued copy lands before the CTA leaves (normally the consumers
      // have waited for all of them already)
      const unsigned long long lim = ok ? tc::kTcWaitNs : tc::kTcDrainNs;
#pragma unroll
      for (int w = 0; w < NW; ++w)
        for (int64_t p = iss[w] > NS ? iss[w] - NS : 0; p < iss[w]; ++p)
          tc::mbar_wait(&full[w * NS + (int)(p % NS)], (uint32_t)((p / NS) & 1), a.err, kStatTimeout, lim);
      if (active) tc::mbar_wait(vbar, 0u, a.err, kStatTimeout, lim);
    }
  } else if (active) {
    const float g = a.gamma_dev ? (float)*a.gamma_dev : a.gamma;
    bool ok = __all_sync(0xffffffffu, wait_fast(vbar, 0u, a.err));
    int64_t p = 0;
    for (int64_t r = warp; ok && r < nrows; r += NW) {
      const int64_t i = i0 + r;
      const float ah = a.Ah[i];
      float S[NA], Cc[NA];
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        S[k] = 0.f;
        Cc[k] = 0.f;
      }
      float mx = 0.f, am = ah;
      bool mx_set = false;
      for (int64_t c = 0; c < T; ++c, ++p) {
        const int slot = warp * NS + (int)(p % NS);
        if (!__all_sync(0xffffffffu, wait_fast(&full[slot], (uint32_t)((p / NS) & 1), a.err))) {
          ok = false;
          break;
        }
        const float* st = ring + (size_t)slot * kStageF;
        const int len = (int)min((int64_t)tw, m - c * tw);
        const float* vb = sv + c * tw;
        if constexpr (!LSE) stage_row_sum<NR, SQM>(st, vb, m, len, lane, ah, g, S, Cc);
        else stage_row_lse(st, vb, m, len, lane, ah, g, mx, am, mx_set, S[0], Cc[0]);
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&empty[slot]);
      }
      if (ok) row_result_f32<NA, LSE, ND>(i, lane, S, Cc, mx, mx_set, epi, wd);
    }
  }
  if (!active) return;  // uniform over the grid: no CTA reaches the dot finish
  pdl_trigger();
  cta_dot_finish<ND, Epi, NW + 1>(wd, blockIdx.x, gridDim.x, a.dotpart, a.cnt_dot, epi);
}

// ----------------------------------------------------------------------------
// Column sweep: grid = (S strips of kColSW columns, R = a.nrowblk row blocks of
// BR = a.rows_per_block rows, a multiple of kColRB); kColThreads threads, warp
// kColWarps is the producer; one 2-D tensor copy (kColSW x kColRB, map `tmap`
// over the n x m cost) per 16 KB stage; dynamic shared memory kBarBytes +
// a.stages * 16 KB + the block's row vectors (3 BR floats).
// ----------------------------------------------------------------------------
template <int NC, bool LSE, class Epi>
__global__ void __launch_bounds__(kColThreads, 1)
    col_bulk_kernel(SweepArgs<float> a, Epi epi, const __grid_constant__ CUtensorMap tmap) {
  constexpr int NT = kColWarps * 32;  // consumer threads
  constexpr int NP = LSE ? 2 : NC;    // partial arrays
  constexpr int ND = Epi::kDot;
  constexpr int SW = kColSW, RBs = kColRB;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int NS = a.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + kColMaxStages;
  float* ring = reinterpret_cast<float*>(smem + kBarBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t strip = blockIdx.x, S = gridDim.x;
  const int rb = blockIdx.y, R = a.nrowblk;
  const int64_t j0 = strip * SW;
  const int sw = (int)min((int64_t)SW, a.m - j0);
  const int64_t r0 = (int64_t)rb * a.rows_per_block;
  const int64_t r1 = min(a.n, r0 + (int64_t)a.rows_per_block);
  const int64_t nstg = (r1 - r0 + RBs - 1) / RBs;
  float* sAh = ring + (size_t)NS * kStageF;  // [BR] row offsets, then [NC][BR] row weights
  const uint64_t pol = cost_policy(a.keep_l2);

  if (threadIdx.x == 0) {
    for (int k = 0; k < NS; ++k) {
      tc::mbar_init(&full[k], 1);
      tc::mbar_init(&empty[k], kColWarps);
    }
    tc::mbar_fence_init();
  }
  __syncthreads();

  const bool producer = warp == kColWarps && lane == 0;
  int64_t iss = 0;
  auto issue = [&]() {
    const int64_t q = iss++;
    const int slot = (int)(q % NS);
    tc::mbar_arrive_expect_tx(&full[slot], (uint32_t)kStageBytes);
    tensor_load(ring + (size_t)slot * kStageF, &tmap, (int)j0, (int)(r0 + q * RBs), &full[slot], pol);
  };
  const bool hint = !(a.active && *(volatile const double*)a.active == 0.0);
  if (producer && hint)
    while (iss < NS && iss < nstg) issue();
  pdl_wait();
  const bool active = !(a.active && *a.active == 0.0);

  // consumer thread t: column group cg (4 columns), rows rl, rl + RP, ... of each stage
  constexpr int G4 = SW / 4, RP = NT / G4;
  const int cg = threadIdx.x % G4, rl = threadIdx.x / G4;
  const int64_t j = j0 + cg * 4;
  const bool jv = warp < kColWarps && cg * 4 < sw;
  float tot[NP][4], cmp[NP][4], mx[4];
#pragma unroll
  for (int k = 0; k < NP; ++k)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      tot[k][e] = 0.f;
      cmp[k][e] = 0.f;
    }
#pragma unroll
  for (int e = 0; e < 4; ++e) mx[e] = 0.f;

  if (warp == kColWarps) {
    if (producer) {
      bool ok = active;
      while (ok && iss < nstg) {
        const int64_t q = iss;
        if (q >= NS && !wait_fast(&empty[q % NS], (uint32_t)(((q / NS) - 1) & 1), a.err)) {
          ok = false;
          break;
        }
        issue();
      }
      const unsigned long long lim = ok ? tc::kTcWaitNs : tc::kTcDrainNs;
      for (int64_t q = iss > NS ? iss - NS : 0; q < iss; ++q)
        tc::mbar_wait(&full[q % NS], (uint32_t)((q / NS) & 1), a.err, kStatTimeout, lim);
    }
  } else if (active) {
    // the block's row offsets and weights, staged once
    const int64_t br = r1 - r0;
    for (int64_t q = threadIdx.x; q < br; q += NT) {
      sAh[q] = a.Ah[r0 + q];
#pragma unroll
      for (int k = 0; k < NC; ++k) sAh[(1 + k) * (int64_t)a.rows_per_block + q] = a.wr[k][r0 + q];
    }
    consumers_sync(NT);
    const float g = a.gamma_dev ? (float)*a.gamma_dev : a.gamma;
    float b[4] = {0.f, 0.f, 0.f, 0.f}, bm[4];
    if (jv) {
      const float4 bb = __ldg(reinterpret_cast<const float4*>(a.Bh + j));
      b[0] = bb.x; b[1] = bb.y; b[2] = bb.z; b[3] = bb.w;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) bm[e] = b[e];
    bool mx_set = false;
    for (int64_t q = 0; q < nstg; ++q) {
      const int slot = (int)(q % NS);
      if (!__all_sync(0xffffffffu, wait_fast(&full[slot], (uint32_t)((q / NS) & 1), a.err))) break;
      const float* st = ring + (size_t)slot * kStageF;
      const int64_t lr0 = q * RBs;  // block-local first row of the stage
      const int rows = (int)min((int64_t)RBs, (r1 - r0) - lr0);
      float acc[NP][4];
#pragma unroll
      for (int k = 0; k < NP; ++k)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[k][e] = 0.f;
      if (jv) {
        if constexpr (!LSE) {
          for (int rr = rl; rr < rows; rr += RP) {
            const float4 c = *reinterpret_cast<const float4*>(st + rr * SW + cg * 4);
            const float cc[4] = {c.x, c.y, c.z, c.w};
            const float hh = sAh[lr0 + rr];
            const float x0 = sAh[(int64_t)a.rows_per_block + lr0 + rr];
            float x1 = 0.f;
            if constexpr (NC > 1) x1 = sAh[2 * (int64_t)a.rows_per_block + lr0 + rr];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float x = expT(fmaf(-g, cc[e], hh + b[e]));
              acc[0][e] = fmaf(x, x0, acc[0][e]);
              if constexpr (NC > 1) acc[1][e] = fmaf(x, x1, acc[1][e]);
            }
          }
        } else {
          // per column: the stage's t (4 rows per thread at every SW), the
          // running max raised at most 4 times (as in col_sweep_kernel), then
          // the weighted sum
          for (int rr0 = rl; rr0 < rows; rr0 += 4 * RP) {
            float cv[4][4], hv[4], xv[4];
            int nr = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int rr = rr0 + u * RP;
              if (rr < rows) {
                const float4 c = *reinterpret_cast<const float4*>(st + rr * SW + cg * 4);
                cv[u][0] = c.x; cv[u][1] = c.y; cv[u][2] = c.z; cv[u][3] = c.w;
                hv[u] = sAh[lr0 + rr];
                xv[u] = sAh[(int64_t)a.rows_per_block + lr0 + rr];
                nr = u + 1;
              }
            }
            if (!mx_set) {
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                mx[e] = ceil_grid(fmaf(-g, cv[0][e], hv[0] + b[e]));
                bm[e] = b[e] - mx[e];
              }
              mx_set = true;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              float t[4];
              float tmax = -3.0e38f;
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                t[u] = fmaf(-g, cv[u][e], hv[u] + bm[e]);
                if (u < nr) tmax = fmaxf(tmax, t[u]);
              }
              for (int k = 0; k < 4 && tmax > kTheta; ++k) {
                const float dlt = ceil_grid(tmax);
                mx[e] += dlt;
                bm[e] = b[e] - mx[e];
                const float f = expT(-dlt);
                tot[1][e] *= f;
                cmp[1][e] *= f;
                acc[1][e] *= f;
                tmax = -3.0e38f;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  t[u] = fmaf(-g, cv[u][e], hv[u] + bm[e]);
                  if (u < nr) tmax = fmaxf(tmax, t[u]);
                }
              }
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (u < nr) acc[1][e] = fmaf(expT(t[u]), xv[u], acc[1][e]);
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < NP; ++k)
#pragma unroll
        for (int e = 0; e < 4; ++e) kadd(tot[k][e], cmp[k][e], acc[k][e]);
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&empty[slot]);
    }
  }
  if (!active) return;  // uniform over the grid
  pdl_trigger();
  // ---- combine the RP row lanes of each column (the ring is free now) ----
  __syncthreads();
  float* fsum = ring;                 // [NP][RP][SW]
  float* fcmp = fsum + NP * NT * 4;   // [NP][RP][SW]
  float* fmx = fcmp + NP * NT * 4;    // [RP][SW]
  if (warp < kColWarps) {
#pragma unroll
    for (int k = 0; k < NP; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        fsum[(k * RP + rl) * SW + cg * 4 + e] = tot[k][e];
        fcmp[(k * RP + rl) * SW + cg * 4 + e] = cmp[k][e];
      }
    if constexpr (LSE) {
#pragma unroll
      for (int e = 0; e < 4; ++e) fmx[rl * SW + cg * 4 + e] = mx[e];
    }
  }
  __syncthreads();
  float2* cp2 = reinterpret_cast<float2*>(a.colpart);
  for (int cc = threadIdx.x; cc < sw; cc += kColThreads) {
    const int64_t jj = j0 + cc;
    if constexpr (!LSE) {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        float s0 = 0.f, c0 = 0.f;
        for (int w = 0; w < RP; ++w) {
          kadd(s0, c0, fsum[(k * RP + w) * SW + cc]);
          c0 += fcmp[(k * RP + w) * SW + cc];
        }
        cp2[((int64_t)k * R + rb) * a.m + jj] = make_float2(s0, c0);
      }
    } else {
      float M = -INFINITY;
      for (int w = 0; w < RP; ++w)
        if (fsum[(RP + w) * SW + cc] != 0.f || fcmp[(RP + w) * SW + cc] != 0.f) M = fmaxf(M, fmx[w * SW + cc]);
      float s0 = 0.f, c0 = 0.f;
      for (int w = 0; w < RP; ++w) {
        const float sv = fsum[(RP + w) * SW + cc], cv = fcmp[(RP + w) * SW + cc];
        if (sv == 0.f && cv == 0.f) continue;
        const float f = expT(fmx[w * SW + cc] - M);
        kadd(s0, c0, sv * f);
        c0 += cv * f;
      }
      cp2[((int64_t)0 * R + rb) * a.m + jj] = make_float2(M, 0.f);
      cp2[((int64_t)1 * R + rb) * a.m + jj] = make_float2(s0, c0);
    }
  }

  // ---- ticket: the last CTA of the strip combines the R partials ----
  __shared__ int last_strip;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last_strip = (atomicAdd(a.cnt_strip + strip, 1) == R - 1);
  }
  __syncthreads();
  if (last_strip) {
    __threadfence();
    double wd[ND > 0 ? ND : 1];
#pragma unroll
    for (int k = 0; k < (ND > 0 ? ND : 1); ++k) wd[k] = 0.0;
    for (int cc = threadIdx.x; cc < sw; cc += kColThreads) {
      DotArr<ND> d;
      col_combine_f32<NC, LSE>(cp2, R, a.m, j0 + cc, epi, d.v);
#pragma unroll
      for (int k = 0; k < ND; ++k) wd[k] += d.v[k];
    }
    if (threadIdx.x == 0) a.cnt_strip[strip] = 0;
    if constexpr (ND > 0) {
#pragma unroll
      for (int k = 0; k < ND; ++k) wd[k] = warp_sum(wd[k]);
      cta_dot_finish<ND, Epi, kColWarps + 1>(wd, strip, S, a.dotpart, a.cnt_dot, epi);
    }
  }
}

}  // namespace bulk
}  // namespace eot
