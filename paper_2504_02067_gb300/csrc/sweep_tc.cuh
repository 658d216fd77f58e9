// Point-cloud sweeps whose cross term x_i . y_j runs on the tensor cores
// (tcgen05, kind::f16 on BF16, FP32 accumulation in TMEM), for the mixed path at
// larger d (up to 64 coordinates).
//
// Exactness (an exact-slice / Ozaki-style splitting). Both point sets are moved
// by one common centre (exact in FP64; distances are unchanged). Each point x is then scaled by
// 2^-e (e from its largest coordinate, so |x_k| < 2^e) and each coordinate cut
// into five signed 8-bit digits:  x_k = 2^e sum_s d_sk 2^-8(s+1)  (to 2^-40 of
// the largest coordinate). A digit is an integer of magnitude <= 255, exact in
// BF16; a digit product is an integer below 2^16, and a dot product over 64
// coordinates stays below 2^22, so every MMA of digit slices is EXACT in the FP32
// accumulator. The 15 slice pairs (s, t) with s + t <= 4 are added into five
// "level" accumulators S_L = sum_{s+t=L} D_s D_t^T, each below 5 * 2^22 < 2^24 and
// still exact; then
//     x . y = 2^(e_x + e_y - 16) (S_0 + 2^-8 S_1 + 2^-16 S_2 + 2^-24 S_3 + 2^-32 S_4)
// to ~2^-38 relative (pairs with s + t >= 5 and the 2^-40 digit truncation).
// The epilogue forms |x - y|^2 = |x|^2 + |y|^2 - 2 x.y as an FP32 pair (TwoSum,
// with |x|^2 precomputed as an FP32 pair from FP64), then the exponent exactly
// as the SIMT point sweep does (expo), exp, and the reductions.
//
// CTA roles (320 threads, one CTA per SM: 177 KB of shared memory):
//   warp 0, lane 0: bulk copies (the own 128 points' slices once; the other
//     side's 48-point tiles into two buffers) and the MMAs of each tile into one
//     of two TMEM accumulator buffers (5 levels x 48 columns each);
//   warp 1: TMEM allocation (512 columns) and release;
//   warps 2-9: epilogue. Warp w reads TMEM lanes 32 (w mod 4) .. +31 (one own
//     point per thread) and half (24) of the tile's 48 columns.
// The other side's per-point data (h, scale, |y|^2, weights) are read by the
// epilogue straight from global memory (the same address in all lanes: one L1
// broadcast).
// Hand-offs are mbarriers: full[b] (copies landed), mmad[b] (MMAs of buffer b
// done: accumulators readable and the slice buffer reusable), tfree[b] (the 8
// epilogue warps have read buffer b). Every wait is bounded (tc.cuh).
#pragma once
#include <cuda_bf16.h>

#include "sweep_pts.cuh"
#include "tc.cuh"

namespace eot {
namespace tc {

constexpr int kM = 128;     // own points per CTA = TMEM lanes = MMA M
constexpr int kN = 48;      // other-side points per tile = MMA N
constexpr int kSlices = 5;  // 8-bit digits per coordinate
constexpr int kLevels = 5;  // s + t = 0 .. 4
constexpr int kEpiWarps = 8;                  // 2 per TMEM lane quarter
constexpr int kParts = kEpiWarps / 4;          // column parts of a tile
constexpr int kPartCols = kN / kParts;         // 24 columns per epilogue warp and tile
constexpr int kTcThreads = 32 * (2 + kEpiWarps);
constexpr int kTcWarps = kTcThreads / 32;
constexpr uint32_t kRowB = 128;    // bytes per point and slice: 64 BF16 coordinates
constexpr uint32_t kOwnSlice = kM * kRowB;                          // 16 KB
constexpr uint32_t kOthSlice = kN * kRowB;                          // 6 KB
constexpr uint32_t kOffOth = kSlices * kOwnSlice;                   // 80 KB
constexpr int kSliceBufs = 3;                                       // tile tt: slice buffer tt % 3
constexpr uint32_t kOffCol = kOffOth + kSliceBufs * kSlices * kOthSlice;  // + 90 KB
constexpr uint32_t kOffBar = kOffCol;
constexpr uint32_t kSmemBytes = kOffBar + 128 + 1024;               // barriers + 1024-byte alignment slack
constexpr int kBufCols = kLevels * kN;                              // 240 TMEM columns per buffer
constexpr uint32_t kTmemCols = 512;
constexpr int64_t kPadRows = 384;                                   // lcm(kM, kN)
constexpr uint32_t kIdesc = idesc_bf16_f32(kM, kN);
constexpr int kMinD = 17;  // the tensor-core path serves d >= kMinD

// Precomputed per point set (fixed for a problem).
struct Side {
  const __nv_bfloat16* slices;  // [kSlices][npad][64], 128-byte swizzle per 8-row atom
  const float* sc;              // [npad] 2^e
  const float* nxh;             // [npad] |x|^2 as an FP32 pair
  const float* nxl;
  int64_t npad;
};
struct TcArgs {
  Side X, Y;
  int* err;  // status word: kStatTimeout on a wait that ran out
};

__host__ __device__ inline int64_t pad_rows(int64_t n) { return (n + kPadRows - 1) / kPadRows * kPadRows; }

// One warp per point (rows >= n and coordinates >= d are zero). Both point sets
// are first moved by the same centre (the first point of X): |x - y|^2 does not
// change, but |x|^2, |y|^2 and x.y become bounded by the data's extent, so the
// expansion |x|^2 + |y|^2 - 2 x.y keeps its relative accuracy however far the
// clouds lie from the origin. The differences are exact in FP64.
static __global__ void tc_prep_kernel(const float* X, int64_t n, int d, int64_t npad, const float* centre,
                                      __nv_bfloat16* sl, float* sc, float* nxh, float* nxl) {
  pdl_wait();
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= npad) return;
  double xv[2] = {0.0, 0.0};
  if (row < n) {
    if (lane < d) xv[0] = (double)X[row * d + lane] - (double)centre[lane];
    if (lane + 32 < d) xv[1] = (double)X[row * d + lane + 32] - (double)centre[lane + 32];
  }
  double mx = fmax(fabs(xv[0]), fabs(xv[1]));
  double q = xv[0] * xv[0] + xv[1] * xv[1];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    q += __shfl_xor_sync(0xffffffffu, q, o);
  }
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1): every |x_k| < 2^e
  if (lane == 0) {
    sc[row] = ldexpf(1.f, e);
    const float h = (float)q;
    nxh[row] = h;
    nxl[row] = (float)(q - (double)h);
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int k = lane + 32 * c;
    const double Qd = trunc(ldexp(xv[c], 40 - e));  // |Q| < 2^40
    const long long Q = (long long)Qd;
    const unsigned long long aQ = (unsigned long long)(Q < 0 ? -Q : Q);
    const float sgn = Q < 0 ? -1.f : 1.f;
    const int64_t idx = row * 64 + (((k >> 3) ^ (int)(row & 7)) << 3) + (k & 7);
#pragma unroll
    for (int s = 0; s < kSlices; ++s) {
      const unsigned dig = (unsigned)((aQ >> (8 * (kSlices - 1 - s))) & 255ull);
      sl[(int64_t)s * npad * 64 + idx] = __float2bfloat16_rn(sgn * (float)dig);
    }
  }
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = add_rn(a, b);
  const float z = sub_rn(s, a);
  e = add_rn(sub_rn(a, sub_rn(s, z)), sub_rn(b, z));
}

// Waits by lane 0 only, result broadcast: keeps the warp converged before the
// .sync.aligned TMEM loads.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int* err) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, err, kStatTimeout) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

template <int NR, bool LSE, int SQM, bool ROWS, class Epi>
__global__ void __launch_bounds__(kTcThreads, 1) tc_sweep_kernel(SweepArgs<float> a, TcArgs ta, Epi epi) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + kOffBar);  // [3] per slice buffer
  uint64_t* mmad = full + 3;                   // [2] per TMEM buffer
  uint64_t* tfree = full + 5;                  // [2] per TMEM buffer
  uint64_t* ownf = full + 7;
  uint32_t* tslot = (uint32_t*)(full + 8);
  constexpr int NA = LSE ? 1 : NR;
  constexpr int NW = LSE ? 1 : NR;
  constexpr int ND = Epi::kDot;
  __shared__ float hsum[kParts - 1][NA][kM], hcmp[kParts - 1][NA][kM], hmax[kParts - 1][kM];
  __shared__ int last_blk;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_own = ROWS ? a.n : a.m, n_oth = ROWS ? a.m : a.n;
  const Side so = ROWS ? ta.X : ta.Y;
  const Side sq = ROWS ? ta.Y : ta.X;
  const int64_t blk = blockIdx.x, sidx = blockIdx.y, S = gridDim.y;
  const int64_t j0 = sidx * a.chunk, j1 = min(n_oth, j0 + a.chunk);
  const int T = (int)((j1 - j0 + kN - 1) / kN);

  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&full[2], 1);
    mbar_init(&mmad[0], 1);
    mbar_init(&mmad[1], 1);
    mbar_init(&tfree[0], kEpiWarps);
    mbar_init(&tfree[1], kEpiWarps);
    mbar_init(ownf, 1);
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(tslot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *(volatile uint32_t*)tslot;
  pdl_wait();
  if (a.active && *a.active == 0.0) {  // CG stopped: nothing to do (uniform over the grid)
    __syncthreads();
    if (warp == 1) tmem_free(tbase, kTmemCols);
    return;
  }

  // per-thread results of the epilogue (own point r of this CTA, one column part)
  const int q = warp & 3, part = warp >= 2 ? (warp - 2) >> 2 : 0;
  const int r = 32 * q + lane;
  const int64_t e = blk * kM + r;
  const bool ev = warp >= 2 && e < n_own;
  float Sa[NA], Ca[NA], mx = 0.f;
  bool mx_set = false;
#pragma unroll
  for (int k = 0; k < NA; ++k) {
    Sa[k] = 0.f;
    Ca[k] = 0.f;
  }

  const float* ht = ROWS ? a.Bh : a.Ah;
  const float* const* wt = ROWS ? a.wc : a.wr;
  if (warp == 0) {
    // ---------------- copies and MMAs (one thread) ----------------
    if (lane == 0) {
      const unsigned char* own_src = (const unsigned char*)so.slices + blk * (int64_t)kM * kRowB;
      const unsigned char* oth_src = (const unsigned char*)sq.slices;
      mbar_arrive_expect_tx(ownf, kSlices * kOwnSlice);
      for (int s = 0; s < kSlices; ++s)
        bulk_g2s(sm + s * kOwnSlice, own_src + (int64_t)s * so.npad * kRowB, kOwnSlice, ownf);
      // tile tt: its slices into buffer tt % 2, its per-point data into slot tt % 4
      // (48 floats per array; the arrays hold at least 47 entries past n, and
      // the epilogue masks j >= j1)
      auto issue = [&](int tt) {
        const int sb = tt % kSliceBufs;
        const int64_t jt = j0 + (int64_t)tt * kN;
        mbar_arrive_expect_tx(&full[sb], kSlices * kOthSlice);
        const unsigned char* src = oth_src + jt * kRowB;
        for (int s = 0; s < kSlices; ++s)
          bulk_g2s(sm + kOffOth + (sb * kSlices + s) * kOthSlice, src + (int64_t)s * sq.npad * kRowB, kOthSlice,
                   &full[sb]);
      };
      // Schedule: tiles 0 and 1 are prefetched; after committing tile tt the
      // copies of tile tt + 2 go into the slice buffer of tile tt - 1 once its
      // MMAs are done (queued before tile tt's, so the tensor pipe stays busy)
      // and into the column slot of tile tt - 2, whose epilogue finished before
      // the MMAs of tile tt were issued.
      int issued = 0, landed = 0, committed = 0, retired = 0;
      for (; issued < 2 && issued < T; ++issued) issue(issued);
      const bool own_ok = mbar_wait(ownf, 0, ta.err, kStatTimeout);
      const uint32_t own_s = smem_u32(sm);
      for (int tt = 0; own_ok && tt < T; ++tt) {
        const int b = tt & 1, sb = tt % kSliceBufs;
        if (!mbar_wait(&full[sb], (tt / kSliceBufs) & 1, ta.err, kStatTimeout)) break;
        landed = tt + 1;
        if (tt >= 2 && !mbar_wait(&tfree[b], ((tt - 2) >> 1) & 1, ta.err, kStatTimeout)) break;
        tc_fence_after();
        const uint32_t oth_s = smem_u32(sm + kOffOth + sb * kSlices * kOthSlice);
#pragma unroll 1
        for (int L = 0; L < kLevels; ++L) {
          const uint32_t d_tmem = tbase + (uint32_t)(b * kBufCols + L * kN);
          uint32_t acc = 0;
          for (int s = (L > kSlices - 1 ? L - (kSlices - 1) : 0); s <= L && s < kSlices; ++s) {
            const int t = L - s;
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
              mma_bf16(d_tmem, desc_sw128(own_s + s * kOwnSlice + k4 * 32),
                       desc_sw128(oth_s + t * kOthSlice + k4 * 32), kIdesc, acc);
              acc = 1;
            }
          }
        }
        mma_commit(&mmad[b]);
        committed = tt + 1;
        if (tt + 2 < T) {
          if (tt >= 1) {
            if (!mbar_wait(&mmad[(tt - 1) & 1], ((tt - 1) >> 1) & 1, ta.err, kStatTimeout)) break;
            retired = tt;
          }
          issue(tt + 2);
          ++issued;
        }
      }
      // leave nothing in flight (bounded waits that ignore the error flag):
      // copies issued but not seen landed, and the MMAs not seen retired
      if (!own_ok) mbar_wait(ownf, 0, ta.err, 0, kTcDrainNs);
      for (int tt = landed; tt < issued; ++tt)
        mbar_wait(&full[tt % kSliceBufs], (tt / kSliceBufs) & 1, ta.err, 0, kTcDrainNs);
      for (int tt = (retired > committed - 2 ? retired : committed - 2); tt < committed; ++tt)
        if (tt >= 0) mbar_wait(&mmad[tt & 1], (tt >> 1) & 1, ta.err, 0, kTcDrainNs);
    }
    __syncwarp();
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const float* ho = ROWS ? a.Ah : a.Bh;
    const float h = ev ? ho[e] : 0.f;
    float hm = h;
    const float sc_own = so.sc[e], nxh = so.nxh[e], nxl = so.nxl[e];  // e < npad
    const float g = a.gamma_dev ? (float)*a.gamma_dev : a.gamma;
    float Kh, Kl;
    split_k<float>((double)g * a.sC, Kh, Kl);
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    for (int tt = 0; tt < T; ++tt) {
      const int b = tt & 1;
      if (!warp_wait(&mmad[b], (tt >> 1) & 1, ta.err)) break;  // also covers the tile's copies
      tc_fence_after();
      const int64_t jt = j0 + (int64_t)tt * kN;
#pragma unroll 1
      for (int c = 0; c < kPartCols / 8; ++c) {
        const int col0 = part * kPartCols + c * 8;
        uint32_t lv[kLevels][8];
#pragma unroll
        for (int L = 0; L < kLevels; ++L)
          tmem_ld8(tbase + lane_base + (uint32_t)(b * kBufCols + L * kN + col0), lv[L]);
        tmem_ld_wait();
        float acc[NA];
#pragma unroll
        for (int k = 0; k < NA; ++k) acc[k] = 0.f;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int cj = col0 + jj;
          if (j0 + (int64_t)tt * kN + cj >= j1) break;  // uniform across the warp
          const int64_t j = jt + cj;
          const float hb = ht[j];
          const float f = sc_own * sq.sc[j] * 0x1p-16f;  // powers of two: exact
          float gh, gl;
          two_sum(__uint_as_float(lv[0][jj]), __uint_as_float(lv[1][jj]) * 0x1p-8f, gh, gl);
          gl += __uint_as_float(lv[2][jj]) * 0x1p-16f +
                (__uint_as_float(lv[3][jj]) * 0x1p-24f + __uint_as_float(lv[4][jj]) * 0x1p-32f);
          gh *= f;
          gl *= f;
          float s1, e1, Dh, e2;
          two_sum(nxh, sq.nxh[j], s1, e1);
          two_sum(s1, -2.f * gh, Dh, e2);
          const float Dl = e2 + ((e1 + (nxl + sq.nxl[j])) - 2.f * gl);
          if constexpr (!LSE) {
            const float ex = expT(expo<true>(h + hb, Kh, Kl, Dh, Dl));
#pragma unroll
            for (int k = 0; k < NR; ++k) {
              const float w = wt[k][j];
              if ((SQM >> k) & 1) acc[k] = fmaf(ex * ex, w, acc[k]);
              else acc[k] = fmaf(ex, w, acc[k]);
            }
          } else {
            if (!mx_set) {  // the running max starts at the first element
              mx = ceil_grid(expo<true>(h + hb, Kh, Kl, Dh, Dl));
              hm = h - mx;
              mx_set = true;
            }
            float tv = expo<true>(hm + hb, Kh, Kl, Dh, Dl);
            for (int k = 0; k < 4 && tv > kTheta; ++k) {
              const float dlt = ceil_grid(tv);
              mx += dlt;
              hm = h - mx;
              const float fsc = expT(-dlt);
              acc[0] *= fsc;
              Sa[0] *= fsc;
              Ca[0] *= fsc;
              tv = expo<true>(hm + hb, Kh, Kl, Dh, Dl);
            }
            acc[0] = fmaf(expT(tv), wt[0][j], acc[0]);
          }
        }
#pragma unroll
        for (int k = 0; k < NA; ++k) kadd(Sa[k], Ca[k], acc[k]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tfree[b]);
    }
    if (part > 0) {  // parts 1-3 hand their sums to part 0
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        hsum[part - 1][k][r] = Sa[k];
        hcmp[part - 1][k][r] = Ca[k];
      }
      hmax[part - 1][r] = mx_set ? mx : 0.f;
    }
  }
  pdl_trigger();
  tc_fence_before();
  __syncthreads();  // every TMEM read and MMA is done; the halves are in shared memory
  if (warp == 1) {
    tc_fence_after();
    tmem_free(tbase, kTmemCols);
  }
  if (warp >= 2 && part == 0 && ev) {
    if constexpr (!LSE) {
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        double v = (double)Sa[k] + (double)Ca[k];
#pragma unroll
        for (int pp = 0; pp < kParts - 1; ++pp) v += (double)hsum[pp][k][r] + (double)hcmp[pp][k][r];
        a.rowpart[((int64_t)k * S + sidx) * n_own + e] = v;
      }
    } else {
      LsePair p{0.0, 0.0};
      const double s0 = (double)Sa[0] + (double)Ca[0];
      if (s0 > 0.0) p = lse_combine<float>(p, LsePair{(double)mx, s0});
#pragma unroll
      for (int pp = 0; pp < kParts - 1; ++pp) {
        const double sp = (double)hsum[pp][0][r] + (double)hcmp[pp][0][r];
        if (sp > 0.0) p = lse_combine<float>(p, LsePair{(double)hmax[pp][r], sp});
      }
      a.rowpart[((int64_t)0 * S + sidx) * n_own + e] = p.m;
      a.rowpart[((int64_t)1 * S + sidx) * n_own + e] = p.s;
    }
  }
  __syncthreads();

  // ---- the last CTA of this own block adds the S partials in fixed order ----
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
  if (threadIdx.x < kM) {
    const int64_t ee = blk * kM + threadIdx.x;
    if (ee < n_own) {
      DotArr<ND> dd;
      if constexpr (!LSE) {
        double tot[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          double v = 0.0;
          ordered_loads(a.rowpart + (int64_t)k * S * n_own + ee, n_own, S, [&](double q) { v += q; });
          tot[k] = v;
        }
        if constexpr (ROWS) epi.row(ee, tot, dd.v);
        else epi.col(ee, tot, dd.v);
      } else {
        LsePair p{0.0, 0.0};
        ordered_loads2(a.rowpart + ee, a.rowpart + S * n_own + ee, n_own, S,
                       [&](double qm, double qs) { p = lse_combine<float>(p, LsePair{qm, qs}); });
        if constexpr (ROWS) epi.row_lse(ee, p.m, p.s, dd.v);
        else epi.col_lse(ee, p.m, p.s, dd.v);
      }
#pragma unroll
      for (int k = 0; k < ND; ++k) wd[k] = dd.v[k];
    }
  }
  if (threadIdx.x == 0) a.cnt_rowblk[blk] = 0;
  if constexpr (ND > 0) {
#pragma unroll
    for (int k = 0; k < ND; ++k) wd[k] = warp_sum(wd[k]);
    cta_dot_finish<ND, Epi, kTcWarps>(wd, blk, gridDim.x, a.dotpart, a.cnt_dot, epi);
  }
}

}  // namespace tc
}  // namespace eot
