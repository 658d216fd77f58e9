// Point-cloud sweeps whose cross term x_i . y_j runs on the tensor cores
// (tcgen05, kind::f16 on BF16, FP32 accumulation in TMEM), for the mixed path at
// larger d (up to 64 coordinates).
//
// Exactness (an exact-slice / Ozaki-style splitting). Both point sets are moved
// by one common centre c (the first point of X; exact in FP64, distances do not
// change). Each cloud gets one exponent E (every centred coordinate |x_k| < 2^E)
// and every coordinate is cut into five signed 8-bit digits
//     x_k = 2^E sum_s d_sk 2^-8(s+1)      (to 2^(E-40)).
// A digit is an integer of magnitude <= 255, exact in BF16; a digit product is an
// integer below 2^16 and a dot product over 64 coordinates stays below 2^22, so
// every MMA of two digit slices is exact in the FP32 accumulator. The 15 slice
// pairs (s, t) with s + t <= 4 are added into five "level" accumulators
// S_L = sum_{s+t=L} D_s D_t^T (levels 0-3 hold at most four pairs, below 2^24,
// and stay exact; level 4 may round by one unit, 2^-32 of a level-0 unit), and
//     x . y = 2^(Ex + Ey - 16) G,   G = S_0 + 2^-8 S_1 + 2^-16 S_2 + 2^-24 S_3 + 2^-32 S_4
// to about 2^-38 of the largest |x||y| (the dropped pairs s + t >= 5 and the
// digit truncation).
//
// Exponent algebra. In base-2 units (t2 = t log2 e) the exponent of the plan is
//     t2_ij = P_i + Q_j + kappa G_ij,   P_i = (A_i - K |x_i|^2) log2 e,
//     Q_j = (B_j - K |y_j|^2) log2 e,   kappa = 2 K 2^(Ex+Ey-16) log2 e,
// with K = gamma s_C and A, B the high parts of the potentials. A small kernel
// before each sweep (tc_sweep_prep_kernel) forms P and Q in FP64 and splits each
// into a high part on the 1/8 grid and a low part below 1/16: the other side's
// low part is folded into its weights (w_j 2^ql_j, one record per point:
// {Qh, w0} in 8 bytes for one weight, {Qh, w0, w1, w2} in 16) and the own side's into one FP64 factor 2^pl_i that
// the finishing CTA applies to the row's total. Per entry the epilogue then
// needs G as an FP32 pair (Fast2Sum of the two top levels plus three FMAs) and
//     t2 = fma(kh, gh, Ph + Qh) + fma(kl, gh, kh gl)
// (Ph + Qh exact on the grid, the big product exact inside the FMA): about a
// dozen FP32 instructions and one MUFU ex2, t2 rounded twice at its own scale.
//
// Tile width. A tcgen05.mma of M = 128, K = 16 costs about 50 cycles whatever
// its N up to ~96 (measured on GB300: 55 cycles at N = 32, 48 and 96; 96 at
// N = 192), so the tile is 96 points wide: the five level accumulators then
// fill 480 of the 512 TMEM columns, one buffer, handed over level by level.
//
// CTA roles (480 threads, one CTA per SM: about 215 KB of shared memory):
//   warp 0, lane 0 and warp 14, lane 0: the 60 MMAs of each tile, level by
//     level (levels 0, 1, 4 and levels 2, 3), with a commit per level group. A
//     tcgen05.mma blocks its thread while the tensor unit's short queue is
//     full, so these threads do nothing else: any other work in them, or a
//     lost issue slot, leaves the tensor unit idle;
//   warp 1: TMEM allocation (512 columns) and release; lane 0 issues the bulk
//     copies (the own 128 points' slices once; the other side's 96-point
//     tiles into two slice buffers and their records into four record slots);
//   warps 2-13: epilogue. Warp w reads TMEM lanes 32 (w mod 4) .. +31 (one own
//     point per thread) and a third (32) of the tile's 96 columns.
// Hand-offs are mbarriers: full[sb] (the slices of buffer sb landed), sfree[sb][i]
// (issuer i's MMAs reading buffer sb are done), rec[s] (records landed), lvl[g] (the
// MMAs of level group g = {0,1}, {2,3}, {4} are done: accumulators readable),
// lfree[0] / lfree[1] (the 12 epilogue warps have loaded levels 0-3 / level 4
// into registers; the next tile's MMAs may overwrite them). Every wait is
// bounded (tc.cuh).
#pragma once
#include <cuda_bf16.h>

#include "sweep_pts.cuh"
#include "tc.cuh"

namespace eot {
namespace tc {

constexpr int kM = 128;     // own points per CTA = TMEM lanes = MMA M
constexpr int kN = 96;      // other-side points per tile = MMA N
constexpr int kSlices = 5;  // 8-bit digits per coordinate
constexpr int kLevels = 5;  // s + t = 0 .. 4
constexpr int kEpiWarps = 12;                  // 3 per TMEM lane quarter
constexpr int kParts = kEpiWarps / 4;          // column parts of a tile
constexpr int kPartCols = kN / kParts;         // 32 columns per epilogue warp and tile
constexpr int kGroups = kPartCols / 8;         // groups of 8 columns in the arithmetic
constexpr int kMmaWarpB = 2 + kEpiWarps;      // the second MMA-issuing warp (after the epilogue warps)
constexpr int kTcThreads = 32 * (3 + kEpiWarps);
constexpr int kTcWarps = kTcThreads / 32;
constexpr uint32_t kRowB = 128;    // bytes per point and slice: 64 BF16 coordinates
constexpr uint32_t kOwnSlice = kM * kRowB;                          // 16 KB
constexpr uint32_t kOthSlice = kN * kRowB;                          // 12 KB
constexpr uint32_t kOffOth = kSlices * kOwnSlice;                   // 80 KB
constexpr int kSliceBufs = 2;                                       // tile tt: slice buffer tt % 2
constexpr int kRecSlots = 4;                                        // tile tt: record slot tt % 4
constexpr uint32_t kRecBytes = kN * 16;                             // 1.5 KB: a slot at the widest record
constexpr uint32_t kOffRec = kOffOth + kSliceBufs * kSlices * kOthSlice;  // + 120 KB
constexpr uint32_t kOffBar = kOffRec + kRecSlots * kRecBytes;            // + 6 KB
constexpr uint32_t kSmemBytes = kOffBar + 256 + 1024;               // barriers, TMEM slot; 1024-byte alignment slack
constexpr uint32_t kTmemCols = 512;                                 // 5 levels x 96 columns used
constexpr int64_t kPadRows = 384;                                   // lcm(kM, kN)
constexpr uint32_t kIdesc = idesc_bf16_f32(kM, kN);
static_assert(kLevels * kN <= (int)kTmemCols, "level accumulators exceed TMEM");
constexpr int kMinD = 17;  // the tensor-core path serves d >= kMinD
constexpr double kLog2eD = 1.4426950408889634;
constexpr double kLn2D = 0.6931471805599453;
constexpr float kTheta2 = 12.0f;       // lazy-rescale threshold of the online max (base 2)
constexpr float kPadQ = -8388608.0f;   // -2^23: Qh of padded points (weights 0), and the LSE max's start
constexpr double kQLimit = 1048576.0;  // |P|, |Q| < 2^20: sums of grid values stay exact in FP32

// Per-sweep data of an own point (written by tc_sweep_prep_kernel).
struct OwnRec {
  float ph;   // high part of P on the 1/8 grid
  float pad;
  double pl;  // P - ph, |pl| <= 1/16
  double f1;  // 2^pl
  double f2;  // 2^(2 pl): sums of squared entries
};

// Per point set: the fixed digit slices and |x - c|^2 (per problem), and the
// per-sweep records of the point set in either role.
struct Side {
  const __nv_bfloat16* slices;  // [kSlices][npad][64], 128-byte swizzle per 8-row atom
  const double* nx;             // [npad] |x - c|^2 (0 for padding)
  float* rec;                   // [npad][rec_floats(NR)] as the other side: {Qh, w0 2^ql[, w1 2^ql, w2 2^ql]}
  OwnRec* own;                  // [npad] as the own side
  int64_t npad;
};
struct TcArgs {
  Side X, Y;
  const unsigned long long* emax;  // [2] bits of the FP64 max |x_k - c_k| of X and of Y
  float* kappa;                    // [2] kappa as an FP32 pair (per sweep)
  int* err;                        // status word: kStatTimeout on a wait that ran out, kStatRange
};

__host__ __device__ inline int64_t pad_rows(int64_t n) { return (n + kPadRows - 1) / kPadRows * kPadRows; }
// Floats per record: sweeps with one weight (the CG halves, the LSE sweeps)
// read 8 bytes per column, so one 16-byte shared load serves two columns.
__host__ __device__ constexpr int rec_floats(int nr) { return nr == 1 ? 2 : 4; }

// E with every centred coordinate |x_k| < 2^E (0 for a cloud of one point).
__device__ __forceinline__ int cloud_exp(unsigned long long bits) {
  const double mx = __longlong_as_double((long long)bits);
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
  return e;
}

// max_{i,k} |x_ik - c_k| of one cloud (FP64, exact differences) into *emax as
// the bits of a non-negative double (ordered like the values). *emax starts at 0.
static __global__ void tc_extent_kernel(const float* X, int64_t n, int d, const float* centre,
                                        unsigned long long* emax) {
  pdl_wait();
  double mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * d;
       i += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, fabs((double)X[i] - (double)centre[i % d]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(emax, (unsigned long long)__double_as_longlong(mx));
}

// One warp per point (rows >= n and coordinates >= d are zero): the five digit
// slices in the swizzled K-major layout and |x - c|^2 in FP64. Centring keeps
// |x|^2, |y|^2 and x.y bounded by the data's extent, so the expansion
// |x|^2 + |y|^2 - 2 x.y keeps its accuracy however far the clouds lie from the
// origin.
static __global__ void tc_prep_kernel(const float* X, int64_t n, int d, int64_t npad, const float* centre,
                                      const unsigned long long* emax, __nv_bfloat16* sl, double* nx) {
  pdl_wait();
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= npad) return;
  double xv[2] = {0.0, 0.0};
  if (row < n) {
    if (lane < d) xv[0] = (double)X[row * d + lane] - (double)centre[lane];
    if (lane + 32 < d) xv[1] = (double)X[row * d + lane + 32] - (double)centre[lane + 32];
  }
  double q = xv[0] * xv[0] + xv[1] * xv[1];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  const int e = cloud_exp(*emax);
  if (lane == 0) nx[row] = q;
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

// Before each sweep: kappa, the other side's records (all npad of them; padded
// points get Qh = -2^23 and weights 0, so no tile needs a mask) and the own
// side's P split. The same gamma as the sweep: (float) of the device value.
template <int NR, int SQM, bool ROWS>
__global__ void tc_sweep_prep_kernel(SweepArgs<float> a, TcArgs ta) {
  pdl_wait();
  if (a.active && *a.active == 0.0) return;
  const Side so = ROWS ? ta.X : ta.Y;
  const Side sq = ROWS ? ta.Y : ta.X;
  const int64_t n_own = ROWS ? a.n : a.m, n_oth = ROWS ? a.m : a.n;
  const float g = a.gamma_dev ? (float)*a.gamma_dev : a.gamma;
  const double K = (double)g * a.sC;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i == 0) {
    const double kap = 2.0 * K * ldexp(1.0, cloud_exp(ta.emax[0]) + cloud_exp(ta.emax[1]) - 16) * kLog2eD;
    const float kh = (float)kap;
    ta.kappa[0] = kh;
    ta.kappa[1] = (float)(kap - (double)kh);
  }
  if (i < sq.npad) {
    constexpr int RW = rec_floats(NR);
    float4 r = make_float4(kPadQ, 0.f, 0.f, 0.f);
    if (i < n_oth) {
      const float* hq = ROWS ? a.Bh : a.Ah;
      const double Q = ((double)hq[i] - K * sq.nx[i]) * kLog2eD;
      if (!(fabs(Q) < kQLimit)) atomicOr(ta.err, kStatRange);
      const double qh = rint(Q * 8.0) * kGrid;
      const double ql = Q - qh;
      const double f1 = exp2(ql);
      const double f2 = SQM ? exp2(2.0 * ql) : 0.0;
      const float* const* wt = ROWS ? a.wc : a.wr;
      r.x = (float)qh;
      r.y = (float)((double)wt[0][i] * ((SQM & 1) ? f2 : f1));
      if constexpr (NR > 1) r.z = (float)((double)wt[1][i] * ((SQM & 2) ? f2 : f1));
      if constexpr (NR > 2) r.w = (float)((double)wt[2][i] * ((SQM & 4) ? f2 : f1));
    }
    if constexpr (RW == 2) reinterpret_cast<float2*>(sq.rec)[i] = make_float2(r.x, r.y);
    else reinterpret_cast<float4*>(sq.rec)[i] = r;
  } else if (i < sq.npad + so.npad) {
    const int64_t e = i - sq.npad;
    OwnRec o{0.f, 0.f, 0.0, 1.0, 1.0};
    if (e < n_own) {
      const float* ho = ROWS ? a.Ah : a.Bh;
      const double P = ((double)ho[e] - K * so.nx[e]) * kLog2eD;
      if (!(fabs(P) < kQLimit)) atomicOr(ta.err, kStatRange);
      const double ph = rint(P * 8.0) * kGrid;
      o.ph = (float)ph;
      o.pl = P - ph;
      o.f1 = exp2(o.pl);
      o.f2 = SQM ? exp2(2.0 * o.pl) : 1.0;
    }
    so.own[e] = o;
  }
}

// t2 = hq + kappa G with hq = Ph + Qh (or Ph - max + Qh), exact on the grid.
__device__ __forceinline__ float entry_t2(float hq, float gh, float gl, float kh, float kl) {
  const float b = fmaf(kh, gh, hq);
  const float c = fmaf(kl, gh, __fmul_rn(kh, gl));
  return __fadd_rn(b, c);
}

// Base-2 log-sum-exp pairs (m on the 1/8 grid, s >= 0; s == 0: empty). The
// exponent difference is exact, so the FP32 ex2 rounds once.
__device__ __forceinline__ void lse2_add(double& M, double& s, double qm, double qs) {
  if (!(qs > 0.0)) return;
  if (!(s > 0.0)) {
    M = qm;
    s = qs;
    return;
  }
  const double Mn = fmax(M, qm);
  s = s * (double)ex2_approx((float)(M - Mn)) + qs * (double)ex2_approx((float)(qm - Mn));
  M = Mn;
}

// Waits by lane 0 only, result broadcast: keeps the warp converged before the
// .sync.aligned TMEM loads.
// Each poll may sleep up to kEpiSleepNs, so that waiting epilogue warps leave
// the issue slots of their SM sub-partition to the MMA-issuing thread.
constexpr uint32_t kEpiSleepNs = 200;
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, int* err) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, err, kStatTimeout, kTcWaitNs, kEpiSleepNs) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

template <int NR, bool LSE, int SQM, bool ROWS, class Epi>
__global__ void __launch_bounds__(kTcThreads, 1) tc_sweep_kernel(SweepArgs<float> a, TcArgs ta, Epi epi) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(sm + kOffBar);  // [2] the five slices of the slice buffer landed
  uint64_t* sfree = full + 2;                  // [2][2] per issuer: its MMAs reading the slice buffer done
  uint64_t* lvl = full + 6;                    // [3] MMAs of levels {0,1}, {2,3}, {4} done
  uint64_t* lfree = full + 9;                  // [2] levels 0-3, level 4 loaded by all epilogue warps
  uint64_t* recf = full + 11;                  // [4] records of the slot landed
  uint64_t* ownf = full + 15;
  uint32_t* tslot = (uint32_t*)(full + 16);
  constexpr int NA = LSE ? 1 : NR;
  constexpr int ND = Epi::kDot;
  constexpr int RW = rec_floats(NR);
  constexpr uint32_t kTileRec = kN * RW * 4;  // record bytes of a tile
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
    for (int k = 0; k < kSliceBufs; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&sfree[2 * k], 1);
      mbar_init(&sfree[2 * k + 1], 1);
    }
    for (int g = 0; g < 3; ++g) mbar_init(&lvl[g], 1);
    for (int g = 0; g < 2; ++g) mbar_init(&lfree[g], kEpiWarps);
    for (int k = 0; k < kRecSlots; ++k) mbar_init(&recf[k], 1);
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
  const bool epi_warp = warp >= 2 && warp < 2 + kEpiWarps;
  const int q = warp & 3, part = epi_warp ? (warp - 2) >> 2 : 0;
  const int r = 32 * q + lane;
  const int64_t e = blk * kM + r;
  const bool ev = epi_warp && e < n_own;
  float Sa[NA], Ca[NA], mx = kPadQ;
#pragma unroll
  for (int k = 0; k < NA; ++k) {
    Sa[k] = 0.f;
    Ca[k] = 0.f;
  }

  if (warp == 1) {
    // ---------------- bulk copies (one thread) ----------------
    // The own 128 points' slices once; tile tt's five slices into buffer tt % 2
    // and its records into slot tt % 4. Tiles 0 and 1 go at once; tile tt >= 2 once the MMAs of tile
    // tt - 2 are done (sfree), by when the epilogue had loaded tile tt - 3 and
    // so finished tile tt - 4, the previous user of the record slot.
    if (lane == 0) {
      const unsigned char* own_src = (const unsigned char*)so.slices + blk * (int64_t)kM * kRowB;
      const unsigned char* oth_src = (const unsigned char*)sq.slices;
      mbar_arrive_expect_tx(ownf, kSlices * kOwnSlice);
      for (int s = 0; s < kSlices; ++s)
        bulk_g2s(sm + s * kOwnSlice, own_src + (int64_t)s * so.npad * kRowB, kOwnSlice, ownf);
      int issued = 0;
      for (int tt = 0; tt < T; ++tt) {
        const int sb = tt % kSliceBufs, rs = tt % kRecSlots;
        const uint32_t opar = (uint32_t)((tt - kSliceBufs) / kSliceBufs) & 1u;  // tile tt - 2's phase
        if (tt >= kSliceBufs &&
            (!mbar_wait(&sfree[2 * sb], opar, ta.err, kStatTimeout, kTcWaitNs, kEpiSleepNs) ||
             !mbar_wait(&sfree[2 * sb + 1], opar, ta.err, kStatTimeout, kTcWaitNs, kEpiSleepNs)))
          break;
        const int64_t jt = j0 + (int64_t)tt * kN;
        const unsigned char* src = oth_src + jt * kRowB;
        mbar_arrive_expect_tx(&full[sb], kSlices * kOthSlice);
        for (int s = 0; s < kSlices; ++s)
          bulk_g2s(sm + kOffOth + (sb * kSlices + s) * kOthSlice, src + (int64_t)s * sq.npad * kRowB, kOthSlice,
                   &full[sb]);
        mbar_arrive_expect_tx(&recf[rs], kTileRec);
        bulk_g2s(sm + kOffRec + rs * kRecBytes, sq.rec + jt * RW, kTileRec, &recf[rs]);
        issued = tt + 1;
      }
      // leave no copy in flight (bounded waits that ignore the error flag): the
      // own slices, the slices of the last two tiles issued (a buffer was
      // reused only after the MMAs had read its previous tile) and the records
      // of the last four
      mbar_wait(ownf, 0, ta.err, 0, kTcDrainNs);
      for (int tt = (issued > kSliceBufs ? issued - kSliceBufs : 0); tt < issued; ++tt)
        mbar_wait(&full[tt % kSliceBufs], (tt / kSliceBufs) & 1, ta.err, 0, kTcDrainNs);
      for (int tt = (issued > kRecSlots ? issued - kRecSlots : 0); tt < issued; ++tt)
        mbar_wait(&recf[tt % kRecSlots], (tt / kRecSlots) & 1, ta.err, 0, kTcDrainNs);
    }
    __syncwarp();
  } else if (warp == 0 || warp == kMmaWarpB) {
    // ---------------- MMAs (two threads) ----------------
    // Issuer A (warp 0) owns levels 0, 1 and 4, issuer B (the last warp)
    // levels 2 and 3: each level's accumulation chain stays in one thread, and
    // with the issuers on two SM sub-partitions the tensor unit's short queue
    // stays fed while the epilogue warps compete for issue slots (one issuer
    // loses ~25 % of the MMA rate to them). Per tile each waits for the slices
    // and for the epilogue to have loaded levels 0-3 of the previous tile; A
    // commits levels {0,1}, waits for level 4 of the previous tile to be loaded,
    // and commits level 4; B commits levels {2,3}; each commits its use of the
    // slice buffer (sfree[buffer][issuer]).
    if (lane == 0) {
      const int who = warp == 0 ? 0 : 1;
      const bool own_ok = mbar_wait(ownf, 0, ta.err, kStatTimeout);
      // descriptors of the first own slice and of the first other-side slice;
      // every MMA adds a compile-time offset (all unrolled)
      const uint64_t adesc0 = desc_sw128(smem_u32(sm));
      const uint64_t bdesc0 = desc_sw128(smem_u32(sm + kOffOth));
      auto level = [&](uint64_t bdesc, int L) {
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4)
#pragma unroll
          for (int s = 0; s < kSlices; ++s) {
            const int t = L - s;
            if (t < 0 || t >= kSlices) continue;
            mma_bf16(tbase + (uint32_t)(L * kN), adesc0 + (uint64_t)((s * kOwnSlice + k4 * 32) >> 4),
                     bdesc + (uint64_t)((t * kOthSlice + k4 * 32) >> 4), kIdesc,
                     (k4 == 0 && s == (L > kSlices - 1 ? L - (kSlices - 1) : 0)) ? 0u : 1u);
          }
      };
      int committed = 0;
      bool ok = own_ok;
      for (int tt = 0; ok && tt < T; ++tt) {
        const int sb = tt % kSliceBufs;
        const uint32_t fpar = (uint32_t)(tt / kSliceBufs) & 1u;
        const uint32_t ppar = (uint32_t)(tt - 1) & 1u;
        const uint64_t bdesc = bdesc0 + (uint64_t)((sb * kSlices * kOthSlice) >> 4);
        if (!mbar_wait(&full[sb], fpar, ta.err, kStatTimeout) ||
            (tt >= 1 && !mbar_wait(&lfree[0], ppar, ta.err, kStatTimeout))) {
          ok = false;
        } else if (who == 0) {
          tc_fence_after();
          level(bdesc, 0);
          level(bdesc, 1);
          mma_commit(&lvl[0]);
          if (tt >= 1 && !mbar_wait(&lfree[1], ppar, ta.err, kStatTimeout)) {
            ok = false;
          } else {
            tc_fence_after();
            level(bdesc, 4);
            mma_commit(&lvl[2]);
          }
        } else {
          tc_fence_after();
          level(bdesc, 2);
          level(bdesc, 3);
          mma_commit(&lvl[1]);
        }
        uint64_t* sf = &sfree[2 * sb + who];
        mma_commit(sf);  // also after a partly issued tile: its MMAs end before the CTA does
        if (ok) {
          committed = tt + 1;
        } else {  // that commit covers every MMA this thread issued: wait for it alone
          mbar_wait(sf, fpar, ta.err, 0, kTcDrainNs);
          committed = 0;
        }
      }
      // this issuer's MMAs of the last two committed tiles (earlier ones were
      // seen done by the copy thread before it reused their buffer)
      for (int tt = (committed > kSliceBufs ? committed - kSliceBufs : 0); tt < committed; ++tt)
        mbar_wait(&sfree[2 * (tt % kSliceBufs) + who], (tt / kSliceBufs) & 1, ta.err, 0, kTcDrainNs);
    }
    __syncwarp();
  } else if (epi_warp) {
    // ---------------- epilogue ----------------
    const float ph = so.own[e].ph;  // e < npad: padded rows have records
    const float kh = ta.kappa[0], kl = ta.kappa[1];
    // LSE: hm = ph - mx. The max starts at -2^23, far below every entry, so the
    // first group of columns raises it to its own maximum (the one inexact step,
    // it only chooses the shift); from then on ph and mx are on the grid and
    // hm is exact.
    float hm = LSE ? ph - mx : ph;
    const uint32_t tcol = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(part * kPartCols);
    const float* recs = (const float*)(sm + kOffRec);
    for (int tt = 0; tt < T; ++tt) {
      const uint32_t par = (uint32_t)tt & 1u;
      // G as an FP32 pair per column, folded level by level; each level goes
      // back to the MMAs of the next tile as soon as it is in registers
      uint32_t gh[kPartCols], gl[kPartCols], u[kPartCols];
      if (!warp_wait(&lvl[0], par, ta.err)) break;  // levels 0 and 1
      tc_fence_after();
      tmem_ld32(tcol, gh);
      tmem_ld32(tcol + (uint32_t)kN, gl);
      tmem_ld_wait();
      // G = S_0 + 2^-8 S_1 + ... as an FP32 pair (gh, gl). S_0 is an integer
      // below 2^22 and 2^-8 S_1 a multiple of 2^-8 below 2^15: where
      // |S_0| >= |2^-8 S_1| Fast2Sum is exact, and otherwise the sum lies below
      // 2^16 on the 2^-8 grid and is exact already (z = 2^-8 S_1, error 0).
#pragma unroll
      for (int c = 0; c < kPartCols; ++c) {
        const float s0 = __uint_as_float(gh[c]), s1 = __uint_as_float(gl[c]);
        const float h = fmaf(s1, 0x1p-8f, s0);
        const float z = __fsub_rn(h, s0);
        gh[c] = __float_as_uint(h);
        gl[c] = __float_as_uint(fmaf(s1, 0x1p-8f, -z));
      }
      if (!warp_wait(&lvl[1], par, ta.err)) break;  // levels 2 and 3
      tc_fence_after();
      bool ok = true;
#pragma unroll
      for (int L = 2; L < kLevels; ++L) {
        if (L == 4) {
          if (!warp_wait(&lvl[2], par, ta.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        tmem_ld32(tcol + (uint32_t)(L * kN), u);
        tmem_ld_wait();
        if (L >= 3) {  // levels 0-3, then level 4, go back to the MMAs
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&lfree[L - 3]);
        }
        const float sc = L == 2 ? 0x1p-16f : (L == 3 ? 0x1p-24f : 0x1p-32f);
#pragma unroll
        for (int c = 0; c < kPartCols; ++c)
          gl[c] = __float_as_uint(fmaf(__uint_as_float(u[c]), sc, __uint_as_float(gl[c])));
      }
      if (!ok) break;
      const int rs = tt % kRecSlots;
      if (!warp_wait(&recf[rs], (uint32_t)(tt / kRecSlots) & 1u, ta.err)) break;
      const float* rt = recs + rs * (kRecBytes / 4) + part * kPartCols * RW;
#pragma unroll
      for (int c = 0; c < kGroups; ++c) {
        float acc[NA];
#pragma unroll
        for (int k = 0; k < NA; ++k) acc[k] = 0.f;
        // the group's records: Qh and the weights of its 8 columns
        float qh[8], w[NR][8];
        if constexpr (RW == 2) {
#pragma unroll
          for (int jj = 0; jj < 8; jj += 2) {
            const float4 R = *reinterpret_cast<const float4*>(rt + (c * 8 + jj) * 2);
            qh[jj] = R.x;
            w[0][jj] = R.y;
            qh[jj + 1] = R.z;
            w[0][jj + 1] = R.w;
          }
        } else {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const float4 R = *reinterpret_cast<const float4*>(rt + (c * 8 + jj) * 4);
            qh[jj] = R.x;
            const float ws[3] = {R.y, R.z, R.w};
#pragma unroll
            for (int k = 0; k < NR; ++k) w[k][jj] = ws[k];
          }
        }
        if constexpr (!LSE) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const float ex = ex2_approx(entry_t2(__fadd_rn(hm, qh[jj]), __uint_as_float(gh[c * 8 + jj]),
                                                 __uint_as_float(gl[c * 8 + jj]), kh, kl));
#pragma unroll
            for (int k = 0; k < NR; ++k) acc[k] = fmaf(((SQM >> k) & 1) ? ex * ex : ex, w[k][jj], acc[k]);
          }
        } else {
          float t[8];
          float tmax = -3.0e38f;
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            t[jj] = entry_t2(__fadd_rn(hm, qh[jj]), __uint_as_float(gh[c * 8 + jj]),
                             __uint_as_float(gl[c * 8 + jj]), kh, kl);
            tmax = fmaxf(tmax, t[jj]);
          }
          for (int k = 0; k < 4 && tmax > kTheta2; ++k) {  // raise the max (rare after the first group)
            const float dlt = ceil_grid(tmax);
            mx += dlt;
            hm = ph - mx;
            const float f = ex2_approx(-dlt);
            Sa[0] *= f;
            Ca[0] *= f;
            tmax = -3.0e38f;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              t[jj] = entry_t2(__fadd_rn(hm, qh[jj]), __uint_as_float(gh[c * 8 + jj]),
                               __uint_as_float(gl[c * 8 + jj]), kh, kl);
              tmax = fmaxf(tmax, t[jj]);
            }
          }
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) acc[0] = fmaf(ex2_approx(t[jj]), w[0][jj], acc[0]);
        }
#pragma unroll
        for (int k = 0; k < NA; ++k) kadd(Sa[k], Ca[k], acc[k]);
      }
    }
    if (part > 0) {  // parts 1 and 2 hand their sums to part 0
#pragma unroll
      for (int k = 0; k < NA; ++k) {
        hsum[part - 1][k][r] = Sa[k];
        hcmp[part - 1][k][r] = Ca[k];
      }
      hmax[part - 1][r] = mx;
    }
  }
  pdl_trigger();
  tc_fence_before();
  __syncthreads();  // every TMEM read and MMA is done; the parts are in shared memory
  if (warp == 1) {
    tc_fence_after();
    tmem_free(tbase, kTmemCols);
  }
  if (epi_warp && part == 0 && ev) {
    if constexpr (!LSE) {
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        double v = (double)Sa[k] + (double)Ca[k];
#pragma unroll
        for (int pp = 0; pp < kParts - 1; ++pp) v += (double)hsum[pp][k][r] + (double)hcmp[pp][k][r];
        a.rowpart[((int64_t)k * S + sidx) * n_own + e] = v;
      }
    } else {
      double M = 0.0, s = 0.0;
      lse2_add(M, s, (double)mx, (double)Sa[0] + (double)Ca[0]);
#pragma unroll
      for (int pp = 0; pp < kParts - 1; ++pp)
        lse2_add(M, s, (double)hmax[pp][r], (double)hsum[pp][0][r] + (double)hcmp[pp][0][r]);
      a.rowpart[((int64_t)0 * S + sidx) * n_own + e] = M;
      a.rowpart[((int64_t)1 * S + sidx) * n_own + e] = s;
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
      const OwnRec o = so.own[ee];
      DotArr<ND> dd;
      if constexpr (!LSE) {
        double tot[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          double v = 0.0;
          ordered_loads(a.rowpart + (int64_t)k * S * n_own + ee, n_own, S, [&](double qv) { v += qv; });
          tot[k] = v * (((SQM >> k) & 1) ? o.f2 : o.f1);
        }
        if constexpr (ROWS) epi.row(ee, tot, dd.v);
        else epi.col(ee, tot, dd.v);
      } else {
        double M = 0.0, s = 0.0;
        ordered_loads2(a.rowpart + ee, a.rowpart + S * n_own + ee, n_own, S,
                       [&](double qm, double qs) { lse2_add(M, s, qm, qs); });
        const double m_nat = s > 0.0 ? (M + o.pl) * kLn2D : 0.0;
        if constexpr (ROWS) epi.row_lse(ee, m_nat, s, dd.v);
        else epi.col_lse(ee, m_nat, s, dd.v);
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
