// eot_marginals_noalloc: the marginals r(P), c(P) without a handle and without
// any device allocation, for callers that cannot allocate GPU memory (a host
// thread that must not call cudaMalloc while another component owns the
// allocator or a fixed memory budget, or code running where an allocation would
// synchronise the device). Its scratch space is one file-scope __device__ array
// of fixed size, loaded with the library and held by every GPU that loads it
// until the process exits.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress and caches it; make that first
// call before any stream capture. Every call on a device shares the array, so
// calls that overlap on the GPU (different streams, or concurrent host threads)
// race and must be ordered by the caller.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "handle.cuh"

namespace {

using namespace eot;

constexpr int64_t kNoAllocMax = 16384;  // largest n and m accepted
constexpr int kNoAllocRowBlocks = 8;     // row blocks of the column sweep
constexpr int kMaxDevices = 64;

// byte offsets of the regions inside the scratch array (all 256-byte aligned)
constexpr size_t kVec = kNoAllocMax * 8;                               // one vector, 8 B per entry
constexpr size_t kOffAh = 0, kOffBh = kVec, kOffAl = 2 * kVec, kOffBl = 3 * kVec;
constexpr size_t kOffEwr = 4 * kVec, kOffEwc = 5 * kVec;
constexpr size_t kOffColpart = 6 * kVec;
constexpr size_t kColpartBytes = 2 * kNoAllocRowBlocks * kNoAllocMax * 8;
constexpr size_t kOffCnt = kOffColpart + kColpartBytes;               // strip tickets, dot ticket
constexpr size_t kCntInts = kNoAllocMax / 32 + 2 + 64;
constexpr size_t kOffDot = kOffCnt + ((kCntInts * 4 + 255) / 256) * 256;
constexpr size_t kDotSlots = kNoAllocMax / kWarps + 1;
constexpr size_t kOffSc = kOffDot + ((kDotSlots * 2 * 8 + 255) / 256) * 256;
constexpr size_t kScratchBytes = kOffSc + 512;  // SC_COUNT doubles, then the status word

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceScratch {
  unsigned char* base = nullptr;
  int sms = 0;
};
std::mutex g_mu;
DeviceScratch g_dev[kMaxDevices];

// Device address of the scratch array for the current device (set-up on first use).
DeviceScratch scratch_for_current_device() {
  int dev = 0;
  EOT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw EotError{EOT_ERR_INVALID_ARG, "device index out of range"};
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev[dev].base) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      throw EotError{EOT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)};
    int sms = 0;
    EOT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    g_dev[dev].base = (unsigned char*)p;
    g_dev[dev].sms = sms;
  }
  return g_dev[dev];
}

__global__ void copy_status_kernel(const int* src, int* dst) {
  pdl_wait();
  *dst = *src;
}

template <class T>
void marginals_noalloc(const eot_problem* P, const double* u, const double* v, double gamma,
                       double* r_out, double* c_out, int* status_out, cudaStream_t st) {
  constexpr int VEC = 16 / (int)sizeof(T);
  const DeviceScratch ds = scratch_for_current_device();
  unsigned char* b = ds.base;
  const int64_t n = P->n, m = P->m, ldc = P->ldc;
  const T* C = (const T*)P->C;
  T* Ah = (T*)(b + kOffAh);
  T* Bh = (T*)(b + kOffBh);
  double* Al = (double*)(b + kOffAl);
  double* Bl = (double*)(b + kOffBl);
  T* ewr = (T*)(b + kOffEwr);
  T* ewc = (T*)(b + kOffEwc);
  double* colpart = (double*)(b + kOffColpart);
  int* cnt = (int*)(b + kOffCnt);
  double* dotpart = (double*)(b + kOffDot);
  double* sc = (double*)(b + kOffSc);
  int* status = (int*)(sc + SC_COUNT);
  const bool plain = P->precision == EOT_PREC_PLAIN_FP32;

  // the array keeps the last call's contents: clear the tickets and the status
  EOT_CUDA(cudaMemsetAsync(cnt, 0, kCntInts * sizeof(int), st));
  EOT_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));

  const bool aligned = ((uintptr_t)C % 16) == 0;
  const int V = (aligned && (m % VEC) == 0 && (ldc % VEC) == 0) ? VEC : 1;
  const int vg_n = vec_grid(n), vg_m = vec_grid(m);
  // column-sweep geometry: S strips of 32 V columns, R <= 8 row blocks, one wave
  const int64_t S = (m + 32 * V - 1) / (32 * V);
  int64_t R = ((int64_t)kColCtasPerSm * ds.sms) / S;
  R = std::max<int64_t>(1, std::min<int64_t>({R, kNoAllocRowBlocks, (n + 31) / 32}));
  int64_t BR = ((n + R - 1) / R + 31) / 32 * 32;
  R = (n + BR - 1) / BR;

  SweepArgs<T> a{};
  a.C = C;
  a.n = n;
  a.m = m;
  a.ldc = ldc;
  a.Ah = Ah;
  a.Bh = Bh;
  a.gamma = (T)gamma;
  a.colpart = colpart;
  a.rowpart = nullptr;
  a.cnt_strip = cnt;
  a.cnt_rowblk = cnt + (kNoAllocMax / 32 + 2);
  a.cnt_dot = cnt + (kNoAllocMax / 32 + 1);
  a.dotpart = dotpart;
  a.rows_per_block = (int)BR;
  a.nrowblk = (int)R;
  a.gamma_dev = nullptr;
  a.active = nullptr;
  a.keep_l2 = 0;

  // log r(P) = LSE_j(u_i + v_j - gamma C_ij): rows split, columns split with weights exp(Bl)
  launch_k(split_kernel<T>, dim3(vg_n), dim3(kThreads), st, n, u, (const double*)nullptr, 0.0,
           (const double*)nullptr, plain ? 1 : 0, Ah, Al, (T*)nullptr, (double*)nullptr,
           (const double*)nullptr, status);
  launch_k(split_kernel<T>, dim3(vg_m), dim3(kThreads), st, m, v, (const double*)nullptr, 0.0,
           (const double*)nullptr, plain ? 1 : 0, Bh, Bl, ewc, (double*)nullptr,
           (const double*)nullptr, status);
  {
    SweepArgs<T> ar = a;
    ar.wc[0] = ewc;
    RowLseEpi e{nullptr, Al, r_out, nullptr, nullptr, sc, SC_MASS, SC_AUX1};
    const dim3 grid((unsigned)((n + kWarps - 1) / kWarps));
    if (V == VEC) launch_k(row_sweep_kernel<T, VEC, 1, true, 0, RowLseEpi>, grid, dim3(kThreads), st, ar, e);
    else launch_k(row_sweep_kernel<T, 1, 1, true, 0, RowLseEpi>, grid, dim3(kThreads), st, ar, e);
  }
  // log c(P) = LSE_i(u_i + v_j - gamma C_ij): rows split with weights exp(Al)
  launch_k(split_kernel<T>, dim3(vg_n), dim3(kThreads), st, n, u, (const double*)nullptr, 0.0,
           (const double*)nullptr, plain ? 1 : 0, Ah, Al, ewr, (double*)nullptr,
           (const double*)nullptr, status);
  {
    SweepArgs<T> ac = a;
    ac.wr[0] = ewr;
    ColLseEpi e{Bl, nullptr, c_out, 0, sc, SC_AUX0, 0.0};
    const dim3 grid((unsigned)S, (unsigned)R);
    if (V == VEC) launch_k(col_sweep_kernel<T, VEC, 1, true, 0, ColLseEpi>, grid, dim3(kThreads), st, ac, e);
    else launch_k(col_sweep_kernel<T, 1, 1, true, 0, ColLseEpi>, grid, dim3(kThreads), st, ac, e);
  }
  // the sweeps wrote log r(P), log c(P) into the outputs; exponentiate in place
  launch_k(exp_kernel, dim3(vg_n), dim3(kThreads), st, n, (const double*)r_out, r_out);
  launch_k(exp_kernel, dim3(vg_m), dim3(kThreads), st, m, (const double*)c_out, c_out);
  if (status_out) launch_k(copy_status_kernel, dim3(1), dim3(1), st, (const int*)status, status_out);
}

}  // namespace

extern "C" eot_status eot_marginals_noalloc(const eot_problem* prob, const double* u,
                                            const double* v, double gamma, double* r_out,
                                            double* c_out, int32_t* status_out, void* stream) {
  try {
    if (!prob || !u || !v || !r_out || !c_out) return EOT_ERR_INVALID_ARG;
    if (prob->n < 1 || prob->m < 1 || prob->n > kNoAllocMax || prob->m > kNoAllocMax)
      return EOT_ERR_INVALID_ARG;  // sizes beyond the fixed scratch are rejected
    if (!prob->C || prob->ldc < prob->m) return EOT_ERR_INVALID_ARG;
    if (!(gamma > 0.0) || !std::isfinite(gamma) || gamma >= kSplitLimit) return EOT_ERR_INVALID_ARG;
    const cudaStream_t st = (cudaStream_t)stream;
    if (prob->kind == EOT_COST_DENSE_F64 && prob->precision == EOT_PREC_FP64) {
      marginals_noalloc<double>(prob, u, v, gamma, r_out, c_out, status_out, st);
    } else if (prob->kind == EOT_COST_DENSE_F32 &&
               (prob->precision == EOT_PREC_MIXED || prob->precision == EOT_PREC_PLAIN_FP32)) {
      marginals_noalloc<float>(prob, u, v, (double)(float)gamma, r_out, c_out, status_out, st);
    } else {
      return EOT_ERR_UNSUPPORTED;
    }
    return EOT_OK;
  } catch (const EotError& e) {
    return e.st;
  } catch (...) {
    return EOT_ERR_CUDA;
  }
}
