// Handle and workspace of the C ABI (include/eot.h). The handle owns every
// scratch buffer of the sweeps and of the solver; caller buffers are never kept.
#pragma once
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <utility>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/eot.h"
#include "kernels.cuh"

struct EotError {
  eot_status st;
  std::string msg;
};

#define EOT_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      throw EotError{EOT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define EOT_LAUNCH_CHECK()                                                               \
  do {                                                                                   \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess)                                                               \
      throw EotError{EOT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)}; \
  } while (0)

// A captured device-controlled program (one stage of Alg. 1, or one NewtonSolve),
// keyed by everything baked into its kernel arguments. The kernels of its top
// level and of each conditional body are counted at capture time, so that the
// kernels a launch ran follow from the device's loop counters.
typedef std::tuple<int, int, int, int64_t, int64_t, int64_t, uintptr_t> ProgKey;
constexpr int kProgBodies = 8;
struct ProgGraph {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int64_t top_kernels = 0;
  int64_t body_kernels[kProgBodies] = {};
};

struct eot_handle_s {
  int device = 0;
  int sms = 152;
  int64_t l2_bytes = 0;
  int64_t cap_n = 0, cap_m = 0, cap_rowpart = 0;
  std::string err = "no error";
  int64_t launches = 0;
  std::vector<void*> allocs;

  // scalars and status
  double* sc = nullptr;     // device [SC_TOTAL]
  double* h_sc = nullptr;   // pinned host [SC_TOTAL + 1]
  int* status = nullptr;    // device
  int* h_status = nullptr;  // pinned host
  // sweep scratch
  int *cnt_strip = nullptr, *cnt_rowblk = nullptr, *cnt_dot = nullptr;
  double *colpart = nullptr, *rowpart = nullptr, *dotpart = nullptr;
  int64_t max_strips = 0, max_rowblk = 64, dot_slots = 0, rowblk_slots = 0;
  double* maxbuf = nullptr;  // per-CTA candidates of the point-cost maximum
  int64_t maxbuf_len = 0;
  // FP64 n-vectors
  double *Al = nullptr, *rowfac = nullptr, *rP = nullptr, *logrP = nullptr, *rowmax = nullptr;
  double *rt = nullptr, *logrt = nullptr, *du = nullptr, *x = nullptr, *res = nullptr;
  double *z = nullptr, *p = nullptr, *q = nullptr, *y = nullptr, *Yx = nullptr, *M = nullptr;
  double *diag = nullptr, *y0 = nullptr, *du0 = nullptr, *nt0 = nullptr, *nt1 = nullptr;
  double* rPs = nullptr;  // row sums of the factorised plan used inside F_r
  double* U = nullptr;    // working potentials of the device-controlled programs
  // FP64 m-vectors
  double *Bl = nullptr, *colfac = nullptr, *cP = nullptr, *logcP = nullptr, *ct = nullptr;
  double *logct = nullptr, *dv = nullptr, *mt0 = nullptr, *mt1 = nullptr;
  double* V = nullptr;
  double* wprev = nullptr;  // dense CG: P^T (rowfac p) of the previous iteration
  // v-blocks of the full-system NewtonSolve's PCG vectors (x, res, z, p, q)
  double *fxv = nullptr, *frv = nullptr, *fzv = nullptr, *fpv = nullptr, *fqv = nullptr;
  double* cgpart = nullptr; // dense CG: per-CTA (<res, z>, ||res||_1) partials of the update kernel
  // element-type vectors (8 bytes per entry, used as float or double)
  void *Ah = nullptr, *Bh = nullptr, *xw0 = nullptr, *xw1 = nullptr, *zf = nullptr;
  void *wsq = nullptr, *ewr = nullptr, *ewc = nullptr;

  std::map<ProgKey, ProgGraph> graphs;
  cudaStream_t cap_streams[8] = {};  // one capture stream per nesting depth of a program

  // eot_solve_batched: its own device block (not in `allocs`: growing the
  // single-problem buffers must not free it) and the autotuner's choices
  void* rd_mem = nullptr;  // Round: FP64 vectors and column partials (own block)
  size_t rd_bytes = 0;
  void* tc_mem = nullptr;  // tensor-core point path: digit slices and row data (own block)
  size_t tc_bytes = 0;
  void* bt_mem = nullptr;
  size_t bt_bytes = 0;
  std::map<std::string, std::pair<int, int>> bt_tune;  // batch shape -> (G, elements per thread)
  int bt_last[3] = {0, 0, 0};                          // G, elements per thread, groups of the last launch
};

namespace eot {

// Kernel launch with programmatic stream serialisation (PDL): the kernel may
// begin while its predecessor in the stream drains; every kernel of this
// library calls pdl_wait() before touching data of earlier kernels.
// EOT_PDL=0 in the environment turns the attribute off. A captured launch that
// directly follows a conditional graph node gets a plain edge (programmatic
// edges join kernel nodes only): the capture sets pdl_skip_next.
inline bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("EOT_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}
inline thread_local bool pdl_skip_next = false;
inline unsigned pdl_attrs() {
  const bool on = pdl_enabled() && !pdl_skip_next;
  pdl_skip_next = false;
  return on ? 1u : 0u;
}
// launch_k with dynamic shared memory
template <typename... KArgs, typename... Args>
inline void launch_kd(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                      Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_attrs();
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  if (e != cudaSuccess)
    throw EotError{EOT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e)};
}
// launch_k in thread-block clusters of (1, cy, 1) CTAs
template <typename... KArgs, typename... Args>
inline void launch_kc(void (*kernel)(KArgs...), dim3 grid, dim3 block, unsigned cy, cudaStream_t st,
                      Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 1;
  at[0].val.clusterDim.y = cy;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1 + pdl_attrs();
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  if (e != cudaSuccess)
    throw EotError{EOT_ERR_CUDA, std::string("cluster kernel launch: ") + cudaGetErrorString(e)};
}
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_attrs();
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
  if (e != cudaSuccess)
    throw EotError{EOT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e)};
}

inline void* dev_alloc(eot_handle h, size_t bytes) {
  void* p = nullptr;
  EOT_CUDA(cudaMalloc(&p, bytes < 256 ? 256 : bytes));
  h->allocs.push_back(p);
  return p;
}

void ensure_capacity(eot_handle h, int64_t n, int64_t m);
void ensure_rowpart(eot_handle h, int64_t n, int64_t strips);
void ensure_rowpart_elems(eot_handle h, int64_t elems);
void free_graphs(eot_handle h);

// sweep geometry
struct ColGeo {
  int64_t S;
  int R, BR;
};
inline ColGeo col_geo(eot_handle h, int64_t n, int64_t m, int V, int64_t rcap = 1 << 30) {
  ColGeo g;
  g.S = (m + 32 * V - 1) / (32 * V);
  // one wave: S * R <= resident CTAs
  const int64_t target = (int64_t)kColCtasPerSm * h->sms;
  int64_t R = target / g.S;
  int64_t rmax = (n + 31) / 32;
  if (R > rmax) R = rmax;
  if (R > h->max_rowblk) R = h->max_rowblk;
  if (R > rcap) R = rcap;
  if (R < 1) R = 1;
  int64_t BR = (n + R - 1) / R;
  BR = (BR + 31) / 32 * 32;
  g.BR = (int)BR;
  g.R = (int)((n + BR - 1) / BR);
  return g;
}
// one row per warp: ceil(n / 8) CTAs
inline int row_grid(int64_t n) {
  int64_t g = (n + kWarps - 1) / kWarps;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace eot
