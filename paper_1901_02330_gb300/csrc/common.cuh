// Shared definitions of the vemsolve CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/vemsolve.h"

namespace vem {

// Device error flags (bit set by kernels, read back by the host).
enum : int {
  DEVERR_DEGENERATE_FACE = 1,
  DEVERR_DEGENERATE_CELL = 2,
  DEVERR_NONCONVEX = 4,
  DEVERR_ADJACENCY = 8,
  DEVERR_NONFINITE = 16,
  DEVERR_SINGULAR_LOCAL = 32,
  DEVERR_AMG_DIAG = 64,        // AMG: non-positive diagonal or pivot
  DEVERR_AMG_ROW = 128,        // AMG: a product row exceeds its column list
  DEVERR_NONPOSITIVE = 256,    // a coefficient K <= 0
  DEVERR_LAYOUT = 512,         // a flux row couples to more pressure DOFs than its cells hold
};

struct Status {
  vem_status code = VEM_OK;
  std::string msg;
};

// A device buffer owned by the handle.
template <class T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
};

// Sliced ELL matrix (slices of 32 rows, column-major inside a slice).
struct SellMat {
  int64_t rows = 0, nslices = 0, stored = 0, nnz = 0;
  int64_t *off = nullptr;   // [nslices + 1] element offset of each slice
  int32_t *len = nullptr;   // [nslices * 32] true row lengths (0 for ghost rows)
  int32_t *col = nullptr;   // [stored] column ids (padding: 0)
  double *val = nullptr;    // [stored] values (padding: 0)
};

__device__ __forceinline__ int64_t sell_pos(const int64_t *off, int64_t r, int j) {
  return off[r >> 5] + ((int64_t)j << 5) + (r & 31);
}

// Launch geometry: a multiple of the SM count.
int num_sms();

// Process-wide count of kernel launches issued by the library.
void count_launch();
void count_launches(int64_t n);   // n may be negative (launches recorded into a graph)
int64_t launch_count();

// ---- programmatic dependent launch -----------------------------------------
// The latency-bound chains (V-cycle and inner-CG kernels) are launched with
// programmatic stream serialisation: a kernel's blocks may be scheduled while
// the previous kernel of the stream drains, and every such kernel first
// waits (griddepcontrol.wait) until that kernel has completed and its memory
// is visible, before it reads or writes anything.  Without the launch
// attribute the wait returns at once.
__device__ __forceinline__ void pdl_wait() {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 900)
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---- reductions -----------------------------------------------------------
// Deterministic two-pass reductions: every block writes its partial sums to
// part[slot * kMaxBlocks + block]; a consumer sums the partials of a slot in
// block order.
constexpr int kRedThreads = 256;
constexpr int kMaxBlocks = 1216;   // 8 x 152 SMs
constexpr int kMaxSlots = 300;     // FGMRES(m <= 256) needs m + 2 slots
constexpr int kBtRow = 8;          // B^T entries kept per flux row (two cells x 4 P1 moments)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of the nb partials of one slot, evaluated identically by every caller.
__device__ __forceinline__ double sum_partials(const double *part, int nb) {
  // every thread sums a strided subset, then a fixed-order tree over the block
  __shared__ double red_s[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v += part[i];
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red_s[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (l < (int)(blockDim.x >> 5)) ? red_s[l] : 0.0;
    t = warp_sum(t);
    if (l == 0) red_s[0] = t;
  }
  __syncthreads();
  double r = red_s[0];
  __syncthreads();
  return r;
}

// Block-wide sum written to part[blockIdx.x] (fixed order).
__device__ __forceinline__ void block_partial(double v, double *part) {
  __shared__ double bp_s[32];
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) bp_s[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (l < (int)(blockDim.x >> 5)) ? bp_s[l] : 0.0;
    t = warp_sum(t);
    if (l == 0) part[blockIdx.x] = t;
  }
  __syncthreads();
}

// Row (32 s + lane) of a SELL-32 matrix times x, one FMA chain per row
// (GB300 issues FP64 at 1/16 of the lane rate, so combining partial
// accumulators would cost FP64 adds per row); T = double or float (values,
// x and arithmetic share the type).  Entries go in batches: all (col, val)
// loads of a batch, then its gathers, then its FMAs.  Unpredicated: batches
// of four and a one-at-a-time tail.  kPred: batches of kB, the last one
// predicated on the slice width (uniform across the warp), so a row of up
// to kB entries costs one round trip.
#ifndef VEM_CG_KB
#define VEM_CG_KB 8
#endif
#ifndef VEM_CG_PRED
#define VEM_CG_PRED 1
#endif
template <class T, int kB = 4, bool kPred = false>
__device__ __forceinline__ T sell_row_dot(const int64_t *__restrict__ off,
                                          const int32_t *__restrict__ col,
                                          const T *__restrict__ val, const T *__restrict__ x,
                                          int64_t s, int lane) {
  const int64_t o = off[s];
  const int w = (int)((off[s + 1] - o) >> 5);
  const T *vp = val + o + lane;
  const int32_t *cp = col + o + lane;
  T acc = 0;
  int j = 0;
  if constexpr (kPred) {
    for (; j < w; j += kB) {
      int32_t c[kB];
      T v[kB], xv[kB];
#pragma unroll
      for (int k = 0; k < kB; ++k) {
        c[k] = 0;
        v[k] = xv[k] = 0;
        if (j + k < w) {
          c[k] = __ldcs(cp + 32 * (j + k));
          v[k] = __ldcs(vp + 32 * (j + k));
        }
      }
#pragma unroll
      for (int k = 0; k < kB; ++k)
        if (j + k < w) xv[k] = __ldg(x + c[k]);
#pragma unroll
      for (int k = 0; k < kB; ++k)
        if (j + k < w) acc += v[k] * xv[k];
    }
  } else {
    static_assert(kB == 4, "the unpredicated form issues four entries per batch");
    for (; j + 3 < w; j += 4) {
      const int32_t c0 = __ldcs(cp + 32 * j), c1 = __ldcs(cp + 32 * (j + 1));
      const int32_t c2 = __ldcs(cp + 32 * (j + 2)), c3 = __ldcs(cp + 32 * (j + 3));
      const T v0 = __ldcs(vp + 32 * j), v1 = __ldcs(vp + 32 * (j + 1));
      const T v2 = __ldcs(vp + 32 * (j + 2)), v3 = __ldcs(vp + 32 * (j + 3));
      const T x0 = __ldg(x + c0), x1 = __ldg(x + c1), x2 = __ldg(x + c2), x3 = __ldg(x + c3);
      acc += v0 * x0;
      acc += v1 * x1;
      acc += v2 * x2;
      acc += v3 * x3;
    }
    for (; j < w; ++j) acc += __ldcs(vp + 32 * j) * __ldg(x + __ldcs(cp + 32 * j));
  }
  return acc;
}

// Last-block-done pattern: after each block has stored its partials, the
// block that arrives last at *counter returns true and may read them all
// (then sums them in a fixed order, so results stay deterministic).  It
// resets the counter for the next use.
__device__ __forceinline__ bool last_block(unsigned int *counter) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
    if (is_last) *counter = 0u;
  }
  __syncthreads();
  const bool r = is_last != 0;
  if (r) __threadfence();
  return r;
}

// Fixed-order sum of nb partials read through L2 (for use by the last block).
__device__ __forceinline__ double sum_partials_cg(const double *part, int nb) {
  __shared__ double rs[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v += __ldcg(part + i);
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) rs[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (l < (int)(blockDim.x >> 5)) ? rs[l] : 0.0;
    t = warp_sum(t);
    if (l == 0) rs[0] = t;
  }
  __syncthreads();
  const double out = rs[0];
  __syncthreads();
  return out;
}

}  // namespace vem
