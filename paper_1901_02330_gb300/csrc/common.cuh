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

struct Handle;

// Launch geometry: a multiple of the SM count.
int num_sms();

// Process-wide count of kernel launches issued by the library.
void count_launch();
int64_t launch_count();

// ---- reductions -----------------------------------------------------------
// Deterministic two-pass reductions: every block writes its partial sums to
// part[slot * kMaxBlocks + block]; a consumer sums the partials of a slot in
// block order.
constexpr int kRedThreads = 256;
constexpr int kMaxBlocks = 1216;   // 8 x 152 SMs
constexpr int kMaxSlots = 300;     // FGMRES(m <= 256) needs m + 2 slots

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

}  // namespace vem
