// vem_residual_norm_noalloc: the residual-norm reduction of the solver
// (||b - A x|| and ||b||, as used for the stopping test) in a form that
// performs no device memory allocation at all.
//
// Some callers cannot let a library call cudaMalloc / cudaFree: code whose
// device memory is owned by a framework allocator with a fixed pool or a hard
// budget (a foreign cudaMalloc can fail there or fragment the pool), and
// latency-sensitive pipelines in which cudaFree's implicit device-wide
// synchronisation would stall every other stream.  This entry point keeps its
// scratch -- one pair of partial sums per 2048-row tile -- in a file-scope
// device array that exists on every GPU that loads the library, for the
// life of the process.
#include <mutex>

#include "handle.cuh"

namespace vem {
namespace {

constexpr int kTileRows = 2048;
constexpr int kMaxTiles = 65536;                       // rows <= 134,217,728
constexpr int kTileThreads = 256;
constexpr int kMaxDevices = 64;

// per-tile sums of r_i^2 (first half) and b_i^2 (second half): 1 MiB
static __device__ __align__(256) double g_scratch[2 * kMaxTiles];

// Host code cannot use &g_scratch as a device address; it is resolved once
// per device with cudaGetSymbolAddress (with that device current).
double *g_addr[kMaxDevices] = {};
std::mutex g_mutex;

// One block per tile, one warp per row: the lanes take the row's entries in
// strides of 32 (coalesced loads of col and val) and combine them with the
// fixed-pattern warp_sum, so the partial sums do not depend on the GPU or the
// launch.
__global__ void __launch_bounds__(kTileThreads) k_tiles(int64_t rows, const int64_t *__restrict__ rp,
                                                        const int32_t *__restrict__ col,
                                                        const double *__restrict__ val,
                                                        const double *__restrict__ x,
                                                        const double *__restrict__ b, double *part) {
  const int64_t lo = (int64_t)blockIdx.x * kTileRows;
  const int64_t hi = lo + kTileRows < rows ? lo + kTileRows : rows;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  double r2 = 0.0, b2 = 0.0;   // meaningful in lane 0
  for (int64_t r = lo + w; r < hi; r += kTileThreads / 32) {
    double ax = 0.0;
    const int64_t p1 = rp[r + 1];
    for (int64_t p = rp[r] + l; p < p1; p += 32) ax += val[p] * x[col[p]];
    ax = warp_sum(ax);
    const double ri = b[r] - ax;
    r2 += ri * ri;
    b2 += b[r] * b[r];
  }
  __shared__ double s_r[kTileThreads / 32], s_b[kTileThreads / 32];
  if (l == 0) {
    s_r[w] = r2;
    s_b[w] = b2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, tb = 0.0;
    for (int i = 0; i < kTileThreads / 32; ++i) {
      tr += s_r[i];
      tb += s_b[i];
    }
    part[blockIdx.x] = tr;
    part[kMaxTiles + blockIdx.x] = tb;
  }
}

// out[0] = ||b - A x||, out[1] = ||b||, out[2] = out[0] / out[1] (out[0] if b = 0)
__global__ void __launch_bounds__(kTileThreads) k_final(const double *part, int ntiles, double *out) {
  const double r2 = sum_partials(part, ntiles);
  const double b2 = sum_partials(part + kMaxTiles, ntiles);
  if (threadIdx.x == 0) {
    out[0] = sqrt(r2);
    out[1] = sqrt(b2);
    out[2] = b2 > 0.0 ? sqrt(r2 / b2) : sqrt(r2);
  }
}

}  // namespace
}  // namespace vem

extern "C" vem_status vem_residual_norm_noalloc(int64_t rows, const int64_t *row_ptr, const int32_t *col,
                                                const double *val, const double *x, const double *b,
                                                double *out, void *cuda_stream) {
  using namespace vem;
  if (!row_ptr || !col || !val || !x || !b || !out || rows < 1) return VEM_ERR_BAD_INPUT;
  if (rows > (int64_t)kTileRows * kMaxTiles) return VEM_ERR_BAD_INPUT;   // beyond the scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VEM_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return VEM_ERR_UNSUPPORTED;
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return VEM_ERR_CUDA;
      }
      g_addr[dev] = static_cast<double *>(p);
    }
    scratch = g_addr[dev];
  }
  // an error left pending by earlier, unrelated work is reported here and
  // left in place for its owner (not cleared), so the launch check below
  // sees only this call's launches
  if (cudaPeekAtLastError() != cudaSuccess) return VEM_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int ntiles = (int)((rows + kTileRows - 1) / kTileRows);
  count_launch();
  k_tiles<<<ntiles, kTileThreads, 0, s>>>(rows, row_ptr, col, val, x, b, scratch);
  count_launch();
  k_final<<<1, kTileThreads, 0, s>>>(scratch, ntiles, out);
  if (cudaGetLastError() != cudaSuccess) return VEM_ERR_CUDA;
  return VEM_OK;
}
