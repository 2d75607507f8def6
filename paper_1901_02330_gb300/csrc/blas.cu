// Sparse and dense vector kernels of the Krylov loop: CSR SpMV with a group
// of L lanes per row (optionally fused with the dot product x . (A x)), and
// deterministic partial dot products.
#include <atomic>

#include "handle.cuh"

namespace vem {

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(); }

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 152;
  }
  return n;
}

int grid_for(int64_t n, int threads, int per_sm) {
  int64_t b = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * per_sm;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

int nblocks_vec(int64_t n) {
  int64_t b = (n + kRedThreads - 1) / kRedThreads;
  int64_t cap = (int64_t)num_sms() * 4;
  if (cap > kMaxBlocks) cap = kMaxBlocks;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// y = A x for a SELL-32 matrix: one warp per slice, one thread per row, one
// FP64 FMA per stored element and lane (no shuffles), coalesced loads of the
// matrix (streamed, evict-first) and read-only-path gathers of x.  With
// dot_part, also the partials of x . (A x).
__global__ void __launch_bounds__(256) k_sell_spmv(int64_t rows, int64_t nslices,
                                                   const int64_t *__restrict__ off,
                                                   const int32_t *__restrict__ col,
                                                   const double *__restrict__ val,
                                                   const double *__restrict__ x, double *__restrict__ y,
                                                   double *dot_part) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dacc = 0.0;
  for (int64_t s = warp; s < nslices; s += nwarps) {
    const double t = sell_row_dot<double>(off, col, val, x, s, lane);
    const int64_t r = 32 * s + lane;
    if (r < rows) {
      y[r] = t;
      if (dot_part) dacc += t * x[r];
    }
  }
  if (dot_part) block_partial(dacc, dot_part);
}

// Blocks of 256 threads that fit on the GPU at once for this kernel: grid-
// stride kernels launched with exactly one wave avoid a partial second wave.
int one_wave_blocks(const void *kernel) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, 0) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 4;
  }
  int64_t cap = (int64_t)num_sms() * occ;
  if (cap > kMaxBlocks) cap = kMaxBlocks;
  return (int)cap;
}

int spmv_nblocks(const SellMat &A, int nbatch) {
  static int cap = 0;
  if (cap == 0) cap = one_wave_blocks((const void *)k_sell_spmv);
  int64_t b = (A.nslices * nbatch + 7) / 8;   // one warp per slice, 8 warps per block
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

void spmv(cudaStream_t s, const SellMat &A, const double *x, double *y, double *dot_part) {
  count_launch();
  k_sell_spmv<<<spmv_nblocks(A, 1), 256, 0, s>>>(A.rows, A.nslices, A.off, A.col, A.val, x, y, dot_part);
}

// Batched y = A_b x_b for nb systems sharing one SELL structure (column ids
// read once per system from the shared arrays), values of system b at
// vals + b * stored.  Stacked vector layout: local index i < split of system
// b at b * split + i, the others at nb * split + b * (rows - split) + (i - split).
__global__ void __launch_bounds__(256) k_sell_spmv_b(int64_t rows, int64_t nslices, int nb, int64_t split,
                                                     int64_t stored, const int64_t *__restrict__ off,
                                                     const int32_t *__restrict__ col,
                                                     const double *__restrict__ vals,
                                                     const double *__restrict__ x, double *__restrict__ y,
                                                     double *dot_part) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double dacc = 0.0;
  const int64_t tasks = nslices * nb;
  for (int64_t tk = warp; tk < tasks; tk += nwarps) {
    const int64_t b = tk / nslices, s = tk - b * nslices;
    const int64_t olo = b * split, ohi = (int64_t)(nb - 1) * split + b * (rows - split);
    const int64_t o = off[s];
    const int w = (int)((off[s + 1] - o) >> 5);
    const double *vp = vals + b * stored + o + lane;
    const int32_t *cp = col + o + lane;
    double t = 0.0;
    int j = 0;
    for (; j + 1 < w; j += 2) {
      const int64_t c0 = __ldcs(cp + 32 * j), c1 = __ldcs(cp + 32 * (j + 1));
      const double v0 = __ldcs(vp + 32 * j), v1 = __ldcs(vp + 32 * (j + 1));
      const double x0 = __ldg(x + c0 + (c0 < split ? olo : ohi)), x1 = __ldg(x + c1 + (c1 < split ? olo : ohi));
      t += v0 * x0;
      t += v1 * x1;
    }
    if (j < w) {
      const int64_t c0 = __ldcs(cp + 32 * j);
      t += __ldcs(vp + 32 * j) * __ldg(x + c0 + (c0 < split ? olo : ohi));
    }
    const int64_t r = 32 * s + lane;
    if (r < rows) {
      const int64_t R = r + (r < split ? olo : ohi);
      y[R] = t;
      if (dot_part) dacc += t * x[R];
    }
  }
  if (dot_part) block_partial(dacc, dot_part);
}

void spmv_batched(cudaStream_t s, const SellMat &A, int nb, int64_t split, const double *vals,
                  const double *x, double *y, double *dot_part) {
  count_launch();
  k_sell_spmv_b<<<spmv_nblocks(A, nb), 256, 0, s>>>(A.rows, A.nslices, nb, split, A.stored, A.off, A.col, vals,
                                                    x, y, dot_part);
}

__global__ void __launch_bounds__(kRedThreads) k_dot(int64_t n, const double *__restrict__ x,
                                                     const double *__restrict__ y, double *part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * y[i];
  block_partial(s, part);
}

void dot_partials(cudaStream_t s, int64_t n, const double *x, const double *y, double *part) {
  count_launch(); k_dot<<<nblocks_vec(n), kRedThreads, 0, s>>>(n, x, y, part);
}

}  // namespace vem
