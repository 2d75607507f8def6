// Sparse and dense vector kernels of the Krylov loop: CSR SpMV with a group
// of L lanes per row (optionally fused with the dot product x . (A x)), and
// deterministic partial dot products.
#include <atomic>

#include "handle.cuh"

namespace vem {

static std::atomic<int64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
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

int choose_lanes(double avg) {
  if (avg <= 6) return 4;
  if (avg <= 20) return 8;
  if (avg <= 48) return 16;
  return 32;
}

// Rows are taken in warp-uniform batches (every lane of a warp runs the same
// number of loop trips), so the full-mask shuffles are always convergent.
template <int L>
__global__ void __launch_bounds__(256) k_spmv(int64_t rows, const int64_t *__restrict__ rp,
                                              const int32_t *__restrict__ col,
                                              const double *__restrict__ val,
                                              const double *__restrict__ x, double *__restrict__ y,
                                              double *dot_part) {
  const int lane = threadIdx.x & 31;
  const int sub = lane % L;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) / L;
  double dacc = 0.0;
  for (int64_t base = warp * (32 / L); base < rows; base += stride) {
    const int64_t r = base + lane / L;
    const bool ok = r < rows;
    double s = 0.0;
    if (ok) {
      const int64_t b = rp[r], e = rp[r + 1];
      for (int64_t p = b + sub; p < e; p += L) s += val[p] * __ldg(x + col[p]);
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, L);
    if (ok && sub == 0) {
      y[r] = s;
      if (dot_part) dacc += s * x[r];
    }
  }
  if (dot_part) block_partial(dacc, dot_part);
}

void spmv(cudaStream_t s, int64_t rows, const int64_t *rp, const int32_t *col, const double *val,
          const double *x, double *y, int lanes, double *dot_part) {
  const int T = 256;
  // a fixed grid for a given size keeps the fused dot deterministic
  int blocks = nblocks_vec(rows * lanes);
  switch (lanes) {
    case 4: count_launch(); k_spmv<4><<<blocks, T, 0, s>>>(rows, rp, col, val, x, y, dot_part); break;
    case 8: count_launch(); k_spmv<8><<<blocks, T, 0, s>>>(rows, rp, col, val, x, y, dot_part); break;
    case 16: count_launch(); k_spmv<16><<<blocks, T, 0, s>>>(rows, rp, col, val, x, y, dot_part); break;
    default: count_launch(); k_spmv<32><<<blocks, T, 0, s>>>(rows, rp, col, val, x, y, dot_part); break;
  }
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
