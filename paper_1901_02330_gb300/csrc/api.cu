// C-ABI entry points of include/vemsolve.h: argument checking, device
// memory, and the order of the assembly / solve phases.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

#include "handle.cuh"

namespace vem {

vem_status fail(vem_handle *h, vem_status code, const char *fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    h->last_error = buf;
  }
  return code;
}

vem_status cuda_check(vem_handle *h, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return VEM_OK;
  cudaGetLastError();   // clear a non-sticky error
  if (e == cudaErrorMemoryAllocation)
    return fail(h, VEM_ERR_OOM, "%s: out of device memory", what);
  return fail(h, VEM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Device memory comes from one stream-ordered pool per device that keeps
// freed memory reserved (release threshold: unlimited), so a handle created
// after another one was destroyed reuses its memory without cudaMalloc or
// cudaFree (which synchronise the device).  vem_release_memory returns the
// unused part to the system.
static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

static cudaError_t device_pool(cudaMemPool_t *out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool;
  e = cudaMemPoolCreate(&pool, &props);
  if (e != cudaSuccess) return e;
  uint64_t thr = ~0ull;
  e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  if (e != cudaSuccess) return e;
  g_pools[dev] = pool;
  *out = pool;
  return cudaSuccess;
}

// Small pinned host buffers (scalar read-backs) are kept for the next handle
// too: cudaMallocHost / cudaFreeHost are slow and may synchronise.
static std::mutex g_pinned_mu;
static std::vector<std::pair<void *, size_t>> g_pinned_free;

static cudaError_t pinned_alloc(void **p, size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    for (size_t i = 0; i < g_pinned_free.size(); ++i)
      if (g_pinned_free[i].second >= bytes) {
        *p = g_pinned_free[i].first;
        g_pinned_free.erase(g_pinned_free.begin() + (std::ptrdiff_t)i);
        return cudaSuccess;
      }
  }
  return cudaMallocHost(p, bytes);
}

static void pinned_free(void *p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  g_pinned_free.emplace_back(p, bytes);
}

vem_status dalloc(vem_handle *h, void **p, size_t bytes) {
  *p = nullptr;
  cudaMemPool_t pool;
  cudaError_t e = device_pool(&pool);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, pool, h->stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(h, e == cudaErrorMemoryAllocation ? VEM_ERR_OOM : VEM_ERR_CUDA,
                "device allocation (%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  h->allocations.push_back(*p);
  return VEM_OK;
}

void dfree(vem_handle *h, void *p) {
  if (!p) return;
  auto it = std::find(h->allocations.begin(), h->allocations.end(), p);
  if (it != h->allocations.end()) h->allocations.erase(it);
  cudaFreeAsync(p, h->stream);
}

vem_status check_device_errors(vem_handle *h, const char *what) {
  VEM_CUDA(h, cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  VEM_CUDA(h, cudaStreamSynchronize(h->stream));
  const int e = *h->h_err;
  if (e == 0) return VEM_OK;
  VEM_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  if (e & DEVERR_ADJACENCY)
    return fail(h, VEM_ERR_BAD_INPUT, "%s: a face is not shared by one or two cells as its flag says", what);
  if (e & DEVERR_DEGENERATE_FACE) return fail(h, VEM_ERR_DEGENERATE_MESH, "%s: zero-area face", what);
  if (e & DEVERR_DEGENERATE_CELL) return fail(h, VEM_ERR_DEGENERATE_MESH, "%s: zero-volume cell", what);
  if (e & DEVERR_NONCONVEX) return fail(h, VEM_ERR_DEGENERATE_MESH, "%s: non-convex cell", what);
  if (e & DEVERR_SINGULAR_LOCAL) return fail(h, VEM_ERR_DEGENERATE_MESH, "%s: singular local Gram matrix", what);
  if (e & DEVERR_NONFINITE) return fail(h, VEM_ERR_NONFINITE, "%s: NaN or Inf in data", what);
  if (e & DEVERR_NONPOSITIVE) return fail(h, VEM_ERR_BAD_INPUT, "%s: K <= 0", what);
  if (e & DEVERR_LAYOUT) return fail(h, VEM_ERR_BAD_INPUT, "%s: flux row with too many pressure couplings", what);
  if (e & DEVERR_AMG_DIAG) return fail(h, VEM_ERR_BREAKDOWN, "%s: non-positive diagonal or pivot", what);
  if (e & DEVERR_AMG_ROW)
    return fail(h, VEM_ERR_UNSUPPORTED, "%s: a row of an AMG product has too many distinct columns", what);
  return fail(h, VEM_ERR_CUDA, "%s: device error flags %d", what, e);
}

static vem_status check_options(vem_handle *h, const vem_options *o) {
  if (o->element != VEM_ELEMENT_E0 && o->element != VEM_ELEMENT_K1 && o->element != VEM_ELEMENT_K2)
    return fail(h, VEM_ERR_BAD_INPUT, "unknown element %d", o->element);
  if (o->krylov != VEM_KRYLOV_MINRES && o->krylov != VEM_KRYLOV_FGMRES)
    return fail(h, VEM_ERR_BAD_INPUT, "unknown Krylov method %d", o->krylov);
  if (o->precond != VEM_PREC_BLOCK_DIAG && o->precond != VEM_PREC_BLOCK_TRI && o->precond != VEM_PREC_BLOCK_REG)
    return fail(h, VEM_ERR_BAD_INPUT, "unknown preconditioner %d", o->precond);
  if (o->krylov == VEM_KRYLOV_MINRES && o->precond == VEM_PREC_BLOCK_TRI)
    return fail(h, VEM_ERR_BAD_INPUT, "MINRES needs an SPD block-diagonal preconditioner");
  if (!(o->reg_gamma >= 0.0) || !std::isfinite(o->reg_gamma))
    return fail(h, VEM_ERR_BAD_INPUT, "reg_gamma %g", o->reg_gamma);
  if (o->inner != VEM_INNER_PCG && o->inner != VEM_INNER_AMG && o->inner != VEM_INNER_BLOCK_AMG)
    return fail(h, VEM_ERR_BAD_INPUT, "unknown inner solver %d", o->inner);
  if (o->inner_smoother != VEM_SMOOTH_JACOBI && o->inner_smoother != VEM_SMOOTH_CHEBYSHEV)
    return fail(h, VEM_ERR_BAD_INPUT, "unknown inner smoother %d", o->inner_smoother);
  if (o->reg_cycle != VEM_REG_SCALAR_AMG && o->reg_cycle != VEM_REG_CONDENSED)
    return fail(h, VEM_ERR_BAD_INPUT, "unknown Block-Reg cycle %d", o->reg_cycle);
  if (o->precision != VEM_PRECISION_FP64 && o->precision != VEM_PRECISION_MIXED)
    return fail(h, VEM_ERR_BAD_INPUT, "unknown precision %d", o->precision);
  if (o->precision == VEM_PRECISION_MIXED && o->krylov != VEM_KRYLOV_FGMRES)
    return fail(h, VEM_ERR_BAD_INPUT, "mixed precision needs FGMRES (its FP32 inner solve is not a fixed operator)");
  if (o->restart < 1 || o->restart > 256) return fail(h, VEM_ERR_BAD_INPUT, "restart %d", o->restart);
  if (o->reuse != 0 && o->reuse != 1) return fail(h, VEM_ERR_BAD_INPUT, "reuse %d", o->reuse);
  if (!(o->rtol > 0.0) || !(o->inner_rtol > 0.0) || o->maxit < 1 || o->inner_maxit < 1)
    return fail(h, VEM_ERR_BAD_INPUT, "tolerances and iteration caps must be positive");
  return VEM_OK;
}

static void set_layout(vem_handle *h) {
  h->nq = 1;
  if (h->opt.element == VEM_ELEMENT_K2) {
    h->nfd = 6;
    h->nid = 14;
    h->nq = 4;
  } else if (h->opt.element == VEM_ELEMENT_K1) {
    h->nfd = 3;
    h->nid = 3;
  } else {
    h->nfd = 1;
    h->nid = 0;
  }
  h->n_u = h->nfd * h->nf + h->nid * h->nc;
  h->n_p = (int64_t)h->nq * h->nc;
  h->n = h->n_u + h->n_p;
}

template <class T>
static vem_status upload(vem_handle *h, T **dst, const T *src, size_t n) {
  VEM_TRY(dalloc_n(h, dst, n));
  VEM_CUDA(h, cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  return VEM_OK;
}

// ---- mesh checks on the device (the arrays are uploaded first; these
// kernels read them sequentially, no index is followed before it passed) ----
enum {
  MS_ERR = 0,        // error bits MSE_*
  MS_BAD_FACE, MS_BAD_CELL, MS_BAD_FV, MS_BAD_CF, MS_BAD_X,   // smallest offending index
  MS_MAXNV, MS_MAXNF, MS_NFLUX, MS_NDIR,
  MS_LO, MS_HI = MS_LO + 3,                                      // ordered bits of min / max coordinates
  MS_COUNT = MS_HI + 3
};
enum { MSE_FACE_NV = 1, MSE_FLAG = 2, MSE_CELL_NF = 4, MSE_VTX = 8, MSE_FACE = 16, MSE_COORD = 32 };

// order-preserving map of a double to an unsigned integer
__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
static double from_ordered(unsigned long long k) {
  const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  double d;
  std::memcpy(&d, &u, sizeof(d));
  return d;
}

__device__ __forceinline__ void warp_add(unsigned long long v, unsigned long long *out) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

// flag[i] = 1 where cnt[i] > 0, else 0 (in place)
__global__ void k_flag_positive(int64_t n, int64_t *cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    cnt[i] = cnt[i] > 0 ? 1 : 0;
}

// ids[pos[i]] = i where flag[i] (pos: exclusive scan of flag)
__global__ void k_compact_ids(int64_t n, const int64_t *__restrict__ flag, const int64_t *__restrict__ pos,
                              int32_t *ids) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flag[i]) ids[pos[i]] = (int32_t)i;
}

__global__ void k_check_faces(int64_t nf, const int64_t *__restrict__ fvp, const int8_t *__restrict__ fbc,
                              unsigned long long *ms, int64_t *bq_cnt, int ppt) {
  unsigned long long nflux = 0, ndir = 0, mx = 0;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = fvp[f + 1] - fvp[f];
    const int fl = fbc[f];
    if (k < 3 || k > 4096) {
      atomicOr(&ms[MS_ERR], (unsigned long long)MSE_FACE_NV);
      atomicMin(&ms[MS_BAD_FACE], (unsigned long long)f);
    }
    if (fl < 0 || fl > 2) {
      atomicOr(&ms[MS_ERR], (unsigned long long)MSE_FLAG);
      atomicMin(&ms[MS_BAD_FACE], (unsigned long long)f);
    }
    nflux += fl == 2;
    ndir += fl == 1;
    if (k > 0 && (unsigned long long)k > mx) mx = (unsigned long long)k;
    bq_cnt[f] = (fl != 0 && k > 0) ? ppt * k : 0;   // boundary-face load points: ppt per fan triangle
  }
  warp_add(nflux, &ms[MS_NFLUX]);
  warp_add(ndir, &ms[MS_NDIR]);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(&ms[MS_MAXNV], mx);
}

__global__ void k_check_cells(int64_t nc, const int64_t *__restrict__ cfp, unsigned long long *ms) {
  unsigned long long mx = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = cfp[c + 1] - cfp[c];
    if (k < 4 || k > 256) {
      atomicOr(&ms[MS_ERR], (unsigned long long)MSE_CELL_NF);
      atomicMin(&ms[MS_BAD_CELL], (unsigned long long)c);
    }
    if (k > 0 && (unsigned long long)k > mx) mx = (unsigned long long)k;
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(&ms[MS_MAXNF], mx);
}

__global__ void k_check_ids(int64_t n, const int32_t *__restrict__ ids, int64_t lim, int bit, int slot,
                            unsigned long long *ms) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = ids[i];
    if (v < 0 || v >= lim) {
      atomicOr(&ms[MS_ERR], (unsigned long long)bit);
      atomicMin(&ms[slot], (unsigned long long)i);
    }
  }
}

__global__ void k_check_coords(int64_t nv, const double *__restrict__ xyz, unsigned long long *ms) {
  unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    for (int d = 0; d < 3; ++d) {
      const double v = xyz[3 * i + d];
      if (!isfinite(v)) {
        atomicOr(&ms[MS_ERR], (unsigned long long)MSE_COORD);
        atomicMin(&ms[MS_BAD_X], (unsigned long long)i);
        continue;
      }
      const unsigned long long b = ordered_bits(v);
      lo[d] = min(lo[d], b);
      hi[d] = max(hi[d], b);
    }
  }
  for (int d = 0; d < 3; ++d) {
    unsigned long long a = lo[d], b = hi[d];
    for (int o = 16; o > 0; o >>= 1) {
      a = min(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&ms[MS_LO + d], a);
      atomicMax(&ms[MS_HI + d], b);
    }
  }
}

__global__ void k_fill_value(int64_t n, double v, double *a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

static vem_status create_impl(vem_handle *h, const vem_mesh *m) {
  if (!m || !m->xyz || !m->face_vtx_ptr || !m->face_vtx || !m->cell_face_ptr || !m->cell_face || !m->face_bc)
    return fail(h, VEM_ERR_BAD_INPUT, "mesh: NULL array");
  if (m->n_vertices < 4 || m->n_faces < 4 || m->n_cells < 1)
    return fail(h, VEM_ERR_BAD_INPUT, "mesh: too few vertices/faces/cells");
  if (m->n_faces > INT32_MAX / 4 || m->n_cells > INT32_MAX / 4 || m->n_vertices > INT32_MAX)
    return fail(h, VEM_ERR_UNSUPPORTED, "mesh too large for 32-bit indices");
  h->nv = m->n_vertices;
  h->nf = m->n_faces;
  h->nc = m->n_cells;
  if (m->face_vtx_ptr[0] != 0 || m->cell_face_ptr[0] != 0)
    return fail(h, VEM_ERR_BAD_INPUT, "mesh: pointers must start at 0");
  h->n_fv = m->face_vtx_ptr[h->nf];
  h->n_cf = m->cell_face_ptr[h->nc];
  if (h->n_fv < 3 * h->nf || h->n_fv > 4096 * h->nf || h->n_cf < 4 * h->nc || h->n_cf > 256 * h->nc)
    return fail(h, VEM_ERR_BAD_INPUT, "mesh: face_vtx_ptr / cell_face_ptr totals out of range");
  set_layout(h);

  VEM_CUDA(h, pinned_alloc(reinterpret_cast<void **>(&h->h_err), 64));
  VEM_CUDA(h, pinned_alloc(reinterpret_cast<void **>(&h->h_scal), 8192 * sizeof(double)));
  VEM_TRY(upload(h, &h->xyz, m->xyz, 3 * (size_t)h->nv));
  VEM_TRY(upload(h, &h->fv_ptr, m->face_vtx_ptr, (size_t)h->nf + 1));
  VEM_TRY(upload(h, &h->fv, m->face_vtx, (size_t)h->n_fv));
  VEM_TRY(upload(h, &h->cf_ptr, m->cell_face_ptr, (size_t)h->nc + 1));
  VEM_TRY(upload(h, &h->cf, m->cell_face, (size_t)h->n_cf));
  VEM_TRY(upload(h, &h->fbc, m->face_bc, (size_t)h->nf));
  // checks and summaries of the mesh, one read-back
  {
    cudaStream_t s = h->stream;
    unsigned long long *ms = nullptr;
    VEM_TRY(dalloc_n(h, &ms, (size_t)MS_COUNT));
    unsigned long long init[MS_COUNT];
    for (int i = 0; i < MS_COUNT; ++i) init[i] = 0;
    for (int i = MS_BAD_FACE; i <= MS_BAD_X; ++i) init[i] = ~0ull;
    for (int d = 0; d < 3; ++d) init[MS_LO + d] = ~0ull;
    VEM_CUDA(h, cudaMemcpyAsync(ms, init, sizeof(init), cudaMemcpyHostToDevice, s));
    int64_t *bq_cnt = nullptr;
    VEM_TRY(dalloc_n(h, &bq_cnt, (size_t)h->nf + 1));
    // the boundary-data rule: Radon's 7 points per fan triangle at k = 2, Dunavant's 6 otherwise
    h->bq_ppt = h->opt.element == VEM_ELEMENT_K2 ? 7 : 6;
    count_launch(); k_check_faces<<<grid_for(h->nf, 256), 256, 0, s>>>(h->nf, h->fv_ptr, h->fbc, ms, bq_cnt,
                                                                       h->bq_ppt);
    count_launch(); k_check_cells<<<grid_for(h->nc, 256), 256, 0, s>>>(h->nc, h->cf_ptr, ms);
    count_launch(); k_check_ids<<<grid_for(h->n_fv, 256), 256, 0, s>>>(h->n_fv, h->fv, h->nv, MSE_VTX, MS_BAD_FV, ms);
    count_launch(); k_check_ids<<<grid_for(h->n_cf, 256), 256, 0, s>>>(h->n_cf, h->cf, h->nf, MSE_FACE, MS_BAD_CF, ms);
    count_launch(); k_check_coords<<<grid_for(h->nv, 256), 256, 0, s>>>(h->nv, h->xyz, ms);
    VEM_CUDA(h, cudaGetLastError());
    unsigned long long r[MS_COUNT];
    VEM_CUDA(h, cudaMemcpyAsync(r, ms, sizeof(r), cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    dfree(h, ms);
    const unsigned long long e = r[MS_ERR];
    if (e & MSE_FACE_NV) return fail(h, VEM_ERR_BAD_INPUT, "mesh: face %llu needs 3..4096 vertices", r[MS_BAD_FACE]);
    if (e & MSE_FLAG) return fail(h, VEM_ERR_BAD_INPUT, "mesh: face %llu has a flag outside 0..2", r[MS_BAD_FACE]);
    if (e & MSE_CELL_NF) return fail(h, VEM_ERR_BAD_INPUT, "mesh: cell %llu needs 4..256 faces", r[MS_BAD_CELL]);
    if (e & MSE_VTX) return fail(h, VEM_ERR_BAD_INPUT, "mesh: vertex index out of range (face_vtx[%llu])", r[MS_BAD_FV]);
    if (e & MSE_FACE) return fail(h, VEM_ERR_BAD_INPUT, "mesh: face index out of range (cell_face[%llu])", r[MS_BAD_CF]);
    if (e & MSE_COORD) return fail(h, VEM_ERR_NONFINITE, "mesh: non-finite coordinate (vertex %llu)", r[MS_BAD_X]);
    h->max_nv_face = (int)r[MS_MAXNV];
    h->max_nf_cell = (int)r[MS_MAXNF];
    h->n_flux_faces = (int64_t)r[MS_NFLUX];
    h->n_dir_faces = (int64_t)r[MS_NDIR];
    double ext2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double w = from_ordered(r[MS_HI + d]) - from_ordered(r[MS_LO + d]);
      ext2 += w * w;
    }
    h->lref = std::sqrt(ext2);
    if (!(h->lref > 0.0)) return fail(h, VEM_ERR_DEGENERATE_MESH, "mesh: zero extent");
    // boundary-face quadrature offsets from the per-face counts
    VEM_TRY(dalloc_n(h, &h->bqp_off, (size_t)h->nf + 1));
    VEM_TRY(scan_counts(h, h->nf, bq_cnt, h->bqp_off, &h->n_bqp));
    // the boundary faces in increasing order, so that the boundary-load
    // kernels give a thread to every boundary face instead of scanning all
    // faces (about 1 in 64 of a 128^3 cube's faces is on the boundary)
    count_launch(); k_flag_positive<<<grid_for(h->nf, 256), 256, 0, s>>>(h->nf, bq_cnt);
    int64_t *bpos = nullptr;
    VEM_TRY(dalloc_n(h, &bpos, (size_t)h->nf + 1));
    VEM_TRY(scan_counts(h, h->nf, bq_cnt, bpos, &h->n_bface));
    VEM_TRY(dalloc_n(h, &h->bface, (size_t)std::max<int64_t>(h->n_bface, 1)));
    count_launch(); k_compact_ids<<<grid_for(h->nf, 256), 256, 0, s>>>(h->nf, bq_cnt, bpos, h->bface);
    VEM_CUDA(h, cudaGetLastError());
    dfree(h, bpos);
    dfree(h, bq_cnt);
  }
  h->multiplier = h->n_flux_faces > 0 && h->n_dir_faces == 0;
  VEM_TRY(dalloc_n(h, &h->f_area, h->nf));
  VEM_TRY(dalloc_n(h, &h->f_cent, 3 * h->nf));
  VEM_TRY(dalloc_n(h, &h->f_norm, 3 * h->nf));
  VEM_TRY(dalloc_n(h, &h->f_t1, 3 * h->nf));
  VEM_TRY(dalloc_n(h, &h->f_diam, h->nf));
  VEM_TRY(dalloc_n(h, &h->f_cell, 2 * h->nf));
  VEM_TRY(dalloc_n(h, &h->f_loc, 2 * h->nf));
  VEM_TRY(dalloc_n(h, &h->c_vol, h->nc));
  VEM_TRY(dalloc_n(h, &h->c_cent, 3 * h->nc));
  VEM_TRY(dalloc_n(h, &h->c_diam, h->nc));
  VEM_TRY(dalloc_n(h, &h->cf_sigma, h->n_cf));
  VEM_TRY(dalloc_n(h, &h->d_err, 1));
  VEM_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  VEM_TRY(dalloc_n(h, &h->part, (size_t)kMaxSlots * kMaxBlocks));
  VEM_TRY(dalloc_n(h, &h->scal, 8192));
  VEM_TRY(dalloc_n(h, &h->ctr, 64));
  VEM_CUDA(h, cudaMemsetAsync(h->ctr, 0, 64 * sizeof(unsigned int), h->stream));
  VEM_CUDA(h, cudaMemsetAsync(h->scal, 0, 8192 * sizeof(double), h->stream));
  VEM_TRY(dalloc_n(h, &h->bqp_xyz, 3 * (size_t)std::max<int64_t>(h->n_bqp, 1)));
  // coefficient nu = 1/K, default K = 1
  VEM_TRY(dalloc_n(h, &h->nu, h->nc));
  count_launch(); k_fill_value<<<grid_for(h->nc, 256), 256, 0, h->stream>>>(h->nc, 1.0, h->nu);
  VEM_CUDA(h, cudaGetLastError());
  h->have_coef = true;
  VEM_TRY(dalloc_n(h, &h->f_qp, h->nc));
  VEM_TRY(dalloc_n(h, &h->gD_qp, std::max<int64_t>(h->n_bqp, 1)));
  VEM_CUDA(h, cudaMemsetAsync(h->f_qp, 0, sizeof(double) * h->nc, h->stream));
  VEM_CUDA(h, cudaMemsetAsync(h->gD_qp, 0, sizeof(double) * std::max<int64_t>(h->n_bqp, 1), h->stream));
  VEM_CUDA(h, cudaEventCreate(&h->ev0));
  VEM_CUDA(h, cudaEventCreate(&h->ev1));
  VEM_CUDA(h, cudaEventCreate(&h->ev2));
  VEM_CUDA(h, cudaEventCreate(&h->ev3));
  for (auto &e : h->tev) VEM_CUDA(h, cudaEventCreate(&e));
  for (auto &e : h->aev) VEM_CUDA(h, cudaEventCreate(&e));
  VEM_TRY(geometry_build(h));
  return classify_cells(h);   // congruence classes: a property of the mesh
}

static vem_status ensure_rhs(vem_handle *h) {
  if (!h->rhs) VEM_TRY(dalloc_n(h, &h->rhs, (size_t)h->n));
  if (!h->rhs_ready) VEM_TRY(assemble_rhs(h));
  return VEM_OK;
}

static vem_status assemble_impl(vem_handle *h) {
  amg_invalidate(h->amg);
  amg_invalidate(h->amg_reg);
  h->areg_valid = false;
  VEM_CUDA(h, cudaEventRecord(h->ev0, h->stream));
  VEM_TRY(classify_cells(h));
  VEM_CUDA(h, cudaEventRecord(h->ev2, h->stream));
  VEM_TRY(assemble_local(h));
  VEM_CUDA(h, cudaEventRecord(h->ev3, h->stream));
  VEM_TRY(assemble_global(h));
  h->rhs_ready = false;
  VEM_TRY(ensure_rhs(h));
  VEM_CUDA(h, cudaEventRecord(h->ev1, h->stream));
  VEM_CUDA(h, cudaEventSynchronize(h->ev1));
  float ms = 0.f, me = 0.f, mg = 0.f;
  VEM_CUDA(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
  VEM_CUDA(h, cudaEventElapsedTime(&me, h->ev2, h->ev3));
  VEM_CUDA(h, cudaEventElapsedTime(&mg, h->ev3, h->ev1));
  h->t_assemble_ms = ms;
  h->t_element_ms = me;
  h->t_scatter_ms = mg;
  h->assembled = true;
  return VEM_OK;
}

// nu = 1/K (K may alias nu); non-finite K raise DEVERR_NONFINITE, K <= 0
// DEVERR_NONPOSITIVE.
__global__ void k_invert_check(int64_t n, const double *K, double *nu, int *err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double k = K[i];
    if (!isfinite(k)) atomicOr(err, DEVERR_NONFINITE);
    else if (!(k > 0.0)) atomicOr(err, DEVERR_NONPOSITIVE);
    nu[i] = 1.0 / k;
  }
}

// nu = exp(-theta) = 1/K from theta = log K; a theta whose K or nu is not a
// finite positive double raises DEVERR_NONFINITE.
__global__ void k_nu_from_log(int64_t n, const double *theta, double *nu, int *err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = exp(-theta[i]);
    if (!isfinite(theta[i]) || !isfinite(v) || !(v > 0.0)) atomicOr(err, DEVERR_NONFINITE);
    nu[i] = v;
  }
}

// Non-finite entries of a vector raise DEVERR_NONFINITE.
__global__ void k_check_finite(int64_t n, const double *__restrict__ a, int *err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(a[i])) atomicOr(err, DEVERR_NONFINITE);
}

__global__ void k_export_x(int64_t nu, int64_t np, const double *x, double *u, double *p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nu + np;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < nu) {
      if (u) u[i] = x[i];
    } else if (p) {
      p[i - nu] = -x[i];
    }
  }
}

__global__ void k_import_x(int64_t nu, int64_t n, const double *x0, double *x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = x0 ? (i < nu ? x0[i] : -x0[i]) : 0.0;
}

// Euclidean norm of each stacked system's entries (one block per system).
__global__ void k_segment_norms(int nb, int64_t nu1, int64_t np1, const double *__restrict__ v, double *out) {
  const int64_t b = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < nu1; i += blockDim.x) {
    const double t = v[b * nu1 + i];
    s += t * t;
  }
  for (int64_t i = threadIdx.x; i < np1; i += blockDim.x) {
    const double t = v[(int64_t)nb * nu1 + b * np1 + i];
    s += t * t;
  }
  block_partial(s, out);
  if (threadIdx.x == 0) out[blockIdx.x] = sqrt(out[blockIdx.x]);
}

__global__ void k_sub(int64_t n, const double *__restrict__ a, const double *__restrict__ b, double *c) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c[i] = a[i] - b[i];
}

template <class T>
static vem_status batch_buf(vem_handle *h, T **p, size_t n, bool grow) {
  if (grow || !*p) {
    dfree(h, *p);
    *p = nullptr;
    VEM_TRY(dalloc_n(h, p, n));
  }
  return VEM_OK;
}

}  // namespace vem

using namespace vem;

extern "C" {

vem_status vem_default_options(vem_options *o) {
  if (!o) return VEM_ERR_BAD_INPUT;
  std::memset(o, 0, sizeof(*o));
  o->element = VEM_ELEMENT_E0;
  o->krylov = VEM_KRYLOV_FGMRES;
  o->restart = 30;
  o->rtol = 1e-12;
  o->maxit = 2000;
  o->precond = VEM_PREC_BLOCK_DIAG;
  o->inner = VEM_INNER_PCG;
  o->inner_rtol = 1e-12;
  o->inner_maxit = 2000;
  o->precision = VEM_PRECISION_FP64;
  o->device_io = 0;
  o->reuse = 1;
  return VEM_OK;
}

vem_status vem_create(const vem_mesh *mesh, const vem_options *opt, void *stream, vem_handle **out) {
  if (!out) return VEM_ERR_BAD_INPUT;
  *out = nullptr;
  vem_handle *h = new (std::nothrow) vem_handle();
  if (!h) return VEM_ERR_OOM;
  if (opt) {
    h->opt = *opt;
  } else {
    vem_default_options(&h->opt);
  }
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  vem_status st = check_options(h, &h->opt);
  if (st == VEM_OK) st = create_impl(h, mesh);
  if (st != VEM_OK) {
    vem_destroy(h);
    return st;
  }
  *out = h;
  return VEM_OK;
}

vem_status vem_set_options(vem_handle *h, const vem_options *opt) {
  if (!h || !opt) return VEM_ERR_BAD_INPUT;
  VEM_TRY(check_options(h, opt));
  const bool elem_changed = opt->element != h->opt.element;
  if (elem_changed || opt->reg_gamma != h->opt.reg_gamma) h->areg_valid = false;
  h->opt = *opt;
  if (elem_changed) {
    set_layout(h);
    const int ppt = opt->element == VEM_ELEMENT_K2 ? 7 : 6;
    if (ppt != h->bq_ppt) VEM_TRY(rebuild_bface_points(h, ppt));
    h->assembled = false;
    h->local_ready = false;
    h->rhs_ready = false;
    h->have_solution = false;
    dfree(h, h->rhs);
    h->rhs = nullptr;
    dfree(h, h->lam);
    h->lam = nullptr;
    dfree(h, h->arhs);
    h->arhs = nullptr;
    dfree(h, h->diagM);
    h->diagM = nullptr;
    dfree(h, h->dinvM);
    h->dinvM = nullptr;
    dfree(h, h->xsol);
    h->xsol = nullptr;
    dfree(h, h->cnt_buf);
    h->cnt_buf = nullptr;
  }
  return VEM_OK;
}

vem_status vem_sizes(const vem_handle *h, int64_t *n_u, int64_t *n_p) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (n_u) *n_u = h->n_u;
  if (n_p) *n_p = h->n_p;
  return VEM_OK;
}

// cell points: one per cell (its barycentre) for E0 / K1, the fan-tetrahedron
// rule of the k = 2 loads otherwise
static int64_t n_cell_points(const vem_handle *h) { return h->nq > 1 ? h->n_cqp : h->nc; }

static vem_status ensure_cell_points(vem_handle *h) {
  if (h->nq == 1) return VEM_OK;
  const bool had = h->cqp_valid;
  VEM_TRY(cell_points_k2(h));
  if (!had) {
    // the source buffer holds one value per cell point
    dfree(h, h->f_qp);
    h->f_qp = nullptr;
    VEM_TRY(dalloc_n(h, &h->f_qp, (size_t)std::max<int64_t>(h->n_cqp, 1)));
    VEM_CUDA(h, cudaMemsetAsync(h->f_qp, 0, sizeof(double) * std::max<int64_t>(h->n_cqp, 1), h->stream));
    h->rhs_ready = false;
  }
  return VEM_OK;
}

vem_status vem_quadrature_count(const vem_handle *hc, int which, int64_t *n) {
  if (!hc || !n) return VEM_ERR_BAD_INPUT;
  vem_handle *h = const_cast<vem_handle *>(hc);   // the k = 2 points are built on first use
  if (which == VEM_QP_CELL) {
    VEM_TRY(ensure_cell_points(h));
    *n = n_cell_points(h);
  } else if (which == VEM_QP_BFACE) *n = h->n_bqp;
  else return VEM_ERR_BAD_INPUT;
  return VEM_OK;
}
vem_status vem_quadrature_points(vem_handle *h, int which, double *xyz_out) {
  if (!h || !xyz_out) return h ? fail(h, VEM_ERR_BAD_INPUT, "NULL output") : VEM_ERR_BAD_INPUT;
  const double *src = nullptr;
  int64_t n = 0;
  if (which == VEM_QP_CELL) {
    VEM_TRY(ensure_cell_points(h));
    src = h->nq > 1 ? h->cqp_x : h->c_cent;
    n = n_cell_points(h);
  } else if (which == VEM_QP_BFACE) {
    src = h->bqp_xyz;
    n = h->n_bqp;
  } else {
    return fail(h, VEM_ERR_BAD_INPUT, "unknown quadrature set %d", which);
  }
  if (n > 0)
    VEM_CUDA(h, cudaMemcpyAsync(xyz_out, src, 3 * n * sizeof(double), cudaMemcpyDefault, h->stream));
  VEM_CUDA(h, cudaStreamSynchronize(h->stream));
  return VEM_OK;
}

// K (device) -> nu = 1/K with the checks on the device; on a bad K the old
// nu is kept (the new values go to a scratch first).
static vem_status set_nu_from_device(vem_handle *h, const double *K, bool log_k = false) {
  double *tmp = nullptr;
  VEM_TRY(dalloc_n(h, &tmp, (size_t)h->nc));
  count_launch();
  if (log_k) k_nu_from_log<<<grid_for(h->nc, 256), 256, 0, h->stream>>>(h->nc, K, tmp, h->d_err);
  else k_invert_check<<<grid_for(h->nc, 256), 256, 0, h->stream>>>(h->nc, K, tmp, h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  VEM_CUDA(h, cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  VEM_CUDA(h, cudaStreamSynchronize(h->stream));
  const int e = *h->h_err;
  if (e & (DEVERR_NONFINITE | DEVERR_NONPOSITIVE)) {
    VEM_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
    dfree(h, tmp);
    if (e & DEVERR_NONFINITE) return fail(h, VEM_ERR_NONFINITE, "K is not finite");
    return fail(h, VEM_ERR_BAD_INPUT, "K <= 0");
  }
  VEM_CUDA(h, cudaMemcpyAsync(h->nu, tmp, sizeof(double) * h->nc, cudaMemcpyDeviceToDevice, h->stream));
  dfree(h, tmp);
  h->assembled = false;
  h->have_solution = false;
  return check_device_errors(h, "coefficient");
}

vem_status vem_set_coefficient(vem_handle *h, const double *K) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (!K) return fail(h, VEM_ERR_BAD_INPUT, "K: NULL");
  double *Kd = nullptr;
  VEM_TRY(dalloc_n(h, &Kd, (size_t)h->nc));
  vem_status st = cuda_check(h, cudaMemcpyAsync(Kd, K, sizeof(double) * h->nc, cudaMemcpyHostToDevice, h->stream),
                             "K upload");
  if (st == VEM_OK) st = set_nu_from_device(h, Kd);
  dfree(h, Kd);
  return st;
}

vem_status vem_set_coefficient_device(vem_handle *h, const double *K) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (!K) return fail(h, VEM_ERR_BAD_INPUT, "K: NULL");
  return set_nu_from_device(h, K);
}

vem_status vem_set_log_coefficient_device(vem_handle *h, const double *logK) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (!logK) return fail(h, VEM_ERR_BAD_INPUT, "log K: NULL");
  return set_nu_from_device(h, logK, true);
}

vem_status vem_set_source(vem_handle *h, const double *f_qp, const double *gD_qp) {
  if (!h) return VEM_ERR_BAD_INPUT;
  cudaStream_t s = h->stream;
  // the new data go to scratch buffers and are checked on the device; the
  // handle's data change only when they are finite
  double *fs = nullptr, *gs = nullptr;
  VEM_TRY(ensure_cell_points(h));
  const int64_t ncp = n_cell_points(h);
  if (f_qp) {
    VEM_TRY(dalloc_n(h, &fs, (size_t)ncp));
    VEM_CUDA(h, cudaMemcpyAsync(fs, f_qp, sizeof(double) * ncp, cudaMemcpyHostToDevice, s));
    count_launch(); k_check_finite<<<grid_for(ncp, 256), 256, 0, s>>>(ncp, fs, h->d_err);
  }
  if (h->n_bqp > 0 && gD_qp) {
    VEM_TRY(dalloc_n(h, &gs, (size_t)h->n_bqp));
    VEM_CUDA(h, cudaMemcpyAsync(gs, gD_qp, sizeof(double) * h->n_bqp, cudaMemcpyHostToDevice, s));
    count_launch(); k_check_finite<<<grid_for(h->n_bqp, 256), 256, 0, s>>>(h->n_bqp, gs, h->d_err);
  }
  VEM_CUDA(h, cudaGetLastError());
  VEM_CUDA(h, cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaStreamSynchronize(s));
  if (*h->h_err & DEVERR_NONFINITE) {
    VEM_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
    dfree(h, fs);
    dfree(h, gs);
    return fail(h, VEM_ERR_NONFINITE, "f or g_D is not finite at a quadrature point");
  }
  if (fs) VEM_CUDA(h, cudaMemcpyAsync(h->f_qp, fs, sizeof(double) * ncp, cudaMemcpyDeviceToDevice, s));
  else VEM_CUDA(h, cudaMemsetAsync(h->f_qp, 0, sizeof(double) * ncp, s));
  if (h->n_bqp > 0) {
    if (gs) VEM_CUDA(h, cudaMemcpyAsync(h->gD_qp, gs, sizeof(double) * h->n_bqp, cudaMemcpyDeviceToDevice, s));
    else VEM_CUDA(h, cudaMemsetAsync(h->gD_qp, 0, sizeof(double) * h->n_bqp, s));
  }
  dfree(h, fs);
  dfree(h, gs);
  h->rhs_ready = false;
  if (h->n_flux_faces > 0) h->assembled = false;   // the flux data is eliminated at assembly
  return VEM_OK;
}

vem_status vem_set_source_device(vem_handle *h, const double *f_qp, const double *gD_qp) {
  if (!h) return VEM_ERR_BAD_INPUT;
  VEM_TRY(ensure_cell_points(h));
  const int64_t ncp = n_cell_points(h);
  if (f_qp)
    VEM_CUDA(h, cudaMemcpyAsync(h->f_qp, f_qp, sizeof(double) * ncp, cudaMemcpyDeviceToDevice, h->stream));
  else
    VEM_CUDA(h, cudaMemsetAsync(h->f_qp, 0, sizeof(double) * ncp, h->stream));
  if (h->n_bqp > 0) {
    if (gD_qp)
      VEM_CUDA(h, cudaMemcpyAsync(h->gD_qp, gD_qp, sizeof(double) * h->n_bqp, cudaMemcpyDeviceToDevice, h->stream));
    else
      VEM_CUDA(h, cudaMemsetAsync(h->gD_qp, 0, sizeof(double) * h->n_bqp, h->stream));
  }
  h->rhs_ready = false;
  if (h->n_flux_faces > 0) h->assembled = false;   // the flux data is eliminated at assembly
  return VEM_OK;
}

vem_status vem_assemble(vem_handle *h) {
  if (!h) return VEM_ERR_BAD_INPUT;
  return assemble_impl(h);
}

vem_status vem_assemble_local(vem_handle *h) {
  if (!h) return VEM_ERR_BAD_INPUT;
  VEM_CUDA(h, cudaEventRecord(h->ev2, h->stream));
  VEM_TRY(classify_cells(h));
  VEM_TRY(assemble_local(h));
  VEM_CUDA(h, cudaEventRecord(h->ev3, h->stream));
  VEM_CUDA(h, cudaEventSynchronize(h->ev3));
  float me = 0.f;
  VEM_CUDA(h, cudaEventElapsedTime(&me, h->ev2, h->ev3));
  h->t_element_ms = me;
  h->local_ready = true;
  return VEM_OK;
}

vem_status vem_local_time(const vem_handle *h, double *element_ms, int64_t *n_classes) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (element_ms) *element_ms = h->t_element_ms;
  if (n_classes) *n_classes = h->ncls;
  return VEM_OK;
}

vem_status vem_solve(vem_handle *h, const double *x0, double *u_out, double *p_out, vem_stats *stats) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (!u_out || !p_out) return fail(h, VEM_ERR_BAD_INPUT, "u_out / p_out: NULL");
  if (!h->assembled) VEM_TRY(assemble_impl(h));
  VEM_TRY(ensure_rhs(h));
  cudaStream_t s = h->stream;
  if (!h->xsol) VEM_TRY(dalloc_n(h, &h->xsol, (size_t)h->n));
  double *x = h->xsol;
  vem_stats st{};
  st.n_u = h->n_u;
  st.n_p = h->n_p;
  st.nnz_A = h->A.nnz;
  st.nnz_S = h->S.nnz;
  st.t_assemble_ms = h->t_assemble_ms;
  st.t_element_ms = h->t_element_ms;
  st.t_scatter_ms = h->t_scatter_ms;
  st.n_classes = h->ncls;
  vem_status r = VEM_OK;
  do {
    const double *x0d = nullptr;
    double *tmp = nullptr;
    if (x0 && !h->opt.device_io) {
      r = dalloc_n(h, &tmp, (size_t)h->n);
      if (r != VEM_OK) break;
      cudaError_t e = cudaMemcpyAsync(tmp, x0, sizeof(double) * h->n, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) { r = cuda_check(h, e, "x0"); break; }
      x0d = tmp;
    } else if (x0) {
      x0d = x0;
    }
    count_launch(); k_import_x<<<grid_for(h->n, 256), 256, 0, s>>>(h->n_u, h->n, x0d, x);
    h->x_zero = x0d == nullptr;
    h->t_schur_spmv_ms = 0.0;
    h->n_schur_spmv = 0;
    h->t_vc_resid_ms = h->t_vc_post_ms = 0.0;
    h->n_vc_resid = h->n_vc_post = 0;
    h->t_saddle_spmv_ms = 0.0;
    h->n_saddle_spmv = 0;
    const bool had_amg = amg_valid(h->amg), had_reg = amg_valid(h->amg_reg);
    cudaEventRecord(h->ev0, s);
    r = krylov_solve(h, single_op(h), h->rhs, x, &st);
    cudaEventRecord(h->ev1, s);
    cudaEventSynchronize(h->ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    st.t_solve_ms = ms;
    st.t_schur_spmv_ms = h->t_schur_spmv_ms;
    st.n_schur_spmv = h->n_schur_spmv;
    const bool reg = h->opt.precond == VEM_PREC_BLOCK_REG;
    st.t_amg_setup_ms = ((!had_amg && amg_valid(h->amg)) ? amg_setup_ms(h->amg) : 0.0) +
                        ((!had_reg && amg_valid(h->amg_reg)) ? amg_setup_ms(h->amg_reg) : 0.0);
    st.amg_levels = reg ? amg_levels(h->amg_reg) : amg_levels(h->amg);
    st.reg_gamma = reg ? h->reg_gamma : 0.0;
    st.nnz_reg = reg && h->areg_valid ? h->Areg.nnz : 0;
    st.t_saddle_spmv_ms = h->t_saddle_spmv_ms;
    st.n_saddle_spmv = h->n_saddle_spmv;
    st.t_vc_resid_ms = h->t_vc_resid_ms;
    st.n_vc_resid = h->n_vc_resid;
    st.t_vc_post_ms = h->t_vc_post_ms;
    st.n_vc_post = h->n_vc_post;
    if (tmp) dfree(h, tmp);
    if (r != VEM_OK && r != VEM_ERR_NOT_CONVERGED) break;
    {
      const vem_status sh = neumann_shift(h, x + h->n_u);   // mean-zero pressure
      if (sh != VEM_OK) { r = sh; break; }
    }
    st.multiplier = h->lambda;
    h->have_solution = true;
    vem_status w = VEM_OK;
    if (h->opt.device_io) {
      count_launch(); k_export_x<<<grid_for(h->n, 256), 256, 0, s>>>(h->n_u, h->n_p, x, u_out, p_out);
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) w = cuda_check(h, e, "export");
    } else {
      cudaError_t e = cudaMemcpyAsync(u_out, x, sizeof(double) * h->n_u, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(p_out, x + h->n_u, sizeof(double) * h->n_p, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) w = cuda_check(h, e, "export");
      else
        for (int64_t i = 0; i < h->n_p; ++i) p_out[i] = -p_out[i];
    }
    if (w != VEM_OK) r = w;
  } while (0);
  if (stats) *stats = st;
  return r;
}

__global__ void k_adjoint_rhs(int64_t nu, int64_t n, const double *gu, const double *gp, double *r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = i < nu ? (gu ? gu[i] : 0.0) : (gp ? -gp[i - nu] : 0.0);
}

vem_status vem_adjoint(vem_handle *h, const double *dL_du, const double *dL_dp, double *dL_dlogK,
                       vem_stats *stats) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (!dL_dlogK) return fail(h, VEM_ERR_BAD_INPUT, "dL_dlogK: NULL");
  if (!h->have_solution || !h->assembled)
    return fail(h, VEM_ERR_BAD_INPUT, "vem_adjoint needs a preceding vem_solve with the same K");
  if (h->n_flux_faces > 0) return fail(h, VEM_ERR_UNSUPPORTED, "adjoint with prescribed-flux faces");
  cudaStream_t s = h->stream;
  if (!h->lam) VEM_TRY(dalloc_n(h, &h->lam, (size_t)h->n));
  if (!h->arhs) VEM_TRY(dalloc_n(h, &h->arhs, (size_t)h->n));
  if (!h->grad) VEM_TRY(dalloc_n(h, &h->grad, (size_t)h->nc));
  const double *gu = dL_du, *gp = dL_dp;
  double *tmp = nullptr;
  if (!h->opt.device_io && (dL_du || dL_dp)) {
    VEM_TRY(dalloc_n(h, &tmp, (size_t)h->n));
    if (dL_du) VEM_CUDA(h, cudaMemcpyAsync(tmp, dL_du, sizeof(double) * h->n_u, cudaMemcpyHostToDevice, s));
    if (dL_dp) VEM_CUDA(h, cudaMemcpyAsync(tmp + h->n_u, dL_dp, sizeof(double) * h->n_p, cudaMemcpyHostToDevice, s));
    gu = dL_du ? tmp : nullptr;
    gp = dL_dp ? tmp + h->n_u : nullptr;
  }
  count_launch();
  k_adjoint_rhs<<<grid_for(h->n, 256), 256, 0, s>>>(h->n_u, h->n, gu, gp, h->arhs);
  VEM_CUDA(h, cudaGetLastError());
  count_launch();
  k_import_x<<<grid_for(h->n, 256), 256, 0, s>>>(h->n_u, h->n, nullptr, h->lam);
  vem_stats st{};
  st.n_u = h->n_u;
  st.n_p = h->n_p;
  st.nnz_A = h->A.nnz;
  st.nnz_S = h->S.nnz;
  cudaEventRecord(h->ev0, s);
  vem_status r = krylov_solve(h, single_op(h), h->arhs, h->lam, &st);
  cudaEventRecord(h->ev1, s);
  cudaEventSynchronize(h->ev1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  st.t_solve_ms = ms;
  if (tmp) dfree(h, tmp);
  if (stats) *stats = st;
  if (r != VEM_OK) return r;
  VEM_TRY(adjoint_contract(h, h->lam, h->xsol, h->grad));
  if (h->opt.device_io) {
    VEM_CUDA(h, cudaMemcpyAsync(dL_dlogK, h->grad, sizeof(double) * h->nc, cudaMemcpyDeviceToDevice, s));
  } else {
    VEM_CUDA(h, cudaMemcpyAsync(dL_dlogK, h->grad, sizeof(double) * h->nc, cudaMemcpyDeviceToHost, s));
  }
  VEM_CUDA(h, cudaStreamSynchronize(s));
  return VEM_OK;
}

vem_status vem_solve_batched(vem_handle *h, int64_t nbatch, const double *K, const double *f_qp,
                             const double *gD_qp, double *u_out, double *p_out, double *relres_out,
                             vem_stats *stats) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (nbatch < 1 || nbatch > 65535) return fail(h, VEM_ERR_BAD_INPUT, "nbatch %lld", (long long)nbatch);
  if (!K || !u_out || !p_out) return fail(h, VEM_ERR_BAD_INPUT, "K / u_out / p_out: NULL");
  if (h->opt.inner != VEM_INNER_PCG)
    return fail(h, VEM_ERR_UNSUPPORTED, "the AMG inner solvers are single-system (no batched solves)");
  if (h->opt.precond == VEM_PREC_BLOCK_REG)
    return fail(h, VEM_ERR_UNSUPPORTED, "Block-Reg is single-system (no batched solves)");
  if (h->n_flux_faces > 0)
    return fail(h, VEM_ERR_UNSUPPORTED, "prescribed-flux faces in batched solves");
  cudaStream_t s = h->stream;
  const int nb = (int)nbatch;
  const bool dev = h->opt.device_io != 0;
  // structure of A and S from a single-system assembly
  if (!h->assembled) VEM_TRY(assemble_impl(h));
  VEM_TRY(ensure_cell_points(h));
  const int64_t ncp = n_cell_points(h);   // f_qp entries per system (n_cells below k = 2)
  const bool grow = nb > h->b_cap || ncp != h->b_ncp;
  const int64_t nbq = std::max<int64_t>(h->n_bqp, 1);
  VEM_TRY(batch_buf(h, &h->b_nu, (size_t)nb * h->nc, grow));
  VEM_TRY(batch_buf(h, &h->b_fqp, (size_t)nb * std::max(ncp, h->nc), grow));
  VEM_TRY(batch_buf(h, &h->b_gqp, (size_t)nb * nbq, grow));
  VEM_TRY(batch_buf(h, &h->b_rhs, (size_t)nb * h->n, grow));
  VEM_TRY(batch_buf(h, &h->b_x, (size_t)nb * h->n, grow));
  VemOp &op = h->bop;
  const bool regrow = grow || op.A.stored != h->A.stored || op.S.stored != h->S.stored || op.n_u1 != h->n_u;
  VEM_TRY(batch_buf(h, &op.A.val, (size_t)nb * h->A.stored, regrow));
  VEM_TRY(batch_buf(h, &op.diagM, (size_t)nb * h->n_u, regrow));
  VEM_TRY(batch_buf(h, &op.dinvM, (size_t)nb * h->n_u, regrow));
  VEM_TRY(batch_buf(h, &op.S.val, (size_t)nb * h->S.stored, regrow));
  VEM_TRY(batch_buf(h, &op.s_dinv, (size_t)nb * h->n_p, regrow));
  VEM_TRY(batch_buf(h, &op.S_val32, (size_t)nb * h->S.stored, regrow));
  VEM_TRY(batch_buf(h, &op.s_dinv32, (size_t)nb * h->n_p, regrow));
  if (grow) {
    h->b_cap = nb;
    h->b_ncp = ncp;
  }
  op.A.rows = h->A.rows; op.A.nslices = h->A.nslices; op.A.stored = h->A.stored; op.A.nnz = h->A.nnz;
  op.A.off = h->A.off; op.A.len = h->A.len; op.A.col = h->A.col;
  op.S.rows = h->S.rows; op.S.nslices = h->S.nslices; op.S.stored = h->S.stored; op.S.nnz = h->S.nnz;
  op.S.off = h->S.off; op.S.len = h->S.len; op.S.col = h->S.col;
  op.n_u1 = h->n_u;
  op.n_p1 = h->n_p;
  op.n_u = (int64_t)nb * h->n_u;
  op.n_p = (int64_t)nb * h->n_p;
  op.n = op.n_u + op.n_p;
  op.nbatch = nb;
  // inputs
  const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  VEM_CUDA(h, cudaMemcpyAsync(h->b_fqp, K, sizeof(double) * nb * h->nc, kind, s));   // staging
  count_launch();
  k_invert_check<<<grid_for((int64_t)nb * h->nc, 256), 256, 0, s>>>((int64_t)nb * h->nc, h->b_fqp, h->b_nu, h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  {
    vem_status e = check_device_errors(h, "batched coefficient");
    if (e == VEM_ERR_NONFINITE) return fail(h, VEM_ERR_BAD_INPUT, "K must be finite and > 0");
    if (e != VEM_OK) return e;
  }
  if (f_qp) VEM_CUDA(h, cudaMemcpyAsync(h->b_fqp, f_qp, sizeof(double) * nb * ncp, kind, s));
  else VEM_CUDA(h, cudaMemsetAsync(h->b_fqp, 0, sizeof(double) * nb * ncp, s));
  if (gD_qp && h->n_bqp > 0) VEM_CUDA(h, cudaMemcpyAsync(h->b_gqp, gD_qp, sizeof(double) * nb * h->n_bqp, kind, s));
  else VEM_CUDA(h, cudaMemsetAsync(h->b_gqp, 0, sizeof(double) * nb * nbq, s));
  // geometry-only local matrices (nu = 1), then the per-system values
  cudaEventRecord(h->ev0, s);
  VEM_TRY(classify_cells(h));
  VEM_TRY(assemble_local(h));
  VEM_TRY(assemble_batched_values(h, nb, h->b_nu, op));
  for (int b = 0; b < nb; ++b)
    VEM_TRY(assemble_rhs_into(h, h->b_fqp + (int64_t)b * ncp, (gD_qp && h->n_bqp > 0) ? h->b_gqp + (int64_t)b * nbq : nullptr,
                              h->b_rhs + (int64_t)b * h->n_u, h->b_rhs + op.n_u + (int64_t)b * h->n_p));
  VEM_TRY(check_device_errors(h, "batched right-hand side"));
  cudaEventRecord(h->ev1, s);
  cudaEventSynchronize(h->ev1);
  float tas = 0.f;
  cudaEventElapsedTime(&tas, h->ev0, h->ev1);
  // per-system right-hand-side norms.  FGMRES: every system runs its own
  // Krylov process and stops on its own test.  MINRES: one process on the
  // stacked system, stopped when ||r|| <= rtol min_b ||b_b||, so that every
  // system meets rtol.
  std::vector<double> bn(nb), rn(nb);
  double *dn = h->part;   // nb <= 65535 norms fit in the partial-sum buffer
  count_launch();
  k_segment_norms<<<nb, 256, 0, s>>>(nb, h->n_u, h->n_p, h->b_rhs, dn);
  VEM_CUDA(h, cudaMemcpyAsync(bn.data(), dn, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaStreamSynchronize(s));
  double bmin = 0.0, btot = 0.0;
  for (int b = 0; b < nb; ++b) {
    btot += bn[b] * bn[b];
    if (bn[b] > 0.0) bmin = (bmin == 0.0) ? bn[b] : std::min(bmin, bn[b]);
  }
  btot = std::sqrt(btot);
  const double rtol = h->opt.rtol;
  const bool per_system = h->opt.krylov == VEM_KRYLOV_FGMRES;
  if (!per_system && btot > 0.0 && bmin > 0.0) h->opt.rtol = rtol * bmin / btot;
  count_launch();
  k_import_x<<<grid_for(op.n, 256), 256, 0, s>>>(op.n_u, op.n, nullptr, h->b_x);
  vem_stats st{};
  st.n_u = op.n_u;
  st.n_p = op.n_p;
  st.nnz_A = h->A.nnz;
  st.nnz_S = h->S.nnz;
  st.t_assemble_ms = tas;
  cudaEventRecord(h->ev0, s);
  vem_status r = per_system ? run_fgmres_systems(h, op, h->b_rhs, h->b_x, &st, nullptr)
                            : krylov_solve(h, op, h->b_rhs, h->b_x, &st);
  cudaEventRecord(h->ev1, s);
  cudaEventSynchronize(h->ev1);
  h->opt.rtol = rtol;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev0, h->ev1);
  st.t_solve_ms = ms;
  st.schur_tile = h->schur_tile;
  if (r != VEM_OK && r != VEM_ERR_NOT_CONVERGED) {
    if (stats) *stats = st;
    return r;
  }
  // per-system true relative residuals
  double *tmp = nullptr;
  VEM_TRY(dalloc_n(h, &tmp, (size_t)op.n));
  spmv_batched(s, op.A, nb, h->n_u, op.A.val, h->b_x, tmp);
  count_launch();
  k_sub<<<grid_for(op.n, 256), 256, 0, s>>>(op.n, h->b_rhs, tmp, tmp);
  count_launch();
  k_segment_norms<<<nb, 256, 0, s>>>(nb, h->n_u, h->n_p, tmp, dn);
  VEM_CUDA(h, cudaMemcpyAsync(rn.data(), dn, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaStreamSynchronize(s));
  dfree(h, tmp);
  double worst = 0.0;
  for (int b = 0; b < nb; ++b) {
    rn[b] = bn[b] > 0.0 ? rn[b] / bn[b] : rn[b];
    worst = std::max(worst, rn[b]);
  }
  st.relres = worst;
  if (stats) *stats = st;
  if (relres_out) std::memcpy(relres_out, rn.data(), sizeof(double) * nb);
  // outputs: u_b contiguous, p_b = -p~_b
  if (dev) {
    count_launch();
    k_export_x<<<grid_for(op.n, 256), 256, 0, s>>>(op.n_u, op.n_p, h->b_x, u_out, p_out);
    VEM_CUDA(h, cudaStreamSynchronize(s));
  } else {
    VEM_CUDA(h, cudaMemcpyAsync(u_out, h->b_x, sizeof(double) * op.n_u, cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaMemcpyAsync(p_out, h->b_x + op.n_u, sizeof(double) * op.n_p, cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    for (int64_t i = 0; i < op.n_p; ++i) p_out[i] = -p_out[i];
  }
  if (r == VEM_OK && worst > rtol)
    return fail(h, VEM_ERR_NOT_CONVERGED, "batched solve: worst relres %.3e", worst);
  return r;
}

vem_status vem_get_geometry(vem_handle *h, double *fa, double *fc, double *fn, double *fd, double *cv,
                            double *cc, double *cd) {
  if (!h) return VEM_ERR_BAD_INPUT;
  cudaStream_t s = h->stream;
  if (fa) VEM_CUDA(h, cudaMemcpyAsync(fa, h->f_area, sizeof(double) * h->nf, cudaMemcpyDeviceToHost, s));
  if (fc) VEM_CUDA(h, cudaMemcpyAsync(fc, h->f_cent, sizeof(double) * 3 * h->nf, cudaMemcpyDeviceToHost, s));
  if (fn) VEM_CUDA(h, cudaMemcpyAsync(fn, h->f_norm, sizeof(double) * 3 * h->nf, cudaMemcpyDeviceToHost, s));
  if (fd) VEM_CUDA(h, cudaMemcpyAsync(fd, h->f_diam, sizeof(double) * h->nf, cudaMemcpyDeviceToHost, s));
  if (cv) VEM_CUDA(h, cudaMemcpyAsync(cv, h->c_vol, sizeof(double) * h->nc, cudaMemcpyDeviceToHost, s));
  if (cc) VEM_CUDA(h, cudaMemcpyAsync(cc, h->c_cent, sizeof(double) * 3 * h->nc, cudaMemcpyDeviceToHost, s));
  if (cd) VEM_CUDA(h, cudaMemcpyAsync(cd, h->c_diam, sizeof(double) * h->nc, cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaStreamSynchronize(s));
  return VEM_OK;
}

static std::vector<int64_t> host_cell_face_ptr(const vem_handle *h) {
  std::vector<int64_t> p(h->nc + 1);
  if (cudaMemcpy(p.data(), h->cf_ptr, sizeof(int64_t) * (h->nc + 1), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    p.assign(h->nc + 1, 0);
  }
  return p;
}

vem_status vem_local_size(const vem_handle *h, int64_t *m_total, int64_t *b_total) {
  if (!h || !m_total || !b_total) return VEM_ERR_BAD_INPUT;
  cudaStreamSynchronize(h->stream);
  const std::vector<int64_t> cfp = host_cell_face_ptr(h);
  int64_t mt = 0;
  for (int64_t c = 0; c < h->nc; ++c) {
    const int64_t nl = h->nfd * (cfp[c + 1] - cfp[c]) + h->nid;
    mt += nl * nl;
  }
  *m_total = mt;
  *b_total = (int64_t)h->nq * (h->nfd * h->n_cf + h->nid * h->nc);
  return VEM_OK;
}

vem_status vem_get_local(vem_handle *h, double *M_out, int64_t *M_offsets, double *B_out) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (!h->assembled && !h->local_ready)
    return fail(h, VEM_ERR_BAD_INPUT, "vem_get_local before vem_assemble / vem_assemble_local");
  cudaStream_t s = h->stream;
  // stored per congruence class with nu = 1: expand to M_P = nu_P Mhat, B_P = Bhat
  std::vector<double> Mc(h->m_total), Bc(h->b_total), nu(h->nc);
  std::vector<int64_t> mo(h->ncls + 1), bo(h->ncls + 1);
  std::vector<int32_t> cls(h->nc);
  VEM_CUDA(h, cudaMemcpyAsync(Mc.data(), h->Mloc, sizeof(double) * h->m_total, cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaMemcpyAsync(Bc.data(), h->Bloc, sizeof(double) * h->b_total, cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaMemcpyAsync(nu.data(), h->nu, sizeof(double) * h->nc, cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaMemcpyAsync(mo.data(), h->m_off, sizeof(int64_t) * (h->ncls + 1), cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaMemcpyAsync(bo.data(), h->b_off, sizeof(int64_t) * (h->ncls + 1), cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaMemcpyAsync(cls.data(), h->cls_of, sizeof(int32_t) * h->nc, cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaStreamSynchronize(s));
  const std::vector<int64_t> cfp = host_cell_face_ptr(h);
  int64_t om = 0, ob = 0;
  for (int64_t c = 0; c < h->nc; ++c) {
    const int64_t nl = h->nfd * (cfp[c + 1] - cfp[c]) + h->nid;
    const int k = cls[c];
    if (M_offsets) M_offsets[c] = om;
    if (M_out)
      for (int64_t e = 0; e < nl * nl; ++e) M_out[om + e] = nu[c] * Mc[mo[k] + e];
    if (B_out)
      for (int64_t e = 0; e < h->nq * nl; ++e) B_out[ob + e] = Bc[bo[k] + e];
    om += nl * nl;
    ob += h->nq * nl;
  }
  if (M_offsets) M_offsets[h->nc] = om;
  return VEM_OK;
}

vem_status vem_get_system(vem_handle *h, int64_t *rp, int32_t *col, double *val, double *rhs) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (!h->assembled) VEM_TRY(assemble_impl(h));
  VEM_TRY(ensure_rhs(h));
  if (rhs) {
    VEM_CUDA(h, cudaMemcpyAsync(rhs, h->rhs, sizeof(double) * h->n, cudaMemcpyDeviceToHost, h->stream));
    VEM_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return sell_to_host_csr(h, h->A, rp, col, val);
}

vem_status vem_get_schur(vem_handle *h, int64_t *rp, int32_t *col, double *val, double *diagM) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (!h->assembled) VEM_TRY(assemble_impl(h));
  if (diagM) {
    VEM_CUDA(h, cudaMemcpyAsync(diagM, h->diagM, sizeof(double) * h->n_u, cudaMemcpyDeviceToHost, h->stream));
    VEM_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  return sell_to_host_csr(h, h->S, rp, col, val);
}

vem_status vem_apply_device(vem_handle *h, const double *x, double *y) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (!x || !y) return fail(h, VEM_ERR_BAD_INPUT, "x / y: NULL");
  if (!h->assembled) VEM_TRY(assemble_impl(h));
  spmv(h->stream, h->A, x, y);
  VEM_CUDA(h, cudaGetLastError());
  VEM_CUDA(h, cudaStreamSynchronize(h->stream));
  return VEM_OK;
}

vem_status vem_launch_count(int64_t *n) {
  if (!n) return VEM_ERR_BAD_INPUT;
  *n = launch_count();
  return VEM_OK;
}

const char *vem_last_error(const vem_handle *h) { return h ? h->last_error.c_str() : "NULL handle"; }

vem_status vem_bface_info(vem_handle *h, double *normals_out, int8_t *flags_out) {
  if (!h) return VEM_ERR_BAD_INPUT;
  if (h->n_bqp == 0) return VEM_OK;
  double *dn = nullptr;
  int8_t *df = nullptr;
  VEM_TRY(dalloc_n(h, &dn, 3 * (size_t)h->n_bqp));
  VEM_TRY(dalloc_n(h, &df, (size_t)h->n_bqp));
  vem_status r = bface_info(h, dn, df);
  if (r == VEM_OK && normals_out)
    r = cuda_check(h, cudaMemcpy(normals_out, dn, sizeof(double) * 3 * h->n_bqp, cudaMemcpyDeviceToHost), "normals");
  if (r == VEM_OK && flags_out)
    r = cuda_check(h, cudaMemcpy(flags_out, df, h->n_bqp, cudaMemcpyDeviceToHost), "flags");
  dfree(h, dn);
  dfree(h, df);
  return r;
}

static AmgState **amg_slot(vem_handle *h, int32_t which) {
  if (which == VEM_AMG_SCHUR) return &h->amg;
  if (which == VEM_AMG_REG) return &h->amg_reg;
  return nullptr;
}

vem_status vem_amg_setup(vem_handle *h, int32_t which) {
  if (!h) return VEM_ERR_BAD_INPUT;
  AmgState **slot = amg_slot(h, which);
  if (!slot) return fail(h, VEM_ERR_BAD_INPUT, "unknown AMG hierarchy %d", which);
  if (!h->assembled) VEM_TRY(assemble_impl(h));
  const bool fp32 = h->opt.precision == VEM_PRECISION_MIXED;
  if (which == VEM_AMG_SCHUR) return schur_amg_setup(h, h->S, h->S_val32);
  (void)fp32;
  amg_invalidate(h->amg_reg);   // rebuilt for the current options
  return ensure_reg(h);
}

vem_status vem_amg_levels(vem_handle *h, int32_t which, int32_t *nlev, int64_t *rows, int64_t *nnz,
                          int64_t *nnz_p) {
  if (!h || !nlev) return VEM_ERR_BAD_INPUT;
  AmgState **slot = amg_slot(h, which);
  if (!slot) return fail(h, VEM_ERR_BAD_INPUT, "unknown AMG hierarchy %d", which);
  int nl = 0;
  VEM_TRY(amg_level_info(h, *slot, &nl, rows, nnz, nnz_p));
  *nlev = nl;
  return VEM_OK;
}

vem_status vem_amg_get_level(vem_handle *h, int32_t which, int32_t level, int64_t *row_ptr, int32_t *col,
                             double *val, int32_t *agg, int64_t *prow_ptr, int32_t *pcol, double *pval) {
  if (!h) return VEM_ERR_BAD_INPUT;
  AmgState **slot = amg_slot(h, which);
  if (!slot) return fail(h, VEM_ERR_BAD_INPUT, "unknown AMG hierarchy %d", which);
  return amg_level_copy(h, *slot, level, row_ptr, col, val, agg, prow_ptr, pcol, pval);
}

vem_status vem_amg_vcycle_device(vem_handle *h, int32_t which, const double *b_dev, double *x_dev) {
  if (!h || !b_dev || !x_dev) return VEM_ERR_BAD_INPUT;
  AmgState **slot = amg_slot(h, which);
  if (!slot) return fail(h, VEM_ERR_BAD_INPUT, "unknown AMG hierarchy %d", which);
  if (!amg_valid(*slot)) return fail(h, VEM_ERR_BAD_INPUT, "no AMG hierarchy: call vem_amg_setup first");
  amg_vcycle(h, *slot, b_dev, x_dev, nullptr);
  VEM_CUDA(h, cudaGetLastError());
  VEM_CUDA(h, cudaStreamSynchronize(h->stream));
  return VEM_OK;
}

vem_status vem_release_memory(void) {
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return VEM_ERR_CUDA;
  }
  cudaMemPool_t pool;
  if (device_pool(&pool) != cudaSuccess || cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
    cudaGetLastError();
    return VEM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  for (auto &b : g_pinned_free) cudaFreeHost(b.first);
  g_pinned_free.clear();
  return VEM_OK;
}

void vem_destroy(vem_handle *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  vem::amg_free(h->amg);
  vem::amg_free(h->amg_reg);
  if (h->pcg_graph) cudaGraphExecDestroy(h->pcg_graph);
  if (h->pcg_graph16) cudaGraphExecDestroy(h->pcg_graph16);
  if (h->bpcg_graph) cudaGraphExecDestroy(h->bpcg_graph);
  if (h->bpcg_graph16) cudaGraphExecDestroy(h->bpcg_graph16);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (void *p : h->allocations) cudaFreeAsync(p, h->stream);
  if (!h->allocations.empty()) cudaStreamSynchronize(h->stream);
  h->allocations.clear();
  pinned_free(h->h_err, 64);
  pinned_free(h->h_scal, 8192 * sizeof(double));
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->ev2) cudaEventDestroy(h->ev2);
  if (h->ev3) cudaEventDestroy(h->ev3);
  for (auto &e : h->tev)
    if (e) cudaEventDestroy(e);
  for (auto &e : h->aev)
    if (e) cudaEventDestroy(e);
  delete h;
}

}  // extern "C"
