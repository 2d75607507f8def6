// Global assembly (paper Sec. 4.3, global forms a_h, b_h, f_h glued across
// cells) into one CSR matrix of the saddle-point operator [M B^T; B 0]
// (Sec. 5), and the Schur approximation S = B diag(M)^{-1} B^T of the
// Block-Schur preconditioner (eq. block_schur).
//
// Row layout: face DOF rows (nfd per face), interior DOF rows (nid per
// cell), pressure rows (one per cell).  A face row gathers the matching
// rows of the (at most two) local matrices of its cells: columns of the
// lower-id cell in its local order, then those of the other cell except the
// shared face, then the pressure columns.  No atomics: every entry is a
// fixed-order sum of at most two local values, so the result is
// deterministic.
#include "handle.cuh"

namespace vem {

struct Layout {
  int nfd, nid;
  int64_t nf, nc, n_u;
  const int64_t *cfp;
  const int32_t *cf;
  const int32_t *f_cell, *f_loc;
  const int64_t *m_off;
  const double *Mloc, *Bloc;
};

__device__ __forceinline__ int nloc(const Layout &L, int64_t c) {
  return L.nfd * (int)(L.cfp[c + 1] - L.cfp[c]) + L.nid;
}
__device__ __forceinline__ int64_t gcol(const Layout &L, int64_t c, int jl) {
  const int k = (int)(L.cfp[c + 1] - L.cfp[c]);
  if (jl < L.nfd * k) return (int64_t)L.nfd * L.cf[L.cfp[c] + jl / L.nfd] + jl % L.nfd;
  return (int64_t)L.nfd * L.nf + (int64_t)L.nid * c + (jl - L.nfd * k);
}
__device__ __forceinline__ int64_t boff(const Layout &L, int64_t c) {
  return L.cfp[c] * L.nfd + (int64_t)L.nid * c;
}

__global__ void k_rowcount(Layout L, int64_t *cnt) {
  const int64_t n = L.n_u + L.nc;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t v;
    if (r < L.nfd * L.nf) {
      const int64_t f = r / L.nfd;
      const int beta = (int)(r % L.nfd);
      const int32_t c0 = L.f_cell[2 * f], c1 = L.f_cell[2 * f + 1];
      v = nloc(L, c0) + (c1 >= 0 ? nloc(L, c1) - L.nfd : 0) + (beta == 0 ? (c1 >= 0 ? 2 : 1) : 0);
    } else if (r < L.n_u) {
      v = nloc(L, (r - L.nfd * L.nf) / L.nid);
    } else {
      const int64_t c = r - L.n_u;
      v = L.cfp[c + 1] - L.cfp[c];
    }
    cnt[r] = v;
  }
}

__global__ void k_fill(Layout L, const int64_t *__restrict__ rp, int32_t *col, double *val,
                       double *diagM) {
  const int64_t n = L.n_u + L.nc;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = rp[r];
    if (r < L.nfd * L.nf) {
      const int64_t f = r / L.nfd;
      const int beta = (int)(r % L.nfd);
      const int32_t c0 = L.f_cell[2 * f], c1 = L.f_cell[2 * f + 1];
      const int l0 = L.f_loc[2 * f], l1 = L.f_loc[2 * f + 1];
      const int n0 = nloc(L, c0);
      const double *M0 = L.Mloc + L.m_off[c0] + (int64_t)(l0 * L.nfd + beta) * n0;
      const double *M1 = nullptr;
      int n1 = 0;
      if (c1 >= 0) {
        n1 = nloc(L, c1);
        M1 = L.Mloc + L.m_off[c1] + (int64_t)(l1 * L.nfd + beta) * n1;
      }
      double dg = 0.0;
      for (int j = 0; j < n0; ++j) {
        double v = M0[j];
        const bool shared = (j < n0 - L.nid) && (j / L.nfd == l0);
        if (c1 >= 0 && shared) v += M1[l1 * L.nfd + j % L.nfd];
        if (shared && j % L.nfd == beta) dg = v;
        col[o] = (int32_t)gcol(L, c0, j);
        val[o] = v;
        ++o;
      }
      if (c1 >= 0) {
        const int k1 = (n1 - L.nid) / L.nfd;
        for (int j = 0; j < n1; ++j) {
          if (j < L.nfd * k1 && j / L.nfd == l1) continue;
          col[o] = (int32_t)gcol(L, c1, j);
          val[o] = M1[j];
          ++o;
        }
      }
      if (beta == 0) {
        col[o] = (int32_t)(L.n_u + c0);
        val[o] = L.Bloc[boff(L, c0) + l0 * L.nfd];
        ++o;
        if (c1 >= 0) {
          col[o] = (int32_t)(L.n_u + c1);
          val[o] = L.Bloc[boff(L, c1) + l1 * L.nfd];
          ++o;
        }
      }
      diagM[r] = dg;
    } else if (r < L.n_u) {
      const int64_t q = r - L.nfd * L.nf;
      const int64_t c = q / L.nid;
      const int l = (int)(q % L.nid);
      const int nl = nloc(L, c);
      const int jr = nl - L.nid + l;
      const double *Mr = L.Mloc + L.m_off[c] + (int64_t)jr * nl;
      for (int j = 0; j < nl; ++j) {
        col[o] = (int32_t)gcol(L, c, j);
        val[o] = Mr[j];
        ++o;
      }
      diagM[r] = Mr[jr];
    } else {
      const int64_t c = r - L.n_u;
      const int k = (int)(L.cfp[c + 1] - L.cfp[c]);
      for (int i = 0; i < k; ++i) {
        col[o] = (int32_t)((int64_t)L.nfd * L.cf[L.cfp[c] + i]);
        val[o] = L.Bloc[boff(L, c) + i * L.nfd];
        ++o;
      }
    }
  }
}

// S = B diag(M)^{-1} B^T: row P holds sum_f B_Pf^2 / M_ff on the diagonal and
// B_Pf B_Qf / M_ff for the neighbour Q across each interior face f.
__global__ void k_schur_count(Layout L, int64_t *cnt) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < L.nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t v = 1;
    for (int64_t p = L.cfp[c]; p < L.cfp[c + 1]; ++p) v += (L.f_cell[2 * L.cf[p] + 1] >= 0);
    cnt[c] = v;
  }
}

__global__ void k_schur_fill(Layout L, const double *__restrict__ diagM, const int64_t *__restrict__ rp,
                             int32_t *col, double *val, double *dinv, int *err) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < L.nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = rp[c];
    const int64_t b = L.cfp[c];
    const int k = (int)(L.cfp[c + 1] - b);
    const int64_t bo = boff(L, c);
    double dg = 0.0;
    const int64_t od = o++;
    for (int i = 0; i < k; ++i) {
      const int f = L.cf[b + i];
      const double bp = L.Bloc[bo + i * L.nfd];
      const double mf = diagM[(int64_t)L.nfd * f];
      dg += bp * bp / mf;
      const int32_t c0 = L.f_cell[2 * f], c1 = L.f_cell[2 * f + 1];
      if (c1 < 0) continue;
      const int32_t q = (c0 == c) ? c1 : c0;
      const int lq = (c0 == c) ? L.f_loc[2 * f + 1] : L.f_loc[2 * f];
      col[o] = q;
      val[o] = bp * L.Bloc[boff(L, q) + lq * L.nfd] / mf;
      ++o;
    }
    col[od] = (int32_t)c;
    val[od] = dg;
    if (!(dg > 0.0) || !isfinite(dg)) atomicOr(err, DEVERR_NONFINITE);
    dinv[c] = 1.0 / dg;
  }
}

// B entries of the (f, 0) DOF in each of the face's two cells (0 for a
// missing second cell), for the block-triangular flux update.
__global__ void k_bt_face(Layout L, double *bt) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < L.nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    for (int s = 0; s < 2; ++s) {
      const int32_t c = L.f_cell[2 * f + s];
      bt[2 * f + s] = c >= 0 ? L.Bloc[boff(L, c) + L.f_loc[2 * f + s] * L.nfd] : 0.0;
    }
  }
}

// ---- exclusive scan of int64 counts: out[0] = 0, out[i+1] = sum_{j<=i} ----
constexpr int kScanBlocks = 1024;
constexpr int kScanThreads = 256;

__device__ int64_t block_incl_scan(int64_t v, int64_t *tot) {
  __shared__ int64_t ws[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) ws[w] = v;
  __syncthreads();
  if (w == 0) {
    int64_t t = (lane < kScanThreads / 32) ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    if (lane < kScanThreads / 32) ws[lane] = t;
  }
  __syncthreads();
  if (w > 0) v += ws[w - 1];
  *tot = ws[kScanThreads / 32 - 1];
  __syncthreads();
  return v;
}

__global__ void k_scan_sums(int64_t n, const int64_t *in, int64_t *bsum) {
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  __shared__ int64_t ws[kScanThreads / 32];
  int64_t s = 0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += in[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int i = 0; i < kScanThreads / 32; ++i) t += ws[i];
    bsum[blockIdx.x] = t;
  }
}

__global__ void k_scan_bsums(int nb, int64_t *bsum) {
  // exclusive scan of nb <= kScanBlocks block sums by one block
  __shared__ int64_t buf[kScanBlocks];
  for (int i = threadIdx.x; i < nb; i += blockDim.x) buf[i] = bsum[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int i = 0; i < nb; ++i) {
      int64_t t = buf[i];
      buf[i] = acc;
      acc += t;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) bsum[i] = buf[i];
}

__global__ void k_scan_apply(int64_t n, const int64_t *in, const int64_t *bsum, int64_t *out) {
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  int64_t carry = bsum[blockIdx.x];
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
  for (int64_t t0 = lo; t0 < hi; t0 += blockDim.x) {
    const int64_t i = t0 + threadIdx.x;
    int64_t v = (i < hi) ? in[i] : 0;
    int64_t tot;
    int64_t inc = block_incl_scan(v, &tot);
    if (i < hi) out[i + 1] = carry + inc;
    carry += tot;
  }
}

static vem_status scan_counts(vem_handle *h, int64_t n, const int64_t *cnt, int64_t *out,
                              int64_t *total) {
  cudaStream_t s = h->stream;
  if (!h->scan_buf) VEM_TRY(dalloc_n(h, &h->scan_buf, kScanBlocks));
  int64_t *bsum = h->scan_buf;
  count_launch(); k_scan_sums<<<kScanBlocks, kScanThreads, 0, s>>>(n, cnt, bsum);
  count_launch(); k_scan_bsums<<<1, 1024, 0, s>>>(kScanBlocks, bsum);
  count_launch(); k_scan_apply<<<kScanBlocks, kScanThreads, 0, s>>>(n, cnt, bsum, out);
  VEM_CUDA(h, cudaGetLastError());
  VEM_CUDA(h, cudaMemcpyAsync(total, out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaStreamSynchronize(s));
  return VEM_OK;
}

vem_status assemble_global(vem_handle *h) {
  cudaStream_t s = h->stream;
  Layout L{h->nfd, h->nid, h->nf, h->nc, h->n_u, h->cf_ptr, h->cf, h->f_cell, h->f_loc,
           h->m_off, h->Mloc, h->Bloc};
  const int T = 256;
  const int64_t n = h->n;
  // ---- [M B^T; B 0] ----
  if (!h->cnt_buf) VEM_TRY(dalloc_n(h, &h->cnt_buf, (size_t)n + 1));
  int64_t *cnt = h->cnt_buf;
  count_launch(); k_rowcount<<<grid_for(n, T), T, 0, s>>>(L, cnt);
  VEM_CUDA(h, cudaGetLastError());
  if (!h->a_rp) VEM_TRY(dalloc_n(h, &h->a_rp, (size_t)n + 1));
  int64_t nnz = 0;
  VEM_TRY(scan_counts(h, n, cnt, h->a_rp, &nnz));
  if (nnz >= (int64_t)1 << 62) return fail(h, VEM_ERR_UNSUPPORTED, "nnz overflow");
  if (h->nnz_a != nnz) {
    dfree(h, h->a_col);
    dfree(h, h->a_val);
    h->a_col = nullptr;
    h->a_val = nullptr;
    VEM_TRY(dalloc_n(h, &h->a_col, (size_t)nnz));
    VEM_TRY(dalloc_n(h, &h->a_val, (size_t)nnz));
    h->nnz_a = nnz;
  }
  if (!h->diagM) VEM_TRY(dalloc_n(h, &h->diagM, (size_t)h->n_u));
  count_launch(); k_fill<<<grid_for(n, T), T, 0, s>>>(L, h->a_rp, h->a_col, h->a_val, h->diagM);
  VEM_CUDA(h, cudaGetLastError());
  h->a_lanes = choose_lanes((double)nnz / (double)n);
  // ---- S ----
  int64_t *scnt = h->cnt_buf;
  count_launch(); k_schur_count<<<grid_for(h->nc, T), T, 0, s>>>(L, scnt);
  VEM_CUDA(h, cudaGetLastError());
  if (!h->s_rp) VEM_TRY(dalloc_n(h, &h->s_rp, (size_t)h->nc + 1));
  int64_t snnz = 0;
  VEM_TRY(scan_counts(h, h->nc, scnt, h->s_rp, &snnz));
  if (h->nnz_s != snnz) {
    dfree(h, h->s_col);
    dfree(h, h->s_val);
    h->s_col = nullptr;
    h->s_val = nullptr;
    VEM_TRY(dalloc_n(h, &h->s_col, (size_t)snnz));
    VEM_TRY(dalloc_n(h, &h->s_val, (size_t)snnz));
    h->nnz_s = snnz;
  }
  if (!h->s_dinv) VEM_TRY(dalloc_n(h, &h->s_dinv, (size_t)h->nc));
  count_launch(); k_schur_fill<<<grid_for(h->nc, T), T, 0, s>>>(L, h->diagM, h->s_rp, h->s_col, h->s_val, h->s_dinv,
                                                 h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  h->s_lanes = choose_lanes((double)snnz / (double)h->nc);
  if (!h->bt_face) VEM_TRY(dalloc_n(h, &h->bt_face, 2 * (size_t)h->nf));
  count_launch(); k_bt_face<<<grid_for(h->nf, T), T, 0, s>>>(L, h->bt_face);
  VEM_CUDA(h, cudaGetLastError());
  return check_device_errors(h, "global assembly");
}

}  // namespace vem
