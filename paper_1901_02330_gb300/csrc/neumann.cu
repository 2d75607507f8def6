// Prescribed-flux faces and the mean-zero pressure (paper Sec. 3: u.n = u_N
// on the boundary, p in Q = {int p = 0}).
//
// The flux DOFs of faces with flag 2 are eliminated at assembly (unit rows,
// zero columns, their coupling A x_fix moved to the right-hand side).  With
// no Dirichlet face the remaining operator is singular (constant pressures);
// the paper's mean-zero Lagrange multiplier lambda is then eliminated too:
// the pressure equations B u + c lambda = F (c_P = |P|) summed over all cells
// give lambda = sum F / sum |P| (B^T 1 = 0), the system is solved with the
// consistent right-hand side F - c lambda, every inner Schur solve works on
// the consistent (mean-free) part of its right-hand side, and the pressure is
// shifted to sum |P| p_P = 0 at the end.
#include <vector>

#include "handle.cuh"

namespace vem {

// rhs_i = x_fix_i on eliminated rows, rhs_i - (A x_fix)_i elsewhere
__global__ void k_apply_fixed(int64_t n, int nfd, int64_t nf, const int8_t *__restrict__ fbc,
                              const double *__restrict__ corr, const double *__restrict__ xfix, double *rhs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool fixed = i < (int64_t)nfd * nf && fbc[i / nfd] == 2;
    rhs[i] = fixed ? xfix[i] : rhs[i] - corr[i];
  }
}

// Block partials of sum a_(i stride), or of sum w_i a_(i stride) when w is
// given (stride: pressure DOFs per cell; entry i stride is cell i's constant
// moment).
__global__ void k_sums(int64_t n, const double *__restrict__ a, const double *__restrict__ w, double *pa,
                       int stride = 1) {
  double sa = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    sa += w ? w[i] * a[i * stride] : a[i * stride];
  block_partial(sa, pa);
}

// y_(i stride) = x_(i stride) - s c_i with s = (sum of the pa partials) /
// (sum of the pw partials, or n when pw is NULL); c = NULL stands for the
// vector of ones.  Every block recomputes s from the partials in the same
// order.  Optionally stores s.  Entries off the stride are not touched.
__global__ void k_sub_scaled(int64_t n, const double *__restrict__ pa, const double *__restrict__ pw, int nb,
                             const double *__restrict__ c, const double *x, double *y, double *s_out,
                             int stride = 1) {
  const double sa = sum_partials(pa, nb);
  const double sw = pw ? sum_partials(pw, nb) : (double)n;
  const double s = sa / sw;
  if (s_out && blockIdx.x == 0 && threadIdx.x == 0) *s_out = s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i * stride] = x[i * stride] - s * (c ? c[i] : 1.0);
}

static vem_status ensure_npart(vem_handle *h) {
  if (!h->npart) VEM_TRY(dalloc_n(h, &h->npart, 2 * (size_t)kMaxBlocks + 2));
  return VEM_OK;
}

vem_status neumann_rhs(vem_handle *h, double *rhs) {
  if (h->n_flux_faces == 0) return VEM_OK;
  cudaStream_t s = h->stream;
  const int64_t n = h->n;
  count_launch();
  k_apply_fixed<<<grid_for(n, 256), 256, 0, s>>>(n, h->nfd, h->nf, h->fbc, h->rhs_corr, h->xfix, rhs);
  VEM_CUDA(h, cudaGetLastError());
  if (!h->multiplier) return VEM_OK;
  // lambda = e^T F / e^T c (e: the constant moments, c: |P| on them);
  // F <- F - c lambda
  VEM_TRY(ensure_npart(h));
  double *F = rhs + h->n_u;
  const int nb = nblocks_vec(h->nc);
  const int q = h->nq;
  double *pa = h->npart, *pw = h->npart + kMaxBlocks, *lam = h->npart + 2 * kMaxBlocks;
  count_launch();
  k_sums<<<nb, kRedThreads, 0, s>>>(h->nc, F, nullptr, pa, q);
  count_launch();
  k_sums<<<nb, kRedThreads, 0, s>>>(h->nc, h->c_vol, nullptr, pw);
  count_launch();
  k_sub_scaled<<<nb, kRedThreads, 0, s>>>(h->nc, pa, pw, nb, h->c_vol, F, F, lam, q);
  VEM_CUDA(h, cudaGetLastError());
  VEM_CUDA(h, cudaMemcpyAsync(&h->lambda, lam, sizeof(double), cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaStreamSynchronize(s));
  return VEM_OK;
}

// out = b minus its component along the constant moments (the consistent
// part: the range of S is orthogonal to them).
vem_status neumann_mean_free(vem_handle *h, int64_t n, const double *b, double *out) {
  VEM_TRY(ensure_npart(h));
  const int q = h->nq;
  const int64_t nc = n / q;
  const int nb = nblocks_vec(nc);
  if (q > 1 && out != b) VEM_CUDA(h, cudaMemcpyAsync(out, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream));
  count_launch();
  k_sums<<<nb, kRedThreads, 0, h->stream>>>(nc, b, nullptr, h->npart, q);
  count_launch();
  k_sub_scaled<<<nb, kRedThreads, 0, h->stream>>>(nc, h->npart, nullptr, nb, nullptr, q > 1 ? out : b, out, nullptr,
                                                  q);
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

vem_status device_sum(vem_handle *h, int64_t n, const double *a, double *out) {
  VEM_TRY(ensure_npart(h));
  const int nb = nblocks_vec(n);
  count_launch();
  k_sums<<<nb, kRedThreads, 0, h->stream>>>(n, a, nullptr, h->npart);
  VEM_CUDA(h, cudaGetLastError());
  std::vector<double> part(nb);
  VEM_CUDA(h, cudaMemcpyAsync(part.data(), h->npart, sizeof(double) * nb, cudaMemcpyDeviceToHost, h->stream));
  VEM_CUDA(h, cudaStreamSynchronize(h->stream));
  double t = 0.0;
  for (int i = 0; i < nb; ++i) t += part[i];
  *out = t;
  return VEM_OK;
}

vem_status neumann_shift(vem_handle *h, double *xp) {
  if (!h->multiplier) return VEM_OK;
  // shift along the constant moments to c^T p = 0
  VEM_TRY(ensure_npart(h));
  const int nb = nblocks_vec(h->nc);
  const int q = h->nq;
  count_launch();
  k_sums<<<nb, kRedThreads, 0, h->stream>>>(h->nc, xp, h->c_vol, h->npart, q);
  count_launch();
  k_sums<<<nb, kRedThreads, 0, h->stream>>>(h->nc, h->c_vol, nullptr, h->npart + kMaxBlocks);
  count_launch();
  k_sub_scaled<<<nb, kRedThreads, 0, h->stream>>>(h->nc, h->npart, h->npart + kMaxBlocks, nb, nullptr, xp, xp,
                                                  nullptr, q);
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

}  // namespace vem
