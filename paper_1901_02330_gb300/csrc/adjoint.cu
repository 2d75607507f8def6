// Adjoint contraction for gradients with respect to per-cell log K.
//
// With theta_P = log K_P and nu_P = exp(-theta_P), the flux block is
// M = sum_P M_P with M_P proportional to nu_P (Sec. 4.3, a_{h,P}), so
// dM/dtheta_P = -M_P.  For A x = b and the adjoint A lambda = dL/dx
// (A is symmetric) the gradient is dL/dtheta_P = lambda_{u,P}^T M_P u_P,
// with the cell's local flux DOFs gathered from the global vectors.  One warp
// per cell; the local vectors are staged in shared memory.
#include "handle.cuh"

namespace vem {

__global__ void k_adjoint_contract(int64_t nc, int nfd, int nid, int64_t nf, int max_nl,
                                   const int64_t *__restrict__ cfp, const int32_t *__restrict__ cf,
                                   const int32_t *__restrict__ cls_of, const double *__restrict__ nu,
                                   const int64_t *__restrict__ m_off, const double *__restrict__ Mloc,
                                   const double *__restrict__ lam, const double *__restrict__ x,
                                   double *g) {
  extern __shared__ double sm[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double *ul = sm + (size_t)warp * 2 * max_nl;
  double *ll = ul + max_nl;
  for (int64_t c = (int64_t)blockIdx.x * wpb + warp; c < nc; c += (int64_t)gridDim.x * wpb) {
    const int64_t b = cfp[c];
    const int k = (int)(cfp[c + 1] - b);
    const int nl = nfd * k + nid;
    for (int j = lane; j < nl; j += 32) {
      const int64_t gj = (j < nfd * k) ? (int64_t)nfd * cf[b + j / nfd] + j % nfd
                                       : (int64_t)nfd * nf + (int64_t)nid * c + (j - nfd * k);
      ul[j] = x[gj];
      ll[j] = lam[gj];
    }
    __syncwarp();
    const double *M = Mloc + m_off[cls_of[c]];   // nu = 1 class matrix
    double acc = 0.0;
    for (int j = lane; j < nl; j += 32) {
      double t = 0.0;
      for (int jp = 0; jp < nl; ++jp) t += M[(int64_t)j * nl + jp] * ul[jp];
      acc += ll[j] * t;
    }
    acc = warp_sum(acc);
    if (lane == 0) g[c] = nu[c] * acc;
    __syncwarp();
  }
}

vem_status adjoint_contract(vem_handle *h, const double *lam, const double *x, double *g) {
  const int max_nl = h->nfd * h->max_nf_cell + h->nid;
  const int wpb = 8;
  const size_t smem = sizeof(double) * 2 * max_nl * wpb;
  if (smem > 48 * 1024)
    VEM_CUDA(h, cudaFuncSetAttribute(k_adjoint_contract, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int64_t blocks = (h->nc + wpb - 1) / wpb;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  count_launch();
  k_adjoint_contract<<<(int)blocks, 32 * wpb, smem, h->stream>>>(h->nc, h->nfd, h->nid, h->nf, max_nl, h->cf_ptr,
                                                                 h->cf, h->cls_of, h->nu, h->m_off, h->Mloc, lam, x, g);
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

}  // namespace vem
