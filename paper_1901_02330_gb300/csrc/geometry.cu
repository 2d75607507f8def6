// Face and cell geometry (paper Sec. 2: barycentres x_f, x_P, diameters
// h_f, h_P and the face frame of the scaled face monomials) and the
// face -> cell adjacency.  One thread per face / per cell.
#include <algorithm>

#include "handle.cuh"
#include "geom_device.cuh"

namespace vem {

__global__ void k_face_geom(int64_t nf, const double *__restrict__ xyz,
                            const int64_t *__restrict__ fvp, const int32_t *__restrict__ fv,
                            double *area, double *cent, double *nrm, double *t1, double *diam,
                            int *err) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = fvp[f];
    const int m = (int)(fvp[f + 1] - b);
    double3 xb = make_double3(0, 0, 0);
    for (int i = 0; i < m; ++i) xb = add3(xb, load3(xyz, fv[b + i]));
    xb = scale3(xb, 1.0 / m);
    // area vector of the loop around its vertex mean
    double3 av = make_double3(0, 0, 0);
    for (int i = 0; i < m; ++i) {
      double3 a = sub3(load3(xyz, fv[b + i]), xb);
      double3 c = sub3(load3(xyz, fv[b + (i + 1) % m]), xb);
      av = add3(av, cross3(a, c));
    }
    const double an = norm3(av);
    double3 n = scale3(av, 1.0 / an);
    double num0 = 0, num1 = 0, num2 = 0, den = 0;
    for (int i = 0; i < m; ++i) {
      double3 A = load3(xyz, fv[b + i]);
      double3 B = load3(xyz, fv[b + (i + 1) % m]);
      double sa = 0.5 * dot3(cross3(sub3(A, xb), sub3(B, xb)), n);
      double3 c = scale3(add3(add3(xb, A), B), 1.0 / 3.0);
      num0 += sa * c.x;
      num1 += sa * c.y;
      num2 += sa * c.z;
      den += sa;
    }
    double dm = 0;
    for (int i = 0; i < m; ++i) {
      double3 A = load3(xyz, fv[b + i]);
      for (int j = i + 1; j < m; ++j) dm = fmax(dm, norm3(sub3(A, load3(xyz, fv[b + j]))));
    }
    double3 e = sub3(load3(xyz, fv[b + 1]), load3(xyz, fv[b]));
    double en = norm3(e);
    if (!(den > 0.0) || !(an > 0.0) || !(en > 0.0) || !isfinite(den) || !isfinite(dm))
      atomicOr(err, DEVERR_DEGENERATE_FACE);
    area[f] = den;
    store3(cent, f, make_double3(num0 / den, num1 / den, num2 / den));
    store3(nrm, f, n);
    store3(t1, f, scale3(e, 1.0 / en));
    diam[f] = dm;
  }
}

// Volume and barycentre from pyramids (x_ref, face): volume |f| h / 3 and
// centroid x_ref + 3/4 (x_f - x_ref); x_ref = mean of the face barycentres.
__global__ void k_cell_geom(int64_t nc, const int64_t *__restrict__ cfp,
                            const int32_t *__restrict__ cf, const int64_t *__restrict__ fvp,
                            const int32_t *__restrict__ fv, const double *__restrict__ xyz,
                            const double *__restrict__ f_area, const double *__restrict__ f_cent,
                            const double *__restrict__ f_norm, double *c_vol, double *c_cent,
                            double *c_diam, int8_t *cf_sigma, int *err) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = cfp[c];
    const int k = (int)(cfp[c + 1] - b);
    double3 xr = make_double3(0, 0, 0);
    for (int i = 0; i < k; ++i) xr = add3(xr, load3(f_cent, cf[b + i]));
    xr = scale3(xr, 1.0 / k);
    double vol = 0, s0 = 0, s1 = 0, s2 = 0;
    for (int i = 0; i < k; ++i) {
      const int f = cf[b + i];
      double3 d = sub3(load3(f_cent, f), xr);
      double hgt = dot3(d, load3(f_norm, f));
      double v = f_area[f] * fabs(hgt) / 3.0;
      vol += v;
      s0 += v * (xr.x + 0.75 * d.x);
      s1 += v * (xr.y + 0.75 * d.y);
      s2 += v * (xr.z + 0.75 * d.z);
      cf_sigma[b + i] = hgt > 0.0 ? 1 : -1;
    }
    double3 xc = make_double3(s0 / vol, s1 / vol, s2 / vol);
    int bad = 0;
    for (int i = 0; i < k; ++i) {
      const int f = cf[b + i];
      double hc = dot3(sub3(load3(f_cent, f), xc), load3(f_norm, f));
      int8_t s = hc > 0.0 ? 1 : -1;
      if (s != cf_sigma[b + i] || hc == 0.0) bad = 1;
    }
    // squared diameter (one square root at the end): the largest distance
    // between two vertices, over the cell's distinct vertices (a vertex is
    // listed by every face that has it); cells with more than kCapV distinct
    // vertices take all pairs of face-vertex references instead (the same
    // maximum)
    constexpr int kCapV = 64;
    int32_t vu[kCapV];
    int nvu = 0;
    bool many = false;
    for (int i = 0; i < k && !many; ++i) {
      const int f = cf[b + i];
      for (int64_t p = fvp[f]; p < fvp[f + 1]; ++p) {
        const int32_t v = fv[p];
        bool seen = false;
        for (int t = 0; t < nvu && !seen; ++t) seen = vu[t] == v;
        if (seen) continue;
        if (nvu == kCapV) {
          many = true;
          break;
        }
        vu[nvu++] = v;
      }
    }
    double dm2 = 0;
    if (!many) {
      for (int a = 0; a < nvu; ++a) {
        const double3 A = load3(xyz, vu[a]);
        for (int t = a + 1; t < nvu; ++t) {
          const double3 d = sub3(A, load3(xyz, vu[t]));
          dm2 = fmax(dm2, dot3(d, d));
        }
      }
    } else {
      for (int i = 0; i < k; ++i) {
        const int f = cf[b + i];
        for (int64_t p = fvp[f]; p < fvp[f + 1]; ++p) {
          double3 A = load3(xyz, fv[p]);
          for (int j = i; j < k; ++j) {
            const int g = cf[b + j];
            for (int64_t q = fvp[g]; q < fvp[g + 1]; ++q) {
              const double3 d = sub3(A, load3(xyz, fv[q]));
              dm2 = fmax(dm2, dot3(d, d));
            }
          }
        }
      }
    }
    const double dm = sqrt(dm2);
    if (!(vol > 0.0) || !isfinite(vol)) atomicOr(err, DEVERR_DEGENERATE_CELL);
    if (bad) atomicOr(err, DEVERR_NONCONVEX);
    c_vol[c] = vol;
    store3(c_cent, c, xc);
    c_diam[c] = dm;
  }
}

__global__ void k_adjacency_count(int64_t nc, const int64_t *__restrict__ cfp,
                                  const int32_t *__restrict__ cf, int *cnt, int32_t *f_cell,
                                  int32_t *f_loc, int *err) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t p = cfp[c]; p < cfp[c + 1]; ++p) {
      const int f = cf[p];
      int slot = atomicAdd(&cnt[f], 1);
      if (slot < 2) {
        f_cell[2 * f + slot] = (int32_t)c;
        f_loc[2 * f + slot] = (int32_t)(p - cfp[c]);
      } else {
        atomicOr(err, DEVERR_ADJACENCY);
      }
    }
  }
}

// Order each face's two cells by id (makes everything downstream
// independent of the atomic slot order) and check the boundary flags.
__global__ void k_adjacency_fix(int64_t nf, const int *cnt, const int8_t *fbc, int32_t *f_cell,
                                int32_t *f_loc, int *err) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int k = cnt[f];
    if (k == 2) {
      if (fbc[f] != 0) atomicOr(err, DEVERR_ADJACENCY);
      if (f_cell[2 * f] > f_cell[2 * f + 1]) {
        int32_t t = f_cell[2 * f];
        f_cell[2 * f] = f_cell[2 * f + 1];
        f_cell[2 * f + 1] = t;
        t = f_loc[2 * f];
        f_loc[2 * f] = f_loc[2 * f + 1];
        f_loc[2 * f + 1] = t;
      }
    } else if (k == 1) {
      if (fbc[f] == 0) atomicOr(err, DEVERR_ADJACENCY);
      f_cell[2 * f + 1] = -1;
      f_loc[2 * f + 1] = -1;
    } else {
      atomicOr(err, DEVERR_ADJACENCY);
    }
  }
}

// Boundary-face load points: the boundary-data rule (ppt points, see
// bface_point) on every fan triangle (x_f, v_i, v_{i+1}) of every Dirichlet
// or prescribed-flux face.
__global__ void k_bface_points(int64_t nf, int ppt, const int8_t *__restrict__ fbc,
                               const int64_t *__restrict__ off, const int64_t *__restrict__ fvp,
                               const int32_t *__restrict__ fv, const double *__restrict__ xyz,
                               const double *__restrict__ f_cent, double *out) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    if (fbc[f] == 0) continue;
    const int64_t b = fvp[f];
    const int m = (int)(fvp[f + 1] - b);
    const double3 xf = load3(f_cent, f);
    int64_t o = off[f];
    for (int i = 0; i < m; ++i) {
      double3 A = load3(xyz, fv[b + i]);
      double3 B = load3(xyz, fv[b + (i + 1) % m]);
      for (int q = 0; q < ppt; ++q) {
        double l0, l1, l2, w;
        bface_point(ppt, q, l0, l1, l2, w);
        store3(out, o++, add3(add3(scale3(xf, l0), scale3(A, l1)), scale3(B, l2)));
      }
    }
  }
}

// Outward unit normal and face flag at every boundary-face load point:
// sigma n_f with sigma the orientation of the face in its one cell.
__global__ void k_bface_info(int64_t nf, const int8_t *__restrict__ fbc, const int64_t *__restrict__ off,
                             const double *__restrict__ f_norm, const int32_t *__restrict__ f_cell,
                             const int32_t *__restrict__ f_loc, const int64_t *__restrict__ cfp,
                             const int8_t *__restrict__ sig, double *nout, int8_t *flag) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    if (fbc[f] == 0) continue;
    const double sg = (double)sig[cfp[f_cell[2 * f]] + f_loc[2 * f]];
    const double3 n = scale3(load3(f_norm, f), sg);
    for (int64_t o = off[f]; o < off[f + 1]; ++o) {
      if (nout) store3(nout, o, n);
      if (flag) flag[o] = fbc[f];
    }
  }
}

vem_status bface_info(vem_handle *h, double *nout, int8_t *flag) {
  count_launch();
  k_bface_info<<<grid_for(h->nf, 128), 128, 0, h->stream>>>(h->nf, h->fbc, h->bqp_off, h->f_norm, h->f_cell,
                                                           h->f_loc, h->cf_ptr, h->cf_sigma, nout, flag);
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

vem_status geometry_build(vem_handle *h) {
  cudaStream_t s = h->stream;
  const int T = 128;
  count_launch(); k_face_geom<<<grid_for(h->nf, T), T, 0, s>>>(h->nf, h->xyz, h->fv_ptr, h->fv, h->f_area,
                                                h->f_cent, h->f_norm, h->f_t1, h->f_diam, h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  count_launch(); k_cell_geom<<<grid_for(h->nc, T), T, 0, s>>>(h->nc, h->cf_ptr, h->cf, h->fv_ptr, h->fv, h->xyz,
                                                h->f_area, h->f_cent, h->f_norm, h->c_vol,
                                                h->c_cent, h->c_diam, h->cf_sigma, h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  int *cnt = nullptr;
  VEM_TRY(dalloc_n(h, &cnt, (size_t)h->nf));
  VEM_CUDA(h, cudaMemsetAsync(cnt, 0, sizeof(int) * h->nf, s));
  count_launch(); k_adjacency_count<<<grid_for(h->nc, T), T, 0, s>>>(h->nc, h->cf_ptr, h->cf, cnt, h->f_cell,
                                                      h->f_loc, h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  count_launch(); k_adjacency_fix<<<grid_for(h->nf, T), T, 0, s>>>(h->nf, cnt, h->fbc, h->f_cell, h->f_loc,
                                                    h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  VEM_TRY(check_device_errors(h, "mesh geometry"));
  dfree(h, cnt);
  if (h->n_bqp > 0) {
    count_launch(); k_bface_points<<<grid_for(h->nf, T), T, 0, s>>>(h->nf, h->bq_ppt, h->fbc, h->bqp_off, h->fv_ptr,
                                                     h->fv, h->xyz, h->f_cent, h->bqp_xyz);
    VEM_CUDA(h, cudaGetLastError());
  }
  return VEM_OK;
}

// Boundary points per face for the rule of ppt points per fan triangle.
__global__ void k_bq_count(int64_t nf, int ppt, const int64_t *__restrict__ fvp, const int8_t *__restrict__ fbc,
                           int64_t *cnt) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x)
    cnt[f] = fbc[f] != 0 ? ppt * (fvp[f + 1] - fvp[f]) : 0;
}

// Rebuild the boundary-face points for another rule (an element change
// between the k = 2 rule and the others): offsets, count, coordinates and a
// zeroed data buffer of the new size.
vem_status rebuild_bface_points(vem_handle *h, int ppt) {
  cudaStream_t s = h->stream;
  const int T = 128;
  int64_t *cnt = nullptr;
  VEM_TRY(dalloc_n(h, &cnt, (size_t)h->nf + 1));
  count_launch(); k_bq_count<<<grid_for(h->nf, T), T, 0, s>>>(h->nf, ppt, h->fv_ptr, h->fbc, cnt);
  VEM_CUDA(h, cudaGetLastError());
  VEM_TRY(scan_counts(h, h->nf, cnt, h->bqp_off, &h->n_bqp));
  dfree(h, cnt);
  h->bq_ppt = ppt;
  dfree(h, h->bqp_xyz);
  dfree(h, h->gD_qp);
  h->bqp_xyz = nullptr;
  h->gD_qp = nullptr;
  const size_t nq = (size_t)std::max<int64_t>(h->n_bqp, 1);
  VEM_TRY(dalloc_n(h, &h->bqp_xyz, 3 * nq));
  VEM_TRY(dalloc_n(h, &h->gD_qp, nq));
  VEM_CUDA(h, cudaMemsetAsync(h->gD_qp, 0, sizeof(double) * nq, s));
  if (h->n_bqp > 0) {
    count_launch(); k_bface_points<<<grid_for(h->nf, T), T, 0, s>>>(h->nf, ppt, h->fbc, h->bqp_off, h->fv_ptr, h->fv,
                                                                    h->xyz, h->f_cent, h->bqp_xyz);
    VEM_CUDA(h, cudaGetLastError());
  }
  return VEM_OK;
}

}  // namespace vem
