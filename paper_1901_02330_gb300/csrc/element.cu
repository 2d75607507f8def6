// Element-batched local matrices (paper Sec. 4.1-4.3), one warp per cell.
//
// For every cell P the kernels build
//   M_P = nu (Pi^T H Pi + |P| (I - D Pi)^T (I - D Pi))   (a_{h,P} with the
//         dofi-dofi stabilisation s_P of Sec. 4.3),
//   B_P = |P| d                                          (b_{h,P}, P0 pressure)
// where Pi = H^{-1} G is the L2 projection onto [P_kp]^3 (Sec. 4.1, third
// bullet), D the DOFs of the vector monomials and d the divergence of the
// basis functions.  M_P is evaluated as
//   M_P = nu (|P| I - |P| (D Pi + Pi^T D^T) + Pi^T W Pi),  W = H + |P| D^T D,
// so each entry costs three length-12 dot products.
//
// E0: face moments against M_0(f) only, Pi^0_0; closed form with
//   N_f = sigma_f |f| (x_f - x_P), D_f = n_f:  Pi = N^T/|P|, H = |P| I.
// K1 (the paper's k = 1): three face moments (M_1(f)), three cross moments
//   (m_I ^ e_q), Pi^0_1 through the decomposition of Props 2.1-2.3.
#include "handle.cuh"
#include "geom_device.cuh"

namespace vem {

// index of y_a * y_d among the degree <= 2 monomials
// (1, y0, y1, y2, y0^2, y0y1, y0y2, y1^2, y1y2, y2^2); a = 0 means 1
__constant__ int c_prod[4][3] = {{1, 2, 3}, {4, 5, 6}, {5, 7, 8}, {6, 8, 9}};
// H1[a][b] = int m_a m_b -> index into the 10 cell moments
__constant__ int c_h1[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};

__device__ __forceinline__ void upper_decode(int e, int n, int &i, int &j) {
  i = 0;
  while (e >= n - i) {
    e -= n - i;
    ++i;
  }
  j = i + e;
}

// ---------------------------------------------------------------- E0 ----
// One warp per congruence class (its representative cell), nu = 1.
__global__ void k_elem_e0(int64_t ncls, int max_nf, const int64_t *__restrict__ cfp,
                          const int32_t *__restrict__ cf, const int8_t *__restrict__ sig,
                          const double *__restrict__ f_area, const double *__restrict__ f_cent,
                          const double *__restrict__ f_norm, const double *__restrict__ c_vol,
                          const double *__restrict__ c_cent, const int32_t *__restrict__ cls_rep,
                          const int64_t *__restrict__ m_off, const int64_t *__restrict__ b_off,
                          double *Mloc, double *Bloc) {
  extern __shared__ double sm[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double *N = sm + (size_t)warp * (6 * max_nf + 9);
  double *nn = N + 3 * max_nf;
  double *Q = nn + 3 * max_nf;
  for (int64_t kk = (int64_t)blockIdx.x * wpb + warp; kk < ncls; kk += (int64_t)gridDim.x * wpb) {
    const int64_t c = cls_rep[kk];
    const int64_t b = cfp[c];
    const int k = (int)(cfp[c + 1] - b);
    const double vol = c_vol[c], nuc = 1.0, ivol = 1.0 / vol;
    const double3 xP = load3(c_cent, c);
    for (int i = lane; i < k; i += 32) {
      const int f = cf[b + i];
      const double s = (double)sig[b + i] * f_area[f];
      const double3 d = sub3(load3(f_cent, f), xP);
      N[3 * i] = s * d.x;
      N[3 * i + 1] = s * d.y;
      N[3 * i + 2] = s * d.z;
      nn[3 * i] = f_norm[3 * f];
      nn[3 * i + 1] = f_norm[3 * f + 1];
      nn[3 * i + 2] = f_norm[3 * f + 2];
      Bloc[b_off[kk] + i] = s;
    }
    __syncwarp();
    if (lane < 9) {
      const int p = lane / 3, q = lane % 3;
      double t = 0;
      for (int i = 0; i < k; ++i) t += nn[3 * i + p] * nn[3 * i + q];
      Q[lane] = t;
    }
    __syncwarp();
    double *M = Mloc + m_off[kk];
    const int T = k * (k + 1) / 2;
    for (int e = lane; e < T; e += 32) {
      int i, j;
      upper_decode(e, k, i, j);
      const double *Ni = N + 3 * i, *Nj = N + 3 * j, *ni = nn + 3 * i, *nj = nn + 3 * j;
      const double nij = Ni[0] * Nj[0] + Ni[1] * Nj[1] + Ni[2] * Nj[2];
      const double cr = (ni[0] * Nj[0] + ni[1] * Nj[1] + ni[2] * Nj[2]) +
                        (Ni[0] * nj[0] + Ni[1] * nj[1] + Ni[2] * nj[2]);
      double nqn = 0;
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) nqn += Ni[p] * Q[3 * p + q] * Nj[q];
      const double v = nuc * ((nij + nqn) * ivol + (i == j ? vol : 0.0) - cr);
      M[(int64_t)i * k + j] = v;
      M[(int64_t)j * k + i] = v;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- K1 ----
// Work per cell is dominated by FP64 instructions (GB300 issues one FP64 warp
// instruction per 16 cycles per SM whatever the number of active lanes), so
// the kernel spreads every phase over as many lanes as possible:
//  * face integrals G_f = int_f m^f m^f and J_f = int_f m^f m_t (degree <= 3)
//    by an exact degree-3 rule (Strang & Fix 4 points: centroid weight
//    -27/48, (3/5, 1/5, 1/5) orbit weight 25/48) on the fan (v0, v_j, v_j+1)
//    of each (convex) face, one (triangle, point) item per lane;
//  * cell moments int_P m_t from the face integrals by Euler's identity for
//    a homogeneous q of degree d: int_P q = (1/(d+3)) sum_f h_f int_f q, with
//    h_f = (x_f - x_P).n_f^out constant on the planar face;
//  * M_P = nu (|P| I + Pi^T V - |P| D Pi),  V = W Pi - |P| D^T,
//    W = H + |P| D^T D  (two length-12 dots per entry).
// Shared-memory layout per warp (doubles):
//   FG[max_nf][8]   sigma, |f|, n_f (3), 1/|f|, h_f, -
//   FA[max_nf][36]  face Gram G_f (6, then its inverse) and J_f[g][t] (30)
//   MU[10] cell moments int_P m_t, H1I[16], W[144]
//   U[...]          chunk buffer (32 x 36) / Pi (12 x nu), D (nu x 12), V (12 x nu)
// plus ints FO[max_nf + 1] (prefix of quadrature items per face).
__host__ __device__ inline int k1_union(int max_nf) {
  const int nu = 3 * max_nf + 3;
  const int a = 32 * 36, b = 36 * nu;
  return a > b ? a : b;
}
__host__ __device__ inline int k1_doubles(int max_nf) {
  return max_nf * 44 + 10 + 16 + 144 + k1_union(max_nf);
}
__host__ __device__ inline int k1_ints(int max_nf) { return ((max_nf + 2) + 1) & ~1; }

__device__ __forceinline__ void sf3_point(int q, double &l0, double &l1, double &l2, double &w) {
  if (q == 0) {
    l0 = l1 = l2 = 1.0 / 3.0;
    w = -27.0 / 48.0;
  } else {
    l0 = (q == 1) ? 0.6 : 0.2;
    l1 = (q == 2) ? 0.6 : 0.2;
    l2 = (q == 3) ? 0.6 : 0.2;
    w = 25.0 / 48.0;
  }
}

__global__ void k_elem_k1(int64_t ncls, int max_nf, const int64_t *__restrict__ cfp,
                          const int32_t *__restrict__ cf, const int8_t *__restrict__ sig,
                          const int64_t *__restrict__ fvp, const int32_t *__restrict__ fv,
                          const double *__restrict__ xyz, const double *__restrict__ f_area,
                          const double *__restrict__ f_cent, const double *__restrict__ f_norm,
                          const double *__restrict__ f_t1, const double *__restrict__ f_diam,
                          const double *__restrict__ c_cent, const double *__restrict__ c_diam,
                          const int32_t *__restrict__ cls_rep, const int64_t *__restrict__ m_off,
                          const int64_t *__restrict__ b_off, double *Mloc, double *Bloc, int *err) {
  extern __shared__ double sm[];
  const int wpb = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nd = k1_doubles(max_nf);
  double *FG = sm + (size_t)warp * nd;
  double *FA = FG + 8 * max_nf;
  double *MU = FA + 36 * max_nf;
  double *H1I = MU + 10;
  double *W = H1I + 16;
  double *U = W + 144;
  int *FO = reinterpret_cast<int *>(sm + (size_t)wpb * nd) + warp * k1_ints(max_nf);

  for (int64_t kk = (int64_t)blockIdx.x * wpb + warp; kk < ncls; kk += (int64_t)gridDim.x * wpb) {
    const int64_t c = cls_rep[kk];
    const int64_t b = cfp[c];
    const int k = (int)(cfp[c + 1] - b);
    const int nu_l = 3 * k + 3;
    const double3 xP = load3(c_cent, c);
    const double hP = c_diam[c], ihP = 1.0 / hP;
    const double nuc = 1.0;

    // (0) per-face data and the prefix of quadrature items (4 per fan triangle)
    for (int i = lane; i < k; i += 32) {
      const int f = cf[b + i];
      const double sg = (double)sig[b + i];
      const double3 n = load3(f_norm, f);
      FG[8 * i] = sg;
      FG[8 * i + 1] = f_area[f];
      FG[8 * i + 2] = n.x;
      FG[8 * i + 3] = n.y;
      FG[8 * i + 4] = n.z;
      FG[8 * i + 5] = 1.0 / f_area[f];
      FG[8 * i + 6] = sg * dot3(sub3(load3(f_cent, f), xP), n);
    }
    for (int e = lane; e < 36 * k; e += 32) FA[e] = 0.0;
    if (lane == 0) {
      int acc = 0;
      for (int i = 0; i < k; ++i) {
        FO[i] = acc;
        const int f = cf[b + i];
        acc += 4 * (int)(fvp[f + 1] - fvp[f] - 2);
      }
      FO[k] = acc;
    }
    __syncwarp();
    const int T = FO[k];

    // (1) face Gram matrices and face-cell integrals J, one quadrature item
    //     per lane, summed per face in item order.
    for (int base = 0; base < T; base += 32) {
      const int p = base + lane;
      double acc[36];
#pragma unroll
      for (int t = 0; t < 36; ++t) acc[t] = 0.0;
      if (p < T) {
        int i = 0;
        while (FO[i + 1] <= p) ++i;
        const int it = p - FO[i];
        const int j = 1 + (it >> 2), q = it & 3;
        const int f = cf[b + i];
        const int64_t vb = fvp[f];
        const double3 A0 = load3(xyz, fv[vb]);
        const double3 A = load3(xyz, fv[vb + j]);
        const double3 B = load3(xyz, fv[vb + j + 1]);
        const double3 xf = load3(f_cent, f);
        const double3 n = make_double3(FG[8 * i + 2], FG[8 * i + 3], FG[8 * i + 4]);
        const double3 t1 = load3(f_t1, f);
        const double3 t2 = cross3(n, t1);
        const double ihf = 1.0 / f_diam[f];
        const double areaT = 0.5 * dot3(cross3(sub3(A, A0), sub3(B, A0)), n);
        double l0, l1, l2, wq;
        sf3_point(q, l0, l1, l2, wq);
        const double3 x = add3(add3(scale3(A0, l0), scale3(A, l1)), scale3(B, l2));
        const double w = wq * areaT;
        const double3 dx = sub3(x, xf);
        const double s1 = dot3(dx, t1) * ihf, s2 = dot3(dx, t2) * ihf;
        const double mf[3] = {w, w * s1, w * s2};   // weighted face monomials
        const double3 y = scale3(sub3(x, xP), ihP);
        const double m3[10] = {1.0, y.x, y.y, y.z, y.x * y.x, y.x * y.y, y.x * y.z,
                               y.y * y.y, y.y * y.z, y.z * y.z};
        acc[0] = mf[0];
        acc[1] = mf[1];
        acc[2] = mf[2];
        acc[3] = mf[1] * s1;
        acc[4] = mf[1] * s2;
        acc[5] = mf[2] * s2;
#pragma unroll
        for (int g = 0; g < 3; ++g)
#pragma unroll
          for (int t = 0; t < 10; ++t) acc[6 + 10 * g + t] = mf[g] * m3[t];
      }
#pragma unroll
      for (int t = 0; t < 36; ++t) U[36 * lane + t] = acc[t];
      __syncwarp();
      const int hi = base + 32 < T ? base + 32 : T;
      for (int e = lane; e < 36 * k; e += 32) {
        const int i = e / 36, t = e - 36 * i;
        const int lo_p = FO[i] > base ? FO[i] : base;
        const int hi_p = FO[i + 1] < hi ? FO[i + 1] : hi;
        double acc_e = FA[e];
        for (int pp = lo_p; pp < hi_p; ++pp) acc_e += U[36 * (pp - base) + t];
        FA[e] = acc_e;
      }
      __syncwarp();
    }
    // cell moments by Euler's identity: int_P m_t = sum_f h_f int_f m_t / (|t| + 3)
    if (lane < 10) {
      double s = 0.0;
      for (int i = 0; i < k; ++i) s += FG[8 * i + 6] * FA[36 * i + 6 + lane];
      const double deg = (lane == 0) ? 3.0 : ((lane < 4) ? 4.0 : 5.0);
      MU[lane] = s / deg;
    }
    // face Gram inverses (symmetric 3x3 by cofactors)
    for (int i = lane; i < k; i += 32) {
      double *G = FA + 36 * i;
      const double a = G[0], bb = G[1], cc = G[2], d = G[3], e2 = G[4], ff = G[5];
      const double A11 = d * ff - e2 * e2, A12 = -(bb * ff - cc * e2), A13 = bb * e2 - cc * d;
      const double A22 = a * ff - cc * cc, A23 = -(a * e2 - bb * cc), A33 = a * d - bb * bb;
      const double det = a * A11 + bb * A12 + cc * A13;
      if (!(fabs(det) > 0.0) || !isfinite(det)) atomicOr(err, DEVERR_SINGULAR_LOCAL);
      const double id = 1.0 / det;
      G[0] = A11 * id;
      G[1] = A12 * id;
      G[2] = A13 * id;
      G[3] = A22 * id;
      G[4] = A23 * id;
      G[5] = A33 * id;
    }
    __syncwarp();
    // H1 = int m_a m_b (a, b <= 1) inverted by cofactors, one per lane
    {
      double cof = 0.0;
      if (lane < 16) {
        const int ri = lane >> 2, cj = lane & 3;
        int rr[3], cc[3];
        for (int q = 0, t = 0; q < 4; ++q)
          if (q != ri) rr[t++] = q;
        for (int q = 0, t = 0; q < 4; ++q)
          if (q != cj) cc[t++] = q;
        double m[3][3];
        for (int a = 0; a < 3; ++a)
          for (int bq = 0; bq < 3; ++bq) m[a][bq] = MU[c_h1[rr[a]][cc[bq]]];
        const double d3 = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                          m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                          m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
        cof = ((ri + cj) & 1) ? -d3 : d3;
      }
      double det = 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) det += MU[c_h1[0][q]] * __shfl_sync(0xffffffffu, cof, q);
      if (lane == 0 && (!(det > 0.0) || !isfinite(det))) atomicOr(err, DEVERR_SINGULAR_LOCAL);
      const double idet = 1.0 / det;
      if (lane < 16) H1I[4 * (lane & 3) + (lane >> 2)] = cof * idet;
    }
    __syncwarp();

    const double vol = MU[0], ivol = 1.0 / vol;
    double *PI = U;                      // [12][nu_l]
    double *DD = U + 12 * nu_l;          // [nu_l][12]
    double *VV = DD + 12 * nu_l;         // [12][nu_l]
    const int nfl = 3 * k;
    const int64_t boff = b_off[kk];

    // (2)-(3) columns j of G, D and B; Pi[:, j] = blockdiag(H1^{-1}) G[:, j]
    for (int j = lane; j < nu_l; j += 32) {
      double Gc[12], Dr[12], Bj = 0.0;
      if (j < nfl) {
        const int i = j / 3, beta = j - 3 * (j / 3);
        const double sa = FG[8 * i] * FG[8 * i + 1], iar = FG[8 * i + 5];
        const double *Gi = FA + 36 * i;
        const double *J = Gi + 6;
        const double gb[3] = {beta == 0 ? Gi[0] : (beta == 1 ? Gi[1] : Gi[2]),
                              beta == 0 ? Gi[1] : (beta == 1 ? Gi[3] : Gi[4]),
                              beta == 0 ? Gi[2] : (beta == 1 ? Gi[4] : Gi[5])};
        double bnd[10];
#pragma unroll
        for (int t = 0; t < 10; ++t) bnd[t] = sa * (gb[0] * J[t] + gb[1] * J[10 + t] + gb[2] * J[20 + t]);
        const double dv = bnd[0] * ivol;     // div(phi_j), constant
        Bj = bnd[0];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          // int phi . grad m_beta by parts, beta = e_c (a = 0) or e_d + e_c (a = 1 + d)
          const int t0 = 1 + cc;
          Gc[4 * cc] = hP * (bnd[t0] - dv * MU[t0]);
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const int t = c_prod[1 + d][cc];
            Gc[4 * cc + 1 + d] = 0.5 * hP * (bnd[t] - dv * MU[t]);
          }
          const double nci = FG[8 * i + 2 + cc] * iar;
#pragma unroll
          for (int a = 0; a < 4; ++a) Dr[4 * cc + a] = nci * J[10 * beta + a];
        }
      } else {
        const int q = j - nfl;
#pragma unroll
        for (int t = 0; t < 12; ++t) Gc[t] = 0.0;
        // Props 2.1-2.3 at degree 1: the m_I ^ e_q coefficients
        if (q == 2) { Gc[0 * 4 + 2] = 0.5 * vol; Gc[1 * 4 + 1] = -0.5 * vol; }
        if (q == 1) { Gc[0 * 4 + 3] = -0.5 * vol; Gc[2 * 4 + 1] = 0.5 * vol; }
        if (q == 0) { Gc[1 * 4 + 3] = 0.5 * vol; Gc[2 * 4 + 2] = -0.5 * vol; }
        // D: (1/|P|) int m_a (m_I ^ e_q)_c
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          int dsel = -1;
          double sgn = 0.0;
          if (q == 0) { if (cc == 1) { dsel = 2; sgn = 1.0; } else if (cc == 2) { dsel = 1; sgn = -1.0; } }
          if (q == 1) { if (cc == 0) { dsel = 2; sgn = -1.0; } else if (cc == 2) { dsel = 0; sgn = 1.0; } }
          if (q == 2) { if (cc == 0) { dsel = 1; sgn = 1.0; } else if (cc == 1) { dsel = 0; sgn = -1.0; } }
#pragma unroll
          for (int a = 0; a < 4; ++a)
            Dr[4 * cc + a] = (dsel < 0) ? 0.0 : sgn * MU[c_prod[a][dsel]] * ivol;
        }
      }
#pragma unroll
      for (int cc = 0; cc < 3; ++cc)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          double s = 0.0;
#pragma unroll
          for (int t = 0; t < 4; ++t) s += H1I[4 * r + t] * Gc[4 * cc + t];
          PI[(4 * cc + r) * nu_l + j] = s;
        }
#pragma unroll
      for (int v = 0; v < 12; ++v) DD[12 * j + v] = Dr[v];
      Bloc[boff + j] = Bj;
    }
    __syncwarp();
    // W = H + |P| D^T D (symmetric, entries v <= w computed once)
    for (int e = lane; e < 78; e += 32) {
      int v, w;
      upper_decode(e, 12, v, w);
      double s = 0.0;
      for (int j = 0; j < nu_l; ++j) s += DD[12 * j + v] * DD[12 * j + w];
      const double hv = (v / 4 == w / 4) ? MU[c_h1[v % 4][w % 4]] : 0.0;
      const double val = hv + vol * s;
      W[12 * v + w] = val;
      W[12 * w + v] = val;
    }
    __syncwarp();
    // V = W Pi - |P| D^T, one (row v, column j) entry per lane
    for (int e = lane; e < 12 * nu_l; e += 32) {
      const int v = e / nu_l, j = e - v * nu_l;
      double s = -vol * DD[12 * j + v];
#pragma unroll
      for (int w = 0; w < 12; ++w) s += W[12 * v + w] * PI[w * nu_l + j];
      VV[e] = s;
    }
    __syncwarp();
    // (4) M_P entries: nu (|P| delta + Pi_j . V_j' - |P| D_j . Pi_j'), j <= j'
    double *M = Mloc + m_off[kk];
    const int TT = nu_l * (nu_l + 1) / 2;
    for (int e = lane; e < TT; e += 32) {
      int j, jp;
      upper_decode(e, nu_l, j, jp);
      double pv = 0.0, dp = 0.0;
#pragma unroll
      for (int v = 0; v < 12; ++v) {
        pv += PI[v * nu_l + j] * VV[v * nu_l + jp];
        dp += DD[12 * j + v] * PI[v * nu_l + jp];
      }
      const double val = nuc * ((j == jp ? vol : 0.0) + pv - vol * dp);
      M[(int64_t)j * nu_l + jp] = val;
      M[(int64_t)jp * nu_l + j] = val;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------- loads ----
// F_P = |P| f(x_P) (midpoint rule at the barycentre).
__global__ void k_rhs_cells(int64_t nc, const double *__restrict__ c_vol,
                            const double *__restrict__ f_qp, double *F, int *err) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const double fv = f_qp ? f_qp[c] : 0.0;
    if (!isfinite(fv)) atomicOr(err, DEVERR_NONFINITE);
    F[c] = c_vol[c] * fv;
  }
}

// g_(f,beta) = -sigma |f| sum_g Ginv[g][beta] int_f g_D m^f_g on Dirichlet
// faces (zero elsewhere), with the Dunavant fan rule of the bface points.
__global__ void k_rhs_faces(int64_t nbf, const int32_t *__restrict__ bface, int ppt, int nfd,
                            const int8_t *__restrict__ fbc,
                            const int64_t *__restrict__ off, const int64_t *__restrict__ fvp,
                            const int32_t *__restrict__ fv, const double *__restrict__ xyz,
                            const double *__restrict__ f_area, const double *__restrict__ f_cent,
                            const double *__restrict__ f_norm, const double *__restrict__ f_t1,
                            const double *__restrict__ f_diam, const int32_t *__restrict__ f_cell,
                            const int32_t *__restrict__ f_loc, const int64_t *__restrict__ cfp,
                            const int8_t *__restrict__ sig, const double *__restrict__ gD, double *g,
                            int *err) {
  // boundary faces only (g is zeroed beforehand)
  for (int64_t ib = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ib < nbf;
       ib += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = bface[ib];
    if (fbc[f] != 1 || gD == nullptr) continue;
    const int64_t vb = fvp[f];
    const int m = (int)(fvp[f + 1] - vb);
    const double3 xf = load3(f_cent, f);
    const double3 n = load3(f_norm, f);
    const double3 t1 = load3(f_t1, f);
    const double3 t2 = cross3(n, t1);
    const double ihf = 1.0 / f_diam[f];
    const double sg = (double)sig[cfp[f_cell[2 * f]] + f_loc[2 * f]];
    double G[6] = {0, 0, 0, 0, 0, 0}, gm[3] = {0, 0, 0};
    int64_t o = off[f];
    for (int i = 0; i < m; ++i) {
      const double3 A = load3(xyz, fv[vb + i]);
      const double3 B = load3(xyz, fv[vb + (i + 1) % m]);
      const double areaT = 0.5 * dot3(cross3(sub3(A, xf), sub3(B, xf)), n);
      for (int q = 0; q < ppt; ++q, ++o) {
        double l0, l1, l2, wq;
        bface_point(ppt, q, l0, l1, l2, wq);
        const double3 x = add3(add3(scale3(xf, l0), scale3(A, l1)), scale3(B, l2));
        const double w = wq * areaT;
        const double3 dx = sub3(x, xf);
        const double mf[3] = {1.0, dot3(dx, t1) * ihf, dot3(dx, t2) * ihf};
        const double gv = gD[o];
        if (!isfinite(gv)) atomicOr(err, DEVERR_NONFINITE);
        G[0] += w * mf[0] * mf[0];
        G[1] += w * mf[0] * mf[1];
        G[2] += w * mf[0] * mf[2];
        G[3] += w * mf[1] * mf[1];
        G[4] += w * mf[1] * mf[2];
        G[5] += w * mf[2] * mf[2];
        gm[0] += w * gv * mf[0];
        gm[1] += w * gv * mf[1];
        gm[2] += w * gv * mf[2];
      }
    }
    const double ar = f_area[f];
    if (nfd == 1) {
      g[f] = -sg * gm[0];
    } else {
      const double a = G[0], bb = G[1], cc = G[2], d = G[3], e = G[4], ff = G[5];
      const double A11 = d * ff - e * e, A12 = -(bb * ff - cc * e), A13 = bb * e - cc * d;
      const double A22 = a * ff - cc * cc, A23 = -(a * e - bb * cc), A33 = a * d - bb * bb;
      const double id = 1.0 / (a * A11 + bb * A12 + cc * A13);
      const double Gi[3][3] = {{A11 * id, A12 * id, A13 * id},
                               {A12 * id, A22 * id, A23 * id},
                               {A13 * id, A23 * id, A33 * id}};
      for (int bta = 0; bta < 3; ++bta)
        g[3 * f + bta] = -sg * ar * (Gi[0][bta] * gm[0] + Gi[1][bta] * gm[1] + Gi[2][bta] * gm[2]);
    }
  }
}

static int warps_per_block(size_t bytes_per_warp, size_t limit = 96 * 1024) {
  int w = (int)(limit / bytes_per_warp);
  if (w > 8) w = 8;
  if (w < 1) w = 1;
  return w;
}

// Geometry-only local matrices (nu = 1), one per congruence class.
vem_status assemble_local(vem_handle *h) {
  cudaStream_t s = h->stream;
  const int mx = h->max_nf_cell;
  const int64_t ncls = h->ncls;
  if (h->opt.element == VEM_ELEMENT_E0) {
    const size_t bpw = sizeof(double) * (6 * mx + 9);
    if (bpw > 200 * 1024) return fail(h, VEM_ERR_UNSUPPORTED, "cell with %d faces", mx);
    const int wpb = warps_per_block(bpw);
    const size_t smem = bpw * wpb;
    VEM_CUDA(h, cudaFuncSetAttribute(k_elem_e0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t blocks = (ncls + wpb - 1) / wpb;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    count_launch();
    k_elem_e0<<<(int)blocks, 32 * wpb, smem, s>>>(ncls, mx, h->cf_ptr, h->cf, h->cf_sigma, h->f_area, h->f_cent,
                                                   h->f_norm, h->c_vol, h->c_cent, h->cls_rep, h->m_off,
                                                   h->b_off, h->Mloc, h->Bloc);
    VEM_CUDA(h, cudaGetLastError());
  } else if (h->opt.element == VEM_ELEMENT_K1) {
    const size_t bpw = sizeof(double) * k1_doubles(mx) + sizeof(int) * k1_ints(mx);
    if (bpw > 200 * 1024) return fail(h, VEM_ERR_UNSUPPORTED, "cell with %d faces", mx);
    const int wpb = warps_per_block(bpw);
    const size_t smem = bpw * wpb;
    VEM_CUDA(h, cudaFuncSetAttribute(k_elem_k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t blocks = (ncls + wpb - 1) / wpb;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    count_launch();
    k_elem_k1<<<(int)blocks, 32 * wpb, smem, s>>>(
        ncls, mx, h->cf_ptr, h->cf, h->cf_sigma, h->fv_ptr, h->fv, h->xyz, h->f_area, h->f_cent, h->f_norm,
        h->f_t1, h->f_diam, h->c_cent, h->c_diam, h->cls_rep, h->m_off, h->b_off, h->Mloc, h->Bloc, h->d_err);
    VEM_CUDA(h, cudaGetLastError());
  } else if (h->opt.element == VEM_ELEMENT_K2) {
    VEM_TRY(element_k2(h));
  } else {
    return fail(h, VEM_ERR_UNSUPPORTED, "element %d", h->opt.element);
  }
  return check_device_errors(h, "element matrices");
}

// Prescribed face DOFs on flux faces (flag 2): (f, beta) = (1/|f|) int_f
// (u.n_f) m^f_beta with u.n_f = sigma u_N (u_N given along the outward
// normal), by the Dunavant fan rule of the bface points; zero elsewhere.
__global__ void k_flux_fixed(int64_t nbf, const int32_t *__restrict__ bface, int ppt, int nfd,
                             const int8_t *__restrict__ fbc,
                             const int64_t *__restrict__ off, const int64_t *__restrict__ fvp,
                             const int32_t *__restrict__ fv, const double *__restrict__ xyz,
                             const double *__restrict__ f_area, const double *__restrict__ f_cent,
                             const double *__restrict__ f_norm, const double *__restrict__ f_t1,
                             const double *__restrict__ f_diam, const int32_t *__restrict__ f_cell,
                             const int32_t *__restrict__ f_loc, const int64_t *__restrict__ cfp,
                             const int8_t *__restrict__ sig, const double *__restrict__ uN, double *xfix,
                             int *err) {
  // boundary faces only (the caller zeroes xfix)
  for (int64_t ib = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ib < nbf;
       ib += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = bface[ib];
    if (fbc[f] != 2 || uN == nullptr) continue;
    const int64_t vb = fvp[f];
    const int m = (int)(fvp[f + 1] - vb);
    const double3 xf = load3(f_cent, f);
    const double3 n = load3(f_norm, f);
    const double3 t1 = load3(f_t1, f);
    const double3 t2 = cross3(n, t1);
    const double ihf = 1.0 / f_diam[f];
    const double sg = (double)sig[cfp[f_cell[2 * f]] + f_loc[2 * f]];
    double mom[6] = {0, 0, 0, 0, 0, 0};
    int64_t o = off[f];
    for (int i = 0; i < m; ++i) {
      const double3 A = load3(xyz, fv[vb + i]);
      const double3 B = load3(xyz, fv[vb + (i + 1) % m]);
      const double areaT = 0.5 * dot3(cross3(sub3(A, xf), sub3(B, xf)), n);
      for (int q = 0; q < ppt; ++q, ++o) {
        double l0, l1, l2, wq;
        bface_point(ppt, q, l0, l1, l2, wq);
        const double3 x = add3(add3(scale3(xf, l0), scale3(A, l1)), scale3(B, l2));
        const double w = wq * areaT;
        const double3 dx = sub3(x, xf);
        const double fs = dot3(dx, t1) * ihf, ft = dot3(dx, t2) * ihf;
        // face monomials of M_2(f): 1, s, t, s^2, s t, t^2 (the first nfd)
        const double mf[6] = {1.0, fs, ft, fs * fs, fs * ft, ft * ft};
        const double un = uN[o];
        if (!isfinite(un)) atomicOr(err, DEVERR_NONFINITE);
        for (int bta = 0; bta < nfd; ++bta) mom[bta] += w * un * mf[bta];
      }
    }
    const double ia = 1.0 / f_area[f];
    for (int bta = 0; bta < nfd; ++bta) xfix[nfd * f + bta] = sg * mom[bta] * ia;
  }
}

vem_status flux_fixed(vem_handle *h, double *xfix) {
  count_launch();
  k_flux_fixed<<<grid_for(h->n_bface, 128), 128, 0, h->stream>>>(
      h->n_bface, h->bface, h->bq_ppt, h->nfd, h->fbc, h->bqp_off, h->fv_ptr, h->fv, h->xyz, h->f_area,
      h->f_cent, h->f_norm, h->f_t1, h->f_diam, h->f_cell, h->f_loc, h->cf_ptr, h->cf_sigma, h->gD_qp, xfix,
      h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

vem_status assemble_rhs_into(vem_handle *h, const double *f_qp, const double *gD_qp, double *g, double *F) {
  if (h->nq > 1) return assemble_rhs_k2(h, f_qp, gD_qp, g, F);
  cudaStream_t s = h->stream;
  const int T = 128;
  VEM_CUDA(h, cudaMemsetAsync(g, 0, sizeof(double) * h->nfd * h->nf, s));
  count_launch(); k_rhs_faces<<<grid_for(h->n_bface, T), T, 0, s>>>(
      h->n_bface, h->bface, h->bq_ppt, h->nfd, h->fbc, h->bqp_off, h->fv_ptr, h->fv, h->xyz, h->f_area,
      h->f_cent, h->f_norm, h->f_t1, h->f_diam, h->f_cell, h->f_loc, h->cf_ptr, h->cf_sigma, gD_qp, g, h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  if (h->nid > 0)
    VEM_CUDA(h, cudaMemsetAsync(g + h->nfd * h->nf, 0, sizeof(double) * h->nid * h->nc, s));
  count_launch(); k_rhs_cells<<<grid_for(h->nc, T), T, 0, s>>>(h->nc, h->c_vol, f_qp, F, h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

vem_status assemble_rhs(vem_handle *h) {
  VEM_TRY(assemble_rhs_into(h, h->f_qp, h->gD_qp, h->rhs, h->rhs + h->n_u));
  VEM_TRY(neumann_rhs(h, h->rhs));   // prescribed flux DOFs and the multiplier
  VEM_TRY(check_device_errors(h, "right-hand side"));
  h->rhs_ready = true;
  return VEM_OK;
}

}  // namespace vem
