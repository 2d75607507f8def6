// Local matrices of the paper's k = 2 element (Sec. 4.1-4.3 at k = 2), one
// block per congruence class (its representative cell), nu = 1:
//   face DOFs      (1/|f|) int_f (v.n_f) m^f_beta, beta in M_2(f)   (6 per face)
//   gradient DOFs  (h_P/|P|) int_P v . grad m_a, |a| = 1             (3)
//   cross DOFs     (1/|P|) int_P v . (m_I ^ e_c m_g), (c, g) in
//                  M^{G,+}_1 (Sec. 2.2)                             (11)
//   pressure       P1 moments                                        (4)
// and, as for k = 1 (element.cu),
//   M_P = |P| I - |P| (D Pi + Pi^T D^T) + Pi^T W Pi,  W = H + |P| D^T D,
//   B_P = |P| d,
// with Pi the L2 projection onto [P_2]^3 (Pi = H^-1 G, G from the
// decomposition [P_2]^3 = grad P_3 (+) m_I ^ [P_1]^3 of Props 2.1-2.4),
// D the DOFs of the vector monomials and d the divergence coefficients
// (H_1 d = r in P_1).
//
// Every integral is of a polynomial: face integrals by the 7-point degree-5
// rule of Radon (1948) on the fan triangles (x_f, v_j, v_j+1); cell
// integrals of monomials through the divergence theorem,
//   int_P m_a = h_P / (3 + |a|) sum_f ((x_f - x_P) . n_f / h_P) int_f m_a,
// (m_a homogeneous of degree |a| in (x - x_P)/h_P), so only face points are
// needed.  Matrices live in shared memory; the dense solves (6x6 face Gram,
// 10x10 H, 4x4 H_1) are Gauss-Jordan on symmetric positive definite
// matrices.
#include <cmath>
#include <cstring>

#include "geom_device.cuh"
#include "handle.cuh"

namespace vem {

namespace {

constexpr int kT = 20;        // test monomials: degree <= 3
constexpr int kMom = 35;      // cell moments: degree <= 4
constexpr int kV = 30;        // vector monomials [P_2]^3
constexpr int kGr = 19;       // gradients: 1 <= |b| <= 3
constexpr int kCr = 11;       // cross DOFs
constexpr int kNid = 14;      // interior DOFs
constexpr int kNfd = 6;       // face DOFs
constexpr int kNq = 4;        // pressure DOFs
constexpr int kThreads = 256;

struct K2Tables {
  int p3[kT][3];              // multi-indices of degree <= 3 (degree order)
  int idx4[5][5][5];          // index of a multi-index of degree <= 4 among kMom
  int a_beta[kV];             // grad m_b of e_c m_a: index of b = a + e_c among the gradients
  double a_coef[kV];          // its coefficient / h_P = 1 / (|a| + 1)
  double c_coef[kV][kCr];     // coefficients of m_I ^ e_comp m_g
  int cr_comp[kCr], cr_g[kCr];   // cross DOF (component, index of g among P_1)
};

__constant__ K2Tables c_k2;

inline int deg(const int a[3]) { return a[0] + a[1] + a[2]; }

// Decomposition of e_c m_a (Props 2.1-2.3): with s = |a| + 1,
//   e_x m_a = (h/s) grad m_{a+e1} - (a3/s) m_I^(0,m_{a-e3},0) + (a2/s) m_I^(0,0,m_{a-e2})
//   e_y m_a = (h/s) grad m_{a+e2} - (a1/s) m_I^(0,0,m_{a-e1}) + (a3/s) m_I^(m_{a-e3},0,0)
//   e_z m_a = (h/s) grad m_{a+e3} - (a2/s) m_I^(m_{a-e2},0,0) + (a1/s) m_I^(0,m_{a-e1},0)
// and an x-component term m_I^(m_g,0,0) with g_1 > 0 (outside N_1) is
// rewritten by Prop 2.4 as -m_I^(0,m_{g-e1+e2},0) - m_I^(0,0,m_{g-e1+e3}).
K2Tables make_tables() {
  K2Tables t;
  std::memset(&t, 0, sizeof(t));
  int n = 0;
  for (int d = 0; d <= 3; ++d)
    for (int a1 = d; a1 >= 0; --a1)
      for (int a2 = d - a1; a2 >= 0; --a2) {
        t.p3[n][0] = a1;
        t.p3[n][1] = a2;
        t.p3[n][2] = d - a1 - a2;
        ++n;
      }
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j)
      for (int k = 0; k < 5; ++k) t.idx4[i][j][k] = -1;
  n = 0;
  for (int d = 0; d <= 4; ++d)
    for (int a1 = d; a1 >= 0; --a1)
      for (int a2 = d - a1; a2 >= 0; --a2) t.idx4[a1][a2][d - a1 - a2] = n++;
  // cross DOFs: x-component over N_1 = {a in P_1 : a_1 = 0}, then y and z over P_1
  int m = 0;
  const int p1_n[3] = {0, 2, 3};   // (000), (010), (001) among the P_3 list
  for (int i = 0; i < 3; ++i) {
    t.cr_comp[m] = 0;
    t.cr_g[m++] = p1_n[i];
  }
  for (int c = 1; c < 3; ++c)
    for (int i = 0; i < 4; ++i) {
      t.cr_comp[m] = c;
      t.cr_g[m++] = i;
    }
  auto p1_index = [&](int g1, int g2, int g3) {
    for (int i = 0; i < 4; ++i)
      if (t.p3[i][0] == g1 && t.p3[i][1] == g2 && t.p3[i][2] == g3) return i;
    return -1;
  };
  auto cross_slot = [&](int comp, int gi) {
    for (int i = 0; i < kCr; ++i)
      if (t.cr_comp[i] == comp && t.cr_g[i] == gi) return i;
    return -1;
  };
  auto add_cross = [&](int r, int comp, int g1, int g2, int g3, double coef) {
    if (coef == 0.0) return;
    if (comp == 0 && g1 > 0) {
      t.c_coef[r][cross_slot(1, p1_index(g1 - 1, g2 + 1, g3))] -= coef;
      t.c_coef[r][cross_slot(2, p1_index(g1 - 1, g2, g3 + 1))] -= coef;
    } else {
      t.c_coef[r][cross_slot(comp, p1_index(g1, g2, g3))] += coef;
    }
  };
  for (int c = 0; c < 3; ++c)
    for (int ai = 0; ai < 10; ++ai) {
      const int r = c * 10 + ai;
      const int *a = t.p3[ai];
      const double s = deg(a) + 1.0;
      int b[3] = {a[0], a[1], a[2]};
      b[c] += 1;
      for (int g = 1; g < kT; ++g)
        if (t.p3[g][0] == b[0] && t.p3[g][1] == b[1] && t.p3[g][2] == b[2]) t.a_beta[r] = g - 1;
      t.a_coef[r] = 1.0 / s;
      if (c == 0) {
        add_cross(r, 1, a[0], a[1], a[2] - 1, -a[2] / s);
        add_cross(r, 2, a[0], a[1] - 1, a[2], a[1] / s);
      } else if (c == 1) {
        add_cross(r, 2, a[0] - 1, a[1], a[2], -a[0] / s);
        add_cross(r, 0, a[0], a[1], a[2] - 1, a[2] / s);
      } else {
        add_cross(r, 0, a[0], a[1] - 1, a[2], -a[1] / s);
        add_cross(r, 1, a[0] - 1, a[1], a[2], a[0] / s);
      }
    }
  return t;
}

__device__ __forceinline__ double ipow(double x, int p) {
  double r = 1.0;
  for (int i = 0; i < p; ++i) r *= x;
  return r;
}

// In-place Gauss-Jordan inverse of an SPD n x n matrix (row-major), one thread.
__device__ void gj_inverse(double *A, int n) {
  for (int k = 0; k < n; ++k) {
    const double ip = 1.0 / A[k * n + k];
    for (int c = 0; c < n; ++c)
      if (c != k) A[k * n + c] *= ip;
    for (int r = 0; r < n; ++r) {
      if (r == k) continue;
      const double f = A[r * n + k];
      for (int c = 0; c < n; ++c)
        if (c != k) A[r * n + c] -= f * A[k * n + c];
      A[r * n + k] = -f * ip;
    }
    A[k * n + k] = ip;
  }
}

}  // namespace

size_t k2_smem_doubles(int max_nf, int max_nv) {
  const size_t nu = (size_t)kNfd * max_nf + kNid;
  const size_t nq = 7 * (size_t)max_nv;
  return 133 * nu + 6 * nq + 120 + 35 + 36 + kMom + 100 + 16 + 4 * kGr + 900 + 8;
}

__global__ void __launch_bounds__(kThreads) k_elem_k2(
    int64_t ncls, int max_nf, int max_nv, const int64_t *__restrict__ cfp, const int32_t *__restrict__ cf,
    const int8_t *__restrict__ sig, const int64_t *__restrict__ fvp, const int32_t *__restrict__ fv,
    const double *__restrict__ xyz, const double *__restrict__ f_area, const double *__restrict__ f_cent,
    const double *__restrict__ f_norm, const double *__restrict__ f_t1, const double *__restrict__ f_diam,
    const double *__restrict__ c_vol, const double *__restrict__ c_cent, const double *__restrict__ c_diam,
    const int32_t *__restrict__ cls_rep, const int64_t *__restrict__ m_off, const int64_t *__restrict__ b_off,
    double *Mloc, double *Bloc, double *hq_inv, double *pm_hat, int *err) {
  extern __shared__ double sm[];
  const int NUmax = kNfd * max_nf + kNid;
  const int NQmax = 7 * max_nv;
  double *bnd = sm;                       // kT x NU
  double *dd = bnd + kT * NUmax;          // kNq x NU
  double *GI = dd + kNq * NUmax;          // kGr x NU
  double *G = GI + kGr * NUmax;           // kV x NU
  double *Pi = G + kV * NUmax;            // kV x NU
  double *D = Pi + kV * NUmax;            // NU x kV
  double *WPi = bnd;                      // kV x NU, reuses bnd, dd, GI once G is formed
  double *qp = D + kV * NUmax;            // face points: y (3), s, t, w
  double *Jf = qp + 6 * NQmax;            // kNfd x kT
  double *Fm = Jf + 120;                  // kMom face integrals of the cell monomials
  double *Gf = Fm + 35;                   // 6 x 6 face Gram, then its inverse
  double *mu = Gf + 36;                   // kMom cell moments
  double *Hp = mu + kMom;                 // 10 x 10, inverted in place
  double *Hq = Hp + 100;                  // 4 x 4, inverted in place
  double *Hqt = Hq + 16;                  // kNq x kGr: int m_g m_b
  double *W = Hqt + 4 * kGr;              // kV x kV
  const int tid = threadIdx.x;

  for (int64_t k = blockIdx.x; k < ncls; k += gridDim.x) {
    const int64_t c = cls_rep[k];
    const int64_t b = cfp[c];
    const int nfc = (int)(cfp[c + 1] - b);
    const int NU = kNfd * nfc + kNid;
    const double3 xP = load3(c_cent, c);
    const double hP = c_diam[c], vol = c_vol[c], ihP = 1.0 / hP;
    if (tid < kMom) mu[tid] = 0.0;
    __syncthreads();

    // ---- faces: Gram matrix, moments against the test monomials, cell-moment terms
    for (int i = 0; i < nfc; ++i) {
      const int f = cf[b + i];
      const int64_t vb = fvp[f];
      const int m = (int)(fvp[f + 1] - vb);
      const double3 xf = load3(f_cent, f), nf = load3(f_norm, f), t1 = load3(f_t1, f);
      const double3 t2 = cross3(nf, t1);
      const double ihf = 1.0 / f_diam[f];
      const double sg = (double)sig[b + i];
      const int np = 7 * m;
      for (int p = tid; p < np; p += blockDim.x) {
        const int tri = p / 7, q = p - 7 * tri;
        const double3 A = load3(xyz, fv[vb + tri]);
        const double3 B = load3(xyz, fv[vb + (tri + 1) % m]);
        const double areaT = 0.5 * dot3(cross3(sub3(A, xf), sub3(B, xf)), nf);
        double l0, l1, l2, wq;
        radon7_point(q, l0, l1, l2, wq);
        const double3 x = add3(add3(scale3(xf, l0), scale3(A, l1)), scale3(B, l2));
        const double3 y = scale3(sub3(x, xP), ihP);
        const double3 dx = sub3(x, xf);
        double *o = qp + 6 * p;
        o[0] = y.x;
        o[1] = y.y;
        o[2] = y.z;
        o[3] = dot3(dx, t1) * ihf;
        o[4] = dot3(dx, t2) * ihf;
        o[5] = wq * areaT;
      }
      __syncthreads();
      // accumulators: 35 monomial integrals, 6 x 20 face-test products, 21 Gram entries
      for (int a = tid; a < kMom + 120 + 21; a += blockDim.x) {
        double acc = 0.0;
        if (a < kMom) {
          // a-th monomial of degree <= 4 (degree order)
          int e[3] = {0, 0, 0}, cnt = 0;
          for (int d = 0; d <= 4; ++d)
            for (int a1 = d; a1 >= 0; --a1)
              for (int a2 = d - a1; a2 >= 0; --a2) {
                if (cnt == a) {
                  e[0] = a1;
                  e[1] = a2;
                  e[2] = d - a1 - a2;
                }
                ++cnt;
              }
          for (int p = 0; p < np; ++p) {
            const double *o = qp + 6 * p;
            acc += o[5] * ipow(o[0], e[0]) * ipow(o[1], e[1]) * ipow(o[2], e[2]);
          }
          Fm[a] = acc;
        } else if (a < kMom + 120) {
          const int bt = (a - kMom) / kT, t = (a - kMom) % kT;
          const int fb[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};
          for (int p = 0; p < np; ++p) {
            const double *o = qp + 6 * p;
            acc += o[5] * ipow(o[3], fb[bt][0]) * ipow(o[4], fb[bt][1]) * ipow(o[0], c_k2.p3[t][0]) *
                   ipow(o[1], c_k2.p3[t][1]) * ipow(o[2], c_k2.p3[t][2]);
          }
          Jf[bt * kT + t] = acc;
        } else {
          int e = a - kMom - 120, r = 0;
          while (e >= 6 - r) {
            e -= 6 - r;
            ++r;
          }
          const int s2 = r + e;
          const int fb[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};
          for (int p = 0; p < np; ++p) {
            const double *o = qp + 6 * p;
            acc += o[5] * ipow(o[3], fb[r][0] + fb[s2][0]) * ipow(o[4], fb[r][1] + fb[s2][1]);
          }
          Gf[r * 6 + s2] = acc;
          Gf[s2 * 6 + r] = acc;
        }
      }
      __syncthreads();
      // cell moments (divergence theorem) and the inverse face Gram matrix
      const double hn = sg * dot3(sub3(xf, xP), nf) * ihP;   // (x_f - x_P) . n_out / h_P
      if (tid < kMom) {
        int d = 0;
        for (int dd2 = 0, cnt = 0; dd2 <= 4; ++dd2) {
          const int len = (dd2 + 1) * (dd2 + 2) / 2;
          if (tid < cnt + len) {
            d = dd2;
            break;
          }
          cnt += len;
        }
        mu[tid] += hP / (3.0 + d) * hn * Fm[tid];
      }
      if (tid == 0) gj_inverse(Gf, 6);
      __syncthreads();
      // face block of bnd: sigma |f| (Jf^T Ginv); face rows of D
      const double ar = f_area[f];
      for (int e = tid; e < kT * kNfd; e += blockDim.x) {
        const int t = e / kNfd, bt = e % kNfd;
        double s = 0.0;
        for (int g = 0; g < kNfd; ++g) s += Jf[g * kT + t] * Gf[g * 6 + bt];
        bnd[t * NUmax + i * kNfd + bt] = sg * ar * s;
      }
      for (int e = tid; e < kNfd * kV; e += blockDim.x) {
        const int bt = e / kV, r = e % kV;
        const int cc = r / 10, a = r % 10;
        D[(i * kNfd + bt) * kV + r] = comp3(nf, cc) * Jf[bt * kT + a] / ar;
      }
      __syncthreads();
    }

    // ---- cell: Gram matrices from the moments
    auto mom = [&](int a1, int a2, int a3) { return mu[c_k2.idx4[a1][a2][a3]]; };
    for (int e = tid; e < 100; e += blockDim.x) {
      const int a = e / 10, bb = e % 10;
      Hp[e] = mom(c_k2.p3[a][0] + c_k2.p3[bb][0], c_k2.p3[a][1] + c_k2.p3[bb][1], c_k2.p3[a][2] + c_k2.p3[bb][2]);
    }
    for (int e = tid; e < 16; e += blockDim.x) {
      const int a = e / 4, bb = e % 4;
      Hq[e] = mom(c_k2.p3[a][0] + c_k2.p3[bb][0], c_k2.p3[a][1] + c_k2.p3[bb][1], c_k2.p3[a][2] + c_k2.p3[bb][2]);
    }
    for (int e = tid; e < 4 * kGr; e += blockDim.x) {
      const int g = e / kGr, bb = e % kGr + 1;
      Hqt[e] = mom(c_k2.p3[g][0] + c_k2.p3[bb][0], c_k2.p3[g][1] + c_k2.p3[bb][1], c_k2.p3[g][2] + c_k2.p3[bb][2]);
    }
    // interior columns of bnd are zero (the interior DOFs have no trace)
    for (int e = tid; e < kT * kNid; e += blockDim.x) bnd[(e / kNid) * NUmax + kNfd * nfc + e % kNid] = 0.0;
    __syncthreads();
    // pressure DOFs (1/|P|) int q m_a of the fields q = 1 and q = x_j - x_P,j
    // (translation invariant; the near-null space of S for the point-block AMG)
    if (pm_hat && tid < 16) {
      const int a = tid / 4, j = tid % 4;
      pm_hat[16 * k + tid] = (j == 0 ? Hq[a] : hP * Hq[j * 4 + a]) / vol;
    }
    __syncthreads();
    if (tid == 0) gj_inverse(Hp, 10);
    if (tid == 32) gj_inverse(Hq, 4);
    __syncthreads();
    if (hq_inv && tid < 16) hq_inv[16 * k + tid] = vol * Hq[tid];   // load map F = |P| H_1^-1 int f m
    const int gcol0 = kNfd * nfc, ccol0 = gcol0 + 3;
    // divergence coefficients d = H_1^-1 r, r_0 = bnd_0, r_a = bnd_a - (|P|/h_P) e_{grad a}
    for (int e = tid; e < kNq * NU; e += blockDim.x) {
      const int q = e / NU, j = e % NU;
      double s = 0.0;
      for (int a = 0; a < kNq; ++a) {
        double r = bnd[a * NUmax + j];
        if (a >= 1 && j == gcol0 + (a - 1)) r -= vol * ihP;
        s += Hq[q * 4 + a] * r;
      }
      dd[q * NUmax + j] = s;
      Bloc[b_off[k] + e] = vol * s;   // B_P = |P| d (row-major kNq x NU)
    }
    __syncthreads();
    // int_P phi_j . grad m_b for the gradients b (|b| = 1: the gradient DOFs)
    for (int e = tid; e < kGr * NU; e += blockDim.x) {
      const int g = e / NU, j = e % NU;
      const int bb = g + 1;
      double v;
      if (bb <= 3) {
        v = (j == gcol0 + (bb - 1)) ? vol * ihP : 0.0;
      } else {
        v = bnd[bb * NUmax + j];
        for (int q = 0; q < kNq; ++q) v -= Hqt[q * kGr + g] * dd[q * NUmax + j];
      }
      GI[g * NUmax + j] = v;
    }
    __syncthreads();
    // G = A GI + C CI (CI: |P| on the cross DOF columns)
    for (int e = tid; e < kV * NU; e += blockDim.x) {
      const int r = e / NU, j = e % NU;
      double v = hP * c_k2.a_coef[r] * GI[c_k2.a_beta[r] * NUmax + j];
      if (j >= ccol0) v += c_k2.c_coef[r][j - ccol0] * vol;
      G[r * NUmax + j] = v;
    }
    __syncthreads();
    // Pi = H^-1 G per component
    for (int e = tid; e < kV * NU; e += blockDim.x) {
      const int r = e / NU, j = e % NU;
      const int cc = r / 10, a = r % 10;
      double s = 0.0;
      for (int bb = 0; bb < 10; ++bb) s += Hp[a * 10 + bb] * G[(cc * 10 + bb) * NUmax + j];
      Pi[r * NUmax + j] = s;
    }
    // interior rows of D: gradient DOFs (|P|^-1 int m_a delta), cross DOFs
    for (int e = tid; e < kNid * kV; e += blockDim.x) {
      const int row = e / kV, r = e % kV;
      const int cc = r / 10, a = r % 10;
      const int *al = c_k2.p3[a];
      double v = 0.0;
      if (row < 3) {
        v = (row == cc) ? mom(al[0], al[1], al[2]) / vol : 0.0;
      } else {
        const int mi = row - 3;
        const int comp = c_k2.cr_comp[mi];
        const int *gm = c_k2.p3[c_k2.cr_g[mi]];
        // (m_I ^ e_comp)_cc = sgn y_dir
        int dir = -1;
        double sgn = 0.0;
        if (comp == 0) {
          if (cc == 1) { dir = 2; sgn = 1.0; }
          if (cc == 2) { dir = 1; sgn = -1.0; }
        } else if (comp == 1) {
          if (cc == 0) { dir = 2; sgn = -1.0; }
          if (cc == 2) { dir = 0; sgn = 1.0; }
        } else {
          if (cc == 0) { dir = 1; sgn = 1.0; }
          if (cc == 1) { dir = 0; sgn = -1.0; }
        }
        if (dir >= 0) {
          int e3[3] = {al[0] + gm[0], al[1] + gm[1], al[2] + gm[2]};
          e3[dir] += 1;
          v = sgn * mom(e3[0], e3[1], e3[2]) / vol;
        }
      }
      D[(gcol0 + row) * kV + r] = v;
    }
    __syncthreads();
    // W = H (block diagonal) + |P| D^T D
    for (int e = tid; e < kV * kV; e += blockDim.x) {
      const int r = e / kV, s2 = e % kV;
      double v = 0.0;
      if (r / 10 == s2 / 10) {
        const int a = r % 10, bb = s2 % 10;
        v = mom(c_k2.p3[a][0] + c_k2.p3[bb][0], c_k2.p3[a][1] + c_k2.p3[bb][1], c_k2.p3[a][2] + c_k2.p3[bb][2]);
      }
      double t = 0.0;
      for (int j = 0; j < NU; ++j) t += D[j * kV + r] * D[j * kV + s2];
      W[e] = v + vol * t;
    }
    __syncthreads();
    for (int e = tid; e < kV * NU; e += blockDim.x) {
      const int r = e / NU, j = e % NU;
      double s = 0.0;
      for (int s2 = 0; s2 < kV; ++s2) s += W[r * kV + s2] * Pi[s2 * NUmax + j];
      WPi[r * NUmax + j] = s;
    }
    __syncthreads();
    // M = |P| I - |P| (D Pi + Pi^T D^T) + Pi^T W Pi;  B = |P| d
    double *Mo = Mloc + m_off[k];
    for (int64_t e = tid; e < (int64_t)NU * NU; e += blockDim.x) {
      const int i2 = (int)(e / NU), j = (int)(e % NU);
      double dp = 0.0, pw = 0.0;
      for (int r = 0; r < kV; ++r) {
        dp += D[i2 * kV + r] * Pi[r * NUmax + j] + D[j * kV + r] * Pi[r * NUmax + i2];
        pw += Pi[r * NUmax + i2] * WPi[r * NUmax + j];
      }
      Mo[e] = (i2 == j ? vol : 0.0) - vol * dp + pw;
    }
    if (tid == 0 && !(Hp[0] > 0.0 && Hq[0] > 0.0 && isfinite(Hp[0]))) atomicOr(err, DEVERR_SINGULAR_LOCAL);
    __syncthreads();
  }
}

vem_status element_k2(vem_handle *h) {
  // the decomposition and index tables (a few KB) go to the current device's
  // constant memory before every launch
  const K2Tables t = make_tables();
  VEM_CUDA(h, cudaMemcpyToSymbolAsync(c_k2, &t, sizeof(t), 0, cudaMemcpyHostToDevice, h->stream));
  const int mx = h->max_nf_cell, mv = h->max_nv_face;
  const size_t bytes = sizeof(double) * k2_smem_doubles(mx, mv);
  if (h->hq_inv_n < h->ncls) {
    dfree(h, h->hq_inv);
    dfree(h, h->pm_hat);
    h->hq_inv = nullptr;
    h->pm_hat = nullptr;
    VEM_TRY(dalloc_n(h, &h->hq_inv, 16 * (size_t)h->ncls));
    VEM_TRY(dalloc_n(h, &h->pm_hat, 16 * (size_t)h->ncls));
    h->hq_inv_n = h->ncls;
  }
  if (mv > 64 || bytes > 220 * 1024)
    return fail(h, VEM_ERR_UNSUPPORTED, "k = 2 element: cell with %d faces / face with %d vertices", mx, mv);
  VEM_CUDA(h, cudaFuncSetAttribute(k_elem_k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  int64_t blocks = h->ncls;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  count_launch();
  k_elem_k2<<<(int)blocks, kThreads, bytes, h->stream>>>(
      h->ncls, mx, mv, h->cf_ptr, h->cf, h->cf_sigma, h->fv_ptr, h->fv, h->xyz, h->f_area, h->f_cent, h->f_norm,
      h->f_t1, h->f_diam, h->c_vol, h->c_cent, h->c_diam, h->cls_rep, h->m_off, h->b_off, h->Mloc, h->Bloc,
      h->hq_inv, h->pm_hat, h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

// ---- loads of the k = 2 element ----
// Cell points: every fan tetrahedron (x_P, x_f, v_j, v_j+1) with the
// collapsed (Duffy) product of 3-point Gauss-Legendre rules in each
// direction (27 points, exact to degree 3: P1 moments of a quadratic f);
// weights signed by the face orientation, so they sum to |P|.
__global__ void k_cell_qp_count(int64_t nc, const int64_t *__restrict__ cfp, const int32_t *__restrict__ cf,
                                const int64_t *__restrict__ fvp, int64_t *cnt) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    int64_t v = 0;
    for (int64_t p = cfp[c]; p < cfp[c + 1]; ++p) v += 27 * (fvp[cf[p] + 1] - fvp[cf[p]]);
    cnt[c] = v;
  }
}

__global__ void k_cell_qp(int64_t nc, const int64_t *__restrict__ off, const int64_t *__restrict__ cfp,
                          const int32_t *__restrict__ cf, const int8_t *__restrict__ sig,
                          const int64_t *__restrict__ fvp, const int32_t *__restrict__ fv,
                          const double *__restrict__ xyz, const double *__restrict__ f_cent,
                          const double *__restrict__ c_cent, double *qx, double *qw) {
  const double g = 0.5 * 0.774596669241483377;   // sqrt(3/5) / 2
  const double s3[3] = {0.5 - g, 0.5, 0.5 + g};
  const double w3[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    int64_t o = off[c];
    const double3 A = load3(c_cent, c);
    for (int64_t p = cfp[c]; p < cfp[c + 1]; ++p) {
      const int f = cf[p];
      const double sg = (double)sig[p];
      const double3 B = load3(f_cent, f);
      const int64_t vb = fvp[f];
      const int m = (int)(fvp[f + 1] - vb);
      for (int j = 0; j < m; ++j) {
        const double3 C = load3(xyz, fv[vb + j]), D = load3(xyz, fv[vb + (j + 1) % m]);
        const double3 e1 = sub3(B, A), e2 = sub3(C, A), e3 = sub3(D, A);
        const double det = dot3(e1, cross3(e2, e3));
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b)
            for (int cc = 0; cc < 3; ++cc, ++o) {
              const double xi = s3[a], eta = s3[b] * (1.0 - s3[a]), zeta = s3[cc] * (1.0 - s3[a]) * (1.0 - s3[b]);
              const double3 x = add3(A, add3(add3(scale3(e1, xi), scale3(e2, eta)), scale3(e3, zeta)));
              store3(qx, o, x);
              qw[o] = sg * det * w3[a] * w3[b] * w3[cc] * (1.0 - s3[a]) * (1.0 - s3[a]) * (1.0 - s3[b]);
            }
      }
    }
  }
}

// F_P = |P| H_1^-1 (int_P f m_r)_r, r in P_1, from f at the cell points.
__global__ void k_rhs_cells_k2(int64_t nc, const int64_t *__restrict__ off, const double *__restrict__ qx,
                               const double *__restrict__ qw, const double *__restrict__ f_qp,
                               const double *__restrict__ c_cent, const double *__restrict__ c_diam,
                               const int32_t *__restrict__ cls_of, const double *__restrict__ hq_inv, double *F,
                               int *err) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    const double3 xP = load3(c_cent, c);
    const double ih = 1.0 / c_diam[c];
    double fm[4] = {0, 0, 0, 0};
    for (int64_t o = off[c]; o < off[c + 1]; ++o) {
      const double fv = f_qp ? f_qp[o] : 0.0;
      if (!isfinite(fv)) atomicOr(err, DEVERR_NONFINITE);
      const double3 y = scale3(sub3(load3(qx, o), xP), ih);
      const double wf = qw[o] * fv;
      fm[0] += wf;
      fm[1] += wf * y.x;
      fm[2] += wf * y.y;
      fm[3] += wf * y.z;
    }
    const double *Hi = hq_inv + 16 * (int64_t)cls_of[c];
    for (int q = 0; q < 4; ++q)
      F[4 * c + q] = Hi[4 * q] * fm[0] + Hi[4 * q + 1] * fm[1] + Hi[4 * q + 2] * fm[2] + Hi[4 * q + 3] * fm[3];
  }
}

// g_(f,beta) = -sigma |f| sum_g Ginv[g][beta] int_f g_D m^f_g on Dirichlet
// faces (zero elsewhere) for the six face moments; the face Gram matrix and
// the load by the boundary-data rule of the boundary-face points (ppt per
// fan triangle: Radon's degree 5 at k = 2, exact for g_D in P_3 times the
// M_2(f) monomials, and for the Gram entries).
__global__ void k_rhs_faces_k2(int64_t nbf, const int32_t *__restrict__ bface, int ppt,
                               const int8_t *__restrict__ fbc, const int64_t *__restrict__ off,
                               const int64_t *__restrict__ fvp, const int32_t *__restrict__ fv,
                               const double *__restrict__ xyz, const double *__restrict__ f_area,
                               const double *__restrict__ f_cent, const double *__restrict__ f_norm,
                               const double *__restrict__ f_t1, const double *__restrict__ f_diam,
                               const int32_t *__restrict__ f_cell, const int32_t *__restrict__ f_loc,
                               const int64_t *__restrict__ cfp, const int8_t *__restrict__ sig,
                               const double *__restrict__ gD, double *g, int *err) {
  const int fb[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};
  // boundary faces only (g is zeroed beforehand)
  for (int64_t ib = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ib < nbf;
       ib += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = bface[ib];
    if (fbc[f] != 1 || gD == nullptr) continue;
    const int64_t vb = fvp[f];
    const int m = (int)(fvp[f + 1] - vb);
    const double3 xf = load3(f_cent, f), n = load3(f_norm, f), t1 = load3(f_t1, f);
    const double3 t2 = cross3(n, t1);
    const double ihf = 1.0 / f_diam[f];
    const double sg = (double)sig[cfp[f_cell[2 * f]] + f_loc[2 * f]];
    double G[36], mom[6];
    for (int e = 0; e < 36; ++e) G[e] = 0.0;
    for (int e = 0; e < 6; ++e) mom[e] = 0.0;
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
        const double s = dot3(dx, t1) * ihf, t = dot3(dx, t2) * ihf;
        double mf[6];
        for (int bt = 0; bt < 6; ++bt) mf[bt] = ipow(s, fb[bt][0]) * ipow(t, fb[bt][1]);
        const double gv = gD[o];
        if (!isfinite(gv)) atomicOr(err, DEVERR_NONFINITE);
        for (int a = 0; a < 6; ++a) {
          mom[a] += w * gv * mf[a];
          for (int b = 0; b < 6; ++b) G[6 * a + b] += w * mf[a] * mf[b];
        }
      }
    }
    gj_inverse(G, 6);
    const double ar = f_area[f];
    for (int bt = 0; bt < 6; ++bt) {
      double v = 0.0;
      for (int a = 0; a < 6; ++a) v += G[6 * a + bt] * mom[a];
      g[6 * f + bt] = -sg * ar * v;
    }
  }
}

vem_status cell_points_k2(vem_handle *h) {
  if (h->cqp_valid) return VEM_OK;
  cudaStream_t s = h->stream;
  if (!h->cqp_off) VEM_TRY(dalloc_n(h, &h->cqp_off, (size_t)h->nc + 1));
  int64_t *cnt = nullptr;
  VEM_TRY(dalloc_n(h, &cnt, (size_t)h->nc + 1));
  count_launch();
  k_cell_qp_count<<<grid_for(h->nc, 256), 256, 0, s>>>(h->nc, h->cf_ptr, h->cf, h->fv_ptr, cnt);
  VEM_CUDA(h, cudaGetLastError());
  VEM_TRY(scan_counts(h, h->nc, cnt, h->cqp_off, &h->n_cqp));
  dfree(h, cnt);
  dfree(h, h->cqp_x);
  dfree(h, h->cqp_w);
  h->cqp_x = h->cqp_w = nullptr;
  VEM_TRY(dalloc_n(h, &h->cqp_x, 3 * (size_t)std::max<int64_t>(h->n_cqp, 1)));
  VEM_TRY(dalloc_n(h, &h->cqp_w, (size_t)std::max<int64_t>(h->n_cqp, 1)));
  count_launch();
  k_cell_qp<<<grid_for(h->nc, 128), 128, 0, s>>>(h->nc, h->cqp_off, h->cf_ptr, h->cf, h->cf_sigma, h->fv_ptr, h->fv,
                                                  h->xyz, h->f_cent, h->c_cent, h->cqp_x, h->cqp_w);
  VEM_CUDA(h, cudaGetLastError());
  h->cqp_valid = true;
  return VEM_OK;
}

// Near-null space of the condensed Block-Reg face system at k = 2: the face
// DOFs (1/|f|) int_f (e_j . n_f) m^f_beta of the three constant fields e_j,
// i.e. n_f[j] times the face mean of m^f_beta.  The means come from the fan
// triangles (x_f, v_i, v_i+1) with the edge-midpoint rule, exact for the
// quadratic face monomials; the triangle areas are signed along n_f, so a
// face centre outside a non-convex face still gives the right sums.
// B: (6 nf) x 3, row (6 f + beta).
__global__ void k_flux_modes_k2(int64_t nf, const int64_t *__restrict__ fvp, const int32_t *__restrict__ fv,
                                const double *__restrict__ xyz, const double *__restrict__ f_area,
                                const double *__restrict__ f_cent, const double *__restrict__ f_norm,
                                const double *__restrict__ f_t1, const double *__restrict__ f_diam, double *B) {
  const int fb[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    const int64_t vb = fvp[f];
    const int m = (int)(fvp[f + 1] - vb);
    const double3 xf = load3(f_cent, f), n = load3(f_norm, f), t1 = load3(f_t1, f);
    const double3 t2 = cross3(n, t1);
    const double ihf = 1.0 / f_diam[f];
    double mean[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < m; ++i) {
      const double3 A = load3(xyz, fv[vb + i]);
      const double3 Bv = load3(xyz, fv[vb + (i + 1) % m]);
      const double w = dot3(cross3(sub3(A, xf), sub3(Bv, xf)), n) / 6.0;   // area / 3 per midpoint
      const double3 mid[3] = {scale3(add3(xf, A), 0.5), scale3(add3(A, Bv), 0.5), scale3(add3(Bv, xf), 0.5)};
      for (int q = 0; q < 3; ++q) {
        const double3 dx = sub3(mid[q], xf);
        const double u = dot3(dx, t1) * ihf, v = dot3(dx, t2) * ihf;
        for (int bt = 0; bt < 6; ++bt) mean[bt] += w * ipow(u, fb[bt][0]) * ipow(v, fb[bt][1]);
      }
    }
    const double ia = 1.0 / f_area[f];
    const double nn[3] = {n.x, n.y, n.z};
    for (int bt = 0; bt < 6; ++bt)
      for (int j = 0; j < 3; ++j) B[(6 * f + bt) * 3 + j] = nn[j] * mean[bt] * ia;
  }
}

vem_status flux_modes_k2(vem_handle *h, double *B) {
  count_launch();
  k_flux_modes_k2<<<grid_for(h->nf, 128), 128, 0, h->stream>>>(h->nf, h->fv_ptr, h->fv, h->xyz, h->f_area,
                                                                h->f_cent, h->f_norm, h->f_t1, h->f_diam, B);
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

vem_status assemble_rhs_k2(vem_handle *h, const double *f_qp, const double *gD_qp, double *g, double *F) {
  cudaStream_t s = h->stream;
  VEM_TRY(cell_points_k2(h));
  VEM_CUDA(h, cudaMemsetAsync(g, 0, sizeof(double) * 6 * h->nf, s));
  count_launch();
  k_rhs_faces_k2<<<grid_for(h->n_bface, 128), 128, 0, s>>>(h->n_bface, h->bface, h->bq_ppt, h->fbc, h->bqp_off,
                                                            h->fv_ptr,
                                                            h->fv, h->xyz, h->f_area, h->f_cent, h->f_norm,
                                                            h->f_t1, h->f_diam, h->f_cell, h->f_loc, h->cf_ptr,
                                                            h->cf_sigma, gD_qp, g, h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  VEM_CUDA(h, cudaMemsetAsync(g + 6 * h->nf, 0, sizeof(double) * 14 * h->nc, s));
  count_launch();
  k_rhs_cells_k2<<<grid_for(h->nc, 128), 128, 0, s>>>(h->nc, h->cqp_off, h->cqp_x, h->cqp_w, f_qp, h->c_cent,
                                                        h->c_diam, h->cls_of, h->hq_inv, F, h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

}  // namespace vem
