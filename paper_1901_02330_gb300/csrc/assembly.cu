// Global assembly (paper Sec. 4.3, global forms a_h, b_h, f_h glued across
// cells) into one sliced-ELL (SELL-32) matrix of the saddle-point operator
// [M B^T; B 0] (Sec. 5), and the Schur approximation S = B diag(M)^{-1} B^T of
// the Block-Schur preconditioner (eq. block_schur), also in SELL-32.
//
// Row layout: face DOF rows (nfd per face), interior DOF rows (nid per
// cell), pressure rows (one per cell).  A face row gathers the matching
// rows of the (at most two) local matrices of its cells: columns of the
// lower-id cell in its local order, then those of the other cell except the
// shared face, then the pressure columns.  No atomics: every entry is a
// fixed-order sum of at most two local values, so the result is
// deterministic.
#include <cmath>

#include "handle.cuh"

namespace vem {

// Local matrices are stored per congruence class with nu = 1: cell c uses
// Mloc + m_off[cls_of[c]] (scaled by its nu) and Bloc + b_off[cls_of[c]].
struct Layout {
  int nfd, nid;
  int64_t nf, nc, n_u;
  const int64_t *cfp;
  const int32_t *cf;
  const int32_t *f_cell, *f_loc;
  const int64_t *m_off, *b_off;
  const int32_t *cls_of;
  const double *Mloc, *Bloc;
  const int8_t *fbc;      // face flags (2: prescribed flux, DOFs eliminated)
};

__device__ __forceinline__ int nloc(const Layout &L, int64_t c) {
  return L.nfd * (int)(L.cfp[c + 1] - L.cfp[c]) + L.nid;
}
__device__ __forceinline__ int64_t gcol(const Layout &L, int64_t c, int jl) {
  const int k = (int)(L.cfp[c + 1] - L.cfp[c]);
  if (jl < L.nfd * k) return (int64_t)L.nfd * L.cf[L.cfp[c] + jl / L.nfd] + jl % L.nfd;
  return (int64_t)L.nfd * L.nf + (int64_t)L.nid * c + (jl - L.nfd * k);
}
__device__ __forceinline__ int64_t boff(const Layout &L, int64_t c) { return L.b_off[L.cls_of[c]]; }
__device__ __forceinline__ const double *mloc(const Layout &L, int64_t c) {
  return L.Mloc + L.m_off[L.cls_of[c]];
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

// One thread per row, consecutive rows on consecutive lanes, so element j of
// the 32 rows of a slice is written by one coalesced store.  Ghost rows of
// the last slice and the padding of short rows get value 0, column 0.
// Batched use (gridDim.y systems): values of system b at val + b * stored,
// diag(M) at diagM + b * n_u (its reciprocal, which the preconditioners
// multiply by, at dinvM + b * n_u), local matrices scaled by nu_scale[b * nc + c]
// (the local matrices then hold nu = 1); col == nullptr skips the (shared)
// column ids.  NFD / NID: face and interior DOFs per face / cell (E0: 1 / 0,
// K1: 3 / 3), so the local-to-global map runs without divisions.
template <int NFD, int NID>
__global__ void k_fill(Layout L, const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                       int64_t nrows_pad, int32_t *col, double *val, double *diagM, double *dinvM,
                       const double *__restrict__ nu_scale, int64_t stored) {
  const int64_t n = L.n_u + L.nc;
  const int64_t nfr = (int64_t)NFD * L.nf;
  const int64_t bb = blockIdx.y;
  val += bb * stored;
  diagM += bb * L.n_u;
  dinvM += bb * L.n_u;
  const double *nsc = nu_scale ? nu_scale + bb * L.nc : nullptr;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows_pad;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s0 = off[r >> 5];
    const int width = (int)((off[(r >> 5) + 1] - s0) >> 5);
    const int64_t lane = r & 31;
    int j = 0;
#define PUT(c_, v_)                          \
  do {                                       \
    const int64_t q_ = s0 + ((int64_t)j << 5) + lane; \
    if (col) col[q_] = (int32_t)(c_);        \
    val[q_] = (v_);                          \
    ++j;                                     \
  } while (0)
    if (r >= n) {
      // ghost row
    } else if (r < nfr) {
      const int64_t f = r / NFD;
      const int beta = (int)(r - f * NFD);
      const int32_t c0 = L.f_cell[2 * f], c1 = L.f_cell[2 * f + 1];
      const int l0 = L.f_loc[2 * f], l1 = L.f_loc[2 * f + 1];
      const int64_t b0 = L.cfp[c0];
      const int k0 = (int)(L.cfp[c0 + 1] - b0);
      const int n0 = NFD * k0 + NID;
      const double *M0 = mloc(L, c0) + (int64_t)(l0 * NFD + beta) * n0;
      const double *M1 = nullptr;
      int64_t b1 = 0;
      int k1 = 0, n1 = 0;
      if (c1 >= 0) {
        b1 = L.cfp[c1];
        k1 = (int)(L.cfp[c1 + 1] - b1);
        n1 = NFD * k1 + NID;
        M1 = mloc(L, c1) + (int64_t)(l1 * NFD + beta) * n1;
      }
      const double w0 = nsc ? nsc[c0] : 1.0, w1 = (nsc && c1 >= 0) ? nsc[c1] : 1.0;
      double dg = 0.0;
      for (int i = 0; i < k0; ++i) {
        const int64_t gc = (int64_t)NFD * L.cf[b0 + i];
#pragma unroll
        for (int bt = 0; bt < NFD; ++bt) {
          double v = w0 * M0[i * NFD + bt];
          if (i == l0) {
            if (c1 >= 0) v += w1 * M1[l1 * NFD + bt];
            if (bt == beta) dg = v;
          }
          PUT(gc + bt, v);
        }
      }
#pragma unroll
      for (int l = 0; l < NID; ++l) PUT(nfr + (int64_t)NID * c0 + l, w0 * M0[NFD * k0 + l]);
      if (c1 >= 0) {
        for (int i = 0; i < k1; ++i) {
          if (i == l1) continue;
          const int64_t gc = (int64_t)NFD * L.cf[b1 + i];
#pragma unroll
          for (int bt = 0; bt < NFD; ++bt) PUT(gc + bt, w1 * M1[i * NFD + bt]);
        }
#pragma unroll
        for (int l = 0; l < NID; ++l) PUT(nfr + (int64_t)NID * c1 + l, w1 * M1[NFD * k1 + l]);
      }
      if (beta == 0) {
        PUT(L.n_u + c0, L.Bloc[boff(L, c0) + l0 * NFD]);
        if (c1 >= 0) PUT(L.n_u + c1, L.Bloc[boff(L, c1) + l1 * NFD]);
      }
      diagM[r] = dg;
      dinvM[r] = 1.0 / dg;
    } else if (r < L.n_u) {
      if constexpr (NID > 0) {
        const int64_t q = r - nfr;
        const int64_t c = q / NID;
        const int l = (int)(q - c * NID);
        const int64_t b0 = L.cfp[c];
        const int k = (int)(L.cfp[c + 1] - b0);
        const int nl = NFD * k + NID;
        const int jr = nl - NID + l;
        const double *Mr = mloc(L, c) + (int64_t)jr * nl;
        const double wc = nsc ? nsc[c] : 1.0;
        for (int i = 0; i < k; ++i) {
          const int64_t gc = (int64_t)NFD * L.cf[b0 + i];
#pragma unroll
          for (int bt = 0; bt < NFD; ++bt) PUT(gc + bt, wc * Mr[i * NFD + bt]);
        }
#pragma unroll
        for (int l2 = 0; l2 < NID; ++l2) PUT(nfr + (int64_t)NID * c + l2, wc * Mr[NFD * k + l2]);
        diagM[r] = wc * Mr[jr];
        dinvM[r] = 1.0 / diagM[r];
      }
    } else {
      const int64_t c = r - L.n_u;
      const int k = (int)(L.cfp[c + 1] - L.cfp[c]);
      for (int i = 0; i < k; ++i) PUT((int64_t)NFD * L.cf[L.cfp[c] + i], L.Bloc[boff(L, c) + i * NFD]);
    }
    while (j < width) PUT(0, 0.0);
#undef PUT
  }
}

static void launch_fill(cudaStream_t s, int nfd, dim3 grid, const Layout &L, const int64_t *off, const int32_t *len,
                        int64_t npad, int32_t *col, double *val, double *diagM, double *dinvM,
                        const double *nu_scale, int64_t stored) {
  count_launch();
  if (nfd == 3) k_fill<3, 3><<<grid, 256, 0, s>>>(L, off, len, npad, col, val, diagM, dinvM, nu_scale, stored);
  else k_fill<1, 0><<<grid, 256, 0, s>>>(L, off, len, npad, col, val, diagM, dinvM, nu_scale, stored);
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

__global__ void k_schur_fill(Layout L, const double *__restrict__ diagM, const int64_t *__restrict__ off,
                             int64_t nrows_pad, int32_t *col, double *val, double *dinv, int *err,
                             int64_t stored) {
  const int64_t bb = blockIdx.y;
  diagM += bb * L.n_u;
  val += bb * stored;
  dinv += bb * L.nc;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nrows_pad;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s0 = off[c >> 5];
    const int width = (int)((off[(c >> 5) + 1] - s0) >> 5);
    const int64_t lane = c & 31;
    int j = 0;
    if (c < L.nc) {
      const int64_t b = L.cfp[c];
      const int k = (int)(L.cfp[c + 1] - b);
      const int64_t bo = boff(L, c);
      double dg = 0.0;
      j = 1;   // slot 0 holds the diagonal
      for (int i = 0; i < k; ++i) {
        const int f = L.cf[b + i];
        if (L.fbc[f] == 2) continue;   // eliminated flux DOF: no column of B
        const double bp = L.Bloc[bo + i * L.nfd];
        const double mf = diagM[(int64_t)L.nfd * f];
        dg += bp * bp / mf;
        const int32_t c0 = L.f_cell[2 * f], c1 = L.f_cell[2 * f + 1];
        if (c1 < 0) continue;
        const int32_t q = (c0 == c) ? c1 : c0;
        const int lq = (c0 == c) ? L.f_loc[2 * f + 1] : L.f_loc[2 * f];
        const int64_t p = s0 + ((int64_t)j << 5) + lane;
        if (col) col[p] = q;
        val[p] = bp * L.Bloc[boff(L, q) + lq * L.nfd] / mf;
        ++j;
      }
      if (col) col[s0 + lane] = (int32_t)c;
      val[s0 + lane] = dg;
      if (!(dg > 0.0) || !isfinite(dg)) atomicOr(err, DEVERR_NONFINITE);
      dinv[c] = 1.0 / dg;
    }
    for (; j < width; ++j) {
      const int64_t p = s0 + ((int64_t)j << 5) + lane;
      if (col) col[p] = 0;
      val[p] = 0.0;
    }
  }
}

// Eliminate the prescribed flux DOFs (faces with flag 2): their rows become
// unit rows, their columns are zeroed elsewhere, diag(M) and its reciprocal
// there are 1 (when diagM / dinvM are given).
__global__ void k_eliminate(int64_t rows, const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                            const int32_t *__restrict__ col, double *val, int nfd, int64_t nf,
                            const int8_t *__restrict__ fbc, double *diagM, double *dinvM) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const bool fixed_row = r < (int64_t)nfd * nf && fbc[r / nfd] == 2;
    const int64_t base = off[r >> 5] + (r & 31);
    const int L = len[r];
    for (int k = 0; k < L; ++k) {
      const int64_t p = base + 32 * (int64_t)k;
      const int64_t c = col[p];
      const bool fixed_col = c < (int64_t)nfd * nf && fbc[c / nfd] == 2;
      if (fixed_row) val[p] = (c == r) ? 1.0 : 0.0;
      else if (fixed_col) val[p] = 0.0;
    }
    if (fixed_row && diagM) diagM[r] = 1.0;
    if (fixed_row && dinvM) dinvM[r] = 1.0;
  }
}

// ---- Block-Reg: A_reg = M + B^T W^-1 B, W = gamma I (paper Sec. 5) ----
// B^T B = sum_P B_P^T B_P couples only DOFs of one cell (the pressure DOF of
// P belongs to P alone), so A_reg has the pattern of M: row r of a face DOF
// gathers the rows of the (at most two) cells of its face, an interior row
// that of its cell, in the column order of the saddle matrix's flux part.
// Entry (r, j) of cell P adds sum_q B_P(q, r) B_P(q, j) / gamma to
// nu_P M_P(r, j), with B_P(q, j) = Bloc[b_off + q n_loc + j] (nq pressure
// DOFs per cell: 1 for k <= 1, the 4 P1 moments for the paper's k = 2).
__global__ void k_reg_count(Layout L, int64_t *cnt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < L.n_u;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t v;
    if (r < L.nfd * L.nf) {
      const int64_t f = r / L.nfd;
      const int32_t c0 = L.f_cell[2 * f], c1 = L.f_cell[2 * f + 1];
      v = nloc(L, c0) + (c1 >= 0 ? nloc(L, c1) - L.nfd : 0);
    } else {
      v = nloc(L, (r - L.nfd * L.nf) / L.nid);
    }
    cnt[r] = v;
  }
}

__global__ void k_reg_fill(Layout L, int nq, const int64_t *__restrict__ off, int64_t nrows_pad, int32_t *col,
                           double *val, const double *__restrict__ nu_scale, double ig) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows_pad;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s0 = off[r >> 5];
    const int width = (int)((off[(r >> 5) + 1] - s0) >> 5);
    const int64_t lane = r & 31;
    int j = 0;
#define PUT(c_, v_)                                   \
  do {                                                \
    const int64_t q_ = s0 + ((int64_t)j << 5) + lane; \
    col[q_] = (int32_t)(c_);                          \
    val[q_] = (v_);                                   \
    ++j;                                              \
  } while (0)
    if (r >= L.n_u) {
      // ghost row
    } else if (r < L.nfd * L.nf) {
      const int64_t f = r / L.nfd;
      const int beta = (int)(r % L.nfd);
      const int32_t c0 = L.f_cell[2 * f], c1 = L.f_cell[2 * f + 1];
      const int l0 = L.f_loc[2 * f], l1 = L.f_loc[2 * f + 1];
      const int n0 = nloc(L, c0);
      const int jr0 = l0 * L.nfd + beta;
      const double *M0 = mloc(L, c0) + (int64_t)jr0 * n0;
      const double *B0 = L.Bloc + boff(L, c0);
      const double w0 = nu_scale[c0];
      double g0[4], g1[4] = {0.0, 0.0, 0.0, 0.0};
      for (int q = 0; q < nq; ++q) g0[q] = ig * B0[q * n0 + jr0];
      const double *M1 = nullptr, *B1 = nullptr;
      int n1 = 0;
      double w1 = 0.0;
      if (c1 >= 0) {
        n1 = nloc(L, c1);
        const int jr1 = l1 * L.nfd + beta;
        M1 = mloc(L, c1) + (int64_t)jr1 * n1;
        B1 = L.Bloc + boff(L, c1);
        w1 = nu_scale[c1];
        for (int q = 0; q < nq; ++q) g1[q] = ig * B1[q * n1 + jr1];
      }
      for (int jl = 0; jl < n0; ++jl) {
        double v = w0 * M0[jl];
        for (int q = 0; q < nq; ++q) v += g0[q] * B0[q * n0 + jl];
        const bool shared = (jl < n0 - L.nid) && (jl / L.nfd == l0);
        if (c1 >= 0 && shared) {
          const int j1 = l1 * L.nfd + jl % L.nfd;
          double v1 = w1 * M1[j1];
          for (int q = 0; q < nq; ++q) v1 += g1[q] * B1[q * n1 + j1];
          v += v1;
        }
        PUT(gcol(L, c0, jl), v);
      }
      if (c1 >= 0) {
        const int k1 = (n1 - L.nid) / L.nfd;
        for (int jl = 0; jl < n1; ++jl) {
          if (jl < L.nfd * k1 && jl / L.nfd == l1) continue;
          double v1 = w1 * M1[jl];
          for (int q = 0; q < nq; ++q) v1 += g1[q] * B1[q * n1 + jl];
          PUT(gcol(L, c1, jl), v1);
        }
      }
    } else {
      const int64_t q = r - L.nfd * L.nf;
      const int64_t c = q / L.nid;
      const int l = (int)(q % L.nid);
      const int nl = nloc(L, c);
      const int jr = nl - L.nid + l;
      const double *Mr = mloc(L, c) + (int64_t)jr * nl;
      const double *Bc = L.Bloc + boff(L, c);
      const double wc = nu_scale[c];
      double gc[4];
      for (int q2 = 0; q2 < nq; ++q2) gc[q2] = ig * Bc[q2 * nl + jr];
      for (int jl = 0; jl < nl; ++jl) {
        double v = wc * Mr[jl];
        for (int q2 = 0; q2 < nq; ++q2) v += gc[q2] * Bc[q2 * nl + jl];
        PUT(gcol(L, c, jl), v);
      }
    }
    while (j < width) PUT(0, 0.0);
#undef PUT
  }
}

__global__ void k_iota32(int64_t n, int32_t *a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

__global__ void k_f64_to_f32(int64_t n, const double *__restrict__ a, float *b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// B entries of the (f, 0) DOF in each of the face's two cells (0 for a
// missing second cell), for the block-triangular flux update.
__global__ void k_bt_face(Layout L, double *bt) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < L.nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    for (int s = 0; s < 2; ++s) {
      const int32_t c = L.f_cell[2 * f + s];
      bt[2 * f + s] = (c >= 0 && L.fbc[f] != 2) ? L.Bloc[boff(L, c) + L.f_loc[2 * f + s] * L.nfd] : 0.0;
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

// Per slice: 32 x (longest row) elements; row lengths copied to int32.
__global__ void k_slice_sizes(int64_t rows, int64_t nslices, const int64_t *__restrict__ cnt,
                              int64_t *ssz, int32_t *len) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslices;
       s += (int64_t)gridDim.x * blockDim.x) {
    int64_t w = 0;
    for (int l = 0; l < 32; ++l) {
      const int64_t r = 32 * s + l;
      const int64_t c = r < rows ? cnt[r] : 0;
      len[r] = (int32_t)c;
      w = c > w ? c : w;
    }
    ssz[s] = 32 * w;
  }
}


// Allocate / lay out a SELL matrix from device row counts cnt[rows].
static vem_status sell_layout(vem_handle *h, SellMat &M, int64_t rows, const int64_t *cnt) {
  const int64_t ns = (rows + 31) / 32;
  if (M.rows != rows) {
    dfree(h, M.off);
    dfree(h, M.len);
    M.off = nullptr;
    M.len = nullptr;
  }
  if (!M.off) VEM_TRY(dalloc_n(h, &M.off, (size_t)ns + 1));
  if (!M.len) VEM_TRY(dalloc_n(h, &M.len, (size_t)ns * 32));
  if (h->slice_buf_n < ns) {
    dfree(h, h->slice_buf);
    h->slice_buf = nullptr;
    VEM_TRY(dalloc_n(h, &h->slice_buf, (size_t)ns));
    h->slice_buf_n = ns;
  }
  int64_t *ssz = h->slice_buf;
  count_launch();
  k_slice_sizes<<<grid_for(ns, 256), 256, 0, h->stream>>>(rows, ns, cnt, ssz, M.len);
  VEM_CUDA(h, cudaGetLastError());
  int64_t stored = 0;
  VEM_TRY(scan_counts(h, ns, ssz, M.off, &stored));
  if (stored != M.stored || !M.val) {
    dfree(h, M.col);
    dfree(h, M.val);
    M.col = nullptr;
    M.val = nullptr;
    VEM_TRY(dalloc_n(h, &M.col, (size_t)stored));
    VEM_TRY(dalloc_n(h, &M.val, (size_t)stored));
  }
  M.rows = rows;
  M.nslices = ns;
  M.stored = stored;
  return VEM_OK;
}

// The same scan in one block for short arrays (the layouts of small meshes,
// coarse AMG levels): every thread sums a run of consecutive entries, the
// run totals are scanned across the block, and each thread writes its run's
// prefix sums.  One launch instead of three.
constexpr int kScanOneThreads = 1024;
constexpr int64_t kScanOneMax = 32768;

__global__ void __launch_bounds__(kScanOneThreads) k_scan_one(int64_t n, const int64_t *__restrict__ in,
                                                              int64_t *out) {
  __shared__ int64_t ws[kScanOneThreads / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t lo = t * per, hi = lo + per < n ? lo + per : n;
  int64_t run = 0;
  for (int64_t i = lo; i < hi; ++i) run += in[i];
  int64_t v = run;   // inclusive scan of the run totals: warp, then across warps
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) ws[w] = v;
  __syncthreads();
  if (w == 0) {
    int64_t x = lane < nw ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    if (lane < nw) ws[lane] = x;
  }
  __syncthreads();
  int64_t acc = v - run + (w > 0 ? ws[w - 1] : 0);   // exclusive prefix of this run
  if (t == 0) out[0] = 0;
  for (int64_t i = lo; i < hi; ++i) {
    acc += in[i];
    out[i + 1] = acc;
  }
}

vem_status scan_counts(vem_handle *h, int64_t n, const int64_t *cnt, int64_t *out, int64_t *total) {
  cudaStream_t s = h->stream;
  if (n <= kScanOneMax) {
    count_launch(); k_scan_one<<<1, kScanOneThreads, 0, s>>>(n, cnt, out);
    VEM_CUDA(h, cudaGetLastError());
    VEM_CUDA(h, cudaMemcpyAsync(total, out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    return VEM_OK;
  }
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

// Sum of true row lengths: one partial per block, added with an integer
// atomic (exact, so the order does not matter).
__global__ void k_len_sum(int64_t n, const int32_t *__restrict__ len, unsigned long long *out) {
  __shared__ int64_t ws[32];
  int64_t s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += len[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += ws[i];
    atomicAdd(out, (unsigned long long)t);
  }
}

static vem_status sell_nnz(vem_handle *h, SellMat &M) {
  // reuse: the per-slice sizes are no longer needed
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(h->slice_buf);
  VEM_CUDA(h, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), h->stream));
  const int64_t n = M.nslices * 32;
  count_launch();
  k_len_sum<<<grid_for(n, 256), 256, 0, h->stream>>>(n, M.len, cnt);
  VEM_CUDA(h, cudaGetLastError());
  unsigned long long t = 0;
  VEM_CUDA(h, cudaMemcpyAsync(&t, cnt, sizeof(t), cudaMemcpyDeviceToHost, h->stream));
  VEM_CUDA(h, cudaStreamSynchronize(h->stream));
  M.nnz = (int64_t)t;
  return VEM_OK;
}

vem_status sell_to_host_csr(vem_handle *h, const SellMat &M, int64_t *rp, int32_t *col, double *val) {
  std::vector<int32_t> len(M.nslices * 32);
  std::vector<int64_t> off(M.nslices + 1);
  VEM_CUDA(h, cudaMemcpyAsync(len.data(), M.len, sizeof(int32_t) * len.size(), cudaMemcpyDeviceToHost, h->stream));
  VEM_CUDA(h, cudaMemcpyAsync(off.data(), M.off, sizeof(int64_t) * off.size(), cudaMemcpyDeviceToHost, h->stream));
  std::vector<int32_t> c;
  std::vector<double> v;
  if (col || val) {
    c.resize(M.stored);
    v.resize(M.stored);
    VEM_CUDA(h, cudaMemcpyAsync(c.data(), M.col, sizeof(int32_t) * M.stored, cudaMemcpyDeviceToHost, h->stream));
    VEM_CUDA(h, cudaMemcpyAsync(v.data(), M.val, sizeof(double) * M.stored, cudaMemcpyDeviceToHost, h->stream));
  }
  VEM_CUDA(h, cudaStreamSynchronize(h->stream));
  int64_t o = 0;
  for (int64_t r = 0; r < M.rows; ++r) {
    if (rp) rp[r] = o;
    const int64_t base = off[r >> 5] + (r & 31);
    for (int j = 0; j < len[r]; ++j, ++o) {
      if (col) col[o] = c[base + 32 * (int64_t)j];
      if (val) val[o] = v[base + 32 * (int64_t)j];
    }
  }
  if (rp) rp[M.rows] = o;
  return VEM_OK;
}

// ---- several pressure DOFs per cell (paper k = 2: NQ = 4) ----
// B_P is NQ x n_loc (row-major at Bloc + b_off): every local DOF couples to
// every pressure DOF of its cell.  Pressure unknown q of cell c sits at
// n_u + NQ c + q.
template <int NFD, int NID, int NQ>
__global__ void k_rowcount_q(Layout L, int64_t *cnt) {
  const int64_t nfr = (int64_t)NFD * L.nf;
  const int64_t n = L.n_u + (int64_t)NQ * L.nc;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t v;
    if (r < nfr) {
      const int64_t f = r / NFD;
      const int32_t c0 = L.f_cell[2 * f], c1 = L.f_cell[2 * f + 1];
      const int64_t k0 = L.cfp[c0 + 1] - L.cfp[c0];
      v = NFD * k0 + NID + NQ;
      if (c1 >= 0) v += NFD * (L.cfp[c1 + 1] - L.cfp[c1]) + NID - NFD + NQ;
    } else if (r < L.n_u) {
      const int64_t c = (r - nfr) / NID;
      v = NFD * (L.cfp[c + 1] - L.cfp[c]) + NID + NQ;
    } else {
      const int64_t c = (r - L.n_u) / NQ;
      v = NFD * (L.cfp[c + 1] - L.cfp[c]) + NID;
    }
    cnt[r] = v;
  }
}

template <int NFD, int NID, int NQ>
// Batched (gridDim.y systems, as k_fill): values of system blockIdx.y at
// val + y stored, diag(M) at diagM + y n_u (1/diag(M) at dinvM + y n_u), its
// nu at nsc + y n_c; col NULL
// writes the values only (the structure is shared).
__global__ void k_fill_q(Layout L, const int64_t *__restrict__ off, int64_t nrows_pad, int32_t *col, double *val,
                         double *diagM, double *dinvM, const double *__restrict__ nsc, int64_t stored) {
  const int64_t nfr = (int64_t)NFD * L.nf;
  const int64_t n = L.n_u + (int64_t)NQ * L.nc;
  const int64_t bb = blockIdx.y;
  val += bb * stored;
  diagM += bb * L.n_u;
  dinvM += bb * L.n_u;
  nsc += bb * L.nc;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows_pad;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s0 = off[r >> 5];
    const int width = (int)((off[(r >> 5) + 1] - s0) >> 5);
    const int64_t lane = r & 31;
    int j = 0;
#define PUT(c_, v_)                                   \
  do {                                                \
    const int64_t q_ = s0 + ((int64_t)j << 5) + lane; \
    if (col) col[q_] = (int32_t)(c_);                 \
    val[q_] = (v_);                                   \
    ++j;                                              \
  } while (0)
    if (r >= n) {
      // ghost row
    } else if (r < nfr) {
      const int64_t f = r / NFD;
      const int beta = (int)(r - f * NFD);
      const int32_t c0 = L.f_cell[2 * f], c1 = L.f_cell[2 * f + 1];
      const int l0 = L.f_loc[2 * f], l1 = L.f_loc[2 * f + 1];
      const int64_t b0 = L.cfp[c0];
      const int k0 = (int)(L.cfp[c0 + 1] - b0);
      const int n0 = NFD * k0 + NID;
      const double *M0 = mloc(L, c0) + (int64_t)(l0 * NFD + beta) * n0;
      const double *B0 = L.Bloc + boff(L, c0);
      const double *M1 = nullptr, *B1 = nullptr;
      int64_t b1 = 0;
      int k1 = 0, n1 = 0;
      if (c1 >= 0) {
        b1 = L.cfp[c1];
        k1 = (int)(L.cfp[c1 + 1] - b1);
        n1 = NFD * k1 + NID;
        M1 = mloc(L, c1) + (int64_t)(l1 * NFD + beta) * n1;
        B1 = L.Bloc + boff(L, c1);
      }
      const double w0 = nsc[c0], w1 = c1 >= 0 ? nsc[c1] : 1.0;
      double dg = 0.0;
      for (int i = 0; i < k0; ++i) {
        const int64_t gc = (int64_t)NFD * L.cf[b0 + i];
        for (int bt = 0; bt < NFD; ++bt) {
          double v = w0 * M0[i * NFD + bt];
          if (i == l0) {
            if (c1 >= 0) v += w1 * M1[l1 * NFD + bt];
            if (bt == beta) dg = v;
          }
          PUT(gc + bt, v);
        }
      }
      for (int l = 0; l < NID; ++l) PUT(nfr + (int64_t)NID * c0 + l, w0 * M0[NFD * k0 + l]);
      if (c1 >= 0) {
        for (int i = 0; i < k1; ++i) {
          if (i == l1) continue;
          const int64_t gc = (int64_t)NFD * L.cf[b1 + i];
          for (int bt = 0; bt < NFD; ++bt) PUT(gc + bt, w1 * M1[i * NFD + bt]);
        }
        for (int l = 0; l < NID; ++l) PUT(nfr + (int64_t)NID * c1 + l, w1 * M1[NFD * k1 + l]);
      }
      for (int q = 0; q < NQ; ++q) PUT(L.n_u + (int64_t)NQ * c0 + q, B0[q * n0 + l0 * NFD + beta]);
      if (c1 >= 0)
        for (int q = 0; q < NQ; ++q) PUT(L.n_u + (int64_t)NQ * c1 + q, B1[q * n1 + l1 * NFD + beta]);
      diagM[r] = dg;
      dinvM[r] = 1.0 / dg;
    } else if (r < L.n_u) {
      const int64_t c = (r - nfr) / NID;
      const int l = (int)(r - nfr - c * NID);
      const int64_t b0 = L.cfp[c];
      const int k = (int)(L.cfp[c + 1] - b0);
      const int nl = NFD * k + NID;
      const int jr = nl - NID + l;
      const double *Mr = mloc(L, c) + (int64_t)jr * nl;
      const double *Bc = L.Bloc + boff(L, c);
      const double wc = nsc[c];
      for (int i = 0; i < k; ++i) {
        const int64_t gc = (int64_t)NFD * L.cf[b0 + i];
        for (int bt = 0; bt < NFD; ++bt) PUT(gc + bt, wc * Mr[i * NFD + bt]);
      }
      for (int l2 = 0; l2 < NID; ++l2) PUT(nfr + (int64_t)NID * c + l2, wc * Mr[NFD * k + l2]);
      for (int q = 0; q < NQ; ++q) PUT(L.n_u + (int64_t)NQ * c + q, Bc[q * nl + jr]);
      diagM[r] = wc * Mr[jr];
      dinvM[r] = 1.0 / diagM[r];
    } else {
      const int64_t c = (r - L.n_u) / NQ;
      const int q = (int)(r - L.n_u - c * NQ);
      const int64_t b0 = L.cfp[c];
      const int k = (int)(L.cfp[c + 1] - b0);
      const int nl = NFD * k + NID;
      const double *Bq = L.Bloc + boff(L, c) + (int64_t)q * nl;
      for (int i = 0; i < k; ++i) {
        const int64_t gc = (int64_t)NFD * L.cf[b0 + i];
        for (int bt = 0; bt < NFD; ++bt) PUT(gc + bt, Bq[i * NFD + bt]);
      }
      for (int l = 0; l < NID; ++l) PUT(nfr + (int64_t)NID * c + l, Bq[NFD * k + l]);
    }
    while (j < width) PUT(0, 0.0);
#undef PUT
  }
}

// S = B diag(M)^-1 B^T with NQ pressure DOFs per cell: row (P, q) holds the
// NQ x NQ block of P (all its local DOFs) and one NQ block per neighbour Q
// across an interior face (that face's NFD DOFs).
template <int NFD, int NID, int NQ>
__global__ void k_schur_count_q(Layout L, int64_t *cnt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < (int64_t)NQ * L.nc;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = r / NQ;
    int64_t v = NQ;
    for (int64_t p = L.cfp[c]; p < L.cfp[c + 1]; ++p) v += (L.f_cell[2 * L.cf[p] + 1] >= 0) ? NQ : 0;
    cnt[r] = v;
  }
}

template <int NFD, int NID, int NQ>
__global__ void k_schur_fill_q(Layout L, const double *__restrict__ diagM, const int64_t *__restrict__ off,
                               int64_t nrows_pad, int32_t *col, double *val, double *dinv, int *err,
                               int64_t stored) {
  const int64_t nfr = (int64_t)NFD * L.nf;
  const int64_t bb = blockIdx.y;   // batched as k_schur_fill; col NULL: values only
  diagM += bb * L.n_u;
  val += bb * stored;
  dinv += bb * (int64_t)NQ * L.nc;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows_pad;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s0 = off[r >> 5];
    const int width = (int)((off[(r >> 5) + 1] - s0) >> 5);
    const int64_t lane = r & 31;
    int j = 0;
    if (r < (int64_t)NQ * L.nc) {
      const int64_t c = r / NQ;
      const int q = (int)(r - c * NQ);
      const int64_t b0 = L.cfp[c];
      const int k = (int)(L.cfp[c + 1] - b0);
      const int nl = NFD * k + NID;
      const double *Bc = L.Bloc + boff(L, c);
      // own block: all local DOFs
      for (int q2 = 0; q2 < NQ; ++q2) {
        double v = 0.0;
        for (int i = 0; i < k; ++i) {
          const int fi = L.cf[b0 + i];
          if (L.fbc[fi] == 2) continue;   // eliminated flux DOFs: no column of B
          const int64_t gc = (int64_t)NFD * fi;
          for (int bt = 0; bt < NFD; ++bt)
            v += Bc[q * nl + i * NFD + bt] * Bc[q2 * nl + i * NFD + bt] / diagM[gc + bt];
        }
        for (int l = 0; l < NID; ++l)
          v += Bc[q * nl + NFD * k + l] * Bc[q2 * nl + NFD * k + l] / diagM[nfr + (int64_t)NID * c + l];
        const int64_t p = s0 + ((int64_t)j << 5) + lane;
        if (col) col[p] = (int32_t)(NQ * c + q2);
        val[p] = v;
        ++j;
        if (q2 == q) {
          if (!(v > 0.0) || !isfinite(v)) atomicOr(err, DEVERR_NONFINITE);
          dinv[r] = 1.0 / v;
        }
      }
      // neighbours across interior faces
      for (int i = 0; i < k; ++i) {
        const int f = L.cf[b0 + i];
        const int32_t f0 = L.f_cell[2 * f], f1 = L.f_cell[2 * f + 1];
        if (f1 < 0) continue;
        const int32_t nb = (f0 == c) ? f1 : f0;
        const int lq = (f0 == c) ? L.f_loc[2 * f + 1] : L.f_loc[2 * f];
        const int kq = (int)(L.cfp[nb + 1] - L.cfp[nb]);
        const int nlq = NFD * kq + NID;
        const double *Bq = L.Bloc + boff(L, nb);
        for (int q2 = 0; q2 < NQ; ++q2) {
          double v = 0.0;
          for (int bt = 0; bt < NFD; ++bt)
            v += Bc[q * nl + i * NFD + bt] * Bq[q2 * nlq + lq * NFD + bt] / diagM[(int64_t)NFD * f + bt];
          const int64_t p = s0 + ((int64_t)j << 5) + lane;
          if (col) col[p] = (int32_t)(NQ * nb + q2);
          val[p] = v;
          ++j;
        }
      }
    }
    for (; j < width; ++j) {
      const int64_t p = s0 + ((int64_t)j << 5) + lane;
      if (col) col[p] = 0;
      val[p] = 0.0;
    }
  }
}

// The B^T part of every flux row of A (its entries in pressure columns, in
// the row's order) copied to kBtRow slots per row (zero-padded; slot k of
// row R at k n_u + R, so a warp's loads of one slot are contiguous), so that
// the block upper-triangular flux update reads 8 entries per row instead of
// the whole row of A (about 100 entries per face row at k = 2).
__global__ void k_bt_rows(int64_t n_u, const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                          const int32_t *__restrict__ col, const double *__restrict__ val, int32_t *bcol,
                          double *bval, int *err) {
  for (int64_t R = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; R < n_u;
       R += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = off[R >> 5] + (R & 31);
    const int L = len[R];
    int k = 0;
    for (int j = 0; j < L; ++j) {
      const int64_t p = base + 32 * (int64_t)j;
      const int64_t c = col[p];
      if (c >= n_u) {
        if (k < kBtRow) {
          bcol[k * n_u + R] = (int32_t)(c - n_u);
          bval[k * n_u + R] = val[p];
        }
        ++k;
      }
    }
    if (k > kBtRow) atomicOr(err, DEVERR_LAYOUT);
    for (; k < kBtRow; ++k) {
      bcol[k * n_u + R] = 0;
      bval[k * n_u + R] = 0.0;
    }
  }
}

static vem_status assemble_global_q(vem_handle *h) {
  cudaStream_t s = h->stream;
  Layout L{h->nfd, h->nid, h->nf, h->nc, h->n_u, h->cf_ptr, h->cf, h->f_cell, h->f_loc,
           h->m_off, h->b_off, h->cls_of, h->Mloc, h->Bloc, h->fbc};
  const int T = 256;
  const int64_t n = h->n;
  if (h->nfd != 6 || h->nid != 14 || h->nq != 4) return fail(h, VEM_ERR_UNSUPPORTED, "element layout");
  if (!h->cnt_buf) VEM_TRY(dalloc_n(h, &h->cnt_buf, (size_t)n + 1));
  int64_t *cnt = h->cnt_buf;
  count_launch(); k_rowcount_q<6, 14, 4><<<grid_for(n, T), T, 0, s>>>(L, cnt);
  VEM_CUDA(h, cudaGetLastError());
  VEM_TRY(sell_layout(h, h->A, n, cnt));
  if (!h->diagM) VEM_TRY(dalloc_n(h, &h->diagM, (size_t)h->n_u));
  if (!h->dinvM) VEM_TRY(dalloc_n(h, &h->dinvM, (size_t)h->n_u));
  const int64_t npad = h->A.nslices * 32;
  count_launch();
  k_fill_q<6, 14, 4><<<grid_for(npad, T), T, 0, s>>>(L, h->A.off, npad, h->A.col, h->A.val, h->diagM, h->dinvM,
                                                     h->nu, h->A.stored);
  VEM_CUDA(h, cudaGetLastError());
  if (h->n_flux_faces > 0) {
    // prescribed flux DOFs: values, A x_fix moved to the right-hand side,
    // symmetric elimination (as for one pressure DOF per cell)
    if (!h->xfix) VEM_TRY(dalloc_n(h, &h->xfix, (size_t)n));
    if (!h->rhs_corr) VEM_TRY(dalloc_n(h, &h->rhs_corr, (size_t)n));
    VEM_CUDA(h, cudaMemsetAsync(h->xfix, 0, sizeof(double) * n, s));
    VEM_TRY(flux_fixed(h, h->xfix));
    spmv(s, h->A, h->xfix, h->rhs_corr);
    count_launch();
    k_eliminate<<<grid_for(n, T), T, 0, s>>>(n, h->A.off, h->A.len, h->A.col, h->A.val, h->nfd, h->nf, h->fbc,
                                            h->diagM, h->dinvM);
    VEM_CUDA(h, cudaGetLastError());
  }
  count_launch(); k_schur_count_q<6, 14, 4><<<grid_for(h->n_p, T), T, 0, s>>>(L, cnt);
  VEM_CUDA(h, cudaGetLastError());
  VEM_TRY(sell_layout(h, h->S, h->n_p, cnt));
  if (!h->s_dinv) VEM_TRY(dalloc_n(h, &h->s_dinv, (size_t)h->n_p));
  const int64_t spad = h->S.nslices * 32;
  count_launch();
  k_schur_fill_q<6, 14, 4><<<grid_for(spad, T), T, 0, s>>>(L, h->diagM, h->S.off, spad, h->S.col, h->S.val,
                                                           h->s_dinv, h->d_err, h->S.stored);
  VEM_CUDA(h, cudaGetLastError());
  if (h->s32_stored != h->S.stored) {
    dfree(h, h->S_val32);
    h->S_val32 = nullptr;
    VEM_TRY(dalloc_n(h, &h->S_val32, (size_t)h->S.stored));
    h->s32_stored = h->S.stored;
  }
  if (!h->s_dinv32) VEM_TRY(dalloc_n(h, &h->s_dinv32, (size_t)h->n_p));
  count_launch(); k_f64_to_f32<<<grid_for(h->S.stored, T), T, 0, s>>>(h->S.stored, h->S.val, h->S_val32);
  count_launch(); k_f64_to_f32<<<grid_for(h->n_p, T), T, 0, s>>>(h->n_p, h->s_dinv, h->s_dinv32);
  VEM_CUDA(h, cudaGetLastError());
  if (h->bt_rows_n != h->n_u) {
    dfree(h, h->bt_col);
    dfree(h, h->bt_val);
    h->bt_col = nullptr;
    h->bt_val = nullptr;
    h->bt_rows_n = 0;
    VEM_TRY(dalloc_n(h, &h->bt_col, (size_t)kBtRow * h->n_u));
    VEM_TRY(dalloc_n(h, &h->bt_val, (size_t)kBtRow * h->n_u));
    h->bt_rows_n = h->n_u;
  }
  count_launch();
  k_bt_rows<<<grid_for(h->n_u, T), T, 0, s>>>(h->n_u, h->A.off, h->A.len, h->A.col, h->A.val, h->bt_col, h->bt_val,
                                              h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  VEM_TRY(check_device_errors(h, "global assembly"));
  VEM_TRY(sell_nnz(h, h->A));
  VEM_TRY(sell_nnz(h, h->S));
  return VEM_OK;
}

vem_status assemble_global(vem_handle *h) {
  if (h->nq > 1) return assemble_global_q(h);
  cudaStream_t s = h->stream;
  Layout L{h->nfd, h->nid, h->nf, h->nc, h->n_u, h->cf_ptr, h->cf, h->f_cell, h->f_loc,
           h->m_off, h->b_off, h->cls_of, h->Mloc, h->Bloc, h->fbc};
  const int T = 256;
  const int64_t n = h->n;
  // ---- [M B^T; B 0] ----
  if (!h->cnt_buf) VEM_TRY(dalloc_n(h, &h->cnt_buf, (size_t)n + 1));
  int64_t *cnt = h->cnt_buf;
  count_launch(); k_rowcount<<<grid_for(n, T), T, 0, s>>>(L, cnt);
  VEM_CUDA(h, cudaGetLastError());
  VEM_TRY(sell_layout(h, h->A, n, cnt));
  if (!h->diagM) VEM_TRY(dalloc_n(h, &h->diagM, (size_t)h->n_u));
  if (!h->dinvM) VEM_TRY(dalloc_n(h, &h->dinvM, (size_t)h->n_u));
  const int64_t npad = h->A.nslices * 32;
  launch_fill(s, h->nfd, dim3(grid_for(npad, T)), L, h->A.off, h->A.len, npad, h->A.col, h->A.val, h->diagM,
              h->dinvM, h->nu, h->A.stored);
  VEM_CUDA(h, cudaGetLastError());
  if (h->n_flux_faces > 0) {
    // prescribed flux DOFs: values, A x_fix with the full matrix (moved to the
    // right-hand side), then the symmetric elimination
    if (!h->xfix) VEM_TRY(dalloc_n(h, &h->xfix, (size_t)n));
    if (!h->rhs_corr) VEM_TRY(dalloc_n(h, &h->rhs_corr, (size_t)n));
    VEM_CUDA(h, cudaMemsetAsync(h->xfix, 0, sizeof(double) * n, s));
    VEM_TRY(flux_fixed(h, h->xfix));
    spmv(s, h->A, h->xfix, h->rhs_corr);
    count_launch();
    k_eliminate<<<grid_for(n, T), T, 0, s>>>(n, h->A.off, h->A.len, h->A.col, h->A.val, h->nfd, h->nf, h->fbc,
                                            h->diagM, h->dinvM);
    VEM_CUDA(h, cudaGetLastError());
  }
  // ---- S ----
  count_launch(); k_schur_count<<<grid_for(h->nc, T), T, 0, s>>>(L, cnt);
  VEM_CUDA(h, cudaGetLastError());
  VEM_TRY(sell_layout(h, h->S, h->nc, cnt));
  if (!h->s_dinv) VEM_TRY(dalloc_n(h, &h->s_dinv, (size_t)h->nc));
  const int64_t spad = h->S.nslices * 32;
  count_launch(); k_schur_fill<<<grid_for(spad, T), T, 0, s>>>(L, h->diagM, h->S.off, spad, h->S.col, h->S.val,
                                                          h->s_dinv, h->d_err, h->S.stored);
  VEM_CUDA(h, cudaGetLastError());
  // FP32 copies of S for the mixed-precision inner solve
  if (h->s32_stored != h->S.stored) {
    dfree(h, h->S_val32);
    h->S_val32 = nullptr;
    VEM_TRY(dalloc_n(h, &h->S_val32, (size_t)h->S.stored));
    h->s32_stored = h->S.stored;
  }
  if (!h->s_dinv32) VEM_TRY(dalloc_n(h, &h->s_dinv32, (size_t)h->nc));
  count_launch(); k_f64_to_f32<<<grid_for(h->S.stored, T), T, 0, s>>>(h->S.stored, h->S.val, h->S_val32);
  count_launch(); k_f64_to_f32<<<grid_for(h->nc, T), T, 0, s>>>(h->nc, h->s_dinv, h->s_dinv32);
  VEM_CUDA(h, cudaGetLastError());
  if (!h->bt_face) VEM_TRY(dalloc_n(h, &h->bt_face, 2 * (size_t)h->nf));
  count_launch(); k_bt_face<<<grid_for(h->nf, T), T, 0, s>>>(L, h->bt_face);
  VEM_CUDA(h, cudaGetLastError());
  VEM_TRY(check_device_errors(h, "global assembly"));
  // true nonzero counts (for statistics)
  VEM_TRY(sell_nnz(h, h->A));
  VEM_TRY(sell_nnz(h, h->S));
  return VEM_OK;
}

vem_status assemble_reg(vem_handle *h, bool fp32) {
  cudaStream_t s = h->stream;
  Layout L{h->nfd, h->nid, h->nf, h->nc, h->n_u, h->cf_ptr, h->cf, h->f_cell, h->f_loc,
           h->m_off, h->b_off, h->cls_of, h->Mloc, h->Bloc, h->fbc};
  const int T = 256;
  amg_invalidate(h->amg_reg);   // its level 0 is a view of the matrix rebuilt here
  h->areg_valid = false;
  // gamma = h^2 with h the mean cell diameter (eq. meshSize), unless given
  double gamma = h->opt.reg_gamma;
  if (!(gamma > 0.0)) {
    double sum = 0.0;
    VEM_TRY(device_sum(h, h->nc, h->c_diam, &sum));
    const double hm = sum / (double)h->nc;
    gamma = hm * hm;
  }
  if (!(gamma > 0.0) || !std::isfinite(gamma)) return fail(h, VEM_ERR_BAD_INPUT, "Block-Reg: gamma %g", gamma);
  h->reg_gamma = gamma;
  if (!h->cnt_buf) VEM_TRY(dalloc_n(h, &h->cnt_buf, (size_t)h->n + 1));
  int64_t *cnt = h->cnt_buf;
  count_launch(); k_reg_count<<<grid_for(h->n_u, T), T, 0, s>>>(L, cnt);
  VEM_CUDA(h, cudaGetLastError());
  VEM_TRY(sell_layout(h, h->Areg, h->n_u, cnt));
  const int64_t npad = h->Areg.nslices * 32;
  count_launch();
  k_reg_fill<<<grid_for(npad, T), T, 0, s>>>(L, h->nq, h->Areg.off, npad, h->Areg.col, h->Areg.val, h->nu,
                                             1.0 / gamma);
  VEM_CUDA(h, cudaGetLastError());
  if (h->n_flux_faces > 0) {
    count_launch();
    k_eliminate<<<grid_for(h->n_u, T), T, 0, s>>>(h->n_u, h->Areg.off, h->Areg.len, h->Areg.col, h->Areg.val,
                                                 h->nfd, h->nf, h->fbc, nullptr, nullptr);
    VEM_CUDA(h, cudaGetLastError());
  }
  if (fp32) {
    if (h->areg32_stored != h->Areg.stored) {
      dfree(h, h->Areg_val32);
      h->Areg_val32 = nullptr;
      VEM_TRY(dalloc_n(h, &h->Areg_val32, (size_t)h->Areg.stored));
      h->areg32_stored = h->Areg.stored;
    }
    count_launch();
    k_f64_to_f32<<<grid_for(h->Areg.stored, T), T, 0, s>>>(h->Areg.stored, h->Areg.val, h->Areg_val32);
    VEM_CUDA(h, cudaGetLastError());
  }
  VEM_TRY(sell_nnz(h, h->Areg));
  h->areg_has32 = fp32;
  h->areg_valid = true;
  return VEM_OK;
}

// ---------------------------------------------------------------- classes --
// Cells that are translates of one another (same vertex offsets from the
// barycentre, same face and vertex order, same orientations) have the same
// geometry-only local matrices.  Each cell gets a key hashed from its vertex
// offsets quantised at 2^-40 of the mesh diagonal; equal keys go to one
// hash-table slot whose smallest cell id represents the class, and every cell
// is checked against its representative exactly (quantised values) before it
// joins the class.
__device__ __forceinline__ uint64_t mix64(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
  h *= 0xff51afd7ed558ccdULL;
  return h ^ (h >> 33);
}

__device__ __forceinline__ long long qcoord(double v, double x, double inv_q) { return llrint((v - x) * inv_q); }

__global__ void k_class_key(int64_t nc, const int64_t *__restrict__ cfp, const int32_t *__restrict__ cf,
                            const int64_t *__restrict__ fvp, const int32_t *__restrict__ fv,
                            const double *__restrict__ xyz, const double *__restrict__ c_cent,
                            const int8_t *__restrict__ sig, double inv_q, uint64_t *key) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = cfp[c];
    const int k = (int)(cfp[c + 1] - b);
    const double x0 = c_cent[3 * c], x1 = c_cent[3 * c + 1], x2 = c_cent[3 * c + 2];
    uint64_t h = mix64(0x1234567ULL, (uint64_t)k);
    for (int i = 0; i < k; ++i) {
      const int f = cf[b + i];
      h = mix64(h, (uint64_t)(sig[b + i] + 2));
      h = mix64(h, (uint64_t)(fvp[f + 1] - fvp[f]));
      for (int64_t p = fvp[f]; p < fvp[f + 1]; ++p) {
        const int64_t v = fv[p];
        h = mix64(h, (uint64_t)qcoord(xyz[3 * v], x0, inv_q));
        h = mix64(h, (uint64_t)qcoord(xyz[3 * v + 1], x1, inv_q));
        h = mix64(h, (uint64_t)qcoord(xyz[3 * v + 2], x2, inv_q));
      }
    }
    key[c] = h | 1ULL;
  }
}

__global__ void k_class_insert(int64_t nc, const uint64_t *__restrict__ key, unsigned long long *tkey,
                               int *trep, uint64_t mask) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = key[c];
    uint64_t s = (k ^ (k >> 31)) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      const unsigned long long prev = atomicCAS(&tkey[s], 0ULL, k);
      if (prev == 0ULL || prev == k) {
        atomicMin(&trep[s], (int)c);
        break;
      }
      s = (s + 1) & mask;
    }
  }
}

// rep[c] from the table, then the exact check against the representative
__global__ void k_class_lookup(int64_t nc, const uint64_t *__restrict__ key,
                               const unsigned long long *__restrict__ tkey, const int *__restrict__ trep,
                               uint64_t mask, const int64_t *__restrict__ cfp, const int32_t *__restrict__ cf,
                               const int64_t *__restrict__ fvp, const int32_t *__restrict__ fv,
                               const double *__restrict__ xyz, const double *__restrict__ c_cent,
                               const int8_t *__restrict__ sig, double inv_q, int32_t *rep) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = key[c];
    uint64_t s = (k ^ (k >> 31)) & mask;
    int r = (int)c;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      if (tkey[s] == k) {
        r = trep[s];
        break;
      }
      s = (s + 1) & mask;
    }
    bool same = r != (int)c;
    if (same) {
      const int64_t b = cfp[c], br = cfp[r];
      const int kc = (int)(cfp[c + 1] - b);
      same = kc == (int)(cfp[r + 1] - br);
      for (int i = 0; same && i < kc; ++i) {
        const int f = cf[b + i], g = cf[br + i];
        const int64_t m = fvp[f + 1] - fvp[f];
        same = sig[b + i] == sig[br + i] && m == fvp[g + 1] - fvp[g];
        for (int64_t p = 0; same && p < m; ++p) {
          const int64_t v = fv[fvp[f] + p], w = fv[fvp[g] + p];
          for (int d = 0; d < 3; ++d)
            same = same && qcoord(xyz[3 * v + d], c_cent[3 * c + d], inv_q) ==
                               qcoord(xyz[3 * w + d], c_cent[3 * r + d], inv_q);
        }
      }
    }
    rep[c] = same ? r : (int)c;
  }
}

__global__ void k_class_flags(int64_t nc, const int32_t *__restrict__ rep, int64_t *flag) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x)
    flag[c] = rep[c] == (int32_t)c ? 1 : 0;
}

// idx = exclusive scan of the flags: class of c = idx[rep[c]]; class sizes
__global__ void k_class_assign(int64_t nc, int nfd, int nid, int nq, const int32_t *__restrict__ rep,
                               const int64_t *__restrict__ idx, const int64_t *__restrict__ cfp,
                               int32_t *cls_of, int32_t *cls_rep, int64_t *msz, int64_t *bsz) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = idx[rep[c]];
    cls_of[c] = (int32_t)k;
    if (rep[c] == (int32_t)c) {
      cls_rep[k] = (int32_t)c;
      const int64_t nl = nfd * (cfp[c + 1] - cfp[c]) + nid;
      msz[k] = nl * nl;
      bsz[k] = nq * nl;
    }
  }
}

vem_status classify_cells(vem_handle *h) {
  // the classes are a property of the mesh (and of the element's local sizes
  // and the reuse option): computed once per handle, with the geometry
  if (h->cls_valid && h->cls_nfd == h->nfd && h->cls_nid == h->nid && h->cls_reuse == h->opt.reuse)
    return VEM_OK;
  h->cls_valid = false;
  cudaStream_t s = h->stream;
  const int T = 256;
  const int64_t nc = h->nc;
  if (!h->cls_of) VEM_TRY(dalloc_n(h, &h->cls_of, (size_t)nc));
  if (!h->cls_rep) VEM_TRY(dalloc_n(h, &h->cls_rep, (size_t)nc));
  if (!h->m_off) VEM_TRY(dalloc_n(h, &h->m_off, (size_t)nc + 1));
  if (!h->b_off) VEM_TRY(dalloc_n(h, &h->b_off, (size_t)nc + 1));
  uint64_t tsize = 1;
  while (tsize < 2 * (uint64_t)nc) tsize <<= 1;
  // persistent scratch (sizes depend on the mesh only)
  const size_t need = sizeof(uint64_t) * (3 * (size_t)tsize / 2 + 6 * (size_t)nc + 8);
  if (h->cls_scratch_bytes < need) {
    dfree(h, h->cls_scratch);
    h->cls_scratch = nullptr;
    VEM_TRY(dalloc(h, &h->cls_scratch, need));
    h->cls_scratch_bytes = need;
  }
  char *sp = static_cast<char *>(h->cls_scratch);
  unsigned long long *tkey = reinterpret_cast<unsigned long long *>(sp);
  sp += sizeof(unsigned long long) * tsize;
  int *trep = reinterpret_cast<int *>(sp);
  sp += sizeof(int) * tsize;
  uint64_t *key = reinterpret_cast<uint64_t *>(sp);
  sp += sizeof(uint64_t) * nc;
  int64_t *flag = reinterpret_cast<int64_t *>(sp);
  sp += sizeof(int64_t) * nc;
  int64_t *idx = reinterpret_cast<int64_t *>(sp);
  sp += sizeof(int64_t) * (nc + 1);
  int64_t *msz = reinterpret_cast<int64_t *>(sp);
  sp += sizeof(int64_t) * nc;
  int64_t *bsz = reinterpret_cast<int64_t *>(sp);
  sp += sizeof(int64_t) * nc;
  int32_t *rep = reinterpret_cast<int32_t *>(sp);
  const double inv_q = 1099511627776.0 / h->lref;   // 2^40 / diagonal
  if (h->opt.reuse) {
    VEM_CUDA(h, cudaMemsetAsync(tkey, 0, sizeof(unsigned long long) * tsize, s));
    VEM_CUDA(h, cudaMemsetAsync(trep, 0x7f, sizeof(int) * tsize, s));
    count_launch();
    k_class_key<<<grid_for(nc, T), T, 0, s>>>(nc, h->cf_ptr, h->cf, h->fv_ptr, h->fv, h->xyz, h->c_cent,
                                               h->cf_sigma, inv_q, key);
    count_launch();
    k_class_insert<<<grid_for(nc, T), T, 0, s>>>(nc, key, tkey, trep, tsize - 1);
    count_launch();
    k_class_lookup<<<grid_for(nc, T), T, 0, s>>>(nc, key, tkey, trep, tsize - 1, h->cf_ptr, h->cf, h->fv_ptr,
                                                  h->fv, h->xyz, h->c_cent, h->cf_sigma, inv_q, rep);
  } else {
    count_launch();
    k_iota32<<<grid_for(nc, T), T, 0, s>>>(nc, rep);
  }
  count_launch();
  k_class_flags<<<grid_for(nc, T), T, 0, s>>>(nc, rep, flag);
  VEM_CUDA(h, cudaGetLastError());
  int64_t ncls = 0;
  VEM_TRY(scan_counts(h, nc, flag, idx, &ncls));
  count_launch();
  k_class_assign<<<grid_for(nc, T), T, 0, s>>>(nc, h->nfd, h->nid, h->nq, rep, idx, h->cf_ptr, h->cls_of, h->cls_rep,
                                                msz, bsz);
  VEM_CUDA(h, cudaGetLastError());
  int64_t mt = 0, bt = 0;
  VEM_TRY(scan_counts(h, ncls, msz, h->m_off, &mt));
  VEM_TRY(scan_counts(h, ncls, bsz, h->b_off, &bt));
  h->ncls = ncls;
  if (h->m_total != mt || !h->Mloc) {
    dfree(h, h->Mloc);
    h->Mloc = nullptr;
    VEM_TRY(dalloc_n(h, &h->Mloc, (size_t)mt));
    h->m_total = mt;
  }
  if (h->b_total != bt || !h->Bloc) {
    dfree(h, h->Bloc);
    h->Bloc = nullptr;
    VEM_TRY(dalloc_n(h, &h->Bloc, (size_t)bt));
    h->b_total = bt;
  }
  h->cls_valid = true;
  h->cls_nfd = h->nfd;
  h->cls_nid = h->nid;
  h->cls_reuse = h->opt.reuse;
  return VEM_OK;
}

// Values of nb systems that share the mesh and the structure of h->A / h->S:
// A_b, diag(M_b) and its reciprocal, S_b, 1/diag(S_b) (and FP32 copies), from local matrices
// computed with nu = 1 and scaled per cell by nu_b = 1/K_b.
vem_status assemble_batched_values(vem_handle *h, int nb, const double *nu_b, VemOp &op) {
  cudaStream_t s = h->stream;
  Layout L{h->nfd, h->nid, h->nf, h->nc, h->n_u, h->cf_ptr, h->cf, h->f_cell, h->f_loc,
           h->m_off, h->b_off, h->cls_of, h->Mloc, h->Bloc, h->fbc};
  const int T = 256;
  const int64_t npad = h->A.nslices * 32, spad = h->S.nslices * 32;
  dim3 ga(grid_for(npad, T, 2), nb), gs(grid_for(spad, T, 2), nb);
  if (h->nq > 1) {
    if (h->nfd != 6 || h->nid != 14 || h->nq != 4) return fail(h, VEM_ERR_UNSUPPORTED, "element layout");
    count_launch();
    k_fill_q<6, 14, 4><<<ga, T, 0, s>>>(L, h->A.off, npad, nullptr, op.A.val, op.diagM, op.dinvM, nu_b,
                                        h->A.stored);
    count_launch();
    k_schur_fill_q<6, 14, 4><<<gs, T, 0, s>>>(L, op.diagM, h->S.off, spad, nullptr, op.S.val, op.s_dinv, h->d_err,
                                              h->S.stored);
  } else {
    launch_fill(s, h->nfd, ga, L, h->A.off, h->A.len, npad, nullptr, op.A.val, op.diagM, op.dinvM, nu_b,
                h->A.stored);
    count_launch();
    k_schur_fill<<<gs, T, 0, s>>>(L, op.diagM, h->S.off, spad, nullptr, op.S.val, op.s_dinv, h->d_err,
                                  h->S.stored);
  }
  count_launch();
  k_f64_to_f32<<<grid_for(nb * h->S.stored, T), T, 0, s>>>(nb * h->S.stored, op.S.val, op.S_val32);
  count_launch();
  k_f64_to_f32<<<grid_for(nb * h->n_p, T), T, 0, s>>>(nb * h->n_p, op.s_dinv, op.s_dinv32);
  VEM_CUDA(h, cudaGetLastError());
  return check_device_errors(h, "batched assembly");
}

}  // namespace vem
