// Smoothed-aggregation algebraic multigrid: the setup (strength of
// connection, distance-2 independent set, aggregates, smoothed prolongator,
// Galerkin coarse operators) and the symmetric V-cycle.  Two hierarchies use
// it: one of the Schur block S (the cycle preconditions the inner CG) and one
// of the regularised flux block A + B^T B / gamma of Block-Reg.
//
// The paper solves S exactly inside Block-Schur and uses a smoothed-
// aggregation AMG (PETSc GAMG) for the velocity block of Block-Reg (Sec. 5);
// this AMG is the library's inner solver option for S and its Block-Reg
// flux-block preconditioner.  Method: Vanek,
// Mandel & Brezina, Computing 56 (1996) (smoothed aggregation); Bell, Dalton &
// Olson, SIAM J. Sci. Comput. 34 (2012) (aggregates from a distance-2 maximal
// independent set found in parallel rounds).  Rules, whose integer decisions
// are exact:
//   strong(i,j): j != i and |a_ij| >= theta sqrt(a_ii a_jj), a_ij read from
//     row i; theta = 0.08 on the finest level, halved on every coarser one;
//   key(i) = ((splitmix64(i) >> 34) << 32) | i (SplitMix64 output function,
//     Steele, Lea & Flood, OOPSLA 2014); a round makes a node a root when its
//     (state, key) is the largest in its distance-2 ball and retires it when
//     a root is in the ball, which yields the greedy set in decreasing key
//     order;
//   isolated nodes (no strong entry) have no aggregate (zero row of P);
//   pass 1: join the smallest root aggregate among the strong neighbours
//     (roots numbered by index, isolated roots not counted);
//   pass 2: join the smallest pass-1 aggregate among the strong neighbours;
//   pass 3: remaining non-isolated nodes become singletons after the roots;
//   P = T - omega_F D^-1 A^F T with A^F = diagonal + strong entries and
//     omega_F = 4 / (3 max_i sum_j |a^F_ij| / a_ii);
//   Jacobi weight omega = 4 / (3 max_i sum_j |a_ij| / a_ii);
//   coarsening stops at <= 64 rows, when a level would keep more than 4/5 of
//     its rows or none, or at 12 levels; the coarsest level is inverted
//     (dense Gauss-Jordan) up to 512 rows, else gets 4 Jacobi sweeps.
// Smoothers: one damped-Jacobi step before and after the coarse correction
// (the S hierarchy), or two steps of Chebyshev acceleration of the Jacobi
// iteration (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed.,
// Alg. 12.1, on [rho/10, rho] with rho the Gershgorin bound above), the
// default smoother of GAMG (the Block-Reg hierarchy).
// The products P, A P and P^T (A P) are formed row by row, one thread per
// row holding the row's distinct columns in a small sorted list and summing
// contributions in a fixed order, so the hierarchy is bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "handle.cuh"

namespace vem {

constexpr int kMaxLevels = 12;
constexpr int kCoarseMax = 64;
constexpr int kDenseMax = 512;
constexpr int kCoarseSweeps = 4;
constexpr double kTheta0 = 0.08;
constexpr int kCapP = 128;       // distinct columns of a row of P
constexpr int kHashBits = 9;     // per-warp hash table of a product row: 512 slots
constexpr int kBigBits = 13;     // rows that overflow it: one warp, 8192 slots
constexpr int kBigMax = 6144;    // distinct columns of a product row
constexpr int kSortMax = 512;    // entries of a row sorted by one warp
constexpr int kProdWarps = 4;    // warps per block of the product kernels
constexpr int kCapThreadRow = 64;  // distinct columns of a thread-per-row product row
constexpr int64_t kSellMinRows = 65536;  // smaller cycle operators stay in CSR
constexpr int kMaxRounds = 200;

constexpr uint64_t kStIn = 2ull << 62, kStUnd = 1ull << 62;

// A CSR matrix in device memory with the capacities of its buffers (grown,
// never shrunk) and the lanes per row used to apply it.
struct CsrBuf {
  int64_t rows = 0, cols = 0, nnz = 0;
  int64_t *rp = nullptr;
  int32_t *col = nullptr;
  double *val = nullptr;
  size_t c_rp = 0, c_nz = 0;
  int lanes = 4;
  float *val32 = nullptr;   // FP32 copy of the values (FP32 cycle)
  size_t c_v32 = 0;
};

// A SELL-32 copy of a CSR matrix for the cycle, with buffer capacities.
struct SellBuf {
  SellMat m;
  size_t c_off = 0, c_len = 0, c_st = 0;
  float *val32 = nullptr;   // FP32 copy of the values (FP32 cycle)
  size_t c_v32 = 0;
};

struct AmgLevel {
  CsrBuf A;                 // levels >= 1 (level 0 is the handle's S in SELL-32)
  CsrBuf P, R;              // prolongator n x nc and restriction R = P^T
  SellBuf As, Rs, Ps;       // SELL-32 copies of A (levels >= 1), R and P for the cycle
  double *dinv = nullptr;
  double *wd = nullptr;     // omega * dinv (the Jacobi step)
  size_t c_wd = 0;
  float *wd32 = nullptr, *vec32 = nullptr;   // FP32 cycle: wd and x, x2, b, r
  size_t c_wd32 = 0, c_vec32 = 0;
  int32_t *agg = nullptr;
  double *vec = nullptr;    // x, x2, b, r (and xc for Chebyshev): vectors of n
  size_t c_dinv = 0, c_agg = 0, c_vec = 0;
  double *wdc = nullptr;    // Chebyshev: (2 rho_1 / delta) D^-1 (the second step)
  size_t c_wdc = 0;
  float *wdc32 = nullptr;
  size_t c_wdc32 = 0;
  double omega = 0.0;
  int mis_rounds = 0;       // MIS-2 rounds this level needed in the last setup
  double rho = 0.0;         // Gershgorin bound of rho(D^-1 A) (point blocks: the estimate below)
  double cheb_c = 0.0;      // Chebyshev: rho_1 rho_0 (the second step)
  // point blocks (block hierarchies): bs x bs diagonal blocks D_I, row-major
  int bs = 1;
  double *dblk = nullptr;   // D_I^-1
  double *lblk = nullptr;   // L_I^-1 with D_I = L_I L_I^T
  size_t c_dblk = 0, c_lblk = 0;
  double *bns = nullptr;    // near-null space of this level (levels >= 1; rows x m)
  size_t c_bns = 0;
  double cheb_theta = 0.0, cheb_w2 = 0.0;   // block Chebyshev: 1 / theta and 2 rho_1 / delta
  int64_t n = 0, nc = 0;
  double *x() const { return vec; }
  double *x2() const { return vec + n; }
  double *b() const { return vec + 2 * n; }
  double *r() const { return vec + 3 * n; }
  template <class T> T *vx(int k) const;
};
template <> double *AmgLevel::vx<double>(int k) const { return vec + k * n; }
template <> float *AmgLevel::vx<float>(int k) const { return vec32 + k * n; }

struct AmgState {
  AmgLevel lv[kMaxLevels];
  int smoother = kSmoothJacobi;
  bool pin_last = false;    // singular level-0 operator (constants): pin the coarsest
  SellMat S0;               // level 0 operator (a view of the handle's S or A_reg)
  const float *S0_val32 = nullptr;   // its FP32 values (the handle's copy)
  bool fp32 = false;                 // cycle in FP32
  int64_t generation = 0;            // counts setups (graphs of the cycle key on it)
  float *cinv32 = nullptr;
  size_t c_cinv32 = 0;
  int nlev = 0;
  bool valid = false;
  double *cinv = nullptr;   // dense inverse of the coarsest level
  size_t c_cinv = 0;
  int csweeps = 0;
  // setup scratch
  uint8_t *flag = nullptr;  size_t c_flag = 0;
  int32_t *nstr = nullptr;  size_t c_nstr = 0;
  uint64_t *tup = nullptr;  size_t c_tup = 0;     // tuples and t1: 2 n
  int64_t *cnt = nullptr;   size_t c_cnt = 0;     // counts (n + 1)
  int *bflag = nullptr;                           // block-row pattern check
  int64_t *scn = nullptr;   size_t c_scn = 0;     // scans (n + 1)
  int32_t *agg1 = nullptr;  size_t c_agg1 = 0;
  double *dg = nullptr;     size_t c_dg = 0;      // diagonal
  unsigned long long *ctr = nullptr;              // [kMaxRounds + 4] counters / maxima
  CsrBuf AP;
  int64_t *cur = nullptr;   size_t c_cur = 0;     // transpose cursors
  uint8_t *big = nullptr;   size_t c_big = 0;     // product rows for the large table
  int64_t *coff = nullptr;  size_t c_coff = 0;    // one-pass product: scratch row offsets
  int32_t *tcol = nullptr;  size_t c_tcol = 0;    //   and the scratch rows
  double *tval = nullptr;   size_t c_tval = 0;
  double t_setup_ms = 0.0;
  // point-block hierarchy: level-0 block size and near-null space (m columns)
  bool block = false;
  int m = 0;
  const double *B0 = nullptr;
  CsrBuf bQ, bQT, bAQ, bN, bT, bZ, bAgg, bAggT, bLm, bLmT, bY, bC;   // block setup scratch
  double *sq = nullptr;     size_t c_sq = 0;      // squared values of the level operator
  double *dgb = nullptr;    size_t c_dgb = 0;     // diagonal of the block graph
  double *dgbi = nullptr;   size_t c_dgbi = 0;
  double *lz = nullptr;     size_t c_lz = 0;      // Lanczos basis (n x 11) and w
  double *lpart = nullptr;  size_t c_lpart = 0;   // partial sums of the Lanczos dots
  // condensed Block-Reg: A_reg's parts, A_ii^-1 and the face system in SELL-32
  bool condensed = false;
  int64_t nfr = 0, nint = 0;
  int nid = 0;
  CsrBuf cAff, cAfi, cAif, cAii, cSf;
  SellBuf cSell;
  double *aii_inv = nullptr; size_t c_aii = 0;
  double *cvec = nullptr;    size_t c_cvec = 0;   // nint + nfr scratch of the apply
  cudaEvent_t tev[4] = {};  // level-0 residual and post-smoothing launches of a timed cycle
  bool timing = false, timed = false;
  cudaEvent_t sev[2] = {};  // the condensed setup's time
  ~AmgState() {
    for (cudaEvent_t &e : tev)
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t &e : sev)
      if (e) cudaEventDestroy(e);
  }
};

template <class T>
static vem_status grow(vem_handle *h, T *&p, size_t &cap, size_t n) {
  if (p && n <= cap) return VEM_OK;
  dfree(h, p);
  p = nullptr;
  cap = 0;
  const size_t c = n + n / 4 + 64;
  VEM_TRY(dalloc_n(h, &p, c));
  cap = c;
  return VEM_OK;
}


// Device view of a SELL-32 (off != nullptr) or CSR matrix: entry k of row i
// sits at position base + stride * k.
struct DMat {
  const int64_t *off = nullptr;
  const int32_t *len = nullptr;
  const int64_t *rp = nullptr;
  const int32_t *col = nullptr;
  const double *val = nullptr;
  int64_t rows = 0, stored = 0;
  __device__ __forceinline__ void row(int64_t i, int64_t &base, int &stride, int &L) const {
    if (off) {
      base = off[i >> 5] + (i & 31);
      stride = 32;
      L = len[i];
    } else {
      base = rp[i];
      stride = 1;
      L = (int)(rp[i + 1] - base);
    }
  }
};

static DMat dview(const SellMat &m) {
  DMat d;
  d.off = m.off;
  d.len = m.len;
  d.col = m.col;
  d.val = m.val;
  d.rows = m.rows;
  d.stored = m.stored;
  return d;
}

static DMat dview(const CsrBuf &m) {
  DMat d;
  d.rp = m.rp;
  d.col = m.col;
  d.val = m.val;
  d.rows = m.rows;
  d.stored = m.nnz;
  return d;
}

// ------------------------------------------------------------ helpers -----
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t node_key(int64_t i) {
  return ((splitmix64((uint64_t)i) >> 34) << 32) | (uint64_t)i;
}

// A row's distinct columns kept sorted, with values summed in arrival order.
template <int CAP>
struct RowMap {
  int32_t key[CAP];
  double val[CAP];
  int n = 0;
  __device__ __forceinline__ bool add(int32_t k, double v) {
    int lo = 0, hi = n;
    while (lo < hi) {
      const int m = (lo + hi) >> 1;
      if (key[m] < k) lo = m + 1;
      else hi = m;
    }
    if (lo < n && key[lo] == k) {
      val[lo] += v;
      return true;
    }
    if (n == CAP) return false;
    for (int t = n; t > lo; --t) {
      key[t] = key[t - 1];
      val[t] = val[t - 1];
    }
    key[lo] = k;
    val[lo] = v;
    ++n;
    return true;
  }
};

#define ROWS_LOOP(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// --------------------------------------------------------- strength -------
__global__ void k_amg_diag(DMat A, double *dg, double *dinv, int *err) {
  ROWS_LOOP(i, A.rows) {
    int64_t base;
    int st, L;
    A.row(i, base, st, L);
    double d = 0.0;
    for (int k = 0; k < L; ++k)
      if (A.col[base + (int64_t)st * k] == (int32_t)i) d = A.val[base + (int64_t)st * k];
    if (!(d > 0.0) || !isfinite(d)) {
      atomicOr(err, DEVERR_AMG_DIAG);
      d = 1.0;
    }
    dg[i] = d;
    dinv[i] = 1.0 / d;
  }
}

// Strong flags per stored entry, strong count per row and the two Gershgorin
// maxima (non-negative doubles compared as their bit patterns).
__global__ void k_amg_strength(DMat A, const double *__restrict__ dg, double theta, uint8_t *flag, int32_t *nstr,
                               unsigned long long *mx) {
  double rho = 0.0, rhof = 0.0;
  ROWS_LOOP(i, A.rows) {
    int64_t base;
    int stp, L;
    A.row(i, base, stp, L);
    const double di = dg[i];
    double sa = 0.0, sf = 0.0;
    int ns = 0;
    for (int k = 0; k < L; ++k) {
      const int64_t p = base + (int64_t)stp * k;
      const int32_t j = A.col[p];
      const double a = fabs(A.val[p]);
      sa += a;
      bool st = false;
      if (j != (int32_t)i) st = a >= theta * sqrt(di * dg[j]);
      else sf += a;
      if (st) {
        sf += a;
        ++ns;
      }
      flag[p] = st ? 1 : 0;
    }
    nstr[i] = ns;
    rho = fmax(rho, sa / di);
    rhof = fmax(rhof, sf / di);
  }
  for (int o = 16; o > 0; o >>= 1) {
    rho = fmax(rho, __shfl_xor_sync(0xffffffffu, rho, o));
    rhof = fmax(rhof, __shfl_xor_sync(0xffffffffu, rhof, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(mx, (unsigned long long)__double_as_longlong(rho));
    atomicMax(mx + 1, (unsigned long long)__double_as_longlong(rhof));
  }
}

// ------------------------------------------------------------ MIS-2 -------
__global__ void k_mis_init(int64_t n, uint64_t *tup) {
  ROWS_LOOP(i, n) tup[i] = kStUnd | node_key(i);
}

__global__ void k_mis_max1(DMat A, const uint8_t *__restrict__ flag, const uint64_t *__restrict__ tup, uint64_t *t1) {
  ROWS_LOOP(i, A.rows) {
    int64_t base;
    int st, L;
    A.row(i, base, st, L);
    uint64_t m = tup[i];
    for (int k = 0; k < L; ++k) {
      const int64_t p = base + (int64_t)st * k;
      if (flag[p]) m = max(m, tup[A.col[p]]);
    }
    t1[i] = m;
  }
}

__global__ void k_mis_max2(DMat A, const uint8_t *__restrict__ flag, const uint64_t *__restrict__ t1, uint64_t *tup,
                           unsigned long long *und) {
  unsigned long long c = 0;
  ROWS_LOOP(i, A.rows) {
    const uint64_t own = tup[i];
    if ((own >> 62) != 1) continue;
    int64_t base;
    int st, L;
    A.row(i, base, st, L);
    uint64_t m = t1[i];
    for (int k = 0; k < L; ++k) {
      const int64_t p = base + (int64_t)st * k;
      if (flag[p]) m = max(m, t1[A.col[p]]);
    }
    const uint64_t key = own & ~(3ull << 62);
    if (m == own) tup[i] = kStIn | key;
    else if ((m >> 62) == 2) tup[i] = key;
    else ++c;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(und, c);
}

// -------------------------------------------------------- aggregates ------
__global__ void k_agg_root(int64_t n, const uint64_t *__restrict__ tup, const int32_t *__restrict__ nstr,
                           int64_t *cnt) {
  ROWS_LOOP(i, n) cnt[i] = ((tup[i] >> 62) == 2 && nstr[i] > 0) ? 1 : 0;
}

__global__ void k_agg_pass1(DMat A, const uint8_t *__restrict__ flag, const uint64_t *__restrict__ tup,
                            const int32_t *__restrict__ nstr, const int64_t *__restrict__ rid, int32_t *agg1) {
  ROWS_LOOP(i, A.rows) {
    int32_t a = -1;
    if (nstr[i] > 0) {
      if ((tup[i] >> 62) == 2) {
        a = (int32_t)rid[i];
      } else {
        int64_t base;
        int st, L;
        A.row(i, base, st, L);
        for (int k = 0; k < L; ++k) {
          const int64_t p = base + (int64_t)st * k;
          if (!flag[p]) continue;
          const int32_t j = A.col[p];
          if ((tup[j] >> 62) == 2 && nstr[j] > 0) {
            const int32_t r = (int32_t)rid[j];
            if (a < 0 || r < a) a = r;
          }
        }
      }
    }
    agg1[i] = a;
  }
}

__global__ void k_agg_pass2(DMat A, const uint8_t *__restrict__ flag, const int32_t *__restrict__ nstr,
                            const int32_t *__restrict__ agg1, int32_t *agg, int64_t *freecnt) {
  ROWS_LOOP(i, A.rows) {
    int32_t a = agg1[i];
    if (a < 0 && nstr[i] > 0) {
      int64_t base;
      int st, L;
      A.row(i, base, st, L);
      for (int k = 0; k < L; ++k) {
        const int64_t p = base + (int64_t)st * k;
        if (!flag[p]) continue;
        const int32_t b = agg1[A.col[p]];
        if (b >= 0 && (a < 0 || b < a)) a = b;
      }
    }
    agg[i] = a;
    freecnt[i] = (a < 0 && nstr[i] > 0) ? 1 : 0;
  }
}

__global__ void k_agg_pass3(int64_t n, int64_t nroot, const int32_t *__restrict__ nstr,
                            const int64_t *__restrict__ fid, int32_t *agg) {
  ROWS_LOOP(i, n) {
    if (agg[i] < 0 && nstr[i] > 0) agg[i] = (int32_t)(nroot + fid[i]);
  }
}

// ------------------------------------------------------- prolongator ------
// Row i of P = T - omega_F D^-1 A^F T: columns agg(i) and agg(j) of the
// strong neighbours j; value [I = agg(i)] - omega_F dinv_i sum a_ij over the
// diagonal and the strong entries with agg(j) = I (stored order).
template <bool kFill>
__global__ void k_p_rows(DMat A, const uint8_t *__restrict__ flag, const double *__restrict__ dinv,
                         const int32_t *__restrict__ agg, double omega_f, int64_t *cnt,
                         const int64_t *__restrict__ rp, int32_t *pcol, double *pval, int *err) {
  ROWS_LOOP(i, A.rows) {
    const int32_t ai = agg[i];
    RowMap<kCapP> m;
    bool ok = true;
    if (ai >= 0) {
      int64_t base;
      int st, L;
      A.row(i, base, st, L);
      for (int k = 0; k < L && ok; ++k) {
        const int64_t p = base + (int64_t)st * k;
        const int32_t j = A.col[p];
        if (j == (int32_t)i) {
          ok = m.add(ai, A.val[p]);
        } else if (flag[p]) {
          const int32_t aj = agg[j];
          if (aj >= 0) ok = m.add(aj, A.val[p]);
        }
      }
    }
    if (!ok) atomicOr(err, DEVERR_AMG_ROW);
    if (!kFill) {
      cnt[i] = ok ? m.n : 0;
    } else if (ok) {
      const double di = dinv[i];
      const int64_t o = rp[i];
      for (int t = 0; t < m.n; ++t) {
        pcol[o + t] = m.key[t];
        pval[o + t] = (m.key[t] == ai ? 1.0 : 0.0) - omega_f * (di * m.val[t]);
      }
    }
  }
}

// --------------------------------------------------------- transpose ------
__global__ void k_t_count(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                          unsigned long long *cnt) {
  ROWS_LOOP(i, n) {
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) atomicAdd(cnt + col[p], 1ull);
  }
}

__global__ void k_t_fill(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                         const double *__restrict__ val, unsigned long long *cur, int32_t *tcol, double *tval) {
  ROWS_LOOP(i, n) {
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const unsigned long long q = atomicAdd(cur + col[p], 1ull);
      tcol[q] = (int32_t)i;
      tval[q] = val[p];
    }
  }
}

// Bitonic sort by key of the first m entries of (key, val) in shared memory,
// padded to a power of two with INT_MAX keys; one warp.
__device__ void warp_sort(int32_t *key, double *val, int m) {
  const int lane = threadIdx.x & 31;
  int np2 = 1;
  while (np2 < m) np2 <<= 1;
  for (int t = m + lane; t < np2; t += 32) {
    key[t] = 0x7fffffff;
    val[t] = 0.0;
  }
  __syncwarp();
  for (int k = 2; k <= np2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < np2; t += 32) {
        const int u = t ^ j;
        if (u > t) {
          const bool up = (t & k) == 0;
          if ((key[t] > key[u]) == up) {
            const int32_t tk = key[t];
            key[t] = key[u];
            key[u] = tk;
            const double tv = val[t];
            val[t] = val[u];
            val[u] = tv;
          }
        }
      }
      __syncwarp();
    }
  }
}

// Sort every row of a CSR matrix by column (distinct columns), one warp per
// row with kCap entries of shared memory (dynamic: values, then keys).  Rows
// longer than kCap are marked (big[i] = 1) for the one-warp pass with the
// large buffer when big is given, else they raise DEVERR_AMG_ROW; only_big
// takes the marked rows alone.
template <int kCap, int kW>
__global__ void __launch_bounds__(32 * kW) k_sort_rows(int64_t n, const int64_t *__restrict__ rp, int32_t *col,
                                                      double *val, int *err, uint8_t *big, bool only_big) {
  extern __shared__ __align__(16) unsigned char sort_smem[];
  double *svb = reinterpret_cast<double *>(sort_smem);
  int32_t *skb = reinterpret_cast<int32_t *>(svb + (size_t)kW * kCap);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * kW + w, nw = (int64_t)gridDim.x * kW;
  double *sv = svb + (size_t)w * kCap;
  int32_t *sk = skb + (size_t)w * kCap;
  for (int64_t i = gw; i < n; i += nw) {
    if (only_big && !big[i]) continue;
    const int64_t lo = rp[i];
    const int m = (int)(rp[i + 1] - lo);
    if (m > kCap) {
      if (lane == 0) {
        if (big && !only_big) big[i] = 1;
        else atomicOr(err, DEVERR_AMG_ROW);
      }
      continue;
    }
    for (int t = lane; t < m; t += 32) {
      sk[t] = col[lo + t];
      sv[t] = val[lo + t];
    }
    __syncwarp();
    warp_sort(sk, sv, m);
    for (int t = lane; t < m; t += 32) {
      col[lo + t] = sk[t];
      val[lo + t] = sv[t];
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------- products ------
// Row r of C = X Y (X in SELL or CSR, Y in CSR), one warp per row: for each
// entry (k, x) of X's row in stored order the lanes take Y's row k (distinct
// columns, so no two lanes meet in one round) and add x * y into a hash table
// in shared memory; every column's sum therefore runs in a fixed order.  The
// count pass stores the number of distinct columns; the fill pass sorts the
// table by column and writes the row.
//
// Two sizes: kW warps with 2^kBits slots each (dynamic shared memory), and
// one warp with 2^kBigBits slots for the rows that overflow the small table
// (the dense-ish coarse operators of wide stencils).  A row overflows when it
// has more than 3/4 of its table's slots of distinct columns.  The small
// count pass marks such rows (big[r] = 1, cnt[r] = 0) when big is given,
// else it raises DEVERR_AMG_ROW; the small fill pass skips marked rows; the
// large passes (only_big) take the marked rows alone.
template <bool kFill, int kBits, int kW>
__global__ void __launch_bounds__(32 * kW) k_prod_rows(DMat X, const int64_t *__restrict__ yrp,
                                                      const int32_t *__restrict__ ycol,
                                                      const double *__restrict__ yval, int64_t *cnt,
                                                      const int64_t *__restrict__ rp, int32_t *ocol,
                                                      double *oval, int *err, uint8_t *big, bool only_big) {
  constexpr int kSlots = 1 << kBits, kMax = 3 * kSlots / 4;
  extern __shared__ __align__(16) unsigned char prod_smem[];
  double *tv = reinterpret_cast<double *>(prod_smem);
  int32_t *tk = reinterpret_cast<int32_t *>(tv + (size_t)kW * kSlots);
  int *tn = reinterpret_cast<int *>(tk + (size_t)kW * kSlots);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * kW + w, nw = (int64_t)gridDim.x * kW;
  int32_t *K = tk + (size_t)w * kSlots;
  double *V = tv + (size_t)w * kSlots;
  for (int64_t r = gw; r < X.rows; r += nw) {
    if (big && (big[r] != 0) != only_big) continue;
    int64_t base;
    int st, L;
    X.row(r, base, st, L);
    // table size: a power of two of at least twice the candidate count
    // (capped), so short rows initialise and compact a small table
    int64_t cand = 0;
    for (int e = lane; e < L; e += 32) {
      const int32_t k = X.col[base + (int64_t)st * e];
      cand += yrp[k + 1] - yrp[k];
    }
    for (int o = 16; o > 0; o >>= 1) cand += __shfl_xor_sync(0xffffffffu, cand, o);
    int bits = 5;
    while (bits < kBits && (1ll << bits) < 2 * cand) ++bits;
    const int slots = 1 << bits;
    for (int t = lane; t < slots; t += 32) {
      K[t] = -1;
      V[t] = 0.0;
    }
    if (lane == 0) tn[w] = 0;
    __syncwarp();
    bool over = false;
    for (int e = 0; e < L; ++e) {
      const int64_t p = base + (int64_t)st * e;
      const int32_t k = X.col[p];
      const double xv = X.val[p];
      const int64_t q0 = yrp[k], q1 = yrp[k + 1];
      for (int64_t q = q0 + lane; q < q1; q += 32) {
        const int32_t c = ycol[q];
        const double v = xv * yval[q];
        unsigned h = ((unsigned)c * 0x9E3779B1u) >> (32 - bits);
        for (int probe = 0; probe < slots; ++probe) {
          const int32_t old = atomicCAS(&K[h], -1, c);
          if (old == -1) atomicAdd(&tn[w], 1);
          if (old == -1 || old == c) {
            V[h] += v;
            break;
          }
          h = (h + 1) & (slots - 1);
        }
      }
      __syncwarp();
      if (tn[w] > kMax) over = true;
      if (over) break;
    }
    __syncwarp();
    const int m = tn[w];
    if (over) {
      if (lane == 0) {
        if (big && !only_big) big[r] = 1;
        else atomicOr(err, DEVERR_AMG_ROW);
        if (cnt) cnt[r] = 0;
      }
      __syncwarp();
      continue;
    }
    if (!kFill) {
      if (lane == 0) cnt[r] = m;
      __syncwarp();
      continue;
    }
    // compact the occupied slots to the front in place (slot order; a slot
    // moves only backwards, and each chunk is read before it is written),
    // then sort by column
    int done = 0;
    for (int t0 = 0; t0 < slots; t0 += 32) {
      const int t = t0 + lane;
      const int32_t kk = K[t];
      const double vv = V[t];
      const bool occ = kk >= 0;
      const unsigned b = __ballot_sync(0xffffffffu, occ);
      __syncwarp();
      if (occ) {
        const int pos = done + __popc(b & ((1u << lane) - 1));
        K[pos] = kk;
        V[pos] = vv;
      }
      done += __popc(b);
      __syncwarp();
    }
    warp_sort(K, V, m);
    const int64_t o = rp[r];
    for (int t = lane; t < m; t += 32) {
      ocol[o + t] = K[t];
      oval[o + t] = V[t];
    }
    if (cnt && lane == 0) cnt[r] = m;
    __syncwarp();
  }
}

// Upper bound of the distinct columns of row r of X Y: the number of
// candidate products sum_{k in row r of X} |row k of Y|.
__global__ void k_prod_cand(DMat X, const int64_t *__restrict__ yrp, int64_t *cand) {
  ROWS_LOOP(r, X.rows) {
    int64_t base;
    int st, L;
    X.row(r, base, st, L);
    int64_t c = 0;
    for (int e = 0; e < L; ++e) {
      const int32_t k = X.col[base + (int64_t)st * e];
      c += yrp[k + 1] - yrp[k];
    }
    cand[r] = c;
  }
}

// Row r's entries from the scratch (at off[r]) to their final place (rp[r]),
// one warp per row.
__global__ void k_compact_rows(int64_t rows, const int64_t *__restrict__ off, const int64_t *__restrict__ rp,
                               const int32_t *__restrict__ tcol, const double *__restrict__ tval, int32_t *col,
                               double *val) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows; r += nwarps) {
    const int64_t src = off[r], dst = rp[r], m = rp[r + 1] - dst;
    for (int64_t t = lane; t < m; t += 32) {
      col[dst + t] = tcol[src + t];
      val[dst + t] = tval[src + t];
    }
  }
}

// Row r of C = X Y with one thread per row (short rows: the finest level's
// A P), the row's distinct columns in a sorted list, contributions summed in
// stored order.
template <bool kFill>
__global__ void k_prod_rows_thread(DMat X, const int64_t *__restrict__ yrp, const int32_t *__restrict__ ycol,
                                   const double *__restrict__ yval, int64_t *cnt, const int64_t *__restrict__ rp,
                                   int32_t *ocol, double *oval, unsigned long long *ovf) {
  ROWS_LOOP(r, X.rows) {
    RowMap<kCapThreadRow> m;
    bool ok = true;
    int64_t base;
    int st, L;
    X.row(r, base, st, L);
    for (int e = 0; e < L && ok; ++e) {
      const int64_t p = base + (int64_t)st * e;
      const int32_t k = X.col[p];
      const double xv = X.val[p];
      for (int64_t q = yrp[k]; q < yrp[k + 1] && ok; ++q) ok = m.add(ycol[q], xv * yval[q]);
    }
    if (!ok) atomicOr(ovf, 1ull);   // the host redoes the product a warp per row
    if (!kFill) {
      cnt[r] = ok ? m.n : 0;
    } else if (ok) {
      if (cnt) cnt[r] = m.n;
      const int64_t o = rp[r];
      for (int t = 0; t < m.n; ++t) {
        ocol[o + t] = m.key[t];
        oval[o + t] = m.val[t];
      }
    }
  }
}

// ------------------------------------------------------ coarsest level ----
__global__ void k_dense_from(DMat A, double *M) {
  const int64_t n = A.rows;
  ROWS_LOOP(i, n) {
    int64_t base;
    int st, L;
    A.row(i, base, st, L);
    for (int64_t c = 0; c < n; ++c) M[i * n + c] = 0.0;
    for (int k = 0; k < L; ++k) M[i * n + A.col[base + (int64_t)st * k]] += A.val[base + (int64_t)st * k];
  }
}

__global__ void k_pin_last(int n, double *M) {
  const int64_t l = n - 1;
  for (int i = threadIdx.x; i < n - 1; i += blockDim.x) {
    M[l * n + i] = 0.0;
    M[(int64_t)i * n + l] = 0.0;
  }
}

// In-place Gauss-Jordan inverse of an SPD n x n matrix (no pivoting needed),
// one block.
__global__ void k_gauss_jordan(int n, double *M, int *err) {
  __shared__ double piv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      piv = M[(int64_t)k * n + k];
      if (!(piv != 0.0) || !isfinite(piv)) {
        atomicOr(err, DEVERR_AMG_DIAG);
        piv = 1.0;
      }
    }
    __syncthreads();
    const double ip = 1.0 / piv;
    // row k scaled; column k of the other rows holds their multipliers
    for (int c = threadIdx.x; c < n; c += blockDim.x)
      if (c != k) M[(int64_t)k * n + c] *= ip;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) {
      const int r = (int)(t / n), c = (int)(t % n);
      if (r == k || c == k) continue;
      M[t] -= M[(int64_t)r * n + k] * M[(int64_t)k * n + c];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      if (r != k) M[(int64_t)r * n + k] *= -ip;
    __syncthreads();
    if (threadIdx.x == 0) M[(int64_t)k * n + k] = ip;
    __syncthreads();
  }
}

// ------------------------------------------------------------ V-cycle -----
__device__ __forceinline__ bool cycle_done(const double *sc) {
  pdl_wait();   // the previous kernel's results first (launch_pdl)
  __shared__ int f;
  if (threadIdx.x == 0) f = (sc && sc[0] != 0.0) ? 1 : 0;
  __syncthreads();
  const bool r = f != 0;
  __syncthreads();
  return r;
}

// Cycle operations on one matrix (row r, t = sum_j a_rj x_j); wd = w D^-1:
//   kResid  y = b - A x
//   kPost   y = x + wd (b - A x)
//   kAdd    y += A x
//   kApply  y = A x
//   kCheb   y = x + c (x - xp) + wd (b - A x)   (xp == nullptr: xp = 0)
// kCheb is the second Chebyshev step: x - xp is the first step's update.
enum { kResid = 0, kPost = 1, kAdd = 2, kApply = 3, kCheb = 4 };

template <int kMode, class T, class Ty>
__device__ __forceinline__ void cycle_out(int64_t r, T t, const T *__restrict__ x, const T *__restrict__ b,
                                          const T *__restrict__ wd, Ty *y, const T *__restrict__ xp, T c) {
  if (kMode == kResid) y[r] = (Ty)(b[r] - t);
  else if (kMode == kPost) y[r] = (Ty)(x[r] + wd[r] * (b[r] - t));
  else if (kMode == kAdd) y[r] += (Ty)t;
  else if (kMode == kCheb) y[r] = (Ty)(x[r] + c * (x[r] - (xp ? xp[r] : (T)0)) + wd[r] * (b[r] - t));
  else y[r] = (Ty)t;
}

template <class T>
__global__ void __launch_bounds__(256) k_vc_pre(int64_t n, const T *__restrict__ b, const T *__restrict__ wd, T *x,
                                                const double *sc) {
  if (cycle_done(sc)) return;
  ROWS_LOOP(i, n) x[i] = wd[i] * b[i];
}

template <class Ta, class Tb>
__global__ void k_vc_convert(int64_t n, const Ta *__restrict__ a, Tb *b, const double *sc) {
  if (cycle_done(sc)) return;
  ROWS_LOOP(i, n) b[i] = (Tb)a[i];
}

// SELL-32: one warp per slice, one thread per row, batches of 8 entries
// predicated on the slice width.
template <class T, class Ty, int kMode>
__global__ void __launch_bounds__(256) k_vc_sell(int64_t rows, int64_t nslices, const int64_t *__restrict__ off,
                                                 const int32_t *__restrict__ col, const T *__restrict__ val,
                                                 const T *__restrict__ x, const T *__restrict__ b,
                                                 const T *__restrict__ wd, Ty *y, const double *sc,
                                                 const T *__restrict__ xp, T c) {
  if (cycle_done(sc)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = warp; s < nslices; s += nwarps) {
    const T acc = sell_row_dot<T, 8, true>(off, col, val, x, s, lane);
    const int64_t r = 32 * s + lane;
    if (r < rows) cycle_out<kMode>(r, acc, x, b, wd, y, xp, c);
  }
}

// CSR with G lanes per row (consecutive rows per warp, so the warp reads one
// contiguous stretch), partial sums combined by shuffles in a fixed pattern:
// the operators of the small levels.
template <int G, class T, class Ty, int kMode>
__global__ void __launch_bounds__(256) k_vc_csr(int64_t rows, const int64_t *__restrict__ rp,
                                                const int32_t *__restrict__ col, const T *__restrict__ val,
                                                const T *__restrict__ x, const T *__restrict__ b,
                                                const T *__restrict__ wd, Ty *y, const double *sc,
                                                const T *__restrict__ xp, T c) {
  if (cycle_done(sc)) return;
  constexpr int R = 32 / G;   // rows per warp
  const int lane = threadIdx.x & 31, sub = lane & (G - 1), grp = lane / G;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = warp * R; r0 < rows; r0 += nwarps * R) {
    const int64_t r = r0 + grp;
    T acc = 0;
    if (r < rows) {
      const int64_t q1 = rp[r + 1];
      for (int64_t q = rp[r] + sub; q < q1; q += G) acc += __ldcs(val + q) * __ldg(x + __ldcs(col + q));
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (r < rows && sub == 0) cycle_out<kMode>(r, acc, x, b, wd, y, xp, c);
  }
}

// x = Minv b with the dense coarsest inverse: one warp per row.
template <class T>
__global__ void __launch_bounds__(256) k_vc_dense(int n, const T *__restrict__ Minv, const T *__restrict__ b, T *x,
                                                  const double *sc) {
  if (cycle_done(sc)) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < n; r += nwarps) {
    T acc = 0;
    for (int c = lane; c < n; c += 32) acc += Minv[(int64_t)r * n + c] * b[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) x[r] = acc;
  }
}

static int rows_grid(int64_t n) { return grid_for(n, 256, 8); }

static int warps_grid(int64_t warps) {   // blocks of 8 warps, one wave at most
  int64_t b = (warps + 7) / 8;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

static int prod_grid(int64_t rows) {     // blocks of kProdWarps warps
  int64_t b = (rows + kProdWarps - 1) / kProdWarps;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// Lanes per row for a CSR matrix: about three entries per lane.
static int lanes_for(int64_t rows, int64_t nnz) {
  const double avg = rows > 0 ? (double)nnz / rows : 1.0;
  int g = 2;
  while (g < 32 && 3.0 * g < avg) g <<= 1;
  return g;
}

template <class T> static const T *vals(const CsrBuf &M);
template <> const double *vals<double>(const CsrBuf &M) { return M.val; }
template <> const float *vals<float>(const CsrBuf &M) { return M.val32; }
template <class T> static const T *vals(const SellBuf &M);
template <> const double *vals<double>(const SellBuf &M) { return M.m.val; }
template <> const float *vals<float>(const SellBuf &M) { return M.val32; }

template <int kMode, class T, class Ty>
static void csr_launch(cudaStream_t s, const CsrBuf &M, const T *x, const T *b, const T *wd, Ty *y,
                       const double *sc, const T *xp = nullptr, T c = 0) {
  const int64_t warps = (M.rows * M.lanes + 31) / 32;
  const int g = warps_grid(warps);
  const T *v = vals<T>(M);
  count_launch();
  switch (M.lanes) {
    case 2: launch_pdl(k_vc_csr<2, T, Ty, kMode>, g, 256, 0, s, M.rows, M.rp, M.col, v, x, b, wd, y, sc, xp, c); break;
    case 4: launch_pdl(k_vc_csr<4, T, Ty, kMode>, g, 256, 0, s, M.rows, M.rp, M.col, v, x, b, wd, y, sc, xp, c); break;
    case 8: launch_pdl(k_vc_csr<8, T, Ty, kMode>, g, 256, 0, s, M.rows, M.rp, M.col, v, x, b, wd, y, sc, xp, c); break;
    case 16: launch_pdl(k_vc_csr<16, T, Ty, kMode>, g, 256, 0, s, M.rows, M.rp, M.col, v, x, b, wd, y, sc, xp, c); break;
    default: launch_pdl(k_vc_csr<32, T, Ty, kMode>, g, 256, 0, s, M.rows, M.rp, M.col, v, x, b, wd, y, sc, xp, c); break;
  }
}

template <int kMode, class T, class Ty>
static void sell_launch(cudaStream_t s, const SellMat &A, const T *val, const T *x, const T *b, const T *wd, Ty *y,
                        const double *sc, const T *xp = nullptr, T c = 0) {
  count_launch();
  launch_pdl(k_vc_sell<T, Ty, kMode>, warps_grid(A.nslices), 256, 0, s, A.rows, A.nslices, A.off, A.col, val, x, b,
             wd, y, sc, xp, c);
}

__global__ void k_rp_counts(int64_t n, const int64_t *__restrict__ rp, int64_t *cnt) {
  ROWS_LOOP(i, n) cnt[i] = rp[i + 1] - rp[i];
}

__global__ void k_sell_slices(int64_t rows, int64_t ns, const int64_t *__restrict__ cnt, int64_t *ssz,
                              int32_t *len) {
  ROWS_LOOP(s, ns) {
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

__global__ void k_csr_to_sell(int64_t ns, const int64_t *__restrict__ rp, int64_t rows,
                              const int32_t *__restrict__ ccol, const double *__restrict__ cval,
                              const int64_t *__restrict__ off, int32_t *scol, double *sval) {
  ROWS_LOOP(t, ns * 32) {
    const int64_t s = t >> 5, lane = t & 31, r = t;
    const int64_t w = (off[s + 1] - off[s]) >> 5;
    const int64_t lo = r < rows ? rp[r] : 0, L = r < rows ? rp[r + 1] - lo : 0;
    for (int64_t k = 0; k < w; ++k) {
      const int64_t p = off[s] + 32 * k + lane;
      scol[p] = k < L ? ccol[lo + k] : 0;
      sval[p] = k < L ? cval[lo + k] : 0.0;
    }
  }
}

__global__ void k_scale_into(int64_t n, const double *__restrict__ a, double w, double *y) {
  ROWS_LOOP(i, n) y[i] = w * a[i];
}

// ------------------------------------------------------ point blocks ------
// Smoothed aggregation on point blocks (several unknowns per node, e.g. the
// four P1 pressure moments of a cell of the paper's k = 2 element): Vanek,
// Mandel & Brezina (1996), the tentative prolongator built from a near-null
// space B orthonormalised per aggregate.  Rules:
//   block graph: N_IJ = Frobenius norm of the bs x bs block (I, J) of A,
//     formed as sqrt(Q^T (A o A) Q) with Q the n x nb block-membership
//     matrix; strong(I, J): N_IJ >= theta sqrt(N_II N_JJ); aggregates from
//     that graph by the scalar rules above;
//   T: for aggregate a with member blocks I_1 < I_2 < ..., the rows of its
//     DOFs (block by block) of B = Q_a R_a with R_a upper triangular,
//     R_jj > 0 (Cholesky of B_a^T B_a, then Q_a = B_a R_a^-1); T holds Q_a in
//     columns a m .. a m + m - 1, the coarse near-null space R_a;
//   D = block diagonal of A = L L^T blockwise; rho = min(Gershgorin bound
//     of C = L^-1 A L^-T, 1.1 x the largest Ritz value of C after 10 Lanczos
//     steps with full reorthogonalisation from v_i = 2 (splitmix64(i) >> 11)
//     2^-53 - 1); omega = 4 / (3 rho);
//   P = T - omega D^-1 (A T); coarse operator P^T A P with block size m;
//   cycle: damped block Jacobi (x = omega D^-1 b; ...) or two Chebyshev
//     steps of block Jacobi on [rho/10, rho].
constexpr int kMaxBs = 8;    // largest block size
constexpr int kMaxM = 6;     // largest near-null space width
constexpr int kMaxInt = 16;  // largest interior block of the condensed cycle (14 at the paper's k = 2)

// D_I^-1 and L_I^-1 (D_I = L_I L_I^T) of every diagonal block (bs <= kN), a
// thread per block.
template <int kN>
__global__ void k_blk_diag(int64_t nb, int bs, DMat A, double *dinvb, double *linvb, int *err) {
  ROWS_LOOP(I, nb) {
    double D[kN][kN], Lc[kN][kN], Li[kN][kN];
    for (int r = 0; r < bs; ++r)
      for (int c = 0; c < bs; ++c) D[r][c] = 0.0, Lc[r][c] = 0.0, Li[r][c] = 0.0;
    const int64_t i0 = I * bs;
    for (int r = 0; r < bs; ++r) {
      int64_t base;
      int st, L;
      A.row(i0 + r, base, st, L);
      for (int k = 0; k < L; ++k) {
        const int64_t p = base + (int64_t)st * k;
        const int64_t j = A.col[p];
        if (j >= i0 && j < i0 + bs) D[r][j - i0] = A.val[p];
      }
    }
    bool ok = true;
    for (int j = 0; j < bs; ++j) {          // Cholesky, column by column
      double d = D[j][j];
      for (int k = 0; k < j; ++k) d -= Lc[j][k] * Lc[j][k];
      if (!(d > 0.0) || !isfinite(d)) {
        ok = false;
        d = 1.0;
      }
      Lc[j][j] = sqrt(d);
      for (int i = j + 1; i < bs; ++i) {
        double v = D[i][j];
        for (int k = 0; k < j; ++k) v -= Lc[i][k] * Lc[j][k];
        Lc[i][j] = v / Lc[j][j];
      }
    }
    if (!ok) atomicOr(err, DEVERR_AMG_DIAG);
    for (int c = 0; c < bs; ++c) {          // L^-1 by forward substitution, column by column
      for (int i = 0; i < bs; ++i) {
        double v = (i == c) ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) v -= Lc[i][k] * Li[k][c];
        Li[i][c] = (i >= c) ? v / Lc[i][i] : 0.0;
      }
    }
    double *dv = dinvb + I * bs * bs, *lv = linvb + I * bs * bs;
    for (int r = 0; r < bs; ++r)
      for (int c = 0; c < bs; ++c) {
        double v = 0.0;                     // (L^-T L^-1)_rc = sum_k Li_kr Li_kc
        for (int k = 0; k < bs; ++k) v += Li[k][r] * Li[k][c];
        dv[r * bs + c] = v;
        lv[r * bs + c] = Li[r][c];
      }
  }
}

__global__ void k_square(int64_t n, const double *__restrict__ a, double *b) {
  ROWS_LOOP(i, n) b[i] = a[i] * a[i];
}

__global__ void k_sqrt_inplace(int64_t n, double *a) {
  ROWS_LOOP(i, n) a[i] = sqrt(a[i]);
}

// Q (n x nb, Q_{i, i / bs} = 1) and Q^T.
__global__ void k_member_rows(int64_t n, int bs, int64_t *rp, int32_t *col, double *val) {
  ROWS_LOOP(i, n) {
    rp[i] = i;
    col[i] = (int32_t)(i / bs);
    val[i] = 1.0;
    if (i == n - 1) rp[n] = n;
  }
}

__global__ void k_member_cols(int64_t nb, int bs, int64_t *rp, int32_t *col, double *val) {
  ROWS_LOOP(I, nb) {
    rp[I] = I * bs;
    for (int k = 0; k < bs; ++k) {
      col[I * bs + k] = (int32_t)(I * bs + k);
      val[I * bs + k] = 1.0;
    }
    if (I == nb - 1) rp[nb] = nb * bs;
  }
}

// The block-diagonal matrix of the blocks blk (row-major bs x bs per block)
// as CSR with full blocks; trans: the transposed blocks.
__global__ void k_blkdiag_rows(int64_t n, int bs, const double *__restrict__ blk, int trans, int64_t *rp,
                               int32_t *col, double *val) {
  ROWS_LOOP(i, n) {
    const int64_t I = i / bs;
    const int r = (int)(i - I * bs);
    rp[i] = i * bs;
    for (int k = 0; k < bs; ++k) {
      col[i * bs + k] = (int32_t)(I * bs + k);
      val[i * bs + k] = trans ? blk[I * bs * bs + k * bs + r] : blk[I * bs * bs + r * bs + k];
    }
    if (i == n - 1) rp[n] = n * bs;
  }
}

// ---- block-diagonal factors applied without a sparse product ----
// When the bs rows of every block row of X hold the same columns in the
// same order (the k = 2 Schur blocks, coarse operators of dense bs x m
// prolongator blocks), L^-1 X L^-T and D^-1 X keep X's pattern and are one
// dense pass over its blocks instead of two hashed products.  bad != 0 if
// some block row differs; with whole_blocks, also if a row's columns do not
// come in whole, ordered blocks of bs.
__global__ void k_blockrow_same(DMat X, int bs, int whole_blocks, int *bad) {
  ROWS_LOOP(i, X.rows) {
    const int64_t i0 = (i / bs) * bs;
    int64_t b, b0;
    int st, st0, L, L0;
    X.row(i, b, st, L);
    X.row(i0, b0, st0, L0);
    bool ok = L == L0 && (!whole_blocks || L % bs == 0);
    for (int k = 0; ok && k < L; ++k) {
      const int32_t c = X.col[b + (int64_t)st * k];
      if (c != X.col[b0 + (int64_t)st0 * k]) ok = false;
      if (whole_blocks) {
        const int kb = k - k % bs;
        if (c % bs != k % bs || c / bs != X.col[b + (int64_t)st * kb] / bs) ok = false;
      }
    }
    if (!ok) atomicOr(bad, 1);
  }
}

__global__ void k_row_lengths(DMat X, int64_t *cnt) {
  ROWS_LOOP(i, X.rows) {
    int64_t b;
    int st, L;
    X.row(i, b, st, L);
    cnt[i] = L;
  }
}

// C = L^-1 A L^-T in A's pattern (CSR rp from A's row lengths):
// C_(I,a),(J,b) = sum_p Li_I[a][p] sum_q A_(I,p),(J,q) Li_J[b][q].
__global__ void k_blk_congruence(DMat A, int bs, const double *__restrict__ li, const int64_t *__restrict__ rp,
                                 int32_t *ccol, double *cval) {
  ROWS_LOOP(i, A.rows) {
    const int64_t I = i / bs;
    const int a = (int)(i - I * bs);
    int64_t bp[kMaxBs];
    int stp[kMaxBs], L = 0;
    for (int p = 0; p < bs; ++p) A.row(I * bs + p, bp[p], stp[p], L);
    const double *LI = li + I * bs * bs;
    const int64_t o = rp[i];
    for (int k = 0; k < L; ++k) {
      const int32_t c = A.col[bp[a] + (int64_t)stp[a] * k];
      const int64_t J = c / bs;
      const int bb = (int)(c - J * bs), kb = k - bb;
      const double *LJ = li + J * bs * bs + bb * bs;
      double sum = 0.0;
      for (int p = 0; p < bs; ++p) {
        double t = 0.0;
        for (int q = 0; q <= bb; ++q) t += A.val[bp[p] + (int64_t)stp[p] * (kb + q)] * LJ[q];
        sum += LI[a * bs + p] * t;
      }
      ccol[o + k] = c;
      cval[o + k] = sum;
    }
  }
}

// C = D^-1 Y in Y's pattern (Y CSR, block rows of identical columns):
// C_(I,a),k = sum_p Dinv_I[a][p] Y_(I,p),k.
__global__ void k_blk_left(int64_t n, int bs, const double *__restrict__ dinv, const int64_t *__restrict__ yrp,
                           const int32_t *__restrict__ ycol, const double *__restrict__ yval, int32_t *ccol,
                           double *cval) {
  ROWS_LOOP(i, n) {
    const int64_t I = i / bs;
    const int a = (int)(i - I * bs);
    const double *DI = dinv + I * bs * bs + a * bs;
    const int64_t o = yrp[i], L = yrp[i + 1] - o;
    for (int64_t k = 0; k < L; ++k) {
      double sum = 0.0;
      for (int p = 0; p < bs; ++p) sum += DI[p] * yval[yrp[I * bs + p] + k];
      ccol[o + k] = ycol[o + k];
      cval[o + k] = sum;
    }
  }
}

// Aggregate membership as a CSR matrix (nb x nc): one entry per aggregated block.
__global__ void k_agg_count(int64_t nb, const int32_t *__restrict__ agg, int64_t *cnt) {
  ROWS_LOOP(I, nb) cnt[I] = agg[I] >= 0 ? 1 : 0;
}

__global__ void k_agg_fill(int64_t nb, const int32_t *__restrict__ agg, const int64_t *__restrict__ rp, int32_t *col,
                           double *val) {
  ROWS_LOOP(I, nb) {
    if (agg[I] >= 0) {
      col[rp[I]] = agg[I];
      val[rp[I]] = 1.0;
    }
  }
}

// Rank test of the near-null space on every aggregate (a thread per
// aggregate): keep[a] = 1 when every pivot of the Cholesky factorisation of
// G = B_a^T B_a, d_j = G_jj - sum_{k<j} R_kj^2, exceeds kRankTol G_jj, else 0
// (the aggregate is then dissolved: with fewer independent modes than m its
// factorisation would give a column of rounding noise).
constexpr double kRankTol = 1e-10;

__global__ void k_tent_rank(int64_t nc, int bs, int m, const int64_t *__restrict__ arp,
                            const int32_t *__restrict__ acol, const double *__restrict__ B, int64_t *keep,
                            int *err) {
  ROWS_LOOP(a, nc) {
    double G[kMaxM][kMaxM], R[kMaxM][kMaxM];
    for (int j = 0; j < m; ++j)
      for (int k = 0; k < m; ++k) G[j][k] = 0.0, R[j][k] = 0.0;
    for (int64_t p = arp[a]; p < arp[a + 1]; ++p)
      for (int c = 0; c < bs; ++c) {
        const double *x = B + ((int64_t)acol[p] * bs + c) * m;
        for (int j = 0; j < m; ++j)
          for (int k = 0; k < m; ++k) G[j][k] += x[j] * x[k];
      }
    int64_t ok = 1;
    for (int j = 0; j < m && ok; ++j) {
      double d = G[j][j];
      for (int k = 0; k < j; ++k) d -= R[k][j] * R[k][j];
      if (!isfinite(d)) atomicOr(err, DEVERR_NONFINITE);
      if (!(d > kRankTol * G[j][j])) {
        ok = 0;
        break;
      }
      R[j][j] = sqrt(d);
      for (int i = j + 1; i < m; ++i) {
        double v = G[j][i];
        for (int k = 0; k < j; ++k) v -= R[k][j] * R[k][i];
        R[j][i] = v / R[j][j];
      }
    }
    keep[a] = ok;
  }
}

// agg[I] -> its aggregate's new number (pos: exclusive scan of keep), or -1
// for a dissolved aggregate.
__global__ void k_agg_renumber(int64_t nb, const int64_t *__restrict__ keep, const int64_t *__restrict__ pos,
                               int32_t *agg) {
  ROWS_LOOP(I, nb) {
    const int32_t a = agg[I];
    if (a >= 0) agg[I] = keep[a] ? (int32_t)pos[a] : -1;
  }
}

__global__ void k_tent_count(int64_t n, int bs, int m, const int32_t *__restrict__ agg, int64_t *cnt) {
  ROWS_LOOP(i, n) cnt[i] = agg[i / bs] >= 0 ? m : 0;
}

// Tentative prolongator, a thread per aggregate: members from the sorted row
// of A^T (agg membership transposed), B_a = Q_a R_a by Cholesky of the Gram
// matrix (R_a = chol(B_a^T B_a)^T, R_jj > 0) and Q_a = B_a R_a^-1.
__global__ void k_tent(int64_t nc, int bs, int m, const int64_t *__restrict__ arp, const int32_t *__restrict__ acol,
                       const double *__restrict__ B, const int64_t *__restrict__ trp, int32_t *tcol, double *tval,
                       double *Bc, int *err) {
  ROWS_LOOP(a, nc) {
    double G[kMaxM][kMaxM], R[kMaxM][kMaxM];
    for (int j = 0; j < m; ++j)
      for (int k = 0; k < m; ++k) G[j][k] = 0.0, R[j][k] = 0.0;
    for (int64_t p = arp[a]; p < arp[a + 1]; ++p)
      for (int c = 0; c < bs; ++c) {
        const double *x = B + ((int64_t)acol[p] * bs + c) * m;
        for (int j = 0; j < m; ++j)
          for (int k = 0; k < m; ++k) G[j][k] += x[j] * x[k];
      }
    bool ok = true;
    for (int j = 0; j < m; ++j) {          // G = R^T R, R upper triangular
      double d = G[j][j];
      for (int k = 0; k < j; ++k) d -= R[k][j] * R[k][j];
      if (!(d > 0.0) || !isfinite(d)) {
        ok = false;
        d = 1.0;
      }
      R[j][j] = sqrt(d);
      for (int i = j + 1; i < m; ++i) {
        double v = G[j][i];
        for (int k = 0; k < j; ++k) v -= R[k][j] * R[k][i];
        R[j][i] = v / R[j][j];
      }
    }
    if (!ok) atomicOr(err, DEVERR_AMG_DIAG);
    for (int64_t p = arp[a]; p < arp[a + 1]; ++p)
      for (int c = 0; c < bs; ++c) {
        const int64_t i = (int64_t)acol[p] * bs + c;
        const double *x = B + i * m;
        double q[kMaxM];
        for (int j = 0; j < m; ++j) {      // q R = x
          double v = x[j];
          for (int k = 0; k < j; ++k) v -= q[k] * R[k][j];
          q[j] = v / R[j][j];
        }
        const int64_t o = trp[i];
        for (int j = 0; j < m; ++j) {
          tcol[o + j] = (int32_t)(a * m + j);
          tval[o + j] = q[j];
        }
      }
    for (int j = 0; j < m; ++j)
      for (int k = 0; k < m; ++k) Bc[(a * m + j) * m + k] = k >= j ? R[j][k] : 0.0;
  }
}

// C = X - w Y for CSR matrices with sorted rows (union pattern).
template <bool kFill>
__global__ void k_sub_rows(int64_t rows, const int64_t *__restrict__ xrp, const int32_t *__restrict__ xc,
                           const double *__restrict__ xv, const int64_t *__restrict__ yrp,
                           const int32_t *__restrict__ yc, const double *__restrict__ yv, double w, int64_t *cnt,
                           const int64_t *__restrict__ crp, int32_t *cc, double *cv) {
  ROWS_LOOP(i, rows) {
    int64_t p = xrp[i], q = yrp[i];
    const int64_t p1 = xrp[i + 1], q1 = yrp[i + 1];
    int64_t o = kFill ? crp[i] : 0;
    int64_t t = 0;
    while (p < p1 || q < q1) {
      const int32_t a = p < p1 ? xc[p] : INT32_MAX, b = q < q1 ? yc[q] : INT32_MAX;
      const int32_t c = a < b ? a : b;
      double v = 0.0;
      if (a == c) v += xv[p++];
      if (b == c) v -= w * yv[q++];
      if (kFill) {
        cc[o + t] = c;
        cv[o + t] = v;
      }
      ++t;
    }
    if (!kFill) cnt[i] = t;
  }
}

// max_i sum_j |a_ij| (as the bit pattern of a non-negative double)
__global__ void k_abs_rowsum_max(int64_t rows, const int64_t *__restrict__ rp, const double *__restrict__ val,
                                 unsigned long long *mx) {
  double m = 0.0;
  ROWS_LOOP(i, rows) {
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += fabs(val[p]);
    m = fmax(m, s);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

// ---- Lanczos ----
__global__ void k_start_vec(int64_t n, double *v) {
  ROWS_LOOP(i, n) v[i] = 2.0 * ((double)(splitmix64((uint64_t)i) >> 11) * 0x1p-53) - 1.0;
}

__global__ void k_csr_spmv(int64_t rows, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ val, const double *__restrict__ x, double *y) {
  ROWS_LOOP(i, rows) {
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += val[p] * x[col[p]];
    y[i] = s;
  }
}

constexpr int kDotBlocks = 256;
// part[j * kDotBlocks + block] = partial sum of V_j . w (V column-major, n rows)
__global__ void __launch_bounds__(256) k_dots_part(int64_t n, int K, const double *__restrict__ V,
                                                   const double *__restrict__ w, double *part) {
  __shared__ double sh[8];
  for (int j = 0; j < K; ++j) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
      s += V[(int64_t)j * n + i] * w[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
      part[j * kDotBlocks + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

__global__ void k_dots_fin(int K, const double *__restrict__ part, double *out) {
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int b = 0; b < kDotBlocks; ++b) t += part[threadIdx.x * kDotBlocks + b];
    out[threadIdx.x] = t;
  }
}

// w -= sum_j h_j V_j (j in order)
__global__ void k_sub_proj(int64_t n, int K, const double *__restrict__ V, const double *__restrict__ hcoef,
                           double *w) {
  ROWS_LOOP(i, n) {
    double v = w[i];
    for (int j = 0; j < K; ++j) v -= hcoef[j] * V[(int64_t)j * n + i];
    w[i] = v;
  }
}

__global__ void k_scale_copy(int64_t n, const double *__restrict__ a, const double *__restrict__ s, double *b) {
  const double f = 1.0 / sqrt(s[0]);
  ROWS_LOOP(i, n) b[i] = a[i] * f;
}

// Block-Jacobi steps of the cycle (y indexes rows; I = i / bs):
//   mode 0: y = s D r;  mode 1: y = x + s D r;  mode 2: y = x + c (x - xp) + s D r (xp == nullptr: 0)
__global__ void __launch_bounds__(256) k_blk_apply(int64_t n, int bs, const double *__restrict__ D, double s,
                                                   const double *__restrict__ r, const double *__restrict__ x,
                                                   const double *__restrict__ xp, double c, double *y, int mode,
                                                   const double *sc) {
  if (cycle_done(sc)) return;
  ROWS_LOOP(i, n) {
    const int64_t I = i / bs;
    const int q = (int)(i - I * bs);
    const double *Dr = D + I * bs * bs + q * bs;
    const double *rr = r + I * bs;
    double t = 0.0;
    for (int k = 0; k < bs; ++k) t += Dr[k] * rr[k];
    t *= s;
    if (mode == 0) y[i] = t;
    else if (mode == 1) y[i] = x[i] + t;
    else y[i] = x[i] + c * (x[i] - (xp ? xp[i] : 0.0)) + t;
  }
}

__global__ void k_pin_row(int n, int k, double *M) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (i != k) {
      M[(int64_t)k * n + i] = 0.0;
      M[(int64_t)i * n + k] = 0.0;
    }
  }
}

// ------------------------------------------------ condensed Block-Reg -----
// A_reg = [A_ff A_fi; A_if A_ii] with the face DOFs (rows < nfr) first; an
// interior DOF couples only to its own cell, so A_ii is block diagonal with
// nid x nid blocks.  The split writes the four parts as CSR (columns of the
// interior parts shifted by -nfr), a count pass then a fill pass.
// Rows r0 .. r0 + nrows - 1; the count pass writes c0/c1 at the global row,
// the fill pass uses rp0/rp1 at the row within the range.
template <bool kFill>
__global__ void k_split(DMat A, int64_t r0, int64_t nrows, int64_t nfr, int64_t *c0, int64_t *c1,
                        const int64_t *__restrict__ rp0, const int64_t *__restrict__ rp1, int32_t *col0,
                        double *val0, int32_t *col1, double *val1) {
  ROWS_LOOP(t, nrows) {
    const int64_t i = r0 + t;
    int64_t base;
    int st, L;
    A.row(i, base, st, L);
    int64_t n0 = 0, n1 = 0;
    const int64_t o0 = kFill ? rp0[t] : 0, o1 = kFill ? rp1[t] : 0;
    for (int k = 0; k < L; ++k) {
      const int64_t p = base + (int64_t)st * k;
      const int64_t j = A.col[p];
      if (j < nfr) {
        if (kFill) {
          col0[o0 + n0] = (int32_t)j;
          val0[o0 + n0] = A.val[p];
        }
        ++n0;
      } else {
        if (kFill) {
          col1[o1 + n1] = (int32_t)(j - nfr);
          val1[o1 + n1] = A.val[p];
        }
        ++n1;
      }
    }
    if (!kFill) {
      c0[i] = n0;
      c1[i] = n1;
    }
  }
}

// Near-null space of the condensed face system of the paper's k = 1 element:
// the face DOFs (1/|f|) int_f (e_j . n_f) m_beta of the constant fields e_j,
// n_f the global normal: n_f[j] for beta = (0, 0), 0 for the two linear face
// monomials (their mean over the face vanishes about its barycentre).
__global__ void k_flux_modes_k1(int64_t nf, const double *__restrict__ f_norm, double *B) {
  ROWS_LOOP(f, nf) {
    for (int b = 0; b < 3; ++b)
      for (int j = 0; j < 3; ++j) B[(3 * f + b) * 3 + j] = b == 0 ? f_norm[3 * f + j] : 0.0;
  }
}

// ------------------------------------------------------------ host --------
// Row counts cnt[rows] -> CSR with that pattern (row pointers from the scan).
static vem_status csr_layout(vem_handle *h, CsrBuf &C, int64_t rows, int64_t cols, const int64_t *cnt) {
  VEM_TRY(grow(h, C.rp, C.c_rp, (size_t)rows + 1));
  int64_t nnz = 0;
  VEM_TRY(scan_counts(h, rows, cnt, C.rp, &nnz));
  if (!C.col || (size_t)nnz + 1 > C.c_nz) {
    dfree(h, C.col);
    dfree(h, C.val);
    C.col = nullptr;
    C.val = nullptr;
    C.c_nz = 0;
    const size_t c = (size_t)nnz + (size_t)nnz / 4 + 64;
    VEM_TRY(dalloc_n(h, &C.col, c));
    VEM_TRY(dalloc_n(h, &C.val, c));
    C.c_nz = c;
  }
  C.rows = rows;
  C.cols = cols;
  C.nnz = nnz;
  C.lanes = lanes_for(rows, nnz);
  return VEM_OK;
}

// SELL-32 copy of a CSR matrix (slice width = longest row of the slice).
static vem_status csr_to_sell(vem_handle *h, AmgState *S, const CsrBuf &C, SellBuf &B) {
  cudaStream_t s = h->stream;
  const int64_t rows = C.rows, ns = (rows + 31) / 32;
  VEM_TRY(grow(h, B.m.off, B.c_off, (size_t)ns + 1));
  VEM_TRY(grow(h, B.m.len, B.c_len, (size_t)ns * 32));
  VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)rows + 1));
  VEM_TRY(grow(h, S->cur, S->c_cur, (size_t)ns + 1));   // per-slice sizes
  count_launch();
  k_rp_counts<<<rows_grid(rows), 256, 0, s>>>(rows, C.rp, S->cnt);
  count_launch();
  k_sell_slices<<<rows_grid(ns), 256, 0, s>>>(rows, ns, S->cnt, S->cur, B.m.len);
  int64_t stored = 0;
  VEM_TRY(scan_counts(h, ns, S->cur, B.m.off, &stored));
  if (!B.m.col || (size_t)stored + 1 > B.c_st) {
    dfree(h, B.m.col);
    dfree(h, B.m.val);
    B.m.col = nullptr;
    B.m.val = nullptr;
    B.c_st = 0;
    const size_t c = (size_t)stored + (size_t)stored / 4 + 64;
    VEM_TRY(dalloc_n(h, &B.m.col, c));
    VEM_TRY(dalloc_n(h, &B.m.val, c));
    B.c_st = c;
  }
  count_launch();
  k_csr_to_sell<<<rows_grid(ns * 32), 256, 0, s>>>(ns, C.rp, rows, C.col, C.val, B.m.off, B.m.col, B.m.val);
  VEM_CUDA(h, cudaGetLastError());
  B.m.rows = rows;
  B.m.nslices = ns;
  B.m.stored = stored;
  B.m.nnz = C.nnz;
  return VEM_OK;
}

static double bits_to_double(unsigned long long b) {
  double d;
  memcpy(&d, &b, sizeof(d));
  return d;
}

static DMat level_op(AmgState *S, int l) { return l == 0 ? dview(S->S0) : dview(S->lv[l].A); }

// dynamic shared memory of k_prod_rows: values, keys, counts
static size_t prod_smem_bytes(int bits, int warps) {
  return (size_t)warps * ((size_t)(1 << bits) * (sizeof(double) + sizeof(int32_t)) + sizeof(int));
}

__global__ void k_count_flags(int64_t n, const uint8_t *__restrict__ f, unsigned long long *out) {
  unsigned long long c = 0;
  ROWS_LOOP(i, n) c += f[i] != 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Sort the rows of a CSR matrix by column: rows of up to kSortMax entries a
// warp each in blocks of kProdWarps, longer ones (up to 2^kBigBits) one warp
// per block with a large shared buffer.
static vem_status sort_rows(vem_handle *h, AmgState *S, int64_t n, const int64_t *rp, int32_t *col, double *val) {
  cudaStream_t s = h->stream;
  constexpr int kBigCap = 1 << kBigBits;
  const size_t sm = (size_t)kProdWarps * kSortMax * (sizeof(double) + sizeof(int32_t));
  const size_t smb = (size_t)kBigCap * (sizeof(double) + sizeof(int32_t));
  VEM_CUDA(h, cudaFuncSetAttribute(k_sort_rows<kBigCap, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb));
  VEM_TRY(grow(h, S->big, S->c_big, (size_t)std::max<int64_t>(n, 1)));
  VEM_CUDA(h, cudaMemsetAsync(S->big, 0, (size_t)n, s));
  count_launch();
  k_sort_rows<kSortMax, kProdWarps><<<prod_grid(n), 32 * kProdWarps, sm, s>>>(n, rp, col, val, h->d_err, S->big,
                                                                              false);
  unsigned long long *nbig = S->ctr + kMaxRounds + 2;
  VEM_CUDA(h, cudaMemsetAsync(nbig, 0, sizeof(*nbig), s));
  count_launch();
  k_count_flags<<<rows_grid(n), 256, 0, s>>>(n, S->big, nbig);
  unsigned long long nb = 0;
  VEM_CUDA(h, cudaMemcpyAsync(&nb, nbig, sizeof(nb), cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaStreamSynchronize(s));
  if (nb) {
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nb, (int64_t)num_sms() * 2));
    count_launch();
    k_sort_rows<kBigCap, 1><<<gb, 32, smb, s>>>(n, rp, col, val, h->d_err, S->big, true);
  }
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

// C = X Y.  One pass when the candidate products fit the scratch budget:
// every row is formed once into a scratch buffer at an upper-bound offset
// (its candidate count), then the rows are compacted; otherwise two passes
// (count, fill).  With short_rows one thread per row (at most 64 distinct
// columns, else the product is redone a warp per row); warp rows that
// overflow the small hash table are redone with the large one.  Both ways
// form each row with the same kernels in the same order, so C is the same
// bit for bit.
constexpr size_t kProdScratchMax = size_t(6) << 30;   // bytes of scratch for the one-pass form

static bool amg_debug() {
  static int v = -1;
  if (v < 0) v = std::getenv("VEM_DEBUG") ? 1 : 0;
  return v == 1;
}

static vem_status product(vem_handle *h, AmgState *S, const DMat &X, const CsrBuf &Y, CsrBuf &C,
                          bool short_rows) {
  cudaStream_t s = h->stream;
  VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)X.rows + 1));
  unsigned long long *ovf = S->ctr + kMaxRounds + 3;
  unsigned long long over = 0;
  const size_t sm = prod_smem_bytes(kHashBits, kProdWarps), smb = prod_smem_bytes(kBigBits, 1);
  VEM_CUDA(h, cudaFuncSetAttribute(k_prod_rows<false, kBigBits, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smb));
  VEM_CUDA(h, cudaFuncSetAttribute(k_prod_rows<true, kBigBits, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smb));
  // ---- one pass through the scratch ----
  VEM_TRY(grow(h, S->coff, S->c_coff, (size_t)X.rows + 1));
  count_launch();
  k_prod_cand<<<rows_grid(X.rows), 256, 0, s>>>(X, Y.rp, S->cnt);
  int64_t ncand = 0;
  VEM_TRY(scan_counts(h, X.rows, S->cnt, S->coff, &ncand));   // synchronises
  if ((size_t)ncand * (sizeof(double) + sizeof(int32_t)) <= kProdScratchMax) {
    VEM_TRY(grow(h, S->tcol, S->c_tcol, (size_t)std::max<int64_t>(ncand, 1)));
    VEM_TRY(grow(h, S->tval, S->c_tval, (size_t)std::max<int64_t>(ncand, 1)));
    bool warp_rows = !short_rows;
    if (short_rows) {
      VEM_CUDA(h, cudaMemsetAsync(ovf, 0, sizeof(*ovf), s));
      count_launch();
      k_prod_rows_thread<true><<<rows_grid(X.rows), 256, 0, s>>>(X, Y.rp, Y.col, Y.val, S->cnt, S->coff, S->tcol,
                                                                 S->tval, ovf);
      VEM_CUDA(h, cudaMemcpyAsync(&over, ovf, sizeof(over), cudaMemcpyDeviceToHost, s));
      VEM_CUDA(h, cudaStreamSynchronize(s));
      warp_rows = over != 0;
    }
    if (warp_rows) {
      const int g = prod_grid(X.rows);
      VEM_TRY(grow(h, S->big, S->c_big, (size_t)X.rows));
      VEM_CUDA(h, cudaMemsetAsync(S->big, 0, (size_t)X.rows, s));
      count_launch();
      k_prod_rows<true, kHashBits, kProdWarps><<<g, 32 * kProdWarps, sm, s>>>(
          X, Y.rp, Y.col, Y.val, S->cnt, S->coff, S->tcol, S->tval, h->d_err, S->big, false);
      unsigned long long *nbig = S->ctr + kMaxRounds + 2;
      VEM_CUDA(h, cudaMemsetAsync(nbig, 0, sizeof(*nbig), s));
      count_launch();
      k_count_flags<<<rows_grid(X.rows), 256, 0, s>>>(X.rows, S->big, nbig);
      unsigned long long nb = 0;
      VEM_CUDA(h, cudaMemcpyAsync(&nb, nbig, sizeof(nb), cudaMemcpyDeviceToHost, s));
      VEM_CUDA(h, cudaStreamSynchronize(s));
      if (amg_debug())
        fprintf(stderr, "[vem] product rows=%lld cols=%lld candidates=%lld wide rows=%llu\n", (long long)X.rows,
                (long long)Y.cols, (long long)ncand, nb);
      if (nb) {
        const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nb, (int64_t)num_sms() * 2));
        count_launch();
        k_prod_rows<true, kBigBits, 1><<<gb, 32, smb, s>>>(X, Y.rp, Y.col, Y.val, S->cnt, S->coff, S->tcol,
                                                            S->tval, h->d_err, S->big, true);
      }
    }
    VEM_TRY(csr_layout(h, C, X.rows, Y.cols, S->cnt));
    count_launch();
    k_compact_rows<<<warps_grid(X.rows), 256, 0, s>>>(X.rows, S->coff, C.rp, S->tcol, S->tval, C.col, C.val);
    VEM_CUDA(h, cudaGetLastError());
    return VEM_OK;
  }
  // ---- two passes ----
  if (short_rows) {
    const int g = rows_grid(X.rows);
    VEM_CUDA(h, cudaMemsetAsync(ovf, 0, sizeof(*ovf), s));
    count_launch();
    k_prod_rows_thread<false><<<g, 256, 0, s>>>(X, Y.rp, Y.col, Y.val, S->cnt, nullptr, nullptr, nullptr, ovf);
    VEM_CUDA(h, cudaMemcpyAsync(&over, ovf, sizeof(over), cudaMemcpyDeviceToHost, s));
    VEM_TRY(csr_layout(h, C, X.rows, Y.cols, S->cnt));   // synchronises
  }
  if (short_rows && !over) {
    count_launch();
    k_prod_rows_thread<true><<<rows_grid(X.rows), 256, 0, s>>>(X, Y.rp, Y.col, Y.val, nullptr, C.rp, C.col, C.val,
                                                               ovf);
  } else {
    const int g = prod_grid(X.rows);
    VEM_TRY(grow(h, S->big, S->c_big, (size_t)X.rows));
    VEM_CUDA(h, cudaMemsetAsync(S->big, 0, (size_t)X.rows, s));
    count_launch();
    k_prod_rows<false, kHashBits, kProdWarps><<<g, 32 * kProdWarps, sm, s>>>(
        X, Y.rp, Y.col, Y.val, S->cnt, nullptr, nullptr, nullptr, h->d_err, S->big, false);
    // rows that overflowed the small tables: count them again with a large one
    unsigned long long *nbig = S->ctr + kMaxRounds + 2;
    VEM_CUDA(h, cudaMemsetAsync(nbig, 0, sizeof(*nbig), s));
    count_launch();
    k_count_flags<<<rows_grid(X.rows), 256, 0, s>>>(X.rows, S->big, nbig);
    unsigned long long nb = 0;
    VEM_CUDA(h, cudaMemcpyAsync(&nb, nbig, sizeof(nb), cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nb, (int64_t)num_sms() * 2));
    if (nb) {
      count_launch();
      k_prod_rows<false, kBigBits, 1><<<gb, 32, smb, s>>>(X, Y.rp, Y.col, Y.val, S->cnt, nullptr, nullptr, nullptr,
                                                           h->d_err, S->big, true);
    }
    VEM_TRY(csr_layout(h, C, X.rows, Y.cols, S->cnt));
    count_launch();
    k_prod_rows<true, kHashBits, kProdWarps><<<g, 32 * kProdWarps, sm, s>>>(
        X, Y.rp, Y.col, Y.val, nullptr, C.rp, C.col, C.val, h->d_err, S->big, false);
    if (nb) {
      count_launch();
      k_prod_rows<true, kBigBits, 1><<<gb, 32, smb, s>>>(X, Y.rp, Y.col, Y.val, nullptr, C.rp, C.col, C.val,
                                                          h->d_err, S->big, true);
    }
  }
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

// Strength of connection on the graph of A (|a_ij| >= theta sqrt(a_ii a_jj)
// with dg the diagonal), the distance-2 maximal independent set in rounds and
// the three aggregation passes: agg[i] (-1 outside the coarse space), the
// number of aggregates nc and the two Gershgorin maxima (mx[0]: of D^-1 A,
// mx[1]: of the filtered D^-1 A^F) as double bit patterns.  mis_rounds: the
// rounds this graph needed in the last setup (updated).
static vem_status aggregate_graph(vem_handle *h, AmgState *S, const DMat &A, const double *dg, double theta,
                                  int32_t *agg, int &mis_rounds, int64_t *nc_out, unsigned long long mx[2]) {
  cudaStream_t s = h->stream;
  const int64_t n = A.rows;
  *nc_out = 0;
  VEM_TRY(grow(h, S->flag, S->c_flag, (size_t)A.stored));
  VEM_TRY(grow(h, S->nstr, S->c_nstr, (size_t)n));
  VEM_TRY(grow(h, S->tup, S->c_tup, 2 * (size_t)n));
  VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)n + 1));
  VEM_TRY(grow(h, S->scn, S->c_scn, (size_t)n + 1));
  VEM_TRY(grow(h, S->agg1, S->c_agg1, (size_t)n));
  const int g = rows_grid(n);

  // strength and the Gershgorin maxima (diagonal and dinv already computed)
  VEM_CUDA(h, cudaMemsetAsync(S->ctr, 0, sizeof(unsigned long long) * (kMaxRounds + 4), s));
  count_launch();
  k_amg_strength<<<g, 256, 0, s>>>(A, dg, theta, S->flag, S->nstr, S->ctr);
  // MIS-2 rounds.  The host reads the undecided counts after a batch of
  // rounds: first as many as this level needed in the last setup (rounds
  // after the set is complete change nothing), then two at a time.
  count_launch();
  k_mis_init<<<g, 256, 0, s>>>(n, S->tup);
  uint64_t *t1 = S->tup + n;
  int round = 0;
  int batch = std::max(2, mis_rounds);
  int needed = 0;
  while (needed == 0) {
    if (round + batch > kMaxRounds) return fail(h, VEM_ERR_CUDA, "AMG aggregation did not finish in %d rounds", kMaxRounds);
    for (int k = 0; k < batch; ++k, ++round) {
      count_launch();
      k_mis_max1<<<g, 256, 0, s>>>(A, S->flag, S->tup, t1);
      count_launch();
      k_mis_max2<<<g, 256, 0, s>>>(A, S->flag, t1, S->tup, S->ctr + 2 + round);
    }
    VEM_CUDA(h, cudaGetLastError());
    unsigned long long und[kMaxRounds];
    VEM_CUDA(h, cudaMemcpyAsync(und, S->ctr + 2 + round - batch, sizeof(und[0]) * batch, cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    for (int k = 0; k < batch && needed == 0; ++k)
      if (und[k] == 0) needed = round - batch + k + 1;
    batch = 2;
  }
  mis_rounds = needed;
  VEM_CUDA(h, cudaMemcpyAsync(mx, S->ctr, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  // aggregates
  count_launch();
  k_agg_root<<<g, 256, 0, s>>>(n, S->tup, S->nstr, S->cnt);
  int64_t nroot = 0;
  VEM_TRY(scan_counts(h, n, S->cnt, S->scn, &nroot));
  count_launch();
  k_agg_pass1<<<g, 256, 0, s>>>(A, S->flag, S->tup, S->nstr, S->scn, S->agg1);
  count_launch();
  k_agg_pass2<<<g, 256, 0, s>>>(A, S->flag, S->nstr, S->agg1, agg, S->cnt);
  int64_t nfree = 0;
  VEM_TRY(scan_counts(h, n, S->cnt, S->scn, &nfree));
  count_launch();
  k_agg_pass3<<<g, 256, 0, s>>>(n, nroot, S->nstr, S->scn, agg);
  VEM_CUDA(h, cudaGetLastError());
  *nc_out = nroot + nfree;
  return VEM_OK;
}

// One level: strength, MIS-2, aggregates, P, R and the coarse operator.
// Returns nc = 0 when the level is not coarsened.
static vem_status coarsen(vem_handle *h, AmgState *S, int l, double theta, int64_t *nc_out) {
  cudaStream_t s = h->stream;
  AmgLevel &L = S->lv[l];
  const DMat A = level_op(S, l);
  const int64_t n = A.rows;
  *nc_out = 0;
  VEM_TRY(grow(h, L.agg, L.c_agg, (size_t)n));
  const int g = rows_grid(n);
  unsigned long long mx[2] = {0, 0};
  int64_t nc = 0;
  VEM_TRY(aggregate_graph(h, S, A, S->dg, theta, L.agg, L.mis_rounds, &nc, mx));
  if (nc == 0 || 5 * nc > 4 * n) return VEM_OK;
  const double rho = bits_to_double(mx[0]), rhof = bits_to_double(mx[1]);
  L.rho = rho;
  L.omega = 4.0 / (3.0 * rho);
  const double omega_f = 4.0 / (3.0 * rhof);

  // P
  count_launch();
  k_p_rows<false><<<g, 256, 0, s>>>(A, S->flag, L.dinv, L.agg, omega_f, S->cnt, nullptr, nullptr, nullptr, h->d_err);
  VEM_TRY(csr_layout(h, L.P, n, nc, S->cnt));
  count_launch();
  k_p_rows<true><<<g, 256, 0, s>>>(A, S->flag, L.dinv, L.agg, omega_f, nullptr, L.P.rp, L.P.col, L.P.val, h->d_err);
  VEM_TRY(check_device_errors(h, "AMG prolongator"));
  // R = P^T, rows sorted by fine index
  VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)nc + 1));
  VEM_CUDA(h, cudaMemsetAsync(S->cnt, 0, sizeof(int64_t) * nc, s));
  count_launch();
  k_t_count<<<g, 256, 0, s>>>(n, L.P.rp, L.P.col, reinterpret_cast<unsigned long long *>(S->cnt));
  VEM_TRY(csr_layout(h, L.R, nc, n, S->cnt));
  VEM_TRY(grow(h, S->cur, S->c_cur, (size_t)nc + 1));
  VEM_CUDA(h, cudaMemcpyAsync(S->cur, L.R.rp, sizeof(int64_t) * nc, cudaMemcpyDeviceToDevice, s));
  count_launch();
  k_t_fill<<<g, 256, 0, s>>>(n, L.P.rp, L.P.col, L.P.val, reinterpret_cast<unsigned long long *>(S->cur), L.R.col,
                             L.R.val);
  count_launch();
  VEM_TRY(sort_rows(h, S, nc, L.R.rp, L.R.col, L.R.val));
  VEM_CUDA(h, cudaGetLastError());
  // A P, then R (A P)
  // the finest level's A P has short rows: try one thread per row first
  VEM_TRY(product(h, S, A, L.P, S->AP, l == 0));
  VEM_TRY(product(h, S, dview(L.R), S->AP, S->lv[l + 1].A, false));
  VEM_TRY(check_device_errors(h, "AMG Galerkin product"));
  L.Rs.m.rows = 0;
  L.Ps.m.rows = 0;
  S->lv[l + 1].As.m.rows = 0;
  if (L.R.rows >= kSellMinRows) VEM_TRY(csr_to_sell(h, S, L.R, L.Rs));
  if (L.P.rows >= kSellMinRows) VEM_TRY(csr_to_sell(h, S, L.P, L.Ps));
  if (nc >= kSellMinRows) VEM_TRY(csr_to_sell(h, S, S->lv[l + 1].A, S->lv[l + 1].As));
  L.nc = nc;
  *nc_out = nc;
  return VEM_OK;
}

// cycle vectors per level: x, x2, b, r, and xc for the Chebyshev smoother
static int nvec(const AmgState *S) { return S->smoother == kSmoothChebyshev ? 5 : 4; }

static vem_status level_vectors(vem_handle *h, AmgState *S, int l) {
  AmgLevel &L = S->lv[l];
  const DMat A = level_op(S, l);
  L.n = A.rows;
  VEM_TRY(grow(h, L.dinv, L.c_dinv, (size_t)L.n));
  VEM_TRY(grow(h, L.vec, L.c_vec, nvec(S) * (size_t)L.n));
  VEM_TRY(grow(h, S->dg, S->c_dg, (size_t)L.n));
  count_launch();
  k_amg_diag<<<rows_grid(L.n), 256, 0, h->stream>>>(A, S->dg, L.dinv, h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

template <class Tb>
static vem_status to_f32(vem_handle *h, float *&dst, size_t &cap, const Tb *src, int64_t n) {
  VEM_TRY(grow(h, dst, cap, (size_t)std::max<int64_t>(n, 1)));
  if (n > 0) {
    count_launch();
    k_vc_convert<Tb, float><<<rows_grid(n), 256, 0, h->stream>>>(n, src, dst, nullptr);
  }
  return VEM_OK;
}

// FP32 copies of everything the cycle reads (values, wd, the coarsest inverse)
static vem_status make_fp32(vem_handle *h, AmgState *S) {
  for (int l = 0; l < S->nlev; ++l) {
    AmgLevel &L = S->lv[l];
    VEM_TRY(to_f32(h, L.wd32, L.c_wd32, L.wd, L.n));
    // the Chebyshev second-step weights exist on the levels above the coarsest
    if (S->smoother == kSmoothChebyshev && l + 1 < S->nlev) VEM_TRY(to_f32(h, L.wdc32, L.c_wdc32, L.wdc, L.n));
    VEM_TRY(grow(h, L.vec32, L.c_vec32, nvec(S) * (size_t)L.n));
    if (l > 0) {
      if (L.As.m.rows) VEM_TRY(to_f32(h, L.As.val32, L.As.c_v32, L.As.m.val, L.As.m.stored));
      else VEM_TRY(to_f32(h, L.A.val32, L.A.c_v32, L.A.val, L.A.nnz));
    }
    if (l + 1 < S->nlev) {
      if (L.Rs.m.rows) VEM_TRY(to_f32(h, L.Rs.val32, L.Rs.c_v32, L.Rs.m.val, L.Rs.m.stored));
      else VEM_TRY(to_f32(h, L.R.val32, L.R.c_v32, L.R.val, L.R.nnz));
      if (L.Ps.m.rows) VEM_TRY(to_f32(h, L.Ps.val32, L.Ps.c_v32, L.Ps.m.val, L.Ps.m.stored));
      else VEM_TRY(to_f32(h, L.P.val32, L.P.c_v32, L.P.val, L.P.nnz));
    }
  }
  if (S->csweeps == 0) {
    const int64_t cn = S->lv[S->nlev - 1].n;
    VEM_TRY(to_f32(h, S->cinv32, S->c_cinv32, S->cinv, cn * cn));
  }
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

vem_status amg_setup(vem_handle *h, AmgState *&slot, const SellMat &Sm, const float *S_val32, bool fp32,
                     bool pin_last, int smoother) {
  if (!slot) slot = new AmgState();
  AmgState *S = slot;
  S->valid = false;
  S->fp32 = fp32;
  S->S0_val32 = S_val32;
  S->pin_last = pin_last;
  S->smoother = smoother;
  S->block = false;
  S->condensed = false;
  if (fp32 && !S_val32) return fail(h, VEM_ERR_BAD_INPUT, "FP32 AMG cycle without FP32 values of the operator");
  cudaStream_t s = h->stream;
  VEM_CUDA(h, cudaEventRecord(h->ev2, s));
  if (!S->ctr) VEM_TRY(dalloc_n(h, &S->ctr, kMaxRounds + 4));
  S->S0 = Sm;
  S->nlev = 1;
  double theta = kTheta0;
  for (int l = 0;; ++l) {
    VEM_TRY(level_vectors(h, S, l));
    AmgLevel &L = S->lv[l];
    if (L.n <= kCoarseMax || l + 1 == kMaxLevels) break;
    int64_t nc = 0;
    VEM_TRY(coarsen(h, S, l, theta, &nc));
    if (nc == 0) break;
    S->nlev = l + 2;
    theta *= 0.5;
  }
  // Jacobi weight of the coarsest level (coarsen() sets it for the others)
  AmgLevel &C = S->lv[S->nlev - 1];
  const DMat CA = level_op(S, S->nlev - 1);
  {
    VEM_TRY(grow(h, S->flag, S->c_flag, (size_t)CA.stored));
    VEM_TRY(grow(h, S->nstr, S->c_nstr, (size_t)C.n));
    VEM_CUDA(h, cudaMemsetAsync(S->ctr, 0, sizeof(unsigned long long) * 2, s));
    count_launch();
    k_amg_strength<<<rows_grid(C.n), 256, 0, s>>>(CA, S->dg, 0.0, S->flag, S->nstr, S->ctr);
    unsigned long long mx[2] = {0, 0};
    VEM_CUDA(h, cudaMemcpyAsync(mx, S->ctr, sizeof(mx), cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    C.rho = bits_to_double(mx[0]);
    C.omega = 4.0 / (3.0 * C.rho);
  }
  for (int l = 0; l < S->nlev; ++l) {
    AmgLevel &L = S->lv[l];
    VEM_TRY(grow(h, L.wd, L.c_wd, (size_t)L.n));
    if (S->smoother == kSmoothChebyshev && l + 1 < S->nlev) {
      // two steps on [lo, hi] = [rho/10, rho]: x1 = x0 + D^-1 r0 / theta,
      // x2 = x1 + rho1 rho0 (x1 - x0) + (2 rho1 / delta) D^-1 r1
      const double hi = L.rho, lo = hi / 10.0;
      const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
      const double rho0 = 1.0 / sigma, rho1 = 1.0 / (2.0 * sigma - rho0);
      L.cheb_c = rho1 * rho0;
      VEM_TRY(grow(h, L.wdc, L.c_wdc, (size_t)L.n));
      count_launch();
      k_scale_into<<<rows_grid(L.n), 256, 0, s>>>(L.n, L.dinv, 1.0 / theta, L.wd);
      count_launch();
      k_scale_into<<<rows_grid(L.n), 256, 0, s>>>(L.n, L.dinv, 2.0 * rho1 / delta, L.wdc);
    } else {
      count_launch();
      k_scale_into<<<rows_grid(L.n), 256, 0, s>>>(L.n, L.dinv, L.omega, L.wd);
    }
  }
  if (C.n <= kDenseMax) {
    VEM_TRY(grow(h, S->cinv, S->c_cinv, (size_t)C.n * C.n));
    count_launch();
    k_dense_from<<<rows_grid(C.n), 256, 0, s>>>(CA, S->cinv);
    if (S->pin_last) {
      // S is singular (constants): keep the diagonal of the last coarse row
      // and column, drop their other entries
      count_launch();
      k_pin_last<<<1, 256, 0, s>>>((int)C.n, S->cinv);
    }
    count_launch();
    k_gauss_jordan<<<1, 256, 0, s>>>((int)C.n, S->cinv, h->d_err);
    S->csweeps = 0;
  } else {
    S->csweeps = kCoarseSweeps;
  }
  VEM_CUDA(h, cudaGetLastError());
  if (fp32) VEM_TRY(make_fp32(h, S));
  VEM_TRY(check_device_errors(h, "AMG setup"));
  VEM_CUDA(h, cudaEventRecord(h->ev3, s));
  VEM_CUDA(h, cudaEventSynchronize(h->ev3));
  float ms = 0.f;
  VEM_CUDA(h, cudaEventElapsedTime(&ms, h->ev2, h->ev3));
  S->t_setup_ms = ms;
  S->valid = true;
  ++S->generation;
  return VEM_OK;
}

// ------------------------------------------------- point-block setup ------
// X^T of a CSR matrix with cols columns, rows sorted by column.
static vem_status transpose_csr(vem_handle *h, AmgState *S, const CsrBuf &X, int64_t cols, CsrBuf &XT) {
  cudaStream_t s = h->stream;
  const int g = rows_grid(X.rows);
  VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)cols + 1));
  VEM_CUDA(h, cudaMemsetAsync(S->cnt, 0, sizeof(int64_t) * cols, s));
  count_launch();
  k_t_count<<<g, 256, 0, s>>>(X.rows, X.rp, X.col, reinterpret_cast<unsigned long long *>(S->cnt));
  VEM_TRY(csr_layout(h, XT, cols, X.rows, S->cnt));
  VEM_TRY(grow(h, S->cur, S->c_cur, (size_t)cols + 1));
  VEM_CUDA(h, cudaMemcpyAsync(S->cur, XT.rp, sizeof(int64_t) * cols, cudaMemcpyDeviceToDevice, s));
  count_launch();
  k_t_fill<<<g, 256, 0, s>>>(X.rows, X.rp, X.col, X.val, reinterpret_cast<unsigned long long *>(S->cur), XT.col,
                             XT.val);
  VEM_TRY(sort_rows(h, S, cols, XT.rp, XT.col, XT.val));
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

// A CSR buffer with exactly rows x (entries per row) stored entries, for
// matrices whose layout a kernel writes directly.
static vem_status csr_fixed(vem_handle *h, CsrBuf &C, int64_t rows, int64_t cols, int64_t nnz) {
  VEM_TRY(grow(h, C.rp, C.c_rp, (size_t)rows + 1));
  if (!C.col || (size_t)nnz + 1 > C.c_nz) {
    dfree(h, C.col);
    dfree(h, C.val);
    C.col = nullptr;
    C.val = nullptr;
    C.c_nz = 0;
    const size_t c = (size_t)nnz + (size_t)nnz / 4 + 64;
    VEM_TRY(dalloc_n(h, &C.col, c));
    VEM_TRY(dalloc_n(h, &C.val, c));
    C.c_nz = c;
  }
  C.rows = rows;
  C.cols = cols;
  C.nnz = nnz;
  C.lanes = lanes_for(rows, nnz);
  return VEM_OK;
}

// Largest eigenvalue of the symmetric tridiagonal matrix (alpha, beta) by
// cyclic Jacobi rotations on its dense form (k <= 11).
static double tridiag_max_eig(const std::vector<double> &al, const std::vector<double> &be) {
  const int k = (int)al.size();
  double M[12][12] = {};
  for (int i = 0; i < k; ++i) M[i][i] = al[i];
  for (int i = 0; i + 1 < k; ++i) M[i][i + 1] = M[i + 1][i] = be[i];
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) {
        tot += M[i][j] * M[i][j];
        if (i != j) off += M[i][j] * M[i][j];
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        if (M[p][q] == 0.0) continue;
        const double th = (M[q][q] - M[p][p]) / (2.0 * M[p][q]);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int r = 0; r < k; ++r) {   // columns p, q
          const double a = M[r][p], b = M[r][q];
          M[r][p] = c * a - sn * b;
          M[r][q] = sn * a + c * b;
        }
        for (int r = 0; r < k; ++r) {   // rows p, q
          const double a = M[p][r], b = M[q][r];
          M[p][r] = c * a - sn * b;
          M[q][r] = sn * a + c * b;
        }
      }
  }
  double mx = M[0][0];
  for (int i = 1; i < k; ++i) mx = std::max(mx, M[i][i]);
  return mx;
}

// Largest Ritz value of C after `steps` Lanczos steps (full
// reorthogonalisation by one classical Gram-Schmidt pass, as stated above).
static vem_status lanczos_max(vem_handle *h, AmgState *S, const CsrBuf &C, int steps, double *ritz) {
  cudaStream_t s = h->stream;
  const int64_t n = C.rows;
  if (steps > n) steps = (int)n;
  VEM_TRY(grow(h, S->lz, S->c_lz, (size_t)n * (steps + 2)));
  VEM_TRY(grow(h, S->lpart, S->c_lpart, (size_t)kDotBlocks * (steps + 1) + 16));
  double *V = S->lz, *w = S->lz + (size_t)n * (steps + 1);
  double *hd = S->lpart + (size_t)kDotBlocks * (steps + 1);
  const int g = rows_grid(n);
  count_launch();
  k_start_vec<<<g, 256, 0, s>>>(n, w);
  count_launch();
  k_dots_part<<<kDotBlocks, 256, 0, s>>>(n, 1, w, w, S->lpart);
  count_launch();
  k_dots_fin<<<1, 32, 0, s>>>(1, S->lpart, hd);
  count_launch();
  k_scale_copy<<<g, 256, 0, s>>>(n, w, hd, V);
  std::vector<double> al, be;
  double hh[16];
  for (int k = 0; k < steps; ++k) {
    count_launch();
    k_csr_spmv<<<g, 256, 0, s>>>(n, C.rp, C.col, C.val, V + (size_t)k * n, w);
    count_launch();
    k_dots_part<<<kDotBlocks, 256, 0, s>>>(n, k + 1, V, w, S->lpart);
    count_launch();
    k_dots_fin<<<1, 32, 0, s>>>(k + 1, S->lpart, hd);
    count_launch();
    k_sub_proj<<<g, 256, 0, s>>>(n, k + 1, V, hd, w);
    count_launch();
    k_dots_part<<<kDotBlocks, 256, 0, s>>>(n, 1, w, w, S->lpart);
    count_launch();
    k_dots_fin<<<1, 32, 0, s>>>(1, S->lpart, hd + k + 1);
    VEM_CUDA(h, cudaMemcpyAsync(hh, hd, sizeof(double) * (k + 2), cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    const double a = hh[k], b = std::sqrt(hh[k + 1]);
    al.push_back(a);
    if (b <= 1e-12 * std::fabs(a) || k == steps - 1) break;
    be.push_back(b);
    count_launch();
    k_scale_copy<<<g, 256, 0, s>>>(n, w, hd + k + 1, V + (size_t)(k + 1) * n);
  }
  VEM_CUDA(h, cudaGetLastError());
  *ritz = tridiag_max_eig(al, be);
  return VEM_OK;
}

// Whether the block rows of X share their pattern (k_blockrow_same).
static vem_status block_rows_uniform(vem_handle *h, AmgState *S, const DMat &X, int bs, bool whole, bool *ok) {
  if (!S->bflag) VEM_TRY(dalloc_n(h, &S->bflag, 1));
  VEM_CUDA(h, cudaMemsetAsync(S->bflag, 0, sizeof(int), h->stream));
  count_launch();
  k_blockrow_same<<<rows_grid(X.rows), 256, 0, h->stream>>>(X, bs, whole ? 1 : 0, S->bflag);
  int bad = 0;
  VEM_CUDA(h, cudaMemcpyAsync(&bad, S->bflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  VEM_CUDA(h, cudaStreamSynchronize(h->stream));
  *ok = bad == 0;
  return VEM_OK;
}

// Diagonal blocks, their inverses and the spectral estimate of D^-1 A for
// level l (block size L.bs).
static vem_status block_level_setup(vem_handle *h, AmgState *S, int l) {
  cudaStream_t s = h->stream;
  AmgLevel &L = S->lv[l];
  const DMat A = level_op(S, l);
  const int bs = L.bs;
  const int64_t n = L.n, nb = n / bs;
  VEM_TRY(grow(h, L.dblk, L.c_dblk, (size_t)nb * bs * bs));
  VEM_TRY(grow(h, L.lblk, L.c_lblk, (size_t)nb * bs * bs));
  count_launch();
  k_blk_diag<kMaxBs><<<rows_grid(nb), 256, 0, s>>>(nb, bs, A, L.dblk, L.lblk, h->d_err);
  VEM_TRY(check_device_errors(h, "point-block AMG diagonal blocks"));
  // C = L^-1 (A L^-T): one pass over A's blocks when its block rows share
  // their pattern, else two sparse products
  bool uniform = false;
  VEM_TRY(block_rows_uniform(h, S, A, bs, true, &uniform));
  if (uniform) {
    VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)n + 1));
    count_launch();
    k_row_lengths<<<rows_grid(n), 256, 0, s>>>(A, S->cnt);
    VEM_TRY(csr_layout(h, S->bC, n, n, S->cnt));
    count_launch();
    k_blk_congruence<<<rows_grid(n), 256, 0, s>>>(A, bs, L.lblk, S->bC.rp, S->bC.col, S->bC.val);
    VEM_CUDA(h, cudaGetLastError());
  } else {
    VEM_TRY(csr_fixed(h, S->bLm, n, n, n * bs));
    VEM_TRY(csr_fixed(h, S->bLmT, n, n, n * bs));
    count_launch();
    k_blkdiag_rows<<<rows_grid(n), 256, 0, s>>>(n, bs, L.lblk, 0, S->bLm.rp, S->bLm.col, S->bLm.val);
    count_launch();
    k_blkdiag_rows<<<rows_grid(n), 256, 0, s>>>(n, bs, L.lblk, 1, S->bLmT.rp, S->bLmT.col, S->bLmT.val);
    VEM_TRY(product(h, S, A, S->bLmT, S->bY, false));
    VEM_TRY(product(h, S, dview(S->bLm), S->bY, S->bC, false));
  }
  unsigned long long *mx = S->ctr + kMaxRounds + 1;
  VEM_CUDA(h, cudaMemsetAsync(mx, 0, sizeof(*mx), s));
  count_launch();
  k_abs_rowsum_max<<<rows_grid(n), 256, 0, s>>>(n, S->bC.rp, S->bC.val, mx);
  unsigned long long gb = 0;
  VEM_CUDA(h, cudaMemcpyAsync(&gb, mx, sizeof(gb), cudaMemcpyDeviceToHost, s));
  double ritz = 0.0;
  VEM_TRY(lanczos_max(h, S, S->bC, 10, &ritz));   // synchronises
  const double gersh = bits_to_double(gb);
  L.rho = std::min(gersh, 1.1 * ritz);
  L.omega = 4.0 / (3.0 * L.rho);
  VEM_TRY(check_device_errors(h, "point-block AMG spectral estimate"));
  return VEM_OK;
}

// One point-block level: block graph, aggregates, tentative and smoothed
// prolongators, restriction and the coarse operator.  nc = 0: not coarsened.
static vem_status block_coarsen(vem_handle *h, AmgState *S, int l, double theta, const double *Bl, int64_t *nc_out) {
  cudaStream_t s = h->stream;
  AmgLevel &L = S->lv[l];
  const DMat A = level_op(S, l);
  const int bs = L.bs, m = S->m;
  const int64_t n = L.n, nb = n / bs;
  *nc_out = 0;
  // N = sqrt(Q^T (A o A) Q)
  VEM_TRY(grow(h, S->sq, S->c_sq, (size_t)std::max<int64_t>(A.stored, 1)));
  count_launch();
  k_square<<<rows_grid(A.stored), 256, 0, s>>>(A.stored, A.val, S->sq);
  DMat A2 = A;
  A2.val = S->sq;
  VEM_TRY(csr_fixed(h, S->bQ, n, nb, n));
  VEM_TRY(csr_fixed(h, S->bQT, nb, n, n));
  count_launch();
  k_member_rows<<<rows_grid(n), 256, 0, s>>>(n, bs, S->bQ.rp, S->bQ.col, S->bQ.val);
  count_launch();
  k_member_cols<<<rows_grid(nb), 256, 0, s>>>(nb, bs, S->bQT.rp, S->bQT.col, S->bQT.val);
  VEM_TRY(product(h, S, A2, S->bQ, S->bAQ, l == 0));
  VEM_TRY(product(h, S, dview(S->bQT), S->bAQ, S->bN, false));
  count_launch();
  k_sqrt_inplace<<<rows_grid(S->bN.nnz), 256, 0, s>>>(S->bN.nnz, S->bN.val);
  // aggregates of the block graph
  const DMat Nv = dview(S->bN);
  VEM_TRY(grow(h, S->dgb, S->c_dgb, (size_t)nb));
  VEM_TRY(grow(h, S->dgbi, S->c_dgbi, (size_t)nb));
  count_launch();
  k_amg_diag<<<rows_grid(nb), 256, 0, s>>>(Nv, S->dgb, S->dgbi, h->d_err);
  VEM_TRY(grow(h, L.agg, L.c_agg, (size_t)nb));
  unsigned long long mx[2] = {0, 0};
  int64_t nc = 0;
  VEM_TRY(aggregate_graph(h, S, Nv, S->dgb, theta, L.agg, L.mis_rounds, &nc, mx));
  if (nc == 0 || 5 * nc > 4 * nb) return VEM_OK;
  // members of every aggregate in increasing block order
  auto members = [&]() -> vem_status {
    VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)nb + 1));
    count_launch();
    k_agg_count<<<rows_grid(nb), 256, 0, s>>>(nb, L.agg, S->cnt);
    VEM_TRY(csr_layout(h, S->bAgg, nb, nc, S->cnt));
    count_launch();
    k_agg_fill<<<rows_grid(nb), 256, 0, s>>>(nb, L.agg, S->bAgg.rp, S->bAgg.col, S->bAgg.val);
    return transpose_csr(h, S, S->bAgg, nc, S->bAggT);
  };
  VEM_TRY(members());
  // dissolve the aggregates on which the near-null space loses rank
  {
    int64_t *keep = S->cnt;   // nc + 1 <= nb + 1 entries, free after the layout above
    VEM_TRY(grow(h, S->scn, S->c_scn, (size_t)nc + 1));
    count_launch();
    k_tent_rank<<<rows_grid(nc), 256, 0, s>>>(nc, bs, m, S->bAggT.rp, S->bAggT.col, Bl, keep, h->d_err);
    int64_t nkeep = 0;
    VEM_TRY(scan_counts(h, nc, keep, S->scn, &nkeep));
    if (nkeep < nc) {
      count_launch();
      k_agg_renumber<<<rows_grid(nb), 256, 0, s>>>(nb, keep, S->scn, L.agg);
      nc = nkeep;
      if (nc == 0) return VEM_OK;
      VEM_TRY(members());
    }
  }
  // T and the coarse near-null space
  AmgLevel &Cl = S->lv[l + 1];
  VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)n + 1));
  count_launch();
  k_tent_count<<<rows_grid(n), 256, 0, s>>>(n, bs, m, L.agg, S->cnt);
  VEM_TRY(csr_layout(h, S->bT, n, nc * m, S->cnt));
  VEM_TRY(grow(h, Cl.bns, Cl.c_bns, (size_t)nc * m * m));
  count_launch();
  k_tent<<<rows_grid(nc), 256, 0, s>>>(nc, bs, m, S->bAggT.rp, S->bAggT.col, Bl, S->bT.rp, S->bT.col, S->bT.val,
                                       Cl.bns, h->d_err);
  VEM_TRY(check_device_errors(h, "point-block AMG tentative prolongator"));
  // P = T - omega D^-1 (A T)
  VEM_TRY(product(h, S, A, S->bT, S->bY, l == 0));
  bool uniform = false;
  VEM_TRY(block_rows_uniform(h, S, dview(S->bY), bs, false, &uniform));
  if (uniform) {
    VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)n + 1));
    count_launch();
    k_row_lengths<<<rows_grid(n), 256, 0, s>>>(dview(S->bY), S->cnt);
    VEM_TRY(csr_layout(h, S->bZ, n, S->bY.cols, S->cnt));
    count_launch();
    k_blk_left<<<rows_grid(n), 256, 0, s>>>(n, bs, L.dblk, S->bY.rp, S->bY.col, S->bY.val, S->bZ.col, S->bZ.val);
    VEM_CUDA(h, cudaGetLastError());
  } else {
    VEM_TRY(csr_fixed(h, S->bLm, n, n, n * bs));
    count_launch();
    k_blkdiag_rows<<<rows_grid(n), 256, 0, s>>>(n, bs, L.dblk, 0, S->bLm.rp, S->bLm.col, S->bLm.val);
    VEM_TRY(product(h, S, dview(S->bLm), S->bY, S->bZ, false));
  }
  count_launch();
  k_sub_rows<false><<<rows_grid(n), 256, 0, s>>>(n, S->bT.rp, S->bT.col, S->bT.val, S->bZ.rp, S->bZ.col, S->bZ.val,
                                                 L.omega, S->cnt, nullptr, nullptr, nullptr);
  VEM_TRY(csr_layout(h, L.P, n, nc * m, S->cnt));
  count_launch();
  k_sub_rows<true><<<rows_grid(n), 256, 0, s>>>(n, S->bT.rp, S->bT.col, S->bT.val, S->bZ.rp, S->bZ.col, S->bZ.val,
                                                L.omega, nullptr, L.P.rp, L.P.col, L.P.val);
  // R = P^T, A P, R (A P)
  VEM_TRY(transpose_csr(h, S, L.P, nc * m, L.R));
  VEM_TRY(product(h, S, A, L.P, S->AP, l == 0));
  VEM_TRY(product(h, S, dview(L.R), S->AP, Cl.A, false));
  VEM_TRY(check_device_errors(h, "point-block AMG Galerkin product"));
  L.Rs.m.rows = 0;
  L.Ps.m.rows = 0;
  Cl.As.m.rows = 0;
  if (L.R.rows >= kSellMinRows) VEM_TRY(csr_to_sell(h, S, L.R, L.Rs));
  if (L.P.rows >= kSellMinRows) VEM_TRY(csr_to_sell(h, S, L.P, L.Ps));
  if (nc * m >= kSellMinRows) VEM_TRY(csr_to_sell(h, S, Cl.A, Cl.As));
  L.nc = nc * m;
  *nc_out = nc;
  return VEM_OK;
}

vem_status amg_setup_block(vem_handle *h, AmgState *&slot, const SellMat &A0, int bs0, const double *B0, int m,
                           bool pin_last, int smoother) {
  if (!slot) slot = new AmgState();
  AmgState *S = slot;
  S->valid = false;
  S->fp32 = false;
  S->S0_val32 = nullptr;
  S->pin_last = pin_last;
  S->smoother = smoother;
  S->block = true;
  S->m = m;
  S->B0 = B0;
  if (bs0 < 1 || bs0 > kMaxBs || m < 1 || m > kMaxM || A0.rows % bs0)
    return fail(h, VEM_ERR_UNSUPPORTED, "point-block AMG: block size %d, near-null space of %d vectors", bs0, m);
  cudaStream_t s = h->stream;
  VEM_CUDA(h, cudaEventRecord(h->ev2, s));
  if (!S->ctr) VEM_TRY(dalloc_n(h, &S->ctr, kMaxRounds + 4));
  S->S0 = A0;
  S->nlev = 1;
  double theta = kTheta0;
  int bs = bs0;
  const double *Bl = B0;
  for (int l = 0;; ++l) {
    VEM_TRY(level_vectors(h, S, l));
    AmgLevel &L = S->lv[l];
    L.bs = bs;
    VEM_TRY(block_level_setup(h, S, l));
    if (L.n / bs <= kCoarseMax || l + 1 == kMaxLevels) break;
    int64_t nc = 0;
    VEM_TRY(block_coarsen(h, S, l, theta, Bl, &nc));
    if (nc == 0) break;
    S->nlev = l + 2;
    theta *= 0.5;
    bs = m;
    Bl = S->lv[l + 1].bns;
  }
  AmgLevel &C = S->lv[S->nlev - 1];
  const DMat CA = level_op(S, S->nlev - 1);
  for (int l = 0; l < S->nlev; ++l) {
    AmgLevel &L = S->lv[l];
    if (S->smoother == kSmoothChebyshev && l + 1 < S->nlev) {
      const double hi = L.rho, lo = hi / 10.0;
      const double th = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = th / delta;
      const double rho0 = 1.0 / sigma, rho1 = 1.0 / (2.0 * sigma - rho0);
      L.cheb_c = rho1 * rho0;
      L.cheb_theta = 1.0 / th;
      L.cheb_w2 = 2.0 * rho1 / delta;
    }
    // scalar omega D^-1 for coarsest-level sweeps (coarsest above the dense size)
    VEM_TRY(grow(h, L.wd, L.c_wd, (size_t)L.n));
    count_launch();
    k_scale_into<<<rows_grid(L.n), 256, 0, s>>>(L.n, L.dinv, L.omega, L.wd);
  }
  if (C.n <= kDenseMax) {
    VEM_TRY(grow(h, S->cinv, S->c_cinv, (size_t)C.n * C.n));
    count_launch();
    k_dense_from<<<rows_grid(C.n), 256, 0, s>>>(CA, S->cinv);
    if (S->pin_last) {
      // the constant pressure is carried by the first component of every
      // block on every level: pin that component of the last block
      count_launch();
      k_pin_row<<<1, 256, 0, s>>>((int)C.n, (int)(C.n - C.bs), S->cinv);
    }
    count_launch();
    k_gauss_jordan<<<1, 256, 0, s>>>((int)C.n, S->cinv, h->d_err);
    S->csweeps = 0;
  } else {
    S->csweeps = kCoarseSweeps;
  }
  VEM_CUDA(h, cudaGetLastError());
  VEM_TRY(check_device_errors(h, "point-block AMG setup"));
  VEM_CUDA(h, cudaEventRecord(h->ev3, s));
  VEM_CUDA(h, cudaEventSynchronize(h->ev3));
  float ms = 0.f;
  VEM_CUDA(h, cudaEventElapsedTime(&ms, h->ev2, h->ev3));
  S->t_setup_ms = ms;
  S->valid = true;
  ++S->generation;
  return VEM_OK;
}

bool amg_valid(const AmgState *S) { return S && S->valid; }
bool amg_is_block(const AmgState *S) { return S && S->block; }
bool amg_is_fp32(const AmgState *S) { return S && S->fp32; }
int64_t amg_generation(const AmgState *S) { return S ? S->generation : 0; }
void amg_invalidate(AmgState *S) {
  if (S) S->valid = false;
}
double amg_setup_ms(const AmgState *S) { return S ? S->t_setup_ms : 0.0; }
int amg_levels(const AmgState *S) { return amg_valid(S) ? S->nlev : 0; }
int amg_smoother(const AmgState *S) { return S ? S->smoother : -1; }

void amg_time_next_cycle(AmgState *S) {
  if (!S) return;
  for (cudaEvent_t &e : S->tev)
    if (!e && cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      e = nullptr;
      return;
    }
  S->timing = true;
}

void amg_collect_timing(vem_handle *h, AmgState *S) {
  if (!S || !S->timed) return;
  S->timed = false;
  float a = 0.f, b = 0.f;
  if (cudaEventElapsedTime(&a, S->tev[0], S->tev[1]) == cudaSuccess &&
      cudaEventElapsedTime(&b, S->tev[2], S->tev[3]) == cudaSuccess) {
    h->t_vc_resid_ms += a;
    h->n_vc_resid += 1;
    h->t_vc_post_ms += b;
    h->n_vc_post += 1;
  }
  cudaGetLastError();
}
void amg_free(AmgState *&S) {
  delete S;   // device buffers are in the handle's allocation list
  S = nullptr;
}

// One operator application of a level (SELL-32: S on level 0, copies above).
template <int kMode, class T, class Ty>
static void op_launch(cudaStream_t s, AmgState *S, int l, const T *x, const T *b, const T *wd, Ty *y,
                      const double *sc, const T *xp = nullptr, T c = 0) {
  if (l == 0) {
    const T *v;
    if constexpr (sizeof(T) == sizeof(double)) v = S->S0.val;
    else v = S->S0_val32;
    sell_launch<kMode>(s, S->S0, v, x, b, wd, y, sc, xp, c);
  } else if (S->lv[l].As.m.rows) {
    sell_launch<kMode>(s, S->lv[l].As.m, vals<T>(S->lv[l].As), x, b, wd, y, sc, xp, c);
  } else {
    csr_launch<kMode>(s, S->lv[l].A, x, b, wd, y, sc, xp, c);
  }
}

template <class T> static const T *wdv(const AmgLevel &L);
template <> const double *wdv<double>(const AmgLevel &L) { return L.wd; }
template <> const float *wdv<float>(const AmgLevel &L) { return L.wd32; }
template <class T> static const T *wdcv(const AmgLevel &L);
template <> const double *wdcv<double>(const AmgLevel &L) { return L.wdc; }
template <> const float *wdcv<float>(const AmgLevel &L) { return L.wdc32; }

// One block-Jacobi step of the point-block cycle (k_blk_apply modes).
static void blk_launch(cudaStream_t s, const AmgLevel &L, double scale, const double *r, const double *x,
                       const double *xp, double c, double *y, int mode, const double *sc) {
  count_launch();
  launch_pdl(k_blk_apply, rows_grid(L.n), 256, 0, s, L.n, L.bs, L.dblk, scale, r, x, xp, c, y, mode, sc);
}

static void coarsest_solve(vem_handle *h, AmgState *S, int l, const double *b, double *x, const double *sc);

// x = V(b) on level l of a point-block hierarchy (FP64): the cycle of the
// scalar hierarchy with the diagonal replaced by the bs x bs blocks.
static void bcycle(vem_handle *h, AmgState *S, int l, const double *b, double *x, const double *sc) {
  cudaStream_t s = h->stream;
  AmgLevel &L = S->lv[l];
  if (l == S->nlev - 1) {
    coarsest_solve(h, S, l, b, x, sc);
    return;
  }
  AmgLevel &C = S->lv[l + 1];
  double *xa = L.vx<double>(0), *r = L.vx<double>(3);
  double *cb = C.vx<double>(2), *cx = C.vx<double>(1);
  const bool tm = l == 0 && S->timing;
  auto mark = [&](int k) {
    if (tm) cudaEventRecord(S->tev[k], s);
  };
  auto restrict_and_recurse = [&](const double *res) {
    if (L.Rs.m.rows) sell_launch<kApply>(s, L.Rs.m, vals<double>(L.Rs), res, (const double *)nullptr,
                                         (const double *)nullptr, cb, sc);
    else csr_launch<kApply>(s, L.R, res, (const double *)nullptr, (const double *)nullptr, cb, sc);
    bcycle(h, S, l + 1, cb, cx, sc);
  };
  auto prolong_add = [&](double *y) {
    if (L.Ps.m.rows) sell_launch<kAdd>(s, L.Ps.m, vals<double>(L.Ps), (const double *)cx, (const double *)nullptr,
                                       (const double *)nullptr, y, sc);
    else csr_launch<kAdd>(s, L.P, (const double *)cx, (const double *)nullptr, (const double *)nullptr, y, sc);
  };
  if (S->smoother == kSmoothChebyshev) {
    double *xc = L.vx<double>(4);
    const double c = L.cheb_c, t = L.cheb_theta, w2 = L.cheb_w2;
    blk_launch(s, L, t, b, nullptr, nullptr, 0.0, xa, 0, sc);                       // xa = D^-1 b / theta
    op_launch<kResid>(s, S, l, (const double *)xa, b, (const double *)nullptr, r, sc);
    blk_launch(s, L, w2, r, xa, nullptr, c, xc, 2, sc);                             // xc = xa + c xa + w2 D^-1 r
    mark(0);
    op_launch<kResid>(s, S, l, (const double *)xc, b, (const double *)nullptr, r, sc);
    mark(1);
    restrict_and_recurse(r);
    prolong_add(xc);
    mark(2);
    op_launch<kResid>(s, S, l, (const double *)xc, b, (const double *)nullptr, r, sc);
    mark(3);
    blk_launch(s, L, t, r, xc, nullptr, 0.0, xa, 1, sc);                            // xa = xc + D^-1 r / theta
    op_launch<kResid>(s, S, l, (const double *)xa, b, (const double *)nullptr, r, sc);
    blk_launch(s, L, w2, r, xa, xc, c, x, 2, sc);                                   // x = xa + c (xa - xc) + ...
  } else {
    blk_launch(s, L, L.omega, b, nullptr, nullptr, 0.0, xa, 0, sc);                 // xa = omega D^-1 b
    mark(0);
    op_launch<kResid>(s, S, l, (const double *)xa, b, (const double *)nullptr, r, sc);
    mark(1);
    restrict_and_recurse(r);
    prolong_add(xa);
    mark(2);
    op_launch<kResid>(s, S, l, (const double *)xa, b, (const double *)nullptr, r, sc);
    mark(3);
    blk_launch(s, L, L.omega, r, xa, nullptr, 0.0, x, 1, sc);                       // x = xa + omega D^-1 r
  }
  if (tm) {
    S->timing = false;
    S->timed = true;
  }
}

// x = V(b) on level l, values and vectors in T; the level's output is Ty
// (FP64 on level 0 of an FP32 cycle, so u needs no conversion pass).
template <class T, class Ty>
static void cycle(vem_handle *h, AmgState *S, int l, const T *b, Ty *x, const double *sc) {
  cudaStream_t s = h->stream;
  AmgLevel &L = S->lv[l];
  if constexpr (sizeof(T) == sizeof(double) && sizeof(Ty) == sizeof(double)) {
    if (S->block) {
      bcycle(h, S, l, (const double *)b, (double *)x, sc);
      return;
    }
  }
  const T *wd = wdv<T>(L);
  if (l == S->nlev - 1) {
    if (S->csweeps == 0) {
      const int g = (int)std::min<int64_t>((L.n + 7) / 8, 1024);
      T *xo = L.vx<T>(1);
      const T *inv;
      if constexpr (sizeof(T) == sizeof(double)) inv = S->cinv;
      else inv = S->cinv32;
      count_launch();
      if constexpr (sizeof(T) == sizeof(Ty)) {
        launch_pdl(k_vc_dense<T>, g, 256, 0, s, (int)L.n, inv, b, x, sc);
      } else {
        launch_pdl(k_vc_dense<T>, g, 256, 0, s, (int)L.n, inv, b, xo, sc);
        count_launch();
        launch_pdl(k_vc_convert<T, Ty>, rows_grid(L.n), 256, 0, s, L.n, (const T *)xo, x, sc);
      }
      return;
    }
    // damped-Jacobi sweeps from zero: x1 = wd b, then x_{k+1} = post(x_k)
    T *xa = L.vx<T>(0), *xb = L.vx<T>(3);
    count_launch();
    launch_pdl(k_vc_pre<T>, rows_grid(L.n), 256, 0, s, L.n, b, wd, xa, sc);
    for (int k = 1; k < S->csweeps; ++k) {
      if (k == S->csweeps - 1) op_launch<kPost>(s, S, l, (const T *)xa, b, wd, x, sc);
      else op_launch<kPost>(s, S, l, (const T *)xa, b, wd, xb, sc);
      std::swap(xa, xb);
    }
    return;
  }
  AmgLevel &C = S->lv[l + 1];
  T *xa = L.vx<T>(0), *r = L.vx<T>(3);
  T *cb = C.vx<T>(2), *cx = C.vx<T>(1);
  const bool cheb = S->smoother == kSmoothChebyshev;
  // events around the level-0 residual and post-smoothing launches of a timed cycle
  const bool tm = l == 0 && S->timing;
  auto mark = [&](int k) {
    if (tm) cudaEventRecord(S->tev[k], s);
  };
  const T cc = (T)L.cheb_c;
  const T *wdc = cheb ? wdcv<T>(L) : nullptr;
  count_launch();
  launch_pdl(k_vc_pre<T>, rows_grid(L.n), 256, 0, s, L.n, b, wd, xa, sc);        // xa = w D^-1 b
  if (cheb) {
    // second Chebyshev step from x0 = 0: xc = xa + c xa + wdc (b - A xa)
    T *xc = L.vx<T>(4);
    op_launch<kCheb>(s, S, l, (const T *)xa, b, wdc, xc, sc, (const T *)nullptr, cc);
    mark(0);
    op_launch<kResid>(s, S, l, (const T *)xc, b, (const T *)nullptr, r, sc);    // r = b - A xc
    mark(1);
    if (L.Rs.m.rows) sell_launch<kApply>(s, L.Rs.m, vals<T>(L.Rs), (const T *)r, (const T *)nullptr,
                                         (const T *)nullptr, cb, sc);
    else csr_launch<kApply>(s, L.R, (const T *)r, (const T *)nullptr, (const T *)nullptr, cb, sc);
    cycle<T, T>(h, S, l + 1, (const T *)cb, cx, sc);
    if (L.Ps.m.rows) sell_launch<kAdd>(s, L.Ps.m, vals<T>(L.Ps), (const T *)cx, (const T *)nullptr,
                                       (const T *)nullptr, xc, sc);              // xc += P x_c
    else csr_launch<kAdd>(s, L.P, (const T *)cx, (const T *)nullptr, (const T *)nullptr, xc, sc);
    mark(2);
    op_launch<kPost>(s, S, l, (const T *)xc, b, wd, xa, sc);                     // xa = xc + wd (b - A xc)
    mark(3);
    op_launch<kCheb>(s, S, l, (const T *)xa, b, wdc, x, sc, (const T *)xc, cc);  // x = xa + c (xa - xc) + ...
    if (tm) {
      S->timing = false;
      S->timed = true;
    }
    return;
  }
  mark(0);
  op_launch<kResid>(s, S, l, (const T *)xa, b, (const T *)nullptr, r, sc);      // r = b - A xa
  mark(1);
  if (L.Rs.m.rows) sell_launch<kApply>(s, L.Rs.m, vals<T>(L.Rs), (const T *)r, (const T *)nullptr,
                                       (const T *)nullptr, cb, sc);
  else csr_launch<kApply>(s, L.R, (const T *)r, (const T *)nullptr, (const T *)nullptr, cb, sc);
  cycle<T, T>(h, S, l + 1, (const T *)cb, cx, sc);
  if (L.Ps.m.rows) sell_launch<kAdd>(s, L.Ps.m, vals<T>(L.Ps), (const T *)cx, (const T *)nullptr,
                                     (const T *)nullptr, xa, sc);                // xa += P x_c
  else csr_launch<kAdd>(s, L.P, (const T *)cx, (const T *)nullptr, (const T *)nullptr, xa, sc);
  mark(2);
  op_launch<kPost>(s, S, l, (const T *)xa, b, wd, x, sc);                        // x = xa + wd (b - A xa)
  mark(3);
  if (tm) {
    S->timing = false;
    S->timed = true;
  }
}

// The coarsest level of an FP64 cycle: the dense inverse, or damped-Jacobi
// sweeps from zero.
static void coarsest_solve(vem_handle *h, AmgState *S, int l, const double *b, double *x, const double *sc) {
  cudaStream_t s = h->stream;
  AmgLevel &L = S->lv[l];
  if (S->csweeps == 0) {
    const int g = (int)std::min<int64_t>((L.n + 7) / 8, 1024);
    count_launch();
    launch_pdl(k_vc_dense<double>, g, 256, 0, s, (int)L.n, (const double *)S->cinv, b, x, sc);
    return;
  }
  double *xa = L.vx<double>(0), *xb = L.vx<double>(3);
  count_launch();
  launch_pdl(k_vc_pre<double>, rows_grid(L.n), 256, 0, s, L.n, b, (const double *)L.wd, xa, sc);
  for (int k = 1; k < S->csweeps; ++k) {
    if (k == S->csweeps - 1) op_launch<kPost>(s, S, l, (const double *)xa, b, (const double *)L.wd, x, sc);
    else op_launch<kPost>(s, S, l, (const double *)xa, b, (const double *)L.wd, xb, sc);
    std::swap(xa, xb);
  }
}

// ------------------------------------------------ condensed Block-Reg -----
// The face system S_f = A_ff - A_fi A_ii^-1 A_if of A_reg (interior DOFs
// eliminated cell by cell, exactly) and the point-block hierarchy of S_f
// with nfd x nfd face blocks and the near-null space Bf (nfr x m).
vem_status amg_setup_condensed(vem_handle *h, AmgState *&slot, const SellMat &Areg, int64_t nfr, int nid, int nfd,
                               const double *Bf, int m, int smoother) {
  if (!slot) slot = new AmgState();
  AmgState *S = slot;
  S->valid = false;
  S->condensed = false;
  if (nid < 1 || nid > kMaxInt || nfd < 1 || nfd > kMaxBs || (Areg.rows - nfr) % nid)
    return fail(h, VEM_ERR_UNSUPPORTED, "condensed Block-Reg cycle: %d interior DOFs per cell", nid);
  cudaStream_t s = h->stream;
  for (cudaEvent_t &e : S->sev)
    if (!e) VEM_CUDA(h, cudaEventCreate(&e));
  VEM_CUDA(h, cudaEventRecord(S->sev[0], s));
  if (!S->ctr) VEM_TRY(dalloc_n(h, &S->ctr, kMaxRounds + 4));
  const int64_t nu = Areg.rows, nint = nu - nfr, nc = nint / nid;
  const DMat A = dview(Areg);
  // split the rows: face rows into A_ff | A_fi, interior rows into A_if | A_ii
  VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)nu + 1));
  VEM_TRY(grow(h, S->scn, S->c_scn, (size_t)nu + 1));
  count_launch();
  k_split<false><<<rows_grid(nu), 256, 0, s>>>(A, 0, nu, nfr, S->cnt, S->scn, nullptr, nullptr, nullptr, nullptr,
                                               nullptr, nullptr);
  // face rows: counts at cnt[0..nfr), scn[0..nfr); interior rows after them
  VEM_TRY(csr_layout(h, S->cAff, nfr, nfr, S->cnt));
  VEM_TRY(csr_layout(h, S->cAfi, nfr, nint, S->scn));
  VEM_TRY(csr_layout(h, S->cAif, nint, nfr, S->cnt + nfr));
  VEM_TRY(csr_layout(h, S->cAii, nint, nint, S->scn + nfr));
  count_launch();
  k_split<true><<<rows_grid(nfr), 256, 0, s>>>(A, 0, nfr, nfr, nullptr, nullptr, S->cAff.rp, S->cAfi.rp,
                                               S->cAff.col, S->cAff.val, S->cAfi.col, S->cAfi.val);
  count_launch();
  k_split<true><<<rows_grid(nint), 256, 0, s>>>(A, nfr, nint, nfr, nullptr, nullptr, S->cAif.rp, S->cAii.rp,
                                                S->cAif.col, S->cAif.val, S->cAii.col, S->cAii.val);
  VEM_TRY(sort_rows(h, S, nfr, S->cAff.rp, S->cAff.col, S->cAff.val));
  VEM_TRY(sort_rows(h, S, nfr, S->cAfi.rp, S->cAfi.col, S->cAfi.val));
  VEM_TRY(sort_rows(h, S, nint, S->cAif.rp, S->cAif.col, S->cAif.val));
  // A_ii^-1 blockwise, then S_f = A_ff - A_fi (A_ii^-1 A_if)
  VEM_TRY(grow(h, S->aii_inv, S->c_aii, (size_t)nint * nid));
  VEM_TRY(grow(h, S->cvec, S->c_cvec, (size_t)nint + nfr));
  double *lscr = nullptr;
  VEM_TRY(dalloc_n(h, &lscr, (size_t)nint * nid));
  count_launch();
  k_blk_diag<kMaxInt><<<rows_grid(nc), 256, 0, s>>>(nc, nid, dview(S->cAii), S->aii_inv, lscr, h->d_err);
  VEM_TRY(check_device_errors(h, "condensed Block-Reg: interior blocks of A_reg"));
  VEM_TRY(csr_fixed(h, S->bLm, nint, nint, nint * nid));
  count_launch();
  k_blkdiag_rows<<<rows_grid(nint), 256, 0, s>>>(nint, nid, S->aii_inv, 0, S->bLm.rp, S->bLm.col, S->bLm.val);
  VEM_TRY(product(h, S, dview(S->bLm), S->cAif, S->bY, false));
  VEM_TRY(product(h, S, dview(S->cAfi), S->bY, S->bZ, false));
  count_launch();
  k_sub_rows<false><<<rows_grid(nfr), 256, 0, s>>>(nfr, S->cAff.rp, S->cAff.col, S->cAff.val, S->bZ.rp, S->bZ.col,
                                                   S->bZ.val, 1.0, S->cnt, nullptr, nullptr, nullptr);
  VEM_TRY(csr_layout(h, S->cSf, nfr, nfr, S->cnt));
  count_launch();
  k_sub_rows<true><<<rows_grid(nfr), 256, 0, s>>>(nfr, S->cAff.rp, S->cAff.col, S->cAff.val, S->bZ.rp, S->bZ.col,
                                                  S->bZ.val, 1.0, nullptr, S->cSf.rp, S->cSf.col, S->cSf.val);
  VEM_TRY(csr_to_sell(h, S, S->cSf, S->cSell));
  dfree(h, lscr);
  VEM_TRY(check_device_errors(h, "condensed Block-Reg: face system"));
  // the point-block hierarchy of S_f; the setup time covers the condensation too
  VEM_TRY(amg_setup_block(h, slot, S->cSell.m, nfd, Bf, m, false, smoother));
  VEM_CUDA(h, cudaEventRecord(S->sev[1], s));
  VEM_CUDA(h, cudaEventSynchronize(S->sev[1]));
  float ms = 0.f;
  VEM_CUDA(h, cudaEventElapsedTime(&ms, S->sev[0], S->sev[1]));
  S->t_setup_ms = ms;
  S->condensed = true;
  S->nfr = nfr;
  S->nint = nint;
  S->nid = nid;
  return VEM_OK;
}

// z = (condensed cycle) r for vectors of n_u = nfr + nint entries.
static void condensed_apply(vem_handle *h, AmgState *S, const double *r, double *z) {
  cudaStream_t s = h->stream;
  const int64_t nfr = S->nfr, nint = S->nint;
  double *t = S->cvec, *rf = S->cvec + nint;
  const double *ri = r + nfr;
  double *zi = z + nfr;
  count_launch();
  k_blk_apply<<<rows_grid(nint), 256, 0, s>>>(nint, S->nid, S->aii_inv, 1.0, ri, nullptr, nullptr, 0.0, t, 0,
                                             nullptr);                                    // t = A_ii^-1 r_i
  csr_launch<kResid>(s, S->cAfi, (const double *)t, r, (const double *)nullptr, rf, nullptr);  // r_f - A_fi t
  bcycle(h, S, 0, rf, z, nullptr);                                                         // z_f = V(S_f) rf
  csr_launch<kResid>(s, S->cAif, (const double *)z, ri, (const double *)nullptr, t, nullptr);  // r_i - A_if z_f
  count_launch();
  k_blk_apply<<<rows_grid(nint), 256, 0, s>>>(nint, S->nid, S->aii_inv, 1.0, t, nullptr, nullptr, 0.0, zi, 0,
                                             nullptr);                                    // z_i = A_ii^-1 t
}

bool amg_is_condensed(const AmgState *S) { return S && S->condensed; }

vem_status flux_modes_k1(vem_handle *h, int64_t nf, const double *f_norm, double *B) {
  count_launch();
  k_flux_modes_k1<<<rows_grid(nf), 256, 0, h->stream>>>(nf, f_norm, B);
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

void amg_vcycle(vem_handle *h, AmgState *S, const double *b, double *x, const double *sc) {
  if (S->condensed) {
    condensed_apply(h, S, b, x);
    return;
  }
  if (!S->fp32) {
    cycle<double, double>(h, S, 0, b, x, sc);
    return;
  }
  AmgLevel &L = S->lv[0];
  float *b32 = L.vx<float>(2);
  count_launch();
  k_vc_convert<double, float><<<rows_grid(L.n), 256, 0, h->stream>>>(L.n, b, b32, sc);
  cycle<float, double>(h, S, 0, (const float *)b32, x, sc);
}

// ---- inspection (host copies for the tests) ----
static vem_status csr_to_host(vem_handle *h, const CsrBuf &C, int64_t *rp, int32_t *col, double *val) {
  if (rp) VEM_CUDA(h, cudaMemcpy(rp, C.rp, sizeof(int64_t) * (C.rows + 1), cudaMemcpyDeviceToHost));
  if (col) VEM_CUDA(h, cudaMemcpy(col, C.col, sizeof(int32_t) * C.nnz, cudaMemcpyDeviceToHost));
  if (val) VEM_CUDA(h, cudaMemcpy(val, C.val, sizeof(double) * C.nnz, cudaMemcpyDeviceToHost));
  return VEM_OK;
}

vem_status amg_level_info(vem_handle *h, const AmgState *S, int *nlev, int64_t *rows, int64_t *nnz,
                          int64_t *nnz_p) {
  if (!amg_valid(S)) return fail(h, VEM_ERR_BAD_INPUT, "no AMG hierarchy: call vem_amg_setup first");
  *nlev = S->nlev;
  for (int l = 0; l < S->nlev; ++l) {
    if (rows) rows[l] = S->lv[l].n;
    if (nnz) nnz[l] = l == 0 ? S->S0.nnz : S->lv[l].A.nnz;
    if (nnz_p) nnz_p[l] = l + 1 < S->nlev ? S->lv[l].P.nnz : 0;
  }
  return VEM_OK;
}

vem_status amg_level_copy(vem_handle *h, AmgState *S, int l, int64_t *rp, int32_t *col, double *val,
                          int32_t *agg, int64_t *prp, int32_t *pcol, double *pval) {
  if (!amg_valid(S)) return fail(h, VEM_ERR_BAD_INPUT, "no AMG hierarchy: call vem_amg_setup first");
  if (l < 0 || l >= S->nlev) return fail(h, VEM_ERR_BAD_INPUT, "AMG level %d of %d", l, S->nlev);
  AmgLevel &L = S->lv[l];
  VEM_CUDA(h, cudaStreamSynchronize(h->stream));
  if (rp || col || val) {
    if (l == 0) VEM_TRY(sell_to_host_csr(h, S->S0, rp, col, val));
    else VEM_TRY(csr_to_host(h, L.A, rp, col, val));
  }
  const bool coarse = l + 1 < S->nlev;
  if (agg && coarse)   // one aggregate per point block
    VEM_CUDA(h, cudaMemcpy(agg, L.agg, sizeof(int32_t) * (S->block ? L.n / L.bs : L.n), cudaMemcpyDeviceToHost));
  if ((prp || pcol || pval) && coarse) VEM_TRY(csr_to_host(h, L.P, prp, pcol, pval));
  return VEM_OK;
}

double amg_omega(const AmgState *S, int l) { return amg_valid(S) && l < S->nlev ? S->lv[l].omega : 0.0; }

}  // namespace vem
