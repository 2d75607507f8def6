// Smoothed-aggregation algebraic multigrid for the Schur block S: the setup
// (strength of connection, distance-2 independent set, aggregates, smoothed
// prolongator, Galerkin coarse operators) and the symmetric V(1,1) cycle that
// preconditions the inner CG.
//
// The paper solves S exactly inside Block-Schur and uses a smoothed-
// aggregation AMG (PETSc GAMG) for the velocity block of Block-Reg (Sec. 5);
// this AMG is the library's inner solver option for S.  Method: Vanek,
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
// The products P, A P and P^T (A P) are formed row by row, one thread per
// row holding the row's distinct columns in a small sorted list and summing
// contributions in a fixed order, so the hierarchy is bitwise reproducible.
#include <algorithm>
#include <cmath>

#include "handle.cuh"

namespace vem {

constexpr int kMaxLevels = 12;
constexpr int kCoarseMax = 64;
constexpr int kDenseMax = 512;
constexpr int kCoarseSweeps = 4;
constexpr double kTheta0 = 0.08;
constexpr int kCapP = 128;     // distinct columns of a row of P
constexpr int kCapAP = 256;    // of a row of A P
constexpr int kCapRAP = 512;   // of a row of P^T A P
constexpr int kMaxRounds = 200;

constexpr uint64_t kStIn = 2ull << 62, kStUnd = 1ull << 62;

// A SELL matrix with the capacities of its buffers (grown, never shrunk).
struct SellBuf {
  SellMat m;
  size_t c_off = 0, c_len = 0, c_st = 0;
};

// A CSR matrix in device memory with capacities.
struct CsrBuf {
  int64_t rows = 0, nnz = 0;
  int64_t *rp = nullptr;
  int32_t *col = nullptr;
  double *val = nullptr;
  size_t c_rp = 0, c_nz = 0;
};

struct AmgLevel {
  SellBuf A, P, R;          // level 0's A is the handle's S (a view, not owned)
  double *dinv = nullptr;
  int32_t *agg = nullptr;
  double *vec = nullptr;    // x, x2, b, r: four vectors of n
  size_t c_dinv = 0, c_agg = 0, c_vec = 0;
  double omega = 0.0;
  int64_t n = 0, nc = 0;
  double *x() const { return vec; }
  double *x2() const { return vec + n; }
  double *b() const { return vec + 2 * n; }
  double *r() const { return vec + 3 * n; }
};

struct AmgState {
  AmgLevel lv[kMaxLevels];
  int nlev = 0;
  bool valid = false;
  double *cinv = nullptr;   // dense inverse of the coarsest level
  size_t c_cinv = 0;
  int csweeps = 0;
  // setup scratch
  uint8_t *flag = nullptr;  size_t c_flag = 0;
  int32_t *nstr = nullptr;  size_t c_nstr = 0;
  uint64_t *tup = nullptr;  size_t c_tup = 0;     // tuples and t1: 2 n
  int64_t *cnt = nullptr;   size_t c_cnt = 0;     // counts (n)
  int64_t *scn = nullptr;   size_t c_scn = 0;     // scans (n + 1)
  int32_t *agg1 = nullptr;  size_t c_agg1 = 0;
  double *dg = nullptr;     size_t c_dg = 0;      // diagonal
  unsigned long long *ctr = nullptr;              // [kMaxRounds + 4] counters / maxima
  CsrBuf Pc, Rc, APc, Ac;
  int64_t *cur = nullptr;   size_t c_cur = 0;     // transpose cursors
  double t_setup_ms = 0.0;
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

static AmgState *state(vem_handle *h) {
  if (!h->amg) h->amg = new AmgState();
  return h->amg;
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
__global__ void k_amg_diag(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                           const int32_t *__restrict__ col, const double *__restrict__ val, double *dg,
                           double *dinv, int *err) {
  ROWS_LOOP(i, n) {
    const int64_t base = off[i >> 5] + (i & 31);
    const int L = len[i];
    double d = 0.0;
    for (int k = 0; k < L; ++k)
      if (col[base + 32 * k] == (int32_t)i) d = val[base + 32 * k];
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
__global__ void k_amg_strength(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                               const int32_t *__restrict__ col, const double *__restrict__ val,
                               const double *__restrict__ dg, double theta, uint8_t *flag, int32_t *nstr,
                               unsigned long long *mx) {
  double rho = 0.0, rhof = 0.0;
  ROWS_LOOP(i, n) {
    const int64_t base = off[i >> 5] + (i & 31);
    const int L = len[i];
    const double di = dg[i];
    double sa = 0.0, sf = 0.0;
    int ns = 0;
    for (int k = 0; k < L; ++k) {
      const int64_t p = base + 32 * k;
      const int32_t j = col[p];
      const double a = fabs(val[p]);
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

__global__ void k_mis_max1(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                           const int32_t *__restrict__ col, const uint8_t *__restrict__ flag,
                           const uint64_t *__restrict__ tup, uint64_t *t1) {
  ROWS_LOOP(i, n) {
    const int64_t base = off[i >> 5] + (i & 31);
    const int L = len[i];
    uint64_t m = tup[i];
    for (int k = 0; k < L; ++k) {
      const int64_t p = base + 32 * k;
      if (flag[p]) m = max(m, tup[col[p]]);
    }
    t1[i] = m;
  }
}

__global__ void k_mis_max2(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                           const int32_t *__restrict__ col, const uint8_t *__restrict__ flag,
                           const uint64_t *__restrict__ t1, uint64_t *tup, unsigned long long *und) {
  unsigned long long c = 0;
  ROWS_LOOP(i, n) {
    const uint64_t own = tup[i];
    if ((own >> 62) != 1) continue;
    const int64_t base = off[i >> 5] + (i & 31);
    const int L = len[i];
    uint64_t m = t1[i];
    for (int k = 0; k < L; ++k) {
      const int64_t p = base + 32 * k;
      if (flag[p]) m = max(m, t1[col[p]]);
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

__global__ void k_agg_pass1(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                            const int32_t *__restrict__ col, const uint8_t *__restrict__ flag,
                            const uint64_t *__restrict__ tup, const int32_t *__restrict__ nstr,
                            const int64_t *__restrict__ rid, int32_t *agg1) {
  ROWS_LOOP(i, n) {
    int32_t a = -1;
    if (nstr[i] > 0) {
      if ((tup[i] >> 62) == 2) {
        a = (int32_t)rid[i];
      } else {
        const int64_t base = off[i >> 5] + (i & 31);
        const int L = len[i];
        for (int k = 0; k < L; ++k) {
          const int64_t p = base + 32 * k;
          if (!flag[p]) continue;
          const int32_t j = col[p];
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

__global__ void k_agg_pass2(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                            const int32_t *__restrict__ col, const uint8_t *__restrict__ flag,
                            const int32_t *__restrict__ nstr, const int32_t *__restrict__ agg1, int32_t *agg,
                            int64_t *freecnt) {
  ROWS_LOOP(i, n) {
    int32_t a = agg1[i];
    if (a < 0 && nstr[i] > 0) {
      const int64_t base = off[i >> 5] + (i & 31);
      const int L = len[i];
      for (int k = 0; k < L; ++k) {
        const int64_t p = base + 32 * k;
        if (!flag[p]) continue;
        const int32_t b = agg1[col[p]];
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
__global__ void k_p_rows(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                         const int32_t *__restrict__ col, const double *__restrict__ val,
                         const uint8_t *__restrict__ flag, const double *__restrict__ dinv,
                         const int32_t *__restrict__ agg, double omega_f, int64_t *cnt,
                         const int64_t *__restrict__ rp, int32_t *pcol, double *pval, int *err) {
  ROWS_LOOP(i, n) {
    const int32_t ai = agg[i];
    RowMap<kCapP> m;
    bool ok = true;
    if (ai >= 0) {
      const int64_t base = off[i >> 5] + (i & 31);
      const int L = len[i];
      for (int k = 0; k < L && ok; ++k) {
        const int64_t p = base + 32 * k;
        const int32_t j = col[p];
        if (j == (int32_t)i) {
          ok = m.add(ai, val[p]);
        } else if (flag[p]) {
          const int32_t aj = agg[j];
          if (aj >= 0) ok = m.add(aj, val[p]);
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

// Insertion sort of every row by column (columns within a row are distinct).
__global__ void k_sort_rows(int64_t n, const int64_t *__restrict__ rp, int32_t *col, double *val) {
  ROWS_LOOP(i, n) {
    const int64_t lo = rp[i], hi = rp[i + 1];
    for (int64_t a = lo + 1; a < hi; ++a) {
      const int32_t c = col[a];
      const double v = val[a];
      int64_t b = a - 1;
      while (b >= lo && col[b] > c) {
        col[b + 1] = col[b];
        val[b + 1] = val[b];
        --b;
      }
      col[b + 1] = c;
      val[b + 1] = v;
    }
  }
}

// ---------------------------------------------------------- products ------
// Row i of A P (A in SELL, P in CSR).
template <bool kFill>
__global__ void k_ap_rows(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                          const int32_t *__restrict__ col, const double *__restrict__ val,
                          const int64_t *__restrict__ prp, const int32_t *__restrict__ pcol,
                          const double *__restrict__ pval, int64_t *cnt, const int64_t *__restrict__ rp,
                          int32_t *ocol, double *oval, int *err) {
  ROWS_LOOP(i, n) {
    RowMap<kCapAP> m;
    bool ok = true;
    const int64_t base = off[i >> 5] + (i & 31);
    const int L = len[i];
    for (int k = 0; k < L && ok; ++k) {
      const int64_t p = base + 32 * k;
      const int32_t j = col[p];
      const double a = val[p];
      for (int64_t q = prp[j]; q < prp[j + 1] && ok; ++q) ok = m.add(pcol[q], a * pval[q]);
    }
    if (!ok) atomicOr(err, DEVERR_AMG_ROW);
    if (!kFill) {
      cnt[i] = ok ? m.n : 0;
    } else if (ok) {
      const int64_t o = rp[i];
      for (int t = 0; t < m.n; ++t) {
        ocol[o + t] = m.key[t];
        oval[o + t] = m.val[t];
      }
    }
  }
}

// Row I of R (A P), R = P^T in CSR with rows sorted by fine index.
template <bool kFill>
__global__ void k_rap_rows(int64_t nc, const int64_t *__restrict__ rrp, const int32_t *__restrict__ rcol,
                           const double *__restrict__ rval, const int64_t *__restrict__ arp,
                           const int32_t *__restrict__ acol, const double *__restrict__ aval, int64_t *cnt,
                           const int64_t *__restrict__ rp, int32_t *ocol, double *oval, int *err) {
  ROWS_LOOP(I, nc) {
    RowMap<kCapRAP> m;
    bool ok = true;
    for (int64_t p = rrp[I]; p < rrp[I + 1] && ok; ++p) {
      const int32_t i = rcol[p];
      const double r = rval[p];
      for (int64_t q = arp[i]; q < arp[i + 1] && ok; ++q) ok = m.add(acol[q], r * aval[q]);
    }
    if (!ok) atomicOr(err, DEVERR_AMG_ROW);
    if (!kFill) {
      cnt[I] = ok ? m.n : 0;
    } else if (ok) {
      const int64_t o = rp[I];
      for (int t = 0; t < m.n; ++t) {
        ocol[o + t] = m.key[t];
        oval[o + t] = m.val[t];
      }
    }
  }
}

// ------------------------------------------------------ CSR <-> SELL ------
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

__global__ void k_dense_from_sell(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ len,
                                  const int32_t *__restrict__ col, const double *__restrict__ val, double *M) {
  ROWS_LOOP(i, n) {
    const int64_t base = off[i >> 5] + (i & 31);
    for (int64_t c = 0; c < n; ++c) M[i * n + c] = 0.0;
    for (int k = 0; k < len[i]; ++k) M[i * n + col[base + 32 * k]] += val[base + 32 * k];
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
  __shared__ int f;
  if (threadIdx.x == 0) f = (sc && sc[0] != 0.0) ? 1 : 0;
  __syncthreads();
  const bool r = f != 0;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256) k_vc_pre(int64_t n, const double *__restrict__ b,
                                                const double *__restrict__ dinv, double omega, double *x,
                                                const double *sc) {
  if (cycle_done(sc)) return;
  ROWS_LOOP(i, n) x[i] = omega * (dinv[i] * b[i]);
}

// mode 0: y = b - A x;  mode 1: y = x + omega dinv (b - A x);  mode 2: y += A x
template <int kMode>
__global__ void __launch_bounds__(256) k_vc_sell(int64_t rows, int64_t nslices, const int64_t *__restrict__ off,
                                                 const int32_t *__restrict__ col, const double *__restrict__ val,
                                                 const double *__restrict__ x, const double *__restrict__ b,
                                                 const double *__restrict__ dinv, double omega, double *y,
                                                 const double *sc) {
  if (cycle_done(sc)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = warp; s < nslices; s += nwarps) {
    const int64_t r = 32 * s + lane;
    double bi = 0.0, xi = 0.0, di = 0.0, yi = 0.0;
    if (r < rows) {
      if (kMode != 2) bi = b[r];
      if (kMode == 1) {
        xi = x[r];
        di = dinv[r];
      }
      if (kMode == 2) yi = y[r];
    }
    const double t = sell_row_dot<double>(off, col, val, x, s, lane);
    if (r < rows) {
      if (kMode == 0) y[r] = bi - t;
      else if (kMode == 1) y[r] = xi + omega * (di * (bi - t));
      else y[r] = yi + t;
    }
  }
}

// y = R x for the restriction (plain SELL SpMV with the cycle's early exit)
__global__ void __launch_bounds__(256) k_vc_spmv(int64_t rows, int64_t nslices, const int64_t *__restrict__ off,
                                                 const int32_t *__restrict__ col, const double *__restrict__ val,
                                                 const double *__restrict__ x, double *y, const double *sc) {
  if (cycle_done(sc)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = warp; s < nslices; s += nwarps) {
    const double t = sell_row_dot<double>(off, col, val, x, s, lane);
    const int64_t r = 32 * s + lane;
    if (r < rows) y[r] = t;
  }
}

// x = Minv b with the dense coarsest inverse: one warp per row.
__global__ void __launch_bounds__(256) k_vc_dense(int n, const double *__restrict__ Minv,
                                                  const double *__restrict__ b, double *x, const double *sc) {
  if (cycle_done(sc)) return;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < n; r += nwarps) {
    double acc = 0.0;
    for (int c = lane; c < n; c += 32) acc += Minv[(int64_t)r * n + c] * b[c];
    acc = warp_sum(acc);
    if (lane == 0) x[r] = acc;
  }
}

static int rows_grid(int64_t n) { return grid_for(n, 256, 8); }

static int sell_grid(const SellMat &A) {
  int64_t b = (A.nslices + 7) / 8;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// ------------------------------------------------------------ host --------
// Row counts cnt[rows] -> CSR with that pattern (row pointers from the scan).
static vem_status csr_layout(vem_handle *h, CsrBuf &C, int64_t rows, const int64_t *cnt) {
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
  C.nnz = nnz;
  return VEM_OK;
}

// CSR -> SELL-32 into a growable SELL buffer.
static vem_status csr_to_sell(vem_handle *h, AmgState *S, const CsrBuf &C, SellBuf &B) {
  cudaStream_t s = h->stream;
  const int64_t rows = C.rows, ns = (rows + 31) / 32;
  VEM_TRY(grow(h, B.m.off, B.c_off, (size_t)ns + 1));
  VEM_TRY(grow(h, B.m.len, B.c_len, (size_t)ns * 32));
  VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)(rows > ns ? rows : ns) + 1));
  count_launch();
  k_rp_counts<<<rows_grid(rows), 256, 0, s>>>(rows, C.rp, S->cnt);
  VEM_TRY(grow(h, S->cur, S->c_cur, (size_t)ns + 1));   // per-slice sizes
  count_launch();
  k_sell_slices<<<rows_grid(ns), 256, 0, s>>>(rows, ns, S->cnt, S->cur, B.m.len);
  int64_t stored = 0;
  VEM_TRY(scan_counts(h, ns, S->cur, B.m.off, &stored));
  if (!B.m.col || (size_t)stored > B.c_st) {
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

// One level: strength, MIS-2, aggregates, P, R and the coarse operator.
// Returns nc = 0 when the level is not coarsened.
static vem_status coarsen(vem_handle *h, AmgState *S, int l, double theta, int64_t *nc_out) {
  cudaStream_t s = h->stream;
  AmgLevel &L = S->lv[l];
  const SellMat &A = L.A.m;
  const int64_t n = A.rows;
  *nc_out = 0;
  VEM_TRY(grow(h, S->flag, S->c_flag, (size_t)A.stored));
  VEM_TRY(grow(h, S->nstr, S->c_nstr, (size_t)n));
  VEM_TRY(grow(h, S->tup, S->c_tup, 2 * (size_t)n));
  VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)n + 1));
  VEM_TRY(grow(h, S->scn, S->c_scn, (size_t)n + 1));
  VEM_TRY(grow(h, S->agg1, S->c_agg1, (size_t)n));
  VEM_TRY(grow(h, S->dg, S->c_dg, (size_t)n));
  VEM_TRY(grow(h, L.agg, L.c_agg, (size_t)n));
  const int g = rows_grid(n);

  // strength and the Gershgorin maxima (diagonal and dinv already computed)
  VEM_CUDA(h, cudaMemsetAsync(S->ctr, 0, sizeof(unsigned long long) * (kMaxRounds + 4), s));
  count_launch();
  k_amg_strength<<<g, 256, 0, s>>>(n, A.off, A.len, A.col, A.val, S->dg, theta, S->flag, S->nstr, S->ctr);
  // MIS-2 rounds; the host reads the undecided count every second round
  count_launch();
  k_mis_init<<<g, 256, 0, s>>>(n, S->tup);
  uint64_t *t1 = S->tup + n;
  int round = 0;
  unsigned long long und = 1;
  while (und != 0) {
    if (round + 2 > kMaxRounds) return fail(h, VEM_ERR_CUDA, "AMG aggregation did not finish in %d rounds", kMaxRounds);
    for (int k = 0; k < 2; ++k, ++round) {
      count_launch();
      k_mis_max1<<<g, 256, 0, s>>>(n, A.off, A.len, A.col, S->flag, S->tup, t1);
      count_launch();
      k_mis_max2<<<g, 256, 0, s>>>(n, A.off, A.len, A.col, S->flag, t1, S->tup, S->ctr + 2 + round);
    }
    VEM_CUDA(h, cudaGetLastError());
    VEM_CUDA(h, cudaMemcpyAsync(&und, S->ctr + 2 + round - 1, sizeof(und), cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
  }
  unsigned long long mx[2] = {0, 0};
  VEM_CUDA(h, cudaMemcpyAsync(mx, S->ctr, sizeof(mx), cudaMemcpyDeviceToHost, s));
  // aggregates
  count_launch();
  k_agg_root<<<g, 256, 0, s>>>(n, S->tup, S->nstr, S->cnt);
  int64_t nroot = 0;
  VEM_TRY(scan_counts(h, n, S->cnt, S->scn, &nroot));
  count_launch();
  k_agg_pass1<<<g, 256, 0, s>>>(n, A.off, A.len, A.col, S->flag, S->tup, S->nstr, S->scn, S->agg1);
  count_launch();
  k_agg_pass2<<<g, 256, 0, s>>>(n, A.off, A.len, A.col, S->flag, S->nstr, S->agg1, L.agg, S->cnt);
  int64_t nfree = 0;
  VEM_TRY(scan_counts(h, n, S->cnt, S->scn, &nfree));
  count_launch();
  k_agg_pass3<<<g, 256, 0, s>>>(n, nroot, S->nstr, S->scn, L.agg);
  VEM_CUDA(h, cudaGetLastError());
  const int64_t nc = nroot + nfree;
  if (nc == 0 || 5 * nc > 4 * n) return VEM_OK;
  const double rho = bits_to_double(mx[0]), rhof = bits_to_double(mx[1]);
  L.omega = 4.0 / (3.0 * rho);
  const double omega_f = 4.0 / (3.0 * rhof);

  // P (CSR, then SELL)
  count_launch();
  k_p_rows<false><<<g, 256, 0, s>>>(n, A.off, A.len, A.col, A.val, S->flag, L.dinv, L.agg, omega_f, S->cnt,
                                    nullptr, nullptr, nullptr, h->d_err);
  VEM_TRY(csr_layout(h, S->Pc, n, S->cnt));
  count_launch();
  k_p_rows<true><<<g, 256, 0, s>>>(n, A.off, A.len, A.col, A.val, S->flag, L.dinv, L.agg, omega_f, nullptr,
                                   S->Pc.rp, S->Pc.col, S->Pc.val, h->d_err);
  VEM_TRY(check_device_errors(h, "AMG prolongator"));
  // R = P^T (CSR with rows sorted by fine index)
  VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)nc + 1));
  VEM_CUDA(h, cudaMemsetAsync(S->cnt, 0, sizeof(int64_t) * nc, s));
  count_launch();
  k_t_count<<<g, 256, 0, s>>>(n, S->Pc.rp, S->Pc.col, reinterpret_cast<unsigned long long *>(S->cnt));
  VEM_TRY(csr_layout(h, S->Rc, nc, S->cnt));
  VEM_TRY(grow(h, S->cur, S->c_cur, (size_t)nc + 1));
  VEM_CUDA(h, cudaMemcpyAsync(S->cur, S->Rc.rp, sizeof(int64_t) * nc, cudaMemcpyDeviceToDevice, s));
  count_launch();
  k_t_fill<<<g, 256, 0, s>>>(n, S->Pc.rp, S->Pc.col, S->Pc.val, reinterpret_cast<unsigned long long *>(S->cur),
                             S->Rc.col, S->Rc.val);
  count_launch();
  k_sort_rows<<<rows_grid(nc), 256, 0, s>>>(nc, S->Rc.rp, S->Rc.col, S->Rc.val);
  VEM_CUDA(h, cudaGetLastError());
  // A P, then P^T (A P)
  VEM_TRY(grow(h, S->cnt, S->c_cnt, (size_t)n + 1));
  count_launch();
  k_ap_rows<false><<<g, 256, 0, s>>>(n, A.off, A.len, A.col, A.val, S->Pc.rp, S->Pc.col, S->Pc.val, S->cnt,
                                     nullptr, nullptr, nullptr, h->d_err);
  VEM_TRY(csr_layout(h, S->APc, n, S->cnt));
  count_launch();
  k_ap_rows<true><<<g, 256, 0, s>>>(n, A.off, A.len, A.col, A.val, S->Pc.rp, S->Pc.col, S->Pc.val, nullptr,
                                    S->APc.rp, S->APc.col, S->APc.val, h->d_err);
  VEM_TRY(check_device_errors(h, "AMG product A P"));
  const int gc = rows_grid(nc);
  count_launch();
  k_rap_rows<false><<<gc, 256, 0, s>>>(nc, S->Rc.rp, S->Rc.col, S->Rc.val, S->APc.rp, S->APc.col, S->APc.val,
                                       S->cnt, nullptr, nullptr, nullptr, h->d_err);
  VEM_TRY(csr_layout(h, S->Ac, nc, S->cnt));
  count_launch();
  k_rap_rows<true><<<gc, 256, 0, s>>>(nc, S->Rc.rp, S->Rc.col, S->Rc.val, S->APc.rp, S->APc.col, S->APc.val,
                                      nullptr, S->Ac.rp, S->Ac.col, S->Ac.val, h->d_err);
  VEM_TRY(check_device_errors(h, "AMG Galerkin product"));
  // SELL copies: P and R for the cycle, the coarse operator as the next A
  VEM_TRY(csr_to_sell(h, S, S->Pc, L.P));
  VEM_TRY(csr_to_sell(h, S, S->Rc, L.R));
  VEM_TRY(csr_to_sell(h, S, S->Ac, S->lv[l + 1].A));
  L.nc = nc;
  *nc_out = nc;
  return VEM_OK;
}

static vem_status level_vectors(vem_handle *h, AmgState *S, int l) {
  AmgLevel &L = S->lv[l];
  L.n = L.A.m.rows;
  VEM_TRY(grow(h, L.dinv, L.c_dinv, (size_t)L.n));
  VEM_TRY(grow(h, L.vec, L.c_vec, 4 * (size_t)L.n));
  VEM_TRY(grow(h, S->dg, S->c_dg, (size_t)L.n));
  const SellMat &A = L.A.m;
  count_launch();
  k_amg_diag<<<rows_grid(L.n), 256, 0, h->stream>>>(L.n, A.off, A.len, A.col, A.val, S->dg, L.dinv, h->d_err);
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

vem_status amg_setup(vem_handle *h, const SellMat &Sm) {
  AmgState *S = state(h);
  S->valid = false;
  cudaStream_t s = h->stream;
  VEM_CUDA(h, cudaEventRecord(h->ev2, s));
  if (!S->ctr) VEM_TRY(dalloc_n(h, &S->ctr, kMaxRounds + 4));
  S->lv[0].A.m = Sm;   // a view of the handle's S
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
  {
    const SellMat &A = C.A.m;
    VEM_TRY(grow(h, S->flag, S->c_flag, (size_t)A.stored));
    VEM_TRY(grow(h, S->nstr, S->c_nstr, (size_t)C.n));
    VEM_CUDA(h, cudaMemsetAsync(S->ctr, 0, sizeof(unsigned long long) * 2, s));
    count_launch();
    k_amg_strength<<<rows_grid(C.n), 256, 0, s>>>(C.n, A.off, A.len, A.col, A.val, S->dg, 0.0, S->flag, S->nstr,
                                                  S->ctr);
    unsigned long long mx[2] = {0, 0};
    VEM_CUDA(h, cudaMemcpyAsync(mx, S->ctr, sizeof(mx), cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    C.omega = 4.0 / (3.0 * bits_to_double(mx[0]));
  }
  if (C.n <= kDenseMax) {
    VEM_TRY(grow(h, S->cinv, S->c_cinv, (size_t)C.n * C.n));
    count_launch();
    k_dense_from_sell<<<rows_grid(C.n), 256, 0, s>>>(C.n, C.A.m.off, C.A.m.len, C.A.m.col, C.A.m.val, S->cinv);
    count_launch();
    k_gauss_jordan<<<1, 256, 0, s>>>((int)C.n, S->cinv, h->d_err);
    S->csweeps = 0;
  } else {
    S->csweeps = kCoarseSweeps;
  }
  VEM_CUDA(h, cudaGetLastError());
  VEM_TRY(check_device_errors(h, "AMG setup"));
  VEM_CUDA(h, cudaEventRecord(h->ev3, s));
  VEM_CUDA(h, cudaEventSynchronize(h->ev3));
  float ms = 0.f;
  VEM_CUDA(h, cudaEventElapsedTime(&ms, h->ev2, h->ev3));
  S->t_setup_ms = ms;
  S->valid = true;
  return VEM_OK;
}

bool amg_valid(const vem_handle *h) { return h->amg && h->amg->valid; }
void amg_invalidate(vem_handle *h) {
  if (h->amg) h->amg->valid = false;
}
double amg_setup_ms(const vem_handle *h) { return h->amg ? h->amg->t_setup_ms : 0.0; }
int amg_levels(const vem_handle *h) { return amg_valid(h) ? h->amg->nlev : 0; }
void amg_free(vem_handle *h) {
  delete h->amg;   // device buffers are in h->allocations
  h->amg = nullptr;
}

// x = V(b) on level l; b and x are device vectors of that level's size.
static void cycle(vem_handle *h, AmgState *S, int l, const double *b, double *x, const double *sc) {
  cudaStream_t s = h->stream;
  AmgLevel &L = S->lv[l];
  const SellMat &A = L.A.m;
  const int gv = rows_grid(L.n), gs = sell_grid(A);
  if (l == S->nlev - 1) {
    if (S->csweeps == 0) {
      count_launch();
      k_vc_dense<<<(int)std::min<int64_t>((L.n + 7) / 8, 1024), 256, 0, s>>>((int)L.n, S->cinv, b, x, sc);
      return;
    }
    double *xa = L.x(), *xb = L.x2();
    count_launch();
    k_vc_pre<<<gv, 256, 0, s>>>(L.n, b, L.dinv, L.omega, xa, sc);
    for (int k = 1; k < S->csweeps; ++k) {
      double *out = (k == S->csweeps - 1) ? x : xb;
      count_launch();
      k_vc_sell<1><<<gs, 256, 0, s>>>(A.rows, A.nslices, A.off, A.col, A.val, xa, b, L.dinv, L.omega, out, sc);
      std::swap(xa, xb);
    }
    return;
  }
  AmgLevel &C = S->lv[l + 1];
  double *xa = L.x();
  count_launch();
  k_vc_pre<<<gv, 256, 0, s>>>(L.n, b, L.dinv, L.omega, xa, sc);
  count_launch();
  k_vc_sell<0><<<gs, 256, 0, s>>>(A.rows, A.nslices, A.off, A.col, A.val, xa, b, nullptr, 0.0, L.r(), sc);
  const SellMat &R = L.R.m, &P = L.P.m;
  count_launch();
  k_vc_spmv<<<sell_grid(R), 256, 0, s>>>(R.rows, R.nslices, R.off, R.col, R.val, L.r(), C.b(), sc);
  cycle(h, S, l + 1, C.b(), C.x2(), sc);
  count_launch();
  k_vc_sell<2><<<sell_grid(P), 256, 0, s>>>(P.rows, P.nslices, P.off, P.col, P.val, C.x2(), nullptr, nullptr, 0.0,
                                            xa, sc);
  count_launch();
  k_vc_sell<1><<<gs, 256, 0, s>>>(A.rows, A.nslices, A.off, A.col, A.val, xa, b, L.dinv, L.omega, x, sc);
}

void amg_vcycle(vem_handle *h, const double *b, double *x, const double *sc) {
  cycle(h, h->amg, 0, b, x, sc);
}

// ---- inspection (host copies for the tests) ----
vem_status amg_level_info(vem_handle *h, int *nlev, int64_t *rows, int64_t *nnz, int64_t *nnz_p) {
  if (!amg_valid(h)) return fail(h, VEM_ERR_BAD_INPUT, "no AMG hierarchy: call vem_amg_setup first");
  AmgState *S = h->amg;
  *nlev = S->nlev;
  for (int l = 0; l < S->nlev; ++l) {
    if (rows) rows[l] = S->lv[l].A.m.rows;
    if (nnz) nnz[l] = S->lv[l].A.m.nnz;
    if (nnz_p) nnz_p[l] = l + 1 < S->nlev ? S->lv[l].P.m.nnz : 0;
  }
  return VEM_OK;
}

vem_status amg_level_copy(vem_handle *h, int l, int64_t *rp, int32_t *col, double *val, int32_t *agg,
                          int64_t *prp, int32_t *pcol, double *pval) {
  if (!amg_valid(h)) return fail(h, VEM_ERR_BAD_INPUT, "no AMG hierarchy: call vem_amg_setup first");
  AmgState *S = h->amg;
  if (l < 0 || l >= S->nlev) return fail(h, VEM_ERR_BAD_INPUT, "AMG level %d of %d", l, S->nlev);
  AmgLevel &L = S->lv[l];
  if (rp || col || val) VEM_TRY(sell_to_host_csr(h, L.A.m, rp, col, val));
  const bool coarse = l + 1 < S->nlev;
  if (agg && coarse)
    VEM_CUDA(h, cudaMemcpy(agg, L.agg, sizeof(int32_t) * L.n, cudaMemcpyDeviceToHost));
  if ((prp || pcol || pval) && coarse) VEM_TRY(sell_to_host_csr(h, L.P.m, prp, pcol, pval));
  return VEM_OK;
}

double amg_omega(const vem_handle *h, int l) { return amg_valid(h) && l < h->amg->nlev ? h->amg->lv[l].omega : 0.0; }

}  // namespace vem
