// Krylov solvers of the saddle-point system (paper Sec. 5): the outer
// Krylov method (preconditioned MINRES or restarted FGMRES) with the block
// preconditioner built on diag(M) and S = B diag(M)^{-1} B^T, and the inner
// Jacobi-PCG on S.
//
// Every scalar of the recurrences lives in device memory; reductions are
// deterministic two-pass sums (block partials, then a fixed-order sum by the
// consumer), so a solve is bitwise reproducible.  The host only polls a
// convergence flag / residual estimate.
//
//   MINRES: Paige & Saunders (1975), preconditioned Lanczos form.
//   FGMRES(m): Saad (1993), right preconditioning, classical Gram-Schmidt
//   for the Arnoldi step with a second pass when the first lost more than
//   1/sqrt(2) of the vector's norm (Daniel, Gragg, Kaufman & Stewart 1976),
//   Givens rotations.
//   PCG: Hestenes & Stiefel (1952) with the Jacobi preconditioner or one
//   V-cycle of the smoothed-aggregation AMG of amg.cu.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "geom_device.cuh"
#include "handle.cuh"

namespace vem {

static bool debug_on() {
  static int v = -1;
  if (v < 0) v = std::getenv("VEM_DEBUG") ? 1 : 0;
  return v == 1;
}

// ---------------------------------------------------------------- slots ----
enum Slot {
  P_RZ0 = 0, P_RZ1, P_PQ, P_RR, P_BB,       // PCG
  P_DELTA, P_G2U, P_G2P, P_R2, P_B2,        // MINRES and residual checks
  P_NRM, P_H0                               // FGMRES: ||w||^2, then h_0..h_m
};
enum Scal {
  S_PCG_DONE = 0, S_PCG_IT, S_PCG_BAD, S_R2 = 4, S_B2 = 5,
  S_MR = 8,   // MINRES: gamma_old, gamma, c_old, c, s_old, s, eta, a1, a2, a3, ceta, inv_gamma
  S_GM = 32,  // FGMRES: beta, inv_beta, est, inv_hnext, bad, then H, cs, sn, g, y, h1, h2
};
enum { MR_GOLD = 0, MR_G, MR_COLD, MR_C, MR_SOLD, MR_S, MR_ETA, MR_A1, MR_A2, MR_A3, MR_CETA,
       MR_IG, MR_BAD };

__host__ __device__ inline double *slot(double *part, int s) { return part + (size_t)s * kMaxBlocks; }


// y = A x for the operator (one system or a stacked batch)
static void op_apply(cudaStream_t s, const VemOp &op, const double *x, double *y, double *dot_part = nullptr) {
  if (op.nbatch == 1) spmv(s, op.A, x, y, dot_part);
  else spmv_batched(s, op.A, op.nbatch, op.n_u1, op.A.val, x, y, dot_part);
}

// op_apply with its launch timed by a pair of CUDA events on the stream
// (the first kTimedA launches of a solve; read back by collect_saddle()).
static void op_apply_timed(vem_handle *h, const VemOp &op, const double *x, double *y,
                           double *dot_part = nullptr) {
  const int k = h->n_saddle_pending;
  if (k < vem_handle::kTimedA) cudaEventRecord(h->aev[2 * k], h->stream);
  op_apply(h->stream, op, x, y, dot_part);
  if (k < vem_handle::kTimedA) {
    cudaEventRecord(h->aev[2 * k + 1], h->stream);
    h->n_saddle_pending = k + 1;
  }
}

// Accumulate the timed saddle SpMV launches (the stream has been synchronised).
static void collect_saddle(vem_handle *h) {
  for (int i = 0; i < h->n_saddle_pending; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->aev[2 * i], h->aev[2 * i + 1]) == cudaSuccess) {
      h->t_saddle_spmv_ms += ms;
      h->n_saddle_spmv += 1;
    }
  }
  cudaGetLastError();
  h->n_saddle_pending = 0;
}

// --------------------------------------------------------------- PCG -------
// Jacobi-preconditioned CG in the single-reduction form of Chronopoulos &
// Gear (J. Comput. Appl. Math. 25, 1989): one fused kernel computes
// w = S u with the three dot products (r,u), (w,u), (r,r), and its
// last-arriving block turns them into alpha, beta and the convergence test;
// one fused kernel then updates p, s, x, r, u.  Two launches per iteration.
enum { CG_ALPHA = 24, CG_BETA, CG_GPREV, CG_APREV, CG_BB, CG_ITER };

// The converged flag read once per block and broadcast, so an early return is
// uniform across the block.
__device__ __forceinline__ bool block_done(const double *sc) {
  pdl_wait();   // the previous kernel's results first (launch_pdl)
  __shared__ int f;
  if (threadIdx.x == 0) f = (sc[S_PCG_DONE] != 0.0);
  __syncthreads();
  const bool r = f != 0;
  __syncthreads();
  return r;
}

template <class T>
__global__ void __launch_bounds__(kRedThreads) k_cg_init(int64_t n, const double *__restrict__ b,
                                                         const T *__restrict__ dinv, T *x, T *r, T *u,
                                                         T *p, T *s, double *part, double *sc,
                                                         unsigned int *ctr) {
  double bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    const T bt = (T)bi;
    x[i] = 0;
    r[i] = bt;
    u[i] = dinv[i] * bt;
    p[i] = 0;
    s[i] = 0;
    bb += (double)bt * (double)bt;
  }
  block_partial(bb, slot(part, P_BB));
  block_partial(bb, slot(part, P_RR));   // ||r_0||^2 for the first convergence test
  if (last_block(ctr)) {
    const double t = sum_partials_cg(slot(part, P_BB), gridDim.x);
    if (threadIdx.x == 0) {
      sc[CG_BB] = t;
      sc[S_PCG_DONE] = (t == 0.0) ? 1.0 : 0.0;
      sc[S_PCG_IT] = 0.0;
      sc[CG_ITER] = 0.0;
      sc[S_PCG_BAD] = isfinite(t) ? 0.0 : 2.0;
      if (!isfinite(t)) sc[S_PCG_DONE] = 1.0;
    }
  }
}

// Block partials of (r,u) and (w,u); the last block to arrive turns them
// and (r,r) (from the update or init kernel) into the convergence test,
// alpha and beta.  The iteration number is a device counter, so every
// iteration launches the same arguments (the launches can be graph-captured).
__device__ __forceinline__ void cg_spmv_finish(double gam, double del, double *part, double *sc,
                                               unsigned int *ctr, double tol2, int nb_rr) {
  block_partial(gam, slot(part, P_RZ0));
  block_partial(del, slot(part, P_RZ1));
  if (!last_block(ctr)) return;
  const double G = sum_partials_cg(slot(part, P_RZ0), gridDim.x);
  const double D = sum_partials_cg(slot(part, P_RZ1), gridDim.x);
  const double R = sum_partials_cg(slot(part, P_RR), nb_rr);
  if (threadIdx.x != 0) return;
  const int it = (int)sc[CG_ITER];
  sc[CG_ITER] = (double)(it + 1);
  if (!isfinite(R) || !isfinite(G) || !isfinite(D)) {
    sc[S_PCG_BAD] = 2.0;
    sc[S_PCG_DONE] = 1.0;
    return;
  }
  sc[S_PCG_IT] = (double)it;
  if (R <= tol2 * sc[CG_BB]) {
    sc[S_PCG_DONE] = 1.0;
    return;
  }
  double beta = 0.0, den = D;
  if (it > 0) {
    beta = G / sc[CG_GPREV];
    den = D - beta * G / sc[CG_APREV];
  }
  if (!(den > 0.0) || !(G > 0.0)) {
    sc[S_PCG_BAD] = 1.0;
    sc[S_PCG_DONE] = 1.0;
    return;
  }
  const double alpha = G / den;
  sc[CG_ALPHA] = alpha;
  sc[CG_BETA] = beta;
  sc[CG_GPREV] = G;
  sc[CG_APREV] = alpha;
}

// w = S u with the partials of (r,u), (w,u) for one system: one warp per
// slice, one thread per row.
#ifndef VEM_CG_MINB
#define VEM_CG_MINB 4
#endif
template <class T>
__global__ void __launch_bounds__(256, VEM_CG_MINB) k_cg_spmv(int64_t rows, int64_t nslices, int64_t stored,
                                                             const int64_t *__restrict__ off,
                                                             const int32_t *__restrict__ col,
                                                             const T *__restrict__ val, const T *__restrict__ u,
                                                             const T *__restrict__ r, T *__restrict__ w,
                                                             double *part, double *sc, unsigned int *ctr,
                                                             double tol2, int nb_rr) {
  if (block_done(sc)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  T gam = 0, del = 0;
  for (int64_t s = warp; s < nslices; s += nwarps) {
    const int64_t i = 32 * s + lane;
    // own-row operands first, so their loads overlap the row's gathers
    T ui = 0, ri = 0;
    if (i < rows) {
      ui = __ldg(u + i);
      ri = __ldg(r + i);
    }
    const T t = sell_row_dot<T, VEM_CG_KB, VEM_CG_PRED>(off, col, val, u, s, lane);
    if (i < rows) {
      w[i] = t;
      gam += ri * ui;
      del += t * ui;
    }
  }
  cg_spmv_finish((double)gam, (double)del, part, sc, ctr, tol2, nb_rr);
}

// The stacked systems of a batch (values of system b at val + b * stored,
// vectors at b * rows), each warp task a tile of one 32-row slice times kR
// consecutive systems: the column ids are read once per tile and serve kR
// value streams and gathers (independent FMA chains).  timing != 0 runs the
// products only (no partials, no scalars), for the autotuner.
template <class T, int kR>
__global__ void __launch_bounds__(256) k_cg_spmv_tiles(int64_t rows, int64_t nslices, int nbatch, int64_t stored,
                                                      const int64_t *__restrict__ off,
                                                      const int32_t *__restrict__ col,
                                                      const T *__restrict__ val, const T *__restrict__ u,
                                                      const T *__restrict__ r, T *__restrict__ w, double *part,
                                                      double *sc, unsigned int *ctr, double tol2, int nb_rr,
                                                      int timing) {
  if (!timing && block_done(sc)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t groups = (nbatch + kR - 1) / kR;
  T gam = 0, del = 0;
  for (int64_t tk = warp; tk < nslices * groups; tk += nwarps) {
    const int64_t g = tk / nslices, s = tk - g * nslices, b0 = g * kR;
    const int64_t o = off[s];
    const int wdt = (int)((off[s + 1] - o) >> 5);
    const int64_t i = 32 * s + lane;
    T acc[kR];
#pragma unroll
    for (int q = 0; q < kR; ++q) acc[q] = 0;
    // kB entries per step (predicated on the slice width): all their column
    // ids, then the kR x kB values and gathers, then the FMAs
    constexpr int kB = kR >= 8 ? 1 : 8 / kR;
    for (int j = 0; j < wdt; j += kB) {
      int32_t c[kB];
#pragma unroll
      for (int t = 0; t < kB; ++t) c[t] = (j + t < wdt) ? __ldcs(col + o + 32 * (int64_t)(j + t) + lane) : 0;
      T v[kR][kB], x[kR][kB];
#pragma unroll
      for (int q = 0; q < kR; ++q)
#pragma unroll
        for (int t = 0; t < kB; ++t) {
          const bool ok = (j + t < wdt) && (b0 + q < nbatch);
          v[q][t] = ok ? __ldcs(val + (b0 + q) * stored + o + 32 * (int64_t)(j + t) + lane) : T(0);
          x[q][t] = ok ? __ldg(u + (b0 + q) * rows + c[t]) : T(0);
        }
#pragma unroll
      for (int q = 0; q < kR; ++q)
#pragma unroll
        for (int t = 0; t < kB; ++t)
          if ((j + t < wdt) && (b0 + q < nbatch)) acc[q] += v[q][t] * x[q][t];
    }
    if (i < rows) {
#pragma unroll
      for (int q = 0; q < kR; ++q) {
        if (b0 + q < nbatch) {
          const int64_t gi = (b0 + q) * rows + i;
          w[gi] = acc[q];
          const T ui = u[gi];
          gam += r[gi] * ui;
          del += acc[q] * ui;
        }
      }
    }
  }
  if (timing) return;
  cg_spmv_finish((double)gam, (double)del, part, sc, ctr, tol2, nb_rr);
}

// p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, and with the
// Jacobi preconditioner u = D^-1 r (the AMG cycle computes u separately)
template <class T, bool kJacobi = true>
__global__ void __launch_bounds__(kRedThreads) k_cg_update(int64_t n, T *x, T *r, T *u, T *p, T *s,
                                                           const T *__restrict__ w,
                                                           const T *__restrict__ dinv,
                                                           const double *sc, double *part) {
  if (block_done(sc)) return;
  const T alpha = (T)sc[CG_ALPHA], beta = (T)sc[CG_BETA];
  T rr = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T pi = u[i] + beta * p[i];
    const T si = w[i] + beta * s[i];
    x[i] += alpha * pi;
    const T ri = r[i] - alpha * si;
    p[i] = pi;
    s[i] = si;
    r[i] = ri;
    if (kJacobi) u[i] = dinv[i] * ri;
    rr += ri * ri;
  }
  block_partial((double)rr, slot(part, P_RR));
}

// The whole Jacobi-PCG inner solve of a small S in one thread block: the
// recurrence, scalars and stopping rule of k_cg_init / k_cg_update /
// k_cg_spmv, with every reduction a block reduction (fixed order), so no
// launch boundary separates the iterations (a small solve is bound by
// latency, not by bytes).  The six vectors live in shared memory (6 n
// entries; global round trips cost ~12 us per iteration on a 512-row S),
// S and D^-1 are read through the read-only cache; x is written out at the
// end.  Rows are dealt as in the SpMV (row 32 s + lane of slice s, slices to
// the warps in turn).  At most maxit updates; the host reads S_PCG_DONE /
// S_PCG_IT / S_PCG_BAD as after the multi-launch form.
// One block pays off while S is small enough for one SM's FP64 rate: about
// 5 us per iteration on 3.6k stored entries (8^3, E0) against ~17 us for the
// two dependent launches, but ~0.8 ns per stored entry, so it loses beyond
// ~20k entries (a 1,000-cell CVT mesh at k = 2, 112k entries: 87 against
// 23 us per iteration).
constexpr int kSmallCgRows = 4096;        // shared-memory capacity (6 vectors)
constexpr int64_t kSmallCgStored = 16384; // stored entries of S
constexpr int kSmallCgThreads = 1024;

// a, b, c summed over the block in a fixed order: a tree over the threads'
// values in shared memory (red: 3 blockDim entries; blockDim a power of two
// >= 32), then the last 32 by shuffles in warp 0.  The sums are valid in
// thread 0 only.  GB300 issues an FP64 warp instruction about every 16
// cycles per SM, so the tree (31 warp additions per value at 1,024 threads)
// is used rather than per-warp shuffle trees (160).
__device__ __forceinline__ void block_sum3(double &a, double &b, double &c, double *red) {
  const int t = threadIdx.x, nt = blockDim.x;
  red[t] = a;
  red[nt + t] = b;
  red[2 * nt + t] = c;
  __syncthreads();
  for (int h = nt >> 1; h >= 32; h >>= 1) {
    if (t < h) {
      red[t] += red[t + h];
      red[nt + t] += red[nt + t + h];
      red[2 * nt + t] += red[2 * nt + t + h];
    }
    __syncthreads();
  }
  if (t < 32) {
    a = red[t];
    b = red[nt + t];
    c = red[2 * nt + t];
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
  }
}

template <class T>
__global__ void __launch_bounds__(kSmallCgThreads) k_cg_block(int64_t n, int64_t nslices,
                                                              const int64_t *__restrict__ off,
                                                              const int32_t *__restrict__ col,
                                                              const T *__restrict__ val, const T *__restrict__ dinv,
                                                              const double *__restrict__ b, T *x_out, double *sc,
                                                              double tol2, int maxit) {
  extern __shared__ unsigned char cg_smem[];
  T *u = reinterpret_cast<T *>(cg_smem);
  T *x = u + n, *r = x + n, *p = r + n, *sv = p + n, *w = sv + n;
  __shared__ double red[3 * kSmallCgThreads];
  __shared__ double bc[3];   // alpha, beta, stop
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double bb = 0.0;
  for (int64_t sl = warp; sl < nslices; sl += nw) {
    const int64_t i = 32 * sl + lane;
    if (i < n) {
      const T bt = (T)b[i];
      x[i] = 0;
      r[i] = bt;
      u[i] = __ldg(dinv + i) * bt;
      p[i] = 0;
      sv[i] = 0;
      w[i] = 0;
      bb += (double)bt * (double)bt;
    }
  }
  double t1 = 0.0, t2 = 0.0;
  block_sum3(bb, t1, t2, red);
  // thread 0's scalars: ||b||^2, the previous gamma and alpha, the state
  double BB = bb, gprev = 0.0, aprev = 0.0, R = bb;
  int it_done = 0, bad = 0, done = 0;
  if (threadIdx.x == 0) {
    done = (BB == 0.0) ? 1 : 0;
    if (!isfinite(BB)) {
      bad = 2;
      done = 1;
    }
    bc[2] = done;
  }
  __syncthreads();
  for (int it = 0; it <= maxit; ++it) {
    if (bc[2] != 0.0) break;
    double rr = 0.0;
    if (it > 0) {
      // p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = D^-1 r
      const T alpha = (T)bc[0], beta = (T)bc[1];
      for (int64_t sl = warp; sl < nslices; sl += nw) {
        const int64_t i = 32 * sl + lane;
        if (i < n) {
          const T pi = u[i] + beta * p[i];
          const T si = w[i] + beta * sv[i];
          x[i] += alpha * pi;
          const T ri = r[i] - alpha * si;
          p[i] = pi;
          sv[i] = si;
          r[i] = ri;
          u[i] = __ldg(dinv + i) * ri;
          rr += (double)(ri * ri);
        }
      }
      __syncthreads();   // u complete before the gathers
    }
    // w = S u with (r, u) and (w, u)
    T gam = 0, del = 0;
    for (int64_t sl = warp; sl < nslices; sl += nw) {
      const int64_t i = 32 * sl + lane;
      const int64_t o = __ldg(off + sl);
      const int wdt = (int)((__ldg(off + sl + 1) - o) >> 5);
      T t = 0;
      for (int j = 0; j < wdt; ++j) {
        const int64_t q = o + 32 * (int64_t)j + lane;
        t += __ldg(val + q) * u[__ldg(col + q)];
      }
      if (i < n) {
        w[i] = t;
        gam += r[i] * u[i];
        del += t * u[i];
      }
    }
    double G = (double)gam, D = (double)del;
    block_sum3(rr, G, D, red);
    if (threadIdx.x == 0) {
      if (it > 0) R = rr;
      if (!isfinite(R) || !isfinite(G) || !isfinite(D)) {
        bad = 2;
        done = 1;
      } else {
        it_done = it;
        if (R <= tol2 * BB) {
          done = 1;
        } else {
          double beta = 0.0, den = D;
          if (it > 0) {
            beta = G / gprev;
            den = D - beta * G / aprev;
          }
          if (!(den > 0.0) || !(G > 0.0)) {
            bad = 1;
            done = 1;
          } else {
            const double alpha = G / den;
            bc[0] = alpha;
            bc[1] = beta;
            gprev = G;
            aprev = alpha;
          }
        }
      }
      // the cap: maxit updates at most
      bc[2] = (done || it == maxit) ? 1.0 : 0.0;
    }
    __syncthreads();
  }
  for (int64_t sl = warp; sl < nslices; sl += nw) {
    const int64_t i = 32 * sl + lane;
    if (i < n) x_out[i] = x[i];
  }
  if (threadIdx.x == 0) {
    sc[S_PCG_DONE] = done ? 1.0 : 0.0;
    sc[S_PCG_IT] = (double)it_done;
    sc[S_PCG_BAD] = (double)bad;
  }
}

__global__ void k_f32_to_f64(int64_t n, const float *__restrict__ a, double *b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// Solve S x = b (length n_p) to relative residual inner_rtol with vectors,
// matrix values and arithmetic in T; returns the iterations.
// Capture the launches of body() on a private stream into the executable
// graph slot (kernels counted once per replay, not at capture).  Returns
// false, with no graph, when capture or instantiation fails.
template <class F>
static bool capture_graph(vem_handle *h, cudaGraphExec_t &slot, int64_t &kernels, F body) {
  if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    if (slot) cudaGraphExecDestroy(slot);
    slot = nullptr;
    return false;
  }
  cudaStream_t saved = h->stream;
  const int64_t l0 = launch_count();
  cudaGraph_t g = nullptr;
  bool ok = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    h->stream = h->cap_stream;
    body();
    h->stream = saved;
    ok = cudaStreamEndCapture(h->cap_stream, &g) == cudaSuccess && g != nullptr;
  }
  const int64_t nk = launch_count() - l0;
  count_launches(-nk);
  // an executable graph of the same topology (the same launch sequence with
  // other arguments, e.g. a rebuilt hierarchy of the same depth) is updated
  // in place, which costs far less than a new instantiation
  bool updated = false;
  if (ok && slot) {
    cudaGraphExecUpdateResultInfo info;
    updated = cudaGraphExecUpdate(slot, g, &info) == cudaSuccess;
    if (!updated) cudaGetLastError();
  }
  if (!updated && slot) {
    cudaGraphExecDestroy(slot);
    slot = nullptr;
  }
  if (ok && !updated) ok = cudaGraphInstantiate(&slot, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    if (slot) cudaGraphExecDestroy(slot);
    slot = nullptr;
    cudaGetLastError();
    return false;
  }
  kernels = nk;
  return true;
}

// The inner PCG's graph of 4 iterations for one set of launch arguments
// (key); the 16-iteration graph of the same key is captured later, on first
// use (pcg_graph16_key).
template <class F>
static bool capture_pcg_graphs(vem_handle *h, const std::vector<uintptr_t> &key, F iteration) {
  h->pcg_graph_key.clear();
  h->pcg_graph16_key.clear();
  const bool ok = capture_graph(h, h->pcg_graph, h->pcg_graph_kernels, [&]() {
    for (int k = 0; k < 4; ++k) iteration();
  });
  if (ok) h->pcg_graph_key = key;
  return ok;
}
// One launch of the tiled batched Schur SpMV with kR systems per tile.
template <class T, int kR>
static void launch_tiles_r(vem_handle *h, const VemOp &op, const T *sval, const T *u, const T *r, T *w,
                           double tol2, int nb_rr, int timing) {
  static int cap = 0;
  if (cap == 0) cap = one_wave_blocks((const void *)k_cg_spmv_tiles<T, kR>);
  const int64_t tasks = op.S.nslices * ((op.nbatch + kR - 1) / kR);
  int64_t g = (tasks + 7) / 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  count_launch();
  k_cg_spmv_tiles<T, kR><<<(int)g, 256, 0, h->stream>>>(op.S.rows, op.S.nslices, op.nbatch, op.S.stored, op.S.off,
                                                        op.S.col, sval, u, r, w, h->part, h->scal, h->ctr + 1, tol2,
                                                        nb_rr, timing);
}

template <class T>
static void launch_tiles(vem_handle *h, const VemOp &op, const T *sval, const T *u, const T *r, T *w, double tol2,
                         int nb_rr, int tile, int timing) {
  switch (tile) {
    case 1: launch_tiles_r<T, 1>(h, op, sval, u, r, w, tol2, nb_rr, timing); break;
    case 2: launch_tiles_r<T, 2>(h, op, sval, u, r, w, tol2, nb_rr, timing); break;
    case 4: launch_tiles_r<T, 4>(h, op, sval, u, r, w, tol2, nb_rr, timing); break;
    default: launch_tiles_r<T, 8>(h, op, sval, u, r, w, tol2, nb_rr, timing); break;
  }
}

// Autotuner of the tile shape of the batched Schur SpMV: on the first solve
// of a shape (rows, slices, systems, value type) every candidate (1, 2, 4, 8
// systems per 32-row tile) runs on the live vectors in timing mode (products
// only), three launches each after one warm-up, timed with CUDA events on the
// stream; the fastest is kept for the process (per device, shape and value
// type; the cache is shared by all handles and guarded by a mutex).
template <class T>
static int tune_tiles(vem_handle *h, const VemOp &op, const T *sval, const T *u, const T *r, T *w, int nb_rr) {
  static std::mutex mu;
  static std::map<std::tuple<int, int64_t, int64_t, int>, int> best;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, op.S.rows, op.S.nslices, op.nbatch);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = best.find(key);
    if (it != best.end()) {
      h->schur_tile = it->second;
      return it->second;
    }
  }
  int pick = 1;
  float pick_ms = 1e30f;
  for (int tile : {1, 2, 4, 8}) {
    if (tile > 1 && tile > op.nbatch) break;
    launch_tiles<T>(h, op, sval, u, r, w, 0.0, nb_rr, tile, 1);
    cudaEventRecord(h->ev2, h->stream);
    for (int k = 0; k < 3; ++k) launch_tiles<T>(h, op, sval, u, r, w, 0.0, nb_rr, tile, 1);
    cudaEventRecord(h->ev3, h->stream);
    cudaEventSynchronize(h->ev3);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev2, h->ev3) == cudaSuccess && ms < pick_ms) {
      pick_ms = ms;
      pick = tile;
    }
  }
  cudaGetLastError();
  {
    std::lock_guard<std::mutex> lk(mu);
    best[key] = pick;
  }
  h->schur_tile = pick;
  if (debug_on()) fprintf(stderr, "[vem] batched Schur SpMV tile: %d systems (%.3f ms / 3)\n", pick, pick_ms);
  return pick;
}

template <class T>
static vem_status pcg_solve_t(vem_handle *h, const VemOp &op, const T *sval, const T *dinv, const double *b,
                              T *x, T *wk, int *iters) {
  cudaStream_t s = h->stream;
  const int64_t n = op.n_p;
  T *r = wk, *u = wk + n, *p = wk + 2 * n, *sv = wk + 3 * n, *w = wk + 4 * n;
  const int nb = nblocks_vec(n);
  static int cap_s = 0;
  if (cap_s == 0) cap_s = one_wave_blocks((const void *)k_cg_spmv<T>);
  int nbs = (int)((op.S.nslices + 7) / 8);
  if (nbs > cap_s) nbs = cap_s;
  if (nbs < 1) nbs = 1;
  double *sc = h->scal;
  const double tol2 = h->opt.inner_rtol * h->opt.inner_rtol;
  // the AMG-preconditioned form replaces u = D^-1 r by one V-cycle u = V(r)
  bool amg = false;
  if constexpr (sizeof(T) == sizeof(double)) amg = h->opt.inner != VEM_INNER_PCG;
  const int maxit = h->opt.inner_maxit;
  if (!amg && op.nbatch == 1 && n <= kSmallCgRows && op.S.stored <= kSmallCgStored) {
    const size_t smem = 6 * (size_t)n * sizeof(T);
    // per call: the attribute belongs to the current device
    VEM_CUDA(h, cudaFuncSetAttribute(k_cg_block<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     6 * kSmallCgRows * (int)sizeof(T)));
    // a warp per slice up to 32 warps (a power of two for the tree sums)
    int nthr = 32;
    while (nthr < kSmallCgThreads && nthr < 32 * op.S.nslices) nthr <<= 1;
    count_launch();
    k_cg_block<T><<<1, nthr, smem, s>>>(n, op.S.nslices, op.S.off, op.S.col, sval, dinv, b, x, sc, tol2, maxit);
    VEM_CUDA(h, cudaGetLastError());
    VEM_CUDA(h, cudaMemcpyAsync(h->h_scal, sc, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    if (h->h_scal[S_PCG_BAD] != 0.0)
      return fail(h, h->h_scal[S_PCG_BAD] == 2.0 ? VEM_ERR_NONFINITE : VEM_ERR_BREAKDOWN, "inner PCG breakdown");
    *iters = h->h_scal[S_PCG_DONE] != 0.0 ? (int)h->h_scal[S_PCG_IT] : maxit;
    h->last_pcg_iters = *iters;
    return VEM_OK;
  }
  count_launch();
  k_cg_init<T><<<nb, kRedThreads, 0, s>>>(n, b, dinv, x, r, u, p, sv, h->part, sc, h->ctr);
  auto precondition = [&]() {
    if constexpr (sizeof(T) == sizeof(double)) amg_vcycle(h, h->amg, r, u, sc);
  };
  if (amg) {
    amg_time_next_cycle(h->amg);   // the finest-level cycle launches of this eager cycle
    precondition();
  }
  // every launch of the Schur SpMV is timed with a pair of events
  int ntimed = 0;
  // stacked systems: the tile shape (systems per tile) chosen by the autotuner
  const int tile = op.nbatch > 1 ? tune_tiles<T>(h, op, sval, u, r, w, nb) : 1;
  auto spmv_it = [&](int) {
    if (ntimed < vem_handle::kTimed) cudaEventRecord(h->tev[2 * ntimed], s);
    if (op.nbatch == 1) {
      count_launch();
      k_cg_spmv<T><<<nbs, 256, 0, s>>>(op.S.rows, op.S.nslices, op.S.stored, op.S.off, op.S.col, sval, u, r, w,
                                       h->part, sc, h->ctr + 1, tol2, nb);
    } else {
      launch_tiles<T>(h, op, sval, u, r, w, tol2, nb, tile, 0);
    }
    if (ntimed < vem_handle::kTimed) cudaEventRecord(h->tev[2 * ntimed + 1], s);
    ++ntimed;
  };
  auto collect = [&]() {
    const int m = ntimed < vem_handle::kTimed ? ntimed : vem_handle::kTimed;
    for (int i = 0; i < m; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, h->tev[2 * i], h->tev[2 * i + 1]) == cudaSuccess) {
        h->t_schur_spmv_ms += ms;
        h->n_schur_spmv += 1;
      }
    }
    cudaGetLastError();
    ntimed = 0;
    if (amg) amg_collect_timing(h, h->amg);
  };
  spmv_it(0);
  // the host polls the convergence flag first after as many iterations as
  // the previous inner solve took (consecutive solves need similar counts),
  // then every 4; launches past convergence return at once
  int chunk = h->last_pcg_iters > 0 ? h->last_pcg_iters : 8;
  // one iteration (update, preconditioner, SpMV) on the handle's current
  // stream; every launch argument is the same in every iteration
  auto iteration = [&]() {
    cudaStream_t cs = h->stream;
    count_launch();
    if (amg) {
      launch_pdl(k_cg_update<T, false>, nb, kRedThreads, 0, cs, n, x, r, u, p, sv, (const T *)w, dinv,
                 (const double *)sc, h->part);
      precondition();
    } else {
      launch_pdl(k_cg_update<T, true>, nb, kRedThreads, 0, cs, n, x, r, u, p, sv, (const T *)w, dinv,
                 (const double *)sc, h->part);
    }
    if (op.nbatch == 1) {
      count_launch();
      launch_pdl(k_cg_spmv<T>, nbs, 256, 0, cs, op.S.rows, op.S.nslices, op.S.stored, op.S.off, op.S.col, sval,
                 (const T *)u, (const T *)r, w, h->part, sc, h->ctr + 1, tol2, nb);
    } else {
      launch_tiles<T>(h, op, sval, u, r, w, tol2, nb, tile, 0);
    }
  };
  // the iterations run from CUDA graphs of 16 and of 4 iterations, captured
  // once per set of launch arguments (eager launches if capture fails): the
  // expected count first (the previous inner solve's), as 16-iteration graphs
  // and the rest in 4s, then 4 at a time between polls of the device flag
  constexpr int kGraphIters = 4, kLongIters = 16;
  uint64_t tol_bits = 0;
  std::memcpy(&tol_bits, &tol2, sizeof(double));
  const std::vector<uintptr_t> key = {
      (uintptr_t)op.S.off, (uintptr_t)op.S.col, (uintptr_t)sval, (uintptr_t)u, (uintptr_t)r, (uintptr_t)w,
      (uintptr_t)x, (uintptr_t)p, (uintptr_t)sv, (uintptr_t)dinv, (uintptr_t)h->part, (uintptr_t)sc,
      (uintptr_t)h->ctr, (uintptr_t)n, (uintptr_t)nb, (uintptr_t)nbs, (uintptr_t)tile,
      (uintptr_t)tol_bits,
      (uintptr_t)amg, (uintptr_t)(amg ? amg_generation(h->amg) : 0), sizeof(T), (uintptr_t)op.nbatch,
      (uintptr_t)op.S.rows, (uintptr_t)op.S.stored};
  bool graph = h->pcg_graph != nullptr && h->pcg_graph_key == key;
  if (!graph) graph = capture_pcg_graphs(h, key, iteration);
  // 16-iteration graphs for the long Jacobi-PCG solves only: with the AMG
  // each iteration holds a whole V-cycle, the key changes with every
  // hierarchy, and capturing 16 cycles costs more than their launches save
  bool g16 = graph && h->pcg_graph16 != nullptr && h->pcg_graph16_key == key;
  int it = 0;
  while (it < maxit) {
    const int end = it + chunk < maxit ? it + chunk : maxit;
    chunk = 4;
    if (graph) {
      if (!g16 && !amg && end - it >= kLongIters) {
        g16 = capture_graph(h, h->pcg_graph16, h->pcg_graph16_kernels, [&]() {
          for (int k = 0; k < kLongIters; ++k) iteration();
        });
        if (g16) h->pcg_graph16_key = key;
      }
      for (; g16 && it + kLongIters <= end; it += kLongIters) {
        VEM_CUDA(h, cudaGraphLaunch(h->pcg_graph16, s));
        count_launches(h->pcg_graph16_kernels);
      }
      for (; it < end; it += kGraphIters) {
        VEM_CUDA(h, cudaGraphLaunch(h->pcg_graph, s));
        count_launches(h->pcg_graph_kernels);
      }
    } else {
      for (; it < end; ++it) iteration();
    }
    VEM_CUDA(h, cudaGetLastError());
    VEM_CUDA(h, cudaMemcpyAsync(h->h_scal, sc, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    collect();
    if (h->h_scal[S_PCG_DONE] != 0.0) break;
  }
  if (h->h_scal[S_PCG_BAD] != 0.0)
    return fail(h, h->h_scal[S_PCG_BAD] == 2.0 ? VEM_ERR_NONFINITE : VEM_ERR_BREAKDOWN,
                "inner PCG breakdown");
  *iters = (int)h->h_scal[S_PCG_IT];
  if (h->h_scal[S_PCG_DONE] == 0.0) *iters = maxit;   // cap reached: use the iterate
  h->last_pcg_iters = *iters;
  if (debug_on()) fprintf(stderr, "[vem] pcg n=%lld iters=%d done=%g\n", (long long)n, *iters, h->h_scal[S_PCG_DONE]);
  return VEM_OK;
}

// The near-null space of S for the paper's k = 2 element: per cell P, the
// pressure DOFs (1/|P|) int q m_a (eq. presMom) of q = 1, x, y, z, from the
// class's moments of 1 and x_j - x_P,j (translation invariant) and the cell's
// barycentre: B[(4P + a) 4 + j].
__global__ void k_pressure_modes(int64_t nc, const int32_t *__restrict__ cls_of, const double *__restrict__ pm_hat,
                                 const double *__restrict__ c_cent, double *B) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    const double *ph = pm_hat + 16 * (int64_t)cls_of[c];
    const double3 xP = load3(c_cent, c);
    const double xs[3] = {xP.x, xP.y, xP.z};
    for (int a = 0; a < 4; ++a)
      for (int j = 0; j < 4; ++j)
        B[(4 * c + a) * 4 + j] = j == 0 ? ph[4 * a] : xs[j - 1] * ph[4 * a] + ph[4 * a + j];
  }
}

// Build the hierarchy of S for the configured inner solver: the scalar AMG,
// or the point-block AMG on the 4 x 4 pressure blocks of the k = 2 element.
vem_status schur_amg_setup(vem_handle *h, const SellMat &S, const float *S_val32) {
  const bool fp32 = h->opt.precision == VEM_PRECISION_MIXED;
  if (h->opt.inner == VEM_INNER_BLOCK_AMG) {
    if (h->nq != 4)
      return fail(h, VEM_ERR_UNSUPPORTED, "the point-block AMG inner solver needs the paper's k = 2 element");
    if (fp32) return fail(h, VEM_ERR_UNSUPPORTED, "the point-block AMG cycle runs in FP64 only");
    if (!h->pmodes) VEM_TRY(dalloc_n(h, &h->pmodes, 16 * (size_t)h->nc));
    count_launch();
    k_pressure_modes<<<grid_for(h->nc, 256), 256, 0, h->stream>>>(h->nc, h->cls_of, h->pm_hat, h->c_cent,
                                                                   h->pmodes);
    VEM_CUDA(h, cudaGetLastError());
    return amg_setup_block(h, h->amg, S, 4, h->pmodes, 4, h->multiplier, schur_smoother(h));
  }
  if (h->multiplier && h->nq > 1)
    return fail(h, VEM_ERR_UNSUPPORTED, "the AMG inner solver with the multiplier needs one pressure DOF per cell");
  return amg_setup(h, h->amg, S, S_val32, fp32, h->multiplier, schur_smoother(h));
}

// S x = b with x, b FP64; the solve runs in FP64 or, with the mixed
// precision option, entirely in FP32 (values, vectors, arithmetic).
static vem_status pcg_solve(vem_handle *h, const VemOp &op, const double *b, double *x, double *wk, int *iters) {
  if (h->multiplier && op.nbatch == 1) {
    // singular S (constant pressures): solve for the consistent part of b
    if (!h->bproj) VEM_TRY(dalloc_n(h, &h->bproj, (size_t)op.n_p));
    VEM_TRY(neumann_mean_free(h, op.n_p, b, h->bproj));
    b = h->bproj;
  }
  if (h->opt.inner == VEM_INNER_AMG || h->opt.inner == VEM_INNER_BLOCK_AMG) {
    // FP64 CG; with the mixed option the scalar V-cycle runs in FP32
    const bool fp32 = h->opt.precision == VEM_PRECISION_MIXED;
    const bool block = h->opt.inner == VEM_INNER_BLOCK_AMG;
    if (!amg_valid(h->amg) || amg_is_fp32(h->amg) != fp32 || amg_smoother(h->amg) != schur_smoother(h) ||
        amg_is_block(h->amg) != block)
      VEM_TRY(schur_amg_setup(h, op.S, op.S_val32));
    return pcg_solve_t<double>(h, op, op.S.val, op.s_dinv, b, x, wk, iters);
  }
  if (h->opt.precision == VEM_PRECISION_MIXED) {
    float *w32 = reinterpret_cast<float *>(wk);
    float *x32 = w32 + 5 * op.n_p;
    VEM_TRY(pcg_solve_t<float>(h, op, op.S_val32, op.s_dinv32, b, x32, w32, iters));
    count_launch();
    k_f32_to_f64<<<grid_for(op.n_p, 256), 256, 0, h->stream>>>(op.n_p, x32, x);
    VEM_CUDA(h, cudaGetLastError());
    return VEM_OK;
  }
  return pcg_solve_t<double>(h, op, op.S.val, op.s_dinv, b, x, wk, iters);
}

// --------------------------------------------------------- vector ops -----
__global__ void k_residual(int64_t n, const double *__restrict__ b, const double *__restrict__ Ax,
                           double *r, double *part_r2, double *part_b2) {
  double rr = 0.0, bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = Ax ? b[i] - Ax[i] : b[i];   // Ax == NULL: x = 0
    r[i] = ri;
    rr += ri * ri;
    bb += b[i] * b[i];
  }
  block_partial(rr, part_r2);
  block_partial(bb, part_b2);
}

__global__ void k_read_sum(const double *part, int nb, double *out) {
  const double v = sum_partials(part, nb);
  if (threadIdx.x == 0) *out = v;
}

// z_u = v_u / diag(M) (first n_u entries) and the partial of v_u . z_u.
// dinv = 1 / diag(M), stored by the assembly: an FP64 division costs several
// FP64-pipe instructions, a product one, and GB300's FP64 pipe (about two
// FMAs per clock per SM) bounds a division per row below the HBM rate.
__global__ void k_diag_scale(int64_t nu, const double *__restrict__ v, const double *__restrict__ dinv,
                             double *z, double *part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nu;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = v[i] * dinv[i];
    z[i] = zi;
    s += v[i] * zi;
  }
  if (part) block_partial(s, part);
}

// Block upper-triangular flux part: z_u = (v_u - B^T z_p) / diag(M), with
// B^T z_p gathered per face from its (at most two) cells (dinv = 1 / diag(M),
// as in k_diag_scale).
// (stacked rows R = b * n_u1 + r; pressure of cell c of system b at b * n_p1 + c)
// NFD: face DOFs per face (1 for E0, 3 for K1), a constant so the face of a
// row is found without a division by a run-time value; kBatch: stacked
// systems (the single system needs no division by n_u1 at all).
template <int NFD, bool kBatch>
__global__ void k_tri_flux(int64_t nf, int64_t n_u, int64_t n_u1, int64_t n_p1,
                           const double *__restrict__ v, const double *__restrict__ dinv,
                           const int32_t *__restrict__ f_cell, const double *__restrict__ bt,
                           const double *__restrict__ zp, double *z) {
  for (int64_t R = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; R < n_u;
       R += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = 0, r = R;
    if (kBatch) {
      b = R / n_u1;
      r = R - b * n_u1;
    }
    double t = v[R];
    if (r < NFD * nf) {
      const int64_t f = r / NFD;
      if (r == f * NFD) {
        const int32_t c0 = f_cell[2 * f], c1 = f_cell[2 * f + 1];
        const double *zb = zp + b * n_p1;
        double g = bt[2 * f] * zb[c0];
        if (c1 >= 0) g += bt[2 * f + 1] * zb[c1];
        t -= g;
      }
    }
    z[R] = t * dinv[R];
  }
}

static void launch_tri_flux(cudaStream_t s, int nfd, bool batch, int64_t nf, int64_t n_u, int64_t n_u1,
                            int64_t n_p1, const double *v, const double *dinv, const int32_t *f_cell,
                            const double *bt, const double *zp, double *z) {
  const int g = grid_for(n_u, 256);
  count_launch();
  if (nfd == 3) {
    if (batch) k_tri_flux<3, true><<<g, 256, 0, s>>>(nf, n_u, n_u1, n_p1, v, dinv, f_cell, bt, zp, z);
    else k_tri_flux<3, false><<<g, 256, 0, s>>>(nf, n_u, n_u1, n_p1, v, dinv, f_cell, bt, zp, z);
  } else {
    if (batch) k_tri_flux<1, true><<<g, 256, 0, s>>>(nf, n_u, n_u1, n_p1, v, dinv, f_cell, bt, zp, z);
    else k_tri_flux<1, false><<<g, 256, 0, s>>>(nf, n_u, n_u1, n_p1, v, dinv, f_cell, bt, zp, z);
  }
}

// The same for several pressure DOFs per cell: B^T z_p of flux row R from
// the pressure-column entries of row R of [M B^T; B 0], which the assembly
// copies to kBtRow slots per row (slot k at k n_u + R; k_bt_rows).
// (stacked systems as in k_tri_flux: row R = b n_u1 + r, the copied B^T
// entries are those of the shared structure, B being independent of K)
template <bool kBatch>
__global__ void k_tri_flux_rows(int64_t n_u, int64_t n_u1, int64_t n_p1, const int32_t *__restrict__ bcol,
                                const double *__restrict__ bval, const double *__restrict__ v,
                                const double *__restrict__ dinv, const double *__restrict__ zp, double *z) {
  for (int64_t R = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; R < n_u;
       R += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = 0, r = R;
    if (kBatch) {
      b = R / n_u1;
      r = R - b * n_u1;
    }
    const double *zb = zp + b * n_p1;
    double t = v[R];
#pragma unroll
    for (int k = 0; k < kBtRow; ++k) t -= bval[k * n_u1 + r] * zb[bcol[k * n_u1 + r]];
    z[R] = t * dinv[R];
  }
}

__global__ void k_negate(int64_t n, double *x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = -x[i];
}

// z = w v and the partial of v . z (the pressure block W^-1 = I / gamma of
// Block-Reg)
__global__ void k_scale_dot(int64_t n, const double *__restrict__ v, double w, double *z, double *part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = w * v[i];
    z[i] = zi;
    s += v[i] * zi;
  }
  if (part) block_partial(s, part);
}

// ------------------------------------------------------------ MINRES -----
__global__ void k_mr_init(double *sc, const double *part, int nbu, int nbp) {
  const double g2 = sum_partials(slot((double *)part, P_G2U), nbu) + sum_partials(slot((double *)part, P_G2P), nbp);
  if (threadIdx.x == 0) {
    double *m = sc + S_MR;
    const double g = sqrt(g2 > 0.0 ? g2 : 0.0);
    m[MR_GOLD] = 1.0;
    m[MR_G] = g;
    m[MR_COLD] = 1.0;
    m[MR_C] = 1.0;
    m[MR_SOLD] = 0.0;
    m[MR_S] = 0.0;
    m[MR_ETA] = g;
    m[MR_IG] = g > 0.0 ? 1.0 / g : 0.0;
    m[MR_BAD] = (g2 >= 0.0 && isfinite(g2)) ? 0.0 : 1.0;
  }
}

__global__ void k_scale_by(int64_t n, double *x, const double *factor) {
  const double f = *factor;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= f;
}

// v_new = Az - (delta/gamma) v - (gamma/gamma_old) v_old, written over v_old.
__global__ void __launch_bounds__(kRedThreads) k_mr_lanczos(int64_t n, const double *__restrict__ Az,
                                                            const double *__restrict__ v, double *vold,
                                                            const double *part, int nbd, const double *sc) {
  const double delta = sum_partials(slot((double *)part, P_DELTA), nbd);
  const double *m = sc + S_MR;
  const double a = delta / m[MR_G], bcoef = m[MR_G] / m[MR_GOLD];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    vold[i] = Az[i] - a * v[i] - bcoef * vold[i];
}

__global__ void k_mr_scalars(double *sc, const double *part, int nbd, int nbu, int nbp) {
  const double delta = sum_partials(slot((double *)part, P_DELTA), nbd);
  const double g2 = sum_partials(slot((double *)part, P_G2U), nbu) + sum_partials(slot((double *)part, P_G2P), nbp);
  if (threadIdx.x != 0) return;
  double *m = sc + S_MR;
  if (!(g2 >= 0.0) || !isfinite(g2) || !isfinite(delta)) {
    m[MR_BAD] = 1.0;
    return;
  }
  const double gn = sqrt(g2);
  const double g = m[MR_G], c = m[MR_C], cold = m[MR_COLD], s = m[MR_S], sold = m[MR_SOLD];
  const double a0 = c * delta - cold * s * g;
  const double a1 = hypot(a0, gn);
  const double a2 = s * delta + cold * c * g;
  const double a3 = sold * g;
  const double cn = a0 / a1, sn = gn / a1;
  m[MR_A1] = a1;
  m[MR_A2] = a2;
  m[MR_A3] = a3;
  m[MR_CETA] = cn * m[MR_ETA];
  m[MR_ETA] = -sn * m[MR_ETA];
  m[MR_GOLD] = g;
  m[MR_G] = gn;
  m[MR_IG] = gn > 0.0 ? 1.0 / gn : 0.0;
  m[MR_COLD] = c;
  m[MR_C] = cn;
  m[MR_SOLD] = s;
  m[MR_S] = sn;
  if (!(a1 > 0.0)) m[MR_BAD] = 2.0;
}

// w_new = (z - a3 w_old - a2 w)/a1 over w_old; x += c eta w_new
__global__ void k_mr_update(int64_t n, const double *__restrict__ z, double *wold,
                            const double *__restrict__ w, double *x, const double *sc) {
  const double *m = sc + S_MR;
  const double ia1 = 1.0 / m[MR_A1], a2 = m[MR_A2], a3 = m[MR_A3], ce = m[MR_CETA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double wn = (z[i] - a3 * wold[i] - a2 * w[i]) * ia1;
    wold[i] = wn;
    x[i] += ce * wn;
  }
}

// ------------------------------------------------------------ FGMRES -----
constexpr int kMD = 8;   // vectors per multi-dot pass

// partials of V_i . w for i in [i0, i0 + cnt), cnt <= kMD
// skip (optional): a device flag; the launch does nothing when it is 0.
__global__ void __launch_bounds__(kRedThreads) k_multidot(int64_t n, const double *__restrict__ V,
                                                          int i0, int cnt,
                                                          const double *__restrict__ w, double *part,
                                                          const double *skip = nullptr) {
  if (skip && *skip == 0.0) return;
  double acc[kMD];
#pragma unroll
  for (int t = 0; t < kMD; ++t) acc[t] = 0.0;
  // four rows of the grid-stride sequence per step, their loads issued
  // together (a thread's sums run in the same row order as one row per step)
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; r + 3 * st < n; r += 4 * st) {
    const double w0 = w[r], w1 = w[r + st], w2 = w[r + 2 * st], w3 = w[r + 3 * st];
#pragma unroll
    for (int t = 0; t < kMD; ++t) {
      if (t < cnt) {
        const double *Vt = V + (size_t)(i0 + t) * n;
        const double v0 = Vt[r], v1 = Vt[r + st], v2 = Vt[r + 2 * st], v3 = Vt[r + 3 * st];
        acc[t] += v0 * w0;
        acc[t] += v1 * w1;
        acc[t] += v2 * w2;
        acc[t] += v3 * w3;
      }
    }
  }
  for (; r < n; r += st) {
    const double wr = w[r];
#pragma unroll
    for (int t = 0; t < kMD; ++t)
      if (t < cnt) acc[t] += V[(size_t)(i0 + t) * n + r] * wr;
  }
#pragma unroll
  for (int t = 0; t < kMD; ++t)
    if (t < cnt) block_partial(acc[t], slot(part, P_H0 + i0 + t));
}

// out[i] = sum of the partials of slot P_H0 + i, one block per i
__global__ void k_multidot_fin(const double *part, int nb, double *out, const double *skip = nullptr) {
  if (skip && *skip == 0.0) return;
  const double v = sum_partials(slot((double *)part, P_H0 + blockIdx.x), nb);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

// w += sgn * sum_i c[i] V_i  (i < cnt), optional partial of ||w||^2
__global__ void __launch_bounds__(kRedThreads) k_multiaxpy(int64_t n, const double *__restrict__ V, int cnt,
                                                           const double *__restrict__ c, double sgn,
                                                           double *w, double *part_nrm,
                                                           const double *skip = nullptr) {
  if (skip && *skip == 0.0) return;
  __shared__ double cs[260];
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) cs[i] = sgn * c[i];
  __syncthreads();
  double nn = 0.0;
  // four rows of the grid-stride sequence per step (each row's sum and the
  // norm's partial run in the same order as one row per step)
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; r + 3 * st < n; r += 4 * st) {
    double t0 = w[r], t1 = w[r + st], t2 = w[r + 2 * st], t3 = w[r + 3 * st];
    for (int i = 0; i < cnt; ++i) {
      const double *Vi = V + (size_t)i * n;
      const double c = cs[i];
      t0 += c * Vi[r];
      t1 += c * Vi[r + st];
      t2 += c * Vi[r + 2 * st];
      t3 += c * Vi[r + 3 * st];
    }
    w[r] = t0;
    w[r + st] = t1;
    w[r + 2 * st] = t2;
    w[r + 3 * st] = t3;
    nn += t0 * t0;
    nn += t1 * t1;
    nn += t2 * t2;
    nn += t3 * t3;
  }
  for (; r < n; r += st) {
    double t = w[r];
    for (int i = 0; i < cnt; ++i) t += cs[i] * V[(size_t)i * n + r];
    w[r] = t;
    nn += t * t;
  }
  if (part_nrm) block_partial(nn, part_nrm);
}

struct GmLayout {
  int m;
  __host__ __device__ int H(int i, int j) const { return S_GM + 16 + i * m + j; }
  __host__ __device__ int CS(int i) const { return S_GM + 16 + (m + 1) * m + i; }
  __host__ __device__ int SN(int i) const { return CS(m) + i; }
  __host__ __device__ int G(int i) const { return SN(m) + i; }
  __host__ __device__ int Y(int i) const { return G(m + 1) + i; }
  __host__ __device__ int H1(int i) const { return Y(m) + i; }
  __host__ __device__ int H2(int i) const { return H1(m + 1) + i; }
  __host__ __device__ int end() const { return H2(m + 1); }
};
enum { GM_BETA = S_GM, GM_IBETA, GM_EST, GM_IHN, GM_BAD, GM_REORTH };

__global__ void k_gm_start(double *sc, const double *part, int nb, GmLayout L) {
  const double r2 = sum_partials(slot((double *)part, P_R2), nb);
  if (threadIdx.x != 0) return;
  const double beta = sqrt(r2);
  sc[GM_BETA] = beta;
  sc[GM_IBETA] = beta > 0.0 ? 1.0 / beta : 0.0;
  sc[GM_EST] = beta;
  sc[GM_BAD] = isfinite(r2) ? 0.0 : 1.0;
  for (int i = 0; i <= L.m; ++i) sc[L.G(i)] = 0.0;
  sc[L.G(0)] = beta;
}

// H[:, j] = h1 + h2, H[j+1, j] = ||w||, apply the rotations, new rotation
// Second Gram-Schmidt pass only when the first lost too much: with w1 the
// vector after the first pass and h its coefficients, reorthogonalise iff
// ||w1|| < ||w0|| / sqrt(2), i.e. ||w1||^2 < ||h||^2 (||w0||^2 = ||w1||^2 +
// ||h||^2); the criterion of Daniel, Gragg, Kaufman & Stewart, Math. Comp. 30
// (1976).  Without it the second-pass coefficients are zero.
__global__ void k_gm_reorth_flag(double *sc, const double *part, int nb, int j, GmLayout L) {
  const double w2 = sum_partials(slot((double *)part, P_NRM), nb);
  if (threadIdx.x != 0) return;
  double h2 = 0.0;
  for (int i = 0; i <= j; ++i) h2 += sc[L.H1(i)] * sc[L.H1(i)];
  const bool again = !(w2 >= h2);   // also on NaN: the second pass then reports it
  sc[GM_REORTH] = again ? 1.0 : 0.0;
  if (!again)
    for (int i = 0; i <= j; ++i) sc[L.H2(i)] = 0.0;
}

__global__ void k_gm_givens(double *sc, const double *part, int nb, int j, GmLayout L) {
  const double w2 = sum_partials(slot((double *)part, P_NRM), nb);
  if (threadIdx.x != 0) return;
  for (int i = 0; i <= j; ++i) sc[L.H(i, j)] = sc[L.H1(i)] + sc[L.H2(i)];
  const double hn = sqrt(w2 > 0.0 ? w2 : 0.0);
  sc[GM_IHN] = hn > 0.0 ? 1.0 / hn : 0.0;
  for (int i = 0; i < j; ++i) {
    const double a = sc[L.H(i, j)], b = sc[L.H(i + 1, j)];
    const double c = sc[L.CS(i)], s = sc[L.SN(i)];
    sc[L.H(i, j)] = c * a + s * b;
    sc[L.H(i + 1, j)] = -s * a + c * b;
  }
  const double a = sc[L.H(j, j)];
  const double den = hypot(a, hn);
  if (!(den > 0.0) || !isfinite(den) || !isfinite(w2)) {
    sc[GM_BAD] = 1.0;
    return;
  }
  const double c = a / den, s = hn / den;
  sc[L.CS(j)] = c;
  sc[L.SN(j)] = s;
  sc[L.H(j, j)] = den;
  const double gj = sc[L.G(j)];
  sc[L.G(j + 1)] = -s * gj;
  sc[L.G(j)] = c * gj;
  sc[GM_EST] = fabs(sc[L.G(j + 1)]);
}

// back substitution H y = g for the leading k x k upper triangle
__global__ void k_gm_solve(double *sc, int k, GmLayout L) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double t = sc[L.G(i)];
    for (int q = i + 1; q < k; ++q) t -= sc[L.H(i, q)] * sc[L.Y(q)];
    sc[L.Y(i)] = t / sc[L.H(i, i)];
  }
}

// ------------------------------------------------------- preconditioner ---
// Block-Reg: A_reg and its AMG hierarchy for the current assembly, gamma and
// precision.
vem_status ensure_reg(vem_handle *h) {
  const bool fp32 = h->opt.precision == VEM_PRECISION_MIXED;
  const bool cond = h->opt.reg_cycle == VEM_REG_CONDENSED;
  if (cond && h->opt.element != VEM_ELEMENT_K1 && h->opt.element != VEM_ELEMENT_K2)
    return fail(h, VEM_ERR_UNSUPPORTED, "the condensed Block-Reg cycle needs the paper's k = 1 or k = 2 element");
  if (cond && fp32) return fail(h, VEM_ERR_UNSUPPORTED, "the condensed Block-Reg cycle runs in FP64 only");
  if (!h->areg_valid || (fp32 && !h->areg_has32)) VEM_TRY(assemble_reg(h, fp32));
  if (amg_valid(h->amg_reg) && amg_is_fp32(h->amg_reg) == fp32 && amg_is_condensed(h->amg_reg) == cond)
    return VEM_OK;
  if (cond) {
    // face DOFs first (nfd per face), nid interior DOFs per cell after them
    if (!h->fmodes) VEM_TRY(dalloc_n(h, &h->fmodes, 3 * (size_t)h->nfd * h->nf));
    if (h->nq > 1) VEM_TRY(flux_modes_k2(h, h->fmodes));
    else VEM_TRY(flux_modes_k1(h, h->nf, h->f_norm, h->fmodes));
    return amg_setup_condensed(h, h->amg_reg, h->Areg, (int64_t)h->nfd * h->nf, h->nid, h->nfd, h->fmodes, 3,
                               kSmoothChebyshev);
  }
  return amg_setup(h, h->amg_reg, h->Areg, h->Areg_val32, fp32, false, kSmoothChebyshev);
}

// z = P^{-1} v for the block preconditioner (diag, upper triangular or
// Block-Reg).  wk: 5 n_p PCG work vectors (FP64 units; the FP32 solve uses
// 6 n_p floats of it).  minres_partials (MINRES) also leaves the partials of
// v.z in slots P_G2U (flux part) and P_G2P (pressure part).
static vem_status precond(vem_handle *h, const VemOp &op, const double *v, double *z, double *wk, int *inner,
                          bool minres_partials) {
  cudaStream_t s = h->stream;
  const int64_t nu = op.n_u, np = op.n_p;
  int it = 0;
  if (h->opt.precond == VEM_PREC_BLOCK_REG) {
    // z_u = V(v_u), one V-cycle of the AMG of A_reg; z_p = v_p / gamma
    amg_vcycle(h, h->amg_reg, v, z, nullptr);
    if (minres_partials) dot_partials(s, nu, v, z, slot(h->part, P_G2U));
    count_launch();
    k_scale_dot<<<nblocks_vec(np), kRedThreads, 0, s>>>(np, v + nu, 1.0 / h->reg_gamma, z + nu,
                                                        minres_partials ? slot(h->part, P_G2P) : nullptr);
    VEM_CUDA(h, cudaGetLastError());
    return VEM_OK;
  }
  if (h->opt.precond == VEM_PREC_BLOCK_DIAG) {
    count_launch();
    k_diag_scale<<<nblocks_vec(nu), kRedThreads, 0, s>>>(nu, v, op.dinvM, z,
                                                         minres_partials ? slot(h->part, P_G2U) : nullptr);
    VEM_TRY(pcg_solve(h, op, v + nu, z + nu, wk, &it));
  } else {
    VEM_TRY(pcg_solve(h, op, v + nu, z + nu, wk, &it));
    count_launch(); k_negate<<<grid_for(np, 256), 256, 0, s>>>(np, z + nu);
    if (h->nq > 1) {
      count_launch();
      if (op.nbatch > 1)
        k_tri_flux_rows<true><<<grid_for(nu, 256), 256, 0, s>>>(nu, op.n_u1, op.n_p1, h->bt_col, h->bt_val, v,
                                                                 op.dinvM, z + nu, z);
      else
        k_tri_flux_rows<false><<<grid_for(nu, 256), 256, 0, s>>>(nu, nu, 0, h->bt_col, h->bt_val, v, op.dinvM,
                                                                  z + nu, z);
    } else {
      launch_tri_flux(s, h->nfd, op.nbatch > 1, h->nf, nu, op.n_u1, op.n_p1, v, op.dinvM, h->f_cell, h->bt_face,
                      z + nu, z);
    }
  }
  VEM_CUDA(h, cudaGetLastError());
  if (minres_partials)
    dot_partials(s, np, v + nu, z + nu, slot(h->part, P_G2P));
  *inner += it;
  return VEM_OK;
}

// true relative residual ||b - A x|| / ||b|| (synchronises)
// ||b - A x|| / ||b||, leaving b - A x in tmp and its partial sums in the
// P_R2 / P_B2 slots.  x_zero: x is known to be 0 (no SpMV).
static vem_status true_relres(vem_handle *h, const VemOp &op, const double *rhs, const double *x, double *tmp,
                              double *rel, bool x_zero = false) {
  cudaStream_t s = h->stream;
  const int64_t n = op.n;
  if (!x_zero) op_apply_timed(h, op, x, tmp);
  const int nb = nblocks_vec(n);
  count_launch(); k_residual<<<nb, kRedThreads, 0, s>>>(n, rhs, x_zero ? nullptr : tmp, tmp, slot(h->part, P_R2),
                                                         slot(h->part, P_B2));
  count_launch(); k_read_sum<<<1, kRedThreads, 0, s>>>(slot(h->part, P_R2), nb, h->scal + S_R2);
  count_launch(); k_read_sum<<<1, kRedThreads, 0, s>>>(slot(h->part, P_B2), nb, h->scal + S_B2);
  VEM_CUDA(h, cudaGetLastError());
  VEM_CUDA(h, cudaMemcpyAsync(h->h_scal + S_R2, h->scal + S_R2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaStreamSynchronize(s));
  const double r2 = h->h_scal[S_R2], b2 = h->h_scal[S_B2];
  if (!std::isfinite(r2)) return fail(h, VEM_ERR_NONFINITE, "non-finite residual");
  *rel = b2 > 0.0 ? std::sqrt(r2 / b2) : std::sqrt(r2);
  return VEM_OK;
}

// ------------------------------------------------------------- drivers ---
static vem_status ensure_work(vem_handle *h, size_t n) {
  if (h->work_n >= n) return VEM_OK;
  dfree(h, h->work);
  h->work = nullptr;
  h->work_n = 0;
  VEM_TRY(dalloc_n(h, &h->work, n));
  h->work_n = n;
  return VEM_OK;
}

static vem_status run_minres(vem_handle *h, const VemOp &op, const double *rhs, double *x, vem_stats *st) {
  cudaStream_t s = h->stream;
  const int64_t n = op.n, nu = op.n_u, np = op.n_p;
  VEM_TRY(ensure_work(h, 8 * (size_t)n + 5 * (size_t)np));
  double *vA = h->work, *vB = vA + n, *z = vB + n, *zn = z + n, *Az = zn + n, *wA = Az + n,
         *wB = wA + n, *tmp = wB + n, *pw = tmp + n;
  double *vold = vA, *v = vB, *wold = wA, *w = wB;
  int inner = 0;
  const int nbn = nblocks_vec(n), nbu = nblocks_vec(nu), nbp = nblocks_vec(np);
  // v = b - A x0
  op_apply_timed(h, op, x, tmp);
  count_launch(); k_residual<<<nbn, kRedThreads, 0, s>>>(n, rhs, tmp, v, slot(h->part, P_R2), slot(h->part, P_B2));
  VEM_CUDA(h, cudaMemsetAsync(vold, 0, sizeof(double) * n, s));
  VEM_CUDA(h, cudaMemsetAsync(wold, 0, sizeof(double) * n, s));
  VEM_CUDA(h, cudaMemsetAsync(w, 0, sizeof(double) * n, s));
  VEM_TRY(precond(h, op, v, z, pw, &inner, true));
  count_launch(); k_mr_init<<<1, kRedThreads, 0, s>>>(h->scal, h->part, nbu, nbp);
  VEM_CUDA(h, cudaGetLastError());
  double rel = 1.0;
  VEM_TRY(true_relres(h, op, rhs, x, tmp, &rel));
  VEM_CUDA(h, cudaMemcpyAsync(h->h_scal + S_MR, h->scal + S_MR, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaStreamSynchronize(s));
  const double eta0 = h->h_scal[S_MR + MR_ETA];
  int it = 0;
  const int nbd = spmv_nblocks(op.A, op.nbatch);
  vem_status result = VEM_ERR_NOT_CONVERGED;
  if (rel <= h->opt.rtol || eta0 == 0.0) result = VEM_OK;
  while (result != VEM_OK && it < h->opt.maxit) {
    ++it;
    count_launch(); k_scale_by<<<grid_for(n, 256), 256, 0, s>>>(n, z, h->scal + S_MR + MR_IG);
    op_apply_timed(h, op, z, Az, slot(h->part, P_DELTA));
    count_launch(); k_mr_lanczos<<<nbn, kRedThreads, 0, s>>>(n, Az, v, vold, h->part, nbd, h->scal);
    VEM_TRY(precond(h, op, vold, zn, pw, &inner, true));
    count_launch(); k_mr_scalars<<<1, kRedThreads, 0, s>>>(h->scal, h->part, nbd, nbu, nbp);
    count_launch(); k_mr_update<<<grid_for(n, 256), 256, 0, s>>>(n, z, wold, w, x, h->scal);
    VEM_CUDA(h, cudaGetLastError());
    // rotate: v_old <- v, v <- v_new (in v_old's buffer); w likewise
    std::swap(vold, v);
    std::swap(wold, w);
    std::swap(z, zn);
    VEM_CUDA(h, cudaMemcpyAsync(h->h_scal + S_MR, h->scal + S_MR, 16 * sizeof(double), cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    const double *m = h->h_scal + S_MR;
    if (debug_on())
      fprintf(stderr, "[vem] minres it=%d eta=%.3e eta0=%.3e gamma=%.3e a1=%.3e bad=%g inner=%d\n", it,
              m[MR_ETA], eta0, m[MR_G], m[MR_A1], m[MR_BAD], inner);
    if (m[MR_BAD] != 0.0)
      return fail(h, m[MR_BAD] == 1.0 ? VEM_ERR_NONFINITE : VEM_ERR_BREAKDOWN, "MINRES breakdown");
    const bool lucky = m[MR_G] == 0.0;
    if (std::fabs(m[MR_ETA]) <= 0.5 * h->opt.rtol * eta0 || lucky) {
      VEM_TRY(true_relres(h, op, rhs, x, tmp, &rel));
      if (rel <= h->opt.rtol) result = VEM_OK;
      else if (lucky) break;
    }
  }
  if (result != VEM_OK) VEM_TRY(true_relres(h, op, rhs, x, tmp, &rel));
  st->iterations = it;
  st->inner_iterations = inner;
  st->relres = rel;
  if (result != VEM_OK) return fail(h, VEM_ERR_NOT_CONVERGED, "MINRES: relres %.3e after %d iterations", rel, it);
  return VEM_OK;
}

static vem_status run_fgmres(vem_handle *h, const VemOp &op, const double *rhs, double *x, vem_stats *st) {
  cudaStream_t s = h->stream;
  const int64_t n = op.n, np = op.n_p;
  const int m = h->opt.restart;
  GmLayout L{m};
  if (L.end() > 8192) return fail(h, VEM_ERR_BAD_INPUT, "restart too large");
  VEM_TRY(ensure_work(h, (size_t)(2 * m + 2) * n + 5 * (size_t)np));
  double *V = h->work, *Z = V + (size_t)(m + 1) * n, *tmp = Z + (size_t)m * n, *pw = tmp + n;
  int inner = 0, it = 0;
  const int nbn = nblocks_vec(n);
  double rel = 1.0;
  VEM_TRY(true_relres(h, op, rhs, x, tmp, &rel, h->x_zero));
  h->x_zero = false;
  vem_status result = rel <= h->opt.rtol ? VEM_OK : VEM_ERR_NOT_CONVERGED;
  double bnorm = std::sqrt(h->h_scal[S_B2]);
  if (bnorm == 0.0) bnorm = 1.0;
  while (result != VEM_OK && it < h->opt.maxit) {
    // V_0 = (b - A x) / beta: the residual and its partial sums are those of
    // the last true_relres (x has not changed since)
    VEM_CUDA(h, cudaMemcpyAsync(V, tmp, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    count_launch(); k_gm_start<<<1, kRedThreads, 0, s>>>(h->scal, h->part, nbn, L);
    count_launch(); k_scale_by<<<grid_for(n, 256), 256, 0, s>>>(n, V, h->scal + GM_IBETA);
    int jd = 0;
    for (int j = 0; j < m && it < h->opt.maxit; ++j) {
      ++it;
      double *Vj = V + (size_t)j * n, *Zj = Z + (size_t)j * n, *w = V + (size_t)(j + 1) * n;
      VEM_TRY(precond(h, op, Vj, Zj, pw, &inner, false));
      op_apply_timed(h, op, Zj, w);
      // classical Gram-Schmidt, the second pass on the device's decision
      for (int pass = 0; pass < 2; ++pass) {
        const double *skip = pass == 1 ? h->scal + GM_REORTH : nullptr;
        for (int i0 = 0; i0 <= j; i0 += kMD) {
          const int cnt = (j + 1 - i0) < kMD ? (j + 1 - i0) : kMD;
          count_launch(); k_multidot<<<nbn, kRedThreads, 0, s>>>(n, V, i0, cnt, w, h->part, skip);
        }
        double *hc = h->scal + (pass == 0 ? L.H1(0) : L.H2(0));
        count_launch(); k_multidot_fin<<<j + 1, kRedThreads, 0, s>>>(h->part, nbn, hc, skip);
        count_launch(); k_multiaxpy<<<nbn, kRedThreads, 0, s>>>(n, V, j + 1, hc, -1.0, w, slot(h->part, P_NRM),
                                                                 skip);
        if (pass == 0) {
          count_launch(); k_gm_reorth_flag<<<1, kRedThreads, 0, s>>>(h->scal, h->part, nbn, j, L);
        }
      }
      count_launch(); k_gm_givens<<<1, kRedThreads, 0, s>>>(h->scal, h->part, nbn, j, L);
      count_launch(); k_scale_by<<<grid_for(n, 256), 256, 0, s>>>(n, w, h->scal + GM_IHN);
      VEM_CUDA(h, cudaGetLastError());
      VEM_CUDA(h, cudaMemcpyAsync(h->h_scal + S_GM, h->scal + S_GM, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
      VEM_CUDA(h, cudaStreamSynchronize(s));
      if (h->h_scal[GM_BAD] != 0.0) {
        // an exactly converged Krylov space (zero new direction) is not an error
        if (h->h_scal[GM_EST] == 0.0) { jd = j + 1; break; }
        return fail(h, VEM_ERR_BREAKDOWN, "FGMRES breakdown at iteration %d", it);
      }
      jd = j + 1;
      if (debug_on())
        fprintf(stderr, "[vem] fgmres it=%d est=%.3e bnorm=%.3e inner=%d\n", it, h->h_scal[GM_EST], bnorm, inner);
      if (h->h_scal[GM_EST] <= 0.5 * h->opt.rtol * bnorm) break;
    }
    count_launch(); k_gm_solve<<<1, 32, 0, s>>>(h->scal, jd, L);
    count_launch(); k_multiaxpy<<<nbn, kRedThreads, 0, s>>>(n, Z, jd, h->scal + L.Y(0), 1.0, x, nullptr);
    VEM_CUDA(h, cudaGetLastError());
    VEM_TRY(true_relres(h, op, rhs, x, tmp, &rel));
    if (rel <= h->opt.rtol) result = VEM_OK;
  }
  st->iterations = it;
  st->inner_iterations = inner;
  st->relres = rel;
  if (result != VEM_OK) return fail(h, VEM_ERR_NOT_CONVERGED, "FGMRES: relres %.3e after %d iterations", rel, it);
  return VEM_OK;
}

// ----------------------------------------------- per-system batched solve --
// nb systems stacked as [u_0 .. u_{nb-1} | p_0 .. p_{nb-1}] (n_u1 flux and
// n_p1 pressure unknowns each).  Every system runs its own FGMRES(m) (its
// own Arnoldi basis coefficients, Givens rotations, stopping test and
// iteration count) and its own inner Jacobi-PCG on its Schur block (its own
// alpha, beta and convergence test); the launches serve all systems at once
// and converged systems are skipped.  Reductions are per system in a fixed
// order: a grid of P x nb blocks writes partial sums, a second pass adds them.

// global row of the t-th unknown (u part, then p part) of system b
__device__ __forceinline__ int64_t sys_row(int64_t t, int b, int nb, int64_t n_u1, int64_t n_p1) {
  return t < n_u1 ? (int64_t)b * n_u1 + t : (int64_t)nb * n_u1 + (int64_t)b * n_p1 + (t - n_u1);
}

// part[(b P + p) K + k] = partial sums of V_{i0+k} . w over system b (K <= 8)
__global__ void __launch_bounds__(256) k_sys_dots(int nb, int64_t n_u1, int64_t n_p1, int64_t N, const double *V,
                                                  int i0, int K, const double *__restrict__ w, double *part,
                                                  const double *skip) {
  __shared__ double sh[8][8];
  if (skip && skip[0] == 0.0) return;
  const int b = blockIdx.y, P = gridDim.x, pb = blockIdx.x;
  const int64_t n1 = n_u1 + n_p1;
  double acc[8];
  for (int k = 0; k < 8; ++k) acc[k] = 0.0;
  for (int64_t t = (int64_t)pb * blockDim.x + threadIdx.x; t < n1; t += (int64_t)P * blockDim.x) {
    const int64_t g = sys_row(t, b, nb, n_u1, n_p1);
    const double wv = w[g];
    for (int k = 0; k < K; ++k) acc[k] += V[(int64_t)(i0 + k) * N + g] * wv;
  }
  const int wi = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int k = 0; k < K; ++k) {
    const double v = warp_sum(acc[k]);
    if (l == 0) sh[k][wi] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[threadIdx.x][q];
    part[((int64_t)b * P + pb) * K + threadIdx.x] = t;
  }
}

// out[b ld + o + k] = sum_p part[(b P + p) K + k]
__global__ void k_sys_dots_fin(int nb, int P, int K, const double *__restrict__ part, double *out, int ld, int o,
                               const double *skip) {
  if (skip && skip[0] == 0.0) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nb * K) return;
  const int b = (int)(t / K), k = (int)(t % K);
  double s = 0.0;
  for (int p = 0; p < P; ++p) s += part[((int64_t)b * P + p) * K + k];
  out[(int64_t)b * ld + o + k] = s;
}

// w[g] += sgn sum_{j < J} coef[b ld + j] V_j[g] for the rows g of every system b
__global__ void k_sys_axpy(int nb, int64_t n_u1, int64_t n_p1, int64_t N, int J, const double *__restrict__ V,
                           const double *__restrict__ coef, int ld, double sgn, double *w, const double *skip) {
  if (skip && skip[0] == 0.0) return;
  const int64_t nu = (int64_t)nb * n_u1;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(g < nu ? g / n_u1 : (g - nu) / n_p1);
    const double *c = coef + (int64_t)b * ld;
    double s = 0.0;
    for (int j = 0; j < J; ++j) s += c[j] * V[(int64_t)j * N + g];
    w[g] += sgn * s;
  }
}

// y[g] = fac[b] x[g]
__global__ void k_sys_scale(int nb, int64_t n_u1, int64_t n_p1, int64_t N, const double *__restrict__ x,
                            const double *__restrict__ fac, int ld, double *y) {
  const int64_t nu = (int64_t)nb * n_u1;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(g < nu ? g / n_u1 : (g - nu) / n_p1);
    y[g] = fac[(int64_t)b * ld] * x[g];
  }
}

// ---- the per-system inner Jacobi-PCG on the stacked Schur blocks ----
// Per-system scalars at bsc[k nb + b]: the slots below; flag[0] = all done.
enum { BC_ALPHA = 0, BC_BETA, BC_GPREV, BC_APREV, BC_BB, BC_IT, BC_DONE, BC_BAD, BC_N };

__device__ __forceinline__ bool all_done(const double *flag) {
  __shared__ int f;
  if (threadIdx.x == 0) f = flag[0] != 0.0;
  __syncthreads();
  const bool r = f != 0;
  __syncthreads();
  return r;
}

// x = 0, r = b, u = D^-1 r, p = s = 0; partials of (b, b) per system (grid P x nb)
template <class T>
__global__ void __launch_bounds__(256) k_bcg_init(int nb, int64_t n1, const double *__restrict__ b,
                                                  const T *__restrict__ dinv, T *x, T *r, T *u, T *p, T *s,
                                                  double *part, double *bsc, const double *__restrict__ active,
                                                  int lda, double *flag) {
  __shared__ double sh[8];
  const int sb = blockIdx.y, P = gridDim.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // this solve's state: systems whose outer iteration is inactive are done
    bsc[BC_DONE * nb + sb] = active[(int64_t)sb * lda] != 0.0 ? 0.0 : 1.0;
    bsc[BC_IT * nb + sb] = 0.0;
    bsc[BC_BAD * nb + sb] = 0.0;
    if (sb == 0) flag[0] = 0.0;
  }
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n1; t += (int64_t)P * blockDim.x) {
    const int64_t i = (int64_t)sb * n1 + t;
    const T bt = (T)b[i];
    x[i] = 0;
    r[i] = bt;
    u[i] = dinv[i] * bt;
    p[i] = 0;
    s[i] = 0;
    acc += (double)bt * (double)bt;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    part[(int64_t)sb * P + blockIdx.x] = t;
  }
}

// w = S u for every system not done, with per-(system, slice) partials of
// (r, u) and (w, u): part_ru[b nsl + s], part_wu[b nsl + s].  A warp task is
// a tile of kS consecutive 32-row slices of kR consecutive systems: each
// column id is read once for kR value streams and gathers, and a thread
// carries kS x kR independent sums.  Tasks whose systems are all done are
// skipped.  flag == nullptr: the autotuner's timing launches (every system
// taken as live).
template <class T, int kR, int kS>
__global__ void __launch_bounds__(256) k_bcg_spmv(int nb, int64_t rows, int64_t nsl, int64_t stored,
                                                  const int64_t *__restrict__ off, const int32_t *__restrict__ col,
                                                  const T *__restrict__ val, const T *__restrict__ u,
                                                  const T *__restrict__ r, T *w, double *part_ru, double *part_wu,
                                                  const double *bsc, const double *flag) {
  if (flag && all_done(flag)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t groups = (nb + kR - 1) / kR, stiles = (nsl + kS - 1) / kS;
  for (int64_t tk = warp; tk < stiles * groups; tk += nwarps) {
    const int64_t g = tk / stiles, st0 = (tk - g * stiles) * kS;
    const int b0 = (int)(g * kR);
    bool live[kR];
    bool any = false;
#pragma unroll
    for (int q = 0; q < kR; ++q) {
      live[q] = (b0 + q < nb) && (!flag || bsc[BC_DONE * nb + b0 + q] == 0.0);
      any = any || live[q];
    }
    if (!any) continue;   // uniform over the warp
#pragma unroll
    for (int k = 0; k < kS; ++k) {
      const int64_t sl = st0 + k;
      if (sl >= nsl) break;
      const int64_t o = off[sl];
      const int wdt = (int)((off[sl + 1] - o) >> 5);
      T acc[kR];
#pragma unroll
      for (int q = 0; q < kR; ++q) acc[q] = 0;
      // kB entries per step (predicated on the slice width): their column
      // ids first, then the kR x kB values and gathers, then the FMAs
      constexpr int kB = kR >= 8 ? 1 : 8 / kR;
      for (int j = 0; j < wdt; j += kB) {
        int32_t c[kB];
#pragma unroll
        for (int t = 0; t < kB; ++t) c[t] = (j + t < wdt) ? __ldcs(col + o + 32 * (int64_t)(j + t) + lane) : 0;
        T v[kR][kB], xg[kR][kB];
#pragma unroll
        for (int q = 0; q < kR; ++q)
#pragma unroll
          for (int t = 0; t < kB; ++t) {
            const bool ok = live[q] && (j + t < wdt);
            v[q][t] = ok ? __ldcs(val + (int64_t)(b0 + q) * stored + o + 32 * (int64_t)(j + t) + lane) : T(0);
            xg[q][t] = ok ? __ldg(u + (int64_t)(b0 + q) * rows + c[t]) : T(0);
          }
#pragma unroll
        for (int q = 0; q < kR; ++q)
#pragma unroll
          for (int t = 0; t < kB; ++t) acc[q] += v[q][t] * xg[q][t];
      }
      const int64_t i = 32 * sl + lane;
#pragma unroll
      for (int q = 0; q < kR; ++q) {
        if (!live[q]) continue;
        // products and the warp's sums in T (no FP64 work per row in the
        // FP32 form); one conversion per slice
        T gam = 0, del = 0;
        if (i < rows) {
          const int64_t gi = (int64_t)(b0 + q) * rows + i;
          w[gi] = acc[q];
          gam = r[gi] * u[gi];
          del = acc[q] * u[gi];
        }
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
          gam += __shfl_xor_sync(0xffffffffu, gam, o2);
          del += __shfl_xor_sync(0xffffffffu, del, o2);
        }
        if (lane == 0) {
          part_ru[(int64_t)(b0 + q) * nsl + sl] = (double)gam;
          part_wu[(int64_t)(b0 + q) * nsl + sl] = (double)del;
        }
      }
    }
  }
}

// One launch of the per-system Schur SpMV with the tile code 100 kS + kR.
template <class T, int kR, int kS>
static void bspmv_launch_t(cudaStream_t s, int nb, const VemOp &op, const T *sval, const T *u, const T *r, T *w,
                           double *ru, double *wu, const double *bsc, const double *flag) {
  static int cap = 0;
  if (cap == 0) cap = one_wave_blocks((const void *)k_bcg_spmv<T, kR, kS>);
  const int64_t nsl = op.S.nslices;
  int64_t g = (((nsl + kS - 1) / kS) * ((nb + kR - 1) / kR) + 7) / 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  count_launch();
  k_bcg_spmv<T, kR, kS><<<(int)g, 256, 0, s>>>(nb, op.n_p1, nsl, op.S.stored, op.S.off, op.S.col, sval, u, r, w, ru,
                                               wu, bsc, flag);
}

template <class T>
static void bspmv_launch(cudaStream_t s, int tile, int nb, const VemOp &op, const T *sval, const T *u, const T *r,
                         T *w, double *ru, double *wu, const double *bsc, const double *flag) {
  switch (tile) {
    case 101: bspmv_launch_t<T, 1, 1>(s, nb, op, sval, u, r, w, ru, wu, bsc, flag); break;
    case 102: bspmv_launch_t<T, 2, 1>(s, nb, op, sval, u, r, w, ru, wu, bsc, flag); break;
    case 108: bspmv_launch_t<T, 8, 1>(s, nb, op, sval, u, r, w, ru, wu, bsc, flag); break;
    case 201: bspmv_launch_t<T, 1, 2>(s, nb, op, sval, u, r, w, ru, wu, bsc, flag); break;
    case 202: bspmv_launch_t<T, 2, 2>(s, nb, op, sval, u, r, w, ru, wu, bsc, flag); break;
    case 204: bspmv_launch_t<T, 4, 2>(s, nb, op, sval, u, r, w, ru, wu, bsc, flag); break;
    case 208: bspmv_launch_t<T, 8, 2>(s, nb, op, sval, u, r, w, ru, wu, bsc, flag); break;
    default: bspmv_launch_t<T, 4, 1>(s, nb, op, sval, u, r, w, ru, wu, bsc, flag); break;
  }
}

// Autotuner of the per-system Schur SpMV's tile (32 or 64 rows x 1, 2, 4 or 8
// systems): on the first solve of a shape (rows, slices, systems, value
// type) every tile runs three timed launches on the live vectors (after one
// warm-up; every system taken as live), with CUDA events on the stream; the
// fastest is kept for the process (per device and shape; a mutex guards the
// shared cache).  The launches write only w and the partial sums, which the
// solve recomputes before reading.
template <class T>
static int tune_bspmv(vem_handle *h, int nb, const VemOp &op, const T *sval, const T *u, const T *r, T *w,
                      double *ru, double *wu) {
  static std::mutex mu;
  static std::map<std::tuple<int, int64_t, int64_t, int, int>, int> best;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, op.S.rows, op.S.nslices, nb, (int)sizeof(T));
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = best.find(key);
    if (it != best.end()) return it->second;
  }
  int pick = 104;
  float pick_ms = 1e30f;
  for (int tile : {101, 102, 104, 108, 201, 202, 204, 208}) {
    if (tile % 100 > 1 && tile % 100 > nb) continue;
    bspmv_launch<T>(h->stream, tile, nb, op, sval, u, r, w, ru, wu, nullptr, nullptr);
    cudaEventRecord(h->ev2, h->stream);
    for (int k = 0; k < 3; ++k) bspmv_launch<T>(h->stream, tile, nb, op, sval, u, r, w, ru, wu, nullptr, nullptr);
    cudaEventRecord(h->ev3, h->stream);
    cudaEventSynchronize(h->ev3);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev2, h->ev3) == cudaSuccess && ms < pick_ms) {
      pick_ms = ms;
      pick = tile;
    }
  }
  cudaGetLastError();
  {
    std::lock_guard<std::mutex> lk(mu);
    best[key] = pick;
  }
  if (debug_on()) fprintf(stderr, "[vem] per-system Schur SpMV tile: %d (%.3f ms / 3)\n", pick, pick_ms);
  return pick;
}

// p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = D^-1 r for
// every system not done; partials of (r, r) per system (grid P x nb)
template <class T>
__global__ void __launch_bounds__(256) k_bcg_update(int nb, int64_t n1, T *x, T *r, T *u, T *p, T *s,
                                                    const T *__restrict__ w, const T *__restrict__ dinv,
                                                    const double *bsc, double *part, const double *flag) {
  __shared__ double sh[8];
  if (all_done(flag)) return;
  const int sb = blockIdx.y, P = gridDim.x;
  if (bsc[BC_DONE * nb + sb] != 0.0) return;   // uniform over the block
  const T alpha = (T)bsc[BC_ALPHA * nb + sb], beta = (T)bsc[BC_BETA * nb + sb];
  T acct = 0;   // (r, r) of this thread's rows in T, as the single-system update
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n1; t += (int64_t)P * blockDim.x) {
    const int64_t i = (int64_t)sb * n1 + t;
    const T pi = u[i] + beta * p[i];
    const T si = w[i] + beta * s[i];
    x[i] += alpha * pi;
    const T ri = r[i] - alpha * si;
    p[i] = pi;
    s[i] = si;
    r[i] = ri;
    u[i] = dinv[i] * ri;
    acct += ri * ri;
  }
  double acc = warp_sum((double)acct);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    part[(int64_t)sb * P + blockIdx.x] = t;
  }
}

// One block per system: (r,u), (w,u) over its slices and (r,r) over its
// update partials, in a fixed order; then the convergence test, alpha and
// beta (the recurrences of the single-system form).  init != 0: the first
// call after k_bcg_init ((r, r) = (b, b) is also stored as BC_BB).  The last
// block to finish sets flag[0] = 1 when every system is done and flag[1] to
// the largest iteration count (ctr: a zeroed counter, reset by that block).
__global__ void __launch_bounds__(256) k_bcg_scalars(int nb, int64_t nsl, int P, const double *__restrict__ part_ru,
                                                     const double *__restrict__ part_wu,
                                                     const double *__restrict__ part_rr, double tol2, double *bsc,
                                                     int init, double *flag, unsigned int *ctr) {
  __shared__ double sh[3][8];
  __shared__ int open;
  __shared__ unsigned long long mx;
  if (all_done(flag)) return;   // uniform over the grid
  const int b = blockIdx.x;
  const bool skip = !init && bsc[BC_DONE * nb + b] != 0.0;
  double g = 0.0, d = 0.0, rr = 0.0;
  if (!skip) {
    for (int64_t s2 = threadIdx.x; s2 < nsl; s2 += blockDim.x) {
      g += part_ru[(int64_t)b * nsl + s2];
      d += part_wu[(int64_t)b * nsl + s2];
    }
    for (int p = threadIdx.x; p < P; p += blockDim.x) rr += part_rr[(int64_t)b * P + p];
  }
  g = warp_sum(g);
  d = warp_sum(d);
  rr = warp_sum(rr);
  const int wi = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sh[0][wi] = g;
    sh[1][wi] = d;
    sh[2][wi] = rr;
  }
  __syncthreads();
  if (threadIdx.x == 0 && !skip) {
    double G = 0.0, D = 0.0, R = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      G += sh[0][q];
      D += sh[1][q];
      R += sh[2][q];
    }
    bool go = true;
    if (init) {
      bsc[BC_BB * nb + b] = R;
      if (R == 0.0) bsc[BC_DONE * nb + b] = 1.0;
      go = bsc[BC_DONE * nb + b] == 0.0;
    }
    if (go) {
      const int it = (int)bsc[BC_IT * nb + b];
      if (!isfinite(R) || !isfinite(G) || !isfinite(D)) {
        bsc[BC_BAD * nb + b] = 2.0;
        bsc[BC_DONE * nb + b] = 1.0;
      } else if (R <= tol2 * bsc[BC_BB * nb + b]) {
        bsc[BC_DONE * nb + b] = 1.0;
      } else {
        double beta = 0.0, den = D;
        if (it > 0) {
          beta = G / bsc[BC_GPREV * nb + b];
          den = D - beta * G / bsc[BC_APREV * nb + b];
        }
        if (!(den > 0.0) || !(G > 0.0)) {
          bsc[BC_BAD * nb + b] = 1.0;
          bsc[BC_DONE * nb + b] = 1.0;
        } else {
          const double alpha = G / den;
          bsc[BC_ALPHA * nb + b] = alpha;
          bsc[BC_BETA * nb + b] = beta;
          bsc[BC_GPREV * nb + b] = G;
          bsc[BC_APREV * nb + b] = alpha;
          bsc[BC_IT * nb + b] = (double)(it + 1);
        }
      }
    }
  }
  if (!last_block(ctr)) return;
  if (threadIdx.x == 0) {
    open = 0;
    mx = 0ull;
  }
  __syncthreads();
  int c = 0;
  double m = 0.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) {
    c += bsc[BC_DONE * nb + q] == 0.0;
    m = fmax(m, bsc[BC_IT * nb + q]);
  }
  atomicAdd(&open, c);
  atomicMax(&mx, (unsigned long long)__double_as_longlong(m));
  __syncthreads();
  if (threadIdx.x == 0) {
    flag[0] = open == 0 ? 1.0 : 0.0;
    flag[1] = __longlong_as_double((long long)mx);
  }
}

// ---- the per-system FGMRES scalars ----
// Per system b at gs + b L: H ((m+1) x m, row-major), cs[m], sn[m], g[m+1],
// y[m], then the slots below.
enum { GS_BETA = 0, GS_BNORM, GS_EST, GS_ACTIVE, GS_JD, GS_DONE, GS_IT, GS_FAC, GS_REL, GS_N };
struct SysLayout {
  int m;
  __host__ __device__ int H(int i, int j) const { return i * m + j; }
  __host__ __device__ int CS(int i) const { return (m + 1) * m + i; }
  __host__ __device__ int SN(int i) const { return (m + 1) * m + m + i; }
  __host__ __device__ int G(int i) const { return (m + 1) * m + 2 * m + i; }
  __host__ __device__ int Y(int i) const { return (m + 1) * m + 3 * m + 1 + i; }
  __host__ __device__ int S(int k) const { return (m + 1) * m + 4 * m + 1 + k; }
  __host__ __device__ int size() const { return (m + 1) * m + 4 * m + 1 + GS_N; }
};

// Restart: beta = ||r_b||, ||b_b||, the relative residual, the stopping test;
// g = beta e_1 and the scale 1 / beta of the new basis vector.  first: the
// first cycle of the solve (sets the iteration count to 0).
__global__ void k_sys_start(int nb, SysLayout L, double rtol, const double *__restrict__ dd, int ldd, int orr,
                            int obb, double *gs, int first) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double *q = gs + (int64_t)b * L.size();
  const double rr = dd[(int64_t)b * ldd + orr], bb = dd[(int64_t)b * ldd + obb];
  const double beta = sqrt(fmax(rr, 0.0)), bn = sqrt(fmax(bb, 0.0));
  const double rel = bn > 0.0 ? beta / bn : beta;
  q[L.S(GS_BETA)] = beta;
  q[L.S(GS_BNORM)] = bn;
  q[L.S(GS_REL)] = rel;
  if (first) q[L.S(GS_IT)] = 0.0;
  const bool done = !(rel > rtol) || beta == 0.0;
  q[L.S(GS_DONE)] = done ? 1.0 : 0.0;
  q[L.S(GS_ACTIVE)] = done ? 0.0 : 1.0;
  q[L.S(GS_JD)] = 0.0;
  q[L.S(GS_FAC)] = done ? 0.0 : 1.0 / beta;
  for (int i = 0; i <= L.m; ++i) q[L.G(i)] = 0.0;
  q[L.G(0)] = beta;
}

// The second Gram-Schmidt pass where the first lost too much (the DGKS test
// of Daniel, Gragg, Kaufman & Stewart, 1976): system b repeats the pass when
// ||w|| after the first is below 0.7 of ||w|| before it (dd at ob and on);
// ro[b] = 1 then; flag[0] = 1 when any system needs it.  Systems without the
// second pass get zero second-pass coefficients.
__global__ void k_sys_reorth(int nb, const double *__restrict__ active, int lda, double *dd, int ldd, int ob, int on,
                             int o2, int jp1, double *ro, double *flag) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int a = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double *h = dd + (int64_t)b * ldd;
    const bool need = active[(int64_t)b * lda] != 0.0 && h[on] < 0.49 * h[ob];
    ro[b] = need ? 1.0 : 0.0;
    a |= need;
  }
  if (a) atomicOr(&any, 1);
  __syncthreads();
  if (threadIdx.x == 0) flag[0] = any ? 1.0 : 0.0;
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (ro[b] == 0.0)
      for (int i = 0; i < jp1; ++i) dd[(int64_t)b * ldd + o2 + i] = 0.0;
}

// Column j of H from the two Gram-Schmidt passes (hh: pass 1 at o1, pass 2
// at o2, ||w||^2 at on, row b at dd + b ldd), the Givens rotations and the
// stopping test of every active system; the scale of V_{j+1}.
__global__ void k_sys_arnoldi(int nb, int j, SysLayout L, double rtol, const double *__restrict__ dd, int ldd, int o1,
                              int o2, int on, double *gs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double *q = gs + (int64_t)b * L.size();
  if (q[L.S(GS_ACTIVE)] == 0.0) {
    q[L.S(GS_FAC)] = 0.0;
    return;
  }
  const double *h = dd + (int64_t)b * ldd;
  for (int i = 0; i <= j; ++i) q[L.H(i, j)] = h[o1 + i] + h[o2 + i];
  const double hn = sqrt(fmax(h[on], 0.0));
  for (int i = 0; i < j; ++i) {
    const double t = q[L.CS(i)] * q[L.H(i, j)] + q[L.SN(i)] * q[L.H(i + 1, j)];
    q[L.H(i + 1, j)] = -q[L.SN(i)] * q[L.H(i, j)] + q[L.CS(i)] * q[L.H(i + 1, j)];
    q[L.H(i, j)] = t;
  }
  const double hjj = q[L.H(j, j)];
  const double den = sqrt(hjj * hjj + hn * hn);
  const double c = den > 0.0 ? hjj / den : 1.0, sn = den > 0.0 ? hn / den : 0.0;
  q[L.CS(j)] = c;
  q[L.SN(j)] = sn;
  q[L.H(j, j)] = den;
  q[L.G(j + 1)] = -sn * q[L.G(j)];
  q[L.G(j)] = c * q[L.G(j)];
  const double est = fabs(q[L.G(j + 1)]);
  q[L.S(GS_EST)] = est;
  q[L.S(GS_IT)] += 1.0;
  q[L.S(GS_JD)] = (double)(j + 1);
  const bool stop = est <= 0.5 * rtol * q[L.S(GS_BNORM)] || hn == 0.0 || den == 0.0;
  if (stop) q[L.S(GS_ACTIVE)] = 0.0;
  q[L.S(GS_FAC)] = (!stop && hn > 0.0) ? 1.0 / hn : 0.0;
}

// y = H^-1 g on the first jd columns (upper triangular), 0 beyond
__global__ void k_sys_solve(int nb, SysLayout L, double *gs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  double *q = gs + (int64_t)b * L.size();
  const int jd = (int)q[L.S(GS_JD)];
  for (int i = L.m - 1; i >= 0; --i) {
    if (i >= jd) {
      q[L.Y(i)] = 0.0;
      continue;
    }
    double v = q[L.G(i)];
    for (int k = i + 1; k < jd; ++k) v -= q[L.H(i, k)] * q[L.Y(k)];
    q[L.Y(i)] = q[L.H(i, i)] != 0.0 ? v / q[L.H(i, i)] : 0.0;
  }
}

// out[0] = systems still active in the cycle, out[1] = systems not done,
// out[2] = the largest iteration count
__global__ void k_sys_flags(int nb, SysLayout L, const double *__restrict__ gs, double *out) {
  __shared__ int na, nn;
  __shared__ unsigned long long mx;
  if (threadIdx.x == 0) {
    na = 0;
    nn = 0;
    mx = 0ull;
  }
  __syncthreads();
  int a = 0, d = 0;
  double m = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const double *q = gs + (int64_t)b * L.size();
    a += q[L.S(GS_ACTIVE)] != 0.0;
    d += q[L.S(GS_DONE)] == 0.0;
    m = fmax(m, q[L.S(GS_IT)]);
  }
  atomicAdd(&na, a);
  atomicAdd(&nn, d);
  atomicMax(&mx, (unsigned long long)__double_as_longlong(m));
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = na;
    out[1] = nn;
    out[2] = __longlong_as_double((long long)mx);
  }
}

// r = b - A x
__global__ void k_sub_vec(int64_t n, const double *__restrict__ b, const double *__restrict__ ax, double *r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - ax[i];
}

// ---- host side of the per-system batched solve ----
static int sys_blocks(int nb, int64_t n1) {
  int64_t P = (4LL * num_sms() + nb - 1) / nb;
  P = std::min<int64_t>(P, (n1 + 255) / 256);
  P = std::max<int64_t>(P, 1);
  return (int)std::min<int64_t>(P, 64);
}

// dd[b ldd + o + k] = V_{i0+k} . w over system b, k < K
static vem_status sys_dots(vem_handle *h, const VemOp &op, const double *V, int i0, int K, const double *w,
                           double *dd, int ldd, int o, const double *skip = nullptr) {
  cudaStream_t s = h->stream;
  const int nb = op.nbatch;
  const int P = sys_blocks(nb, op.n_u1 + op.n_p1);
  for (int c = 0; c < K; c += 8) {
    const int k = std::min(8, K - c);
    count_launch();
    k_sys_dots<<<dim3(P, nb), 256, 0, s>>>(nb, op.n_u1, op.n_p1, op.n, V, i0 + c, k, w, h->sys_part, skip);
    count_launch();
    k_sys_dots_fin<<<grid_for((int64_t)nb * k, 256), 256, 0, s>>>(nb, P, k, h->sys_part, dd, ldd, o + c, skip);
  }
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

// x = S^-1 b for every system whose outer iteration is active (active[b lda]
// != 0), each by its own Jacobi-PCG to inner_rtol; vectors and values in T.
template <class T>
static vem_status bpcg_solve(vem_handle *h, const VemOp &op, const T *sval, const T *dinv, const double *b, T *x,
                             T *wk, const double *active, int lda, int *iters) {
  cudaStream_t s = h->stream;
  const int nb = op.nbatch;
  const int64_t n1 = op.n_p1, nsl = op.S.nslices, N = (int64_t)nb * n1;
  T *r = wk, *u = wk + N, *p = wk + 2 * N, *sv = wk + 3 * N, *w = wk + 4 * N;
  const int P = sys_blocks(nb, n1);
  double *ru = h->bc_part, *wu = ru + (size_t)nb * nsl, *rr = wu + (size_t)nb * nsl;
  double *bsc = h->bc_sc, *flag = h->bc_sc + BC_N * nb;
  unsigned int *tick = reinterpret_cast<unsigned int *>(flag + 2);
  const double tol2 = h->opt.inner_rtol * h->opt.inner_rtol;
  // the tile of the Schur SpMV: the autotuner's choice for this shape
  const int tile = tune_bspmv<T>(h, nb, op, sval, u, r, w, ru, wu);
  h->schur_tile = tile;
  count_launch();
  k_bcg_init<T><<<dim3(P, nb), 256, 0, s>>>(nb, n1, b, dinv, x, r, u, p, sv, rr, bsc, active, lda, flag);
  bspmv_launch<T>(s, tile, nb, op, sval, u, r, w, ru, wu, bsc, flag);
  count_launch();
  k_bcg_scalars<<<nb, 256, 0, s>>>(nb, nsl, P, ru, wu, rr, tol2, bsc, 1, flag, tick);
  auto iteration = [&]() {
    cudaStream_t cs = h->stream;
    count_launch();
    k_bcg_update<T><<<dim3(P, nb), 256, 0, cs>>>(nb, n1, x, r, u, p, sv, w, dinv, bsc, rr, flag);
    bspmv_launch<T>(cs, tile, nb, op, sval, u, r, w, ru, wu, bsc, flag);
    count_launch();
    k_bcg_scalars<<<nb, 256, 0, cs>>>(nb, nsl, P, ru, wu, rr, tol2, bsc, 0, flag, tick);
  };
  uint64_t tol_bits = 0;
  std::memcpy(&tol_bits, &tol2, sizeof(double));
  const std::vector<uintptr_t> key = {(uintptr_t)op.S.off, (uintptr_t)op.S.col, (uintptr_t)sval, (uintptr_t)dinv,
                                      (uintptr_t)x, (uintptr_t)wk, (uintptr_t)bsc, (uintptr_t)ru, (uintptr_t)nb,
                                      (uintptr_t)n1, (uintptr_t)P, (uintptr_t)tile, (uintptr_t)tol_bits,
                                      sizeof(T), (uintptr_t)op.S.stored};
  bool graph = h->bpcg_graph && h->bpcg_graph16 && h->bpcg_key == key;
  if (!graph) {
    h->bpcg_key.clear();
    graph = capture_graph(h, h->bpcg_graph, h->bpcg_kernels, [&]() {
              for (int k = 0; k < 4; ++k) iteration();
            }) &&
            capture_graph(h, h->bpcg_graph16, h->bpcg16_kernels, [&]() {
              for (int k = 0; k < 16; ++k) iteration();
            });
    if (graph) h->bpcg_key = key;
  }
  const int maxit = h->opt.inner_maxit;
  int chunk = h->last_bpcg_iters > 0 ? h->last_bpcg_iters : 8;
  int it = 0;
  while (it < maxit) {
    const int end = it + chunk < maxit ? it + chunk : maxit;
    chunk = 4;
    if (graph) {
      for (; it + 16 <= end; it += 16) {
        VEM_CUDA(h, cudaGraphLaunch(h->bpcg_graph16, s));
        count_launches(h->bpcg16_kernels);
      }
      for (; it < end; it += 4) {
        VEM_CUDA(h, cudaGraphLaunch(h->bpcg_graph, s));
        count_launches(h->bpcg_kernels);
      }
    } else {
      for (; it < end; ++it) iteration();
    }
    VEM_CUDA(h, cudaGetLastError());
    VEM_CUDA(h, cudaMemcpyAsync(h->h_scal, flag, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    if (h->h_scal[0] != 0.0) break;
  }
  std::vector<double> bad(nb);
  VEM_CUDA(h, cudaMemcpyAsync(bad.data(), bsc + BC_BAD * nb, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaStreamSynchronize(s));
  for (int b2 = 0; b2 < nb; ++b2)
    if (bad[b2] != 0.0)
      return fail(h, bad[b2] == 2.0 ? VEM_ERR_NONFINITE : VEM_ERR_BREAKDOWN, "inner PCG breakdown in system %d", b2);
  *iters = (int)h->h_scal[1];
  h->last_bpcg_iters = *iters;
  return VEM_OK;
}

// z = P^-1 v for every system (block-diagonal or block upper-triangular with
// the systems' own inner solves); systems whose outer iteration is inactive
// have v = 0 and get z = 0.
static vem_status sys_precond(vem_handle *h, const VemOp &op, const double *v, double *z, double *pw,
                              const double *active, int lda, int *inner) {
  cudaStream_t s = h->stream;
  const int64_t nu = op.n_u, np = op.n_p;
  int it = 0;
  if (h->opt.precision == VEM_PRECISION_MIXED) {
    float *w32 = reinterpret_cast<float *>(pw);
    float *x32 = w32 + 5 * np;
    VEM_TRY(bpcg_solve<float>(h, op, op.S_val32, op.s_dinv32, v + nu, x32, w32, active, lda, &it));
    count_launch();
    k_f32_to_f64<<<grid_for(np, 256), 256, 0, s>>>(np, x32, z + nu);
  } else {
    VEM_TRY(bpcg_solve<double>(h, op, op.S.val, op.s_dinv, v + nu, z + nu, pw, active, lda, &it));
  }
  *inner += it;
  if (h->opt.precond == VEM_PREC_BLOCK_DIAG) {
    count_launch();
    k_diag_scale<<<nblocks_vec(nu), kRedThreads, 0, s>>>(nu, v, op.dinvM, z, nullptr);
  } else {
    count_launch();
    k_negate<<<grid_for(np, 256), 256, 0, s>>>(np, z + nu);
    if (h->nq > 1) {
      count_launch();
      k_tri_flux_rows<true><<<grid_for(nu, 256), 256, 0, s>>>(nu, op.n_u1, op.n_p1, h->bt_col, h->bt_val, v,
                                                               op.dinvM, z + nu, z);
    } else {
      launch_tri_flux(s, h->nfd, true, h->nf, nu, op.n_u1, op.n_p1, v, op.dinvM, h->f_cell, h->bt_face, z + nu, z);
    }
  }
  VEM_CUDA(h, cudaGetLastError());
  return VEM_OK;
}

// Per-system restarted FGMRES(m) with right preconditioning from x (usually
// 0): system b stops when ||b_b - A_b x_b|| <= rtol ||b_b||.  relres (host,
// nb entries, may be NULL) receives each system's last true relative residual.
vem_status run_fgmres_systems(vem_handle *h, const VemOp &op, const double *rhs, double *x, vem_stats *st,
                              double *relres) {
  cudaStream_t s = h->stream;
  h->n_saddle_pending = 0;
  const int nb = op.nbatch;
  const int64_t N = op.n, np = op.n_p;
  const int m = h->opt.restart;
  const SysLayout L{m};
  // per-system dot rows: pass-1 and pass-2 coefficients, ||w||^2, ||r||^2, ||b||^2
  const int ldd = 2 * (m + 2) + 4, o1 = 0, o2 = m + 2, on = 2 * (m + 2), orr = on + 1, obb = on + 2;
  VEM_TRY(ensure_work(h, (size_t)(2 * m + 2) * N + 5 * (size_t)np));
  double *V = h->work, *Z = V + (size_t)(m + 1) * N, *tmp = Z + (size_t)m * N, *pw = tmp + N;
  const int P = sys_blocks(nb, op.n_u1 + op.n_p1);
  if (h->sys_n < (size_t)nb * L.size()) {
    dfree(h, h->sys_gs);
    h->sys_gs = nullptr;
    VEM_TRY(dalloc_n(h, &h->sys_gs, (size_t)nb * L.size() + 8));
    h->sys_n = (size_t)nb * L.size();
  }
  const size_t ddn = (size_t)nb * ldd + 8 + (size_t)nb;   // dot rows, flags, reorthogonalisation marks
  if (h->sys_dd_n < ddn) {
    dfree(h, h->sys_dd);
    h->sys_dd = nullptr;
    VEM_TRY(dalloc_n(h, &h->sys_dd, ddn));
    h->sys_dd_n = ddn;
  }
  if (h->sys_part_n < (size_t)nb * P * 8) {
    dfree(h, h->sys_part);
    VEM_TRY(dalloc_n(h, &h->sys_part, (size_t)nb * P * 8));
    h->sys_part_n = (size_t)nb * P * 8;
  }
  const size_t bcn = 3 * (size_t)nb * op.S.nslices + (size_t)nb * sys_blocks(nb, op.n_p1) + 16;
  if (h->bc_part_n < bcn) {
    dfree(h, h->bc_part);
    VEM_TRY(dalloc_n(h, &h->bc_part, bcn));
    h->bc_part_n = bcn;
  }
  if (h->bc_sc_n < (size_t)BC_N * nb + 4) {
    dfree(h, h->bc_sc);
    VEM_TRY(dalloc_n(h, &h->bc_sc, (size_t)BC_N * nb + 4));
    h->bc_sc_n = (size_t)BC_N * nb + 4;
    // the scalars kernel's last-block counter (after the two flags) starts at 0
    VEM_CUDA(h, cudaMemsetAsync(h->bc_sc + (size_t)BC_N * nb + 2, 0, sizeof(double), s));
  }
  double *gs = h->sys_gs, *dd = h->sys_dd, *fl = h->sys_dd + (size_t)nb * ldd, *ro = fl + 8;
  const int gnb = grid_for(nb, 128);
  const double rtol = h->opt.rtol;
  // r = b - A x, the norms and the first cycle's start
  op_apply_timed(h, op, x, tmp);
  count_launch();
  k_sub_vec<<<grid_for(N, 256), 256, 0, s>>>(N, rhs, tmp, tmp);
  VEM_TRY(sys_dots(h, op, tmp, 0, 1, tmp, dd, ldd, orr));
  VEM_TRY(sys_dots(h, op, rhs, 0, 1, rhs, dd, ldd, obb));
  count_launch();
  k_sys_start<<<gnb, 128, 0, s>>>(nb, L, rtol, dd, ldd, orr, obb, gs, 1);
  int inner = 0, it = 0;
  double hf[3] = {0, 0, 0};
  auto flags = [&]() -> vem_status {
    count_launch();
    k_sys_flags<<<1, 256, 0, s>>>(nb, L, gs, fl);
    VEM_CUDA(h, cudaMemcpyAsync(hf, fl, sizeof(hf), cudaMemcpyDeviceToHost, s));
    VEM_CUDA(h, cudaStreamSynchronize(s));
    return VEM_OK;
  };
  VEM_TRY(flags());
  while (hf[1] > 0.0 && it < h->opt.maxit) {
    count_launch();
    k_sys_scale<<<grid_for(N, 256), 256, 0, s>>>(nb, op.n_u1, op.n_p1, N, tmp, gs + L.S(GS_FAC), L.size(), V);
    for (int j = 0; j < m && it < h->opt.maxit; ++j) {
      ++it;
      double *Vj = V + (size_t)j * N, *Zj = Z + (size_t)j * N, *w = V + (size_t)(j + 1) * N;
      VEM_TRY(sys_precond(h, op, Vj, Zj, pw, gs + L.S(GS_ACTIVE), L.size(), &inner));
      op_apply_timed(h, op, Zj, w);
      // classical Gram-Schmidt per system; the first pass's dots include
      // w = V_{j+1} itself (||w||^2 before the pass, at o1 + j + 1); the
      // second pass only where the DGKS test asks, decided on the device
      VEM_TRY(sys_dots(h, op, V, 0, j + 2, w, dd, ldd, o1));
      count_launch();
      k_sys_axpy<<<grid_for(N, 256), 256, 0, s>>>(nb, op.n_u1, op.n_p1, N, j + 1, V, dd + o1, ldd, -1.0, w, nullptr);
      VEM_TRY(sys_dots(h, op, w, 0, 1, w, dd, ldd, on));
      count_launch();
      k_sys_reorth<<<1, 256, 0, s>>>(nb, gs + L.S(GS_ACTIVE), L.size(), dd, ldd, o1 + j + 1, on, o2, j + 1, ro,
                                     fl + 4);
      VEM_TRY(sys_dots(h, op, V, 0, j + 1, w, dd, ldd, o2, fl + 4));
      count_launch();
      k_sys_axpy<<<grid_for(N, 256), 256, 0, s>>>(nb, op.n_u1, op.n_p1, N, j + 1, V, dd + o2, ldd, -1.0, w, fl + 4);
      VEM_TRY(sys_dots(h, op, w, 0, 1, w, dd, ldd, on, fl + 4));
      count_launch();
      k_sys_arnoldi<<<gnb, 128, 0, s>>>(nb, j, L, rtol, dd, ldd, o1, o2, on, gs);
      count_launch();
      k_sys_scale<<<grid_for(N, 256), 256, 0, s>>>(nb, op.n_u1, op.n_p1, N, w, gs + L.S(GS_FAC), L.size(), w);
      VEM_TRY(flags());
      if (debug_on()) fprintf(stderr, "[vem] batched fgmres it=%d active=%g open=%g\n", it, hf[0], hf[1]);
      if (hf[0] == 0.0) break;
    }
    // x += Z y per system, then the true residuals and the next start
    count_launch();
    k_sys_solve<<<gnb, 128, 0, s>>>(nb, L, gs);
    count_launch();
    k_sys_axpy<<<grid_for(N, 256), 256, 0, s>>>(nb, op.n_u1, op.n_p1, N, m, Z, gs + L.Y(0), L.size(), 1.0, x,
                                                nullptr);
    op_apply_timed(h, op, x, V);
    count_launch();
    k_sub_vec<<<grid_for(N, 256), 256, 0, s>>>(N, rhs, V, tmp);
    VEM_TRY(sys_dots(h, op, tmp, 0, 1, tmp, dd, ldd, orr));
    count_launch();
    k_sys_start<<<gnb, 128, 0, s>>>(nb, L, rtol, dd, ldd, orr, obb, gs, 0);
    VEM_TRY(flags());
  }
  std::vector<double> q((size_t)nb * L.size());
  VEM_CUDA(h, cudaMemcpyAsync(q.data(), gs, sizeof(double) * q.size(), cudaMemcpyDeviceToHost, s));
  VEM_CUDA(h, cudaStreamSynchronize(s));
  double worst = 0.0;
  int itmax = 0;
  for (int b = 0; b < nb; ++b) {
    const double rel = q[(size_t)b * L.size() + L.S(GS_REL)];
    if (relres) relres[b] = rel;
    worst = std::max(worst, rel);
    itmax = std::max(itmax, (int)q[(size_t)b * L.size() + L.S(GS_IT)]);
  }
  st->iterations = itmax;
  st->inner_iterations = inner;
  st->relres = worst;
  if (cudaStreamSynchronize(s) == cudaSuccess) collect_saddle(h);
  cudaGetLastError();
  if (hf[1] > 0.0)
    return fail(h, VEM_ERR_NOT_CONVERGED, "batched FGMRES: %g systems above rtol after %d iterations", hf[1], it);
  return VEM_OK;
}

VemOp single_op(vem_handle *h) {
  VemOp op;
  op.A = h->A;
  op.S = h->S;
  op.diagM = h->diagM;
  op.dinvM = h->dinvM;
  op.s_dinv = h->s_dinv;
  op.S_val32 = h->S_val32;
  op.s_dinv32 = h->s_dinv32;
  op.n_u = op.n_u1 = h->n_u;
  op.n_p = op.n_p1 = h->n_p;
  op.n = h->n;
  op.nbatch = 1;
  return op;
}

vem_status krylov_solve(vem_handle *h, const VemOp &op, const double *rhs, double *x, vem_stats *st) {
  h->n_saddle_pending = 0;
  vem_status r;
  if (h->opt.precond == VEM_PREC_BLOCK_REG) {
    if (op.nbatch != 1) return fail(h, VEM_ERR_UNSUPPORTED, "Block-Reg is single-system");
    VEM_TRY(ensure_reg(h));
  }
  if (h->opt.krylov == VEM_KRYLOV_MINRES) {
    if (h->opt.precond == VEM_PREC_BLOCK_TRI)
      return fail(h, VEM_ERR_BAD_INPUT, "MINRES needs a block-diagonal preconditioner");
    r = run_minres(h, op, rhs, x, st);
  } else if (h->opt.krylov == VEM_KRYLOV_FGMRES) {
    r = run_fgmres(h, op, rhs, x, st);
  } else {
    return fail(h, VEM_ERR_BAD_INPUT, "unknown Krylov method %d", h->opt.krylov);
  }
  if (cudaStreamSynchronize(h->stream) == cudaSuccess) collect_saddle(h);
  cudaGetLastError();
  h->x_zero = false;
  return r;
}

}  // namespace vem
