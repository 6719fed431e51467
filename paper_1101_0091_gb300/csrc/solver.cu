// Iterative consumers of the product: conjugate gradients (Hestenes-Stiefel)
// and the Lanczos three-term recurrence, each on k independent columns, so that
// every iteration's product is one k-column SpMM through the plan (Sec. 1.3.1
// names Lanczos and Jacobi-Davidson as the methods whose run time the product
// dominates).
//
// Vectors are row-major n x k blocks (ld = k, 16-byte aligned: the vector
// kernels move 16 bytes per access).  The vector work of an iteration is a few
// fused grid-stride kernels on a grid of one wave; each reduces
// its per-column inner products to one partial per CTA, and the CTA that
// finishes last (threadfence + ticket, no waiting) adds the partials in a
// fixed order and updates the per-column scalars in device memory.  Reductions are
// therefore deterministic for a given solver.  Columns freeze on the device the
// iteration they converge (or break down), so the host only polls a counter
// every `check_every` iterations; those iterations are replayed from a CUDA
// graph captured once per (B, X, check_every).
#include <cmath>
#include <cstring>
#include <new>

#include "device.cuh"
#include "internal.h"

namespace spmv {

constexpr int kSolverCtasPerSm = 8;  // upper limit; the occupancy of the update kernel decides
constexpr int kMaxCols = 16;

struct CgScalars {
  double rr[kMaxCols], tol2[kMaxCols], alpha[kMaxCols], beta[kMaxCols];
  int active[kMaxCols], next_active[kMaxCols], iters[kMaxCols], breakdown[kMaxCols];
  int n_active;
};

struct LzScalars {
  double b_prev[kMaxCols], inv_b[kMaxCols], alpha[kMaxCols];
  int live[kMaxCols];
};

// ---------------------------------------------------------------- block walking
// How a thread walks a row-major n x k block, one unit per grid-stride step:
//  PAIRS (k = 1): two consecutive entries, one 16-byte access;
//  VROWS (k = K = 2, 4): one row of K values, K/2 16-byte accesses;
//  VGROUPS (k = K = 8, 16): a group of 4 columns of one row (K/4 units per
//    row), two 16-byte accesses; a thread keeps 4 accumulators instead of K,
//    which keeps these kernels at several CTAs per SM;
//  ROWS (other k): one row, k scalar accesses (K >= k, masked).
// PAIRS, VROWS and VGROUPS need 16-byte aligned blocks (checked on the host).
enum { ROWS = 0, VROWS = 1, PAIRS = 2, VGROUPS = 3 };

template <int K, int MODE>
struct Seg {
  static constexpr int NG = MODE == VGROUPS ? K / 4 : 1;                    // units per row
  static constexpr int W = MODE == PAIRS ? 2 : (MODE == VGROUPS ? 4 : K);  // values per unit
  static constexpr int KC = MODE == PAIRS ? 1 : W;                         // accumulators per thread
  static constexpr int KP = MODE == PAIRS ? 1 : K;                         // columns of the sums
  static_assert(kThreads % NG == 0, "a thread's units must share one column group");
  __device__ static int64_t units(int64_t n) { return MODE == PAIRS ? (n + 1) / 2 : n * NG; }
  // accumulator of value w, and the block column it belongs to in unit u
  __device__ static int acol(int w) { return MODE == PAIRS ? 0 : w; }
  __device__ static int gcol(int64_t u, int w) {
    return MODE == PAIRS ? 0 : (MODE == VGROUPS ? (int)(u % NG) * 4 + w : w);
  }
  __device__ static void load(const double* p, int64_t u, int64_t n, int k, double (&v)[W]) {
    if (MODE == PAIRS) {
      if (2 * u + 1 < n) {
        const double2 t = reinterpret_cast<const double2*>(p)[u];
        v[0] = t.x;
        v[1] = t.y;
      } else {
        v[0] = p[2 * u];
        v[1] = 0.0;
      }
    } else if (MODE == VROWS || MODE == VGROUPS) {
      // VGROUPS: u * 4 is the offset of group u % NG of row u / NG
#pragma unroll
      for (int h = 0; h < W / 2; ++h) {
        const double2 t = reinterpret_cast<const double2*>(p + u * W)[h];
        v[2 * h] = t.x;
        v[2 * h + 1] = t.y;
      }
    } else {
#pragma unroll
      for (int w = 0; w < W; ++w) v[w] = w < k ? p[u * k + w] : 0.0;
    }
  }
  __device__ static void store(double* p, int64_t u, int64_t n, int k, const double (&v)[W]) {
    if (MODE == PAIRS) {
      if (2 * u + 1 < n)
        reinterpret_cast<double2*>(p)[u] = make_double2(v[0], v[1]);
      else
        p[2 * u] = v[0];
    } else if (MODE == VROWS || MODE == VGROUPS) {
#pragma unroll
      for (int h = 0; h < W / 2; ++h) reinterpret_cast<double2*>(p + u * W)[h] = make_double2(v[2 * h], v[2 * h + 1]);
    } else {
#pragma unroll
      for (int w = 0; w < W; ++w)
        if (w < k) p[u * k + w] = v[w];
    }
  }
};

// ---------------------------------------------------------------- reductions
// Per-column sums over a CTA and then over the CTAs, in a fixed order (so a
// solver's results do not depend on timing).

// Writes this CTA's NS x KP column sums of the threads' accumulators
// (G::KC per thread: thread t holds the columns of group t % G::NG, or all
// of them), then returns true in the CTA that finished last (all partials
// visible to it).  Order: xor-shuffle tree within each warp, then warps in
// order.
template <typename G, int NS>
__device__ bool publish_partials(double (&acc)[NS][G::KC], double* partial, uint32_t* counter, int k) {
  constexpr int KP = G::KP, KC = G::KC, R = G::NG;  // R lanes of a warp hold distinct column sets
  __shared__ double sh[kThreads / 32][KP];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
#pragma unroll
    for (int w = 0; w < KC; ++w)
#pragma unroll
      for (int off = 16; off >= R; off >>= 1) acc[s][w] += __shfl_xor_sync(0xffffffffu, acc[s][w], off);
    if (lane < R)
#pragma unroll
      for (int w = 0; w < KC; ++w) sh[warp][lane * KC + w] = acc[s][w];
    __syncthreads();
    if (threadIdx.x < KP && threadIdx.x < k) {
      double t = 0.0;
#pragma unroll
      for (int v = 0; v < kThreads / 32; ++v) t += sh[v][threadIdx.x];
      partial[((size_t)blockIdx.x * NS + s) * kMaxCols + threadIdx.x] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// In the last CTA (all threads): the sums of the CTAs' partials, per sum s
// and column q, into tot[s][q].  Thread t takes column t % KP and adds the
// partials of CTAs t / KP, t / KP + 256 / KP, ... in order; the threads of a
// column are then combined by an xor-shuffle tree and the warps in order.
template <int KP, int NS>
__device__ void finish_partials(const double* partial, int k, double (&tot)[NS][KP]) {
  constexpr int SL = kThreads / KP;  // threads per column
  __shared__ double sh[kThreads / 32][KP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q = threadIdx.x % KP;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double x = 0.0;
    if (q < k)
      for (unsigned b = threadIdx.x / KP; b < gridDim.x; b += SL)
        x += __ldcg(partial + ((size_t)b * NS + s) * kMaxCols + q);
#pragma unroll
    for (int off = 16; off >= KP; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane < KP) sh[warp][lane] = x;
    __syncthreads();
    if (threadIdx.x < KP) {
      double t = 0.0;
#pragma unroll
      for (int v = 0; v < kThreads / 32; ++v) t += sh[v][threadIdx.x];
      tot[s][threadIdx.x] = t;
    }
    __syncthreads();
  }
}

#define UNIT_LOOP(u, n) \
  for (int64_t u = (int64_t)blockIdx.x * kThreads + threadIdx.x; u < G::units(n); u += (int64_t)gridDim.x * kThreads)

// ---------------------------------------------------------------- CG kernels
// R = B - AX (AX in Q), P = R; rr = R.R, tol2 = rtol^2 B.B, active = rr > tol2.
template <int K, int MODE>
__global__ void __launch_bounds__(kThreads) k_cg_init(int64_t n, int k, const double* __restrict__ B,
                                                      const double* __restrict__ Q, double* R, double* P,
                                                      double* partial, uint32_t* counter, CgScalars* S,
                                                      double rtol2) {
  using G = Seg<K, MODE>;
  double acc[2][G::KC];
#pragma unroll
  for (int q = 0; q < G::KC; ++q) acc[0][q] = acc[1][q] = 0.0;
  UNIT_LOOP(u, n) {
    double b[G::W], r[G::W];
    G::load(B, u, n, k, b);
    G::load(Q, u, n, k, r);
#pragma unroll
    for (int w = 0; w < G::W; ++w) {
      r[w] = b[w] - r[w];
      acc[0][G::acol(w)] = fma(r[w], r[w], acc[0][G::acol(w)]);
      acc[1][G::acol(w)] = fma(b[w], b[w], acc[1][G::acol(w)]);
    }
    G::store(R, u, n, k, r);
    G::store(P, u, n, k, r);
  }
  if (!publish_partials<G, 2>(acc, partial, counter, k)) return;
  __shared__ double tot[2][G::KP];
  finish_partials<G::KP, 2>(partial, k, tot);
  if (threadIdx.x < k) {
    const int q = threadIdx.x;
    const double rr = tot[0][q], bb = tot[1][q];
    S->rr[q] = rr;
    S->tol2[q] = rtol2 * bb;
    S->active[q] = rr > rtol2 * bb;
    S->iters[q] = 0;
    S->breakdown[q] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int na = 0;
    for (int q = 0; q < k; ++q) na += S->active[q];
    S->n_active = na;
    *counter = 0;
  }
}

// pq = P.Q; active columns: alpha = rr / pq, or breakdown when pq <= 0.
template <int K, int MODE>
__global__ void __launch_bounds__(kThreads) k_cg_alpha(int64_t n, int k, const double* __restrict__ P,
                                                       const double* __restrict__ Q, double* partial,
                                                       uint32_t* counter, CgScalars* S) {
  using G = Seg<K, MODE>;
  double acc[1][G::KC];
#pragma unroll
  for (int q = 0; q < G::KC; ++q) acc[0][q] = 0.0;
  UNIT_LOOP(u, n) {
    double p[G::W], q2[G::W];
    G::load(P, u, n, k, p);
    G::load(Q, u, n, k, q2);
#pragma unroll
    for (int w = 0; w < G::W; ++w) acc[0][G::acol(w)] = fma(p[w], q2[w], acc[0][G::acol(w)]);
  }
  if (!publish_partials<G, 1>(acc, partial, counter, k)) return;
  __shared__ double tot[1][G::KP];
  finish_partials<G::KP, 1>(partial, k, tot);
  if (threadIdx.x < k) {
    const int q = threadIdx.x;
    const double pq = tot[0][q];
    if (S->active[q] && !(pq > 0.0)) {
      S->breakdown[q] = 1;
      S->active[q] = 0;
    }
    S->alpha[q] = S->active[q] ? S->rr[q] / pq : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0;
}

// Active columns: X += alpha P, R -= alpha Q; rr' = R.R, beta = rr' / rr.
// (Inactive columns are written back unchanged.)
template <int K, int MODE>
__global__ void __launch_bounds__(kThreads) k_cg_update(int64_t n, int k, double* X, double* R,
                                                        const double* __restrict__ P, const double* __restrict__ Q,
                                                        double* partial, uint32_t* counter, CgScalars* S) {
  using G = Seg<K, MODE>;
  __shared__ double s_alpha[G::KP];
  __shared__ int s_active[G::KP];
  if (threadIdx.x < G::KP) {
    s_alpha[threadIdx.x] = threadIdx.x < k ? S->alpha[threadIdx.x] : 0.0;
    s_active[threadIdx.x] = threadIdx.x < k ? S->active[threadIdx.x] : 0;
  }
  __syncthreads();
  double acc[1][G::KC];
#pragma unroll
  for (int q = 0; q < G::KC; ++q) acc[0][q] = 0.0;
  UNIT_LOOP(u, n) {
    double x[G::W], r[G::W], p[G::W], q2[G::W];
    G::load(X, u, n, k, x);
    G::load(R, u, n, k, r);
    G::load(P, u, n, k, p);
    G::load(Q, u, n, k, q2);
#pragma unroll
    for (int w = 0; w < G::W; ++w) {
      const int c = G::gcol(u, w);
      if (s_active[c]) {
        x[w] = fma(s_alpha[c], p[w], x[w]);
        r[w] = fma(-s_alpha[c], q2[w], r[w]);
      }
      acc[0][G::acol(w)] = fma(r[w], r[w], acc[0][G::acol(w)]);
    }
    G::store(X, u, n, k, x);
    G::store(R, u, n, k, r);
  }
  if (!publish_partials<G, 1>(acc, partial, counter, k)) return;
  __shared__ double tot[1][G::KP];
  finish_partials<G::KP, 1>(partial, k, tot);
  if (threadIdx.x < k) {
    const int q = threadIdx.x;
    if (S->active[q]) {
      const double rr = tot[0][q];
      S->beta[q] = rr / S->rr[q];
      S->rr[q] = rr;
      S->iters[q] += 1;
      S->next_active[q] = rr > S->tol2[q];
    } else {
      S->beta[q] = 0.0;
      S->next_active[q] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0;
}

// Active columns: P = R + beta P; then the columns that met the tolerance stop.
template <int K, int MODE>
__global__ void __launch_bounds__(kThreads) k_cg_direction(int64_t n, int k, const double* __restrict__ R,
                                                           double* P, uint32_t* counter, CgScalars* S) {
  using G = Seg<K, MODE>;
  __shared__ double s_beta[G::KP];
  __shared__ int s_active[G::KP];
  __shared__ bool last;
  if (threadIdx.x < G::KP) {
    s_beta[threadIdx.x] = threadIdx.x < k ? S->beta[threadIdx.x] : 0.0;
    s_active[threadIdx.x] = threadIdx.x < k ? S->active[threadIdx.x] : 0;
  }
  __syncthreads();
  UNIT_LOOP(u, n) {
    double r[G::W], p[G::W];
    G::load(R, u, n, k, r);
    G::load(P, u, n, k, p);
#pragma unroll
    for (int w = 0; w < G::W; ++w)
      if (s_active[G::gcol(u, w)]) p[w] = fma(s_beta[G::gcol(u, w)], p[w], r[w]);
    G::store(P, u, n, k, p);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  int na = 0;
  for (int q = 0; q < k; ++q) {
    S->active[q] = S->active[q] && S->next_active[q];
    na += S->active[q];
  }
  S->n_active = na;
  *counter = 0;
}

// ---------------------------------------------------------------- Lanczos kernels
// |V0| per column; live = |V0| > 0; inv_b = 1 / |V0| (consumed by k_lz_scale).
template <int K, int MODE>
__global__ void __launch_bounds__(kThreads) k_lz_norm(int64_t n, int k, const double* __restrict__ V0,
                                                      double* partial, uint32_t* counter, LzScalars* S) {
  using G = Seg<K, MODE>;
  double acc[1][G::KC];
#pragma unroll
  for (int q = 0; q < G::KC; ++q) acc[0][q] = 0.0;
  UNIT_LOOP(u, n) {
    double v[G::W];
    G::load(V0, u, n, k, v);
#pragma unroll
    for (int w = 0; w < G::W; ++w) acc[0][G::acol(w)] = fma(v[w], v[w], acc[0][G::acol(w)]);
  }
  if (!publish_partials<G, 1>(acc, partial, counter, k)) return;
  __shared__ double tot[1][G::KP];
  finish_partials<G::KP, 1>(partial, k, tot);
  if (threadIdx.x < k) {
    const int q = threadIdx.x;
    const double b = sqrt(tot[0][q]);
    S->live[q] = b > 0.0;
    S->b_prev[q] = b;
    S->inv_b[q] = b > 0.0 ? 1.0 / b : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0;
}

// dst = live ? src * (1 / beta) : 0 (one FP64 division per column, in the
// reducing CTA, instead of one per entry); zero_out (if given) = 0.
template <int K, int MODE>
__global__ void __launch_bounds__(kThreads) k_lz_scale(int64_t n, int k, const double* __restrict__ src,
                                                       double* dst, double* zero_out, const LzScalars* S) {
  using G = Seg<K, MODE>;
  __shared__ double s_b[G::KP];
  __shared__ int s_live[G::KP];
  if (threadIdx.x < G::KP) {
    s_b[threadIdx.x] = threadIdx.x < k ? S->inv_b[threadIdx.x] : 0.0;
    s_live[threadIdx.x] = threadIdx.x < k ? S->live[threadIdx.x] : 0;
  }
  __syncthreads();
  UNIT_LOOP(u, n) {
    double v[G::W];
    G::load(src, u, n, k, v);
#pragma unroll
    for (int w = 0; w < G::W; ++w) v[w] = s_live[G::gcol(u, w)] ? v[w] * s_b[G::gcol(u, w)] : 0.0;
    G::store(dst, u, n, k, v);
    if (zero_out) {
#pragma unroll
      for (int w = 0; w < G::W; ++w) v[w] = 0.0;
      G::store(zero_out, u, n, k, v);
    }
  }
}

// W = W - b_prev v_prev; alpha = W.v (live columns), stored to alpha_out.
template <int K, int MODE>
__global__ void __launch_bounds__(kThreads) k_lz_alpha(int64_t n, int k, double* W, const double* __restrict__ v,
                                                       const double* __restrict__ v_prev, double* partial,
                                                       uint32_t* counter, LzScalars* S, double* alpha_out) {
  using G = Seg<K, MODE>;
  __shared__ double s_b[G::KP];
  if (threadIdx.x < G::KP) s_b[threadIdx.x] = threadIdx.x < k ? S->b_prev[threadIdx.x] : 0.0;
  __syncthreads();
  double acc[1][G::KC];
#pragma unroll
  for (int q = 0; q < G::KC; ++q) acc[0][q] = 0.0;
  UNIT_LOOP(u, n) {
    double w_[G::W], vv[G::W], vp[G::W];
    G::load(W, u, n, k, w_);
    G::load(v, u, n, k, vv);
    G::load(v_prev, u, n, k, vp);
#pragma unroll
    for (int w = 0; w < G::W; ++w) {
      w_[w] = fma(-s_b[G::gcol(u, w)], vp[w], w_[w]);
      acc[0][G::acol(w)] = fma(w_[w], vv[w], acc[0][G::acol(w)]);
    }
    G::store(W, u, n, k, w_);
  }
  if (!publish_partials<G, 1>(acc, partial, counter, k)) return;
  __shared__ double tot[1][G::KP];
  finish_partials<G::KP, 1>(partial, k, tot);
  if (threadIdx.x < k) {
    const int q = threadIdx.x;
    const double a = S->live[q] ? tot[0][q] : 0.0;
    S->alpha[q] = a;
    alpha_out[q] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0;
}

// W = W - alpha v; beta = |W| (live columns), stored to beta_out; a column
// whose beta is 0 stops.
template <int K, int MODE>
__global__ void __launch_bounds__(kThreads) k_lz_beta(int64_t n, int k, double* W, const double* __restrict__ v,
                                                      double* partial, uint32_t* counter, LzScalars* S,
                                                      double* beta_out) {
  using G = Seg<K, MODE>;
  __shared__ double s_a[G::KP];
  if (threadIdx.x < G::KP) s_a[threadIdx.x] = threadIdx.x < k ? S->alpha[threadIdx.x] : 0.0;
  __syncthreads();
  double acc[1][G::KC];
#pragma unroll
  for (int q = 0; q < G::KC; ++q) acc[0][q] = 0.0;
  UNIT_LOOP(u, n) {
    double w_[G::W], vv[G::W];
    G::load(W, u, n, k, w_);
    G::load(v, u, n, k, vv);
#pragma unroll
    for (int w = 0; w < G::W; ++w) {
      w_[w] = fma(-s_a[G::gcol(u, w)], vv[w], w_[w]);
      acc[0][G::acol(w)] = fma(w_[w], w_[w], acc[0][G::acol(w)]);
    }
    G::store(W, u, n, k, w_);
  }
  if (!publish_partials<G, 1>(acc, partial, counter, k)) return;
  __shared__ double tot[1][G::KP];
  finish_partials<G::KP, 1>(partial, k, tot);
  if (threadIdx.x < k) {
    const int q = threadIdx.x;
    const double b = S->live[q] ? sqrt(tot[0][q]) : 0.0;
    beta_out[q] = b;
    S->live[q] = S->live[q] && b > 0.0;
    S->b_prev[q] = S->live[q] ? b : 0.0;
    S->inv_b[q] = S->live[q] ? 1.0 / b : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0;
}
#undef UNIT_LOOP

// ---------------------------------------------------------------- dispatch
// k = 1 -> pairs; k = 2, 4 -> vector rows; k = 8, 16 -> 4-column groups;
// other k -> scalar rows.
template <template <int, int> class F, typename... Args>
static cudaError_t by_k(int k, Args... args) {
  switch (k) {
    case 1: return F<1, PAIRS>::run(args...);
    case 2: return F<2, VROWS>::run(args...);
    case 4: return F<4, VROWS>::run(args...);
    case 8: return F<8, VGROUPS>::run(args...);
    case 16: return F<16, VGROUPS>::run(args...);
    default: break;
  }
  if (k <= 4) return F<4, ROWS>::run(args...);
  if (k <= 8) return F<8, ROWS>::run(args...);
  return F<16, ROWS>::run(args...);
}

#define SOLVER_LAUNCHER(NAME, KERNEL)                                \
  template <int K, int MODE>                                         \
  struct NAME {                                                      \
    template <typename... A>                                         \
    static cudaError_t run(unsigned grid, cudaStream_t s, A... a) { \
      KERNEL<K, MODE><<<grid, kThreads, 0, s>>>(a...);               \
      return cudaGetLastError();                                     \
    }                                                                \
  };
SOLVER_LAUNCHER(LCgInit, k_cg_init)
SOLVER_LAUNCHER(LCgAlpha, k_cg_alpha)
SOLVER_LAUNCHER(LCgUpdate, k_cg_update)
SOLVER_LAUNCHER(LCgDirection, k_cg_direction)
SOLVER_LAUNCHER(LLzNorm, k_lz_norm)
SOLVER_LAUNCHER(LLzScale, k_lz_scale)
SOLVER_LAUNCHER(LLzAlpha, k_lz_alpha)
SOLVER_LAUNCHER(LLzBeta, k_lz_beta)
#undef SOLVER_LAUNCHER

// Resident CTAs per SM of each vector kernel (the CG kernels come first,
// then the Lanczos ones, four each).
enum { KI_CG_INIT = 0, KI_CG_ALPHA, KI_CG_UPDATE, KI_CG_DIRECTION, KI_LZ_NORM, KI_LZ_SCALE, KI_LZ_ALPHA,
       KI_LZ_BETA, KI_COUNT };

template <int K, int MODE>
struct LOccupancy {
  static cudaError_t run(int* o) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(o + 0, k_cg_init<K, MODE>, kThreads, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(o + 1, k_cg_alpha<K, MODE>, kThreads, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(o + 2, k_cg_update<K, MODE>, kThreads, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(o + 3, k_cg_direction<K, MODE>, kThreads, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(o + 4, k_lz_norm<K, MODE>, kThreads, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(o + 5, k_lz_scale<K, MODE>, kThreads, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(o + 6, k_lz_alpha<K, MODE>, kThreads, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(o + 7, k_lz_beta<K, MODE>, kThreads, 0);
    return e;
  }
};

}  // namespace spmv

using namespace spmv;

struct spmv_solver {
  spmv_handle A = nullptr;
  int device = 0, k = 0;
  int64_t n = 0;
  unsigned grid[KI_COUNT] = {};    // one-wave grid of each vector kernel
  double *buf[3] = {nullptr, nullptr, nullptr};  // CG: R, P, Q; Lanczos: v_prev, v, W
  double* partial = nullptr;
  uint32_t* counter = nullptr;
  CgScalars* cg = nullptr;
  LzScalars* lz = nullptr;
  double* lz_out = nullptr;        // alpha[m][16], beta[m][16] on the device
  int lz_cap = 0;
  int* host_active = nullptr;      // pinned
  cudaStream_t cap = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t graph = nullptr;
  const double* g_B = nullptr;
  double* g_X = nullptr;
  int g_steps = 0;
  uint64_t g_gen = 0;              // plan generation the graph was captured at
};

static void solver_free(spmv_solver* s) {
  if (s->graph) cudaGraphExecDestroy(s->graph);
  for (double* b : s->buf) if (b) cudaFree(b);
  if (s->partial) cudaFree(s->partial);
  if (s->counter) cudaFree(s->counter);
  if (s->cg) cudaFree(s->cg);
  if (s->lz) cudaFree(s->lz);
  if (s->lz_out) cudaFree(s->lz_out);
  if (s->host_active) cudaFreeHost(s->host_active);
  if (s->cap) cudaStreamDestroy(s->cap);
  if (s->ev) cudaEventDestroy(s->ev);
}

namespace {
struct SolverDeviceGuard {
  int prev = -1;
  explicit SolverDeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~SolverDeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// One CG iteration on stream s: Q = A P, then alpha, the X/R update and the new direction.
spmv_status cg_iteration(spmv_solver* S, double* X, cudaStream_t s) {
  double *R = S->buf[0], *P = S->buf[1], *Q = S->buf[2];
  spmv_status st = spmv_apply_block(S->A, P, S->k, S->k, Q, S->k, s);
  if (st != SPMV_OK) return st;
  cudaError_t e = by_k<LCgAlpha>(S->k, S->grid[KI_CG_ALPHA], s, S->n, S->k, (const double*)P, (const double*)Q,
                                 S->partial, S->counter, S->cg);
  if (e == cudaSuccess)
    e = by_k<LCgUpdate>(S->k, S->grid[KI_CG_UPDATE], s, S->n, S->k, X, R, (const double*)P, (const double*)Q,
                        S->partial, S->counter, S->cg);
  if (e == cudaSuccess)
    e = by_k<LCgDirection>(S->k, S->grid[KI_CG_DIRECTION], s, S->n, S->k, (const double*)R, P, S->counter, S->cg);
  return e == cudaSuccess ? SPMV_OK : cuda_fail(e, "CG kernel launch");
}
}  // namespace

extern "C" {

spmv_status spmv_solver_create(spmv_handle A, int32_t k, spmv_solver_handle* out) {
  if (!A || !out) return fail(SPMV_ERR_ARG, "NULL argument");
  *out = nullptr;
  spmv_info info;
  spmv_status st = spmv_get_info(A, &info);
  if (st != SPMV_OK) return st;
  if (info.n_rows != info.n_cols) return fail(SPMV_ERR_ARG, "the solvers need a square matrix");
  if (k < 1 || k > plan_max_k(A)) return fail(SPMV_ERR_ARG, "k out of range 1..max_k of the plan");
  auto* S = new (std::nothrow) spmv_solver;
  if (!S) return fail(SPMV_ERR_OOM, "host allocation failed");
  S->A = A;
  S->device = plan_device(A);
  S->k = k;
  S->n = info.n_rows;
  SolverDeviceGuard g(S->device);
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device);
  // The kernels of one method (CG: 4, Lanczos: 4) share the one-wave grid of the
  // heaviest of them (measured: 1-2 % faster iterations at k >= 4 than a grid per
  // kernel, and 2 % faster at k = 1 than one grid for all 8 kernels).
  int per_sm[KI_COUNT] = {};
  if (e == cudaSuccess) e = by_k<LOccupancy>(k, per_sm);
  const int64_t want = (S->n + kThreads - 1) / kThreads;
  unsigned max_grid = 1;
  for (int m0 = 0; m0 < KI_COUNT; m0 += 4) {
    int r = kSolverCtasPerSm;
    for (int i = m0; i < m0 + 4; ++i) r = per_sm[i] < r ? per_sm[i] : r;
    r = r < 1 ? 1 : r;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * r;
    const unsigned g = (unsigned)(want < 1 ? 1 : (want < cap ? want : cap));
    for (int i = m0; i < m0 + 4; ++i) S->grid[i] = g;
    max_grid = g > max_grid ? g : max_grid;
  }
  const size_t vec = sizeof(double) * (size_t)(S->n > 0 ? S->n : 1) * (size_t)k;
  for (int b = 0; b < 3 && e == cudaSuccess; ++b) e = cudaMalloc(&S->buf[b], vec);
  if (e == cudaSuccess) e = cudaMalloc(&S->partial, sizeof(double) * max_grid * 2 * kMaxCols);
  if (e == cudaSuccess) e = cudaMalloc(&S->counter, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(S->counter, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&S->cg, sizeof(CgScalars));
  if (e == cudaSuccess) e = cudaMemset(S->cg, 0, sizeof(CgScalars));
  if (e == cudaSuccess) e = cudaMalloc(&S->lz, sizeof(LzScalars));
  if (e == cudaSuccess) e = cudaMallocHost(&S->host_active, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    solver_free(S);
    delete S;
    return e == cudaErrorMemoryAllocation ? fail(SPMV_ERR_OOM, "solver work vectors")
                                          : cuda_fail(e, "solver setup");
  }
  *out = S;
  return SPMV_OK;
}

spmv_status spmv_solver_destroy(spmv_solver_handle S) {
  if (!S) return SPMV_OK;
  {
    SolverDeviceGuard g(S->device);
    cudaDeviceSynchronize();
    solver_free(S);
  }
  delete S;
  return SPMV_OK;
}

spmv_status spmv_cg_solve(spmv_solver_handle S, const double* B_dev, double* X_dev, int32_t max_iter, double rtol,
                          int32_t check_every, void* stream, int32_t* iterations_host, double* rr_host,
                          spmv_cg_summary* summary) {
  if (!S) return fail(SPMV_ERR_ARG, "solver handle is NULL");
  if (max_iter < 0 || check_every < 1 || !(rtol >= 0.0)) return fail(SPMV_ERR_ARG, "bad max_iter, check_every or rtol");
  if (S->n > 0 && (!B_dev || !X_dev)) return fail(SPMV_ERR_ARG, "B or X is NULL");
  if ((((uintptr_t)B_dev) | ((uintptr_t)X_dev)) & 15) return fail(SPMV_ERR_ARG, "B and X must be 16-byte aligned");
  SolverDeviceGuard g(S->device);
  cudaStream_t s = (cudaStream_t)stream;
  CgScalars host{};
  if (S->n > 0) {
    // R = B - A X0, P = R, scalars
    spmv_status st = spmv_apply_block(S->A, X_dev, S->k, S->k, S->buf[2], S->k, s);
    if (st != SPMV_OK) return st;
    cudaError_t e = by_k<LCgInit>(S->k, S->grid[KI_CG_INIT], s, S->n, S->k, B_dev, (const double*)S->buf[2],
                                  S->buf[0], S->buf[1], S->partial, S->counter, S->cg, rtol * rtol);
    if (e != cudaSuccess) return cuda_fail(e, "CG init launch");
    const int steps = check_every < max_iter ? check_every : (max_iter > 0 ? max_iter : 1);
    const uint64_t gen = plan_generation(S->A);
    if (max_iter > 0 &&
        (!S->graph || S->g_B != B_dev || S->g_X != X_dev || S->g_steps != steps || S->g_gen != gen)) {
      if (S->graph) cudaGraphExecDestroy(S->graph);
      S->graph = nullptr;
      cudaGraph_t gr = nullptr;
      SPMV_CUDA(cudaStreamBeginCapture(S->cap, cudaStreamCaptureModeThreadLocal));
      spmv_status cst = SPMV_OK;
      for (int it = 0; it < steps && cst == SPMV_OK; ++it) cst = cg_iteration(S, X_dev, S->cap);
      cudaError_t ce = cudaStreamEndCapture(S->cap, &gr);
      if (cst != SPMV_OK) {
        if (gr) cudaGraphDestroy(gr);
        return cst;
      }
      if (ce != cudaSuccess) return cuda_fail(ce, "CG graph capture");
      ce = cudaGraphInstantiate(&S->graph, gr, 0);
      cudaGraphDestroy(gr);
      if (ce != cudaSuccess) {
        S->graph = nullptr;
        return cuda_fail(ce, "CG graph instantiate");
      }
      S->g_B = B_dev;
      S->g_X = X_dev;
      S->g_steps = steps;
      S->g_gen = gen;
    }
    int done = 0;
    while (done < max_iter) {
      // whole graphs while they fit; the remainder one iteration at a time
      if (max_iter - done >= S->g_steps) {
        SPMV_CUDA(cudaGraphLaunch(S->graph, s));
        done += S->g_steps;
      } else {
        spmv_status ist = cg_iteration(S, X_dev, s);
        if (ist != SPMV_OK) return ist;
        done += 1;
        if (done < max_iter && (done % S->g_steps) != 0) continue;
      }
      SPMV_CUDA(cudaMemcpyAsync(S->host_active, &S->cg->n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
      SPMV_CUDA(cudaEventRecord(S->ev, s));
      SPMV_CUDA(cudaEventSynchronize(S->ev));
      if (*S->host_active == 0) break;
    }
    SPMV_CUDA(cudaMemcpyAsync(&host, S->cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA(cudaStreamSynchronize(s));
  }
  int it_max = 0, conv = 0, bd = 0;
  for (int q = 0; q < S->k; ++q) {
    if (iterations_host) iterations_host[q] = host.iters[q];
    if (rr_host) rr_host[q] = host.rr[q];
    it_max = host.iters[q] > it_max ? host.iters[q] : it_max;
    bd += host.breakdown[q];
    conv += !host.breakdown[q] && !(host.rr[q] > host.tol2[q]);
  }
  if (summary) {
    std::memset(summary, 0, sizeof(*summary));
    summary->iterations = it_max;
    summary->converged = S->n > 0 ? conv : S->k;
    summary->breakdown = bd;
  }
  return SPMV_OK;
}

spmv_status spmv_lanczos(spmv_solver_handle S, const double* V0_dev, int32_t m, double* alpha_host,
                         double* beta_host, void* stream) {
  if (!S) return fail(SPMV_ERR_ARG, "solver handle is NULL");
  if (m < 1) return fail(SPMV_ERR_ARG, "m must be >= 1");
  if (S->n > 0 && !V0_dev) return fail(SPMV_ERR_ARG, "V0 is NULL");
  if (((uintptr_t)V0_dev) & 15) return fail(SPMV_ERR_ARG, "V0 must be 16-byte aligned");
  if (!alpha_host || !beta_host) return fail(SPMV_ERR_ARG, "alpha or beta is NULL");
  SolverDeviceGuard g(S->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int k = S->k;
  if (S->n == 0) {
    std::memset(alpha_host, 0, sizeof(double) * (size_t)m * k);
    std::memset(beta_host, 0, sizeof(double) * (size_t)m * k);
    return SPMV_OK;
  }
  if (S->lz_cap < m) {
    if (S->lz_out) cudaFree(S->lz_out);
    S->lz_out = nullptr;
    S->lz_cap = 0;
    SPMV_CUDA(cudaMalloc(&S->lz_out, sizeof(double) * 2 * (size_t)m * kMaxCols));
    S->lz_cap = m;
  }
  double* a_out = S->lz_out;
  double* b_out = S->lz_out + (size_t)m * kMaxCols;
  double *v_prev = S->buf[0], *v = S->buf[1], *W = S->buf[2];
  cudaError_t e = by_k<LLzNorm>(k, S->grid[KI_LZ_NORM], s, S->n, k, V0_dev, S->partial, S->counter, S->lz);
  if (e == cudaSuccess)
    e = by_k<LLzScale>(k, S->grid[KI_LZ_SCALE], s, S->n, k, V0_dev, v, v_prev, (const LzScalars*)S->lz);
  if (e == cudaSuccess) e = cudaMemsetAsync(S->lz->b_prev, 0, sizeof(double) * kMaxCols, s);
  if (e != cudaSuccess) return cuda_fail(e, "Lanczos start");
  for (int j = 0; j < m; ++j) {
    spmv_status st = spmv_apply_block(S->A, v, k, k, W, k, s);
    if (st != SPMV_OK) return st;
    e = by_k<LLzAlpha>(k, S->grid[KI_LZ_ALPHA], s, S->n, k, W, (const double*)v, (const double*)v_prev, S->partial,
                       S->counter, S->lz, a_out + (size_t)j * kMaxCols);
    if (e == cudaSuccess)
      e = by_k<LLzBeta>(k, S->grid[KI_LZ_BETA], s, S->n, k, W, (const double*)v, S->partial, S->counter, S->lz,
                        b_out + (size_t)j * kMaxCols);
    // v_{j+1} = W / beta_j into the buffer of v_{j-1}, then rotate
    if (e == cudaSuccess)
      e = by_k<LLzScale>(k, S->grid[KI_LZ_SCALE], s, S->n, k, (const double*)W, v_prev, (double*)nullptr,
                         (const LzScalars*)S->lz);
    if (e != cudaSuccess) return cuda_fail(e, "Lanczos kernel launch");
    double* t = v_prev;
    v_prev = v;
    v = t;
  }
  std::vector<double> tmp((size_t)2 * m * kMaxCols);
  SPMV_CUDA(cudaMemcpyAsync(tmp.data(), S->lz_out, sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost, s));
  SPMV_CUDA(cudaStreamSynchronize(s));
  for (int j = 0; j < m; ++j)
    for (int q = 0; q < k; ++q) {
      alpha_host[(size_t)j * k + q] = tmp[(size_t)j * kMaxCols + q];
      beta_host[(size_t)j * k + q] = tmp[(size_t)(m + j) * kMaxCols + q];
    }
  return SPMV_OK;
}

}  // extern "C"
