// Device side of the batched product: member table, work items and the
// persistent kernel (shared by the batch API and its allocation-free entry).
#pragma once

#include "device.cuh"

namespace spmv {

struct BatchMat {
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val;
  const double* B;
  double* C;
  int64_t ldb, ldc;
  int64_t n_rows;
};

// Work item.  mode 0: rows [p0, p1) of member `mat`, bounds from row_ptr.
// mode 1: the rows listed at positions [p0, p1) of the (row, first entry)
// list, all of length `len` (the length-binned rows of the adaptive policy).
// mode 2: listed rows of unequal lengths (ends from row_ptr).
// mode 3: chunks [p0, p1) of the length-sorted SELL-32 copy (sorted policy),
// all of length `len`, stored back to back from slot `base`: one lane per row,
// slots column-major inside a chunk.
// L lanes share one row; 32/L rows per warp pass.
struct BatchItem {
  int32_t mat, p0, p1, len;
  int16_t lanes, mode;
  int32_t pad;
  int64_t base;
};

// Length-sorted SELL-32 copy of the short rows of the members with the sorted
// policy: chunk c holds 32 rows (row index perm[32c + t], -1 for padding) of
// chunk_len[c] slots each at chunk_ptr[c] + 32 j + t.
struct BatchSell {
  const int64_t* chunk_ptr;
  const int32_t* chunk_len;
  const int32_t* perm;
  const int32_t* col;
  const double* val;
};

// C is written once per product: streaming (evict-first) stores leave L2 to
// the B blocks of the members in flight.
__device__ __forceinline__ void st_c(double* p, double x) { __stcs(p, x); }
__device__ __forceinline__ void st_c(double2* p, double2 x) { __stcs(p, x); }

// 16-byte loads of two consecutive right-hand-side values when B rows are
// 16-byte aligned (VEC), else single 8-byte loads.
template <int K, bool VEC>
__device__ __forceinline__ void gather_row(const double* __restrict__ b, int k, double (&g)[K]) {
  if (VEC && K >= 2) {
#pragma unroll
    for (int q = 0; q + 1 < K; q += 2) {
      if (q < k) {
        const double2 t = __ldg(reinterpret_cast<const double2*>(b + q));
        g[q] = t.x;
        g[q + 1] = t.y;
      } else {
        g[q] = 0.0;
        g[q + 1] = 0.0;
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < K; ++q) g[q] = (q < k) ? __ldg(b + q) : 0.0;
  }
}

template <int L, int K, bool VEC>
__device__ __forceinline__ void batch_rows(const BatchMat* __restrict__ Mp, const int2* __restrict__ rowlist,
                                           const BatchItem& item, int k, int lane) {
  const BatchMat& M = *Mp;  // fields are read where used, not held across the item
  constexpr int RPP = 32 / L;  // rows per warp pass
  const int t = lane % L;
  for (int base = item.p0; base < item.p1; base += RPP) {
    const int i = base + lane / L;
    const bool active = i < item.p1;
    int r = 0, rs = 0, re = 0;
    if (active) {
      if (item.mode) {
        const int2 e = __ldg(rowlist + i);
        r = e.x;
        rs = e.y;
        re = item.mode == 1 ? rs + item.len : __ldg(M.row_ptr + r + 1);
      } else {
        r = i;
        rs = __ldg(M.row_ptr + r);
        re = __ldg(M.row_ptr + r + 1);
      }
    }
    double acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = 0.0;
    constexpr int NB = (L == 1 && K <= 2) ? 4 / K : 1;  // gathers issued before their FMAs
    for (int j = rs + t; j < re; j += NB * L) {
      double v[NB];
      const double* b[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int jj = (j + u * L < re) ? j + u * L : j;
        v[u] = ldcs(M.val + jj);
        b[u] = M.B + (int64_t)ldcs(M.col + jj) * M.ldb;
      }
      double g[NB][K];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        if (j + u * L < re) {
          gather_row<K, VEC>(b[u], k, g[u]);
        } else {
#pragma unroll
          for (int q = 0; q < K; ++q) g[u][q] = 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < NB; ++u)
#pragma unroll
        for (int q = 0; q < K; ++q)
          if (j + u * L < re && q < k) acc[q] = fma(v[u], g[u][q], acc[q]);
    }
    if (L > 1) {
#pragma unroll
      for (int q = 0; q < K; ++q) acc[q] = warp_sum_xor(acc[q], L);
    }
    if (active) {
      double* out = M.C + (int64_t)r * M.ldc;
      if (VEC && L == 1 && K >= 2) {
#pragma unroll
        for (int q = 0; q + 1 < K; q += 2)
          if (q < k) st_c(reinterpret_cast<double2*>(out + q), make_double2(acc[q], acc[q + 1]));
      } else {
#pragma unroll
        for (int q = 0; q < K; ++q)
          if (q < k && (L == 1 || t == q % L)) st_c(out + q, acc[q]);
      }
    }
  }
}

// Chunks whose rows all have exactly LEN entries, CH chunks per step; returns
// the first chunk left for the generic loop.  Same FMA order per row as the
// generic loop.
template <int LEN, int CH, int K, bool VEC>
__device__ __forceinline__ int chunks_fixed(const BatchMat* __restrict__ Mp, const double* __restrict__ B,
                                            int64_t ldb, const BatchSell& S, const BatchItem& item, int k,
                                            int lane) {
  int c = item.p0;
  for (; c + CH - 1 < item.p1; c += CH) {
    const int64_t s0 = item.base + (int64_t)(c - item.p0) * 32 * LEN + lane;
    int r[CH];
    double v[CH][LEN];
    const double* b[CH][LEN];
#pragma unroll
    for (int h = 0; h < CH; ++h) {
      r[h] = __ldg(S.perm + (int64_t)(c + h) * 32 + lane);
#pragma unroll
      for (int j = 0; j < LEN; ++j) {
        const int64_t slot = s0 + (int64_t)(h * LEN + j) * 32;
        v[h][j] = ldcs(S.val + slot);
        b[h][j] = B + (int64_t)ldcs(S.col + slot) * ldb;
      }
    }
    double g[CH][LEN][K];
#pragma unroll
    for (int h = 0; h < CH; ++h)
#pragma unroll
      for (int j = 0; j < LEN; ++j) gather_row<K, VEC>(b[h][j], k, g[h][j]);
#pragma unroll
    for (int h = 0; h < CH; ++h) {
      double acc[K];
#pragma unroll
      for (int q = 0; q < K; ++q) acc[q] = 0.0;
#pragma unroll
      for (int j = 0; j < LEN; ++j)
#pragma unroll
        for (int q = 0; q < K; ++q) acc[q] = fma(v[h][j], g[h][j][q], acc[q]);
      if (r[h] < 0) continue;
      double* out = Mp->C + (int64_t)r[h] * Mp->ldc;
      if (VEC && K >= 2) {
#pragma unroll
        for (int q = 0; q + 1 < K; q += 2)
          if (q < k) st_c(reinterpret_cast<double2*>(out + q), make_double2(acc[q], acc[q + 1]));
      } else {
#pragma unroll
        for (int q = 0; q < K; ++q)
          if (q < k) st_c(out + q, acc[q]);
      }
    }
  }
  return c;
}

template <int K, bool VEC>
__device__ __forceinline__ void batch_chunks(const BatchMat* __restrict__ Mp, const BatchSell& S,
                                             const BatchItem& item, int k, int lane) {
  struct {
    const double* B;
    int64_t ldb;
  } M = {Mp->B, Mp->ldb};  // only what the inner loop needs stays in registers
  const int len = item.len;  // every chunk of the item has this length: no per-chunk metadata loads
  int c = item.p0;
  // short rows (most rows of a power-law matrix): a fixed length, several
  // chunks per step, every load and gather of a step in flight together
  if (len == 1) c = chunks_fixed<1, K <= 4 ? 4 : 2, K, VEC>(Mp, M.B, M.ldb, S, item, k, lane);
  else if (len == 2) c = chunks_fixed<2, K <= 4 ? 2 : 1, K, VEC>(Mp, M.B, M.ldb, S, item, k, lane);
  else if (len == 3 && K <= 4) c = chunks_fixed<3, 1, K, VEC>(Mp, M.B, M.ldb, S, item, k, lane);
  else if (len == 4 && K <= 4) c = chunks_fixed<4, 1, K, VEC>(Mp, M.B, M.ldb, S, item, k, lane);
  for (; c < item.p1; ++c) {
    const int64_t base = item.base + (int64_t)(c - item.p0) * 32 * len + lane;
    const int r = __ldg(S.perm + (int64_t)c * 32 + lane);
    double acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = 0.0;
    constexpr int NB = K <= 2 ? 4 / K : 1;  // gathers issued before their FMAs
    if (NB == 1) {
      // one slot per step, software-pipelined: the next slot's val/col load is in flight
      // while this slot's gathers are, so only the gathers stay on the critical path
      double v = len > 0 ? ldcs(S.val + base) : 0.0;
      int32_t cc = len > 0 ? ldcs(S.col + base) : 0;
      for (int j = 0; j < len; ++j) {
        double g[K];
        gather_row<K, VEC>(M.B + (int64_t)cc * M.ldb, k, g);
        const int64_t nxt = base + (int64_t)(j + 1 < len ? j + 1 : j) * 32;
        const double v_n = ldcs(S.val + nxt);
        const int32_t c_n = ldcs(S.col + nxt);
#pragma unroll
        for (int q = 0; q < K; ++q)
          if (q < k) acc[q] = fma(v, g[q], acc[q]);
        v = v_n;
        cc = c_n;
      }
    } else {
      for (int j = 0; j < len; j += NB) {
        double v[NB];
        const double* b[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
          const int64_t slot = base + (int64_t)((j + u < len) ? j + u : j) * 32;
          v[u] = ldcs(S.val + slot);
          b[u] = M.B + (int64_t)ldcs(S.col + slot) * M.ldb;
        }
        double g[NB][K];
#pragma unroll
        for (int u = 0; u < NB; ++u) gather_row<K, VEC>(b[u], k, g[u]);
#pragma unroll
        for (int u = 0; u < NB; ++u)
#pragma unroll
          for (int q = 0; q < K; ++q)
            if (j + u < len && q < k) acc[q] = fma(v[u], g[u][q], acc[q]);
      }
    }
    if (r >= 0) {
      double* out = Mp->C + (int64_t)r * Mp->ldc;
      if (VEC && K >= 2) {
#pragma unroll
        for (int q = 0; q + 1 < K; q += 2)
          if (q < k) st_c(reinterpret_cast<double2*>(out + q), make_double2(acc[q], acc[q + 1]));
      } else {
#pragma unroll
        for (int q = 0; q < K; ++q)
          if (q < k) st_c(out + q, acc[q]);
      }
    }
  }
}

// Threads per CTA of the persistent kernels, and the CTAs per SM the register
// budget is sized for: for k <= 4 at 72 registers seven 128-thread CTAs (28
// warps) stay resident (256-thread CTAs held to 64 registers spilled, and only
// three of them fitted on an SM, not four: 24 warps); the wider gathers of
// k = 8 / 16 keep about 100 registers (four or five CTAs) rather than spill.
constexpr int kBatchThreads = 128;
constexpr int kBatchCtasPerSm = 7;
template <int K>
struct BatchMinCtas {
  static constexpr int value = K <= 4 ? kBatchCtasPerSm : 4;
};

// Persistent kernel: warps take items round-robin (dynamic = 0) or from the
// atomic counter (dynamic = 1, counter zeroed before the launch).
// Next item index of the calling warp: round-robin or from the atomic counter.
__device__ __forceinline__ int next_item(int it, int nw, int dynamic, int* counter, int lane) {
  if (!dynamic) return it + nw;
  int v = 0;
  if (lane == 0) v = atomicAdd(counter, 1);
  return __shfl_sync(0xffffffffu, v, 0);
}

// Persistent kernel over row items (modes 0-2).
template <int K, bool VEC>
__global__ void __launch_bounds__(kBatchThreads, BatchMinCtas<K>::value)
    k_batch_rows(const BatchMat* __restrict__ mats, const BatchItem* __restrict__ items, int n_items,
                 const int2* __restrict__ rowlist, int* __restrict__ counter, int dynamic, int k) {
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * (kBatchThreads / 32) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (kBatchThreads / 32);
  int it = dynamic ? next_item(0, nw, 1, counter, lane) : wid;
  while (it < n_items) {
    const BatchItem item = items[it];
    switch (item.lanes) {
      case 1: batch_rows<1, K, VEC>(mats + item.mat, rowlist, item, k, lane); break;
      case 2: batch_rows<2, K, VEC>(mats + item.mat, rowlist, item, k, lane); break;
      case 4: batch_rows<4, K, VEC>(mats + item.mat, rowlist, item, k, lane); break;
      case 8: batch_rows<8, K, VEC>(mats + item.mat, rowlist, item, k, lane); break;
      case 16: batch_rows<16, K, VEC>(mats + item.mat, rowlist, item, k, lane); break;
      default: batch_rows<32, K, VEC>(mats + item.mat, rowlist, item, k, lane); break;
    }
    it = next_item(it, nw, dynamic, counter, lane);
  }
}

// Persistent kernel over all item modes.  Sorted-chunk items and row items of
// one member stay next to each other in the list, so a member's B block is
// gathered while it is resident in L2 (two separate kernels, one per mode,
// would stream every B block twice).
template <int K, bool VEC>
__global__ void __launch_bounds__(kBatchThreads, BatchMinCtas<K>::value)
    k_batch(const BatchMat* __restrict__ mats, const BatchItem* __restrict__ items, int n_items,
            const int2* __restrict__ rowlist, BatchSell sell, int* __restrict__ counter, int dynamic, int k) {
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * (kBatchThreads / 32) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (kBatchThreads / 32);
  int it = dynamic ? next_item(0, nw, 1, counter, lane) : wid;
  while (it < n_items) {
    const BatchItem item = items[it];
    if (item.mode == 3) {
      batch_chunks<K, VEC>(mats + item.mat, sell, item, k, lane);
    } else {
      switch (item.lanes) {
        case 1: batch_rows<1, K, VEC>(mats + item.mat, rowlist, item, k, lane); break;
        case 2: batch_rows<2, K, VEC>(mats + item.mat, rowlist, item, k, lane); break;
        case 4: batch_rows<4, K, VEC>(mats + item.mat, rowlist, item, k, lane); break;
        case 8: batch_rows<8, K, VEC>(mats + item.mat, rowlist, item, k, lane); break;
        case 16: batch_rows<16, K, VEC>(mats + item.mat, rowlist, item, k, lane); break;
        default: batch_rows<32, K, VEC>(mats + item.mat, rowlist, item, k, lane); break;
      }
    }
    it = next_item(it, nw, dynamic, counter, lane);
  }
}

template <bool VEC>
static const void* batch_rows_kernel_t(int k) {
  if (k <= 1) return (const void*)k_batch_rows<1, false>;
  if (k <= 2) return (const void*)k_batch_rows<2, VEC>;
  if (k <= 4) return (const void*)k_batch_rows<4, VEC>;
  if (k <= 8) return (const void*)k_batch_rows<8, VEC>;
  return (const void*)k_batch_rows<16, VEC>;
}

template <bool VEC>
static const void* batch_kernel_t(int k) {
  if (k <= 1) return (const void*)k_batch<1, false>;
  if (k <= 2) return (const void*)k_batch<2, VEC>;
  if (k <= 4) return (const void*)k_batch<4, VEC>;
  if (k <= 8) return (const void*)k_batch<8, VEC>;
  return (const void*)k_batch<16, VEC>;
}

// The kernels for k right-hand sides; vec: every member's B and C rows are
// 16-byte aligned and k is even (16-byte loads and stores).  The rows-only
// variant serves work lists without sorted chunks.
static inline const void* batch_rows_kernel(int k, bool vec) {
  return vec ? batch_rows_kernel_t<true>(k) : batch_rows_kernel_t<false>(k);
}
static inline const void* batch_kernel(int k, bool vec) {
  return vec ? batch_kernel_t<true>(k) : batch_kernel_t<false>(k);
}

}  // namespace spmv
