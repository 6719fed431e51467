// SELL-C-sigma product, C = 32 (Kreutzer et al. 2014 format; the paper's CRS
// loop of Sec. 1.2 applied to the sliced, sorted, column-major form).
//
// One warp per chunk, one lane per sorted row: slot j of lane t lives at
// chunk_ptr[c] + 32*j + t, so each load instruction of a warp reads 32
// consecutive entries (256 B of FP64 values, 128 B of indices).  Every lane
// runs chunk_len[c] steps; padding slots hold +0.0 and a valid column, so they
// add exactly +0.0 and need no test.  The row sum goes to C[perm[r]].  Sorting
// rows by length inside sigma-windows keeps the padding (idle FP64 issue
// slots) small.
//
// A full, 16-byte aligned block of K >= 2 columns runs k_sell_cols: each
// sorted row is shared by G = K / W lanes (W = 4 columns per lane for K >= 8,
// all K below), every gather is a 16-byte load, and the G lanes of a row read
// one contiguous piece of its B row; a row's slots are still summed in order,
// so the bits equal the scalar form's.
#include "device.cuh"

namespace spmv {

// Bring the slots of chunks [c0, c0 + chunks) into L2 (one thread; chunk
// offsets are multiples of 32 slots, so the ranges are 16-byte aligned).
template <typename VT>
__device__ __forceinline__ void prefetch_chunks(int64_t c0, int64_t chunks, int64_t n_chunks,
                                                const int64_t* __restrict__ chunk_ptr,
                                                const int32_t* __restrict__ col, const VT* __restrict__ val) {
  if (c0 >= n_chunks) return;
  const int64_t c1 = c0 + chunks < n_chunks ? c0 + chunks : n_chunks;
  const int64_t s0 = __ldg(chunk_ptr + c0), s1 = __ldg(chunk_ptr + c1);
  if (s1 > s0) {
    prefetch_l2(val + s0, (uint32_t)((s1 - s0) * (int64_t)sizeof(VT)));
    prefetch_l2(col + s0, (uint32_t)((s1 - s0) * 4));
  }
}

template <typename VT, int K>
__global__ void __launch_bounds__(kThreads)
    k_sell(int64_t n_rows, int64_t n_chunks, const int32_t* __restrict__ perm,
           const int64_t* __restrict__ chunk_ptr, const int32_t* __restrict__ chunk_len,
           const int32_t* __restrict__ col, const VT* __restrict__ val, const double* __restrict__ B,
           int64_t ldb, double* __restrict__ C, int64_t ldc, int k, int prefetch) {
  constexpr int CPC = kThreads / kSellC;  // chunks per CTA
  // bring the slots of the CTA `prefetch` positions ahead into L2
  if (threadIdx.x == 0 && prefetch > 0)
    prefetch_chunks(((int64_t)blockIdx.x + prefetch) * CPC, CPC, n_chunks, chunk_ptr, col, val);
  const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int64_t c = r >> 5;
  if (c >= n_chunks) return;
  const int t = threadIdx.x & 31;
  const int len = __ldg(chunk_len + c);
  const int64_t base = __ldg(chunk_ptr + c) + t;
  double acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0.0;
  // batches of NB slots: all gathers of a batch are issued before its FMAs
  constexpr int NB = K >= 4 ? 1 : 2;
  for (int j = 0; j < len; j += NB) {
    double v[NB];
    const double* b[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int64_t slot = base + (int64_t)((j + u < len) ? j + u : j) * kSellC;
      v[u] = to_f64(ldcs(val + slot));
      b[u] = B + (int64_t)ldcs(col + slot) * ldb;
    }
    double g[NB][K];
#pragma unroll
    for (int u = 0; u < NB; ++u)
#pragma unroll
      for (int q = 0; q < K; ++q) g[u][q] = (j + u < len && q < k) ? __ldg(b[u] + q) : 0.0;
#pragma unroll
    for (int u = 0; u < NB; ++u)
#pragma unroll
      for (int q = 0; q < K; ++q)
        if (j + u < len && q < k) acc[q] = fma(v[u], g[u][q], acc[q]);
  }
  if (r >= n_rows) return;
  double* out = C + (int64_t)__ldg(perm + r) * ldc;
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (q < k) out[q] = acc[q];
}

// Columns per lane of the column-split form.
template <int K>
struct SellColsPerLane {
  static constexpr int value = K >= 8 ? 4 : K;
};

template <typename VT, int K>
__global__ void __launch_bounds__(kThreads, 6)
    k_sell_cols(int64_t n_rows, int64_t n_chunks, const int32_t* __restrict__ perm,
                const int64_t* __restrict__ chunk_ptr, const int32_t* __restrict__ chunk_len,
                const int32_t* __restrict__ col, const VT* __restrict__ val, const double* __restrict__ B,
                int64_t ldb, double* __restrict__ C, int64_t ldc, int prefetch) {
  constexpr int W = SellColsPerLane<K>::value;
  constexpr int G = K / W;                      // lanes per row
  constexpr int CPC = kThreads / (kSellC * G);  // chunks per CTA
  if (threadIdx.x == 0 && prefetch > 0)
    prefetch_chunks(((int64_t)blockIdx.x + prefetch) * CPC, CPC, n_chunks, chunk_ptr, col, val);
  const int64_t ra = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int64_t r = ra / G;  // sorted row
  const int64_t c = r >> 5;
  if (c >= n_chunks) return;
  const int c0 = (int)(ra % G) * W;  // first column of this lane
  const int len = __ldg(chunk_len + c);
  const int64_t base = __ldg(chunk_ptr + c) + (r & (kSellC - 1));
  double acc[W];
#pragma unroll
  for (int q = 0; q < W; ++q) acc[q] = 0.0;
  const double* Bc = B + c0;
  for (int j = 0; j < len; ++j) {
    const int64_t slot = base + (int64_t)j * kSellC;
    const double v = to_f64(ldcs(val + slot));
    const double* b = Bc + (int64_t)ldcs(col + slot) * ldb;
    double g[W];
#pragma unroll
    for (int q = 0; q < W; q += 2) {
      const double2 x = __ldg(reinterpret_cast<const double2*>(b + q));
      g[q] = x.x;
      g[q + 1] = x.y;
    }
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = fma(v, g[q], acc[q]);
  }
  if (r >= n_rows) return;
  double2* out = reinterpret_cast<double2*>(C + (int64_t)__ldg(perm + r) * ldc + c0);
#pragma unroll
  for (int q = 0; q < W; q += 2) out[q / 2] = make_double2(acc[q], acc[q + 1]);
}

template <typename VT, int K>
static cudaError_t launch_sell_t(const SellDev& S, const VT* val, const double* B, int64_t ldb, double* C,
                                 int64_t ldc, int k, cudaStream_t s) {
  if (S.n_chunks == 0) return cudaSuccess;
  if constexpr (K >= 2) {
    // a full block of K columns with 16-byte aligned rows: the column-split form (these
    // products are FP64-pipe-bound; on the eigenproblem-shaped matrix it took K = 2 / 4 / 16
    // from 0.59 / 0.71 / 0.88 to 0.82 / 0.94 / 0.97 of the FP64 peak)
    if (k == K && ldb % 2 == 0 && ldc % 2 == 0 && (((uintptr_t)B | (uintptr_t)C) & 15) == 0) {
      constexpr int G = K / SellColsPerLane<K>::value;
      const int64_t grid = (S.n_chunks * kSellC * G + kThreads - 1) / kThreads;
      k_sell_cols<VT, K><<<(unsigned)grid, kThreads, 0, s>>>(S.n_rows, S.n_chunks, S.perm, S.chunk_ptr,
                                                              S.chunk_len, S.col, val, B, ldb, C, ldc, S.prefetch);
      return cudaGetLastError();
    }
  }
  const int64_t threads = S.n_chunks * kSellC;
  const int64_t grid = (threads + kThreads - 1) / kThreads;
  k_sell<VT, K><<<(unsigned)grid, kThreads, 0, s>>>(S.n_rows, S.n_chunks, S.perm, S.chunk_ptr, S.chunk_len, S.col,
                                                     val, B, ldb, C, ldc, k, S.prefetch);
  return cudaGetLastError();
}

template <typename VT>
static cudaError_t sell_k(const SellDev& S, const VT* val, const double* B, int64_t ldb, double* C, int64_t ldc,
                          int k, cudaStream_t s) {
  if (k <= 1) return launch_sell_t<VT, 1>(S, val, B, ldb, C, ldc, k, s);
  if (k <= 2) return launch_sell_t<VT, 2>(S, val, B, ldb, C, ldc, k, s);
  if (k <= 4) return launch_sell_t<VT, 4>(S, val, B, ldb, C, ldc, k, s);
  if (k <= 8) return launch_sell_t<VT, 8>(S, val, B, ldb, C, ldc, k, s);
  return launch_sell_t<VT, 16>(S, val, B, ldb, C, ldc, k, s);
}

cudaError_t launch_sell(const SellDev& S, bool fp32, const double* B, int64_t ldb, double* C, int64_t ldc, int k,
                        cudaStream_t s) {
  if (fp32 && S.val32_special) return sell_k<float>(S, S.val32, B, ldb, C, ldc, k, s);
  if (fp32) return sell_k<f32n>(S, reinterpret_cast<const f32n*>(S.val32), B, ldb, C, ldc, k, s);
  return sell_k<double>(S, S.val, B, ldb, C, ldc, k, s);
}

}  // namespace spmv
