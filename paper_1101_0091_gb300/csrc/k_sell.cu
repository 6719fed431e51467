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
#include "device.cuh"

namespace spmv {

template <typename VT, int K, bool VEC>
__global__ void __launch_bounds__(kThreads)
    k_sell(int64_t n_rows, int64_t n_chunks, const int32_t* __restrict__ perm,
           const int64_t* __restrict__ chunk_ptr, const int32_t* __restrict__ chunk_len,
           const int32_t* __restrict__ col, const VT* __restrict__ val, const double* __restrict__ B,
           int64_t ldb, double* __restrict__ C, int64_t ldc, int k, int prefetch) {
  constexpr int CPC = kThreads / kSellC;  // chunks per CTA
  if (threadIdx.x == 0 && prefetch > 0) {
    // bring the slots of the CTA `prefetch` positions ahead into L2 (chunk
    // offsets are multiples of 32 slots, so the ranges are 16-byte aligned)
    const int64_t c0 = ((int64_t)blockIdx.x + prefetch) * CPC;
    if (c0 < n_chunks) {
      const int64_t c1 = c0 + CPC < n_chunks ? c0 + CPC : n_chunks;
      const int64_t s0 = __ldg(chunk_ptr + c0), s1 = __ldg(chunk_ptr + c1);
      if (s1 > s0) {
        prefetch_l2(val + s0, (uint32_t)((s1 - s0) * (int64_t)sizeof(VT)));
        prefetch_l2(col + s0, (uint32_t)((s1 - s0) * 4));
      }
    }
  }
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
    if (VEC) {  // k == K >= 8, 16-byte aligned rows of B: one 16-byte gather per two columns
#pragma unroll
      for (int u = 0; u < NB; ++u)
#pragma unroll
        for (int q = 0; q < K; q += 2) {
          const double2 t2 = j + u < len ? __ldg(reinterpret_cast<const double2*>(b[u] + q)) : make_double2(0.0, 0.0);
          g[u][q] = t2.x;
          g[u][q + 1] = t2.y;
        }
    } else {
#pragma unroll
      for (int u = 0; u < NB; ++u)
#pragma unroll
        for (int q = 0; q < K; ++q) g[u][q] = (j + u < len && q < k) ? __ldg(b[u] + q) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < NB; ++u)
#pragma unroll
      for (int q = 0; q < K; ++q)
        if (j + u < len && q < k) acc[q] = fma(v[u], g[u][q], acc[q]);
  }
  if (r >= n_rows) return;
  double* out = C + (int64_t)__ldg(perm + r) * ldc;
  if (VEC) {
#pragma unroll
    for (int q = 0; q < K; q += 2) reinterpret_cast<double2*>(out)[q / 2] = make_double2(acc[q], acc[q + 1]);
    return;
  }
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (q < k) out[q] = acc[q];
}

template <typename VT, int K>
static cudaError_t launch_sell_t(const SellDev& S, const VT* val, const double* B, int64_t ldb, double* C,
                                 int64_t ldc, int k, cudaStream_t s) {
  if (S.n_chunks == 0) return cudaSuccess;
  const int64_t threads = S.n_chunks * kSellC;
  const int64_t grid = (threads + kThreads - 1) / kThreads;
  const bool vec = K >= 8 && k == K && ldb % 2 == 0 && ldc % 2 == 0 && (((uintptr_t)B | (uintptr_t)C) & 15) == 0;
  if (vec)
    k_sell<VT, K, (K >= 8)><<<(unsigned)grid, kThreads, 0, s>>>(S.n_rows, S.n_chunks, S.perm, S.chunk_ptr,
                                                                 S.chunk_len, S.col, val, B, ldb, C, ldc, k,
                                                                 S.prefetch);
  else
    k_sell<VT, K, false><<<(unsigned)grid, kThreads, 0, s>>>(S.n_rows, S.n_chunks, S.perm, S.chunk_ptr,
                                                             S.chunk_len, S.col, val, B, ldb, C, ldc, k, S.prefetch);
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
