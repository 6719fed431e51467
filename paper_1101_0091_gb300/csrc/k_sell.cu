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

template <typename VT, int K>
__global__ void __launch_bounds__(kThreads)
    k_sell(int64_t n_rows, int64_t n_chunks, const int32_t* __restrict__ perm,
           const int64_t* __restrict__ chunk_ptr, const int32_t* __restrict__ chunk_len,
           const int32_t* __restrict__ col, const VT* __restrict__ val, const double* __restrict__ B,
           int64_t ldb, double* __restrict__ C, int64_t ldc, int k) {
  const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int64_t c = r >> 5;
  if (c >= n_chunks) return;
  const int t = threadIdx.x & 31;
  const int len = __ldg(chunk_len + c);
  const int64_t base = __ldg(chunk_ptr + c) + t;
  double acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0.0;
  int j = 0;
  for (; j + 2 <= len; j += 2) {
    const int64_t s0 = base + (int64_t)j * kSellC, s1 = s0 + kSellC;
    const double v0 = to_f64(ldcs(val + s0)), v1 = to_f64(ldcs(val + s1));
    const double* b0 = B + (int64_t)ldcs(col + s0) * ldb;
    const double* b1 = B + (int64_t)ldcs(col + s1) * ldb;
    double g0[K], g1[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      g0[q] = (q < k) ? __ldg(b0 + q) : 0.0;
      g1[q] = (q < k) ? __ldg(b1 + q) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (q < k) acc[q] = fma(v1, g1[q], fma(v0, g0[q], acc[q]));
  }
  if (j < len) {
    const int64_t s0 = base + (int64_t)j * kSellC;
    const double v0 = to_f64(ldcs(val + s0));
    const double* b0 = B + (int64_t)ldcs(col + s0) * ldb;
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (q < k) acc[q] = fma(v0, __ldg(b0 + q), acc[q]);
  }
  if (r >= n_rows) return;
  double* out = C + (int64_t)__ldg(perm + r) * ldc;
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
  k_sell<VT, K><<<(unsigned)grid, kThreads, 0, s>>>(S.n_rows, S.n_chunks, S.perm, S.chunk_ptr, S.chunk_len, S.col,
                                                    val, B, ldb, C, ldc, k);
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
  if (fp32) return sell_k<float>(S, S.val32, B, ldb, C, ldc, k, s);
  return sell_k<double>(S, S.val, B, ldb, C, ldc, k, s);
}

}  // namespace spmv
