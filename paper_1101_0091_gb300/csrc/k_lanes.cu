// CRS_L{1,2,4,8,16,32}: L lanes per row, loads straight from HBM (Sec. 1.2 loop).
//
// A group of L consecutive lanes owns one row; lane t of the group takes
// entries rs + t, rs + t + L, ... (for L >= 8 a group's loads of val/col_idx
// coalesce), gathers B with read-only loads and keeps FP64 partial sums, which
// an xor-shuffle tree of log2(L) steps adds at the end.  L = 1 is the classic
// scalar CRS kernel.  The same kernel with a row list and accumulate = 1 is the
// halo pass of the local/halo split: C[rows[t]] += (halo row t) * B.
#include "device.cuh"

namespace spmv {

template <typename VT, int L, int K>
__global__ void __launch_bounds__(kThreads)
    k_crs_lanes(int64_t n_rows, const int32_t* __restrict__ rows, const int32_t* __restrict__ row_ptr,
                const int32_t* __restrict__ col, const VT* __restrict__ val, const double* __restrict__ B,
                int64_t ldb, double* __restrict__ C, int64_t ldc, int k, int accumulate) {
  const int64_t g = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / L;
  const int t = threadIdx.x % L;
  const bool active = g < n_rows;
  int rs = 0, re = 0;
  if (active) {
    rs = __ldg(row_ptr + g);
    re = __ldg(row_ptr + g + 1);
  }
  double acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0.0;
  int j = rs + t;
  if (L == 1) {
    // two entries per step so that two gathers are in flight
    for (; j + 1 < re; j += 2) {
      const double v0 = to_f64(ldg(val + j)), v1 = to_f64(ldg(val + j + 1));
      const double* b0 = B + (int64_t)ldg(col + j) * ldb;
      const double* b1 = B + (int64_t)ldg(col + j + 1) * ldb;
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
  }
  for (; j < re; j += L) {
    const double v = to_f64(L >= 8 ? ldcs(val + j) : ldg(val + j));
    const double* b = B + (int64_t)(L >= 8 ? ldcs(col + j) : ldg(col + j)) * ldb;
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (q < k) acc[q] = fma(v, __ldg(b + q), acc[q]);
  }
  if (L > 1) {
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = warp_sum_xor(acc[q], L);
  }
  if (!active) return;
  const int64_t row = rows ? (int64_t)__ldg(rows + g) : g;
  double* out = C + row * ldc;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    if (q < k && (L == 1 || t == q % L)) out[q] = accumulate ? out[q] + acc[q] : acc[q];
  }
}

template <typename VT, int L, int K>
static cudaError_t launch_lanes_t(int64_t n_rows, const int32_t* rows, const int32_t* row_ptr,
                                  const int32_t* col, const VT* val, const double* B, int64_t ldb, double* C,
                                  int64_t ldc, int k, bool acc, cudaStream_t s) {
  if (n_rows == 0) return cudaSuccess;
  const int64_t rows_per_cta = kThreads / L;
  const int64_t grid = (n_rows + rows_per_cta - 1) / rows_per_cta;
  k_crs_lanes<VT, L, K><<<(unsigned)grid, kThreads, 0, s>>>(n_rows, rows, row_ptr, col, val, B, ldb, C, ldc, k,
                                                            acc ? 1 : 0);
  return cudaGetLastError();
}

template <typename VT, int L>
static cudaError_t lanes_k(int64_t n, const int32_t* rows, const int32_t* rp, const int32_t* col, const VT* val,
                           const double* B, int64_t ldb, double* C, int64_t ldc, int k, bool acc,
                           cudaStream_t s) {
  if (k <= 1) return launch_lanes_t<VT, L, 1>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, s);
  if (k <= 2) return launch_lanes_t<VT, L, 2>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, s);
  if (k <= 4) return launch_lanes_t<VT, L, 4>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, s);
  if (k <= 8) return launch_lanes_t<VT, L, 8>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, s);
  return launch_lanes_t<VT, L, 16>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, s);
}

template <typename VT>
static cudaError_t lanes_dispatch(int lanes, int64_t n, const int32_t* rows, const int32_t* rp,
                                  const int32_t* col, const VT* val, const double* B, int64_t ldb, double* C,
                                  int64_t ldc, int k, bool acc, cudaStream_t s) {
  switch (lanes) {
    case 1: return lanes_k<VT, 1>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, s);
    case 2: return lanes_k<VT, 2>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, s);
    case 4: return lanes_k<VT, 4>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, s);
    case 8: return lanes_k<VT, 8>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, s);
    case 16: return lanes_k<VT, 16>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, s);
    case 32: return lanes_k<VT, 32>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_crs_lanes(const CsrDev& A, bool fp32, int lanes, const double* B, int64_t ldb, double* C,
                             int64_t ldc, int k, cudaStream_t s) {
  if (fp32) return lanes_dispatch<float>(lanes, A.n_rows, nullptr, A.row_ptr, A.col, A.val32, B, ldb, C, ldc, k,
                                         false, s);
  return lanes_dispatch<double>(lanes, A.n_rows, nullptr, A.row_ptr, A.col, A.val, B, ldb, C, ldc, k, false, s);
}

cudaError_t launch_halo(const HaloDev& H, bool fp32, const double* B, int64_t ldb, double* C, int64_t ldc, int k,
                        cudaStream_t s) {
  if (fp32) return lanes_dispatch<float>(1, H.n_rows, H.rows, H.row_ptr, H.col, H.val32, B, ldb, C, ldc, k, true,
                                         s);
  return lanes_dispatch<double>(1, H.n_rows, H.rows, H.row_ptr, H.col, H.val, B, ldb, C, ldc, k, true, s);
}

}  // namespace spmv
