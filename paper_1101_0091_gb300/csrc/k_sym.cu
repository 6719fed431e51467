// SYM: symmetric CRS (Sec. 1.3.1).  Only the entries of each row with
// col >= row are stored, so val/col_idx traffic is about half that of CRS.
//
// One thread per row i.  A stored entry u(i,j) adds u(i,j)*B(j) to the row's
// FP64 sum (one FMA) and, for j != i, its mirror u(i,j)*B(i) to C(j) through an
// FP64 atomic add whose result is unused (a reduction performed at L2).  The
// row's own sum goes to C(i) the same way at the end, because mirrors from
// other rows reach C(i) at any time.  C is zeroed on the stream first.  The
// order in which the contributions of a row meet is not fixed, so results vary
// by rounding from call to call (integer-valued products stay exact).
#include "device.cuh"

namespace spmv {

template <typename VT, int K>
__global__ void __launch_bounds__(kThreads, (K == 1 ? 6 : 1))
    k_sym(int64_t n_rows, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
          const VT* __restrict__ val, const double* __restrict__ B, int64_t ldb, double* C, int64_t ldc, int k,
          int prefetch) {
  if (threadIdx.x == 0 && prefetch > 0) {
    // bring the val/col slices of the CTA `prefetch` positions ahead into L2
    const int64_t f0 = ((int64_t)blockIdx.x + prefetch) * kThreads;
    if (f0 < n_rows) {
      const int64_t f1 = f0 + kThreads < n_rows ? f0 + kThreads : n_rows;
      const int bs = __ldg(row_ptr + f0), be = __ldg(row_ptr + f1);
      constexpr int VA = 16 / (int)sizeof(VT);
      const int v_lo = bs & ~(VA - 1), v_hi = (be + VA - 1) & ~(VA - 1);
      const int c_lo = bs & ~3, c_hi = (be + 3) & ~3;
      if (be > bs) {
        prefetch_l2(val + v_lo, (uint32_t)(v_hi - v_lo) * (uint32_t)sizeof(VT));
        prefetch_l2(col + c_lo, (uint32_t)(c_hi - c_lo) * 4u);
      }
    }
  }
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n_rows) return;
  const int rs = __ldg(row_ptr + i), re = __ldg(row_ptr + i + 1);
  double xi[K], acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    xi[q] = q < k ? __ldg(B + i * ldb + q) : 0.0;
    acc[q] = 0.0;
  }
  // batches of NB entries: all loads and gathers of a batch are issued before its arithmetic
  // (4 entries per batch keep K = 1 within the 40 registers of 6 resident CTAs)
  constexpr int NB = 4 / K > 0 ? 4 / K : 1;
  for (int j = rs; j < re; j += NB) {
    double v[NB];
    int32_t c[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int jj = (j + u < re) ? j + u : j;
      v[u] = to_f64(ldg(val + jj));
      c[u] = ldg(col + jj);
    }
    double gv[NB][K];
#pragma unroll
    for (int u = 0; u < NB; ++u)
#pragma unroll
      for (int q = 0; q < K; ++q) gv[u][q] = (j + u < re && q < k) ? __ldg(B + (int64_t)c[u] * ldb + q) : 0.0;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      if (j + u < re) {
#pragma unroll
        for (int q = 0; q < K; ++q)
          if (q < k) acc[q] = fma(v[u], gv[u][q], acc[q]);
        if (c[u] != i) {
          double* mirror = C + (int64_t)c[u] * ldc;
#pragma unroll
          for (int q = 0; q < K; ++q)
            if (q < k) atomicAdd(mirror + q, v[u] * xi[q]);
        }
      }
    }
  }
  double* out = C + i * ldc;
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (q < k) atomicAdd(out + q, acc[q]);
}

template <typename VT, int K>
static cudaError_t launch_sym_t(const SymDev& S, const VT* val, const double* B, int64_t ldb, double* C,
                                int64_t ldc, int k, cudaStream_t s) {
  const int64_t grid = (S.n_rows + kThreads - 1) / kThreads;
  k_sym<VT, K><<<(unsigned)grid, kThreads, 0, s>>>(S.n_rows, S.row_ptr, S.col, val, B, ldb, C, ldc, k,
                                                   S.prefetch);
  return cudaGetLastError();
}

template <typename VT>
static cudaError_t sym_k(const SymDev& S, const VT* val, const double* B, int64_t ldb, double* C, int64_t ldc,
                         int k, cudaStream_t s) {
  if (k <= 1) return launch_sym_t<VT, 1>(S, val, B, ldb, C, ldc, k, s);
  if (k <= 2) return launch_sym_t<VT, 2>(S, val, B, ldb, C, ldc, k, s);
  if (k <= 4) return launch_sym_t<VT, 4>(S, val, B, ldb, C, ldc, k, s);
  if (k <= 8) return launch_sym_t<VT, 8>(S, val, B, ldb, C, ldc, k, s);
  return launch_sym_t<VT, 16>(S, val, B, ldb, C, ldc, k, s);
}

cudaError_t launch_sym(const SymDev& S, bool fp32, const double* B, int64_t ldb, double* C, int64_t ldc, int k,
                       cudaStream_t s) {
  if (S.n_rows == 0) return cudaSuccess;
  cudaError_t e = ldc == k ? cudaMemsetAsync(C, 0, sizeof(double) * (size_t)(S.n_rows * k), s)
                           : cudaMemset2DAsync(C, sizeof(double) * (size_t)ldc, 0, sizeof(double) * (size_t)k,
                                               (size_t)S.n_rows, s);
  if (e != cudaSuccess) return e;
  if (fp32 && S.val32_special) return sym_k<float>(S, S.val32, B, ldb, C, ldc, k, s);
  if (fp32) return sym_k<f32n>(S, reinterpret_cast<const f32n*>(S.val32), B, ldb, C, ldc, k, s);
  return sym_k<double>(S, S.val, B, ldb, C, ldc, k, s);
}

}  // namespace spmv
