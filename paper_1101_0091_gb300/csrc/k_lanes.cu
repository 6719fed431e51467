// CRS_L{1,2,4,8,16,32}: L lanes per row, loads straight from HBM (Sec. 1.2 loop).
//
// A group of L consecutive lanes owns one row; lane t of the group takes
// entries rs + t, rs + t + L, ... (for L >= 8 a group's loads of val/col_idx
// coalesce), gathers B with read-only loads and keeps FP64 partial sums, which
// an xor-shuffle tree of log2(L) steps adds at the end.  L = 1 is the classic
// scalar CRS kernel.  The same kernel with a row list and accumulate = 1 is the
// halo pass of the local/halo split: C[rows[t]] += (halo row t) * B.
//
// CRS_L1 on a full, 16-byte aligned block of K >= 2 columns runs k_crs_cols
// instead: the row's entries still go to one lane each in order, but the K
// columns are split over G = K / W lanes (W = 4 columns per lane for K >= 8,
// all K below), so every gather is a 16-byte load and the G lanes of a row
// read one contiguous piece of its B row.  Each column's sum is formed in the
// same order as in the scalar form, so the bits are the same.
#include "device.cuh"

namespace spmv {

// Bring the val/col slices of rows [f0, f0 + rows) into L2 (one thread).
template <typename VT>
__device__ __forceinline__ void prefetch_rows(int64_t f0, int64_t rows, int64_t n_rows,
                                              const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                              const VT* __restrict__ val) {
  if (f0 >= n_rows) return;
  const int64_t f1 = f0 + rows < n_rows ? f0 + rows : n_rows;
  const int bs = __ldg(row_ptr + f0), be = __ldg(row_ptr + f1);
  constexpr int VA = 16 / (int)sizeof(VT);
  const int v_lo = bs & ~(VA - 1), v_hi = (be + VA - 1) & ~(VA - 1);
  const int c_lo = bs & ~3, c_hi = (be + 3) & ~3;
  if (be > bs) {
    prefetch_l2(val + v_lo, (uint32_t)(v_hi - v_lo) * (uint32_t)sizeof(VT));
    prefetch_l2(col + c_lo, (uint32_t)(c_hi - c_lo) * 4u);
  }
}

// VEC (L > 1, a full block of K >= 2 columns with 16-byte aligned B rows): each
// entry's K values are gathered with K / 2 16-byte loads instead of K 8-byte ones.
template <typename VT, int L, int K, bool VEC>
__global__ void __launch_bounds__(kThreads, (K == 1 ? 8 : 1))
    k_crs_lanes(int64_t n_rows, const int32_t* __restrict__ rows, const int32_t* __restrict__ row_ptr,
                const int32_t* __restrict__ col, const VT* __restrict__ val, const double* __restrict__ B,
                int64_t ldb, double* __restrict__ C, int64_t ldc, int k, int accumulate, int prefetch) {
  constexpr int RPC = kThreads / L;  // rows per CTA
  // bring the val/col slices of the CTA `prefetch` positions ahead into L2
  if (threadIdx.x == 0 && prefetch > 0)
    prefetch_rows(((int64_t)blockIdx.x + prefetch) * RPC, RPC, n_rows, row_ptr, col, val);
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
  // batches of NB entries per lane: all gathers of a batch are issued before its FMAs
  constexpr int NB1 = sizeof(VT) == 8 ? 8 : 4;  // single-lane batch (FP32 storage: widening needs registers)
  // (K >= 4: one entry per batch; its K gathers already keep the FP64 pipe fed, and two entries
  // measured 9 % slower at K = 4)
  constexpr int NB = K >= 4 ? 1 : (L >= 4 ? 1 : (L == 2 ? 4 / K : NB1 / K > 0 ? NB1 / K : 1));
  for (int j = rs + t; j < re; j += NB * L) {
    double v[NB];
    const double* b[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int jj = (j + u * L < re) ? j + u * L : j;
      v[u] = to_f64(L >= 8 ? ldcs(val + jj) : ldg(val + jj));
      b[u] = B + (int64_t)(L >= 8 ? ldcs(col + jj) : ldg(col + jj)) * ldb;
    }
    double gv[NB][K];
    if constexpr (VEC) {
#pragma unroll
      for (int u = 0; u < NB; ++u)
#pragma unroll
        for (int q = 0; q < K; q += 2) {
          const double2 x = j + u * L < re ? __ldg(reinterpret_cast<const double2*>(b[u] + q)) : make_double2(0.0, 0.0);
          gv[u][q] = x.x;
          gv[u][q + 1] = x.y;
        }
    } else {
#pragma unroll
      for (int u = 0; u < NB; ++u)
#pragma unroll
        for (int q = 0; q < K; ++q) gv[u][q] = (j + u * L < re && q < k) ? __ldg(b[u] + q) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < NB; ++u)
#pragma unroll
      for (int q = 0; q < K; ++q)
        if (j + u * L < re && q < k) acc[q] = fma(v[u], gv[u][q], acc[q]);
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

// Columns per lane of the column-split form.
template <int K>
struct ColsPerLane {
  static constexpr int value = K >= 8 ? 4 : K;
};

template <typename VT, int K>
__global__ void __launch_bounds__(kThreads, 6)
    k_crs_cols(int64_t n_rows, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
               const VT* __restrict__ val, const double* __restrict__ B, int64_t ldb, double* __restrict__ C,
               int64_t ldc, int prefetch) {
  constexpr int W = ColsPerLane<K>::value;
  constexpr int G = K / W;           // lanes per row
  constexpr int RPC = kThreads / G;  // rows per CTA
  if (threadIdx.x == 0 && prefetch > 0)
    prefetch_rows(((int64_t)blockIdx.x + prefetch) * RPC, RPC, n_rows, row_ptr, col, val);
  const int64_t g = ((int64_t)blockIdx.x * kThreads + threadIdx.x) / G;
  if (g >= n_rows) return;
  const int c0 = (int)(threadIdx.x % G) * W;  // first column of this lane
  const int rs = __ldg(row_ptr + g), re = __ldg(row_ptr + g + 1);
  double acc[W];
#pragma unroll
  for (int q = 0; q < W; ++q) acc[q] = 0.0;
  const double* Bc = B + c0;
  for (int j = rs; j < re; ++j) {
    const double v = to_f64(ldg(val + j));
    const double* b = Bc + (int64_t)ldg(col + j) * ldb;
    double gv[W];
#pragma unroll
    for (int q = 0; q < W; q += 2) {
      const double2 x = __ldg(reinterpret_cast<const double2*>(b + q));
      gv[q] = x.x;
      gv[q + 1] = x.y;
    }
#pragma unroll
    for (int q = 0; q < W; ++q) acc[q] = fma(v, gv[q], acc[q]);
  }
  double2* out = reinterpret_cast<double2*>(C + g * ldc + c0);
#pragma unroll
  for (int q = 0; q < W; q += 2) out[q / 2] = make_double2(acc[q], acc[q + 1]);
}

template <typename VT, int L, int K>
static cudaError_t launch_lanes_t(int64_t n_rows, const int32_t* rows, const int32_t* row_ptr,
                                  const int32_t* col, const VT* val, const double* B, int64_t ldb, double* C,
                                  int64_t ldc, int k, bool acc, int pf, cudaStream_t s) {
  if (n_rows == 0) return cudaSuccess;
  if constexpr (L == 1 && K >= 2) {
    // a full block of K columns with 16-byte aligned rows, not accumulating: the column-split
    // form (16-byte gathers and stores; these products are FP64-pipe-bound, and halving the
    // gather instructions, then sharing each B row among G lanes, took the 3D Poisson product
    // at K = 2 / 16 from 0.82 / 0.81 to 0.95 / 0.98 of the FP64 peak)
    if (k == K && !acc && !rows && ldb % 2 == 0 && ldc % 2 == 0 && (((uintptr_t)B | (uintptr_t)C) & 15) == 0) {
      constexpr int G = K / ColsPerLane<K>::value;
      const int64_t grid = (n_rows * G + kThreads - 1) / kThreads;
      k_crs_cols<VT, K><<<(unsigned)grid, kThreads, 0, s>>>(n_rows, row_ptr, col, val, B, ldb, C, ldc, pf);
      return cudaGetLastError();
    }
  }
  const int64_t rows_per_cta = kThreads / L;
  const int64_t grid = (n_rows + rows_per_cta - 1) / rows_per_cta;
  if constexpr (L > 1 && K >= 2) {
    // several lanes per row on a full block with 16-byte aligned B rows: 16-byte gathers
    if (k == K && ldb % 2 == 0 && (((uintptr_t)B) & 15) == 0) {
      k_crs_lanes<VT, L, K, true><<<(unsigned)grid, kThreads, 0, s>>>(n_rows, rows, row_ptr, col, val, B, ldb, C,
                                                                        ldc, k, acc ? 1 : 0, pf);
      return cudaGetLastError();
    }
  }
  k_crs_lanes<VT, L, K, false><<<(unsigned)grid, kThreads, 0, s>>>(n_rows, rows, row_ptr, col, val, B, ldb, C,
                                                                     ldc, k, acc ? 1 : 0, pf);
  return cudaGetLastError();
}

template <typename VT, int L>
static cudaError_t lanes_k(int64_t n, const int32_t* rows, const int32_t* rp, const int32_t* col, const VT* val,
                           const double* B, int64_t ldb, double* C, int64_t ldc, int k, bool acc,
                           int pf, cudaStream_t s) {
  if (k <= 1) return launch_lanes_t<VT, L, 1>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, pf, s);
  if (k <= 2) return launch_lanes_t<VT, L, 2>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, pf, s);
  if (k <= 4) return launch_lanes_t<VT, L, 4>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, pf, s);
  if (k <= 8) return launch_lanes_t<VT, L, 8>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, pf, s);
  return launch_lanes_t<VT, L, 16>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, pf, s);
}

template <typename VT>
static cudaError_t lanes_dispatch(int lanes, int64_t n, const int32_t* rows, const int32_t* rp,
                                  const int32_t* col, const VT* val, const double* B, int64_t ldb, double* C,
                                  int64_t ldc, int k, bool acc, int pf, cudaStream_t s) {
  switch (lanes) {
    case 1: return lanes_k<VT, 1>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, pf, s);
    case 2: return lanes_k<VT, 2>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, pf, s);
    case 4: return lanes_k<VT, 4>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, pf, s);
    case 8: return lanes_k<VT, 8>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, pf, s);
    case 16: return lanes_k<VT, 16>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, pf, s);
    case 32: return lanes_k<VT, 32>(n, rows, rp, col, val, B, ldb, C, ldc, k, acc, pf, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_crs_lanes(const CsrDev& A, bool fp32, int lanes, const double* B, int64_t ldb, double* C,
                             int64_t ldc, int k, cudaStream_t s) {
  if (fp32 && A.val32_special)
    return lanes_dispatch<float>(lanes, A.n_rows, nullptr, A.row_ptr, A.col, A.val32, B, ldb, C, ldc, k, false,
                                 A.prefetch, s);
  if (fp32)
    return lanes_dispatch<f32n>(lanes, A.n_rows, nullptr, A.row_ptr, A.col, reinterpret_cast<const f32n*>(A.val32),
                                B, ldb, C, ldc, k, false, A.prefetch, s);
  return lanes_dispatch<double>(lanes, A.n_rows, nullptr, A.row_ptr, A.col, A.val, B, ldb, C, ldc, k, false,
                                A.prefetch, s);
}

cudaError_t launch_halo(const HaloDev& H, bool fp32, const double* B, int64_t ldb, double* C, int64_t ldc, int k,
                        cudaStream_t s) {
  if (fp32 && H.val32_special)
    return lanes_dispatch<float>(1, H.n_rows, H.rows, H.row_ptr, H.col, H.val32, B, ldb, C, ldc, k, true, 0, s);
  if (fp32)
    return lanes_dispatch<f32n>(1, H.n_rows, H.rows, H.row_ptr, H.col, reinterpret_cast<const f32n*>(H.val32), B,
                                ldb, C, ldc, k, true, 0, s);
  return lanes_dispatch<double>(1, H.n_rows, H.rows, H.row_ptr, H.col, H.val, B, ldb, C, ldc, k, true, 0, s);
}

}  // namespace spmv
