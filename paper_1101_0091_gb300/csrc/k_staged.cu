// CRS_STAGED: thread-per-row CRS product with bulk-copied tiles (Sec. 1.2 loop).
//
// The row range of the matrix is cut into blocks (host side, build_row_blocks).
// A "tile" block holds up to 256 consecutive rows of at most 64 entries whose
// entries, being contiguous in val/col_idx, fit one shared-memory tile.  One
// elected thread brings the block's val and col_idx slices into shared memory
// with two one-dimensional bulk copies (cp.async.bulk, TMA engine) completing
// on an mbarrier; meanwhile every thread reads its row bounds.  Then each thread
// walks its own row from shared memory, gathers B with read-only loads, and
// accumulates in FP64 with one FMA per entry.  On this GPU the FP64 pipe
// sustains about two FMAs per SM clock, so the kernel does no shuffle
// reductions at all for these rows.  A "warp" block holds up to 8 rows longer
// than 64 entries, one warp per row: lanes stride the row with coalesced loads
// and a 5-step xor-shuffle tree sums their partials.  A full, 16-byte aligned
// block of K >= 8 columns splits each tile row's columns over K / 4 lanes.
#include <mutex>

#include "device.cuh"

namespace spmv {

template <typename VT, int K, bool VEC>
__device__ __forceinline__ void row_warp(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                         const VT* __restrict__ val, int row, const double* __restrict__ B,
                                         int64_t ldb, double* __restrict__ C, int64_t ldc, int k,
                                         int accumulate) {
  const int lane = threadIdx.x & 31;
  const int rs = __ldg(row_ptr + row), re = __ldg(row_ptr + row + 1);
  double acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0.0;
  for (int j = rs + lane; j < re; j += 32) {
    const double v = to_f64(ldcs(val + j));
    const double* b = B + (int64_t)ldcs(col + j) * ldb;
    if constexpr (VEC) {  // k == K >= 2, 16-byte aligned rows of B
#pragma unroll
      for (int q = 0; q < K; q += 2) {
        const double2 x = __ldg(reinterpret_cast<const double2*>(b + q));
        acc[q] = fma(v, x.x, acc[q]);
        acc[q + 1] = fma(v, x.y, acc[q + 1]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < K; ++q)
        if (q < k) acc[q] = fma(v, __ldg(b + q), acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = warp_sum_xor(acc[q], 32);
  double* out = C + (int64_t)row * ldc;
#pragma unroll
  for (int q = 0; q < K; ++q)
    if (q < k && lane == q) out[q] = accumulate ? out[q] + acc[q] : acc[q];
}

// Entries of one row processed per batch: every gather of a batch is issued
// before its FMAs, so short rows keep all their B loads in flight at once.
template <int K>
struct Batch {
  static constexpr int value = K >= 4 ? 1 : 4 / K;
};

// Prefetch into L2 the val/col slices of row block `b` (called `prefetch`
// blocks ahead of the block being processed).
template <typename VT>
__device__ __forceinline__ void prefetch_block(const uint32_t* __restrict__ blk, int64_t b,
                                               const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                               const VT* __restrict__ val) {
  const int r0 = (int)(__ldg(blk + b) & ~kBlockWarpFlag), r1 = (int)(__ldg(blk + b + 1) & ~kBlockWarpFlag);
  const int bs = __ldg(row_ptr + r0), be = __ldg(row_ptr + r1);
  if (be <= bs) return;
  constexpr int VA = 16 / (int)sizeof(VT);
  const int v_lo = bs & ~(VA - 1), v_hi = (be + VA - 1) & ~(VA - 1);
  const int c_lo = bs & ~3, c_hi = (be + 3) & ~3;
  prefetch_l2(val + v_lo, (uint32_t)(v_hi - v_lo) * (uint32_t)sizeof(VT));
  prefetch_l2(col + c_lo, (uint32_t)(c_hi - c_lo) * 4u);
}

template <typename VT, int K, bool VEC>
__global__ void __launch_bounds__(kThreads)
    k_crs_staged(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                 const VT* __restrict__ val, const uint32_t* __restrict__ blk, int64_t n_blk, int tile,
                 int prefetch, const double* __restrict__ B, int64_t ldb, double* __restrict__ C, int64_t ldc,
                 int k, int accumulate, int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar;

  const uint32_t e0 = __ldg(blk + blockIdx.x), e1 = __ldg(blk + blockIdx.x + 1);
  const int r0 = (int)(e0 & ~kBlockWarpFlag), r1 = (int)(e1 & ~kBlockWarpFlag);
  const int tid = threadIdx.x;

  if (tid == 32 && prefetch > 0 && (int64_t)blockIdx.x + prefetch < n_blk)
    prefetch_block(blk, (int64_t)blockIdx.x + prefetch, row_ptr, col, val);

  if (e0 & kBlockWarpFlag) {  // block of long rows: one warp per row
    const int row = r0 + (tid >> 5);
    if (row < r1) row_warp<VT, K, VEC>(row_ptr, col, val, row, B, ldb, C, ldc, k, accumulate);
    return;
  }

  const int bs = __ldg(row_ptr + r0), be = __ldg(row_ptr + r1);
  constexpr int VA = 16 / (int)sizeof(VT);  // value entries per 16 bytes
  const int v_lo = bs & ~(VA - 1), v_hi = (be + VA - 1) & ~(VA - 1);
  const int c_lo = bs & ~3, c_hi = (be + 3) & ~3;
  VT* sval = reinterpret_cast<VT*>(smem);
  const int32_t* scol = reinterpret_cast<const int32_t*>(smem + sizeof(VT) * (size_t)(tile + 8));
  const bool any = be > bs;

  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (any && tid == 0) {
    const uint32_t vb = (uint32_t)(v_hi - v_lo) * (uint32_t)sizeof(VT);
    const uint32_t cb = (uint32_t)(c_hi - c_lo) * 4u;
    mbar_arrive_expect_tx(&bar, vb + cb);
    bulk_g2s(sval, val + v_lo, vb, &bar);
    bulk_g2s(smem + sizeof(VT) * (size_t)(tile + 8), col + c_lo, cb, &bar);
  }

  const int row = r0 + tid;
  int rs = 0, re = 0;
  if (row < r1) {
    rs = __ldg(row_ptr + row);
    re = __ldg(row_ptr + row + 1);
  }
  if (any && !mbar_wait_bounded(&bar, 0, kWaitLimitNs)) {
    atomicExch(status, DEV_WAIT_TIMEOUT);
    mbar_wait_bounded(&bar, 0, kWaitLimitNs);  // let the copies in flight land before exiting
    return;
  }
  if constexpr (VEC && K >= 8) {
    // a full block of K >= 8 columns: each row is shared by G = K / 4 lanes, lane c owning
    // columns 4c .. 4c + 3 (two 16-byte gathers per entry, the G lanes of a row read one
    // contiguous piece of its B row); the block's rows take G passes of 256 / G rows.  Each
    // column's entries are summed in order, as in the thread-per-row form.
    constexpr int G = K / 4, RPP = kThreads / G;
    const int c0 = (tid % G) * 4;
    for (int r = r0 + tid / G; r < r1; r += RPP) {
      const int s0 = __ldg(row_ptr + r), s1 = __ldg(row_ptr + r + 1);
      double a[4] = {0.0, 0.0, 0.0, 0.0};
      for (int j = s0; j < s1; ++j) {
        const double v = to_f64(sval[j - v_lo]);
        const double2* b = reinterpret_cast<const double2*>(B + (int64_t)scol[j - c_lo] * ldb + c0);
        const double2 x = __ldg(b), y = __ldg(b + 1);
        a[0] = fma(v, x.x, a[0]);
        a[1] = fma(v, x.y, a[1]);
        a[2] = fma(v, y.x, a[2]);
        a[3] = fma(v, y.y, a[3]);
      }
      double2* out = reinterpret_cast<double2*>(C + (int64_t)r * ldc + c0);
      out[0] = make_double2(a[0], a[1]);
      out[1] = make_double2(a[2], a[3]);
    }
    return;
  }
  if (row >= r1) return;

  double acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0.0;
  constexpr int NB = VEC ? 1 : Batch<K>::value;  // 16-byte gathers: one entry per step measured fastest
  for (int j = rs; j < re; j += NB) {
    double v[NB];
    const double* b[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int jj = (j + u < re) ? j + u : j;
      v[u] = to_f64(sval[jj - v_lo]);
      b[u] = B + (int64_t)scol[jj - c_lo] * ldb;
    }
    double g[NB][K];
    if (VEC) {  // k == K >= 2, 16-byte aligned rows of B: one 16-byte gather per two columns
#pragma unroll
      for (int u = 0; u < NB; ++u)
#pragma unroll
        for (int q = 0; q < K; q += 2) {
          const double2 t2 = j + u < re ? __ldg(reinterpret_cast<const double2*>(b[u] + q)) : make_double2(0.0, 0.0);
          g[u][q] = t2.x;
          g[u][q + 1] = t2.y;
        }
    } else {
#pragma unroll
      for (int u = 0; u < NB; ++u)
#pragma unroll
        for (int q = 0; q < K; ++q) g[u][q] = (j + u < re && q < k) ? __ldg(b[u] + q) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < NB; ++u)
#pragma unroll
      for (int q = 0; q < K; ++q)
        if (j + u < re && q < k) acc[q] = fma(v[u], g[u][q], acc[q]);
  }
  double* out = C + (int64_t)row * ldc;
  if constexpr (VEC) {
#pragma unroll
    for (int q = 0; q < K; q += 2) reinterpret_cast<double2*>(out)[q / 2] = make_double2(acc[q], acc[q + 1]);
  } else {
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (q < k) out[q] = accumulate ? out[q] + acc[q] : acc[q];
  }
}

template <typename VT, int K, bool VEC>
static cudaError_t launch_staged_v(const CsrDev& A, const VT* val, const double* B, int64_t ldb, double* C,
                                   int64_t ldc, int k, bool accumulate, int* status, cudaStream_t s) {
  const size_t smem = sizeof(VT) * (size_t)(A.tile + 8) + 4 * (size_t)(A.tile + 8);
  auto kern = k_crs_staged<VT, K, VEC>;
  // per device: largest dynamic shared memory size enabled so far (check and set under a lock, so
  // that concurrent host threads never leave the attribute below the recorded size)
  static int smem_set[64] = {0};
  static std::mutex smem_mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(smem_mu);
    if (dev >= 64 || (int)smem > smem_set[dev]) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      if (dev < 64) smem_set[dev] = (int)smem;
    }
  }
  kern<<<(unsigned)A.n_blk, kThreads, smem, s>>>(A.row_ptr, A.col, val, A.blk, A.n_blk, A.tile, A.prefetch, B,
                                                  ldb, C, ldc, k, accumulate ? 1 : 0, status);
  return cudaGetLastError();
}

template <typename VT, int K>
static cudaError_t launch_staged_t(const CsrDev& A, const VT* val, const double* B, int64_t ldb, double* C,
                                   int64_t ldc, int k, bool accumulate, int* status, cudaStream_t s) {
  const bool vec = K >= 2 && k == K && !accumulate && ldb % 2 == 0 && ldc % 2 == 0 &&
                   (((uintptr_t)B | (uintptr_t)C) & 15) == 0;
  if (vec) return launch_staged_v<VT, K, (K >= 2)>(A, val, B, ldb, C, ldc, k, accumulate, status, s);
  return launch_staged_v<VT, K, false>(A, val, B, ldb, C, ldc, k, accumulate, status, s);
}

template <typename VT>
static cudaError_t dispatch_staged(const CsrDev& A, const VT* val, const double* B, int64_t ldb, double* C,
                                   int64_t ldc, int k, bool acc, int* status, cudaStream_t s) {
  if (k <= 1) return launch_staged_t<VT, 1>(A, val, B, ldb, C, ldc, k, acc, status, s);
  if (k <= 2) return launch_staged_t<VT, 2>(A, val, B, ldb, C, ldc, k, acc, status, s);
  if (k <= 4) return launch_staged_t<VT, 4>(A, val, B, ldb, C, ldc, k, acc, status, s);
  if (k <= 8) return launch_staged_t<VT, 8>(A, val, B, ldb, C, ldc, k, acc, status, s);
  return launch_staged_t<VT, 16>(A, val, B, ldb, C, ldc, k, acc, status, s);
}

cudaError_t launch_crs_staged(const CsrDev& A, bool fp32, const double* B, int64_t ldb, double* C,
                              int64_t ldc, int k, bool accumulate, int* status, cudaStream_t s) {
  if (A.n_blk == 0) return cudaSuccess;
  if (fp32 && A.val32_special) return dispatch_staged<float>(A, A.val32, B, ldb, C, ldc, k, accumulate, status, s);
  if (fp32)
    return dispatch_staged<f32n>(A, reinterpret_cast<const f32n*>(A.val32), B, ldb, C, ldc, k, accumulate, status,
                                 s);
  return dispatch_staged<double>(A, A.val, B, ldb, C, ldc, k, accumulate, status, s);
}

}  // namespace spmv
