// C ABI of the reordering: the RCM permutation and the symmetric permutation
// of CRS arrays (host), and a device object that moves k-column blocks between
// the original and the permuted row order (a validated permutation on the
// device, so the gathers and scatters stay in bounds).
#include <new>

#include "device.cuh"
#include "internal.h"

namespace spmv {

// Y[r] = X[perm[r]] (gather) or Y[perm[r]] = X[r] (scatter), k columns per row.
template <bool SCATTER>
__global__ void __launch_bounds__(kThreads) k_permute_rows(int64_t n, int k, const int32_t* __restrict__ perm,
                                                           const double* __restrict__ X, int64_t ldx,
                                                           double* __restrict__ Y, int64_t ldy) {
  const int64_t total = n * k;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < total; e += (int64_t)gridDim.x * kThreads) {
    const int64_t r = e / k;
    const int c = (int)(e - r * k);
    const int64_t o = __ldg(perm + r);
    if (SCATTER)
      Y[o * ldy + c] = __ldg(X + r * ldx + c);
    else
      Y[r * ldy + c] = __ldg(X + o * ldx + c);
  }
}

}  // namespace spmv

using namespace spmv;

struct spmv_reorder {
  int device = 0;
  int64_t n = 0;
  int32_t* perm = nullptr;  // device
  unsigned grid = 0;
};

extern "C" {

spmv_status spmv_rcm(int64_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* perm) {
  if (n < 0 || (n > 0 && (!row_ptr || !perm))) return fail(SPMV_ERR_ARG, "bad size or NULL array");
  std::string why;
  if (!validate_csr(n, n, row_ptr, col_idx, &why)) return fail(SPMV_ERR_CSR, why);
  try {
    rcm_permutation(n, row_ptr, col_idx, perm);
  } catch (const std::bad_alloc&) {
    return fail(SPMV_ERR_OOM, "host allocation failed");
  }
  return SPMV_OK;
}

spmv_status spmv_permute_csr(int64_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                             const int32_t* perm, int32_t* out_row_ptr, int32_t* out_col_idx, double* out_val) {
  if (n < 0 || (n > 0 && (!row_ptr || !perm || !out_row_ptr))) return fail(SPMV_ERR_ARG, "bad size or NULL array");
  std::string why;
  if (!validate_csr(n, n, row_ptr, col_idx, &why)) return fail(SPMV_ERR_CSR, why);
  if (n > 0 && row_ptr[n] > 0 && (!val || !out_col_idx || !out_val)) return fail(SPMV_ERR_ARG, "NULL array");
  try {
    std::vector<int32_t> inv;
    if (!validate_permutation(n, perm, &inv, &why)) return fail(SPMV_ERR_ARG, why);
    if (n == 0) {
      out_row_ptr[0] = 0;
      return SPMV_OK;
    }
    permute_csr(n, row_ptr, col_idx, val, perm, inv, out_row_ptr, out_col_idx, out_val);
  } catch (const std::bad_alloc&) {
    return fail(SPMV_ERR_OOM, "host allocation failed");
  }
  return SPMV_OK;
}

spmv_status spmv_reorder_create(int64_t n, const int32_t* perm, spmv_reorder_handle* out) {
  if (!out || n < 0 || (n > 0 && !perm)) return fail(SPMV_ERR_ARG, "bad argument");
  *out = nullptr;
  std::string why;
  std::vector<int32_t> inv;
  if (!validate_permutation(n, perm, &inv, &why)) return fail(SPMV_ERR_ARG, why);
  auto* h = new (std::nothrow) spmv_reorder;
  if (!h) return fail(SPMV_ERR_OOM, "host allocation failed");
  h->n = n;
  cudaError_t e = cudaGetDevice(&h->device);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->perm, sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(h->perm, perm, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (h->perm) cudaFree(h->perm);
    delete h;
    return cuda_fail(e, "reorder setup");
  }
  h->grid = (unsigned)((sms > 0 ? sms : 1) * 8);
  *out = h;
  return SPMV_OK;
}

spmv_status spmv_reorder_destroy(spmv_reorder_handle h) {
  if (!h) return SPMV_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  cudaFree(h->perm);
  if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
  delete h;
  return SPMV_OK;
}

static spmv_status reorder_move(spmv_reorder_handle h, bool scatter, int32_t k, const double* X, int64_t ldx,
                                double* Y, int64_t ldy, void* stream) {
  if (!h) return fail(SPMV_ERR_ARG, "handle is NULL");
  if (k < 1 || ldx < k || ldy < k) return fail(SPMV_ERR_ARG, "need k >= 1, ldx >= k, ldy >= k");
  if (h->n == 0) return SPMV_OK;
  if (!X || !Y) return fail(SPMV_ERR_ARG, "X or Y is NULL");
  if (X == Y) return fail(SPMV_ERR_ARG, "X and Y must not be the same block");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  if (scatter)
    k_permute_rows<true><<<h->grid, kThreads, 0, (cudaStream_t)stream>>>(h->n, k, h->perm, X, ldx, Y, ldy);
  else
    k_permute_rows<false><<<h->grid, kThreads, 0, (cudaStream_t)stream>>>(h->n, k, h->perm, X, ldx, Y, ldy);
  cudaError_t e = cudaGetLastError();
  if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
  return e == cudaSuccess ? SPMV_OK : cuda_fail(e, "permute launch");
}

spmv_status spmv_reorder_gather(spmv_reorder_handle h, int32_t k, const double* X_dev, int64_t ldx, double* Y_dev,
                                int64_t ldy, void* stream) {
  return reorder_move(h, false, k, X_dev, ldx, Y_dev, ldy, stream);
}

spmv_status spmv_reorder_scatter(spmv_reorder_handle h, int32_t k, const double* X_dev, int64_t ldx, double* Y_dev,
                                 int64_t ldy, void* stream) {
  return reorder_move(h, true, k, X_dev, ldx, Y_dev, ldy, stream);
}

}  // extern "C"
