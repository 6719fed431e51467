// Batched product for callers that cannot allocate device memory.
//
// Same persistent kernel as spmv_batch_apply, but its scratch (the work
// counter, the member table and the work list) lives in one file-scope static
// device array instead of memory from cudaMalloc.  The work list is built on
// the host from the member row counts alone (contiguous row items, fixed lanes
// per row), copied into the array, and the counter is cleared before each
// launch.  See the declaration in include/spmv.h for the contract.
#include <cstring>
#include <mutex>

#include "batch_kernel.cuh"
#include "internal.h"

namespace spmv {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr size_t kNoAllocCounterBytes = 256;
constexpr int kNoAllocMaxMembers = 8192;
constexpr size_t kNoAllocTableBytes = sizeof(BatchMat) * kNoAllocMaxMembers;
constexpr size_t kNoAllocItemsOffset = kNoAllocCounterBytes + kNoAllocTableBytes;
constexpr size_t kNoAllocMaxItems = (kNoAllocScratchBytes - kNoAllocItemsOffset) / sizeof(BatchItem);
constexpr int kNoAllocPasses = 32;  // warp passes per work item

// The scratch: [counter | member table | work items].  Every GPU that loads the
// library holds these 8 MiB until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch, looked up once per device with that device
// current (in host code the array's name is only a host-side stand-in).
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64];

// Host staging of the table and the items.  cudaMemcpyAsync from pageable
// memory returns once the bytes are staged, so the buffer can be refilled by
// the next call; the mutex keeps two host threads from filling it at once.
static unsigned char g_noalloc_host[kNoAllocScratchBytes];

static spmv_status noalloc_scratch(void** out) {
  int dev = 0;
  SPMV_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SPMV_ERR_UNSUPPORTED, "device index beyond 63");
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return SPMV_OK;
}

}  // namespace spmv

using namespace spmv;

extern "C" spmv_status spmv_batch_apply_noalloc(int32_t count, const int64_t* n_rows,
                                                const int32_t* const* row_ptr_dev, const int32_t* const* col_dev,
                                                const double* const* val_dev, const double* const* B_dev,
                                                const int64_t* ldb, double* const* C_dev, const int64_t* ldc,
                                                int32_t k, const int32_t* lanes, void* stream) {
  if (count < 1 || !n_rows || !row_ptr_dev || !col_dev || !val_dev || !B_dev || !C_dev)
    return fail(SPMV_ERR_ARG, "count must be >= 1 with non-NULL per-member arrays");
  if (count > kNoAllocMaxMembers)
    return fail(SPMV_ERR_ARG, "spmv_batch_apply_noalloc: more than 8192 members (scratch limit)");
  if (k < 1 || k > 16) return fail(SPMV_ERR_ARG, "k out of range 1..16");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  // every argument is checked and the work list built before the first CUDA call
  BatchMat* table = reinterpret_cast<BatchMat*>(g_noalloc_host + kNoAllocCounterBytes);
  BatchItem* items = reinterpret_cast<BatchItem*>(g_noalloc_host + kNoAllocItemsOffset);
  size_t n_items = 0;
  bool vec = (k % 2 == 0);
  for (int m = 0; m < count; ++m) {
    const int L = lanes ? lanes[m] : 1;
    if (L != 1 && L != 2 && L != 4 && L != 8 && L != 16 && L != 32)
      return fail(SPMV_ERR_ARG, "lanes per row must be 1, 2, 4, 8, 16 or 32");
    const int64_t lb = ldb ? ldb[m] : k, lc = ldc ? ldc[m] : k;
    if (n_rows[m] < 0 || n_rows[m] > INT32_MAX) return fail(SPMV_ERR_ARG, "n_rows out of range");
    if (lb < k || lc < k) return fail(SPMV_ERR_ARG, "ldb/ldc must be >= k");
    if (n_rows[m] > 0 && (!row_ptr_dev[m] || !col_dev[m] || !val_dev[m] || !B_dev[m] || !C_dev[m]))
      return fail(SPMV_ERR_ARG, "NULL row_ptr, col, val, B or C of member " + std::to_string(m) + " (it has rows)");
    table[m] = BatchMat{row_ptr_dev[m], col_dev[m], val_dev[m], B_dev[m], C_dev[m], lb, lc, n_rows[m]};
    vec = vec && lb % 2 == 0 && lc % 2 == 0 && (uintptr_t)B_dev[m] % 16 == 0 && (uintptr_t)C_dev[m] % 16 == 0;
    const int64_t per = (int64_t)(32 / L) * kNoAllocPasses;
    for (int64_t r0 = 0; r0 < n_rows[m]; r0 += per) {
      if (n_items == kNoAllocMaxItems)
        return fail(SPMV_ERR_ARG, "spmv_batch_apply_noalloc: the work list exceeds the scratch limit");
      const int64_t r1 = r0 + per < n_rows[m] ? r0 + per : n_rows[m];
      items[n_items++] = BatchItem{m, (int32_t)r0, (int32_t)r1, 0, (int16_t)L, 0, 0};
    }
  }
  void* scratch = nullptr;
  spmv_status st = noalloc_scratch(&scratch);
  if (st != SPMV_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* d = static_cast<unsigned char*>(scratch);
  // the counter starts at zero on every call; the table and items overwrite the last call's
  SPMV_CUDA(cudaMemsetAsync(d, 0, kNoAllocCounterBytes, s));
  SPMV_CUDA(cudaMemcpyAsync(d + kNoAllocCounterBytes, table, sizeof(BatchMat) * (size_t)count,
                            cudaMemcpyHostToDevice, s));
  if (n_items == 0) return SPMV_OK;
  SPMV_CUDA(cudaMemcpyAsync(d + kNoAllocItemsOffset, items, sizeof(BatchItem) * n_items, cudaMemcpyHostToDevice,
                            s));
  int dev = 0, sms = 0;
  SPMV_CUDA(cudaGetDevice(&dev));
  SPMV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const BatchMat* mats = reinterpret_cast<const BatchMat*>(d + kNoAllocCounterBytes);
  const BatchItem* ditems = reinterpret_cast<const BatchItem*>(d + kNoAllocItemsOffset);
  const int2* rowlist = nullptr;
  int* counter = reinterpret_cast<int*>(d);
  int ni = (int)n_items, dynamic = 1, kk = k;
  void* args[] = {(void*)&mats, (void*)&ditems, (void*)&ni, (void*)&rowlist, (void*)&counter, (void*)&dynamic,
                  (void*)&kk};
  SPMV_CUDA(cudaLaunchKernel(batch_rows_kernel(k, vec), dim3(sms * kBatchCtasPerSm), dim3(kBatchThreads), args,
                             0, s));
  return SPMV_OK;
}
