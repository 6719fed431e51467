// Bounded waits: the host-side deadline wait on a stream, and a self-test of
// the device-side bounded mbarrier wait's failure path (an mbarrier phase that
// nothing completes), which returns a status instead of hanging.
#include <chrono>
#include <thread>

#include "device.cuh"
#include "internal.h"

namespace spmv {

// One CTA, one thread: init an mbarrier expecting one arrival that never
// comes, wait with the limit, record the outcome.
__global__ void k_wait_selftest(unsigned long long limit_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  const bool done = mbar_wait_bounded(&bar, 0, limit_ns);
  *status = done ? DEV_OK : DEV_WAIT_TIMEOUT;
}

}  // namespace spmv

using namespace spmv;

extern "C" spmv_status spmv_wait(void* stream, int32_t timeout_ms) {
  if (timeout_ms < 0) return fail(SPMV_ERR_ARG, "timeout_ms must be >= 0");
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    const cudaError_t e = cudaStreamQuery((cudaStream_t)stream);
    if (e == cudaSuccess) return SPMV_OK;
    if (e != cudaErrorNotReady) return cuda_fail(e, "cudaStreamQuery");
    if (std::chrono::steady_clock::now() >= deadline)
      return fail(SPMV_ERR_TIMEOUT, "stream work not finished within " + std::to_string(timeout_ms) + " ms");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

extern "C" spmv_status spmv_selftest_wait_timeout(int32_t limit_us) {
  if (limit_us < 1 || limit_us > 1000000) return fail(SPMV_ERR_ARG, "limit_us out of range 1..1e6");
  int* d = nullptr;
  SPMV_CUDA(cudaMalloc(&d, sizeof(int)));
  const int init = -1;
  cudaError_t e = cudaMemcpy(d, &init, sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32>>>((unsigned long long)limit_us * 1000ull, d);
    e = cudaGetLastError();
  }
  int h = -1;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
  if (h == DEV_WAIT_TIMEOUT) return fail(SPMV_ERR_TIMEOUT, "device wait gave up after the limit (expected)");
  if (h == DEV_OK) return SPMV_OK;
  return fail(SPMV_ERR_DEVICE, "wait self-test kernel did not report");
}
