// Measurement probes: the machine side of the balance model.  The paper sets
// the code balance of Eq. 1 against the machine's measured memory bandwidth
// (STREAM, Sec. 2).  On this GPU two more rates bound forms of the product:
// the FP64 fused multiply-add rate (k >= 2 columns, the batch, the solvers)
// and the rate of random 8-byte reads served by L2 (the scattered B gathers of
// the eigenproblem-shaped matrix).  Each probe times its own kernel with CUDA
// events on a private stream and reports the best of `reps` launches.
#include <algorithm>

#include "internal.h"

namespace spmv {

constexpr int kProbeChains = 8;        // independent FMA chains / gathers in flight per thread
constexpr int kProbeFmaIters = 4096;   // ~16 ms of FMA work on the whole GPU
constexpr int kProbeGatherIters = 512;

__device__ __forceinline__ unsigned long long probe_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 of each CTA adds the SM clock cycles and the nanoseconds its CTA
// ran: their ratio over all CTAs is the SM clock during the probe.
__device__ __forceinline__ void probe_span(unsigned long long c0, unsigned long long t0, unsigned long long* span) {
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(span, clock64() - c0);
    atomicAdd(span + 1, probe_ns() - t0);
  }
}

// FMA throughput: kProbeChains independent chains x = x*a + b per thread
// (a < 1, so every chain stays near b / (1 - a): no overflow, no
// subnormals).  a and b are computed per thread so that they live in
// registers: operands read from the constant bank cap the FMA rate lower.
__global__ void __launch_bounds__(kThreads) k_probe_fma(int iters, double* out, unsigned long long* span) {
  const unsigned long long c0 = clock64(), t0 = probe_ns();
  const double a = 1.0 - 1e-6 * (1 + (threadIdx.x & 1)), b = 1e-6 * (1 + (threadIdx.x & 3));
  double x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
  probe_span(c0, t0, span);
}

// Random-read throughput: kProbeChains independent linear congruential
// streams per thread (Numerical Recipes constants 1664525 / 1013904223); the
// top bits of each state pick an index in [0, n) by a 32 x 32 -> high-32
// multiply, and the loaded bits are folded in with an integer xor so that no
// FP64 pipe work competes with the loads.  Read-only (non-coherent) loads, as
// in the product's B gathers.
__global__ void __launch_bounds__(kThreads) k_probe_gather(const double* __restrict__ buf, uint32_t n, int iters,
                                                           unsigned long long* out, unsigned long long* span) {
  const unsigned long long c0 = clock64(), t0 = probe_ns();
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = (tid * kProbeChains + c) * 2654435761u + 12345u;
  unsigned long long acc = 0;
#pragma unroll 2
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) {
      const uint32_t idx = __umulhi(x[c], n);
      acc ^= (unsigned long long)__double_as_longlong(__ldg(buf + idx));
      x[c] = x[c] * 1664525u + 1013904223u;
    }
  }
  out[tid] = acc;
  probe_span(c0, t0, span);
}

static spmv_status probe_grid(int* sms, int* grid) {
  int dev = 0, per_sm = 0;
  SPMV_CUDA(cudaGetDevice(&dev));
  SPMV_CUDA(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
  int max_threads = 0;
  SPMV_CUDA(cudaDeviceGetAttribute(&max_threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
  per_sm = std::max(1, max_threads / kThreads);
  *grid = *sms * per_sm;
  return SPMV_OK;
}

// Runs `launch` (which writes its clock span into span[0:2]) and returns the
// best time and the SM clock (MHz) of that best launch.
template <class F>
static spmv_status probe_run(F launch, cudaStream_t s, int reps, unsigned long long* span, float* best_ms,
                             double* mhz) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  double best_mhz = 0.0;
  if (e == cudaSuccess) e = cudaMemsetAsync(span, 0, 16, s);
  if (e == cudaSuccess) e = launch();  // untimed
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaMemsetAsync(span, 0, 16, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, span, 16, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && ms < best) {
      best = ms;
      best_mhz = h[1] ? 1e3 * (double)h[0] / (double)h[1] : 0.0;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "probe timing");
  *best_ms = best;
  *mhz = best_mhz;
  return SPMV_OK;
}

}  // namespace spmv

using namespace spmv;

extern "C" spmv_status spmv_probe_fp64(int32_t reps, double* gflops, double* ms, int32_t* sm_count, double* sm_mhz) {
  if (reps < 1 || reps > 1000) return fail(SPMV_ERR_ARG, "reps out of range 1..1000");
  int sms = 0, grid = 0;
  spmv_status st = probe_grid(&sms, &grid);
  if (st != SPMV_OK) return st;
  double* out = nullptr;
  unsigned long long* span = nullptr;
  cudaStream_t s = nullptr;
  SPMV_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaError_t e = cudaMalloc(&out, sizeof(double) * (size_t)grid * kThreads);
  if (e == cudaSuccess) e = cudaMalloc(&span, 16);
  if (e != cudaSuccess) {
    cudaFree(out);
    cudaStreamDestroy(s);
    return cuda_fail(e, "probe buffer");
  }
  float best = 0.f;
  double mhz = 0.0;
  st = probe_run(
      [&]() {
        k_probe_fma<<<grid, kThreads, 0, s>>>(kProbeFmaIters, out, span);
        return cudaGetLastError();
      },
      s, reps, span, &best, &mhz);
  cudaFree(out);
  cudaFree(span);
  cudaStreamDestroy(s);
  if (st != SPMV_OK) return st;
  const double flops = 2.0 * kProbeChains * (double)kProbeFmaIters * (double)grid * kThreads;
  if (gflops) *gflops = flops / (best * 1e-3) / 1e9;
  if (ms) *ms = best;
  if (sm_count) *sm_count = sms;
  if (sm_mhz) *sm_mhz = mhz;
  return SPMV_OK;
}

extern "C" spmv_status spmv_probe_gather(int64_t n_elems, int32_t reps, double* gathers_per_s, double* ms,
                                         double* sm_mhz) {
  if (n_elems < 1 || n_elems > INT32_MAX) return fail(SPMV_ERR_ARG, "n_elems out of range 1..2^31-1");
  if (reps < 1 || reps > 1000) return fail(SPMV_ERR_ARG, "reps out of range 1..1000");
  int sms = 0, grid = 0;
  spmv_status st = probe_grid(&sms, &grid);
  if (st != SPMV_OK) return st;
  double* buf = nullptr;
  unsigned long long *out = nullptr, *span = nullptr;
  cudaStream_t s = nullptr;
  SPMV_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaError_t e = cudaMalloc(&buf, sizeof(double) * (size_t)n_elems);
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(unsigned long long) * (size_t)grid * kThreads);
  if (e == cudaSuccess) e = cudaMalloc(&span, 16);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, sizeof(double) * (size_t)n_elems, s);
  if (e != cudaSuccess) {
    cudaFree(buf);
    cudaFree(out);
    cudaFree(span);
    cudaStreamDestroy(s);
    return cuda_fail(e, "probe buffers");
  }
  float best = 0.f;
  double mhz = 0.0;
  const uint32_t n = (uint32_t)n_elems;
  st = probe_run(
      [&]() {
        k_probe_gather<<<grid, kThreads, 0, s>>>(buf, n, kProbeGatherIters, out, span);
        return cudaGetLastError();
      },
      s, reps, span, &best, &mhz);
  cudaFree(buf);
  cudaFree(out);
  cudaFree(span);
  cudaStreamDestroy(s);
  if (st != SPMV_OK) return st;
  const double gathers = (double)kProbeChains * kProbeGatherIters * (double)grid * kThreads;
  if (gathers_per_s) *gathers_per_s = gathers / (best * 1e-3);
  if (ms) *ms = best;
  if (sm_mhz) *sm_mhz = mhz;
  return SPMV_OK;
}
