// Device helpers shared by the kernels: PTX wrappers for mbarriers and bulk
// copies, a bounded mbarrier wait, value loads, and the exact float->double
// widening used by the FP32-value forms.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace spmv {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes the mbarrier initialisation visible to the async (bulk copy) proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// One-dimensional bulk copy global -> shared (TMA engine, no tensor map).
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier, giving up after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// FP32-stored values come in two storage types with the same layout:
//  - f32n: every value is zero or a normal float (the plan checks this on the
//    host when it rounds the values).  Widened exactly in the integer pipe from
//    the IEEE 754 formats: with sign s, biased exponent e and 23-bit fraction m,
//    a normal float is 2^(e-127) * 1.m, the same number as the double with
//    exponent e + (1023 - 127) and fraction m << 29; zero keeps its sign.
//    On this GPU the hardware f32->f64 conversion issues on the FP64 pipe that
//    the FMAs already saturate, so this path avoids it.
//  - float: values that include subnormal, infinite or NaN floats; widened by
//    the hardware conversion (exact for every input).
struct f32n {
  float v;
};

__device__ __forceinline__ double widen_f32n(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7fffffffu;
  const uint32_t hi = a ? ((u & 0x80000000u) | ((a >> 3) + (896u << 20))) : (u & 0x80000000u);
  const uint32_t lo = a ? (u << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}

// Fire-and-forget bulk prefetch of [p, p + bytes) into L2 (TMA engine).  p and
// bytes must be multiples of 16 and the range inside the allocation.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  if (bytes == 0) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(f32n v) { return widen_f32n(v.v); }

// Read-only loads through the non-coherent path.
__device__ __forceinline__ double ldg(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldg(const float* p) { return __ldg(p); }
__device__ __forceinline__ f32n ldg(const f32n* p) { return f32n{__ldg(reinterpret_cast<const float*>(p))}; }
__device__ __forceinline__ int32_t ldg(const int32_t* p) { return __ldg(p); }

// Streaming loads (evict-first): matrix entries are used once per product.
__device__ __forceinline__ double ldcs(const double* p) { return __ldcs(p); }
__device__ __forceinline__ float ldcs(const float* p) { return __ldcs(p); }
__device__ __forceinline__ f32n ldcs(const f32n* p) { return f32n{__ldcs(reinterpret_cast<const float*>(p))}; }
__device__ __forceinline__ int32_t ldcs(const int32_t* p) { return __ldcs(p); }

__device__ __forceinline__ double warp_sum_xor(double x, int width) {
  for (int off = width >> 1; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
  return x;
}

}  // namespace spmv
