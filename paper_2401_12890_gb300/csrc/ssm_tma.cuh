// TMA (cp.async.bulk.tensor) and mbarrier helpers for the solver's kernels, plus the
// host-side tensor-map encoder (driver entry point fetched through the runtime, so
// the library does not link libcuda directly).
//
// Every wait on an mbarrier is bounded: after kWaitLimit polls it gives up and the
// caller records SSM_ETIMEOUT in the plan's device error word instead of hanging.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ssm {

constexpr unsigned kWaitLimit = 1u << 24;   // polls before a wait is declared failed

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

// make barrier initialisation visible to the async proxy (TMA) and the cluster
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for the phase with the given parity to complete; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity,
                                          unsigned limit = kWaitLimit) {
  for (unsigned i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// As mbar_try_wait, but a thread whose phase has not completed is suspended for up to
// `suspend_ns` nanoseconds (it resumes as soon as the phase completes), so a waiting warp
// does not take issue slots from working ones by polling.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, unsigned parity,
                                                    unsigned suspend_ns) {
  unsigned ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(suspend_ns)
      : "memory");
  return ok != 0;
}

// bounded wait with suspension between polls: at most `limit` polls of up to 20 us each
// (the default bounds the wait by about 1.3 s); false on timeout
constexpr unsigned kSleepPollLimit = 1u << 16;
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* bar, unsigned parity,
                                                unsigned limit = kSleepPollLimit) {
  for (unsigned i = 0; i < limit; ++i)
    if (mbar_try_wait_sleep(bar, parity, 20000u)) return true;
  return false;
}

// 2D tiled TMA load of one box into shared memory, completing on `bar`
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// 2D tiled TMA prefetch of one box into L2 (no shared memory, no completion to wait for;
// coordinates outside the tensor are ignored like a load's)
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global [%0, {%1, %2}];\n" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}

__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ------------------------------------------------------------------------------------
// host: 2D row-major FP32/BF16 tensor map, dim0 = columns (contiguous), dim1 = rows
// ------------------------------------------------------------------------------------
// Returns cudaSuccess or an error; rows have `ld` elements of `elem` bytes.
cudaError_t encode_2d(CUtensorMap* map, CUtensorMapDataType dtype, size_t elem, const void* base,
                      uint64_t cols, uint64_t rows, uint64_t ld, unsigned box_cols,
                      unsigned box_rows, CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_NONE);

}  // namespace ssm
