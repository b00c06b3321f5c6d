// lbm_tma.cuh -- Tensor Memory Accelerator (TMA) tile loads and mbarrier
// waits for sm_103a, in inline PTX.
//
// A tile's inputs are brought into shared memory by cp.async.bulk.tensor
// (one thread issues them; the copies complete on an mbarrier with a
// transaction count), so that the loads of the next tile run while the CTA
// computes the current one.  Every wait is bounded: after kSpinLimit
// polls a wait gives up and reports it, so a lost copy can never hang the
// GPU; the caller then records an error and drains.  No multicast and no
// cluster: every copy reads this GPU's own memory into its own CTA.
#pragma once

#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

namespace lbmk {

// A wait gives up after about a second of GPU time (%globaltimer), or
// after kSpinLimit polls, whichever comes first.
constexpr unsigned kSpinLimit = 1u << 26;
constexpr unsigned long long kWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

// make the barrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses of the same memory
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// One poll of phase `parity`; true when that phase has completed.
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

// Bounded wait; false if the phase did not complete within the bound.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned k = 0; k < kSpinLimit; k++) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((k & 255u) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// 3-D tiled TMA load of the box at (x, y, z) into shared memory; completes on
// `bar` with the box's bytes.  x must be a multiple of 16 bytes' worth of
// elements (the caller's tiles guarantee it).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y,
                                            int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

}  // namespace lbmk
