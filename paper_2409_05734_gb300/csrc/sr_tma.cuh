// Tensor-memory-access (TMA) and mbarrier helpers written as inline PTX for
// sm_100-family GPUs: 2D tiled bulk loads from global into shared memory with
// 128-byte swizzle, completion through a transaction-counting mbarrier, and a
// bounded wait that gives up (instead of spinning forever) after a fixed
// number of polls.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sr {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// subsequent async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrive on the barrier and add `bytes` to the transactions the current phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for phase `parity` of the barrier for at most kWaitNs nanoseconds of
// the global timer; false on give-up (the caller records an error and stops).
constexpr uint64_t kWaitNs = 100ull * 1000 * 1000;
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

// As mbar_wait_bounded, for threads that expect a long wait (the end of a whole
// main loop): they poll every `sleep_ns` nanoseconds and leave the shared-memory
// pipe to the barrier traffic of the threads that keep the loop going.
__device__ __forceinline__ bool mbar_wait_bounded_sleep(uint32_t bar, uint32_t parity, unsigned sleep_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    __nanosleep(sleep_ns);
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

// 2D tiled TMA load of one box at element coordinates (x, y) into shared
// memory at `dst`, completing `bytes` transactions on barrier `bar`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Byte offset of element (row t, position q) of a tile loaded as boxes of
// 16 complex values (128 bytes) x T rows with CU_TENSOR_MAP_SWIZZLE_128B into a
// 1024-byte-aligned buffer: box q/16 starts at (q/16) * box_stride (a multiple
// of 1024), row t of a box sits at t*128, and the 16-byte chunk index (address
// bits 4..6) is XORed with the 128-byte row index modulo 8 (bits 7..9).
__device__ __forceinline__ uint32_t swz128_offset(int box_stride, int t, int q) {
  const uint32_t lin = (uint32_t)((q >> 4) * box_stride + (t << 7) + ((q & 15) << 3));
  return lin ^ (((lin >> 7) & 7u) << 4);
}

}  // namespace sr
