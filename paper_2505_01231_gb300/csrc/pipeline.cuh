// pipeline.cuh -- shared-memory staging helpers for sm_103a: mbarriers, 1-D TMA
// bulk copies (cp.async.bulk) and bounded waits, plus the balanced static
// schedule of (tile, group range) work used by the persistent pair kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ss {

// Device status codes written to the plan's status word.
enum : int { kStatusOk = 0, kStatusWaitTimeout = 1 };

// A wait on an mbarrier gives up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
// Limit of the wait that the timeout test injects (on a barrier nothing completes).
constexpr unsigned long long kInjectedWaitNs = 1000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// First 1024-byte aligned address at or after p in shared memory (destinations
// of 128-byte-swizzled TMA loads; kernels reserve 1024 spare bytes).
template <typename T>
__device__ __forceinline__ T* align1024(void* p) {
  const uint32_t a = smem_addr(p);
  return reinterpret_cast<T*>(static_cast<char*>(p) + ((1024u - (a & 1023u)) & 1023u));
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// make barrier initialisation and prior generic smem writes visible to the async proxy
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared, completion counted on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// 2-D tiled TMA load of one box of a tensor map (coordinates {x, y}, x the
// innermost; x * element size must be a multiple of 16 bytes); bins outside the
// tensor are filled with zeros.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// 3-D tiled TMA load (coordinates {x, y, z}).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// 4-D tiled TMA load (coordinates {x, y, z, w}).
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            int w, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
      : "memory");
}

// Byte offset, inside a 1024-byte aligned shared buffer written by a TMA load
// with 128-byte swizzling, of the 16-byte chunk holding logical offset `off`:
// the chunk index (bits 4-6) is XOR-ed with the 128-byte row index (bits 7-9).
__device__ __forceinline__ uint32_t swz128(uint32_t off) {
  return off ^ (((off >> 7) & 7u) << 4);
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false (and records
// kStatusWaitTimeout) if the phase does not complete within limit_ns
// nanoseconds (kWaitLimitNs; the injected wait of the timeout test is shorter).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_timer_ns() - t0 > limit_ns) {
      if (status) atomicExch(status, kStatusWaitTimeout);
      return false;
    }
  }
  return true;
}

// Work description of one tile of (k, l) grid points: its origin, how many of
// the CTA's eight 32 x 16 warp sub-tiles touch the domain (CUDA-core kernels)
// and its number of l columns (tensor-core kernel, a multiple of 16).
struct TileInfo {
  int k0, l0, active_warps, ncols;
};

// Dynamic work queue of the persistent pair kernels.  Item i is (group chunk
// i / n_tiles, tile i % n_tiles): group-major, so the CTAs working at the same
// time share one chunk of centred spectra in L2.  A CTA takes the next item
// with one atomicAdd on a counter that the host zeroes before the launch.
struct WorkQueue {
  int* counter;
  int n_tiles;
  int group_chunk;
  int n_items;
};

// Returns the next item for the calling CTA (all threads receive it) or -1.
__device__ __forceinline__ int next_item(const WorkQueue& q, int* s_slot) {
  __syncthreads();  // the previous item's readers of *s_slot are done
  if (threadIdx.x == 0) *s_slot = atomicAdd(q.counter, 1);
  __syncthreads();
  const int it = *s_slot;
  return it < q.n_items ? it : -1;
}

}  // namespace ss
