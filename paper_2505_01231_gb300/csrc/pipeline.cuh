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

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// First 128-byte aligned address at or after p in shared memory (tiled TMA
// destinations need 128-byte alignment; kernels reserve 128 spare bytes).
template <typename T>
__device__ __forceinline__ T* align128(void* p) {
  const uint32_t a = smem_addr(p);
  return reinterpret_cast<T*>(static_cast<char*>(p) + ((128u - (a & 127u)) & 127u));
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
// kStatusWaitTimeout) if the phase does not complete within kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_timer_ns() - t0 > kWaitLimitNs) {
      if (status) atomicExch(status, kStatusWaitTimeout);
      return false;
    }
  }
  return true;
}

// Scheduling cost of one (tile, group) unit: the warps of the CTA whose
// sub-tile touches the domain, plus a fixed part for staging and barriers that
// every group pays whatever the tile's shape.
constexpr int kTileFixedCost = 3;

// Work description of one tile of (k, l) grid points: origin and per-group
// weight (number of warps of the CTA whose sub-tile touches the domain).
// `prefix` is the sum of the weights of all earlier tiles.
struct TileInfo {
  int k0, l0, weight, prefix;
};

// Balanced static schedule: the work units are (tile t, group g) with weight
// w_t each, laid out tile-major; CTA c of n takes the weight range
// [c W / n, (c+1) W / n).  Group g of tile t belongs to the CTA whose range holds
// the unit's first weight position P_t G + g w_t, so every unit is taken once.
// Calls f(tile_index, g_begin, g_end) for each tile segment of the CTA's range.
template <typename F>
__device__ __forceinline__ void for_each_segment(const TileInfo* __restrict__ tiles, int n_tiles,
                                                 int G, int cta, int n_cta, F&& f) {
  const long long total_w = (long long)(tiles[n_tiles - 1].prefix + tiles[n_tiles - 1].weight) * G;
  const long long x0 = total_w * cta / n_cta;
  const long long x1 = total_w * (cta + 1) / n_cta;
  for (int t = 0; t < n_tiles; ++t) {
    const long long w = tiles[t].weight;
    if (w == 0) continue;
    const long long p0 = (long long)tiles[t].prefix * G;
    const long long p1 = p0 + w * G;
    if (p1 <= x0) continue;
    if (p0 >= x1) break;
    const long long a = x0 > p0 ? x0 - p0 : 0;
    const long long b = (x1 < p1 ? x1 : p1) - p0;
    const int ga = (int)((a + w - 1) / w);
    const int gb = (int)((b + w - 1) / w);
    if (gb > ga) f(t, ga, gb);
  }
}

}  // namespace ss
