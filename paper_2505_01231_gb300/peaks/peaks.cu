// peaks.cu -- microbenchmarks of the two compute peaks the polyspectrum kernels
// are measured against: FP32 FMA on the CUDA cores (the bispectrum and the FP32
// trispectrum) and tcgen05 dense products of kind::tf32 and kind::f16 (BF16
// inputs) with FP32 accumulators in tensor memory (the tensor-core trispectrum).
// Built as its own small library (libsspeaks.so) and used by the bench only;
// the estimator library does not depend on it.
//
//   ssp_fma_peak  -- every SM runs 2048 threads of 16 independent FMA chains.
//   ssp_mma_peak  -- one CTA per SM; one thread issues M = 128, N = 256 products
//                    from shared-memory operands (K-major, no swizzle) into two
//                    alternating TMEM accumulators, then waits (bounded) for
//                    their completion.
//   ssp_mma_rate  -- the same with N = 32, 64, 96, 128 or 256: the rate of narrow
//                    products, whose operand reads from shared memory rather
//                    than the multipliers set the pace.
// Both time the kernel with CUDA events on a stream of their own and return the
// rate in FLOP/s (an FMA counts two).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kFmaThreads = 256, kFmaChains = 16;

__global__ void __launch_bounds__(kFmaThreads)
k_fma(int iters, float seed, float* __restrict__ out) {
  float a[kFmaChains];
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) a[c] = seed + 0.001f * (threadIdx.x + c);
  const float x = 0.9999f, y = 1e-7f * seed;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int c = 0; c < kFmaChains; ++c) a[c] = fmaf(a[c], x, y);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kFmaChains; ++c) s += a[c];
  if (s == 12345.678f) out[blockIdx.x] = s;  // keeps the chains live
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// no-swizzle shared-memory matrix descriptor: start, leading (K) and stride
// (8-row group) byte offsets
__device__ __forceinline__ uint64_t mdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

constexpr int kMmaM = 128;
constexpr uint32_t kRowBytes = 128;                       // K bytes per operand row
constexpr uint32_t kABytes = kMmaM * kRowBytes;            // 16 KB
constexpr uint32_t kPad = 96u << 10;                       // keeps one CTA per SM
constexpr unsigned long long kMmaWaitNs = 20000000000ull;  // 20 s

// kType: 0 = TF32 (kind::tf32), 1 = BF16, 2 = FP16 (both kind::f16); kMmaN: N
template <int kType, int kMmaN>
__global__ void __launch_bounds__(128, 1)
k_mma(int iters, int* __restrict__ status) {
  constexpr uint32_t kBBytes = kMmaN * kRowBytes;
  constexpr bool kBF16 = kType != 0;  // a 16-bit kind::f16 type
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tslot;
  unsigned char* base = smem + ((1024u - (smem_u32(smem) & 1023u)) & 1023u);
  // operands: small non-zero values (layout: [8-row group][16-byte K group][8 rows][16 B])
  for (uint32_t i = threadIdx.x; i < (kABytes + kBBytes) / 4; i += blockDim.x) {
    const uint32_t h = (i * 2654435761u) >> 9;
    float v = 0.25f + (float)(h & 1023u) * (1.0f / 4096.0f);
    uint32_t w = __float_as_uint(v);
    if (kType == 1) w = (w >> 16) | (w & 0xFFFF0000u);  // two BF16 values of about v
    if (kType == 2) {                                    // two FP16 values of about v
      const uint32_t hbits = __half_as_ushort(__float2half_rn(v));
      w = hbits | (hbits << 16);
    }
    reinterpret_cast<uint32_t*>(base)[i] = w;
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  if (threadIdx.x == 0) {
    // D f32 (bit 4), A/B format (bits 7-9, 10-12: tf32 = 2, bf16 = 1), K-major
    // A and B, N / 8 at bit 17, M / 16 at bit 24
    const uint32_t fmt = kType == 1 ? ((1u << 7) | (1u << 10))
                         : kType == 2 ? 0u
                                      : ((2u << 7) | (2u << 10));
    const uint32_t idesc = (1u << 4) | fmt | ((uint32_t)(kMmaN >> 3) << 17) |
                           ((uint32_t)(kMmaM >> 4) << 24);
    const uint64_t a0 = mdesc(smem_u32(base), 128, 8 * kRowBytes);
    const uint64_t b0 = mdesc(smem_u32(base) + kABytes, 128, 8 * kRowBytes);
    // one product consumes 32 bytes of K (8 TF32 or 16 BF16 values): 4 per row
    for (int it = 0; it < iters; ++it) {
      const uint32_t d = tmem + (uint32_t)(it & 1) * kMmaN;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint64_t off = (uint64_t)((ks * 256) >> 4);
        const uint32_t acc = (it > 1 || ks > 0) ? 1u : 0u;
        if (kBF16)
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
              "l"(a0 + off), "l"(b0 + off), "r"(idesc), "r"(acc));
        else
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
              "l"(a0 + off), "l"(b0 + off), "r"(idesc), "r"(acc));
      }
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&done))
        : "memory");
    // bounded wait for the products
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
      uint32_t ok;
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(ok)
          : "r"(smem_u32(&done))
          : "memory");
      if (ok) break;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > kMmaWaitNs) {
        atomicExch(status, 1);
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

int timed(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double* seconds) {
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess) return -1;
  if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1;
  *seconds = ms * 1e-3;
  (void)s;
  return 0;
}

}  // namespace

extern "C" {

// FP32 FMA rate of the whole device: returns 0 and fills seconds / flops_per_s.
int ssp_fma_peak(int iters, double* seconds, double* flops_per_s) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const int grid = nsm * (2048 / kFmaThreads);
  float* out = nullptr;
  cudaStream_t s;
  cudaEvent_t e0, e1;
  if (cudaMalloc(&out, grid * sizeof(float)) != cudaSuccess) return -1;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma<<<grid, kFmaThreads, 0, s>>>(iters / 10 + 1, 1.0f, out);  // warm-up
  cudaEventRecord(e0, s);
  k_fma<<<grid, kFmaThreads, 0, s>>>(iters, 1.0f, out);
  cudaEventRecord(e1, s);
  int rc = cudaGetLastError() == cudaSuccess ? timed(s, e0, e1, seconds) : -1;
  if (rc == 0)
    *flops_per_s = 2.0 * grid * kFmaThreads * (double)iters * 8 * kFmaChains / *seconds;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  cudaFree(out);
  return rc;
}

// tcgen05 dense product rate of the whole device for products of M = 128 and the
// given N, kind 0 = kind::tf32, 1 = kind::f16 with BF16 inputs, 2 = kind::f16 with
// FP16 inputs; returns 0, 1 if a bounded wait ran out, -1 on an error (or an N
// other than 32, 64, 96, 128, 256).
int ssp_mma_rate(int kind, int n, int iters, double* seconds, double* flops_per_s) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (iters < 2) iters = 2;
  if (kind < 0 || kind > 2) return -1;
  void (*kern)(int, int*) = nullptr;
#define SSP_PICK(N)                                                              \
  if (n == N) kern = kind == 1 ? k_mma<1, N> : kind == 2 ? k_mma<2, N> : k_mma<0, N>;
  SSP_PICK(32)
  SSP_PICK(64)
  SSP_PICK(96)
  SSP_PICK(128)
  SSP_PICK(256)
#undef SSP_PICK
  if (!kern) return -1;
  int* status = nullptr;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) return -1;
  cudaMemset(status, 0, sizeof(int));
  const size_t smem = kABytes + (size_t)n * kRowBytes + 1024 + kPad;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaFree(status);
    return -1;
  }
  cudaStream_t s;
  cudaEvent_t e0, e1;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  kern<<<nsm, 128, smem, s>>>(iters / 10 + 2, status);  // warm-up
  cudaEventRecord(e0, s);
  kern<<<nsm, 128, smem, s>>>(iters, status);
  cudaEventRecord(e1, s);
  int rc = cudaGetLastError() == cudaSuccess ? timed(s, e0, e1, seconds) : -1;
  int st = 0;
  if (rc == 0 && cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = -1;
  if (rc == 0 && st != 0) rc = 1;
  if (rc == 0) {
    const double k = kind == 0 ? 8.0 : 16.0;  // K of one product
    *flops_per_s = 2.0 * kMmaM * n * k * 4.0 * (double)iters * nsm / *seconds;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  cudaFree(status);
  return rc;
}

// the dense peak: products of M = 128, N = 256
int ssp_mma_peak(int kind, int iters, double* seconds, double* flops_per_s) {
  return ssp_mma_rate(kind, 256, iters, seconds, flops_per_s);
}

}  // extern "C"
