// k_trispec_tc.cu -- K3 on the tensor cores: the fourth-order moment sums of the
// trispectrum cut (Eq. 31, factorised estimator of App. H, Eq. 85) as tcgen05
// matrix products with accumulators in TMEM.
//
// Per group and per 128 x 48 tile of (k, l), with centred coefficients
// da = ar + j ai and P = |da|^2 over the group's frames j (the K dimension):
//   RR = Ar_k^T Ar_l, II = Ai_k^T Ai_l, X = Ar_k^T Ai_l, Xt = Ai_k^T Ar_l,
//   Q' = (alpha P_k)^T P_l,  alpha = m(m+1) / (2(m-1)),
// five real products of [128 x K] by [K x 48].  Then
//   c4 / (2 pb) = Q' - (Sk/sqrt2)(Sl/sqrt2) - (RR^2 + II^2 + X^2 + Xt^2),
// pb = 1/((m-2)(m-3)), Sk = sum_j P_jk, which is the factorised c4 of Eq. 85
// (the same algebra as the CUDA-core kernel k_trispec.cu, with the prefactors
// folded into the operands); the 2 pb factor is applied when the sums are
// flushed.
//
// Precision: operands are split as x = hi + lo in TF32 (or BF16) and each
// product is formed from three MMAs hi*hi + hi*lo + lo*hi accumulated in FP32
// in TMEM (one MMA per product in the plain BF16 mode).
//
// The operands come ready-made: K1 writes, once per group and chunk of <= 16
// frames, the hi/lo parts of Re, Im and |.|^2 in the K-major core-matrix layout
// the tensor cores read (the "operand image", see OperandImage), and the sums
// sum_j |.|^2 / sqrt2 per bin.  Pipeline of a CTA over its (group chunk, tile)
// items, per step = (group, chunk):
//   1-D TMA bulk copies of the image rows of the 128 bins at k0 and the 48 at
//   l0 into one of kTcStages stages -> one thread issues the 30 (or 15 / 5)
//   MMAs straight from the stage into the group's TMEM buffer (two buffers of
//   5 x 48 columns) and commits them to the stage's mbarrier -> when the
//   products of the previous step are complete its stage is refilled, and, at a
//   group boundary, all threads read the finished group's accumulators from
//   TMEM (tcgen05.ld), form c4 and update the float32 sums of their 24 grid
//   points while the tensor cores work on the next group.  Every wait is
//   bounded; a CTA that gives up drains its copies and products and frees its
//   TMEM before returning.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "pipeline.cuh"

namespace ss {
namespace {

constexpr int kTM = 128, kTN = 48, kKpad = 16, kTcThreads = 256;
constexpr int kTcStages = 3;
constexpr uint32_t kTmemCols = 512;  // two buffers of 5 x 48 fp32 columns

// Operand formats.  A matrix of a row group is CB bytes: its core matrices
// (8 rows x 16 bytes) for consecutive 16-byte frame groups, 128 bytes apart
// (LBO); consecutive row groups are 6 CB apart (SBO, the six matrices of a row
// group are adjacent).
template <bool kBF16>
struct OpFmt;

template <>
struct OpFmt<false> {  // TF32 operands, K = 8 per MMA
  static constexpr uint32_t kCB = 512, kLBO = 128, kSBO = 6 * 512, kKstepBytes = 256;
  static constexpr int kKsteps = 2;
  static constexpr uint32_t kIdescAB = (2u << 7) | (2u << 10);
};

template <>
struct OpFmt<true> {  // BF16 operands, K = 16 per MMA
  static constexpr uint32_t kCB = 256, kLBO = 128, kSBO = 6 * 256, kKstepBytes = 0;
  static constexpr int kKsteps = 1;
  static constexpr uint32_t kIdescAB = (1u << 7) | (1u << 10);
};

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // start address, leading / stride byte offsets (>> 4), descriptor version 1,
  // no swizzle
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          bool accumulate, bool bf16) {
  if (bf16)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)accumulate));
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <bool kBF16>
__global__ void __launch_bounds__(kTcThreads, 1)
k3_trispec_tc(const unsigned char* __restrict__ img, const float* __restrict__ ps, int G, int m,
              int nch, int M, int Mp, long long chunk_bytes, const TileInfo* __restrict__ tiles,
              WorkQueue wq, float alpha, float scale2pb, int passes, double* __restrict__ acc,
              long long plane, int* __restrict__ status) {
  using F = OpFmt<kBF16>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];  // + 1024 spare bytes
  __shared__ __align__(8) uint64_t full[kTcStages];
  __shared__ __align__(8) uint64_t mma_bar[kTcStages];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_item;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr uint32_t kRowGroupBytes = 6 * F::kCB;
  constexpr uint32_t kKBytes = (kTM / 8) * kRowGroupBytes;   // 16 row groups at k0
  constexpr uint32_t kLBytes = (kTN / 8) * kRowGroupBytes;   // 6 row groups at l0
  constexpr uint32_t kStageBytes = kKBytes + kLBytes;
  unsigned char* base = align1024<unsigned char>(smem_raw);
  const int R = Mp / 8;  // row groups per chunk of the image

  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&mma_bar[s], 1);
    }
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = tmem_slot;
  const uint32_t idesc = (1u << 4) | F::kIdescAB | ((uint32_t)(kTN >> 3) << 17) |
                         ((uint32_t)(kTM >> 4) << 24);
  const int q = warp & 3, h = warp >> 2;  // epilogue: TMEM lane quadrant, column half
  uint32_t qs = 0;    // running step counter: stage qs % kTcStages, barrier parities
  uint32_t gcnt = 0;  // running group counter: TMEM buffer gcnt % 2
  bool failed = false;
  long long last_commit[kTcStages];
  for (int s = 0; s < kTcStages; ++s) last_commit[s] = -1;
  uint32_t tma_next = 0, tma_issued = 0;

  for (int item; !failed && (item = next_item(wq, &s_item)) >= 0;) {
    const int t = item % wq.n_tiles;
    const int ga = (item / wq.n_tiles) * wq.group_chunk;
    const int gb = min(G, ga + wq.group_chunk);
    const int k0 = tiles[t].k0, l0 = tiles[t].l0;
    const int nsteps = (gb - ga) * nch;
    const uint32_t kb = (uint32_t)min(kTM / 8, R - (k0 >> 3)) * kRowGroupBytes;
    const uint32_t lb = (uint32_t)min(kTN / 8, R - (l0 >> 3)) * kRowGroupBytes;
    float sum[24], sq[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) sum[i] = sq[i] = 0.f;

    auto issue_tma = [&](int i) {
      const uint32_t Q = qs + i;
      const int s = Q % kTcStages;
      const int g = ga + i / nch, ch = i % nch;
      const unsigned char* src = img + ((size_t)g * nch + ch) * (size_t)chunk_bytes;
      unsigned char* st = base + (size_t)s * kStageBytes;
      mbar_arrive_expect_tx(&full[s], kb + lb);
      tma_load_1d(st, src + (size_t)(k0 >> 3) * kRowGroupBytes, kb, &full[s]);
      tma_load_1d(st + kKBytes, src + (size_t)(l0 >> 3) * kRowGroupBytes, lb, &full[s]);
    };
    // epilogue of group g held in TMEM buffer b (its products are complete)
    auto epilogue = [&](int g, uint32_t b) {
      const float* psg = ps + (long long)g * Mp;
      const int kr = k0 + 32 * q + lane;
      const float skr = kr < Mp ? __ldg(psg + kr) : 0.f;
      tc_fence_after();
      const uint32_t tb = taddr + ((uint32_t)(32 * q) << 16) + b * 5 * kTN + 24 * h;
#pragma unroll
      for (int c0 = 0; c0 < 24; c0 += 8) {
        float rr[8], ii[8], xx[8], xt[8], qq[8], sl[8];
        tmem_ld8(tb + 0 * kTN + c0, rr);
        tmem_ld8(tb + 1 * kTN + c0, ii);
        tmem_ld8(tb + 2 * kTN + c0, xx);
        tmem_ld8(tb + 3 * kTN + c0, xt);
        tmem_ld8(tb + 4 * kTN + c0, qq);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int lc = l0 + 24 * h + c0 + i;
          sl[i] = lc < Mp ? __ldg(psg + lc) : 0.f;
        }
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float u = rr[i] * rr[i];
          u = fmaf(ii[i], ii[i], u);
          u = fmaf(xx[i], xx[i], u);
          u = fmaf(xt[i], xt[i], u);
          u = fmaf(skr, sl[i], u);
          const float c = fmaf(alpha, qq[i], -u);
          sum[c0 + i] += c;
          sq[c0 + i] = fmaf(c, c, sq[c0 + i]);
        }
      }
      tc_fence_before();
    };

    if (tid == 0) {
      fence_async_smem();
      for (int i = 0; i < kTcStages && i < nsteps; ++i) issue_tma(i);
    }
    tma_next = qs;
    tma_issued = qs + (uint32_t)min(kTcStages, nsteps);
    for (int i = 0; i < nsteps; ++i) {
      const uint32_t Q = qs + i;
      const int s = Q % kTcStages;
      const int gi = i / nch, ch = i % nch;
      const uint32_t tb = (gcnt + gi) & 1u;
      const bool ok = mbar_wait_bounded(&full[s], (Q / kTcStages) & 1u, status);
      tma_next = Q + 1;
      // all threads are past the previous epilogue (TMEM reads done) and agree on success
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc_fence_after();
      last_commit[s] = Q;
      if (tid == 0) {
        const uint32_t d0 = taddr + tb * 5 * kTN;
        const uint32_t ka = smem_addr(base + (size_t)s * kStageBytes), la = ka + kKBytes;
        // products: (k-side, l-side) = RR (Re,Re), II (Im,Im), X (Re,Im), Xt (Im,Re),
        // Q (P,P); the six matrices of a row group are Re hi, Re lo, Im hi, Im lo,
        // P hi, P lo
#pragma unroll
        for (int pr = 0; pr < 5; ++pr) {
          const int pa = pr < 4 ? (pr & 1) : 2;
          const int pl = pr < 4 ? ((pr ^ (pr >> 1)) & 1) : 2;
          for (int ps_ = 0; ps_ < passes; ++ps_) {
            const int ha = (ps_ == 2) ? 1 : 0, hb = (ps_ == 1) ? 1 : 0;
#pragma unroll
            for (int kst = 0; kst < F::kKsteps; ++kst) {
              const uint64_t ad = smem_desc(ka + (pa * 2 + ha) * F::kCB + kst * F::kKstepBytes,
                                            F::kLBO, F::kSBO);
              const uint64_t bd = smem_desc(la + (pl * 2 + hb) * F::kCB + kst * F::kKstepBytes,
                                            F::kLBO, F::kSBO);
              const bool accum = !(ch == 0 && ps_ == 0 && kst == 0);
              mma_issue(d0 + pr * kTN, ad, bd, idesc, accum, kBF16);
            }
          }
        }
        mma_commit(&mma_bar[s]);
      }
      if (i > 0) {
        // the previous step's products are complete: refill its stage, and if it
        // closed a group, run that group's epilogue while this step's products run
        const uint32_t Qp = Q - 1;
        const int sp = Qp % kTcStages;
        const bool okp = mbar_wait_bounded(&mma_bar[sp], (Qp / kTcStages) & 1u, status);
        if (__syncthreads_or(!okp)) {
          failed = true;
          break;
        }
        if (tid == 0 && (i - 1) + kTcStages < nsteps) {
          fence_async_smem();
          issue_tma((i - 1) + kTcStages);
        }
        if ((i - 1) + kTcStages < nsteps) tma_issued = Qp + kTcStages + 1;
        if (ch == 0) epilogue(ga + gi - 1, (gcnt + gi - 1) & 1u);
      }
    }
    if (!failed && nsteps > 0) {
      const uint32_t Ql = qs + nsteps - 1;
      const bool okl = mbar_wait_bounded(&mma_bar[Ql % kTcStages], (Ql / kTcStages) & 1u, status);
      if (__syncthreads_or(!okl))
        failed = true;
      else
        epilogue(gb - 1, (gcnt + (gb - ga) - 1) & 1u);
    }
    if (failed) break;
    qs += nsteps;
    gcnt += gb - ga;
    // flush the item's sums (scaled back by 2 pb) into the float64 accumulators
    const int k = k0 + 32 * q + lane;
#pragma unroll
    for (int c = 0; c < 24; ++c) {
      const int l = l0 + 24 * h + c;
      if (k > l || l >= M) continue;
      const long long o = (long long)k * M + l;
      atomicAdd(acc + o, (double)sum[c] * scale2pb);
      atomicAdd(acc + 2 * plane + o, (double)sq[c] * scale2pb * scale2pb);
    }
  }
  if (failed && tid == 0) {
    // drain with bounded waits: the last products committed on each barrier and
    // the copies issued but not consumed, before the TMEM is freed
    for (int b = 0; b < kTcStages; ++b)
      if (last_commit[b] >= 0)
        mbar_wait_bounded(&mma_bar[b], ((uint32_t)last_commit[b] / kTcStages) & 1u, nullptr);
    for (uint32_t Q = tma_next; Q < tma_issued; ++Q)
      mbar_wait_bounded(&full[Q % kTcStages], (Q / kTcStages) & 1u, nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(kTmemCols));
  }
}

size_t tc_smem_bytes(bool bf16) {
  const size_t cb = bf16 ? OpFmt<true>::kCB : OpFmt<false>::kCB;
  return (size_t)kTcStages * (kTM / 8 + kTN / 8) * 6 * cb + 1024;
}

}  // namespace

size_t k3tc_smem_bytes(int precision) { return tc_smem_bytes(precision != SS_PREC_TF32X3); }

cudaError_t launch_k3_trispec_tc(const OperandImage& oi, int channel, int G, int m, int M, int Mp,
                                 const TileInfo* tiles, int n_tiles, int precision, double* acc,
                                 long long plane, int nsm, int* counter, int* status,
                                 cudaStream_t stream) {
  if (G <= 0 || n_tiles <= 0) return cudaSuccess;
  const bool bf16 = precision != SS_PREC_TF32X3;
  const int passes = precision == SS_PREC_BF16 ? 1 : 3;
  const size_t smem = tc_smem_bytes(bf16);
  auto kern = bf16 ? k3_trispec_tc<true> : k3_trispec_tc<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // one CTA per SM: each CTA allocates all 512 TMEM columns
  const int n_cta = nsm;
  WorkQueue wq;
  wq.counter = counter;
  wq.n_tiles = n_tiles;
  wq.group_chunk = work_group_chunk(G, n_tiles, n_cta);
  wq.n_items = n_tiles * ((G + wq.group_chunk - 1) / wq.group_chunk);
  e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  const double md = m;
  const float alpha = (float)(md * (md + 1.0) / (2.0 * (md - 1.0)));
  const float scale2pb = (float)(2.0 / ((md - 2.0) * (md - 3.0)));
  const unsigned char* img = static_cast<const unsigned char*>(oi.img) + (size_t)channel * oi.chan_bytes;
  const float* ps = oi.ps + (size_t)channel * oi.chan_ps;
  kern<<<n_cta, kTcThreads, smem, stream>>>(img, ps, G, m, oi.nch, M, Mp, oi.chunk_bytes, tiles, wq,
                                            alpha, scale2pb, passes, acc, plane, status);
  return cudaGetLastError();
}

}  // namespace ss
