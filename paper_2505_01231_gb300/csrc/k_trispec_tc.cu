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
// sum_j |.|^2 / sqrt2 per bin.
//
// Warp roles (288 threads).  Warp 8, the producer: takes (group chunk, tile)
// items from the queue; for every step = (group, chunk of <= 16 frames) it
// issues 1-D TMA bulk copies of the image rows of the 128 bins at k0 and the 48
// at l0 into one of kTcStages stages, then the 30 (or 15 / 5) MMAs straight
// from the stage into the group's TMEM buffer (two buffers of 5 x 48 columns),
// commits them to the stage's mbarrier (stage reuse) and, after the group's last
// chunk, to the buffer's "full" mbarrier with a record of the group in shared
// memory.  Warps 0-7, the epilogue: for each group in order they wait for its
// buffer, read the five accumulators from TMEM (tcgen05.ld, TMEM lane quadrant
// = warp % 4, column half = warp / 4), form c4 and update the float32 sums of
// their 24 grid points, release the buffer, and at the end of an item add the
// sums to the float64 accumulators.  Producer and epilogue meet only on
// mbarriers, so copies, products and epilogue of consecutive groups overlap.
// Every wait is bounded; on a failure the CTA stops, drains its copies and
// products and frees its TMEM before returning.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "pipeline.cuh"

namespace ss {
namespace {

constexpr int kTM = 128, kTN = 48, kKpad = 16, kTcThreads = 288, kEpiWarps = 8;
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

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

struct GroupRec {
  int k0, l0, g, flags;  // flags: 1 = last group of its item, 2 = stop
};

template <bool kBF16>
__global__ void __launch_bounds__(kTcThreads, 1)
k3_trispec_tc(const unsigned char* __restrict__ img, const float* __restrict__ ps, int G, int m,
              int nch, int M, int Mp, long long chunk_bytes, const TileInfo* __restrict__ tiles,
              WorkQueue wq, float alpha, float scale2pb, int passes, double* __restrict__ acc,
              long long plane, int* __restrict__ status) {
  using F = OpFmt<kBF16>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];  // + 1024 spare bytes
  __shared__ __align__(8) uint64_t full[kTcStages];       // stage loaded (TMA)
  __shared__ __align__(8) uint64_t sdone[kTcStages];      // stage's products complete
  __shared__ __align__(8) uint64_t afull[2];              // TMEM buffer holds a finished group
  __shared__ __align__(8) uint64_t aempty[2];             // TMEM buffer read by the epilogue
  __shared__ GroupRec rec[2];
  // sums of |.|^2 / sqrt 2 of the group in each TMEM buffer: 128 k-bins, then 48 l-bins
  __shared__ __align__(16) float psb[2][kTM + kTN];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
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
      mbar_init(&sdone[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&afull[b], 2);  // the products' commit + the producer's record arrive
      mbar_init(&aempty[b], kEpiWarps);
    }
    s_fail = 0;
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

  if (warp == kEpiWarps) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | F::kIdescAB | ((uint32_t)(kTN >> 3) << 17) |
                             ((uint32_t)(kTM >> 4) << 24);
      uint32_t Q = 0;      // steps issued (stage Q % kTcStages)
      uint32_t gc = 0;     // groups issued (TMEM buffer gc % 2)
      bool ok = true;
      // per stage: the step last loaded into it (for the stage-reuse wait)
      long long stage_step[kTcStages];
      for (int s = 0; s < kTcStages; ++s) stage_step[s] = -1;
      auto load_step = [&](uint32_t q, int k0, int l0, int g, int ch) -> bool {
        const int s = q % kTcStages;
        if (stage_step[s] >= 0 &&  // the stage's previous products must be complete
            !mbar_wait_bounded(&sdone[s], ((uint32_t)stage_step[s] / kTcStages) & 1u, status))
          return false;
        stage_step[s] = q;
        const uint32_t kb = (uint32_t)min(kTM / 8, R - (k0 >> 3)) * kRowGroupBytes;
        const uint32_t lb = (uint32_t)min(kTN / 8, R - (l0 >> 3)) * kRowGroupBytes;
        const unsigned char* src = img + ((size_t)g * nch + ch) * (size_t)chunk_bytes;
        unsigned char* st = base + (size_t)s * kStageBytes;
        fence_async_smem();
        mbar_arrive_expect_tx(&full[s], kb + lb);
        tma_load_1d(st, src + (size_t)(k0 >> 3) * kRowGroupBytes, kb, &full[s]);
        tma_load_1d(st + kKBytes, src + (size_t)(l0 >> 3) * kRowGroupBytes, lb, &full[s]);
        return true;
      };
      for (;;) {
        const int item = atomicAdd(wq.counter, 1);
        if (item >= wq.n_items || *(volatile int*)&s_fail) break;
        const int t = item % wq.n_tiles;
        const int ga = (item / wq.n_tiles) * wq.group_chunk;
        const int gb = min(G, ga + wq.group_chunk);
        const int k0 = tiles[t].k0, l0 = tiles[t].l0;
        const int nsteps = (gb - ga) * nch;
        // keep kTcStages - 1 steps of copies ahead of the products
        int loaded = 0;
        for (; loaded < nsteps && loaded < kTcStages - 1 && ok; ++loaded)
          ok = load_step(Q + loaded, k0, l0, ga + loaded / nch, loaded % nch);
        for (int i = 0; i < nsteps && ok; ++i) {
          const uint32_t q = Q + i;
          const int s = q % kTcStages;
          const int ch = i % nch, gi = i / nch;
          const uint32_t b = (gc + gi) & 1u;
          if (ch == 0) {
            // the TMEM buffer (and its slot of P sums) is free once the epilogue has
            // read the group before last
            const uint32_t use = (gc + gi) >> 1;  // earlier uses of buffer b
            if (use > 0 && !mbar_wait_bounded(&aempty[b], (use - 1) & 1u, status)) {
              ok = false;
              break;
            }
            // stage the group's P sums for the epilogue; the copies count on afull[b]
            const float* psg = ps + (long long)(ga + gi) * Mp;
            const uint32_t pk = (uint32_t)min(kTM, Mp - k0) * 4u, pl = (uint32_t)min(kTN, Mp - l0) * 4u;
            asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(
                             smem_addr(&afull[b])),
                         "r"(pk + pl)
                         : "memory");
            tma_load_1d(&psb[b][0], psg + k0, pk, &afull[b]);
            tma_load_1d(&psb[b][kTM], psg + l0, pl, &afull[b]);
          }
          if (!mbar_wait_bounded(&full[s], (q / kTcStages) & 1u, status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d0 = taddr + b * 5 * kTN;
          const uint32_t ka = smem_addr(base + (size_t)s * kStageBytes), la = ka + kKBytes;
          // products (k-side, l-side): RR (Re,Re), II (Im,Im), X (Re,Im), Xt (Im,Re),
          // Q (P,P); a row group's six matrices are Re hi, Re lo, Im hi, Im lo, P hi, P lo
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
                mma_issue(d0 + pr * kTN, ad, bd, idesc, !(ch == 0 && ps_ == 0 && kst == 0),
                          kBF16);
              }
            }
          }
          mma_commit(&sdone[s]);
          if (ch == nch - 1) {
            const int g = ga + gi;
            rec[b].k0 = k0;
            rec[b].l0 = l0;
            rec[b].g = g;
            rec[b].flags = (g == gb - 1) ? 1 : 0;
            mma_commit(&afull[b]);  // arrives when the group's products are complete
            asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(
                             smem_addr(&afull[b]))
                         : "memory");
          }
          // refill the stage freed by the previous step while this step's products run
          if (loaded < nsteps) {
            ok = load_step(Q + loaded, k0, l0, ga + loaded / nch, loaded % nch);
            ++loaded;
          }
        }
        if (!ok) break;
        Q += nsteps;
        gc += gb - ga;
      }
      if (!ok) {
        atomicExch(&s_fail, 1);
        // drain: every stage's last copy and products, with bounded waits
        for (int s = 0; s < kTcStages; ++s)
          if (stage_step[s] >= 0) {
            mbar_wait_bounded(&full[s], ((uint32_t)stage_step[s] / kTcStages) & 1u, nullptr);
          }
      }
      // stop record: wait until the next buffer is free, then release it without products
      const uint32_t b = gc & 1u, use = gc >> 1;
      if (use > 0) mbar_wait_bounded(&aempty[b], (use - 1) & 1u, nullptr);
      rec[b].flags = 2;
      asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0], 2;" ::"r"(
                       smem_addr(&afull[b]))
                   : "memory");
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3, h = warp >> 2;
    float sum[24], sq[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) sum[i] = sq[i] = 0.f;
    for (uint32_t gc = 0;; ++gc) {
      const uint32_t b = gc & 1u;
      if (!mbar_wait_bounded(&afull[b], (gc >> 1) & 1u, status)) {
        atomicExch(&s_fail, 1);
        break;
      }
      const GroupRec r = rec[b];
      if (r.flags & 2) break;
      tc_fence_after();
      const uint32_t tb = taddr + ((uint32_t)(32 * q) << 16) + b * 5 * kTN + 24 * h;
      const int kr = r.k0 + 32 * q + lane;
      const int lc0 = r.l0 + 24 * h;
      const float skr = psb[b][32 * q + lane];
      // two rounds of 12 columns keep the live accumulator values within the
      // register budget of three warps per scheduler
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int cb = 12 * half;
        float v[5][12];
#pragma unroll
        for (int pr = 0; pr < 5; ++pr) {
          float t8[8], t4[4];
          tmem_ld8(tb + pr * kTN + cb, t8);
          tmem_ld4(tb + pr * kTN + cb + 8, t4);
#pragma unroll
          for (int e = 0; e < 8; ++e) v[pr][e] = t8[e];
#pragma unroll
          for (int e = 0; e < 4; ++e) v[pr][8 + e] = t4[e];
        }
        // sums of |.|^2 / sqrt 2 of the 12 columns (the same for the whole warp)
        float sl[12];
#pragma unroll
        for (int c = 0; c < 12; c += 4) {
          const float4 w = *reinterpret_cast<const float4*>(&psb[b][kTM + 24 * h + cb + c]);
          sl[c] = w.x; sl[c + 1] = w.y; sl[c + 2] = w.z; sl[c + 3] = w.w;
        }
        tmem_wait_ld();
        if (half == 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0)  // this warp has read the buffer
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&aempty[b]))
                         : "memory");
        }
#pragma unroll
        for (int i = 0; i < 12; ++i) {
          float u = v[0][i] * v[0][i];
          u = fmaf(v[1][i], v[1][i], u);
          u = fmaf(v[2][i], v[2][i], u);
          u = fmaf(v[3][i], v[3][i], u);
          u = fmaf(skr, sl[i], u);
          const float c = fmaf(alpha, v[4][i], -u);
          sum[cb + i] += c;
          sq[cb + i] = fmaf(c, c, sq[cb + i]);
        }
      }
      if (r.flags & 1) {
        // end of the item: add the sums (scaled back by 2 pb) to the float64 accumulators
#pragma unroll
        for (int c = 0; c < 24; ++c) {
          const int l = lc0 + c;
          if (kr <= l && l < M) {
            const long long o = (long long)kr * M + l;
            atomicAdd(acc + o, (double)sum[c] * scale2pb);
            atomicAdd(acc + 2 * plane + o, (double)sq[c] * scale2pb * scale2pb);
          }
          sum[c] = sq[c] = 0.f;
        }
      }
    }
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
