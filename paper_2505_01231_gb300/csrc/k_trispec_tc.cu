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
// Pipeline of a CTA over its (group chunk, tile) items, per step = (group,
// chunk of <= 16 frames):
//   TMA loads of the complex coefficients (128 bins at k0, 48 at l0) into one
//   of two stages -> all threads convert them into K-major split operands in
//   one of two operand buffers -> one thread issues the 30 (or 10 / 5) MMAs into
//   the group's TMEM buffer (two buffers of 5 x 48 columns) and commits them to
//   an mbarrier -> while those run, all threads read the previous group's
//   accumulators from TMEM (tcgen05.ld), form c4 and update the float32 sums of
//   their 24 grid points.  Every wait is bounded; a CTA that gives up drains
//   its copies and products and frees its TMEM before returning.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "pipeline.cuh"

namespace ss {
namespace {

constexpr int kTM = 128, kTN = 48, kKpad = 16, kTcThreads = 256;
constexpr int kTcStages = 2;
constexpr uint32_t kTmemCols = 512;  // two buffers of 5 x 48 fp32 columns

template <bool kBF16>
struct OpFmt;

template <>
struct OpFmt<false> {  // TF32 operands, K = 8 per MMA
  static constexpr uint32_t kMatK = kTM * kKpad * 4, kMatL = kTN * kKpad * 4;
  static constexpr uint32_t kLBO = 128, kSBO = 512, kKstepBytes = 256;
  static constexpr int kKsteps = 2;
  static constexpr uint32_t kIdescAB = (2u << 7) | (2u << 10);
  // byte offset of element (row r, frame k) in the no-swizzle K-major layout of
  // 8-row x 16-byte core matrices, K-adjacent cores 128 bytes apart
  __device__ static uint32_t off(int r, int k) {
    return ((r >> 3) * 4 + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4;
  }
};

template <>
struct OpFmt<true> {  // BF16 operands, K = 16 per MMA
  static constexpr uint32_t kMatK = kTM * kKpad * 2, kMatL = kTN * kKpad * 2;
  static constexpr uint32_t kLBO = 128, kSBO = 256, kKstepBytes = 0;
  static constexpr int kKsteps = 1;
  static constexpr uint32_t kIdescAB = (1u << 7) | (1u << 10);
  __device__ static uint32_t off(int r, int k) {
    return ((r >> 3) * 2 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
  }
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

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t t;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
  return t;
}

// split x = hi + lo in the operand format; returns the bits of (hi, lo)
template <bool kBF16>
__device__ __forceinline__ void split(float x, uint32_t& hi, uint32_t& lo) {
  if constexpr (kBF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
  } else {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
  }
}

struct TcSmem {
  unsigned char* stage[kTcStages];  // [FC][8][16] float2 at k0 | [FC][3][16] float2 at l0
  uint32_t lside_off;               // offset of the l-side box inside a stage
  unsigned char* ops[2];            // split operands: 6 k-side then 6 l-side matrices
  float* sk;                        // [2][128] sum_j P / sqrt 2 per TMEM buffer
  float* sl;                        // [2][48]
};

template <bool kBF16>
__global__ void __launch_bounds__(kTcThreads, 1)
k3_trispec_tc(const __grid_constant__ CUtensorMap tm128, const __grid_constant__ CUtensorMap tm48,
              int row0, int G, int m, int FC, int M, const TileInfo* __restrict__ tiles,
              WorkQueue wq, float alpha, float scale2pb, int passes,
              double* __restrict__ acc, long long plane, int* __restrict__ status) {
  using F = OpFmt<kBF16>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];  // + 1024 spare bytes
  __shared__ __align__(8) uint64_t full[kTcStages];
  __shared__ __align__(8) uint64_t mma_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_item;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  unsigned char* base = align1024<unsigned char>(smem_raw);
  const uint32_t k_bytes = (uint32_t)FC * 1024u;
  const uint32_t l_bytes = ((uint32_t)FC * 384u + 1023u) & ~1023u;
  const uint32_t stage_bytes = k_bytes + l_bytes;
  const uint32_t op_bytes = 6 * F::kMatK + 6 * F::kMatL;  // multiples of 1024
  TcSmem S;
  S.stage[0] = base;
  S.stage[1] = base + stage_bytes;
  S.lside_off = k_bytes;
  S.ops[0] = base + 2 * stage_bytes;
  S.ops[1] = S.ops[0] + op_bytes;
  S.sk = reinterpret_cast<float*>(S.ops[1] + op_bytes);
  S.sl = S.sk + 2 * kTM;

  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) mbar_init(&full[s], 1);
    mbar_init(&mma_bar[0], 1);
    mbar_init(&mma_bar[1], 1);
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
  const int nch = (m + FC - 1) / FC;
  // epilogue role: TMEM lane quadrant q (rows 32q..32q+31), column half h
  const int q = warp & 3, h = warp >> 2;
  uint32_t qs = 0;   // running step counter: TMA stage q % 2, mbarrier parities
  uint32_t gcnt = 0; // running group counter: TMEM / sk buffer gcnt % 2
  bool failed = false;
  // for a bounded drain after a failure: last committed step per product
  // barrier, and the TMA steps issued but not yet waited for
  long long last_commit[2] = {-1, -1};
  uint32_t tma_next = 0, tma_issued = 0;

  for (int item; !failed && (item = next_item(wq, &s_item)) >= 0;) {
    const int t = item % wq.n_tiles;
    const int ga = (item / wq.n_tiles) * wq.group_chunk;
    const int gb = min(G, ga + wq.group_chunk);
    const int k0 = tiles[t].k0, l0 = tiles[t].l0;
    const int nsteps = (gb - ga) * nch;
    float sum[24], sq[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) sum[i] = sq[i] = 0.f;

    auto issue_tma = [&](int i) {
      const uint32_t Q = qs + i;
      const int s = Q % kTcStages;
      const int g = ga + i / nch, j0 = (i % nch) * FC;
      mbar_arrive_expect_tx(&full[s], (uint32_t)FC * (1024u + 384u));
      tma_load_3d(S.stage[s], &tm128, 0, k0 >> 4, row0 + g * m + j0, &full[s]);
      tma_load_3d(S.stage[s] + S.lside_off, &tm48, 0, l0 >> 4, row0 + g * m + j0, &full[s]);
    };
    // epilogue of the group held in TMEM buffer b (its products are complete)
    auto epilogue = [&](int b) {
      tc_fence_after();
      const float skr = S.sk[b * kTM + 32 * q + lane];
      const uint32_t tb = taddr + ((uint32_t)(32 * q) << 16) + (uint32_t)b * 5 * kTN + 24 * h;
#pragma unroll
      for (int c0 = 0; c0 < 24; c0 += 8) {
        float rr[8], ii[8], xx[8], xt[8], qq[8];
        tmem_ld8(tb + 0 * kTN + c0, rr);
        tmem_ld8(tb + 1 * kTN + c0, ii);
        tmem_ld8(tb + 2 * kTN + c0, xx);
        tmem_ld8(tb + 3 * kTN + c0, xt);
        tmem_ld8(tb + 4 * kTN + c0, qq);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float u = rr[i] * rr[i];
          u = fmaf(ii[i], ii[i], u);
          u = fmaf(xx[i], xx[i], u);
          u = fmaf(xt[i], xt[i], u);
          u = fmaf(skr, S.sl[b * kTN + 24 * h + c0 + i], u);
          const float c = qq[i] - u;
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
    for (int i = 0; i < nsteps && !failed; ++i) {
      const uint32_t Q = qs + i;
      const int s = Q % kTcStages;
      const int gi = i / nch, ch = i % nch;
      const int nf = min(FC, m - ch * FC);
      const uint32_t tb = (gcnt + gi) & 1u;  // TMEM / sk buffer of this group
      bool ok = mbar_wait_bounded(&full[s], (Q / kTcStages) & 1u, status);
      tma_next = Q + 1;
      // operand buffer Q % 2 is free once the products of step Q-2 are complete
      if (ok && Q >= 2 && i >= 2) ok = mbar_wait_bounded(&mma_bar[Q & 1], ((Q - 2) >> 1) & 1u, status);
      // ---- convert: complex coefficients -> K-major split operands
      unsigned char* ops = S.ops[Q & 1];
      const unsigned char* st = S.stage[s];
      if (tid < kTM + kTN) {
        const bool kside = tid < kTM;
        const int r = kside ? tid : tid - kTM;
        const uint32_t rowb = kside ? 1024u : 384u;
        const unsigned char* src = st + (kside ? 0u : S.lside_off);
        unsigned char* dst = ops + (kside ? 0u : 6 * F::kMatK);
        const uint32_t mat = kside ? F::kMatK : F::kMatL;
        const float sc = kside ? alpha : 1.f;
        float psum = 0.f;
        constexpr int kPer = kBF16 ? 8 : 4;  // K elements per 16-byte core-matrix row
#pragma unroll
        for (int kg = 0; kg < kKpad / kPer; ++kg) {
          uint32_t w[6][kPer];
#pragma unroll
          for (int e = 0; e < kPer; ++e) {
            const int j = kg * kPer + e;
            float re = 0.f, im = 0.f;
            if (j < nf) {
              const float2 v = *reinterpret_cast<const float2*>(src + swz128(j * rowb + r * 8));
              re = v.x;
              im = v.y;
            }
            const float p = fmaf(re, re, im * im);
            psum += p;
            split<kBF16>(re, w[0][e], w[1][e]);
            split<kBF16>(im, w[2][e], w[3][e]);
            split<kBF16>(p * sc, w[4][e], w[5][e]);
          }
#pragma unroll
          for (int mt = 0; mt < 6; ++mt) {
            uint4 pk;
            if constexpr (kBF16) {
              pk = make_uint4(w[mt][0] | (w[mt][1] << 16), w[mt][2] | (w[mt][3] << 16),
                              w[mt][4] | (w[mt][5] << 16), w[mt][6] | (w[mt][7] << 16));
            } else {
              pk = make_uint4(w[mt][0], w[mt][1], w[mt][2], w[mt][3]);
            }
            *reinterpret_cast<uint4*>(dst + mt * mat + F::off(r, kg * kPer)) = pk;
          }
        }
        float* sx = kside ? &S.sk[tb * kTM + r] : &S.sl[tb * kTN + r];
        const float v = psum * 0.70710678118654752f;
        *sx = (ch == 0) ? v : *sx + v;
      }
      fence_async_smem();
      // a failed wait anywhere stops the CTA (after this barrier all agree)
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      tc_fence_after();
      last_commit[Q & 1] = Q;
      if (i + kTcStages < nsteps) tma_issued = Q + kTcStages + 1;
      if (tid == 0) {
        // refill the TMA stage just consumed
        if (i + kTcStages < nsteps) issue_tma(i + kTcStages);
        const uint32_t d0 = taddr + tb * 5 * kTN;
        const uint32_t ka = smem_addr(ops), la = ka + 6 * F::kMatK;
        // products: (k-side matrix, l-side matrix) = RR (Ar,Ar), II (Ai,Ai), X (Ar,Ai),
        // Xt (Ai,Ar), Q (P,P); matrices are ordered hi, lo for Ar, Ai, P
#pragma unroll
        for (int pr = 0; pr < 5; ++pr) {
          const int pa = pr < 4 ? (pr & 1) : 2;              // Ar, Ai, Ar, Ai, P
          const int pl = pr < 4 ? ((pr ^ (pr >> 1)) & 1) : 2;  // Ar, Ai, Ai, Ar, P
          for (int ps = 0; ps < passes; ++ps) {
            const int ha = (ps == 2) ? 1 : 0, hb = (ps == 1) ? 1 : 0;
#pragma unroll
            for (int kst = 0; kst < F::kKsteps; ++kst) {
              const uint64_t ad = smem_desc(ka + (pa * 2 + ha) * F::kMatK + kst * F::kKstepBytes,
                                            F::kLBO, F::kSBO);
              const uint64_t bd = smem_desc(la + (pl * 2 + hb) * F::kMatL + kst * F::kKstepBytes,
                                            F::kLBO, F::kSBO);
              const bool accum = !(ch == 0 && ps == 0 && kst == 0);
              mma_issue(d0 + pr * kTN, ad, bd, idesc, accum, kBF16);
            }
          }
        }
        mma_commit(&mma_bar[Q & 1]);
      }
      // epilogue of the previous group while this step's products run
      if (ch == 0 && gi > 0) {
        const uint32_t Qp = Q - 1;  // last step of the previous group
        const bool okp = mbar_wait_bounded(&mma_bar[Qp & 1], (Qp >> 1) & 1u, status);
        if (__syncthreads_or(!okp)) {
          failed = true;
          break;
        }
        epilogue((gcnt + gi - 1) & 1u);
      }
    }
    if (!failed && nsteps > 0) {
      const uint32_t Ql = qs + nsteps - 1;
      const bool okl = mbar_wait_bounded(&mma_bar[Ql & 1], (Ql >> 1) & 1u, status);
      if (__syncthreads_or(!okl)) {
        failed = true;
      } else {
        epilogue((gcnt + (gb - ga) - 1) & 1u);
      }
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
    for (int b = 0; b < 2; ++b)
      if (last_commit[b] >= 0)
        mbar_wait_bounded(&mma_bar[b], ((uint32_t)last_commit[b] >> 1) & 1u, nullptr);
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

size_t tc_smem_bytes(int FC, bool bf16) {
  const size_t k_bytes = (size_t)FC * 1024;
  const size_t l_bytes = ((size_t)FC * 384 + 1023) & ~(size_t)1023;
  const size_t mk = bf16 ? OpFmt<true>::kMatK : OpFmt<false>::kMatK;
  const size_t ml = bf16 ? OpFmt<true>::kMatL : OpFmt<false>::kMatL;
  return 2 * (k_bytes + l_bytes) + 2 * (6 * mk + 6 * ml) + (2 * kTM + 2 * kTN) * sizeof(float) +
         1024;
}

}  // namespace

size_t k3tc_smem_bytes(int FC, int precision) {
  return tc_smem_bytes(FC, precision != SS_PREC_TF32X3);
}

cudaError_t launch_k3_trispec_tc(const CUtensorMap& tm128, const CUtensorMap& tm48, int row0,
                                 int G, int m, int FC, int M, const TileInfo* tiles, int n_tiles,
                                 int precision, double* acc, long long plane, int nsm,
                                 int* counter, int* status, cudaStream_t stream) {
  if (G <= 0 || n_tiles <= 0) return cudaSuccess;
  const bool bf16 = precision != SS_PREC_TF32X3;
  const int passes = precision == SS_PREC_BF16 ? 1 : 3;
  const size_t smem = tc_smem_bytes(FC, bf16);
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
  kern<<<n_cta, kTcThreads, smem, stream>>>(tm128, tm48, row0, G, m, FC, M, tiles, wq, alpha,
                                            scale2pb, passes, acc, plane, status);
  return cudaGetLastError();
}

}  // namespace ss
