// k_trispec_tc.cu -- K3 on the tensor cores: the trispectrum cut (Eq. 31) with
// the factorised fourth k-statistic (App. H, Eq. 85) as one tcgen05 contraction
// per group, with accumulators and running sums in TMEM.
//
// With the centred coefficients d_j of a group and the frame Gram of bin k,
// G^k_jj' = Re(d_jk d_j'k*), the bracket of Eq. 85 for (a_k, a_k*, a_l, a_l*) is
//   B(k, l) = m(m+1) sum_j P_jk P_jl - (m-1)(|U|^2 + |V|^2)
//           = sum_{j<=j'} w_jj' G^k_jj' G^l_jj',
//   w_jj = m^2 - m + 2,  w_jj' = -4(m-1) for j < j',
// with P = |d|^2, U = sum_j d_jk d_jl, V = sum_j d_jk d_jl* (the cross terms of
// |U|^2 + |V|^2 regroup as 2 sum_{j,j'} G^k_jj' G^l_jj'), and
//   c4 = [B(k, l) - (m-1) Sk Sl] / ((m-1)(m-2)(m-3)),  Sk = sum_j P_jk.
// K1 writes the operand image of sqrt(|w| r) G (m(m+1)/2 entries in chunks of
// 16, see OperandImage), r = 1/((m-1)(m-2)(m-3)), followed by the entry
// ps = sqrt((m-1) r) Sk.  This kernel forms D = A_k A_l^T over K for every
// 128 x 128 tile of (k, l), negating the pair chunks (and with them ps_k ps_l)
// through the MMA's negate-A bit, in FP32 accumulators in TMEM: D is c4 itself
// (FP16: times s_k s_l, the rows' scales).
// Operands are split hi + lo (TF32 or BF16) and each chunk takes three MMAs
// hi*hi + hi*lo + lo*hi (one in the plain BF16 mode).
//
// Warp roles (608 threads), coupled only by mbarriers.  Warp 16, TMA: takes
// (group chunk, tile) items from the queue; per group it writes a record of the
// group into a ring of kPsSlots slots (FP16: with the tile's row scales),
// and per stage (group, kChunks consecutive K chunks) it loads two boxes of the
// operand image through a 4-D tensor map: the 16 row groups of the k-block and
// the 16 of the l-block.  Warps 17 and 18, MMA: warp 17 + w takes every other
// group (w = group index mod 2; TMEM buffer group index mod 4 of 128 columns, so
// the products run up to three groups ahead of the epilogue), reads the group's
// record from the ring, and per stage issues the MMAs of its chunks, commits
// them to the stage's barrier (the stage is then free for the next load) and,
// after the group's last stage, to the buffer's barrier; one warp's waits and
// commits overlap the other's products.  Warps 0-15, the epilogue: TMEM lane
// quadrant warp % 4, columns 32 (warp / 4) .. + 31.  For each group they read D
// in two halves of 16 columns (FP16: divided by the scales) and update the
// running sums and sums of squares of their 32 grid points, held in registers;
// at the end of an item they add both to the float64 accumulators.  Tiles of the last l-block are as
// narrow as the bins left (N a multiple of 16).  Every wait is bounded; on a
// failure the CTA stops, drains its copies and products and frees its TMEM.
#include "internal.cuh"
#include "pipeline.cuh"

namespace ss {
namespace {

constexpr int kTM = 128, kTN = 128, kEpiWarps = 16, kMmaWarps = 2;
constexpr int kTcThreads = 32 * (kEpiWarps + 1 + kMmaWarps);
constexpr uint32_t kTmemCols = 512;  // D0 | D1 | D2 | D3
constexpr int kBufs = 4;  // TMEM accumulator buffers: group g uses buffer g mod 4

__device__ __forceinline__ uint32_t buf_col(uint32_t b) { return b * kTN; }
constexpr int kEpiCols = kTN / (kEpiWarps / 4);  // columns of an epilogue warp (32)

// Operand formats.  In the image and in a stage, a row group (8 bins) holds,
// per K chunk, a hi block and a lo block of CB bytes; a block holds the core
// matrices (8 rows x 16 bytes) of the chunk's 16-byte entry groups, 128 bytes
// apart (LBO).  A stage holds kChunks chunks of 16 row groups, so row groups
// are kChunks * 2 CB apart (SBO).  Every stage is 64 KB.
template <int kFmt>
struct OpFmt;

template <>
struct OpFmt<kImageGramTF32> {  // TF32: K = 8 per MMA, two K steps of two core matrices
  static constexpr uint32_t kCB = 512, kKstepBytes = 256;
  static constexpr int kKsteps = 2, kChunks = 2, kStages = 3;
  static constexpr uint32_t kIdescAB = (2u << 7) | (2u << 10);
  static constexpr bool kF16Kind = false, kScaled = false;
};

template <>
struct OpFmt<kImageGramBF16> {  // BF16: K = 16 per MMA, one K step
  static constexpr uint32_t kCB = 256, kKstepBytes = 0;
  static constexpr int kKsteps = 1, kChunks = 4, kStages = 3;
  static constexpr uint32_t kIdescAB = (1u << 7) | (1u << 10);
  static constexpr bool kF16Kind = true, kScaled = false;
};

template <>
struct OpFmt<kImageGramF16> {  // FP16 (rows scaled by powers of two): as BF16, A/B type 0
  static constexpr uint32_t kCB = 256, kKstepBytes = 0;
  static constexpr int kKsteps = 1, kChunks = 4, kStages = 3;
  static constexpr uint32_t kIdescAB = 0u;
  static constexpr bool kF16Kind = true, kScaled = true;
};

// Shared-memory matrix descriptor, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

template <bool kF16Kind>
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          bool accumulate) {
  if constexpr (kF16Kind)
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Record of a group for the MMA warps and the epilogue (FP16: with its row scales).
struct GroupRec {
  int k0, l0, n, flags;  // n = tile columns; flags: 1 = last group of its item, 2 = stop
};

constexpr int kPsSlots = 8;  // ring of per-group records (a power of two)

// kPasses: 3 (hi*hi + hi*lo + lo*hi) or 1 (hi*hi, plain BF16).  rsc (FP16): the
// group's row scales 1/s_k at rsc + g * Mp.
template <int kFmt, int kPasses>
__global__ void __launch_bounds__(kTcThreads, 1)
k3_trispec_tc(const __grid_constant__ CUtensorMap tm_img, const float* __restrict__ rsc,
              int G, int nkc, int ndc, int M, int Mp,
              const TileInfo* __restrict__ tiles, WorkQueue wq, double* __restrict__ acc,
              long long plane, int* __restrict__ status) {
  using F = OpFmt<kFmt>;
  constexpr int S = F::kStages, KC = F::kChunks;
  constexpr uint32_t kChunkBytes = 2 * F::kCB;               // hi and lo blocks of a chunk
  constexpr uint32_t kRowGroupBytes = KC * kChunkBytes;      // a row group in a stage
  constexpr uint32_t kABytes = (kTM / 8) * kRowGroupBytes;   // box of 16 row groups
  constexpr uint32_t kStageBytes = 2 * kABytes;
  extern __shared__ __align__(1024) unsigned char smem_raw[];  // + 1024 spare bytes
  __shared__ __align__(8) uint64_t full[S];             // stage loaded (TMA)
  __shared__ __align__(8) uint64_t sdone[S];            // stage's products complete
  __shared__ __align__(8) uint64_t psfull[kPsSlots];    // group slot written (FP16: scales loaded)
  __shared__ __align__(8) uint64_t psempty[kPsSlots];   // group slot read by the epilogue
  __shared__ __align__(8) uint64_t afull[kBufs];        // TMEM buffer holds a finished group
  __shared__ __align__(8) uint64_t aempty[kBufs];       // TMEM buffer read by the epilogue
  __shared__ GroupRec prec[kPsSlots];
  // FP16: the row scales 1/s of the tile's k rows, then of its l columns
  __shared__ __align__(16) float psr[kPsSlots][F::kScaled ? kTM + kTN : 4];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* base = align1024<unsigned char>(smem_raw);

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&sdone[s], 1);
    }
    for (int p = 0; p < kPsSlots; ++p) {
      mbar_init(&psfull[p], 1);
      mbar_init(&psempty[p], kEpiWarps);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(&afull[b], 1);
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
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm_img))
                   : "memory");
      uint32_t q = 0, gq = 0;  // stages and groups issued
      int s = 0;               // stage of load q
      uint32_t ph = 0;         // parity of stage s's current use
      bool ok = true;
      for (;;) {
        const int item = atomicAdd(wq.counter, 1);
        if (item >= wq.n_items || *(volatile int*)&s_fail) break;
        const int t = item % wq.n_tiles;
        const int ga = (item / wq.n_tiles) * wq.group_chunk;
        const int gb = min(G, ga + wq.group_chunk);
        const TileInfo ti = tiles[t];
        const uint32_t pk = (uint32_t)min(kTM, Mp - ti.k0) * 4u;
        const uint32_t pl = (uint32_t)min(ti.ncols, Mp - ti.l0) * 4u;
        for (int g = ga; g < gb && ok; ++g) {
          // the group's record (FP16: and the tile's row scales)
          const int p = gq & (kPsSlots - 1);
          if (gq >= kPsSlots &&
              !mbar_wait_bounded(&psempty[p], ((gq / kPsSlots) - 1) & 1u, status)) {
            ok = false;
            break;
          }
          prec[p] = GroupRec{ti.k0, ti.l0, ti.ncols, (g == gb - 1) ? 1 : 0};
          if constexpr (F::kScaled) {
            const float* rg = rsc + (long long)g * Mp;
            mbar_arrive_expect_tx(&psfull[p], pk + pl);
            tma_load_1d(&psr[p][0], rg + ti.k0, pk, &psfull[p]);
            tma_load_1d(&psr[p][kTM], rg + ti.l0, pl, &psfull[p]);
          } else {
            asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(
                             smem_addr(&psfull[p]))
                         : "memory");
          }
          ++gq;
          // its stages of KC chunks (chunks past nkc and rows past Mp read as zeros)
          for (int kc0 = 0; kc0 < nkc; kc0 += KC) {
            if (q >= (uint32_t)S && !mbar_wait_bounded(&sdone[s], ph ^ 1u, status)) {
              ok = false;
              break;
            }
            unsigned char* st = base + (size_t)s * kStageBytes;
            mbar_arrive_expect_tx(&full[s], kStageBytes);
            tma_load_4d(st, &tm_img, 0, kc0, ti.k0 >> 3, g, &full[s]);
            tma_load_4d(st + kABytes, &tm_img, 0, kc0, ti.l0 >> 3, g, &full[s]);
            ++q;
            if (++s == S) {
              s = 0;
              ph ^= 1u;
            }
          }
        }
        if (!ok) break;
      }
      if (!ok) atomicExch(&s_fail, 1);
      // every copy this warp issued has landed before the CTA may exit (waited
      // before the stop records below move the barriers to their next phase)
      for (uint32_t i = q > (uint32_t)S ? q - S : 0; i < q; ++i)
        mbar_wait_bounded(&full[i % S], (i / S) & 1u, status);
      for (uint32_t i = gq > (uint32_t)kPsSlots ? gq - kPsSlots : 0; i < gq; ++i)
        mbar_wait_bounded(&psfull[i % kPsSlots], (i / kPsSlots) & 1u, status);
      // stop records (plain arrivals, no bytes) in the next two group slots: the
      // epilogue reads the first, each MMA warp the one of its next group
      for (uint32_t gs = gq; gs < gq + kMmaWarps; ++gs) {
        const int p = gs & (kPsSlots - 1);
        if (gs >= kPsSlots) mbar_wait_bounded(&psempty[p], ((gs / kPsSlots) - 1) & 1u, status);
        prec[p].flags = 2;
        asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(
                         smem_addr(&psfull[p]))
                     : "memory");
      }
    }
    __syncwarp();
  } else if (warp > kEpiWarps) {
    // ------------------------------------------------------------ MMA issuers
    // MMA warp w takes the groups gc = w, w + 2, ... (TMEM buffer w), so that one
    // warp's waits and commits overlap the other's products
    if (lane == 0) {
      const uint32_t w = (uint32_t)(warp - kEpiWarps - 1);
      const uint32_t idesc0 = (1u << 4) | F::kIdescAB | ((uint32_t)(kTM >> 4) << 24);
      // descriptors of stage 0; a stage adds kStageBytes >> 4 to the address field
      const uint64_t a_desc0 = smem_desc(smem_addr(base), 128, kRowGroupBytes);
      const uint64_t b_desc0 = smem_desc(smem_addr(base) + kABytes, 128, kRowGroupBytes);
      const uint32_t nst = (uint32_t)((nkc + KC - 1) / KC);  // stages per group
      int last_s = -1;
      uint32_t last_ph = 0;
      for (uint32_t gc = w;; gc += kMmaWarps) {
        // the group's record (tile columns, or stop)
        const int p = gc & (kPsSlots - 1);
        if (!mbar_wait_bounded(&psfull[p], (gc / kPsSlots) & 1u, status)) break;
        const GroupRec r = prec[p];
        if (r.flags & 2) break;
        const uint32_t b = gc % kBufs;
        const uint32_t d = taddr + buf_col(b);
        const uint32_t idesc = idesc0 | ((uint32_t)(r.n >> 3) << 17);
        // the buffer is free once the epilogue has read its previous group, gc - 3
        if (gc >= kBufs && !mbar_wait_bounded(&aempty[b], ((gc / kBufs) - 1) & 1u, status))
          break;
        // order the group's products after the epilogue's reads of the buffer; the
        // staged operands need no fence (TMA writes and MMA reads are both
        // async-proxy accesses ordered by the stage barrier)
        tc_fence_after();
        bool stop = false;
        for (uint32_t i = 0; i < nst; ++i) {
          const uint32_t q = gc * nst + i;  // the group's stages are loaded in order
          const int s = (int)(q % S);
          const uint32_t ph = (q / S) & 1u;
          if (!mbar_wait_bounded(&full[s], ph, status)) {
            stop = true;
            break;
          }
          const int kc0 = (int)i * KC;
          // descriptors of the stage; every MMA adds a compile-time offset
          const uint64_t sa = a_desc0 + (uint64_t)((s * kStageBytes) >> 4);
          const uint64_t sb = b_desc0 + (uint64_t)((s * kStageBytes) >> 4);
          const int nck = min(KC, nkc - kc0);
#pragma unroll
          for (int j = 0; j < KC; ++j) {
            if (j < nck) {
              const int kc = kc0 + j;
              const uint32_t id = kc < ndc ? idesc : (idesc | (1u << 13));  // negate A: pairs
#pragma unroll
              for (int pa = 0; pa < kPasses; ++pa) {
                constexpr uint64_t kLo = F::kCB >> 4;
#pragma unroll
                for (int kst = 0; kst < F::kKsteps; ++kst) {
                  const uint64_t off = (uint64_t)((j * kChunkBytes + kst * F::kKstepBytes) >> 4);
                  mma_issue<F::kF16Kind>(d, sa + off + (pa == 2 ? kLo : 0u),
                                   sb + off + (pa == 1 ? kLo : 0u), id,
                                   kc > 0 || pa > 0 || kst > 0);
                }
              }
            }
          }
          mma_commit(&sdone[s]);
          last_s = s;
          last_ph = ph;
        }
        if (stop) break;
        mma_commit(&afull[b]);  // arrives when the group's products are complete
      }
      if (*(volatile int*)status != 0) atomicExch(&s_fail, 1);
      // the products issued must be complete before the TMEM is freed
      if (last_s >= 0) mbar_wait_bounded(&sdone[last_s], last_ph, status);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3, h = warp >> 2;
    const uint32_t lane_addr = taddr + ((uint32_t)(32 * q) << 16);
    const int col0 = kEpiCols * h;  // this warp's 32 columns of the tile
    // running sums and sums of squares over the item's groups of this thread's
    // 32 points (row 32 q + lane, columns col0 ..)
    float sm[kEpiCols], sq[kEpiCols];
#pragma unroll
    for (int i = 0; i < kEpiCols; ++i) sm[i] = sq[i] = 0.f;
    for (uint32_t gc = 0;; ++gc) {
      const int p = gc & (kPsSlots - 1);
      const uint32_t b = gc % kBufs;
      // one decision per warp: the TMEM accesses below are warp-collective
      if (!__all_sync(0xffffffffu,
                      mbar_wait_bounded(&psfull[p], (gc / kPsSlots) & 1u, status))) {
        if (lane == 0) atomicExch(&s_fail, 1);
        break;
      }
      const GroupRec r = prec[p];
      if (r.flags & 2) break;
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&afull[b], (gc / kBufs) & 1u, status))) {
        if (lane == 0) atomicExch(&s_fail, 1);
        break;
      }
      tc_fence_after();
      // FP16: the row scales of k and l undo the operands' scaling, applied one at a
      // time (their product alone may leave the float range)
      const float rk = F::kScaled ? psr[p][32 * q + lane] : 1.f;
      // 16-column halves of this warp that meet the tile (the tile width is a
      // multiple of 16; columns past it hold no products and are never flushed)
      const int nh = min(kEpiCols / 16, max(0, (r.n - col0) >> 4));
#pragma unroll
      for (int hh = 0; hh < kEpiCols / 16; ++hh) {
        if (hh < nh) {
          const uint32_t col = col0 + 16 * hh;
          float d[16];
          tmem_ld16(lane_addr + buf_col(b) + col, d);
          tmem_wait_ld();
#pragma unroll
          for (int c = 0; c < 16; c += 4) {
            float rl[4] = {1.f, 1.f, 1.f, 1.f};
            if constexpr (F::kScaled) {
              const float4 r4 = *reinterpret_cast<const float4*>(&psr[p][kTM + col + c]);
              rl[0] = r4.x; rl[1] = r4.y; rl[2] = r4.z; rl[3] = r4.w;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              // c4 = D (FP16: D / s_k / s_l)
              const float v = F::kScaled ? (d[c + i] * rk) * rl[i] : d[c + i];
              sm[16 * hh + c + i] += v;
              sq[16 * hh + c + i] = fmaf(v, v, sq[16 * hh + c + i]);
            }
          }
        }
      }
      // this warp has read its part of the buffer and of the ps slot
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&aempty[b]))
                     : "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&psempty[p]))
                     : "memory");
      }
      if (r.flags & 1) {
        // end of an item: add the sums to the float64 accumulators.  Point (k, l),
        // k <= l, is stored at [l][k], so a warp's 32 rows k are 32 consecutive
        // doubles.
        const int k = r.k0 + 32 * q + lane;
#pragma unroll
        for (int i = 0; i < kEpiCols; ++i) {
          const int l = r.l0 + col0 + i;
          if (i < 16 * nh && k <= l && l < M) {
            const long long o = (long long)l * M + k;
            atomicAdd(acc + o, (double)sm[i]);
            atomicAdd(acc + 2 * plane + o, (double)sq[i]);
          }
          sm[i] = sq[i] = 0.f;
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

template <int kFmt>
size_t tc_smem_bytes_t() {
  using F = OpFmt<kFmt>;
  return (size_t)F::kStages * 2 * (kTM / 8) * F::kChunks * 2 * F::kCB + 1024;
}

}  // namespace

size_t k3tc_smem_bytes(int precision) {
  return precision == SS_PREC_TF32X3 ? tc_smem_bytes_t<kImageGramTF32>()
                                     : tc_smem_bytes_t<kImageGramBF16>();
}

int k3tc_stage_chunks(int precision) {
  return precision == SS_PREC_TF32X3 ? OpFmt<kImageGramTF32>::kChunks
                                     : OpFmt<kImageGramBF16>::kChunks;
}

cudaError_t launch_k3_trispec_tc(const CUtensorMap& tm_img, const OperandImage& oi, int channel,
                                 int G, int m, int M, int Mp, const TileInfo* tiles, int n_tiles,
                                 int precision, double* acc, long long plane, int nsm,
                                 int* counter, int* status, cudaStream_t stream) {
  if (G <= 0 || n_tiles <= 0) return cudaSuccess;
  if (m < 4 || m > kMaxGramM || (Mp & 15)) return cudaErrorInvalidValue;
  const size_t smem = k3tc_smem_bytes(precision);
  auto kern = precision == SS_PREC_TF32X3   ? k3_trispec_tc<kImageGramTF32, 3>
              : precision == SS_PREC_BF16X3 ? k3_trispec_tc<kImageGramBF16, 3>
              : precision == SS_PREC_FP16X3 ? k3_trispec_tc<kImageGramF16, 3>
                                            : k3_trispec_tc<kImageGramBF16, 1>;
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
  const float* rsc = oi.rsc ? oi.rsc + (size_t)channel * oi.chan_rsc : nullptr;
  kern<<<n_cta, kTcThreads, smem, stream>>>(tm_img, rsc, G, oi.nkc, oi.ndc, M, Mp,
                                            tiles, wq, acc, plane, status);
  return cudaGetLastError();
}

}  // namespace ss
