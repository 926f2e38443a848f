// k_trispec_cross_tc.cu -- K3 for several channels on the tcgen05 tensor cores:
// per-group trispectrum-cut k-statistics C4(a_k, b_k*, c_l, d_l*) (Sec. 7,
// Eq. 50) in the factorised form of App. H, Eq. 85.
//
// Per group and combination (a, b, c, d), with centred coefficients and
// x_j = da_jk, y_j = db_jk*, z_j = dc_jl, w_j = dd_jl* (a_{-k} = a_k*):
//   c4(k, l) = pref [fmm P - fm1 (Sxy Szw + Sxz Syw + Sxw Syz)],
//   P = sum_j x_j y_j z_j w_j,   Suv = sum_j u_j v_j   (j over the m frames).
// Over a tile of 128 rows k and 24 columns l, Sxz, Sxw, Syz, Syw and P are
// complex matrix products with the frames as K:
//   rows x (128 x m) and rows y (128 x m) times columns [z | w] (m x 48), and
//   rows xy (128 x m) times columns zw (m x 24).
// Each complex product is a real one with K = 2m (real and imaginary part of
// frame j at 2j and 2j + 1): a row u is (ur_j, ui_j); the column giving Re(u v)
// is (vr_j, -vi_j) and the one giving Im(u v) is (vi_j, vr_j), so [z | w] is 96
// real columns and zw 48.  The products run in three passes (hi hi + hi lo + lo
// hi) accumulated in FP32 in TMEM, as TF32 hi/lo (kind::tf32, stages of 4 frames)
// or, for FP16X3, as FP16 hi/lo (kind::f16, stages of 8 frames) of operands
// scaled per group and bin by powers of two that keep them below 2^14: x sx,
// y sy, (x sx)(y sy) 2^-14 and z tz, w tw, (z tz)(w tw) 2^-14, with the scales
// written by K1; the epilogue undoes them one power of two at a time.  Sxy and
// Szw depend on one bin each and are summed, unscaled, by the threads that build
// the operands.
//
// Building the operands is the limit: an M = 128, N <= 128 product reads its
// operands from shared memory at about 120 bytes per clock, so the tile is as
// wide as two TMEM buffers allow, and the builders' staging reads and operand
// stores are kept to one pass each, free of bank conflicts.
//
// Grid: one persistent CTA per SM (all 512 TMEM columns).  Items (group chunk,
// combination, tile) come from a group-major queue.  Warp roles, coupled only by
// mbarriers:
// - warp 17 takes the items and, per stage, stages the coefficients the tile
//   needs with four 2-D tensor-map boxes (the stage's frame rows of a and of b
//   over the bins |k| of the tile's rows, at most 131 consecutive bins from a
//   multiple of 4; of c and of d over its 24 bins) into a ring, with the stage's
//   record; FP16: with a group's first stage also the bins' row scales;
// - warps 8-15 build each stage from them: the hi and lo parts of x, y, xy for
//   the tile's 128 rows (a thread: one row, half the stage's frames) and of the
//   [z | w] and zw columns (144 tasks of one operand, one bin and half the
//   frames, writing its Re and Im columns), in the K-major core-matrix layout of
//   the MMA descriptors (no copy of the operands exists in HBM), plus the group's
//   Sxy, Szw, scales and record in a ring of slots;
// - warp 16 issues, per stage, the nine MMAs (3 products x 3 passes) into the
//   group's TMEM buffer (two buffers of 240 columns, alternating by group), and
//   commits the stage (free again) and, after the group's last stage, the buffer;
// - warps 0-7 (TMEM lane quadrant warp % 4, 12 of the 24 columns each) read the
//   buffer, form c4 and keep each point's sums of Re, Im, Re^2 and Im^2 over the
//   item's groups in registers; at the end of an item they add them to the
//   float64 accumulators.
// Rows: r = k + M - 1 in [1, 2M - 2] (k from -(M - 2) to M - 1).  The row r = 0
// (k = -(M - 1)) equals the row r = 2M - 2: for a real signal the Nyquist
// coefficient X(M - 1) is real, so x, y at k = -(M - 1) are those at k = M - 1;
// a small kernel copies that row's sums after every batch.  Every wait is
// bounded; on a failure the CTA stops, waits for the copies and products it
// issued and frees its TMEM.
#include <cuda_fp16.h>

#include "internal.cuh"
#include "pipeline.cuh"

namespace ss {
namespace {

constexpr int kXT = 128;     // rows of a tile
constexpr int kXL = kCrossTileCols;  // columns of a tile (24)
constexpr int kXLw = kXL / 2;        // columns of an epilogue warp
constexpr int kXEpiWarps = 8, kXBuildWarps = 8;
constexpr int kXMmaWarp = kXEpiWarps + kXBuildWarps, kXLoadWarp = kXMmaWarp + 1;
constexpr int kXThreads = 32 * (kXLoadWarp + 1);
constexpr int kXSlots = 4;
constexpr uint32_t kXTmemCols = 512;
// TMEM buffer b starts at column 256 b: 24 columns (one per l) each of Re Sxz,
// Im Sxz, Re Sxw, Im Sxw, then of Re Syz, Im Syz, Re Syw, Im Syw at +96, then of
// Re P, Im P at +192 (the B rows are ordered the same way: type-major)
constexpr uint32_t kXBufCols = 256, kColY = 4 * kXL, kColP = 8 * kXL;

// A stage: for each matrix a hi block, then a lo block.  A matrix of R rows and
// 32 bytes of K per row is R/8 row groups of two core matrices (8 rows x 16
// bytes: the first and the second half of the stage's frames, Re and Im), 128
// bytes apart (LBO); row groups are 256 bytes apart (SBO).  TF32: 4 frames per
// stage (K = 8); FP16: 8 frames (K = 16).
constexpr uint32_t kAMat = kXT * 32;                      // 4 KB
constexpr uint32_t kBXYMat = 4 * kXL * 32, kBPMat = 2 * kXL * 32;
constexpr uint32_t kOffAX = 0, kOffAY = 2 * kAMat, kOffAP = 4 * kAMat;
constexpr uint32_t kOffBXY = 6 * kAMat, kOffBP = kOffBXY + 2 * kBXYMat;
constexpr uint32_t kXStageBytes = kOffBP + 2 * kBPMat;    // 33 KB

// Operand formats.  TF32 hi/lo of the values; FP16 hi/lo of the values scaled
// by a power of two per row (bin and operand) that keeps them below 2^14.
// A stage of staged coefficients holds kF frames: the bins of a and b that the
// tile's rows need (at most 131 consecutive bins from a bin that is a multiple
// of 4; boxes of kF rows x min(kRawK, Mp) bins, rows rawk bins apart), then the
// 24 bins of c and d (boxes of kF rows x kColBox bins) and, for FP16, the
// group's row scales of each of those bins (boxes of one row).  The box widths
// put the rows of a thread's two frame chunks (kHalf frames apart) 64 bytes
// apart modulo 128: on other banks.
template <bool kF16>
struct XFmt {
  static constexpr int kF = kF16 ? 8 : 4;           // frames per stage
  static constexpr int kHalf = kF / 2;              // frames per 16-byte chunk of a row
  static constexpr int kStages = kF16 ? 3 : 4;      // operand stages
  static constexpr int kRaw = kF16 ? 4 : 6;         // staged-coefficient stages
  static constexpr int kRawK = kF16 ? kCrossBoxBinsH : kCrossBoxBins;
  static constexpr int kColBox = kF16 ? kCrossColBoxH : kCrossColBox;
  static constexpr uint32_t kRawA = 0, kRawB = kF * kRawK * 8, kRawC = 2 * kF * kRawK * 8,
                            kRawD = kRawC + kF * kColBox * 8, kRawEnd = kRawD + kF * kColBox * 8;
  static constexpr uint32_t kRawSA = kRawEnd, kRawSB = kRawSA + 640, kRawSC = kRawSB + 640,
                            kRawSD = kRawSC + 128;
  static constexpr uint32_t kRawBytes = kF16 ? kRawSD + 128 : kRawEnd;
  static constexpr size_t kSmem = (size_t)kStages * kXStageBytes + (size_t)kRaw * kRawBytes + 128;
};
static_assert(XFmt<false>::kRawBytes % 128 == 0 && XFmt<true>::kRawBytes % 128 == 0 &&
                  XFmt<true>::kRawSA % 128 == 0 && XFmt<true>::kRawSB % 128 == 0 &&
                  XFmt<true>::kRawSC % 128 == 0 && XFmt<true>::kRawSD % 128 == 0,
              "staging regions start on 128-byte boundaries");
static_assert(XFmt<false>::kSmem <= 227 * 1024 - 12 * 1024 && XFmt<true>::kSmem <= 227 * 1024 - 12 * 1024,
              "shared memory");

enum : int { kRecFirst = 1, kRecLast = 2, kRecStop = 4, kRecItemEnd = 8 };

struct StageRec {
  int flags;
};

struct RawRec {  // a staged stage: its tile, combination, first staged bin, frames
  int r0, l0, combo, bstart, st, flags;
};

struct CrossSlot {  // one group: its one-bin sums, scales and record, for the epilogue
  float2 sxy[kXT];
  float2 szw[2][kXL];   // over the first and the second half of each stage's frames
  float2 rxy[kXT];      // FP16: 1 / (row scales of x and y)
  float2 rzw[kXL];      // FP16: 1 / (column scales of z and w)
  int r0, l0, combo, flags;
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t t;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
  return t;
}

// hi and lo TF32 parts of four values into the hi and lo blocks at byte `off`
__device__ __forceinline__ void put_split(unsigned char* blk, uint32_t lo_off, uint32_t off, float a,
                                          float b, float c, float d) {
  uint4 h, l;
  h.x = to_tf32(a);
  h.y = to_tf32(b);
  h.z = to_tf32(c);
  h.w = to_tf32(d);
  l.x = to_tf32(a - __uint_as_float(h.x));
  l.y = to_tf32(b - __uint_as_float(h.y));
  l.z = to_tf32(c - __uint_as_float(h.z));
  l.w = to_tf32(d - __uint_as_float(h.w));
  *reinterpret_cast<uint4*>(blk + off) = h;
  *reinterpret_cast<uint4*>(blk + lo_off + off) = l;
}

// hi and lo FP16 parts of eight values (two at a time, each rounded to nearest)
__device__ __forceinline__ void put_split16(unsigned char* blk, uint32_t lo_off, uint32_t off,
                                            const float (&v)[8]) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const __half2 hh = __floats2half2_rn(v[2 * t], v[2 * t + 1]);
    const float2 hf = __half22float2(hh);
    const __half2 ll = __floats2half2_rn(v[2 * t] - hf.x, v[2 * t + 1] - hf.y);
    h[t] = *reinterpret_cast<const uint32_t*>(&hh);
    l[t] = *reinterpret_cast<const uint32_t*>(&ll);
  }
  *reinterpret_cast<uint4*>(blk + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(blk + lo_off + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// 1 / s for a normal power of two s (exact): the exponent field mirrored
__device__ __forceinline__ float pow2_inv(float s) {
  return __int_as_float((254 << 23) - __float_as_int(s));
}

// byte offset of row n's 16-byte chunk c in a matrix block
__device__ __forceinline__ uint32_t core_off(int n, int c) {
  return (uint32_t)((n >> 3) * 256 + c * 128 + (n & 7) * 16);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void cmacf(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

__device__ __forceinline__ uint64_t smem_desc_x(uint32_t addr) {
  // K-major, no swizzle: LBO 128 bytes, SBO 256 bytes
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(256u >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)accumulate));
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)accumulate));
}

__device__ __forceinline__ void mma_commit_x(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float (&v)[2]) {
  uint32_t r[2];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(taddr));
  v[0] = __uint_as_float(r[0]);
  v[1] = __uint_as_float(r[1]);
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_x(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

struct CrossQueue {
  int* counter;
  int n_items, n_tiles, n_combos, n_cb, group_chunk;
};

template <bool kF16>
__global__ void __launch_bounds__(kXThreads, 1)
k3_trispec_cross_tc(const __grid_constant__ CUtensorMap tm_ab,
                    const __grid_constant__ CUtensorMap tm_cd,
                    const __grid_constant__ CUtensorMap tm_sab,
                    const __grid_constant__ CUtensorMap tm_scd, int chan_rows, int grp_rows,
                    int rawk, int sabk, int G, int m, int M, int Mp,
                    const int4* __restrict__ combos, CrossQueue wq, float pref, float fmm,
                    float fm1, double* __restrict__ acc, long long plane, long long combo_stride,
                    int* __restrict__ status) {
  using F = XFmt<kF16>;
  constexpr int kSt = F::kStages, kRw = F::kRaw, kH = F::kHalf;
  constexpr float kPairScale = 1.f / 16384.f;  // FP16: products of two scaled values x 2^-14
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kSt];           // stage built
  __shared__ __align__(8) uint64_t sdone[kSt];          // stage's products complete
  __shared__ __align__(8) uint64_t slotfull[kXSlots];   // group slot written
  __shared__ __align__(8) uint64_t slotempty[kXSlots];  // group slot read by the epilogue
  __shared__ __align__(8) uint64_t bfull[2];            // TMEM buffer holds a finished group
  __shared__ __align__(8) uint64_t bempty[2];           // TMEM buffer read by the epilogue
  __shared__ __align__(8) uint64_t rfull[kRw];          // coefficients staged (tensor copies)
  __shared__ __align__(8) uint64_t rempty[kRw];         // staged coefficients read
  __shared__ StageRec srec[kSt];
  __shared__ RawRec rrec[kRw];
  __shared__ __align__(16) CrossSlot slot[kXSlots];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* stages =
      smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);  // 128-byte aligned

  if (tid == 0) {
    for (int s = 0; s < kSt; ++s) {
      mbar_init(&full[s], kXBuildWarps);
      mbar_init(&sdone[s], 1);
    }
    for (int p = 0; p < kXSlots; ++p) {
      mbar_init(&slotfull[p], kXBuildWarps);
      mbar_init(&slotempty[p], kXEpiWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bfull[b], 1);
      mbar_init(&bempty[b], kXEpiWarps);
    }
    for (int i = 0; i < kRw; ++i) {
      mbar_init(&rfull[i], 1);
      mbar_init(&rempty[i], kXBuildWarps);
    }
    s_fail = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kXTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t taddr = tmem_slot;
  const int rows_hi = 2 * M - 2;  // last row r of the tiles
  const int nst = (m + F::kF - 1) / F::kF;

  unsigned char* raws = stages + (size_t)kSt * kXStageBytes;
  if (warp >= kXEpiWarps && warp < kXMmaWarp) {
    // ------------------------------------------------------------ builders
    // Builder warp wb, lane: row R = 16 wb + lane % 8 + 8 (lane / 16) of the tile,
    // the first or second half of every stage's frames, fp = lane / 8 % 2 (one
    // 16-byte chunk of the row), so that 8 consecutive lanes fill one 128-byte core
    // matrix.  The column rows: 3 operands (z, w, zw) x 24 bins x 2 chunks = 144
    // tasks, thread bt < 144 taking task bt: operand bt / 48, chunk bt / 24 % 2, bin
    // bt % 24; a task writes the operand's Re and Im columns (8 consecutive tasks
    // fill one core matrix).  Each warp waits and arrives on its own.
    constexpr int kTasks = 3 * 2 * kXL;
    const int bt = tid - 32 * kXEpiWarps, wb = bt >> 5;
    const int R = 16 * wb + (lane & 7) + 8 * (lane >> 4), fp = (lane >> 3) & 1;
    const int top = bt < kTasks ? bt / (2 * kXL) : -1;  // 0: z, 1: w, 2: zw; -1: none
    const int tli = bt % kXL, tfq = (bt / kXL) & 1;
    const float2 zero = make_float2(0.f, 0.f);
    uint32_t rq = 0, q = 0, gs = 0;
    bool ok = true;
    float2 sxy = zero, szw = zero;  // szw: the zw task, if any
    // FP16: the current group's scales of this thread's row (x, y) and column (z, w)
    float sx = 1.f, sy = 1.f, tz = 1.f, tw = 1.f;
    for (;;) {
      const int rs = (int)(rq % kRw);
      ok = __all_sync(0xffffffffu, mbar_wait_bounded(&rfull[rs], (rq / kRw) & 1u, status));
      if (!ok) break;
      const RawRec rec = rrec[rs];
      if (rec.flags & kRecStop) break;
      const int r = rec.r0 + R, k = r - (M - 1);
      const bool rv = r <= rows_hi;
      const int kb = k < 0 ? -k : k;
      const int j0 = rec.st * F::kF;  // first frame of the stage
      const unsigned char* rbase = raws + (size_t)rs * F::kRawBytes;
      const float2* raw = reinterpret_cast<const float2*>(rbase);
      float2 va[kH], vb[kH], vc[kH], vd[kH];
      const bool lv = top >= 0 && rec.l0 + tli < M;
#pragma unroll
      for (int jj = 0; jj < kH; ++jj) {
        const int fj = kH * fp + jj;  // frame within the stage
        const bool v = rv && j0 + fj < m;
        va[jj] = v ? raw[F::kRawA / 8 + fj * rawk + kb - rec.bstart] : zero;
        vb[jj] = v ? raw[F::kRawB / 8 + fj * rawk + kb - rec.bstart] : zero;
        const int fk = kH * tfq + jj;
        const bool w = lv && j0 + fk < m;
        vc[jj] = w && top != 1 ? raw[F::kRawC / 8 + fk * F::kColBox + tli] : zero;
        vd[jj] = w && top != 0 ? raw[F::kRawD / 8 + fk * F::kColBox + tli] : zero;
      }
      if constexpr (kF16) {
        if (rec.flags & kRecFirst) {  // the group's row scales, staged with its first stage
          const float* ssc = reinterpret_cast<const float*>(rbase);
          sx = rv ? ssc[F::kRawSA / 4 + kb - rec.bstart] : 1.f;
          sy = rv ? ssc[F::kRawSB / 4 + kb - rec.bstart] : 1.f;
          tz = lv ? ssc[F::kRawSC / 4 + tli] : 1.f;
          tw = lv ? ssc[F::kRawSD / 4 + tli] : 1.f;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive_x(&rempty[rs]);  // the warp's coefficients are in registers
      ++rq;
      const int s = (int)(q % kSt);
      ok = __all_sync(0xffffffffu,
                      q < (uint32_t)kSt ||
                          mbar_wait_bounded(&sdone[s], ((q / kSt) & 1u) ^ 1u, status));
      if (!ok) break;
      if (rec.flags & kRecFirst) sxy = szw = zero;
      unsigned char* stg = stages + (size_t)s * kXStageBytes;
      // rows: k < 0: x = a_{|k|}*, y = b_{|k|};  k >= 0: x = a_k, y = b_k*
      float2 x[kH], y[kH], xy[kH];
#pragma unroll
      for (int jj = 0; jj < kH; ++jj) {
        x[jj] = k < 0 ? make_float2(va[jj].x, -va[jj].y) : va[jj];
        y[jj] = k < 0 ? vb[jj] : make_float2(vb[jj].x, -vb[jj].y);
        xy[jj] = cmulf(x[jj], y[jj]);
        sxy.x += xy[jj].x;
        sxy.y += xy[jj].y;
      }
      const uint32_t o = core_off(R, fp);
      if constexpr (!kF16) {
        put_split(stg + kOffAX, kAMat, o, x[0].x, x[0].y, x[1].x, x[1].y);
        put_split(stg + kOffAY, kAMat, o, y[0].x, y[0].y, y[1].x, y[1].y);
        put_split(stg + kOffAP, kAMat, o, xy[0].x, xy[0].y, xy[1].x, xy[1].y);
      } else {
        // scaled rows: x sx, y sy and (x sx)(y sy) 2^-14, each below 2^14
        float ex[8], ey[8], ep[8];
#pragma unroll
        for (int jj = 0; jj < kH; ++jj) {
          const float2 xs = make_float2(x[jj].x * sx, x[jj].y * sx);
          const float2 ys = make_float2(y[jj].x * sy, y[jj].y * sy);
          const float2 ps = cmulf(xs, ys);
          ex[2 * jj] = xs.x;
          ex[2 * jj + 1] = xs.y;
          ey[2 * jj] = ys.x;
          ey[2 * jj + 1] = ys.y;
          ep[2 * jj] = ps.x * kPairScale;
          ep[2 * jj + 1] = ps.y * kPairScale;
        }
        put_split16(stg + kOffAX, kAMat, o, ex);
        put_split16(stg + kOffAY, kAMat, o, ey);
        put_split16(stg + kOffAP, kAMat, o, ep);
      }
      if (top >= 0) {
        // operand top of bin l: z = c_l, w = d_l*, zw; its Re column (ur, -ui) and
        // its Im column (ui, ur)
        float2 v[kH];
#pragma unroll
        for (int jj = 0; jj < kH; ++jj) {
          float2 z = vc[jj], w = make_float2(vd[jj].x, -vd[jj].y);
          if (top == 2) {
            const float2 zw = cmulf(z, w);
            szw.x += zw.x;
            szw.y += zw.y;
          }
          if constexpr (kF16) {
            z = make_float2(z.x * tz, z.y * tz);
            w = make_float2(w.x * tw, w.y * tw);
            const float2 zws = cmulf(z, w);
            v[jj] = top == 0 ? z
                             : (top == 1 ? w : make_float2(zws.x * kPairScale, zws.y * kPairScale));
          } else {
            v[jj] = top == 0 ? z : (top == 1 ? w : cmulf(z, w));
          }
        }
        const uint32_t cre = top < 2 ? kOffBXY + core_off(kXL * (2 * top) + tli, tfq)
                                     : kOffBP + core_off(tli, tfq);
        const uint32_t cim = top < 2 ? kOffBXY + core_off(kXL * (2 * top + 1) + tli, tfq)
                                     : kOffBP + core_off(kXL + tli, tfq);
        const uint32_t lo = top < 2 ? kBXYMat : kBPMat;
        if constexpr (!kF16) {
          put_split(stg, lo, cre, v[0].x, -v[0].y, v[1].x, -v[1].y);
          put_split(stg, lo, cim, v[0].y, v[0].x, v[1].y, v[1].x);
        } else {
          float er[8], ei[8];
#pragma unroll
          for (int jj = 0; jj < kH; ++jj) {
            er[2 * jj] = v[jj].x;
            er[2 * jj + 1] = -v[jj].y;
            ei[2 * jj] = v[jj].y;
            ei[2 * jj + 1] = v[jj].x;
          }
          put_split16(stg, lo, cre, er);
          put_split16(stg, lo, cim, ei);
        }
      }
      if (bt == 0) srec[s] = StageRec{rec.flags & (kRecFirst | kRecLast)};
      // the generic-proxy writes become visible to the tensor cores' reads
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive_x(&full[s]);
      ++q;
      if (rec.flags & kRecLast) {
        // the group's one-bin sums (the two chunks of a row are lanes 8 apart; the
        // column sums go per chunk), its scales and its record, for the epilogue
        const float2 sxy_o = make_float2(__shfl_xor_sync(0xffffffffu, sxy.x, 8),
                                         __shfl_xor_sync(0xffffffffu, sxy.y, 8));
        const int p = (int)(gs % kXSlots);
        ok = __all_sync(0xffffffffu, gs < (uint32_t)kXSlots ||
                                         mbar_wait_bounded(&slotempty[p],
                                                           ((gs / kXSlots) - 1) & 1u, status));
        if (!ok) break;
        if (fp == 0) slot[p].sxy[R] = make_float2(sxy.x + sxy_o.x, sxy.y + sxy_o.y);
        if (top == 2) slot[p].szw[tfq][tli] = szw;
        if constexpr (kF16) {
          if (fp == 0) slot[p].rxy[R] = make_float2(pow2_inv(sx), pow2_inv(sy));
          if (top == 2 && tfq == 0) slot[p].rzw[tli] = make_float2(pow2_inv(tz), pow2_inv(tw));
        }
        if (bt == 0) {
          slot[p].r0 = rec.r0;
          slot[p].l0 = rec.l0;
          slot[p].combo = rec.combo;
          slot[p].flags = rec.flags & kRecItemEnd;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_x(&slotfull[p]);
        ++gs;
      }
    }
    if (!ok && lane == 0) atomicExch(&s_fail, 1);
    // stop records: the next stage (for the MMA warp) and the next slot (epilogue)
    {
      const int s = (int)(q % kSt);
      if (q >= (uint32_t)kSt) mbar_wait_bounded(&sdone[s], ((q / kSt) & 1u) ^ 1u, status);
      if (bt == 0) srec[s] = StageRec{kRecStop};
      __syncwarp();
      if (lane == 0) mbar_arrive_x(&full[s]);
      const int p = (int)(gs % kXSlots);
      if (gs >= (uint32_t)kXSlots)
        mbar_wait_bounded(&slotempty[p], ((gs / kXSlots) - 1) & 1u, status);
      if (bt == 0) slot[p].flags = kRecStop;
      __syncwarp();
      if (lane == 0) mbar_arrive_x(&slotfull[p]);
    }
  } else if (warp == kXMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t sbase = smem_addr(stages);
      // D FP32; A, B TF32 (format 2) or FP16 (format 0 of kind::f16); K-major
      const uint32_t fmt = kF16 ? 0u : ((2u << 7) | (2u << 10));
      const uint32_t idesc0 = (1u << 4) | fmt | ((uint32_t)(kXT >> 4) << 24);
      uint32_t q = 0, gc = 0;
      int last_s = -1;
      uint32_t last_ph = 0;
      for (;; ++q) {
        const int s = (int)(q % kSt);
        const uint32_t ph = (q / kSt) & 1u;
        if (!mbar_wait_bounded(&full[s], ph, status)) break;
        const StageRec rec = srec[s];
        if (rec.flags & kRecStop) break;
        const uint32_t b = gc & 1u;
        if (rec.flags & kRecFirst) {
          // the buffer is free once the epilogue has read the group two before
          if (gc >= 2 && !mbar_wait_bounded(&bempty[b], ((gc >> 1) - 1) & 1u, status)) break;
          tc_after();
        }
        const uint32_t d = taddr + b * kXBufCols;
        // N = 96 ([z | w] columns) and 48 (zw), whatever the tile's width (columns
        // of bins past M - 1 are zero)
        const uint32_t idx = idesc0 | ((uint32_t)((4 * kXL) >> 3) << 17);
        const uint32_t idp = idesc0 | ((uint32_t)((2 * kXL) >> 3) << 17);
        const uint32_t sa = sbase + (uint32_t)s * kXStageBytes;
        const bool first = (rec.flags & kRecFirst) != 0;
#pragma unroll
        for (int pa = 0; pa < 3; ++pa) {
          // passes hi*hi, hi*lo, lo*hi
          const uint32_t ao = pa == 2 ? kAMat : 0u;
          const uint32_t bxo = pa == 1 ? kBXYMat : 0u, bpo = pa == 1 ? kBPMat : 0u;
          const bool accum = !(first && pa == 0);
          const uint64_t ax = smem_desc_x(sa + kOffAX + ao), ay = smem_desc_x(sa + kOffAY + ao);
          const uint64_t ap = smem_desc_x(sa + kOffAP + ao);
          const uint64_t bxy = smem_desc_x(sa + kOffBXY + bxo), bp = smem_desc_x(sa + kOffBP + bpo);
          if constexpr (kF16) {
            mma_f16(d, ax, bxy, idx, accum);
            mma_f16(d + kColY, ay, bxy, idx, accum);
            mma_f16(d + kColP, ap, bp, idp, accum);
          } else {
            mma_tf32(d, ax, bxy, idx, accum);
            mma_tf32(d + kColY, ay, bxy, idx, accum);
            mma_tf32(d + kColP, ap, bp, idp, accum);
          }
        }
        mma_commit_x(&sdone[s]);
        last_s = s;
        last_ph = ph;
        if (rec.flags & kRecLast) {
          mma_commit_x(&bfull[b]);
          ++gc;
        }
      }
      if (*(volatile int*)status != 0) atomicExch(&s_fail, 1);
      // the products issued must be complete before the TMEM is freed
      if (last_s >= 0) mbar_wait_bounded(&sdone[last_s], last_ph, status);
    }
    __syncwarp();
  } else if (warp == kXLoadWarp) {
    // ------------------------------------------------------------ loader
    // takes the items and stages, per stage of kF frames, the coefficients the
    // builders need (tensor-map boxes of whole bin ranges) with the stage's record;
    // FP16: with a group's first stage also the bins' largest |coefficient|^2
    if (lane == 0) {
      uint32_t rq = 0;
      bool ok = true;
      const int per_chunk = wq.n_tiles * wq.n_combos;
      for (;;) {
        const int item = *(volatile int*)&s_fail ? wq.n_items : atomicAdd(wq.counter, 1);
        if (item >= wq.n_items) break;
        const int chunk = item / per_chunk, rest = item - chunk * per_chunk;
        const int combo = rest / wq.n_tiles, tile = rest - combo * wq.n_tiles;
        const int r0 = 1 + (tile / wq.n_cb) * kXT, l0 = (tile % wq.n_cb) * kXL;
        const int g0 = chunk * wq.group_chunk, g1 = min(G, g0 + wq.group_chunk);
        const int4 cb = combos[combo];
        // bins |k| of the tile's rows: one range of at most 128 bins, staged from a
        // multiple of 4 (x times 8 bytes, and times 4 for the maxima, a multiple of
        // 16: the boxes' alignment rule)
        const int klo = r0 - (M - 1), khi = min(r0 + kXT - 1, rows_hi) - (M - 1);
        const int blo = klo >= 0 ? klo : (khi <= 0 ? -khi : 0);
        const int bstart = blo & ~3;
        const uint32_t stage_bytes = 2u * (uint32_t)F::kF * 8u * (uint32_t)(rawk + F::kColBox);
        const uint32_t scale_bytes = kF16 ? 2u * 4u * (uint32_t)(sabk + kCrossScaleCols) : 0u;
        for (int g = g0; g < g1 && ok; ++g) {
          for (int st = 0; st < nst; ++st) {
            const int rs = (int)(rq % kRw);
            if (rq >= (uint32_t)kRw &&
                !mbar_wait_bounded(&rempty[rs], ((rq / kRw) - 1) & 1u, status)) {
              ok = false;
              break;
            }
            const int last = st == nst - 1;
            rrec[rs] = RawRec{r0, l0, combo, bstart, st,
                              (st == 0 ? kRecFirst : 0) | (last ? kRecLast : 0) |
                                  (last && g == g1 - 1 ? kRecItemEnd : 0)};
            unsigned char* dst = raws + (size_t)rs * F::kRawBytes;
            // kF frame rows of each channel (rows past the group's m frames are not
            // used; rows and bins past the spectra read as zeros)
            const int fr = g * m + st * F::kF;
            mbar_arrive_expect_tx(&rfull[rs], stage_bytes + (st == 0 ? scale_bytes : 0u));
            tma_load_2d(dst + F::kRawA, &tm_ab, bstart, cb.x * chan_rows + fr, &rfull[rs]);
            tma_load_2d(dst + F::kRawB, &tm_ab, bstart, cb.y * chan_rows + fr, &rfull[rs]);
            tma_load_2d(dst + F::kRawC, &tm_cd, l0, cb.z * chan_rows + fr, &rfull[rs]);
            tma_load_2d(dst + F::kRawD, &tm_cd, l0, cb.w * chan_rows + fr, &rfull[rs]);
            if (kF16 && st == 0) {
              tma_load_2d(dst + F::kRawSA, &tm_sab, bstart, cb.x * grp_rows + g, &rfull[rs]);
              tma_load_2d(dst + F::kRawSB, &tm_sab, bstart, cb.y * grp_rows + g, &rfull[rs]);
              tma_load_2d(dst + F::kRawSC, &tm_scd, l0, cb.z * grp_rows + g, &rfull[rs]);
              tma_load_2d(dst + F::kRawSD, &tm_scd, l0, cb.w * grp_rows + g, &rfull[rs]);
            }
            ++rq;
          }
        }
        if (!ok) break;
      }
      if (!ok) atomicExch(&s_fail, 1);
      // every copy issued has landed before the CTA may exit (waited before the stop
      // record moves the barrier to its next phase)
      for (uint32_t i = rq > (uint32_t)kRw ? rq - kRw : 0; i < rq; ++i)
        mbar_wait_bounded(&rfull[i % kRw], (i / kRw) & 1u, status);
      const int rs = (int)(rq % kRw);
      if (rq >= (uint32_t)kRw) mbar_wait_bounded(&rempty[rs], ((rq / kRw) - 1) & 1u, status);
      rrec[rs].flags = kRecStop;
      asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(
                       smem_addr(&rfull[rs]))
                   : "memory");
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int qd = warp & 3, h = warp >> 2;
    const int R = 32 * qd + lane;
    const uint32_t lane_addr = taddr + ((uint32_t)(32 * qd) << 16);
    // FP16: P' carries the two factors 2^-14 of the scaled products xy and zw
    const float fmm_p = kF16 ? fmm * 268435456.f : fmm;  // 2^28
    float sre[kXLw], sim[kXLw], qre[kXLw], qim[kXLw];
#pragma unroll
    for (int i = 0; i < kXLw; ++i) sre[i] = sim[i] = qre[i] = qim[i] = 0.f;
    for (uint32_t gc = 0;; ++gc) {
      const int p = (int)(gc % kXSlots);
      const uint32_t b = gc & 1u;
      // one decision per warp: the TMEM accesses below are warp-collective
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&slotfull[p], (gc / kXSlots) & 1u, status))) {
        if (lane == 0) atomicExch(&s_fail, 1);
        break;
      }
      const int flags = slot[p].flags;
      if (flags & kRecStop) break;
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bfull[b], (gc >> 1) & 1u, status))) {
        if (lane == 0) atomicExch(&s_fail, 1);
        break;
      }
      tc_after();
      // the whole record is read before the slot is released below
      const int l0 = slot[p].l0, r0 = slot[p].r0, combo = slot[p].combo;
      const float2 sxy = slot[p].sxy[R];
      const float2 rxy = kF16 ? slot[p].rxy[R] : make_float2(1.f, 1.f);
      const uint32_t tb = lane_addr + b * kXBufCols;
#pragma unroll
      for (int hh = 0; hh < kXLw / 2; ++hh) {
        const int li0 = kXLw * h + 2 * hh;
        if (l0 + li0 < M) {  // warp-uniform
          // columns li0, li0 + 1 of each of the ten product types
          float d[10][2];
#pragma unroll
          for (int t = 0; t < 10; ++t) tmem_ld2(tb + kXL * t + li0, d[t]);
          tc_wait_ld();
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const float2 szw = make_float2(slot[p].szw[0][li0 + i].x + slot[p].szw[1][li0 + i].x,
                                           slot[p].szw[0][li0 + i].y + slot[p].szw[1][li0 + i].y);
            const float2 xz = make_float2(d[0][i], d[1][i]), xw = make_float2(d[2][i], d[3][i]);
            const float2 yz = make_float2(d[4][i], d[5][i]), yw = make_float2(d[6][i], d[7][i]);
            float cr, ci;
            if constexpr (kF16) {
              // the scaled products: [fmm P - fm1 (Sxz Syw + Sxw Syz)] sx sy tz tw, undone
              // one power of two at a time (their product alone may leave the float
              // range); Sxy Szw is unscaled
              float2 t = cmulf(xz, yw);
              cmacf(t, xw, yz);
              const float2 rzw = slot[p].rzw[li0 + i];
              float ur = fmaf(fmm_p, d[8][i], -fm1 * t.x), ui = fmaf(fmm_p, d[9][i], -fm1 * t.y);
              ur = ur * rxy.x * rxy.y * rzw.x * rzw.y;
              ui = ui * rxy.x * rxy.y * rzw.x * rzw.y;
              const float2 u = cmulf(sxy, szw);
              cr = pref * fmaf(-fm1, u.x, ur);
              ci = pref * fmaf(-fm1, u.y, ui);
            } else {
              float2 t = cmulf(sxy, szw);
              cmacf(t, xz, yw);
              cmacf(t, xw, yz);
              cr = pref * fmaf(fmm_p, d[8][i], -fm1 * t.x);
              ci = pref * fmaf(fmm_p, d[9][i], -fm1 * t.y);
            }
            const int e = 2 * hh + i;
            sre[e] += cr;
            sim[e] += ci;
            qre[e] = fmaf(cr, cr, qre[e]);
            qim[e] = fmaf(ci, ci, qim[e]);
          }
        }
      }
      // this warp has read its part of the buffer and of the slot
      tc_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive_x(&bempty[b]);
        mbar_arrive_x(&slotempty[p]);
      }
      if (flags & kRecItemEnd) {
        const int r = r0 + R;
        const long long cbase = (long long)combo * combo_stride;
#pragma unroll
        for (int e = 0; e < kXLw; ++e) {
          const int lc = l0 + kXLw * h + e;
          if (r <= rows_hi && lc < M) {
            const long long o = cbase + (long long)r * M + lc;
            atomicAdd(acc + o, (double)sre[e]);
            atomicAdd(acc + plane + o, (double)sim[e]);
            atomicAdd(acc + 2 * plane + o, (double)qre[e]);
            atomicAdd(acc + 3 * plane + o, (double)qim[e]);
          }
          sre[e] = sim[e] = qre[e] = qim[e] = 0.f;
        }
      }
    }
  }
  tc_before();
  __syncthreads();
  if (warp == 0) {
    tc_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr),
                 "r"(kXTmemCols));
  }
}

// row r = 0 (k = -(M - 1)) of every plane and combination <- row r = 2M - 2
__global__ void k3_cross_row0(double* __restrict__ acc, int n, int M, long long combo_stride,
                              long long plane) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int l = i % M, pc = i / M;
  const int c = pc >> 2, pl = pc & 3;
  double* a = acc + pl * plane + (long long)c * combo_stride;
  a[l] = a[(long long)(2 * M - 2) * M + l];
}

}  // namespace

cudaError_t launch_k3_trispec_cross_tc(const CrossViews& v, int G, int m, int M, int Mp,
                                       const int4* combos, int n_combos, double* acc,
                                       long long plane, int nsm, bool natural, int* counter,
                                       int* status, cudaStream_t stream) {
  if (G <= 0 || n_combos <= 0) return cudaSuccess;
  if (m < 1 || M < 2 || nsm <= 0 || (Mp & 15) || Mp < M) return cudaErrorInvalidValue;
  if (v.f16 && (!v.tm_sab || !v.tm_scd)) return cudaErrorInvalidValue;
  const int n_rb = (2 * M - 2 + kXT - 1) / kXT, n_cb = (M + kXL - 1) / kXL;
  const long long n_tiles = (long long)n_rb * n_cb;
  CrossQueue wq;
  wq.counter = counter;
  wq.n_tiles = (int)n_tiles;
  wq.n_combos = n_combos;
  wq.n_cb = n_cb;
  wq.group_chunk = work_group_chunk(G, (int)std::min<long long>(n_tiles * n_combos, 1 << 30), nsm);
  const long long n_chunks = (G + wq.group_chunk - 1) / wq.group_chunk;
  const long long n_items = n_chunks * n_tiles * n_combos;
  if (n_items > 0x7fffffffll) return cudaErrorInvalidValue;
  wq.n_items = (int)n_items;
  auto kern = v.f16 ? k3_trispec_cross_tc<true> : k3_trispec_cross_tc<false>;
  const size_t smem = v.f16 ? XFmt<true>::kSmem : XFmt<false>::kSmem;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  const double md = m;
  // c4 = pref [fmm P - fm1 (...)]: the k-statistic (Eq. 85) or the natural estimator
  const float pref =
      (float)(natural ? 1.0 / (md * md) : 1.0 / ((md - 1.0) * (md - 2.0) * (md - 3.0)));
  const float fmm = (float)(natural ? md : md * (md + 1.0));
  const float fm1 = (float)(natural ? 1.0 : md - 1.0);
  const long long combo_stride = (long long)(2 * M - 1) * M;
  const int rawk = std::min(v.f16 ? XFmt<true>::kRawK : XFmt<false>::kRawK, Mp);  // tm_ab's box
  const int sabk = std::min(kCrossScaleBins, Mp);    // the box width of tm_sab
  const CUtensorMap& tsab = v.f16 ? *v.tm_sab : *v.tm_ab;  // not read by the TF32 form
  const CUtensorMap& tscd = v.f16 ? *v.tm_scd : *v.tm_cd;
  kern<<<nsm, kXThreads, smem, stream>>>(*v.tm_ab, *v.tm_cd, tsab, tscd, v.chan_rows, v.grp_rows,
                                         rawk, sabk, G, m, M, Mp, combos, wq, pref, fmm, fm1, acc,
                                         plane, combo_stride, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n = 4 * n_combos * M;
  k3_cross_row0<<<(n + 255) / 256, 256, 0, stream>>>(acc, n, M, combo_stride, plane);
  return cudaGetLastError();
}

}  // namespace ss
