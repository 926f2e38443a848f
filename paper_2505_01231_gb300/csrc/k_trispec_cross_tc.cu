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
// real columns and zw 48.  The products run as TF32 hi/lo splits in three passes
// (hi hi + hi lo + lo hi) accumulated in FP32 in TMEM.  Sxy and Szw depend on one
// bin each and are summed by the threads that build the operands.
//
// The products are bound by shared-memory bandwidth: an M = 128, N <= 128 TF32
// product reads its operands at about 120 bytes per clock, the port's rate, so
// the tile is as wide as two TMEM buffers allow and every other shared-memory
// access (staging, building) is kept to one pass, free of bank conflicts.
//
// Grid: one persistent CTA per SM (all 512 TMEM columns).  Items (group chunk,
// combination, tile) come from a group-major queue.  Warp roles, coupled only by
// mbarriers:
// - warp 17 takes the items and, per stage of 4 frames, stages the coefficients
//   the tile needs with four 2-D tensor-map boxes (4 frame rows of a and of b over
//   the bins |k| of the tile's rows, at most 130 consecutive bins from an even
//   bin; 4 frame rows of c and of d over its 24 bins) into a ring of 6, with the
//   stage's record;
// - warps 8-15 build each stage from them: the TF32 hi and lo parts of x, y, xy
//   for the tile's 128 rows (a thread: one row, two frames) and of the [z | w]
//   and zw columns (288 tasks of one column row and two frames), written to
//   shared memory in the K-major core-matrix layout of the MMA descriptors (no
//   copy of the operands exists in HBM), plus the group's Sxy and Szw and its
//   record in a ring of slots;
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
#include "internal.cuh"
#include "pipeline.cuh"

namespace ss {
namespace {

constexpr int kXT = 128;     // rows of a tile
constexpr int kXL = kCrossTileCols;  // columns of a tile (24)
constexpr int kXLw = kXL / 2;        // columns of an epilogue warp
constexpr int kXF = 4;       // frames per stage: K = 8 TF32 values, one MMA K step
constexpr int kXStages = 4;  // operand stages
constexpr int kXRaw = 6;     // stages of staged coefficients
constexpr int kXEpiWarps = 8, kXBuildWarps = 8;
constexpr int kXMmaWarp = kXEpiWarps + kXBuildWarps, kXLoadWarp = kXMmaWarp + 1;
constexpr int kXThreads = 32 * (kXLoadWarp + 1);
constexpr int kXSlots = 4;
constexpr uint32_t kXTmemCols = 512;
// TMEM buffer b starts at column 256 b: 24 columns (one per l) each of Re Sxz,
// Im Sxz, Re Sxw, Im Sxw, then of Re Syz, Im Syz, Re Syw, Im Syw at +96, then of
// Re P, Im P at +192 (the B rows are ordered the same way: type-major)
constexpr uint32_t kXBufCols = 256, kColY = 4 * kXL, kColP = 8 * kXL;

// A stage: for each matrix a hi block, then a lo block.  A matrix of R rows x 8
// TF32 values is R/8 row groups of two core matrices (8 rows x 16 bytes: frames
// 2c and 2c + 1 of the stage, Re and Im), 128 bytes apart (LBO); row groups are
// 256 bytes apart (SBO).
constexpr uint32_t kAMat = kXT * 32;                      // 4 KB
constexpr uint32_t kBXYMat = 4 * kXL * 32, kBPMat = 2 * kXL * 32;
constexpr uint32_t kOffAX = 0, kOffAY = 2 * kAMat, kOffAP = 4 * kAMat;
constexpr uint32_t kOffBXY = 6 * kAMat, kOffBP = kOffBXY + 2 * kBXYMat;
constexpr uint32_t kXStageBytes = kOffBP + 2 * kBPMat;    // 30 KB
// A stage of staged coefficients (4 frames): the bins of a and b that the tile's
// rows need (at most 130 consecutive bins from an even bin; a box of 4 rows x
// min(kRawK, Mp) bins, rows rawk bins apart), then the 24 bins of c and d of its
// columns (boxes of 4 rows x kCrossColBox bins).
constexpr int kRawK = kCrossBoxBins;
constexpr uint32_t kRawA = 0, kRawB = kXF * kRawK * 8, kRawC = 2 * kXF * kRawK * 8,
                   kRawD = kRawC + kXF * kCrossColBox * 8;
constexpr uint32_t kXRawBytes = kRawD + kXF * kCrossColBox * 8;  // 10.5 KB
constexpr size_t kXSmemBytes =
    (size_t)kXStages * kXStageBytes + (size_t)kXRaw * kXRawBytes + 128;

enum : int { kRecFirst = 1, kRecLast = 2, kRecStop = 4, kRecItemEnd = 8 };

struct StageRec {
  int flags;
};

struct RawRec {  // a staged stage: its tile, combination, first staged bin, frames
  int r0, l0, combo, bstart, st, flags;
};

struct CrossSlot {  // one group: its one-bin sums and record, for the epilogue
  float2 sxy[kXT];
  float2 szw[2][kXL];  // over frames 4i, 4i + 1 and over 4i + 2, 4i + 3
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

__global__ void __launch_bounds__(kXThreads, 1)
k3_trispec_cross_tc(const __grid_constant__ CUtensorMap tm_ab,
                    const __grid_constant__ CUtensorMap tm_cd, int chan_rows, int rawk, int G,
                    int m, int M, int Mp, const int4* __restrict__ combos, CrossQueue wq,
                    float pref, float fmm, float fm1, double* __restrict__ acc, long long plane,
                    long long combo_stride, int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kXStages];      // stage built
  __shared__ __align__(8) uint64_t sdone[kXStages];     // stage's products complete
  __shared__ __align__(8) uint64_t slotfull[kXSlots];   // group slot written
  __shared__ __align__(8) uint64_t slotempty[kXSlots];  // group slot read by the epilogue
  __shared__ __align__(8) uint64_t bfull[2];            // TMEM buffer holds a finished group
  __shared__ __align__(8) uint64_t bempty[2];           // TMEM buffer read by the epilogue
  __shared__ __align__(8) uint64_t rfull[kXRaw];       // coefficients staged (bulk copies)
  __shared__ __align__(8) uint64_t rempty[kXRaw];      // staged coefficients read
  __shared__ StageRec srec[kXStages];
  __shared__ RawRec rrec[kXRaw];
  __shared__ __align__(16) CrossSlot slot[kXSlots];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* stages =
      smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);  // 128-byte aligned

  if (tid == 0) {
    for (int s = 0; s < kXStages; ++s) {
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
    for (int i = 0; i < kXRaw; ++i) {
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
  const int nst = (m + kXF - 1) / kXF;

  unsigned char* raws = stages + (size_t)kXStages * kXStageBytes;
  if (warp >= kXEpiWarps && warp < kXMmaWarp) {
    // ------------------------------------------------------------ builders
    // Builder warp wb, lane: row R = 16 wb + lane % 8 + 8 (lane / 16) of the tile,
    // frames 2 fp and 2 fp + 1 of every stage, fp = lane / 8 % 2 (one 16-byte chunk
    // of the row), so that 8 consecutive lanes fill one 128-byte core matrix.  The
    // column rows are 6 types (Re and Im columns of z, of w, of zw) x 24 bins x 2
    // chunks = 288 tasks: thread bt takes tasks bt and bt + 256, task i being type
    // i / 48, chunk i / 24 % 2, bin i % 24 (8 consecutive tasks fill one core
    // matrix).  Each warp waits and arrives on its own.
    constexpr int kTasks = 6 * 2 * kXL;
    const int bt = tid - 32 * kXEpiWarps, wb = bt >> 5;
    const int R = 16 * wb + (lane & 7) + 8 * (lane >> 4), fp = (lane >> 3) & 1;
    int tt[2], tli[2], tfq[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int i = bt + u * 32 * kXBuildWarps;
      tt[u] = i < kTasks ? i / (2 * kXL) : -1;
      tli[u] = i % kXL;
      tfq[u] = (i / kXL) & 1;
    }
    const float2 zero = make_float2(0.f, 0.f);
    uint32_t rq = 0, q = 0, gs = 0;
    bool ok = true;
    float2 sxy = zero, szw = zero;  // szw: the task of type 4 (Re zw), if any
    for (;;) {
      const int rs = (int)(rq % kXRaw);
      ok = __all_sync(0xffffffffu, mbar_wait_bounded(&rfull[rs], (rq / kXRaw) & 1u, status));
      if (!ok) break;
      const RawRec rec = rrec[rs];
      if (rec.flags & kRecStop) break;
      const int r = rec.r0 + R, k = r - (M - 1);
      const bool rv = r <= rows_hi;
      const int kb = k < 0 ? -k : k;
      const int j0 = rec.st * kXF;  // first frame of the stage
      const float2* raw = reinterpret_cast<const float2*>(raws + (size_t)rs * kXRawBytes);
      float2 va[2], vb[2], vc[2][2], vd[2][2];
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        const int fj = 2 * fp + jj;  // frame within the stage
        const bool v = rv && j0 + fj < m;
        va[jj] = v ? raw[kRawA / 8 + fj * rawk + kb - rec.bstart] : zero;
        vb[jj] = v ? raw[kRawB / 8 + fj * rawk + kb - rec.bstart] : zero;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int fk = 2 * tfq[u] + jj;
          const bool w = tt[u] >= 0 && rec.l0 + tli[u] < M && j0 + fk < m;
          vc[u][jj] = w ? raw[kRawC / 8 + fk * kCrossColBox + tli[u]] : zero;
          vd[u][jj] = w ? raw[kRawD / 8 + fk * kCrossColBox + tli[u]] : zero;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive_x(&rempty[rs]);  // the warp's coefficients are in registers
      ++rq;
      const int s = (int)(q % kXStages);
      ok = __all_sync(0xffffffffu, q < (uint32_t)kXStages ||
                                       mbar_wait_bounded(&sdone[s], ((q / kXStages) & 1u) ^ 1u,
                                                         status));
      if (!ok) break;
      if (rec.flags & kRecFirst) sxy = szw = zero;
      unsigned char* stg = stages + (size_t)s * kXStageBytes;
      // rows: k < 0: x = a_{|k|}*, y = b_{|k|};  k >= 0: x = a_k, y = b_k*
      float2 x[2], y[2], xy[2];
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        x[jj] = k < 0 ? make_float2(va[jj].x, -va[jj].y) : va[jj];
        y[jj] = k < 0 ? vb[jj] : make_float2(vb[jj].x, -vb[jj].y);
        xy[jj] = cmulf(x[jj], y[jj]);
        sxy.x += xy[jj].x;
        sxy.y += xy[jj].y;
      }
      const uint32_t o = core_off(R, fp);
      put_split(stg + kOffAX, kAMat, o, x[0].x, x[0].y, x[1].x, x[1].y);
      put_split(stg + kOffAY, kAMat, o, y[0].x, y[0].y, y[1].x, y[1].y);
      put_split(stg + kOffAP, kAMat, o, xy[0].x, xy[0].y, xy[1].x, xy[1].y);
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int t = tt[u];
        if (t < 0) continue;
        // column row of type t of bin l: z = c_l (t 0, 1), w = d_l* (2, 3), zw (4, 5);
        // an even t gives the Re column (ur, -ui), an odd one the Im column (ui, ur)
        float2 v[2];
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const float2 z = vc[u][jj], w = make_float2(vd[u][jj].x, -vd[u][jj].y);
          const float2 zw = cmulf(z, w);
          if (t == 4) {
            szw.x += zw.x;
            szw.y += zw.y;
          }
          v[jj] = t < 2 ? z : (t < 4 ? w : zw);
        }
        const uint32_t co = t < 4 ? kOffBXY + core_off(kXL * t + tli[u], tfq[u])
                                  : kOffBP + core_off(kXL * (t - 4) + tli[u], tfq[u]);
        const uint32_t lo = t < 4 ? kBXYMat : kBPMat;
        if (t & 1)
          put_split(stg, lo, co, v[0].y, v[0].x, v[1].y, v[1].x);
        else
          put_split(stg, lo, co, v[0].x, -v[0].y, v[1].x, -v[1].y);
      }
      if (bt == 0) srec[s] = StageRec{rec.flags & (kRecFirst | kRecLast)};
      // the generic-proxy writes become visible to the tensor cores' reads
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive_x(&full[s]);
      ++q;
      if (rec.flags & kRecLast) {
        // the group's one-bin sums (the two chunks of a row are lanes 8 apart; the
        // column sums go per chunk) and its record, for the epilogue
        const float2 sxy_o = make_float2(__shfl_xor_sync(0xffffffffu, sxy.x, 8),
                                         __shfl_xor_sync(0xffffffffu, sxy.y, 8));
        const int p = (int)(gs % kXSlots);
        ok = __all_sync(0xffffffffu, gs < (uint32_t)kXSlots ||
                                         mbar_wait_bounded(&slotempty[p],
                                                           ((gs / kXSlots) - 1) & 1u, status));
        if (!ok) break;
        if (fp == 0) slot[p].sxy[R] = make_float2(sxy.x + sxy_o.x, sxy.y + sxy_o.y);
        if (tt[0] == 4) slot[p].szw[tfq[0]][tli[0]] = szw;
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
      const int s = (int)(q % kXStages);
      if (q >= (uint32_t)kXStages)
        mbar_wait_bounded(&sdone[s], ((q / kXStages) & 1u) ^ 1u, status);
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
      const uint32_t idesc0 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kXT >> 4) << 24);
      uint32_t q = 0, gc = 0;
      int last_s = -1;
      uint32_t last_ph = 0;
      for (;; ++q) {
        const int s = (int)(q % kXStages);
        const uint32_t ph = (q / kXStages) & 1u;
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
        // N = 64 ([z | w] columns) and 32 (zw), whatever the tile's width (columns
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
          mma_tf32(d, smem_desc_x(sa + kOffAX + ao), smem_desc_x(sa + kOffBXY + bxo), idx, accum);
          mma_tf32(d + kColY, smem_desc_x(sa + kOffAY + ao), smem_desc_x(sa + kOffBXY + bxo), idx,
                   accum);
          mma_tf32(d + kColP, smem_desc_x(sa + kOffAP + ao), smem_desc_x(sa + kOffBP + bpo), idp,
                   accum);
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
    // takes the items and stages, per 4 frames, the coefficients the builders need
    // (bulk copies of whole bin ranges), with the stage's record
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
        // bins |k| of the tile's rows: one range of at most 128 bins, staged from an
        // even bin (x 8 bytes a multiple of 16: the boxes' alignment rule)
        const int klo = r0 - (M - 1), khi = min(r0 + kXT - 1, rows_hi) - (M - 1);
        const int blo = klo >= 0 ? klo : (khi <= 0 ? -khi : 0);
        const int bstart = blo & ~1;
        const uint32_t stage_bytes = 2u * 4u * 8u * (uint32_t)(rawk + kCrossColBox);
        for (int g = g0; g < g1 && ok; ++g) {
          for (int st = 0; st < nst; ++st) {
            const int rs = (int)(rq % kXRaw);
            if (rq >= (uint32_t)kXRaw &&
                !mbar_wait_bounded(&rempty[rs], ((rq / kXRaw) - 1) & 1u, status)) {
              ok = false;
              break;
            }
            const int last = st == nst - 1;
            rrec[rs] = RawRec{r0, l0, combo, bstart, st,
                              (st == 0 ? kRecFirst : 0) | (last ? kRecLast : 0) |
                                  (last && g == g1 - 1 ? kRecItemEnd : 0)};
            unsigned char* dst = raws + (size_t)rs * kXRawBytes;
            // 4 frame rows of each channel (rows past the group's m frames are not
            // used; rows and bins past the spectra read as zeros)
            const int fr = g * m + st * kXF;
            mbar_arrive_expect_tx(&rfull[rs], stage_bytes);
            tma_load_2d(dst + kRawA, &tm_ab, bstart, cb.x * chan_rows + fr, &rfull[rs]);
            tma_load_2d(dst + kRawB, &tm_ab, bstart, cb.y * chan_rows + fr, &rfull[rs]);
            tma_load_2d(dst + kRawC, &tm_cd, l0, cb.z * chan_rows + fr, &rfull[rs]);
            tma_load_2d(dst + kRawD, &tm_cd, l0, cb.w * chan_rows + fr, &rfull[rs]);
            ++rq;
          }
        }
        if (!ok) break;
      }
      if (!ok) atomicExch(&s_fail, 1);
      // every copy issued has landed before the CTA may exit (waited before the stop
      // record moves the barrier to its next phase)
      for (uint32_t i = rq > (uint32_t)kXRaw ? rq - kXRaw : 0; i < rq; ++i)
        mbar_wait_bounded(&rfull[i % kXRaw], (i / kXRaw) & 1u, status);
      const int rs = (int)(rq % kXRaw);
      if (rq >= (uint32_t)kXRaw) mbar_wait_bounded(&rempty[rs], ((rq / kXRaw) - 1) & 1u, status);
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
            float2 t = cmulf(sxy, szw);
            cmacf(t, xz, yw);
            cmacf(t, xw, yz);
            const float cr = pref * fmaf(fmm, d[8][i], -fm1 * t.x);
            const float ci = pref * fmaf(fmm, d[9][i], -fm1 * t.y);
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

cudaError_t launch_k3_trispec_cross_tc(const CUtensorMap& tm_ab, const CUtensorMap& tm_cd,
                                       int chan_rows, int G, int m, int M, int Mp,
                                       const int4* combos, int n_combos, double* acc,
                                       long long plane, int nsm, bool natural, int* counter,
                                       int* status, cudaStream_t stream) {
  if (G <= 0 || n_combos <= 0) return cudaSuccess;
  if (m < 1 || M < 2 || nsm <= 0 || (Mp & 15) || Mp < M) return cudaErrorInvalidValue;
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
  auto kern = k3_trispec_cross_tc;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kXSmemBytes);
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
  const int rawk = std::min(kRawK, Mp);  // the box width of tm_ab
  kern<<<nsm, kXThreads, kXSmemBytes, stream>>>(tm_ab, tm_cd, chan_rows, rawk, G, m, M, Mp,
                                                combos, wq, pref, fmm, fm1, acc, plane,
                                                combo_stride, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n = 4 * n_combos * M;
  k3_cross_row0<<<(n + 255) / 256, 256, 0, stream>>>(acc, n, M, combo_stride, plane);
  return cudaGetLastError();
}

}  // namespace ss
