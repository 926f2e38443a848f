// k_bispec.cu -- K2: per-group bispectrum k-statistics on CUDA cores (FP32).
//
// For every group and every grid point (k, l) of the domain it forms
//   c3(a_k, b_l, c_{k+l}*) = m/((m-1)(m-2)) sum_j da_jk db_jl dc*_j,k+l
// -- Eq. 33 written with centred samples (the group means are removed by K1),
// the form equivalent to the raw-moment expression -- and accumulates the sum
// and the sums of squares of its real and imaginary parts over groups
// (Sec. 4.2, Eq. 35-36).  The window and dt normalisation (Eq. 28, Eq. 48) is
// applied by the finalize kernel.
//
// Work split: persistent CTAs take (group chunk, 64 x 64 tile of (k, l)) items
// from a group-major work queue.  A group's frames are taken in chunks of FC
// frames; for each chunk one thread issues three 3-D TMA box loads (FC frames x
// 64 bins at k0, at l0, and FC x 128 bins at k0 + l0, as 128-byte blocks of 16
// bins with 128-byte swizzling; bins past the spectrum read as zero) into one of
// kStages shared-memory stages, so loads run kStages-1 chunks ahead of the
// arithmetic.  Each thread evaluates a 4 x 4 micro-tile of grid points with
// 128-bit shared loads; the thread layout (a quarter-warp covers 4 k-threads x
// 2 l-threads) together with the swizzle keeps every quarter-warp on distinct
// banks.  The per-item float32 sums over groups of the four parts (Re, Im and
// their squares) live in tensor memory, 128 columns per CTA (warp w: TMEM lane
// quadrant w % 4, columns 64 (w / 4) ..), read and written with tcgen05.ld/st
// once per group, which keeps the kernel within 128 registers and two CTAs per
// SM; they are added to the float64 accumulators when the item ends.  Warps whose 32 x 16 sub-tile lies outside
// the domain skip the arithmetic.  All waits on the stage barriers are bounded.
//
// Domains: one channel (cross = 0): 0 <= k <= l, k + l <= M-1 (the rest follows
// from S3(k, l) = S3(l, k), Sec. 9).  Several channels (cross = 1):
// -(M-1) <= k <= M-1, 0 <= l <= M-1, |k + l| <= M-1, using X_{-k} = X_k*; tiles
// that reach negative bins are staged by the threads (conjugated), not by TMA.
#include <algorithm>

#include "internal.cuh"
#include "pipeline.cuh"

namespace ss {
namespace {

constexpr int kStages = 4;

__device__ __forceinline__ float2 coef(const float2* __restrict__ row, int k, int M) {
  if (k >= 0) return k < M ? row[k] : make_float2(0.f, 0.f);
  if (-k < M) {
    const float2 v = row[-k];
    return make_float2(v.x, -v.y);
  }
  return make_float2(0.f, 0.f);
}

__device__ __forceinline__ bool in_domain3(int k, int l, int M, int cross) {
  if (cross) return l >= 0 && l < M && k > -M && k < M && (k + l) < M && (k + l) > -M;
  return k >= 0 && k <= l && k + l < M;
}

// bytes of one [FC][64] float2 array rounded up to the 1024-byte swizzle atom
__host__ __device__ __forceinline__ uint32_t arr64_bytes(int FC) {
  return ((uint32_t)FC * 512u + 1023u) & ~1023u;
}
__host__ __device__ __forceinline__ uint32_t stage_bytes(int FC) {
  return 2u * arr64_bytes(FC) + (uint32_t)FC * 1024u;
}

__device__ __forceinline__ float4 lds128(const unsigned char* p) {
  return *reinterpret_cast<const float4*>(p);
}

// 16-byte load from a shared-memory address (the .shared window, 32 bits)
__device__ __forceinline__ float4 lds128_s(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a));
  return v;
}

constexpr uint32_t kTmemCols = 128;  // per CTA: 2 warps per lane quadrant x 64 columns

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
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
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// kFC > 0: the frames per staged chunk fixed at compile time (the frame loop of a
// full chunk is unrolled with constant shared-memory offsets); 0: taken from FC.
// kSt stages; kMinCtas resident CTAs per SM the register budget is set for (two
// with four stages: 128 registers; three with three stages: 85)
template <int kFC, int kSt = kStages, int kMinCtas = 2>
__global__ void __launch_bounds__(kThreadsPair, kMinCtas)
k2_bispec(const __grid_constant__ CUtensorMap tm64, const __grid_constant__ CUtensorMap tm128,
          const float2* __restrict__ sa, const float2* __restrict__ sb,
          const float2* __restrict__ sc, int rowA, int rowB, int rowC, int G, int m, int FC_rt,
          int M, int Mp, const TileInfo* __restrict__ tiles, WorkQueue wq, int cross,
          float pref3, double* __restrict__ acc, long long plane, int koff,
          int* __restrict__ status, int inject_timeout) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];  // + 1024 spare bytes
  __shared__ __align__(8) uint64_t full[kSt];
  __shared__ __align__(8) uint64_t never;  // completed by nothing (timeout test)
  __shared__ int s_item;
  __shared__ uint32_t tmem_slot;
  unsigned char* sbase = align1024<unsigned char>(smem_raw);
  const int FC = kFC > 0 ? kFC : FC_rt;
  const uint32_t sbytes = stage_bytes(FC), a64 = arr64_bytes(FC);
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int qw = lane >> 3, r8 = lane & 7;
  const int tx = (warp & 1) * 8 + (r8 & 3) + 4 * (qw & 1);    // 16 threads along k
  const int ty = (warp >> 1) * 4 + (r8 >> 2) + 2 * (qw >> 1);  // 16 threads along l
  const int kt = 4 * tx, lt = 4 * ty;
  const int nch = (m + FC - 1) / FC;
  // swizzled byte offsets of this thread's operands (even / odd frame of a pair)
  const uint32_t oA0 = swz128(kt * 8), oA1 = swz128(kt * 8 + 16);
  const uint32_t oA0o = swz128(512 + kt * 8), oA1o = swz128(512 + kt * 8 + 16);
  const uint32_t oB0 = swz128(lt * 8), oB1 = swz128(lt * 8 + 16);
  const uint32_t oB0o = swz128(512 + lt * 8), oB1o = swz128(512 + lt * 8 + 16);
  uint32_t oC[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) oC[d] = swz128((kt + lt) * 8 + 16 * d);

  if (tid == 0) {
    for (int s = 0; s < kSt; ++s) mbar_init(&full[s], 1);
    mbar_init(&never, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // this warp's 64 columns of per-item sums: Re, Im, Re^2, Im^2 of 16 points
  const uint32_t tsum = tmem_slot + ((uint32_t)(32 * (warp & 3)) << 16) + 64u * (warp >> 2);
  {
    float z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) z[i] = 0.f;
#pragma unroll
    for (int part = 0; part < 4; ++part) tmem_st16(tsum + 16 * part, z);
  }
  uint32_t qbase = 0;  // TMA steps consumed so far (stage = q % kSt)
  bool failed = false;

  for (int item; !failed && (item = next_item(wq, &s_item)) >= 0;) {
    const int t = item % wq.n_tiles;
    const int ga = (item / wq.n_tiles) * wq.group_chunk;
    const int gb = min(G, ga + wq.group_chunk);
    const int k0 = tiles[t].k0, l0 = tiles[t].l0;
    const bool use_tma = k0 >= 0 && k0 + l0 >= 0;
    const int kw = k0 + 32 * (warp & 1), lw = l0 + 16 * (warp >> 1);
    bool active = false;
    for (int a = 0; a < 32 && !active; ++a)
      for (int b = 0; b < 16 && !active; ++b) active = in_domain3(kw + a, lw + b, M, cross);
    const int nsteps = (gb - ga) * nch;
    auto issue = [&](int i) {
      const int s = (int)((qbase + i) % kSt);
      const int g = ga + i / nch, j0 = (i % nch) * FC;
      unsigned char* st = sbase + (size_t)s * sbytes;
      mbar_arrive_expect_tx(&full[s], (uint32_t)FC * 256u * 8u);
      tma_load_3d(st, &tm64, 0, k0 >> 4, rowA + g * m + j0, &full[s]);
      tma_load_3d(st + a64, &tm64, 0, l0 >> 4, rowB + g * m + j0, &full[s]);
      tma_load_3d(st + 2 * a64, &tm128, 0, (k0 + l0) >> 4, rowC + g * m + j0, &full[s]);
    };

    float ar[16], ai[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) ar[i] = ai[i] = 0.f;

    if (use_tma && tid == 0) {
      fence_async_smem();
      for (int i = 0; i < kSt && i < nsteps; ++i) issue(i);
    }
    bool ok = true;
    for (int i = 0; i < nsteps; ++i) {
      const int g = ga + i / nch, ch = i % nch, j0 = ch * FC;
      const int nf = min(FC, m - j0);
      const int s = use_tma ? (int)((qbase + i) % kSt) : (i & 1);
      const unsigned char* sA = sbase + (size_t)s * sbytes;
      const unsigned char* sB = sA + a64;
      const unsigned char* sC = sA + 2 * a64;
      if (use_tma) {
        ok = mbar_wait_bounded(&full[s], ((qbase + i) / kSt) & 1u, status);
      } else {
        unsigned char* w = sbase + (size_t)s * sbytes;
        for (int idx = tid; idx < nf * 4 * kTile; idx += blockDim.x) {
          const int j = idx / (4 * kTile);
          const int e = idx - j * 4 * kTile;
          const long long rr = ((long long)g * m + j0 + j) * Mp;
          float2 v;
          uint32_t off;
          if (e < kTile) {
            v = coef(sa + rr, k0 + e, M);
            off = swz128(j * 512 + e * 8);
          } else if (e < 2 * kTile) {
            v = coef(sb + rr, l0 + e - kTile, M);
            off = a64 + swz128(j * 512 + (e - kTile) * 8);
          } else {
            v = coef(sc + rr, k0 + l0 + e - 2 * kTile, M);
            off = 2 * a64 + swz128(j * 1024 + (e - 2 * kTile) * 8);
          }
          *reinterpret_cast<float2*>(w + off) = v;
        }
        __syncthreads();
      }
      // timeout test (inject_timeout): the CTA that takes the first item waits, at
      // its first step, on a barrier that nothing completes; the wait runs out and
      // the CTA stops as after any failed wait (the copies already issued drain)
      if (inject_timeout && item == 0 && i == 0 && tid == 0)
        ok = mbar_wait_bounded(&never, 0u, status, kInjectedWaitNs) && ok;
      if (active) {
        auto frame = [&](int j, uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1) {
          const unsigned char* pa = sA + (j & ~1) * 512;
          const unsigned char* pb = sB + (j & ~1) * 512;
          const unsigned char* pc = sC + j * 1024;
          const float4 a01 = lds128(pa + a0), a23 = lds128(pa + a1);
          const float4 b01 = lds128(pb + b0), b23 = lds128(pb + b1);
          const float4 c01 = lds128(pc + oC[0]), c23 = lds128(pc + oC[1]);
          const float4 c45 = lds128(pc + oC[2]), c67 = lds128(pc + oC[3]);
          const float2 ak[4] = {{a01.x, a01.y}, {a01.z, a01.w}, {a23.x, a23.y}, {a23.z, a23.w}};
          const float2 al[4] = {{b01.x, b01.y}, {b01.z, b01.w}, {b23.x, b23.y}, {b23.z, b23.w}};
          const float2 ac[7] = {{c01.x, c01.y}, {c01.z, c01.w}, {c23.x, c23.y}, {c23.z, c23.w},
                                {c45.x, c45.y}, {c45.z, c45.w}, {c67.x, c67.y}};
#pragma unroll
          for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              // p = a_k b_l ; accumulate p * conj(c_{k+l})
              const float px = fmaf(ak[a].x, al[b].x, -ak[a].y * al[b].y);
              const float py = fmaf(ak[a].x, al[b].y, ak[a].y * al[b].x);
              const float2 c = ac[a + b];
              ar[a * 4 + b] = fmaf(px, c.x, fmaf(py, c.y, ar[a * 4 + b]));
              ai[a * 4 + b] = fmaf(py, c.x, fmaf(-px, c.y, ai[a * 4 + b]));
            }
          }
        };
        if (kFC > 0 && nf == kFC) {
#pragma unroll
          for (int j = 0; j < kFC; j += 2) {
            frame(j, oA0, oA1, oB0, oB1);
            if (j + 1 < kFC) frame(j + 1, oA0o, oA1o, oB0o, oB1o);
          }
        } else {
          int j = 0;
          for (; j + 1 < nf; j += 2) {
            frame(j, oA0, oA1, oB0, oB1);
            frame(j + 1, oA0o, oA1o, oB0o, oB1o);
          }
          if (j < nf) frame(j, oA0, oA1, oB0, oB1);
        }
        if (ch == nch - 1) {  // end of a group: c3 into the per-item sums
          float t[16];
          tmem_ld16(tsum, t);
#pragma unroll
          for (int q = 0; q < 16; ++q) t[q] = fmaf(ar[q], pref3, t[q]);
          tmem_st16(tsum, t);
          tmem_ld16(tsum + 16, t);
#pragma unroll
          for (int q = 0; q < 16; ++q) t[q] = fmaf(ai[q], pref3, t[q]);
          tmem_st16(tsum + 16, t);
          tmem_ld16(tsum + 32, t);
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float v = ar[q] * pref3;
            t[q] = fmaf(v, v, t[q]);
          }
          tmem_st16(tsum + 32, t);
          tmem_ld16(tsum + 48, t);
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float v = ai[q] * pref3;
            t[q] = fmaf(v, v, t[q]);
            ar[q] = ai[q] = 0.f;
          }
          tmem_st16(tsum + 48, t);
        }
      }
      // every thread is done with stage s; a failed wait anywhere stops the CTA.
      // Before it gives up, the copies issued so far (steps i .. i + kSt - 1,
      // the one whose wait ran out included) must have landed: those drain waits
      // keep the full limit, so no copy is in flight when the CTA exits.
      if (__syncthreads_or(!ok)) {
        if (use_tma)
          for (int q = i; q < nsteps && q < i + kSt; ++q)
            mbar_wait_bounded(&full[(qbase + q) % kSt], ((qbase + q) / kSt) & 1u, status);
        failed = true;
        break;
      }
      if (use_tma && tid == 0 && i + kSt < nsteps) {
        fence_async_smem();
        issue(i + kSt);
      }
    }
    if (failed) break;
    if (use_tma) qbase += nsteps;
    if (!active) continue;
    // end of the item: the sums of each part go to the float64 accumulators
#pragma unroll 1
    for (int part = 0; part < 4; ++part) {
      float t[16], z[16];
      tmem_ld16(tsum + 16 * part, t);
      double* dst = acc + (long long)part * plane;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int k = k0 + kt + (q >> 2), l = l0 + lt + (q & 3);
        if (in_domain3(k, l, M, cross))
          atomicAdd(dst + (long long)(k + koff) * M + l, (double)t[q]);
        z[q] = 0.f;
      }
      tmem_st16(tsum + 16 * part, z);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot),
                 "r"(kTmemCols));
  }
}

// ---------------------------------------------------------------------------
// K2 with 8 x 4 micro-tiles (k2_bispec84).  Same items, staging and sums as
// k2_bispec, smaller CTAs: 4 warps of 32 x 32 grid points on the 64 x 64 tile,
// each thread 8 k-bins x 4 l-bins, so a frame costs 12 shared-memory loads of
// 16 bytes per 32 points (256 FP instructions) instead of 8 per 16 points: the
// shared-memory wavefronts per FP instruction drop from 0.25 to 0.19.  Lanes map
// to (tx, ty) = (lane & 3, bit 3 | bit 2 << 1 | bit 4 << 2 of the lane), which
// with the 128-byte swizzle puts every quarter-warp's loads of a_k, b_l and
// c_{k+l} on distinct bank groups (checked with a bank model for every load of a
// frame).  Warps whose 32 x 32 sub-tile lies outside the domain skip the
// arithmetic.  The per-item sums of the warp's 32 points (four parts) live in
// 128 TMEM columns of its lane quadrant.  kSt stages of FC frames.
constexpr int kThreads84 = 128;

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
      "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
      "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
      "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
      "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
      "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// resident CTAs per SM the register budget is set for: four with two stages
// (128 registers), three with three (168)
template <int kSt>
constexpr int k84_min_ctas() { return kSt == 2 ? 4 : 3; }

template <int kFC, int kSt>
__global__ void __launch_bounds__(kThreads84, k84_min_ctas<kSt>())
k2_bispec84(const __grid_constant__ CUtensorMap tm64, const __grid_constant__ CUtensorMap tm128,
            const float2* __restrict__ sa, const float2* __restrict__ sb,
            const float2* __restrict__ sc, int rowA, int rowB, int rowC, int G, int m,
            int FC_rt, int M, int Mp, const TileInfo* __restrict__ tiles, WorkQueue wq,
            int cross, float pref3, double* __restrict__ acc, long long plane, int koff,
            int* __restrict__ status, int inject_timeout) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];  // + 1024 spare bytes
  __shared__ __align__(8) uint64_t full[kSt];
  __shared__ __align__(8) uint64_t never;  // completed by nothing (timeout test)
  __shared__ int s_item;
  __shared__ uint32_t tmem_slot;
  unsigned char* sbase = align1024<unsigned char>(smem_raw);
  const int FC = kFC > 0 ? kFC : FC_rt;
  const uint32_t sbytes = stage_bytes(FC), a64 = arr64_bytes(FC);
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tx = lane & 3;
  const int ty = ((lane >> 3) & 1) | (((lane >> 2) & 1) << 1) | (((lane >> 4) & 1) << 2);
  const int wk = warp & 1, wl = warp >> 1;
  const int kt = 32 * wk + 8 * tx, lt = 32 * wl + 4 * ty;  // micro-tile origin in the tile
  const int nch = (m + FC - 1) / FC;
  // byte offsets of the thread's loads in frame row 0 before the swizzle; the
  // rows of the 64-bin arrays are 512 bytes, so an odd row flips bit 6 of the
  // swizzled offset (bit 9 of the row start enters the swizzle), the 1024-byte
  // rows of c_{k+l} do not
  const uint32_t oa0 = kt * 8, ob0 = lt * 8, oc0 = (kt + lt) * 8;

  if (tid == 0) {
    for (int s = 0; s < kSt; ++s) mbar_init(&full[s], 1);
    mbar_init(&never, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // this warp's 128 columns of per-item sums in its lane quadrant: Re, Im, Re^2,
  // Im^2 of its 32 points (point q = 4 a + b at column 32 part + q)
  const uint32_t tsum = tmem_slot + ((uint32_t)(32 * warp) << 16);
  {
    float z[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) z[i] = 0.f;
#pragma unroll
    for (int part = 0; part < 4; ++part) tmem_st32(tsum + 32 * part, z);
  }
  uint32_t qbase = 0;  // TMA steps consumed so far (stage = q % kSt)
  bool failed = false;

  for (int item; !failed && (item = next_item(wq, &s_item)) >= 0;) {
    const int t = item % wq.n_tiles;
    const int ga = (item / wq.n_tiles) * wq.group_chunk;
    const int gb = min(G, ga + wq.group_chunk);
    const int k0 = tiles[t].k0, l0 = tiles[t].l0;
    const bool use_tma = k0 >= 0 && k0 + l0 >= 0;
    const int kw = k0 + 32 * wk, lw = l0 + 32 * wl;
    bool active = false;
    for (int a = 0; a < 32 && !active; ++a)
      for (int b = 0; b < 32 && !active; ++b) active = in_domain3(kw + a, lw + b, M, cross);
    const int nsteps = (gb - ga) * nch;
    auto issue = [&](int i) {
      const int s = (int)((qbase + i) % kSt);
      const int g = ga + i / nch, j0 = (i % nch) * FC;
      unsigned char* st = sbase + (size_t)s * sbytes;
      mbar_arrive_expect_tx(&full[s], (uint32_t)FC * 256u * 8u);
      tma_load_3d(st, &tm64, 0, k0 >> 4, rowA + g * m + j0, &full[s]);
      tma_load_3d(st + a64, &tm64, 0, l0 >> 4, rowB + g * m + j0, &full[s]);
      tma_load_3d(st + 2 * a64, &tm128, 0, (k0 + l0) >> 4, rowC + g * m + j0, &full[s]);
    };

    float ar[32], ai[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) ar[i] = ai[i] = 0.f;

    if (use_tma && tid == 0) {
      fence_async_smem();
      for (int i = 0; i < kSt && i < nsteps; ++i) issue(i);
    }
    bool ok = true;
    for (int i = 0; i < nsteps; ++i) {
      const int g = ga + i / nch, ch = i % nch, j0 = ch * FC;
      const int nf = min(FC, m - j0);
      const int s = use_tma ? (int)((qbase + i) % kSt) : (i & 1);
      const unsigned char* sA = sbase + (size_t)s * sbytes;
      const unsigned char* sB = sA + a64;
      const unsigned char* sC = sA + 2 * a64;
      if (use_tma) {
        ok = mbar_wait_bounded(&full[s], ((qbase + i) / kSt) & 1u, status);
      } else {
        unsigned char* w = sbase + (size_t)s * sbytes;
        for (int idx = tid; idx < nf * 4 * kTile; idx += blockDim.x) {
          const int j = idx / (4 * kTile);
          const int e = idx - j * 4 * kTile;
          const long long rr = ((long long)g * m + j0 + j) * Mp;
          float2 v;
          uint32_t off;
          if (e < kTile) {
            v = coef(sa + rr, k0 + e, M);
            off = swz128(j * 512 + e * 8);
          } else if (e < 2 * kTile) {
            v = coef(sb + rr, l0 + e - kTile, M);
            off = a64 + swz128(j * 512 + (e - kTile) * 8);
          } else {
            v = coef(sc + rr, k0 + l0 + e - 2 * kTile, M);
            off = 2 * a64 + swz128(j * 1024 + (e - 2 * kTile) * 8);
          }
          *reinterpret_cast<float2*>(w + off) = v;
        }
        __syncthreads();
      }
      if (inject_timeout && item == 0 && i == 0 && tid == 0)
        ok = mbar_wait_bounded(&never, 0u, status, kInjectedWaitNs) && ok;
      if (active) {
        auto frame = [&](int j) {
          const unsigned char* pa = sA + j * 512;
          const unsigned char* pb = sB + j * 512;
          const unsigned char* pc = sC + j * 1024;
          const uint32_t odd = (uint32_t)(j & 1) << 6;
          float2 al[4], ac[12];
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const float4 v = lds128(pb + (swz128(ob0 + 16 * q) ^ odd));
            al[2 * q] = make_float2(v.x, v.y);
            al[2 * q + 1] = make_float2(v.z, v.w);
          }
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            const float4 v = lds128(pc + swz128(oc0 + 16 * q));
            ac[2 * q] = make_float2(v.x, v.y);
            ac[2 * q + 1] = make_float2(v.z, v.w);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 v = lds128(pa + (swz128(oa0 + 16 * q) ^ odd));
            const float2 ak2[2] = {make_float2(v.x, v.y), make_float2(v.z, v.w)};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int a = 2 * q + h;
#pragma unroll
              for (int b = 0; b < 4; ++b) {
                // p = a_k b_l ; accumulate p * conj(c_{k+l})
                const float px = fmaf(ak2[h].x, al[b].x, -ak2[h].y * al[b].y);
                const float py = fmaf(ak2[h].x, al[b].y, ak2[h].y * al[b].x);
                const float2 c = ac[a + b];
                ar[a * 4 + b] = fmaf(px, c.x, fmaf(py, c.y, ar[a * 4 + b]));
                ai[a * 4 + b] = fmaf(py, c.x, fmaf(-px, c.y, ai[a * 4 + b]));
              }
            }
          }
        };
        if (kFC > 0 && nf == kFC) {
#pragma unroll 1
          for (int j = 0; j < kFC; ++j) frame(j);
        } else {
          for (int j = 0; j < nf; ++j) frame(j);
        }
        if (ch == nch - 1) {  // end of a group: c3 into the per-item sums
#pragma unroll
          for (int h = 0; h < 2; ++h) {  // halves of 16 points keep the registers low
            float tt[16];
            tmem_ld16(tsum + 16 * h, tt);
#pragma unroll
            for (int q = 0; q < 16; ++q) tt[q] = fmaf(ar[16 * h + q], pref3, tt[q]);
            tmem_st16(tsum + 16 * h, tt);
            tmem_ld16(tsum + 32 + 16 * h, tt);
#pragma unroll
            for (int q = 0; q < 16; ++q) tt[q] = fmaf(ai[16 * h + q], pref3, tt[q]);
            tmem_st16(tsum + 32 + 16 * h, tt);
            tmem_ld16(tsum + 64 + 16 * h, tt);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const float v = ar[16 * h + q] * pref3;
              tt[q] = fmaf(v, v, tt[q]);
            }
            tmem_st16(tsum + 64 + 16 * h, tt);
            tmem_ld16(tsum + 96 + 16 * h, tt);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const float v = ai[16 * h + q] * pref3;
              tt[q] = fmaf(v, v, tt[q]);
              ar[16 * h + q] = ai[16 * h + q] = 0.f;
            }
            tmem_st16(tsum + 96 + 16 * h, tt);
          }
        }
      }
      // every thread is done with stage s; a failed wait anywhere stops the CTA
      // after the copies issued so far (steps i .. i + kSt - 1) have landed
      if (__syncthreads_or(!ok)) {
        if (use_tma)
          for (int q = i; q < nsteps && q < i + kSt; ++q)
            mbar_wait_bounded(&full[(qbase + q) % kSt], ((qbase + q) / kSt) & 1u, status);
        failed = true;
        break;
      }
      if (use_tma && tid == 0 && i + kSt < nsteps) {
        fence_async_smem();
        issue(i + kSt);
      }
    }
    if (failed) break;
    if (use_tma) qbase += nsteps;
    if (!active) continue;
    // end of the item: the sums of each part go to the float64 accumulators
#pragma unroll 1
    for (int part = 0; part < 4; ++part) {
      float tt[32], z[32];
      tmem_ld32(tsum + 32 * part, tt);
      double* dst = acc + (long long)part * plane;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int k = k0 + kt + (q >> 2), l = l0 + lt + (q & 3);
        if (in_domain3(k, l, M, cross))
          atomicAdd(dst + (long long)(k + koff) * M + l, (double)tt[q]);
        z[q] = 0.f;
      }
      tmem_st32(tsum + 32 * part, z);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot),
                 "r"(kTmemCols));
  }
}

// ---------------------------------------------------------------------------
// K2 with independent warps (k2_bispec84w, one channel).  Each warp of a
// 128-thread CTA is a worker of its own: it takes (group chunk, 32 x 32
// sub-tile) items from the queue, stages the item's frame rows kFS84w at a
// time into its own ring of kSt84w stages (a: 32 bins, b: 32 bins, c: 64 bins
// per frame, three 3-D TMA boxes with 128-byte swizzling, refilled by its lane
// 0 as soon as the warp leaves a stage) and evaluates 8 x 4 micro-tiles as
// k2_bispec84 does, with the same lane layout (conflict-free for these 256- and
// 512-byte frame rows too, checked with a bank model).  No block barrier: a warp
// never waits for another.  The frames of an item's groups are contiguous rows,
// so the stages run across group boundaries and a group ends at the frame where
// its m-th row is consumed.  Per-item sums: 128 TMEM columns of the warp's lane
// quadrant; four CTAs per SM fill the 512 columns.
constexpr int kThreads84w = 128;
constexpr int kFS84w = kFrames84w;  // frames per stage
constexpr int kSt84w = 3;   // stages per warp
constexpr uint32_t kStage84w = kFS84w * (256u + 256u + 512u);  // a | b | c
constexpr uint32_t kRing84w = kSt84w * kStage84w;

__global__ void __launch_bounds__(kThreads84w, 4)
k2_bispec84w(const __grid_constant__ CUtensorMap tm32, const __grid_constant__ CUtensorMap tm64,
             int row0, int m, int M, int G, const TileInfo* __restrict__ tiles, WorkQueue wq,
             float pref3, double* __restrict__ acc, long long plane, int* __restrict__ status,
             int inject_timeout) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];  // + 1024 spare bytes
  __shared__ __align__(8) uint64_t full[kThreads84w / 32][kSt84w];
  __shared__ __align__(8) uint64_t never;  // completed by nothing (timeout test)
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char* ring = align1024<unsigned char>(smem_raw) + (size_t)warp * kRing84w;
  const int tx = lane & 3;
  const int ty = ((lane >> 3) & 1) | (((lane >> 2) & 1) << 1) | (((lane >> 4) & 1) << 2);
  const int kt = 8 * tx, lt = 4 * ty;  // micro-tile origin in the sub-tile
  // Swizzled byte offsets of the thread's loads in frame 0 of an array: frame f of
  // a or b (256-byte rows) XORs them with 32 f, of c (512-byte rows) with 64 (f & 1).
  // For a and b the q-th 16-byte load of a thread stays in the 128-byte row of the
  // first (their chunk is 0 or 4, resp. even), so its offset is the first's XOR 16 q;
  // with array and frame bases free of the offset bits, an address is the frame
  // base XOR one per-thread constant, one logic operation a load.
  const uint32_t sa0 = swz128(kt * 8), sb0 = swz128(lt * 8);
  uint32_t sc[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) sc[q] = swz128((kt + lt) * 8 + 16 * q);
  const uint32_t ring_s = smem_addr(ring);

  if (tid == 0) {
    for (int w = 0; w < kThreads84w / 32; ++w)
      for (int s = 0; s < kSt84w; ++s) mbar_init(&full[w][s], 1);
    mbar_init(&never, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tsum = tmem_slot + ((uint32_t)(32 * warp) << 16);
  {
    float z[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) z[i] = 0.f;
#pragma unroll
    for (int part = 0; part < 4; ++part) tmem_st32(tsum + 32 * part, z);
  }
  uint32_t qb = 0;  // stages this warp has consumed (stage = q % kSt84w)
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(wq.counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= wq.n_items) break;
    const int t = item % wq.n_tiles;
    const int ga = (item / wq.n_tiles) * wq.group_chunk;
    const int gb = min(G, ga + wq.group_chunk);
    const int k0 = tiles[t].k0, l0 = tiles[t].l0;
    const int rows = (gb - ga) * m;  // the item's frames, consecutive rows from r0
    const int r0 = row0 + ga * m;
    const int nst = (rows + kFS84w - 1) / kFS84w;
    auto issue = [&](int i) {  // lane 0: stage of step i (kFS84w rows from r0 + i kFS84w)
      const int s = (int)((qb + i) % kSt84w);
      unsigned char* st = ring + (size_t)s * kStage84w;
      const int r = r0 + i * kFS84w;
      mbar_arrive_expect_tx(&full[warp][s], kStage84w);
      tma_load_3d(st, &tm32, 0, k0 >> 4, r, &full[warp][s]);
      tma_load_3d(st + kFS84w * 256, &tm32, 0, l0 >> 4, r, &full[warp][s]);
      tma_load_3d(st + kFS84w * 512, &tm64, 0, (k0 + l0) >> 4, r, &full[warp][s]);
    };
    float ar[32], ai[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) ar[i] = ai[i] = 0.f;
    if (lane == 0) {
      fence_async_smem();
      for (int i = 0; i < kSt84w && i < nst; ++i) issue(i);
    }
    __syncwarp();
    bool ok = true;
    int jg = 0;  // frames of the current group consumed
    for (int i = 0; i < nst && ok; ++i) {
      const int s = (int)((qb + i) % kSt84w);
      ok = mbar_wait_bounded(&full[warp][s], ((qb + i) / kSt84w) & 1u, status);
      // timeout test: the warp that takes the first item waits, at its first
      // step, on a barrier that nothing completes
      if (inject_timeout && item == 0 && i == 0 && lane == 0)
        ok = mbar_wait_bounded(&never, 0u, status, kInjectedWaitNs) && ok;
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        // the copies issued and not consumed (steps i .. i + kSt84w - 1) land
        // before the warp stops; those waits keep the full limit
        if (lane == 0)
          for (int q = i; q < nst && q < i + kSt84w; ++q)
            mbar_wait_bounded(&full[warp][(qb + q) % kSt84w], ((qb + q) / kSt84w) & 1u, status);
        break;
      }
      const uint32_t sA = ring_s + (uint32_t)s * kStage84w;  // 1024-byte aligned
      const uint32_t sB = sA + kFS84w * 256;
      const uint32_t sC = sA + kFS84w * 512;
      const int nf = min(kFS84w, rows - i * kFS84w);
#pragma unroll 1
      for (int f = 0; f < nf; ++f) {
        const uint32_t fab = (uint32_t)f << 5, fc = (uint32_t)(f & 1) << 6;
        const uint32_t pa = (sA + f * 256) | (sa0 ^ fab);
        const uint32_t pb = (sB + f * 256) | (sb0 ^ fab);
        const uint32_t pc = (sC + f * 512) ^ fc;
        float2 al[4], ac[12];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float4 v = lds128_s(pb ^ (16u * q));
          al[2 * q] = make_float2(v.x, v.y);
          al[2 * q + 1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const float4 v = lds128_s(pc ^ sc[q]);
          ac[2 * q] = make_float2(v.x, v.y);
          ac[2 * q + 1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 v = lds128_s(pa ^ (16u * q));
          const float2 ak2[2] = {make_float2(v.x, v.y), make_float2(v.z, v.w)};
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int a = 2 * q + h;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              // p = a_k b_l ; accumulate p * conj(c_{k+l})
              const float px = fmaf(ak2[h].x, al[b].x, -ak2[h].y * al[b].y);
              const float py = fmaf(ak2[h].x, al[b].y, ak2[h].y * al[b].x);
              const float2 c = ac[a + b];
              ar[a * 4 + b] = fmaf(px, c.x, fmaf(py, c.y, ar[a * 4 + b]));
              ai[a * 4 + b] = fmaf(py, c.x, fmaf(-px, c.y, ai[a * 4 + b]));
            }
          }
        }
        if (++jg == m) {  // end of a group: c3 into the per-item sums
          jg = 0;
#pragma unroll
          for (int h = 0; h < 2; ++h) {  // halves of 16 points keep the registers low
            float tt[16];
            tmem_ld16(tsum + 16 * h, tt);
#pragma unroll
            for (int q = 0; q < 16; ++q) tt[q] = fmaf(ar[16 * h + q], pref3, tt[q]);
            tmem_st16(tsum + 16 * h, tt);
            tmem_ld16(tsum + 32 + 16 * h, tt);
#pragma unroll
            for (int q = 0; q < 16; ++q) tt[q] = fmaf(ai[16 * h + q], pref3, tt[q]);
            tmem_st16(tsum + 32 + 16 * h, tt);
            tmem_ld16(tsum + 64 + 16 * h, tt);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const float v = ar[16 * h + q] * pref3;
              tt[q] = fmaf(v, v, tt[q]);
            }
            tmem_st16(tsum + 64 + 16 * h, tt);
            tmem_ld16(tsum + 96 + 16 * h, tt);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              const float v = ai[16 * h + q] * pref3;
              tt[q] = fmaf(v, v, tt[q]);
              ar[16 * h + q] = ai[16 * h + q] = 0.f;
            }
            tmem_st16(tsum + 96 + 16 * h, tt);
          }
        }
      }
      // the warp is done with stage s: its lane 0 loads the stage's next step
      __syncwarp();
      if (lane == 0 && i + kSt84w < nst) {
        fence_async_smem();
        issue(i + kSt84w);
      }
    }
    if (!ok) break;
    qb += nst;
    // end of the item: the sums of each part go to the float64 accumulators
#pragma unroll 1
    for (int part = 0; part < 4; ++part) {
      float tt[32], z[32];
      tmem_ld32(tsum + 32 * part, tt);
      double* dst = acc + (long long)part * plane;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int k = k0 + kt + (q >> 2), l = l0 + lt + (q & 3);
        if (in_domain3(k, l, M, 0)) atomicAdd(dst + (long long)k * M + l, (double)tt[q]);
        z[q] = 0.f;
      }
      tmem_st32(tsum + 32 * part, z);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot),
                 "r"(kTmemCols));
  }
}

// Isolated grid points of one channel (the tiles that hold a single point of
// the domain, where the edge k + l = M - 1 passes a tile corner): each thread
// evaluates c3 at one point for one group at a time, reading the centred
// coefficients from global memory, and the block sums over its groups in
// float64 before one atomic add per part.
constexpr int kPointThreads = 128;

__global__ void __launch_bounds__(kPointThreads)
k2_points(const float2* __restrict__ spec, int Mp, int G, int m, const int2* __restrict__ pts,
          int M, float pref3, double* __restrict__ acc, long long plane) {
  __shared__ double red[4][kPointThreads / 32];
  const int2 pt = pts[blockIdx.x];
  const int k = pt.x, l = pt.y;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int g = blockIdx.y * kPointThreads + threadIdx.x; g < G;
       g += gridDim.y * kPointThreads) {
    const float2* row = spec + (long long)g * m * Mp;
    float ar = 0.f, ai = 0.f;
    for (int j = 0; j < m; ++j, row += Mp) {
      const float2 a = row[k], b = row[l], c = row[k + l];
      const float px = fmaf(a.x, b.x, -a.y * b.y);
      const float py = fmaf(a.x, b.y, a.y * b.x);
      ar = fmaf(px, c.x, fmaf(py, c.y, ar));
      ai = fmaf(py, c.x, fmaf(-px, c.y, ai));
    }
    const double vr = (double)(ar * pref3), vi = (double)(ai * pref3);
    s[0] += vr;
    s[1] += vi;
    s[2] += vr * vr;
    s[3] += vi * vi;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double v = s[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[q][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int i = 0; i < kPointThreads / 32; ++i) v += red[threadIdx.x][i];
    atomicAdd(acc + (long long)threadIdx.x * plane + (long long)k * M + l, v);
  }
}

}  // namespace

size_t k2_smem_bytes(int FC) { return (size_t)kStages * stage_bytes(FC) + 1024; }

namespace {

// resident CTAs per SM of one kernel, from its registers and shared memory (the
// occupancy query reports fewer for these kernels than both limits allow),
// capped at max_ctas (the CTAs whose TMEM allocations fit an SM together)
template <typename Kern>
cudaError_t ctas_per_sm(Kern kern, int threads, size_t smem, int max_ctas, int* occ_out) {
  cudaFuncAttributes fa;
  int dev = 0, sm_smem = 0, sm_regs = 0, rsv = 0;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e != cudaSuccess) return e;
  const int regs = ((fa.numRegs + 7) & ~7) * threads;
  const int by_regs = regs > 0 ? sm_regs / regs : 1;
  const int by_smem = sm_smem / (int)(smem + fa.sharedSizeBytes + rsv);
  *occ_out = std::max(1, std::min(max_ctas, std::min(by_regs, by_smem)));
  return cudaSuccess;
}

// shared memory of the 8 x 4 variant with kSt stages of FC frames
size_t k84_smem_bytes(int FC, int kSt) { return (size_t)kSt * stage_bytes(FC) + 1024; }

// One launcher for both tilings: kVar = 0 is k2_bispec (4 x 4 micro-tiles, 256
// threads, 4 stages), kVar = 2 or 3 is k2_bispec84 with that many stages.
template <int kFC, int kVar>
cudaError_t launch_k2_t(const CUtensorMap& tm64, const CUtensorMap& tm128, const float2* spec_a,
                        const float2* spec_b, const float2* spec_c, int rowA, int rowB, int rowC,
                        int G, int m, int FC, int M, int Mp, const TileInfo* tiles, int n_tiles,
                        int cross, float pref3, double* acc, long long plane, int rows, int nsm,
                        int* counter, int* status, int inject_timeout,
                        cudaStream_t stream) {
  // kVar: 0 = 4 x 4 with 4 stages (two CTAs per SM), 1 = 4 x 4 with 3 stages (three
  // CTAs per SM), 2 / 3 = 8 x 4 with that many stages
  constexpr bool k44 = kVar < 2;
  constexpr int kSt = kVar == 0 ? kStages : kVar == 1 ? 3 : kVar;
  auto kern = [] {
    if constexpr (kVar == 0) return k2_bispec<kFC>;
    else if constexpr (kVar == 1) return k2_bispec<kFC, 3, 3>;
    else return k2_bispec84<kFC, kSt>;
  }();
  const int threads = k44 ? kThreadsPair : kThreads84;
  const size_t smem = k84_smem_bytes(FC, kSt);
  // one fixed limit per instantiation (the function attribute is shared by all
  // launches): the chunk size of the instantiation, or the largest one
  const size_t limit = k84_smem_bytes(kFC > 0 ? kFC : kMaxFC, kSt);
  if (FC < 1 || FC > kMaxFC || smem > limit) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)limit);
  if (e != cudaSuccess) return e;
  // the whole unified L1 as shared memory, so that several CTAs fit per SM
  e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  // TMEM: 128 columns per CTA of either tiling, 512 per SM
  int occ = 1;
  e = ctas_per_sm(kern, threads, smem, kVar == 0 ? 2 : kVar == 1 ? 3 : k84_min_ctas<kSt>(),
                  &occ);
  if (e != cudaSuccess) return e;
  const int n_cta = nsm * occ;
  WorkQueue wq;
  wq.counter = counter;
  wq.n_tiles = n_tiles;
  wq.group_chunk = work_group_chunk(G, n_tiles, n_cta);
  wq.n_items = n_tiles * ((G + wq.group_chunk - 1) / wq.group_chunk);
  e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  const int koff = (rows == M) ? 0 : (M - 1);
  kern<<<n_cta, threads, smem, stream>>>(tm64, tm128, spec_a, spec_b, spec_c, rowA, rowB, rowC,
                                         G, m, FC, M, Mp, tiles, wq, cross, pref3, acc, plane,
                                         koff, status, inject_timeout);
  return cudaGetLastError();
}

template <int kVar>
cudaError_t launch_k2_fc(const CUtensorMap& tm64, const CUtensorMap& tm128, const float2* spec_a,
                         const float2* spec_b, const float2* spec_c, int rowA, int rowB, int rowC,
                         int G, int m, int FC, int M, int Mp, const TileInfo* tiles, int n_tiles,
                         int cross, float pref3, double* acc, long long plane, int rows, int nsm,
                         int* counter, int* status, int inject_timeout, cudaStream_t stream) {
#define K2_ARGS tm64, tm128, spec_a, spec_b, spec_c, rowA, rowB, rowC, G, m, FC, M, Mp, tiles, \
                n_tiles, cross, pref3, acc, plane, rows, nsm, counter, status, inject_timeout, stream
  switch (FC) {
    case 8: return launch_k2_t<8, kVar>(K2_ARGS);
    case 10: return launch_k2_t<10, kVar>(K2_ARGS);
    case 16: return launch_k2_t<16, kVar>(K2_ARGS);
    default: return launch_k2_t<0, kVar>(K2_ARGS);
  }
#undef K2_ARGS
}

}  // namespace

cudaError_t launch_k2_bispec84w(const CUtensorMap& tm32, const CUtensorMap& tm64w, int row0,
                                int G, int m, int M, const TileInfo* tiles, int n_tiles,
                                float pref3, double* acc, long long plane, int nsm, int* counter,
                                int* status, int inject_timeout, cudaStream_t stream) {
  if (G <= 0 || n_tiles <= 0) return cudaSuccess;
  const size_t smem = (size_t)(kThreads84w / 32) * kRing84w + 1024;
  cudaError_t e = cudaFuncSetAttribute(k2_bispec84w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k2_bispec84w, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  // TMEM: 128 columns per CTA, 512 per SM
  int occ = 1;
  e = ctas_per_sm(k2_bispec84w, kThreads84w, smem, 4, &occ);
  if (e != cudaSuccess) return e;
  const int n_cta = nsm * occ;
  WorkQueue wq;  // items per warp
  wq.counter = counter;
  wq.n_tiles = n_tiles;
  // about 8 items per warp (half the pair kernels' 16): each item ends with a
  // flush of its warp's 32 x 32 sub-tile, so longer items halve the atomics
  wq.group_chunk = work_group_chunk(G, n_tiles, n_cta * (kThreads84w / 32) / 2);
  wq.n_items = n_tiles * ((G + wq.group_chunk - 1) / wq.group_chunk);
  e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  k2_bispec84w<<<n_cta, kThreads84w, smem, stream>>>(tm32, tm64w, row0, m, M, G, tiles, wq,
                                                     pref3, acc, plane, status, inject_timeout);
  return cudaGetLastError();
}

cudaError_t launch_k2_bispec(const CUtensorMap& tm64, const CUtensorMap& tm128,
                             const float2* spec_a, const float2* spec_b, const float2* spec_c,
                             int rowA, int rowB, int rowC, int G, int m, int FC, int M, int Mp,
                             const TileInfo* tiles, int n_tiles, int cross, float pref3,
                             double* acc, long long plane, int rows, int nsm, int* counter,
                             int* status, int inject_timeout, int variant, cudaStream_t stream) {
  if (G <= 0 || n_tiles <= 0) return cudaSuccess;
#define K2_ARGS tm64, tm128, spec_a, spec_b, spec_c, rowA, rowB, rowC, G, m, FC, M, Mp, tiles, \
                n_tiles, cross, pref3, acc, plane, rows, nsm, counter, status, inject_timeout, stream
  switch (variant) {
    case kK2Tile84Stages2: return launch_k2_fc<2>(K2_ARGS);
    case kK2Tile84Stages3: return launch_k2_fc<3>(K2_ARGS);
    case kK2Tile44: return launch_k2_fc<0>(K2_ARGS);
    case kK2Tile44Stages3: return launch_k2_fc<1>(K2_ARGS);
    default: return cudaErrorInvalidValue;
  }
#undef K2_ARGS
}

cudaError_t launch_k2_points(const float2* spec, int Mp, int G, int m, const int2* pts,
                             int n_pts, int M, float pref3, double* acc, long long plane,
                             cudaStream_t stream) {
  if (G <= 0 || n_pts <= 0) return cudaSuccess;
  const int gy = std::min(256, (G + kPointThreads - 1) / kPointThreads);
  k2_points<<<dim3((unsigned)n_pts, (unsigned)gy), kPointThreads, 0, stream>>>(
      spec, Mp, G, m, pts, M, pref3, acc, plane);
  return cudaGetLastError();
}

}  // namespace ss
