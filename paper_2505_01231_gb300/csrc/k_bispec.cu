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
// Work split: a persistent CTA walks a balanced list of (64 x 64 tile of (k, l),
// range of groups) segments.  Per group, one thread issues 1-D TMA bulk copies
// of the m frames' coefficients at k0..k0+63, l0..l0+63 and k0+l0..k0+l0+127
// into one of two shared-memory stages (mbarrier completion, bounded waits), so
// the copy of group g+2 overlaps the arithmetic of group g+1.  Each thread
// evaluates a 4 x 4 micro-tile of grid points with 128-bit shared loads,
// looping over the frames; its float32 sums over the segment's groups are added
// to the float64 accumulators when the segment ends.  Warps whose 32 x 16
// sub-tile lies outside the domain skip the arithmetic.
//
// Domains: one channel (cross = 0): 0 <= k <= l, k + l <= M-1 (the rest follows
// from S3(k, l) = S3(l, k), Sec. 9).  Several channels (cross = 1):
// -(M-1) <= k <= M-1, 0 <= l <= M-1, |k + l| <= M-1, using X_{-k} = X_k*; tiles
// that reach negative bins are staged by the threads (conjugated), not by TMA.
#include "internal.cuh"
#include "pipeline.cuh"

namespace ss {
namespace {

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

struct Stage {
  float2* a;  // [m][64]
  float2* b;  // [m][64]
  float2* c;  // [m][128]
};

__device__ __forceinline__ Stage stage_ptr(float2* base, int s, int m) {
  float2* p = base + (size_t)s * m * 4 * kTile;
  return Stage{p, p + m * kTile, p + 2 * m * kTile};
}

// bytes of a bulk copy of n coefficients starting at bin k0 of a row of Mp
__device__ __forceinline__ uint32_t seg_bytes(int k0, int n, int Mp) {
  const int len = min(n, Mp - k0);
  return len > 0 ? (uint32_t)len * sizeof(float2) : 0u;
}

__global__ void __launch_bounds__(kThreadsPair, 1)
k2_bispec(const float2* __restrict__ sa, const float2* __restrict__ sb,
          const float2* __restrict__ sc, int G, int m, int M, int Mp,
          const TileInfo* __restrict__ tiles, int n_tiles, int cross, float pref3,
          double* __restrict__ acc, long long plane, int koff, int* __restrict__ status) {
  extern __shared__ __align__(128) float4 smem_raw[];
  __shared__ __align__(8) uint64_t full[2];
  float2* sbase = reinterpret_cast<float2*>(smem_raw);
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tx = (warp & 1) * 8 + (lane & 7);     // 16 threads along k
  const int ty = (warp >> 1) * 4 + (lane >> 3);   // 16 threads along l
  const int kt = 4 * tx, lt = 4 * ty;

  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    fence_mbar_init();
  }
  for (int i = tid; i < 2 * m * 4 * kTile; i += blockDim.x) sbase[i] = make_float2(0.f, 0.f);
  fence_async_smem();
  __syncthreads();
  uint32_t phase = 0;  // bit s = parity of the next wait on stage s
  bool aborted = false;

  for_each_segment(tiles, n_tiles, G, blockIdx.x, gridDim.x, [&](int t, int ga, int gb) {
    if (aborted) return;
    const int k0 = tiles[t].k0, l0 = tiles[t].l0;
    const bool use_tma = k0 >= 0 && k0 + l0 >= 0;
    const int kw = k0 + 32 * (warp & 1), lw = l0 + 16 * (warp >> 1);
    bool active = false;
    for (int a = 0; a < 32 && !active; ++a)
      for (int b = 0; b < 16 && !active; ++b) active = in_domain3(kw + a, lw + b, M, cross);

    const uint32_t ba = seg_bytes(k0, kTile, Mp), bb = seg_bytes(l0, kTile, Mp);
    const uint32_t bc = use_tma ? seg_bytes(k0 + l0, 2 * kTile, Mp) : 0u;
    auto issue = [&](int s, int g) {
      const Stage st = stage_ptr(sbase, s, m);
      mbar_arrive_expect_tx(&full[s], (uint32_t)m * (ba + bb + bc));
      for (int j = 0; j < m; ++j) {
        const long long r = ((long long)g * m + j) * Mp;
        if (ba) tma_load_1d(st.a + j * kTile, sa + r + k0, ba, &full[s]);
        if (bb) tma_load_1d(st.b + j * kTile, sb + r + l0, bb, &full[s]);
        if (bc) tma_load_1d(st.c + j * 2 * kTile, sc + r + k0 + l0, bc, &full[s]);
      }
    };

    float sr[16], si[16], qr[16], qi[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) sr[i] = si[i] = qr[i] = qi[i] = 0.f;

    if (use_tma && tid == 0) {
      fence_async_smem();
      issue(0, ga);
      if (ga + 1 < gb) issue(1, ga + 1);
    }
    for (int g = ga; g < gb; ++g) {
      const int s = (g - ga) & 1;
      const Stage st = stage_ptr(sbase, s, m);
      bool ok = true;
      if (use_tma) {
        ok = mbar_wait_bounded(&full[s], (phase >> s) & 1u, status);
        phase ^= 1u << s;
      } else {
        const long long gbase = (long long)g * m * Mp;
        for (int idx = tid; idx < m * 4 * kTile; idx += blockDim.x) {
          const int j = idx / (4 * kTile);
          const int e = idx - j * 4 * kTile;
          const long long r = gbase + (long long)j * Mp;
          if (e < kTile) st.a[j * kTile + e] = coef(sa + r, k0 + e, M);
          else if (e < 2 * kTile) st.b[j * kTile + e - kTile] = coef(sb + r, l0 + e - kTile, M);
          else st.c[j * 2 * kTile + e - 2 * kTile] = coef(sc + r, k0 + l0 + e - 2 * kTile, M);
        }
        __syncthreads();
      }
      if (active) {
        float ar[16], ai[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) ar[i] = ai[i] = 0.f;
#pragma unroll 2
        for (int j = 0; j < m; ++j) {
          const float4* pa = reinterpret_cast<const float4*>(st.a + j * kTile + kt);
          const float4* pb = reinterpret_cast<const float4*>(st.b + j * kTile + lt);
          const float4* pc = reinterpret_cast<const float4*>(st.c + j * 2 * kTile + kt + lt);
          const float4 a01 = pa[0], a23 = pa[1], b01 = pb[0], b23 = pb[1];
          const float4 c01 = pc[0], c23 = pc[1], c45 = pc[2], c67 = pc[3];
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
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float vr = ar[i] * pref3, vi = ai[i] * pref3;
          sr[i] += vr;
          si[i] += vi;
          qr[i] = fmaf(vr, vr, qr[i]);
          qi[i] = fmaf(vi, vi, qi[i]);
        }
      }
      // every thread is done with stage s; a failed wait anywhere stops the CTA
      if (__syncthreads_or(!ok)) {
        // drain the other stage's copy, if one is in flight, then give up
        if (use_tma && g + 1 < gb) mbar_wait_bounded(&full[s ^ 1], (phase >> (s ^ 1)) & 1u, status);
        aborted = true;
        return;
      }
      if (use_tma && tid == 0 && g + 2 < gb) {
        fence_async_smem();
        issue(s, g + 2);
      }
    }
    if (!active) return;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int k = k0 + kt + a, l = l0 + lt + b;
        if (!in_domain3(k, l, M, cross)) continue;
        const long long o = (long long)(k + koff) * M + l;
        const int i = a * 4 + b;
        atomicAdd(acc + o, (double)sr[i]);
        atomicAdd(acc + plane + o, (double)si[i]);
        atomicAdd(acc + 2 * plane + o, (double)qr[i]);
        atomicAdd(acc + 3 * plane + o, (double)qi[i]);
      }
    }
  });
}

}  // namespace

cudaError_t launch_k2_bispec(const float2* spec_a, const float2* spec_b, const float2* spec_c,
                             int G, int m, int M, int Mp, const TileInfo* tiles, int n_tiles,
                             int cross, float pref3, double* acc, long long plane, int rows,
                             int nsm, int* status, cudaStream_t stream) {
  if (G <= 0 || n_tiles <= 0) return cudaSuccess;
  const size_t smem = (size_t)2 * m * 4 * kTile * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k2_bispec, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k2_bispec, kThreadsPair, smem);
  if (e != cudaSuccess) return e;
  const int n_cta = nsm * (occ > 0 ? occ : 1);
  const int koff = (rows == M) ? 0 : (M - 1);
  k2_bispec<<<n_cta, kThreadsPair, smem, stream>>>(spec_a, spec_b, spec_c, G, m, M, Mp, tiles,
                                                   n_tiles, cross, pref3, acc, plane, koff,
                                                   status);
  return cudaGetLastError();
}

}  // namespace ss
