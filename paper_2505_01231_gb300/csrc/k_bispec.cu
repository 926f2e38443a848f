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
// Work split: a CTA owns one 64 x 64 tile of (k, l) and a contiguous range of
// groups.  Per group it stages the m frames' coefficients at k, at l and at
// k + l in shared memory, then each thread evaluates a 4 x 4 micro-tile of grid
// points, looping over the frames with the group sums in registers.  Warps whose
// 32 x 16 sub-tile lies entirely outside the domain skip the arithmetic.
// At the end the CTA adds its float32 partial sums to the float64 accumulators.
//
// Domains: one channel (cross = 0): 0 <= k <= l, k + l <= M-1 (the rest follows
// from S3(k, l) = S3(l, k), Sec. 9).  Several channels (cross = 1):
// -(M-1) <= k <= M-1, 0 <= l <= M-1, |k + l| <= M-1, using X_{-k} = X_k*.
#include "internal.cuh"

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

__global__ void __launch_bounds__(kThreadsPair)
k2_bispec(const float2* __restrict__ sa, const float2* __restrict__ sb,
          const float2* __restrict__ sc, int G, int m, int M, int Mp,
          const int2* __restrict__ tiles, int cross, int groups_per_cta, float pref3,
          double* __restrict__ acc, long long plane, int koff) {
  extern __shared__ float4 smem_raw[];
  float2* sA = reinterpret_cast<float2*>(smem_raw);   // [m][64]   coefficients at k
  float2* sB = sA + m * kTile;                          // [m][64]   at l
  float2* sC = sB + m * kTile;                          // [m][128]  at k + l

  const int2 tile = tiles[blockIdx.x];
  const int k0 = tile.x, l0 = tile.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tx = (warp & 1) * 8 + (lane & 7);     // 16 threads along k
  const int ty = (warp >> 1) * 4 + (lane >> 3);   // 16 threads along l
  const int kt = 4 * tx, lt = 4 * ty;

  // does this warp's 32 x 16 sub-tile touch the domain?
  bool active = false;
  {
    const int kw = k0 + 32 * (warp & 1), lw = l0 + 16 * (warp >> 1);
    for (int a = 0; a < 32 && !active; ++a)
      for (int b = 0; b < 16 && !active; ++b) active = in_domain3(kw + a, lw + b, M, cross);
  }

  float sr[16], si[16], qr[16], qi[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) sr[i] = si[i] = qr[i] = qi[i] = 0.f;

  const int g0 = blockIdx.y * groups_per_cta;
  const int g1 = min(G, g0 + groups_per_cta);
  for (int g = g0; g < g1; ++g) {
    __syncthreads();
    const long long gbase = (long long)g * m * Mp;
    for (int idx = threadIdx.x; idx < m * 4 * kTile; idx += blockDim.x) {
      const int j = idx / (4 * kTile);
      const int e = idx - j * 4 * kTile;
      const long long r = gbase + (long long)j * Mp;
      if (e < kTile) {
        sA[j * kTile + e] = coef(sa + r, k0 + e, M);
      } else if (e < 2 * kTile) {
        sB[j * kTile + e - kTile] = coef(sb + r, l0 + e - kTile, M);
      } else {
        sC[j * 2 * kTile + e - 2 * kTile] = coef(sc + r, k0 + l0 + e - 2 * kTile, M);
      }
    }
    __syncthreads();
    if (!active) continue;

    float ar[16], ai[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) ar[i] = ai[i] = 0.f;
    for (int j = 0; j < m; ++j) {
      float2 ak[4], al[4], ac[7];
#pragma unroll
      for (int a = 0; a < 4; ++a) ak[a] = sA[j * kTile + kt + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) al[b] = sB[j * kTile + lt + b];
#pragma unroll
      for (int d = 0; d < 7; ++d) ac[d] = sC[j * 2 * kTile + kt + lt + d];
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
}

}  // namespace

cudaError_t launch_k2_bispec(const float2* spec_a, const float2* spec_b, const float2* spec_c,
                             int G, int m, int M, int Mp, const int2* tiles, int n_tiles,
                             int cross, int group_splits, float pref3, double* acc,
                             long long plane, int rows, cudaStream_t stream) {
  if (G <= 0 || n_tiles <= 0) return cudaSuccess;
  if (group_splits > G) group_splits = G;
  const int gpc = (G + group_splits - 1) / group_splits;
  const int splits = (G + gpc - 1) / gpc;
  const size_t smem = (size_t)m * 4 * kTile * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k2_bispec, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int koff = (rows == M) ? 0 : (M - 1);
  dim3 grid(n_tiles, splits);
  k2_bispec<<<grid, kThreadsPair, smem, stream>>>(spec_a, spec_b, spec_c, G, m, M, Mp, tiles,
                                                  cross, gpc, pref3, acc, plane, koff);
  return cudaGetLastError();
}

}  // namespace ss
