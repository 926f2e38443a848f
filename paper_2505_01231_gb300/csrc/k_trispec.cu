// k_trispec.cu -- K3: per-group trispectrum-cut k-statistics on CUDA cores (FP32).
//
// Single channel, cumulant arguments (x, y, z, w) = (a_k, a_k*, a_l, a_l*) of
// Eq. 31.  With centred coefficients da = ar + j ai (K1) and, per group,
//   SQ  = sum_j P_jk P_jl           (P = |da|^2)
//   Sk  = sum_j P_jk, Sl = sum_j P_jl
//   RR  = sum_j ar_k ar_l,  II = sum_j ai_k ai_l,
//   X   = sum_j ar_k ai_l,  Xt = sum_j ai_k ar_l,
// the factorised estimator of App. H, Eq. 85 becomes
//   c4 = [m(m+1) SQ - (m-1)(Sk Sl + |U|^2 + |V|^2)] / ((m-1)(m-2)(m-3)),
// because mean(dx dy) mean(dz dw) = Sk Sl / m^2, mean(dx dz) mean(dy dw) =
// |U|^2 / m^2 with U = sum_j da_k da_l, mean(dx dw) mean(dy dz) = |V|^2 / m^2 with
// V = sum_j da_k da_l*, and |U|^2 + |V|^2 = 2 (RR^2 + II^2 + X^2 + Xt^2).
// The cut is real for a real channel (Sec. 9), so only the real part, its sum
// and its sum of squares over groups are accumulated (Eq. 35-36).
//
// This is the plain FP32 CUDA-core form of the fourth-order moment sums: five
// length-m dot products per grid point and group.  Work split as in K2: 64 x 64
// tiles of the upper triangle k <= l, 4 x 4 micro-tiles per thread.
#include "internal.cuh"

namespace ss {
namespace {

__global__ void __launch_bounds__(kThreadsPair)
k3_trispec(const float2* __restrict__ spec, int G, int m, int M, int Mp,
           const int2* __restrict__ tiles, int groups_per_cta, float pref_a, float pref_b,
           double* __restrict__ acc, long long plane) {
  extern __shared__ float4 smem_raw[];
  float2* sA = reinterpret_cast<float2*>(smem_raw);   // [m][64] da at k
  float2* sB = sA + m * kTile;                          // [m][64] da at l
  float* pA = reinterpret_cast<float*>(sB + m * kTile); // [m][64] |da|^2 at k
  float* pB = pA + m * kTile;                           // [m][64] |da|^2 at l

  const int2 tile = tiles[blockIdx.x];
  const int k0 = tile.x, l0 = tile.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tx = (warp & 1) * 8 + (lane & 7);
  const int ty = (warp >> 1) * 4 + (lane >> 3);
  const int kt = 4 * tx, lt = 4 * ty;
  const int kw = k0 + 32 * (warp & 1), lw = l0 + 16 * (warp >> 1);
  // sub-tile touches k <= l, l < M ?
  const bool active = (kw <= lw + 15) && (lw < M) && (kw < M);

  float sum[16], sq[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) sum[i] = sq[i] = 0.f;

  const int g0 = blockIdx.y * groups_per_cta;
  const int g1 = min(G, g0 + groups_per_cta);
  for (int g = g0; g < g1; ++g) {
    __syncthreads();
    const long long gbase = (long long)g * m * Mp;
    for (int idx = threadIdx.x; idx < m * 2 * kTile; idx += blockDim.x) {
      const int j = idx / (2 * kTile);
      const int e = idx - j * 2 * kTile;
      const float2* row = spec + gbase + (long long)j * Mp;
      const int k = (e < kTile) ? k0 + e : l0 + e - kTile;
      const float2 v = (k < M) ? row[k] : make_float2(0.f, 0.f);
      const float p = fmaf(v.x, v.x, v.y * v.y);
      if (e < kTile) {
        sA[j * kTile + e] = v;
        pA[j * kTile + e] = p;
      } else {
        sB[j * kTile + e - kTile] = v;
        pB[j * kTile + e - kTile] = p;
      }
    }
    __syncthreads();
    if (!active) continue;

    float q[16], rr[16], ii[16], xx[16], xt[16], sk[4], sl[4];
#pragma unroll
    for (int i = 0; i < 16; ++i) q[i] = rr[i] = ii[i] = xx[i] = xt[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) sk[i] = sl[i] = 0.f;
    for (int j = 0; j < m; ++j) {
      float2 ak[4], al[4];
      float pk[4], pl[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        ak[a] = sA[j * kTile + kt + a];
        pk[a] = pA[j * kTile + kt + a];
        al[a] = sB[j * kTile + lt + a];
        pl[a] = pB[j * kTile + lt + a];
        sk[a] += pk[a];
        sl[a] += pl[a];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = a * 4 + b;
          q[i] = fmaf(pk[a], pl[b], q[i]);
          rr[i] = fmaf(ak[a].x, al[b].x, rr[i]);
          ii[i] = fmaf(ak[a].y, al[b].y, ii[i]);
          xx[i] = fmaf(ak[a].x, al[b].y, xx[i]);
          xt[i] = fmaf(ak[a].y, al[b].x, xt[i]);
        }
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int i = a * 4 + b;
        float uv = fmaf(rr[i], rr[i], ii[i] * ii[i]);
        uv = fmaf(xx[i], xx[i], uv);
        uv = fmaf(xt[i], xt[i], uv);
        const float pair = fmaf(2.f, uv, sk[a] * sl[b]);
        const float c4 = fmaf(pref_a, q[i], -pref_b * pair);
        sum[i] += c4;
        sq[i] = fmaf(c4, c4, sq[i]);
      }
    }
  }

  if (!active) return;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int k = k0 + kt + a, l = l0 + lt + b;
      if (k > l || l >= M) continue;
      const long long o = (long long)k * M + l;
      atomicAdd(acc + o, (double)sum[a * 4 + b]);
      atomicAdd(acc + 2 * plane + o, (double)sq[a * 4 + b]);
    }
  }
}

}  // namespace

cudaError_t launch_k3_trispec(const float2* spec, int G, int m, int M, int Mp, const int2* tiles,
                              int n_tiles, int group_splits, float pref4a, float pref4b,
                              double* acc, long long plane, cudaStream_t stream) {
  if (G <= 0 || n_tiles <= 0) return cudaSuccess;
  if (group_splits > G) group_splits = G;
  const int gpc = (G + group_splits - 1) / group_splits;
  const int splits = (G + gpc - 1) / gpc;
  const size_t smem = (size_t)m * 2 * kTile * (sizeof(float2) + sizeof(float));
  cudaError_t e = cudaFuncSetAttribute(k3_trispec, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(n_tiles, splits);
  k3_trispec<<<grid, kThreadsPair, smem, stream>>>(spec, G, m, M, Mp, tiles, gpc, pref4a, pref4b,
                                                   acc, plane);
  return cudaGetLastError();
}

}  // namespace ss
