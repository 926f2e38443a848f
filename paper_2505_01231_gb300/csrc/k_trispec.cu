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
// length-m dot products per grid point and group.  Work split as in K2: a
// persistent CTA walks balanced (64 x 64 tile of the upper triangle k <= l,
// group range) segments; the m frames' coefficients at k0.. and l0.. arrive by
// 1-D TMA bulk copies into two shared-memory stages; 4 x 4 micro-tiles.
#include "internal.cuh"
#include "pipeline.cuh"

namespace ss {
namespace {

__device__ __forceinline__ uint32_t seg_bytes(int k0, int n, int Mp) {
  const int len = min(n, Mp - k0);
  return len > 0 ? (uint32_t)len * sizeof(float2) : 0u;
}

__global__ void __launch_bounds__(kThreadsPair, 1)
k3_trispec(const float2* __restrict__ spec, int G, int m, int M, int Mp,
           const TileInfo* __restrict__ tiles, int n_tiles, float pref_a, float pref_b,
           double* __restrict__ acc, long long plane, int* __restrict__ status) {
  extern __shared__ __align__(128) float4 smem_raw[];
  __shared__ __align__(8) uint64_t full[2];
  float2* sbase = reinterpret_cast<float2*>(smem_raw);       // 2 stages x [2][m][64] float2
  float* pA = reinterpret_cast<float*>(sbase + 2 * 2 * m * kTile);  // [m][64]
  float* pB = pA + m * kTile;                                        // [m][64]
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int tx = (warp & 1) * 8 + (lane & 7);
  const int ty = (warp >> 1) * 4 + (lane >> 3);
  const int kt = 4 * tx, lt = 4 * ty;

  if (tid == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    fence_mbar_init();
  }
  for (int i = tid; i < 2 * 2 * m * kTile; i += blockDim.x) sbase[i] = make_float2(0.f, 0.f);
  fence_async_smem();
  __syncthreads();
  uint32_t phase = 0;
  bool aborted = false;

  for_each_segment(tiles, n_tiles, G, blockIdx.x, gridDim.x, [&](int t, int ga, int gb) {
    if (aborted) return;
    const int k0 = tiles[t].k0, l0 = tiles[t].l0;
    const int kw = k0 + 32 * (warp & 1), lw = l0 + 16 * (warp >> 1);
    const bool active = (kw <= lw + 15) && (lw < M) && (kw < M);
    const uint32_t ba = seg_bytes(k0, kTile, Mp), bb = seg_bytes(l0, kTile, Mp);
    auto issue = [&](int s, int g) {
      float2* sa = sbase + (size_t)s * 2 * m * kTile;
      float2* sb = sa + m * kTile;
      mbar_arrive_expect_tx(&full[s], (uint32_t)m * (ba + bb));
      for (int j = 0; j < m; ++j) {
        const long long r = ((long long)g * m + j) * Mp;
        if (ba) tma_load_1d(sa + j * kTile, spec + r + k0, ba, &full[s]);
        if (bb) tma_load_1d(sb + j * kTile, spec + r + l0, bb, &full[s]);
      }
    };

    float sum[16], sq[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) sum[i] = sq[i] = 0.f;
    if (tid == 0) {
      fence_async_smem();
      issue(0, ga);
      if (ga + 1 < gb) issue(1, ga + 1);
    }
    for (int g = ga; g < gb; ++g) {
      const int s = (g - ga) & 1;
      const float2* sA = sbase + (size_t)s * 2 * m * kTile;
      const float2* sB = sA + m * kTile;
      const bool ok = mbar_wait_bounded(&full[s], (phase >> s) & 1u, status);
      phase ^= 1u << s;
      for (int i = tid; i < 2 * m * kTile; i += blockDim.x) {
        const float2 v = sA[i];  // sA and sB are contiguous: [2][m][64]
        const float p = fmaf(v.x, v.x, v.y * v.y);
        if (i < m * kTile) pA[i] = p; else pB[i - m * kTile] = p;
      }
      __syncthreads();
      if (active) {
        float q[16], rr[16], ii[16], xx[16], xt[16], sk[4], sl[4];
#pragma unroll
        for (int i = 0; i < 16; ++i) q[i] = rr[i] = ii[i] = xx[i] = xt[i] = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) sk[i] = sl[i] = 0.f;
#pragma unroll 2
        for (int j = 0; j < m; ++j) {
          const float4* a4 = reinterpret_cast<const float4*>(sA + j * kTile + kt);
          const float4* b4 = reinterpret_cast<const float4*>(sB + j * kTile + lt);
          const float4 a01 = a4[0], a23 = a4[1], b01 = b4[0], b23 = b4[1];
          const float4 pk4 = *reinterpret_cast<const float4*>(pA + j * kTile + kt);
          const float4 pl4 = *reinterpret_cast<const float4*>(pB + j * kTile + lt);
          const float2 ak[4] = {{a01.x, a01.y}, {a01.z, a01.w}, {a23.x, a23.y}, {a23.z, a23.w}};
          const float2 al[4] = {{b01.x, b01.y}, {b01.z, b01.w}, {b23.x, b23.y}, {b23.z, b23.w}};
          const float pk[4] = {pk4.x, pk4.y, pk4.z, pk4.w};
          const float pl[4] = {pl4.x, pl4.y, pl4.z, pl4.w};
#pragma unroll
          for (int a = 0; a < 4; ++a) {
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
      if (__syncthreads_or(!ok)) {
        if (g + 1 < gb) mbar_wait_bounded(&full[s ^ 1], (phase >> (s ^ 1)) & 1u, status);
        aborted = true;
        return;
      }
      if (tid == 0 && g + 2 < gb) {
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
        if (k > l || l >= M) continue;
        const long long o = (long long)k * M + l;
        atomicAdd(acc + o, (double)sum[a * 4 + b]);
        atomicAdd(acc + 2 * plane + o, (double)sq[a * 4 + b]);
      }
    }
  });
}

}  // namespace

cudaError_t launch_k3_trispec(const float2* spec, int G, int m, int M, int Mp,
                              const TileInfo* tiles, int n_tiles, float pref4a, float pref4b,
                              double* acc, long long plane, int nsm, int* status,
                              cudaStream_t stream) {
  if (G <= 0 || n_tiles <= 0) return cudaSuccess;
  const size_t smem = (size_t)2 * 2 * m * kTile * sizeof(float2) +
                      (size_t)2 * m * kTile * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k3_trispec, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k3_trispec, kThreadsPair, smem);
  if (e != cudaSuccess) return e;
  const int n_cta = nsm * (occ > 0 ? occ : 1);
  k3_trispec<<<n_cta, kThreadsPair, smem, stream>>>(spec, G, m, M, Mp, tiles, n_tiles, pref4a,
                                                    pref4b, acc, plane, status);
  return cudaGetLastError();
}

}  // namespace ss
