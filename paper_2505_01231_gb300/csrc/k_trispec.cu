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
// length-m dot products per grid point and group.  Work split as in K2:
// persistent CTAs take (group chunk, 64 x 64 tile of the upper triangle k <= l)
// items from a group-major queue; chunks of FC frames of the coefficients at
// k0.. and l0.. arrive by 128-byte-swizzled 3-D TMA box loads into kStages
// shared-memory stages, |da|^2 is formed once per staged chunk, and each thread
// evaluates a 4 x 4 micro-tile (quarter-warps of 4 k-threads x 2 l-threads).
#include <algorithm>

#include "internal.cuh"
#include "pipeline.cuh"

namespace ss {
namespace {

constexpr int kStages = 4;

__host__ __device__ __forceinline__ uint32_t arr64_bytes(int FC) {
  return ((uint32_t)FC * 512u + 1023u) & ~1023u;
}

__device__ __forceinline__ float4 lds128(const void* p) {
  return *reinterpret_cast<const float4*>(p);
}

__global__ void __launch_bounds__(kThreadsPair, 1)
k3_trispec(const __grid_constant__ CUtensorMap tm64, int row0, int G, int m, int FC, int M,
           const TileInfo* __restrict__ tiles, WorkQueue wq, float pref_a, float pref_b,
           double* __restrict__ acc, long long plane, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];  // + 1024 spare bytes
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ int s_item;
  unsigned char* sbase = align1024<unsigned char>(smem_raw);
  const uint32_t a64 = arr64_bytes(FC), sbytes = 2 * a64;   // stage: [FC][64] at k, at l
  float* pA = reinterpret_cast<float*>(sbase + kStages * sbytes);  // [FC][64] |da_k|^2
  float* pB = pA + FC * kTile;                                      // [FC][64] |da_l|^2
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int qw = lane >> 3, r8 = lane & 7;
  const int tx = (warp & 1) * 8 + (r8 & 3) + 4 * (qw & 1);
  const int ty = (warp >> 1) * 4 + (r8 >> 2) + 2 * (qw >> 1);
  const int kt = 4 * tx, lt = 4 * ty;
  const int nch = (m + FC - 1) / FC;
  const uint32_t oA0 = swz128(kt * 8), oA1 = swz128(kt * 8 + 16);
  const uint32_t oA0o = swz128(512 + kt * 8), oA1o = swz128(512 + kt * 8 + 16);
  const uint32_t oB0 = swz128(lt * 8), oB1 = swz128(lt * 8 + 16);
  const uint32_t oB0o = swz128(512 + lt * 8), oB1o = swz128(512 + lt * 8 + 16);

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  fence_async_smem();
  __syncthreads();
  uint32_t qbase = 0;

  for (int item; (item = next_item(wq, &s_item)) >= 0;) {
    const int t = item % wq.n_tiles;
    const int ga = (item / wq.n_tiles) * wq.group_chunk;
    const int gb = min(G, ga + wq.group_chunk);
    const int k0 = tiles[t].k0, l0 = tiles[t].l0;
    const int kw = k0 + 32 * (warp & 1), lw = l0 + 16 * (warp >> 1);
    const bool active = (kw <= lw + 15) && (lw < M) && (kw < M);
    const int nsteps = (gb - ga) * nch;
    auto issue = [&](int i) {
      const int s = (int)((qbase + i) % kStages);
      const int g = ga + i / nch, j0 = (i % nch) * FC;
      unsigned char* st = sbase + (size_t)s * sbytes;
      mbar_arrive_expect_tx(&full[s], (uint32_t)FC * 128u * 8u);
      tma_load_3d(st, &tm64, 0, k0 >> 4, row0 + g * m + j0, &full[s]);
      tma_load_3d(st + a64, &tm64, 0, l0 >> 4, row0 + g * m + j0, &full[s]);
    };

    float sum[16], sq[16], q[16], rr[16], ii[16], xx[16], xt[16], sk[4], sl[4];
#pragma unroll
    for (int i = 0; i < 16; ++i) sum[i] = sq[i] = q[i] = rr[i] = ii[i] = xx[i] = xt[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) sk[i] = sl[i] = 0.f;
    if (tid == 0) {
      fence_async_smem();
      for (int i = 0; i < kStages && i < nsteps; ++i) issue(i);
    }
    for (int i = 0; i < nsteps; ++i) {
      const int ch = i % nch;
      const int nf = min(FC, m - ch * FC);
      const int s = (int)((qbase + i) % kStages);
      const unsigned char* sA = sbase + (size_t)s * sbytes;
      const unsigned char* sB = sA + a64;
      const bool ok = mbar_wait_bounded(&full[s], ((qbase + i) / kStages) & 1u, status);
      for (int e = tid; e < 2 * FC * kTile; e += blockDim.x) {
        const int arr = e >= FC * kTile;
        const int rem = e - arr * FC * kTile;
        const int j = rem >> 6, bin = rem & 63;
        const float2 v = *reinterpret_cast<const float2*>(sA + arr * a64 + swz128(j * 512 + bin * 8));
        (arr ? pB : pA)[rem] = fmaf(v.x, v.x, v.y * v.y);
      }
      __syncthreads();
      if (active) {
        auto frame = [&](int j, uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1) {
          const unsigned char* pa = sA + (j & ~1) * 512;
          const unsigned char* pb = sB + (j & ~1) * 512;
          const float4 a01 = lds128(pa + a0), a23 = lds128(pa + a1);
          const float4 b01 = lds128(pb + b0), b23 = lds128(pb + b1);
          const float4 pk4 = lds128(pA + j * kTile + kt);
          const float4 pl4 = lds128(pB + j * kTile + lt);
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
              const int r = a * 4 + b;
              q[r] = fmaf(pk[a], pl[b], q[r]);
              rr[r] = fmaf(ak[a].x, al[b].x, rr[r]);
              ii[r] = fmaf(ak[a].y, al[b].y, ii[r]);
              xx[r] = fmaf(ak[a].x, al[b].y, xx[r]);
              xt[r] = fmaf(ak[a].y, al[b].x, xt[r]);
            }
          }
        };
        int j = 0;
        for (; j + 1 < nf; j += 2) {
          frame(j, oA0, oA1, oB0, oB1);
          frame(j + 1, oA0o, oA1o, oB0o, oB1o);
        }
        if (j < nf) frame(j, oA0, oA1, oB0, oB1);
        if (ch == nch - 1) {
#pragma unroll
          for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const int r = a * 4 + b;
              float uv = fmaf(rr[r], rr[r], ii[r] * ii[r]);
              uv = fmaf(xx[r], xx[r], uv);
              uv = fmaf(xt[r], xt[r], uv);
              const float pair = fmaf(2.f, uv, sk[a] * sl[b]);
              const float c4 = fmaf(pref_a, q[r], -pref_b * pair);
              sum[r] += c4;
              sq[r] = fmaf(c4, c4, sq[r]);
              q[r] = rr[r] = ii[r] = xx[r] = xt[r] = 0.f;
            }
          }
#pragma unroll
          for (int a = 0; a < 4; ++a) sk[a] = sl[a] = 0.f;
        }
      }
      if (__syncthreads_or(!ok)) {
        for (int r = i + 1; r < nsteps && r < i + kStages; ++r)
          mbar_wait_bounded(&full[(qbase + r) % kStages], ((qbase + r) / kStages) & 1u, status);
        return;
      }
      if (tid == 0 && i + kStages < nsteps) {
        fence_async_smem();
        issue(i + kStages);
      }
    }
    qbase += nsteps;
    if (!active) continue;
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
}

}  // namespace

size_t k3_smem_bytes(int FC) {
  return (size_t)kStages * 2 * arr64_bytes(FC) + (size_t)2 * FC * kTile * sizeof(float) + 1024;
}

cudaError_t launch_k3_trispec(const CUtensorMap& tm64, int row0, int G, int m, int FC, int M,
                              const TileInfo* tiles, int n_tiles, float pref4a, float pref4b,
                              double* acc, long long plane, int nsm, int* counter, int* status,
                              cudaStream_t stream) {
  if (G <= 0 || n_tiles <= 0) return cudaSuccess;
  const size_t smem = k3_smem_bytes(FC);
  // one fixed limit for the function (the attribute is shared by all launches)
  if (FC < 1 || FC > kMaxFC) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k3_trispec, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)k3_smem_bytes(kMaxFC));
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k3_trispec, kThreadsPair, smem);
  if (e != cudaSuccess) return e;
  const int n_cta = nsm * (occ > 0 ? occ : 1);
  WorkQueue wq;
  wq.counter = counter;
  wq.n_tiles = n_tiles;
  wq.group_chunk = work_group_chunk(G, n_tiles, n_cta);
  wq.n_items = n_tiles * ((G + wq.group_chunk - 1) / wq.group_chunk);
  e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  k3_trispec<<<n_cta, kThreadsPair, smem, stream>>>(tm64, row0, G, m, FC, M, tiles, wq, pref4a,
                                                    pref4b, acc, plane, status);
  return cudaGetLastError();
}

// The last column l = M - 1 of the one-channel cut for every k (the tensor-core
// tiles leave it out when it is the only column of its block): one thread per
// k, the same five length-m sums as above per group, reading the centred
// coefficients from global memory (consecutive k are consecutive addresses; the
// bin-l values are the same address across a warp).  Written at [l][k], the
// layout of the tensor-core kernel's accumulators.
constexpr int kColThreads = 128;

__global__ void __launch_bounds__(kColThreads)
k3_column(const float2* __restrict__ spec, int Mp, int G, int m, int M, float pref_a,
          float pref_b, double* __restrict__ acc, long long plane) {
  const int k = blockIdx.x * kColThreads + threadIdx.x;
  const int l = M - 1;
  if (k >= M) return;
  float sum = 0.f, sq = 0.f;
  for (int g = blockIdx.y; g < G; g += gridDim.y) {
    const float2* row = spec + (long long)g * m * Mp;
    float q = 0.f, sk = 0.f, sl = 0.f, rr = 0.f, ii = 0.f, xx = 0.f, xt = 0.f;
    for (int j = 0; j < m; ++j, row += Mp) {
      const float2 a = __ldg(row + k), b = __ldg(row + l);
      const float pk = fmaf(a.x, a.x, a.y * a.y), pl = fmaf(b.x, b.x, b.y * b.y);
      q = fmaf(pk, pl, q);
      sk += pk;
      sl += pl;
      rr = fmaf(a.x, b.x, rr);
      ii = fmaf(a.y, b.y, ii);
      xx = fmaf(a.x, b.y, xx);
      xt = fmaf(a.y, b.x, xt);
    }
    float uv = fmaf(rr, rr, ii * ii);
    uv = fmaf(xx, xx, uv);
    uv = fmaf(xt, xt, uv);
    const float pair = fmaf(2.f, uv, sk * sl);
    const float c4 = fmaf(pref_a, q, -pref_b * pair);
    sum += c4;
    sq = fmaf(c4, c4, sq);
  }
  const long long o = (long long)l * M + k;
  atomicAdd(acc + o, (double)sum);
  atomicAdd(acc + 2 * plane + o, (double)sq);
}

cudaError_t launch_k3_column(const float2* spec, int Mp, int G, int m, int M, float pref4a,
                             float pref4b, double* acc, long long plane, cudaStream_t stream) {
  if (G <= 0 || M <= 0) return cudaSuccess;
  const int gx = (M + kColThreads - 1) / kColThreads;
  // at most kMaxFp32Groups groups in a thread's float32 sums (grid y <= 65535)
  const int gy = std::min(G, std::min(65535, std::max(1024, (G + kMaxFp32Groups - 1) / kMaxFp32Groups)));
  k3_column<<<dim3((unsigned)gx, (unsigned)gy), kColThreads, 0, stream>>>(
      spec, Mp, G, m, M, pref4a, pref4b, acc, plane);
  return cudaGetLastError();
}

}  // namespace ss
