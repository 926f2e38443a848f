// k_trispec_cross.cu -- K3 for several channels: per-group trispectrum-cut
// k-statistics C4(a_k, b_k*, c_l, d_l*) (Sec. 7, Eq. 50) on CUDA cores (FP32).
//
// Domain: k in [-(M-1), M-1] (row r = k + M - 1 of the output grid), l in
// [0, M-1], with a_{-k} = a_k* (real channels).  With centred coefficients and,
// per group, x_j = da_jk, y_j = db_jk*, z_j = dc_jl, w_j = dd_jl*, the
// factorised estimator of App. H, Eq. 85 is
//   c4 = [m(m+1) sum xyzw - (m-1)(sum xy sum zw + sum xz sum yw + sum xw sum yz)]
//        / ((m-1)(m-2)(m-3)),
// all sums over the group's m frames and all products complex.  Per grid point
// and frame that is five complex multiply-adds (20 FFMA); sum xy and sum zw
// depend on one bin only.  The cut is complex for distinct channels, so the
// real and imaginary parts, their sums and their sums of squares over groups
// are accumulated (Eq. 35-36).
//
// Work split: CTA = (16 x 64 tile of (r, l), run of groups, combination).
// Chunks of up to 16 frames of the four channels' coefficients are staged in
// shared memory as x, y, xy for the tile's 16 rows and z, w, zw for its 64
// columns; each thread evaluates 1 row x 4 columns.  Sums over groups stay in
// FP32 registers for at most kFlushGroups groups, then go to the float64
// accumulators with atomics.
#include "internal.cuh"

namespace ss {
namespace {

constexpr int kRT = 16, kLT = 64, kFrames = 16, kThreads = 256, kFlushGroups = 64;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

__global__ void __launch_bounds__(kThreads, 2)
k3_trispec_cross(const float2* __restrict__ spec, long long chan_stride, int G, int m, int M,
                 int Mp, const int4* __restrict__ combos, int tiles_l, int groups_per_cta,
                 float pref, float fmm, float fm1, double* __restrict__ acc, long long plane,
                 long long combo_stride) {
  __shared__ __align__(16) float2 sx[kFrames][kRT], sy[kFrames][kRT], sxy[kFrames][kRT];
  __shared__ __align__(16) float2 sz[kFrames][kLT], sw[kFrames][kLT], szw[kFrames][kLT];
  const int tid = threadIdx.x;
  const int tile = blockIdx.x;
  const int r0 = (tile / tiles_l) * kRT, l0 = (tile % tiles_l) * kLT;
  const int g0 = blockIdx.y * groups_per_cta;
  const int g1 = min(G, g0 + groups_per_cta);
  if (g0 >= g1) return;
  const int4 cb = combos[blockIdx.z];
  const float2* A = spec + cb.x * chan_stride;
  const float2* B = spec + cb.y * chan_stride;
  const float2* C = spec + cb.z * chan_stride;
  const float2* D = spec + cb.w * chan_stride;
  const int rows = 2 * M - 1;
  const int ti = tid & (kRT - 1), tj = tid >> 4;  // row ti, columns 4 tj .. 4 tj + 3
  const int r = r0 + ti, lc = l0 + 4 * tj;

  float sre[4], sim[4], qre[4], qim[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) sre[i] = sim[i] = qre[i] = qim[i] = 0.f;
  int since_flush = 0;

  auto flush = [&]() {
    if (r < rows) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int l = lc + i;
        if (l < M) {
          const long long o = (long long)blockIdx.z * combo_stride + (long long)r * M + l;
          atomicAdd(acc + o, (double)sre[i]);
          atomicAdd(acc + plane + o, (double)sim[i]);
          atomicAdd(acc + 2 * plane + o, (double)qre[i]);
          atomicAdd(acc + 3 * plane + o, (double)qim[i]);
        }
        sre[i] = sim[i] = qre[i] = qim[i] = 0.f;
      }
    }
  };

  for (int g = g0; g < g1; ++g) {
    float2 a_xyzw[4], a_xz[4], a_yw[4], a_xw[4], a_yz[4], a_zw[4], a_xy;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      a_xyzw[i] = a_xz[i] = a_yw[i] = a_xw[i] = a_yz[i] = a_zw[i] = make_float2(0.f, 0.f);
    a_xy = make_float2(0.f, 0.f);
    const long long gbase = (long long)g * m * Mp;
    for (int f0 = 0; f0 < m; f0 += kFrames) {
      const int nf = min(kFrames, m - f0);
      __syncthreads();  // the previous chunk has been read
      for (int idx = tid; idx < nf * kRT; idx += kThreads) {
        const int f = idx / kRT, i = idx - f * kRT;
        const int rr = r0 + i, k = rr - (M - 1);
        float2 x = make_float2(0.f, 0.f), y = x;
        if (rr < rows) {
          const int kb = k < 0 ? -k : k;
          const long long o = gbase + (long long)(f0 + f) * Mp + kb;
          float2 va = A[o], vb = B[o];
          if (k < 0) {
            va = conjf2(va);
            vb = conjf2(vb);
          }
          x = va;
          y = conjf2(vb);
        }
        sx[f][i] = x;
        sy[f][i] = y;
        sxy[f][i] = cmul(x, y);
      }
      for (int idx = tid; idx < nf * kLT; idx += kThreads) {
        const int f = idx / kLT, i = idx - f * kLT;
        const int l = l0 + i;
        float2 z = make_float2(0.f, 0.f), w = z;
        if (l < M) {
          const long long o = gbase + (long long)(f0 + f) * Mp + l;
          z = C[o];
          w = conjf2(D[o]);
        }
        sz[f][i] = z;
        sw[f][i] = w;
        szw[f][i] = cmul(z, w);
      }
      __syncthreads();
      for (int f = 0; f < nf; ++f) {
        const float2 x = sx[f][ti], y = sy[f][ti], xy = sxy[f][ti];
        const float4 z01 = *reinterpret_cast<const float4*>(&sz[f][4 * tj]);
        const float4 z23 = *reinterpret_cast<const float4*>(&sz[f][4 * tj + 2]);
        const float4 w01 = *reinterpret_cast<const float4*>(&sw[f][4 * tj]);
        const float4 w23 = *reinterpret_cast<const float4*>(&sw[f][4 * tj + 2]);
        const float4 p01 = *reinterpret_cast<const float4*>(&szw[f][4 * tj]);
        const float4 p23 = *reinterpret_cast<const float4*>(&szw[f][4 * tj + 2]);
        const float2 zz[4] = {make_float2(z01.x, z01.y), make_float2(z01.z, z01.w),
                              make_float2(z23.x, z23.y), make_float2(z23.z, z23.w)};
        const float2 ww[4] = {make_float2(w01.x, w01.y), make_float2(w01.z, w01.w),
                              make_float2(w23.x, w23.y), make_float2(w23.z, w23.w)};
        const float2 pp[4] = {make_float2(p01.x, p01.y), make_float2(p01.z, p01.w),
                              make_float2(p23.x, p23.y), make_float2(p23.z, p23.w)};
        a_xy.x += xy.x;
        a_xy.y += xy.y;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          cmac(a_xyzw[i], xy, pp[i]);
          cmac(a_xz[i], x, zz[i]);
          cmac(a_yw[i], y, ww[i]);
          cmac(a_xw[i], x, ww[i]);
          cmac(a_yz[i], y, zz[i]);
          a_zw[i].x += pp[i].x;
          a_zw[i].y += pp[i].y;
        }
      }
    }
    // c4 of this group at the thread's four points
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 t = cmul(a_xy, a_zw[i]);
      cmac(t, a_xz[i], a_yw[i]);
      cmac(t, a_xw[i], a_yz[i]);
      const float cr = pref * fmaf(fmm, a_xyzw[i].x, -fm1 * t.x);
      const float ci = pref * fmaf(fmm, a_xyzw[i].y, -fm1 * t.y);
      sre[i] += cr;
      sim[i] += ci;
      qre[i] = fmaf(cr, cr, qre[i]);
      qim[i] = fmaf(ci, ci, qim[i]);
    }
    if (++since_flush == kFlushGroups) {
      flush();
      since_flush = 0;
    }
  }
  if (since_flush) flush();
}

}  // namespace

cudaError_t launch_k3_trispec_cross(const float2* spec, long long chan_stride, int G, int m, int M,
                                    int Mp, const int4* combos, int n_combos, double* acc,
                                    long long plane, int nsm, bool natural, cudaStream_t stream) {
  if (G <= 0 || n_combos <= 0) return cudaSuccess;
  const int rows = 2 * M - 1;
  const int tiles_r = (rows + kRT - 1) / kRT, tiles_l = (M + kLT - 1) / kLT;
  const long long tiles = (long long)tiles_r * tiles_l;
  // enough CTAs for about four waves of two CTAs per SM
  long long chunks = (8ll * nsm + tiles * n_combos - 1) / (tiles * n_combos);
  if (chunks < 1) chunks = 1;
  if (chunks > G) chunks = G;
  if (chunks > 65535) chunks = 65535;
  const int gpc = (int)((G + chunks - 1) / chunks);
  chunks = (G + gpc - 1) / gpc;
  if (tiles > 0x7fffffffll || n_combos > 65535) return cudaErrorInvalidValue;
  const double md = m;
  // c4 = pref [fmm sum xyzw - fm1 (sum xy sum zw + ...)]: the k-statistic (Eq. 85),
  // or the natural estimator 1/m sum xyzw - 1/m^2 (...)
  const float pref =
      (float)(natural ? 1.0 / (md * md) : 1.0 / ((md - 1.0) * (md - 2.0) * (md - 3.0)));
  const float fmm = (float)(natural ? md : md * (md + 1.0));
  const float fm1 = (float)(natural ? 1.0 : md - 1.0);
  dim3 grid((unsigned)tiles, (unsigned)chunks, (unsigned)n_combos);
  k3_trispec_cross<<<grid, kThreads, 0, stream>>>(spec, chan_stride, G, m, M, Mp, combos, tiles_l,
                                                  gpc, pref, fmm, fm1, acc, plane,
                                                  (long long)rows * M);
  return cudaGetLastError();
}

}  // namespace ss
