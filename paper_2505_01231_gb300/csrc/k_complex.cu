// k_complex.cu -- spectra of complex-valued signals (App. D) and S4 planes
// shifted off the cut (App. E), on CUDA cores (FP32, float64 across groups).
//
// A complex signal z = x + j y is carried as its two real channels, so K1's
// centred half spectra serve it: by the linearity of Eq. 18 and of the
// centring, the transform of z at a signed bin k is Z(k) = X(k) + j Y(k), with
// X(-k) = X(k)* for the real parts; the transform of z* at k is
// Z(-k)* = X(k) - j Y(k).  An operand is (real channel, imaginary channel or
// -1, conjugate flag): its value at k is X(k) + sigma j Y(k), sigma = +1 or -1.
// The k-statistics of Eq. 32-34 (App. H, Eq. 85 for the fourth order) are then
// taken directly over these complex samples -- the multilinear extension of
// Eq. 47, 48, 50 that App. D writes as sums of 4, 8 or 16 real spectra, formed
// here per group so that the error bars of Eq. 35-36 hold for the combination:
//   S2(k)    = c2(A(k), B(-k)),                      k in [-(M-1), M-1]
//   S3(k, l) = c3(A(k), B(l), C(-k-l)),              |k|, |l|, |k+l| <= M-1
//   S4(k, l) = c4(A(k+s), B(-k-s), C(l-s), D(-l+s)), |k|, |l| <= M-1
// (the window and dt normalisation is applied by K4).  s shifts the S4 plane
// of the 3-D trispectrum (App. E); bins are taken mod T (the transform of a
// frame is periodic in k).  Outputs: row r holds k = r - (M-1), column c holds
// l = c - (M-1).
//
// Work split: CTA = (tile, run of at most kMaxFp32Groups groups, combination).
// Per chunk of up to 16 frames the operands of the tile's rows and columns are
// formed in shared memory; each thread evaluates one row x four columns, with
// float32 sums over its groups flushed to the float64 accumulators.
#include <algorithm>

#include "internal.cuh"

namespace ss {
namespace {

constexpr int kRT = 16, kLT = 64, kFrames = 16, kThreads = 256;

__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void cmacc(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

// signed bin k wrapped into [-(T/2), T/2] (T = 2 (M - 1))
__device__ __forceinline__ int wrap_bin(int k, int M) {
  const int T = 2 * (M - 1);
  int r = (k + (M - 1)) % T;
  if (r < 0) r += T;
  return r - (M - 1);
}

// coefficient of a real channel's centred half spectrum at a signed bin
__device__ __forceinline__ float2 half_coef(const float2* __restrict__ row, int k) {
  if (k >= 0) return row[k];
  const float2 v = row[-k];
  return make_float2(v.x, -v.y);
}

// value of operand o (re channel, im channel or -1, sign of j) at signed bin k of
// frame row `off` (group g, frame j: (g m + j) Mp)
__device__ __forceinline__ float2 operand(const float2* __restrict__ spec, long long chan_stride,
                                          int4 o, long long off, int k, int M) {
  k = wrap_bin(k, M);
  float2 v = half_coef(spec + o.x * chan_stride + off, k);
  if (o.y >= 0) {
    const float2 w = half_coef(spec + o.y * chan_stride + off, k);
    // v + sigma j w
    v.x -= (float)o.z * w.y;
    v.y += (float)o.z * w.x;
  }
  return v;
}

__device__ __forceinline__ void flush4(double* __restrict__ acc, long long plane, long long o,
                                       float sr, float si, float qr, float qi) {
  atomicAdd(acc + o, (double)sr);
  atomicAdd(acc + plane + o, (double)si);
  atomicAdd(acc + 2 * plane + o, (double)qr);
  atomicAdd(acc + 3 * plane + o, (double)qi);
}

// S2: thread = (bin, combination), blockIdx.y = run of groups
__global__ void k5_cplx_s2(const float2* __restrict__ spec, long long chan_stride, int G, int m,
                           int M, int Mp, const int4* __restrict__ ops, int groups_per_cta,
                           float pref2, double* __restrict__ acc, long long plane) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int rows = 2 * M - 1;
  if (r >= rows) return;
  const int k = r - (M - 1);
  const int4 a = ops[2 * blockIdx.z], b = ops[2 * blockIdx.z + 1];
  const int g0 = blockIdx.y * groups_per_cta, g1 = min(G, g0 + groups_per_cta);
  float sr = 0.f, si = 0.f, qr = 0.f, qi = 0.f;
  for (int g = g0; g < g1; ++g) {
    float2 c = make_float2(0.f, 0.f);
    for (int j = 0; j < m; ++j) {
      const long long off = ((long long)g * m + j) * Mp;
      cmacc(c, operand(spec, chan_stride, a, off, k, M), operand(spec, chan_stride, b, off, -k, M));
    }
    c.x *= pref2;
    c.y *= pref2;
    sr += c.x;
    si += c.y;
    qr = fmaf(c.x, c.x, qr);
    qi = fmaf(c.y, c.y, qi);
  }
  flush4(acc, plane, (long long)blockIdx.z * rows + r, sr, si, qr, qi);
}

// S3 over the full plane: CTA = (16 x 64 tile, run of groups, combination)
__global__ void __launch_bounds__(kThreads)
k5_cplx_s3(const float2* __restrict__ spec, long long chan_stride, int G, int m, int M, int Mp,
           const int4* __restrict__ ops, int tiles_l, int groups_per_cta, float pref3,
           double* __restrict__ acc, long long plane) {
  __shared__ __align__(16) float2 sa[kFrames][kRT], sb[kFrames][kLT], sc[kFrames][kRT + kLT];
  const int tid = threadIdx.x;
  const int n = 2 * M - 1;
  const int r0 = (blockIdx.x / tiles_l) * kRT, c0 = (blockIdx.x % tiles_l) * kLT;
  const int g0 = blockIdx.y * groups_per_cta, g1 = min(G, g0 + groups_per_cta);
  if (g0 >= g1) return;
  const int4 oa = ops[3 * blockIdx.z], ob = ops[3 * blockIdx.z + 1], oc = ops[3 * blockIdx.z + 2];
  const int ti = tid & (kRT - 1), tj = tid >> 4;
  const int r = r0 + ti, k = r - (M - 1);
  float sr[4], si[4], qr[4], qi[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) sr[i] = si[i] = qr[i] = qi[i] = 0.f;
  const int kmin = r0 - (M - 1), lmin = c0 - (M - 1);
  for (int g = g0; g < g1; ++g) {
    float2 s[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) s[i] = make_float2(0.f, 0.f);
    for (int f0 = 0; f0 < m; f0 += kFrames) {
      const int nf = min(kFrames, m - f0);
      __syncthreads();  // the previous chunk has been read
      for (int idx = tid; idx < nf * (kRT + kLT + kRT + kLT); idx += kThreads) {
        const int f = idx / (2 * (kRT + kLT)), e = idx - f * 2 * (kRT + kLT);
        const long long off = ((long long)g * m + f0 + f) * Mp;
        if (e < kRT) {
          sa[f][e] = operand(spec, chan_stride, oa, off, kmin + e, M);
        } else if (e < kRT + kLT) {
          sb[f][e - kRT] = operand(spec, chan_stride, ob, off, lmin + e - kRT, M);
        } else {
          // C(-(k + l)) for k + l = kmin + lmin + q (q = ti + column, < kRT + kLT - 1)
          const int q = e - kRT - kLT;
          sc[f][q] = operand(spec, chan_stride, oc, off, -(kmin + lmin + q), M);
        }
      }
      __syncthreads();
      for (int f = 0; f < nf; ++f) {
        const float2 a = sa[f][ti];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int cl = 4 * tj + i;
          cmacc(s[i], cmulc(a, sb[f][cl]), sc[f][ti + cl]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float cr = s[i].x * pref3, ci = s[i].y * pref3;
      sr[i] += cr;
      si[i] += ci;
      qr[i] = fmaf(cr, cr, qr[i]);
      qi[i] = fmaf(ci, ci, qi[i]);
    }
  }
  if (r >= n) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int c = c0 + 4 * tj + i;
    const int l = c - (M - 1);
    if (c < n && abs(k + l) <= M - 1)
      flush4(acc, plane, (long long)blockIdx.z * n * n + (long long)r * n + c, sr[i], si[i], qr[i],
             qi[i]);
  }
}

// S4 plane over the full (k, l) plane: CTA = (16 x 64 tile, run of groups, combination)
__global__ void __launch_bounds__(kThreads)
k5_cplx_s4(const float2* __restrict__ spec, long long chan_stride, int G, int m, int M, int Mp,
           const int4* __restrict__ ops, int tiles_l, int groups_per_cta, int shift, float pref,
           float fmm, float fm1, double* __restrict__ acc, long long plane) {
  __shared__ __align__(16) float2 sx[kFrames][kRT], sy[kFrames][kRT], sxy[kFrames][kRT];
  __shared__ __align__(16) float2 sz[kFrames][kLT], sw[kFrames][kLT], szw[kFrames][kLT];
  const int tid = threadIdx.x;
  const int n = 2 * M - 1;
  const int r0 = (blockIdx.x / tiles_l) * kRT, c0 = (blockIdx.x % tiles_l) * kLT;
  const int g0 = blockIdx.y * groups_per_cta, g1 = min(G, g0 + groups_per_cta);
  if (g0 >= g1) return;
  const int4 oa = ops[4 * blockIdx.z], ob = ops[4 * blockIdx.z + 1];
  const int4 oc = ops[4 * blockIdx.z + 2], od = ops[4 * blockIdx.z + 3];
  const int ti = tid & (kRT - 1), tj = tid >> 4;
  const int r = r0 + ti;
  float sr[4], si[4], qr[4], qi[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) sr[i] = si[i] = qr[i] = qi[i] = 0.f;
  for (int g = g0; g < g1; ++g) {
    float2 a_xyzw[4], a_xz[4], a_yw[4], a_xw[4], a_yz[4], a_zw[4], a_xy;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      a_xyzw[i] = a_xz[i] = a_yw[i] = a_xw[i] = a_yz[i] = a_zw[i] = make_float2(0.f, 0.f);
    a_xy = make_float2(0.f, 0.f);
    for (int f0 = 0; f0 < m; f0 += kFrames) {
      const int nf = min(kFrames, m - f0);
      __syncthreads();  // the previous chunk has been read
      for (int idx = tid; idx < nf * (kRT + kLT); idx += kThreads) {
        const int f = idx / (kRT + kLT), e = idx - f * (kRT + kLT);
        const long long off = ((long long)g * m + f0 + f) * Mp;
        if (e < kRT) {
          const int k = r0 + e - (M - 1);
          const float2 x = operand(spec, chan_stride, oa, off, k + shift, M);
          const float2 y = operand(spec, chan_stride, ob, off, -k - shift, M);
          sx[f][e] = x;
          sy[f][e] = y;
          sxy[f][e] = cmulc(x, y);
        } else {
          const int l = c0 + e - kRT - (M - 1);
          const float2 z = operand(spec, chan_stride, oc, off, l - shift, M);
          const float2 w = operand(spec, chan_stride, od, off, -l + shift, M);
          sz[f][e - kRT] = z;
          sw[f][e - kRT] = w;
          szw[f][e - kRT] = cmulc(z, w);
        }
      }
      __syncthreads();
      for (int f = 0; f < nf; ++f) {
        const float2 x = sx[f][ti], y = sy[f][ti], xy = sxy[f][ti];
        a_xy.x += xy.x;
        a_xy.y += xy.y;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int cl = 4 * tj + i;
          const float2 z = sz[f][cl], w = sw[f][cl], zw = szw[f][cl];
          cmacc(a_xyzw[i], xy, zw);
          cmacc(a_xz[i], x, z);
          cmacc(a_yw[i], y, w);
          cmacc(a_xw[i], x, w);
          cmacc(a_yz[i], y, z);
          a_zw[i].x += zw.x;
          a_zw[i].y += zw.y;
        }
      }
    }
    // c4 (App. H, Eq. 85 with complex samples) at the thread's four points
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float2 t = cmulc(a_xy, a_zw[i]);
      cmacc(t, a_xz[i], a_yw[i]);
      cmacc(t, a_xw[i], a_yz[i]);
      const float cr = pref * fmaf(fmm, a_xyzw[i].x, -fm1 * t.x);
      const float ci = pref * fmaf(fmm, a_xyzw[i].y, -fm1 * t.y);
      sr[i] += cr;
      si[i] += ci;
      qr[i] = fmaf(cr, cr, qr[i]);
      qi[i] = fmaf(ci, ci, qi[i]);
    }
  }
  if (r >= n) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int c = c0 + 4 * tj + i;
    if (c < n)
      flush4(acc, plane, (long long)blockIdx.z * n * n + (long long)r * n + c, sr[i], si[i], qr[i],
             qi[i]);
  }
}

// runs of at most kMaxFp32Groups groups, enough CTAs for a few waves
int group_runs(int G, long long ctas_per_run, int nsm) {
  long long runs = (8ll * nsm + ctas_per_run - 1) / std::max(1ll, ctas_per_run);
  runs = std::max(runs, (long long)(G + kMaxFp32Groups - 1) / kMaxFp32Groups);
  runs = std::min<long long>(std::min<long long>(runs, G), 65535);
  return (int)std::max(1ll, runs);
}

}  // namespace

cudaError_t launch_k5_complex(const float2* spec, long long chan_stride, int G, int m, int M,
                              int Mp, int order, const int4* ops, int n_combos, int shift,
                              bool natural, double* acc, long long plane, int nsm,
                              cudaStream_t stream) {
  if (G <= 0 || n_combos <= 0) return cudaSuccess;
  if (n_combos > 65535) return cudaErrorInvalidValue;
  const double md = m;
  const int n = 2 * M - 1;
  if (order == 2) {
    const int bx = (n + 127) / 128;
    const int runs = group_runs(G, (long long)bx * n_combos, nsm);
    const int gpc = (G + runs - 1) / runs;
    const float pref2 = (float)(natural ? 1.0 / md : 1.0 / (md - 1.0));
    k5_cplx_s2<<<dim3(bx, (G + gpc - 1) / gpc, n_combos), 128, 0, stream>>>(
        spec, chan_stride, G, m, M, Mp, ops, gpc, pref2, acc, plane);
    return cudaGetLastError();
  }
  const int tiles_r = (n + kRT - 1) / kRT, tiles_l = (n + kLT - 1) / kLT;
  const long long tiles = (long long)tiles_r * tiles_l;
  if (tiles > 0x7fffffffll) return cudaErrorInvalidValue;
  const int runs = group_runs(G, tiles * n_combos, nsm);
  const int gpc = (G + runs - 1) / runs;
  const dim3 grid((unsigned)tiles, (unsigned)((G + gpc - 1) / gpc), (unsigned)n_combos);
  if (order == 3) {
    const float pref3 = (float)(natural ? 1.0 / md : md / ((md - 1.0) * (md - 2.0)));
    k5_cplx_s3<<<grid, kThreads, 0, stream>>>(spec, chan_stride, G, m, M, Mp, ops, tiles_l, gpc,
                                              pref3, acc, plane);
  } else {
    const float pref =
        (float)(natural ? 1.0 / (md * md) : 1.0 / ((md - 1.0) * (md - 2.0) * (md - 3.0)));
    const float fmm = (float)(natural ? md : md * (md + 1.0));
    const float fm1 = (float)(natural ? 1.0 : md - 1.0);
    k5_cplx_s4<<<grid, kThreads, 0, stream>>>(spec, chan_stride, G, m, M, Mp, ops, tiles_l, gpc,
                                              shift, pref, fmm, fm1, acc, plane);
  }
  return cudaGetLastError();
}

}  // namespace ss
