// k_spectra.cu -- K1: frame, window, real FFT, group centring and S2.
//
// One CTA handles one group of m consecutive frames at a time (persistent loop
// over groups).  For every channel and frame j of the group it
//   1. reads the T samples of the frame (Sec. 3, Eq. 16) from the concatenation
//      carry-over | chunk and multiplies them by the window g_i / sqrt(sum g^2)
//      (Eq. 17; the scale is undone in the finalize step),
//   2. packs them as N = T/2 complex points y_n = x_{2n} + j x_{2n+1} and runs a
//      Stockham autosort FFT with the POSITIVE exponent of Eq. 18 (radix-8/4/2
//      butterflies in registers, ping-pong buffers in shared memory),
//   3. splits the half-length transform into the T/2+1 coefficients
//      X_k = E_k + e^{+2 pi j k/T} O_k of the real frame, and writes them.
// After the m frames it subtracts the group mean of every bin (the centred
// samples of the factorised k-statistics, App. H, Eq. 85), and forms the
// per-group S2 estimate c2 = 1/(m-1) sum_j |dX_jk|^2 (Eq. 32 with y = x*),
// whose sum and sum of squares over groups are accumulated for Eq. 35-36.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "internal.cuh"

namespace ss {
namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// multiplication by +j
__device__ __forceinline__ float2 cj(float2 a) { return make_float2(-a.y, a.x); }

// Radix-R DFT with the positive exponent, V_q = sum_r v_r e^{+2 pi j rq/R}.
__device__ __forceinline__ void dft4(float2& v0, float2& v1, float2& v2, float2& v3) {
  const float2 s02 = cadd(v0, v2), d02 = csub(v0, v2);
  const float2 s13 = cadd(v1, v3), d13 = cj(csub(v1, v3));
  v0 = cadd(s02, s13);
  v2 = csub(s02, s13);
  v1 = cadd(d02, d13);
  v3 = csub(d02, d13);
}

template <int R>
__device__ __forceinline__ void dft(float2 (&v)[R]);

template <>
__device__ __forceinline__ void dft<2>(float2 (&v)[2]) {
  const float2 a = v[0];
  v[0] = cadd(a, v[1]);
  v[1] = csub(a, v[1]);
}

template <>
__device__ __forceinline__ void dft<4>(float2 (&v)[4]) {
  dft4(v[0], v[1], v[2], v[3]);
}

template <>
__device__ __forceinline__ void dft<8>(float2 (&v)[8]) {
  // even/odd split: V_q = E_q + w^q O_q, V_{q+4} = E_q - w^q O_q, w = e^{+2 pi j/8}
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  const float h = 0.70710678118654752f;
  o1 = make_float2((o1.x - o1.y) * h, (o1.x + o1.y) * h);    // * (1 + j)/sqrt 2
  o2 = cj(o2);                                                // * j
  o3 = make_float2((-o3.x - o3.y) * h, (o3.x - o3.y) * h);   // * (-1 + j)/sqrt 2
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

// One Stockham pass: sub-transforms of length Ns are combined R at a time into
// length Ns*R.  x, y: N complex points in shared memory; tw[a] = e^{+2 pi j a/T}.
template <int R>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ x, float2* __restrict__ y,
                                              int N, int Ns, const float2* __restrict__ tw,
                                              int T) {
  const int NR = N / R;
  const int tw_scale = T / (Ns * R);
  for (int j = threadIdx.x; j < NR; j += blockDim.x) {
    const int k = j & (Ns - 1);
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[j + r * NR];
    if (Ns > 1) {
      const int step = k * tw_scale;
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(&tw[r * step]));
    }
    dft<R>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) y[base + q * Ns] = v[q];
  }
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t t;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
  return t;
}

// Write one bin's row of one K chunk (16 entries) of the Gram operand image:
// the hi and lo parts of the entries, in the K-major core-matrix layout the
// tensor cores read (8 rows x 16 bytes per core matrix, 16-byte entry groups
// 128 bytes apart; the hi block of a row group's chunk is followed by its lo
// block).  `row` is the bin's 16-byte slot in the chunk's first hi matrix.
template <int FMT>
__device__ __forceinline__ void write_gram_row(unsigned char* row, const float (&e)[16]) {
  constexpr uint32_t CB = FMT == kImageGramTF32 ? 512u : 256u;
  if constexpr (FMT == kImageGramF16) {
#pragma unroll
    for (int kg = 0; kg < 2; ++kg) {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        // two entries per conversion (each rounded to nearest, as one at a time)
        const float v0 = e[8 * kg + 2 * t], v1 = e[8 * kg + 2 * t + 1];
        const __half2 h = __floats2half2_rn(v0, v1);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
        hi[t] = *reinterpret_cast<const uint32_t*>(&h);
        lo[t] = *reinterpret_cast<const uint32_t*>(&l);
      }
      *reinterpret_cast<uint4*>(row + kg * 128) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(row + CB + kg * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
  } else if constexpr (FMT == kImageGramTF32) {
#pragma unroll
    for (int kg = 0; kg < 4; ++kg) {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        hi[t] = to_tf32(e[4 * kg + t]);
        lo[t] = to_tf32(e[4 * kg + t] - __uint_as_float(hi[t]));
      }
      *reinterpret_cast<uint4*>(row + kg * 128) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(row + CB + kg * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
  } else {
#pragma unroll
    for (int kg = 0; kg < 2; ++kg) {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float v0 = e[8 * kg + 2 * t], v1 = e[8 * kg + 2 * t + 1];
        const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
        hi[t] = *reinterpret_cast<const uint32_t*>(&h);
        lo[t] = *reinterpret_cast<const uint32_t*>(&l);
      }
      *reinterpret_cast<uint4*>(row + kg * 128) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(row + CB + kg * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

// Several channels in FP16X3: the row scale of a bin whose largest |d_j|^2 over
// the group is mx2, a power of two that brings sqrt(mx2) below 2^14, within
// [2^-60, 2^60] (1 for a zero bin).
__device__ __forceinline__ float cross_row_scale(float mx2) {
  if (!(mx2 > 0.f)) return 1.f;
  int e;
  frexpf(sqrtf(mx2), &e);  // sqrt(mx2) < 2^e
  return ldexpf(1.f, min(60, max(-60, 14 - e)));
}

// FP16 operand image: the power of two that brings a bin's largest entry (the
// weighted Gram products and ps), bounded by `bound`, below 2^14 (1 for an
// all-zero bin).
__device__ __forceinline__ float f16_row_scale(float bound) {
  if (!(bound > 0.f)) return 1.f;
  int e;
  frexpf(bound, &e);  // bound < 2^e
  return ldexpf(1.f, 14 - e);
}

template <int DTYPE>
__device__ __forceinline__ float load_sample(const SampleSource& s, int c, long long idx) {
  if (idx < s.carry_n) {
    const long long o = (long long)c * s.carry_stride + idx;
    if (DTYPE == SS_F32) return __ldg(static_cast<const float*>(s.carry) + o);
    return (float)__ldg(static_cast<const short*>(s.carry) + o);
  }
  const long long o = (long long)c * s.chunk_stride + (idx - s.carry_n);
  if (DTYPE == SS_F32) return __ldg(static_cast<const float*>(s.chunk) + o);
  return (float)__ldg(static_cast<const short*>(s.chunk) + o);
}

// First-order spectrum of one group (Sec. 4, App. G): the group mean of the
// zero-frequency coefficient (divided by sum g at finalize); its sum and sums of
// squares over the CTA's groups.  Called by the thread that centres bin 0.
__device__ __forceinline__ void add_s1(float* s1, float2 mean) {
  s1[0] += mean.x;
  s1[1] += mean.y;
  s1[2] = fmaf(mean.x, mean.x, s1[2]);
  s1[3] = fmaf(mean.y, mean.y, s1[3]);
}

// Centre bin k over the group's m frames (subtract the mean, the samples of the
// factorised k-statistics, App. H, Eq. 85), store the centred coefficients,
// add the per-group S2 estimate c2 = 1/(m-1) sum_j |d_j|^2 (Eq. 32) to the
// CTA's float32 sums, and, with an operand image, write the bin's weighted Gram
// products (diagonal chunks sqrt(w_jj r) |d_j|^2, then the pairs j < j' in
// lexicographic order, sqrt(4(m-1) r) Re(d_j d_j'*), 16 per chunk, zero-padded)
// and its ps value.  fetch(j) gives frame j's coefficient, store(j, d) keeps the
// centred one.
template <int FMT, class Fetch, class Store>
__device__ __forceinline__ void centre_bin(int k, bool valid, float2 mean, int m, int c, int g,
                                           int Mp, const OperandImage& oi, Fetch fetch,
                                           Store store, float* s2sum, float* s2sq, float pref2) {
  float p = 0.f;
  if constexpr (FMT == kImageNone) {
    float mx = 0.f;  // max_j |d_j|^2 (several channels in FP16X3: the bin's row scale)
    for (int j = 0; j < m; ++j) {
      const float2 d = valid ? csub(fetch(j), mean) : make_float2(0.f, 0.f);
      store(j, d);
      p = fmaf(d.x, d.x, fmaf(d.y, d.y, p));
      mx = fmaxf(mx, fmaf(d.x, d.x, d.y * d.y));
    }
    if (oi.rmax) oi.rmax[(long long)c * oi.chan_rmax + (long long)g * Mp + k] = cross_row_scale(mx);
  } else {
    float dr[kMaxGramM], di[kMaxGramM];
    float mx = 0.f;  // max_j |d_j|^2
    for (int j = 0; j < m; ++j) {
      const float2 d = valid ? csub(fetch(j), mean) : make_float2(0.f, 0.f);
      store(j, d);
      dr[j] = d.x;
      di[j] = d.y;
      const float pj = fmaf(d.x, d.x, d.y * d.y);
      p += pj;
      mx = fmaxf(mx, pj);
    }
    const float sc =
        FMT == kImageGramF16 ? f16_row_scale(fmaxf(fmaxf(oi.sd, oi.so) * mx, oi.sp * p)) : 1.f;
    const float sd = oi.sd * sc, so = oi.so * sc, sps = oi.sp * p * sc;
    const int npair = m * (m - 1) / 2;
    int pj = 0, pk = 1;  // next off-diagonal pair (j, j'), lexicographic
    if (k < oi.img_bins) {  // rows the tensor-core S4 reads
      constexpr int kChunkBytes = FMT == kImageGramTF32 ? 1024 : 512;  // 2 CB
      unsigned char* rbase = static_cast<unsigned char*>(oi.img) + (size_t)c * oi.chan_bytes +
                             (size_t)g * oi.group_bytes + (size_t)(k >> 3) * oi.rg_bytes +
                             (k & 7) * 16;
      for (int ch = 0; ch < oi.nkc; ++ch) {
        float e[16];
        if (ch < oi.ndc) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int j = ch * 16 + t;
            e[t] = j < m ? sd * fmaf(dr[j], dr[j], di[j] * di[j]) : 0.f;
          }
        } else {
          const int p0 = (ch - oi.ndc) * 16;
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            if (p0 + t < npair) {
              e[t] = so * fmaf(dr[pj], dr[pk], di[pj] * di[pk]);
              if (++pk == m) {
                ++pj;
                pk = pj + 1;
              }
            } else {
              e[t] = p0 + t == npair ? sps : 0.f;  // ps after the pairs (negated with them)
            }
          }
        }
        write_gram_row<FMT>(rbase + ch * kChunkBytes, e);
      }
      if (FMT == kImageGramF16)  // exact: a power of two
        oi.rsc[(long long)c * oi.chan_rsc + (long long)g * Mp + k] = 1.f / sc;
    }
  }
  if (valid && s2sum) {
    const float c2 = p * pref2;
    s2sum[k] += c2;
    s2sq[k] = fmaf(c2, c2, s2sq[k]);
  }
}

// Add the CTA's float32 sums of S2 (and S1) over its last groups to the float64
// accumulators and clear them.  Each thread flushes the bins it centres (bin k
// belongs to thread k mod blockDim.x; S1 to thread 0), so no barrier is needed.
__device__ __forceinline__ void flush_k1_sums(int C, int M, const int* __restrict__ s2_auto,
                                              double* __restrict__ acc2, int n_s2, float* s2sum,
                                              float* s2sq, float (*s1s)[4], double* acc1) {
  const long long plane = (long long)n_s2 * M;
  for (int c = 0; c < C; ++c) {
    const int ia = s2_auto[c];
    if (ia < 0) continue;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
      atomicAdd(acc2 + 0 * plane + (long long)ia * M + k, (double)s2sum[c * M + k]);
      atomicAdd(acc2 + 2 * plane + (long long)ia * M + k, (double)s2sq[c * M + k]);
      s2sum[c * M + k] = 0.f;
      s2sq[c * M + k] = 0.f;
    }
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < C; ++c)
      for (int q = 0; q < 4; ++q) {
        if (acc1) atomicAdd(acc1 + q * C + c, (double)s1s[c][q]);
        s1s[c][q] = 0.f;
      }
}

template <int DTYPE, int FMT>
__global__ void __launch_bounds__(kThreadsK1)
k1_spectra(SampleSource src, long long sample0, int G, int C, int T, int m, int M, int Mp,
           const float* __restrict__ win, const float2* __restrict__ tw,
           float2* __restrict__ spec, long long chan_stride, const int* __restrict__ s2_auto,
           double* __restrict__ acc2, int n_s2, float pref2, OperandImage oi,
           double* __restrict__ acc1) {
  extern __shared__ float4 smem_raw[];
  const int N = T / 2;
  float2* bufA = reinterpret_cast<float2*>(smem_raw);
  float2* bufB = bufA + N;
  float2* gsum = bufB + N;                                        // [M]
  float* s2sum = reinterpret_cast<float*>(gsum + M);             // [C][M]
  float* s2sq = s2sum + C * M;                                    // [C][M]

  __shared__ float s1s[4][4];  // per channel: sums of Re, Im, Re^2, Im^2 of S1 (thread 0)
  for (int i = threadIdx.x; i < 2 * C * M; i += blockDim.x) s2sum[i] = 0.f;
  if (threadIdx.x < 16) s1s[threadIdx.x >> 2][threadIdx.x & 3] = 0.f;

  int ngroups = 0;  // groups in the float32 sums since the last flush
  for (int g = blockIdx.x; g < G; g += gridDim.x) {
    for (int c = 0; c < C; ++c) {
      float2* grow = spec + (long long)c * chan_stride + (long long)g * m * Mp;
      for (int k = threadIdx.x; k < M; k += blockDim.x) gsum[k] = make_float2(0.f, 0.f);
      for (int j = 0; j < m; ++j) {
        const long long s0 = sample0 + ((long long)g * m + j) * T;
        __syncthreads();  // bufA is free (previous frame's post-processing done)
        for (int n = threadIdx.x; n < N; n += blockDim.x) {
          const float x0 = load_sample<DTYPE>(src, c, s0 + 2 * n);
          const float x1 = load_sample<DTYPE>(src, c, s0 + 2 * n + 1);
          bufA[n] = make_float2(x0 * __ldg(&win[2 * n]), x1 * __ldg(&win[2 * n + 1]));
        }
        __syncthreads();
        float2* x = bufA;
        float2* y = bufB;
        int Ns = 1;
        int rem = N;
        while (rem > 1) {
          if (rem % 8 == 0 && rem != 16) {
            stockham_pass<8>(x, y, N, Ns, tw, T);
            Ns *= 8; rem /= 8;
          } else if (rem % 4 == 0) {
            stockham_pass<4>(x, y, N, Ns, tw, T);
            Ns *= 4; rem /= 4;
          } else {
            stockham_pass<2>(x, y, N, Ns, tw, T);
            Ns *= 2; rem /= 2;
          }
          __syncthreads();
          float2* t = x; x = y; y = t;
        }
        // x holds Y_n; X_k = 1/2 [(Y_k + Y*_{N-k}) - j w^k (Y_k - Y*_{N-k})], w = e^{+2 pi j/T}
        float2* row = grow + (long long)j * Mp;
        for (int k = threadIdx.x; k < M; k += blockDim.x) {
          const float2 yk = x[k == N ? 0 : k];
          const float2 yr = x[k == 0 ? 0 : N - k];
          const float2 yc = make_float2(yr.x, -yr.y);
          const float2 s = cadd(yk, yc);
          const float2 wd = cmul(__ldg(&tw[k]), csub(yk, yc));
          const float2 X = make_float2(0.5f * (s.x + wd.y), 0.5f * (s.y - wd.x));
          row[k] = X;
          gsum[k] = cadd(gsum[k], X);
        }
      }
      // centre each bin over the group and form the per-group S2 estimate; with an
      // operand image, also write the split tensor-core operands chunk by chunk
      const float inv_m = 1.0f / (float)m;
      const int ia = s2_auto[c];
      for (int k = threadIdx.x; k < Mp; k += blockDim.x) {
        const bool valid = k < M;
        const float2 mean = valid ? make_float2(gsum[k].x * inv_m, gsum[k].y * inv_m)
                                  : make_float2(0.f, 0.f);
        if (k == 0) add_s1(s1s[c], mean);
        centre_bin<FMT>(
            k, valid, mean, m, c, g, Mp, oi,
            [&](int j) { return grow[(long long)j * Mp + k]; },
            [&](int j, float2 d) { grow[(long long)j * Mp + k] = d; },
            ia >= 0 ? s2sum + c * M : nullptr, ia >= 0 ? s2sq + c * M : nullptr, pref2);
      }
    }
    if (++ngroups == kMaxFp32Groups) {
      flush_k1_sums(C, M, s2_auto, acc2, n_s2, s2sum, s2sq, s1s, acc1);
      ngroups = 0;
    }
  }
  // the CTA's remaining float32 partial sums into the float64 accumulators
  if (ngroups) flush_k1_sums(C, M, s2_auto, acc2, n_s2, s2sum, s2sq, s1s, acc1);
}

// Stockham pass over a batch of FB frames of N points (frame f at x + f sx, its
// output at y + f sy); all threads share the FB * N/R butterflies of the pass.
template <int R>
__device__ __forceinline__ void stockham_pass_batch(const float2* __restrict__ x,
                                                    float2* __restrict__ y, int N, int Ns,
                                                    const float2* __restrict__ tw, int T, int FB,
                                                    int sx, int sy) {
  const int NR = N / R;
  const int lg = __ffs(NR) - 1;  // NR is a power of two
  const int tw_scale = T / (Ns * R);
  for (int idx = threadIdx.x; idx < FB * NR; idx += blockDim.x) {
    const int f = idx >> lg, j = idx & (NR - 1);
    const float2* xf = x + f * sx;
    float2* yf = y + f * sy;
    const int k = j & (Ns - 1);
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = xf[j + r * NR];
    if (Ns > 1) {
      const int step = k * tw_scale;
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[r * step]);
    }
    dft<R>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) yf[base + q * Ns] = v[q];
  }
}

// K1, resident forms: with the group's m coefficient rows of channel c in shared
// memory (Xs, [m][Mp]), thread = bin: subtract the bin's group mean (the centred
// samples of the factorised k-statistics, App. H, Eq. 85), write the centred
// column to the spectra once, add the per-group S2 estimate to the CTA's float32
// sums and, with an operand image, write the bin's weighted Gram products and its
// ps value.
template <int FMT>
__device__ __forceinline__ void centre_resident(float2* Xs, float2* __restrict__ grow, int c, int g,
                                                int m, int M, int Mp, const OperandImage& oi,
                                                int ia, float* s2sum, float* s2sq, float* s1,
                                                float pref2) {
  const float inv_m = 1.0f / (float)m;
  for (int k = threadIdx.x; k < Mp; k += blockDim.x) {
    // thread = bin: centre the column in place, write it out once
    const bool valid = k < M;
    float2 mean = make_float2(0.f, 0.f);
    if (valid) {
      for (int j = 0; j < m; ++j) mean = cadd(mean, Xs[j * Mp + k]);
      mean = make_float2(mean.x * inv_m, mean.y * inv_m);
    }
    if (k == 0) add_s1(s1, mean);
    float p = 0.f, mx = 0.f;  // sum and max over j of |d_j|^2
    for (int j = 0; j < m; ++j) {
      const float2 d = valid ? csub(Xs[j * Mp + k], mean) : make_float2(0.f, 0.f);
      Xs[j * Mp + k] = d;
      grow[(long long)j * Mp + k] = d;
      const float pj = fmaf(d.x, d.x, d.y * d.y);
      p += pj;
      mx = fmaxf(mx, pj);
    }
    // several channels in FP16X3: the bin's row scale
    if (oi.rmax) oi.rmax[(long long)c * oi.chan_rmax + (long long)g * Mp + k] = cross_row_scale(mx);
    if (FMT != kImageNone && k < oi.img_bins) {  // rows the tensor-core S4 reads
      const float sc =
        FMT == kImageGramF16 ? f16_row_scale(fmaxf(fmaxf(oi.sd, oi.so) * mx, oi.sp * p)) : 1.f;
      const float sd = oi.sd * sc, so = oi.so * sc, sps = oi.sp * p * sc;
      // weighted Gram products of the bin in K order, read from the centred column
      const int npair = m * (m - 1) / 2;
      int pj = 0, pk = 1;
      float2 dj = Xs[k];
      constexpr int kChunkBytes = FMT == kImageGramTF32 ? 1024 : 512;  // 2 CB
      unsigned char* rbase = static_cast<unsigned char*>(oi.img) + (size_t)c * oi.chan_bytes +
                             (size_t)g * oi.group_bytes + (size_t)(k >> 3) * oi.rg_bytes +
                             (k & 7) * 16;
      for (int ch = 0; ch < oi.nkc; ++ch) {
        float e[16];
        if (ch < oi.ndc) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int j = ch * 16 + t;
            const float2 d = j < m ? Xs[j * Mp + k] : make_float2(0.f, 0.f);
            e[t] = sd * fmaf(d.x, d.x, d.y * d.y);
          }
        } else {
          const int p0 = (ch - oi.ndc) * 16;
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            if (p0 + t < npair) {
              const float2 d2 = Xs[pk * Mp + k];
              e[t] = so * fmaf(dj.x, d2.x, dj.y * d2.y);
              if (++pk == m) {
                ++pj;
                pk = pj + 1;
                dj = Xs[pj * Mp + k];
              }
            } else {
              e[t] = p0 + t == npair ? sps : 0.f;  // ps after the pairs (negated with them)
            }
          }
        }
        write_gram_row<FMT>(rbase + ch * kChunkBytes, e);
      }
      if (FMT == kImageGramF16)  // exact: a power of two
        oi.rsc[(long long)c * oi.chan_rsc + (long long)g * Mp + k] = 1.f / sc;
    }
    if (valid && ia >= 0) {
      const float c2 = p * pref2;
      s2sum[c * M + k] += c2;
      s2sq[c * M + k] = fmaf(c2, c2, s2sq[c * M + k]);
    }
  }
}

// K1 for groups whose coefficients fit in shared memory: the group's m frames
// are transformed FB at a time (every Stockham pass covers all FB frames, so a
// frame costs a fraction of the barriers), the coefficients X_jk stay in shared
// memory, and the centred coefficients are written to the spectra once.  The
// passes of a batch alternate between the batch's own coefficient rows and one
// buffer of FB frames (a second buffer would halve FB within the same shared
// memory); the split into X_k reads the last pass's output and writes the rows,
// in place (one thread per pair k, N - k) when the rows hold that output.  Same
// results as k1_spectra; the samples of a batch are contiguous and are read
// with 16-byte (float32) or 8-byte (int16) loads when aligned.
template <int DTYPE, int FMT>
__global__ void __launch_bounds__(kThreadsK1, 3)
k1_spectra_res(SampleSource src, long long sample0, int G, int C, int T, int m, int M, int Mp,
               int FB, const float* __restrict__ win, const float2* __restrict__ tw,
               float2* __restrict__ spec, long long chan_stride, const int* __restrict__ s2_auto,
               double* __restrict__ acc2, int n_s2, float pref2, OperandImage oi,
           double* __restrict__ acc1) {
  extern __shared__ float4 smem_raw[];
  const int N = T / 2;
  float2* buf = reinterpret_cast<float2*>(smem_raw);  // [FB][N]
  float2* Xs = buf + FB * N;                          // [m][Mp]
  float2* tws = Xs + m * Mp;                           // [T] twiddles e^{+2 pi j a/T}
  float* wins = reinterpret_cast<float*>(tws + T);     // [T] window / sqrt(sum g^2)
  float* s2sum = wins + T;                             // [C][M]
  float* s2sq = s2sum + C * M;                         // [C][M]
  constexpr int kVec = DTYPE == SS_F32 ? 16 : 8;        // bytes per vector load (4 samples)

  __shared__ float s1s[4][4];  // per channel: sums of Re, Im, Re^2, Im^2 of S1 (thread 0)
  for (int i = threadIdx.x; i < 2 * C * M; i += blockDim.x) s2sum[i] = 0.f;
  if (threadIdx.x < 16) s1s[threadIdx.x >> 2][threadIdx.x & 3] = 0.f;
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    tws[i] = __ldg(&tw[i]);
    wins[i] = __ldg(&win[i]);
  }

  // float32 samples of the next batch, loaded into registers while the current
  // batch is transformed (when the batch is aligned, past the carry-over, and at
  // most kPre vectors per thread)
  constexpr int kPre = 4;
  float4 pre[kPre];
  auto prefetch = [&](int gg, int cc, int jj) -> bool {
    if constexpr (DTYPE != SS_F32) return false;
    const int nq = min(FB, m - jj) * T / 4;
    if (nq > kPre * (int)blockDim.x) return false;
    const long long off = sample0 + ((long long)gg * m + jj) * T - src.carry_n;
    const float4* p4 = reinterpret_cast<const float4*>(
        static_cast<const float*>(src.chunk) + (long long)cc * src.chunk_stride + off);
    if (off < 0 || ((uintptr_t)p4 % 16) != 0) return false;
#pragma unroll
    for (int r = 0; r < kPre; ++r) {
      const int q = threadIdx.x + r * blockDim.x;
      if (q < nq) pre[r] = __ldg(p4 + q);
    }
    return true;
  };
  bool have = blockIdx.x < G && prefetch(blockIdx.x, 0, 0);  // pre holds the batch's samples
  int ngroups = 0;  // groups in the float32 sums since the last flush
  for (int g = blockIdx.x; g < G; g += gridDim.x) {
    for (int c = 0; c < C; ++c) {
      float2* grow = spec + (long long)c * chan_stride + (long long)g * m * Mp;
      for (int j0 = 0; j0 < m; j0 += FB) {
        const int nf = min(FB, m - j0);
        const long long s0 = sample0 + ((long long)g * m + j0) * T;  // first sample of the batch
        __syncthreads();  // the buffers are free (previous batch split, previous group centred)
        const long long off = s0 - src.carry_n;
        const char* cbase = static_cast<const char*>(src.chunk) +
                            ((long long)c * src.chunk_stride + off) * (DTYPE == SS_F32 ? 4 : 2);
        if (have) {
#pragma unroll
          for (int r = 0; r < kPre; ++r) {
            const int q = threadIdx.x + r * blockDim.x;
            if (q < nf * T / 4) {
              const int i = (4 * q) & (T - 1), f = (4 * q) / T;
              const float4 w = *reinterpret_cast<const float4*>(wins + i);
              float2* d = Xs + (j0 + f) * Mp + i / 2;
              d[0] = make_float2(pre[r].x * w.x, pre[r].y * w.y);
              d[1] = make_float2(pre[r].z * w.z, pre[r].w * w.w);
            }
          }
        } else if (off >= 0 && ((uintptr_t)cbase % kVec) == 0) {
          for (int q = threadIdx.x; q < nf * T / 4; q += blockDim.x) {
            const int i = (4 * q) & (T - 1), f = (4 * q) / T;
            float x0, x1, x2, x3;
            if constexpr (DTYPE == SS_F32) {
              const float4 v = __ldg(reinterpret_cast<const float4*>(cbase) + q);
              x0 = v.x; x1 = v.y; x2 = v.z; x3 = v.w;
            } else {
              const short4 v = __ldg(reinterpret_cast<const short4*>(cbase) + q);
              x0 = v.x; x1 = v.y; x2 = v.z; x3 = v.w;
            }
            const float4 w = *reinterpret_cast<const float4*>(wins + i);
            float2* d = Xs + (j0 + f) * Mp + i / 2;
            d[0] = make_float2(x0 * w.x, x1 * w.y);
            d[1] = make_float2(x2 * w.z, x3 * w.w);
          }
        } else {
          for (int q = threadIdx.x; q < nf * N; q += blockDim.x) {
            const int f = q / N, n = q - f * N;
            const long long si = s0 + (long long)f * T + 2 * n;
            Xs[(j0 + f) * Mp + n] = make_float2(load_sample<DTYPE>(src, c, si) * wins[2 * n],
                                                load_sample<DTYPE>(src, c, si + 1) * wins[2 * n + 1]);
          }
        }
        {  // the next batch: this group's next frames, the next channel or the next group
          int gn = g, cn = c, jn = j0 + FB;
          if (jn >= m) {
            jn = 0;
            if (++cn == C) {
              cn = 0;
              gn += gridDim.x;
            }
          }
          have = gn < G && prefetch(gn, cn, jn);
        }
        __syncthreads();
        float2* rows = Xs + j0 * Mp;
        float2* x = rows;  // the pass input and its frame stride
        float2* y = buf;
        int sx = Mp, sy = N;
        int Ns = 1;
        int rem = N;
        while (rem > 1) {
          if (rem % 8 == 0 && rem != 16) {
            stockham_pass_batch<8>(x, y, N, Ns, tws, T, nf, sx, sy);
            Ns *= 8; rem /= 8;
          } else if (rem % 4 == 0) {
            stockham_pass_batch<4>(x, y, N, Ns, tws, T, nf, sx, sy);
            Ns *= 4; rem /= 4;
          } else {
            stockham_pass_batch<2>(x, y, N, Ns, tws, T, nf, sx, sy);
            Ns *= 2; rem /= 2;
          }
          __syncthreads();
          float2* t = x; x = y; y = t;
          const int ts = sx; sx = sy; sy = ts;
        }
        // X_k = 1/2 [(Y_k + Y*_{N-k}) - j w^k (Y_k - Y*_{N-k})], w = e^{+2 pi j/T},
        // Y_N = Y_0: each thread takes a pair k, N - k (k = 0 also gives X_N from
        // Y_0), reads both Y and writes both X, so the split may work in place
        auto split = [&](float2 yk, float2 yr, int k) {
          const float2 yc = make_float2(yr.x, -yr.y);
          const float2 sm = cadd(yk, yc);
          const float2 wd = cmul(tws[k], csub(yk, yc));
          return make_float2(0.5f * (sm.x + wd.y), 0.5f * (sm.y - wd.x));
        };
        const int NH = N / 2 + 1;  // pairs per frame
        for (int idx = threadIdx.x; idx < nf * NH; idx += blockDim.x) {
          const int f = idx / NH, k = idx - f * NH;
          const float2* xf = x + f * sx;
          float2* xr = rows + f * Mp;
          const float2 a = xf[k], b = xf[k == 0 ? 0 : N - k];
          xr[k] = split(a, b, k);
          xr[N - k] = split(b, a, N - k);
        }
      }
      __syncthreads();  // the group's coefficients are in shared memory
      centre_resident<FMT>(Xs, grow, c, g, m, M, Mp, oi, s2_auto[c], s2sum, s2sq, s1s[c], pref2);
    }
    if (++ngroups == kMaxFp32Groups) {
      flush_k1_sums(C, M, s2_auto, acc2, n_s2, s2sum, s2sq, s1s, acc1);
      ngroups = 0;
    }
  }
  if (ngroups) flush_k1_sums(C, M, s2_auto, acc2, n_s2, s2sum, s2sq, s1s, acc1);
}

// One Stockham pass of a warp's own frame (N points in the warp's shared buffer,
// transformed in place): every lane first reads the inputs of its butterflies
// (j = lane + 32 b), the warp synchronises, then each lane writes its outputs.
// N / R <= 32 * (16 / R), i.e. N <= 512: at most 16 points per lane.
template <int R>
__device__ __forceinline__ void warp_stockham_pass(float2* buf, int N, int Ns,
                                                   const float2* __restrict__ tw, int T, int lane) {
  constexpr int kB = 16 / R;  // butterflies per lane
  const int NR = N / R;
  const int tw_scale = T / (Ns * R);
  float2 v[kB][R];
#pragma unroll
  for (int b = 0; b < kB; ++b) {
    const int j = lane + 32 * b;
    if (j < NR) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = buf[j + r * NR];
    }
  }
  __syncwarp();
#pragma unroll
  for (int b = 0; b < kB; ++b) {
    const int j = lane + 32 * b;
    if (j < NR) {
      const int k = j & (Ns - 1);
      if (Ns > 1) {
        const int step = k * tw_scale;
#pragma unroll
        for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], tw[r * step]);
      }
      dft<R>(v[b]);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int q = 0; q < R; ++q) buf[base + q * Ns] = v[b][q];
    }
  }
  __syncwarp();
}

// K1 with a warp per frame (T <= 1024): the group's coefficients stay resident as
// in k1_spectra_res, but each warp windows, transforms and splits whole frames in
// a buffer of its own, synchronising only itself (no block barrier per pass);
// the block synchronises once per group before and after the centring.
template <int DTYPE, int FMT>
__global__ void __launch_bounds__(kThreadsK1, 2)
k1_spectra_warp(SampleSource src, long long sample0, int G, int C, int T, int m, int M, int Mp,
                const float* __restrict__ win, const float2* __restrict__ tw,
                float2* __restrict__ spec, long long chan_stride, const int* __restrict__ s2_auto,
                double* __restrict__ acc2, int n_s2, float pref2, OperandImage oi,
                double* __restrict__ acc1) {
  extern __shared__ float4 smem_raw[];
  const int N = T / 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kWarps = kThreadsK1 / 32;
  float2* Xs = reinterpret_cast<float2*>(smem_raw);  // [m][Mp]
  float2* bufs = Xs + m * Mp;                         // [kWarps][N]
  float2* tws = bufs + kWarps * N;                    // [T] twiddles e^{+2 pi j a/T}
  float* wins = reinterpret_cast<float*>(tws + T);   // [T] window / sqrt(sum g^2)
  float* s2sum = wins + T;                            // [C][M]
  float* s2sq = s2sum + C * M;                        // [C][M]
  float2* buf = bufs + warp * N;
  constexpr int kVec = DTYPE == SS_F32 ? 16 : 8;       // bytes per vector load (4 samples)

  __shared__ float s1s[4][4];  // per channel: sums of Re, Im, Re^2, Im^2 of S1 (thread 0)
  for (int i = threadIdx.x; i < 2 * C * M; i += blockDim.x) s2sum[i] = 0.f;
  if (threadIdx.x < 16) s1s[threadIdx.x >> 2][threadIdx.x & 3] = 0.f;
  for (int i = threadIdx.x; i < T; i += blockDim.x) {
    tws[i] = __ldg(&tw[i]);
    wins[i] = __ldg(&win[i]);
  }
  __syncthreads();

  int ngroups = 0;  // groups in the float32 sums since the last flush
  for (int g = blockIdx.x; g < G; g += gridDim.x) {
    for (int c = 0; c < C; ++c) {
      float2* grow = spec + (long long)c * chan_stride + (long long)g * m * Mp;
      for (int j = warp; j < m; j += kWarps) {
        // the frame's samples times the window, packed as N complex points
        const long long s0 = sample0 + ((long long)g * m + j) * T;
        const long long off = s0 - src.carry_n;
        const char* cbase = static_cast<const char*>(src.chunk) +
                            ((long long)c * src.chunk_stride + off) * (DTYPE == SS_F32 ? 4 : 2);
        if (off >= 0 && ((uintptr_t)cbase % kVec) == 0) {
          for (int q = lane; q < T / 4; q += 32) {
            float x0, x1, x2, x3;
            if constexpr (DTYPE == SS_F32) {
              const float4 v = __ldg(reinterpret_cast<const float4*>(cbase) + q);
              x0 = v.x; x1 = v.y; x2 = v.z; x3 = v.w;
            } else {
              const short4 v = __ldg(reinterpret_cast<const short4*>(cbase) + q);
              x0 = v.x; x1 = v.y; x2 = v.z; x3 = v.w;
            }
            const float4 w = *reinterpret_cast<const float4*>(wins + 4 * q);
            buf[2 * q] = make_float2(x0 * w.x, x1 * w.y);
            buf[2 * q + 1] = make_float2(x2 * w.z, x3 * w.w);
          }
        } else {
          for (int n = lane; n < N; n += 32)
            buf[n] = make_float2(load_sample<DTYPE>(src, c, s0 + 2 * n) * wins[2 * n],
                                 load_sample<DTYPE>(src, c, s0 + 2 * n + 1) * wins[2 * n + 1]);
        }
        __syncwarp();
        int Ns = 1, rem = N;
        while (rem > 1) {
          if (rem % 8 == 0 && rem != 16) {
            warp_stockham_pass<8>(buf, N, Ns, tws, T, lane);
            Ns *= 8; rem /= 8;
          } else if (rem % 4 == 0) {
            warp_stockham_pass<4>(buf, N, Ns, tws, T, lane);
            Ns *= 4; rem /= 4;
          } else {
            warp_stockham_pass<2>(buf, N, Ns, tws, T, lane);
            Ns *= 2; rem /= 2;
          }
        }
        // X_k = 1/2 [(Y_k + Y*_{N-k}) - j w^k (Y_k - Y*_{N-k})], w = e^{+2 pi j/T}
        float2* xr = Xs + j * Mp;
        for (int k = lane; k < M; k += 32) {
          const float2 yk = buf[k == N ? 0 : k];
          const float2 yr = buf[k == 0 ? 0 : N - k];
          const float2 yc = make_float2(yr.x, -yr.y);
          const float2 sm = cadd(yk, yc);
          const float2 wd = cmul(tws[k], csub(yk, yc));
          xr[k] = make_float2(0.5f * (sm.x + wd.y), 0.5f * (sm.y - wd.x));
        }
        __syncwarp();  // the buffer is free for the warp's next frame
      }
      __syncthreads();  // the group's coefficients are in shared memory
      centre_resident<FMT>(Xs, grow, c, g, m, M, Mp, oi, s2_auto[c], s2sum, s2sq, s1s[c], pref2);
      __syncthreads();  // Xs is free for the next channel or group
    }
    if (++ngroups == kMaxFp32Groups) {
      flush_k1_sums(C, M, s2_auto, acc2, n_s2, s2sum, s2sq, s1s, acc1);
      ngroups = 0;
    }
  }
  if (ngroups) flush_k1_sums(C, M, s2_auto, acc2, n_s2, s2sum, s2sq, s1s, acc1);
}

// Cross-channel S2 (Sec. 7, Eq. 47): c2(a_k, b_k*) = 1/(m-1) sum_j da_jk db_jk*
// per group, from the centred spectra K1 wrote.  Thread = (combination, bin);
// blockIdx.y splits the groups; float32 sums per CTA, float64 accumulation.
__global__ void k1_cross_s2(const float2* __restrict__ spec, long long chan_stride, int G, int m,
                            int M, int Mp, const int4* __restrict__ pairs, int groups_per_cta,
                            float pref2, double* __restrict__ acc2, long long plane) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  const int4 pr = pairs[blockIdx.z];
  const float2* A = spec + pr.x * chan_stride;
  const float2* B = spec + pr.y * chan_stride;
  const int g0 = blockIdx.y * groups_per_cta;
  const int g1 = min(G, g0 + groups_per_cta);
  float sr = 0.f, si = 0.f, qr = 0.f, qi = 0.f;
  for (int g = g0; g < g1; ++g) {
    float cr = 0.f, ci = 0.f;
    for (int j = 0; j < m; ++j) {
      const long long o = ((long long)g * m + j) * Mp + k;
      const float2 a = A[o], b = B[o];
      cr = fmaf(a.x, b.x, fmaf(a.y, b.y, cr));
      ci = fmaf(a.y, b.x, fmaf(-a.x, b.y, ci));
    }
    cr *= pref2;
    ci *= pref2;
    sr += cr;
    si += ci;
    qr = fmaf(cr, cr, qr);
    qi = fmaf(ci, ci, qi);
  }
  const long long o = (long long)pr.z * M + k;
  atomicAdd(acc2 + o, (double)sr);
  atomicAdd(acc2 + plane + o, (double)si);
  atomicAdd(acc2 + 2 * plane + o, (double)qr);
  atomicAdd(acc2 + 3 * plane + o, (double)qi);
}

}  // namespace

// Dynamic shared memory of the frame-at-a-time K1 for T samples and C channels,
// and its largest value (T = kMaxT, C = kMaxChannels).
constexpr size_t k1_smem(int T, int C) {
  return (size_t)(T / 2) * 2 * sizeof(float2) + (size_t)(T / 2 + 1) * sizeof(float2) +
         (size_t)2 * C * (T / 2 + 1) * sizeof(float);
}
constexpr size_t kK1MaxSmem = k1_smem(kMaxT, kMaxChannels);

// The dynamic shared-memory limit of a kernel is an attribute of the function,
// shared by every plan, stream and captured graph that launches it; each
// kernel therefore gets one fixed limit, the largest amount any of its
// launches can ask for, so that no launch depends on which launch set it last.
template <typename Kern>
cudaError_t set_smem_limit(Kern kern, size_t limit) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)limit);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                              cudaSharedmemCarveoutMaxShared);
}

// resident CTAs per SM of a K1 kernel with `smem` bytes of dynamic shared memory,
// from its own registers and shared memory (one wave is launched)
template <typename Kern>
cudaError_t k1_occupancy(Kern kern, size_t smem, int* occ) {
  int dev = 0, sm_smem = 0, sm_regs = 0, rsv = 0;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e != cudaSuccess) return e;
  const int by_smem = sm_smem / (int)(smem + fa.sharedSizeBytes + rsv);
  const int by_regs = sm_regs / std::max(1, ((fa.numRegs + 7) & ~7) * kThreadsK1);
  *occ = std::max(1, std::min(std::min(by_smem, by_regs), 2048 / kThreadsK1));
  return cudaSuccess;
}

template <int DTYPE, int FMT>
cudaError_t launch_k1_t(const SampleSource& src, long long sample0, int G, int C, int T, int m,
                        int M, int Mp, const float* win, const float2* tw, float2* spec,
                        long long spec_chan_stride, const int* s2_auto, double* acc2, int n_s2,
                        float pref2, const OperandImage& oi, int grid, size_t smem,
                        cudaStream_t stream, double* acc1, int mode) {
  // a group whose coefficients fit beside a batch of FFT buffers stays resident
  const size_t fixed = (size_t)m * Mp * sizeof(float2) + (size_t)2 * C * M * sizeof(float) +
                       (size_t)T * (sizeof(float2) + sizeof(float));  // + twiddles and window
  const size_t per_frame = (size_t)(T / 2) * sizeof(float2);  // one buffer of T/2 points
  // kK1Auto: three CTAs per SM with a smaller batch of frames beat two with a
  // larger one (T = 1024, m = 10: 2.59 vs 2.69 ms per step), else the 96 KB
  // budget; kK1Resident96: the 96 KB budget; kK1Frames: frame at a time
  // a warp per frame: the group's coefficients, a buffer of T/2 points per warp;
  // shapes it does not take (T > 1024, or a group beyond 96 KB) use kK1Auto
  const size_t wsmem = fixed + (size_t)(kThreadsK1 / 32) * (T / 2) * sizeof(float2);
  if (mode == kK1Warp && (T > 1024 || wsmem > kK1ResidentBytes)) mode = kK1Auto;
  if (mode == kK1Warp) {
    auto kern = k1_spectra_warp<DTYPE, FMT>;
    cudaError_t e = set_smem_limit(kern, kK1ResidentBytes);
    if (e != cudaSuccess) return e;
    int occ = 1;
    e = k1_occupancy(kern, wsmem, &occ);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 1;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int rgrid = std::max(1, std::min(G, nsm * occ));
    kern<<<rgrid, kThreadsK1, wsmem, stream>>>(src, sample0, G, C, T, m, M, Mp, win, tw, spec,
                                               spec_chan_stride, s2_auto, acc2, n_s2, pref2, oi,
                                               acc1);
    return cudaGetLastError();
  }
  const size_t budget = mode == kK1Frames ? 0
                        : (mode == kK1Auto && fixed + per_frame <= kK1ResidentBytes3)
                            ? kK1ResidentBytes3
                            : kK1ResidentBytes;
  if (fixed + per_frame <= budget) {
    const int FB = (int)std::min<size_t>((size_t)m, (budget - fixed) / per_frame);
    const size_t rsmem = fixed + (size_t)FB * per_frame;
    if (rsmem > kK1ResidentBytes) return cudaErrorInvalidValue;  // never: budget <= the limit
    auto kern = k1_spectra_res<DTYPE, FMT>;
    cudaError_t e = set_smem_limit(kern, kK1ResidentBytes);
    if (e != cudaSuccess) return e;
    // one wave: as many CTAs as are resident at once, from the kernel's own
    // registers and shared memory
    int dev = 0, nsm = 1, sm_smem = 0, sm_regs = 0, rsv = 0;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e != cudaSuccess) return e;
    const int by_smem = sm_smem / (int)(rsmem + fa.sharedSizeBytes + rsv);
    const int by_regs = sm_regs / std::max(1, ((fa.numRegs + 7) & ~7) * kThreadsK1);
    const int occ = std::max(1, std::min(std::min(by_smem, by_regs), 2048 / kThreadsK1));
    const int rgrid = std::max(1, std::min(G, nsm * occ));
    kern<<<rgrid, kThreadsK1, rsmem, stream>>>(
        src, sample0, G, C, T, m, M, Mp, FB, win, tw, spec, spec_chan_stride, s2_auto, acc2, n_s2,
        pref2, oi, acc1);
    return cudaGetLastError();
  }
  if (smem > kK1MaxSmem) return cudaErrorInvalidValue;
  cudaError_t e = set_smem_limit(k1_spectra<DTYPE, FMT>, kK1MaxSmem);
  if (e != cudaSuccess) return e;
  k1_spectra<DTYPE, FMT><<<grid, kThreadsK1, smem, stream>>>(src, sample0, G, C, T, m, M, Mp, win,
                                                             tw, spec, spec_chan_stride, s2_auto,
                                                             acc2, n_s2, pref2, oi, acc1);
  return cudaGetLastError();
}

cudaError_t launch_k1_spectra(const SampleSource& src, long long sample0, int G, int C, int T,
                              int m, int M, int Mp, const float* win, const float2* tw,
                              float2* spec, long long spec_chan_stride, const int* s2_auto,
                              double* acc2, int n_s2, float pref2, int grid, cudaStream_t stream,
                              const OperandImage& oi, double* acc1, int mode) {
  if (G <= 0) return cudaSuccess;
  if (mode < kK1Auto || mode >= kK1Modes) return cudaErrorInvalidValue;
  const size_t smem = k1_smem(T, C);
  if (grid > G) grid = G;
  const bool f32 = src.dtype == SS_F32;
#define K1_ARGS src, sample0, G, C, T, m, M, Mp, win, tw, spec, spec_chan_stride, s2_auto, acc2, \
                n_s2, pref2, oi, grid, smem, stream, acc1, mode
  switch (oi.fmt) {
    case kImageGramTF32:
      return f32 ? launch_k1_t<SS_F32, kImageGramTF32>(K1_ARGS)
                 : launch_k1_t<SS_I16, kImageGramTF32>(K1_ARGS);
    case kImageGramBF16:
      return f32 ? launch_k1_t<SS_F32, kImageGramBF16>(K1_ARGS)
                 : launch_k1_t<SS_I16, kImageGramBF16>(K1_ARGS);
    case kImageGramF16:
      return f32 ? launch_k1_t<SS_F32, kImageGramF16>(K1_ARGS)
                 : launch_k1_t<SS_I16, kImageGramF16>(K1_ARGS);
    default:
      return f32 ? launch_k1_t<SS_F32, kImageNone>(K1_ARGS)
                 : launch_k1_t<SS_I16, kImageNone>(K1_ARGS);
  }
#undef K1_ARGS
}

cudaError_t launch_k1_cross_s2(const float2* spec, long long chan_stride, int G, int m, int M,
                               int Mp, const int4* pairs, int n_pairs, float pref2, double* acc2,
                               long long plane, int nsm, cudaStream_t stream) {
  if (G <= 0 || n_pairs <= 0) return cudaSuccess;
  const int bx = (M + 127) / 128;
  int splits = std::max(1, (4 * nsm) / std::max(1, bx * n_pairs));
  splits = std::min(splits, std::max(1, G / 8));
  // at most kMaxFp32Groups groups in a thread's float32 sums (grid y <= 65535)
  splits = std::min(65535, std::max(splits, (G + kMaxFp32Groups - 1) / kMaxFp32Groups));
  const int gpc = (G + splits - 1) / splits;
  splits = (G + gpc - 1) / gpc;
  dim3 grid(bx, splits, n_pairs);
  k1_cross_s2<<<grid, 128, 0, stream>>>(spec, chan_stride, G, m, M, Mp, pairs, gpc, pref2, acc2,
                                        plane);
  return cudaGetLastError();
}

}  // namespace ss
