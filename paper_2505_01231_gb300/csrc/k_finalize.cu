// k_finalize.cu -- K4: mean over groups and standard errors, in float64; and the
// element-wise float64 addition that merges the group sums of two plans.
//
// For every output grid point it reads the float64 sums over the G groups of
// S_g (real and imaginary part) and of their squares, applies the window and
// dt normalisation `norm` of Eq. 23, 28, 31 (and Eq. 47, 48, 50), and writes
//   mean = norm sum / G
//   err  = sqrt( G/(G-1) (norm^2 sumsq / G - mean^2) / G )   (Eq. 35-36)
// for the real and the imaginary part.  One-channel grids that were computed
// on the k <= l half are mirrored with S(k, l) = S(l, k) (Sec. 9), whether the
// sums of (k, l) are stored at [k][l] or at [l][k]; bispectrum points with
// k + l > M-1 are set to zero.
#include "internal.cuh"

namespace ss {
namespace {

__global__ void k4_finalize(const double* __restrict__ acc, const double* __restrict__ prev,
                            int n_combos, int rows, int M, int layout, long long G, double norm,
                            double* __restrict__ out, double* __restrict__ err) {
  const long long per = (long long)rows * M;
  const long long total = per * n_combos;
  const long long plane = total;
  const double invG = 1.0 / (double)G;
  const double bessel = (double)G / (double)(G - 1);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long cmb = i / per;
    const long long p = i - cmb * per;
    int r = (int)(p / M), l = (int)(p - (long long)r * M);
    bool zero = false;
    if (layout == kLayoutS3Single) {
      if (r + l > M - 1) zero = true;
      if (r > l) { const int t = r; r = l; l = t; }
    } else if (layout == kLayoutS4Single) {
      if (r > l) { const int t = r; r = l; l = t; }
    } else if (layout == kLayoutS4Lower) {
      if (r < l) { const int t = r; r = l; l = t; }
    }
    double mr = 0.0, mi = 0.0, er = 0.0, ei = 0.0;
    if (!zero) {
      const long long o = cmb * per + (long long)r * M + l;
      // the sums of the groups since the snapshot `prev` (a block of sequential
      // spectra), or of all groups
      double s[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) s[q] = acc[q * plane + o] - (prev ? prev[q * plane + o] : 0.0);
      mr = norm * s[0] * invG;
      mi = norm * s[1] * invG;
      const double vr = bessel * (norm * norm * s[2] * invG - mr * mr);
      const double vi = bessel * (norm * norm * s[3] * invG - mi * mi);
      er = sqrt(fmax(vr, 0.0) * invG);
      ei = sqrt(fmax(vi, 0.0) * invG);
    }
    if (out) { out[2 * i] = mr; out[2 * i + 1] = mi; }
    if (err) { err[2 * i] = er; err[2 * i + 1] = ei; }
  }
}

__global__ void k_add_f64(double* __restrict__ dst, const double* __restrict__ src, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] += src[i];
}

}  // namespace

cudaError_t launch_add_f64(double* dst, const double* src, long long n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  long long grid = (n + 255) / 256;
  if (grid > 4096) grid = 4096;
  k_add_f64<<<(int)grid, 256, 0, stream>>>(dst, src, n);
  return cudaGetLastError();
}

cudaError_t launch_k4_finalize(const double* acc, int n_combos, int rows, int M, int layout,
                               long long G, double norm, double* out, double* err,
                               cudaStream_t stream, const double* prev) {
  const long long total = (long long)n_combos * rows * M;
  if (total == 0) return cudaSuccess;
  int grid = (int)((total + 255) / 256);
  if (grid > 4096) grid = 4096;
  k4_finalize<<<grid, 256, 0, stream>>>(acc, prev, n_combos, rows, M, layout, G, norm, out, err);
  return cudaGetLastError();
}

}  // namespace ss
