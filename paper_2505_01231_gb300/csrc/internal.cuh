// internal.cuh -- definitions shared by the kernels and the host runtime of the
// polyspectrum library (not part of the public ABI; see include/polyspec.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pipeline.cuh"
#include "polyspec.h"

namespace ss {

// Size of the static scratch array of ss_s2_noalloc.
constexpr size_t kNoallocScratchBytes = SS_NOALLOC_SCRATCH_BYTES;

// Tile edge of the bispectrum and trispectrum kernels in (k, l) grid points.
constexpr int kTile = 64;
// Threads per CTA of the frame/FFT kernel and of the pair kernels.
constexpr int kThreadsK1 = 256;
constexpr int kThreadsPair = 256;

// Accumulator planes per grid point: sum Re S_g, sum Im S_g, sum (Re S_g)^2,
// sum (Im S_g)^2, all float64 (Sec. 4.2, Eq. 35-36 need the first and second
// power sums over the parts).
constexpr int kPlanes = 4;

// Where the samples of one batch come from: the plan's carry-over buffer
// (samples left from earlier chunks) followed by the caller's chunk.  Sample s
// of channel c in the concatenated record is carry[c*carry_stride + s] for
// s < carry_n and chunk[c*chunk_stride + s - carry_n] otherwise.
struct SampleSource {
  const void* carry;
  long long carry_n;
  long long carry_stride;
  const void* chunk;
  long long chunk_stride;
  int dtype;  // SS_F32 or SS_I16
};

// One channel combination of one order; channels as in the ABI records.
struct Combo {
  int order;
  int c[4];
};

// Optional second output of K1 for the tensor-core S4 kernel: per channel,
// group and chunk of FC frames (zero-padded to 16), the hi/lo split of Re, Im
// and |.|^2 of the centred coefficients, laid out as the tensor cores read
// K-major operands: rows (bins) in groups of 8; for each row group the six
// matrices (Re hi, Re lo, Im hi, Im lo, P hi, P lo) of `CB` bytes each, where a
// matrix holds the row group's core matrices (8 rows x 16 bytes) for
// consecutive 16-byte frame groups, 128 bytes apart (TF32: 4 frame groups,
// CB = 512; BF16: 2, CB = 256).  ps holds sum_j |.|^2 / sqrt 2 per bin.
enum { kImageNone = 0, kImageTF32 = 1, kImageBF16 = 2 };
struct OperandImage {
  void* img = nullptr;
  float* ps = nullptr;
  int fmt = kImageNone;
  int FC = 0, nch = 0;
  long long chunk_bytes = 0;  // (Mp / 8) * 6 * CB
  long long chan_bytes = 0;   // Gb_max * nch * chunk_bytes
  long long chan_ps = 0;      // Gb_max * Mp floats
};

// Kernel launchers (each returns the launch status; all work on `stream`).
cudaError_t launch_k1_spectra(const SampleSource& src, long long sample0, int G, int C, int T,
                              int m, int M, int Mp, const float* win, const float2* tw,
                              float2* spec, long long spec_chan_stride, const int* s2_auto,
                              double* acc2, int n_s2, float pref2, int grid, cudaStream_t stream,
                              const OperandImage& oi = OperandImage());

cudaError_t launch_k1_cross_s2(const float2* spec, long long chan_stride, int G, int m, int M,
                               int Mp, const int4* pairs, int n_pairs, float pref2, double* acc2,
                               long long plane, int nsm, cudaStream_t stream);

// Pair kernels run persistent grids of nsm x (resident CTAs per SM) CTAs that
// take (group chunk, tile) items from a queue (see pipeline.cuh); `counter` is
// a device int the launcher zeroes on the stream.  acc points at the
// combination's first accumulator plane; `plane` is the distance in doubles
// between the four planes (sum Re, sum Im, sumsq Re, sumsq Im).  `status` is
// the plan's device status word (a bounded wait that gives up writes to it).
// The tensor maps view the centred spectra as [rows][Mp/16][16] float2 with
// 128-byte swizzling; tm64 has boxes of 4 blocks (64 bins), tm128 of 8.
cudaError_t launch_k2_bispec(const CUtensorMap& tm64, const CUtensorMap& tm128,
                             const float2* spec_a, const float2* spec_b, const float2* spec_c,
                             int rowA, int rowB, int rowC, int G, int m, int FC, int M, int Mp,
                             const TileInfo* tiles, int n_tiles, int cross, float pref3,
                             double* acc, long long plane, int rows, int nsm, int* counter,
                             int* status, cudaStream_t stream);

cudaError_t launch_k3_trispec(const CUtensorMap& tm64, int row0, int G, int m, int FC, int M,
                              const TileInfo* tiles, int n_tiles, float pref4a, float pref4b,
                              double* acc, long long plane, int nsm, int* counter, int* status,
                              cudaStream_t stream);

// Tensor-core form of K3 (SS_PREC_TF32X3, SS_PREC_BF16X3, SS_PREC_BF16): tiles of
// 128 k-bins x 48 l-bins fed from K1's operand image of `channel`.
constexpr int kTcTileM = 128, kTcTileN = 48;
cudaError_t launch_k3_trispec_tc(const OperandImage& oi, int channel, int G, int m, int M, int Mp,
                                 const TileInfo* tiles, int n_tiles, int precision, double* acc,
                                 long long plane, int nsm, int* counter, int* status,
                                 cudaStream_t stream);
size_t k3tc_smem_bytes(int precision);

// Groups per work item: about 16 items per CTA, whole groups, at least one.
inline int work_group_chunk(int G, int n_tiles, int n_cta) {
  const long long units = (long long)G * n_tiles;
  const long long target = 16ll * n_cta;
  long long gc = (units + target - 1) / target;
  if (gc < 1) gc = 1;
  if (gc > G) gc = G;
  return (int)gc;
}

// dynamic shared memory of the pair kernels for FC frames per stage
size_t k2_smem_bytes(int FC);
size_t k3_smem_bytes(int FC);

cudaError_t launch_k4_finalize(const double* acc, int n_combos, int rows, int M, int layout,
                               long long G, double norm, double* out, double* err,
                               cudaStream_t stream);

// Layout codes of launch_k4_finalize.
enum { kLayoutVector = 0,       // S2: [M]
       kLayoutS3Single = 1,     // one channel, computed for k <= l, mirrored; k+l <= M-1
       kLayoutS4Single = 2,     // one channel, computed for k <= l, mirrored
       kLayoutCross = 3 };      // full [2M-1][M] grid, no mirroring

}  // namespace ss
