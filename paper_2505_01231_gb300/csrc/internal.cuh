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
// shared memory of the resident form of K1 (group coefficients + FFT batch)
constexpr size_t kK1ResidentBytes = 96u << 10;
// a tighter budget tried first: three resident CTAs per SM
constexpr size_t kK1ResidentBytes3 = 74u << 10;
constexpr int kTile = 64;
// Largest frame length and channel count a plan takes (the kernels' fixed
// dynamic shared-memory limits are sized for them).
constexpr int kMaxT = 4096, kMaxChannels = 4;
// Largest frames per staged chunk of the pair kernels.
constexpr int kMaxFC = 16;
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

// Optional second output of K1 for the tensor-core S4 kernel: the operand
// image of the weighted frame Gram of every bin.  With centred coefficients d_j
// of a group, G_jj' = Re(d_j d_j'*), the bracket of the factorised fourth
// k-statistic (App. H, Eq. 85) for the cut (a_k, a_k*, a_l, a_l*) is
//   m(m+1) Q - (m-1)(|U|^2 + |V|^2) = sum_{j<=j'} w_jj' G^k_jj' G^l_jj',
//   w_jj = m^2 - m + 2,  w_jj' = -4(m-1) (j < j'),
// one real contraction over K = m(m+1)/2, and c4 = r [that - (m-1) Sk Sl] with
// r = 1/((m-1)(m-2)(m-3)), Sk = sum_j |d_jk|^2.  The K entries come in chunks
// of 16: the diagonal chunks first, scaled by sd = sqrt(w_jj r), then the pairs
// j < j' in lexicographic order, scaled by so = sqrt(4(m-1) r), then one entry
// ps_k = sp Sk, sp = sqrt((m-1) r), zero-padded (the tensor-core kernel negates
// the pair chunks, so ps_k ps_l is subtracted with them and the contraction is
// c4 itself; K = m(m+1)/2 + 1).  Each entry is split hi + lo.  Layout per
// channel and group: rows (bins) in groups of 8; per row group, for each chunk,
// a hi block and a lo block of CB bytes, each holding the row group's core
// matrices (8 rows x 16 bytes) of the chunk's 16-byte entry groups 128 bytes
// apart (TF32: CB = 512; BF16, FP16: CB = 256).  So a chunk of a row group is
// 2 CB bytes, a row group rg_bytes = nkc * 2 CB, a group group_bytes =
// (Mp / 8) * rg_bytes.
// FP16: each bin's row is first multiplied by a power of two s_k that brings its
// largest entry (at most max(max(sd, so) max_j |d_jk|^2, sp Sk)) below 2^14, so
// that hi and lo stay inside the FP16 range; rsc holds 1/s_k per group and bin,
// and the kernel divides D by s_k and by s_l (exactly: powers of two).
enum { kImageNone = 0, kImageGramTF32 = 1, kImageGramBF16 = 2, kImageGramF16 = 3 };
constexpr int kMaxGramM = 32;  // largest m of the tensor-core S4 path
struct OperandImage {
  void* img = nullptr;
  float* rsc = nullptr;       // FP16: per group and bin, 1 / the bin's row scale
  int fmt = kImageNone;
  int nkc = 0, ndc = 0;       // K chunks, of which diagonal
  float sd = 0.f, so = 0.f, sp = 0.f;
  long long rg_bytes = 0;     // nkc * 2 * CB
  long long group_bytes = 0;  // (Mp / 8) * rg_bytes
  long long chan_bytes = 0;   // Gb_max * group_bytes
  long long chan_rsc = 0;     // Gb_max * Mp floats (FP16)
  int img_bins = 0;           // bins whose image rows and scales the tensor-core S4 reads
                              // (M - 1 when k3_column takes the last column, else Mp)
  // several channels in FP16X3: per channel, group and bin the power of two that
  // brings the bin's coefficients over the group's frames below 2^14 (within
  // [2^-60, 2^60]; 1 for a zero bin), at rmax[channel * chan_rmax + group * Mp + bin]
  float* rmax = nullptr;
  long long chan_rmax = 0;
};

// K1 forms (the autotuner's choice per plan): groups resident in shared memory
// within 74 KB (three CTAs per SM) when they fit, else 96 KB (kK1Auto); always
// the 96 KB budget (kK1Resident96); one frame at a time (kK1Frames); resident
// groups with a warp per frame (kK1Warp, T <= 1024 and the group within 96 KB).
enum { kK1Auto = 0, kK1Resident96 = 1, kK1Frames = 2, kK1Warp = 3, kK1Modes = 4 };

// Kernel launchers (each returns the launch status; all work on `stream`).
cudaError_t launch_k1_spectra(const SampleSource& src, long long sample0, int G, int C, int T,
                              int m, int M, int Mp, const float* win, const float2* tw,
                              float2* spec, long long spec_chan_stride, const int* s2_auto,
                              double* acc2, int n_s2, float pref2, int grid, cudaStream_t stream,
                              const OperandImage& oi = OperandImage(), double* acc1 = nullptr,
                              int mode = kK1Auto);

cudaError_t launch_k1_cross_s2(const float2* spec, long long chan_stride, int G, int m, int M,
                               int Mp, const int4* pairs, int n_pairs, float pref2, double* acc2,
                               long long plane, int nsm, cudaStream_t stream);

// Pair kernels run persistent grids of nsm x (resident CTAs per SM) CTAs that
// take (group chunk, tile) items from a queue (see pipeline.cuh); `counter` is
// a device int the launcher zeroes on the stream.  acc points at the
// combination's first accumulator plane; `plane` is the distance in doubles
// between the four planes (sum Re, sum Im, sumsq Re, sumsq Im).  `status` is
// the plan's device status word (a bounded wait that gives up writes to it);
// inject_timeout != 0 makes K2 run one wait out on purpose (timeout test).
// The tensor maps view the centred spectra as [rows][Mp/16][16] float2 with
// 128-byte swizzling; tm64 has boxes of 4 blocks (64 bins), tm128 of 8.
// K2 tilings (the autotuner's choice per plan): 4 x 4 micro-tiles in CTAs of 256
// threads with 4 stages (two CTAs per SM) or 3 stages (three CTAs per SM, 85
// registers), or 8 x 4 micro-tiles in CTAs of 128 threads with 2 or 3 stages;
// all take the same 64 x 64 tiles and give the same sums.  kK2Warp84 (one channel;
// the plan takes kK2Tile84Stages2 for several) runs k2_bispec84w: 8 x 4 micro-tiles
// in warps that work independently on 32 x 32 sub-tiles, each with its own stages.
enum { kK2Tile44 = 0, kK2Tile84Stages2 = 1, kK2Tile84Stages3 = 2, kK2Tile44Stages3 = 3,
       kK2Warp84 = 4, kK2Variants = 5 };
cudaError_t launch_k2_bispec(const CUtensorMap& tm64, const CUtensorMap& tm128,
                             const float2* spec_a, const float2* spec_b, const float2* spec_c,
                             int rowA, int rowB, int rowC, int G, int m, int FC, int M, int Mp,
                             const TileInfo* tiles, int n_tiles, int cross, float pref3,
                             double* acc, long long plane, int rows, int nsm, int* counter,
                             int* status, int inject_timeout, int variant, cudaStream_t stream);

cudaError_t launch_k3_trispec(const CUtensorMap& tm64, int row0, int G, int m, int FC, int M,
                              const TileInfo* tiles, int n_tiles, float pref4a, float pref4b,
                              double* acc, long long plane, int nsm, int* counter, int* status,
                              cudaStream_t stream);

// Tensor-core form of K3 (SS_PREC_TF32X3, SS_PREC_BF16X3, SS_PREC_BF16): tiles of
// 128 x 128 (k, l) bins, the weighted frame-Gram contraction fed from K1's
// operand image of `channel` through tm_img, a 4-D view of that channel's
// image [group][row group][chunk][2 CB bytes] in 8-byte elements with boxes of
// k3tc_stage_chunks(precision) chunks x 16 row groups; needs 4 <= m <= kMaxGramM.
constexpr int kTcTileM = 128, kTcTileN = 128;
cudaError_t launch_k3_trispec_tc(const CUtensorMap& tm_img, const OperandImage& oi, int channel,
                                 int G, int m, int M, int Mp,
                                 const TileInfo* tiles, int n_tiles, int precision, double* acc,
                                 long long plane, int nsm, int* counter, int* status,
                                 cudaStream_t stream);
size_t k3tc_smem_bytes(int precision);

// K3 for several channels (FP32 CUDA cores): C4(a_k, b_k*, c_l, d_l*) of every
// combination (combos: device array of n_combos (a, b, c, d)) on the grid
// k in [-(M-1), M-1] x l in [0, M-1], accumulated at acc[plane][combo][k+M-1][l].
cudaError_t launch_k3_trispec_cross(const float2* spec, long long chan_stride, int G, int m, int M,
                                    int Mp, const int4* combos, int n_combos, double* acc,
                                    long long plane, int nsm, bool natural, cudaStream_t stream);
int k3tc_stage_chunks(int precision);

// The same on the tcgen05 tensor cores: tiles of 128 rows k x 24 columns l,
// operands built in shared memory from the centred spectra.  TF32 hi/lo in three
// passes for SS_PREC_TF32X3, SS_PREC_BF16X3 and SS_PREC_BF16; with SS_PREC_FP16X3
// FP16 hi/lo in three passes of operands scaled per bin by powers of two, the
// bins' row scales per group that K1 writes (OperandImage::rmax).
// The spectra are read through 2-D views [rows][Mp] (8-byte elements, no swizzle):
// tm_ab with boxes of kF rows x min(box bins, Mp) bins, tm_cd with boxes of kF
// rows x col box bins (kF = 4 frames, 8 for FP16); a channel's rows start at
// channel x chan_rows.  FP16 also reads the row scales [channel x grp_rows +
// group][Mp] (float) through tm_sab (boxes of min(kCrossScaleBins, Mp) bins) and
// tm_scd (kCrossScaleCols bins).  The row k = -(M-1) is copied from k = M-1 (equal
// for real signals).  counter and status as for the pair kernels.
// Box widths (bins) of tm_ab and tm_cd, TF32 and FP16 forms: wider than the bins
// used, so that the rows of a thread's two frame chunks fall on other banks.
constexpr int kCrossBoxBins = 140, kCrossBoxBinsH = 142, kCrossColBox = 28, kCrossColBoxH = 30;
constexpr int kCrossTileCols = 24, kCrossScaleBins = 144, kCrossScaleCols = 28;
struct CrossViews {
  const CUtensorMap* tm_ab = nullptr;
  const CUtensorMap* tm_cd = nullptr;
  const CUtensorMap* tm_sab = nullptr;
  const CUtensorMap* tm_scd = nullptr;
  int chan_rows = 0, grp_rows = 0;
  bool f16 = false;
};
cudaError_t launch_k3_trispec_cross_tc(const CrossViews& v, int G, int m, int M, int Mp,
                                       const int4* combos, int n_combos, double* acc,
                                       long long plane, int nsm, bool natural, int* counter,
                                       int* status, cudaStream_t stream);

// Most groups whose per-group estimates a kernel adds up in float32 before the
// run goes to the float64 accumulators (bounds the float32 rounding of the sums
// over groups of Sec. 4.2 whatever the record length).
constexpr int kMaxFp32Groups = 64;

// Groups per work item: about 16 items per CTA, whole groups, at least one, at
// most kMaxFp32Groups (the pair kernels sum an item's groups in float32).
inline int work_group_chunk(int G, int n_tiles, int n_cta) {
  const long long units = (long long)G * n_tiles;
  const long long target = 16ll * n_cta;
  long long gc = (units + target - 1) / target;
  if (gc < 1) gc = 1;
  if (gc > kMaxFp32Groups) gc = kMaxFp32Groups;
  if (gc > G) gc = G;
  return (int)gc;
}

// Spectra of complex-valued signals (App. D) and shifted S4 planes (App. E) on
// the full (k, l) plane: n_combos combinations of `order` operands each, operand
// i of combination q at ops[order q + i] = (real channel, imaginary channel or
// -1, sign of j: -1 for the conjugate signal, else 1); accumulated at
// acc[plane][q][rows][cols] with rows = cols = 2M - 1 (S2: [q][2M - 1]).
cudaError_t launch_k5_complex(const float2* spec, long long chan_stride, int G, int m, int M,
                              int Mp, int order, const int4* ops, int n_combos, int shift,
                              bool natural, double* acc, long long plane, int nsm,
                              cudaStream_t stream);

// K2 for isolated grid points of one channel (pts: n_pts (k, l) pairs)
// One channel: independent warps on 32 x 32 sub-tiles (the plan's list of those
// with more than 8 points of the domain; k2_points takes the others' points).
// tm32 / tm64w: boxes of 2 / 4 blocks (32 / 64 bins) x kFrames84w frame rows.
constexpr int kFrames84w = 4;
cudaError_t launch_k2_bispec84w(const CUtensorMap& tm32, const CUtensorMap& tm64w, int row0,
                                int G, int m, int M, const TileInfo* tiles, int n_tiles,
                                float pref3, double* acc, long long plane, int nsm, int* counter,
                                int* status, int inject_timeout, cudaStream_t stream);
cudaError_t launch_k2_points(const float2* spec, int Mp, int G, int m, const int2* pts,
                             int n_pts, int M, float pref3, double* acc, long long plane,
                             cudaStream_t stream);

// the one-channel S4 cut at l = M - 1 for every k, stored at [l][k]
cudaError_t launch_k3_column(const float2* spec, int Mp, int G, int m, int M, float pref4a,
                             float pref4b, double* acc, long long plane, cudaStream_t stream);

// dynamic shared memory of the pair kernels for FC frames per stage
size_t k2_smem_bytes(int FC);
size_t k3_smem_bytes(int FC);

// K4: mean and standard error over G groups of the float64 sums in acc, or, with
// prev, of the sums acc - prev (the groups since a snapshot: sequential spectra).
cudaError_t launch_k4_finalize(const double* acc, int n_combos, int rows, int M, int layout,
                               long long G, double norm, double* out, double* err,
                               cudaStream_t stream, const double* prev = nullptr);

// dst[i] += src[i], i < n (device pointers): merges exported group sums.
cudaError_t launch_add_f64(double* dst, const double* src, long long n, cudaStream_t stream);

// Layout codes of launch_k4_finalize.
enum { kLayoutVector = 0,       // S2: [M]
       kLayoutS3Single = 1,     // one channel, computed for k <= l, mirrored; k+l <= M-1
       kLayoutS4Single = 2,     // one channel, computed for k <= l, mirrored
       kLayoutCross = 3,        // full [2M-1][M] grid, no mirroring
       kLayoutS4Lower = 4 };    // one channel, point (k, l), k <= l, stored at [l][k]

}  // namespace ss
