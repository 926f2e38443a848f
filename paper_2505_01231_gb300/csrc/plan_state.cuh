// plan_state.cuh -- the plan object behind ss_plan_t, shared by the host
// runtime (plan.cu) and the autotuner (tune.cu); not part of the public ABI.
#pragma once

#include <string>
#include <vector>

#include "internal.cuh"

namespace ss {
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
};
}  // namespace ss

struct ss_plan_s {
  // configuration
  int C = 1, T = 0, M = 0, Mp = 0, m = 0, window = 0, dtype = 0, precision = 0;
  unsigned orders = 0;
  double dt = 1.0, win_param = 0.14;
  cudaStream_t stream = nullptr;
  cudaStream_t copy_stream = nullptr;
  int device = 0, nsm = 1;
  size_t elem = 4;
  std::vector<ss::Combo> c2, c3, c4;
  int rows3 = 0, rows4 = 0;
  // normalisation (Eq. 23, 28, 31 with the window scaled by 1/sqrt(sum g^2))
  double sg2 = 0, sg3 = 0, sg4 = 0, norm2 = 0, norm3 = 0, norm4 = 0;
  // device tables and buffers
  float* d_win = nullptr;
  float2* d_tw = nullptr;
  void* d_carry = nullptr;
  long long carry_n = 0;
  float2* d_spec = nullptr;
  int Gb_max = 0, Gb_user = 0;
  double *d_acc1 = nullptr, *d_acc2 = nullptr, *d_acc3 = nullptr, *d_acc4 = nullptr;
  size_t n_acc1 = 0, n_acc2 = 0, n_acc3 = 0, n_acc4 = 0;
  int estimator = SS_EST_UNBIASED;
  // interlaced spectra (Sec. 3): a plan fed the same record without its first
  // T/2 samples, whose groups are pooled with this plan's at finalize
  ss_plan_s* shadow = nullptr;
  long long skip = 0;       // samples still to drop (in the shadow plan)
  double* d_pool = nullptr;  // pooled accumulators of the two plans
  double sg1 = 0, norm1 = 0;  // sum g and the S1 scale sqrt(sum g^2) / sum g
  int* d_s2auto = nullptr;
  int4* d_s2cross = nullptr;
  int n_s2cross = 0;
  ss::TileInfo *d_tiles3 = nullptr, *d_tiles4 = nullptr;
  int* d_status = nullptr;
  int inject_timeout = 0;          // timeout test: K2 runs one bounded wait out
  int k2_variant = ss::kK2Tile84Stages2;  // K2 tiling (set by the autotuner or ss_set_tuning)
  int k1_mode = ss::kK1Auto;              // K1 form (likewise)
  float tune_ms[ss::kK1Modes + ss::kK2Variants] = {};  // last ss_autotune: pass ms per form
  // sequential spectra (Sec. 8): every seq_B groups, the block's means and errors
  // go to seq_out (blocks past seq_cap are counted, not written)
  int seq_B = 0;
  double* seq_out = nullptr;
  long long seq_cap = 0, seq_blocks = 0;
  double* d_prev = nullptr;  // the S2/S3/S4 sums at the end of the last block
  // complex-valued signals (App. D) and shifted S4 planes (App. E): per order
  // (index order - 2) the operands of its combinations, their float64 sums, and
  // each record's order and place in the caller's record list
  std::vector<int4> cx_ops[3];
  int4* d_cx_ops[3] = {nullptr, nullptr, nullptr};
  double* d_cx_acc[3] = {nullptr, nullptr, nullptr};
  size_t n_cx_acc[3] = {0, 0, 0};
  std::vector<int> cx_order;  // order of each record, in the caller's order
  int cx_shift = 0;
  int* d_counter = nullptr;        // work-queue counter of the pair kernels
  int FC = 0;                      // frames per staged chunk of the pair kernels
  CUtensorMap tm64{}, tm128{}, tm48{};  // 3-D views [rows = C*Gb_max*m][Mp/16][16] of the spectra
  CUtensorMap tm32w{}, tm64w{};          // the same with boxes of kFrames84w rows (k2_bispec84w)
  CUtensorMap tmx_ab{}, tmx_cd{};        // 2-D views [rows][Mp] (several channels, tensor cores)
  CUtensorMap tmx_sab{}, tmx_scd{};      // FP16X3: views of the bins' maxima [rows][Mp]
  CUtensorMap tm_img[4]{};               // 4-D views of each channel's Gram operand image
  ss::TileInfo* d_tiles4tc = nullptr;  // tiles of the tensor-core S4 kernel (one channel)
  int4* d_c4cross = nullptr;       // (a, b, c, d) of each S4 combination (several channels)
  int n_tiles4tc = 0;
  ss::OperandImage oi;                 // K1's second output for the tensor-core S4 kernel
  int n_tiles3 = 0, n_tiles4 = 0;
  int2* d_pts3 = nullptr;  // isolated S3 grid points of one channel (k2_points)
  // the independent-warp K2 form: its 32 x 32 sub-tiles and their isolated points
  ss::TileInfo* d_tiles3w = nullptr;
  int2* d_pts3w = nullptr;
  int n_tiles3w = 0, n_pts3w = 0;
  bool col4 = false;       // the S4 column l = M - 1 is left to k3_column
  int n_pts3 = 0;
  long long pairs3 = 0, pairs4 = 0;
  void* d_stage[2] = {nullptr, nullptr};
  long long stage_n = 0;
  cudaEvent_t ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  double* d_out = nullptr;
  size_t out_doubles = 0;
  size_t device_bytes = 0;
  // progress
  long long groups = 0, samples = 0;
  // timing
  bool timing = false;
  std::vector<ss::EventPair> ev[5];
  long long launches[5] = {0, 0, 0, 0, 0};
  // errors
  bool broken = false;
  std::string err;
};


namespace ss {
// K1 -> K2 -> K3 over n samples per channel already on the device (channel c
// at ptr + c * stride elements), with carry-over; defined in plan.cu.
ss_status run_device_chunk(ss_plan_s* p, const void* ptr, long long n, long long stride);
// zero the accumulators, the carry-over and the statistics (stream-ordered)
ss_status reset_state(ss_plan_s* p);
// record a failure on the plan (or the thread's plan-less error) and return st
ss_status plan_fail(ss_plan_s* p, ss_status st, const std::string& msg);
}  // namespace ss
