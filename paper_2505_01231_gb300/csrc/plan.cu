// plan.cu -- host runtime behind the C ABI of include/polyspec.h.
//
// A plan owns the window and twiddle tables, the carry-over of samples that do
// not yet complete a group, the scratch of centred spectra for one batch of
// groups, and the float64 accumulators (sum and sum of squares of every
// per-group estimate, Sec. 4.2).  ss_accumulate cuts the concatenation
// carry-over | chunk into whole groups of m frames (Sec. 3, Eq. 16) and runs,
// batch after batch on the plan's stream,
//   K1 frame/window/FFT/centre + S2 -> K2 bispectrum (per S3 combination)
//   -> K3 trispectrum cut (per S4 combination);
// ss_finalize runs K4 (mean and standard error, Eq. 35-36) and copies out.
// Host chunks are copied to the device through two staging buffers on a
// separate copy stream, so the copy of one piece overlaps the kernels of the
// previous one.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include <cudaTypedefs.h>

#include "internal.cuh"
#include "plan_state.cuh"

using namespace ss;

namespace {

thread_local std::string g_plan_error;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

}  // namespace


namespace {

ss_status fail(ss_plan_s* p, ss_status st, const std::string& msg) {
  if (p) {
    p->err = msg;
    if (st == SS_ECUDA) p->broken = true;
  } else {
    g_plan_error = msg;
  }
  return st;
}

ss_status cuda_fail(ss_plan_s* p, cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a non-sticky error
  return fail(p, e == cudaErrorMemoryAllocation ? SS_ENOMEM : SS_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define SS_TRY(p, call)                                        \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail((p), e_, #call);   \
  } while (0)

template <typename T>
cudaError_t dev_alloc(ss_plan_s* p, T** ptr, size_t bytes) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), bytes);
  if (e == cudaSuccess) p->device_bytes += bytes;
  return e;
}

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Default combinations (Sec. 9): every multiset for S2 and S3, every unordered
// pair of unordered channel pairs for the S4 cut C4(a_k, b_k*, c_l, d_l*).
void default_combos(ss_plan_s* p) {
  const int C = p->C;
  if (p->orders & SS_ORDER2)
    for (int a = 0; a < C; ++a)
      for (int b = a; b < C; ++b) p->c2.push_back({2, {a, b, -1, -1}});
  if (p->orders & SS_ORDER3)
    for (int a = 0; a < C; ++a)
      for (int b = a; b < C; ++b)
        for (int c = b; c < C; ++c) p->c3.push_back({3, {a, b, c, -1}});
  if (p->orders & SS_ORDER4) {
    std::vector<std::pair<int, int>> pairs;
    for (int a = 0; a < C; ++a)
      for (int b = a; b < C; ++b) pairs.push_back({a, b});
    for (size_t i = 0; i < pairs.size(); ++i)
      for (size_t j = i; j < pairs.size(); ++j)
        p->c4.push_back({4, {pairs[i].first, pairs[i].second, pairs[j].first, pairs[j].second}});
  }
}

bool in_domain3(int k, int l, int M, bool cross) {
  if (cross) return l >= 0 && l < M && k > -M && k < M && k + l < M && k + l > -M;
  return k >= 0 && k <= l && k + l < M;
}

// Tiles of the tensor-core S4 kernel that touch the upper triangle k <= l < M:
// 128 k-bins by up to 128 l-bins; the last l-block is cut to the bins left,
// rounded up to the 16-column granule of the MMA.
// Tensor-core tiles of the upper triangle k <= l.  A last column block that
// holds only the column l = M - 1 (M = T/2 + 1 with T a multiple of 256) is
// left to k3_column (*last_col = true): a 16-column tile per k block would
// cost a full operand load per group for one column.
std::vector<TileInfo> build_tc_tiles(int M, bool* last_col) {
  std::vector<TileInfo> t;
  *last_col = false;
  for (int k0 = 0; k0 < M; k0 += kTcTileM)
    for (int l0 = 0; l0 < M; l0 += kTcTileN) {
      const int n = std::min(kTcTileN, (M - l0 + 15) & ~15);
      if (M - l0 == 1 && M > 1) {
        *last_col = true;
        continue;
      }
      if (k0 <= l0 + n - 1) t.push_back(TileInfo{k0, l0, 8, n});
    }
  return t;
}

// Tiles of 64 x 64 grid points that touch the domain, with the number of
// their 32 x 16 warp sub-tiles that touch it (the kernels skip the others).
// A one-channel S3 tile holding at most this many domain points (the corner
// tiles cut by k + l = M - 1) is left to k2_points.
constexpr int kIsolatedPoints = 8;

void build_tiles(int M, bool cross, std::vector<TileInfo>& t3, std::vector<TileInfo>& t4,
                 std::vector<int2>& pts3, long long* pairs3, long long* pairs4) {
  *pairs3 = 0;
  *pairs4 = 0;
  auto warps = [&](int k0, int l0, auto in_dom) {
    int w = 0;
    for (int wi = 0; wi < kThreadsPair / 32; ++wi) {
      const int kw = k0 + 32 * (wi & 1), lw = l0 + 16 * (wi >> 1);
      bool any = false;
      for (int a = 0; a < 32 && !any; ++a)
        for (int b = 0; b < 16 && !any; ++b) any = in_dom(kw + a, lw + b);
      w += any ? 1 : 0;
    }
    return w;
  };
  auto dom3 = [&](int k, int l) { return in_domain3(k, l, M, cross); };
  auto dom4 = [&](int k, int l) {
    return cross ? (l >= 0 && l < M && k > -M && k < M) : (k >= 0 && k <= l && l < M);
  };
  const int kmin = cross ? -((M - 1 + kTile - 1) / kTile) * kTile : 0;
  for (int k0 = kmin; k0 < M; k0 += kTile)
    for (int l0 = 0; l0 < M; l0 += kTile) {
      const int w3 = warps(k0, l0, dom3), w4 = warps(k0, l0, dom4);
      std::vector<int2> in3;
      if (w3 && !cross)
        for (int a = 0; a < kTile && (int)in3.size() <= kIsolatedPoints; ++a)
          for (int b = 0; b < kTile && (int)in3.size() <= kIsolatedPoints; ++b)
            if (dom3(k0 + a, l0 + b)) in3.push_back(make_int2(k0 + a, l0 + b));
      if (w3 && !cross && (int)in3.size() <= kIsolatedPoints)
        pts3.insert(pts3.end(), in3.begin(), in3.end());
      else if (w3)
        t3.push_back(TileInfo{k0, l0, w3, 0});
      if (w4) t4.push_back(TileInfo{k0, l0, w4, 0});
    }
  for (int k = -(M - 1); k < M; ++k)
    for (int l = 0; l < M; ++l) {
      if (dom3(k, l)) ++*pairs3;
      if (dom4(k, l)) ++*pairs4;
    }
}

// One channel, k2_bispec84w: the 32 x 32 sub-tiles that hold more than
// kIsolatedPoints points of the S3 domain (0 <= k <= l, k + l <= M - 1), and the
// points of the others (where the edge k + l = M - 1 passes a sub-tile corner),
// which k2_points evaluates.
void build_warp_tiles(int M, std::vector<TileInfo>& t, std::vector<int2>& pts) {
  constexpr int kW = 32;
  for (int k0 = 0; k0 < M; k0 += kW)
    for (int l0 = 0; l0 < M; l0 += kW) {
      std::vector<int2> in;
      for (int a = 0; a < kW && (int)in.size() <= kIsolatedPoints; ++a)
        for (int b = 0; b < kW && (int)in.size() <= kIsolatedPoints; ++b)
          if (in_domain3(k0 + a, l0 + b, M, 0)) in.push_back(make_int2(k0 + a, l0 + b));
      if ((int)in.size() > kIsolatedPoints)
        t.push_back(TileInfo{k0, l0, 1, kW});
      else
        pts.insert(pts.end(), in.begin(), in.end());
    }
}

void record(ss_plan_s* p, int stage, cudaStream_t s, bool start) {
  if (!p->timing) return;
  if (start) {
    EventPair e;
    cudaEventCreate(&e.a);
    cudaEventCreate(&e.b);
    cudaEventRecord(e.a, s);
    p->ev[stage].push_back(e);
  } else {
    cudaEventRecord(p->ev[stage].back().b, s);
    ++p->launches[stage];
  }
}

void clear_events(ss_plan_s* p) {
  for (auto& v : p->ev) {
    for (auto& e : v) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    v.clear();
  }
  for (auto& l : p->launches) l = 0;
}

// Sequential spectra (Sec. 8): the block of seq_B groups that just ended gives
// its means and standard errors (the sums since the snapshot, over seq_B groups)
// in the finalize layout at block index seq_blocks of seq_out; then the snapshot
// moves to the current sums.
ss_status emit_block(ss_plan_s* p) {
  const long long b = p->seq_blocks++;
  const size_t n2 = p->c2.size() * p->M * 2;
  const size_t n3 = p->c3.size() * p->rows3 * p->M * 2;
  const size_t n4 = p->c4.size() * p->rows4 * p->M * 2;
  if (b < p->seq_cap) {
    double* o2 = p->seq_out + (size_t)b * 2 * (n2 + n3 + n4);
    double* e2 = o2 + n2;
    double* o3 = e2 + n2;
    double* e3 = o3 + n3;
    double* o4 = e3 + n3;
    double* e4 = o4 + n4;
    const double* q2 = p->d_prev;
    const double* q3 = q2 + p->n_acc2;
    const double* q4 = q3 + p->n_acc3;
    if (n2)
      SS_TRY(p, launch_k4_finalize(p->d_acc2, (int)p->c2.size(), 1, p->M, kLayoutVector,
                                   p->seq_B, p->norm2, o2, e2, p->stream, q2));
    if (n3)
      SS_TRY(p, launch_k4_finalize(p->d_acc3, (int)p->c3.size(), p->rows3, p->M,
                                   p->C == 1 ? kLayoutS3Single : kLayoutCross, p->seq_B,
                                   p->norm3, o3, e3, p->stream, q3));
    if (n4)
      SS_TRY(p, launch_k4_finalize(p->d_acc4, (int)p->c4.size(), p->rows4, p->M,
                                   p->C != 1                        ? kLayoutCross
                                   : p->precision == SS_PREC_FP32 ? kLayoutS4Single
                                                                   : kLayoutS4Lower,
                                   p->seq_B, p->norm4, o4, e4, p->stream, q4));
  }
  const std::pair<const double*, size_t> parts[3] = {
      {p->d_acc2, p->n_acc2}, {p->d_acc3, p->n_acc3}, {p->d_acc4, p->n_acc4}};
  double* q = p->d_prev;
  for (const auto& pr : parts) {
    if (pr.second)
      SS_TRY(p, cudaMemcpyAsync(q, pr.first, pr.second * sizeof(double),
                                cudaMemcpyDeviceToDevice, p->stream));
    q += pr.second;
  }
  return SS_OK;
}

// Process n samples per channel that are already on the device (channel c at
// ptr + c * stride elements).
ss_status process_device(ss_plan_s* p, const void* ptr, long long n, long long stride) {
  const long long per_group = (long long)p->m * p->T;
  const long long total = p->carry_n + n;
  const long long Gn = total / per_group;
  const char* base = static_cast<const char*>(ptr);
  if (Gn > 0) {
    const long long nb = (Gn + p->Gb_max - 1) / p->Gb_max;
    const long long gb = (Gn + nb - 1) / nb;
    SampleSource src;
    src.carry = p->d_carry;
    src.carry_n = p->carry_n;
    src.carry_stride = per_group;
    src.chunk = ptr;
    src.chunk_stride = stride;
    src.dtype = p->dtype;
    const long long chan_stride = (long long)p->Gb_max * p->m * p->Mp;
    // prefactors of c2, c3 and the two parts of c4 over the centred sums: the
    // k-statistics (Eq. 32-34, 85) or the natural estimators
    const double md = p->m;
    const bool nat = p->estimator == SS_EST_NATURAL;
    const float pref2 = (float)(nat ? 1.0 / md : 1.0 / (md - 1));
    const float pref3 = (float)(nat ? 1.0 / md : md / ((md - 1) * (md - 2)));
    const float pref4a =
        (float)(nat ? 1.0 / md : md * (md + 1) / ((md - 1) * (md - 2) * (md - 3)));
    const float pref4b = (float)(nat ? 1.0 / (md * md) : 1.0 / ((md - 2) * (md - 3)));
    for (long long g0 = 0; g0 < Gn;) {
      long long take = std::min(gb, Gn - g0);
      // sequential spectra: a batch ends where a block of seq_B groups ends
      if (p->seq_B > 0) take = std::min(take, p->seq_B - (p->groups + g0) % p->seq_B);
      const int cnt = (int)take;
      record(p, 0, p->stream, true);
      SS_TRY(p, launch_k1_spectra(src, g0 * per_group, cnt, p->C, p->T, p->m, p->M, p->Mp,
                                  p->d_win, p->d_tw, p->d_spec, chan_stride, p->d_s2auto,
                                  p->d_acc2, (int)p->c2.size(), pref2, 4 * p->nsm, p->stream,
                                  p->oi, p->d_acc1, p->k1_mode));
      if (p->n_s2cross > 0)
        SS_TRY(p, launch_k1_cross_s2(p->d_spec, chan_stride, cnt, p->m, p->M, p->Mp,
                                     p->d_s2cross, p->n_s2cross, pref2, p->d_acc2,
                                     (long long)p->c2.size() * p->M, p->nsm, p->stream));
      record(p, 0, p->stream, false);
      if (!p->c3.empty()) {
        record(p, 1, p->stream, true);
        const long long plane = (long long)p->c3.size() * p->rows3 * p->M;
        for (size_t i = 0; i < p->c3.size(); ++i) {
          const Combo& cb = p->c3[i];
          const int row_stride = p->Gb_max * p->m;
          double* acc3 = p->d_acc3 + (long long)i * p->rows3 * p->M;
          const bool warps = p->k2_variant == kK2Warp84 && p->C == 1;
          if (warps)
            SS_TRY(p, launch_k2_bispec84w(p->tm32w, p->tm64w, cb.c[0] * row_stride, cnt, p->m,
                                          p->M, p->d_tiles3w, p->n_tiles3w, pref3, acc3, plane,
                                          p->nsm, p->d_counter, p->d_status, p->inject_timeout,
                                          p->stream));
          else
            SS_TRY(p, launch_k2_bispec(p->tm64, p->tm128, p->d_spec + cb.c[0] * chan_stride,
                                       p->d_spec + cb.c[1] * chan_stride,
                                       p->d_spec + cb.c[2] * chan_stride, cb.c[0] * row_stride,
                                       cb.c[1] * row_stride, cb.c[2] * row_stride, cnt, p->m,
                                       p->FC, p->M, p->Mp, p->d_tiles3, p->n_tiles3,
                                       p->C > 1 ? 1 : 0, pref3, acc3, plane, p->rows3, p->nsm,
                                       p->d_counter, p->d_status, p->inject_timeout,
                                       p->k2_variant == kK2Warp84 ? kK2Tile84Stages2
                                                                  : p->k2_variant,
                                       p->stream));
          const int2* pts = warps ? p->d_pts3w : p->d_pts3;
          const int npts = warps ? p->n_pts3w : p->n_pts3;
          if (p->C == 1 && npts > 0)
            SS_TRY(p, launch_k2_points(p->d_spec + cb.c[0] * chan_stride, p->Mp, cnt, p->m, pts,
                                       npts, p->M, pref3, acc3, plane, p->stream));
        }
        record(p, 1, p->stream, false);
      }
      if (!p->c4.empty()) {
        record(p, 2, p->stream, true);
        const long long plane = (long long)p->c4.size() * p->rows4 * p->M;
        if (p->C > 1 && p->precision == SS_PREC_FP32)
          SS_TRY(p, launch_k3_trispec_cross(p->d_spec, chan_stride, cnt, p->m, p->M, p->Mp,
                                            p->d_c4cross, (int)p->c4.size(), p->d_acc4, plane,
                                            p->nsm, nat, p->stream));
        else if (p->C > 1) {
          CrossViews v;
          v.tm_ab = &p->tmx_ab;
          v.tm_cd = &p->tmx_cd;
          v.tm_sab = p->oi.rmax ? &p->tmx_sab : nullptr;
          v.tm_scd = p->oi.rmax ? &p->tmx_scd : nullptr;
          v.chan_rows = p->Gb_max * p->m;
          v.grp_rows = p->Gb_max;
          v.f16 = p->oi.rmax != nullptr;
          SS_TRY(p, launch_k3_trispec_cross_tc(v, cnt, p->m, p->M, p->Mp, p->d_c4cross,
                                               (int)p->c4.size(), p->d_acc4, plane, p->nsm, nat,
                                               p->d_counter, p->d_status, p->stream));
        }
        for (size_t i = 0; i < p->c4.size() && p->C == 1; ++i) {
          const Combo& cb = p->c4[i];
          if (p->precision == SS_PREC_FP32)
            SS_TRY(p, launch_k3_trispec(p->tm64, cb.c[0] * p->Gb_max * p->m, cnt, p->m, p->FC,
                                        p->M, p->d_tiles4, p->n_tiles4, pref4a, pref4b,
                                        p->d_acc4 + (long long)i * p->rows4 * p->M, plane,
                                        p->nsm, p->d_counter, p->d_status, p->stream));
          else
            SS_TRY(p, launch_k3_trispec_tc(p->tm_img[cb.c[0]], p->oi, cb.c[0], cnt, p->m, p->M,
                                           p->Mp,
                                           p->d_tiles4tc, p->n_tiles4tc, p->precision,
                                           p->d_acc4 + (long long)i * p->rows4 * p->M, plane,
                                           p->nsm, p->d_counter, p->d_status, p->stream));
          if (p->precision != SS_PREC_FP32 && p->col4)
            SS_TRY(p, launch_k3_column(p->d_spec + cb.c[0] * chan_stride, p->Mp, cnt, p->m,
                                       p->M, pref4a, pref4b,
                                       p->d_acc4 + (long long)i * p->rows4 * p->M, plane,
                                       p->stream));
        }
        record(p, 2, p->stream, false);
      }
      // spectra of complex-valued signals and shifted S4 planes (App. D, E)
      for (int o = 0; o < 3; ++o) {
        if (p->cx_ops[o].empty()) continue;
        record(p, 2, p->stream, true);
        const int n_cx = (int)(p->cx_ops[o].size() / (o + 2));
        const long long cplane = (long long)p->n_cx_acc[o] / kPlanes;
        SS_TRY(p, launch_k5_complex(p->d_spec, chan_stride, cnt, p->m, p->M, p->Mp, o + 2,
                                    p->d_cx_ops[o], n_cx, p->cx_shift, nat, p->d_cx_acc[o],
                                    cplane, p->nsm, p->stream));
        record(p, 2, p->stream, false);
      }
      g0 += take;
      if (p->seq_B > 0 && (p->groups + g0) % p->seq_B == 0) {
        ss_status st = emit_block(p);
        if (st != SS_OK) return st;
      }
    }
  }
  // keep the samples that do not complete a group
  const long long left = total - Gn * per_group;
  const size_t e = p->elem;
  char* carry = static_cast<char*>(p->d_carry);
  for (int c = 0; c < p->C; ++c) {
    char* dst = carry + (size_t)c * per_group * e;
    const char* src = base + (size_t)c * stride * e;
    if (Gn == 0) {
      if (n > 0)
        SS_TRY(p, cudaMemcpyAsync(dst + p->carry_n * e, src, n * e, cudaMemcpyDeviceToDevice,
                                  p->stream));
    } else if (left > 0) {
      SS_TRY(p, cudaMemcpyAsync(dst, src + (n - left) * e, left * e, cudaMemcpyDeviceToDevice,
                                p->stream));
    }
  }
  p->carry_n = left;
  p->groups += Gn;
  p->samples += n;
  return SS_OK;
}

// A kernel whose bounded wait gave up leaves a non-zero device status; the
// sums of that launch are incomplete, so the plan is marked unusable.
ss_status check_status(ss_plan_s* p) {
  int st = 0;
  if (p->shadow) {
    SS_TRY(p, cudaMemcpy(&st, p->shadow->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != kStatusOk) {
      p->broken = true;
      return fail(p, SS_ETIMEOUT, "a device-side wait for staged data gave up; results discarded");
    }
  }
  SS_TRY(p, cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != kStatusOk) {
    p->broken = true;
    return fail(p, SS_ETIMEOUT, "a device-side wait for staged data gave up; results discarded");
  }
  return SS_OK;
}

ss_status ensure_stage(ss_plan_s* p) {
  if (p->d_stage[0]) return SS_OK;
  // one device batch of samples per staging buffer (within 32 Mi and 256 Mi
  // samples per channel), so a staged piece runs as one full batch of groups
  const long long batch = (long long)p->Gb_max * p->m * p->T;
  p->stage_n = std::max(32ll << 20, std::min(256ll << 20, batch)) / std::max(1, p->C);
  for (int i = 0; i < 2; ++i) {
    SS_TRY(p, dev_alloc(p, &p->d_stage[i], (size_t)p->stage_n * p->C * p->elem));
    SS_TRY(p, cudaEventCreateWithFlags(&p->ev_ready[i], cudaEventDisableTiming));
    SS_TRY(p, cudaEventCreateWithFlags(&p->ev_free[i], cudaEventDisableTiming));
  }
  SS_TRY(p, cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
  return SS_OK;
}

// Pass samples on to the interlaced window set: the same stream, less its
// first T/2 samples.
ss_status feed_shadow(ss_plan_s* p, const void* ptr, long long n, long long stride) {
  ss_plan_s* s = p->shadow;
  if (!s || n <= 0) return SS_OK;
  const long long skip = std::min(s->skip, n);
  s->skip -= skip;
  if (n - skip <= 0) return SS_OK;
  ss_status st = process_device(s, static_cast<const char*>(ptr) + (size_t)skip * s->elem,
                                n - skip, stride);
  if (st != SS_OK) return fail(p, st, "interlaced window set: " + s->err);
  return SS_OK;
}

ss_status process_host(ss_plan_s* p, const void* chunk, long long n) {
  ss_status st = ensure_stage(p);
  if (st != SS_OK) return st;
  const char* src = static_cast<const char*>(chunk);
  const size_t e = p->elem;
  // pieces of about a quarter of the call in whole groups (at least 32 Mi
  // samples, at most a staging buffer), so that the copies of all but the first
  // piece overlap the kernels of the one before
  const long long per_group = (long long)p->m * p->T;
  long long step = (n + 3) / 4;
  step = (step + per_group - 1) / per_group * per_group;
  step = std::min(p->stage_n, std::max(step, std::min(p->stage_n, (32ll << 20) / p->C)));
  int piece = 0;
  for (long long off = 0; off < n; off += step, ++piece) {
    const int b = piece & 1;
    const long long len = std::min(step, n - off);
    SS_TRY(p, cudaStreamWaitEvent(p->copy_stream, p->ev_free[b], 0));
    record(p, 4, p->copy_stream, true);
    for (int c = 0; c < p->C; ++c)
      SS_TRY(p, cudaMemcpyAsync(static_cast<char*>(p->d_stage[b]) + (size_t)c * p->stage_n * e,
                                src + ((size_t)c * n + off) * e, len * e,
                                cudaMemcpyHostToDevice, p->copy_stream));
    record(p, 4, p->copy_stream, false);
    SS_TRY(p, cudaEventRecord(p->ev_ready[b], p->copy_stream));
    SS_TRY(p, cudaStreamWaitEvent(p->stream, p->ev_ready[b], 0));
    st = process_device(p, p->d_stage[b], len, p->stage_n);
    if (st == SS_OK) st = feed_shadow(p, p->d_stage[b], len, p->stage_n);
    if (st != SS_OK) return st;
    SS_TRY(p, cudaEventRecord(p->ev_free[b], p->stream));
  }
  // the caller may reuse its buffer once every copy out of it has finished
  SS_TRY(p, cudaStreamSynchronize(p->copy_stream));
  return SS_OK;
}

ss_status zero_state(ss_plan_s* p) {
  if (p->d_status) SS_TRY(p, cudaMemsetAsync(p->d_status, 0, sizeof(int), p->stream));
  if (p->d_acc1) SS_TRY(p, cudaMemsetAsync(p->d_acc1, 0, p->n_acc1 * sizeof(double), p->stream));
  if (p->d_acc2) SS_TRY(p, cudaMemsetAsync(p->d_acc2, 0, p->n_acc2 * sizeof(double), p->stream));
  if (p->d_acc3) SS_TRY(p, cudaMemsetAsync(p->d_acc3, 0, p->n_acc3 * sizeof(double), p->stream));
  if (p->d_acc4) SS_TRY(p, cudaMemsetAsync(p->d_acc4, 0, p->n_acc4 * sizeof(double), p->stream));
  if (p->d_prev)
    SS_TRY(p, cudaMemsetAsync(p->d_prev, 0,
                              (p->n_acc2 + p->n_acc3 + p->n_acc4) * sizeof(double), p->stream));
  for (int o = 0; o < 3; ++o)
    if (p->d_cx_acc[o])
      SS_TRY(p, cudaMemsetAsync(p->d_cx_acc[o], 0, p->n_cx_acc[o] * sizeof(double), p->stream));
  p->seq_blocks = 0;
  p->carry_n = 0;
  p->groups = 0;
  p->samples = 0;
  clear_events(p);
  return SS_OK;
}

// 3-D tensor maps over the centred spectra: element (x, y, z) is bin 16 y + x of
// frame row z (rows of channel c start at c * Gb_max * m).  Boxes are 16 bins x
// 4 or 8 blocks x FC rows, written to shared memory with 128-byte swizzling;
// blocks past the row read as zero.
ss_status encode_maps(ss_plan_s* p) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(p, SS_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t rows = (cuuint64_t)p->C * p->Gb_max * p->m;
  const cuuint64_t dims[3] = {16, (cuuint64_t)p->Mp / 16, rows};
  const cuuint64_t strides[2] = {16 * sizeof(float2), (cuuint64_t)p->Mp * sizeof(float2)};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int blocks : {3, 4, 8}) {
    const cuuint32_t box[3] = {16, (cuuint32_t)blocks, (cuuint32_t)p->FC};
    CUtensorMap* map = blocks == 3 ? &p->tm48 : blocks == 4 ? &p->tm64 : &p->tm128;
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                        p->d_spec, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      return fail(p, SS_ECUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string(r));
  }
  for (int blocks : {2, 4}) {  // boxes of kFrames84w rows for k2_bispec84w
    const cuuint32_t box[3] = {16, (cuuint32_t)blocks, (cuuint32_t)kFrames84w};
    CUresult r = encode(blocks == 2 ? &p->tm32w : &p->tm64w, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                        p->d_spec, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      return fail(p, SS_ECUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string(r));
  }
  if (p->C > 1) {
    // 2-D views [rows][Mp] for the tensor-core cross S4: boxes of 4 frame rows (8 for
    // FP16X3) by min(box bins, Mp) bins (rows of a and b) or by the column box
    // (c and d); the widths differ between the two forms
    const cuuint32_t fr = p->precision == SS_PREC_FP16X3 ? 8 : 4;
    const cuuint64_t d2[2] = {(cuuint64_t)p->Mp, rows};
    const cuuint64_t s2[1] = {(cuuint64_t)p->Mp * sizeof(float2)};
    const cuuint32_t e2[2] = {1, 1};
    const bool h = p->precision == SS_PREC_FP16X3;
    const cuuint32_t bab[2] = {(cuuint32_t)std::min(h ? kCrossBoxBinsH : kCrossBoxBins, p->Mp), fr};
    const cuuint32_t bcd[2] = {(cuuint32_t)(h ? kCrossColBoxH : kCrossColBox), fr};
    for (int i = 0; i < 2; ++i) {
      CUresult r = encode(i == 0 ? &p->tmx_ab : &p->tmx_cd, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                          p->d_spec, d2, s2, i == 0 ? bab : bcd, e2,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return fail(p, SS_ECUDA,
                    "cuTensorMapEncodeTiled (cross views) failed with code " + std::to_string(r));
    }
  }
  if (p->oi.rmax) {
    // the bins' row scales: [channel x Gb_max + group][Mp] floats, boxes of one row
    const cuuint64_t d2[2] = {(cuuint64_t)p->Mp, (cuuint64_t)p->C * p->Gb_max};
    const cuuint64_t s2[1] = {(cuuint64_t)p->Mp * sizeof(float)};
    const cuuint32_t e2[2] = {1, 1};
    const cuuint32_t bab[2] = {(cuuint32_t)std::min(kCrossScaleBins, p->Mp), 1};
    const cuuint32_t bcd[2] = {(cuuint32_t)kCrossScaleCols, 1};
    for (int i = 0; i < 2; ++i) {
      CUresult r = encode(i == 0 ? &p->tmx_sab : &p->tmx_scd, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                          p->oi.rmax, d2, s2, i == 0 ? bab : bcd, e2,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return fail(p, SS_ECUDA,
                    "cuTensorMapEncodeTiled (cross maxima) failed with code " + std::to_string(r));
    }
  }
  if (p->oi.img) {
    // Gram operand image of each channel as [group][row group][chunk][2 CB bytes]
    // in 8-byte elements; a box is the stage's chunks of 16 row groups of one group
    const cuuint64_t cbytes = p->oi.rg_bytes / p->oi.nkc;  // 2 CB
    const cuuint64_t idims[4] = {cbytes / 8, (cuuint64_t)p->oi.nkc, (cuuint64_t)p->Mp / 8,
                                 (cuuint64_t)p->Gb_max};
    const cuuint64_t istr[3] = {cbytes, (cuuint64_t)p->oi.rg_bytes,
                                (cuuint64_t)p->oi.group_bytes};
    const cuuint32_t ibox[4] = {(cuuint32_t)(cbytes / 8),
                                (cuuint32_t)k3tc_stage_chunks(p->precision), 16, 1};
    const cuuint32_t iestr[4] = {1, 1, 1, 1};
    for (int c = 0; c < p->C; ++c) {
      CUresult r = encode(&p->tm_img[c], CU_TENSOR_MAP_DATA_TYPE_UINT64, 4,
                          static_cast<char*>(p->oi.img) + (size_t)c * p->oi.chan_bytes, idims,
                          istr, ibox, iestr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return fail(p, SS_ECUDA,
                    "cuTensorMapEncodeTiled (operand image) failed with code " + std::to_string(r));
    }
  }
  return SS_OK;
}

// Weights of the Gram contraction of the tensor-core S4 with the prefactor r
// folded in (see OperandImage): for the k-statistic (Eq. 85) w_jj = m^2 - m + 2,
// w_jj' = -4(m-1), S_k S_l weight m-1, r = 1/((m-1)(m-2)(m-3)); for the natural
// estimator, c4 = [(m-2) sum_j P_jk P_jl - 4 sum_{j<j'} G G - S_k S_l] / m^2
// (the same regrouping of |U|^2 + |V|^2), so w_jj = m-2, w_jj' = -4, weight 1,
// r = 1/m^2.
void set_image_scales(ss_plan_s* p) {
  const double md = p->m;
  if (p->estimator == SS_EST_NATURAL) {
    const double r = 1.0 / (md * md);
    p->oi.sd = (float)std::sqrt((md - 2.0) * r);
    p->oi.so = (float)std::sqrt(4.0 * r);
    p->oi.sp = (float)std::sqrt(r);
  } else {
    const double r = 1.0 / ((md - 1.0) * (md - 2.0) * (md - 3.0));
    p->oi.sd = (float)std::sqrt((md * md - md + 2.0) * r);
    p->oi.so = (float)std::sqrt(4.0 * (md - 1.0) * r);
    p->oi.sp = (float)std::sqrt((md - 1.0) * r);
  }
}

ss_status alloc_spec(ss_plan_s* p) {
  auto release = [&](void*& ptr, size_t bytes) {
    if (ptr) {
      cudaFree(ptr);
      p->device_bytes -= bytes;
      ptr = nullptr;
    }
  };
  const size_t spec_group = (size_t)p->C * p->m * p->Mp * sizeof(float2);
  const bool image = p->C == 1 && !p->c4.empty() && p->precision != SS_PREC_FP32;
  // Gram image: ceil(m/16) diagonal chunks, then ceil((m(m-1)/2 + 1) / 16) chunks
  // of the pairs and ps
  const int ndc = (p->m + 15) / 16;
  const int nkc = ndc + (p->m * (p->m - 1) / 2 + 16) / 16;
  const size_t cb = p->precision == SS_PREC_TF32X3 ? 512 : 256;
  const size_t rg_bytes = (size_t)nkc * 2 * cb;
  const size_t group_bytes = (size_t)(p->Mp / 8) * rg_bytes;
  const size_t img_group = image ? (size_t)p->C * group_bytes : 0;
  // FP16: the bins' row scales per group
  const bool scaled = image && p->precision == SS_PREC_FP16X3;
  const size_t rsc_group = scaled ? (size_t)p->C * p->Mp * sizeof(float) : 0;
  // several channels in FP16X3: the bins' row scales per group
  const bool cross16 = p->C > 1 && !p->c4.empty() && p->precision == SS_PREC_FP16X3;
  const size_t rmax_group = cross16 ? (size_t)p->C * p->Mp * sizeof(float) : 0;
  {
    void* r = p->oi.rmax;
    release(r, rmax_group * p->Gb_max);
    p->oi.rmax = nullptr;
    void* v = p->d_spec;
    release(v, spec_group * p->Gb_max);
    p->d_spec = nullptr;
    release(p->oi.img, img_group * p->Gb_max);
    void* w = p->oi.rsc;
    release(w, rsc_group * p->Gb_max);
    p->oi.rsc = nullptr;
  }
  const size_t per_group = spec_group + img_group + rsc_group + rmax_group;
  int gb = p->Gb_user;
  if (gb <= 0) {
    // about 4 GiB of per-batch scratch, at least one group
    gb = (int)std::max<size_t>(1, (size_t)(4096ull << 20) / per_group);
  }
  // the 3-D views index rows with 32-bit coordinates
  const long long max_rows = (1ll << 31) - 1;
  if ((long long)p->C * gb * p->m > max_rows) gb = (int)(max_rows / ((long long)p->C * p->m));
  p->Gb_max = gb;
  SS_TRY(p, dev_alloc(p, &p->d_spec, spec_group * gb));
  p->oi = OperandImage();
  if (image) {
    SS_TRY(p, dev_alloc(p, &p->oi.img, img_group * gb));
    if (scaled) SS_TRY(p, dev_alloc(p, &p->oi.rsc, rsc_group * gb));
    p->oi.fmt = p->precision == SS_PREC_TF32X3   ? kImageGramTF32
                : p->precision == SS_PREC_FP16X3 ? kImageGramF16
                                                 : kImageGramBF16;
    p->oi.nkc = nkc;
    p->oi.ndc = ndc;
    set_image_scales(p);
    p->oi.rg_bytes = (long long)rg_bytes;
    p->oi.group_bytes = (long long)group_bytes;
    p->oi.chan_bytes = (long long)gb * group_bytes;
    p->oi.chan_rsc = (long long)gb * p->Mp;
    // no tile reads the rows of bins from M - 1 on when k3_column takes that column
    p->oi.img_bins = p->col4 ? p->M - 1 : p->Mp;
  }
  if (cross16) {
    SS_TRY(p, dev_alloc(p, &p->oi.rmax, rmax_group * gb));
    p->oi.chan_rmax = (long long)gb * p->Mp;
  }
  return encode_maps(p);
}

void destroy(ss_plan_s* p) {
  if (!p) return;
  if (p->shadow) destroy(p->shadow);
  p->shadow = nullptr;
  cudaFree(p->d_pool);
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->copy_stream) {
    cudaStreamSynchronize(p->copy_stream);
    cudaStreamDestroy(p->copy_stream);
  }
  clear_events(p);
  for (int i = 0; i < 2; ++i) {
    if (p->ev_ready[i]) cudaEventDestroy(p->ev_ready[i]);
    if (p->ev_free[i]) cudaEventDestroy(p->ev_free[i]);
    cudaFree(p->d_stage[i]);
  }
  cudaFree(p->d_win);
  cudaFree(p->d_tw);
  cudaFree(p->d_carry);
  cudaFree(p->d_spec);
  cudaFree(p->oi.img);
  cudaFree(p->oi.rsc);
  cudaFree(p->oi.rmax);
  cudaFree(p->d_acc1);
  cudaFree(p->d_acc2);
  cudaFree(p->d_acc3);
  cudaFree(p->d_acc4);
  cudaFree(p->d_s2auto);
  cudaFree(p->d_s2cross);
  cudaFree(p->d_tiles3);
  cudaFree(p->d_pts3);
  cudaFree(p->d_tiles3w);
  cudaFree(p->d_pts3w);
  cudaFree(p->d_tiles4);
  cudaFree(p->d_tiles4tc);
  cudaFree(p->d_c4cross);
  cudaFree(p->d_status);
  cudaFree(p->d_counter);
  cudaFree(p->d_out);
  cudaFree(p->d_prev);
  for (int o = 0; o < 3; ++o) {
    cudaFree(p->d_cx_ops[o]);
    cudaFree(p->d_cx_acc[o]);
  }
  delete p;
}

}  // namespace

namespace ss {
ss_status run_device_chunk(ss_plan_s* p, const void* ptr, long long n, long long stride) {
  return process_device(p, ptr, n, stride);
}
ss_status reset_state(ss_plan_s* p) { return zero_state(p); }
ss_status plan_fail(ss_plan_s* p, ss_status st, const std::string& msg) { return fail(p, st, msg); }
}  // namespace ss

extern "C" {

const char* ss_version(void) { return "polyspec-gb300 0.1 (sm_103a)"; }

const char* ss_last_error(ss_plan_t plan) {
  return plan ? plan->err.c_str() : g_plan_error.c_str();
}

// ss_plan with a cap on groups per device batch applied before the scratch is
// allocated (0 = automatic).
static ss_status plan_create(ss_plan_t* out, int channels, int T, double dt, int m, int window,
                             double win_param, unsigned orders, int dtype, int precision,
                             const int* combos, int n_combos, void* stream, int batch) {
  if (!out) return fail(nullptr, SS_EINVAL, "out is NULL");
  *out = nullptr;
  if (channels < 1 || channels > 4) return fail(nullptr, SS_EINVAL, "channels must be 1..4");
  if (!is_pow2(T) || T < 8 || T > 4096)
    return fail(nullptr, SS_EINVAL, "T must be a power of two in [8, 4096]");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, SS_EINVAL, "dt must be > 0");
  if (orders == 0 || (orders & ~(unsigned)(SS_ORDER1 | SS_ORDER2 | SS_ORDER3 | SS_ORDER4)))
    return fail(nullptr, SS_EINVAL, "orders must be a non-empty OR of SS_ORDER1/2/3/4");
  if (m < 2) return fail(nullptr, SS_EINVAL, "S2 needs m >= 2 (Eq. 32)");
  if ((orders & SS_ORDER3) && m < 3) return fail(nullptr, SS_EINVAL, "S3 needs m >= 3 (Eq. 33)");
  if ((orders & SS_ORDER4) && m < 4) return fail(nullptr, SS_EINVAL, "S4 needs m >= 4 (Eq. 34)");
  if (window != SS_WIN_HANN && window != SS_WIN_ACG)
    return fail(nullptr, SS_EINVAL, "unknown window");
  if (window == SS_WIN_ACG && !(win_param > 0.0 && win_param < 10.0))
    return fail(nullptr, SS_EINVAL, "sigma_t of the confined Gaussian must be in (0, 10)");
  if (dtype != SS_F32 && dtype != SS_I16) return fail(nullptr, SS_EINVAL, "unknown dtype");
  if (precision < SS_PREC_FP32 || precision > SS_PREC_FP16X3)
    return fail(nullptr, SS_EINVAL, "unknown precision");
  if (combos && n_combos <= 0) return fail(nullptr, SS_EINVAL, "n_combos must be > 0");

  ss_plan_s* p = new ss_plan_s();
  p->C = channels;
  p->T = T;
  p->M = T / 2 + 1;
  p->Mp = (p->M + 15) & ~15;  // whole 128-byte blocks of 16 bins per row
  p->m = m;
  p->dt = dt;
  p->window = window;
  p->win_param = win_param;
  p->orders = orders;
  p->dtype = dtype;
  p->precision = precision;
  p->elem = dtype == SS_F32 ? 4 : 2;
  {
    const int nch = (m + 15) / 16;
    p->FC = (m + nch - 1) / nch;  // chunks of at most 16 frames, as even as possible
  }
  p->stream = static_cast<cudaStream_t>(stream);

  if (combos) {
    for (int i = 0; i < n_combos; ++i) {
      const int* r = combos + 5 * i;
      Combo cb{r[0], {r[1], r[2], r[3], r[4]}};
      const int n = cb.order;
      if (n < 2 || n > 4 || !(orders & (1u << n))) {
        delete p;
        return fail(nullptr, SS_EINVAL, "combination of an order the plan does not compute");
      }
      for (int q = 0; q < n; ++q)
        if (cb.c[q] < 0 || cb.c[q] >= channels) {
          delete p;
          return fail(nullptr, SS_EINVAL, "combination names a channel out of range");
        }
      (n == 2 ? p->c2 : n == 3 ? p->c3 : p->c4).push_back(cb);
    }
  } else {
    default_combos(p);
  }
  if (channels == 1 && !p->c4.empty() && precision != SS_PREC_FP32 && m > kMaxGramM) {
    delete p;
    return fail(nullptr, SS_EUNSUPPORTED,
                "the tensor-core S4 precisions take m <= 32 frames per group; use fp32");
  }
  p->rows3 = channels == 1 ? p->M : 2 * p->M - 1;
  p->rows4 = channels == 1 ? p->M : 2 * p->M - 1;

  ss_status st;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    st = cuda_fail(nullptr, e, "cudaGetDevice");
    delete p;
    return st;
  }
  cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device);

  // window (Eq. 17 / App. B) and its power sums, in float64
  std::vector<double> g(T);
  for (int i = 0; i < T; ++i) {
    if (window == SS_WIN_HANN) {
      g[i] = 0.5 - 0.5 * std::cos(2.0 * M_PI * i / T);
    } else {
      const double N = T, s = win_param, c = (N - 1.0) / 2.0;
      auto G = [&](double x) { return std::exp(-(x - c) * (x - c) / (4.0 * N * N * s * s)); };
      g[i] = G(i) - G(-0.5) * (G(i + N) + G(i - N)) / (G(-0.5 + N) + G(-0.5 - N));
    }
  }
  for (int i = 0; i < T; ++i) {
    p->sg1 += g[i];
    p->sg2 += g[i] * g[i];
    p->sg3 += g[i] * g[i] * g[i];
    p->sg4 += g[i] * g[i] * g[i] * g[i];
  }
  // S1 = mean X_0 / sum g with the kernels' window scaled by 1/sqrt(sum g^2)
  p->norm1 = std::sqrt(p->sg2) / p->sg1;
  p->norm2 = dt;
  p->norm3 = dt * dt * std::pow(p->sg2, 1.5) / p->sg3;
  p->norm4 = dt * dt * dt * p->sg2 * p->sg2 / p->sg4;
  std::vector<float> gw(T);
  for (int i = 0; i < T; ++i) gw[i] = (float)(g[i] / std::sqrt(p->sg2));
  std::vector<float2> tw(T);
  for (int a = 0; a < T; ++a)
    tw[a] = make_float2((float)std::cos(2.0 * M_PI * a / T), (float)std::sin(2.0 * M_PI * a / T));

  std::vector<int> s2auto(channels, -1);
  std::vector<int4> s2cross;
  for (size_t i = 0; i < p->c2.size(); ++i) {
    const Combo& cb = p->c2[i];
    if (cb.c[0] == cb.c[1] && s2auto[cb.c[0]] < 0)
      s2auto[cb.c[0]] = (int)i;
    else
      s2cross.push_back(make_int4(cb.c[0], cb.c[1], (int)i, 0));
  }
  p->n_s2cross = (int)s2cross.size();
  std::vector<TileInfo> t3, t4;
  std::vector<int2> pts3;
  build_tiles(p->M, channels > 1, t3, t4, pts3, &p->pairs3, &p->pairs4);
  std::vector<TileInfo> t4tc;
  if (channels == 1 && !p->c4.empty() && precision != SS_PREC_FP32)
    t4tc = build_tc_tiles(p->M, &p->col4);
  p->n_tiles4tc = (int)t4tc.size();
  if (p->c3.empty()) {
    t3.clear();
    pts3.clear();
  }
  if (p->c4.empty() || channels > 1) t4.clear();  // several channels: k3_trispec_cross
  std::vector<TileInfo> t3w;
  std::vector<int2> pts3w;
  if (channels == 1 && !p->c3.empty()) build_warp_tiles(p->M, t3w, pts3w);
  p->n_tiles3 = (int)t3.size();
  p->n_tiles4 = (int)t4.size();
  p->n_pts3 = (int)pts3.size();
  p->n_tiles3w = (int)t3w.size();
  p->n_pts3w = (int)pts3w.size();

#define PLAN_TRY(call)                           \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) {                     \
      st = cuda_fail(nullptr, e_, #call);        \
      destroy(p);                                \
      return st;                                 \
    }                                            \
  } while (0)

  PLAN_TRY(dev_alloc(p, &p->d_win, T * sizeof(float)));
  PLAN_TRY(dev_alloc(p, &p->d_tw, T * sizeof(float2)));
  PLAN_TRY(dev_alloc(p, &p->d_carry, (size_t)channels * m * T * p->elem));
  PLAN_TRY(dev_alloc(p, &p->d_s2auto, channels * sizeof(int)));
  if (!s2cross.empty()) PLAN_TRY(dev_alloc(p, &p->d_s2cross, s2cross.size() * sizeof(int4)));
  p->n_acc1 = (orders & SS_ORDER1) ? (size_t)kPlanes * channels : 0;
  p->n_acc2 = (size_t)kPlanes * p->c2.size() * p->M;
  p->n_acc3 = (size_t)kPlanes * p->c3.size() * p->rows3 * p->M;
  p->n_acc4 = (size_t)kPlanes * p->c4.size() * p->rows4 * p->M;
  if (p->n_acc1) PLAN_TRY(dev_alloc(p, &p->d_acc1, p->n_acc1 * sizeof(double)));
  if (p->n_acc2) PLAN_TRY(dev_alloc(p, &p->d_acc2, p->n_acc2 * sizeof(double)));
  if (p->n_acc3) PLAN_TRY(dev_alloc(p, &p->d_acc3, p->n_acc3 * sizeof(double)));
  if (p->n_acc4) PLAN_TRY(dev_alloc(p, &p->d_acc4, p->n_acc4 * sizeof(double)));
  if (!t3.empty()) PLAN_TRY(dev_alloc(p, &p->d_tiles3, t3.size() * sizeof(TileInfo)));
  if (!pts3.empty()) PLAN_TRY(dev_alloc(p, &p->d_pts3, pts3.size() * sizeof(int2)));
  if (!t3w.empty()) PLAN_TRY(dev_alloc(p, &p->d_tiles3w, t3w.size() * sizeof(TileInfo)));
  if (!pts3w.empty()) PLAN_TRY(dev_alloc(p, &p->d_pts3w, pts3w.size() * sizeof(int2)));
  if (!t4.empty()) PLAN_TRY(dev_alloc(p, &p->d_tiles4, t4.size() * sizeof(TileInfo)));
  if (!t4tc.empty()) PLAN_TRY(dev_alloc(p, &p->d_tiles4tc, t4tc.size() * sizeof(TileInfo)));
  std::vector<int4> c4x;
  if (channels > 1)
    for (const Combo& cb : p->c4) c4x.push_back(make_int4(cb.c[0], cb.c[1], cb.c[2], cb.c[3]));
  if (!c4x.empty()) {
    PLAN_TRY(dev_alloc(p, &p->d_c4cross, c4x.size() * sizeof(int4)));
    PLAN_TRY(cudaMemcpy(p->d_c4cross, c4x.data(), c4x.size() * sizeof(int4),
                        cudaMemcpyHostToDevice));
  }
  PLAN_TRY(dev_alloc(p, &p->d_status, sizeof(int)));
  PLAN_TRY(dev_alloc(p, &p->d_counter, sizeof(int)));
  PLAN_TRY(cudaMemcpy(p->d_win, gw.data(), T * sizeof(float), cudaMemcpyHostToDevice));
  PLAN_TRY(cudaMemcpy(p->d_tw, tw.data(), T * sizeof(float2), cudaMemcpyHostToDevice));
  PLAN_TRY(cudaMemcpy(p->d_s2auto, s2auto.data(), channels * sizeof(int),
                      cudaMemcpyHostToDevice));
  if (!s2cross.empty())
    PLAN_TRY(cudaMemcpy(p->d_s2cross, s2cross.data(), s2cross.size() * sizeof(int4),
                        cudaMemcpyHostToDevice));
  if (!t3.empty())
    PLAN_TRY(cudaMemcpy(p->d_tiles3, t3.data(), t3.size() * sizeof(TileInfo),
                        cudaMemcpyHostToDevice));
  if (!pts3.empty())
    PLAN_TRY(cudaMemcpy(p->d_pts3, pts3.data(), pts3.size() * sizeof(int2),
                        cudaMemcpyHostToDevice));
  if (!t3w.empty())
    PLAN_TRY(cudaMemcpy(p->d_tiles3w, t3w.data(), t3w.size() * sizeof(TileInfo),
                        cudaMemcpyHostToDevice));
  if (!pts3w.empty())
    PLAN_TRY(cudaMemcpy(p->d_pts3w, pts3w.data(), pts3w.size() * sizeof(int2),
                        cudaMemcpyHostToDevice));
  if (!t4.empty())
    PLAN_TRY(cudaMemcpy(p->d_tiles4, t4.data(), t4.size() * sizeof(TileInfo),
                        cudaMemcpyHostToDevice));
  if (!t4tc.empty())
    PLAN_TRY(cudaMemcpy(p->d_tiles4tc, t4tc.data(), t4tc.size() * sizeof(TileInfo),
                        cudaMemcpyHostToDevice));
  p->Gb_user = batch;
  st = alloc_spec(p);
  if (st != SS_OK) {
    g_plan_error = p->err;
    destroy(p);
    return st;
  }
  st = zero_state(p);
  if (st == SS_OK && p->stream == nullptr) {
    cudaError_t e2 = cudaStreamSynchronize(nullptr);
    if (e2 != cudaSuccess) st = cuda_fail(p, e2, "cudaStreamSynchronize");
  }
  if (st != SS_OK) {
    g_plan_error = p->err;
    destroy(p);
    return st;
  }
#undef PLAN_TRY
  *out = p;
  return SS_OK;
}

ss_status ss_plan(ss_plan_t* out, int channels, int T, double dt, int m, int window,
                  double win_param, unsigned orders, int dtype, int precision,
                  const int* combos, int n_combos, void* stream) {
  return plan_create(out, channels, T, dt, m, window, win_param, orders, dtype, precision,
                     combos, n_combos, stream, 0);
}

ss_status ss_accumulate(ss_plan_t p, const void* chunk, size_t n_samples) {
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  if (p->broken) return fail(p, SS_ESTATE, "plan is unusable after a CUDA failure: " + p->err);
  if (n_samples == 0) return SS_OK;
  if (!chunk) return fail(p, SS_EINVAL, "chunk is NULL");
  if (n_samples > (size_t)1 << 46) return fail(p, SS_EINVAL, "n_samples too large");
  DeviceGuard guard(p->device);
  if (is_device_ptr(chunk)) {
    ss_status st = process_device(p, chunk, (long long)n_samples, (long long)n_samples);
    if (st == SS_OK) st = feed_shadow(p, chunk, (long long)n_samples, (long long)n_samples);
    return st;
  }
  return process_host(p, chunk, (long long)n_samples);
}

// The sums to finalize or export: the plan's own, or with an interlaced window
// set the element-wise sum of both plans' sums and groups.
struct Pooled {
  double *a1, *a2, *a3, *a4;
  long long groups, samples;
};

static ss_status pooled(ss_plan_s* p, Pooled* out) {
  *out = Pooled{p->d_acc1, p->d_acc2, p->d_acc3, p->d_acc4, p->groups, p->samples};
  ss_plan_s* s = p->shadow;
  if (!s) return SS_OK;
  const size_t n = p->n_acc1 + p->n_acc2 + p->n_acc3 + p->n_acc4;
  if (!p->d_pool) SS_TRY(p, dev_alloc(p, &p->d_pool, n * sizeof(double)));
  double* q = p->d_pool;
  double** dst[4] = {&out->a1, &out->a2, &out->a3, &out->a4};
  const double* mine[4] = {p->d_acc1, p->d_acc2, p->d_acc3, p->d_acc4};
  const double* theirs[4] = {s->d_acc1, s->d_acc2, s->d_acc3, s->d_acc4};
  const size_t cnt[4] = {p->n_acc1, p->n_acc2, p->n_acc3, p->n_acc4};
  for (int i = 0; i < 4; ++i) {
    if (!cnt[i]) continue;
    SS_TRY(p, cudaMemcpyAsync(q, mine[i], cnt[i] * sizeof(double), cudaMemcpyDeviceToDevice,
                              p->stream));
    SS_TRY(p, launch_add_f64(q, theirs[i], (long long)cnt[i], p->stream));
    *dst[i] = q;
    q += cnt[i];
  }
  out->groups += s->groups;
  out->samples += s->samples;
  return SS_OK;
}

// The finalize buffer: means and errors of every spectrum (complex doubles).
static ss_status ensure_out(ss_plan_s* p) {
  const size_t n2 = p->c2.size() * p->M * 2;
  const size_t n3 = p->c3.size() * p->rows3 * p->M * 2;
  const size_t n4 = p->c4.size() * p->rows4 * p->M * 2;
  const size_t need = 2 * (n2 + n3 + n4);
  if (p->out_doubles < need) {
    if (p->d_out) {
      cudaFree(p->d_out);
      p->device_bytes -= p->out_doubles * sizeof(double);
      p->d_out = nullptr;
      p->out_doubles = 0;
    }
    SS_TRY(p, dev_alloc(p, &p->d_out, need * sizeof(double)));
    p->out_doubles = need;
  }
  return SS_OK;
}

// K4 and the copies to the caller's buffers, stream-ordered (no synchronisation).
static ss_status finalize_launch(ss_plan_s* p, double* S2, double* S3, double* S4,
                                 double* S2_err, double* S3_err, double* S4_err) {
  ss_status st0 = ensure_out(p);
  if (st0 != SS_OK) return st0;
  Pooled pl;
  st0 = pooled(p, &pl);
  if (st0 != SS_OK) return st0;
  const size_t n2 = p->c2.size() * p->M * 2;
  const size_t n3 = p->c3.size() * p->rows3 * p->M * 2;
  const size_t n4 = p->c4.size() * p->rows4 * p->M * 2;
  double* o2 = p->d_out;
  double* e2 = o2 + n2;
  double* o3 = e2 + n2;
  double* e3 = o3 + n3;
  double* o4 = e3 + n3;
  double* e4 = o4 + n4;
  const bool single = p->C == 1;
  record(p, 3, p->stream, true);
  if (n2)
    SS_TRY(p, launch_k4_finalize(pl.a2, (int)p->c2.size(), 1, p->M, kLayoutVector,
                                 pl.groups, p->norm2, o2, e2, p->stream));
  if (n3)
    SS_TRY(p, launch_k4_finalize(pl.a3, (int)p->c3.size(), p->rows3, p->M,
                                 single ? kLayoutS3Single : kLayoutCross, pl.groups, p->norm3,
                                 o3, e3, p->stream));
  if (n4)
    SS_TRY(p, launch_k4_finalize(pl.a4, (int)p->c4.size(), p->rows4, p->M,
                                 !single ? kLayoutCross
                                 : p->precision == SS_PREC_FP32 ? kLayoutS4Single : kLayoutS4Lower,
                                 pl.groups, p->norm4,
                                 o4, e4, p->stream));
  record(p, 3, p->stream, false);
  const std::pair<double*, std::pair<const double*, size_t>> copies[6] = {
      {S2, {o2, n2}}, {S2_err, {e2, n2}}, {S3, {o3, n3}},
      {S3_err, {e3, n3}}, {S4, {o4, n4}}, {S4_err, {e4, n4}}};
  for (const auto& c : copies)
    if (c.first && c.second.second)
      SS_TRY(p, cudaMemcpyAsync(c.first, c.second.first, c.second.second * sizeof(double),
                                cudaMemcpyDefault, p->stream));
  return SS_OK;
}

ss_status ss_finalize(ss_plan_t p, double* S2, double* S3, double* S4, double* S2_err,
                      double* S3_err, double* S4_err) {
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  if (p->broken) return fail(p, SS_ESTATE, "plan is unusable after a CUDA failure: " + p->err);
  if (p->groups + (p->shadow ? p->shadow->groups : 0) < 2)
    return fail(p, SS_ESTATE, "fewer than two groups accumulated: no error estimate (Eq. 35)");
  DeviceGuard guard(p->device);
  ss_status st = finalize_launch(p, S2, S3, S4, S2_err, S3_err, S4_err);
  if (st != SS_OK) return st;
  SS_TRY(p, cudaStreamSynchronize(p->stream));
  return check_status(p);
}

ss_status ss_finalize_s1(ss_plan_t p, double* S1, double* S1_err) {
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  if (p->broken) return fail(p, SS_ESTATE, "plan is unusable after a CUDA failure: " + p->err);
  if (!p->d_acc1) return fail(p, SS_ESTATE, "the plan was made without SS_ORDER1");
  if (p->groups + (p->shadow ? p->shadow->groups : 0) < 2)
    return fail(p, SS_ESTATE, "fewer than two groups accumulated: no error estimate (Eq. 35)");
  DeviceGuard guard(p->device);
  ss_status st = ensure_out(p);
  if (st != SS_OK) return st;
  Pooled pl;
  st = pooled(p, &pl);
  if (st != SS_OK) return st;
  const size_t n1 = (size_t)p->C * 2;
  double* o1 = p->d_out;
  double* e1 = o1 + n1;
  SS_TRY(p, launch_k4_finalize(pl.a1, p->C, 1, 1, kLayoutVector, pl.groups, p->norm1, o1,
                               e1, p->stream));
  if (S1) SS_TRY(p, cudaMemcpyAsync(S1, o1, n1 * sizeof(double), cudaMemcpyDefault, p->stream));
  if (S1_err)
    SS_TRY(p, cudaMemcpyAsync(S1_err, e1, n1 * sizeof(double), cudaMemcpyDefault, p->stream));
  SS_TRY(p, cudaStreamSynchronize(p->stream));
  return check_status(p);
}

ss_status ss_set_estimator(ss_plan_t p, int estimator) {
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  if (estimator != SS_EST_UNBIASED && estimator != SS_EST_NATURAL)
    return fail(p, SS_EINVAL, "unknown estimator");
  if (p->groups != 0 || p->carry_n != 0)
    return fail(p, SS_ESTATE, "ss_set_estimator is valid only before the first ss_accumulate");
  for (ss_plan_s* q = p; q; q = q->shadow) {
    q->estimator = estimator;
    if (q->oi.img) set_image_scales(q);
  }
  return SS_OK;
}

ss_status ss_set_sequential(ss_plan_t p, int block_groups, double* out, long long max_blocks) {
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  if (block_groups < 0 || block_groups == 1)
    return fail(p, SS_EINVAL, "block_groups must be 0 (off) or at least 2 (Eq. 35 needs two parts)");
  if (p->groups != 0 || p->carry_n != 0)
    return fail(p, SS_ESTATE, "ss_set_sequential is valid only before the first ss_accumulate");
  if (block_groups > 0 && p->shadow)
    return fail(p, SS_EUNSUPPORTED, "sequential spectra of interlaced window sets");
  if (block_groups > 0 && max_blocks > 0 && (!out || !is_device_ptr(out)))
    return fail(p, SS_EINVAL, "out must be device memory");
  if (max_blocks < 0) return fail(p, SS_EINVAL, "max_blocks must be >= 0");
  DeviceGuard guard(p->device);
  p->seq_B = block_groups;
  p->seq_out = block_groups > 0 ? out : nullptr;
  p->seq_cap = block_groups > 0 ? max_blocks : 0;
  p->seq_blocks = 0;
  const size_t n = p->n_acc2 + p->n_acc3 + p->n_acc4;
  if (block_groups > 0 && !p->d_prev && n) SS_TRY(p, dev_alloc(p, &p->d_prev, n * sizeof(double)));
  if (p->d_prev) SS_TRY(p, cudaMemsetAsync(p->d_prev, 0, n * sizeof(double), p->stream));
  return SS_OK;
}

ss_status ss_sequential_info(ss_plan_t p, size_t* block_doubles, long long* blocks_done) {
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  const size_t n2 = p->c2.size() * p->M * 2;
  const size_t n3 = p->c3.size() * p->rows3 * p->M * 2;
  const size_t n4 = p->c4.size() * p->rows4 * p->M * 2;
  if (block_doubles) *block_doubles = 2 * (n2 + n3 + n4);
  if (blocks_done) *blocks_done = p->seq_blocks;
  return SS_OK;
}

ss_status ss_set_complex(ss_plan_t p, const int* recs, int n, int s4_shift) {
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  if (n < 0 || (n > 0 && !recs)) return fail(p, SS_EINVAL, "records missing");
  if (p->groups != 0 || p->carry_n != 0)
    return fail(p, SS_ESTATE, "ss_set_complex is valid only before the first ss_accumulate");
  if (n > 0 && p->shadow)
    return fail(p, SS_EUNSUPPORTED, "complex-signal spectra of interlaced window sets");
  std::vector<int4> ops[3];
  std::vector<int> order;
  for (int i = 0; i < n; ++i) {
    const int* r = recs + 13 * i;
    const int o = r[0];
    if (o < 2 || o > 4) return fail(p, SS_EINVAL, "record order must be 2, 3 or 4");
    if (o == 3 && p->m < 3) return fail(p, SS_EINVAL, "S3 needs m >= 3 (Eq. 33)");
    if (o == 4 && p->m < 4) return fail(p, SS_EINVAL, "S4 needs m >= 4 (Eq. 34)");
    for (int q = 0; q < o; ++q) {
      const int re = r[1 + 3 * q], im = r[2 + 3 * q], cj = r[3 + 3 * q];
      if (re < 0 || re >= p->C || im < -1 || im >= p->C || (cj != 0 && cj != 1))
        return fail(p, SS_EINVAL, "operand names a channel out of range or a bad conjugate flag");
      ops[o - 2].push_back(make_int4(re, im, cj ? -1 : 1, 0));
    }
    order.push_back(o);
  }
  DeviceGuard guard(p->device);
  const long long nn = 2ll * p->M - 1;
  for (int o = 0; o < 3; ++o) {
    cudaFree(p->d_cx_ops[o]);
    cudaFree(p->d_cx_acc[o]);
    p->d_cx_ops[o] = nullptr;
    p->d_cx_acc[o] = nullptr;
    p->n_cx_acc[o] = 0;
    p->cx_ops[o] = ops[o];
    if (ops[o].empty()) continue;
    const size_t combos = ops[o].size() / (o + 2);
    p->n_cx_acc[o] = (size_t)kPlanes * combos * (o == 0 ? nn : nn * nn);
    SS_TRY(p, dev_alloc(p, &p->d_cx_ops[o], ops[o].size() * sizeof(int4)));
    SS_TRY(p, cudaMemcpy(p->d_cx_ops[o], ops[o].data(), ops[o].size() * sizeof(int4),
                         cudaMemcpyHostToDevice));
    SS_TRY(p, dev_alloc(p, &p->d_cx_acc[o], p->n_cx_acc[o] * sizeof(double)));
    SS_TRY(p, cudaMemsetAsync(p->d_cx_acc[o], 0, p->n_cx_acc[o] * sizeof(double), p->stream));
  }
  p->cx_order = order;
  p->cx_shift = s4_shift;
  return SS_OK;
}

ss_status ss_complex_size(ss_plan_t p, size_t* n_doubles) {
  if (!p || !n_doubles) return fail(p, SS_EINVAL, "NULL argument");
  const size_t nn = 2 * (size_t)p->M - 1;
  size_t n = 0;
  for (int o : p->cx_order) n += 2 * (o == 2 ? nn : nn * nn);
  *n_doubles = n;
  return SS_OK;
}

ss_status ss_finalize_complex(ss_plan_t p, double* S, double* S_err) {
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  if (p->broken) return fail(p, SS_ESTATE, "plan is unusable after a CUDA failure: " + p->err);
  if (p->cx_order.empty()) return fail(p, SS_ESTATE, "no complex-signal combinations set");
  if (p->groups < 2)
    return fail(p, SS_ESTATE, "fewer than two groups accumulated: no error estimate (Eq. 35)");
  DeviceGuard guard(p->device);
  size_t total = 0;
  ss_status st = ss_complex_size(p, &total);
  if (st != SS_OK) return st;
  // the finalize buffer holds means and errors (grown to fit)
  if (p->out_doubles < 2 * total) {
    if (p->d_out) {
      cudaFree(p->d_out);
      p->device_bytes -= p->out_doubles * sizeof(double);
      p->d_out = nullptr;
      p->out_doubles = 0;
    }
    SS_TRY(p, dev_alloc(p, &p->d_out, 2 * total * sizeof(double)));
    p->out_doubles = 2 * total;
  }
  const int nn = 2 * p->M - 1;
  const double norms[3] = {p->norm2, p->norm3, p->norm4};
  // each order's combinations in one K4 launch over its block of the buffer
  double* mean[3];
  double* err[3];
  size_t off = 0;
  for (int o = 0; o < 3; ++o) {
    const size_t combos = p->cx_ops[o].size() / (o + 2);
    const size_t per = 2 * (o == 0 ? (size_t)nn : (size_t)nn * nn);
    mean[o] = p->d_out + off;
    err[o] = p->d_out + total + off;
    if (combos)
      SS_TRY(p, launch_k4_finalize(p->d_cx_acc[o], (int)combos, o == 0 ? 1 : nn, nn,
                                   kLayoutCross, p->groups, norms[o], mean[o], err[o], p->stream));
    off += combos * per;
  }
  // to the caller in record order
  size_t seen[3] = {0, 0, 0};
  size_t out_off = 0;
  for (int o : p->cx_order) {
    const size_t per = 2 * (o == 2 ? (size_t)nn : (size_t)nn * nn);
    const int i = o - 2;
    if (S)
      SS_TRY(p, cudaMemcpyAsync(S + out_off, mean[i] + seen[i] * per, per * sizeof(double),
                                cudaMemcpyDefault, p->stream));
    if (S_err)
      SS_TRY(p, cudaMemcpyAsync(S_err + out_off, err[i] + seen[i] * per, per * sizeof(double),
                                cudaMemcpyDefault, p->stream));
    ++seen[i];
    out_off += per;
  }
  SS_TRY(p, cudaStreamSynchronize(p->stream));
  return check_status(p);
}

ss_status ss_inject_timeout(ss_plan_t p, int on) {
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  for (ss_plan_s* q = p; q; q = q->shadow) q->inject_timeout = on ? 1 : 0;
  return SS_OK;
}

ss_status ss_set_interlace(ss_plan_t p, int on) {
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  if (p->groups != 0 || p->carry_n != 0)
    return fail(p, SS_ESTATE, "ss_set_interlace is valid only before the first ss_accumulate");
  DeviceGuard guard(p->device);
  if (!on) {
    if (p->shadow) {
      destroy(p->shadow);
      p->shadow = nullptr;
    }
    return SS_OK;
  }
  if (p->shadow) return SS_OK;
  if (p->seq_B > 0)
    return fail(p, SS_EUNSUPPORTED, "interlaced window sets with sequential spectra");
  if (!p->cx_order.empty())
    return fail(p, SS_EUNSUPPORTED, "interlaced window sets with complex-signal spectra");
  // the same configuration and combinations, fed from T/2 samples on
  std::vector<int> recs;
  for (const auto* list : {&p->c2, &p->c3, &p->c4})
    for (const Combo& cb : *list) {
      recs.push_back(cb.order);
      for (int q = 0; q < 4; ++q) recs.push_back(q < cb.order ? cb.c[q] : -1);
    }
  ss_plan_t s = nullptr;
  ss_status st = plan_create(&s, p->C, p->T, p->dt, p->m, p->window, p->win_param, p->orders,
                             p->dtype, p->precision, recs.empty() ? nullptr : recs.data(),
                             (int)(recs.size() / 5), p->stream, p->Gb_user);
  if (st != SS_OK) return fail(p, st, "interlaced window set: " + g_plan_error);
  s->estimator = p->estimator;
  s->inject_timeout = p->inject_timeout;
  if (s->oi.img) set_image_scales(s);
  s->skip = p->T / 2;
  p->shadow = s;
  return SS_OK;
}

ss_status ss_reset(ss_plan_t p) {
  if (p && p->shadow && !p->broken) {
    ss_status st = ss_reset(p->shadow);
    if (st != SS_OK) return fail(p, st, "interlaced window set: " + p->shadow->err);
    p->shadow->skip = p->T / 2;
  }
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  if (p->broken) return fail(p, SS_ESTATE, "plan is unusable after a CUDA failure: " + p->err);
  DeviceGuard guard(p->device);
  SS_TRY(p, cudaStreamSynchronize(p->stream));
  return zero_state(p);
}

ss_status ss_query(ss_plan_t p, ss_info* info) {
  if (!p || !info) return fail(p, SS_EINVAL, "NULL argument");
  info->channels = p->C;
  info->T = p->T;
  info->M = p->M;
  info->m = p->m;
  info->n_s2 = (int)p->c2.size();
  info->n_s3 = (int)p->c3.size();
  info->n_s4 = (int)p->c4.size();
  info->rows3 = p->rows3;
  info->rows4 = p->rows4;
  info->groups = p->groups + (p->shadow ? p->shadow->groups : 0);
  info->samples = p->samples;
  info->carried = p->carry_n;
  info->groups_per_batch = p->Gb_max;
  info->device_bytes = p->device_bytes;
  info->kernels_per_batch = 1 + (p->n_s2cross > 0 ? 1 : 0) +
                            (int)p->c3.size() * (1 + (p->C == 1 && p->n_pts3 > 0 ? 1 : 0)) +
                            (p->C > 1 ? (p->c4.empty() ? 0 : p->precision == SS_PREC_FP32 ? 1 : 2)
                                      : (int)p->c4.size() *
                                            (1 + (p->precision != SS_PREC_FP32 && p->col4 ? 1 : 0)));
  return SS_OK;
}

ss_status ss_layout(int channels, int T, int* s3_tiles, int max3, int* n3, int* s3_points,
                    int maxp, int* np, int* s4_tiles, int max4, int* n4, int* last_col) {
  if (channels < 1 || channels > 4 || T < 8 || T > 4096 || !is_pow2(T))
    return fail(nullptr, SS_EINVAL, "channels in [1, 4] and T a power of two in [8, 4096]");
  if (!n3 || !np || !n4 || !last_col) return fail(nullptr, SS_EINVAL, "NULL count argument");
  const int M = T / 2 + 1;
  std::vector<TileInfo> t3, t4;
  std::vector<int2> pts3;
  long long pairs3 = 0, pairs4 = 0;
  build_tiles(M, channels > 1, t3, t4, pts3, &pairs3, &pairs4);
  *n3 = (int)t3.size();
  *np = (int)pts3.size();
  for (int i = 0; i < *n3 && i < max3 && s3_tiles; ++i) {
    s3_tiles[2 * i] = t3[i].k0;
    s3_tiles[2 * i + 1] = t3[i].l0;
  }
  for (int i = 0; i < *np && i < maxp && s3_points; ++i) {
    s3_points[2 * i] = pts3[i].x;
    s3_points[2 * i + 1] = pts3[i].y;
  }
  bool col = false;
  std::vector<TileInfo> tc;
  if (channels == 1) tc = build_tc_tiles(M, &col);
  *n4 = (int)tc.size();
  *last_col = col ? 1 : 0;
  for (int i = 0; i < *n4 && i < max4 && s4_tiles; ++i) {
    s4_tiles[3 * i] = tc[i].k0;
    s4_tiles[3 * i + 1] = tc[i].l0;
    s4_tiles[3 * i + 2] = tc[i].ncols;
  }
  return SS_OK;
}

ss_status ss_layout_warps(int T, int* tiles, int max_tiles, int* n, int* points, int maxp,
                          int* np) {
  if (T < 8 || T > 4096 || !is_pow2(T))
    return fail(nullptr, SS_EINVAL, "T a power of two in [8, 4096]");
  if (!n || !np) return fail(nullptr, SS_EINVAL, "NULL count argument");
  std::vector<TileInfo> t;
  std::vector<int2> pts;
  build_warp_tiles(T / 2 + 1, t, pts);
  *n = (int)t.size();
  *np = (int)pts.size();
  for (int i = 0; i < *n && i < max_tiles && tiles; ++i) {
    tiles[2 * i] = t[i].k0;
    tiles[2 * i + 1] = t[i].l0;
  }
  for (int i = 0; i < *np && i < maxp && points; ++i) {
    points[2 * i] = pts[i].x;
    points[2 * i + 1] = pts[i].y;
  }
  return SS_OK;
}

ss_status ss_combos(ss_plan_t p, int* out, int max_records) {
  if (!p || (!out && max_records > 0)) return fail(p, SS_EINVAL, "NULL argument");
  int r = 0;
  for (const auto* v : {&p->c2, &p->c3, &p->c4})
    for (const Combo& cb : *v) {
      if (r >= max_records) return fail(p, SS_EINVAL, "max_records too small");
      out[5 * r] = cb.order;
      for (int q = 0; q < 4; ++q) out[5 * r + 1 + q] = q < cb.order ? cb.c[q] : -1;
      ++r;
    }
  return SS_OK;
}

ss_status ss_set_timing(ss_plan_t p, int enable) {
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  p->timing = enable != 0;
  return SS_OK;
}

ss_status ss_stats(ss_plan_t p, ss_stats_t* s) {
  if (!p || !s) return fail(p, SS_EINVAL, "NULL argument");
  DeviceGuard guard(p->device);
  SS_TRY(p, cudaStreamSynchronize(p->stream));
  if (p->copy_stream) SS_TRY(p, cudaStreamSynchronize(p->copy_stream));
  for (int i = 0; i < 5; ++i) {
    double ms = 0.0;
    for (const EventPair& e : p->ev[i]) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) ms += t;
    }
    s->ms[i] = ms;
    s->launches[i] = p->launches[i];
  }
  s->pairs3 = p->pairs3;
  s->pairs4 = p->pairs4;
  return SS_OK;
}

ss_status ss_set_batch(ss_plan_t p, int groups_per_batch) {
  if (!p) return fail(nullptr, SS_EINVAL, "plan is NULL");
  if (groups_per_batch < 0) return fail(p, SS_EINVAL, "groups_per_batch must be >= 0");
  if (p->groups != 0 || p->carry_n != 0)
    return fail(p, SS_ESTATE, "ss_set_batch is valid only before the first ss_accumulate");
  DeviceGuard guard(p->device);
  SS_TRY(p, cudaStreamSynchronize(p->stream));
  p->Gb_user = groups_per_batch;
  if (p->shadow) {
    p->shadow->Gb_user = groups_per_batch;
    ss_status st = alloc_spec(p->shadow);
    if (st != SS_OK) return fail(p, st, "interlaced window set: " + p->shadow->err);
  }
  return alloc_spec(p);
}

namespace {

constexpr double kStateLayoutVersion = 2.0;  // 2: S1 sums before the S2 sums
constexpr int kStateCfgWords = 14;  // header words that must match; 14 = groups, 15 = samples

// FNV-1a over the combination records, cut to 52 bits (exact in a double)
double combos_hash(const ss_plan_s* p) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](int v) {
    for (int b = 0; b < 4; ++b) {
      h ^= (uint64_t)((v >> (8 * b)) & 0xff);
      h *= 1099511628211ull;
    }
  };
  for (const auto* list : {&p->c2, &p->c3, &p->c4})
    for (const Combo& c : *list) {
      mix(c.order);
      for (int q = 0; q < 4; ++q) mix(q < c.order ? c.c[q] : -1);
    }
  return (double)(h & ((1ull << 52) - 1));
}

void state_header(const ss_plan_s* p, double* h) {
  for (int i = 0; i < SS_STATE_HEADER; ++i) h[i] = 0.0;
  h[0] = p->C;
  h[1] = p->T;
  h[2] = p->m;
  h[3] = p->orders | (p->shadow ? 1u : 0u);  // bit 0: interlaced
  h[4] = p->precision;
  h[5] = p->window;
  h[6] = p->window == SS_WIN_ACG ? p->win_param : 0.0;
  h[7] = p->dt;
  h[8] = (double)p->c2.size();
  h[9] = (double)p->c3.size();
  h[10] = (double)p->c4.size();
  h[11] = combos_hash(p);
  h[12] = kStateLayoutVersion;
  h[13] = p->estimator;
  h[14] = (double)p->groups;
  h[15] = (double)p->samples;
}

}  // namespace

ss_status ss_state_size(ss_plan_t p, size_t* n) {
  if (!p || !n) return fail(p, SS_EINVAL, "NULL argument");
  *n = SS_STATE_HEADER + p->n_acc1 + p->n_acc2 + p->n_acc3 + p->n_acc4;
  return SS_OK;
}

ss_status ss_export_state(ss_plan_t p, double* dst) {
  if (!p || !dst) return fail(p, SS_EINVAL, "NULL argument");
  if (p->broken) return fail(p, SS_ESTATE, "plan is unusable after a CUDA failure: " + p->err);
  DeviceGuard guard(p->device);
  ss_status st = check_status(p);
  if (st != SS_OK) return st;
  Pooled pl;  // with an interlaced window set, the sums of both
  st = pooled(p, &pl);
  if (st != SS_OK) return st;
  double h[SS_STATE_HEADER];
  state_header(p, h);
  h[14] = (double)pl.groups;
  h[15] = (double)pl.samples;
  SS_TRY(p, cudaMemcpyAsync(dst, h, sizeof(h), cudaMemcpyDefault, p->stream));
  double* o = dst + SS_STATE_HEADER;
  const std::pair<const double*, size_t> parts[4] = {
      {pl.a1, p->n_acc1}, {pl.a2, p->n_acc2}, {pl.a3, p->n_acc3}, {pl.a4, p->n_acc4}};
  for (const auto& pr : parts) {
    if (pr.second)
      SS_TRY(p, cudaMemcpyAsync(o, pr.first, pr.second * sizeof(double), cudaMemcpyDefault,
                                p->stream));
    o += pr.second;
  }
  SS_TRY(p, cudaStreamSynchronize(p->stream));
  return SS_OK;
}

ss_status ss_merge_state(ss_plan_t p, const double* src) {
  if (!p || !src) return fail(p, SS_EINVAL, "NULL argument");
  if (p->broken) return fail(p, SS_ESTATE, "plan is unusable after a CUDA failure: " + p->err);
  DeviceGuard guard(p->device);
  double mine[SS_STATE_HEADER], theirs[SS_STATE_HEADER];
  state_header(p, mine);
  SS_TRY(p, cudaMemcpyAsync(theirs, src, sizeof(theirs), cudaMemcpyDefault, p->stream));
  SS_TRY(p, cudaStreamSynchronize(p->stream));
  for (int i = 0; i < kStateCfgWords; ++i)
    if (mine[i] != theirs[i])
      return fail(p, SS_EINVAL, "state of a plan with another configuration (header word " +
                                    std::to_string(i) + ")");
  if (!(theirs[14] >= 0.0) || !(theirs[15] >= 0.0))
    return fail(p, SS_EINVAL, "state with a negative group or sample count");
  const size_t n = p->n_acc1 + p->n_acc2 + p->n_acc3 + p->n_acc4;
  const double* payload = src + SS_STATE_HEADER;
  if (n) {
    const double* dsrc = payload;
    if (!is_device_ptr(src)) {
      if (p->out_doubles < n) {  // the finalize buffer doubles as the staging buffer
        if (p->d_out) {
          cudaFree(p->d_out);
          p->device_bytes -= p->out_doubles * sizeof(double);
          p->d_out = nullptr;
          p->out_doubles = 0;
        }
        SS_TRY(p, dev_alloc(p, &p->d_out, n * sizeof(double)));
        p->out_doubles = n;
      }
      SS_TRY(p, cudaMemcpyAsync(p->d_out, payload, n * sizeof(double), cudaMemcpyHostToDevice,
                                p->stream));
      dsrc = p->d_out;
    }
    const std::pair<double*, size_t> parts[4] = {
        {p->d_acc1, p->n_acc1}, {p->d_acc2, p->n_acc2}, {p->d_acc3, p->n_acc3},
        {p->d_acc4, p->n_acc4}};
    for (const auto& pr : parts) {
      if (pr.second) SS_TRY(p, launch_add_f64(pr.first, dsrc, (long long)pr.second, p->stream));
      dsrc += pr.second;
    }
    SS_TRY(p, cudaStreamSynchronize(p->stream));  // a host src may be reused on return
  }
  p->groups += (long long)theirs[14];
  p->samples += (long long)theirs[15];
  return SS_OK;
}

ss_status ss_destroy(ss_plan_t p) {
  if (!p) return SS_OK;
  DeviceGuard guard(p->device);
  destroy(p);
  return SS_OK;
}

// ------------------------------------------------------------------------
// Many independent recordings (single channel each, frame lengths and record
// lengths of their own) processed as one CUDA graph: per recording ss_reset,
// ss_accumulate of the whole record from device memory and ss_finalize into
// device buffers, the recordings one after the other on one stream of the
// graph (longest first), each recording's kernels in the forms the autotuner
// chose for its frame length.  The graph is captured on the first ss_run_many
// and replayed while the inputs and outputs stay the same.
}  // extern "C"

namespace {
// Streams the recordings are captured on.  One: every kernel sizes its
// persistent grid for a whole GPU, which holds only when the recordings run one
// after the other.  (Four concurrent branches ended in an unexplained launch
// failure on the 64-recording workload; that form is not used.)
constexpr int kBranches = 1;
constexpr size_t kManyScratch = 6ull << 30;  // per-batch scratch of all recordings together
thread_local std::string g_many_error;
}  // namespace

struct ss_many_s {
  std::vector<ss_plan_s*> plans;
  std::vector<long long> max_n;
  std::vector<int> order;  // recordings by decreasing length (branch assignment)
  cudaStream_t stream = nullptr;   // the caller's: the graph is launched on it
  cudaStream_t cap = nullptr;      // own stream the graph is captured on
  cudaStream_t branch[kBranches] = {};
  cudaEvent_t fork = nullptr, join[kBranches] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> cap_in;
  std::vector<size_t> cap_n;
  std::vector<double*> cap_out;  // 6 per recording
  int device = 0;
  std::string err;
};

namespace {

ss_status many_fail(ss_many_s* mp, ss_status st, const std::string& msg) {
  if (mp)
    mp->err = msg;
  else
    g_many_error = msg;
  return st;
}

void many_release(ss_many_s* mp) {
  if (!mp) return;
  if (mp->exec) cudaGraphExecDestroy(mp->exec);
  if (mp->graph) cudaGraphDestroy(mp->graph);
  mp->exec = nullptr;
  mp->graph = nullptr;
  for (ss_plan_s* p : mp->plans) destroy(p);
  mp->plans.clear();
  for (int b = 0; b < kBranches; ++b) {
    if (mp->branch[b]) cudaStreamDestroy(mp->branch[b]);
    if (mp->join[b]) cudaEventDestroy(mp->join[b]);
  }
  if (mp->fork) cudaEventDestroy(mp->fork);
  if (mp->cap) cudaStreamDestroy(mp->cap);
}

bool device_or_pinned(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged ||
         a.type == cudaMemoryTypeHost;
}

}  // namespace

extern "C" {

ss_status ss_plan_many(ss_many_t* out, int n_rec, const int* T, const size_t* max_samples,
                       double dt, int m, int window, double win_param, unsigned orders,
                       int precision, void* stream) {
  if (!out) return many_fail(nullptr, SS_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_rec < 1 || !T || !max_samples)
    return many_fail(nullptr, SS_EINVAL, "need n_rec >= 1 and the T and max_samples arrays");
  std::vector<long long> groups(n_rec);
  double total = 0.0;
  for (int i = 0; i < n_rec; ++i) {
    if (T[i] < 8 || T[i] > 4096 || (T[i] & (T[i] - 1)))
      return many_fail(nullptr, SS_EINVAL,
                       "recording " + std::to_string(i) + ": T must be a power of two in [8, 4096]");
    if (m < 2) return many_fail(nullptr, SS_EINVAL, "m >= 2 required");
    groups[i] = (long long)(max_samples[i] / ((size_t)m * T[i]));
    if (groups[i] < 2)
      return many_fail(nullptr, SS_EINVAL,
                       "recording " + std::to_string(i) + " holds fewer than two groups");
    const int Mp = ((T[i] / 2 + 1) + 15) & ~15;
    total += (double)groups[i] * m * Mp * 8.0 * (precision == SS_PREC_FP32 ? 1.0 : 5.0);
  }
  ss_many_s* mp = new ss_many_s();
  mp->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&mp->device);
  for (int i = 0; i < n_rec; ++i) {
    // the scratch budget is shared in proportion to each recording's groups
    long long gb = groups[i];
    if (total > (double)kManyScratch)
      gb = std::max(1ll, (long long)((double)groups[i] * (double)kManyScratch / total));
    ss_plan_t p = nullptr;
    ss_status st = plan_create(&p, 1, T[i], dt, m, window, win_param, orders, SS_F32, precision,
                               nullptr, 0, stream, (int)std::min<long long>(gb, 1 << 30));
    if (st == SS_OK) st = ensure_out(p);
    if (st != SS_OK) {
      const std::string why = p ? p->err : g_plan_error;
      if (p) destroy(p);
      many_release(mp);
      delete mp;
      return many_fail(nullptr, st, "recording " + std::to_string(i) + ": " + why);
    }
    mp->plans.push_back(p);
    mp->max_n.push_back((long long)max_samples[i]);
  }
  mp->order.resize(n_rec);
  for (int i = 0; i < n_rec; ++i) mp->order[i] = i;
  std::stable_sort(mp->order.begin(), mp->order.end(),
                   [&](int a, int b) { return max_samples[a] > max_samples[b]; });
  // the kernel forms per frame length: the autotuner on the first plan of each T,
  // its choice applied to the other plans of that T
  for (int i = 0; i < n_rec; ++i) {
    int first = -1;
    for (int j = 0; j < i && first < 0; ++j)
      if (T[j] == T[i]) first = j;
    ss_status st = SS_OK;
    if (first < 0) {
      st = ss_autotune(mp->plans[i], nullptr);
    } else {
      mp->plans[i]->k1_mode = mp->plans[first]->k1_mode;
      mp->plans[i]->k2_variant = mp->plans[first]->k2_variant;
    }
    if (st != SS_OK) {
      const std::string why = mp->plans[i]->err;
      many_release(mp);
      delete mp;
      return many_fail(nullptr, st, "recording " + std::to_string(i) + " autotune: " + why);
    }
  }
  cudaError_t e = cudaEventCreateWithFlags(&mp->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&mp->cap, cudaStreamNonBlocking);
  for (int b = 0; b < kBranches && e == cudaSuccess; ++b) {
    e = cudaStreamCreateWithFlags(&mp->branch[b], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&mp->join[b], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    many_release(mp);
    delete mp;
    return many_fail(nullptr, SS_ECUDA, std::string("stream set-up: ") + cudaGetErrorString(e));
  }
  *out = mp;
  return SS_OK;
}

ss_status ss_run_many(ss_many_t mp, const void* const* chunks, const size_t* n_samples,
                      double* const* S2, double* const* S3, double* const* S4,
                      double* const* S2_err, double* const* S3_err, double* const* S4_err) {
  if (!mp) return many_fail(nullptr, SS_EINVAL, "handle is NULL");
  if (!chunks || !n_samples) return many_fail(mp, SS_EINVAL, "chunks and n_samples are required");
  DeviceGuard guard(mp->device);
  const int n = (int)mp->plans.size();
  std::vector<double*> outs(6 * (size_t)n, nullptr);
  double* const* lists[6] = {S2, S2_err, S3, S3_err, S4, S4_err};
  for (int i = 0; i < n; ++i) {
    ss_plan_s* p = mp->plans[i];
    if (p->broken) return many_fail(mp, SS_ESTATE, "recording " + std::to_string(i) + ": " + p->err);
    if (!chunks[i] || !is_device_ptr(chunks[i]))
      return many_fail(mp, SS_EINVAL, "recording " + std::to_string(i) + ": chunk must be device memory");
    if ((long long)n_samples[i] > mp->max_n[i])
      return many_fail(mp, SS_EINVAL, "recording " + std::to_string(i) + ": more samples than planned");
    if ((long long)(n_samples[i] / ((size_t)p->m * p->T)) < 2)
      return many_fail(mp, SS_EINVAL, "recording " + std::to_string(i) + ": fewer than two groups");
    for (int k = 0; k < 6; ++k) {
      double* o = lists[k] ? lists[k][i] : nullptr;
      if (o && !device_or_pinned(o))
        return many_fail(mp, SS_EINVAL, "recording " + std::to_string(i) +
                                            ": outputs must be device or page-locked host memory");
      outs[6 * (size_t)i + k] = o;
    }
  }
  const bool same = mp->exec && mp->cap_n.size() == (size_t)n &&
                    std::equal(mp->cap_n.begin(), mp->cap_n.end(), n_samples) &&
                    std::equal(mp->cap_in.begin(), mp->cap_in.end(), chunks) &&
                    mp->cap_out == outs;
  if (!same) {
    if (mp->exec) cudaGraphExecDestroy(mp->exec);
    if (mp->graph) cudaGraphDestroy(mp->graph);
    mp->exec = nullptr;
    mp->graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(mp->cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess)
      return many_fail(mp, SS_ECUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    ss_status st = SS_OK;
    e = cudaEventRecord(mp->fork, mp->cap);
    for (int b = 0; b < kBranches && e == cudaSuccess; ++b)
      e = cudaStreamWaitEvent(mp->branch[b], mp->fork, 0);
    if (e != cudaSuccess) st = many_fail(mp, SS_ECUDA, cudaGetErrorString(e));
    for (int r = 0; r < n && st == SS_OK; ++r) {
      const int i = mp->order[r];
      ss_plan_s* p = mp->plans[i];
      const cudaStream_t own = p->stream;
      p->stream = mp->branch[r % kBranches];
      st = zero_state(p);
      if (st == SS_OK) st = process_device(p, chunks[i], (long long)n_samples[i], (long long)n_samples[i]);
      if (st == SS_OK)
        st = finalize_launch(p, outs[6 * i + 0], outs[6 * i + 2], outs[6 * i + 4],
                             outs[6 * i + 1], outs[6 * i + 3], outs[6 * i + 5]);
      p->stream = own;
      if (st != SS_OK) st = many_fail(mp, st, "recording " + std::to_string(i) + ": " + p->err);
    }
    for (int b = 0; b < kBranches && st == SS_OK; ++b) {
      e = cudaEventRecord(mp->join[b], mp->branch[b]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(mp->cap, mp->join[b], 0);
      if (e != cudaSuccess) st = many_fail(mp, SS_ECUDA, cudaGetErrorString(e));
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(mp->cap, &g);
    if (st != SS_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess)
      return many_fail(mp, SS_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    mp->graph = g;
    e = cudaGraphInstantiate(&mp->exec, g, 0);
    if (e != cudaSuccess) {
      mp->exec = nullptr;
      return many_fail(mp, SS_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    mp->cap_in.assign(chunks, chunks + n);
    mp->cap_n.assign(n_samples, n_samples + n);
    mp->cap_out = outs;
  }
  cudaError_t e = cudaGraphLaunch(mp->exec, mp->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(mp->stream);
  if (e != cudaSuccess)
    return many_fail(mp, SS_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  for (int i = 0; i < n; ++i) {
    ss_status st = check_status(mp->plans[i]);
    if (st != SS_OK)
      return many_fail(mp, st, "recording " + std::to_string(i) + ": " + mp->plans[i]->err);
  }
  mp->err.clear();
  return SS_OK;
}

ss_status ss_many_plan(ss_many_t mp, int i, ss_plan_t* plan) {
  if (!mp || !plan) return many_fail(mp, SS_EINVAL, "NULL argument");
  if (i < 0 || i >= (int)mp->plans.size()) return many_fail(mp, SS_EINVAL, "index out of range");
  *plan = mp->plans[i];
  return SS_OK;
}

ss_status ss_destroy_many(ss_many_t mp) {
  if (!mp) return SS_OK;
  DeviceGuard guard(mp->device);
  if (mp->stream) cudaStreamSynchronize(mp->stream);
  many_release(mp);
  delete mp;
  return SS_OK;
}

const char* ss_many_last_error(ss_many_t mp) {
  return mp ? mp->err.c_str() : g_many_error.c_str();
}

}  // extern "C"
