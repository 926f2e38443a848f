// tune.cu -- the autotuner of the plan's kernel forms, and the text form of its
// choices ("wisdom"): ss_autotune, ss_get_tuning, ss_set_tuning.
//
// A plan's results do not depend on these choices; only its speed does.  Two
// stages have alternative forms:
//   K1 (frame/window/FFT/centre): groups resident in shared memory within 74 KB
//       (three CTAs per SM) or 96 KB (two), or one frame at a time;
//   K2 (bispectrum): 4 x 4 micro-tiles in CTAs of 256 threads (4 stages), or
//       8 x 4 micro-tiles in CTAs of 128 threads with 2 or 3 stages.
// ss_autotune times every form on the plan's own shapes (frame length, group
// size, channels, precision) on this GPU, on a synthetic record of Gaussian
// noise generated on the device, and keeps the fastest of each stage.  The
// choice is keyed by the configuration and the GPU, so that a saved string can
// be applied to later plans of the same shape (ss_set_tuning), as FFTW applies
// its wisdom.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "internal.cuh"
#include "plan_state.cuh"

using namespace ss;

namespace {

const char* const kK1Names[kK1Modes] = {"auto", "r96", "frames", "warp"};
const char* const kK2Names[kK2Variants] = {"44", "84s2", "84s3", "44s3", "84w"};

// Gaussian noise (counter-based: SplitMix64 of the element index, Box-Muller),
// float32 or int16 (scaled by 1000, saturated), for timing only.
__global__ void k_tune_noise(void* out, long long n, int dtype, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u1 = ((float)(z >> 40) + 0.5f) * (1.0f / 16777216.0f);
    const float u2 = ((float)((z >> 16) & 0xFFFFFFull) + 0.5f) * (1.0f / 16777216.0f);
    const float g = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    if (dtype == SS_F32)
      static_cast<float*>(out)[i] = g;
    else
      static_cast<short*>(out)[i] = (short)fmaxf(-32768.f, fminf(32767.f, rintf(1000.f * g)));
  }
}

std::string key_of(const ss_plan_s* p) {
  cudaDeviceProp prop;
  std::string gpu = "unknown";
  if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) gpu = prop.name;
  for (char& c : gpu)
    if (c == ' ') c = '_';
  static const char* const prec[] = {"fp32", "tf32x3", "bf16x3", "bf16", "fp16x3"};
  char buf[256];
  std::snprintf(buf, sizeof(buf), "T=%d m=%d C=%d dtype=%s prec=%s sms=%d gpu=%s", p->T, p->m,
                p->C, p->dtype == SS_F32 ? "f32" : "i16", prec[p->precision], p->nsm,
                gpu.c_str());
  return buf;
}

std::string tuning_of(const ss_plan_s* p) {
  std::string s = "polyspec-tuning 1 " + key_of(p) + " | k1=" + kK1Names[p->k1_mode] +
                  " k2=" + kK2Names[p->k2_variant];
  if (p->tune_ms[0] > 0.f) {  // the pass times of the last ss_autotune
    char buf[64];
    s += " | ms";
    for (int i = 0; i < kK1Modes + kK2Variants; ++i) {
      if (p->tune_ms[i] <= 0.f) continue;
      std::snprintf(buf, sizeof(buf), " %s:%s=%.4f", i < kK1Modes ? "k1" : "k2",
                    i < kK1Modes ? kK1Names[i] : kK2Names[i - kK1Modes], p->tune_ms[i]);
      s += buf;
    }
  }
  return s;
}

// value of "name=" in s (up to the next blank), or "" if absent
std::string field(const std::string& s, const char* name) {
  const std::string pat = std::string(name) + "=";
  size_t at = 0;
  while ((at = s.find(pat, at)) != std::string::npos) {
    if (at == 0 || s[at - 1] == ' ') {
      const size_t b = at + pat.size();
      const size_t e = s.find(' ', b);
      return s.substr(b, e == std::string::npos ? std::string::npos : e - b);
    }
    at += pat.size();
  }
  return "";
}

// device time of one pass of the plan's K1-K3 over the synthetic record
ss_status time_pass(ss_plan_s* p, const void* rec, long long n, cudaEvent_t e0, cudaEvent_t e1,
                    float* ms) {
  ss_status st = reset_state(p);
  if (st != SS_OK) return st;
  if (cudaEventRecord(e0, p->stream) != cudaSuccess) return SS_ECUDA;
  st = run_device_chunk(p, rec, n, n);
  if (st != SS_OK) return st;
  if (cudaEventRecord(e1, p->stream) != cudaSuccess) return SS_ECUDA;
  if (cudaEventSynchronize(e1) != cudaSuccess) return SS_ECUDA;
  return cudaEventElapsedTime(ms, e0, e1) == cudaSuccess ? SS_OK : SS_ECUDA;
}

}  // namespace

extern "C" {

ss_status ss_get_tuning(ss_plan_t p, char* out, size_t cap) {
  if (!p || !out || cap == 0) return plan_fail(p, SS_EINVAL, "NULL argument");
  const std::string s = tuning_of(p);
  if (s.size() + 1 > cap)
    return plan_fail(p, SS_EINVAL, "buffer too small: " + std::to_string(s.size() + 1) + " bytes");
  std::memcpy(out, s.c_str(), s.size() + 1);
  return SS_OK;
}

ss_status ss_set_tuning(ss_plan_t p, const char* text) {
  if (!p || !text) return plan_fail(p, SS_EINVAL, "NULL argument");
  const std::string s(text);
  // a keyed string applies only to a plan of the same configuration on the same GPU
  const size_t bar = s.find(" | ");
  const std::string body = bar == std::string::npos ? s : s.substr(bar + 3);
  if (bar != std::string::npos) {
    const std::string key = s.substr(0, bar);
    const std::string mine = key_of(p);
    if (key.size() < mine.size() || key.compare(key.size() - mine.size(), mine.size(), mine) != 0)
      return plan_fail(p, SS_EINVAL, "tuning of another configuration or GPU: " + key);
  }
  int k1 = p->k1_mode, k2 = p->k2_variant;
  const std::string v1 = field(body, "k1"), v2 = field(body, "k2");
  if (!v1.empty()) {
    k1 = -1;
    for (int i = 0; i < kK1Modes; ++i)
      if (v1 == kK1Names[i]) k1 = i;
  }
  if (!v2.empty()) {
    k2 = -1;
    for (int i = 0; i < kK2Variants; ++i)
      if (v2 == kK2Names[i]) k2 = i;
  }
  if (k1 < 0 || k2 < 0) return plan_fail(p, SS_EINVAL, "unknown kernel form in: " + s);
  for (ss_plan_s* q = p; q; q = q->shadow) {
    q->k1_mode = k1;
    q->k2_variant = k2;
  }
  return SS_OK;
}

ss_status ss_autotune(ss_plan_t p, double* best_ms) {
  if (!p) return plan_fail(nullptr, SS_EINVAL, "plan is NULL");
  if (p->broken) return plan_fail(p, SS_ESTATE, "plan is unusable after a CUDA failure: " + p->err);
  if (p->groups != 0 || p->carry_n != 0)
    return plan_fail(p, SS_ESTATE, "ss_autotune is valid only before the first ss_accumulate");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != p->device) cudaSetDevice(p->device);
  struct Restore {
    int dev;
    ~Restore() {
      if (dev >= 0) cudaSetDevice(dev);
    }
  } restore{prev};
  // enough groups for several waves of every kernel, within one batch: 64 per SM,
  // so that the pair kernels' items hold about as many groups as in a full batch
  // (with 16 per SM, the items of the 128-thread tilings were a fifth of their
  // full-batch size and their float64 flushes weighed several times more)
  const long long per_group = (long long)p->m * p->T;
  const long long G = std::min<long long>(p->Gb_max, std::max(8, 64 * p->nsm));
  const long long n = G * per_group;
  void* rec = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool timing = p->timing;
  p->timing = false;
  ss_status st = SS_OK;
  auto done = [&](ss_status s) {
    if (rec) cudaFree(rec);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    p->timing = timing;
    return s;
  };
  if (cudaMalloc(&rec, (size_t)n * p->C * p->elem) != cudaSuccess) {
    cudaGetLastError();
    return done(plan_fail(p, SS_ENOMEM, "autotune: no device memory for the synthetic record"));
  }
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return done(plan_fail(p, SS_ECUDA, "autotune: cudaEventCreate failed"));
  k_tune_noise<<<4 * p->nsm, 256, 0, p->stream>>>(rec, n * p->C, p->dtype, 0x5EEDull);
  if (cudaGetLastError() != cudaSuccess)
    return done(plan_fail(p, SS_ECUDA, "autotune: noise kernel launch failed"));
  // the fastest of `count` forms: one untimed pass, then the best of three
  auto pick = [&](int* slot, int count, float* times) -> ss_status {
    float best = 1e30f;
    int arg = *slot;
    for (int v = 0; v < count; ++v) {
      *slot = v;
      float t = 0.f, tmin = 1e30f;
      ss_status s = time_pass(p, rec, n, e0, e1, &t);
      if (s == SS_ECUDA && !p->broken) {  // a form this plan's shapes cannot take
        cudaGetLastError();
        continue;
      }
      for (int r = 0; r < 3 && s == SS_OK; ++r) {
        s = time_pass(p, rec, n, e0, e1, &t);
        tmin = std::min(tmin, t);
      }
      if (s != SS_OK) return s;
      times[v] = tmin;
      if (tmin < best) {
        best = tmin;
        arg = v;
      }
    }
    *slot = arg;
    if (best_ms) *best_ms = best;
    return SS_OK;
  };
  for (float& t : p->tune_ms) t = 0.f;
  st = pick(&p->k1_mode, kK1Modes, p->tune_ms);
  if (st == SS_OK && !p->c3.empty()) st = pick(&p->k2_variant, kK2Variants, p->tune_ms + kK1Modes);
  if (st == SS_OK) st = reset_state(p);
  if (st == SS_OK && cudaStreamSynchronize(p->stream) != cudaSuccess)
    st = plan_fail(p, SS_ECUDA, "autotune: stream synchronisation failed");
  if (st == SS_OK && p->shadow) {
    p->shadow->k1_mode = p->k1_mode;
    p->shadow->k2_variant = p->k2_variant;
  }
  return done(st);
}

}  // extern "C"
