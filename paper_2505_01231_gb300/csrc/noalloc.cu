// noalloc.cu -- ss_s2_noalloc: the power spectrum of one float32 channel computed
// without any device allocation.
//
// Some callers cannot call cudaMalloc: a process whose device memory is owned up
// front by a framework's caching allocator or by a fixed memory budget, or a
// latency-critical loop that must not pay for an allocation (cudaMalloc can
// synchronise the device) or handle its failure.  For them this entry point
// runs the frame/window/FFT/centre + S2 kernel (K1) and the finalize kernel
// (K4) with all intermediate data in one file-scope static device array of
// kNoallocScratchBytes bytes, which every GPU that loads the library holds
// until the process exits.  The caller passes the input and the outputs.
#include <cmath>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace ss {
namespace {

// Layout of the scratch array: tables and accumulators first, then the centred
// spectra of all groups of one call.
constexpr size_t kTableBytes = 128 << 10;
constexpr size_t kWinOff = 0;                        // float  [4096]  window / sqrt(sum g^2)
constexpr size_t kTwOff = 16 << 10;                  // float2 [4096]  e^{+2 pi j a/T}
constexpr size_t kAccOff = 48 << 10;                 // double [4][2049] sums over groups
constexpr size_t kAutoOff = kAccOff + 4 * 2049 * 8;  // int    s2 combination index (0)
constexpr size_t kSpecOff = kTableBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_mu;
void* g_addr[64] = {};  // device address of the array, per device ordinal

thread_local std::string g_err;

ss_status fail(ss_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

// Device or managed memory (checked before anything is enqueued, so that a host
// pointer is refused instead of reaching a kernel).
bool on_device(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The window scaled by 1/sqrt(sum g^2) and the twiddles e^{+2 pi j a/T}, built on
// the device in float64 (the same definitions ss_plan evaluates on the host), so
// that a call enqueues kernels and memsets only.  One block.
constexpr int kTableThreads = 256;

__global__ void __launch_bounds__(kTableThreads)
k0_tables(int T, int window, double sigma, float* __restrict__ win, float2* __restrict__ tw) {
  __shared__ double red[kTableThreads];
  auto g_at = [&](int i) {
    if (window == SS_WIN_HANN) return 0.5 - 0.5 * cospi(2.0 * i / T);
    const double N = T, c = (N - 1.0) / 2.0, d = 4.0 * N * N * sigma * sigma;
    auto G = [&](double x) { return exp(-(x - c) * (x - c) / d); };
    return G(i) - G(-0.5) * (G(i + N) + G(i - N)) / (G(-0.5 + N) + G(-0.5 - N));
  };
  double s = 0.0;
  for (int i = threadIdx.x; i < T; i += kTableThreads) {
    const double g = g_at(i);
    s += g * g;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = kTableThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  const double scale = 1.0 / sqrt(red[0]);
  for (int i = threadIdx.x; i < T; i += kTableThreads) {
    win[i] = (float)(g_at(i) * scale);
    double sn, cs;
    sincospi(2.0 * i / T, &sn, &cs);
    tw[i] = make_float2((float)cs, (float)sn);
  }
}

}  // namespace

const char* noalloc_last_error() { return g_err.c_str(); }

}  // namespace ss

using namespace ss;

extern "C" ss_status ss_s2_noalloc(const float* d_signal, size_t n_samples, int T, double dt,
                                   int m, int window, double win_param, double* d_S2,
                                   double* d_S2_err, void* stream) {
  if (!d_signal || !d_S2) return fail(SS_EINVAL, "d_signal and d_S2 must not be NULL");
  if (!on_device(d_signal) || !on_device(d_S2) || (d_S2_err && !on_device(d_S2_err)))
    return fail(SS_EINVAL, "d_signal, d_S2 and d_S2_err must be device (or managed) memory");
  if (T < 8 || T > 4096 || (T & (T - 1))) return fail(SS_EINVAL, "T must be a power of two in [8, 4096]");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(SS_EINVAL, "dt must be > 0");
  if (m < 2) return fail(SS_EINVAL, "S2 needs m >= 2 (Eq. 32)");
  if (window != SS_WIN_HANN && window != SS_WIN_ACG) return fail(SS_EINVAL, "unknown window");
  if (window == SS_WIN_ACG && !(win_param > 0.0 && win_param < 10.0))
    return fail(SS_EINVAL, "sigma_t of the confined Gaussian must be in (0, 10)");
  const int M = T / 2 + 1, Mp = (M + 3) & ~3;
  const long long G = (long long)(n_samples / ((size_t)m * T));
  if (G < 2) return fail(SS_ESTATE, "fewer than two groups: no error estimate (Eq. 35)");
  const size_t spec_bytes = (size_t)G * m * Mp * sizeof(float2);
  if (spec_bytes > kNoallocScratchBytes - kSpecOff)
    return fail(SS_EINVAL, "input too long for the static scratch: " + std::to_string(G) +
                               " groups need " + std::to_string(spec_bytes) +
                               " bytes of spectra, the scratch holds " +
                               std::to_string(kNoallocScratchBytes - kSpecOff));
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // set-up, once per device, with that device current: the device address of the
  // static array (its name in host code is only a host-side stand-in)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(SS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return fail(SS_EUNSUPPORTED, "device ordinal above 63");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return fail(SS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_addr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_addr[dev]);
  }

  float* d_win = reinterpret_cast<float*>(base + kWinOff);
  float2* d_tw = reinterpret_cast<float2*>(base + kTwOff);
  double* d_acc = reinterpret_cast<double*>(base + kAccOff);
  int* d_auto = reinterpret_cast<int*>(base + kAutoOff);
  float2* d_spec = reinterpret_cast<float2*>(base + kSpecOff);
#define NA_TRY(call)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return fail(SS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
  k0_tables<<<1, kTableThreads, 0, s>>>(T, window, win_param, d_win, d_tw);
  NA_TRY(cudaGetLastError());
  // the array keeps the previous call's contents: clear the sums and the index
  NA_TRY(cudaMemsetAsync(d_acc, 0, (size_t)4 * M * sizeof(double), s));
  NA_TRY(cudaMemsetAsync(d_auto, 0, sizeof(int), s));
  int nsm = 1;
  NA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  SampleSource src;
  src.carry = nullptr;
  src.carry_n = 0;
  src.carry_stride = 0;
  src.chunk = d_signal;
  src.chunk_stride = (long long)n_samples;
  src.dtype = SS_F32;
  NA_TRY(launch_k1_spectra(src, 0, (int)G, 1, T, m, M, Mp, d_win, d_tw, d_spec,
                           (long long)G * m * Mp, d_auto, d_acc, 1, 1.0f / (float)(m - 1),
                           4 * nsm, s));
  NA_TRY(launch_k4_finalize(d_acc, 1, 1, M, kLayoutVector, G, dt, d_S2, d_S2_err, s));
#undef NA_TRY
  g_err.clear();
  return SS_OK;
}

extern "C" const char* ss_noalloc_last_error(void) { return ss::noalloc_last_error(); }
