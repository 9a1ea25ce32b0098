// Per-phase CUDA-event timing and the launch counter (see hz.h).
#include <stdlib.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "hz_internal.h"

namespace hz {
namespace {

const char* kNames[PH_COUNT] = {"fft_row_fwd", "fft_line", "fft_sym_inv", "fft_row_inv_acc",
                                "stencil", "cgs2_dots", "cgs2_update", "givens",
                                "solution_update", "residual", "norm"};

struct Pending {
  cudaEvent_t e0, e1;
  Phase ph;
  double bytes, flops;
  int launches;
  bool live;
  SolveSink* sink;
};

struct Acc {
  long long launches = 0;
  double ms = 0, bytes = 0, flops = 0;
};

std::atomic<unsigned long long> g_launches{0};
// NVTX ranges named after the phases around their launches, for timeline
// tools, when the environment sets HZ_NVTX=1 (read once)
bool nvtx_on() {
  static const bool on = [] {
    const char* e = getenv("HZ_NVTX");
    return e && e[0] == '1';
  }();
  return on;
}
std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Pending> g_pend;
std::vector<int> g_free_slots;
Acc g_acc[PH_COUNT];
thread_local SolveSink* g_tls_sink = nullptr;

// only: resolve only the entries of this sink (nullptr: every entry)
void resolve_locked(SolveSink* only = nullptr) {
  for (size_t i = 0; i < g_pend.size(); ++i) {
    Pending& p = g_pend[i];
    if (!p.live) continue;
    if (only && p.sink != only) continue;
    float ms = 0.f;
    if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      Acc& a = g_acc[p.ph];
      a.launches += p.launches;
      a.ms += ms;
      a.bytes += p.bytes;
      a.flops += p.flops;
      if (p.sink) {
        p.sink->ms[p.ph] += ms;
        p.sink->bytes[p.ph] += p.bytes;
      }
    } else {
      cudaGetLastError();
    }
    p.live = false;
    g_free_slots.push_back(int(i));
  }
}

// 8 independent FMA chains per thread; the result is stored so that no
// chain is dead code.
__global__ void fma_probe_kernel(double* out, double a, double b, int iters) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5,
         x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace

void count_launches(int k) {
  g_launches.fetch_add((unsigned long long)(long long)k, std::memory_order_relaxed);
}
bool profiling() { return g_on.load(std::memory_order_relaxed); }

void set_solve_sink(SolveSink* sink) { g_tls_sink = sink; }

void resolve_solve_sink(SolveSink* sink) {
  if (!sink) return;
  std::lock_guard<std::mutex> lk(g_mu);
  resolve_locked(sink);
}

PhaseScope::PhaseScope(cudaStream_t s, Phase p, double b, double f, int l)
    : st(s), ph(p), bytes(b), flops(f), launches(l) {
  count_launches(l);
  if (nvtx_on()) nvtxRangePushA(kNames[p]);
  if (!profiling()) return;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;  // no timing inside a graph capture
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_free_slots.empty() && g_pend.size() >= 4096) resolve_locked();
  if (g_free_slots.empty()) {
    Pending np{};
    if (cudaEventCreate(&np.e0) != cudaSuccess || cudaEventCreate(&np.e1) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    g_pend.push_back(np);
    g_free_slots.push_back(int(g_pend.size()) - 1);
  }
  slot = g_free_slots.back();
  g_free_slots.pop_back();
  sink = g_tls_sink;
  cudaEventRecord(g_pend[slot].e0, st);
}

PhaseScope::~PhaseScope() {
  if (nvtx_on()) nvtxRangePop();
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Pending& p = g_pend[slot];
  cudaEventRecord(p.e1, st);
  p.ph = ph;
  p.bytes = bytes;
  p.flops = flops;
  p.launches = launches;
  p.sink = sink;
  p.live = true;
}

}  // namespace hz

using namespace hz;

extern "C" hz_status hz_profile_enable(int on) {
  g_on.store(on != 0);
  return HZ_OK;
}

extern "C" hz_status hz_profile_read(hz_phase_stats* out, int max, int* count, int reset) {
  std::lock_guard<std::mutex> lk(g_mu);
  resolve_locked();
  int c = 0;
  for (int i = 0; i < PH_COUNT; ++i) {
    if (g_acc[i].launches == 0) continue;
    if (out && c < max) {
      memset(out[c].name, 0, sizeof(out[c].name));
      strncpy(out[c].name, kNames[i], sizeof(out[c].name) - 1);
      out[c].launches = g_acc[i].launches;
      out[c].ms = g_acc[i].ms;
      out[c].bytes = g_acc[i].bytes;
      out[c].flops = g_acc[i].flops;
    }
    ++c;
  }
  if (count) *count = c;
  if (reset)
    for (auto& a : g_acc) a = Acc();
  return HZ_OK;
}

extern "C" unsigned long long hz_launch_count(void) { return g_launches.load(); }

extern "C" hz_status hz_measure_fp64_peak(double* gflops) {
  if (!gflops) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  int dev = 0, sms = 0;
  HZ_CUDA(cudaGetDevice(&dev));
  HZ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 8000;
  double* out = nullptr;
  HZ_CUDA(cudaMalloc(&out, size_t(blocks) * threads * sizeof(double)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_probe_kernel<<<blocks, threads>>>(out, 0.999, 1e-3, 200);
  cudaEventRecord(e0);
  fma_probe_kernel<<<blocks, threads>>>(out, 0.999, 1e-3, iters);
  cudaEventRecord(e1);
  cudaError_t ce = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (ce != cudaSuccess) return cuda_error(ce, "fp64 probe");
  *gflops = 2.0 * 8.0 * iters * double(blocks) * threads / (double(ms) * 1e6);
  return HZ_OK;
}
