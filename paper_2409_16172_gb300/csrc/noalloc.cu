// Allocation-free preconditioner apply.
//
// hz_apply_preconditioner keeps its work arrays (the transformed input and
// the K symbol planes) in a plan that the library allocates.  Some callers
// cannot allocate device memory at the point where they need the apply: a
// solver embedded in another runtime that owns the GPU's memory through its
// own pool and forbids raw cudaMalloc, or a real-time loop where cudaMalloc /
// cudaFree would stall (they synchronise the device).  This entry point runs
// the same kernels with its work arrays in one file-scope device array of
// fixed size, so the call itself allocates nothing.  The array is part of the
// library's device image: every GPU that loads the library holds it until the
// process exits.
#include <cuda.h>

#include <mutex>

#include "hz_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The array's device address belongs to the CUDA context that loaded the
// library's module on that device.  A context can be destroyed and a new one
// created on the same device (cudaDeviceReset, or the primary context
// released and retained again); the new context holds its own copy of the
// array at an address that may differ.  So the cached address is keyed on the
// context's unique id (cuCtxGetId, never reused within a process), not on the
// device ordinal alone, and is looked up again when the id changes.
struct ScratchSlot {
  unsigned long long ctx_id = 0;  // 0: nothing cached
  void* ptr = nullptr;
};
std::mutex g_mu;
ScratchSlot g_slot[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Id of the calling thread's current context (after cudaGetDevice has made
// the device's primary context current if there was none).
hz_status current_context_id(unsigned long long* id) {
  if (!g_ctx_current || !g_ctx_id) {
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    void* f1 = nullptr;
    void* f2 = nullptr;
    const cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                           cudaEnableDefault, &q1);
    const cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000,
                                                           cudaEnableDefault, &q2);
    if (e1 != cudaSuccess || e2 != cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
        q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return hz::set_error(HZ_ERR_CUDA, "driver entry points cuCtxGetCurrent / cuCtxGetId not found");
    g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx)
    return hz::set_error(HZ_ERR_CUDA, "no current CUDA context");
  unsigned long long cid = 0;
  if (g_ctx_id(ctx, &cid) != CUDA_SUCCESS || cid == 0)
    return hz::set_error(HZ_ERR_CUDA, "cuCtxGetId failed");
  *id = cid;
  return HZ_OK;
}

}  // namespace

using namespace hz;

extern "C" hz_status hz_apply_preconditioner_noalloc(const hz_medium* med, const void* x, void* y,
                                                     int nrhs, int precision, void* stream) {
  if (!med || !x || !y) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  if (nrhs < 1) return set_error(HZ_ERR_INVALID_ARG, "nrhs must be >= 1");
  if (precision != 0 && precision != 1) return set_error(HZ_ERR_INVALID_ARG, "precision must be 0 or 1");
  const long n = med->n;
  const size_t es = precision == 0 ? 16 : 8;
  const size_t tmp_bytes = align256(size_t(nrhs) * n * es);
  const size_t need = tmp_bytes + size_t(nrhs) * med->K * n * es;
  if (need > kScratchBytes)
    return set_error(HZ_ERR_INVALID_ARG,
                     "allocation-free apply needs %zu bytes of scratch (nrhs * n * (K + 1) * %zu); "
                     "the static limit is %zu bytes",
                     need, es, kScratchBytes);

  // Set-up, once per device and context with that device current: the
  // host-side name of the array is not a device address; ask the runtime
  // for it, and ask again when the context has changed.
  int dev = 0;
  HZ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(HZ_ERR_INVALID_ARG, "device id %d too large", dev);
  if (dev != med->device)
    return set_error(HZ_ERR_INVALID_ARG, "the medium lives on device %d but device %d is current",
                     med->device, dev);
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned long long cid = 0;
    HZ_TRY(current_context_id(&cid));
    ScratchSlot& slot = g_slot[dev];
    if (slot.ctx_id != cid || !slot.ptr) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(scratch)");
      slot.ctx_id = cid;
      slot.ptr = p;
    }
    scratch = slot.ptr;
  }
  unsigned char* base = static_cast<unsigned char*>(scratch);
  void* tmp = base;
  void* planes = base + tmp_bytes;

  // Same passes as the plan-based apply: x forward, forward along the other
  // axes, symbol * inverse along the last axis per node, 3D y inverse, and
  // the x inverse with the weighted sum (Eqn. 103 / 403).  Every scratch
  // element a pass reads was written earlier in the same call (the planes
  // only on the rows / slabs that use the node), so nothing needs clearing.
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int prec = precision;
  const int nx = med->nx, ny = med->ny, nz = med->nz;
  const FftOps* ox = fft_ops(nx);
  const FftOps* oy = fft_ops(ny);
  const AxisTables& tx = med->ax[0];
  const AxisTables& ty = med->ax[1];
  auto tw = [&](const AxisTables& t) -> const void* { return prec == 0 ? (const void*)t.tw64 : (const void*)t.tw32; };
  auto tw2 = [&](const AxisTables& t) -> const void* { return prec == 0 ? nullptr : (const void*)t.tw32p; };
  auto xi = [&](const AxisTables& t) -> const void* { return prec == 0 ? (const void*)t.xi2_64 : (const void*)t.xi2_32; };
  const void* A = prec == 0 ? (const void*)med->symA64 : (const void*)med->symA32;
  const void* G = prec == 0 ? (const void*)med->symG64 : (const void*)med->symG32;
  const void* D = prec == 0 ? (const void*)med->symD64 : (const void*)med->symD32;
  const void* rec = prec == 0 ? (const void*)med->rec64 : (const void*)med->rec32;
  const long rows = n / nx;
  const long slab = long(nx) * ny;
  HZ_TRY(ox->row_fwd(prec, static_cast<const double2*>(x), nullptr, rows, rows * nrhs, tw(tx), tmp, st,
                     nullptr, nullptr, 0));
  HZ_TRY(oy->line_pass(prec, -1, tmp, nx, nz, nx, slab, n, nrhs, nullptr, med->K, tw(ty), st, nullptr, 1));
  int launches = 2;
  if (med->dim == 2) {
    HZ_TRY(oy->line_sym_inv(prec, tmp, planes, nx, 1, nx, 0, n, med->K, nrhs, xi(tx), nullptr, xi(ty),
                            A, G, D, med->rowmask, 0, 1, tw(ty), tw2(ty), st, nullptr, 1, 1));
    launches += 1;
  } else {
    const FftOps* oz = fft_ops(nz);
    const AxisTables& tz = med->ax[2];
    HZ_TRY(oz->line_pass(prec, -1, tmp, nx, ny, slab, nx, n, nrhs, nullptr, med->K, tw(tz), st,
                         nullptr, 1));
    HZ_TRY(oz->line_sym_inv(prec, tmp, planes, nx, ny, slab, nx, n, med->K, nrhs, xi(tx), xi(ty),
                            xi(tz), A, G, D, med->slabmask, 0, 1, tw(tz), tw2(tz), st, nullptr, 1, 1));
    HZ_TRY(oy->line_pass(prec, +1, planes, nx, nz, nx, slab, n, nrhs * med->K, med->slabmask, med->K,
                         tw(ty), st, nullptr, med->K));
    launches += 3;
  }
  HZ_TRY(ox->row_inv_acc(prec, 1, planes, rec, med->segtab, med->nseg, med->rowmask, med->K, rows,
                         rows * nrhs, n, 1.0 / double(n), tw(tx), y, st, nullptr, 0, nullptr, 0, med->gnode,
                         prec == 0 ? (const void*)med->gw64 : (const void*)med->gw32));
  count_launches(launches + 1);
  return HZ_OK;
}
