// C ABI: errors, allocator, plans, operator / preconditioner apply and the
// restarted (F)GMRES driver (Section 5, "GMRES implementation"; right and
// flexible preconditioning with Q_M of Eqn. 103 / 403).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "hz_internal.h"
#include "kernels.h"

namespace hz {

// ---------------------------------------------------------------------------
// errors and allocation
// ---------------------------------------------------------------------------
namespace {
thread_local std::string g_err;
void* (*g_alloc)(size_t, void*) = nullptr;
void (*g_free)(void*, void*) = nullptr;
void* g_ctx = nullptr;
}  // namespace

hz_status set_error(hz_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

hz_status cuda_error(cudaError_t e, const char* what) {
  const hz_status st = e == cudaErrorMemoryAllocation ? HZ_ERR_OOM : HZ_ERR_CUDA;
  return set_error(st, "%s: %s", what, cudaGetErrorString(e));
}

namespace {
thread_local cudaStream_t g_tls_stream = nullptr;
thread_local bool g_tls_async = false;
}  // namespace

cudaStream_t tls_stream() { return g_tls_stream; }
void set_tls_stream(cudaStream_t st, bool async_alloc) {
  g_tls_stream = st;
  g_tls_async = async_alloc;
}

void* dev_alloc(size_t bytes) {
  if (g_alloc) return g_alloc(bytes, g_ctx);
  void* p = nullptr;
  const cudaError_t e = g_tls_async ? cudaMallocAsync(&p, bytes, g_tls_stream) : cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void* p) {
  if (!p) return;
  if (g_free) g_free(p, g_ctx);
  else if (g_tls_async) cudaFreeAsync(p, g_tls_stream);
  else cudaFree(p);
}

const FftOps* fft_ops_8();
const FftOps* fft_ops_12();
const FftOps* fft_ops_16();
const FftOps* fft_ops_24();
const FftOps* fft_ops_32();
const FftOps* fft_ops_48();
const FftOps* fft_ops_64();
const FftOps* fft_ops_96();
const FftOps* fft_ops_128();
const FftOps* fft_ops_192();
const FftOps* fft_ops_256();
const FftOps* fft_ops_512();
const FftOps* fft_ops_1024();
const FftOps* fft_ops_2048();
const FftOps* fft_ops_20();
const FftOps* fft_ops_40();
const FftOps* fft_ops_60();
const FftOps* fft_ops_120();
const FftOps* fft_ops_180();
const FftOps* fft_ops_240();
const FftOps* fft_ops_360();
const FftOps* fft_ops_480();
const FftOps* fft_ops_720();
const FftOps* fft_ops_960();
const FftOps* fft_ops_1440();
const FftOps* fft_ops_1920();
const FftOps* fft_ops_2400();
const FftOps* fft_ops_2880();
const FftOps* fft_ops_3600();
const FftOps* fft_ops_4800();

const FftOps* fft_ops(int N) {
  switch (N) {
    case 8: return fft_ops_8();
    case 12: return fft_ops_12();
    case 16: return fft_ops_16();
    case 24: return fft_ops_24();
    case 32: return fft_ops_32();
    case 48: return fft_ops_48();
    case 64: return fft_ops_64();
    case 96: return fft_ops_96();
    case 128: return fft_ops_128();
    case 192: return fft_ops_192();
    case 256: return fft_ops_256();
    case 512: return fft_ops_512();
    case 1024: return fft_ops_1024();
    case 2048: return fft_ops_2048();
    case 20: return fft_ops_20();
    case 40: return fft_ops_40();
    case 60: return fft_ops_60();
    case 120: return fft_ops_120();
    case 180: return fft_ops_180();
    case 240: return fft_ops_240();
    case 360: return fft_ops_360();
    case 480: return fft_ops_480();
    case 720: return fft_ops_720();
    case 960: return fft_ops_960();
    case 1440: return fft_ops_1440();
    case 1920: return fft_ops_1920();
    case 2400: return fft_ops_2400();
    case 2880: return fft_ops_2880();
    case 3600: return fft_ops_3600();
    case 4800: return fft_ops_4800();
    default: return nullptr;
  }
}

// ---------------------------------------------------------------------------
// preconditioner apply: Q_M v = sum_k w_k IFFT(q_k FFT(v)) / n
// ---------------------------------------------------------------------------
static hz_status ensure_planes(hz_plan* p, int prec) {
  if (p->planes && p->planes_prec <= prec) return HZ_OK;  // c128 buffer also fits c64
  const hz_medium* m = p->med;
  const size_t es = prec == 0 ? 16 : 8;
  void* np = dev_alloc(size_t(p->max_nrhs) * m->K * m->n * es);
  if (!np) return set_error(HZ_ERR_OOM, "no memory for %d x %d symbol planes", p->max_nrhs, m->K);
  if (p->planes) {
    auto it = std::find(p->arena.ptrs.begin(), p->arena.ptrs.end(), p->planes);
    if (it != p->arena.ptrs.end()) p->arena.ptrs.erase(it);
    dev_free(p->planes);
  }
  p->arena.ptrs.push_back(np);
  p->arena.bytes += size_t(p->max_nrhs) * m->K * m->n * es;
  p->planes = np;
  p->planes_prec = prec;
  return HZ_OK;
}

// in: nrhs c128 vectors at stride n, each scaled by scale[b] (NULL = 1).
// out_kind 0: c64 output, 1: c128 output.  prec 0: complex128 arithmetic.
hz_status precond_apply(hz_plan* p, int prec, const double2* in, const double* scale, int nrhs,
                        void* out, int out_kind, cudaStream_t st, const int* active) {
  const hz_medium* m = p->med;
  HZ_TRY(ensure_planes(p, prec));
  const int nx = m->nx, ny = m->ny, nz = m->nz;
  const long n = m->n;
  const FftOps* ox = fft_ops(nx);
  const FftOps* oy = fft_ops(ny);
  const AxisTables& tx = m->ax[0];
  const AxisTables& ty = m->ax[1];
  auto tw = [&](const AxisTables& t) -> const void* { return prec == 0 ? (const void*)t.tw64 : (const void*)t.tw32; };
  // paired (two columns per thread) complex64 symbol pass unless tuned off
  auto tw2 = [&](const AxisTables& t) -> const void* {
    return prec == 1 && p->tune.col_pair ? (const void*)t.tw32p : nullptr;
  };
  auto xi = [&](const AxisTables& t) -> const void* { return prec == 0 ? (const void*)t.xi2_64 : (const void*)t.xi2_32; };
  const void* A = prec == 0 ? (const void*)m->symA64 : (const void*)m->symA32;
  const void* G = prec == 0 ? (const void*)m->symG64 : (const void*)m->symG32;
  const void* D = prec == 0 ? (const void*)m->symD64 : (const void*)m->symD32;
  const void* rec = prec == 0 ? (const void*)m->rec64 : (const void*)m->rec32;
  const long rows = n / nx;
  const double s = prec == 0 ? 16.0 : 8.0;          // working complex element
  const double so = out_kind == 1 ? 16.0 : 8.0;     // output element
  const double rb = prec == 0 ? 8.0 : 4.0;          // interpolation record
  const double B = nrhs, K = m->K, dn = double(n);
  auto l2 = [](int N) { return std::log2(double(N)); };
  // the scattering x-inverse pass adds into out: cleared by the x-forward pass
  const bool scatter = p->tune.rowinv_mode == 3;
  {
    PhaseScope ps(st, PH_ROW_FWD, B * dn * (16.0 + s + (scatter ? so : 0.0)),
                  B * 5.0 * dn * l2(nx));
    HZ_TRY(ox->row_fwd(prec, in, scale, rows, rows * nrhs, tw(tx), p->tmp, st, active,
                       scatter ? out : nullptr, long(nx) * long(so)));
  }
  // forward FFT along every axis but x, in place on tmp
  {
    PhaseScope ps(st, PH_LINE, B * 2.0 * s * dn, B * 5.0 * dn * l2(ny));
    HZ_TRY(oy->line_pass(prec, -1, p->tmp, nx, nz, nx, long(nx) * ny, n, nrhs, nullptr, m->K,
                         tw(ty), st, active, 1));
  }
  if (m->dim == 2) {
    PhaseScope ps(st, PH_SYMINV, B * (dn * s + m->rowk_used * nx * s),
                  B * K * (5.0 * dn * l2(ny) + 14.0 * dn));
    HZ_TRY(oy->line_sym_inv(prec, p->tmp, p->planes, nx, 1, nx, 0, n, m->K, nrhs, xi(tx), nullptr,
                            xi(ty), A, G, D, m->rowmask, 0, 1, tw(ty), tw2(ty), st, active,
                            p->tune.syminv_kpb, p->tune.col_pair));
  } else {
    const FftOps* oz = fft_ops(nz);
    const AxisTables& tz = m->ax[2];
    const long slab = long(nx) * ny;
    {
      PhaseScope ps(st, PH_LINE, B * 2.0 * s * dn, B * 5.0 * dn * l2(nz));
      HZ_TRY(oz->line_pass(prec, -1, p->tmp, nx, ny, slab, nx, n, nrhs, nullptr, m->K, tw(tz), st,
                           active, 1));
    }
    {
      PhaseScope ps(st, PH_SYMINV, B * (dn * s + m->slabk_used * slab * s),
                    B * K * (5.0 * dn * l2(nz) + 14.0 * dn));
      HZ_TRY(oz->line_sym_inv(prec, p->tmp, p->planes, nx, ny, slab, nx, n, m->K, nrhs, xi(tx),
                              xi(ty), xi(tz), A, G, D, m->slabmask, 0, 1, tw(tz), tw2(tz), st,
                              active, p->tune.syminv_kpb, p->tune.col_pair));
    }
    {
      PhaseScope ps(st, PH_LINE, B * 2.0 * s * m->slabk_used * slab,
                    B * 5.0 * m->slabk_used * slab * l2(ny));
      HZ_TRY(oy->line_pass(prec, +1, p->planes, nx, nz, nx, slab, n, nrhs * m->K, m->slabmask, m->K,
                           tw(ty), st, active, m->K));
    }
  }
  {
    PhaseScope ps(st, PH_ROW_INV, B * (m->rowk_used * nx * s + dn * (rb + so)),
                  B * (m->rowk_used * 5.0 * nx * l2(nx) + 8.0 * dn));
    HZ_TRY(ox->row_inv_acc(prec, out_kind, p->planes, rec, m->segtab, m->nseg, m->rowmask, m->K,
                           rows, rows * nrhs, n, 1.0 / double(n), tw(tx), out, st, active,
                           p->tune.rowinv_mode, m->rowitems, m->nitems, m->gnode,
                           prec == 0 ? (const void*)m->gw64 : (const void*)m->gw32));
  }
  return HZ_OK;
}

}  // namespace hz

using namespace hz;

extern "C" const char* hz_last_error(void) { return g_err.c_str(); }

extern "C" const char* hz_version(void) { return "hz-pdo 0.1 (sm_103a)"; }

extern "C" hz_status hz_set_allocator(void* (*alloc)(size_t, void*), void (*release)(void*, void*),
                                      void* ctx) {
  if ((alloc == nullptr) != (release == nullptr))
    return set_error(HZ_ERR_INVALID_ARG, "alloc and release must both be set or both be NULL");
  g_alloc = alloc;
  g_free = release;
  g_ctx = ctx;
  return HZ_OK;
}

extern "C" hz_status hz_plan_create(hz_medium* med, const hz_solver_opts* opts, int max_nrhs,
                                    hz_plan** out) {
  if (!med || !opts || !out) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (max_nrhs < 1) return set_error(HZ_ERR_INVALID_ARG, "max_nrhs must be >= 1");
  if (opts->precision != 0 && opts->precision != 1)
    return set_error(HZ_ERR_INVALID_ARG, "precision must be 0 or 1");
  if (opts->no_precond != 0 && opts->no_precond != 1)
    return set_error(HZ_ERR_INVALID_ARG, "no_precond must be 0 or 1");
  if (opts->left != 0 && opts->left != 1) return set_error(HZ_ERR_INVALID_ARG, "left must be 0 or 1");
  if (opts->restart < 1 || opts->restart > HZ_MAX_RESTART)
    return set_error(HZ_ERR_INVALID_ARG, "restart must be in [1, %d]", HZ_MAX_RESTART);
  if (!(opts->tol > 0) || opts->maxit < 1) return set_error(HZ_ERR_INVALID_ARG, "need tol > 0, maxit >= 1");
  hz_plan* p = new hz_plan();
  p->med = med;
  p->opts = *opts;
  p->max_nrhs = max_nrhs;
  const long n = med->n;
  const int m = opts->restart;
  const int B = max_nrhs;
  auto fail = [&](hz_status s) {
    p->arena.release();
    delete p;
    return s;
  };
  hz_status st;
  const size_t es = opts->precision == 0 ? 16 : 8;
  void* tmp = nullptr;
  if ((st = p->arena.alloc(reinterpret_cast<char**>(&tmp), size_t(B) * n * 16)) != HZ_OK) return fail(st);
  p->tmp = tmp;
  if ((st = ensure_planes(p, opts->precision)) != HZ_OK) return fail(st);
  if ((st = p->arena.alloc(&p->V, size_t(m + 1) * B * n)) != HZ_OK) return fail(st);
  // Z: FGMRES basis (c64); the FP64 path keeps one c128 work vector per rhs
  void* Z = nullptr;
  const size_t zlen = opts->precision == 1 ? size_t(m) * B * n * es : size_t(B) * n * 16;
  if ((st = p->arena.alloc(reinterpret_cast<char**>(&Z), zlen)) != HZ_OK) return fail(st);
  p->Z = Z;
  if ((st = p->arena.alloc(&p->u, size_t(B) * n)) != HZ_OK) return fail(st);
  if ((st = p->arena.alloc(&p->f, size_t(B) * n)) != HZ_OK) return fail(st);
  // block partial sums: the stencil residual (one per block), the CGS2 dot
  // partials (2 (j+1) nblk doubles per rhs with at most 4 x 152 blocks over
  // the launch, 8 vectors per chunk) and the update norms (<= 8 x 152 blocks)
  const int nblk = std::max(stencil_blocks(n), krylov_blocks(n, 1, 1));
  p->partial_len = size_t(B) * (m + 2) * std::max(nblk, 1024) * 2;
  if ((st = p->arena.alloc(&p->partial, p->partial_len)) != HZ_OK) return fail(st);
  *out = p;
  return HZ_OK;
}

extern "C" hz_status hz_plan_bytes(const hz_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  *bytes = plan->arena.bytes;
  return HZ_OK;
}

extern "C" hz_status hz_destroy_plan(hz_plan* plan) {
  if (!plan) return HZ_OK;
  solve_ws_destroy(plan);
  plan->arena.release();
  delete plan;
  return HZ_OK;
}

// The medium's arrays live on the device that was current when it was
// created; every call that launches work on them must run with that device
// current.
hz_status hz::check_device(const hz_medium* med) {
  int dev = 0;
  HZ_CUDA(cudaGetDevice(&dev));
  if (dev != med->device)
    return set_error(HZ_ERR_INVALID_ARG, "the medium lives on device %d but device %d is current",
                     med->device, dev);
  return HZ_OK;
}

extern "C" hz_status hz_apply_operator(hz_plan* plan, const void* x, void* y, int nrhs,
                                       int precision, void* stream) {
  if (!plan || !x || !y) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  if (nrhs < 1 || nrhs > plan->max_nrhs) return set_error(HZ_ERR_INVALID_ARG, "nrhs out of range");
  if (precision != 0 && precision != 1) return set_error(HZ_ERR_INVALID_ARG, "precision must be 0 or 1");
  if (x == y) return set_error(HZ_ERR_INVALID_ARG, "x and y must not alias");
  HZ_TRY(check_device(plan->med));
  const long n = plan->med->n;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double sin = precision == 0 ? 16.0 : 8.0;
  PhaseScope ps(st, PH_STENCIL, double(nrhs) * n * (sin + 32.0 + (plan->med->a ? 8.0 : 0.0)),
                double(nrhs) * n * (plan->med->dim == 3 ? 30.0 : 26.0));
  return launch_stencil(plan->med, precision, x, n, static_cast<double2*>(y), n, nrhs, nullptr, st);
}

extern "C" hz_status hz_apply_preconditioner(hz_plan* plan, const void* x, void* y, int nrhs,
                                             int precision, void* stream) {
  if (!plan || !x || !y) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  if (nrhs < 1 || nrhs > plan->max_nrhs) return set_error(HZ_ERR_INVALID_ARG, "nrhs out of range");
  if (precision != 0 && precision != 1) return set_error(HZ_ERR_INVALID_ARG, "precision must be 0 or 1");
  HZ_TRY(check_device(plan->med));
  return precond_apply(plan, precision, static_cast<const double2*>(x), nullptr, nrhs, y, 1,
                       static_cast<cudaStream_t>(stream), nullptr);
}
