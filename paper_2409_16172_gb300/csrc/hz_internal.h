// Internal definitions shared by the library's translation units.
#pragma once
#include <utility>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hz.h"

#define HZ_MAX_K 64     // symbol planes (node bit masks are 64-bit)
#define HZ_MAX_SEG 72   // interpolation segments incl. the two end entries
#define HZ_MAX_RESTART 128

namespace hz {

hz_status set_error(hz_status st, const char* fmt, ...);
hz_status cuda_error(cudaError_t e, const char* what);

#define HZ_CUDA(call)                                            \
  do {                                                           \
    cudaError_t e_ = (call);                                     \
    if (e_ != cudaSuccess) return ::hz::cuda_error(e_, #call);   \
  } while (0)

#define HZ_TRY(call)                         \
  do {                                       \
    hz_status s_ = (call);                   \
    if (s_ != HZ_OK) return s_;              \
  } while (0)

void* dev_alloc(size_t bytes);
void dev_free(void* p);

// Per-thread stream for the library's own set-up work and stream-ordered
// allocation (server workers set it; elsewhere it is the legacy stream and
// allocation uses cudaMalloc).
cudaStream_t tls_stream();
void set_tls_stream(cudaStream_t st, bool async_alloc);

// RAII list of device allocations owned by a medium or plan.
struct DevArena {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  template <typename T>
  hz_status alloc(T** out, size_t count) {
    size_t b = count * sizeof(T);
    if (b == 0) b = 16;
    void* p = dev_alloc(b);
    if (!p) return set_error(HZ_ERR_OOM, "device allocation of %zu bytes failed", b);
    ptrs.push_back(p);
    bytes += b;
    *out = static_cast<T*>(p);
    return HZ_OK;
  }
  void release() {
    for (void* p : ptrs) dev_free(p);
    ptrs.clear();
    bytes = 0;
  }
};

// Supported axis lengths.
bool fft_size_supported(int N);

// Per-axis tables for one FFT length.
struct AxisTables {
  int N = 0;
  double2* tw64 = nullptr;  // exp(-2 pi i j / N)
  float2* tw32 = nullptr;
  float4* tw32p = nullptr;  // (re, re, im, im) of tw32, for paired lines
  double* xi2_64 = nullptr;  // squared wavenumber per bin
  float* xi2_32 = nullptr;
};

#ifdef __CUDACC__
// Programmatic dependent launch.  Every hot-path kernel starts with
// pdl_wait() (griddepcontrol.wait), which returns once the kernel before it
// on the stream has finished and its writes are visible, and touches no
// global memory before it; launched with launch_pdl, a kernel's launch and
// block scheduling then overlap the tail of the previous kernel (also as
// programmatic edges inside captured graphs).  Without a PDL predecessor the
// wait returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
#endif

#ifdef __CUDACC__
// float -> double by moving the bit fields with integer operations, so that
// the conversion does not occupy the FP64 pipe (the limit of the FP64
// kernels that read complex64 data).
// Exact for normal numbers, zeros, infinities and NaNs; single-precision
// subnormals (|x| < 1.2e-38) are read as signed zeros.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long ed = e == 0u ? 0ull : (e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u));
  const unsigned long long m = e == 0u ? 0ull : (unsigned long long)(u & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(sign | (ed << 52) | m));
}

#endif

}  // namespace hz

struct hz_medium {
  int device = 0;  // CUDA device that holds the medium's arrays (current at create time)
  int dim = 2;
  int nx = 0, ny = 1, nz = 1;
  long n = 0;
  double L = 1.0, omega = 0.0;
  hz_interp interp{};
  // node table
  int K = 0, M = 0, Mt = 0, m_o = -1;
  double c_min = 0, c_max = 0, zeta_max = 0;
  std::vector<double> gamma_re, gamma_im, a_k, c_real, zeta_nodes;
  int nseg = 0;
  std::vector<uchar2> segtab_h;
  // bivariate (c, a) interpolation and the quadratic basis: Ma damping nodes
  // (node k = s * Ma + j), and per-point (node, weight) records instead of
  // the (segment, t) record
  int Ma = 1, basis = 0;
  bool generic = false;
  std::vector<double> a_nodes;
  // device data
  hz::DevArena arena;
  double2* gamma2 = nullptr;        // per point gamma^2 / h_x^2 (Eqn. Complex_wave_speed squared)
  double* a = nullptr;              // per point operator damping (NULL when a == 0)
  double* rec64 = nullptr;          // per point segment + t (complex128 path)
  uint32_t* rec32 = nullptr;        // per point segment:8 | t:24 (complex64 path)
  unsigned long long* rowmask = nullptr;   // per x-row: nodes with a non-zero weight
  unsigned long long* slabmask = nullptr;  // 3D: per z-slab OR of its rows
  uchar4* gnode = nullptr;          // generic: up to 4 nodes per point (0xFF: unused)
  float4* gw32 = nullptr;           // generic: their weights (complex64 path)
  double2* gw64 = nullptr;          // generic: their weights, two double2 per point
  unsigned long long* rowitems = nullptr;  // (row << 8) | k for every set bit of rowmask, row-major
  long nitems = 0;
  uchar2* segtab = nullptr;
  double2* symA64 = nullptr;        // w^2 + i w a_k
  double2* symG64 = nullptr;        // gamma_k^2
  float2* symA32 = nullptr;
  float2* symG32 = nullptr;
  // cubic Hermite (basis 2): per plane 0 for the symbol q_k, 2 c_k for its
  // derivative in c, dq/dc = 2 c |xi|^2 q^2 (NULL when no plane is one)
  std::vector<double> dcoef;
  double* symD64 = nullptr;
  float* symD32 = nullptr;
  hz::AxisTables ax[3];
  double inv_h2[3] = {0, 0, 0};
  // sum over x-rows (3D: also z-slabs) of the number of nodes used there;
  // the symbol planes are only written and read for these (row, k) pairs
  double rowk_used = 0, slabk_used = 0;
};

namespace hz {

// Launchers of the FFT passes for one axis length N (one translation unit per
// N, see fft_inst.cu).  V = float2 (prec 1) or double2 (prec 0).
struct FftOps {
  int N;
  // forward FFT along x, c128 input (optionally scaled per rhs)
  // active (nullable): per-rhs flags; work of retired right-hand sides is skipped
  // zero (nullable): rows of zero_row_bytes bytes (row gr at gr * zero_row_bytes)
  // set to 0 for every row transformed, after its input has been read
  hz_status (*row_fwd)(int prec, const double2* in, const double* scale, long rows_per_rhs,
                       long nrows, const void* tw, void* out, cudaStream_t st, const int* active,
                       void* zero, long zero_row_bytes);
  // inverse FFT along x of the K planes + weighted sum; out_kind 0: c64, 1: c128
  // mode 0: by size, 1: in-place inverse then gather (planes overwritten),
  // 2: fused inverse + weighted sum, 3: one line per (row, node) item of
  // items[0 .. nitems) adding its weighted line into out, which must be zero.
  // gnode (nullable): per-point (node, weight) records gnode / gw (float4 or
  // two double2 per point) replace rec / segtab; mode 3 then scatters and
  // every other mode transforms in place and gathers
  hz_status (*row_inv_acc)(int prec, int out_kind, const void* planes, const void* rec,
                           const uchar2* segtab, int nseg, const unsigned long long* rowmask,
                           int K, long rows_per_rhs, long nrows, long n, double inv_n,
                           const void* tw, void* out, cudaStream_t st, const int* active,
                           int mode, const unsigned long long* items, long nitems,
                           const uchar4* gnode, const void* gw);
  // FFT along a strided axis, in place; sign -1 forward, +1 inverse
  hz_status (*line_pass)(int prec, int sign, void* data, int nx, long outer, long S,
                         long ostride, long bstride, int batch,
                         const unsigned long long* omask, int K, const void* tw,
                         cudaStream_t st, const int* active, int per_rhs);
  // last axis: symbol multiply of the spectrum and inverse FFT, one plane per k
  // (symD, nullable: per plane 0, or 2 c_k for a Hermite derivative plane);
  // tw2 (complex64 only, nullable): the paired twiddle table, selects the
  // two-columns-per-thread kernel when nx is even; pair > 1 halves its blocks
  hz_status (*line_sym_inv)(int prec, const void* vhat, void* planes, int nx, long outer, long S,
                            long ostride, long n, int K, int batch, const void* xi2_x,
                            const void* xi2_o, const void* xi2_l, const void* symA,
                            const void* symG, const void* symD, const unsigned long long* smask,
                            long smO, long smS, const void* tw, const void* tw2, cudaStream_t st,
                            const int* active, int kpb, int pair);
};

const FftOps* fft_ops(int N);

// ---- measurement (profile.cu) ----
enum Phase {
  PH_ROW_FWD = 0, PH_LINE, PH_SYMINV, PH_ROW_INV, PH_STENCIL, PH_DOTS, PH_UPDATE, PH_GIVENS,
  PH_SOLUPD, PH_RESID, PH_NORM, PH_COUNT
};
void count_launches(int k);
bool profiling();
// Per-solve sums of the phases timed while a SolveSink is installed on the
// calling thread (profiling on, launches outside graph capture).
struct SolveSink {
  double ms[PH_COUNT] = {};
  double bytes[PH_COUNT] = {};
};
void set_solve_sink(SolveSink* sink);   // thread-local; nullptr to remove
void resolve_solve_sink(SolveSink* sink);  // waits for and adds this sink's events
// HZ_ERR_INVALID_ARG unless the medium's device is the current one
hz_status check_device(const hz_medium* med);
// Records an event pair around the launches made while it is alive.
struct PhaseScope {
  PhaseScope(cudaStream_t st, Phase ph, double bytes, double flops, int launches = 1);
  ~PhaseScope();
  cudaStream_t st;
  Phase ph;
  double bytes, flops;
  int launches;
  int slot = -1;
  SolveSink* sink = nullptr;
};

}  // namespace hz

namespace hz {
struct SolveWs;

// Launch shapes the autotuner chooses per plan (defaults are the untuned
// choice): blocks per SM of the CGS2 dot and update kernels, basis vectors
// per dot block, and nodes per block of the last-axis symbol pass.
struct Tune {
  int dots_bps = 2;
  int dots_vc = 8;
  int upd_bps = 4;
  int syminv_kpb = 1;
  int rowinv_mode = 0;  // FftOps::row_inv_acc mode (0..3)
  int col_pair = 1;     // complex64 symbol pass: two columns per thread (2: in
                        // half-size blocks)
};
}

namespace hz {
// Sets plan->tune from the autotuner's process cache (no timing); false
// when no entry of the same grid, K, restart and precision exists.
bool tune_from_cache(hz_plan* plan);
}

struct hz_plan {
  hz_medium* med = nullptr;
  hz_solver_opts opts{};
  int max_nrhs = 1;
  hz::DevArena arena;
  // preconditioner workspace
  void* tmp = nullptr;     // working-precision transform of the input [max_nrhs][n]
  void* planes = nullptr;  // [max_nrhs][K][n] in the working precision
  int planes_prec = 1;     // precision the planes buffer is sized for (0 = c128)
  // Krylov workspace (FP64)
  double2* V = nullptr;    // [(m+1)][max_nrhs][n] unnormalised basis vectors
  void* Z = nullptr;       // [m][max_nrhs][n] preconditioned vectors (c64 or unused)
  double2* u = nullptr;    // staged solution for host buffers [max_nrhs][n]
  double2* f = nullptr;    // staged right-hand side for host buffers
  double* partial = nullptr;     // block partial sums
  size_t partial_len = 0;
  hz::SolveWs* ws = nullptr;     // small Krylov state, created by the first solve
  hz::Tune tune;                 // launch shapes (hz_plan_autotune)
};
