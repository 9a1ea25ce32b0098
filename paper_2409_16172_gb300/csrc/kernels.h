// Launchers of the non-FFT kernels (stencil.cu, krylov.cu).
#pragma once
#include <functional>

#include "hz_internal.h"

namespace hz {

// Device-side small Krylov state, one entry per right-hand side b.
struct KsDev {
  int m;            // restart length
  int ldsig;        // leading dimension of sigma ([i][b])
  double tol;
  double2* H;       // [b][j][m+1] rotated Hessenberg columns (R factor)
  double2* S1;      // [b][m+1] first CGS sums
  double2* S2;      // [b][m+1] second CGS sums
  double* sigma;    // [i][b] scale of stored basis vector i
  double* nrm2;     // [b] |w|^2 after the second pass
  double* cs;       // [b][m] rotation cosines
  double2* sn;      // [b][m] rotation sines
  double2* g;       // [b][m+1] rotated right-hand side
  double* est;      // [b] |g_{j+1}|
  double* hist;     // [b][m] est / ||f|| after each step of the cycle
  double2* Hraw;    // [b][j][m+1] Hessenberg columns of the cycle before rotation
  double* bnorm;    // [b] ||f||
  int* jend;        // [b] columns built in this cycle
  int* active;      // [b] 1 while the cycle continues
  int* status;      // [b] hz_status
  int* n_active;    // number of active right-hand sides
};

// Per-plan solve workspace (allocated once, reused by every solve).
struct SolveWs {
  DevArena ar;
  KsDev ks{};
  double* rnorm2 = nullptr;   // [B]
  double2* y = nullptr;       // [B][m]
  int* h_nact = nullptr;      // pinned, 2 slots
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaGraphExec_t cyc_exec = nullptr;  // captured Arnoldi cycle (opts.graphs)
  int cyc_nrhs = 0, cyc_kernels = 0;
  cudaStream_t gstream = nullptr;      // stream the cycle graph is captured on / replayed from
  cudaEvent_t gev[2] = {nullptr, nullptr};
};
hz_status solve_ws_create(hz_plan* p);
void solve_ws_destroy(hz_plan* p);

// Restart-boundary control of a batched solve (continuous batching): each of
// the plan's max_nrhs slots holds one right-hand side that joins at a
// restart boundary and leaves once it has converged or failed; the others
// keep iterating.  Every kernel computes per slot, with launch shapes fixed
// by the slot count, so a slot's iterates do not depend on the other slots.
struct BatchCtl {
  hz_plan* plan = nullptr;
  cudaStream_t st = nullptr;
  long n = 0;
  int B = 0;
  double2* f = nullptr;  // device right-hand sides, slot b at f + b n
  double2* u = nullptr;  // device iterates (zero on admission), slot b at u + b n
  // per-slot state at this boundary
  const int* busy = nullptr;      // 1 while the slot holds a right-hand side
  const int* done = nullptr;      // its iteration has ended (converged or failed)
  const int* conv = nullptr;
  const int* iters = nullptr;
  const int* restarts = nullptr;
  const int* status = nullptr;
  const double* rel = nullptr;    // true relative residual at this boundary
  const double* est = nullptr;    // last Givens estimate / ||f||
  // admit(b): the caller has written f + b n (and zeroed u + b n) on st;
  // computes ||f_b|| and starts the slot.  release(b): frees a done slot.
  std::function<hz_status(int)> admit;
  std::function<void(int)> release;
};
// Runs restarted (F)GMRES over the plan's slots until no slot is live and
// boundary() admits none.  boundary(ctl) is called at every restart
// boundary after the residual check; it returns 1 when it admitted slots
// (their residuals are then computed before the next cycle), 0 when not, or
// -status on an error.  Right / flexible preconditioning only.
hz_status gmres_batch(hz_plan* plan, cudaStream_t st,
                      const std::function<int(BatchCtl&)>& boundary);

int stencil_blocks(long n);
hz_status launch_stencil(const hz_medium* m, int in_prec, const void* x, long in_stride,
                         double2* y, long out_stride, int nrhs, const int* active,
                         cudaStream_t st);
hz_status launch_residual(const hz_medium* m, const double2* u, const double2* f, double2* r,
                          long stride, int nrhs, const int* active, double* partial,
                          cudaStream_t st);

int krylov_blocks(long n, int nrhs, int nchunk);
hz_status launch_dots(const double2* V, long ldb, const double2* w, long wstride, long n, int j,
                      int nrhs, const int* active, double2* partial, const Tune& tn, double2* S,
                      int ldS, cudaStream_t st);
hz_status launch_update(const double2* V, long ldb, double2* w, long wstride, long n, int j,
                        int nrhs, const double2* S, int ldS, const double* sigma, int ldsig,
                        const int* active, bool norm, double* partial, const Tune& tn, double* nrm2,
                        cudaStream_t st);
hz_status launch_givens(const KsDev& ks, int j, int nrhs, cudaStream_t st);
hz_status launch_solution_update(int zprec, const void* Z, long ldb, double2* u, long ustride,
                                 long n, int nrhs, const double2* y, int ldy, const int* jn,
                                 cudaStream_t st);
hz_status launch_combine(const double2* V, long ldb, double2* out, long ostride, long n, int nrhs,
                         const double2* y, int ldy, const double* sigma, int ldsig, const int* jn,
                         cudaStream_t st);
hz_status launch_scale_copy(const double2* V, const double* sigma, double2* out, long n, int nrhs,
                           const int* active, cudaStream_t st);
hz_status launch_axpy(double2* u, const double2* t, long stride, long n, int nrhs, const int* jn,
                      cudaStream_t st);
hz_status launch_norm2(const double2* x, long stride, long n, int nrhs, double* partial, int nblk,
                       double* out, cudaStream_t st);
hz_status launch_reduce_r(const double* partial, int nblk, int nq, double* out, cudaStream_t st);

}  // namespace hz
