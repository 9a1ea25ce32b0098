// Restarted (F)GMRES(m) driver (Section 5, "GMRES implementation"):
//   r = f - P_N u;  v_0 = r / ||r||;  for j < m:
//     z_j = Q_M v_j                          (complex64 or complex128 apply)
//     w   = P_N z_j                          (FP64 stencil)
//     CGS2: h = V^H w, w -= V h; h' = V^H w, w -= V h'; h += h'
//     h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
//     Givens rotation of column j, residual estimate |g_{j+1}|
//   u += Z y (flexible, precision 1) or u += Q_M (V y) (precision 0),
//   then the true FP64 residual decides whether to stop or restart.
// All right-hand sides of a call advance in lock step; each one retires on
// its own device-side flag.  The host waits on the device once per Arnoldi
// step (one step behind the launches) and once per cycle.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <limits>
#include <complex>
#include <vector>

#include "hz_internal.h"
#include "kernels.h"

namespace hz {
hz_status precond_apply(hz_plan* p, int prec, const double2* in, const double* scale, int nrhs,
                        void* out, int out_kind, cudaStream_t st, const int* active);
}

using namespace hz;

namespace {

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace hz {

hz_status solve_ws_create(hz_plan* p) {
  if (p->ws) return HZ_OK;
  SolveWs* w = new SolveWs();
  const int m = p->opts.restart, B = p->max_nrhs;
  KsDev& ks = w->ks;
  ks.m = m;
  ks.ldsig = B;
  ks.tol = p->opts.tol;
  hz_status st = HZ_OK;
  auto A = [&](hz_status s) { if (st == HZ_OK) st = s; };
  A(w->ar.alloc(&ks.H, size_t(B) * m * (m + 1)));
  A(w->ar.alloc(&ks.S1, size_t(B) * (m + 1)));
  A(w->ar.alloc(&ks.S2, size_t(B) * (m + 1)));
  A(w->ar.alloc(&ks.sigma, size_t(B) * (m + 1)));
  A(w->ar.alloc(&ks.nrm2, B));
  A(w->ar.alloc(&ks.cs, size_t(B) * m));
  A(w->ar.alloc(&ks.sn, size_t(B) * m));
  A(w->ar.alloc(&ks.g, size_t(B) * (m + 1)));
  A(w->ar.alloc(&ks.est, B));
  A(w->ar.alloc(&ks.hist, size_t(B) * m));
  A(w->ar.alloc(&ks.Hraw, size_t(B) * m * (m + 1)));
  A(w->ar.alloc(&ks.bnorm, B));
  A(w->ar.alloc(&ks.jend, B));
  A(w->ar.alloc(&ks.active, B));
  A(w->ar.alloc(&ks.status, B));
  A(w->ar.alloc(&ks.n_active, 1));
  A(w->ar.alloc(&w->rnorm2, B));
  A(w->ar.alloc(&w->y, size_t(B) * m));
  if (st == HZ_OK && cudaMallocHost(&w->h_nact, 2 * sizeof(int)) != cudaSuccess)
    st = set_error(HZ_ERR_OOM, "pinned host allocation failed");
  for (auto& e : w->ev)
    if (st == HZ_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      st = set_error(HZ_ERR_CUDA, "event creation failed");
  if (st == HZ_OK && (cudaEventCreate(&w->t0) != cudaSuccess || cudaEventCreate(&w->t1) != cudaSuccess))
    st = set_error(HZ_ERR_CUDA, "event creation failed");
  p->ws = w;
  if (st != HZ_OK) {
    cudaGetLastError();
    solve_ws_destroy(p);
  }
  return st;
}

void solve_ws_destroy(hz_plan* p) {
  SolveWs* w = p->ws;
  if (!w) return;
  w->ar.release();
  if (w->h_nact) cudaFreeHost(w->h_nact);
  for (auto& e : w->ev)
    if (e) cudaEventDestroy(e);
  if (w->t0) cudaEventDestroy(w->t0);
  if (w->t1) cudaEventDestroy(w->t1);
  if (w->cyc_exec) cudaGraphExecDestroy(w->cyc_exec);
  for (auto& e : w->gev)
    if (e) cudaEventDestroy(e);
  if (w->gstream) cudaStreamDestroy(w->gstream);
  delete w;
  p->ws = nullptr;
}

}  // namespace hz

namespace {
hz_status gmres_solve(hz_plan* plan, const void* f_in, void* u_io, int nrhs, hz_solve_stats* stats,
                      double* history, int hlen, void* stream,
                      const std::function<int(BatchCtl&)>* boundary = nullptr) {
  if (!plan || !f_in || !u_io) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  if (nrhs < 1 || nrhs > plan->max_nrhs) return set_error(HZ_ERR_INVALID_ARG, "nrhs out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  hz_plan* p = plan;
  const hz_medium* med = p->med;
  const long n = med->n;
  const int m = p->opts.restart;
  const int B = p->max_nrhs;
  const int prec = p->opts.precision;
  const double tol = p->opts.tol;
  const long ldb = B;  // basis vector i of rhs b at V + (i * B + b) * n

  HZ_TRY(check_device(med));
  HZ_TRY(solve_ws_create(p));
  SolveWs& w = *p->ws;
  // per-solve phase times (only while profiling is on; nothing is timed
  // inside a captured graph)
  SolveSink sink;
  struct SinkGuard {
    SolveSink* s;
    bool on;
    void finish() {
      if (!on) return;
      set_solve_sink(nullptr);
      resolve_solve_sink(s);
      on = false;
    }
    ~SinkGuard() { finish(); }
  } sink_guard{&sink, profiling()};
  if (sink_guard.on) set_solve_sink(&sink);
  KsDev& ks = w.ks;
  (void)tol;
  HZ_CUDA(cudaEventRecord(w.t0, st));

  // stage f and u
  const bool f_dev = is_device_ptr(f_in), u_dev = is_device_ptr(u_io);
  const double2* f = f_dev ? static_cast<const double2*>(f_in) : p->f;
  double2* u = u_dev ? static_cast<double2*>(u_io) : p->u;
  const size_t vbytes = size_t(nrhs) * n * sizeof(double2);
  if (!f_dev) HZ_CUDA(cudaMemcpyAsync(p->f, f_in, vbytes, cudaMemcpyHostToDevice, st));
  if (!u_dev) HZ_CUDA(cudaMemcpyAsync(p->u, u_io, vbytes, cudaMemcpyHostToDevice, st));

  const int nblk_r = stencil_blocks(n);
  const int nblk_n = krylov_blocks(n, nrhs, 1);
  const double Bn = double(nrhs) * n;
  {
    PhaseScope ps(st, PH_NORM, 16.0 * Bn, 4.0 * Bn, 2);
    HZ_TRY(launch_norm2(f, n, n, nrhs, p->partial, nblk_n, ks.bnorm, st));
  }
  std::vector<double> bnorm(nrhs), rn2(nrhs);
  HZ_CUDA(cudaMemcpyAsync(bnorm.data(), ks.bnorm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
  HZ_CUDA(cudaStreamSynchronize(st));
  for (auto& b : bnorm) b = std::sqrt(b);
  const std::vector<double> fnorm = bnorm;  // ||f||
  // The paper's left form (Eqn. MainDiscretePrecond): GMRES on Q_M P_N u =
  // Q_M f; residuals are measured after Q_M, relative to ||Q_M f||.
  const bool left = p->opts.left != 0 && p->opts.no_precond == 0;
  if (left) {
    HZ_TRY(precond_apply(p, prec, f, nullptr, nrhs, p->V, 1, st, nullptr));
    {
      PhaseScope ps(st, PH_NORM, 16.0 * Bn, 4.0 * Bn, 2);
      HZ_TRY(launch_norm2(p->V, n, n, nrhs, p->partial, nblk_n, ks.bnorm, st));
    }
    HZ_CUDA(cudaMemcpyAsync(bnorm.data(), ks.bnorm, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    HZ_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < nrhs; ++b) bnorm[b] = fnorm[b] == 0.0 ? 0.0 : std::sqrt(bnorm[b]);
  }
  HZ_CUDA(cudaMemcpyAsync(ks.bnorm, bnorm.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st));

  std::vector<int> done(nrhs, 0), conv(nrhs, 0), iters(nrhs, 0), restarts(nrhs, 0),
      status(nrhs, HZ_OK);
  std::vector<double> rel(nrhs, 0.0), est(nrhs, 0.0);
  for (int b = 0; b < nrhs; ++b) {
    if (bnorm[b] == 0.0) {  // the solution is zero
      HZ_CUDA(cudaMemsetAsync(u + long(b) * n, 0, n * sizeof(double2), st));
      done[b] = conv[b] = 1;
    }
  }
  std::vector<int> h_active(nrhs), h_jend(nrhs), h_status(nrhs);
  std::vector<double> h_sigma0(B, 0.0);
  std::vector<double2> h_g(size_t(nrhs) * (m + 1)), h_H(size_t(nrhs) * m * (m + 1)), h_y(size_t(B) * m);
  std::vector<double> h_est(nrhs);
  const bool noq = p->opts.no_precond != 0;
  std::vector<double> h_hist(history ? size_t(nrhs) * m : 0);
  std::vector<std::vector<double>> hist_b(history ? nrhs : 0);
  int total_iters = 0;

  // continuous batching: slots join and leave at restart boundaries
  std::vector<int> busy(nrhs, 0);
  BatchCtl ctl;
  if (boundary) {
    ctl.plan = p;
    ctl.st = st;
    ctl.n = n;
    ctl.B = nrhs;
    ctl.f = const_cast<double2*>(f);
    ctl.u = u;
    ctl.busy = busy.data();
    ctl.done = done.data();
    ctl.conv = conv.data();
    ctl.iters = iters.data();
    ctl.restarts = restarts.data();
    ctl.status = status.data();
    ctl.rel = rel.data();
    ctl.est = est.data();
    const int nblk1 = krylov_blocks(n, 1, 1);
    ctl.admit = [&, nblk1](int b) -> hz_status {
      double nb = 0.0;
      HZ_TRY(launch_norm2(f + long(b) * n, n, n, 1, p->partial, nblk1, ks.bnorm + b, st));
      HZ_CUDA(cudaMemcpyAsync(&nb, ks.bnorm + b, sizeof(double), cudaMemcpyDeviceToHost, st));
      HZ_CUDA(cudaStreamSynchronize(st));
      nb = std::sqrt(nb);
      HZ_CUDA(cudaMemcpyAsync(ks.bnorm + b, &nb, sizeof(double), cudaMemcpyHostToDevice, st));
      HZ_CUDA(cudaStreamSynchronize(st));
      bnorm[b] = nb;
      busy[b] = 1;
      done[b] = conv[b] = nb == 0.0 ? 1 : 0;  // a zero right-hand side: u = 0
      iters[b] = restarts[b] = 0;
      status[b] = HZ_OK;
      rel[b] = est[b] = 0.0;
      return HZ_OK;
    };
    ctl.release = [&](int b) {
      busy[b] = 0;
      done[b] = 1;
      bnorm[b] = 0.0;
    };
  }

  for (;;) {
    // true FP64 residual r = f - P u into V_0
    {
      PhaseScope ps(st, PH_RESID, 64.0 * Bn + (med->a ? 8.0 * Bn : 0.0), 30.0 * Bn, 2);
      HZ_TRY(launch_residual(med, u, f, p->V, n, nrhs, nullptr, p->partial, st));
      HZ_TRY(launch_reduce_r(p->partial, nblk_r, nrhs, w.rnorm2, st));
    }
    if (left) {
      // r <- Q_M r in place, and its norm
      HZ_TRY(precond_apply(p, prec, p->V, nullptr, nrhs, p->V, 1, st, nullptr));
      PhaseScope ps(st, PH_NORM, 16.0 * Bn, 4.0 * Bn, 2);
      HZ_TRY(launch_norm2(p->V, n, n, nrhs, p->partial, nblk_n, w.rnorm2, st));
    }
    HZ_CUDA(cudaMemcpyAsync(rn2.data(), w.rnorm2, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    HZ_CUDA(cudaStreamSynchronize(st));
    int live = 0;
    for (int b = 0; b < nrhs; ++b) {
      if (bnorm[b] == 0.0) continue;
      rel[b] = std::sqrt(rn2[b]) / bnorm[b];
      if (done[b]) continue;
      if (!std::isfinite(rel[b])) {
        done[b] = 1;
        status[b] = HZ_ERR_BREAKDOWN;
      } else if (rel[b] <= tol) {
        done[b] = conv[b] = 1;
      } else if (iters[b] >= p->opts.maxit) {
        done[b] = 1;
        status[b] = HZ_ERR_NOT_CONVERGED;
      }
      live += !done[b];
    }
    if (boundary) {
      const int a = (*boundary)(ctl);
      if (a < 0) return hz_status(-a);
      if (a > 0) continue;  // residuals of the admitted slots first
    }
    if (!live) break;

    // start a cycle for the live right-hand sides
    std::fill(h_g.begin(), h_g.end(), make_double2(0.0, 0.0));
    for (int b = 0; b < nrhs; ++b) {
      h_active[b] = !done[b];
      const double r = std::sqrt(rn2[b]);
      h_sigma0[b] = (!done[b] && r > 0) ? 1.0 / r : 0.0;
      h_g[size_t(b) * (m + 1)] = make_double2(done[b] ? 0.0 : r, 0.0);
      h_status[b] = HZ_OK;
    }
    HZ_CUDA(cudaMemcpyAsync(ks.active, h_active.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
    HZ_CUDA(cudaMemcpyAsync(ks.status, h_status.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
    HZ_CUDA(cudaMemcpyAsync(ks.sigma, h_sigma0.data(), B * sizeof(double), cudaMemcpyHostToDevice, st));
    HZ_CUDA(cudaMemcpyAsync(ks.g, h_g.data(), h_g.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    HZ_CUDA(cudaMemsetAsync(ks.jend, 0, nrhs * sizeof(int), st));
    HZ_CUDA(cudaMemcpyAsync(ks.n_active, &live, sizeof(int), cudaMemcpyHostToDevice, st));
    HZ_CUDA(cudaStreamSynchronize(st));  // host vectors above are reused next cycle

    int maxit_left = 0;
    for (int b = 0; b < nrhs; ++b)
      if (!done[b]) maxit_left = std::max(maxit_left, p->opts.maxit - iters[b]);
    const int jmax = std::min(m, maxit_left);
    // one Arnoldi step for every live right-hand side (no host interaction)
    auto step = [&](int j, cudaStream_t st) -> hz_status {
      const double2* Vj = p->V + long(j) * ldb * n;
      double2* Vn = p->V + long(j + 1) * ldb * n;
      const double* sig_j = ks.sigma + long(j) * B;
      const double stb = Bn * ((prec == 1 ? 8.0 : 16.0) + 32.0 + (med->a ? 8.0 : 0.0));
      const double stf = Bn * (med->dim == 3 ? 30.0 : 26.0);
      if (noq) {
        // unpreconditioned: w = P_N (sigma_j V_j)
        double2* zt = static_cast<double2*>(p->Z);
        {
          PhaseScope ps(st, PH_SOLUPD, 32.0 * Bn, 2.0 * Bn);
          HZ_TRY(launch_scale_copy(Vj, sig_j, zt, n, nrhs, ks.active, st));
        }
        PhaseScope ps(st, PH_STENCIL, stb, stf);
        HZ_TRY(launch_stencil(med, 0, zt, n, Vn, n, nrhs, ks.active, st));
      } else if (left) {
        // left: v_{j+1} = Q_M (P_N (sigma_j V_j)); the FP64 stencil writes
        // P_N V_j, the preconditioner scales it by sigma_j and works in place
        {
          PhaseScope ps(st, PH_STENCIL, Bn * (16.0 + 32.0 + (med->a ? 8.0 : 0.0)), stf);
          HZ_TRY(launch_stencil(med, 0, Vj, n, Vn, n, nrhs, ks.active, st));
        }
        HZ_TRY(precond_apply(p, prec, Vn, sig_j, nrhs, Vn, 1, st, ks.active));
      } else if (prec == 1) {
        float2* Zj = static_cast<float2*>(p->Z) + long(j) * ldb * n;
        HZ_TRY(precond_apply(p, 1, Vj, sig_j, nrhs, Zj, 0, st, ks.active));
        PhaseScope ps(st, PH_STENCIL, stb, stf);
        HZ_TRY(launch_stencil(med, 1, Zj, n, Vn, n, nrhs, ks.active, st));
      } else {
        double2* zt = static_cast<double2*>(p->Z);
        HZ_TRY(precond_apply(p, 0, Vj, sig_j, nrhs, zt, 1, st, ks.active));
        PhaseScope ps(st, PH_STENCIL, stb, stf);
        HZ_TRY(launch_stencil(med, 0, zt, n, Vn, n, nrhs, ks.active, st));
      }
      // CGS2: two passes of classical Gram-Schmidt against v_0 .. v_j
      const double db = 16.0 * Bn * (j + 2), ub = 16.0 * Bn * (j + 3), fl = 8.0 * Bn * (j + 1);
      for (int pass = 0; pass < 2; ++pass) {
        double2* S = pass == 0 ? ks.S1 : ks.S2;
        {
          PhaseScope ps(st, PH_DOTS, db, fl, 2);
          HZ_TRY(launch_dots(p->V, ldb, Vn, n, n, j, nrhs, ks.active,
                             reinterpret_cast<double2*>(p->partial), p->tune, S, m + 1, st));
        }
        PhaseScope ps(st, PH_UPDATE, ub, fl + (pass ? 4.0 * Bn : 0.0), pass ? 2 : 1);
        HZ_TRY(launch_update(p->V, ldb, Vn, n, n, j, nrhs, S, m + 1, ks.sigma, B, ks.active, pass == 1,
                             p->partial, p->tune, ks.nrm2, st));
      }
      PhaseScope ps(st, PH_GIVENS, 0.0, 0.0);
      HZ_TRY(launch_givens(ks, j, nrhs, st));
      return HZ_OK;
    };
    if (p->opts.graphs && jmax == m && !history) {
      // The whole cycle as one CUDA graph, captured once per plan and right-
      // hand-side count and replayed; steps after a right-hand side retires
      // return at once on its device-side flag.
      // captured on and replayed from the plan's own stream (the legacy
      // default stream cannot be captured), ordered after / before st
      if (!w.gstream) HZ_CUDA(cudaStreamCreateWithFlags(&w.gstream, cudaStreamNonBlocking));
      if (!w.gev[0]) {
        HZ_CUDA(cudaEventCreateWithFlags(&w.gev[0], cudaEventDisableTiming));
        HZ_CUDA(cudaEventCreateWithFlags(&w.gev[1], cudaEventDisableTiming));
      }
      if (!w.cyc_exec || w.cyc_nrhs != nrhs) {
        if (w.cyc_exec) cudaGraphExecDestroy(w.cyc_exec);
        w.cyc_exec = nullptr;
        const unsigned long long l0 = hz_launch_count();
        HZ_CUDA(cudaStreamBeginCapture(w.gstream, cudaStreamCaptureModeThreadLocal));
        hz_status cst = HZ_OK;
        for (int j = 0; j < m && cst == HZ_OK; ++j) cst = step(j, w.gstream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(w.gstream, &graph);
        const unsigned long long captured = hz_launch_count() - l0;
        count_launches(-int(captured));  // recorded, not run
        if (cst != HZ_OK) {
          if (graph) cudaGraphDestroy(graph);
          return cst;
        }
        HZ_CUDA(ce);
        const cudaError_t ie = cudaGraphInstantiate(&w.cyc_exec, graph, 0);
        cudaGraphDestroy(graph);
        HZ_CUDA(ie);
        w.cyc_nrhs = nrhs;
        w.cyc_kernels = int(captured);
      }
      HZ_CUDA(cudaEventRecord(w.gev[0], st));
      HZ_CUDA(cudaStreamWaitEvent(w.gstream, w.gev[0], 0));
      HZ_CUDA(cudaGraphLaunch(w.cyc_exec, w.gstream));
      HZ_CUDA(cudaEventRecord(w.gev[1], w.gstream));
      HZ_CUDA(cudaStreamWaitEvent(st, w.gev[1], 0));
      count_launches(w.cyc_kernels);
    } else {
      for (int j = 0; j < jmax; ++j) {
        HZ_TRY(step(j, st));
        HZ_CUDA(cudaMemcpyAsync(&w.h_nact[j & 1], ks.n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        HZ_CUDA(cudaEventRecord(w.ev[j & 1], st));
        if (j >= 1) {
          HZ_CUDA(cudaEventSynchronize(w.ev[(j - 1) & 1]));
          if (w.h_nact[(j - 1) & 1] == 0) break;
        }
      }
    }
    HZ_CUDA(cudaMemcpyAsync(h_jend.data(), ks.jend, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
    HZ_CUDA(cudaMemcpyAsync(h_status.data(), ks.status, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
    HZ_CUDA(cudaMemcpyAsync(h_est.data(), ks.est, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    HZ_CUDA(cudaMemcpyAsync(h_H.data(), ks.H, h_H.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
    HZ_CUDA(cudaMemcpyAsync(h_g.data(), ks.g, h_g.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
    if (history)
      HZ_CUDA(cudaMemcpyAsync(h_hist.data(), ks.hist, h_hist.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, st));
    HZ_CUDA(cudaStreamSynchronize(st));

    // back substitution R y = g on the host (m <= 128)
    std::fill(h_y.begin(), h_y.end(), make_double2(0.0, 0.0));
    std::vector<int> jn(nrhs, 0);
    for (int b = 0; b < nrhs; ++b) {
      if (done[b]) continue;
      const int J = h_jend[b];
      jn[b] = J;
      iters[b] += J;
      if (history)
        for (int i = 0; i < J; ++i) hist_b[b].push_back(h_hist[size_t(b) * m + i]);
      restarts[b] += 1;
      est[b] = h_est[b] / bnorm[b];
      if (h_status[b] != HZ_OK) {
        status[b] = h_status[b];
        done[b] = 1;
        jn[b] = 0;
        continue;
      }
      std::vector<std::complex<double>> yy(J);
      auto Hc = [&](int i, int jj) {
        const double2 v = h_H[(size_t(b) * m + jj) * (m + 1) + i];
        return std::complex<double>(v.x, v.y);
      };
      for (int i = J - 1; i >= 0; --i) {
        std::complex<double> s(h_g[size_t(b) * (m + 1) + i].x, h_g[size_t(b) * (m + 1) + i].y);
        for (int k = i + 1; k < J; ++k) s -= Hc(i, k) * yy[k];
        yy[i] = s / Hc(i, i);
      }
      for (int i = 0; i < J; ++i) h_y[size_t(b) * m + i] = make_double2(yy[i].real(), yy[i].imag());
    }
    total_iters += *std::max_element(jn.begin(), jn.end());
    int* d_jn = ks.jend;  // reuse: per-rhs number of columns to add (0 = skip)
    HZ_CUDA(cudaMemcpyAsync(d_jn, jn.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
    HZ_CUDA(cudaMemcpyAsync(w.y, h_y.data(), size_t(nrhs) * m * sizeof(double2), cudaMemcpyHostToDevice, st));
    const int Jmax = *std::max_element(jn.begin(), jn.end());
    if (prec == 1 && !noq && !left) {
      PhaseScope ps(st, PH_SOLUPD, Bn * (8.0 * Jmax + 32.0), Bn * 8.0 * Jmax);
      HZ_TRY(launch_solution_update(1, p->Z, ldb, u, n, n, nrhs, w.y, m, d_jn, st));
    } else if (noq || left) {
      // u += V (sigma y)
      double2* t = p->V + long(m) * ldb * n;
      PhaseScope ps(st, PH_SOLUPD, Bn * (16.0 * Jmax + 64.0), Bn * (8.0 * Jmax + 2.0));
      HZ_TRY(launch_combine(p->V, ldb, t, n, n, nrhs, w.y, m, ks.sigma, B, d_jn, st));
      HZ_TRY(launch_axpy(u, t, n, n, nrhs, d_jn, st));
    } else {
      // t = V (sigma y), then u += Q_M t in complex128
      double2* t = p->V + long(m) * ldb * n;  // V_m is free once the cycle is over
      {
        PhaseScope ps(st, PH_SOLUPD, Bn * (16.0 * Jmax + 16.0), Bn * 8.0 * Jmax);
        HZ_TRY(launch_combine(p->V, ldb, t, n, n, nrhs, w.y, m, ks.sigma, B, d_jn, st));
      }
      double2* zt = static_cast<double2*>(p->Z);
      HZ_TRY(precond_apply(p, 0, t, nullptr, nrhs, zt, 1, st, nullptr));
      PhaseScope ps(st, PH_SOLUPD, Bn * 48.0, Bn * 2.0);
      HZ_TRY(launch_axpy(u, zt, n, n, nrhs, d_jn, st));
    }
    HZ_CUDA(cudaStreamSynchronize(st));
  }
  if (boundary) return HZ_OK;  // each slot was reported at the boundary it finished

  // the left form stopped on the preconditioned residual; report the true one
  std::vector<double> rel_true = rel;
  if (left) {
    {
      PhaseScope ps(st, PH_RESID, 64.0 * Bn + (med->a ? 8.0 * Bn : 0.0), 30.0 * Bn, 2);
      HZ_TRY(launch_residual(med, u, f, p->V, n, nrhs, nullptr, p->partial, st));
      HZ_TRY(launch_reduce_r(p->partial, nblk_r, nrhs, w.rnorm2, st));
    }
    HZ_CUDA(cudaMemcpyAsync(rn2.data(), w.rnorm2, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    HZ_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < nrhs; ++b) rel_true[b] = fnorm[b] == 0.0 ? 0.0 : std::sqrt(rn2[b]) / fnorm[b];
  }
  if (!u_dev) HZ_CUDA(cudaMemcpyAsync(u_io, p->u, vbytes, cudaMemcpyDeviceToHost, st));
  HZ_CUDA(cudaEventRecord(w.t1, st));
  HZ_CUDA(cudaEventSynchronize(w.t1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, w.t0, w.t1);
  sink_guard.finish();
  const float ms_pre = float(sink.ms[PH_ROW_FWD] + sink.ms[PH_LINE] + sink.ms[PH_SYMINV] +
                             sink.ms[PH_ROW_INV]);
  const float ms_op = float(sink.ms[PH_STENCIL] + sink.ms[PH_RESID]);
  const float ms_arn = float(sink.ms[PH_DOTS] + sink.ms[PH_UPDATE] + sink.ms[PH_GIVENS] +
                             sink.ms[PH_NORM] + sink.ms[PH_SOLUPD]);
  const double pre_bytes = sink.bytes[PH_ROW_FWD] + sink.bytes[PH_LINE] + sink.bytes[PH_SYMINV] +
                           sink.bytes[PH_ROW_INV];
  hz_status ret = HZ_OK;
  for (int b = 0; b < nrhs; ++b) {
    if (stats) {
      stats[b].iters = iters[b];
      stats[b].restarts = restarts[b];
      stats[b].status = conv[b] ? HZ_OK : (status[b] == HZ_OK ? HZ_ERR_NOT_CONVERGED : status[b]);
      stats[b].converged = conv[b];
      stats[b].rel_true_resid = rel_true[b];
      stats[b].rel_est_resid = est[b];
      stats[b].ms_total = ms;
      stats[b].ms_precond = ms_pre;
      stats[b].ms_stencil = ms_op;
      stats[b].ms_arnoldi = ms_arn;
      stats[b].model_bytes_precond = pre_bytes;
    }
    if (!conv[b]) {
      const hz_status sb = status[b] == HZ_OK ? HZ_ERR_NOT_CONVERGED : hz_status(status[b]);
      if (ret == HZ_OK || sb == HZ_ERR_BREAKDOWN) ret = sb;
    }
  }
  (void)total_iters;
  if (history) {
    for (int b = 0; b < nrhs; ++b)
      for (int s = 0; s < hlen; ++s)
        history[size_t(b) * hlen + s] =
            s < int(hist_b[b].size()) ? hist_b[b][s] : std::numeric_limits<double>::quiet_NaN();
  }
  if (ret != HZ_OK) set_error(ret, "%s", ret == HZ_ERR_BREAKDOWN ? "Krylov breakdown (NaN/Inf)" : "not converged within maxit");
  return ret;
}
}  // namespace

hz_status hz::gmres_batch(hz_plan* plan, cudaStream_t st,
                          const std::function<int(BatchCtl&)>& boundary) {
  if (!plan) return set_error(HZ_ERR_INVALID_ARG, "null plan");
  if (plan->opts.left) return set_error(HZ_ERR_INVALID_ARG, "batched solves are right-preconditioned");
  const size_t vb = size_t(plan->max_nrhs) * plan->med->n * sizeof(double2);
  // every slot starts free, with a zero right-hand side and iterate
  HZ_CUDA(cudaMemsetAsync(plan->f, 0, vb, st));
  HZ_CUDA(cudaMemsetAsync(plan->u, 0, vb, st));
  return gmres_solve(plan, plan->f, plan->u, plan->max_nrhs, nullptr, nullptr, 0, st, &boundary);
}

extern "C" hz_status hz_gmres_solve(hz_plan* plan, const void* f_in, void* u_io, int nrhs,
                                    hz_solve_stats* stats, void* stream) {
  return gmres_solve(plan, f_in, u_io, nrhs, stats, nullptr, 0, stream);
}

extern "C" hz_status hz_plan_hessenberg(const hz_plan* plan, int rhs, void* H, int* cols) {
  if (!plan || !H || !cols) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  if (!plan->ws) return set_error(HZ_ERR_INVALID_ARG, "no solve has run on this plan");
  if (rhs < 0 || rhs >= plan->max_nrhs) return set_error(HZ_ERR_INVALID_ARG, "rhs out of range");
  const int m = plan->opts.restart;
  const KsDev& ks = plan->ws->ks;
  int J = 0;
  HZ_CUDA(cudaMemcpy(&J, ks.jend + rhs, sizeof(int), cudaMemcpyDeviceToHost));
  J = std::max(0, std::min(J, m));
  *cols = J;
  if (J > 0) {
    HZ_CUDA(cudaMemcpy(H, ks.Hraw + long(rhs) * m * (m + 1), size_t(J) * (m + 1) * sizeof(double2),
                       cudaMemcpyDeviceToHost));
    // below the subdiagonal: zero (those entries are never written)
    double2* h = static_cast<double2*>(H);
    for (int j = 0; j < J; ++j)
      for (int i = j + 2; i <= m; ++i) h[size_t(j) * (m + 1) + i] = make_double2(0.0, 0.0);
  }
  return HZ_OK;
}

extern "C" hz_status hz_gmres_solve_history(hz_plan* plan, const void* f_in, void* u_io, int nrhs,
                                            hz_solve_stats* stats, double* history,
                                            int history_len, void* stream) {
  if (!history || history_len < 1) return set_error(HZ_ERR_INVALID_ARG, "history buffer required");
  return gmres_solve(plan, f_in, u_io, nrhs, stats, history, history_len, stream);
}
