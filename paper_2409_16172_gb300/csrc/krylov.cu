// FP64 Krylov kernels of restarted (F)GMRES (Section 5, "GMRES
// implementation"): CGS2 Arnoldi (classical Gram-Schmidt applied twice),
// complex Givens rotations on the Hessenberg column, the solution update and
// the deterministic reductions they need.
//
// The basis is stored unnormalised: the true basis vector is
// v_i = sigma_i * V_i, sigma_i = 1 / ||w_i||.  Then
//   h_i   = <v_i, w> = sigma_i * sum conj(V_i) w          (dots)
//   w    -= sum_i h_i v_i = sum_i (sigma_i h_i) V_i         (update)
// so no pass ever rescales a stored vector.
// Layout: V[(i * ldb + b) * n + p] for basis vector i, right-hand side b.
#include <math.h>

#include "hz_internal.h"
#include "kernels.h"

namespace hz {
namespace {

constexpr int KT = 256;   // threads per block
constexpr int VC = 8;     // basis vectors per dots block

// fixed-order block sum of NV doubles per thread; result in sh[0..NV-1]
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh) {
#pragma unroll
  for (int c = 0; c < NV; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < NV; ++c) sh[warp * NV + c] = v[c];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < KT / 32; ++w) s += sh[w * NV + threadIdx.x];
    sh[KT / 32 * NV + threadIdx.x] = s;
  }
  __syncthreads();
}

// S[b][i] partials: raw sums sum_p conj(V_i[p]) w[p] for i in [i0, i0 + VC),
// i <= j.  grid = (nblk, nrhs, nchunk).  partial layout
// [(b * (j+1) + i) * nblk + blk] as double2.
__global__ void __launch_bounds__(KT)
dots_kernel(const double2* __restrict__ V, long ldb, const double2* __restrict__ w, long wstride,
            long n, int j, const int* __restrict__ active, double2* __restrict__ partial) {
  const int b = blockIdx.y;
  const int i0 = blockIdx.z * VC;
  const int nv = min(VC, j + 1 - i0);
  double acc[2 * VC];
#pragma unroll
  for (int c = 0; c < 2 * VC; ++c) acc[c] = 0.0;
  const bool on = active[b] != 0;
  if (on) {
    const double2* wb = w + b * wstride;
    for (long p = long(blockIdx.x) * KT + threadIdx.x; p < n; p += long(gridDim.x) * KT) {
      const double2 x = wb[p];
#pragma unroll
      for (int c = 0; c < VC; ++c) {
        if (c < nv) {
          const double2 v = V[(long(i0 + c) * ldb + b) * n + p];
          acc[2 * c] = fma(v.x, x.x, fma(v.y, x.y, acc[2 * c]));
          acc[2 * c + 1] = fma(v.x, x.y, fma(-v.y, x.x, acc[2 * c + 1]));
        }
      }
    }
  }
  __shared__ double sh[(KT / 32 + 1) * 2 * VC];
  block_sum<2 * VC>(acc, sh);
  if (threadIdx.x < nv) {
    const double* r = sh + (KT / 32) * 2 * VC;
    partial[(long(b) * (j + 1) + i0 + threadIdx.x) * gridDim.x + blockIdx.x] =
        make_double2(r[2 * threadIdx.x], r[2 * threadIdx.x + 1]);
  }
}

// Sum partials in a fixed order: q = b * jp1 + i,
// out[b * ldo + i] = sum_blk part[q * nblk + blk].
__global__ void __launch_bounds__(KT)
reduce_c_kernel(const double2* __restrict__ part, int nblk, int jp1, int ldo,
                double2* __restrict__ out) {
  const long q = blockIdx.x;
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < nblk; i += KT) {
    const double2 p = part[q * nblk + i];
    v[0] += p.x;
    v[1] += p.y;
  }
  __shared__ double sh[(KT / 32 + 1) * 2];
  block_sum<2>(v, sh);
  if (threadIdx.x == 0)
    out[(q / jp1) * ldo + q % jp1] = make_double2(sh[(KT / 32) * 2], sh[(KT / 32) * 2 + 1]);
}

__global__ void __launch_bounds__(KT)
reduce_r_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  const long q = blockIdx.x;
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < nblk; i += KT) v[0] += part[q * nblk + i];
  __shared__ double sh[(KT / 32 + 1)];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) out[q] = sh[KT / 32];
}

// w -= sum_{i <= j} sigma_i^2 S[b][i] V_i, optionally |w|^2 partials.
template <bool NORM>
__global__ void __launch_bounds__(KT)
update_kernel(const double2* __restrict__ V, long ldb, double2* __restrict__ w, long wstride,
              long n, int j, const double2* __restrict__ S, int ldS, const double* __restrict__ sigma,
              int ldsig, const int* __restrict__ active, double* __restrict__ partial) {
  const int b = blockIdx.y;
  __shared__ double2 coef[HZ_MAX_RESTART + 1];
  const bool on = active[b] != 0;
  if (on) {
    for (int i = threadIdx.x; i <= j; i += KT) {
      const double s = sigma[long(i) * ldsig + b];
      const double2 h = S[long(b) * ldS + i];
      coef[i] = make_double2(s * s * h.x, s * s * h.y);
    }
  }
  __syncthreads();
  double nrm[1] = {0.0};
  if (on) {
    double2* wb = w + b * wstride;
    for (long p = long(blockIdx.x) * KT + threadIdx.x; p < n; p += long(gridDim.x) * KT) {
      double2 x = wb[p];
      for (int i = 0; i <= j; ++i) {
        const double2 v = V[(long(i) * ldb + b) * n + p];
        const double2 c = coef[i];
        x.x = fma(-c.x, v.x, fma(c.y, v.y, x.x));
        x.y = fma(-c.x, v.y, fma(-c.y, v.x, x.y));
      }
      wb[p] = x;
      if (NORM) nrm[0] = fma(x.x, x.x, fma(x.y, x.y, nrm[0]));
    }
  }
  if (NORM) {
    __shared__ double sh[KT / 32 + 1];
    block_sum<1>(nrm, sh);
    if (threadIdx.x == 0) partial[long(b) * gridDim.x + blockIdx.x] = sh[KT / 32];
  }
}

__device__ __forceinline__ double2 cmul_d(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conj_d(double2 a) { return make_double2(a.x, -a.y); }

// One thread per right-hand side: form column j of the Hessenberg matrix,
// apply the earlier rotations, build the new one (c real, G [a;b] = [r;0]),
// update g and the residual estimate, and retire converged / broken rows.
__global__ void givens_kernel(KsDev ks, int j, int nrhs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nrhs || !ks.active[b]) return;
  const int m = ks.m;
  double2* col = ks.H + (long(b) * m + j) * (m + 1);
  const double2* S1 = ks.S1 + long(b) * (m + 1);
  const double2* S2 = ks.S2 + long(b) * (m + 1);
  bool bad = false;
  double hmax = 0.0;
  for (int i = 0; i <= j; ++i) {
    const double s = ks.sigma[long(i) * ks.ldsig + b];
    col[i] = make_double2(s * (S1[i].x + S2[i].x), s * (S1[i].y + S2[i].y));
    hmax = fmax(hmax, hypot(col[i].x, col[i].y));
    bad |= !isfinite(col[i].x) || !isfinite(col[i].y);
  }
  const double hn = sqrt(ks.nrm2[b]);
  bad |= !isfinite(hn);
  col[j + 1] = make_double2(hn, 0.0);
  const bool happy = hn <= 1e-14 * hmax;
  ks.sigma[long(j + 1) * ks.ldsig + b] = (hn > 0.0 && !happy) ? 1.0 / hn : 0.0;
  double* cs = ks.cs + long(b) * m;
  double2* sn = ks.sn + long(b) * m;
  double2* g = ks.g + long(b) * (m + 1);
  for (int i = 0; i < j; ++i) {
    const double2 t = make_double2(cs[i] * col[i].x, cs[i] * col[i].y);
    const double2 u = cmul_d(sn[i], col[i + 1]);
    const double2 lo = cmul_d(conj_d(sn[i]), col[i]);
    col[i + 1] = make_double2(cs[i] * col[i + 1].x - lo.x, cs[i] * col[i + 1].y - lo.y);
    col[i] = make_double2(t.x + u.x, t.y + u.y);
  }
  const double2 a = col[j];
  const double aa = hypot(a.x, a.y);
  double c;
  double2 s, r;
  if (hn == 0.0) {
    c = 1.0; s = make_double2(0.0, 0.0); r = a;
  } else if (aa == 0.0) {
    c = 0.0; s = make_double2(1.0, 0.0); r = make_double2(hn, 0.0);
  } else {
    const double rho = hypot(aa, hn);
    c = aa / rho;
    const double2 ph = make_double2(a.x / aa, a.y / aa);
    s = make_double2(ph.x * hn / rho, ph.y * hn / rho);   // ph * conj(hn) / rho, hn real
    r = make_double2(ph.x * rho, ph.y * rho);
  }
  cs[j] = c;
  sn[j] = s;
  col[j] = r;
  col[j + 1] = make_double2(0.0, 0.0);
  const double2 gj = g[j];
  g[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));  // -conj(s) g_j
  g[j] = make_double2(c * gj.x, c * gj.y);
  const double est = hypot(g[j + 1].x, g[j + 1].y);
  ks.est[b] = est;
  ks.jend[b] = j + 1;
  bad |= !isfinite(est) || !isfinite(r.x) || !isfinite(r.y);
  if (bad) {
    ks.status[b] = HZ_ERR_BREAKDOWN;
    ks.active[b] = 0;
  } else if (est <= ks.tol * ks.bnorm[b] || happy) {
    ks.active[b] = 0;
  }
  if (!ks.active[b]) atomicSub(ks.n_active, 1);
}

// u += sum_{i < jn} y[b][i] Z_i  (Z in c64 or c128), one pass.
template <typename ZT>
__global__ void __launch_bounds__(KT)
solution_update_kernel(const ZT* __restrict__ Z, long ldb, double2* __restrict__ u, long ustride,
                       long n, const double2* __restrict__ y, int ldy, const int* __restrict__ jn) {
  const int b = blockIdx.y;
  const int J = jn[b];
  if (J <= 0) return;
  __shared__ double2 ys[HZ_MAX_RESTART];
  for (int i = threadIdx.x; i < J; i += KT) ys[i] = y[long(b) * ldy + i];
  __syncthreads();
  double2* ub = u + b * ustride;
  for (long p = long(blockIdx.x) * KT + threadIdx.x; p < n; p += long(gridDim.x) * KT) {
    double2 x = ub[p];
    for (int i = 0; i < J; ++i) {
      const ZT zv = Z[(long(i) * ldb + b) * n + p];
      const double zr = double(zv.x), zi = double(zv.y);
      const double2 c = ys[i];
      x.x = fma(c.x, zr, fma(-c.y, zi, x.x));
      x.y = fma(c.x, zi, fma(c.y, zr, x.y));
    }
    ub[p] = x;
  }
}

// out[b] = sum_{i < J} (sigma_i y_i) V_i  (FP64 path: the combination that is
// then preconditioned).
__global__ void __launch_bounds__(KT)
combine_kernel(const double2* __restrict__ V, long ldb, double2* __restrict__ out, long ostride,
               long n, const double2* __restrict__ y, int ldy, const double* __restrict__ sigma,
               int ldsig, const int* __restrict__ jn) {
  const int b = blockIdx.y;
  const int J = jn[b];
  __shared__ double2 ys[HZ_MAX_RESTART];
  for (int i = threadIdx.x; i < J; i += KT) {
    const double s = sigma[long(i) * ldsig + b];
    const double2 yy = y[long(b) * ldy + i];
    ys[i] = make_double2(s * yy.x, s * yy.y);
  }
  __syncthreads();
  double2* ob = out + b * ostride;
  for (long p = long(blockIdx.x) * KT + threadIdx.x; p < n; p += long(gridDim.x) * KT) {
    double2 x = make_double2(0.0, 0.0);
    for (int i = 0; i < J; ++i) {
      const double2 v = V[(long(i) * ldb + b) * n + p];
      const double2 c = ys[i];
      x.x = fma(c.x, v.x, fma(-c.y, v.y, x.x));
      x.y = fma(c.x, v.y, fma(c.y, v.x, x.y));
    }
    ob[p] = x;
  }
}

// u += t (element-wise, FP64), for active right-hand sides with jn > 0
__global__ void axpy_kernel(double2* __restrict__ u, const double2* __restrict__ t, long stride,
                            long n, const int* __restrict__ jn) {
  const int b = blockIdx.y;
  if (jn[b] <= 0) return;
  for (long p = long(blockIdx.x) * KT + threadIdx.x; p < n; p += long(gridDim.x) * KT) {
    const double2 a = u[b * stride + p], c = t[b * stride + p];
    u[b * stride + p] = make_double2(a.x + c.x, a.y + c.y);
  }
}

// |x|^2 partials of nrhs vectors
__global__ void __launch_bounds__(KT)
norm2_kernel(const double2* __restrict__ x, long stride, long n, double* __restrict__ partial) {
  const int b = blockIdx.y;
  double v[1] = {0.0};
  for (long p = long(blockIdx.x) * KT + threadIdx.x; p < n; p += long(gridDim.x) * KT) {
    const double2 a = x[b * stride + p];
    v[0] = fma(a.x, a.x, fma(a.y, a.y, v[0]));
  }
  __shared__ double sh[KT / 32 + 1];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) partial[long(b) * gridDim.x + blockIdx.x] = sh[KT / 32];
}

}  // namespace

int krylov_blocks(long n, int nrhs, int nchunk) {
  // aim at ~4 blocks per SM over the whole launch, >= 4 points per thread
  long per = (4L * 152 + long(nrhs) * nchunk - 1) / (long(nrhs) * nchunk);
  long maxb = (n + 4L * KT - 1) / (4L * KT);
  if (per > maxb) per = maxb;
  if (per < 1) per = 1;
  return int(per);
}

hz_status launch_dots(const double2* V, long ldb, const double2* w, long wstride, long n, int j,
                      int nrhs, const int* active, double2* partial, int nblk, double2* S, int ldS,
                      cudaStream_t st) {
  const int nchunk = (j + 1 + VC - 1) / VC;
  dots_kernel<<<dim3(nblk, nrhs, nchunk), KT, 0, st>>>(V, ldb, w, wstride, n, j, active, partial);
  reduce_c_kernel<<<unsigned(nrhs * (j + 1)), KT, 0, st>>>(partial, nblk, j + 1, ldS, S);
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_update(const double2* V, long ldb, double2* w, long wstride, long n, int j,
                        int nrhs, const double2* S, int ldS, const double* sigma, int ldsig,
                        const int* active, bool norm, double* partial, int nblk, double* nrm2,
                        cudaStream_t st) {
  if (norm) {
    update_kernel<true><<<dim3(nblk, nrhs), KT, 0, st>>>(V, ldb, w, wstride, n, j, S, ldS, sigma,
                                                          ldsig, active, partial);
    reduce_r_kernel<<<unsigned(nrhs), KT, 0, st>>>(partial, nblk, nrm2);
  } else {
    update_kernel<false><<<dim3(nblk, nrhs), KT, 0, st>>>(V, ldb, w, wstride, n, j, S, ldS, sigma,
                                                           ldsig, active, nullptr);
  }
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_givens(const KsDev& ks, int j, int nrhs, cudaStream_t st) {
  givens_kernel<<<(nrhs + 63) / 64, 64, 0, st>>>(ks, j, nrhs);
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_solution_update(int zprec, const void* Z, long ldb, double2* u, long ustride,
                                 long n, int nrhs, const double2* y, int ldy, const int* jn,
                                 cudaStream_t st) {
  const int nblk = krylov_blocks(n, nrhs, 1);
  if (zprec == 0)
    solution_update_kernel<double2><<<dim3(nblk, nrhs), KT, 0, st>>>(
        static_cast<const double2*>(Z), ldb, u, ustride, n, y, ldy, jn);
  else
    solution_update_kernel<float2><<<dim3(nblk, nrhs), KT, 0, st>>>(
        static_cast<const float2*>(Z), ldb, u, ustride, n, y, ldy, jn);
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_combine(const double2* V, long ldb, double2* out, long ostride, long n, int nrhs,
                         const double2* y, int ldy, const double* sigma, int ldsig, const int* jn,
                         cudaStream_t st) {
  const int nblk = krylov_blocks(n, nrhs, 1);
  combine_kernel<<<dim3(nblk, nrhs), KT, 0, st>>>(V, ldb, out, ostride, n, y, ldy, sigma, ldsig, jn);
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_axpy(double2* u, const double2* t, long stride, long n, int nrhs, const int* jn,
                      cudaStream_t st) {
  const int nblk = krylov_blocks(n, nrhs, 1);
  axpy_kernel<<<dim3(nblk, nrhs), KT, 0, st>>>(u, t, stride, n, jn);
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_norm2(const double2* x, long stride, long n, int nrhs, double* partial, int nblk,
                       double* out, cudaStream_t st) {
  norm2_kernel<<<dim3(nblk, nrhs), KT, 0, st>>>(x, stride, n, partial);
  reduce_r_kernel<<<unsigned(nrhs), KT, 0, st>>>(partial, nblk, out);
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_reduce_r(const double* partial, int nblk, int nq, double* out, cudaStream_t st) {
  reduce_r_kernel<<<unsigned(nq), KT, 0, st>>>(partial, nblk, out);
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

}  // namespace hz
