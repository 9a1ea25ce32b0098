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
constexpr int VCMAX = 8;  // basis vectors per dots block (at most)

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

// S[b][i] partials: raw sums sum_p conj(V_i[p]) w[p] for i in [i0, i0 + nv),
// chunks of vpc = ceil((j+1) / nchunk) <= VC vectors, i0 = chunk * vpc,
// nv = min(vpc, j + 1 - i0).  grid = (nblk, nrhs, nchunk).  partial layout
// [(b * (j+1) + i) * nblk + blk] as double2.  The next point's operands are
// loaded before the current point's FMAs so that the FP64 pipe, the limit
// here, does not wait on memory.  With VC <= 4 every product has its own
// accumulator (re*re, im*im, re*im, im*re), so that no FMA waits on another
// FMA of the same point; with VC = 8 (register budget) two per vector.  Only
// the nv live sums are reduced.
template <int VC> struct DotsCfg {
  static constexpr int NA = VC <= 4 ? 4 : 2;  // accumulators per vector
  static constexpr int MINB = VC <= 2 ? 4 : (VC <= 4 ? 3 : 2);
};

template <int VC>
__global__ void __launch_bounds__(KT, DotsCfg<VC>::MINB)
dots_kernel(const double2* __restrict__ V, long ldb, const double2* __restrict__ w, long wstride,
            long n, int j, int vpc, const int* __restrict__ active, double2* __restrict__ partial) {
  pdl_wait();
  constexpr int NA = DotsCfg<VC>::NA;
  const int b = blockIdx.y;
  const int i0 = blockIdx.z * vpc;
  const int nv = min(vpc, j + 1 - i0);
  double acc[NA * VC];
#pragma unroll
  for (int c = 0; c < NA * VC; ++c) acc[c] = 0.0;
  const bool on = active[b] != 0;
  if (on) {
    const double2* wb = w + b * wstride;
    const double2* Vb = V + (long(i0) * ldb + b) * n;
    const long vs = ldb * n;
    const long step = long(gridDim.x) * KT;
    long p = long(blockIdx.x) * KT + threadIdx.x;
    double2 x, v[VC];
    if (p < n) {
      x = wb[p];
#pragma unroll
      for (int c = 0; c < VC; ++c)
        if (c < nv) v[c] = Vb[c * vs + p];
    }
    while (p < n) {
      const long q = p + step;
      double2 xn, vn[VC];
      if (q < n) {
        xn = wb[q];
#pragma unroll
        for (int c = 0; c < VC; ++c)
          if (c < nv) vn[c] = Vb[c * vs + q];
      }
#pragma unroll
      for (int c = 0; c < VC; ++c) {
        if (c < nv) {
          if constexpr (NA == 4) {
            acc[4 * c] = fma(v[c].x, x.x, acc[4 * c]);
            acc[4 * c + 1] = fma(v[c].y, x.y, acc[4 * c + 1]);
            acc[4 * c + 2] = fma(v[c].x, x.y, acc[4 * c + 2]);
            acc[4 * c + 3] = fma(v[c].y, x.x, acc[4 * c + 3]);
          } else {
            acc[2 * c] = fma(v[c].x, x.x, fma(v[c].y, x.y, acc[2 * c]));
            acc[2 * c + 1] = fma(v[c].x, x.y, fma(-v[c].y, x.x, acc[2 * c + 1]));
          }
        }
      }
      p = q;
      x = xn;
#pragma unroll
      for (int c = 0; c < VC; ++c) v[c] = vn[c];
    }
  }
  // conj(v) x = (re re + im im) + i (re im - im re)
  double sum[2 * VC];
#pragma unroll
  for (int c = 0; c < VC; ++c) {
    if constexpr (NA == 4) {
      sum[2 * c] = acc[4 * c] + acc[4 * c + 1];
      sum[2 * c + 1] = acc[4 * c + 2] - acc[4 * c + 3];
    } else {
      sum[2 * c] = acc[2 * c];
      sum[2 * c + 1] = acc[2 * c + 1];
    }
  }
  // block reduction of the 2 nv live sums (warp shuffles, then one value per warp)
  __shared__ double sh[(KT / 32) * 2 * VC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < 2 * VC; ++c) {
    if (c < 2 * nv) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum[c] += __shfl_down_sync(0xffffffffu, sum[c], o);
      if (lane == 0) sh[warp * 2 * VC + c] = sum[c];
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * nv) {
    double s = 0.0;
    for (int wi = 0; wi < KT / 32; ++wi) s += sh[wi * 2 * VC + threadIdx.x];
    sh[threadIdx.x] = s;  // rows 0..: warp 0's slots are no longer needed
  }
  __syncthreads();
  if (threadIdx.x < nv)
    partial[(long(b) * (j + 1) + i0 + threadIdx.x) * gridDim.x + blockIdx.x] =
        make_double2(sh[2 * threadIdx.x], sh[2 * threadIdx.x + 1]);
}

// Sum partials in a fixed order: q = b * jp1 + i,
// out[b * ldo + i] = sum_blk part[q * nblk + blk].
__global__ void __launch_bounds__(KT)
reduce_c_kernel(const double2* __restrict__ part, int nblk, int jp1, int ldo,
                double2* __restrict__ out) {
  pdl_wait();
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
  pdl_wait();
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
  pdl_wait();
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
    const double2* Vb = V + long(b) * n;
    const long vs = ldb * n;  // stride between basis vectors
    for (long p = long(blockIdx.x) * KT + threadIdx.x; p < n; p += long(gridDim.x) * KT) {
      // d = sum_i c_i V_i[p] in two interleaved partial sums; loads hoisted
      double dr0 = 0.0, di0 = 0.0, dr1 = 0.0, di1 = 0.0;
      int i = 0;
      for (; i + 3 <= j; i += 4) {
        const double2 v0 = Vb[(i + 0) * vs + p], v1 = Vb[(i + 1) * vs + p];
        const double2 v2 = Vb[(i + 2) * vs + p], v3 = Vb[(i + 3) * vs + p];
        const double2 c0 = coef[i], c1 = coef[i + 1], c2 = coef[i + 2], c3 = coef[i + 3];
        dr0 = fma(c0.x, v0.x, fma(-c0.y, v0.y, dr0));
        di0 = fma(c0.x, v0.y, fma(c0.y, v0.x, di0));
        dr1 = fma(c1.x, v1.x, fma(-c1.y, v1.y, dr1));
        di1 = fma(c1.x, v1.y, fma(c1.y, v1.x, di1));
        dr0 = fma(c2.x, v2.x, fma(-c2.y, v2.y, dr0));
        di0 = fma(c2.x, v2.y, fma(c2.y, v2.x, di0));
        dr1 = fma(c3.x, v3.x, fma(-c3.y, v3.y, dr1));
        di1 = fma(c3.x, v3.y, fma(c3.y, v3.x, di1));
      }
      for (; i <= j; ++i) {
        const double2 v = Vb[i * vs + p];
        const double2 c = coef[i];
        dr0 = fma(c.x, v.x, fma(-c.y, v.y, dr0));
        di0 = fma(c.x, v.y, fma(c.y, v.x, di0));
      }
      double2 x = wb[p];
      x.x -= dr0 + dr1;
      x.y -= di0 + di1;
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

__device__ __forceinline__ double2 cfma_d(double2 a, double2 b, double2 c) {  // a b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// 1/sqrt(x) for x > 0: the MUFU approximation refined by three Newton-Raphson
// steps y <- y + y (1 - x y^2) / 2 (each doubles the correct bits).  The
// Givens kernel runs in one warp, where every FP64 instruction holds the
// sub-partition's FP64 unit for ~64 cycles; this takes fewer of them than a
// square root followed by a division.
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
#pragma unroll
  for (int it = 0; it < 3; ++it) {
    const double e = fma(-x * y, y, 1.0);
    y = fma(0.5 * y, e, y);
  }
  return y;
}
// max(|a|, |b|) of finite doubles as an integer max of the magnitude bits
// (IEEE order of non-negative doubles is that of their bit patterns), off the
// FP64 pipe
__device__ __forceinline__ long long absbits(double a) {
  return __double_as_longlong(a) & 0x7fffffffffffffffLL;
}

__device__ __forceinline__ double2 shfl_up_d2(double2 v, int o) {
  return make_double2(__shfl_up_sync(0xffffffffu, v.x, o), __shfl_up_sync(0xffffffffu, v.y, o));
}

// One warp per right-hand side: form column j of the Hessenberg matrix,
// apply the earlier rotations, build the new one (c real, G [a;b] = [r;0]),
// update g and the residual estimate, and retire converged / broken rows.
// Applying rotations 0..j-1 is a linear recurrence on the running entry,
//   x_0 = h_0,  x_{i+1} = -conj(s_i) x_i + c_i h_{i+1},  r_i = c_i x_i + s_i h_{i+1},
// evaluated as a warp scan of affine maps (each lane composes a contiguous
// chunk, a shuffle scan composes the chunks) instead of j serial steps.
__global__ void givens_kernel(KsDev ks, int j, int nrhs) {
  pdl_wait();
  const int b = blockIdx.x;
  const int lane = threadIdx.x;
  if (b >= nrhs || !ks.active[b]) return;
  const int m = ks.m;
  __shared__ double2 col[HZ_MAX_RESTART + 2];   // h, the new column before rotation
  __shared__ double2 rcol[HZ_MAX_RESTART + 2];  // rotated column
  double2* colg = ks.H + (long(b) * m + j) * (m + 1);
  const double2* S1 = ks.S1 + long(b) * (m + 1);
  const double2* S2 = ks.S2 + long(b) * (m + 1);
  double* cs = ks.cs + long(b) * m;
  double2* sn = ks.sn + long(b) * m;
  double2* g = ks.g + long(b) * (m + 1);
  long long hbits = 0;  // bits of max |Re h|, |Im h|
  bool bad = false;
  for (int i = lane; i <= j; i += 32) {
    const double s = ks.sigma[long(i) * ks.ldsig + b];
    const double2 h = make_double2(s * (S1[i].x + S2[i].x), s * (S1[i].y + S2[i].y));
    col[i] = h;
    ks.Hraw[(long(b) * m + j) * (m + 1) + i] = h;
    hbits = max(hbits, max(absbits(h.x), absbits(h.y)));
    bad |= !isfinite(h.x) || !isfinite(h.y);
  }
  const double hn2 = ks.nrm2[b];  // |w|^2 after orthogonalisation
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) hbits = max(hbits, __shfl_xor_sync(0xffffffffu, hbits, o));
  const double hmax = __longlong_as_double(hbits);
  bad = __any_sync(0xffffffffu, bad) || !isfinite(hn2);
  __syncwarp();
  // chunk of maps i in [i0, i1) of this lane; composite F(x) = A x + B
  const int per = (j + 31) / 32;
  const int i0 = min(j, lane * per), i1 = min(j, i0 + per);
  double2 A = make_double2(1.0, 0.0), B = make_double2(0.0, 0.0);
  for (int i = i0; i < i1; ++i) {
    const double2 al = make_double2(-sn[i].x, sn[i].y);  // -conj(s_i)
    const double c = cs[i];
    const double2 be = make_double2(c * col[i + 1].x, c * col[i + 1].y);
    A = cmul_d(al, A);
    B = cfma_d(al, B, be);
  }
  // inclusive scan over lanes: G_l = F_l o F_{l-1} o ... o F_0
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double2 Ap = shfl_up_d2(A, o), Bp = shfl_up_d2(B, o);
    if (lane >= o) {
      B = cfma_d(A, Bp, B);
      A = cmul_d(A, Ap);
    }
  }
  const double2 h0 = col[0];
  double2 Ae = shfl_up_d2(A, 1), Be = shfl_up_d2(B, 1);
  if (lane == 0) {
    Ae = make_double2(1.0, 0.0);
    Be = make_double2(0.0, 0.0);
  }
  double2 x = cfma_d(Ae, h0, Be);  // x_{i0}
  for (int i = i0; i < i1; ++i) {
    const double c = cs[i];
    const double2 sv = sn[i], h1 = col[i + 1];
    rcol[i] = cfma_d(sv, h1, make_double2(c * x.x, c * x.y));
    x = cfma_d(make_double2(-sv.x, sv.y), x, make_double2(c * h1.x, c * h1.y));
  }
  const double2 xall = cfma_d(A, h0, B);  // lane 31 holds the full composition
  const double2 a = make_double2(__shfl_sync(0xffffffffu, xall.x, 31), __shfl_sync(0xffffffffu, xall.y, 31));
  __syncwarp();
  if (lane == 0) {
    // h_{j+1,j} = hn = |w|; sigma_{j+1} = 1 / hn normalises the next vector
    const double inv_hn = hn2 > 0.0 ? rsqrt_nr(hn2) : 0.0;
    const double hn = hn2 * inv_hn;
    ks.Hraw[(long(b) * m + j) * (m + 1) + j + 1] = make_double2(hn, 0.0);
    const bool happy = hn <= 1e-14 * hmax;
    ks.sigma[long(j + 1) * ks.ldsig + b] = (hn > 0.0 && !happy) ? inv_hn : 0.0;
    const double aa2 = fma(a.x, a.x, a.y * a.y);
    double c;
    double2 s, r;
    if (hn == 0.0) {
      c = 1.0; s = make_double2(0.0, 0.0); r = a;
    } else if (aa2 == 0.0) {
      c = 0.0; s = make_double2(1.0, 0.0); r = make_double2(hn, 0.0);
    } else {
      // rho = sqrt(|a|^2 + hn^2); c = |a| / rho; s = (a / |a|) hn / rho;
      // r = (a / |a|) rho
      const double rho2 = aa2 + hn2;
      const double inv_aa = rsqrt_nr(aa2), inv_rho = rsqrt_nr(rho2);
      const double aa = aa2 * inv_aa, rho = rho2 * inv_rho;
      c = aa * inv_rho;
      const double2 ph = make_double2(a.x * inv_aa, a.y * inv_aa);
      const double hr = hn * inv_rho;
      s = make_double2(ph.x * hr, ph.y * hr);  // ph conj(hn) / rho
      r = make_double2(ph.x * rho, ph.y * rho);
    }
    cs[j] = c;
    sn[j] = s;
    rcol[j] = r;
    rcol[j + 1] = make_double2(0.0, 0.0);
    const double2 gj = g[j];
    const double2 gn = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    g[j + 1] = gn;  // -conj(s) g_j
    g[j] = make_double2(c * gj.x, c * gj.y);
    const double gn2 = fma(gn.x, gn.x, gn.y * gn.y);
    const double est = gn2 > 0.0 ? gn2 * rsqrt_nr(gn2) : 0.0;
    ks.est[b] = est;
    ks.hist[long(b) * m + j] = est / ks.bnorm[b];
    ks.jend[b] = j + 1;
    bad |= !isfinite(est) || !isfinite(r.x) || !isfinite(r.y);
    int act = 1;
    if (bad) {
      ks.status[b] = HZ_ERR_BREAKDOWN;
      act = 0;
    } else if (est <= ks.tol * ks.bnorm[b] || happy) {
      act = 0;
    }
    if (!act) {
      ks.active[b] = 0;
      atomicSub(ks.n_active, 1);
    }
  }
  __syncwarp();
  for (int i = lane; i <= j + 1; i += 32) colg[i] = rcol[i];
}

__device__ __forceinline__ double2 widen(double2 v) { return v; }
__device__ __forceinline__ double2 widen(float2 v) { return make_double2(f2d_bits(v.x), f2d_bits(v.y)); }

// u += sum_{i < jn} y[b][i] Z_i  (Z in c64 or c128), one pass.
template <typename ZT>
__global__ void __launch_bounds__(KT)
solution_update_kernel(const ZT* __restrict__ Z, long ldb, double2* __restrict__ u, long ustride,
                       long n, const double2* __restrict__ y, int ldy, const int* __restrict__ jn) {
  pdl_wait();
  const int b = blockIdx.y;
  const int J = jn[b];
  if (J <= 0) return;
  __shared__ double2 ys[HZ_MAX_RESTART];
  for (int i = threadIdx.x; i < J; i += KT) ys[i] = y[long(b) * ldy + i];
  __syncthreads();
  double2* ub = u + b * ustride;
  for (long p = long(blockIdx.x) * KT + threadIdx.x; p < n; p += long(gridDim.x) * KT) {
    // two interleaved partial sums; complex64 Z widened by integer bit moves
    // (off the FP64 pipe, the limit here)
    double2 x = ub[p], x1 = make_double2(0.0, 0.0);
    int i = 0;
    for (; i + 1 < J; i += 2) {
      const double2 z0 = widen(Z[(long(i) * ldb + b) * n + p]);
      const double2 z1 = widen(Z[(long(i + 1) * ldb + b) * n + p]);
      const double2 c0 = ys[i], c1 = ys[i + 1];
      x.x = fma(c0.x, z0.x, fma(-c0.y, z0.y, x.x));
      x.y = fma(c0.x, z0.y, fma(c0.y, z0.x, x.y));
      x1.x = fma(c1.x, z1.x, fma(-c1.y, z1.y, x1.x));
      x1.y = fma(c1.x, z1.y, fma(c1.y, z1.x, x1.y));
    }
    if (i < J) {
      const double2 z0 = widen(Z[(long(i) * ldb + b) * n + p]);
      const double2 c0 = ys[i];
      x.x = fma(c0.x, z0.x, fma(-c0.y, z0.y, x.x));
      x.y = fma(c0.x, z0.y, fma(c0.y, z0.x, x.y));
    }
    ub[p] = make_double2(x.x + x1.x, x.y + x1.y);
  }
}

// out[b] = sum_{i < J} (sigma_i y_i) V_i  (FP64 path: the combination that is
// then preconditioned).
__global__ void __launch_bounds__(KT)
combine_kernel(const double2* __restrict__ V, long ldb, double2* __restrict__ out, long ostride,
               long n, const double2* __restrict__ y, int ldy, const double* __restrict__ sigma,
               int ldsig, const int* __restrict__ jn) {
  pdl_wait();
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
  pdl_wait();
  const int b = blockIdx.y;
  if (jn[b] <= 0) return;
  for (long p = long(blockIdx.x) * KT + threadIdx.x; p < n; p += long(gridDim.x) * KT) {
    const double2 a = u[b * stride + p], c = t[b * stride + p];
    u[b * stride + p] = make_double2(a.x + c.x, a.y + c.y);
  }
}

// out[b] = sigma[b] V[b]: the operator input of an unpreconditioned step
__global__ void scale_copy_kernel(const double2* __restrict__ V, const double* __restrict__ sigma,
                                  double2* __restrict__ out, long n, const int* __restrict__ active) {
  pdl_wait();
  const int b = blockIdx.y;
  if (!active[b]) return;
  const double s = sigma[b];
  for (long p = long(blockIdx.x) * KT + threadIdx.x; p < n; p += long(gridDim.x) * KT) {
    const double2 v = V[b * n + p];
    out[b * n + p] = make_double2(s * v.x, s * v.y);
  }
}

// |x|^2 partials of nrhs vectors
__global__ void __launch_bounds__(KT)
norm2_kernel(const double2* __restrict__ x, long stride, long n, double* __restrict__ partial) {
  pdl_wait();
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

// Blocks per right-hand side of the element-wise FP64 kernels: bps blocks
// per SM over the whole launch, but at least one point per thread.  Short
// vectors thus still spread over every SM: an FP64 warp instruction holds a
// sub-partition's FP64 unit for ~64 cycles, so a few long-running warps
// would serialise the work.
int krylov_blocks_bps(long n, int nrhs, int nchunk, int bps) {
  long per = (long(bps) * 152 + long(nrhs) * nchunk - 1) / (long(nrhs) * nchunk);
  long maxb = (n + KT - 1) / KT;
  if (per > maxb) per = maxb;
  if (per < 1) per = 1;
  return int(per);
}

int krylov_blocks(long n, int nrhs, int nchunk) { return krylov_blocks_bps(n, nrhs, nchunk, 4); }

hz_status launch_dots(const double2* V, long ldb, const double2* w, long wstride, long n, int j,
                      int nrhs, const int* active, double2* partial, const Tune& tn, double2* S,
                      int ldS, cudaStream_t st) {
  // balanced chunks of at most vc vectors; one wave of tn.dots_bps blocks
  // per SM (the register budget allows two)
  const int vc = tn.dots_vc <= 2 ? 2 : (tn.dots_vc <= 4 ? 4 : VCMAX);
  int nchunk = (j + 1 + vc - 1) / vc;
  const int vpc = (j + 1 + nchunk - 1) / nchunk;
  nchunk = (j + 1 + vpc - 1) / vpc;  // no empty chunk
  long per = (long(tn.dots_bps) * 152) / (long(nrhs) * nchunk);
  const long cap = (n + KT - 1) / KT;  // at least one point per thread
  if (per > cap) per = cap;
  const int nblk = int(per < 1 ? 1 : per);
  if (vc == 2)
    HZ_CUDA(launch_pdl(dots_kernel<2>, dim3(nblk, nrhs, nchunk), dim3(KT), 0, st, V, ldb, w,
                       wstride, n, j, vpc, active, partial));
  else if (vc == 4)
    HZ_CUDA(launch_pdl(dots_kernel<4>, dim3(nblk, nrhs, nchunk), dim3(KT), 0, st, V, ldb, w,
                       wstride, n, j, vpc, active, partial));
  else
    HZ_CUDA(launch_pdl(dots_kernel<VCMAX>, dim3(nblk, nrhs, nchunk), dim3(KT), 0, st, V, ldb, w,
                       wstride, n, j, vpc, active, partial));
  HZ_CUDA(launch_pdl(reduce_c_kernel, dim3(unsigned(nrhs * (j + 1))), dim3(KT), 0, st, partial,
                     nblk, j + 1, ldS, S));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_update(const double2* V, long ldb, double2* w, long wstride, long n, int j,
                        int nrhs, const double2* S, int ldS, const double* sigma, int ldsig,
                        const int* active, bool norm, double* partial, const Tune& tn, double* nrm2,
                        cudaStream_t st) {
  const int nblk = krylov_blocks_bps(n, nrhs, 1, tn.upd_bps);
  if (norm) {
    HZ_CUDA(launch_pdl(update_kernel<true>, dim3(nblk, nrhs), dim3(KT), 0, st, V, ldb, w, wstride,
                       n, j, S, ldS, sigma, ldsig, active, partial));
    HZ_CUDA(launch_pdl(reduce_r_kernel, dim3(unsigned(nrhs)), dim3(KT), 0, st, partial, nblk,
                       nrm2));
  } else {
    HZ_CUDA(launch_pdl(update_kernel<false>, dim3(nblk, nrhs), dim3(KT), 0, st, V, ldb, w, wstride,
                       n, j, S, ldS, sigma, ldsig, active, nullptr));
  }
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_givens(const KsDev& ks, int j, int nrhs, cudaStream_t st) {
  HZ_CUDA(launch_pdl(givens_kernel, dim3(nrhs), dim3(32), 0, st, ks, j, nrhs));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_solution_update(int zprec, const void* Z, long ldb, double2* u, long ustride,
                                 long n, int nrhs, const double2* y, int ldy, const int* jn,
                                 cudaStream_t st) {
  const int nblk = krylov_blocks(n, nrhs, 1);
  if (zprec == 0)
    HZ_CUDA(launch_pdl(solution_update_kernel<double2>, dim3(nblk, nrhs), dim3(KT), 0, st,
                       static_cast<const double2*>(Z), ldb, u, ustride, n, y, ldy, jn));
  else
    HZ_CUDA(launch_pdl(solution_update_kernel<float2>, dim3(nblk, nrhs), dim3(KT), 0, st,
                       static_cast<const float2*>(Z), ldb, u, ustride, n, y, ldy, jn));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_combine(const double2* V, long ldb, double2* out, long ostride, long n, int nrhs,
                         const double2* y, int ldy, const double* sigma, int ldsig, const int* jn,
                         cudaStream_t st) {
  const int nblk = krylov_blocks(n, nrhs, 1);
  HZ_CUDA(launch_pdl(combine_kernel, dim3(nblk, nrhs), dim3(KT), 0, st, V, ldb, out, ostride, n, y,
                     ldy, sigma, ldsig, jn));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_scale_copy(const double2* V, const double* sigma, double2* out, long n, int nrhs,
                           const int* active, cudaStream_t st) {
  const int nblk = krylov_blocks(n, nrhs, 1);
  HZ_CUDA(launch_pdl(scale_copy_kernel, dim3(nblk, nrhs), dim3(KT), 0, st, V, sigma, out, n,
                     active));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_axpy(double2* u, const double2* t, long stride, long n, int nrhs, const int* jn,
                      cudaStream_t st) {
  const int nblk = krylov_blocks(n, nrhs, 1);
  HZ_CUDA(launch_pdl(axpy_kernel, dim3(nblk, nrhs), dim3(KT), 0, st, u, t, stride, n, jn));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_norm2(const double2* x, long stride, long n, int nrhs, double* partial, int nblk,
                       double* out, cudaStream_t st) {
  HZ_CUDA(launch_pdl(norm2_kernel, dim3(nblk, nrhs), dim3(KT), 0, st, x, stride, n, partial));
  HZ_CUDA(launch_pdl(reduce_r_kernel, dim3(unsigned(nrhs)), dim3(KT), 0, st, partial, nblk, out));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_reduce_r(const double* partial, int nblk, int nq, double* out, cudaStream_t st) {
  HZ_CUDA(launch_pdl(reduce_r_kernel, dim3(unsigned(nq)), dim3(KT), 0, st, partial, nblk, out));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

}  // namespace hz
