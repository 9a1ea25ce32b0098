// Finite-difference Helmholtz operator P_N (Eqn. 001 discretised as in
// Section 5: second-order centred differences, periodic boundaries), FP64:
//   (P x)_j = gamma_j^2 sum_axes (x_{j+e} - 2 x_j + x_{j-e}) / h_axis^2
//             + (omega^2 + i omega a_j) x_j,
// with gamma^2 = c^2 (1 - i zeta)^2 (Eqn. Complex_wave_speed).
// Mode RESID computes r = f - P x and per-block partial sums of |r|^2.
#include "hz_internal.h"
#include "kernels.h"

namespace hz {
namespace {

constexpr int ST_THREADS = 256;

__device__ __forceinline__ double2 ld2(const double2* p, long i) { return p[i]; }
__device__ __forceinline__ double2 ld2(const float2* p, long i) {
  const float2 v = p[i];
  return make_double2(f2d_bits(v.x), f2d_bits(v.y));
}

// The stencil in the form that takes the fewest FP64 instructions per point
// (the FP64 pipe is this kernel's limit): with g = gamma^2 / h_x^2 (stored
// so by the medium), rho_a = h_x^2 / h_a^2 and diag = 2 sum_a rho_a,
//   (P x)_j = g_j [ (x_{j-ex} + x_{j+ex}) + rho_y (x_{j-ey} + x_{j+ey})
//                  (+ rho_z (...)) - diag x_j ] + (omega^2 + i omega a_j) x_j.
template <typename InT, bool RESID>
__global__ void __launch_bounds__(ST_THREADS)
stencil_kernel(const InT* __restrict__ x, double2* __restrict__ y, const double2* __restrict__ f,
               const double2* __restrict__ gs, const double* __restrict__ a, double omega,
               double w2, double rho_y, double rho_z, double diag, int nx, int ny, int nz, long n,
               long in_stride, long out_stride, const int* __restrict__ active,
               double* __restrict__ partial) {
  pdl_wait();
  const int b = blockIdx.y;
  double nrm = 0.0;
  const bool on = !active || active[b];
  if (on) {
    const InT* xb = x + b * in_stride;
    const long i = long(blockIdx.x) * ST_THREADS + threadIdx.x;
    if (i < n) {
      // n < 2^31 per right-hand side: 32-bit division
      const unsigned ui = unsigned(i);
      const unsigned r = ui / unsigned(nx);
      const int ix = int(ui - r * unsigned(nx));
      const unsigned rz = r / unsigned(ny);
      const int iy = int(r - rz * unsigned(ny));
      const int iz = int(rz);
      const long xl = ix == 0 ? i + nx - 1 : i - 1;
      const long xr = ix == nx - 1 ? i - (nx - 1) : i + 1;
      const long sy = nx;
      const long yd = iy == 0 ? i + sy * (ny - 1) : i - sy;
      const long yu = iy == ny - 1 ? i - sy * (ny - 1) : i + sy;
      const double2 c = ld2(xb, i);
      const double2 vxl = ld2(xb, xl), vxr = ld2(xb, xr), vyd = ld2(xb, yd), vyu = ld2(xb, yu);
      double sr = fma(rho_y, vyd.x + vyu.x, vxl.x + vxr.x);
      double si = fma(rho_y, vyd.y + vyu.y, vxl.y + vxr.y);
      if (nz > 1) {
        const long sz = long(nx) * ny;
        const long zd = iz == 0 ? i + sz * (nz - 1) : i - sz;
        const long zu = iz == nz - 1 ? i - sz * (nz - 1) : i + sz;
        const double2 vzd = ld2(xb, zd), vzu = ld2(xb, zu);
        sr = fma(rho_z, vzd.x + vzu.x, sr);
        si = fma(rho_z, vzd.y + vzu.y, si);
      }
      sr = fma(-diag, c.x, sr);
      si = fma(-diag, c.y, si);
      const double2 g = gs[i];
      // g * lap + (w^2 + i w a) x
      double yr = fma(g.x, sr, fma(-g.y, si, w2 * c.x));
      double yi = fma(g.x, si, fma(g.y, sr, w2 * c.y));
      if (a) {
        const double wa = omega * a[i];
        yr = fma(-wa, c.y, yr);
        yi = fma(wa, c.x, yi);
      }
      if (RESID) {
        const double2 fv = f[b * out_stride + i];
        yr = fv.x - yr;
        yi = fv.y - yi;
        nrm = yr * yr + yi * yi;
      }
      y[b * out_stride + i] = make_double2(yr, yi);
    }
  }
  if (RESID) {
    // fixed-shape block reduction of |r|^2
    __shared__ double sh[ST_THREADS];
    sh[threadIdx.x] = nrm;
    __syncthreads();
    for (int s = ST_THREADS / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[long(b) * gridDim.x + blockIdx.x] = sh[0];
  }
}

}  // namespace

int stencil_blocks(long n) { return int((n + ST_THREADS - 1) / ST_THREADS); }

namespace {
struct StencilConsts {
  double w2, rho_y, rho_z, diag;
};
StencilConsts stencil_consts(const hz_medium* m) {
  StencilConsts k;
  k.w2 = m->omega * m->omega;
  k.rho_y = m->inv_h2[1] / m->inv_h2[0];
  k.rho_z = m->dim == 3 ? m->inv_h2[2] / m->inv_h2[0] : 0.0;
  k.diag = 2.0 * (1.0 + k.rho_y + k.rho_z);
  return k;
}
}  // namespace

hz_status launch_stencil(const hz_medium* m, int in_prec, const void* x, long in_stride,
                         double2* y, long out_stride, int nrhs, const int* active,
                         cudaStream_t st) {
  dim3 grid(unsigned(stencil_blocks(m->n)), unsigned(nrhs));
  const StencilConsts k = stencil_consts(m);
  if (in_prec == 0)
    HZ_CUDA(launch_pdl(stencil_kernel<double2, false>, dim3(grid), dim3(ST_THREADS), 0, st,
                       static_cast<const double2*>(x), y, nullptr, m->gamma2, m->a, m->omega, k.w2,
                       k.rho_y, k.rho_z, k.diag, m->nx, m->ny, m->nz, m->n, in_stride, out_stride,
                       active, nullptr));
  else
    HZ_CUDA(launch_pdl(stencil_kernel<float2, false>, dim3(grid), dim3(ST_THREADS), 0, st,
                       static_cast<const float2*>(x), y, nullptr, m->gamma2, m->a, m->omega, k.w2,
                       k.rho_y, k.rho_z, k.diag, m->nx, m->ny, m->nz, m->n, in_stride, out_stride,
                       active, nullptr));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status launch_residual(const hz_medium* m, const double2* u, const double2* f, double2* r,
                          long stride, int nrhs, const int* active, double* partial,
                          cudaStream_t st) {
  dim3 grid(unsigned(stencil_blocks(m->n)), unsigned(nrhs));
  const StencilConsts k = stencil_consts(m);
  HZ_CUDA(launch_pdl(stencil_kernel<double2, true>, dim3(grid), dim3(ST_THREADS), 0, st, u, r, f,
                     m->gamma2, m->a, m->omega, k.w2, k.rho_y, k.rho_z, k.diag, m->nx, m->ny, m->nz,
                     m->n, stride, stride, active, partial));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

}  // namespace hz
