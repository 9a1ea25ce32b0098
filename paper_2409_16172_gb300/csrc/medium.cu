// Medium set-up (plan time): validation, the node table of Section 4.1 /
// Section 4.4, per-point interpolation records of Eqn. 405, gamma^2 of
// Eqn. Complex_wave_speed, row / slab node masks, FFT twiddles and the
// per-axis |xi|^2 tables.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "hz_internal.h"

namespace hz {
namespace {

constexpr int VAL_THREADS = 256;

struct ValPartial {
  double cmin, cmax, zmax, amin, amax;
  unsigned long long bad_c, bad_zeta, bad_layer, bad_a;
};

// One pass over the medium: min/max of c, max of zeta and counts of the
// points that violate Section 3 (c > 0, finite) and Section 4.4 (zeta >= 0,
// c = c_o where zeta > 0).
__global__ void validate_kernel(const double* __restrict__ c, const double* __restrict__ zeta,
                                const double* __restrict__ a, long n, double c_o,
                                ValPartial* __restrict__ part) {
  double cmin = INFINITY, cmax = -INFINITY, zmax = 0.0, amin = INFINITY, amax = -INFINITY;
  unsigned long long bc = 0, bz = 0, bl = 0, ba = 0;
  for (long i = blockIdx.x * long(blockDim.x) + threadIdx.x; i < n; i += long(gridDim.x) * blockDim.x) {
    const double ci = c[i];
    const double zi = zeta ? zeta[i] : 0.0;
    if (!(ci > 0.0) || !isfinite(ci)) {
      ++bc;
    } else {
      cmin = fmin(cmin, ci);
      cmax = fmax(cmax, ci);
    }
    if (!(zi >= 0.0) || !isfinite(zi)) ++bz;
    else zmax = fmax(zmax, zi);
    if (zi > 0.0 && fabs(ci - c_o) > 1e-12 * c_o) ++bl;
    if (a) {
      if (!isfinite(a[i])) {
        ++ba;
      } else {
        amin = fmin(amin, a[i]);
        amax = fmax(amax, a[i]);
      }
    }
  }
  __shared__ ValPartial sh[VAL_THREADS];
  sh[threadIdx.x] = ValPartial{cmin, cmax, zmax, amin, amax, bc, bz, bl, ba};
  __syncthreads();
  for (int s = VAL_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      ValPartial& p = sh[threadIdx.x];
      const ValPartial& q = sh[threadIdx.x + s];
      p.cmin = fmin(p.cmin, q.cmin);
      p.cmax = fmax(p.cmax, q.cmax);
      p.zmax = fmax(p.zmax, q.zmax);
      p.amin = fmin(p.amin, q.amin);
      p.amax = fmax(p.amax, q.amax);
      p.bad_c += q.bad_c;
      p.bad_zeta += q.bad_zeta;
      p.bad_layer += q.bad_layer;
      p.bad_a += q.bad_a;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

struct NodeDev {
  double c_real[HZ_MAX_K];
  double zeta_nodes[HZ_MAX_K + 1];
  double a_nodes[HZ_MAX_K];
  int M, Mt, Ma, basis;
  uchar2 seg[HZ_MAX_SEG];
};

// Per point: the hat segment and t of Eqn. 405 (real hats in c where
// zeta = 0, hats in zeta on the layer segment where zeta > 0), gamma^2,
// and the row mask bits of the nodes with a non-zero weight.
__global__ void record_kernel(const double* __restrict__ c, const double* __restrict__ zeta,
                              long n, int nx, NodeDev nd, double* __restrict__ rec64,
                              uint32_t* __restrict__ rec32, double2* __restrict__ gamma2,
                              double ih2x, unsigned long long* __restrict__ rowmask) {
  const long i = blockIdx.x * long(blockDim.x) + threadIdx.x;
  unsigned long long bits = 0ull;
  long row = -1;
  if (i < n) {
    const double ci = c[i];
    const double zi = zeta ? zeta[i] : 0.0;
    int seg;
    double t;
    if (zi > 0.0) {
      int m = 0;
      while (m + 1 < nd.Mt && zi >= nd.zeta_nodes[m + 1]) ++m;
      t = (zi - nd.zeta_nodes[m]) / (nd.zeta_nodes[m + 1] - nd.zeta_nodes[m]);
      seg = nd.M + m;
    } else if (nd.M == 1) {
      seg = 0;
      t = 0.0;
    } else {
      int m = 0;
      while (m + 2 < nd.M && ci >= nd.c_real[m + 1]) ++m;
      t = (ci - nd.c_real[m]) / (nd.c_real[m + 1] - nd.c_real[m]);
      seg = m;
    }
    t = fmin(fmax(t, 0.0), 1.0);
    const double r = double(seg) + t;
    rec64[i] = r;
    rec32[i] = uint32_t(llrint(r * 16777216.0));
    const uchar2 kk = nd.seg[seg];
    if (t < 1.0) bits |= 1ull << kk.x;
    if (t > 0.0) bits |= 1ull << kk.y;
    // gamma^2 = c^2 (1 - i zeta)^2, stored times 1 / h_x^2 for the stencil
    const double c2 = ci * ci;
    gamma2[i] = make_double2(c2 * (1.0 - zi * zi) * ih2x, -2.0 * c2 * zi * ih2x);
    row = i / nx;
  }
  // OR the bits of the warp's points that share a row, then one atomic each
  const unsigned full = __activemask();
  const long row0 = __shfl_sync(full, row, 0);
  const bool same = __all_sync(full, row == row0);
  if (same && row0 >= 0) {
    const unsigned lo = __reduce_or_sync(full, unsigned(bits & 0xFFFFFFFFull));
    const unsigned hi = __reduce_or_sync(full, unsigned(bits >> 32));
    if ((threadIdx.x & 31) == 0) atomicOr(&rowmask[row0], (unsigned long long)lo | ((unsigned long long)hi << 32));
  } else if (row >= 0 && bits) {
    atomicOr(&rowmask[row], bits);
  }
}

// Per point, for the bivariate and quadratic forms: the non-zero weights of
// node k = s * Ma + j as (node, weight) pairs, speed weight of node s times
// the hat of a(x) on damping node j.  Speed weights: hats in zeta on the
// layer segment where zeta > 0 (Eqn. 405), else hats in c (basis 0) or the
// degree-2 Lagrange polynomials of the element [c_2e, c_2e+2] containing c
// (basis 1).  Also gamma^2 and the row mask bits of the nodes used.
__global__ void gen_record_kernel(const double* __restrict__ c, const double* __restrict__ zeta,
                                  const double* __restrict__ a, long n, int nx, NodeDev nd,
                                  uchar4* __restrict__ gnode, float4* __restrict__ gw32,
                                  double2* __restrict__ gw64, double2* __restrict__ gamma2,
                                  double ih2x, unsigned long long* __restrict__ rowmask) {
  const long i = blockIdx.x * long(blockDim.x) + threadIdx.x;
  unsigned long long bits = 0ull;
  long row = -1;
  if (i < n) {
    const double ci = c[i];
    const double zi = zeta ? zeta[i] : 0.0;
    const double ai = a ? a[i] : 0.0;
    int sk[4] = {0, 0, 0, 0};
    double sw[4] = {0.0, 0.0, 0.0, 0.0};
    int ns = 0;
    if (zi > 0.0) {
      int m = 0;
      while (m + 1 < nd.Mt && zi >= nd.zeta_nodes[m + 1]) ++m;
      double t = (zi - nd.zeta_nodes[m]) / (nd.zeta_nodes[m + 1] - nd.zeta_nodes[m]);
      t = fmin(fmax(t, 0.0), 1.0);
      const uchar2 kk = nd.seg[nd.M + m];
      sk[0] = kk.x; sw[0] = 1.0 - t;
      sk[1] = kk.y; sw[1] = t;
      ns = 2;
    } else if (nd.M == 1) {
      sk[0] = 0; sw[0] = 1.0;
      ns = 1;
    } else {
      int m = 0;
      while (m + 2 < nd.M && ci >= nd.c_real[m + 1]) ++m;
      if (nd.basis == 2) {
        // cubic Hermite on [c_m, c_m+1]: values h00, h01, derivative
        // planes (after the M + Mt value planes) h h10, h h11
        const double h = nd.c_real[m + 1] - nd.c_real[m];
        double t = (ci - nd.c_real[m]) / h;
        t = fmin(fmax(t, 0.0), 1.0);
        const double t2 = t * t, t3 = t2 * t;
        const int nv = nd.M + nd.Mt;
        sk[0] = m;          sw[0] = 2.0 * t3 - 3.0 * t2 + 1.0;
        sk[1] = m + 1;      sw[1] = 3.0 * t2 - 2.0 * t3;
        sk[2] = nv + m;     sw[2] = h * (t3 - 2.0 * t2 + t);
        sk[3] = nv + m + 1; sw[3] = h * (t3 - t2);
        ns = 4;
      } else if (nd.basis == 1) {
        const int e = min(m / 2, (nd.M - 1) / 2 - 1);
        const double c0 = nd.c_real[2 * e], c1 = nd.c_real[2 * e + 1], c2 = nd.c_real[2 * e + 2];
        sk[0] = 2 * e;     sw[0] = (ci - c1) * (ci - c2) / ((c0 - c1) * (c0 - c2));
        sk[1] = 2 * e + 1; sw[1] = (ci - c0) * (ci - c2) / ((c1 - c0) * (c1 - c2));
        sk[2] = 2 * e + 2; sw[2] = (ci - c0) * (ci - c1) / ((c2 - c0) * (c2 - c1));
        ns = 3;
      } else {
        double t = (ci - nd.c_real[m]) / (nd.c_real[m + 1] - nd.c_real[m]);
        t = fmin(fmax(t, 0.0), 1.0);
        sk[0] = m;     sw[0] = 1.0 - t;
        sk[1] = m + 1; sw[1] = t;
        ns = 2;
      }
    }
    int dk[2] = {0, 0};
    double dw[2] = {1.0, 0.0};
    int na = 1;
    if (nd.Ma > 1) {
      int j = 0;
      while (j + 2 < nd.Ma && ai >= nd.a_nodes[j + 1]) ++j;
      double t = (ai - nd.a_nodes[j]) / (nd.a_nodes[j + 1] - nd.a_nodes[j]);
      t = fmin(fmax(t, 0.0), 1.0);
      dk[0] = j;     dw[0] = 1.0 - t;
      dk[1] = j + 1; dw[1] = t;
      na = 2;
    }
    unsigned char kn[4] = {0xFF, 0xFF, 0xFF, 0xFF};
    double wv[4] = {0.0, 0.0, 0.0, 0.0};
    int used = 0;
    for (int s = 0; s < ns; ++s) {
      for (int d = 0; d < na; ++d) {
        const double w = sw[s] * dw[d];
        if (w != 0.0 && used < 4) {
          const int k = sk[s] * nd.Ma + dk[d];
          kn[used] = (unsigned char)k;
          wv[used] = w;
          bits |= 1ull << k;
          ++used;
        }
      }
    }
    gnode[i] = make_uchar4(kn[0], kn[1], kn[2], kn[3]);
    gw32[i] = make_float4(float(wv[0]), float(wv[1]), float(wv[2]), float(wv[3]));
    gw64[2 * i] = make_double2(wv[0], wv[1]);
    gw64[2 * i + 1] = make_double2(wv[2], wv[3]);
    const double c2 = ci * ci;
    gamma2[i] = make_double2(c2 * (1.0 - zi * zi) * ih2x, -2.0 * c2 * zi * ih2x);
    row = i / nx;
  }
  const unsigned full = __activemask();
  const long row0 = __shfl_sync(full, row, 0);
  const bool same = __all_sync(full, row == row0);
  if (same && row0 >= 0) {
    const unsigned lo = __reduce_or_sync(full, unsigned(bits & 0xFFFFFFFFull));
    const unsigned hi = __reduce_or_sync(full, unsigned(bits >> 32));
    if ((threadIdx.x & 31) == 0) atomicOr(&rowmask[row0], (unsigned long long)lo | ((unsigned long long)hi << 32));
  } else if (row >= 0 && bits) {
    atomicOr(&rowmask[row], bits);
  }
}

// 3D: slabmask[z] = OR over y of rowmask[z * ny + y].
__global__ void slab_kernel(const unsigned long long* __restrict__ rowmask, int ny, int nz,
                            unsigned long long* __restrict__ slabmask) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nz) return;
  unsigned long long m = 0ull;
  for (int y = 0; y < ny; ++y) m |= rowmask[long(z) * ny + y];
  slabmask[z] = m;
}

// exp(-2 pi i j / N) with the angle reduced to the first quadrant so that
// every entry is accurate to a few ulp.
void twiddles(int N, std::vector<double2>& w) {
  w.resize(N);
  for (int j = 0; j < N; ++j) {
    const int q = (4 * j) / N;          // quadrant (N is a multiple of 4)
    const int r = j - q * (N / 4);
    const double th = 2.0 * M_PI * double(r) / double(N);
    const double c = std::cos(th), s = std::sin(th);
    double cr, sr;  // cos/sin of 2 pi j / N
    switch (q) {
      case 0: cr = c; sr = s; break;
      case 1: cr = -s; sr = c; break;
      case 2: cr = -c; sr = -s; break;
      default: cr = s; sr = -c; break;
    }
    w[j] = make_double2(cr, -sr);
  }
}

void xi2_table(int N, double L, int kind, std::vector<double>& t) {
  t.resize(N);
  for (int k = 0; k < N; ++k) {
    if (kind == 0) {
      const int ks = (k <= (N - 1) / 2) ? k : k - N;
      const double xi = 2.0 * M_PI * double(ks) / L;
      t[k] = xi * xi;
    } else {
      const double h = L / N;
      const double s = std::sin(M_PI * double(k) / double(N));
      t[k] = 4.0 / (h * h) * s * s;
    }
  }
}

template <typename T>
hz_status upload(DevArena& ar, T** d, const std::vector<T>& h, cudaStream_t cs) {
  HZ_TRY(ar.alloc(d, h.size()));
  // pageable source: the call returns once the data has been staged
  HZ_CUDA(cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, cs));
  return HZ_OK;
}

// Real nodes (Lemma 3: equispaced, c_1 = c_lo, c_M = c_hi).  With force_co
// the background speed c_o is a node (Section 4.4): a c_o strictly inside
// the range splits it into two equispaced segments of s1 and M-1-s1
// intervals, s1 = clamp(round((M-1)(c_o-c_lo)/(c_hi-c_lo)), 1, M-2).
// basis 1 (quadratic elements of two intervals): M odd, and the split gives
// each segment an even number of intervals,
// s1 = clamp(2 round((M-1)(c_o-c_lo)/(2(c_hi-c_lo))), 2, M-3).
hz_status real_nodes(double c_lo, double c_hi, int M, bool force_co, double c_o, int basis,
                     std::vector<double>& out) {
  out.clear();
  if (M == 1) {
    out.push_back(force_co ? c_o : c_lo);
    return HZ_OK;
  }
  if (c_hi - c_lo <= 1e-12 * c_hi) {
    out.push_back(c_lo);
    return HZ_OK;
  }
  if (basis == 1 && M % 2 == 0)
    return set_error(HZ_ERR_INVALID_ARG, "the quadratic basis needs an odd number of real nodes");
  if (force_co && c_lo < c_o && c_o < c_hi) {
    if (M < (basis == 1 ? 5 : 3))
      return set_error(HZ_ERR_MEDIUM, "c_o inside (c_min, c_max) needs more real nodes");
    int s1;
    if (basis == 1) {
      s1 = 2 * int(std::floor((M - 1) * (c_o - c_lo) / (2.0 * (c_hi - c_lo)) + 0.5));
      s1 = std::min(std::max(s1, 2), M - 3);
    } else {
      s1 = int(std::floor((M - 1) * (c_o - c_lo) / (c_hi - c_lo) + 0.5));
      s1 = std::min(std::max(s1, 1), M - 2);
    }
    const int s2 = (M - 1) - s1;
    for (int i = 0; i < s1; ++i) out.push_back(c_lo + (c_o - c_lo) * i / s1);
    for (int i = 0; i < s2; ++i) out.push_back(c_o + (c_hi - c_o) * i / s2);
    out.push_back(c_hi);
    return HZ_OK;
  }
  for (int i = 0; i < M - 1; ++i) out.push_back(c_lo + (c_hi - c_lo) * i / (M - 1));
  out.push_back(c_hi);
  return HZ_OK;
}

}  // namespace

bool fft_size_supported(int N) {
  switch (N) {
    case 8: case 12: case 16: case 24: case 32: case 48: case 64: case 96: case 128:
    case 192: case 256: case 512: case 1024: case 2048:
    case 20: case 40: case 60: case 120: case 180: case 240: case 360: case 480: case 720:
    case 960: case 1440: case 1920: case 2400: case 2880: case 3600: case 4800:
      return true;
    default:
      return false;
  }
}

}  // namespace hz

using namespace hz;

extern "C" hz_status hz_create_medium(const hz_grid* grid, const double* c, const double* zeta,
                                      const double* a, double omega, const hz_interp* interp,
                                      hz_medium** out) {
  if (!grid || !c || !interp || !out) return set_error(HZ_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (grid->dim != 2 && grid->dim != 3) return set_error(HZ_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (!(grid->L > 0) || !std::isfinite(grid->L)) return set_error(HZ_ERR_INVALID_ARG, "L must be > 0");
  for (int d = 0; d < grid->dim; ++d) {
    if (!fft_size_supported(grid->n[d]))
      return set_error(HZ_ERR_INVALID_ARG, "unsupported axis length %d", grid->n[d]);
  }
  if (grid->dim == 3 && grid->n[2] > 1024)
    return set_error(HZ_ERR_INVALID_ARG, "z axis longer than 1024");
  {
    // kernels index one right-hand side's points with 32-bit integers
    const long long pts = (long long)grid->n[0] * grid->n[1] * (grid->dim == 3 ? grid->n[2] : 1);
    if (pts >= (1LL << 31)) return set_error(HZ_ERR_INVALID_ARG, "grid has %lld >= 2^31 points", pts);
  }
  if (!(omega > 0) || !std::isfinite(omega)) return set_error(HZ_ERR_INVALID_ARG, "omega must be > 0");
  if (interp->M < 1 || interp->Mt < 0 || interp->M + interp->Mt > HZ_MAX_K)
    return set_error(HZ_ERR_INVALID_ARG, "need 1 <= M and M + Mt <= %d", HZ_MAX_K);
  if (!(interp->c_o > 0) || interp->alpha < 0 || interp->a_node < 0 ||
      (interp->symbol_kind != 0 && interp->symbol_kind != 1))
    return set_error(HZ_ERR_INVALID_ARG, "bad interpolation options");
  if (interp->Ma < 0 || interp->basis < 0 || interp->basis > 2 ||
      (interp->basis >= 1 && interp->Ma > 1) ||
      (interp->M + interp->Mt) * std::max(interp->Ma, 1) + (interp->basis == 2 ? interp->M : 0) >
          HZ_MAX_K)
    return set_error(HZ_ERR_INVALID_ARG,
                     "need Ma >= 0, basis 0, 1 or 2 (1 and 2 only with Ma <= 1), at most %d planes",
                     HZ_MAX_K);

  int dev = 0;
  {
    const cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return cuda_error(de, "cudaGetDevice");
  }
  hz_medium* m = new hz_medium();
  m->device = dev;
  m->dim = grid->dim;
  m->nx = grid->n[0];
  m->ny = grid->n[1];
  m->nz = grid->dim == 3 ? grid->n[2] : 1;
  m->n = long(m->nx) * m->ny * m->nz;
  m->L = grid->L;
  m->omega = omega;
  m->interp = *interp;
  const long n = m->n;
  auto fail = [&](hz_status s) {
    m->arena.release();
    delete m;
    return s;
  };

  // stage the medium on the device (dc, dz, dpart live in a scratch arena)
  DevArena scratch;
  struct ScratchGuard {
    DevArena& s;
    ~ScratchGuard() { s.release(); }
  } guard{scratch};
  double *dc = nullptr, *dz = nullptr;
  hz_status st = scratch.alloc(&dc, n);
  if (st == HZ_OK && zeta) st = scratch.alloc(&dz, n);
  if (st == HZ_OK && a) st = m->arena.alloc(&m->a, n);
  if (st != HZ_OK) return fail(st);
  // all work of the set-up runs on the calling thread's stream (the legacy
  // default stream unless a server worker set its own)
  cudaStream_t cs = tls_stream();
  cudaError_t ce = cudaMemcpyAsync(dc, c, n * sizeof(double), cudaMemcpyHostToDevice, cs);
  if (ce == cudaSuccess && zeta) ce = cudaMemcpyAsync(dz, zeta, n * sizeof(double), cudaMemcpyHostToDevice, cs);
  if (ce == cudaSuccess && a) ce = cudaMemcpyAsync(m->a, a, n * sizeof(double), cudaMemcpyHostToDevice, cs);
  if (ce != cudaSuccess) return fail(cuda_error(ce, "medium upload"));

  // validation and ranges
  const int vblocks = 304;
  ValPartial* dpart = nullptr;
  if ((st = scratch.alloc(&dpart, vblocks)) != HZ_OK) return fail(st);
  validate_kernel<<<vblocks, VAL_THREADS, 0, cs>>>(dc, dz, m->a, n, interp->c_o, dpart);
  count_launches(1);
  std::vector<ValPartial> hp(vblocks);
  ce = cudaMemcpyAsync(hp.data(), dpart, vblocks * sizeof(ValPartial), cudaMemcpyDeviceToHost, cs);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(cs);
  if (ce != cudaSuccess) return fail(cuda_error(ce, "validate"));
  double cmin = INFINITY, cmax = -INFINITY, zmax = 0, amin = INFINITY, amax = -INFINITY;
  unsigned long long bc = 0, bz = 0, bl = 0, ba = 0;
  for (const auto& p : hp) {
    cmin = std::min(cmin, p.cmin);
    cmax = std::max(cmax, p.cmax);
    zmax = std::max(zmax, p.zmax);
    amin = std::min(amin, p.amin);
    amax = std::max(amax, p.amax);
    bc += p.bad_c; bz += p.bad_zeta; bl += p.bad_layer; ba += p.bad_a;
  }
  if (bc) return fail(set_error(HZ_ERR_MEDIUM, "%llu points with c <= 0 or not finite", bc));
  if (bz) return fail(set_error(HZ_ERR_MEDIUM, "%llu points with zeta < 0 or not finite", bz));
  if (bl) return fail(set_error(HZ_ERR_MEDIUM, "%llu layer points with c != c_o", bl));
  if (ba) return fail(set_error(HZ_ERR_MEDIUM, "%llu points with a not finite", ba));
  m->c_min = cmin;
  m->c_max = cmax;

  // node table (Section 4.1 / 4.4)
  const bool layer = zmax > 0 && interp->Mt > 0;
  if (zmax > 0 && interp->Mt == 0)
    return fail(set_error(HZ_ERR_MEDIUM, "medium has a layer (zeta > 0) but Mt == 0"));
  double c_lo = cmin, c_hi = cmax;
  if (layer) {
    c_lo = std::min(c_lo, interp->c_o);
    c_hi = std::max(c_hi, interp->c_o);
  }
  if ((st = real_nodes(c_lo, c_hi, interp->M, layer || interp->M == 1, interp->c_o,
                       interp->basis == 1 ? 1 : 0, m->c_real)) != HZ_OK)
    return fail(st);
  m->M = int(m->c_real.size());
  m->m_o = -1;
  m->zeta_nodes.assign(1, 0.0);
  if (layer) {
    for (int i = 0; i < m->M; ++i)
      if (m->c_real[i] == interp->c_o) m->m_o = i;
    if (m->m_o < 0) return fail(set_error(HZ_ERR_MEDIUM, "c_o is not a node"));
    double zm = interp->zeta_max > 0 ? interp->zeta_max : zmax;
    if (zm < zmax) return fail(set_error(HZ_ERR_MEDIUM, "zeta_max below max(zeta)"));
    for (int i = 1; i < interp->Mt; ++i) m->zeta_nodes.push_back(i * zm / interp->Mt);
    m->zeta_nodes.push_back(zm);
    m->zeta_max = zm;
  }
  m->Mt = int(m->zeta_nodes.size()) - 1;
  const int Ks = m->M + m->Mt;  // speed nodes
  // damping nodes: bivariate form only (Ma >= 2), equispaced on [min a, max a]
  m->a_nodes.clear();
  if (interp->Ma >= 2) {
    const double lo = a ? amin : 0.0, hi = a ? amax : 0.0;
    if (hi - lo <= 1e-12 * std::max(std::fabs(hi), 1.0)) {
      m->a_nodes.push_back(lo);
    } else {
      for (int j = 0; j < interp->Ma - 1; ++j) m->a_nodes.push_back(lo + (hi - lo) * j / (interp->Ma - 1));
      m->a_nodes.push_back(hi);
    }
  } else {
    m->a_nodes.push_back(interp->a_node);
  }
  m->Ma = int(m->a_nodes.size());
  m->basis = interp->basis;
  m->generic = m->Ma > 1 || (m->basis >= 1 && m->M > 1);
  m->K = Ks * m->Ma;
  m->gamma_re.clear();
  m->gamma_im.clear();
  m->a_k.clear();
  for (int s = 0; s < Ks; ++s) {
    // gamma = c_s for real nodes, c_o (1 - i zeta_m) for layer nodes
    const double gr = s < m->M ? m->c_real[s] : interp->c_o;
    const double gi = s < m->M ? 0.0 : -interp->c_o * m->zeta_nodes[s - m->M + 1];
    for (int j = 0; j < m->Ma; ++j) {
      m->gamma_re.push_back(gr);
      m->gamma_im.push_back(gi);
      m->a_k.push_back(m->a_nodes[j] + interp->alpha * omega);
    }
  }
  // cubic Hermite: one plane per real node with the symbol's derivative in
  // the wave speed, dq/dc = 2 c |xi|^2 q^2, after the value planes
  m->dcoef.assign(m->K, 0.0);
  if (m->basis == 2 && m->M > 1) {
    for (int s = 0; s < m->M; ++s) {
      m->gamma_re.push_back(m->c_real[s]);
      m->gamma_im.push_back(0.0);
      m->a_k.push_back(m->a_nodes[0] + interp->alpha * omega);
      m->dcoef.push_back(2.0 * m->c_real[s]);
    }
    m->K += m->M;
  }

  // segment table: real segments, end entry, layer segments, end entry
  m->segtab_h.clear();
  for (int s = 0; s + 1 < m->M; ++s) m->segtab_h.push_back(make_uchar2(s, s + 1));
  m->segtab_h.push_back(make_uchar2(m->M - 1, m->M - 1));
  if (m->Mt > 0) {
    std::vector<int> node_of(m->Mt + 1);
    node_of[0] = m->m_o;
    for (int i = 1; i <= m->Mt; ++i) node_of[i] = m->M + i - 1;
    for (int i = 0; i < m->Mt; ++i) m->segtab_h.push_back(make_uchar2(node_of[i], node_of[i + 1]));
    m->segtab_h.push_back(make_uchar2(Ks - 1, Ks - 1));
  }
  m->nseg = int(m->segtab_h.size());

  NodeDev nd;
  memset(&nd, 0, sizeof(nd));
  nd.M = m->M;
  nd.Mt = m->Mt;
  nd.Ma = m->Ma;
  nd.basis = m->basis;
  for (int j = 0; j < m->Ma; ++j) nd.a_nodes[j] = m->a_nodes[j];
  for (int i = 0; i < m->M; ++i) nd.c_real[i] = m->c_real[i];
  for (int i = 0; i <= m->Mt; ++i) nd.zeta_nodes[i] = m->zeta_nodes[i];
  for (int i = 0; i < m->nseg; ++i) nd.seg[i] = m->segtab_h[i];

  const long nrows = n / m->nx;
  st = m->arena.alloc(&m->rec64, n);
  if (st == HZ_OK) st = m->arena.alloc(&m->rec32, n);
  if (st == HZ_OK) st = m->arena.alloc(&m->gamma2, n);
  if (st == HZ_OK) st = m->arena.alloc(&m->rowmask, nrows);
  if (st == HZ_OK) st = m->arena.alloc(&m->slabmask, m->nz);
  if (st == HZ_OK && m->generic) st = m->arena.alloc(&m->gnode, n);
  if (st == HZ_OK && m->generic) st = m->arena.alloc(&m->gw32, n);
  if (st == HZ_OK && m->generic) st = m->arena.alloc(&m->gw64, 2 * n);
  if (st != HZ_OK) return fail(st);
  ce = cudaMemsetAsync(m->rowmask, 0, nrows * sizeof(unsigned long long), cs);
  if (ce != cudaSuccess) return fail(cuda_error(ce, "memset"));
  const double hx = m->L / m->nx;
  if (m->generic) {
    gen_record_kernel<<<unsigned((n + 255) / 256), 256, 0, cs>>>(dc, dz, m->a, n, m->nx, nd, m->gnode,
                                                                m->gw32, m->gw64, m->gamma2,
                                                                1.0 / (hx * hx), m->rowmask);
  } else {
    record_kernel<<<unsigned((n + 255) / 256), 256, 0, cs>>>(dc, dz, n, m->nx, nd, m->rec64, m->rec32,
                                                            m->gamma2, 1.0 / (hx * hx), m->rowmask);
  }
  slab_kernel<<<(m->nz + 127) / 128, 128, 0, cs>>>(m->rowmask, m->ny, m->nz, m->slabmask);
  count_launches(2);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return fail(cuda_error(ce, "record kernel"));
  {
    std::vector<unsigned long long> rm(nrows), sm(m->nz);
    ce = cudaMemcpyAsync(rm.data(), m->rowmask, nrows * sizeof(unsigned long long), cudaMemcpyDeviceToHost, cs);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(sm.data(), m->slabmask, m->nz * sizeof(unsigned long long), cudaMemcpyDeviceToHost, cs);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(cs);
    if (ce != cudaSuccess) return fail(cuda_error(ce, "mask readback"));
    double ru = 0, su = 0;
    for (auto v : rm) ru += __builtin_popcountll(v);
    for (auto v : sm) su += __builtin_popcountll(v);
    m->rowk_used = ru;
    m->slabk_used = su;
    // the (row, node) pairs in use, for the scattering x-inverse pass
    std::vector<unsigned long long> items;
    items.reserve(size_t(ru));
    for (long r = 0; r < nrows; ++r)
      for (unsigned long long b = rm[r]; b; b &= b - 1)
        items.push_back((static_cast<unsigned long long>(r) << 8) |
                        static_cast<unsigned long long>(__builtin_ctzll(b)));
    m->nitems = long(items.size());
    if ((st = upload(m->arena, &m->rowitems, items, cs)) != HZ_OK) return fail(st);
  }

  // symbol constants A_k = w^2 + i w a_k, G_k = gamma_k^2
  std::vector<double2> A(m->K), G(m->K);
  std::vector<float2> Af(m->K), Gf(m->K);
  for (int k = 0; k < m->K; ++k) {
    A[k] = make_double2(omega * omega, omega * m->a_k[k]);
    const double gr = m->gamma_re[k], gi = m->gamma_im[k];
    G[k] = make_double2(gr * gr - gi * gi, 2.0 * gr * gi);
    Af[k] = make_float2(float(A[k].x), float(A[k].y));
    Gf[k] = make_float2(float(G[k].x), float(G[k].y));
  }
  if ((st = upload(m->arena, &m->symA64, A, cs)) != HZ_OK) return fail(st);
  if ((st = upload(m->arena, &m->symG64, G, cs)) != HZ_OK) return fail(st);
  if ((st = upload(m->arena, &m->symA32, Af, cs)) != HZ_OK) return fail(st);
  if ((st = upload(m->arena, &m->symG32, Gf, cs)) != HZ_OK) return fail(st);
  if (m->basis == 2 && m->M > 1) {
    std::vector<float> Df(m->K);
    for (int k = 0; k < m->K; ++k) Df[k] = float(m->dcoef[k]);
    if ((st = upload(m->arena, &m->symD64, m->dcoef, cs)) != HZ_OK) return fail(st);
    if ((st = upload(m->arena, &m->symD32, Df, cs)) != HZ_OK) return fail(st);
  }
  if ((st = upload(m->arena, &m->segtab, m->segtab_h, cs)) != HZ_OK) return fail(st);

  // per-axis tables
  const int nax[3] = {m->nx, m->ny, m->nz};
  for (int d = 0; d < m->dim; ++d) {
    const int N = nax[d];
    std::vector<double2> tw;
    std::vector<double> xi;
    twiddles(N, tw);
    xi2_table(N, m->L, interp->symbol_kind, xi);
    std::vector<float2> twf(N);
    std::vector<float4> twp(N);
    std::vector<float> xif(N);
    for (int j = 0; j < N; ++j) {
      twf[j] = make_float2(float(tw[j].x), float(tw[j].y));
      twp[j] = make_float4(twf[j].x, twf[j].x, twf[j].y, twf[j].y);
      xif[j] = float(xi[j]);
    }
    AxisTables& t = m->ax[d];
    t.N = N;
    if ((st = upload(m->arena, &t.tw64, tw, cs)) != HZ_OK) return fail(st);
    if ((st = upload(m->arena, &t.tw32, twf, cs)) != HZ_OK) return fail(st);
    if ((st = upload(m->arena, &t.tw32p, twp, cs)) != HZ_OK) return fail(st);
    if ((st = upload(m->arena, &t.xi2_64, xi, cs)) != HZ_OK) return fail(st);
    if ((st = upload(m->arena, &t.xi2_32, xif, cs)) != HZ_OK) return fail(st);
    const double h = m->L / N;
    m->inv_h2[d] = 1.0 / (h * h);
  }
  ce = cudaStreamSynchronize(cs);
  if (ce != cudaSuccess) return fail(cuda_error(ce, "create_medium"));
  *out = m;
  return HZ_OK;
}

extern "C" hz_status hz_medium_info(const hz_medium* med, int* K, int* M, int* Mt, double* gamma_re,
                                    double* gamma_im, double* a_k, double* c_min, double* c_max) {
  if (!med) return set_error(HZ_ERR_INVALID_ARG, "null medium");
  if (K) *K = med->K;
  if (M) *M = med->M;
  if (Mt) *Mt = med->Mt;
  for (int k = 0; k < med->K; ++k) {
    if (gamma_re) gamma_re[k] = med->gamma_re[k];
    if (gamma_im) gamma_im[k] = med->gamma_im[k];
    if (a_k) a_k[k] = med->a_k[k];
  }
  if (c_min) *c_min = med->c_min;
  if (c_max) *c_max = med->c_max;
  return HZ_OK;
}

extern "C" hz_status hz_destroy_medium(hz_medium* med) {
  if (!med) return HZ_OK;
  med->arena.release();
  delete med;
  return HZ_OK;
}
