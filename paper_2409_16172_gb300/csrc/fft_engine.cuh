// Shared-memory Stockham FFT engine for one line of length N per group of
// TPL threads, E = N / TPL complex elements per thread in registers.
//
// The transform convention is the discrete form of the symmetric Fourier
// pair (Section 2, Eqn. FT): forward X[k] = sum_j x[j] e^{-2 pi i jk/N}
// (sign -1), inverse with e^{+2 pi i jk/N} (sign +1) and no scaling; the 1/n
// of the inverse is applied once at the end of the preconditioner.
//
// Stage s has radix R and Ns = product of the earlier radices.  Butterfly j
// (0 <= j < N/R) reads x[j + r N/R], multiplies input r by w_{Ns R}^{r (j mod Ns)},
// runs an R-point DFT and writes y[(j / Ns) Ns R + (j mod Ns) + r Ns]; after
// the last stage the line is in natural order (mixed-radix Stockham autosort).
// Thread t of a line runs butterflies j = t + b TPL, b = 0 .. E/R - 1.
//
// Shared memory holds a line padded by one element every 16 elements (32 for
// plans with a radix-32 stage) so that the stride-R writes of the early
// stages spread over the banks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hz {

template <typename R> struct cvec;
template <> struct cvec<float> { using T = float2; };
template <> struct cvec<double> { using T = double2; };

template <typename V> __device__ __forceinline__ V cmk(decltype(V::x) a, decltype(V::x) b) {
  V r; r.x = a; r.y = b; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  return cmk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return cmk<V>(a.x * s, a.y * s); }
// multiply by S*i  (S = +1: i a, S = -1: -i a)
template <int S, typename V> __device__ __forceinline__ V cmul_si(V a) {
  return (S > 0) ? cmk<V>(-a.y, a.x) : cmk<V>(a.y, -a.x);
}

// Twiddle loads through the read-only path, kept where they are written: a
// kernel that runs several transforms per thread (one per node) would
// otherwise keep every twiddle of every stage live in registers across them.
__device__ __forceinline__ float2 ld_twiddle(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ double2 ld_twiddle(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}

// ---------------------------------------------------------------------------
// Small DFTs, X[m] = sum_n x[n] e^{S 2 pi i n m / R}, in place on x[0..R-1].
// ---------------------------------------------------------------------------
template <int S, typename V> __device__ __forceinline__ void dft2(V* x) {
  V a = x[0], b = x[1];
  x[0] = cadd(a, b); x[1] = csub(a, b);
}

template <int S, typename V> __device__ __forceinline__ void dft3(V* x) {
  using R = decltype(V::x);
  const R h = R(0.86602540378443864676);  // sin(2 pi / 3)
  V s = cadd(x[1], x[2]);
  V d = csub(x[1], x[2]);
  V t = cmk<V>(x[0].x - R(0.5) * s.x, x[0].y - R(0.5) * s.y);
  V e = cmul_si<S>(cscale(d, h));
  x[0] = cadd(x[0], s);
  x[1] = cadd(t, e);
  x[2] = csub(t, e);
}

// 5-point DFT from its definition, folded by the symmetry of the constants
// c_m = cos(2 pi m / 5), s_m = sin(2 pi m / 5): with t1 = x1 + x4,
// t2 = x2 + x3, t3 = x1 - x4, t4 = x2 - x3,
//   X0     = x0 + t1 + t2
//   X1, X4 = x0 + c1 t1 + c2 t2 +- S i (s1 t3 + s2 t4)
//   X2, X3 = x0 + c2 t1 + c1 t2 +- S i (s2 t3 - s1 t4)
template <int S, typename V> __device__ __forceinline__ void dft5(V* x) {
  using R = decltype(V::x);
  const R c1 = R(0.30901699437494742410), c2 = R(-0.80901699437494742410);
  const R s1 = R(0.95105651629515357212), s2 = R(0.58778525229247312917);
  const V t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
  const V t3 = csub(x[1], x[4]), t4 = csub(x[2], x[3]);
  const V a1 = cmk<V>(x[0].x + c1 * t1.x + c2 * t2.x, x[0].y + c1 * t1.y + c2 * t2.y);
  const V a2 = cmk<V>(x[0].x + c2 * t1.x + c1 * t2.x, x[0].y + c2 * t1.y + c1 * t2.y);
  const V b1 = cmul_si<S>(cmk<V>(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
  const V b2 = cmul_si<S>(cmk<V>(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
  x[0] = cadd(x[0], cadd(t1, t2));
  x[1] = cadd(a1, b1);
  x[4] = csub(a1, b1);
  x[2] = cadd(a2, b2);
  x[3] = csub(a2, b2);
}

template <int S, typename V> __device__ __forceinline__ void dft4(V* x) {
  V a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
  V c = cadd(x[1], x[3]), d = cmul_si<S>(csub(x[1], x[3]));
  x[0] = cadd(a, c); x[2] = csub(a, c);
  x[1] = cadd(b, d); x[3] = csub(b, d);
}

template <int S, typename V> __device__ __forceinline__ void dft8(V* x) {
  using R = decltype(V::x);
  const R r2 = R(0.70710678118654752440);
  V e[4] = {x[0], x[2], x[4], x[6]};
  V o[4] = {x[1], x[3], x[5], x[7]};
  dft4<S>(e);
  dft4<S>(o);
  // w8^1 = r2 (1 + S i), w8^2 = S i, w8^3 = r2 (-1 + S i)
  V o1 = cscale(cadd(o[1], cmul_si<S>(o[1])), r2);
  V o2 = cmul_si<S>(o[2]);
  V o3 = cscale(csub(cmul_si<S>(o[3]), o[3]), r2);
  x[0] = cadd(e[0], o[0]); x[4] = csub(e[0], o[0]);
  x[1] = cadd(e[1], o1);   x[5] = csub(e[1], o1);
  x[2] = cadd(e[2], o2);   x[6] = csub(e[2], o2);
  x[3] = cadd(e[3], o3);   x[7] = csub(e[3], o3);
}

// w16^m = cos(2 pi m / 16) + S i sin(2 pi m / 16)
template <int S, typename V> __device__ __forceinline__ V w16mul(V a, int m) {
  using R = decltype(V::x);
  const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173);
  const R r2 = R(0.70710678118654752440);
  R c, s;
  switch (m) {
    case 0: return a;
    case 1: c = c1; s = s1; break;
    case 2: c = r2; s = r2; break;
    case 3: c = s1; s = c1; break;
    case 4: return cmul_si<S>(a);
    case 6: c = -r2; s = r2; break;
    case 9: c = -c1; s = -s1; break;
    default: c = R(1); s = R(0); break;  // not reached for the 4x4 split
  }
  return cmul(a, cmk<V>(c, R(S) * s));
}

template <int S, typename V> __device__ __forceinline__ void dft16(V* x) {
  V y[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    V t[4] = {x[n2], x[n2 + 4], x[n2 + 8], x[n2 + 12]};
    dft4<S>(t);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) y[n2 * 4 + k1] = w16mul<S>(t[k1], n2 * k1);
  }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    V t[4] = {y[k1], y[4 + k1], y[8 + k1], y[12 + k1]};
    dft4<S>(t);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = t[k2];
  }
}

// w32^k = cos(2 pi k / 32) + S i sin(2 pi k / 32), k = 0..15
template <int S, typename V> __device__ __forceinline__ V w32mul(V a, int k) {
  using R = decltype(V::x);
  constexpr double C[8] = {1.0,
                           0.980785280403230449126182, 0.923879532511286756128183,
                           0.831469612302545237078788, 0.707106781186547524400844,
                           0.555570233019602224742831, 0.382683432365089771728460,
                           0.195090322016128267848285};
  if (k == 0) return a;
  if (k == 8) return cmul_si<S>(a);
  if (k < 8) return cmul(a, cmk<V>(R(C[k]), R(S) * R(C[8 - k])));
  // w^(8 + m) = S i w^m
  return cmul_si<S>(cmul(a, cmk<V>(R(C[k - 8]), R(S) * R(C[16 - k]))));
}

// 32-point DFT as two 16-point DFTs of the even and odd samples.
template <int S, typename V> __device__ __forceinline__ void dft32(V* x) {
  V e[16], o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    e[i] = x[2 * i];
    o[i] = x[2 * i + 1];
  }
  dft16<S>(e);
  dft16<S>(o);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const V t = w32mul<S>(o[k], k);
    x[k] = cadd(e[k], t);
    x[k + 16] = csub(e[k], t);
  }
}

// Twiddle multiply of the Stockham stages: x * w (forward, S = -1) or
// x * conj(w) (inverse, S = +1), w = exp(-2 pi i m / N) from the table.
template <typename V> struct TwiddleOf { using T = V; };
template <int S, typename V> __device__ __forceinline__ V twiddle_mul(V a, V w) {
  return S > 0 ? cmulc(a, w) : cmul(a, w);
}

// ---------------------------------------------------------------------------
// Paired complex FP32: two independent lines transformed by one thread.  PV
// holds the real parts of the two lines' values in x and the imaginary parts
// in y, each an f32x2 pair, so that every butterfly add, subtract and multiply
// is one packed FP32 instruction (PTX add/sub/mul/fma.rn.f32x2) for both
// lines.
// ---------------------------------------------------------------------------
struct __align__(8) f2 {
  unsigned long long v;
};
__device__ __forceinline__ f2 f2_make(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ f2 f2_splat(float a) { return f2_make(a, a); }
__device__ __forceinline__ float f2_lo(f2 p) { return __uint_as_float(unsigned(p.v)); }
__device__ __forceinline__ float f2_hi(f2 p) { return __uint_as_float(unsigned(p.v >> 32)); }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {  // a b + c
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ f2 neg2(f2 a) { return f2_splat(0.0f) - a; }

struct __align__(16) PV {
  f2 x, y;
};
// twiddles for pairs: (re, re, im, im) of exp(-2 pi i m / N)
template <> struct TwiddleOf<PV> { using T = float4; };
__device__ __forceinline__ float4 ld_twiddle(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
template <int S> __device__ __forceinline__ PV twiddle_mul(PV a, float4 w) {
  const f2 wr = f2_make(w.x, w.y), wi = f2_make(w.z, w.w);
  PV r;
  if constexpr (S > 0) {  // a conj(w)
    r.x = fma2(a.y, wi, a.x * wr);
    r.y = a.y * wr - a.x * wi;
  } else {  // a w
    r.x = a.x * wr - a.y * wi;
    r.y = fma2(a.x, wi, a.y * wr);
  }
  return r;
}
__device__ __forceinline__ PV cmul(PV a, PV b) {
  PV r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = fma2(a.x, b.y, a.y * b.x);
  return r;
}
__device__ __forceinline__ PV cmulc(PV a, PV b) {  // a conj(b)
  PV r;
  r.x = fma2(a.x, b.x, a.y * b.y);
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
// a (c + i s) for constants c, s
__device__ __forceinline__ PV cmul_const(PV a, float c, float s) {
  const f2 C = f2_splat(c), Sv = f2_splat(s), NS = f2_splat(-s);
  PV r;
  r.x = fma2(a.y, NS, a.x * C);
  r.y = fma2(a.x, Sv, a.y * C);
  return r;
}
template <int S> __device__ __forceinline__ PV cmul_si(PV a) {
  PV r;
  if constexpr (S > 0) { r.x = neg2(a.y); r.y = a.x; }
  else { r.x = a.y; r.y = neg2(a.x); }
  return r;
}
// b + S i e and b - S i e without forming S i e
template <int S> __device__ __forceinline__ PV cadd_si(PV b, PV e) {
  PV r;
  if constexpr (S > 0) { r.x = b.x - e.y; r.y = b.y + e.x; }
  else { r.x = b.x + e.y; r.y = b.y - e.x; }
  return r;
}
template <int S> __device__ __forceinline__ PV csub_si(PV b, PV e) {
  PV r;
  if constexpr (S > 0) { r.x = b.x + e.y; r.y = b.y - e.x; }
  else { r.x = b.x - e.y; r.y = b.y + e.x; }
  return r;
}

template <int S> __device__ __forceinline__ void dft3(PV* x) {
  const float h = 0.86602540378443864676f;  // sin(2 pi / 3)
  const PV s = cadd(x[1], x[2]), d = csub(x[1], x[2]);
  const f2 mh = f2_splat(-0.5f);
  PV t;
  t.x = fma2(s.x, mh, x[0].x);
  t.y = fma2(s.y, mh, x[0].y);
  // e = S i h d:  x1 = t + e, x2 = t - e
  const f2 pH = f2_splat(float(S) * h), nH = f2_splat(-float(S) * h);
  x[0] = cadd(x[0], s);
  PV a, b;
  a.x = fma2(d.y, nH, t.x);
  a.y = fma2(d.x, pH, t.y);
  b.x = fma2(d.y, pH, t.x);
  b.y = fma2(d.x, nH, t.y);
  x[1] = a;
  x[2] = b;
}

template <int S> __device__ __forceinline__ void dft4(PV* x) {
  const PV a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
  const PV c = cadd(x[1], x[3]), e = csub(x[1], x[3]);
  x[0] = cadd(a, c);
  x[2] = csub(a, c);
  x[1] = cadd_si<S>(b, e);
  x[3] = csub_si<S>(b, e);
}

template <int S> __device__ __forceinline__ void dft8(PV* x) {
  const float r2 = 0.70710678118654752440f;
  PV e[4] = {x[0], x[2], x[4], x[6]};
  PV o[4] = {x[1], x[3], x[5], x[7]};
  dft4<S>(e);
  dft4<S>(o);
  const f2 R2 = f2_splat(r2), NR2 = f2_splat(-r2);
  // o1 w8^1 = r2 (o1 + S i o1); o3 w8^3 = r2 (S i o3 - o3)
  PV o1, o3;
  if constexpr (S > 0) {
    o1.x = (o[1].x - o[1].y) * R2;
    o1.y = (o[1].y + o[1].x) * R2;
    o3.x = (o[3].x + o[3].y) * NR2;
    o3.y = (o[3].x - o[3].y) * R2;
  } else {
    o1.x = (o[1].x + o[1].y) * R2;
    o1.y = (o[1].y - o[1].x) * R2;
    o3.x = (o[3].y - o[3].x) * R2;
    o3.y = (o[3].x + o[3].y) * NR2;
  }
  x[0] = cadd(e[0], o[0]); x[4] = csub(e[0], o[0]);
  x[1] = cadd(e[1], o1);   x[5] = csub(e[1], o1);
  x[2] = cadd_si<S>(e[2], o[2]); x[6] = csub_si<S>(e[2], o[2]);
  x[3] = cadd(e[3], o3);   x[7] = csub(e[3], o3);
}

template <int S> __device__ __forceinline__ PV w16mul(PV a, int m) {
  const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
  const float r2 = 0.70710678118654752440f;
  switch (m) {
    case 0: return a;
    case 1: return cmul_const(a, c1, float(S) * s1);
    case 2: return cmul_const(a, r2, float(S) * r2);
    case 3: return cmul_const(a, s1, float(S) * c1);
    case 4: return cmul_si<S>(a);
    case 6: return cmul_const(a, -r2, float(S) * r2);
    case 9: return cmul_const(a, -c1, -float(S) * s1);
    default: return a;  // not reached for the 4x4 split
  }
}

template <int S> __device__ __forceinline__ PV w32mul(PV a, int k) {
  constexpr double C[9] = {1.0,
                           0.980785280403230449126182, 0.923879532511286756128183,
                           0.831469612302545237078788, 0.707106781186547524400844,
                           0.555570233019602224742831, 0.382683432365089771728460,
                           0.195090322016128267848285, 0.0};
  if (k == 0) return a;
  if (k == 8) return cmul_si<S>(a);
  if (k < 8) return cmul_const(a, float(C[k]), float(S) * float(C[8 - k]));
  // w^k = S i w^(k-8): (c + i S s) S i = -s' + i S c' with c' = C[k-8], s' = C[16-k]
  return cmul_const(a, -float(C[16 - k]), float(S) * float(C[k - 8]));
}

template <int S> __device__ __forceinline__ void dft5(PV* x) {
  const f2 C1 = f2_splat(0.30901699437494742410f), C2 = f2_splat(-0.80901699437494742410f);
  const f2 S1 = f2_splat(0.95105651629515357212f), S2 = f2_splat(0.58778525229247312917f);
  const f2 NS1 = f2_splat(-0.95105651629515357212f);
  const PV t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
  const PV t3 = csub(x[1], x[4]), t4 = csub(x[2], x[3]);
  PV a1, a2, u1, u2;
  a1.x = fma2(t1.x, C1, fma2(t2.x, C2, x[0].x));
  a1.y = fma2(t1.y, C1, fma2(t2.y, C2, x[0].y));
  a2.x = fma2(t1.x, C2, fma2(t2.x, C1, x[0].x));
  a2.y = fma2(t1.y, C2, fma2(t2.y, C1, x[0].y));
  u1.x = fma2(t3.x, S1, t4.x * S2);
  u1.y = fma2(t3.y, S1, t4.y * S2);
  u2.x = fma2(t4.x, NS1, t3.x * S2);
  u2.y = fma2(t4.y, NS1, t3.y * S2);
  x[0] = cadd(x[0], cadd(t1, t2));
  x[1] = cadd_si<S>(a1, u1);
  x[4] = csub_si<S>(a1, u1);
  x[2] = cadd_si<S>(a2, u2);
  x[3] = csub_si<S>(a2, u2);
}

// cos and sin of 2 pi m / RR for the in-radix twiddles of the composite
// radices below (RR = 6, 10, 12, 15, 20; 0 <= m < RR)
__host__ __device__ constexpr double wr_cos(int RR, int m) {
  return RR == 6    ? (m == 0 ? 1.0 : (m == 1 || m == 5) ? 0.5 : (m == 3 ? -1.0 : -0.5))
         : RR == 10 ? (m == 0 ? 1.0 : m == 5 ? -1.0
                       : (m == 1 || m == 9) ? 0.80901699437494742410
                       : (m == 2 || m == 8) ? 0.30901699437494742410
                       : (m == 3 || m == 7) ? -0.30901699437494742410 : -0.80901699437494742410)
                    : 0.0;
}
__host__ __device__ constexpr double wr_sin(int RR, int m) {
  return RR == 6    ? (m == 0 || m == 3 ? 0.0 : m < 3 ? 0.86602540378443864676 : -0.86602540378443864676)
         : RR == 10 ? (m == 0 || m == 5 ? 0.0
                       : (m == 1 || m == 4) ? 0.58778525229247312917
                       : (m == 2 || m == 3) ? 0.95105651629515357212
                       : (m == 6 || m == 9) ? -0.58778525229247312917 : -0.95105651629515357212)
                    : 0.0;
}
// a * exp(S 2 pi i m / RR)
template <int RR, int S, typename V> __device__ __forceinline__ V wrmul(V a, int m) {
  using R = decltype(V::x);
  m %= RR;
  if (m == 0) return a;
  if (4 * m == RR) return cmul_si<S>(a);
  if (2 * m == RR) return cmk<V>(-a.x, -a.y);
  if (4 * m == 3 * RR) return cmul_si<-S>(a);
  return cmul(a, cmk<V>(R(wr_cos(RR, m)), R(S) * R(wr_sin(RR, m))));
}
template <int RR, int S> __device__ __forceinline__ PV wrmul(PV a, int m) {
  m %= RR;
  if (m == 0) return a;
  if (4 * m == RR) return cmul_si<S>(a);
  if (2 * m == RR) return cmk<PV>(neg2(a.x), neg2(a.y));
  if (4 * m == 3 * RR) return cmul_si<-S>(a);
  return cmul_const(a, float(wr_cos(RR, m)), float(S) * float(wr_sin(RR, m)));
}

template <int RAD, int S, typename V> __device__ __forceinline__ void dftR(V* x);

// Composite radix R1 R2 by one Cooley-Tukey split: with n = n2 + R2 n1 and
// k = k1 + R1 k2, X[k] = sum_n2 w_{R1R2}^{n2 k1} (sum_n1 x[n] w_{R1}^{n1 k1})
// w_{R2}^{n2 k2}: R2 DFTs of length R1, the twiddles, then R1 of length R2.
template <int R1, int R2, int S, typename V> __device__ __forceinline__ void dft_split(V* x) {
  constexpr int RR = R1 * R2;
  V y[RR];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    V t[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) t[n1] = x[n2 + R2 * n1];
    dftR<R1, S>(t);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) y[n2 * R1 + k1] = wrmul<RR, S>(t[k1], n2 * k1);
  }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    V t[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) t[n2] = y[n2 * R1 + k1];
    dftR<R2, S>(t);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) x[k1 + R1 * k2] = t[k2];
  }
}

template <int RAD, int S, typename V> __device__ __forceinline__ void dftR(V* x) {
  if constexpr (RAD == 2) dft2<S>(x);
  else if constexpr (RAD == 3) dft3<S>(x);
  else if constexpr (RAD == 4) dft4<S>(x);
  else if constexpr (RAD == 5) dft5<S>(x);
  else if constexpr (RAD == 6) dft_split<2, 3, S>(x);
  else if constexpr (RAD == 8) dft8<S>(x);
  else if constexpr (RAD == 10) dft_split<2, 5, S>(x);
  else if constexpr (RAD == 16) dft16<S>(x);
  else if constexpr (RAD == 32) dft32<S>(x);
  else static_assert(RAD == 2, "unsupported radix");
}

// ---------------------------------------------------------------------------
// Radix plans: N = prod(radices); E is a multiple of every radix.
// ---------------------------------------------------------------------------
template <int N> struct FftPlan;
#define HZ_PLAN(NN, EE, ...) HZ_PLAN_T(FftPlan<NN>, NN, EE, __VA_ARGS__)
#define HZ_PLAN_T(NAME, NN, EE, ...)                                       \
  template <> struct NAME {                                                \
    static constexpr int E = EE;                                           \
    static constexpr int rads[] = {__VA_ARGS__};                           \
    static constexpr int NST = sizeof(rads) / sizeof(int);                 \
    __host__ __device__ static constexpr int rad(int s) { return rads[s]; } \
  };
HZ_PLAN(8, 8, 8)
HZ_PLAN(12, 12, 4, 3)
HZ_PLAN(16, 16, 16)
HZ_PLAN(24, 24, 8, 3)
HZ_PLAN(32, 8, 8, 4)
HZ_PLAN(48, 12, 4, 4, 3)
HZ_PLAN(64, 8, 8, 8)
HZ_PLAN(96, 24, 8, 4, 3)
HZ_PLAN(128, 16, 16, 8)
HZ_PLAN(192, 24, 8, 8, 3)
HZ_PLAN(256, 16, 16, 16)
HZ_PLAN(512, 8, 8, 8, 8)
HZ_PLAN(1024, 16, 16, 16, 4)
HZ_PLAN(2048, 16, 16, 16, 8)
// Lengths with a factor 5 (the grids of the paper's Example 1 and Tables
// 1-2): radices 10, 6 (and 2, 3) so that 30 elements per thread are a
// multiple of every radix (10 for the lengths without a factor 3)
HZ_PLAN(20, 10, 10, 2)
HZ_PLAN(40, 10, 10, 2, 2)
HZ_PLAN(60, 30, 10, 6)
HZ_PLAN(120, 30, 10, 6, 2)
HZ_PLAN(180, 30, 10, 6, 3)
HZ_PLAN(240, 30, 10, 6, 2, 2)
HZ_PLAN(360, 30, 10, 6, 6)
HZ_PLAN(480, 30, 10, 6, 2, 2, 2)
HZ_PLAN(720, 30, 10, 6, 6, 2)
HZ_PLAN(960, 30, 10, 6, 2, 2, 2, 2)
HZ_PLAN(1440, 30, 10, 6, 6, 2, 2)
HZ_PLAN(1920, 30, 10, 6, 2, 2, 2, 2, 2)
HZ_PLAN(2400, 30, 10, 10, 6, 2, 2)
HZ_PLAN(2880, 30, 10, 6, 6, 2, 2, 2)
HZ_PLAN(3600, 30, 10, 10, 6, 6)
HZ_PLAN(4800, 30, 10, 10, 6, 2, 2, 2)

// Row plans (contiguous lines, complex64): 32 threads per line for N = 512
// and 1024 so that a line is one warp and its stage barriers are warp
// barriers.  Other lengths and complex128 use the plans above.
template <typename R, int N> struct RowPlan { using P = FftPlan<N>; };
template <int N> struct FftPlanW;
HZ_PLAN_T(FftPlanW<512>, 512, 16, 16, 16, 2)
HZ_PLAN_T(FftPlanW<1024>, 1024, 32, 32, 32)
template <> struct RowPlan<float, 512> { using P = FftPlanW<512>; };
template <> struct RowPlan<float, 1024> { using P = FftPlanW<1024>; };

// Strided-axis (column) kernels use FftPlan, except as below.
template <typename R, int N> struct ColPlan { using P = FftPlan<N>; };
// complex64 columns of 512: three stages (16, 16, 2) instead of four radix-8
// stages, one shared-memory exchange fewer
template <> struct ColPlan<float, 512> { using P = FftPlanW<512>; };
// The paired complex64 symbol pass: the column plan, except two radix-32
// stages (32 pairs per thread) for 1024.
template <typename R, int N> struct PairPlan { using P = typename ColPlan<R, N>::P; };
template <> struct PairPlan<float, 1024> { using P = FftPlanW<1024>; };

// FP64 lines up to 256 points: radix-4 (and 2, 3) stages with 4 or 12
// elements per thread.  An FP64 instruction occupies a sub-partition's FP64
// unit for many cycles on this part, so a short line is transformed by more
// threads with shorter per-thread chains; the extra stages cost shared
// memory traffic, not FP64 work.
template <int N> struct FftPlanD;
HZ_PLAN_T(FftPlanD<8>, 8, 4, 4, 2)
HZ_PLAN_T(FftPlanD<16>, 16, 4, 4, 4)
HZ_PLAN_T(FftPlanD<24>, 24, 12, 4, 2, 3)
HZ_PLAN_T(FftPlanD<32>, 32, 4, 4, 4, 2)
HZ_PLAN_T(FftPlanD<64>, 64, 4, 4, 4, 4)
HZ_PLAN_T(FftPlanD<96>, 96, 12, 4, 4, 2, 3)
HZ_PLAN_T(FftPlanD<128>, 128, 4, 4, 4, 4, 2)
HZ_PLAN_T(FftPlanD<192>, 192, 12, 4, 4, 4, 3)
HZ_PLAN_T(FftPlanD<256>, 256, 4, 4, 4, 4, 4)
#define HZ_DPLAN(NN)                                                       \
  template <> struct RowPlan<double, NN> { using P = FftPlanD<NN>; };      \
  template <> struct ColPlan<double, NN> { using P = FftPlanD<NN>; };
HZ_DPLAN(8)
HZ_DPLAN(16)
HZ_DPLAN(24)
HZ_DPLAN(32)
HZ_DPLAN(64)
HZ_DPLAN(96)
HZ_DPLAN(128)
HZ_DPLAN(192)
HZ_DPLAN(256)
#undef HZ_DPLAN
#undef HZ_PLAN
#undef HZ_PLAN_T

constexpr int PAD_SHIFT = 4;
// shared-memory elements of one padded line (enough for either padding)
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> PAD_SHIFT) + 1; }

// LS: distance in elements between consecutive positions of a line in shared
// memory (1 for a private line, TB when TB lines are interleaved).
// WS: the threads of a line lie in one warp (TPL <= 32 and lines laid out
// warp by warp), so the stage barriers are warp barriers.
template <typename R, int N, int S, int LS = 1, bool WS = false, typename PL = FftPlan<N>,
          typename VT = typename cvec<R>::T>
struct LineFFT {
  using V = VT;                        // one complex value, or a pair (PV)
  using TW = typename TwiddleOf<V>::T;  // twiddle table entry
  using P = PL;
  static constexpr int E = P::E;
  static constexpr int TPL = N / E;
  static constexpr int R0 = P::rad(0);
  // shared-memory padding: one element per 16, or per 32 for plans with a
  // radix-32 stage, whose stride-32 writes would otherwise put every eighth
  // lane on the same banks (padded_len(N) covers both)
  static constexpr int max_rad() {
    int m = 0;
    for (int s = 0; s < P::NST; ++s) m = P::rad(s) > m ? P::rad(s) : m;
    return m;
  }
  static constexpr int PS = max_rad() >= 32 ? 5 : PAD_SHIFT;
  __device__ static __forceinline__ int pad(int i) { return i + (i >> PS); }
  // For i >= 0 and a step m that is a multiple of 2^PS, pad(i + r m) =
  // pad(i) + r padstep(m): the addresses of a stage's elements are then one
  // per-thread base plus compile-time offsets.
  static constexpr bool affine(int m) { return m % (1 << PS) == 0; }
  static constexpr int padstep(int m) { return m + (m >> PS); }
  static_assert(!WS || TPL <= 32, "warp-synchronous lines need TPL <= 32");

  // lanes of the warp that exist: a block smaller than a warp holds lanes
  // 0 .. blockDim.x - 1 only
  __device__ static __forceinline__ unsigned lane_mask() {
    return blockDim.x >= 32 ? 0xffffffffu : ((1u << blockDim.x) - 1u);
  }
  __device__ static __forceinline__ void sync() {
    if constexpr (WS) __syncwarp(lane_mask());
    else __syncthreads();
  }

  // Frequency / position index held in x[e] before stage 0 (the stage-0
  // read pattern): b = e / R0, r = e % R0, j = t + b TPL, index = j + r N/R0.
  __device__ static __forceinline__ int stage0_index(int t, int e) {
    return (t + (e / R0) * TPL) + (e % R0) * (N / R0);
  }

  __device__ static __forceinline__ void load_stage0(const V* line, int t, V (&x)[E]) {
    if constexpr (affine(TPL) && affine(N / R0)) {
      const int pt = pad(t);
#pragma unroll
      for (int e = 0; e < E; ++e)
        x[e] = line[(pt + (e / R0) * padstep(TPL) + (e % R0) * padstep(N / R0)) * LS];
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) x[e] = line[pad(stage0_index(t, e)) * LS];
    }
  }

  template <int STAGE, int NS, bool KEEP>
  __device__ static __forceinline__ void stage(V* line, int t, V (&x)[E], const TW* __restrict__ tw) {
    if constexpr (STAGE < P::NST) {
      constexpr int RAD = P::rad(STAGE);
      if constexpr (STAGE > 0) {
#pragma unroll
        for (int b = 0; b < E / RAD; ++b) {
          const int j = t + b * TPL;
          if constexpr (affine(N / RAD)) {
            const int pj = affine(TPL) ? pad(t) + b * padstep(TPL) : pad(j);
#pragma unroll
            for (int r = 0; r < RAD; ++r) x[b * RAD + r] = line[(pj + r * padstep(N / RAD)) * LS];
          } else {
#pragma unroll
            for (int r = 0; r < RAD; ++r) x[b * RAD + r] = line[pad(j + r * (N / RAD)) * LS];
          }
        }
        sync();
      }
#pragma unroll
      for (int b = 0; b < E / RAD; ++b) {
        const int j = t + b * TPL;
        const int k = j % NS;
        if constexpr (NS > 1) {
#pragma unroll
          for (int r = 1; r < RAD; ++r) {
            x[b * RAD + r] = twiddle_mul<S>(x[b * RAD + r], ld_twiddle(&tw[r * k * (N / (NS * RAD))]));
          }
        }
        dftR<RAD, S>(&x[b * RAD]);
        if constexpr (!(KEEP && STAGE == P::NST - 1)) {
          const int d = (j / NS) * NS * RAD + k;
          if constexpr (affine(NS)) {
            const int pd = pad(d);
#pragma unroll
            for (int r = 0; r < RAD; ++r) line[(pd + r * padstep(NS)) * LS] = x[b * RAD + r];
          } else {
#pragma unroll
            for (int r = 0; r < RAD; ++r) line[pad(d + r * NS) * LS] = x[b * RAD + r];
          }
        }
      }
      if constexpr (!(KEEP && STAGE == P::NST - 1)) sync();
      stage<STAGE + 1, NS * RAD, KEEP>(line, t, x, tw);
    }
  }

  // Runs the whole transform.  On entry x holds the stage-0 inputs and every
  // thread of the line has finished reading it (the caller syncs).  On exit
  // the line holds the result in natural order and the line's threads (the
  // block, unless WS) are synchronised.  tw[i] = exp(-2 pi i * i / N) for i < N.
  __device__ static __forceinline__ void run(V* line, int t, V (&x)[E], const TW* __restrict__ tw) {
    stage<0, 1, false>(line, t, x, tw);
  }

  // Same transform, but the last stage leaves its outputs in registers:
  // x[e] holds output position out_index(t, e).  The line's shared memory is
  // free again on return (the last stage's reads are behind a barrier), so
  // the next transform on the same line needs no barrier of the caller.
  static constexpr int RL = P::rad(P::NST - 1);
  __device__ static __forceinline__ int out_index(int t, int e) {
    return t + (e / RL) * TPL + (e % RL) * (N / RL);
  }
  __device__ static __forceinline__ void run_regs(V* line, int t, V (&x)[E], const TW* __restrict__ tw) {
    stage<0, 1, true>(line, t, x, tw);
  }
};

}  // namespace hz
