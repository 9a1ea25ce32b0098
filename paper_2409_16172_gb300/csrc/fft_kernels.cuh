// FFT pass kernels of the preconditioner apply Q_M v (Eqn. 103 / 403):
//
//   row_fwd       forward FFT along x of the input vector (c128 in, scaled by
//                 the Krylov normalisation, rounded to the working precision;
//                 optionally clears the rows of the scattering pass's output)
//   line_pass     forward or inverse FFT along a strided axis (y, and z in 3D)
//   line_sym_inv  last axis, one block per (column tile, group of 1/2/4 nodes):
//                 read vhat, multiply by q_k(|xi|^2) =
//                 1 / (w^2 + i w a_k - gamma_k^2 |xi|^2) (Eqn. 021, recomputed,
//                 never stored), inverse FFT along the axis, write plane k on
//                 the rows / slabs that use node k; complex64 also with two
//                 columns per thread in packed f32x2 arithmetic
//   row_inv_acc   inverse FFT along x of every plane a row needs, then the
//                 weighted sum z = (1/n) sum_k w_k(x) plane_k(x) (Eqn. 405:
//                 two non-zero hat weights per point); or an in-place
//                 inverse of every used (row, node) line and a gather (also
//                 the 4-weight gather of the bivariate / quadratic records);
//                 or one line per used (row, node) adding its weighted
//                 result into an output cleared by row_fwd (row_inv_scatter)
//
// Layout: vectors [rhs][z][y][x] (x fastest); planes [rhs][k][z][y][x].
// Every kernel reads its inputs straight into registers in the transform's
// first-stage order, exchanges through padded shared memory between stages
// (Stockham engine of fft_engine.cuh) and writes from registers after the
// last stage; global accesses are coalesced along x (rows directly, strided
// axes in tiles of TB adjacent columns whose lines are interleaved in shared
// memory).  Every kernel begins with pdl_wait() (programmatic dependent
// launch).
#pragma once
#include "fft_engine.cuh"
#include "hz_internal.h"

#include <type_traits>

namespace hz {

// Launch shapes.  Row kernels: ROW_THREADS threads, ROW_THREADS / TPL lines.
// Strided kernels: TB adjacent columns x TPL threads, TB chosen so that a
// block moves at least 64 contiguous bytes per row, has >= 128 threads, at
// most 512, and its shared memory stays under ~200 KB.
template <typename R, int N> struct LineCfg {
  using CP = typename ColPlan<R, N>::P;           // strided kernels
  static constexpr int TPL = N / CP::E;
  using RP = typename RowPlan<R, N>::P;           // row kernels
  static constexpr int TPL_ROW = N / RP::E;
  // whole lines per block: about 128 threads, at least one line
  static constexpr int ROW_LINES = TPL_ROW >= 128 ? 1 : 128 / TPL_ROW;
  static constexpr int ROW_THREADS = ROW_LINES * TPL_ROW;
  // row kernels: a line's threads sit in one warp (TPL_ROW divides 32, so
  // no line straddles two warps) -> warp barriers
  static constexpr bool WS = TPL_ROW <= 32 && 32 % TPL_ROW == 0;
  static constexpr int VB = int(2 * sizeof(R));
  static constexpr int tb_calc() {
    int tb = 32 / VB;                 // one 32-byte sector per row at least
    if (tb < 1) tb = 1;
    if (tb * TPL < 128) tb = 128 / TPL;
    while (tb > 1 && tb * TPL > 256) tb /= 2;
    while (tb > 1 && long(tb) * padded_len(N) * VB > 100 * 1024) tb /= 2;
    return tb;
  }
  static constexpr int TB = tb_calc();
  static constexpr int COL_THREADS = TB * TPL;
  static constexpr size_t row_smem(int lines = ROW_LINES) { return size_t(lines) * padded_len(N) * VB; }
  // row_inv_acc: padded work lines, then (16-byte aligned for cp.async) two
  // unpadded staging rows per line
  static constexpr size_t stage_offset(int lines = ROW_LINES) { return (row_smem(lines) + 15) / 16 * 16; }
  static constexpr size_t row_acc_smem(int lines = ROW_LINES) {
    return stage_offset(lines) + size_t(lines) * 2 * N * VB;
  }
  static constexpr size_t col_smem() { return size_t(TB) * padded_len(N) * VB; }
  static constexpr size_t col_pair_smem(int tb) { return size_t(tb) * padded_len(N) * 16; }
  // The paired complex64 symbol pass.  One-node blocks use PairPlan (two
  // radix-32 stages for columns of 1024), blocks of several nodes, which keep
  // the spectrum across nodes, the column plan.  tb_p column pairs per block
  // (>= 128 threads), or half as many; one-node blocks aim at 512 resident
  // threads per SM, 384 when a thread holds 32 pairs.
  template <int KPB>
  using PPK = typename std::conditional<KPB == 1, typename PairPlan<R, N>::P, CP>::type;
  template <int KPB> static constexpr int tpl_p() { return N / PPK<KPB>::E; }
  template <int KPB> static constexpr int tb_p() {
    return tpl_p<KPB>() == TPL ? TB : (tpl_p<KPB>() >= 128 ? 1 : 128 / tpl_p<KPB>());
  }
  template <int KPB> static constexpr int tb_p_half() { return tb_p<KPB>() > 1 ? tb_p<KPB>() / 2 : 1; }
  template <int KPB> static constexpr int pair_min_blocks(int tb) {
    return KPB > 1 ? 1
                   : (PPK<KPB>::E >= 32 ? (tb * tpl_p<KPB>() >= 384 ? 1 : 384 / (tb * tpl_p<KPB>()))
                                        : (tb * tpl_p<KPB>() >= 512 ? 1 : 512 / (tb * tpl_p<KPB>())));
  }
};

// 16-byte asynchronous global -> shared copies (L2 only), in groups.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = unsigned(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Per-point interpolation record, complex64 path: segment in the top 8 bits,
// t in [0, 1) as a 24-bit fraction.  The segment table maps a segment to
// (k_lo, k_hi); w_{k_lo} = 1 - t, w_{k_hi} = t.
__device__ __forceinline__ void decode_rec(uint32_t rec, int& seg, float& t) {
  seg = int(rec >> 24);
  t = float(rec & 0xFFFFFFu) * (1.0f / 16777216.0f);
}
__device__ __forceinline__ void decode_rec(double rec, int& seg, double& t) {
  seg = int(rec);
  t = rec - double(seg);
}

// Nodes per block of the symbol pass: 1, 2 or 4 (compiled variants).
constexpr int SYM_KPB_MAX = 4;

// 1/x for the symbol.  FP32: one MUFU reciprocal (PTX rcp.approx, at most
// 1 ulp).
__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// FP64: the MUFU approximation refined by three Newton-Raphson steps for
// 1/x, r <- r + r (1 - x r), each of which doubles the number of correct bits.
__device__ __forceinline__ double recip(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
#pragma unroll
  for (int it = 0; it < 3; ++it) r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

template <typename R> struct RecT;
template <> struct RecT<float> { using T = uint32_t; };
template <> struct RecT<double> { using T = double; };

// Per-point (node, weight) records of the bivariate and quadratic forms:
// gnode[p] holds up to four node indices (0xFF: unused slot) and gw their
// weights, one float4 (complex64 path) or two double2 (complex128) per point.
template <typename R> struct GwT;
template <> struct GwT<float> { using T = float4; };
template <> struct GwT<double> { using T = double2; };
__device__ __forceinline__ void load_gw(const float4* gw, long p, float (&w)[4]) {
  const float4 v = gw[p];
  w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
}
__device__ __forceinline__ void load_gw(const double2* gw, long p, double (&w)[4]) {
  const double2 u = gw[2 * p], v = gw[2 * p + 1];
  w[0] = u.x; w[1] = u.y; w[2] = v.x; w[3] = v.y;
}

// ---------------------------------------------------------------------------
// Forward FFT along x.  in: c128 rows (row gr at gr * N); scale[rhs] (or
// NULL) multiplies the input; out: working-precision rows.  zero (or NULL):
// rows of zchunks 16-byte chunks cleared for every row transformed (the
// output of the scattering x-inverse pass of the same apply; it may alias in).
// ---------------------------------------------------------------------------
template <typename R, int N, int LPB>
__global__ void __launch_bounds__(LPB * LineCfg<R, N>::TPL_ROW)
row_fwd_kernel(const double2* __restrict__ in, const double* __restrict__ scale,
               long rows_per_rhs, long nrows, const typename cvec<R>::T* __restrict__ tw,
               typename cvec<R>::T* __restrict__ out, const int* __restrict__ active,
               uint4* zero, int zchunks) {
  pdl_wait();
  using V = typename cvec<R>::T;
  using F = LineFFT<R, N, -1, 1, LineCfg<R, N>::WS, typename LineCfg<R, N>::RP>;
  constexpr int TPL = F::TPL, E = F::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  const int li = threadIdx.x / TPL, t = threadIdx.x % TPL;
  const long row = long(blockIdx.x) * LPB + li;
  // rows of retired right-hand sides (active[rhs] == 0) are skipped
  const bool valid = row < nrows && (!active || active[row / rows_per_rhs]);
  V* line = sm + li * padded_len(N);
  V x[E];
  // the Krylov scale is applied after rounding to the working precision
  R s = R(1);
  if (valid && scale) s = R(scale[row / rows_per_rhs]);
  const double2* src = in + row * N;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    double2 v = valid ? src[F::stage0_index(t, e)] : make_double2(0.0, 0.0);
    x[e] = cmk<V>(R(v.x) * s, R(v.y) * s);
  }
  F::run_regs(line, t, x, tw);
  if (valid) {
    V* dst = out + row * N;
#pragma unroll
    for (int e = 0; e < E; ++e) dst[F::out_index(t, e)] = x[e];
    // every thread of the line has read its input (the transform's first
    // barrier is behind the loads), so an aliased row may be cleared now
    if (zero) {
      uint4* z = zero + row * zchunks;
      for (int c = t; c < zchunks; c += TPL) z[c] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

// ---------------------------------------------------------------------------
// Inverse FFT along x of the K planes and the weighted sum.
// planes: [rhs][K][n]; rec: per-point record (shared by all rhs); segtab:
// (k_lo, k_hi) per segment; rowmask[row % rows_per_rhs] bit k = some point of
// the row has a non-zero weight on node k (only those planes were written).
// out[rhs][n] = inv_n * sum_k w_k plane_k.  The block walks the planes its
// rows need; the next plane's rows are copied into a shared staging buffer
// with cp.async while the current plane is transformed.
// ---------------------------------------------------------------------------
template <typename R, int N, typename OutT, int LPB>
__global__ void __launch_bounds__(LPB * LineCfg<R, N>::TPL_ROW)
row_inv_acc_kernel(const typename cvec<R>::T* __restrict__ planes,
                   const typename RecT<R>::T* __restrict__ rec, const uchar2* __restrict__ segtab,
                   int nseg, const unsigned long long* __restrict__ rowmask, int K,
                   long rows_per_rhs, long nrows, long n, R inv_n,
                   const typename cvec<R>::T* __restrict__ tw, OutT* __restrict__ out,
                   const int* __restrict__ active) {
  pdl_wait();
  using V = typename cvec<R>::T;
  constexpr bool WS = LineCfg<R, N>::WS;
  using F = LineFFT<R, N, +1, 1, WS, typename LineCfg<R, N>::RP>;
  constexpr int TPL = F::TPL, E = F::E;
  constexpr int CH = N * int(sizeof(V)) / 16;  // 16-byte chunks per row
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  __shared__ uchar2 seg_s[HZ_MAX_SEG];
  __shared__ unsigned long long cta_mask;
  for (int i = threadIdx.x; i < nseg; i += blockDim.x) seg_s[i] = segtab[i];
  const int li = threadIdx.x / TPL, t = threadIdx.x % TPL;
  const long row = long(blockIdx.x) * LPB + li;
  const bool valid = row < nrows && (!active || active[row / rows_per_rhs]);
  const long rhs = valid ? row / rows_per_rhs : 0;
  const long lrow = valid ? row - rhs * rows_per_rhs : 0;
  unsigned long long mymask = valid ? rowmask[lrow] : 0ull;
  if (threadIdx.x == 0) cta_mask = 0ull;
  __syncthreads();
  if (t == 0 && mymask) atomicOr(&cta_mask, mymask);
  V* line = sm + li * padded_len(N);
  // two staging rows of this line; cp.async needs 16-byte aligned destinations
  V* stg = reinterpret_cast<V*>(smem_raw + LineCfg<R, N>::stage_offset(LPB)) + li * 2 * N;
  typename RecT<R>::T r_[E];
  V acc[E];
  // this thread's output positions are those the transform's last stage
  // leaves in its registers
#pragma unroll
  for (int e = 0; e < E; ++e) {
    r_[e] = valid ? rec[lrow * N + F::out_index(t, e)] : typename RecT<R>::T(0);
    acc[e] = cmk<V>(R(0), R(0));
  }
  __syncthreads();
  // planes to transform: those any line of the block needs, or with
  // warp-synchronous lines only those the lines of this warp need
  unsigned long long cm = cta_mask;
  if constexpr (WS) {
    const unsigned lm = F::lane_mask();
    const unsigned lo = __reduce_or_sync(lm, unsigned(mymask & 0xFFFFFFFFull));
    const unsigned hi = __reduce_or_sync(lm, unsigned(mymask >> 32));
    cm = (unsigned long long)lo | ((unsigned long long)hi << 32);
  }
  const V* pbase = planes + (rhs * K) * n + lrow * N;
  auto issue = [&](int kk, int buf) {
    if ((mymask >> kk) & 1ull) {
      const char* src = reinterpret_cast<const char*>(pbase + long(kk) * n);
      char* dst = reinterpret_cast<char*>(stg + buf * N);
      for (int c = t; c < CH; c += TPL) cp_async16(dst + 16 * c, src + 16 * c);
    }
    cp_async_commit();
  };
  unsigned long long todo = cm;
  int kc = todo ? __ffsll((long long)todo) - 1 : -1;
  if (kc >= 0) {
    todo &= todo - 1;
    issue(kc, 0);
  }
  int buf = 0;
  while (kc >= 0) {
    const int kn = todo ? __ffsll((long long)todo) - 1 : -1;
    if (kn >= 0) {
      todo &= todo - 1;
      issue(kn, buf ^ 1);
    } else {
      cp_async_commit();  // keep one group in flight per step
    }
    cp_async_wait1();   // this thread's copies of plane kc are done
    F::sync();          // ... and the line's
    const bool need = (mymask >> kc) & 1ull;
    V x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = need ? stg[buf * N + F::stage0_index(t, e)] : cmk<V>(R(0), R(0));
    // Multi-stage plans: the transform's barriers also order these staging
    // reads before the next iteration's copies into the same buffer.  A
    // single-stage plan has one thread per line, which reads only what it
    // copied itself.
    F::run_regs(line, t, x, tw);
    if (need) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        int seg;
        R tf;
        decode_rec(r_[e], seg, tf);
        const uchar2 kk = seg_s[seg];
        R w = R(0);
        if (kk.x == kc) w += R(1) - tf;
        if (kk.y == kc) w += tf;
        acc[e].x += w * x[e].x;
        acc[e].y += w * x[e].y;
      }
    }
    kc = kn;
    buf ^= 1;
  }
  if (valid) {
    OutT* dst = out + rhs * n + lrow * N;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      OutT o;
      o.x = acc[e].x * inv_n;
      o.y = acc[e].y * inv_n;
      dst[F::out_index(t, e)] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// The same pass in two kernels, for grids with too few rows to fill the GPU
// with one block per row: the inverse FFT along x of every (row, node) line
// that the row's points weight, in place in the planes, one line per thread
// group (grid: row blocks x K); then the weighted sum as a gather of the two
// weighted planes per point (Eqn. 405), in the same order as the fused
// kernel: (1 - t) plane_lo first, then + t plane_hi.
// ---------------------------------------------------------------------------
template <typename R, int N, int LPB>
__global__ void __launch_bounds__(LPB * LineCfg<R, N>::TPL_ROW)
row_inv_inplace_kernel(typename cvec<R>::T* __restrict__ planes,
                       const unsigned long long* __restrict__ rowmask, int K, long rows_per_rhs,
                       long nrows, long n, const typename cvec<R>::T* __restrict__ tw,
                       const int* __restrict__ active) {
  pdl_wait();
  using V = typename cvec<R>::T;
  using F = LineFFT<R, N, +1, 1, LineCfg<R, N>::WS, typename LineCfg<R, N>::RP>;
  constexpr int TPL = F::TPL, E = F::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  const int li = threadIdx.x / TPL, t = threadIdx.x % TPL;
  const long row = long(blockIdx.x) * LPB + li;
  const int k = blockIdx.y;
  const long rhs = row < nrows ? row / rows_per_rhs : 0;
  const long lrow = row - rhs * rows_per_rhs;
  const bool valid = row < nrows && (!active || active[rhs]) && ((rowmask[lrow] >> k) & 1ull);
  V* g = planes + (rhs * K + k) * n + lrow * N;
  V x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) x[e] = valid ? g[F::stage0_index(t, e)] : cmk<V>(R(0), R(0));
  // every thread of the block takes part in the transform's barriers; the
  // line's reads are behind them before any of its writes
  F::run_regs(sm + li * padded_len(N), t, x, tw);
  if (valid) {
#pragma unroll
    for (int e = 0; e < E; ++e) g[F::out_index(t, e)] = x[e];
  }
}

template <typename R, typename OutT>
__global__ void __launch_bounds__(256)
weighted_gather_kernel(const typename cvec<R>::T* __restrict__ planes,
                       const typename RecT<R>::T* __restrict__ rec, const uchar2* __restrict__ segtab,
                       int K, long n, long total, R inv_n, OutT* __restrict__ out,
                       const int* __restrict__ active) {
  pdl_wait();
  using V = typename cvec<R>::T;
  for (long i = long(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += long(gridDim.x) * blockDim.x) {
    const long rhs = i / n, e = i - rhs * n;
    if (active && !active[rhs]) continue;
    int seg;
    R tf;
    decode_rec(rec[e], seg, tf);
    const uchar2 kk = segtab[seg];
    const V* pl = planes + rhs * K * n + e;
    V acc = cmk<V>(R(0), R(0));
    if (kk.x == kk.y) {
      acc = pl[long(kk.x) * n];
    } else {
      const R wl = R(1) - tf;
      if (wl != R(0)) {
        const V a = pl[long(kk.x) * n];
        acc = cmk<V>(wl * a.x, wl * a.y);
      }
      if (tf != R(0)) {
        const V b = pl[long(kk.y) * n];
        acc = cmk<V>(fma(tf, b.x, acc.x), fma(tf, b.y, acc.y));
      }
    }
    OutT o;
    o.x = acc.x * inv_n;
    o.y = acc.y * inv_n;
    out[i] = o;
  }
}

// The gather for per-point (node, weight) records: z = (1/n) sum over the
// point's used slots of w_slot plane_node (slots in increasing node order).
template <typename R, typename OutT>
__global__ void __launch_bounds__(256)
weighted_gather4_kernel(const typename cvec<R>::T* __restrict__ planes,
                        const uchar4* __restrict__ gnode, const typename GwT<R>::T* __restrict__ gw,
                        int K, long n, long total, R inv_n, OutT* __restrict__ out,
                        const int* __restrict__ active) {
  pdl_wait();
  using V = typename cvec<R>::T;
  for (long i = long(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += long(gridDim.x) * blockDim.x) {
    const long rhs = i / n, e = i - rhs * n;
    if (active && !active[rhs]) continue;
    const uchar4 nd = gnode[e];
    R w[4];
    load_gw(gw, e, w);
    const unsigned char ks[4] = {nd.x, nd.y, nd.z, nd.w};
    const V* pl = planes + rhs * K * n + e;
    R ax = R(0), ay = R(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (ks[j] != 0xFF) {
        const V a = pl[long(ks[j]) * n];
        ax = fma(w[j], a.x, ax);
        ay = fma(w[j], a.y, ay);
      }
    }
    OutT o;
    o.x = ax * inv_n;
    o.y = ay * inv_n;
    out[i] = o;
  }
}

// ---------------------------------------------------------------------------
// The same pass with one line per (row, node) item: items[i] = (row << 8) | k
// lists every pair of rowmask in use (grid.x: item blocks, grid.y: rhs).  A
// line inverse-transforms plane k along its row and adds w_k(x) / n times the
// result into out (Eqn. 405), which the apply cleared beforehand.  Each point
// receives at most two additions (its nodes k_lo and k_hi) onto an exact zero;
// floating-point addition commutes, so the sum does not depend on which
// arrives first.  Many independent short lines keep more warps resident than
// the fused kernel, whose row loops hold the accumulator in registers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void add_out(float2* p, float x, float y) {
  atomicAdd(p, make_float2(x, y));
}
__device__ __forceinline__ void add_out(double2* p, double x, double y) {
  atomicAdd(&p->x, x);
  atomicAdd(&p->y, y);
}

// GEN: the weights come from the per-point (node, weight) records gnode / gw.
// A point then receives up to four additions; with three or more the
// rounding of the sum depends on their arrival order, so results can differ
// between runs by rounding (the gather form does not).
template <typename R, int N, typename OutT, int LPB, bool GEN>
__global__ void __launch_bounds__(LPB * LineCfg<R, N>::TPL_ROW,
                                  sizeof(R) == 4 && LPB * LineCfg<R, N>::TPL_ROW < 512
                                      ? 512 / (LPB * LineCfg<R, N>::TPL_ROW) : 1)
row_inv_scatter_kernel(const typename cvec<R>::T* __restrict__ planes,
                       const typename RecT<R>::T* __restrict__ rec,
                       const uchar2* __restrict__ segtab, int nseg,
                       const unsigned long long* __restrict__ items, long nitems, int K, long n,
                       R inv_n, const typename cvec<R>::T* __restrict__ tw, OutT* out,
                       const int* __restrict__ active, const uchar4* __restrict__ gnode,
                       const typename GwT<R>::T* __restrict__ gw) {
  pdl_wait();
  using V = typename cvec<R>::T;
  using F = LineFFT<R, N, +1, 1, LineCfg<R, N>::WS, typename LineCfg<R, N>::RP>;
  constexpr int TPL = F::TPL, E = F::E;
  const long rhs = blockIdx.y;
  if (active && !active[rhs]) return;  // the whole block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  const int li = threadIdx.x / TPL, t = threadIdx.x % TPL;
  const long it = long(blockIdx.x) * LPB + li;
  const bool valid = it < nitems;
  const unsigned long long item = valid ? items[it] : 0ull;
  const long row = long(item >> 8);
  const int kc = int(item & 0xFFull);
  // the line's weight of node kc on segment s, as w = a + b t (already / n):
  // a = [k_lo == kc], b = [k_hi == kc] - a; HZ_MAX_SEG entries per line
  // after the lines' transform buffers
  V* wtab = reinterpret_cast<V*>(smem_raw + LineCfg<R, N>::row_smem(LPB)) + li * HZ_MAX_SEG;
  if constexpr (!GEN) {
    for (int i = t; i < nseg; i += TPL) {
      const uchar2 kk = segtab[i];
      const R a = kk.x == kc ? R(1) : R(0);
      const R b = (kk.y == kc ? R(1) : R(0)) - a;
      wtab[i] = cmk<V>(a * inv_n, b * inv_n);
    }
  }
  const V* src = planes + (rhs * K + kc) * n + row * N;
  V x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) x[e] = valid ? src[F::stage0_index(t, e)] : cmk<V>(R(0), R(0));
  // the records of this thread's output points, loaded with the line so that
  // no global load waits behind the transform
  using RT = typename RecT<R>::T;
  RT rv[GEN ? 1 : E];
  if constexpr (!GEN) {
    const RT* rr = rec + row * N;
#pragma unroll
    for (int e = 0; e < E; ++e) rv[e] = valid ? rr[F::out_index(t, e)] : RT(0);
  }
  __syncthreads();  // wtab
  F::run_regs(sm + li * padded_len(N), t, x, tw);
  if (valid) {
    OutT* dst = out + rhs * n + row * N;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = F::out_index(t, e);
      R w = R(0);
      if constexpr (GEN) {
        const uchar4 nd = gnode[row * N + p];
        R ws[4];
        load_gw(gw, row * N + p, ws);
        if (nd.x == kc) w += ws[0];
        if (nd.y == kc) w += ws[1];
        if (nd.z == kc) w += ws[2];
        if (nd.w == kc) w += ws[3];
      } else {
        int seg;
        R tf;
        decode_rec(rv[e], seg, tf);
        const V ab = wtab[seg];
        w = fma(ab.y, tf, ab.x);  // already / n
      }
      if (w != R(0)) {
        if constexpr (GEN) w *= inv_n;
        add_out(dst + p, w * x[e].x, w * x[e].y);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Strided-axis kernels.  A line has N elements at stride S; a block handles
// TB lines at adjacent x (thread = t * TB + column), so that loads and stores
// move TB contiguous elements, and keeps them interleaved in shared memory
// (position p of column col at pad(p) * TB + col).  Line (x, o, b) starts
// at b * bstride + o * ostride + x; grid.x = ceil(nx / TB) * outer.
// ---------------------------------------------------------------------------
template <typename R, int N, int SIGN>
__global__ void __launch_bounds__(LineCfg<R, N>::COL_THREADS)
line_pass_kernel(typename cvec<R>::T* __restrict__ data, int nx, int ntile, long S, long ostride,
                 long bstride, const unsigned long long* __restrict__ omask, int K,
                 const typename cvec<R>::T* __restrict__ tw, const int* __restrict__ active,
                 int per_rhs) {
  pdl_wait();
  using V = typename cvec<R>::T;
  constexpr int TB = LineCfg<R, N>::TB;
  using F = LineFFT<R, N, SIGN, TB, false, typename LineCfg<R, N>::CP>;
  constexpr int E = F::E;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  const int col = threadIdx.x % TB, t = threadIdx.x / TB;
  const int tile = blockIdx.x % ntile;
  const long o = blockIdx.x / ntile;
  const int x = tile * TB + col;
  const bool valid = x < nx;
  // omask (planes only): skip outer slices o that no row of plane k needs
  if (omask && !((omask[o] >> (blockIdx.z % K)) & 1ull)) return;
  if (active && !active[blockIdx.z / per_rhs]) return;
  V* base = data + long(blockIdx.z) * bstride + o * ostride + x;
  V* line = sm + col;
  V v[E];
#pragma unroll
  // offsets along the line fit in 32 bits
  for (int e = 0; e < E; ++e) v[e] = valid ? base[F::stage0_index(t, e) * int(S)] : cmk<V>(R(0), R(0));
  F::run_regs(line, t, v, tw);
  if (valid) {
#pragma unroll
    for (int e = 0; e < E; ++e) base[F::out_index(t, e) * int(S)] = v[e];
  }
}

// Last axis, one block per (column tile and outer index, group of kpb nodes,
// rhs): the spectrum vhat (transformed along every axis) times q_k, inverse
// FFT along the axis, written to plane k, for each node of the group (the
// spectrum is read once per block).  |xi|^2 = xi2_x[x] + xi2_o[o] + xi2_l[p].
// Plane k is only stored where smask[o smO + p smS] has bit k: per row in 2D
// (the next pass is the x inverse), per z-slab in 3D (the next pass is the y
// inverse, which needs the whole slab).
template <typename R, int N, int KPB, bool HERM>
__global__ void __launch_bounds__(LineCfg<R, N>::COL_THREADS)
line_sym_inv_kernel(const typename cvec<R>::T* __restrict__ vhat,
                    typename cvec<R>::T* __restrict__ planes, int nx, int ntile, long S,
                    long ostride, long n, int K, const R* __restrict__ xi2_x,
                    const R* __restrict__ xi2_o, const R* __restrict__ xi2_l,
                    const typename cvec<R>::T* __restrict__ symA,
                    const typename cvec<R>::T* __restrict__ symG, const R* __restrict__ symD,
                    const unsigned long long* __restrict__ smask, long smO, long smS,
                    const typename cvec<R>::T* __restrict__ tw, const int* __restrict__ active) {
  pdl_wait();
  using V = typename cvec<R>::T;
  constexpr int TB = LineCfg<R, N>::TB;
  using F = LineFFT<R, N, +1, TB, false, typename LineCfg<R, N>::CP>;
  constexpr int E = F::E;
  static_assert(KPB == 1 || KPB == 2 || KPB == 4, "nodes per block");
  if (active && !active[blockIdx.z]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sm = reinterpret_cast<V*>(smem_raw);
  const int col = threadIdx.x % TB, t = threadIdx.x / TB;
  const int tile = blockIdx.x % ntile;
  const long o = blockIdx.x / ntile;
  const int k0 = blockIdx.y * KPB;
  const int k1 = min(K, k0 + KPB);
  const long rhs = blockIdx.z;
  const int x = tile * TB + col;
  const bool valid = x < nx;
  const long off = o * ostride + x;
  const V* src = vhat + rhs * n + off;
  const R sxo = (valid ? xi2_x[x] : R(0)) + (xi2_o ? xi2_o[o] : R(0));
  V spec[E];
  R s2[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = F::stage0_index(t, e);
    spec[e] = valid ? src[p * int(S)] : cmk<V>(R(0), R(0));
    s2[e] = sxo + xi2_l[p];
  }
  // plane-store bits of this block's nodes for the rows this thread writes
  constexpr int MW = (E * KPB + 31) / 32;
  uint32_t mb[MW];
#pragma unroll
  for (int w = 0; w < MW; ++w) mb[w] = 0u;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int p = F::out_index(t, e);
    const uint32_t bits = uint32_t(smask[o * smO + p * int(smS)] >> k0) & ((1u << KPB) - 1u);
    mb[(e * KPB) / 32] |= bits << ((e * KPB) % 32);
  }
#pragma unroll 1
  for (int k = k0; k < k1; ++k) {
    const V A = symA[k], G = symG[k];
    const R D = HERM ? symD[k] : R(0);
    const int kk = k - k0;
    V v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      // vhat q_k = vhat conj(den) / |den|^2,  den = A - G |xi|^2
      const V den = cmk<V>(A.x - G.x * s2[e], A.y - G.y * s2[e]);
      const R inv = recip(den.x * den.x + den.y * den.y);
      V r = cscale(cmulc(spec[e], den), inv);
      if (HERM && D != R(0)) {
        // derivative plane of the Hermite basis: vhat dq/dc = vhat q (D |xi|^2 q),
        // D = 2 c_k (HERM: a medium with such planes; compiled out otherwise)
        r = cscale(cmul(r, cmk<V>(den.x * inv, -den.y * inv)), D * s2[e]);
      }
      v[e] = r;
    }
    F::run_regs(sm + col, t, v, tw);
    if (valid) {
      // offsets within one plane fit in 32 bits
      V* dst = planes + (rhs * K + k) * n + off;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        if ((mb[(e * KPB) / 32] >> ((e * KPB) % 32 + (KPB == 1 ? 0 : kk))) & 1u) dst[F::out_index(t, e) * int(S)] = v[e];
      }
    }
  }
}


// The complex64 symbol pass with two adjacent columns per thread (x, x + 1;
// nx even), their values paired in f32x2 registers (PV): the same arithmetic
// per column as line_sym_inv_kernel, in packed FP32 instructions, 16-byte
// global accesses, and tw2 = the (re, re, im, im) twiddle table.  TB: column
// pairs per block (the scalar kernel's TB, or half of it: the same registers
// per thread, smaller blocks).  SC > 0: the line stride S is SC (a square 2D
// grid, S = nx = N), so that every load and store offset of a thread is a
// compile-time constant from one base address.
template <int N, int KPB, int TB, bool HERM, int SC = 0>
__global__ void __launch_bounds__(TB * LineCfg<float, N>::template tpl_p<KPB>(),
                                  LineCfg<float, N>::template pair_min_blocks<KPB>(TB))
line_sym_inv_pair_kernel(const float2* __restrict__ vhat, float2* __restrict__ planes, int nx,
                         int ntile, long S, long ostride, long n, int K,
                         const float* __restrict__ xi2_x, const float* __restrict__ xi2_o,
                         const float* __restrict__ xi2_l, const float2* __restrict__ symA,
                         const float2* __restrict__ symG, const float* __restrict__ symD,
                         const unsigned long long* __restrict__ smask, long smO, long smS,
                         const float4* __restrict__ tw2, const int* __restrict__ active) {
  pdl_wait();
  using F = LineFFT<float, N, +1, TB, false, typename LineCfg<float, N>::template PPK<KPB>, PV>;
  constexpr int E = F::E;
  static_assert(KPB == 1 || KPB == 2 || KPB == 4, "nodes per block");
  if (active && !active[blockIdx.z]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PV* sm = reinterpret_cast<PV*>(smem_raw);
  const int col = threadIdx.x % TB, t = threadIdx.x / TB;
  const int tile = blockIdx.x % ntile;
  const long o = blockIdx.x / ntile;
  const int k0 = blockIdx.y * KPB;
  const int k1 = min(K, k0 + KPB);
  const long rhs = blockIdx.z;
  const int x = 2 * (tile * TB + col);
  const bool valid = x < nx;
  const long off = o * ostride + x;
  const float2* src = vhat + rhs * n + off;
  // line stride: compile-time when SC > 0 (then S == SC)
  const int Sl = SC > 0 ? SC : int(S);
  const float so = xi2_o ? xi2_o[o] : 0.0f;
  const float sx0 = (valid ? xi2_x[x] : 0.0f) + so, sx1 = (valid ? xi2_x[x + 1] : 0.0f) + so;
  constexpr int MW = (E * KPB + 31) / 32;
  uint32_t mb[MW];
  constexpr int TPLP = LineCfg<float, N>::template tpl_p<KPB>();
  // one node, E dividing 32: the block's warps build the E-bit store mask of
  // every t by ballots (lane = (t, e) pair, E lanes per t), one entry of
  // smask per (t, e) instead of E per thread
  constexpr bool BALLOT = KPB == 1 && E <= 32 && 32 % E == 0 && TPLP % (32 / E) == 0 &&
                          (TB * TPLP) % 32 == 0;
  if constexpr (BALLOT) {
    __shared__ uint32_t mwords[TPLP];
    constexpr int TPW = 32 / E;                        // t values per warp round
    constexpr int NW = TB * TPLP / 32;                 // warps per block
    constexpr int ROUNDS = (TPLP + NW * TPW - 1) / (NW * TPW);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, e = lane % E;
    // every round's entry loaded before the first ballot
    unsigned bit[ROUNDS];
#pragma unroll
    for (int i = 0; i < ROUNDS; ++i) {
      const int tt = (warp + i * NW) * TPW + lane / E;
      bit[i] = tt < TPLP ? unsigned(smask[o * smO + F::out_index(tt, e) * int(smS)] >> k0) & 1u : 0u;
    }
#pragma unroll
    for (int i = 0; i < ROUNDS; ++i) {
      const int tt = (warp + i * NW) * TPW + lane / E;
      if ((warp + i * NW) * TPW < TPLP) {  // warp-uniform
        const unsigned bal = __ballot_sync(0xffffffffu, bit[i]);
        if (e == 0) mwords[tt] = E == 32 ? bal : (bal >> lane) & ((1u << (E & 31)) - 1u);
      }
    }
    __syncthreads();
    mb[0] = mwords[t];
  } else {
#pragma unroll
    for (int w = 0; w < MW; ++w) mb[w] = 0u;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int p = F::out_index(t, e);
      const uint32_t bits = uint32_t(smask[o * smO + p * int(smS)] >> k0) & ((1u << KPB) - 1u);
      mb[(e * KPB) / 32] |= bits << ((e * KPB) % 32);
    }
  }
  // vhat q_k = vhat conj(den) / |den|^2,  den = A - G |xi|^2
  auto symbol = [](const PV& sp, f2 s2, f2 AX, f2 AY, f2 NGX, f2 NGY, float D) {
    PV den;
    den.x = fma2(NGX, s2, AX);
    den.y = fma2(NGY, s2, AY);
    const f2 nrm = fma2(den.x, den.x, den.y * den.y);
    const f2 inv = f2_make(recip(f2_lo(nrm)), recip(f2_hi(nrm)));
    const PV q = cmulc(sp, den);
    PV r;
    r.x = q.x * inv;
    r.y = q.y * inv;
    if (HERM && D != 0.0f) {
      // derivative plane of the Hermite basis: vhat dq/dc = vhat q (D |xi|^2 q)
      PV qv;
      qv.x = den.x * inv;
      qv.y = neg2(den.y) * inv;
      r = cmul(r, qv);
      const f2 ds = f2_splat(D) * s2;
      r.x = r.x * ds;
      r.y = r.y * ds;
    }
    return r;
  };
  auto store = [&](int k, int kk, PV (&v)[E]) {
    if (!valid) return;
    float2* dst = planes + (rhs * K + k) * n + off;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if ((mb[(e * KPB) / 32] >> ((e * KPB) % 32 + (KPB == 1 ? 0 : kk))) & 1u)
        *reinterpret_cast<float4*>(dst + F::out_index(t, e) * Sl) =
            make_float4(f2_lo(v[e].x), f2_lo(v[e].y), f2_hi(v[e].x), f2_hi(v[e].y));
    }
  };
  auto load = [&](int e, PV& sp, f2& s2) {
    const int p = F::stage0_index(t, e);
    // the spectrum streams past L1 (.cg), which keeps the twiddle table
    const float4 a = valid ? __ldcg(reinterpret_cast<const float4*>(src + p * Sl))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
    sp.x = f2_make(a.x, a.z);
    sp.y = f2_make(a.y, a.w);
    const float xl = xi2_l[p];
    s2 = f2_make(sx0 + xl, sx1 + xl);
  };
  if constexpr (KPB == 1) {
    // one node: the symbol product straight from the loads (no copy of the
    // spectrum kept across nodes)
    const float2 A = symA[k0], G = symG[k0];
    const float D = HERM ? symD[k0] : 0.0f;
    const f2 AX = f2_splat(A.x), AY = f2_splat(A.y), NGX = f2_splat(-G.x), NGY = f2_splat(-G.y);
    PV v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      PV sp;
      f2 s2;
      load(e, sp, s2);
      v[e] = symbol(sp, s2, AX, AY, NGX, NGY, D);
    }
    F::run_regs(sm + col, t, v, tw2);
    store(k0, 0, v);
  } else {
    PV spec[E];
    f2 s2[E];
#pragma unroll
    for (int e = 0; e < E; ++e) load(e, spec[e], s2[e]);
#pragma unroll 1
    for (int k = k0; k < k1; ++k) {
      const float2 A = symA[k], G = symG[k];
      const float D = HERM ? symD[k] : 0.0f;
      const f2 AX = f2_splat(A.x), AY = f2_splat(A.y), NGX = f2_splat(-G.x), NGY = f2_splat(-G.y);
      PV v[E];
#pragma unroll
      for (int e = 0; e < E; ++e) v[e] = symbol(spec[e], s2[e], AX, AY, NGX, NGY, D);
      F::run_regs(sm + col, t, v, tw2);
      store(k, k - k0, v);
    }
  }
}

}  // namespace hz
