// Instantiates the FFT pass kernels for one axis length, HZ_FFT_N, and
// exposes them as an FftOps table.  The build compiles this file once per
// supported length, in parallel.
#include <algorithm>
#include <type_traits>

#include "fft_kernels.cuh"

#ifndef HZ_FFT_N
#error "HZ_FFT_N must be defined"
#endif

namespace hz {
namespace {

constexpr int N = HZ_FFT_N;

template <typename K>
hz_status smem_attr(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) {
    HZ_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)));
  }
  return HZ_OK;
}

template <typename R>
hz_status row_fwd_t(const double2* in, const double* scale, long rows_per_rhs, long nrows,
                    const void* tw, void* out, cudaStream_t st, const int* active, void* zero,
                    long zero_row_bytes) {
  if (zero && zero_row_bytes % 16 != 0) return HZ_ERR_INVALID_ARG;
  uint4* z = static_cast<uint4*>(zero);
  const int zc = int(zero_row_bytes / 16);
  using C = LineCfg<R, N>;
  using V = typename cvec<R>::T;
  // blocks of ROW_LINES lines, or one line per block when that leaves the
  // GPU under-filled (few rows)
  const bool small = (nrows + C::ROW_LINES - 1) / C::ROW_LINES < 2L * 152;
  if (small) {
    auto k = row_fwd_kernel<R, N, 1>;
    HZ_TRY(smem_attr(k, C::row_smem(1)));
    HZ_CUDA(launch_pdl(k, dim3(unsigned(nrows)), dim3(C::TPL_ROW), C::row_smem(1), st, in, scale,
                       rows_per_rhs, nrows, static_cast<const V*>(tw), static_cast<V*>(out),
                       active, z, zc));
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
  }
  constexpr int lines = C::ROW_LINES;
  auto k = row_fwd_kernel<R, N, C::ROW_LINES>;
  HZ_TRY(smem_attr(k, C::row_smem(lines)));
  const long blocks = (nrows + lines - 1) / lines;
  HZ_CUDA(launch_pdl(k, dim3(unsigned(blocks)), dim3(lines * C::TPL_ROW), C::row_smem(lines), st,
                     in, scale, rows_per_rhs, nrows, static_cast<const V*>(tw),
                     static_cast<V*>(out), active, z, zc));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status row_fwd(int prec, const double2* in, const double* scale, long rows_per_rhs, long nrows,
                  const void* tw, void* out, cudaStream_t st, const int* active, void* zero,
                  long zero_row_bytes) {
  return prec == 0 ? row_fwd_t<double>(in, scale, rows_per_rhs, nrows, tw, out, st, active, zero,
                                       zero_row_bytes)
                   : row_fwd_t<float>(in, scale, rows_per_rhs, nrows, tw, out, st, active, zero,
                                      zero_row_bytes);
}

template <typename R, typename OutT>
hz_status row_inv_acc_t(const void* planes, const void* rec, const uchar2* segtab, int nseg,
                        const unsigned long long* rowmask, int K, long rows_per_rhs, long nrows,
                        long n, double inv_n, const void* tw, void* out, cudaStream_t st,
                        const int* active, int mode, const unsigned long long* items,
                        long nitems, const uchar4* gnode, const void* gw) {
  using C = LineCfg<R, N>;
  using V = typename cvec<R>::T;
  using GW = typename GwT<R>::T;
  if (gnode && mode != 3) {
    // per-point (node, weight) records: lines in place, then the gather
    auto ki = row_inv_inplace_kernel<R, N, C::ROW_LINES>;
    HZ_TRY(smem_attr(ki, C::row_smem()));
    dim3 grid(unsigned((nrows + C::ROW_LINES - 1) / C::ROW_LINES), unsigned(K));
    HZ_CUDA(launch_pdl(ki, dim3(grid), dim3(C::ROW_THREADS), C::row_smem(), st,
                       static_cast<V*>(const_cast<void*>(planes)), rowmask, K, rows_per_rhs, nrows,
                       n, static_cast<const V*>(tw), active));
    HZ_CUDA(cudaGetLastError());
    const long total = nrows * N;
    const long gblocks = std::min<long>((total + 255) / 256, 152L * 16);
    HZ_CUDA(launch_pdl(weighted_gather4_kernel<R, OutT>, dim3(unsigned(gblocks)), dim3(256), 0, st,
                       static_cast<const V*>(planes), gnode, static_cast<const GW*>(gw), K, n,
                       total, R(inv_n), static_cast<OutT*>(out), active));
    HZ_CUDA(cudaGetLastError());
    count_launches(1);  // the phase counts one
    return HZ_OK;
  }
  if (mode == 3) {
    // one line per (row, node) item, added into the cleared output
    if (!items || nitems <= 0) return nitems == 0 ? HZ_OK : HZ_ERR_INVALID_ARG;
    const long rhs = nrows / rows_per_rhs;
    if (rhs > 65535) return HZ_ERR_INVALID_ARG;
    auto ks = gnode ? row_inv_scatter_kernel<R, N, OutT, C::ROW_LINES, true>
                    : row_inv_scatter_kernel<R, N, OutT, C::ROW_LINES, false>;
    // line buffers, then (two-node records) one weight table per line
    const size_t smem = C::row_smem() + (gnode ? 0 : size_t(C::ROW_LINES) * HZ_MAX_SEG * sizeof(V));
    HZ_TRY(smem_attr(ks, smem));
    dim3 grid(unsigned((nitems + C::ROW_LINES - 1) / C::ROW_LINES), unsigned(rhs));
    HZ_CUDA(launch_pdl(ks, dim3(grid), dim3(C::ROW_THREADS), smem, st,
                       static_cast<const V*>(planes), static_cast<const typename RecT<R>::T*>(rec),
                       segtab, nseg, items, nitems, K, n, R(inv_n), static_cast<const V*>(tw),
                       static_cast<OutT*>(out), active, gnode, static_cast<const GW*>(gw)));
    HZ_CUDA(cudaGetLastError());
    return HZ_OK;
  }
  // fewer blocks of ROW_LINES rows than SMs: few rows
  const bool small = (nrows + C::ROW_LINES - 1) / C::ROW_LINES < 152L;
  // the fused pass holds three E-element arrays per thread; complex128 with
  // 30 elements per thread (lengths with a factor 5) would spill, so those
  // take the in-place pass and the gather
  constexpr bool fused_ok = !(sizeof(R) == 8 && C::RP::E > 16);
  if (mode == 1 || (mode == 0 && small) || !fused_ok) {
    // few rows: (row, node) lines in parallel, in place, then the gather
    auto ki = row_inv_inplace_kernel<R, N, C::ROW_LINES>;
    HZ_TRY(smem_attr(ki, C::row_smem()));
    dim3 grid(unsigned((nrows + C::ROW_LINES - 1) / C::ROW_LINES), unsigned(K));
    HZ_CUDA(launch_pdl(ki, dim3(grid), dim3(C::ROW_THREADS), C::row_smem(), st,
                       static_cast<V*>(const_cast<void*>(planes)), rowmask, K, rows_per_rhs, nrows,
                       n, static_cast<const V*>(tw), active));
    HZ_CUDA(cudaGetLastError());
    const long total = nrows * N;
    const long gblocks = std::min<long>((total + 255) / 256, 152L * 16);
    HZ_CUDA(launch_pdl(weighted_gather_kernel<R, OutT>, dim3(unsigned(gblocks)), dim3(256), 0, st,
                       static_cast<const V*>(planes), static_cast<const typename RecT<R>::T*>(rec),
                       segtab, K, n, total, R(inv_n), static_cast<OutT*>(out), active));
    HZ_CUDA(cudaGetLastError());
    count_launches(1);  // the phase counts one
    return HZ_OK;
  }
  if constexpr (fused_ok) {
    constexpr int lines = C::ROW_LINES;
    auto k = row_inv_acc_kernel<R, N, OutT, C::ROW_LINES>;
    HZ_TRY(smem_attr(k, C::row_acc_smem(lines)));
    const long blocks = (nrows + lines - 1) / lines;
    HZ_CUDA(launch_pdl(k, dim3(unsigned(blocks)), dim3(lines * C::TPL_ROW), C::row_acc_smem(lines),
                       st, static_cast<const V*>(planes),
                       static_cast<const typename RecT<R>::T*>(rec), segtab, nseg, rowmask, K,
                       rows_per_rhs, nrows, n, R(inv_n), static_cast<const V*>(tw),
                       static_cast<OutT*>(out), active));
    HZ_CUDA(cudaGetLastError());
  }
  return HZ_OK;
}

hz_status row_inv_acc(int prec, int out_kind, const void* planes, const void* rec,
                      const uchar2* segtab, int nseg, const unsigned long long* rowmask, int K,
                      long rows_per_rhs, long nrows, long n, double inv_n, const void* tw,
                      void* out, cudaStream_t st, const int* active, int mode,
                      const unsigned long long* items, long nitems, const uchar4* gnode,
                      const void* gw) {
  if (prec == 0)
    return row_inv_acc_t<double, double2>(planes, rec, segtab, nseg, rowmask, K, rows_per_rhs,
                                          nrows, n, inv_n, tw, out, st, active, mode, items, nitems, gnode, gw);
  if (out_kind == 0)
    return row_inv_acc_t<float, float2>(planes, rec, segtab, nseg, rowmask, K, rows_per_rhs,
                                        nrows, n, inv_n, tw, out, st, active, mode, items, nitems, gnode, gw);
  return row_inv_acc_t<float, double2>(planes, rec, segtab, nseg, rowmask, K, rows_per_rhs,
                                       nrows, n, inv_n, tw, out, st, active, mode, items, nitems, gnode, gw);
}

template <typename R, int SIGN>
hz_status line_pass_t(void* data, int nx, long outer, long S, long ostride, long bstride,
                      int batch, const unsigned long long* omask, int K, const void* tw,
                      cudaStream_t st, const int* active, int per_rhs) {
  using C = LineCfg<R, N>;
  using V = typename cvec<R>::T;
  auto k = line_pass_kernel<R, N, SIGN>;
  HZ_TRY(smem_attr(k, C::col_smem()));
  const int ntile = (nx + C::TB - 1) / C::TB;
  dim3 grid(unsigned(ntile * outer), 1, unsigned(batch));
  HZ_CUDA(launch_pdl(k, dim3(grid), dim3(C::COL_THREADS), C::col_smem(), st, static_cast<V*>(data),
                     nx, ntile, S, ostride, bstride, omask, K, static_cast<const V*>(tw), active,
                     per_rhs));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status line_pass(int prec, int sign, void* data, int nx, long outer, long S, long ostride,
                    long bstride, int batch, const unsigned long long* omask, int K,
                    const void* tw, cudaStream_t st, const int* active, int per_rhs) {
  if (prec == 0)
    return sign < 0 ? line_pass_t<double, -1>(data, nx, outer, S, ostride, bstride, batch, omask, K, tw, st, active, per_rhs)
                    : line_pass_t<double, +1>(data, nx, outer, S, ostride, bstride, batch, omask, K, tw, st, active, per_rhs);
  return sign < 0 ? line_pass_t<float, -1>(data, nx, outer, S, ostride, bstride, batch, omask, K, tw, st, active, per_rhs)
                  : line_pass_t<float, +1>(data, nx, outer, S, ostride, bstride, batch, omask, K, tw, st, active, per_rhs);
}

template <typename R>
hz_status line_sym_inv_t(const void* vhat, void* planes, int nx, long outer, long S, long ostride,
                         long n, int K, int batch, const void* xi2_x, const void* xi2_o,
                         const void* xi2_l, const void* symA, const void* symG,
                         const void* symD, const unsigned long long* smask, long smO, long smS,
                         const void* tw, const void* tw2, cudaStream_t st, const int* active,
                         int kpb, int pair) {
  using C = LineCfg<R, N>;
  using V = typename cvec<R>::T;
  // nodes per block: 1, 2 or 4
  kpb = kpb >= 4 ? 4 : (kpb >= 2 ? 2 : 1);
  if constexpr (std::is_same<R, float>::value) {
    if (tw2 && nx % 2 == 0) {
      // pair > 1: half-size blocks
      const bool half = pair > 1;
      constexpr int T1 = C::template tb_p<1>(), T1H = C::template tb_p_half<1>();
      constexpr int Tn = C::template tb_p<2>(), TnH = C::template tb_p_half<2>();
      // the Hermite derivative planes (symD) are a compiled variant, so
      // that other media run without their test
      // a square 2D grid (line stride N): the one-node form with compile-time offsets
      const bool sq = kpb == 1 && !half && outer == 1 && S == N;
      auto k = sq ? (symD ? line_sym_inv_pair_kernel<N, 1, T1, true, N>
                          : line_sym_inv_pair_kernel<N, 1, T1, false, N>)
             : symD ? (kpb == 1 ? (half ? line_sym_inv_pair_kernel<N, 1, T1H, true>
                                        : line_sym_inv_pair_kernel<N, 1, T1, true>)
                       : kpb == 2 ? (half ? line_sym_inv_pair_kernel<N, 2, TnH, true>
                                          : line_sym_inv_pair_kernel<N, 2, Tn, true>)
                                  : (half ? line_sym_inv_pair_kernel<N, 4, TnH, true>
                                          : line_sym_inv_pair_kernel<N, 4, Tn, true>))
                    : (kpb == 1 ? (half ? line_sym_inv_pair_kernel<N, 1, T1H, false>
                                        : line_sym_inv_pair_kernel<N, 1, T1, false>)
                       : kpb == 2 ? (half ? line_sym_inv_pair_kernel<N, 2, TnH, false>
                                          : line_sym_inv_pair_kernel<N, 2, Tn, false>)
                                  : (half ? line_sym_inv_pair_kernel<N, 4, TnH, false>
                                          : line_sym_inv_pair_kernel<N, 4, Tn, false>));
      const int tb = kpb == 1 ? (half ? T1H : T1) : (half ? TnH : Tn);
      const int tpl = kpb == 1 ? C::template tpl_p<1>() : C::template tpl_p<2>();
      HZ_TRY(smem_attr(k, C::col_pair_smem(tb)));
      const int ntile = (nx / 2 + tb - 1) / tb;
      dim3 grid(unsigned(ntile * outer), unsigned((K + kpb - 1) / kpb), unsigned(batch));
      HZ_CUDA(launch_pdl(k, dim3(grid), dim3(tb * tpl), C::col_pair_smem(tb), st,
                         static_cast<const float2*>(vhat), static_cast<float2*>(planes), nx, ntile,
                         S, ostride, n, K, static_cast<const float*>(xi2_x),
                         static_cast<const float*>(xi2_o), static_cast<const float*>(xi2_l),
                         static_cast<const float2*>(symA), static_cast<const float2*>(symG),
                         static_cast<const float*>(symD), smask, smO, smS,
                         static_cast<const float4*>(tw2), active));
      HZ_CUDA(cudaGetLastError());
      return HZ_OK;
    }
  }
  auto k = symD ? (kpb == 4 ? line_sym_inv_kernel<R, N, 4, true>
                            : (kpb == 2 ? line_sym_inv_kernel<R, N, 2, true>
                                        : line_sym_inv_kernel<R, N, 1, true>))
                : (kpb == 4 ? line_sym_inv_kernel<R, N, 4, false>
                            : (kpb == 2 ? line_sym_inv_kernel<R, N, 2, false>
                                        : line_sym_inv_kernel<R, N, 1, false>));
  HZ_TRY(smem_attr(k, C::col_smem()));
  const int ntile = (nx + C::TB - 1) / C::TB;
  dim3 grid(unsigned(ntile * outer), unsigned((K + kpb - 1) / kpb), unsigned(batch));
  HZ_CUDA(launch_pdl(k, dim3(grid), dim3(C::COL_THREADS), C::col_smem(), st,
                     static_cast<const V*>(vhat), static_cast<V*>(planes), nx, ntile, S, ostride, n,
                     K, static_cast<const R*>(xi2_x), static_cast<const R*>(xi2_o),
                     static_cast<const R*>(xi2_l), static_cast<const V*>(symA),
                     static_cast<const V*>(symG), static_cast<const R*>(symD), smask, smO, smS,
                     static_cast<const V*>(tw), active));
  HZ_CUDA(cudaGetLastError());
  return HZ_OK;
}

hz_status line_sym_inv(int prec, const void* vhat, void* planes, int nx, long outer, long S,
                       long ostride, long n, int K, int batch, const void* xi2_x,
                       const void* xi2_o, const void* xi2_l, const void* symA, const void* symG,
                       const void* symD, const unsigned long long* smask, long smO, long smS,
                       const void* tw, const void* tw2, cudaStream_t st, const int* active,
                       int kpb, int pair) {
  return prec == 0
             ? line_sym_inv_t<double>(vhat, planes, nx, outer, S, ostride, n, K, batch, xi2_x,
                                      xi2_o, xi2_l, symA, symG, symD, smask, smO, smS, tw, nullptr,
                                      st, active, kpb, 0)
             : line_sym_inv_t<float>(vhat, planes, nx, outer, S, ostride, n, K, batch, xi2_x,
                                     xi2_o, xi2_l, symA, symG, symD, smask, smO, smS, tw, tw2, st,
                                     active, kpb, pair);
}

const FftOps ops = {N, row_fwd, row_inv_acc, line_pass, line_sym_inv};

}  // namespace

#define HZ_CAT2(a, b) a##b
#define HZ_CAT(a, b) HZ_CAT2(a, b)
const FftOps* HZ_CAT(fft_ops_, HZ_FFT_N)() { return &ops; }

}  // namespace hz
