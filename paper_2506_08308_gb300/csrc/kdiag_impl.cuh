// k-space diagonal operators y = IDFT diag(g(|mu|^2)) DFT x over the whole
// grid, g(k2) = 1 / (shift + scale * k2).  Used as the preconditioner
// T_sigma = (1/2 |mu|^2 + sigma)^-1 of the subspace iteration and as the
// implicit kinetic step (1/tau + alpha - 1/2 Lap)^-1 of the ground-state
// flow (Section 3.1, eq. laplace_approx, for the Fourier symbols).
//
// The transform is separable: forward line FFTs along every axis but the
// slowest (natural-order spectra written back), then along the slowest axis
// forward, multiply, inverse, then the inverse passes in reverse order.
#pragma once

#include "common.cuh"
#include "fft.cuh"
#include "kdiag.cuh"

namespace bdg {

enum { KD_FWD = 0, KD_INV = 1, KD_FMI = 2 };

struct KdCoef {
  double shift, scale;   // g = 1 / (shift + scale * sum_a kappa_a k_a^2)
  double kappa[3];       // (2 pi / len_a)^2
  int n[3];
  double norm;           // 1 / N_p
};

// Contiguous lines (last axis): warp-mapped, 8 warps per CTA.  x may equal y
// (each line is read completely before it is written).
template <int N, typename R>
__global__ void __launch_bounds__(256) k_kd_contig(const typename CT<R>::T* x,
                                                   typename CT<R>::T* y, long long nlines,
                                                   const typename CT<R>::T* __restrict__ twg, int mode,
                                                   KdCoef c, int axis) {
  typedef typename CT<R>::T T;
  typedef Line<N, T, WarpSync> L;
  constexpr int N1 = L::N1, N2 = L::N2, LPW = 32 / N1, LPC = 8 * LPW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tw = reinterpret_cast<T*>(smem_raw);
  T* exb = tw + N;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = twg[i];
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, lw = lane / N1, t = lane - lw * N1;
  const long long line = (long long)blockIdx.x * LPC + warp * LPW + lw;
  const bool act = line < nlines;
  T* ex = exb + (warp * LPW + lw) * N;
  const T* xl = x + (act ? line : 0) * N;
  T a[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) a[n2] = act ? xl[t + N1 * n2] : mk((R)0, (R)0);
  T b[L::S][N1];
  if (mode == KD_INV) {
    // natural spectrum in -> spectral columns
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) ex[t + N1 * n2] = a[n2];
    __syncwarp();
    L::fromNatural(b, t, ex, WarpSync());
  } else {
    L::fwdA(a, t, ex, tw, WarpSync());
    L::fwdB(b, t, ex);
  }
  if (mode == KD_FMI) {
#pragma unroll
    for (int s = 0; s < L::S; ++s)
#pragma unroll
      for (int k2 = 0; k2 < N1; ++k2) {
        const int kk = kidx<N>(t + N1 * s + N2 * k2);
        // the symbol in the arithmetic precision R (FP64 division runs at a
        // small fraction of the FP32 rate on this part)
        const R d = (R)c.shift + (R)(c.scale * c.kappa[axis]) * (R)(kk * kk);
        b[s][k2] = b[s][k2] * ((R)c.norm / d);
      }
  }
  if (mode == KD_FWD) {
    L::toNatural(b, t, ex, WarpSync());
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) a[n2] = ex[t + N1 * n2];
  } else {
    L::invB(b, t, ex, WarpSync());
    L::invA(a, t, ex, tw);
  }
  if (act) {
    T* yl = y + line * N;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) yl[t + N1 * n2] = a[n2];
  }
}

// Strided lines (axis with stride st > 1): W adjacent lines per CTA.
// For KD_FMI this is the slowest axis (axis 0) and the other axes' spectral
// indices come from the position within the plane.
template <int N, typename R, int W>
__global__ void __launch_bounds__(W * Split<N>::N1) k_kd_strided(const typename CT<R>::T* x,
                                                                typename CT<R>::T* y,
                                                                long long npts, long long st,
                                                                long long tiles_per_plane,
                                                                const typename CT<R>::T* __restrict__ twg,
                                                                int mode, KdCoef c) {
  typedef typename CT<R>::T T;
  typedef Line<N, T, BlockSync> L;
  constexpr int N1 = L::N1, N2 = L::N2, LS = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tw = reinterpret_cast<T*>(smem_raw);
  T* exb = tw + N;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = twg[i];
  const long long plane = blockIdx.x / tiles_per_plane;
  const long long tile = blockIdx.x - plane * tiles_per_plane;
  const long long tiles_inner = st / W;
  const long long outer = tile / tiles_inner, inner0 = (tile - outer * tiles_inner) * W;
  const int w = tid % W, j = tid / W;
  const long long inner = inner0 + w;
  const long long base = plane * npts + outer * (long long)N * st + inner;
  const T* xl = x + base;
  T a[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) a[n2] = xl[(long long)(j + N1 * n2) * st];
  T* ex = exb + w * LS;
  __syncthreads();
  T b[L::S][N1];
  if (mode == KD_INV) {
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) ex[j + N1 * n2] = a[n2];
    __syncthreads();
    L::fromNatural(b, j, ex, BlockSync());
  } else {
    L::fwdA(a, j, ex, tw, BlockSync());
    L::fwdB(b, j, ex);
  }
  if (mode == KD_FMI) {
    // spectral indices of the faster axes from `inner`
    double extra = 0.0;
    if (c.n[2] > 1) {
      const int i2 = (int)(inner % c.n[2]), i1 = (int)(inner / c.n[2]);
      const int k1 = i1 < c.n[1] / 2 ? i1 : i1 - c.n[1];
      const int k2 = i2 < c.n[2] / 2 ? i2 : i2 - c.n[2];
      extra = c.kappa[1] * (double)(k1 * k1) + c.kappa[2] * (double)(k2 * k2);
    } else {
      const int i1 = (int)inner;
      const int k1 = i1 < c.n[1] / 2 ? i1 : i1 - c.n[1];
      extra = c.kappa[1] * (double)(k1 * k1);
    }
    // the symbol in the arithmetic precision R, per-thread constants hoisted
    const R base_d = (R)(c.shift + c.scale * extra), sk0 = (R)(c.scale * c.kappa[0]);
#pragma unroll
    for (int s = 0; s < L::S; ++s)
#pragma unroll
      for (int k2 = 0; k2 < N1; ++k2) {
        const int kk = kidx<N>(j + N1 * s + N2 * k2);
        const R d = base_d + sk0 * (R)(kk * kk);
        b[s][k2] = b[s][k2] * ((R)c.norm / d);
      }
  }
  if (mode == KD_FWD) {
    L::toNatural(b, j, ex, BlockSync());
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) a[n2] = ex[j + N1 * n2];
  } else {
    L::invB(b, j, ex, BlockSync());
    L::invA(a, j, ex, tw);
  }
  T* yl = y + base;
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) yl[(long long)(j + N1 * n2) * st] = a[n2];
}

template <int N, typename R>
static cudaError_t kd_contig(const KdArgs<R>& g, const KdCoef& c, const typename CT<R>::T* x,
                             typename CT<R>::T* y, int mode) {
  typedef typename CT<R>::T T;
  constexpr int N1 = Split<N>::N1, LPC = 8 * (32 / N1);
  const size_t sm = sizeof(T) * ((size_t)N + (size_t)LPC * N);
  auto kern = k_kd_contig<N, R>;
  cudaError_t e = allow_dynamic_smem((const void*)kern, sm);
  if (e != cudaSuccess) return e;
  const int ax = g.grid->dim - 1;
  const long long nlines = g.grid->npts / N * g.nplanes;
  kern<<<(unsigned)((nlines + LPC - 1) / LPC), 256, sm, g.stream>>>(x, y, nlines, g.tw[ax], mode, c, ax);
  return cudaGetLastError();
}

template <int N, typename R, int W>
static cudaError_t kd_strided_w(const KdArgs<R>& g, const KdCoef& c, int ax, long long st,
                                const typename CT<R>::T* x, typename CT<R>::T* y, int mode) {
  typedef typename CT<R>::T T;
  constexpr int N1 = Split<N>::N1;
  const size_t sm = sizeof(T) * ((size_t)N + (size_t)W * (N + 1));
  auto kern = k_kd_strided<N, R, W>;
  cudaError_t e = allow_dynamic_smem((const void*)kern, sm);
  if (e != cudaSuccess) return e;
  const long long tiles = g.grid->npts / ((long long)N * W);
  kern<<<(unsigned)(tiles * g.nplanes), W * N1, sm, g.stream>>>(x, y, g.grid->npts, st, tiles, g.tw[ax],
                                                               mode, c);
  return cudaGetLastError();
}

template <int N, typename R>
static cudaError_t kd_strided(const KdArgs<R>& g, const KdCoef& c, int ax, const typename CT<R>::T* x,
                              typename CT<R>::T* y, int mode) {
  typedef typename CT<R>::T T;
  long long st = 1;
  for (int a = ax + 1; a < g.grid->dim; ++a) st *= g.grid->n[a];
  const size_t per_line = sizeof(T) * (N + 1);
  long long w = per_line * 16 <= 80 * 1024 ? 16 : per_line * 8 <= 80 * 1024 ? 8 : 4;
  if (w > st) w = st;
  if (w >= 16) return kd_strided_w<N, R, 16>(g, c, ax, st, x, y, mode);
  if (w >= 8) return kd_strided_w<N, R, 8>(g, c, ax, st, x, y, mode);
  return kd_strided_w<N, R, 4>(g, c, ax, st, x, y, mode);
}

#define BDG_KD_DISPATCH(nval, FN, ...)                    \
  switch (nval) {                                         \
    case 8: return FN<8, R>(__VA_ARGS__);                 \
    case 16: return FN<16, R>(__VA_ARGS__);               \
    case 32: return FN<32, R>(__VA_ARGS__);               \
    case 64: return FN<64, R>(__VA_ARGS__);               \
    case 128: return FN<128, R>(__VA_ARGS__);             \
    case 256: return FN<256, R>(__VA_ARGS__);             \
    case 512: return FN<512, R>(__VA_ARGS__);             \
    case 1024: return FN<1024, R>(__VA_ARGS__);           \
    default: return cudaErrorInvalidValue;                \
  }

template <typename R>
static cudaError_t kd_contig_d(const KdArgs<R>& g, const KdCoef& c, const typename CT<R>::T* x,
                               typename CT<R>::T* y, int mode) {
  BDG_KD_DISPATCH(g.grid->n[g.grid->dim - 1], kd_contig, g, c, x, y, mode)
}
template <typename R>
static cudaError_t kd_strided_d(const KdArgs<R>& g, const KdCoef& c, int ax, const typename CT<R>::T* x,
                                typename CT<R>::T* y, int mode) {
  BDG_KD_DISPATCH(g.grid->n[ax], kd_strided, g, c, ax, x, y, mode)
}

template <typename R>
cudaError_t kdiag_launch(const KdArgs<R>& g) {
  if (g.nplanes <= 0) return cudaSuccess;
  KdCoef c;
  c.shift = g.shift;
  c.scale = g.scale;
  for (int a = 0; a < 3; ++a) {
    const double k0 = 2.0 * M_PI / g.grid->len[a];
    c.kappa[a] = k0 * k0;
    c.n[a] = g.grid->n[a];
  }
  c.norm = 1.0 / (double)g.grid->npts;
  const int d = g.grid->dim;
  cudaError_t e;
  if (d == 1) return kd_contig_d<R>(g, c, g.x, g.y, KD_FMI);
  // forward passes: last axis (contiguous), then the middle axes
  if ((e = kd_contig_d<R>(g, c, g.x, g.y, KD_FWD))) return e;
  for (int ax = d - 2; ax >= 1; --ax)
    if ((e = kd_strided_d<R>(g, c, ax, g.y, g.y, KD_FWD))) return e;
  if ((e = kd_strided_d<R>(g, c, 0, g.y, g.y, KD_FMI))) return e;
  for (int ax = 1; ax <= d - 2; ++ax)
    if ((e = kd_strided_d<R>(g, c, ax, g.y, g.y, KD_INV))) return e;
  return kd_contig_d<R>(g, c, g.y, g.y, KD_INV);
}

}  // namespace bdg
