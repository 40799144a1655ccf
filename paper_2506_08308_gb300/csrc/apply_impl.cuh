// Matrix-free BdG product y = M x (Section 3.2; eqs. BdG-d / lrep-d).
//
// M = -1/2 Lap (x) diag(+1,+1,+1,s,s,s) + pointwise 6x6 coupling, with
// s = -1 in the UV form and +1 in the FG form.  The spectral Laplacian is a
// sum over axes of one-dimensional operators (eq. laplace_approx):
//   -1/2 Lap x = sum_a IDFT_a diag(1/2 mu_k^2) DFT_a x,
// so each axis is one pass of line FFTs: forward, multiply, inverse, all in
// registers and shared memory.
//
// Pass "row" (last, contiguous axis): a CTA takes RR grid rows of all six
// components of one vector, stages them in shared memory, computes the
// pointwise coupling from (phi_1, phi_0, phi_-1, V) there, runs the six
// line transforms and writes y = s_c T_last x_c + (C x)_c.
// Pass "axis" (each strided axis): a CTA takes W adjacent lines of one
// component, lanes mapped across lines for coalescing, and adds s_c T_a x_c
// into y.
//
// Pointwise coupling (eqs. def_A, def_B for real Phi = (a, b, c), rho =
// a^2+b^2+c^2, plus the Zeeman diagonal; the closed-form entries):
//   A11 = V + q - p - mu_1 + bn (rho + a^2) + bs (2a^2 + b^2 - c^2)
//   A22 = V - mu_0 + bn (rho + b^2) + bs (a^2 + c^2)
//   A33 = V + q + p - mu_-1 + bn (rho + c^2) + bs (2c^2 + b^2 - a^2)
//   A12 = bn ab + bs b (a + 2c),  A23 = bn bc + bs b (2a + c),  A13 = (bn - bs) ac
//   B11 = (bn + bs) a^2,  B22 = bn b^2 + 2 bs ac,  B33 = (bn + bs) c^2
//   B12 = (bn + bs) ab,  B23 = (bn + bs) bc,  B13 = bn ac + bs (b^2 - ac)
//   UV: (A u + B v, -(B u + A v));  FG: ((A + B) f, (A - B) g).
#pragma once

#include "apply.cuh"
#include "fft.cuh"

namespace bdg {

template <typename R>
struct Sym3 {
  R d0, d1, d2, o01, o12, o02;
};

template <typename R, typename T>
__device__ __forceinline__ T sym3_row0(const Sym3<R>& m, T x0, T x1, T x2) {
  return mk(m.d0 * x0.x + m.o01 * x1.x + m.o02 * x2.x, m.d0 * x0.y + m.o01 * x1.y + m.o02 * x2.y);
}
template <typename R, typename T>
__device__ __forceinline__ T sym3_row1(const Sym3<R>& m, T x0, T x1, T x2) {
  return mk(m.o01 * x0.x + m.d1 * x1.x + m.o12 * x2.x, m.o01 * x0.y + m.d1 * x1.y + m.o12 * x2.y);
}
template <typename R, typename T>
__device__ __forceinline__ T sym3_row2(const Sym3<R>& m, T x0, T x1, T x2) {
  return mk(m.o02 * x0.x + m.o12 * x1.x + m.d2 * x2.x, m.o02 * x0.y + m.o12 * x1.y + m.d2 * x2.y);
}

// Pointwise A and B at one node.
template <typename R, typename Q>
__device__ __forceinline__ void coupling_blocks(const Q pv, const Coupling<R>& cp, Sym3<R>& A,
                                                Sym3<R>& B) {
  const R a = (R)pv.x, b = (R)pv.y, c = (R)pv.z, V = (R)pv.w;
  const R bn = cp.beta_n, bs = cp.beta_s;
  const R a2 = a * a, b2 = b * b, c2 = c * c, ac = a * c;
  const R rho = a2 + b2 + c2;
  const R bnbs = bn + bs;
  A.d0 = V + cp.d1 + bn * (rho + a2) + bs * (2 * a2 + b2 - c2);
  A.d1 = V + cp.d0 + bn * (rho + b2) + bs * (a2 + c2);
  A.d2 = V + cp.dm + bn * (rho + c2) + bs * (2 * c2 + b2 - a2);
  A.o01 = bn * a * b + bs * b * (a + 2 * c);
  A.o12 = bn * b * c + bs * b * (2 * a + c);
  A.o02 = (bn - bs) * ac;
  B.d0 = bnbs * a2;
  B.d1 = bn * b2 + 2 * bs * ac;
  B.d2 = bnbs * c2;
  B.o01 = bnbs * a * b;
  B.o12 = bnbs * b * c;
  B.o02 = bn * ac + bs * (b2 - ac);
}

template <typename R>
__device__ __forceinline__ Sym3<R> sym_add(const Sym3<R>& A, const Sym3<R>& B, R s) {
  Sym3<R> o;
  o.d0 = A.d0 + s * B.d0; o.d1 = A.d1 + s * B.d1; o.d2 = A.d2 + s * B.d2;
  o.o01 = A.o01 + s * B.o01; o.o12 = A.o12 + s * B.o12; o.o02 = A.o02 + s * B.o02;
  return o;
}

// ---------------------------------------------------------------------------
// Row pass: last axis + coupling.  192 threads = 6 warps; warp w = component
// w; each warp holds RR = 32/N1 rows of that component.
// ---------------------------------------------------------------------------
#ifndef BDG_ROW_MIN_CTAS
#define BDG_ROW_MIN_CTAS 4   // FP32 row pass: 4 CTAs per SM (85 registers) measured 5 % faster than 3
#endif
#ifndef BDG_AXIS_MIN_CTAS
#define BDG_AXIS_MIN_CTAS 512 / (W * Split<N>::N1)
#endif
template <int N, typename R>
__global__ void __launch_bounds__(192, sizeof(R) == 4 ? BDG_ROW_MIN_CTAS : 1) k_row(const typename CT<R>::T* __restrict__ x,
                                             typename CT<R>::T* __restrict__ y, long long nunits,
                                             int rows_per_vec, long long npts,
                                             const typename CT<R>::Q* __restrict__ phiv,
                                             const typename CT<R>::T* __restrict__ twg,
                                             Coupling<R> cp, R kscale, int mode) {
  typedef typename CT<R>::T T;
  typedef Line<N, T, WarpSync> L;
  constexpr int N1 = L::N1, N2 = L::N2, RR = 32 / N1, NL = 6 * RR, NT = 192;
  static_assert(NL * N == NT * N2, "the staging loop gives every thread N2 elements");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tw = reinterpret_cast<T*>(smem_raw);
  T* xbuf = tw + N;         // [NL][N]
  T* cbuf = xbuf + NL * N;  // [NL][N]
  const int tid = threadIdx.x;
  const long long u0 = (long long)blockIdx.x * RR;

  for (int i = tid; i < N; i += NT) tw[i] = twg[i];
  // stage x (line l = c*RR + r): NL*N = NT*N2 elements, N2 per thread, in
  // batches of KB loads issued before their stores so that the latencies
  // overlap; the per-point table of the coupling loop below is fetched first
  constexpr int NP = (RR * N + NT - 1) / NT;   // coupling points per thread
  typename CT<R>::Q q[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int pidx = tid + k * NT;
    const int r = pidx / N, i = pidx - r * N;
    const long long u = u0 + r;
    if (pidx < RR * N && u < nunits) q[k] = phiv[(u % rows_per_vec) * N + i];
  }
  constexpr int KB = N2 >= 8 ? 8 : N2;
  static_assert(N2 % KB == 0, "whole batches");
#pragma unroll
  for (int k0 = 0; k0 < N2; k0 += KB) {
    T v[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const int idx = tid + (k0 + k) * NT;
      const int l = idx / N, i = idx - l * N;
      const int c = l / RR, r = l - c * RR;
      const long long u = u0 + r;
      v[k] = mk((R)0, (R)0);
      if (u < nunits) {
        const long long vec = u / rows_per_vec, row = u - vec * rows_per_vec;
        v[k] = x[(vec * 6 + c) * npts + row * N + i];
      }
    }
#pragma unroll
    for (int k = 0; k < KB; ++k) xbuf[tid + (k0 + k) * NT] = v[k];
  }
  __syncthreads();
  // pointwise coupling
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int pidx = tid + k * NT;
    if (pidx >= RR * N) break;
    const int r = pidx / N, i = pidx - r * N;
    const long long u = u0 + r;
    if (u >= nunits) continue;
    Sym3<R> A, B;
    coupling_blocks<R>(q[k], cp, A, B);
    const T x0 = xbuf[(0 * RR + r) * N + i], x1 = xbuf[(1 * RR + r) * N + i],
            x2 = xbuf[(2 * RR + r) * N + i], x3 = xbuf[(3 * RR + r) * N + i],
            x4 = xbuf[(4 * RR + r) * N + i], x5 = xbuf[(5 * RR + r) * N + i];
    T y0, y1, y2, y3, y4, y5;
    if (mode == BDG_UV) {
      y0 = sym3_row0(A, x0, x1, x2) + sym3_row0(B, x3, x4, x5);
      y1 = sym3_row1(A, x0, x1, x2) + sym3_row1(B, x3, x4, x5);
      y2 = sym3_row2(A, x0, x1, x2) + sym3_row2(B, x3, x4, x5);
      y3 = mk((R)0, (R)0) - (sym3_row0(B, x0, x1, x2) + sym3_row0(A, x3, x4, x5));
      y4 = mk((R)0, (R)0) - (sym3_row1(B, x0, x1, x2) + sym3_row1(A, x3, x4, x5));
      y5 = mk((R)0, (R)0) - (sym3_row2(B, x0, x1, x2) + sym3_row2(A, x3, x4, x5));
    } else {
      const Sym3<R> P = sym_add(A, B, (R)1), M = sym_add(A, B, (R)-1);
      y0 = sym3_row0(P, x0, x1, x2);
      y1 = sym3_row1(P, x0, x1, x2);
      y2 = sym3_row2(P, x0, x1, x2);
      y3 = sym3_row0(M, x3, x4, x5);
      y4 = sym3_row1(M, x3, x4, x5);
      y5 = sym3_row2(M, x3, x4, x5);
    }
    cbuf[(0 * RR + r) * N + i] = y0;
    cbuf[(1 * RR + r) * N + i] = y1;
    cbuf[(2 * RR + r) * N + i] = y2;
    cbuf[(3 * RR + r) * N + i] = y3;
    cbuf[(4 * RR + r) * N + i] = y4;
    cbuf[(5 * RR + r) * N + i] = y5;
  }
  __syncthreads();
  // line transforms: warp = component, lane/N1 = row
  const int lane = tid & 31, c = tid >> 5, r = lane / N1, t = lane - r * N1;
  const int l = c * RR + r;
  T* ex = xbuf + l * N;
  T a[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) a[n2] = ex[t + N1 * n2];
  L::fwdA(a, t, ex, tw, WarpSync());
  T b[L::S][N1];
  L::fwdB(b, t, ex);
#pragma unroll
  for (int s = 0; s < L::S; ++s)
#pragma unroll
    for (int k2 = 0; k2 < N1; ++k2) {
      const int kk = kidx<N>(t + N1 * s + N2 * k2);
      b[s][k2] = b[s][k2] * (kscale * (R)(kk * kk));
    }
  L::invB(b, t, ex, WarpSync());
  L::invA(a, t, ex, tw);
  const long long u = u0 + r;
  if (u < nunits) {
    const R sg = (mode == BDG_UV && c >= 3) ? (R)-1 : (R)1;
    const long long vec = u / rows_per_vec, row = u - vec * rows_per_vec;
    T* yl = y + (vec * 6 + c) * npts + row * N;
    const T* cl = cbuf + l * N;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      const int i = t + N1 * n2;
      yl[i] = cfma(a[n2], sg, cl[i]);
    }
  }
}

// ---------------------------------------------------------------------------
// Strided-axis pass: y += s_c T_a x for lines of length N with stride st.
// W adjacent lines per CTA, thread (w, j): w = tid % W, j = tid / W.
// ---------------------------------------------------------------------------
template <int N, typename R, int W>
__global__ void __launch_bounds__(W * Split<N>::N1, (sizeof(R) == 4 && N <= 256) ? BDG_AXIS_MIN_CTAS : 1) k_axis(const typename CT<R>::T* __restrict__ x,
                                                          typename CT<R>::T* __restrict__ y,
                                                          long long npts, long long st,
                                                          long long tiles_per_comp,
                                                          const typename CT<R>::T* __restrict__ twg,
                                                          R kscale, int mode) {
  typedef typename CT<R>::T T;
  typedef Line<N, T, BlockSync> L;
  constexpr int N1 = L::N1, N2 = L::N2, LS = N + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tw = reinterpret_cast<T*>(smem_raw);
  T* exb = tw + N;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += blockDim.x) tw[i] = twg[i];
  const long long vc = blockIdx.x / tiles_per_comp;  // vector*6 + component
  const long long tile = blockIdx.x - vc * tiles_per_comp;
  const long long tiles_inner = st / W;
  const long long outer = tile / tiles_inner, inner0 = (tile - outer * tiles_inner) * W;
  const int w = tid % W, j = tid / W;
  const long long base = vc * npts + outer * (long long)N * st + inner0 + w;
  const T* xl = x + base;
  T a[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) a[n2] = xl[(long long)(j + N1 * n2) * st];
  T* ex = exb + w * LS;
  __syncthreads();  // twiddles
  L::fwdA(a, j, ex, tw, BlockSync());
  T b[L::S][N1];
  L::fwdB(b, j, ex);
#pragma unroll
  for (int s = 0; s < L::S; ++s)
#pragma unroll
    for (int k2 = 0; k2 < N1; ++k2) {
      const int kk = kidx<N>(j + N1 * s + N2 * k2);
      b[s][k2] = b[s][k2] * (kscale * (R)(kk * kk));
    }
  L::invB(b, j, ex, BlockSync());
  L::invA(a, j, ex, tw);
  const int c = (int)(vc % 6);
  const R sg = (mode == BDG_UV && c >= 3) ? (R)-1 : (R)1;
  T* yl = y + base;
  // all N2 reads of y first: with a runtime stride the compiler cannot tell
  // the elements apart, and a read-add-write per element would wait out one
  // memory latency per element
  T yv[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) yv[n2] = yl[(long long)(j + N1 * n2) * st];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) yl[(long long)(j + N1 * n2) * st] = cfma(a[n2], sg, yv[n2]);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <int N, typename R>
static cudaError_t launch_row(const ApplyArgs<R>& g, cudaStream_t s) {
  typedef typename CT<R>::T T;
  constexpr int N1 = Split<N>::N1, RR = 32 / N1;
  const size_t sm = sizeof(T) * (size_t)N * (1 + 2 * 6 * RR);
  auto kern = k_row<N, R>;
  cudaError_t e = allow_dynamic_smem((const void*)kern, sm);
  if (e != cudaSuccess) return e;
  const int nlast = g.grid->n[g.grid->dim - 1];
  const long long rows_per_vec = g.grid->npts / nlast;
  const long long nunits = rows_per_vec * g.nvec;
  const long long blocks = (nunits + RR - 1) / RR;
  kern<<<(unsigned)blocks, 192, sm, s>>>(g.x, g.y, nunits, (int)rows_per_vec, g.grid->npts,
                                         g.phiv, g.tw[g.grid->dim - 1], g.cp,
                                         g.kscale[g.grid->dim - 1], g.mode);
  return cudaGetLastError();
}

template <int N, typename R, int W>
static cudaError_t launch_axis_w(const ApplyArgs<R>& g, int ax, long long st, cudaStream_t s) {
  typedef typename CT<R>::T T;
  constexpr int N1 = Split<N>::N1;
  const size_t sm = sizeof(T) * ((size_t)N + (size_t)W * (N + 1));
  auto kern = k_axis<N, R, W>;
  cudaError_t e = allow_dynamic_smem((const void*)kern, sm);
  if (e != cudaSuccess) return e;
  const long long tiles = g.grid->npts / ((long long)N * W);
  const long long blocks = tiles * 6 * g.nvec;
  kern<<<(unsigned)blocks, W * N1, sm, s>>>(g.x, g.y, g.grid->npts, st, tiles, g.tw[ax],
                                            g.kscale[ax], g.mode);
  return cudaGetLastError();
}

// W adjacent lines per CTA: 16 when their exchange areas fit in 80 KB, else
// fewer; never more than the stride (the number of adjacent lines).
template <int N, typename R>
static cudaError_t launch_axis(const ApplyArgs<R>& g, int ax, cudaStream_t s) {
  typedef typename CT<R>::T T;
  long long st = 1;
  for (int a = ax + 1; a < g.grid->dim; ++a) st *= g.grid->n[a];
  const size_t per_line = sizeof(T) * (N + 1);
  long long w = per_line * 16 <= 80 * 1024 ? 16 : per_line * 8 <= 80 * 1024 ? 8 : 4;
  if (w > st) w = st;
  if (w >= 16) return launch_axis_w<N, R, 16>(g, ax, st, s);
  if (w >= 8) return launch_axis_w<N, R, 8>(g, ax, st, s);
  return launch_axis_w<N, R, 4>(g, ax, st, s);
}

#define BDG_DISPATCH_N(nval, FN, ...)                         \
  switch (nval) {                                             \
    case 8: return FN<8, R>(__VA_ARGS__);                     \
    case 16: return FN<16, R>(__VA_ARGS__);                   \
    case 32: return FN<32, R>(__VA_ARGS__);                   \
    case 64: return FN<64, R>(__VA_ARGS__);                   \
    case 128: return FN<128, R>(__VA_ARGS__);                 \
    case 256: return FN<256, R>(__VA_ARGS__);                 \
    case 512: return FN<512, R>(__VA_ARGS__);                 \
    case 1024: return FN<1024, R>(__VA_ARGS__);               \
    default: return cudaErrorInvalidValue;                    \
  }

template <typename R>
static cudaError_t row_dispatch(const ApplyArgs<R>& g, cudaStream_t s) {
  BDG_DISPATCH_N(g.grid->n[g.grid->dim - 1], launch_row, g, s)
}
template <typename R>
static cudaError_t axis_dispatch(const ApplyArgs<R>& g, int ax, cudaStream_t s) {
  BDG_DISPATCH_N(g.grid->n[ax], launch_axis, g, ax, s)
}

template <typename R>
cudaError_t apply_launch(const ApplyArgs<R>& g, cudaStream_t s) {
  if (g.nvec <= 0) return cudaSuccess;
  cudaError_t e = row_dispatch<R>(g, s);
  if (e != cudaSuccess) return e;
  for (int ax = g.grid->dim - 2; ax >= 0; --ax) {
    e = axis_dispatch<R>(g, ax, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}


}  // namespace bdg
