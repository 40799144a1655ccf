// Line FFTs for the Fourier pseudospectral operators (Section 3.1,
// eqs. FT_3 and laplace_approx), written for SIMT FP32/FP64 on sm_103a.
//
// A line of N = N1 * N2 points (powers of two, 8..1024) is handled by N1
// threads, each holding N2 complex values in registers (four-step
// Cooley-Tukey):
//   n = t + N1 n2  (t < N1, n2 < N2),   k = k1 + N2 k2  (k1 < N2, k2 < N1)
//   stage A  (thread t)  : DFT_N2 over n2, twiddle W_N^{t k1}
//   exchange (shared mem): element (t, k1) stored at t*N2 + (k1 ^ t)
//   stage B  (thread owns k1 = t + N1 s): DFT_N1 over t -> X[k1 + N2 k2]
// The inverse runs the same steps backwards.  Between stage B forward and
// stage B inverse every thread holds whole spectral columns, so a diagonal
// k-space multiplier costs no extra exchange.  The XOR swizzle keeps both
// exchange directions free of shared-memory bank conflicts for a line
// handled by one half-warp (FP32) or quarter-warp (FP64).
//
// In-register DFTs are radix-2 decimation in frequency with compile-time
// twiddles (cos(2 pi q/32) constants written out below).
#pragma once

#include "common.cuh"

namespace bdg {

__host__ __device__ constexpr double cos32_q(int q) {  // cos(2 pi q / 32), 0 <= q <= 8
  return q == 0 ? 1.0
       : q == 1 ? 0.9807852804032304
       : q == 2 ? 0.9238795325112867
       : q == 3 ? 0.8314696123025452
       : q == 4 ? 0.7071067811865476
       : q == 5 ? 0.5555702330196023
       : q == 6 ? 0.38268343236508984
       : q == 7 ? 0.19509032201612833
       : 0.0;
}
__host__ __device__ constexpr double cos32(int q) {
  return (q & 31) <= 8 ? cos32_q(q & 31)
       : (q & 31) <= 16 ? -cos32_q(16 - (q & 31))
       : (q & 31) <= 24 ? -cos32_q((q & 31) - 16)
       : cos32_q(32 - (q & 31));
}
__host__ __device__ constexpr double sin32(int q) { return cos32(q - 8); }

__host__ __device__ constexpr int bitrev(int k, int nbits) {
  return nbits == 0 ? 0 : ((k & 1) << (nbits - 1)) | bitrev(k >> 1, nbits - 1);
}
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// a * exp(i * DIR * 2 pi q / 32); q is a compile-time constant after unrolling.
template <int DIR, typename T>
__device__ __forceinline__ T rot32(T a, int q) {
  typedef decltype(a.x) R;
  q &= 31;
  if (q == 0) return a;
  if (q == 16) return mk(-a.x, -a.y);
  if (q == 8) return DIR > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
  if (q == 24) return DIR > 0 ? mk(a.y, -a.x) : mk(-a.y, a.x);
  const double c = cos32(q), s = DIR * sin32(q);
  if ((q & 7) == 4) {  // |c| = |s| = sqrt(1/2)
    const R h = (R)0.7071067811865476;
    const R xr = c > 0 ? a.x : -a.x, yr = c > 0 ? a.y : -a.y;
    const R xs = s > 0 ? a.x : -a.x, ys = s > 0 ? a.y : -a.y;
    return mk((xr - ys) * h, (yr + xs) * h);
  }
  const R cr = (R)c, sr = (R)s;
  return mk(fma(a.x, cr, -a.y * sr), fma(a.x, sr, a.y * cr));
}

// One radix-2 decimation-in-frequency stage of half-size SPAN, then the next.
template <int NR, int SPAN, int DIR, typename T>
struct DifStage {
  __device__ __forceinline__ static void run(T (&a)[NR]) {
#pragma unroll
    for (int blk = 0; blk < NR; blk += 2 * SPAN) {
#pragma unroll
      for (int j = 0; j < SPAN; ++j) {
        const T u = a[blk + j], v = a[blk + j + SPAN];
        a[blk + j] = u + v;
        a[blk + j + SPAN] = rot32<DIR>(u - v, j * (32 / (2 * SPAN)));
      }
    }
    DifStage<NR, SPAN / 2, DIR, T>::run(a);
  }
};
template <int NR, int DIR, typename T>
struct DifStage<NR, 0, DIR, T> {
  __device__ __forceinline__ static void run(T (&)[NR]) {}
};

// In-register DFT of size NR (2..32), DIR = -1 forward / +1 inverse,
// natural order in and out, unnormalized.
template <int NR, int K, typename T>
struct BitRevCopy {  // b[k] = a[bitrev(k)] for k >= K, indices fixed at compile time
  __device__ __forceinline__ static void run(const T (&a)[NR], T (&b)[NR]) {
    b[K] = a[bitrev(K, ilog2(NR))];
    BitRevCopy<NR, K + 1, T>::run(a, b);
  }
};
template <int NR, typename T>
struct BitRevCopy<NR, NR, T> {
  __device__ __forceinline__ static void run(const T (&)[NR], T (&)[NR]) {}
};

template <int NR, int DIR, typename T>
__device__ __forceinline__ void dft_reg(T (&a)[NR]) {
  DifStage<NR, NR / 2, DIR, T>::run(a);
  T b[NR];
  BitRevCopy<NR, 0, T>::run(a, b);
#pragma unroll
  for (int k = 0; k < NR; ++k) a[k] = b[k];
}

template <int N> struct Split;
template <> struct Split<8> { static constexpr int N1 = 2, N2 = 4; };
template <> struct Split<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct Split<32> { static constexpr int N1 = 4, N2 = 8; };
template <> struct Split<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct Split<128> { static constexpr int N1 = 8, N2 = 16; };
template <> struct Split<256> { static constexpr int N1 = 16, N2 = 16; };
template <> struct Split<512> { static constexpr int N1 = 16, N2 = 32; };
template <> struct Split<1024> { static constexpr int N1 = 32, N2 = 32; };

struct WarpSync {
  __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Signed wavenumber index of DFT slot k (k < N/2 -> k, else k - N).
template <int N>
__device__ __forceinline__ int kidx(int k) { return k < N / 2 ? k : k - N; }

template <int N, typename T, typename Sync>
struct Line {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, S = N2 / N1;
  typedef decltype(T().x) R;

  // a[n2] = x[t + N1 n2] (natural)  ->  exchange area holds twiddled stage-A output.
  __device__ __forceinline__ static void fwdA(T (&a)[N2], int t, T* ex, const T* tw, Sync sync) {
    dft_reg<N2, -1>(a);
    sync();  // previous readers of ex are done
#pragma unroll
    for (int k1 = 0; k1 < N2; ++k1) ex[t * N2 + (k1 ^ t)] = cmul(a[k1], tw[(t * k1) & (N - 1)]);
    sync();
  }
  // b[s][k2] = X[(t + N1 s) + N2 k2]
  __device__ __forceinline__ static void fwdB(T (&b)[S][N1], int t, const T* ex) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int k1 = t + N1 * s;
#pragma unroll
      for (int j = 0; j < N1; ++j) b[s][j] = ex[j * N2 + (k1 ^ j)];
      dft_reg<N1, -1>(b[s]);
    }
  }
  // inverse of fwdB; leaves the exchange area ready for invA.
  __device__ __forceinline__ static void invB(T (&b)[S][N1], int t, T* ex, Sync sync) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      dft_reg<N1, +1>(b[s]);
      const int k1 = t + N1 * s;
#pragma unroll
      for (int j = 0; j < N1; ++j) ex[j * N2 + (k1 ^ j)] = b[s][j];
    }
    sync();
  }
  // exchange area -> a[n2] = (unnormalized inverse)[t + N1 n2]
  __device__ __forceinline__ static void invA(T (&a)[N2], int t, const T* ex, const T* tw) {
#pragma unroll
    for (int k1 = 0; k1 < N2; ++k1) a[k1] = cmulc(ex[t * N2 + (k1 ^ t)], tw[(t * k1) & (N - 1)]);
    dft_reg<N2, +1>(a);
  }
  // spectral columns -> natural order in ex (for a forward-only transform)
  __device__ __forceinline__ static void toNatural(const T (&b)[S][N1], int t, T* ex, Sync sync) {
    sync();
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int k2 = 0; k2 < N1; ++k2) ex[t + N1 * s + N2 * k2] = b[s][k2];
    sync();
  }
  // natural order in ex -> spectral columns (for an inverse-only transform).
  // Ends with a barrier: the read pattern differs from the write pattern of
  // invB, which follows, so every thread must finish reading first.
  __device__ __forceinline__ static void fromNatural(T (&b)[S][N1], int t, const T* ex, Sync sync) {
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int k2 = 0; k2 < N1; ++k2) b[s][k2] = ex[t + N1 * s + N2 * k2];
    sync();
  }
};

}  // namespace bdg
