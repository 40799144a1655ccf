// Tall-skinny block kernels (SIMT): pair Gram with FP64 cross-chunk
// reduction, block update with FP64 coefficients, conversions.
#include <algorithm>

#include "blas.cuh"

namespace bdg {

namespace {

constexpr int GT = 64;      // output tile (real columns) per CTA, both sides
constexpr int GK = 32;      // rows per shared-memory stage
constexpr int GROWS = 2048; // rows per chunk (partial sums per chunk)

// Partial Gram over one row chunk: part[chunk][i][j] for real columns
// i < 2P, j < 2Q.  256 threads, thread (ty, tx) owns rows 4ty.., cols 4tx..
template <typename R>
__global__ void __launch_bounds__(256) k_gram_partial(PairBlock<R> A, PairBlock<R> B,
                                                      double* __restrict__ part) {
  typedef typename CT<R>::T T;
  __shared__ R sA[GK][GT + 4];
  __shared__ R sB[GK][GT + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;  // real-column tile origins
  const long long r_begin = (long long)blockIdx.z * GROWS;
  const long long r_end = min(A.n, r_begin + GROWS);
  const int P2 = 2 * A.cols, Q2 = 2 * B.cols;
  R acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (R)0;
  for (long long r0 = r_begin; r0 < r_end; r0 += GK) {
    // load GK rows x 32 pairs of A and B: element e = (pair pp, row rr)
    for (int e = tid; e < GK * (GT / 2); e += 256) {
      const int rr = e % GK, pp = e / GK;
      const long long r = r0 + rr;
      const int pa = i0 / 2 + pp, pb = j0 / 2 + pp;
      T va = mk((R)0, (R)0), vb = mk((R)0, (R)0);
      if (r < r_end && pa < A.cols) va = A.p[(long long)pa * A.ld + r];
      if (r < r_end && pb < B.cols) vb = B.p[(long long)pb * B.ld + r];
      sA[rr][2 * pp] = va.x;
      sA[rr][2 * pp + 1] = va.y;
      sB[rr][2 * pp] = vb.x;
      sB[rr][2 * pp + 1] = vb.y;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < GK; ++k) {
      R a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = sA[k][4 * ty + q];
        b[q] = sB[k][4 * tx + q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
  double* out = part + (long long)blockIdx.z * P2 * Q2;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + 4 * ty + p, j = j0 + 4 * tx + q;
      if (i < P2 && j < Q2) out[(long long)i * Q2 + j] = (double)acc[p][q];
    }
}

// ---------------------------------------------------------------------------
// FP64 blocks on the FP32 pipes.  GB300 runs FP64 FMAs at about 1/60 of the
// FP32 rate, so the FP64 contractions use double-float arithmetic: every FP64
// operand is split into hi + lo floats (48 significant bits), products are
// formed exactly with an FMA (Dekker's product) plus the two cross terms,
// and sums are error-free two-sums (Knuth) renormalized at every step, so a
// partial sum carries about 2^-48 relative error per term -- the same order
// as an FP64 dot product of the chunk lengths used here -- at roughly a
// quarter of the FP32 rate instead of 1/60.
struct DF {
  float h, l;
};
// (the _rn intrinsics keep the compiler from contracting a product into a
// following sum, which would break the exactness of the two-sums)
__device__ __forceinline__ DF df_split(double v) {
  const float h = __double2float_rn(v);
  return DF{h, __double2float_rn(__dsub_rn(v, (double)h))};
}
// (sh, sl) += (ah + al) * (bh + bl), dropping al * bl
__device__ __forceinline__ void df_fma(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float t = __fadd_rn(__fadd_rn(sl, err), e);
  const float u = __fadd_rn(s, t);
  sl = __fsub_rn(t, __fsub_rn(u, s));
  sh = u;
}

// Partial Gram over one row chunk in double-float (layout as k_gram_partial),
// output tile (16 MP) x (16 MQ) real columns so that narrow and 48-wide
// blocks waste no arithmetic; with upper set (A and B tiled alike) only the
// tiles on or above the diagonal are formed.
template <int MP, int MQ>
__global__ void __launch_bounds__(256) k_gram_partial_df(PairBlock<double> A, PairBlock<double> B,
                                                         double* __restrict__ part, int upper, long long crows) {
  constexpr int TP = 16 * MP, TQ = 16 * MQ;
  if (upper && blockIdx.y < blockIdx.x) return;
  __shared__ float sAh[GK][TP + 4], sAl[GK][TP + 4];
  __shared__ float sBh[GK][TQ + 4], sBl[GK][TQ + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * TP, j0 = blockIdx.y * TQ;
  const long long r_begin = (long long)blockIdx.z * crows;
  const long long r_end = min(A.n, r_begin + crows);
  const int P2 = 2 * A.cols, Q2 = 2 * B.cols;
  float ah_[MP][MQ], al_[MP][MQ];
#pragma unroll
  for (int a = 0; a < MP; ++a)
#pragma unroll
    for (int b = 0; b < MQ; ++b) ah_[a][b] = al_[a][b] = 0.f;
  for (long long r0 = r_begin; r0 < r_end; r0 += GK) {
    for (int e = tid; e < GK * (TP / 2); e += 256) {
      const int rr = e % GK, pp = e / GK;
      const long long r = r0 + rr;
      const int pa = i0 / 2 + pp;
      double2 va = make_double2(0.0, 0.0);
      if (r < r_end && pa < A.cols) va = A.p[(long long)pa * A.ld + r];
      DF t;
      t = df_split(va.x); sAh[rr][2 * pp] = t.h; sAl[rr][2 * pp] = t.l;
      t = df_split(va.y); sAh[rr][2 * pp + 1] = t.h; sAl[rr][2 * pp + 1] = t.l;
    }
    for (int e = tid; e < GK * (TQ / 2); e += 256) {
      const int rr = e % GK, pp = e / GK;
      const long long r = r0 + rr;
      const int pb = j0 / 2 + pp;
      double2 vb = make_double2(0.0, 0.0);
      if (r < r_end && pb < B.cols) vb = B.p[(long long)pb * B.ld + r];
      DF t;
      t = df_split(vb.x); sBh[rr][2 * pp] = t.h; sBl[rr][2 * pp] = t.l;
      t = df_split(vb.y); sBh[rr][2 * pp + 1] = t.h; sBl[rr][2 * pp + 1] = t.l;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < GK; ++k) {
      float xh[MP], xl[MP], yh[MQ], yl[MQ];
#pragma unroll
      for (int q = 0; q < MP; ++q) {
        xh[q] = sAh[k][MP * ty + q];
        xl[q] = sAl[k][MP * ty + q];
      }
#pragma unroll
      for (int q = 0; q < MQ; ++q) {
        yh[q] = sBh[k][MQ * tx + q];
        yl[q] = sBl[k][MQ * tx + q];
      }
#pragma unroll
      for (int p = 0; p < MP; ++p)
#pragma unroll
        for (int q = 0; q < MQ; ++q) df_fma(ah_[p][q], al_[p][q], xh[p], xl[p], yh[q], yl[q]);
    }
    __syncthreads();
  }
  double* out = part + (long long)blockIdx.z * P2 * Q2;
#pragma unroll
  for (int p = 0; p < MP; ++p)
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
      const int i = i0 + MP * ty + p, j = j0 + MQ * tx + q;
      if (i < P2 && j < Q2) out[(long long)i * Q2 + j] = (double)ah_[p][q] + (double)al_[p][q];
    }
}

// tile multiple m (tile 16 m) for n real columns: least padded work, then the larger tile
inline int tile_mult(int n) {
  int best = 4;
  long long bw = -1;
  for (int m = 4; m >= 1; --m) {
    const long long w = (long long)((n + 16 * m - 1) / (16 * m)) * 16 * m;
    if (bw < 0 || w < bw) {
      bw = w;
      best = m;
    }
  }
  return best;
}

// G = sum over chunks; with tile > 0, entries below the diagonal tiles are
// read from their mirror (upper-triangle Grams)
// in a fixed order: thread (x, y) of a 32 x 8 block sums chunks y, y + 8,
// ... of one output (independent loads in flight), then the eight sums are
// added in order of y
__global__ void __launch_bounds__(256) k_gram_reduce_upper(const double* __restrict__ part, int nchunks, int P2,
                                                           int Q2, int tile, double* __restrict__ G) {
  __shared__ double t[8][33];
  const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + x, nout = P2 * Q2;
  double s = 0.0;
  if (e < nout) {
    const int i = e / Q2, j = e - i * Q2;
    const int src = (i / tile > j / tile) ? j * Q2 + i : e;
#pragma unroll 4
    for (int c = y; c < nchunks; c += 8) s += part[(long long)c * nout + src];
  }
  t[y][x] = s;
  __syncthreads();
  if (y == 0 && e < nout) {
    double g = t[0][x];
#pragma unroll
    for (int q = 1; q < 8; ++q) g += t[q][x];
    G[e] = g;
  }
}

__global__ void __launch_bounds__(256) k_gram_reduce(const double* __restrict__ part, int nchunks, int nout,
                                                     double* __restrict__ G) {
  __shared__ double t[8][33];
  const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + x;
  double s = 0.0;
  if (e < nout)
#pragma unroll 4
    for (int c = y; c < nchunks; c += 8) s += part[(long long)c * nout + e];
  t[y][x] = s;
  __syncthreads();
  if (y == 0 && e < nout) {
    double g = t[0][x];
#pragma unroll
    for (int q = 1; q < 8; ++q) g += t[q][x];
    G[e] = g;
  }
}

// One thread per row, 16 real output columns (8 pairs) per CTA column group.
constexpr int UCOLS = 16;
template <typename R>
__global__ void __launch_bounds__(256) k_update(PairBlock<R> A, const double* __restrict__ C, int ldc,
                                                double beta, typename CT<R>::T* __restrict__ Y,
                                                long long ldy, int Q, double alpha) {
  typedef typename CT<R>::T T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sC = reinterpret_cast<R*>(smem_raw);  // [2P][UCOLS]
  const int P2 = 2 * A.cols;
  const int j0 = blockIdx.y * UCOLS;       // first real output column
  const int Q2 = 2 * Q;
  for (int e = threadIdx.x; e < P2 * UCOLS; e += blockDim.x) {
    const int k = e / UCOLS, j = e - k * UCOLS;
    sC[e] = (j0 + j < Q2) ? (R)(alpha * C[(long long)k * ldc + j0 + j]) : (R)0;
  }
  __syncthreads();
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= A.n) return;
  R acc[UCOLS];
#pragma unroll
  for (int j = 0; j < UCOLS; ++j) acc[j] = (R)0;
  for (int p = 0; p < A.cols; ++p) {
    const T a = A.p[(long long)p * A.ld + r];
    const R* c0 = sC + (2 * p) * UCOLS;
    const R* c1 = c0 + UCOLS;
#pragma unroll
    for (int j = 0; j < UCOLS; ++j) acc[j] = fma(a.x, c0[j], fma(a.y, c1[j], acc[j]));
  }
#pragma unroll
  for (int q = 0; q < UCOLS / 2; ++q) {
    const int qq = j0 / 2 + q;
    if (qq >= Q) break;
    T* yp = Y + (long long)qq * ldy + r;
    T v = mk(acc[2 * q], acc[2 * q + 1]);
    if (beta != 0.0) {
      const T o = *yp;
      v = mk(fma((R)beta, o.x, v.x), fma((R)beta, o.y, v.y));
    }
    *yp = v;
  }
}

// k_update for FP64 blocks in double-float (see df_fma)
__global__ void __launch_bounds__(256) k_update_df(PairBlock<double> A, const double* __restrict__ C, int ldc,
                                                   double beta, double2* __restrict__ Y, long long ldy, int Q,
                                                   double alpha) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sCh = reinterpret_cast<float*>(smem_raw);  // [2P][UCOLS]
  const int P2 = 2 * A.cols;
  float* sCl = sCh + P2 * UCOLS;
  const int j0 = blockIdx.y * UCOLS;
  const int Q2 = 2 * Q;
  for (int e = threadIdx.x; e < P2 * UCOLS; e += blockDim.x) {
    const int k = e / UCOLS, j = e - k * UCOLS;
    const DF t = df_split((j0 + j < Q2) ? alpha * C[(long long)k * ldc + j0 + j] : 0.0);
    sCh[e] = t.h;
    sCl[e] = t.l;
  }
  __syncthreads();
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= A.n) return;
  float hh[UCOLS], ll[UCOLS];
#pragma unroll
  for (int j = 0; j < UCOLS; ++j) hh[j] = ll[j] = 0.f;
  for (int p = 0; p < A.cols; ++p) {
    const double2 a = A.p[(long long)p * A.ld + r];
    const DF ax = df_split(a.x), ay = df_split(a.y);
    const float* c0h = sCh + (2 * p) * UCOLS;
    const float* c0l = sCl + (2 * p) * UCOLS;
    const float* c1h = c0h + UCOLS;
    const float* c1l = c0l + UCOLS;
#pragma unroll
    for (int j = 0; j < UCOLS; ++j) {
      df_fma(hh[j], ll[j], ax.h, ax.l, c0h[j], c0l[j]);
      df_fma(hh[j], ll[j], ay.h, ay.l, c1h[j], c1l[j]);
    }
  }
#pragma unroll
  for (int q = 0; q < UCOLS / 2; ++q) {
    const int qq = j0 / 2 + q;
    if (qq >= Q) break;
    double2* yp = Y + (long long)qq * ldy + r;
    double2 v = make_double2((double)hh[2 * q] + (double)ll[2 * q], (double)hh[2 * q + 1] + (double)ll[2 * q + 1]);
    if (beta != 0.0) {
      const double2 o = *yp;
      v = make_double2(fma(beta, o.x, v.x), fma(beta, o.y, v.y));
    }
    *yp = v;
  }
}

template <typename RI, typename RO>
__global__ void k_convert(const typename CT<RI>::T* __restrict__ X, long long ldx,
                          typename CT<RO>::T* __restrict__ Y, long long ldy, long long n, int cols) {
  const long long total = n * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / n, r = e - c * n;
    const typename CT<RI>::T v = X[c * ldx + r];
    Y[c * ldy + r] = mk((RO)v.x, (RO)v.y);
  }
}

template <typename R>
__global__ void k_scale(typename CT<R>::T* __restrict__ Y, long long ldy, long long n, int cols,
                        const double* __restrict__ alpha, double alpha_const) {
  const long long total = n * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / n, r = e - c * n;
    const R s = (R)(alpha ? alpha[c] : alpha_const);
    typename CT<R>::T v = Y[c * ldy + r];
    Y[c * ldy + r] = mk(v.x * s, v.y * s);
  }
}

unsigned grid_for(long long total) {
  long long b = (total + 255) / 256;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

size_t gram_workspace_bytes(int P, int Q, long long n) {
  const long long nchunks = (n + GROWS - 1) / GROWS;
  return sizeof(double) * (size_t)nchunks * (size_t)(2 * P) * (size_t)(2 * Q);
}

template <typename R>
cudaError_t gram_pairs(const PairBlock<R>& A, const PairBlock<R>& B, double* G_dev, void* ws,
                       size_t ws_bytes, cudaStream_t s, bool upper) {
  if (A.n != B.n) return cudaErrorInvalidValue;
  const int P2 = 2 * A.cols, Q2 = 2 * B.cols;
  if (P2 == 0 || Q2 == 0) return cudaSuccess;
  if (A.n == 0) return cudaMemsetAsync(G_dev, 0, sizeof(double) * P2 * Q2, s);
  const long long nchunks = (A.n + GROWS - 1) / GROWS;
  if (ws_bytes < gram_workspace_bytes(A.cols, B.cols, A.n)) return cudaErrorInvalidValue;
  dim3 grid((P2 + GT - 1) / GT, (Q2 + GT - 1) / GT, (unsigned)nchunks);
  if (sizeof(R) == 8) {
    const PairBlock<double>& A8 = *reinterpret_cast<const PairBlock<double>*>(&A);
    const PairBlock<double>& B8 = *reinterpret_cast<const PairBlock<double>*>(&B);
    int mp = tile_mult(P2), mq = tile_mult(Q2);
    const bool up = upper && P2 == Q2;
    if (up) mp = mq = std::max(mp, mq);
    // narrow blocks have few output tiles: shorter row chunks (more CTAs, up
    // to about four per SM) as far as the workspace holds their partial sums
    const long long tiles = (long long)((P2 + 16 * mp - 1) / (16 * mp)) * ((Q2 + 16 * mq - 1) / (16 * mq));
    long long crows = GROWS, nch = nchunks;
    const long long want = (4 * 152 + tiles - 1) / tiles;
    if (want > nch) {
      const long long cap = (long long)(ws_bytes / (sizeof(double) * (size_t)P2 * Q2));
      long long target = std::min(want, cap);
      if (target > nch) {
        crows = ((A.n + target - 1) / target + GK - 1) / GK * GK;
        nch = (A.n + crows - 1) / crows;
      }
    }
    dim3 g8((P2 + 16 * mp - 1) / (16 * mp), (Q2 + 16 * mq - 1) / (16 * mq), (unsigned)nch);
#define BDG_GDF(MP_, MQ_) \
  if (mp == MP_ && mq == MQ_) k_gram_partial_df<MP_, MQ_><<<g8, 256, 0, s>>>(A8, B8, (double*)ws, up ? 1 : 0, crows);
    BDG_GDF(1, 1) BDG_GDF(1, 2) BDG_GDF(1, 3) BDG_GDF(1, 4)
    BDG_GDF(2, 1) BDG_GDF(2, 2) BDG_GDF(2, 3) BDG_GDF(2, 4)
    BDG_GDF(3, 1) BDG_GDF(3, 2) BDG_GDF(3, 3) BDG_GDF(3, 4)
    BDG_GDF(4, 1) BDG_GDF(4, 2) BDG_GDF(4, 3) BDG_GDF(4, 4)
#undef BDG_GDF
    cudaError_t e8 = cudaGetLastError();
    if (e8 != cudaSuccess) return e8;
    const int nout8 = P2 * Q2;
    k_gram_reduce_upper<<<(nout8 + 31) / 32, 256, 0, s>>>((const double*)ws, (int)nch, P2, Q2,
                                                            up ? 16 * mp : (1 << 30), G_dev);
    return cudaGetLastError();
  }
  k_gram_partial<R><<<grid, 256, 0, s>>>(A, B, (double*)ws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nout = P2 * Q2;
  k_gram_reduce<<<(nout + 31) / 32, 256, 0, s>>>((const double*)ws, (int)nchunks, nout, G_dev);
  return cudaGetLastError();
}

template <typename R>
cudaError_t update_pairs(const PairBlock<R>& A, const double* C_dev, int ldc, double beta,
                         typename CT<R>::T* Y, long long ldy, int Q, cudaStream_t s, double alpha) {
  if (Q <= 0 || A.n == 0) return cudaSuccess;
  if (A.cols == 0) {
    return scale_pairs<R>(Y, ldy, A.n, Q, nullptr, beta, s);
  }
  const size_t sm = sizeof(R) * (size_t)(2 * A.cols) * UCOLS;   // double: hi + lo floats, same size
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((A.n + 255) / 256), (unsigned)((2 * Q + UCOLS - 1) / UCOLS));
  cudaError_t e;
  if (sizeof(R) == 8) {
    e = allow_dynamic_smem((const void*)k_update_df, sm);
    if (e != cudaSuccess) return e;
    k_update_df<<<grid, 256, sm, s>>>(*reinterpret_cast<const PairBlock<double>*>(&A), C_dev, ldc, beta,
                                      reinterpret_cast<double2*>(Y), ldy, Q, alpha);
  } else {
    e = allow_dynamic_smem((const void*)k_update<R>, sm);
    if (e != cudaSuccess) return e;
    k_update<R><<<grid, 256, sm, s>>>(A, C_dev, ldc, beta, Y, ldy, Q, alpha);
  }
  return cudaGetLastError();
}

template <typename RI, typename RO>
cudaError_t convert_pairs(const typename CT<RI>::T* X, long long ldx, typename CT<RO>::T* Y,
                          long long ldy, long long n, int cols, cudaStream_t s) {
  if (n * cols == 0) return cudaSuccess;
  k_convert<RI, RO><<<grid_for(n * cols), 256, 0, s>>>(X, ldx, Y, ldy, n, cols);
  return cudaGetLastError();
}

template <typename R>
cudaError_t scale_pairs(typename CT<R>::T* Y, long long ldy, long long n, int cols,
                        const double* alpha_dev, double alpha_const, cudaStream_t s) {
  if (n * cols == 0) return cudaSuccess;
  k_scale<R><<<grid_for(n * cols), 256, 0, s>>>(Y, ldy, n, cols, alpha_dev, alpha_const);
  return cudaGetLastError();
}

template cudaError_t gram_pairs<float>(const PairBlock<float>&, const PairBlock<float>&, double*,
                                       void*, size_t, cudaStream_t, bool);
template cudaError_t gram_pairs<double>(const PairBlock<double>&, const PairBlock<double>&, double*,
                                        void*, size_t, cudaStream_t, bool);
template cudaError_t update_pairs<float>(const PairBlock<float>&, const double*, int, double,
                                         float2*, long long, int, cudaStream_t, double);
template cudaError_t update_pairs<double>(const PairBlock<double>&, const double*, int, double,
                                          double2*, long long, int, cudaStream_t, double);
template cudaError_t convert_pairs<double, float>(const double2*, long long, float2*, long long,
                                                  long long, int, cudaStream_t);
template cudaError_t convert_pairs<float, double>(const float2*, long long, double2*, long long,
                                                  long long, int, cudaStream_t);
template cudaError_t convert_pairs<double, double>(const double2*, long long, double2*, long long,
                                                   long long, int, cudaStream_t);
template cudaError_t convert_pairs<float, float>(const float2*, long long, float2*, long long,
                                                 long long, int, cudaStream_t);
template cudaError_t scale_pairs<float>(float2*, long long, long long, int, const double*, double,
                                        cudaStream_t);
template cudaError_t scale_pairs<double>(double2*, long long, long long, int, const double*, double,
                                         cudaStream_t);

}  // namespace bdg
