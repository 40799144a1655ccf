// Tall-skinny block kernels (SIMT): pair Gram with FP64 cross-chunk
// reduction, block update with FP64 coefficients, conversions.
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

__global__ void k_gram_reduce(const double* __restrict__ part, int nchunks, int nout,
                              double* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nout) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += part[(long long)c * nout + i];
  G[i] = s;
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
                       size_t ws_bytes, cudaStream_t s) {
  if (A.n != B.n) return cudaErrorInvalidValue;
  const int P2 = 2 * A.cols, Q2 = 2 * B.cols;
  if (P2 == 0 || Q2 == 0) return cudaSuccess;
  if (A.n == 0) return cudaMemsetAsync(G_dev, 0, sizeof(double) * P2 * Q2, s);
  const long long nchunks = (A.n + GROWS - 1) / GROWS;
  if (ws_bytes < gram_workspace_bytes(A.cols, B.cols, A.n)) return cudaErrorInvalidValue;
  dim3 grid((P2 + GT - 1) / GT, (Q2 + GT - 1) / GT, (unsigned)nchunks);
  k_gram_partial<R><<<grid, 256, 0, s>>>(A, B, (double*)ws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nout = P2 * Q2;
  k_gram_reduce<<<(nout + 255) / 256, 256, 0, s>>>((const double*)ws, (int)nchunks, nout, G_dev);
  return cudaGetLastError();
}

template <typename R>
cudaError_t update_pairs(const PairBlock<R>& A, const double* C_dev, int ldc, double beta,
                         typename CT<R>::T* Y, long long ldy, int Q, cudaStream_t s, double alpha) {
  if (Q <= 0 || A.n == 0) return cudaSuccess;
  if (A.cols == 0) {
    return scale_pairs<R>(Y, ldy, A.n, Q, nullptr, beta, s);
  }
  const size_t sm = sizeof(R) * (size_t)(2 * A.cols) * UCOLS;
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_update<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((A.n + 255) / 256), (unsigned)((2 * Q + UCOLS - 1) / UCOLS));
  k_update<R><<<grid, 256, sm, s>>>(A, C_dev, ldc, beta, Y, ldy, Q, alpha);
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
                                       void*, size_t, cudaStream_t);
template cudaError_t gram_pairs<double>(const PairBlock<double>&, const PairBlock<double>&, double*,
                                        void*, size_t, cudaStream_t);
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
