// Tall-skinny block kernels used by the Gram-Schmidt and Rayleigh-Ritz steps.
//
// Blocks are "pair blocks": P complex columns of length n, column c starting
// at base + c*ld (complex elements), stored (re, im) interleaved.  Seen as
// real data they are 2P real columns: real column 2c+s (s = 0 real part,
// s = 1 imaginary part).  Both a complex Gram F^H G and the real Gram of
// real vectors packed two per complex column come out of the one real
// 2P x 2Q product.
#pragma once

#include "common.cuh"

namespace bdg {

template <typename R>
struct PairBlock {
  const typename CT<R>::T* p;  // first column
  long long ld;                // column stride in complex elements
  long long n;                 // rows (complex elements per column)
  int cols;                    // complex columns
};

// G (2P x 2Q, row-major, FP64) = A^T B over real columns; partial sums per
// row chunk are accumulated in R (FP64 blocks: double-float) and reduced
// across chunks in FP64.  ws must hold gram_workspace_bytes(P, Q, n) bytes.
// upper (FP64 blocks with P == Q): G is known to be symmetric; only the
// tiles on and above the diagonal are formed and the rest mirrored.
template <typename R>
cudaError_t gram_pairs(const PairBlock<R>& A, const PairBlock<R>& B, double* G_dev, void* ws,
                       size_t ws_bytes, cudaStream_t s, bool upper = false);
size_t gram_workspace_bytes(int P, int Q, long long n);

// The same Gram (full, no triangle) on the tensor cores with split-BF16
// operands and FP32 accumulation: FP32 accuracy for FP32 or FP64 blocks.
// Needs 2 B.cols <= 160; ws as for gram_pairs.
bool gram_tc_supported(int P, int Q);
template <typename R>
cudaError_t gram_pairs_tc(const PairBlock<R>& A, const PairBlock<R>& B, double* G_dev, void* ws,
                          size_t ws_bytes, cudaStream_t s);

// Y[:, q].t = beta * Y[:, q].t + alpha * sum_{p,s} A[:, p].s * C[(2p+s) * ldc + 2q+t]
// C is FP64 on the device (row-major 2P x 2Q with leading dimension ldc);
// A and Y must not overlap.
template <typename R>
cudaError_t update_pairs(const PairBlock<R>& A, const double* C_dev, int ldc, double beta,
                         typename CT<R>::T* Y, long long ldy, int Q, cudaStream_t s, double alpha = 1.0);

// Y = convert(X) column by column (FP64 <-> FP32 or same type), n complex
// elements per column, cols columns.
template <typename RI, typename RO>
cudaError_t convert_pairs(const typename CT<RI>::T* X, long long ldx, typename CT<RO>::T* Y,
                          long long ldy, long long n, int cols, cudaStream_t s);

// Y[:, q] = alpha_q * Y[:, q] (real scale per complex column) -- also zeroes.
template <typename R>
cudaError_t scale_pairs(typename CT<R>::T* Y, long long ldy, long long n, int cols,
                        const double* alpha_dev, double alpha_const, cudaStream_t s);

}  // namespace bdg
