// Small dense FP64 linear algebra on the device for the projected problems
// of the Gram-Schmidt and Rayleigh-Ritz steps (sizes up to SMALL_MAX).
#pragma once

#include "common.cuh"

namespace bdg {

constexpr int SMALL_MAX = 160;  // largest projected dimension (shared-memory Jacobi)

// C = alpha * op(A) * op(B) + beta * C, FP64, row-major with leading
// dimensions; op = transpose when ta / tb.  Sizes m x k times k x n.
cudaError_t dgemm_small(bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
                        const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t s);

// Symmetric eigen-decomposition A = V diag(w) V^T of an n x n FP64 matrix
// (row-major, lda), ascending w.  Parallel cyclic Jacobi in FP32 on one CTA
// gives a first V; Ogita-Aishima refinement steps in FP64 (SIAM J. Sci.
// Comput. 2018 "Iterative refinement for symmetric eigenvalue
// decomposition") bring it to FP64 accuracy.  ws: workspace of
// eigh_workspace_doubles(n) doubles.  V is n x n row-major (ld n).
size_t eigh_workspace_doubles(int n);
// floor_rel > 0: eigenvalues with |lambda| < floor_rel max|lambda| are
// returned orthonormal but not resolved from each other (for callers that
// discard them).  from_identity: start the refinement from V = I instead of
// the Jacobi basis, for matrices that are diagonal up to small off-diagonal
// entries (the refinement then resolves every pair whose gap exceeds a
// hundred times its coupling).
cudaError_t eigh(int n, const double* A, int lda, double* w, double* V, double* ws, int refine_steps,
                 cudaStream_t s, double floor_rel = 0.0, bool from_identity = false);

// Rank-revealing Cholesky factorization with symmetric pivoting of a
// symmetric positive semidefinite n x n FP64 matrix A (row-major, lda):
// P A P^T = [L1; L2] [L1; L2]^T, pivoting on the largest remaining
// diagonal and stopping at the first pivot <= tol * max_i A_ii.  Writes, in
// the original row order and with leading dimension ldo (>= n, columns
// r .. n-1 zero): L = P^T [L1; L2] (A ~ L L^T) and M = P^T [L1^-T; 0]
// (L^T M = I_r); the rank r goes to *rank_dev (device).  One CTA, the
// matrix staged in shared memory (n <= SMALL_MAX).
cudaError_t pchol(int n, const double* A, int lda, double tol, double* L, double* M, int ldo, int* rank_dev,
                  cudaStream_t s);

// Elementwise helpers on small matrices (row-major).
// B[i][j] = A[i][j] * dl[i] * dr[j]  (dl / dr may be NULL = ones)
cudaError_t dscale_small(int m, int n, const double* A, int lda, const double* dl, const double* dr,
                         double* B, int ldb, cudaStream_t s);

// A = (A + A^T) / 2 in place (n x n, lda)
cudaError_t dsym_small(int n, double* A, int lda, cudaStream_t s);

// B = 0 (m x n, ldb)
cudaError_t dzero_small(int m, int n, double* B, int ldb, cudaStream_t s);

}  // namespace bdg
