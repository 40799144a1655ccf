// Small dense FP64 kernels: GEMM, symmetric eigen-decomposition (FP32
// Jacobi + FP64 Ogita-Aishima refinement), scaling.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <vector>

#include "dense.cuh"

namespace bdg {

namespace {

constexpr int TB = 16;

__global__ void k_dgemm(bool ta, bool tb, int m, int n, int k, double alpha, const double* __restrict__ A,
                        int lda, const double* __restrict__ B, int ldb, double beta, double* __restrict__ C,
                        int ldc) {
  __shared__ double sA[TB][TB + 1];
  __shared__ double sB[TB][TB + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.y * TB + ty, j = blockIdx.x * TB + tx;
  double acc = 0.0;
  for (int l0 = 0; l0 < k; l0 += TB) {
    {  // A tile: rows i (block), cols l0 + tx
      const int ii = blockIdx.y * TB + ty, ll = l0 + tx;
      double v = 0.0;
      if (ii < m && ll < k) v = ta ? A[(long long)ll * lda + ii] : A[(long long)ii * lda + ll];
      sA[ty][tx] = v;
    }
    {  // B tile: rows l0 + ty, cols j
      const int ll = l0 + ty, jj = blockIdx.x * TB + tx;
      double v = 0.0;
      if (ll < k && jj < n) v = tb ? B[(long long)jj * ldb + ll] : B[(long long)ll * ldb + jj];
      sB[ty][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < TB; ++l) acc = fma(sA[ty][l], sB[l][tx], acc);
    __syncthreads();
  }
  if (i < m && j < n) {
    double* c = C + (long long)i * ldc + j;
    *c = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * *c);
  }
}

// ---------------------------------------------------------------------------
// Parallel cyclic Jacobi (FP32) on one CTA: round-robin ordering, each round
// rotates n/2 disjoint (p, q) planes, rows then columns.  Rotation of
// Golub & Van Loan (sym.schur2): tau = (a_qq - a_pp) / (2 a_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2), s = t c.
// Output ascending eigenvalues and the matching columns of V (FP64 copies).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_jacobi(int n, const double* __restrict__ Ag, int lda,
                                                 double* __restrict__ w, double* __restrict__ Vg,
                                                 int max_sweeps, float off_tol) {
  extern __shared__ float sm[];
  const int ld = n + 1;
  float* A = sm;                 // [n][ld]
  float* V = A + n * ld;         // [n][ld]
  float* cs = V + n * ld;        // [npair][2]
  int* pq = (int*)(cs + 2 * (n / 2 + 1));  // [npair][2]
  float* red = (float*)(pq + 2 * (n / 2 + 1));  // [64]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int np2 = (n + 1) & ~1;  // even count including a dummy index
  const int npair = np2 / 2;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e - i * n;
    A[i * ld + j] = (float)Ag[(long long)i * lda + j];
    V[i * ld + j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // off-diagonal and total Frobenius norms
    float off = 0.f, tot = 0.f;
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e - i * n;
      const float v = A[i * ld + j];
      tot += v * v;
      if (i != j) off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((tid & 31) == 0) { red[tid >> 5] = off; red[32 + (tid >> 5)] = tot; }
    __syncthreads();
    if (tid == 0) {
      float so = 0.f, st = 0.f;
      for (int q = 0; q < (nt + 31) / 32; ++q) { so += red[q]; st += red[32 + q]; }
      red[0] = so;
      red[32] = st;
    }
    __syncthreads();
    const bool done = red[0] <= off_tol * red[32];
    __syncthreads();
    if (done) break;
    for (int r = 0; r < np2 - 1; ++r) {
      if (tid < npair) {
        const int k = tid;
        int p = (r + k) % (np2 - 1);
        int q = (k == 0) ? (np2 - 1) : (r - k + np2 - 1) % (np2 - 1);
        if (p > q) { const int t = p; p = q; q = t; }
        float c = 1.f, s = 0.f;
        if (q < n) {
          const float apq = A[p * ld + q];
          const float app = A[p * ld + p], aqq = A[q * ld + q];
          if (fabsf(apq) > 1e-30f && fabsf(apq) > 1e-9f * sqrtf(fabsf(app * aqq))) {
            const float tau = (aqq - app) / (2.f * apq);
            const float t = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = rsqrtf(1.f + t * t);
            s = t * c;
          }
        } else {
          q = p;  // dummy: no rotation
        }
        pq[2 * k] = p;
        pq[2 * k + 1] = q;
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
      }
      __syncthreads();
      // A <- J^T A J and V <- V J in one pass: a work item is the 2 x 2 block
      // (row pair k, column pair l) of A -- rows first, then columns, as the
      // two one-sided updates would do -- or the rows of V's column pair l.
      // Warps take row pairs (or V's column pairs), lanes column pairs (or
      // rows): no index division, and the row pair's indices and rotation
      // are broadcast loads.  A dummy pair (odd n) has p == q and c = 1,
      // s = 0, which makes its duplicate reads and writes agree.
      const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
      for (int k = warp; k < npair; k += nwarp) {
        const int p = pq[2 * k], q = pq[2 * k + 1];
        const float ck = cs[2 * k], sk = cs[2 * k + 1];
        float* Ap = A + p * ld;
        float* Aq = A + q * ld;
        for (int l = lane; l < npair; l += 32) {
          const int u = pq[2 * l], v = pq[2 * l + 1];
          const float cl = cs[2 * l], sl = cs[2 * l + 1];
          const float x00 = Ap[u], x01 = Ap[v], x10 = Aq[u], x11 = Aq[v];
          const float r00 = ck * x00 - sk * x10, r01 = ck * x01 - sk * x11;
          const float r10 = sk * x00 + ck * x10, r11 = sk * x01 + ck * x11;
          Ap[u] = cl * r00 - sl * r01;
          Ap[v] = sl * r00 + cl * r01;
          Aq[u] = cl * r10 - sl * r11;
          Aq[v] = sl * r10 + cl * r11;
        }
      }
      for (int l = warp; l < npair; l += nwarp) {
        const int u = pq[2 * l], v = pq[2 * l + 1];
        if (u == v) continue;
        const float cl = cs[2 * l], sl = cs[2 * l + 1];
        for (int i = lane; i < n; i += 32) {
          const float vp = V[i * ld + u], vq = V[i * ld + v];
          V[i * ld + u] = cl * vp - sl * vq;
          V[i * ld + v] = sl * vp + cl * vq;
        }
      }
      __syncthreads();
    }
  }
  // ascending order by rank of the diagonal
  for (int j = tid; j < n; j += nt) {
    const float dj = A[j * ld + j];
    int rank = 0;
    for (int l = 0; l < n; ++l) {
      const float dl = A[l * ld + l];
      rank += (dl < dj) || (dl == dj && l < j);
    }
    w[rank] = (double)dj;
    for (int i = 0; i < n; ++i) Vg[(long long)i * n + rank] = (double)V[i * ld + j];
  }
}

// One Ogita-Aishima correction (SIAM J. Sci. Comput. 2018), given R = X^T X
// and S = X^T A X: lam_i = s_ii / (1 - r_ii), with r = I - X^T X;
// E_ij = (s_ij + lam_j r_ij) / (lam_j - lam_i) for pairs the current X
// resolves, else r_ij / 2 (orthogonalization only).  A pair counts as
// resolved when its corrections are small, |E_ij|, |E_ji| < 1/100, and its gap is above
// the rounding level of S (16 eps sqrt(n) |A|_F).  The pairwise test replaces the
// paper's global threshold 2 (|S - diag(lam)| + |A| |R|), which for graded
// spectra lumps every eigenvalue below eps_32 |A| into one cluster and stalls
// the refinement there.  On entry R holds X^T X; E is written over S.
__global__ void __launch_bounds__(1024) k_oa_correction(int n, double* __restrict__ R,
                                                        double* __restrict__ S,
                                                        const double* __restrict__ anorm_p,
                                                        double* __restrict__ lam) {
  const double anorm = *anorm_p;
  const int tid = threadIdx.x, nt = blockDim.x;
  // Symmetrize both products first: X^T (A X) carries a rounding asymmetry of
  // about eps n |A|, and the antisymmetric part of S would enter the
  // correction as (s_ij - s_ji) / (lam_j - lam_i) -- a loss of orthogonality
  // of eps n |A| / gap for small, graded eigenvalues.
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e - i * n;
    if (i > j) continue;
    const double r = 0.5 * (R[e] + R[j * n + i]);
    const double sv = 0.5 * (S[e] + S[j * n + i]);
    R[e] = (i == j ? 1.0 : 0.0) - r;
    R[j * n + i] = R[e];
    S[e] = sv;
    S[j * n + i] = sv;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) lam[i] = S[i * n + i] / (1.0 - R[i * n + i]);
  __syncthreads();
  const double floor_gap = 16.0 * 2.220446049250313e-16 * sqrt((double)n) * anorm;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e - i * n;
    const double r = R[e];
    double ev = 0.5 * r;
    if (i != j) {
      // the test is symmetric in (i, j) so that E_ij + E_ji = r_ij holds for
      // every pair and the update stays orthogonal to first order
      const double num = S[e] + lam[j] * r;
      const double numt = S[e] + lam[i] * r;
      const double den = lam[j] - lam[i];
      if (fabs(den) > floor_gap && 100.0 * fmax(fabs(num), fabs(numt)) < fabs(den)) ev = num / den;
    }
    S[e] = ev;
  }
}

__global__ void k_frob(int n, const double* __restrict__ A, int lda, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    const double v = A[(long long)i * lda + j];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x + 31) / 32; ++q) t += red[q];
    *out = sqrt(t);
  }
}

// sort (w, V columns) ascending after refinement (n small; one CTA)
__global__ void k_sort_eig(int n, const double* __restrict__ w, const double* __restrict__ V,
                           double* __restrict__ w2, double* __restrict__ V2) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double dj = w[j];
    int rank = 0;
    for (int l = 0; l < n; ++l) rank += (w[l] < dj) || (w[l] == dj && l < j);
    w2[rank] = dj;
    for (int i = 0; i < n; ++i) V2[(long long)i * n + rank] = V[(long long)i * n + j];
  }
}

__global__ void k_dscale(int m, int n, const double* __restrict__ A, int lda, const double* __restrict__ dl,
                         const double* __restrict__ dr, double* __restrict__ B, int ldb) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e - i * n;
    double v = A[(long long)i * lda + j];
    if (dl) v *= dl[i];
    if (dr) v *= dr[j];
    B[(long long)i * ldb + j] = v;
  }
}

__global__ void k_dsym(int n, double* A, int lda) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e - i * n;
    if (j >= i) continue;
    const double v = 0.5 * (A[(long long)i * lda + j] + A[(long long)j * lda + i]);
    A[(long long)i * lda + j] = v;
    A[(long long)j * lda + i] = v;
  }
}

__global__ void k_dzero(int m, int n, double* B, int ldb) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e - i * n;
    B[(long long)i * ldb + j] = 0.0;
  }
}

}  // namespace

cudaError_t dsym_small(int n, double* A, int lda, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  k_dsym<<<(n * n + 255) / 256, 256, 0, s>>>(n, A, lda);
  return cudaGetLastError();
}

cudaError_t dzero_small(int m, int n, double* B, int ldb, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  k_dzero<<<(m * n + 255) / 256, 256, 0, s>>>(m, n, B, ldb);
  return cudaGetLastError();
}

cudaError_t dgemm_small(bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
                        const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  dim3 grid((n + TB - 1) / TB, (m + TB - 1) / TB), block(TB, TB);
  k_dgemm<<<grid, block, 0, s>>>(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
  return cudaGetLastError();
}

cudaError_t dscale_small(int m, int n, const double* A, int lda, const double* dl, const double* dr,
                         double* B, int ldb, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  k_dscale<<<(m * n + 255) / 256, 256, 0, s>>>(m, n, A, lda, dl, dr, B, ldb);
  return cudaGetLastError();
}


__global__ void k_add_diag(int n, double* A, int lda, double c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[(long long)i * lda + i] += c;
}
// M = (3 I - G) / 2, one Newton-Schulz step toward (G)^-1/2 for G = V^T V near I
__global__ void k_newton_schulz(int n, double* G) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e - i * n;
    G[e] = (i == j ? 1.5 : 0.0) - 0.5 * G[e];
  }
}
__global__ void k_add_vec(int n, double* w, double c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] += c;
}

size_t eigh_workspace_doubles(int n) { return (size_t)48 * n * n + 128 * n + 256; }

namespace {

// ---------------------------------------------------------------------------
// All clusters of an FP32 Jacobi basis resolved in one launch.  CTA b takes
// the run of columns [start, start + size) of V (n x n, ld n) with midpoint
// shift c: two FP64 Newton-Schulz steps orthonormalize the columns, the
// shifted projection G = Vs^T (A - c I) Vs (norm about half the run's
// spread) is diagonalized by parallel cyclic Jacobi in FP64 (rotations of
// Golub & Van Loan, round-robin pairs as in k_jacobi), and the rotated
// columns and eigenvalues (ascending within the run) replace the old ones.
// ---------------------------------------------------------------------------
constexpr int RC_MAX_CLUSTERS = 96;   // runs of two or more columns: at most n / 2
constexpr int RC_NS_MAX = 48;         // wider runs keep the sequential path
struct ClusterList {
  int count;
  int start[RC_MAX_CLUSTERS];
  int size[RC_MAX_CLUSTERS];
  double shift[RC_MAX_CLUSTERS];
};

size_t resolve_smem_bytes(int n, int ns) {
  const int np2 = (ns + 1) & ~1;
  return sizeof(double) * (2 * (size_t)n * ns + 2 * (size_t)ns * ns + 2 * (size_t)np2 + 64) +
         sizeof(int) * ((size_t)np2 + 2 * (size_t)ns + 8);
}

__global__ void __launch_bounds__(256) k_resolve_clusters(int n, const double* __restrict__ A, int lda,
                                                          double* __restrict__ w, double* __restrict__ V,
                                                          ClusterList cl) {
  extern __shared__ double rsm[];
  const int i0 = cl.start[blockIdx.x], ns = cl.size[blockIdx.x];
  const double c = cl.shift[blockIdx.x];
  const int np2 = (ns + 1) & ~1, npair = np2 / 2;
  double* Vs = rsm;                       // [n][ns]
  double* T = Vs + (size_t)n * ns;        // [n][ns]
  double* G = T + (size_t)n * ns;         // [ns][ns]
  double* Z = G + (size_t)ns * ns;        // [ns][ns]
  double* cs = Z + (size_t)ns * ns;       // [npair][2]
  double* red = cs + np2;                 // [64]
  int* pq = reinterpret_cast<int*>(red + 64);   // [npair][2]
  int* rank = pq + np2;                   // [ns]
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * ns; e += nt) {
    const int i = e / ns, j = e - i * ns;
    Vs[e] = V[(long long)i * n + i0 + j];
  }
  __syncthreads();
  // Vs <- Vs (3 I - Vs^T Vs) / 2, twice
  for (int it = 0; it < 2; ++it) {
    for (int e = tid; e < ns * ns; e += nt) {
      const int a = e / ns, b = e - a * ns;
      double sacc = 0.0;
      for (int i = 0; i < n; ++i) sacc = fma(Vs[i * ns + a], Vs[i * ns + b], sacc);
      G[e] = (a == b ? 1.5 : 0.0) - 0.5 * sacc;
    }
    __syncthreads();
    for (int e = tid; e < n * ns; e += nt) {
      const int i = e / ns, b = e - i * ns;
      double sacc = 0.0;
      for (int a = 0; a < ns; ++a) sacc = fma(Vs[i * ns + a], G[a * ns + b], sacc);
      T[e] = sacc;
    }
    __syncthreads();
    for (int e = tid; e < n * ns; e += nt) Vs[e] = T[e];
    __syncthreads();
  }
  // T = (A - c I) Vs, G = Vs^T T symmetrized
  for (int e = tid; e < n * ns; e += nt) {
    const int i = e / ns, b = e - i * ns;
    const double* Ai = A + (long long)i * lda;
    double sacc = -c * Vs[i * ns + b];
    for (int k = 0; k < n; ++k) sacc = fma(Ai[k], Vs[k * ns + b], sacc);
    T[e] = sacc;
  }
  __syncthreads();
  for (int e = tid; e < ns * ns; e += nt) {
    const int a = e / ns, b = e - a * ns;
    double sacc = 0.0;
    for (int i = 0; i < n; ++i) sacc = fma(Vs[i * ns + a], T[i * ns + b], sacc);
    Z[e] = sacc;
  }
  __syncthreads();
  double fro = 0.0;
  for (int e = tid; e < ns * ns; e += nt) {
    const int a = e / ns, b = e - a * ns;
    const double v = 0.5 * (Z[a * ns + b] + Z[b * ns + a]);
    G[e] = v;
    fro += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  if ((tid & 31) == 0) red[tid >> 5] = fro;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < (nt + 31) / 32; ++q) t += red[q];
    red[32] = sqrt(t);
  }
  for (int e = tid; e < ns * ns; e += nt) Z[e] = (e / ns == e % ns) ? 1.0 : 0.0;
  __syncthreads();
  const double tiny = 1e-18 * red[32];
  // parallel cyclic Jacobi in FP64
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0;
    for (int e = tid; e < ns * ns; e += nt) {
      const int a = e / ns, b = e - a * ns;
      if (a != b) off += G[e] * G[e];
    }
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = off;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int q = 0; q < (nt + 31) / 32; ++q) t += red[q];
      red[33] = t;
    }
    __syncthreads();
    if (!(red[33] > 1e-32 * red[32] * red[32]) || !(red[33] > tiny * tiny)) break;
    for (int r = 0; r < np2 - 1; ++r) {
      if (tid < npair) {
        const int k = tid;
        int p = (r + k) % (np2 - 1);
        int q = (k == 0) ? (np2 - 1) : (r - k + np2 - 1) % (np2 - 1);
        if (p > q) { const int t = p; p = q; q = t; }
        double cc = 1.0, ss = 0.0;
        if (q < ns) {
          const double apq = G[p * ns + q], app = G[p * ns + p], aqq = G[q * ns + q];
          if (fabs(apq) > tiny) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            cc = 1.0 / sqrt(1.0 + t * t);
            ss = t * cc;
          }
        } else {
          q = p;
        }
        pq[2 * k] = p;
        pq[2 * k + 1] = q;
        cs[2 * k] = cc;
        cs[2 * k + 1] = ss;
      }
      __syncthreads();
      const int nblk = npair * npair;
      for (int e = tid; e < nblk + npair * ns; e += nt) {
        if (e < nblk) {
          const int k = e / npair, l = e - k * npair;
          const int p = pq[2 * k], q = pq[2 * k + 1], u = pq[2 * l], v = pq[2 * l + 1];
          const double ck = cs[2 * k], sk = cs[2 * k + 1], cl_ = cs[2 * l], sl = cs[2 * l + 1];
          const double x00 = G[p * ns + u], x01 = G[p * ns + v], x10 = G[q * ns + u], x11 = G[q * ns + v];
          const double r00 = ck * x00 - sk * x10, r01 = ck * x01 - sk * x11;
          const double r10 = sk * x00 + ck * x10, r11 = sk * x01 + ck * x11;
          G[p * ns + u] = cl_ * r00 - sl * r01;
          G[p * ns + v] = sl * r00 + cl_ * r01;
          G[q * ns + u] = cl_ * r10 - sl * r11;
          G[q * ns + v] = sl * r10 + cl_ * r11;
        } else {
          const int f = e - nblk, l = f / ns, i = f - l * ns;
          const int u = pq[2 * l], v = pq[2 * l + 1];
          if (u == v) continue;
          const double cl_ = cs[2 * l], sl = cs[2 * l + 1];
          const double zp = Z[i * ns + u], zq = Z[i * ns + v];
          Z[i * ns + u] = cl_ * zp - sl * zq;
          Z[i * ns + v] = sl * zp + cl_ * zq;
        }
      }
      __syncthreads();
    }
  }
  // ascending order within the run, new columns Vs Z, eigenvalues + c
  for (int j = tid; j < ns; j += nt) {
    const double dj = G[j * ns + j];
    int rk = 0;
    for (int l = 0; l < ns; ++l) {
      const double dl = G[l * ns + l];
      rk += (dl < dj) || (dl == dj && l < j);
    }
    rank[j] = rk;
    w[i0 + rk] = dj + c;
  }
  __syncthreads();
  for (int e = tid; e < n * ns; e += nt) {
    const int i = e / ns, j = e - i * ns;
    double sacc = 0.0;
    for (int a = 0; a < ns; ++a) sacc = fma(Vs[i * ns + a], Z[a * ns + j], sacc);
    V[(long long)i * n + i0 + rank[j]] = sacc;
  }
}

// FP32 Jacobi start for A (n x n, lda) into (w, V), with clusters resolved
// by recursion.  FP32 separates eigenvalues only down to about 1e-7 max|w|;
// every run of consecutive eigenvalues closer than 1e-4 max|w| (a cluster
// around its midpoint c -- which includes the eigenvalues near zero of a
// graded matrix) is re-solved on the FP64 projection V_s^T (A - c I) V_s,
// whose norm is about the spread, and rotated back.  Runs are disjoint, so
// the workspace is reused from one to the next.
cudaError_t jacobi_multilevel(int n, const double* A, int lda, double* w, double* V, double* ws, int depth,
                              double floor, double shift, cudaStream_t s) {
  const size_t sm = sizeof(float) * (2 * (size_t)n * (n + 1) + 2 * (n / 2 + 1)) +
                    sizeof(int) * 2 * (n / 2 + 1) + sizeof(float) * 64;
  cudaError_t e = allow_dynamic_smem((const void*)k_jacobi, sm);
  if (e != cudaSuccess) return e;
  static const bool prof = getenv("BDG_PROFILE_EIGH") != nullptr;
  cudaEvent_t pj[2] = {};
  if (prof) {
    cudaEventCreate(&pj[0]);
    cudaEventCreate(&pj[1]);
    cudaEventRecord(pj[0], s);
  }
  // converged to off(A) <= 1e-12 |A|^2: the FP64 refinement needs a start
  // this close (a stop at 1e-7 left backward errors up to 5e-2)
  k_jacobi<<<1, 1024, sm, s>>>(n, A, lda, w, V, 30, 1e-12f);
  if ((e = cudaGetLastError())) return e;
  if (prof) {
    cudaEventRecord(pj[1], s);
    cudaEventSynchronize(pj[1]);
    float t = 0;
    cudaEventElapsedTime(&t, pj[0], pj[1]);
    fprintf(stderr, "[bdg]   jacobi n %d depth %d %.3f ms\n", n, depth, t);
    cudaEventDestroy(pj[0]);
    cudaEventDestroy(pj[1]);
  }
  if (depth >= 4 || n < 2) return cudaSuccess;
  std::vector<double> hw(n);
  if ((e = cudaMemcpyAsync(hw.data(), w, sizeof(double) * n, cudaMemcpyDeviceToHost, s))) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  double amax = 0.0;
  for (double v : hw) amax = std::max(amax, std::fabs(v));
  if (!(amax > 0)) return cudaSuccess;
  if (depth == 0) floor *= amax;   // the caller's floor is relative at the top level
  const double tau = 1e-4 * amax;
  // runs of at most RC_NS_MAX columns are resolved by one launch (FP64
  // Jacobi per run); wider runs re-solve in turn on their projection
  ClusterList cl;
  cl.count = 0;
  int ns_max = 0;
  for (int i0 = 0; i0 < n;) {
    int i1 = i0 + 1;
    while (i1 < n && hw[i1] - hw[i1 - 1] < tau) ++i1;
    const int ns = i1 - i0;
    // a run whose spread is at the FP64 rounding level -- of its own values
    // or of the whole matrix -- is degenerate to working precision: any
    // orthonormal basis of it is an eigenbasis and nothing is re-solved
    const double spread = hw[i1 - 1] - hw[i0];
    const double mag = std::max(std::fabs(hw[i0]), std::fabs(hw[i1 - 1]));
    const bool degenerate = spread <= 1e-12 * mag || spread <= 64 * 2.220446049250313e-16 * amax;
    // runs whose eigenvalues all lie below the caller's floor (|lambda| of the
    // original matrix) are not needed resolved: the caller discards them
    const double top = std::max(std::fabs(hw[i0] + shift), std::fabs(hw[i1 - 1] + shift));
    if (ns >= 2 && spread > 0 && !degenerate && !(top < floor) && ns <= RC_NS_MAX &&
        cl.count < RC_MAX_CLUSTERS) {
      cl.start[cl.count] = i0;
      cl.size[cl.count] = ns;
      cl.shift[cl.count] = 0.5 * (hw[i0] + hw[i1 - 1]);
      cl.count++;
      ns_max = std::max(ns_max, ns);
    } else if (ns >= 2 && spread > 0 && !degenerate && !(top < floor)) {
      const double c = 0.5 * (hw[i0] + hw[i1 - 1]);  // midpoint: the shifted norm is half the spread
      double* Vs = ws;                         // n x ns
      double* AVs = Vs + (size_t)n * ns;       // n x ns
      double* As = AVs + (size_t)n * ns;       // ns x ns
      double* w2 = As + (size_t)ns * ns;       // ns
      double* V2 = w2 + ns + 8;                // ns x ns
      double* Vn = V2 + (size_t)ns * ns;       // n x ns
      double* rest = Vn + (size_t)n * ns;
      // V's columns i0 .. i1-1 are contiguous: gather with a strided copy
      if ((e = cudaMemcpy2DAsync(Vs, sizeof(double) * ns, V + i0, sizeof(double) * n, sizeof(double) * ns, n,
                                 cudaMemcpyDeviceToDevice, s)))
        return e;
      // FP64 orthonormalization of the FP32 columns (two Newton-Schulz
      // steps): with c != 0 the projection would otherwise carry
      // c (V^T V - I) ~ 1e-7 c, which can exceed the spread being resolved
      for (int it = 0; it < 2; ++it) {
        if ((e = dgemm_small(true, false, ns, ns, n, 1.0, Vs, ns, Vs, ns, 0.0, As, ns, s))) return e;
        k_newton_schulz<<<(ns * ns + 255) / 256, 256, 0, s>>>(ns, As);
        if ((e = cudaGetLastError())) return e;
        if ((e = dgemm_small(false, false, n, ns, ns, 1.0, Vs, ns, As, ns, 0.0, Vn, ns, s))) return e;
        if ((e = cudaMemcpyAsync(Vs, Vn, sizeof(double) * n * ns, cudaMemcpyDeviceToDevice, s))) return e;
      }
      if ((e = dgemm_small(false, false, n, ns, n, 1.0, A, lda, Vs, ns, 0.0, AVs, ns, s))) return e;
      if ((e = dgemm_small(true, false, ns, ns, n, 1.0, Vs, ns, AVs, ns, 0.0, As, ns, s))) return e;
      if ((e = dsym_small(ns, As, ns, s))) return e;
      k_add_diag<<<(ns + 127) / 128, 128, 0, s>>>(ns, As, ns, -c);
      if ((e = cudaGetLastError())) return e;
      if ((e = jacobi_multilevel(ns, As, ns, w2, V2, rest, depth + 1, floor, shift + c, s))) return e;
      k_add_vec<<<(ns + 127) / 128, 128, 0, s>>>(ns, w2, c);
      if ((e = cudaGetLastError())) return e;
      if ((e = dgemm_small(false, false, n, ns, ns, 1.0, Vs, ns, V2, ns, 0.0, Vn, ns, s))) return e;
      if ((e = cudaMemcpy2DAsync(V + i0, sizeof(double) * n, Vn, sizeof(double) * ns, sizeof(double) * ns, n,
                                 cudaMemcpyDeviceToDevice, s)))
        return e;
      if ((e = cudaMemcpyAsync(w + i0, w2, sizeof(double) * ns, cudaMemcpyDeviceToDevice, s))) return e;
    }
    i0 = i1;
  }
  if (prof && depth == 0)
    fprintf(stderr, "[bdg]   clusters n %d: %d batched (widest %d)\n", n, cl.count, ns_max);
  if (cl.count > 0) {
    const size_t smr = resolve_smem_bytes(n, ns_max);
    if ((e = allow_dynamic_smem((const void*)k_resolve_clusters, smr))) return e;
    k_resolve_clusters<<<cl.count, 256, smr, s>>>(n, A, lda, w, V, cl);
    if ((e = cudaGetLastError())) return e;
  }
  return cudaSuccess;
}

}  // namespace

// ---------------------------------------------------------------------------
// Rank-revealing pivoted Cholesky (see dense.cuh), one CTA of 1024 threads:
// right-looking, the lower triangle of the working matrix S in shared
// memory; step k pivots the largest remaining diagonal to position k, forms
// column k of L and updates the trailing lower triangle.  The inverse of L1
// comes from row-wise forward substitution, X_i = (e_i - sum_{j<i} L_ij X_j)
// / L_ii.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_pchol(int n, const double* __restrict__ A, int lda, double tol,
                                                double* __restrict__ L, double* __restrict__ M, int ldo,
                                                int* __restrict__ rank_dev) {
  extern __shared__ double psm[];
  double* S = psm;                           // [n][n]
  double* dinv = S + (size_t)n * n;          // [n]: 1 / L_ii
  int* perm = reinterpret_cast<int*>(dinv + n);
  __shared__ double sh_d0;
  __shared__ int sh_p, sh_r;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e - i * n;
    S[e] = A[(long long)i * lda + j];
  }
  for (int i = tid; i < n; i += nt) perm[i] = i;
  if (tid == 0) sh_r = n;
  __syncthreads();
  if (tid < 32) {
    double m = 0.0;
    for (int i = tid; i < n; i += 32) m = fmax(m, S[i * n + i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (tid == 0) sh_d0 = m;
  }
  __syncthreads();
  const double dmin = tol * sh_d0;
  for (int k = 0; k < n; ++k) {
    if (tid < 32) {   // pivot: largest remaining diagonal (first index on ties)
      double m = -1.0;
      int p = k;
      for (int i = k + tid; i < n; i += 32) {
        const double d = S[i * n + i];
        if (d > m) { m = d; p = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double m2 = __shfl_xor_sync(0xffffffffu, m, o);
        const int p2 = __shfl_xor_sync(0xffffffffu, p, o);
        if (m2 > m || (m2 == m && p2 < p)) { m = m2; p = p2; }
      }
      if (tid == 0) {
        sh_p = p;
        if (!(m > dmin) || !(sh_d0 > 0.0)) sh_r = k;
      }
    }
    __syncthreads();
    if (sh_r == k) break;
    const int p = sh_p;
    if (p != k) {   // symmetric swap of rows / columns k and p (full matrix)
      for (int j = tid; j < n; j += nt) {
        const double t = S[k * n + j];
        S[k * n + j] = S[p * n + j];
        S[p * n + j] = t;
      }
      __syncthreads();
      for (int i = tid; i < n; i += nt) {
        const double t = S[i * n + k];
        S[i * n + k] = S[i * n + p];
        S[i * n + p] = t;
      }
      if (tid == 0) {
        const int t = perm[k];
        perm[k] = perm[p];
        perm[p] = t;
      }
      __syncthreads();
    }
    const double lkk = sqrt(S[k * n + k]);
    __syncthreads();
    for (int i = k + 1 + tid; i < n; i += nt) S[i * n + k] /= lkk;
    if (tid == 0) S[k * n + k] = lkk;
    __syncthreads();
    // trailing update of the lower triangle and its mirror (rows and columns
    // of later pivots are read in full by the swaps above)
    const int m = n - k - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      S[i * n + j] -= S[i * n + k] * S[j * n + k];
    }
    __syncthreads();
  }
  const int r = sh_r;
  // L in the original row order: row perm[i] of L is row i of the factor
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, c = e - i * n;
    L[(long long)perm[i] * ldo + c] = (c < r && c <= i) ? S[i * n + c] : 0.0;
    M[(long long)i * ldo + c] = 0.0;
  }
  __syncthreads();
  // X = L1^-1 (r x r, lower), row by row: X_ii = 1 / L_ii in dinv, X_ic
  // (c < i) in the strictly upper triangle of S at S[c * n + i] (free once
  // the factor was copied out; L1 stays in the lower triangle)
  for (int i = tid; i < r; i += nt) dinv[i] = 1.0 / S[i * n + i];
  __syncthreads();
  for (int i = 1; i < r; ++i) {
    for (int c = tid; c < i; c += nt) {
      double acc = -S[i * n + c] * dinv[c];
      for (int j = c + 1; j < i; ++j) acc -= S[i * n + j] * S[c * n + j];
      S[c * n + i] = acc * dinv[i];
    }
    __syncthreads();
  }
  // M = P^T [L1^-T; 0]: row perm[i] (i < r) holds (L1^-T)_{i c} = X_{c i}
  for (int e = tid; e < r * r; e += nt) {
    const int i = e / r, c = e - i * r;
    M[(long long)perm[i] * ldo + c] = c == i ? dinv[i] : (c > i ? S[i * n + c] : 0.0);
  }
  if (tid == 0) *rank_dev = r;
}

// X = I, lam = diag(A): the start for nearly diagonal matrices
__global__ void k_identity_start(int n, const double* __restrict__ A, int lda, double* __restrict__ X,
                                 double* __restrict__ lam) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e - i * n;
    X[e] = i == j ? 1.0 : 0.0;
    if (i == j) lam[i] = A[(long long)i * lda + i];
  }
}

cudaError_t pchol(int n, const double* A, int lda, double tol, double* L, double* M, int ldo, int* rank_dev,
                  cudaStream_t s) {
  if (n <= 0 || n > SMALL_MAX || ldo < n) return cudaErrorInvalidValue;
  const size_t sm = sizeof(double) * ((size_t)n * n + n) + sizeof(int) * (size_t)n;
  cudaError_t e = allow_dynamic_smem((const void*)k_pchol, sm);
  if (e != cudaSuccess) return e;
  k_pchol<<<1, 1024, sm, s>>>(n, A, lda, tol, L, M, ldo, rank_dev);
  return cudaGetLastError();
}

cudaError_t eigh(int n, const double* A, int lda, double* w, double* V, double* ws, int refine_steps,
                 cudaStream_t s, double floor_rel, bool from_identity) {
  if (n <= 0) return cudaSuccess;
  if (n > SMALL_MAX) return cudaErrorInvalidValue;
  cudaError_t e;
  double* X = ws;                 // n x n current eigenvectors
  double* X2 = X + n * n;         // n x n
  double* R = X2 + n * n;         // n x n
  double* S = R + n * n;          // n x n
  double* AX = S + n * n;         // n x n
  double* lam = AX + n * n;       // n
  double* lam2 = lam + n;         // n
  double* anorm = lam2 + n;       // 8
  double* rest = anorm + 8;
  // diagnostics (BDG_PROFILE_EIGH): device time of the start, the refinement
  // and the ordering of this call, printed per call
  static const bool prof = getenv("BDG_PROFILE_EIGH") != nullptr;
  cudaEvent_t pe[4] = {};
  if (prof)
    for (auto& x : pe) cudaEventCreate(&x);
  if (prof) cudaEventRecord(pe[0], s);
  if (from_identity) {
    k_identity_start<<<(n * n + 255) / 256, 256, 0, s>>>(n, A, lda, X, lam2);
    if ((e = cudaGetLastError())) return e;
  } else if ((e = jacobi_multilevel(n, A, lda, lam2, X, rest, 0, floor_rel, 0.0, s))) {
    return e;
  }
  if (prof) cudaEventRecord(pe[1], s);
  k_frob<<<1, 1024, 0, s>>>(n, A, lda, anorm);
  double* cur = X;
  double* nxt = X2;
  for (int it = 0; it < refine_steps; ++it) {
    if ((e = dgemm_small(true, false, n, n, n, 1.0, cur, n, cur, n, 0.0, R, n, s))) return e;
    if ((e = dgemm_small(false, false, n, n, n, 1.0, A, lda, cur, n, 0.0, AX, n, s))) return e;
    if ((e = dgemm_small(true, false, n, n, n, 1.0, cur, n, AX, n, 0.0, S, n, s))) return e;
    k_oa_correction<<<1, 1024, 0, s>>>(n, R, S, anorm, lam);
    if ((e = cudaGetLastError())) return e;
    // X <- X + X E
    if ((e = cudaMemcpyAsync(nxt, cur, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, s))) return e;
    if ((e = dgemm_small(false, false, n, n, n, 1.0, cur, n, S, n, 1.0, nxt, n, s))) return e;
    double* t = cur; cur = nxt; nxt = t;
  }
  // Rotations driven by rounding noise (pairs just above the gap floor)
  // leave a second-order loss of orthogonality; two Newton-Schulz steps
  // X <- X (3 I - X^T X) / 2 remove it without rotating.
  for (int it = 0; refine_steps > 0 && it < 2; ++it) {
    if ((e = dgemm_small(true, false, n, n, n, 1.0, cur, n, cur, n, 0.0, R, n, s))) return e;
    k_newton_schulz<<<(n * n + 255) / 256, 256, 0, s>>>(n, R);
    if ((e = cudaGetLastError())) return e;
    if ((e = dgemm_small(false, false, n, n, n, 1.0, cur, n, R, n, 0.0, nxt, n, s))) return e;
    double* t = cur; cur = nxt; nxt = t;
  }
  if (prof) cudaEventRecord(pe[2], s);
  k_sort_eig<<<1, 256, 0, s>>>(n, refine_steps > 0 ? lam : lam2, cur, w, V);
  if (prof) {
    cudaEventRecord(pe[3], s);
    cudaEventSynchronize(pe[3]);
    float t0 = 0, t1 = 0, t2 = 0;
    cudaEventElapsedTime(&t0, pe[0], pe[1]);
    cudaEventElapsedTime(&t1, pe[1], pe[2]);
    cudaEventElapsedTime(&t2, pe[2], pe[3]);
    fprintf(stderr, "[bdg] eigh n %d %s start %.3f refine %.3f sort %.3f ms\n", n, from_identity ? "identity" : "jacobi",
            t0, t1, t2);
    for (auto& x : pe) cudaEventDestroy(x);
  }
  return cudaGetLastError();
}

}  // namespace bdg
