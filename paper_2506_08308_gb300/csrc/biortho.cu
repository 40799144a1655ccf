// bdg_biortho: stable bi-orthogonal Gram-Schmidt of complex blocks (Section
// 3.2; Theorem "Biorthogonality"), all arithmetic on the device.
//
//   twice  F <- F - Fl (Gl^H F),  G <- G - Gl (Fl^H G)          (CGS2)
//   S = F^H G = X Sigma Y^H,  keep sigma_i >= rtol sigma_max,
//   F <- F X Sigma^-1/2,  G <- G Y Sigma^-1/2                   (F^H G = I)
//
// Complex Grams come from the real Grams of the (re, im) columns (FP64
// accumulation).  The SVD of S is read off the Hermitian Jordan-Wielandt
// matrix H = [[0, S], [S^H, 0]] (eigenvalues +-sigma, eigenvectors
// [x; y] / sqrt2), itself solved through its real embedding
// R = [[Re H, -Im H], [Im H, Re H]] whose eigenvalues come in equal pairs
// (the vectors v and i v); one vector per complex direction is kept by a
// Gram-Schmidt against the kept vectors and their images under i.  The step
// runs twice; the second pass restores F^H G = I to working precision after
// the rounding of the first.
#include <cmath>
#include <vector>

#include "blas.cuh"
#include "dense.cuh"
#include "plan.cuh"

namespace bdg {
namespace {

constexpr int BIO_MAX_COLS = SMALL_MAX / 4;  // the real embedding of H is 4 ncol wide

// Complex matrix C (a x b) from the real Gram G (2a x 2b) of complex columns:
// C = A^H B (conj = 1) or A^T B (conj = 0); written as the real pair-layout
// coefficient matrix K (2a x 2b) of the product by C, scaled by alpha:
// y_re += alpha (a_re Cr - a_im Ci), y_im += alpha (a_re Ci + a_im Cr).
__global__ void k_cplx_coef(const double* __restrict__ G, int a, int b, double alpha, double* __restrict__ K) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < a * b; e += gridDim.x * blockDim.x) {
    const int p = e / b, q = e - p * b;
    const int Q2 = 2 * b;
    const double rr = G[(2 * p) * Q2 + 2 * q], ii = G[(2 * p + 1) * Q2 + 2 * q + 1];
    const double ri = G[(2 * p) * Q2 + 2 * q + 1], ir = G[(2 * p + 1) * Q2 + 2 * q];
    const double cr = alpha * (rr + ii), ci = alpha * (ri - ir);   // conj(a) . b
    K[(2 * p) * Q2 + 2 * q] = cr;
    K[(2 * p + 1) * Q2 + 2 * q] = -ci;
    K[(2 * p) * Q2 + 2 * q + 1] = ci;
    K[(2 * p + 1) * Q2 + 2 * q + 1] = cr;
  }
}

// R = real embedding of H = [[0, S], [S^H, 0]], S = F^H G (n x n complex from
// the real Gram G, 2n x 2n).  H is 2n x 2n, R is 4n x 4n (row-major).
__global__ void k_jw_embed(const double* __restrict__ G, int n, double* __restrict__ R) {
  const int m = 2 * n, M = 4 * n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * M; e += gridDim.x * blockDim.x) {
    const int i = e / M, j = e - i * M;
    const int bi = i / m, bj = j / m, hi = i - bi * m, hj = j - bj * m;  // block of R, entry of H
    double hr = 0.0, him = 0.0;                                          // H[hi][hj]
    if (hi < n && hj >= n) {                                             // S[hi][hj - n]
      const int p = hi, q = hj - n, Q2 = 2 * n;
      hr = G[(2 * p) * Q2 + 2 * q] + G[(2 * p + 1) * Q2 + 2 * q + 1];
      him = G[(2 * p) * Q2 + 2 * q + 1] - G[(2 * p + 1) * Q2 + 2 * q];
    } else if (hi >= n && hj < n) {                                      // conj(S[hj][hi - n])
      const int p = hj, q = hi - n, Q2 = 2 * n;
      hr = G[(2 * p) * Q2 + 2 * q] + G[(2 * p + 1) * Q2 + 2 * q + 1];
      him = -(G[(2 * p) * Q2 + 2 * q + 1] - G[(2 * p + 1) * Q2 + 2 * q]);
    }
    double v;
    if (bi == bj) v = hr;
    else if (bi == 0) v = -him;   // upper right: -Im H
    else v = him;                 // lower left: Im H
    R[e] = v;
  }
}

// Choice of one real eigenvector per complex direction.  R commutes with J,
// J [a; b] = [-b; a] (multiplication by i), so each eigenspace is J-invariant
// and a complex eigenvector v = a + i b shows up as the real pair (e, J e).
// Candidates are taken from the largest eigenvalue down and kept when they
// are not (numerically) in the span of the kept vectors and their J-images
// -- a Gram-Schmidt against both, which also handles degenerate clusters
// where the eigensolver returns an arbitrary real basis of the eigenspace.
// One CTA; out: E (M x M row-major, kept vectors in columns 0..), wsel, *count.
__global__ void k_jw_select(const double* __restrict__ V, const double* __restrict__ w, int M, int c_lo,
                            int max_keep, double* __restrict__ E, double* __restrict__ wsel, int* count) {
  extern __shared__ double sh[];
  double* e = sh;            // [M]
  double* red = sh + M;      // [32]
  const int tid = threadIdx.x, h = M / 2;
  int kept = 0;
  for (int c = M - 1; c >= c_lo && kept < max_keep; --c) {
    for (int i = tid; i < M; i += blockDim.x) e[i] = V[(long long)i * M + c];
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int j = 0; j < kept; ++j) {
        // d1 = E_j . e, d2 = (J E_j) . e with J E_j = [-E_j(h:); E_j(:h)]
        double d1 = 0.0, d2 = 0.0;
        for (int i = tid; i < M; i += blockDim.x) {
          const double ej = E[(long long)i * M + j];
          const double jej = i < h ? -E[(long long)(i + h) * M + j] : E[(long long)(i - h) * M + j];
          d1 += ej * e[i];
          d2 += jej * e[i];
        }
        for (int o = 16; o > 0; o >>= 1) {
          d1 += __shfl_xor_sync(0xffffffffu, d1, o);
          d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        }
        if ((tid & 31) == 0) { red[tid >> 5] = d1; red[16 + (tid >> 5)] = d2; }
        __syncthreads();
        if (tid == 0) {
          double a = 0.0, b = 0.0;
          for (int q = 0; q < (int)blockDim.x / 32; ++q) { a += red[q]; b += red[16 + q]; }
          red[0] = a;
          red[16] = b;
        }
        __syncthreads();
        d1 = red[0];
        d2 = red[16];
        __syncthreads();
        for (int i = tid; i < M; i += blockDim.x) {
          const double ej = E[(long long)i * M + j];
          const double jej = i < h ? -E[(long long)(i + h) * M + j] : E[(long long)(i - h) * M + j];
          e[i] -= d1 * ej + d2 * jej;
        }
        __syncthreads();
      }
    }
    double nn = 0.0;
    for (int i = tid; i < M; i += blockDim.x) nn += e[i] * e[i];
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    if ((tid & 31) == 0) red[tid >> 5] = nn;
    __syncthreads();
    if (tid == 0) {
      double a = 0.0;
      for (int q = 0; q < (int)blockDim.x / 32; ++q) a += red[q];
      red[0] = a;
    }
    __syncthreads();
    const double nrm = sqrt(red[0]);
    __syncthreads();
    if (nrm > 0.5) {   // a unit candidate mostly outside the kept span
      for (int i = tid; i < M; i += blockDim.x) E[(long long)i * M + kept] = e[i] / nrm;
      if (tid == 0) wsel[kept] = w[c];
      ++kept;
    }
    __syncthreads();
  }
  if (tid == 0) *count = kept;
}

// From the selected eigenvectors e_k = [a; b] of R (4n x 4n, columns idx[k]):
// v = a + i b, x = sqrt2 v[0:n], y = sqrt2 v[n:2n], scaled by sc[k]; written
// as pair-layout coefficient matrices KX, KY (2n x 2r, ld 2r) of F X and G Y.
__global__ void k_jw_coef(const double* __restrict__ V, int n, int r, const int* __restrict__ idx,
                          const double* __restrict__ sc, double* __restrict__ KX, double* __restrict__ KY) {
  const int M = 4 * n, R2 = 2 * r;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * r; e += gridDim.x * blockDim.x) {
    const int p = e / r, k = e - p * r;
    const int c = idx[k];
    const double s = 1.4142135623730951 * sc[k];
    for (int part = 0; part < 2; ++part) {
      const int row = part * n + p;                 // entry of v
      const double cr = s * V[(long long)row * M + c];
      const double ci = s * V[(long long)(2 * n + row) * M + c];
      double* K = part ? KY : KX;
      K[(2 * p) * R2 + 2 * k] = cr;
      K[(2 * p + 1) * R2 + 2 * k] = -ci;
      K[(2 * p) * R2 + 2 * k + 1] = ci;
      K[(2 * p + 1) * R2 + 2 * k + 1] = cr;
    }
  }
}

template <typename R>
struct Bio {
  typedef typename CT<R>::T T;
  bdg_plan_t plan;
  cudaStream_t s;
  long long n3;
  double* small = nullptr;   // matrices
  double* ews = nullptr;     // eigensolver workspace
  void* gws = nullptr;
  size_t gws_bytes = 0;
  T* tmp = nullptr;          // 2 ncol columns

  PairBlock<R> blk(const void* p, int cols) const { return PairBlock<R>{(const T*)p, n3, n3, cols}; }

  bdg_status gram(const void* A, int a, const void* B, int b, double* G) {
    BDG_CUDA_TRY(plan, gram_pairs<R>(blk(A, a), blk(B, b), G, gws, gws_bytes, s));
    return BDG_OK;
  }

  // Y (cols b) += -Bk (Ck^H Y) for the locked pair, twice, on both blocks
  bdg_status cgs2(void* F, void* G, int ncol, const void* Fl, const void* Gl, int nlock) {
    double* Gm = small;
    double* K = small + 4 * 256 * 256;
    for (int pass = 0; pass < 2; ++pass) {
      for (int side = 0; side < 2; ++side) {
        void* Y = side ? G : F;
        const void* Bk = side ? Gl : Fl;   // the block that spans Y's space
        const void* Ck = side ? Fl : Gl;   // its bi-orthogonal partner
        bdg_status st = gram(Ck, nlock, Y, ncol, Gm);
        if (st) return st;
        k_cplx_coef<<<(nlock * ncol + 255) / 256, 256, 0, s>>>(Gm, nlock, ncol, 1.0, K);
        BDG_CUDA_TRY(plan, cudaGetLastError());
        BDG_CUDA_TRY(plan, update_pairs<R>(blk(Bk, nlock), K, 2 * ncol, 1.0, (T*)Y, n3, ncol, s, -1.0));
      }
    }
    return BDG_OK;
  }

  // one bi-orthonormalization of the first ncol columns of F, G; *rank out
  bdg_status biortho_once(void* F, void* G, int ncol, double rtol, int* rank) {
    *rank = 0;
    double* Gm = small;                       // 2n x 2n real Gram
    double* Rm = small + 4 * 256 * 256;       // 4n x 4n
    double* Vm = Rm + 160 * 160;              // eigenvectors
    double* w = Vm + 160 * 160;               // eigenvalues
    double* KX = w + 256;                     // 2n x 2r
    double* KY = KX + 80 * 80;
    double* sc = KY + 80 * 80;
    int* didx = (int*)(sc + 128);
    bdg_status st = gram(F, ncol, G, ncol, Gm);
    if (st) return st;
    const int M = 4 * ncol;
    k_jw_embed<<<(M * M + 255) / 256, 256, 0, s>>>(Gm, ncol, Rm);
    BDG_CUDA_TRY(plan, cudaGetLastError());
    BDG_CUDA_TRY(plan, eigh(M, Rm, M, w, Vm, ews, 3, s));
    std::vector<double> hw(M);
    BDG_CUDA_TRY(plan, cudaMemcpyAsync(hw.data(), w, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
    BDG_CUDA_TRY(plan, cudaStreamSynchronize(s));
    const double smax = hw[M - 1];
    if (!(smax > 0)) return BDG_OK;
    int c_lo = M - 1;
    while (c_lo > 0 && hw[c_lo - 1] >= rtol * smax) --c_lo;
    double* E = sc + 256;                      // M x M (kept vectors in its first columns)
    double* wsel = E + 160 * 160;
    int* dcount = (int*)(wsel + 128);
    k_jw_select<<<1, 256, sizeof(double) * (M + 32), s>>>(Vm, w, M, c_lo, ncol, E, wsel, dcount);
    BDG_CUDA_TRY(plan, cudaGetLastError());
    int r = 0;
    std::vector<double> hsel(ncol);
    BDG_CUDA_TRY(plan, cudaMemcpyAsync(&r, dcount, sizeof(int), cudaMemcpyDeviceToHost, s));
    BDG_CUDA_TRY(plan, cudaMemcpyAsync(hsel.data(), wsel, sizeof(double) * ncol, cudaMemcpyDeviceToHost, s));
    BDG_CUDA_TRY(plan, cudaStreamSynchronize(s));
    if (r == 0) return BDG_OK;
    std::vector<int> idx(r);
    std::vector<double> scale(r);
    for (int k = 0; k < r; ++k) {
      idx[k] = k;
      scale[k] = 1.0 / std::sqrt(hsel[k]);
    }
    BDG_CUDA_TRY(plan, cudaMemcpyAsync(didx, idx.data(), sizeof(int) * r, cudaMemcpyHostToDevice, s));
    BDG_CUDA_TRY(plan, cudaMemcpyAsync(sc, scale.data(), sizeof(double) * r, cudaMemcpyHostToDevice, s));
    k_jw_coef<<<(ncol * r + 255) / 256, 256, 0, s>>>(E, ncol, r, didx, sc, KX, KY);
    BDG_CUDA_TRY(plan, cudaGetLastError());
    // F X, G Y into tmp, then back, the remaining columns zeroed
    T* tf = tmp;
    T* tg = tmp + (long long)ncol * n3;
    BDG_CUDA_TRY(plan, update_pairs<R>(blk(F, ncol), KX, 2 * r, 0.0, tf, n3, r, s));
    BDG_CUDA_TRY(plan, update_pairs<R>(blk(G, ncol), KY, 2 * r, 0.0, tg, n3, r, s));
    const size_t colb = sizeof(T) * (size_t)n3;
    BDG_CUDA_TRY(plan, cudaMemcpyAsync(F, tf, colb * r, cudaMemcpyDeviceToDevice, s));
    BDG_CUDA_TRY(plan, cudaMemcpyAsync(G, tg, colb * r, cudaMemcpyDeviceToDevice, s));
    if (r < ncol) {
      BDG_CUDA_TRY(plan, cudaMemsetAsync((char*)F + colb * r, 0, colb * (ncol - r), s));
      BDG_CUDA_TRY(plan, cudaMemsetAsync((char*)G + colb * r, 0, colb * (ncol - r), s));
    }
    *rank = r;
    return BDG_OK;
  }
};

template <typename R>
bdg_status biortho_run(bdg_plan_t plan, void* F, void* G, int ncol, const void* Fl, const void* Gl, int nlock,
                       int* rank, cudaStream_t s) {
  Bio<R> b;
  b.plan = plan;
  b.s = s;
  b.n3 = 3 * plan->grid.npts;
  const int wide = std::max(ncol, nlock);
  b.gws_bytes = gram_workspace_bytes(wide, wide, b.n3);
  const size_t small_doubles = 4 * 256 * 256 + 3 * 160 * 160 + 2 * 80 * 80 + 2048;
  bdg_status st;
  if ((st = ensure(plan, SLOT_GRAM_WS, b.gws_bytes)) || (st = ensure(plan, SLOT_SMALL, sizeof(double) * small_doubles)) ||
      (st = ensure(plan, SLOT_AUX, sizeof(double) * eigh_workspace_doubles(SMALL_MAX))) ||
      (st = ensure(plan, SLOT_VEC_A, sizeof(typename CT<R>::T) * 2 * (size_t)ncol * b.n3)))
    return st;
  b.gws = plan->scratch[SLOT_GRAM_WS].ptr;
  b.small = (double*)plan->scratch[SLOT_SMALL].ptr;
  b.ews = (double*)plan->scratch[SLOT_AUX].ptr;
  b.tmp = (typename CT<R>::T*)plan->scratch[SLOT_VEC_A].ptr;
  if (nlock > 0 && (st = b.cgs2(F, G, ncol, Fl, Gl, nlock))) return st;
  const double rtol = sizeof(R) == 8 ? 1e-12 : 1e-6;
  int r1 = 0, r2 = 0;
  if ((st = b.biortho_once(F, G, ncol, rtol, &r1))) return st;
  if (r1 > 0 && (st = b.biortho_once(F, G, r1, rtol, &r2))) return st;
  *rank = r2;
  if (r2 == 0) return fail(plan, BDG_ERR_BREAKDOWN, "F^H G has no nonzero singular value");
  return BDG_OK;
}

}  // namespace
}  // namespace bdg

using namespace bdg;

extern "C" bdg_status bdg_biortho(bdg_plan_t plan, int dtype, void* F, void* G, int ncol, const void* Fl,
                                  const void* Gl, int nlock, int* rank, void* stream) {
  if (!plan) return fail(nullptr, BDG_ERR_INVALID, "plan is NULL");
  if (!rank) return fail(plan, BDG_ERR_INVALID, "rank must be a host pointer");
  *rank = 0;
  if (dtype != BDG_C128 && dtype != BDG_C64) return fail(plan, BDG_ERR_INVALID, "dtype must be BDG_C128 or BDG_C64");
  if (ncol < 1 || nlock < 0) return fail(plan, BDG_ERR_INVALID, "need ncol >= 1 and nlock >= 0");
  if (ncol > BIO_MAX_COLS)
    return fail(plan, BDG_ERR_UNSUPPORTED, "bdg_biortho handles at most " + std::to_string(BIO_MAX_COLS) + " columns");
  if (nlock > 256) return fail(plan, BDG_ERR_UNSUPPORTED, "at most 256 locked columns");
  if (!F || !G || (nlock > 0 && (!Fl || !Gl))) return fail(plan, BDG_ERR_INVALID, "F, G (and Fl, Gl) must be device pointers");
  const size_t esz = dtype == BDG_C128 ? 16 : 8;
  if (((uintptr_t)F | (uintptr_t)G | (uintptr_t)Fl | (uintptr_t)Gl) % esz)
    return fail(plan, BDG_ERR_INVALID, "blocks not aligned to the element size");
  const size_t bytes = esz * 3 * (size_t)plan->grid.npts * ncol;
  const char *fb = (const char*)F, *gb = (const char*)G;
  if (fb < gb + bytes && gb < fb + bytes) return fail(plan, BDG_ERR_INVALID, "F and G overlap");
  if (bdg_status sd = check_device(plan)) return sd;
  plan->last_stream = stream;
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == BDG_C128) return biortho_run<double>(plan, F, G, ncol, Fl, Gl, nlock, rank, s);
  return biortho_run<float>(plan, F, G, ncol, Fl, Gl, nlock, rank, s);
}
