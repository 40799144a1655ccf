// bdg_solve: the structure-preserving subspace iteration for
// the k smallest positive excitations (Sections 2.2-2.3, 3.1-3.2).
//
// The operator is real for a real ground state (Section 2.2), so the
// iteration works with real vectors; two real FG vectors share one complex
// vector (real and imaginary parts), which is how the complex product
// kernels apply M to both at once.  A block of 2P real columns is a
// PairBlock of P complex columns; the f-part of every column holds a
// u-side basis vector (U) and the g-part a v-side basis vector (V).
//
// One iteration (block structure-preserving Rayleigh-Ritz, after the
// LOBP4dCG family the paper's eigensolver builds on):
//   Ritz block (F, G) with F^T G = I, images HF = H_+ F, HG = H_- G,
//   residuals R_f = HF - G w, R_g = HG - F w (components of G along Z_f and
//   of F along Z_g, invisible to the projected pencil, set in closed form),
//   directions D = T_sigma R for the unconverged columns, deflated against
//   Z_f / Z_g, and the previous update P;
//   CGS2 of [D P] against (F, G), SVD bi-orthonormalization inside [D P]
//   (rank cut), projected pencil K_+ = U^T H_+ U, K_- = V^T H_- V on
//   U = [F D P], V = [G D P], eigen-decomposition
//   K_+ = Q L Q^T, C = L^1/2 Q^T K_- Q L^1/2 = Z W^2 Z^T, and the m smallest
//   positive w with coefficients p = Q L^-1/2 Z, q = Q L^1/2 Z / w.
// Precision: FP64 runs everything in FP64.  MIXED runs the iteration with
// FP32 vectors and products (Gram entries still summed in FP64) until the
// FP32 floor, then continues in FP64 from the FP32 Ritz vectors.  All
// projected problems are solved in FP64 accuracy (dense.cuh).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "apply.cuh"
#include "blas.cuh"
#include "common.cuh"
#include "dense.cuh"
#include "inner.cuh"
#include "kdiag.cuh"
#include "plan.cuh"

namespace bdg {

namespace {

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
// counter-based normal deviates: SplitMix64 (Steele, Lea & Flood 2014) of
// (seed, index), Box-Muller on two 53-bit uniforms.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

template <typename R>
__global__ void k_random_block(typename CT<R>::T* out, long long total, unsigned long long seed) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long a = splitmix64(seed ^ splitmix64(2 * i));
    const unsigned long long b = splitmix64(seed ^ splitmix64(2 * i + 1));
    const double u1 = ((a >> 11) + 1) * (1.0 / 9007199254740993.0);
    const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    const double r = sqrt(-2.0 * log(u1));
    out[i] = mk((R)(r * cos(2.0 * M_PI * u2)), (R)(r * sin(2.0 * M_PI * u2)));
  }
}

// pack real parts of complex FG vectors X0[2p], X0[2p+1] into pair p
template <typename R>
__global__ void k_pack_real(const double2* __restrict__ X0, int ncols, long long vlen,
                            typename CT<R>::T* __restrict__ out) {
  const long long npairs = (ncols + 1) / 2;
  const long long total = npairs * vlen;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long p = e / vlen, r = e - p * vlen;
    const R a = (R)X0[(2 * p) * vlen + r].x;
    const R b = (2 * p + 1 < ncols) ? (R)X0[(2 * p + 1) * vlen + r].x : (R)0;
    out[e] = mk(a, b);
  }
}

// (u, v) = (f + g, f - g) of real column c of a pair bank, as complex128 with zero imaginary part
template <typename R>
__global__ void k_unpack_uv(const typename CT<R>::T* __restrict__ bank, long long np, int k,
                            const double* __restrict__ scale, double2* __restrict__ UV) {
  const long long total = (long long)k * 3 * np;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long c = e / (3 * np), r = e - c * 3 * np;
    const long long p = c / 2;
    const int part = (int)(c & 1);
    const typename CT<R>::T f2 = bank[p * 6 * np + r];
    const typename CT<R>::T g2 = bank[p * 6 * np + 3 * np + r];
    const double f = part ? (double)f2.y : (double)f2.x;
    const double g = part ? (double)g2.y : (double)g2.x;
    const double s = scale[c];
    UV[c * 6 * np + r] = make_double2(s * (f + g), 0.0);
    UV[c * 6 * np + 3 * np + r] = make_double2(s * (f - g), 0.0);
  }
}

// per real column: sum of squares over rows of a pair block (pair p, part s -> col 2p+s),
// as partial sums per CTA row range: part[(p * gridDim.x + blockIdx.x) * 2 + s]
constexpr int CN_BLOCKS = 64;
template <typename R>
__global__ void k_colnorm2(const typename CT<R>::T* __restrict__ A, long long ld, long long n, int pairs,
                           double* __restrict__ part) {
  __shared__ double red[2][32];
  const int p = blockIdx.y;
  double s0 = 0.0, s1 = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    const typename CT<R>::T v = A[(long long)p * ld + r];
    s0 += (double)v.x * (double)v.x;
    s1 += (double)v.y * (double)v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = s0; red[1][threadIdx.x >> 5] = s1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < (int)blockDim.x / 32; ++q) { a += red[0][q]; b += red[1][q]; }
    part[((long long)p * gridDim.x + blockIdx.x) * 2] = a;
    part[((long long)p * gridDim.x + blockIdx.x) * 2 + 1] = b;
  }
}

// out[2p + s] = sum of the nb partials of k_colnorm2 in a fixed order
__global__ void k_colnorm_reduce(const double* __restrict__ part, int nb, int pairs, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= 2 * pairs) return;
  const int p = c / 2, s = c - 2 * p;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += part[((long long)p * nb + b) * 2 + s];
  out[c] = t;
}

// scale the f-part of real column c by af[c] and the g-part by ag[c]
template <typename R>
__global__ void k_scale_parts(typename CT<R>::T* __restrict__ bank, long long np, int pairs,
                              const double* __restrict__ af, const double* __restrict__ ag) {
  const long long vlen = 6 * np, total = (long long)pairs * vlen;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long p = e / vlen, r = e - p * vlen;
    const double* a = r < 3 * np ? af : ag;
    typename CT<R>::T v = bank[e];
    bank[e] = mk((R)(v.x * a[2 * p]), (R)(v.y * a[2 * p + 1]));
  }
}

// Symmetric diagonal scaling Kt = D^-1/2 K D^-1/2 with D_ii = K_ii for
// i >= nfix and 1 below (the Ritz block, whose K block is already diag(omega):
// scaling it to I would make a cluster at 1); rows with K_ii <= 0 (zero
// columns of the basis) become zero.  dsq = D^1/2, dinv = D^-1/2.
__global__ void k_diag_scale(int n, int nfix, const double* __restrict__ K, int ldk, double* __restrict__ Kt,
                             double* __restrict__ dsq, double* __restrict__ dinv) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e - i * n;
    const double di = i < nfix ? 1.0 : K[(long long)i * ldk + i];
    const double dj = j < nfix ? 1.0 : K[(long long)j * ldk + j];
    const double si = di > 0 ? 1.0 / sqrt(di) : 0.0, sj = dj > 0 ? 1.0 / sqrt(dj) : 0.0;
    Kt[e] = K[(long long)i * ldk + j] * si * sj;
    if (j == 0) {
      dsq[i] = di > 0 ? sqrt(di) : 0.0;
      dinv[i] = si;
    }
  }
}

// Jordan-Wielandt matrix J = [[0, S], [S^T, 0]] (2n x 2n) of S (n x n, lds)
__global__ void k_jordan_wielandt(int n, const double* __restrict__ S, int lds, double* __restrict__ J) {
  const int m = 2 * n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    const int i = e / m, j = e - i * m;
    double v = 0.0;
    if (i < n && j >= n) v = S[(long long)i * lds + (j - n)];
    else if (i >= n && j < n) v = S[(long long)j * lds + (i - n)];
    J[e] = v;
  }
}
// From eigenvectors V (2n x 2n, ld 2n) of J, columns c0.., r of them:
// Tf[i][k] = sqrt2 V[i][c0+k] * sc[k], Tg[i][k] = sqrt2 V[n+i][c0+k] * sc[k]  (i < n)
__global__ void k_jw_split(int n, int r, int c0, const double* __restrict__ V, const double* __restrict__ sc,
                           double* __restrict__ Tf, double* __restrict__ Tg, int ldt) {
  const int m = 2 * n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * r; e += gridDim.x * blockDim.x) {
    const int i = e / r, k = e - i * r;
    const double s2 = 1.4142135623730951 * sc[k];
    Tf[(long long)i * ldt + k] = s2 * V[(long long)i * m + c0 + k];
    Tg[(long long)i * ldt + k] = s2 * V[(long long)(n + i) * m + c0 + k];
  }
}

unsigned nblk(long long total) {
  long long b = (total + 255) / 256;
  if (b > 152LL * 8) b = 152LL * 8;
  return (unsigned)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------------------
// host-side helpers for small matrices
// ---------------------------------------------------------------------------
struct HostMat {
  int r = 0, c = 0;
  std::vector<double> a;
  HostMat() {}
  HostMat(int r_, int c_) : r(r_), c(c_), a((size_t)r_ * c_, 0.0) {}
  double& operator()(int i, int j) { return a[(size_t)i * c + j]; }
  double operator()(int i, int j) const { return a[(size_t)i * c + j]; }
};

}  // namespace

// ---------------------------------------------------------------------------
// The solver
// ---------------------------------------------------------------------------
template <typename R>
class Solver {
 public:
  typedef typename CT<R>::T T;

  Solver(bdg_plan_t plan, cudaStream_t s, int m) : plan_(plan), s_(s), m_(m) {
    np_ = plan->grid.npts;
    n3_ = 3 * np_;
    vlen_ = 6 * np_;
    mp_ = (m + 1) / 2;                 // pairs of the Ritz block
    cap_ = 3 * mp_ + 1;                // pairs of a basis bank
  }
  ~Solver() { release(); }

  bdg_status init_buffers() {
    const size_t vb = sizeof(T) * (size_t)vlen_;
    void* p = nullptr;
    for (int b = 0; b < 2; ++b) {
      if (alloc(&p, vb * cap_)) return fail(plan_, BDG_ERR_NOMEM, "solver basis allocation failed");
      U_[b] = (T*)p;
      if (alloc(&p, vb * cap_)) return fail(plan_, BDG_ERR_NOMEM, "solver basis allocation failed");
      HU_[b] = (T*)p;
    }
    if (alloc(&p, vb * mp_)) return fail(plan_, BDG_ERR_NOMEM, "solver residual allocation failed");
    Rb_ = (T*)p;
    if (alloc(&p, vb * 2 * mp_)) return fail(plan_, BDG_ERR_NOMEM, "solver work allocation failed");
    Wb_ = (T*)p;
    if (alloc(&p, vb * 2 * mp_)) return fail(plan_, BDG_ERR_NOMEM, "solver work allocation failed");
    HWb_ = (T*)p;
    if (alloc(&p, vb * mp_)) return fail(plan_, BDG_ERR_NOMEM, "solver work allocation failed");
    Pb_ = (T*)p;
    if (alloc(&p, vb * mp_)) return fail(plan_, BDG_ERR_NOMEM, "solver work allocation failed");
    HPb_ = (T*)p;
    big_ = 2 * cap_;
    bdg_status sl = alloc_lane();
    if (sl) return sl;
    if (overlap_) {
      if (cudaStreamCreateWithFlags(&lane2_.s, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&ev_fork_, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ev_join_, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ev_img_, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(plan_, BDG_ERR_CUDA, "second solver stream could not be created");
      }
      swap_lane(lane2_);
      sl = alloc_lane();
      swap_lane(lane2_);
      if (sl) return sl;
    }
    zf_ = (const T*)(sizeof(R) == 8 ? (const void*)plan_->zf64 : (const void*)plan_->zf32);
    zg_ = (const T*)(sizeof(R) == 8 ? (const void*)plan_->zg64 : (const void*)plan_->zg32);
    if (inner_steps_ > 0) {
      auto al = [this](void** q, size_t b) { return alloc(q, b); };
      bdg_status st = inner_fp32_ ? in32_.init(plan_, mp_, al) : in64_.init(plan_, mp_, al);
      if (st) return st;
    }
    return BDG_OK;
  }

  // Gram workspace, small matrices, column-norm partials and pinned staging
  // of the current lane
  bdg_status alloc_lane() {
    void* p = nullptr;
    gws_bytes_ = gram_workspace_bytes(cap_, cap_, n3_);
    if (alloc(&p, gws_bytes_)) return fail(plan_, BDG_ERR_NOMEM, "gram workspace allocation failed");
    gws_ = p;
    const size_t mat = (size_t)big_ * big_;
    const size_t sd = NMAT * mat + eigh_workspace_doubles(SMALL_MAX) + 64 * (size_t)big_;
    if (alloc(&p, sizeof(double) * sd)) return fail(plan_, BDG_ERR_NOMEM, "small workspace allocation failed");
    dsm_ = (double*)p;
    for (int i = 0; i < NMAT; ++i) dmat_[i] = dsm_ + i * mat;
    dvec_ = dsm_ + NMAT * mat;
    dws_ = dvec_ + 64 * (size_t)big_;
    if (alloc(&p, sizeof(double) * 2 * CN_BLOCKS * (size_t)cap_))
      return fail(plan_, BDG_ERR_NOMEM, "column-norm workspace allocation failed");
    cnpart_ = (double*)p;
    if (alloc(&p, 256)) return fail(plan_, BDG_ERR_NOMEM, "solver workspace allocation failed");
    dint_ = (int*)p;
    if (cudaMallocHost((void**)&pinned_, sizeof(double) * PIN_DOUBLES) != cudaSuccess) {
      cudaGetLastError();
      pinned_ = nullptr;
      return fail(plan_, BDG_ERR_NOMEM, "pinned staging allocation failed");
    }
    pin_off_ = 0;
    return BDG_OK;
  }

  // search directions D = (H_+^-1 r_f, H_-^-1 r_g) approximated by inner PCG
  // in FP32 or FP64, or T_sigma r when the inner solver is off
  bdg_status directions(T* W, int pairs) {
    if (inner_steps_ <= 0) return precondition(W, W, pairs);
    if (inner_fp32_) return in32_.template run<R>(W, W, pairs, inner_steps_, sigma_, s_);
    if constexpr (sizeof(R) == 8) return in64_.template run<R>(W, W, pairs, inner_steps_, sigma_, s_);
    return fail(plan_, BDG_ERR_INVALID, "an FP32 phase runs its inner solver in FP32");
  }

  // ---- block views ------------------------------------------------------
  PairBlock<R> fpart(const T* bank, int pair0, int pairs) const {
    return PairBlock<R>{bank + (long long)pair0 * vlen_, vlen_, n3_, pairs};
  }
  PairBlock<R> gpart(const T* bank, int pair0, int pairs) const {
    return PairBlock<R>{bank + (long long)pair0 * vlen_ + n3_, vlen_, n3_, pairs};
  }
  T* fptr(T* bank, int pair0) const { return bank + (long long)pair0 * vlen_; }
  T* gptr(T* bank, int pair0) const { return bank + (long long)pair0 * vlen_ + n3_; }

  // ---- primitive wrappers ----------------------------------------------
  // G (2P x 2Q) of real columns, FP64 on device
  // Grams for which FP32 accuracy suffices -- every Gram of the FP32 phase,
  // and the first pass of the two-pass Gram-Schmidt, whose second pass
  // (double-float) removes what the first leaves -- run on the tensor cores
  // (split-BF16 slices, FP32 accumulation); the rest in double-float.
  bool tc_ = !getenv("BDG_GRAM_TC") || atoi(getenv("BDG_GRAM_TC")) != 0;
  static constexpr long long TC_MIN_ROWS = 2048;
  bdg_status gram(const PairBlock<R>& A, const PairBlock<R>& B, double* G, bool upper = false,
                  bool fp32_enough = sizeof(R) == 4) {
    if (tc_ && fp32_enough && A.n >= TC_MIN_ROWS && gram_tc_supported(A.cols, B.cols)) {
      BDG_CUDA_TRY(plan_, gram_pairs_tc<R>(A, B, G, gws_, gws_bytes_, s_));
      return BDG_OK;
    }
    BDG_CUDA_TRY(plan_, gram_pairs<R>(A, B, G, gws_, gws_bytes_, s_, upper));
    return BDG_OK;
  }
  // Y (Q pairs at y) = beta Y + A C with C on the device (2P rows used, ldc)
  bdg_status update_dev(const PairBlock<R>& A, const double* dC, int ldc, double beta, T* y, int Q,
                        double alpha = 1.0) {
    if (Q == 0) return BDG_OK;
    BDG_CUDA_TRY(plan_, update_pairs<R>(A, dC, ldc, beta, y, vlen_, Q, s_, alpha));
    if (sizeof(R) == 8) plan_->stats.flops_update_df += 2.0 * (double)A.n * (2.0 * A.cols) * (2.0 * Q);
    return BDG_OK;
  }
  // the same with a host matrix (small data-movement matrices: diagonals, selections)
  bdg_status update(const PairBlock<R>& A, const HostMat& C, double beta, T* y, int Q) {
    if (Q == 0) return BDG_OK;
    double* dC = dmat_[MAT_HOST];
    bdg_status st = upload(dC, C.a.data(), C.a.size());
    if (st) return st;
    return update_dev(A, dC, C.c, beta, y, Q);
  }
  bdg_status apply_fg(const T* x, T* y, int pairs) {
    if (pairs == 0) return BDG_OK;
    bdg_status st = apply_internal(plan_, BDG_FG, sizeof(R) == 8 ? BDG_C128 : BDG_C64, x, y, pairs, s_, nullptr);
    if (sizeof(R) == 8) plan_->stats.applies_fp64 += 2 * pairs;
    else plan_->stats.applies_fp32 += 2 * pairs;
    return st;
  }
  bdg_status precondition(const T* x, T* y, int pairs) {
    if (pairs == 0) return BDG_OK;
    KdArgs<R> g;
    g.grid = &plan_->grid;
    g.x = x;
    g.y = y;
    g.nplanes = 6LL * pairs;
    for (int a = 0; a < 3; ++a)
      g.tw[a] = (const T*)(sizeof(R) == 8 ? (const void*)plan_->tw64[a] : (const void*)plan_->tw32[a]);
    g.shift = sigma_;
    g.scale = 0.5;
    g.stream = s_;
    BDG_CUDA_TRY(plan_, kdiag_launch<R>(g));
    return BDG_OK;
  }
  // Host <-> device copies of small data go through a pinned staging arena:
  // a copy from pageable memory would make the stream drain first.  Staged
  // uploads stay queued behind the work in flight; the arena is recycled at
  // every point where the host waits for the stream anyway.
  bdg_status sync_stream() {
    BDG_CUDA_TRY(plan_, cudaStreamSynchronize(s_));
    pin_off_ = 0;
    return BDG_OK;
  }
  double* stage(size_t n) {
    if (pin_off_ + n > PIN_DOUBLES) {
      if (sync_stream()) return nullptr;
      if (n > PIN_DOUBLES) return nullptr;
    }
    double* p = pinned_ + pin_off_;
    pin_off_ += (n + 7) & ~(size_t)7;
    return p;
  }
  bdg_status download(const double* d, std::vector<double>& h, size_t n) {
    double* p = stage(n);
    if (!p) return fail(plan_, BDG_ERR_INVALID, "staging arena too small for a download");
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(p, d, sizeof(double) * n, cudaMemcpyDeviceToHost, s_));
    bdg_status st = sync_stream();
    if (st) return st;
    h.assign(p, p + n);
    return BDG_OK;
  }
  bdg_status upload(double* d, const double* h, size_t n) {
    if (n == 0) return BDG_OK;
    double* p = stage(n);
    if (!p) return fail(plan_, BDG_ERR_INVALID, "staging arena too small for an upload");
    memcpy(p, h, sizeof(double) * n);
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(d, p, sizeof(double) * n, cudaMemcpyHostToDevice, s_));
    return BDG_OK;
  }
  bdg_status upload(double* d, const std::vector<double>& h) { return upload(d, h.data(), h.size()); }
  // Gram of real columns, leading na x nb block copied to the host
  bdg_status gram_host(const PairBlock<R>& A, int na, const PairBlock<R>& B, int nb, HostMat& out) {
    double* G = dmat_[MAT_G1];
    bdg_status st = gram(A, B, G);
    if (st) return st;
    std::vector<double> full;
    if ((st = download(G, full, (size_t)(2 * A.cols) * (2 * B.cols)))) return st;
    out = HostMat(na, nb);
    for (int i = 0; i < na; ++i)
      for (int j = 0; j < nb; ++j) out(i, j) = full[(size_t)i * (2 * B.cols) + j];
    return BDG_OK;
  }
  bdg_status cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) return fail(plan_, BDG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return BDG_OK;
  }
  // symmetric eigen-decomposition of the n x n device matrix A (ld lda),
  // ascending w to the host, V to dV (n x n, ld n)
  bdg_status eigh_dev(int n, const double* A, int lda, double* dw, double* dV, std::vector<double>& w,
                      double floor_rel = 0.0, bool from_identity = false) {
    if (n > SMALL_MAX) return fail(plan_, BDG_ERR_UNSUPPORTED, "projected problem larger than supported");
    int si_;
    cudaEvent_t se_ = sec_begin(from_identity ? "  eigh (identity start)" : (n > 100 ? "  eigh n>100" : "  eigh n<=100"), &si_);
    bdg_status st = cuda(eigh(n, A, lda, dw, dV, dws_, 3, s_, floor_rel, from_identity), "eigh");
    sec_end(se_);
    if (st) return st;
    if ((st = download(dw, w, n))) return st;
    if (dbg_eigh_) check_eigh(n, A, lda, dV, w);
    return BDG_OK;
  }
  void check_eigh(int n, const double* A, int lda, const double* dV, const std::vector<double>& w) {
    std::vector<double> a((size_t)n * lda), v((size_t)n * n);
    cudaMemcpy(a.data(), A, sizeof(double) * ((size_t)(n - 1) * lda + n), cudaMemcpyDeviceToHost);
    cudaMemcpy(v.data(), dV, sizeof(double) * n * n, cudaMemcpyDeviceToHost);
    double an = 0, res = 0, orth = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) an += a[(size_t)i * lda + j] * a[(size_t)i * lda + j];
    an = std::sqrt(an);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        double s = 0, o = 0;
        for (int l = 0; l < n; ++l) s += a[(size_t)i * lda + l] * v[(size_t)l * n + j];
        res = std::max(res, std::fabs(s - w[j] * v[(size_t)i * n + j]));
        for (int l = 0; l < n; ++l) o += v[(size_t)l * n + i] * v[(size_t)l * n + j];
        orth = std::max(orth, std::fabs(o - (i == j)));
      }
    if (res > 1e-13 * an || orth > 1e-12) {
      fprintf(stderr, "[bdg]   EIGH BAD n %d |A| %.3e res %.3e orth %.3e w0 %.3e wn %.3e\n", n, an, res / an, orth,
              w[0], w[n - 1]);
    }
  }

  // debug: max |A_f^T B_g - delta| over na x nb columns (delta if diag)
  double dbg_bi(const T* A, int pa, int na, const T* B, int pb, int nb, bool diag) {
    HostMat G;
    if (gram_host(fpart(A, 0, pa), na, gpart(B, 0, pb), nb, G)) return -1;
    double d = 0.0;
    for (int i = 0; i < na; ++i)
      for (int j = 0; j < nb; ++j) d = std::max(d, std::fabs(G(i, j) - ((diag && i == j) ? 1.0 : 0.0)));
    return d;
  }
  bool dbg_ = getenv("BDG_DEBUG") != nullptr;
  // debug: worst |H X - HX| / |H X| over the real columns of `pairs` pairs
  double dbg_img(const T* Xb, const T* HXb, int pairs) {
    if (!dbg_buf_ && alloc((void**)&dbg_buf_, sizeof(T) * vlen_ * cap_)) return -1;
    if (apply_fg(Xb, dbg_buf_, pairs)) return -1;
    double worst = 0.0;
    PairBlock<R> A{dbg_buf_, vlen_, vlen_, pairs}, B{HXb, vlen_, vlen_, pairs};
    HostMat a, c, d;
    gram_host(A, 2 * pairs, A, 2 * pairs, a);
    gram_host(B, 2 * pairs, A, 2 * pairs, c);
    gram_host(B, 2 * pairs, B, 2 * pairs, d);
    for (int i = 0; i < 2 * pairs; ++i)
      worst = std::max(worst, std::sqrt(std::fabs(a(i, i) - 2 * c(i, i) + d(i, i)) / std::max(a(i, i), 1e-300)));
    return worst;
  }

  // ---- deflation: X_f -= Z_f (Z_f^T X_f), X_g -= Z_g (Z_g^T X_g) ----------
  bdg_status deflate(T* bank, int pair0, int pairs) {
    if (pairs == 0) return BDG_OK;
    for (int side = 0; side < 2; ++side) {
      const int nz = side == 0 ? plan_->nzf : plan_->nzg;
      if (nz == 0) continue;
      const T* Z = side == 0 ? zf_ : zg_;
      PairBlock<R> Zb{Z, n3_, n3_, nz};
      PairBlock<R> Xb = side == 0 ? fpart(bank, pair0, pairs) : gpart(bank, pair0, pairs);
      double* G = dmat_[MAT_G1];
      bdg_status st = gram(Zb, Xb, G);
      if (st) return st;
      // X -= Z G  (G is 2nz x 2pairs)
      if ((st = update_dev(Zb, G, 2 * pairs, 1.0, side == 0 ? fptr(bank, pair0) : gptr(bank, pair0), pairs,
                           -1.0)))
        return st;
    }
    return BDG_OK;
  }

  // unit f- and g-parts for every real column of the block (zero columns stay zero)
  bdg_status normalize_parts(T* W, T* HW, int pairs) {
    std::vector<double> nf, ng;
    bdg_status st = colnorms_part(W, pairs, 0, nf);
    if (st) return st;
    if ((st = colnorms_part(W, pairs, 1, ng))) return st;
    std::vector<double> af(2 * pairs), ag(2 * pairs);
    for (int c = 0; c < 2 * pairs; ++c) {
      af[c] = nf[c] > 0 ? 1.0 / std::sqrt(nf[c]) : 0.0;
      ag[c] = ng[c] > 0 ? 1.0 / std::sqrt(ng[c]) : 0.0;
    }
    double* daf = dvec_ + 8 * big_;
    double* dag = daf + big_;
    if ((st = upload(daf, af)) || (st = upload(dag, ag))) return st;
    k_scale_parts<R><<<nblk((long long)pairs * vlen_), 256, 0, s_>>>(W, np_, pairs, daf, dag);
    if (HW) k_scale_parts<R><<<nblk((long long)pairs * vlen_), 256, 0, s_>>>(HW, np_, pairs, daf, dag);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    return BDG_OK;
  }

  // ---- S = F^T G bi-orthonormalization of the ncols columns of W ----------
  // S = X Sig Y^T via S^T S = Y Sig^2 Y^T; keep sigma >= rtol sigma_max;
  // dst_f = W_f S Y_r Sig^-3/2, dst_g = W_g Y_r Sig^-1/2 (and the images).
  bdg_status biortho_block(T* W, T* HW, int pairs, int ncols, T* dst, T* Hdst, double rtol, int* rank) {
    *rank = 0;
    if (ncols == 0) return BDG_OK;
    bdg_status st = normalize_parts(W, HW, pairs);
    if (st) return st;
    double* S = dmat_[MAT_G1];  // 2pairs x 2pairs, ld 2pairs
    const int ld = 2 * pairs;
    if ((st = gram(fpart(W, 0, pairs), gpart(W, 0, pairs), S))) return st;
    // S = X Sigma Y^T from the symmetric eigenproblem of [[0, S], [S^T, 0]]
    // (eigenvalues +-sigma, eigenvectors [x; y] / sqrt2): no squaring of the
    // condition number, so small singular values keep FP64 resolution.
    const int n2 = 2 * ncols;
    if (n2 > SMALL_MAX) return fail(plan_, BDG_ERR_UNSUPPORTED, "block too wide for the projected solver");
    double* J = dmat_[MAT_A];
    double* Vj = dmat_[MAT_B];
    k_jordan_wielandt<<<(n2 * n2 + 255) / 256, 256, 0, s_>>>(ncols, S, ld, J);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    std::vector<double> w;
    if ((st = eigh_dev(n2, J, n2, dvec_, Vj, w, 0.1 * rtol))) return st;   // sigma < rtol sigma_max is dropped
    const double smax = std::max(w[n2 - 1], 0.0);
    if (log_)
      fprintf(stderr, "[bdg]   biortho ncols %d sigma [%.3e, %.3e]", ncols, std::max(w[ncols], 0.0), smax);
    if (!(smax > 0)) return BDG_OK;
    int c0 = n2;
    while (c0 > ncols && w[c0 - 1] >= rtol * smax) --c0;
    const int r = n2 - c0;
    if (log_) fprintf(stderr, " rank %d\n", r);
    std::vector<double> sc(r);
    for (int k = 0; k < r; ++k) sc[k] = 1.0 / std::sqrt(w[c0 + k]);
    double* dsc = dvec_ + big_;
    if ((st = upload(dsc, sc))) return st;
    const int rp = (r + 1) / 2;
    double* Tf = dmat_[MAT_P];
    double* Tg = dmat_[MAT_Q];
    const int ldt = 2 * rp;
    if ((st = cuda(dzero_small(2 * pairs, ldt, Tf, ldt, s_), "zero"))) return st;
    if ((st = cuda(dzero_small(2 * pairs, ldt, Tg, ldt, s_), "zero"))) return st;
    k_jw_split<<<(ncols * r + 255) / 256 + 1, 256, 0, s_>>>(ncols, r, c0, Vj, dsc, Tf, Tg, ldt);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    if ((st = update_dev(fpart(W, 0, pairs), Tf, ldt, 0.0, dst, rp))) return st;
    if ((st = update_dev(gpart(W, 0, pairs), Tg, ldt, 0.0, dst + n3_, rp))) return st;
    if (HW) {
      if ((st = update_dev(fpart(HW, 0, pairs), Tf, ldt, 0.0, Hdst, rp))) return st;
      if ((st = update_dev(gpart(HW, 0, pairs), Tg, ldt, 0.0, Hdst + n3_, rp))) return st;
    }
    *rank = r;
    return BDG_OK;
  }

  // ---- projected pencil (device) --------------------------------------------
  // One small LREP solve: K_+ (n x n, ldp) = Q L Q^T keeping L > 1e-10 L_max,
  // C = L^1/2 Q^T K_- Q L^1/2 = Z W^2 Z^T, the mm <= mmax smallest w^2 above
  // the zero-mode cut max(1e-12, 1e-13 |C|) (zero modes of the projected
  // problem come out at the rounding level of C):
  //   Pc = Q L^-1/2 Z W^1/2, Qc = Q L^1/2 Z W^-1/2  (p^T q = 1, K_+ p = w q,
  //   K_- q = w p), written n x mm with leading dimension ldc (zero-filled
  //   to zrows x ldc first).
  bdg_status small_lrep(int n, const double* Kp, int ldp, const double* Km, int ldm, int mmax, int zrows,
                        bool scale, int nfix, double* Pc, double* Qc, int ldc_fixed, std::vector<double>& om,
                        int* ldc_out) {
    // K_+ = D^1/2 Kt D^1/2 with unit-diagonal Kt = Q diag(lam) Q^T: the
    // diagonal scaling takes out the column scales of the basis, so that
    // lam spans only the conditioning of H_+ on it.  L = D^1/2 Q_r lam^1/2.
    // (scale = false: D = I, for a K_+ that is already nearly diagonal.)
    double* Q = dmat_[MAT_A];
    double* dsq = nullptr;
    double* dinv = nullptr;
    const double* Kt = Kp;
    int ldt = ldp;
    if (scale) {
      double* Ks = dmat_[MAT_D];
      dsq = dvec_ + 11 * big_;
      dinv = dvec_ + 12 * big_;
      k_diag_scale<<<(n * n + 255) / 256, 256, 0, s_>>>(n, nfix, Kp, ldp, Ks, dsq, dinv);
      BDG_CUDA_TRY(plan_, cudaGetLastError());
      Kt = Ks;
      ldt = n;
    }
    // Factor K_+ = Lh Lh^T on its numerical range with a right inverse Minv
    // (Lh^T Minv = I): stage 1 by the rank-revealing pivoted Cholesky of the
    // unit-diagonal Kt (pivots <= 1e-10 of the largest are cut), stage 2
    // (scale == false, a Kt diagonal up to the rounding of stage 1) by its
    // eigen-decomposition refined from the identity,
    // Kt = Q diag(lam) Q^T, lam <= 1e-10 lam_max cut.
    double* Lh = dmat_[MAT_B];    // n x r
    double* Minv = dmat_[MAT_M];  // n x r
    bdg_status st = BDG_OK;
    int r = 0;
    if (scale && pchol_) {
      double* Lc = dmat_[MAT_A];
      double* Mc = dmat_[MAT_E];
      { int si_; cudaEvent_t se_ = sec_begin("  pivoted Cholesky", &si_);
        st = cuda(pchol(n, Kt, ldt, 1e-10, Lc, Mc, n, dint_, s_), "pchol");
        sec_end(se_); if (st) return st; }
      std::vector<double> rr;
      int rk = 0;
      BDG_CUDA_TRY(plan_, cudaMemcpyAsync(&rk, dint_, sizeof(int), cudaMemcpyDeviceToHost, s_));
      if ((st = sync_stream())) return st;
      r = rk;
      if (r <= 0) return fail(plan_, BDG_ERR_BREAKDOWN, "projected H_+ is not positive");
      if ((st = cuda(dscale_small(n, r, Lc, n, dsq, nullptr, Lh, r, s_), "scale")) ||
          (st = cuda(dscale_small(n, r, Mc, n, dinv, nullptr, Minv, r, s_), "scale")))
        return st;
    } else {
      std::vector<double> lam;
      // stage 2 re-solves matrices that are diagonal up to the rounding of
      // stage 1: the refinement starts from the identity
      st = eigh_dev(n, Kt, ldt, dvec_, Q, lam, 1e-11, !scale);   // lam <= 1e-10 lam_max is cut
      if (st) return st;
      const double lmax = lam[n - 1];
      if (!(lmax > 0)) return fail(plan_, BDG_ERR_BREAKDOWN, "projected H_+ is not positive");
      int i0 = 0;
      while (i0 < n && !(lam[i0] > 1e-10 * lmax)) ++i0;
      r = n - i0;
      std::vector<double> sl(r), isl(r);
      for (int a = 0; a < r; ++a) {
        sl[a] = std::sqrt(lam[i0 + a]);
        isl[a] = 1.0 / sl[a];
      }
      double* dsl = dvec_ + big_;
      double* disl = dsl + big_;
      if ((st = upload(dsl, sl)) || (st = upload(disl, isl))) return st;
      // Lh = D^1/2 Q_r diag(sqrt(lam)), Minv = D^-1/2 Q_r diag(1/sqrt(lam))
      if ((st = cuda(dscale_small(n, r, Q + i0, n, dsq, dsl, Lh, r, s_), "scale")) ||
          (st = cuda(dscale_small(n, r, Q + i0, n, dinv, disl, Minv, r, s_), "scale")))
        return st;
    }
    double* KL = dmat_[MAT_C];   // n x r
    double* C = dmat_[MAT_D];    // r x r
    if ((st = cuda(dgemm_small(false, false, n, r, n, 1.0, Km, ldm, Lh, r, 0.0, KL, r, s_), "gemm"))) return st;
    if ((st = cuda(dgemm_small(true, false, r, r, n, 1.0, Lh, r, KL, r, 0.0, C, r, s_), "gemm"))) return st;
    if ((st = cuda(dsym_small(r, C, r, s_), "sym"))) return st;
    double* Z = dmat_[MAT_E];
    std::vector<double> w2;
    if ((st = eigh_dev(r, C, r, dvec_, Z, w2, 0.0, !scale))) return st;
    const double cut = zero_tol2_;
    int j0 = 0;
    while (j0 < r && !(w2[j0] > cut)) ++j0;
    const int mm = std::min(mmax, r - j0);
    om.assign(mm, 0.0);
    std::vector<double> sw(mm), isw(mm);
    for (int j = 0; j < mm; ++j) {
      om[j] = std::sqrt(w2[j0 + j]);
      sw[j] = std::sqrt(om[j]);
      isw[j] = 1.0 / sw[j];
    }
    const int ldc = ldc_fixed > 0 ? ldc_fixed : 2 * ((mm + 1) / 2);
    *ldc_out = ldc;
    if ((st = cuda(dzero_small(zrows, ldc, Pc, ldc, s_), "zero")) ||
        (st = cuda(dzero_small(zrows, ldc, Qc, ldc, s_), "zero")))
      return st;
    if (mm == 0) return BDG_OK;
    double* dsw = dvec_ + 3 * big_;
    double* disw = dsw + big_;
    if ((st = upload(dsw, sw)) || (st = upload(disw, isw))) return st;
    double* ZS = dmat_[MAT_C];   // Z_sel diag(sqrt(w)) then diag(1/sqrt(w))
    // Pc = Minv Z_sel W^1/2, Qc = Lh Z_sel W^-1/2
    if ((st = cuda(dscale_small(r, mm, Z + j0, r, nullptr, dsw, ZS, mm, s_), "scale"))) return st;
    if ((st = cuda(dgemm_small(false, false, n, mm, r, 1.0, Minv, r, ZS, mm, 0.0, Pc, ldc, s_), "gemm"))) return st;
    if ((st = cuda(dscale_small(r, mm, Z + j0, r, nullptr, disw, ZS, mm, s_), "scale"))) return st;
    if ((st = cuda(dgemm_small(false, false, n, mm, r, 1.0, Lh, r, ZS, mm, 0.0, Qc, ldc, s_), "gemm"))) return st;
    return BDG_OK;
  }

  // Rayleigh-Ritz on the basis (U, HU) of nu real columns.  Stage 1 solves
  // the projected pencil on the whole basis and keeps the m smallest Ritz
  // pairs; stage 2 re-solves the pencil restricted to those m pairs, whose
  // spectrum spans only [w_1^2, w_m^2], so the small eigenvalues come out to
  // full FP64 relative accuracy (stage 1 alone is limited to eps |C| with
  // |C| ~ w_max^2).  Coefficients go to dmat_[MAT_P] / [MAT_Q] in pair layout
  // (2 pu rows, ldc = 2 mmp).
  bdg_status rayleigh_ritz(const T* U, const T* HU, int nu, int nfix, int mmax, std::vector<double>& om) {
    const int pu = (nu + 1) / 2, ldg = 2 * pu;
    bdg_status st = BDG_OK;
    if (dbg_) {
      // images: |H U - HU| per real column relative to |H U| over all nu columns
      if (!dbg_buf_ && alloc((void**)&dbg_buf_, sizeof(T) * vlen_ * cap_)) return BDG_ERR_NOMEM;
      if ((st = apply_fg(U, dbg_buf_, pu))) return st;
      std::vector<double> bad;
      for (int part = 0; part < 2; ++part) {
        HostMat a, c, d;
        PairBlock<R> Wp = part ? gpart(dbg_buf_, 0, pu) : fpart(dbg_buf_, 0, pu);
        PairBlock<R> Hp = part ? gpart(HU, 0, pu) : fpart(HU, 0, pu);
        if ((st = gram_host(Wp, nu, Wp, nu, a)) || (st = gram_host(Hp, nu, Wp, nu, c)) ||
            (st = gram_host(Hp, nu, Hp, nu, d)))
          return st;
        for (int i = 0; i < nu; ++i) {
          const double e = std::sqrt(std::fabs(a(i, i) - 2 * c(i, i) + d(i, i)) / std::max(a(i, i), 1e-300));
          if (e > 1e-6) bad.push_back(i + 1000 * part);
        }
      }
      fprintf(stderr, "[bdg]   dbg images bad columns:");
      for (double b : bad) fprintf(stderr, " %d", (int)b);
      fprintf(stderr, "\n");
    }
    double* Kp = dmat_[MAT_G1];
    double* Km = dmat_[MAT_G2];
    { int si_; cudaEvent_t se_ = sec_begin("  RR grams", &si_);
      // K_+ = U^T H_+ U and K_- = V^T H_- V are symmetric: the tiles on and
      // above the diagonal are formed, the rest mirrored
      st = gram(fpart(U, 0, pu), fpart(HU, 0, pu), Kp, true);
      if (!st) st = gram(gpart(U, 0, pu), gpart(HU, 0, pu), Km, true);
      sec_end(se_); if (st) return st; }
    if ((st = cuda(dsym_small(nu, Kp, ldg, s_), "sym")) || (st = cuda(dsym_small(nu, Km, ldg, s_), "sym")))
      return st;
    // stage 1
    double* P1 = dmat_[MAT_P1];
    double* Q1 = dmat_[MAT_Q1];
    std::vector<double> om1;
    int ld1 = 0;
    if ((st = small_lrep(nu, Kp, ldg, Km, ldg, mmax, nu, true, nfix, P1, Q1, 0, om1, &ld1))) return st;
    const int mm = (int)om1.size();
    if (log_) fprintf(stderr, "[bdg]   RR nu %d mm %d omega1 [%.6g .. %.6g]\n", nu, mm, mm ? om1[0] : 0.0,
                      mm ? om1[mm - 1] : 0.0);
    if (mm == 0) {
      om.clear();
      return BDG_OK;
    }
    // stage 2: K_+2 = P1^T K_+ P1, K_-2 = Q1^T K_- Q1 (mm x mm)
    double* T1 = dmat_[MAT_T];
    double* Kp2 = dmat_[MAT_K2P];
    double* Km2 = dmat_[MAT_K2M];
    if ((st = cuda(dgemm_small(false, false, nu, mm, nu, 1.0, Kp, ldg, P1, ld1, 0.0, T1, mm, s_), "gemm")))
      return st;
    if ((st = cuda(dgemm_small(true, false, mm, mm, nu, 1.0, P1, ld1, T1, mm, 0.0, Kp2, mm, s_), "gemm")))
      return st;
    if ((st = cuda(dgemm_small(false, false, nu, mm, nu, 1.0, Km, ldg, Q1, ld1, 0.0, T1, mm, s_), "gemm")))
      return st;
    if ((st = cuda(dgemm_small(true, false, mm, mm, nu, 1.0, Q1, ld1, T1, mm, 0.0, Km2, mm, s_), "gemm")))
      return st;
    if ((st = cuda(dsym_small(mm, Kp2, mm, s_), "sym")) || (st = cuda(dsym_small(mm, Km2, mm, s_), "sym")))
      return st;
    double* P2 = dmat_[MAT_P2];
    double* Q2 = dmat_[MAT_Q2];
    int ld2 = 0;
    if ((st = small_lrep(mm, Kp2, mm, Km2, mm, mm, mm, false, 0, P2, Q2, mm, om, &ld2))) return st;
    const int m2 = (int)om.size();
    const int mmp = (m2 + 1) / 2, ldc = 2 * mmp;
    double* Pc = dmat_[MAT_P];
    double* Qc = dmat_[MAT_Q];
    if ((st = cuda(dzero_small(2 * pu, ldc, Pc, ldc, s_), "zero")) ||
        (st = cuda(dzero_small(2 * pu, ldc, Qc, ldc, s_), "zero")))
      return st;
    if (m2 == 0) return BDG_OK;
    if ((st = cuda(dgemm_small(false, false, nu, m2, mm, 1.0, P1, ld1, P2, ld2, 0.0, Pc, ldc, s_), "gemm")))
      return st;
    if ((st = cuda(dgemm_small(false, false, nu, m2, mm, 1.0, Q1, ld1, Q2, ld2, 0.0, Qc, ldc, s_), "gemm")))
      return st;
    return BDG_OK;
  }

  // ---- one solve phase ---------------------------------------------------
  // The Ritz block enters in bank U_[cur_] columns [0, nx_) with images.
  // stop_floor > 0 (FP32 phase): return once the worst of the first k
  // residuals is below it, or after fp32_stall_ iterations (1 unless
  // BDG_FP32_STALL says otherwise) without a 30% gain.
  bdg_status iterate(int k, double tol, int maxit, double stop_floor, int* iters_out, bool* converged) {
    *converged = false;
    int nu = nx_;   // basis columns
    int nxb = 0;    // where the [D P] part starts (0: the basis is the Ritz block alone)
    double best = INFINITY;
    int stall = 0;
    bool refresh_next = false;
    int refreshed_at = -1;
    for (int it = 0; it < maxit; ++it) {
      plan_->stats.iterations++;
      if (sizeof(R) == 4) plan_->stats.iterations_fp32++;
      std::vector<double> om;
      int si_rr;
      cudaEvent_t se_rr = sec_begin("rayleigh-ritz", &si_rr);
      bdg_status st = rayleigh_ritz(U_[cur_], HU_[cur_], nu, nxb, m_, om);
      sec_end(se_rr);
      if (st) return st;
      const int mm = (int)om.size();
      if (mm == 0) return fail(plan_, BDG_ERR_BREAKDOWN, "no positive Ritz values");
      const int pu = (nu + 1) / 2, mmp = (mm + 1) / 2, ldc = 2 * mmp;
      const int nxt = 1 - cur_;
      const double* Pc = dmat_[MAT_P];
      const double* Qc = dmat_[MAT_Q];
      // previous update P: the [D P]-part of the basis times its coefficient
      // rows; the new Ritz block is then X-part + P, which spares the [D P]
      // columns a second pass
      bool haveP = nxb > 0 && nu > nxb;
      int si_ex;
      cudaEvent_t se_ex = sec_begin("extraction", &si_ex);
      if (haveP) {
        const int p0 = nxb / 2, pp = pu - p0;
        const double* Pd = Pc + (size_t)nxb * ldc;
        const double* Qd = Qc + (size_t)nxb * ldc;
        if ((st = update_dev(fpart(U_[cur_], p0, pp), Pd, ldc, 0.0, fptr(Pb_, 0), mmp))) return st;
        if ((st = update_dev(gpart(U_[cur_], p0, pp), Qd, ldc, 0.0, gptr(Pb_, 0), mmp))) return st;
        if (!exact_images_) {
          if ((st = update_dev(fpart(HU_[cur_], p0, pp), Pd, ldc, 0.0, fptr(HPb_, 0), mmp))) return st;
          if ((st = update_dev(gpart(HU_[cur_], p0, pp), Qd, ldc, 0.0, gptr(HPb_, 0), mmp))) return st;
        }
        const size_t bytes = sizeof(T) * (size_t)vlen_ * mmp;
        BDG_CUDA_TRY(plan_, cudaMemcpyAsync(U_[nxt], Pb_, bytes, cudaMemcpyDeviceToDevice, s_));
        if (!exact_images_) BDG_CUDA_TRY(plan_, cudaMemcpyAsync(HU_[nxt], HPb_, bytes, cudaMemcpyDeviceToDevice, s_));
        if ((st = update_dev(fpart(U_[cur_], 0, p0), Pc, ldc, 1.0, fptr(U_[nxt], 0), mmp))) return st;
        if ((st = update_dev(gpart(U_[cur_], 0, p0), Qc, ldc, 1.0, gptr(U_[nxt], 0), mmp))) return st;
        if (!exact_images_) {
          if ((st = update_dev(fpart(HU_[cur_], 0, p0), Pc, ldc, 1.0, fptr(HU_[nxt], 0), mmp))) return st;
          if ((st = update_dev(gpart(HU_[cur_], 0, p0), Qc, ldc, 1.0, gptr(HU_[nxt], 0), mmp))) return st;
        }
      } else {
        // new Ritz block into the other bank
        if ((st = update_dev(fpart(U_[cur_], 0, pu), Pc, ldc, 0.0, fptr(U_[nxt], 0), mmp))) return st;
        if ((st = update_dev(gpart(U_[cur_], 0, pu), Qc, ldc, 0.0, gptr(U_[nxt], 0), mmp))) return st;
        if (!exact_images_) {
          if ((st = update_dev(fpart(HU_[cur_], 0, pu), Pc, ldc, 0.0, fptr(HU_[nxt], 0), mmp))) return st;
          if ((st = update_dev(gpart(HU_[cur_], 0, pu), Qc, ldc, 0.0, gptr(HU_[nxt], 0), mmp))) return st;
        }
      }
      sec_end(se_ex);
      if (dbg_ && haveP && !exact_images_)
        fprintf(stderr, "[bdg]   dbg P images after extraction %.3e\n", dbg_img(Pb_, HPb_, mmp));
      cur_ = nxt;
      T* X = U_[cur_];
      T* HX = HU_[cur_];
      if (exact_images_) {
        // images of the new Ritz block by the product itself: every residual
        // and every projected matrix then holds to the rounding of one product
        { int si_; cudaEvent_t se_ = sec_begin("apply ritz block", &si_); st = apply_fg(X, HX, mmp); sec_end(se_); if (st) return st; }
        refreshed_at = it;
      }
      // The images HX are carried by linear combination; their rounding
      // drifts slowly away from H X.  Recompute them exactly every 20
      // iterations and before a convergence claim is accepted.  (A refresh
      // on every stall dropped the previous-update block P again and again
      // near the floor and could keep the iteration from recovering.)
      const bool refresh = !exact_images_ && (refresh_next || (it > 0 && it % 20 == 0));
      if (refresh) {
        if ((st = apply_fg(X, HX, mmp))) return st;
        haveP = false;  // P's images were drifted the same way
        refreshed_at = it;
      }
      refresh_next = false;
      if (dbg_) fprintf(stderr, "[bdg]   dbg ritz X_f^T X_g - I %.3e\n", dbg_bi(X, mmp, mm, X, mmp, mm, true));
      int si_res;
      cudaEvent_t se_res = sec_begin("residuals", &si_res);
      // residuals R_f = HF - G w, R_g = HG - F w
      BDG_CUDA_TRY(plan_, cudaMemcpyAsync(Rb_, HX, sizeof(T) * vlen_ * mmp, cudaMemcpyDeviceToDevice, s_));
      HostMat Dw(2 * mmp, 2 * mmp);
      for (int j = 0; j < mm; ++j) Dw(j, j) = -om[j];
      if ((st = update(gpart(X, 0, mmp), Dw, 1.0, fptr(Rb_, 0), mmp))) return st;
      if ((st = update(fpart(X, 0, mmp), Dw, 1.0, gptr(Rb_, 0), mmp))) return st;
      // components of G along Z_f (and F along Z_g) in closed form:
      // G += Z_f (Z_f^T R_f) / w, R_f -= Z_f (Z_f^T R_f)
      for (int side = 0; side < 2; ++side) {
        const int nz = side == 0 ? plan_->nzf : plan_->nzg;
        if (nz == 0) continue;
        const T* Z = side == 0 ? zf_ : zg_;
        PairBlock<R> Zb{Z, n3_, n3_, nz};
        HostMat c;
        if ((st = gram_host(Zb, 2 * nz, side == 0 ? fpart(Rb_, 0, mmp) : gpart(Rb_, 0, mmp), 2 * mmp, c)))
          return st;
        HostMat cw = c, cn = c;
        for (int i = 0; i < 2 * nz; ++i)
          for (int j = 0; j < 2 * mmp; ++j) {
            cw(i, j) = j < mm ? c(i, j) / om[j] : 0.0;
            cn(i, j) = -c(i, j);
          }
        if ((st = update(Zb, cw, 1.0, side == 0 ? gptr(X, 0) : fptr(X, 0), mmp))) return st;
        if ((st = update(Zb, cn, 1.0, side == 0 ? fptr(Rb_, 0) : gptr(Rb_, 0), mmp))) return st;
      }
      if (dbg_) fprintf(stderr, "[bdg]   dbg after null fix X_f^T X_g - I %.3e\n", dbg_bi(X, mmp, mm, X, mmp, mm, true));
      sec_end(se_res);
      // residual norms
      std::vector<double> nr, nx;
      if ((st = colnorms(Rb_, mmp, nr))) return st;
      if ((st = colnorms(X, mmp, nx))) return st;
      resid_.assign(mm, 0.0);
      omega_ = om;
      int nconv = 0;
      double worst = 0.0;
      for (int j = 0; j < mm; ++j) {
        resid_[j] = std::sqrt(nr[j]) / (om[j] * std::sqrt(nx[j]));
        if (!std::isfinite(resid_[j])) return fail(plan_, BDG_ERR_NAN, "NaN in the iteration");
      }
      for (int j = 0; j < std::min(k, mm); ++j) {
        worst = std::max(worst, resid_[j]);
        if (resid_[j] <= tol) nconv++;
      }
      mm_ = mm;
      nx_ = mm;
      *iters_out = it + 1;
      if (mm >= k && nconv == k && refreshed_at != it) {
        // verify with exact images before accepting convergence
        refresh_next = true;
        nconv = 0;
      }
      if (log_) {
        fprintf(stderr, "[bdg] it %d prec %d nu %d nxb %d mm %d worst %.3e omega[0..2] %.6g %.6g %.6g\n", it,
                (int)sizeof(R) * 8, nu, nxb, mm, worst, om[0], mm > 1 ? om[1] : 0.0, mm > 2 ? om[2] : 0.0);
      }
      if (mm >= k && nconv == k) {
        *converged = true;
        return BDG_OK;
      }
      if (stop_floor > 0) {
        if (mm >= k && worst < stop_floor) return BDG_OK;
        if (worst < 0.7 * best) {
          best = worst;
          stall = 0;
        } else if (++stall >= fp32_stall_) {
          return BDG_OK;
        }
      }
      if (it + 1 == maxit) break;
      // active columns: D = T_sigma R_act, with P_act beside it in W
      std::vector<int> act;
      for (int j = 0; j < mm; ++j)
        if (resid_[j] > tol) act.push_back(j);
      const int na = (int)act.size();
      const int nap = (na + 1) / 2;
      if (log_) fprintf(stderr, "[bdg]   active %d of %d, P %d\n", na, mm, haveP ? 1 : 0);
      if (na == 0) {
        // Every Ritz pair meets tol, so there is no search direction.  This
        // happens when the block is wide enough that its extra pairs converge
        // with the wanted ones.  The pending check re-runs the Ritz step on
        // the block alone, with exact images.
        if (!refresh_next)
          return fail(plan_, BDG_ERR_BREAKDOWN, "all Ritz pairs converged but fewer than k were found");
        nxb = 0;
        nu = mm;
        continue;
      }
      if (dbg_ && haveP && !exact_images_)
        fprintf(stderr, "[bdg]   dbg P images before gather %.3e\n", dbg_img(Pb_, HPb_, mmp));
      if (dbg_ && haveP) {
        // gather check on a copy: G = P Sel must equal the selected columns
        HostMat Sel2(2 * mmp, 2 * nap);
        for (int jj = 0; jj < na; ++jj) Sel2(act[jj], jj) = 1.0;
        if (!dbg_buf_) alloc((void**)&dbg_buf_, sizeof(T) * vlen_ * cap_);
        PairBlock<R> Pa{Pb_, vlen_, vlen_, mmp};
        update(Pa, Sel2, 0.0, dbg_buf_, nap);
        std::vector<double> ng, np_;
        colnorms(dbg_buf_, nap, ng);
        colnorms(Pb_, mmp, np_);
        fprintf(stderr, "[bdg]   dbg gather |P Sel|_j vs |P|_act[j]:");
        for (int jj = 0; jj < na; ++jj) fprintf(stderr, " (%.3e %.3e)", std::sqrt(ng[jj]), std::sqrt(np_[act[jj]]));
        fprintf(stderr, "\n");
      }
      HostMat Sel(2 * mmp, 2 * nap);
      for (int jj = 0; jj < na; ++jj) Sel(act[jj], jj) = 1.0;
      if ((st = update_full(Rb_, mmp, Sel, Wb_, nap))) return st;
      // The previous-update block P (gathered into the second half of W,
      // Gram-Schmidt against X, bi-orthonormalized behind X) does not depend
      // on the new directions: with exact images it runs on the second lane
      // while the inner PCG of the directions runs on this one.
      const bool fork = overlap_ && lane2_.s && exact_images_ && haveP;
      bool p_images = false;   // images of P' formed on the second lane
      if (fork) BDG_CUDA_TRY(plan_, cudaEventRecord(ev_fork_, s_));
      { int si_; cudaEvent_t se_ = sec_begin("inner directions", &si_); st = directions(Wb_, nap); sec_end(se_); if (st) return st; }
      int nw = 2 * nap;
      int rp = 0;
      T* const HWx = exact_images_ ? nullptr : HWb_;   // images carried only without exact products
      auto p_chain = [&]() -> bdg_status {
        bdg_status sp = BDG_OK;
        if (haveP) {
          // previous-update columns that carry information: |P_j| >= 1e-12 |X_j|
          // (near convergence P is a cancellation-level difference whose image
          // is consistent with it only to eps |X| / |P|; such columns are left out)
          std::vector<double> npn;
          if ((sp = colnorms(Pb_, mmp, npn))) return sp;
          std::vector<int> actp;
          for (int j : act)
            if (npn[j] >= 1e-24 * nx[j]) actp.push_back(j);
          const int npa = (int)actp.size();
          if (npa > 0) {
            HostMat SelP(2 * mmp, 2 * nap);
            for (int jj = 0; jj < npa; ++jj) SelP(actp[jj], jj) = 1.0;
            if ((sp = update_full(Pb_, mmp, SelP, Wb_ + (long long)nap * vlen_, nap))) return sp;
            if (!exact_images_ && (sp = update_full(HPb_, mmp, SelP, HWb_ + (long long)nap * vlen_, nap)))
              return sp;
            nw = 4 * nap;
          }
        }
        // Bi-orthogonal Gram-Schmidt in two stages: P against X, then
        // bi-orthonormalize P; D against [X, P'], then bi-orthonormalize D.
        // Each block holds at most 2 nap columns, so its Jordan-Wielandt
        // problem stays within the projected solver's size.
        if (nw > 2 * nap) {
          T* WP = Wb_ + (long long)nap * vlen_;
          T* HWP = HWx ? HWx + (long long)nap * vlen_ : nullptr;
          { int si_; cudaEvent_t se_ = sec_begin("cgs2 P", &si_); sp = cgs2(X, HX, mmp, WP, HWP, nap); sec_end(se_); if (sp) return sp; }
          { int si_; cudaEvent_t se_ = sec_begin("biortho P", &si_);
            sp = biortho_block(WP, HWP, nap, 2 * nap, fptr(X, mmp), HWP ? fptr(HX, mmp) : nullptr, rtol_, &rp);
            sec_end(se_); if (sp) return sp; }
        }
        return BDG_OK;
      };
      if (fork) {
        BDG_CUDA_TRY(plan_, cudaStreamWaitEvent(lane2_.s, ev_fork_, 0));
        {
          swap_lane(lane2_);
          LaneGuard back{this};
          st = p_chain();
          if (!st && cudaEventRecord(ev_join_, s_) != cudaSuccess) st = fail(plan_, BDG_ERR_CUDA, "join event");
          // the images of P' need nothing from the directions either: their
          // product also runs on this lane, joined before the next
          // Rayleigh-Ritz step
          if (!st && rp > 0) {
            int si_;
            cudaEvent_t se_ = sec_begin("apply new columns P", &si_);
            st = apply_fg(fptr(X, mmp), fptr(HX, mmp), (rp + 1) / 2);
            sec_end(se_);
            if (!st && cudaEventRecord(ev_img_, s_) != cudaSuccess) st = fail(plan_, BDG_ERR_CUDA, "image event");
            p_images = !st;
          }
        }
        if (st) return st;
        BDG_CUDA_TRY(plan_, cudaStreamWaitEvent(s_, ev_join_, 0));
      }
      { int si_; cudaEvent_t se_ = sec_begin("deflate D", &si_); st = deflate(Wb_, 0, nap); sec_end(se_); if (st) return st; }
      // unit f- and g-parts before the product: the two real columns sharing
      // a complex vector then have equal norms, so the rounding crosstalk
      // between them in the FFTs stays at eps relative to each column
      { int si_; cudaEvent_t se_ = sec_begin("normalize D", &si_); st = normalize_parts(Wb_, nullptr, nap); sec_end(se_); if (st) return st; }
      if (!exact_images_ && (st = apply_fg(Wb_, HWb_, nap))) return st;
      if (!fork && (st = p_chain())) return st;
      const int rpp = (rp + 1) / 2;
      { int si_; cudaEvent_t se_ = sec_begin("cgs2 D", &si_); st = cgs2(X, HX, mmp + rpp, Wb_, HWx, nap); sec_end(se_); if (st) return st; }
      int rd = 0;
      { int si_; cudaEvent_t se_ = sec_begin("biortho D", &si_);
        st = biortho_block(Wb_, HWx, nap, 2 * nap, fptr(X, mmp + rpp), HWx ? fptr(HX, mmp + rpp) : nullptr, rtol_, &rd);
        sec_end(se_); if (st) return st; }
      if (log_) fprintf(stderr, "[bdg]   block ranks P %d D %d\n", rp, rd);
      if (rp + rd == 0) return fail(plan_, BDG_ERR_BREAKDOWN, "search directions lost rank");
      // images of the new basis columns [P', D'] by one product
      if (exact_images_) {
        int si_;
        cudaEvent_t se_ = sec_begin("apply new columns", &si_);
        if (p_images) {
          st = apply_fg(fptr(X, mmp + rpp), fptr(HX, mmp + rpp), (rd + 1) / 2);
          if (!st && cudaStreamWaitEvent(s_, ev_img_, 0) != cudaSuccess) st = fail(plan_, BDG_ERR_CUDA, "image join");
        } else {
          st = apply_fg(fptr(X, mmp), fptr(HX, mmp), rpp + (rd + 1) / 2);
        }
        sec_end(se_);
        if (st) return st;
      }
      nxb = 2 * mmp;
      nu = 2 * (mmp + rpp) + rd;
    }
    return BDG_OK;
  }

  // Twice: W_f -= B_f (B_g^T W_f), W_g -= B_g (B_f^T W_g), images alike, for
  // the bi-orthonormal basis B = the first bp pairs of (Bk, HBk).
  bdg_status cgs2(const T* Bk, const T* HBk, int bp, T* W, T* HW, int wp) {
    bdg_status st = BDG_OK;
    const int nw = 2 * wp;
    for (int pass = 0; pass < cgs_passes_; ++pass) {
      double* c1 = dmat_[MAT_G1];
      double* c2 = dmat_[MAT_G2];
      const bool first_of_two = pass == 0 && cgs_passes_ >= 2;
      if ((st = gram(gpart(Bk, 0, bp), fpart(W, 0, wp), c1, false, sizeof(R) == 4 || first_of_two))) return st;
      if ((st = gram(fpart(Bk, 0, bp), gpart(W, 0, wp), c2, false, sizeof(R) == 4 || first_of_two))) return st;
      // (the updates stay in double-float in both passes: rounding errors of
      // an FP32 update lie outside span(B), where the second pass cannot
      // remove them, and near convergence W is mostly along B, so they
      // swamp its remaining part -- tried, and the solves stalled)
      if ((st = update_dev(fpart(Bk, 0, bp), c1, nw, 1.0, fptr(W, 0), wp, -1.0))) return st;
      if (HW && (st = update_dev(fpart(HBk, 0, bp), c1, nw, 1.0, fptr(HW, 0), wp, -1.0))) return st;
      if ((st = update_dev(gpart(Bk, 0, bp), c2, nw, 1.0, gptr(W, 0), wp, -1.0))) return st;
      if (HW && (st = update_dev(gpart(HBk, 0, bp), c2, nw, 1.0, gptr(HW, 0), wp, -1.0))) return st;
    }
    return BDG_OK;
  }

  // Y (Q pairs) = bank A (P pairs, whole 6-component vectors) C
  bdg_status update_full(const T* bank, int P, const HostMat& C, T* Y, int Q) {
    PairBlock<R> A{bank, vlen_, vlen_, P};
    return update(A, C, 0.0, Y, Q);
  }

  // ---- start block --------------------------------------------------------
  bdg_status start_random(const void* X0, unsigned long long seed) {
    T* X = U_[cur_];
    const long long total = (long long)mp_ * vlen_;
    if (X0) k_pack_real<R><<<nblk(total), 256, 0, s_>>>((const double2*)X0, m_, vlen_, X);
    else k_random_block<R><<<nblk(total), 256, 0, s_>>>(X, total, seed);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    return begin_block(m_);
  }

  // deflate + bi-orthonormalize the ncols columns in U_[cur_], apply H
  bdg_status begin_block(int ncols) {
    T* X = U_[cur_];
    const int pairs = (ncols + 1) / 2;
    bdg_status st = deflate(X, 0, pairs);
    if (st) return st;
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(Wb_, X, sizeof(T) * vlen_ * pairs, cudaMemcpyDeviceToDevice, s_));
    int r = 0;
    if ((st = biortho_block(Wb_, nullptr, pairs, ncols, X, nullptr, rtol_, &r))) return st;
    if (r == 0) return fail(plan_, BDG_ERR_BREAKDOWN, "start block has no bi-orthogonal directions");
    if ((st = apply_fg(X, HU_[cur_], (r + 1) / 2))) return st;
    nx_ = r;
    return BDG_OK;
  }

  // per real column: squared norm of the f-part (part 0) or the g-part (part 1)
  // squared column norms over n rows from offset off of each 6-field column,
  // reduced in a fixed order (the solve is reproducible run to run)
  bdg_status colnorm_dev(const T* bank, long long n, int pairs, double* d) {
    if (pairs > cap_) return fail(plan_, BDG_ERR_INVALID, "column-norm block wider than its workspace");
    k_colnorm2<R><<<dim3(CN_BLOCKS, pairs), 256, 0, s_>>>(bank, vlen_, n, pairs, cnpart_);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    k_colnorm_reduce<<<(2 * pairs + 127) / 128, 128, 0, s_>>>(cnpart_, CN_BLOCKS, pairs, d);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    return BDG_OK;
  }

  bdg_status colnorms_part(const T* bank, int pairs, int part, std::vector<double>& out) {
    double* d = dvec_ + 10 * big_;
    bdg_status st = colnorm_dev(bank + (part ? n3_ : 0), n3_, pairs, d);
    if (st) return st;
    return download(d, out, 2 * pairs);
  }

  bdg_status colnorms(const T* bank, int pairs, std::vector<double>& out) {
    double* d = dvec_ + 6 * big_;
    bdg_status st = colnorm_dev(bank, vlen_, pairs, d);
    if (st) return st;
    return download(d, out, 2 * pairs);
  }

  bdg_status alloc(void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return BDG_ERR_NOMEM;
    }
    owned_.push_back(*p);
    // diagnostics (BDG_POISON): fill new buffers with NaN bytes, so that a
    // read before the first write shows up in the results
    if (poison_ && cudaMemset(*p, 0xFF, bytes) != cudaSuccess) return BDG_ERR_NOMEM;
    return BDG_OK;
  }
  bool poison_ = getenv("BDG_POISON") != nullptr;
  void release() {
    sec_report();
    if (pinned_) {
      cudaStreamSynchronize(s_);
      cudaFreeHost(pinned_);
      pinned_ = nullptr;
    }
    if (lane2_.s) {
      cudaStreamSynchronize(lane2_.s);
      cudaStreamDestroy(lane2_.s);
      lane2_.s = nullptr;
    }
    if (lane2_.pinned) {
      cudaFreeHost(lane2_.pinned);
      lane2_.pinned = nullptr;
    }
    if (ev_fork_) cudaEventDestroy(ev_fork_);
    if (ev_join_) cudaEventDestroy(ev_join_);
    if (ev_img_) cudaEventDestroy(ev_img_);
    ev_fork_ = ev_join_ = ev_img_ = nullptr;
    for (void* p : owned_) cudaFree(p);
    owned_.clear();
  }

  // members
  bdg_plan_t plan_;
  cudaStream_t s_;
  int m_, mp_, cap_;
  long long np_, n3_, vlen_;
  T* U_[2] = {nullptr, nullptr};
  T* HU_[2] = {nullptr, nullptr};
  T *Rb_ = nullptr, *Wb_ = nullptr, *HWb_ = nullptr, *Pb_ = nullptr, *HPb_ = nullptr;
  const T* zf_ = nullptr;
  const T* zg_ = nullptr;
  void* gws_ = nullptr;
  size_t gws_bytes_ = 0;
  double* dsm_ = nullptr;
  enum { MAT_G1, MAT_G2, MAT_A, MAT_B, MAT_C, MAT_D, MAT_E, MAT_P, MAT_Q, MAT_HOST, MAT_P1, MAT_Q1,
         MAT_P2, MAT_Q2, MAT_T, MAT_K2P, MAT_K2M, MAT_M, NMAT };
  double* dmat_[NMAT] = {};
  double* dvec_ = nullptr;
  double* dws_ = nullptr;
  double* cnpart_ = nullptr;
  int* dint_ = nullptr;
  // stage 1 of the Rayleigh-Ritz step factors K_+ by pivoted Cholesky
  // (otherwise by its eigen-decomposition)
  bool pchol_ = getenv("BDG_RR_EIGH") == nullptr;
  static constexpr size_t PIN_DOUBLES = 1 << 20;   // 8 MB of pinned staging
  double* pinned_ = nullptr;
  size_t pin_off_ = 0;
  // A second lane -- a stream of its own with its own Gram workspace, small
  // matrices, column-norm partials and pinned staging -- runs the
  // previous-update block's Gram-Schmidt while the inner PCG of the new
  // directions runs on the solver's stream (BDG_OVERLAP=0 keeps one lane).
  // The two chains touch disjoint buffers, so the results do not change.
  struct Lane {
    cudaStream_t s = nullptr;
    void* gws = nullptr;
    size_t gws_bytes = 0;
    double* dsm = nullptr;
    double* dmat[NMAT] = {};
    double* dvec = nullptr;
    double* dws = nullptr;
    double* cnpart = nullptr;
    int* dint = nullptr;
    double* pinned = nullptr;
    size_t pin_off = 0;
  };
  Lane lane2_;
  bool overlap_ = !getenv("BDG_OVERLAP") || atoi(getenv("BDG_OVERLAP")) != 0;
  cudaEvent_t ev_fork_ = nullptr, ev_join_ = nullptr, ev_img_ = nullptr;
  void swap_lane(Lane& L) {
    std::swap(s_, L.s);
    std::swap(gws_, L.gws);
    std::swap(gws_bytes_, L.gws_bytes);
    std::swap(dsm_, L.dsm);
    for (int i = 0; i < NMAT; ++i) std::swap(dmat_[i], L.dmat[i]);
    std::swap(dvec_, L.dvec);
    std::swap(dws_, L.dws);
    std::swap(cnpart_, L.cnpart);
    std::swap(dint_, L.dint);
    std::swap(pinned_, L.pinned);
    std::swap(pin_off_, L.pin_off);
  }
  struct LaneGuard {
    Solver* S;
    ~LaneGuard() { S->swap_lane(S->lane2_); }
  };
  int big_ = 0;
  bool dbg_eigh_ = getenv("BDG_CHECK_EIGH") != nullptr;
  T* dbg_buf_ = nullptr;
  std::vector<void*> owned_;
  int cur_ = 0, nx_ = 0, mm_ = 0;
  double sigma_ = 1.0;
  // inner PCG steps per search direction (0: the kinetic preconditioner
  // alone); set per precision by bdg_solve
  int inner_steps_ = 10;
  bool inner_fp32_ = sizeof(R) == 4;
  InnerPCG<float> in32_;
  InnerPCG<double> in64_;
  double rtol_ = 1e-10;
  double zero_tol2_ = 1e-12;
  int cgs_passes_ = getenv("BDG_CGS_PASSES") ? atoi(getenv("BDG_CGS_PASSES")) : 2;
  // images H X of the Ritz block and of new basis columns by the product
  // itself (otherwise carried by linear combination, refreshed every 20
  // iterations; carried images drift by eps |coefficients| and stall strong
  // search directions near 1e-7)
  bool exact_images_ = getenv("BDG_CARRY_IMAGES") == nullptr;
  // the FP32 phase hands over after this many iterations without a 30 % gain
  int fp32_stall_ = getenv("BDG_FP32_STALL") ? atoi(getenv("BDG_FP32_STALL")) : 1;
  bool log_ = getenv("BDG_LOG") != nullptr;
  std::vector<double> omega_, resid_;

  // diagnostics (BDG_PROFILE): device time per solver section, from CUDA
  // events on the solver's stream, printed when the solver is released
  bool prof_ = getenv("BDG_PROFILE") != nullptr;
  struct Section { std::string name; std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev; };
  std::vector<Section> sections_;
  cudaEvent_t sec_begin(const char* name, int* idx) {
    if (!prof_) return nullptr;
    int i = 0;
    while (i < (int)sections_.size() && sections_[i].name != name) ++i;
    if (i == (int)sections_.size()) sections_.push_back(Section{name, {}});
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s_);
    sections_[i].ev.push_back({a, b});
    *idx = i;
    return b;
  }
  void sec_end(cudaEvent_t b) {
    if (b) cudaEventRecord(b, s_);
  }
  void sec_report() {
    if (!prof_ || sections_.empty()) return;
    cudaStreamSynchronize(s_);
    for (auto& sc : sections_) {
      double ms = 0.0;
      for (auto& pr : sc.ev) {
        float t = 0.f;
        cudaEventElapsedTime(&t, pr.first, pr.second);
        ms += t;
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
      }
      fprintf(stderr, "[bdg] prof %-3d-bit %-22s %5zu x %9.3f ms\n", (int)sizeof(R) * 8, sc.name.c_str(),
              sc.ev.size(), ms);
    }
    sections_.clear();
  }
};

// ---------------------------------------------------------------------------
// FP64 output: rescale to h^d <f, g> = 1/4, write UV, recompute residuals
// ---------------------------------------------------------------------------
template <typename R>
static bdg_status finish(Solver<R>& S, int k, double* omega, void* UV, double* resid, cudaStream_t s) {
  bdg_plan_t plan = S.plan_;
  const int kk = std::min(k, S.mm_);
  const int kp = (kk + 1) / 2;
  const Grid& g = plan->grid;
  double hd = 1.0;
  for (int a = 0; a < g.dim; ++a) hd *= g.len[a] / g.n[a];
  // f_i^T g_i (diagonal of the Gram)
  HostMat fg;
  bdg_status st = S.gram_host(S.fpart(S.U_[S.cur_], 0, kp), 2 * kp, S.gpart(S.U_[S.cur_], 0, kp), 2 * kp, fg);
  if (st) return st;
  std::vector<double> scale(2 * kp, 0.0);
  for (int i = 0; i < kk; ++i) {
    const double d = hd * fg(i, i);
    scale[i] = std::sqrt(0.25 / std::fabs(d));
  }
  for (int i = 0; i < kk; ++i) omega[i] = S.omega_[i];
  if (resid)
    for (int i = 0; i < kk; ++i) resid[i] = S.resid_[i];
  if (UV) {
    double* dscale = S.dvec_ + 7 * S.big_;
    BDG_CUDA_TRY(plan, cudaMemcpyAsync(dscale, scale.data(), sizeof(double) * 2 * kp, cudaMemcpyHostToDevice, s));
    k_unpack_uv<R><<<nblk((long long)kk * 3 * g.npts), 256, 0, s>>>(S.U_[S.cur_], g.npts, kk, dscale,
                                                                     (double2*)UV);
    BDG_CUDA_TRY(plan, cudaGetLastError());
    BDG_CUDA_TRY(plan, cudaStreamSynchronize(s));
  }
  return BDG_OK;
}

// FP32 Ritz block -> FP64 solver's first bank
static bdg_status transfer(Solver<float>& a, Solver<double>& b, cudaStream_t s) {
  const int pairs = (a.mm_ + 1) / 2;
  BDG_CUDA_TRY(a.plan_, (convert_pairs<float, double>(a.U_[a.cur_], a.vlen_, b.U_[b.cur_], b.vlen_, a.vlen_,
                                                      pairs, s)));
  return b.begin_block(a.mm_);
}

}  // namespace bdg

using namespace bdg;

extern "C" {

bdg_status bdg_solve(bdg_plan_t plan, int k, int m, const void* X0, double* omega, void* UV, double* resid,
                     int* nconv, void* stream) {
  if (!plan) return fail(nullptr, BDG_ERR_INVALID, "plan is NULL");
  if (!omega || !nconv) return fail(plan, BDG_ERR_INVALID, "omega and nconv must be host pointers");
  // the basis [X, P, D] holds at most 2 (mp + mp) + 2 mp = 6 mp real columns
  // (mp = ceil(m / 2) pairs per block), and its projected problem must fit
  // the on-chip eigensolver
  if (k < 1 || m < k || 6 * ((m + 1) / 2) > SMALL_MAX)
    return fail(plan, k < 1 || m < k ? BDG_ERR_INVALID : BDG_ERR_UNSUPPORTED,
                "need 1 <= k <= m <= " + std::to_string(2 * (SMALL_MAX / 6)) +
                    " (three blocks of m rounded up to even within " + std::to_string(SMALL_MAX) +
                    " projected columns)");
  if (bdg_status sd = check_device(plan)) return sd;
  cudaStream_t s = (cudaStream_t)stream;
  plan->last_stream = stream;
  memset(&plan->stats, 0, sizeof(plan->stats));
  *nconv = 0;
  const auto t0 = std::chrono::steady_clock::now();
  const double tol = plan->prm.tol > 0 ? plan->prm.tol : 1e-10;
  const int maxit = plan->prm.maxit > 0 ? plan->prm.maxit : 500;
  const double sigma = std::max(1.0, (plan->mu[0] + plan->mu[1] + plan->mu[2]) / 3.0);
  bdg_status st = BDG_OK;
  bool conv = false;
  int it1 = 0, it2 = 0;
  Solver<double> S64(plan, s, m);
  S64.sigma_ = sigma;
  // rank cut of the bi-orthonormalization: a kept direction with singular
  // value sigma scales the projected matrices by 1 / sigma, and FP64 rounding
  // with it; 1e-5 stalled strong search directions between 1e-7 and 1e-6,
  // 1e-4 ... 1e-2 converged alike (reading P16)
  S64.rtol_ = getenv("BDG_RTOL64") ? atof(getenv("BDG_RTOL64")) : 1e-3;
  S64.inner_fp32_ = plan->prm.prec == BDG_MIXED;   // plain FP64 keeps every kernel in FP64
  // inner steps: each precision at its fastest measured setting on the 2-D
  // 256^2 workload (FP64 inner products cost about twenty FP32 ones)
  const char* env_inner = getenv("BDG_INNER_STEPS");
  S64.inner_steps_ = env_inner ? atoi(env_inner) : (S64.inner_fp32_ ? 12 : 8);
  const bool log_phases = getenv("BDG_LOG") != nullptr;
  auto mark = [&](const char* what) {
    if (log_phases)
      fprintf(stderr, "[bdg] %8.3f ms  %s\n",
              1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(), what);
  };
  if (plan->prm.prec == BDG_MIXED) {
    Solver<float> S32(plan, s, m);
    S32.sigma_ = sigma;
    S32.rtol_ = 1e-4;
    S32.inner_steps_ = env_inner ? atoi(env_inner) : 12;
    if ((st = S32.init_buffers())) return st;
    mark("FP32 buffers");
    if ((st = S32.start_random(X0, plan->prm.seed))) return st;
    mark("FP32 start block");
    const double floor32 = getenv("BDG_FP32_FLOOR") ? atof(getenv("BDG_FP32_FLOOR")) : 3e-4;
    if ((st = S32.iterate(k, tol, maxit, floor32, &it1, &conv))) return st;
    mark("FP32 phase");
    if ((st = S64.init_buffers())) return st;
    mark("FP64 buffers");
    if ((st = transfer(S32, S64, s))) return st;
    mark("transfer");
  } else {
    if ((st = S64.init_buffers())) return st;
    mark("FP64 buffers");
    if ((st = S64.start_random(X0, plan->prm.seed))) return st;
    mark("FP64 start block");
  }
  mark("FP32 solver released");
  st = S64.iterate(k, tol, std::max(1, maxit - it1), 0.0, &it2, &conv);
  if (st) return st;
  mark("FP64 phase");
  std::vector<double> res(k, INFINITY);
  if ((st = finish<double>(S64, k, omega, UV, res.data(), s))) return st;
  mark("finish");
  int nc = 0;
  while (nc < k && nc < S64.mm_ && res[nc] <= tol) nc++;
  *nconv = nc;
  if (resid)
    for (int i = 0; i < k; ++i) resid[i] = res[i];
  plan->stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (nc < k) return fail(plan, BDG_ERR_NOT_CONVERGED, "not converged within maxit");
  return BDG_OK;
}

}  // extern "C"

// Independent problems back to back on one stream (the batched workload of
// many parameter sets and grids): each plan is solved as by bdg_solve; the
// first failing status is returned after every plan has been attempted, and
// nconv[i] is filled for every plan.
extern "C" bdg_status bdg_solve_batched(bdg_plan_t* plans, int count, const int* k, const int* m,
                                        double** omega, void** UV, double** resid, int* nconv, void* stream) {
  if (count < 0 || (count > 0 && (!plans || !k || !m || !omega || !nconv)))
    return fail(nullptr, BDG_ERR_INVALID, "plans, k, m, omega and nconv must hold count entries");
  for (int i = 0; i < count; ++i)
    if (!plans[i] || !omega[i]) return fail(nullptr, BDG_ERR_INVALID, "plan or omega entry is NULL");
  if (count == 0) return BDG_OK;
  {
    std::vector<bdg_plan_t> seen(plans, plans + count);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
      return fail(nullptr, BDG_ERR_INVALID, "a plan appears twice (its solves would share its scratch)");
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, BDG_ERR_CUDA, "cudaGetDevice failed");
  for (int i = 0; i < count; ++i)
    if (bdg_status sd = check_device(plans[i])) {
      set_thread_error("plan " + std::to_string(i) + ": " + plans[i]->err);
      return sd;
    }
  // Work queue over the instances, largest grids first so that the small
  // ones fill in at the end.  Several host threads take instances from it,
  // each solving on a stream of its own, so that the kernels of small
  // instances (which fill a fraction of the SMs) and the host decisions of
  // one solve overlap with the work of others.  Grids above 2^20 points fill
  // the GPU alone and are solved one at a time (their banks are large).
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return plans[a]->grid.npts * m[a] > plans[b]->grid.npts * m[b]; });
  long long biggest = 0;
  for (int i = 0; i < count; ++i) biggest = std::max(biggest, plans[i]->grid.npts);
  int workers = getenv("BDG_BATCH_WORKERS") ? atoi(getenv("BDG_BATCH_WORKERS")) : 8;
  if (biggest > (1LL << 20)) workers = 1;
  workers = std::max(1, std::min(workers, count));
  std::vector<bdg_status> st(count, BDG_OK);
  auto run_one = [&](int i, cudaStream_t s) {
    st[i] = bdg_solve(plans[i], k[i], m[i], nullptr, omega[i], UV ? UV[i] : nullptr, resid ? resid[i] : nullptr,
                      &nconv[i], s);
    // bdg_solve has synchronized its stream; the plan must not keep a
    // worker's stream, which is destroyed when the worker ends
    plans[i]->last_stream = stream;
  };
  if (workers == 1) {
    for (int j = 0; j < count; ++j) run_one(order[j], (cudaStream_t)stream);
  } else {
    // the workers' streams start after the work already queued on the caller's stream
    cudaEvent_t ready = nullptr;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ready, (cudaStream_t)stream) != cudaSuccess)
      return fail(nullptr, BDG_ERR_CUDA, "event on the caller's stream failed");
    std::atomic<int> next{0};
    std::vector<cudaError_t> werr(workers, cudaSuccess);
    auto work = [&](int w) {
      cudaStream_t ws = nullptr;
      cudaError_t e = cudaSetDevice(dev);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(ws, ready, 0);
      if (e != cudaSuccess) {
        werr[w] = e;
        return;
      }
      for (int j; (j = next.fetch_add(1)) < count;) run_one(order[j], ws);
      cudaStreamSynchronize(ws);
      cudaStreamDestroy(ws);
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < workers; ++w) pool.emplace_back(work, w);
    for (auto& t : pool) t.join();
    cudaEventDestroy(ready);
    // a worker that could not start leaves its instances to the others; the
    // call fails only if none drained the queue
    if (next.load() < count) {
      cudaError_t e = cudaErrorUnknown;
      for (int w = 0; w < workers; ++w)
        if (werr[w] != cudaSuccess) e = werr[w];
      return fail(nullptr, BDG_ERR_CUDA, std::string("no batch worker could start: ") + cudaGetErrorString(e));
    }
  }
  bdg_status first = BDG_OK;
  for (int i = 0; i < count; ++i)
    if (st[i] != BDG_OK && first == BDG_OK) {
      first = st[i];
      set_thread_error("plan " + std::to_string(i) + ": " + plans[i]->err);
    }
  return first;
}
