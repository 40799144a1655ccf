// C ABI: plan life cycle, the BdG product, chemical potentials and the
// deflation bases (Sections 2.3 and 3.1).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "apply.cuh"
#include "blas.cuh"
#include "common.cuh"
#include "plan.cuh"

namespace bdg {

static thread_local std::string g_thread_error = "no error";

void set_thread_error(const std::string& msg) { g_thread_error = msg; }
const char* thread_error() { return g_thread_error.c_str(); }

cudaError_t allow_dynamic_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> granted;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& g = granted[{func, dev}];
  if (bytes <= g) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) g = bytes;
  return e;
}

bdg_status fail(bdg_plan_t plan, bdg_status st, const std::string& msg) {
  if (plan) plan->err = msg;
  set_thread_error(msg);
  return st;
}

bdg_status check_device(bdg_plan_t plan) {
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(plan, BDG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != plan->device)
    return fail(plan, BDG_ERR_INVALID, "the current device is " + std::to_string(dev) + " but the plan lives on device " +
                                           std::to_string(plan->device) + "; make the plan's device current first");
  return BDG_OK;
}

bdg_status ensure(bdg_plan_t plan, int slot, size_t bytes) {
  Buffer& b = plan->scratch[slot];
  if (b.bytes >= bytes) return BDG_OK;
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.bytes = 0;
  const size_t want = bytes < 256 ? 256 : bytes;
  if (cudaMalloc(&b.ptr, want) != cudaSuccess) {
    cudaGetLastError();
    return fail(plan, BDG_ERR_NOMEM, "device allocation of " + std::to_string(want) + " bytes failed");
  }
  b.bytes = want;
  // diagnostics (BDG_POISON): NaN bytes in new scratch, as for the solver's buffers
  if (getenv("BDG_POISON") && cudaMemset(b.ptr, 0xFF, want) != cudaSuccess)
    return fail(plan, BDG_ERR_CUDA, "scratch fill failed");
  return BDG_OK;
}

// ---------------------------------------------------------------------------
// argument helpers
// ---------------------------------------------------------------------------
static bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static bdg_status validate(const bdg_params* p, Grid* g, std::string* why) {
  if (!p) { *why = "params is NULL"; return BDG_ERR_INVALID; }
  if (p->dim < 1 || p->dim > 3) { *why = "dim must be 1, 2 or 3"; return BDG_ERR_INVALID; }
  g->dim = p->dim;
  g->npts = 1;
  for (int a = 0; a < p->dim; ++a) {
    if (!pow2(p->n[a]) || p->n[a] < 8 || p->n[a] > 1024) {
      *why = "n[" + std::to_string(a) + "] must be a power of two in [8, 1024]";
      return p->n[a] > 1024 || (pow2(p->n[a]) && p->n[a] < 8) ? BDG_ERR_UNSUPPORTED : BDG_ERR_INVALID;
    }
    if (!(std::isfinite(p->lo[a]) && std::isfinite(p->hi[a]) && p->hi[a] > p->lo[a])) {
      *why = "box axis " + std::to_string(a) + " must satisfy lo < hi (finite)";
      return BDG_ERR_INVALID;
    }
    g->n[a] = p->n[a];
    g->len[a] = p->hi[a] - p->lo[a];
    g->lo[a] = p->lo[a];
    g->npts *= p->n[a];
  }
  for (int a = p->dim; a < 3; ++a) { g->n[a] = 1; g->len[a] = 1.0; g->lo[a] = 0.0; }
  if (g->npts > (1LL << 27)) { *why = "more than 2^27 grid points"; return BDG_ERR_UNSUPPORTED; }
  const double sc[4] = {p->beta_n, p->beta_s, p->p, p->q};
  for (double v : sc)
    if (!std::isfinite(v)) { *why = "beta_n, beta_s, p, q must be finite"; return BDG_ERR_INVALID; }
  return BDG_OK;
}

// exp(-2 pi i r / N) in FP64 with the angle reduced to the first octant.
static void twiddles(int N, std::vector<double>& re, std::vector<double>& im) {
  re.resize(N);
  im.resize(N);
  for (int r = 0; r < N; ++r) {
    // angle 2 pi r / N = (pi/4) * (8 r / N); reduce r modulo N/8 octants
    const long long num = 8LL * r;  // in units of (pi/4)/N
    const int oct = (int)(num / N);
    const long long rem = num - (long long)oct * N;  // 0 <= rem < N
    const double t = (M_PI / 4.0) * (double)rem / (double)N;
    double c, s;
    // exact rotation by oct * pi/4 applied to (cos t, sin t)
    const double ct = std::cos(t), st = std::sin(t);
    const double h = 0.70710678118654752440;
    switch (oct & 7) {
      case 0: c = ct; s = st; break;
      case 1: c = h * (ct - st); s = h * (ct + st); break;
      case 2: c = -st; s = ct; break;
      case 3: c = -h * (ct + st); s = h * (ct - st); break;
      case 4: c = -ct; s = -st; break;
      case 5: c = -h * (ct - st); s = -h * (ct + st); break;
      case 6: c = st; s = -ct; break;
      default: c = h * (ct + st); s = -h * (ct - st); break;
    }
    re[r] = c;
    im[r] = -s;
  }
}

template <typename R>
static ApplyArgs<R> make_args(bdg_plan_t plan, int mode, const void* x, void* y, int nvec,
                              const double* mu) {
  ApplyArgs<R> g;
  g.grid = &plan->grid;
  g.x = (const typename CT<R>::T*)x;
  g.y = (typename CT<R>::T*)y;
  g.nvec = nvec;
  g.mode = mode;
  g.phiv = (const typename CT<R>::Q*)(sizeof(R) == 8 ? (const void*)plan->phiv64 : (const void*)plan->phiv32);
  for (int a = 0; a < 3; ++a) {
    g.tw[a] = (const typename CT<R>::T*)(sizeof(R) == 8 ? (const void*)plan->tw64[a] : (const void*)plan->tw32[a]);
    const double k0 = 2.0 * M_PI / plan->grid.len[a];
    g.kscale[a] = (R)(0.5 * k0 * k0 / plan->grid.n[a]);
  }
  const bdg_params& p = plan->prm;
  g.cp.beta_n = (R)p.beta_n;
  g.cp.beta_s = (R)p.beta_s;
  g.cp.d1 = (R)(p.q - p.p - mu[0]);
  g.cp.d0 = (R)(-mu[1]);
  g.cp.dm = (R)(p.q + p.p - mu[2]);
  return g;
}

bdg_status apply_internal(bdg_plan_t plan, int mode, int dtype, const void* x, void* y, int nvec,
                          cudaStream_t s, const double* mu_override) {
  const double* mu = mu_override ? mu_override : plan->mu;
  cudaError_t e;
  if (dtype == BDG_C128) e = apply_launch<double>(make_args<double>(plan, mode, x, y, nvec, mu), s);
  else e = apply_launch<float>(make_args<float>(plan, mode, x, y, nvec, mu), s);
  if (e != cudaSuccess) return fail(plan, BDG_ERR_CUDA, std::string("apply launch: ") + cudaGetErrorString(e));
  return BDG_OK;
}

// real dot product <a, b> of complex columns of length n (sum of re*re + im*im)
template <typename R>
static bdg_status dot_cols(bdg_plan_t plan, const void* a, const void* b, long long n, double* out,
                           cudaStream_t s) {
  PairBlock<R> A{(const typename CT<R>::T*)a, n, n, 1};
  PairBlock<R> B{(const typename CT<R>::T*)b, n, n, 1};
  bdg_status st = ensure(plan, SLOT_GRAM_WS, gram_workspace_bytes(1, 1, n));
  if (st) return st;
  st = ensure(plan, SLOT_SMALL, 64 * sizeof(double));
  if (st) return st;
  double* G = (double*)plan->scratch[SLOT_SMALL].ptr;
  BDG_CUDA_TRY(plan, gram_pairs<R>(A, B, G, plan->scratch[SLOT_GRAM_WS].ptr,
                                   plan->scratch[SLOT_GRAM_WS].bytes, s));
  double h[4];
  BDG_CUDA_TRY(plan, cudaMemcpyAsync(h, G, sizeof(h), cudaMemcpyDeviceToHost, s));
  BDG_CUDA_TRY(plan, cudaStreamSynchronize(s));
  *out = h[0] + h[3];
  return BDG_OK;
}

// Build the real vectors used at set-up from (phi_1, phi_0, phi_-1, V):
// kind 0: [0,0,0, phi] (FG vector), 1: Phi, 2: S_z Phi, 3: -i S_y Phi,
// 4: S_x Phi (f-part 3 x N_p complex with zero imaginary parts).
__global__ void k_build(const dquad* __restrict__ pv, long long np, int kind, double2* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
       i += (long long)gridDim.x * blockDim.x) {
    const dquad v = pv[i];
    double c0, c1, c2;
    if (kind == 0 || kind == 1) { c0 = v.x; c1 = v.y; c2 = v.z; }
    else if (kind == 2) { c0 = v.x; c1 = 0.0; c2 = -v.z; }
    else if (kind == 3) { const double h = 0.70710678118654752440; c0 = -h * v.y; c1 = h * (v.x - v.z); c2 = h * v.y; }
    else { const double h = 0.70710678118654752440; c0 = h * v.y; c1 = h * (v.x + v.z); c2 = h * v.y; }
    if (kind == 0) {
      out[i] = make_double2(0.0, 0.0);
      out[np + i] = make_double2(0.0, 0.0);
      out[2 * np + i] = make_double2(0.0, 0.0);
      out[3 * np + i] = make_double2(c0, 0.0);
      out[4 * np + i] = make_double2(c1, 0.0);
      out[5 * np + i] = make_double2(c2, 0.0);
    } else {
      out[i] = make_double2(c0, 0.0);
      out[np + i] = make_double2(c1, 0.0);
      out[2 * np + i] = make_double2(c2, 0.0);
    }
  }
}

static unsigned blocks_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b));
}

// Chemical potentials by eq. chem-formula: with mu = 0, the FG product of
// (0, Phi) gives (H_- Phi) = H Phi; mu_j = <phi_j, (H Phi)_j> / |phi_j|^2,
// and the relation mu_1 + mu_-1 = 2 mu_0 fills components with
// |phi_j|^2 < 1e-20 |Phi|^2 (unweighted grid sums): a component that small
// is the decayed remnant of the ground-state iteration, and its own Rayleigh
// quotient (the energy of its slowest mode) would shift the whole m = j
// branch of the operator.
static bdg_status compute_mu(bdg_plan_t plan, cudaStream_t s, double* mu) {
  const long long np = plan->grid.npts;
  bdg_status st = ensure(plan, SLOT_VEC_A, sizeof(double2) * 6 * np);
  if (st) return st;
  st = ensure(plan, SLOT_VEC_B, sizeof(double2) * 6 * np);
  if (st) return st;
  double2* x = (double2*)plan->scratch[SLOT_VEC_A].ptr;
  double2* y = (double2*)plan->scratch[SLOT_VEC_B].ptr;
  k_build<<<blocks_for(np), 256, 0, s>>>(plan->phiv64, np, 0, x);
  BDG_CUDA_TRY(plan, cudaGetLastError());
  const double zero[3] = {0.0, 0.0, 0.0};
  st = apply_internal(plan, BDG_FG, BDG_C128, x, y, 1, s, zero);
  if (st) return st;
  double num[3], den[3];
  for (int j = 0; j < 3; ++j) {
    st = dot_cols<double>(plan, x + (3 + j) * np, y + (3 + j) * np, np, &num[j], s);
    if (st) return st;
    st = dot_cols<double>(plan, x + (3 + j) * np, x + (3 + j) * np, np, &den[j], s);
    if (st) return st;
  }
  const double tiny = 1e-20 * (den[0] + den[1] + den[2]);
  bool z[3];
  for (int j = 0; j < 3; ++j) {
    z[j] = den[j] < tiny;
    mu[j] = z[j] ? NAN : num[j] / den[j];
  }
  if (z[1] && !z[0] && !z[2]) mu[1] = 0.5 * (mu[0] + mu[2]);
  else if (z[0] && z[2] && !z[1]) mu[0] = mu[2] = mu[1];
  else if (z[0] && !z[2] && !z[1]) mu[0] = 2 * mu[1] - mu[2];
  else if (z[2] && !z[0] && !z[1]) mu[2] = 2 * mu[1] - mu[0];
  for (int j = 0; j < 3; ++j)
    if (!std::isfinite(mu[j])) return fail(plan, BDG_ERR_INVALID, "Phi has no nonzero component");
  return BDG_OK;
}

// z -= w (w . z) for the unit column w, as pair coefficients (imaginary parts zero)
static bdg_status subtract_projection(bdg_plan_t plan, const double2* w, double2* z, long long n3,
                                      cudaStream_t s) {
  double d;
  bdg_status st = dot_cols<double>(plan, w, z, n3, &d, s);
  if (st) return st;
  double hC[4] = {-d, 0.0, 0.0, -d};
  st = ensure(plan, SLOT_SMALL, 64 * sizeof(double));
  if (st) return st;
  double* C = (double*)plan->scratch[SLOT_SMALL].ptr;
  BDG_CUDA_TRY(plan, cudaMemcpyAsync(C, hC, sizeof(hC), cudaMemcpyHostToDevice, s));
  PairBlock<double> A{w, n3, n3, 1};
  BDG_CUDA_TRY(plan, update_pairs<double>(A, C, 2, 1.0, z, n3, 1, s));
  BDG_CUDA_TRY(plan, cudaStreamSynchronize(s));
  return BDG_OK;
}

// Deflation bases (Section 2.3; Theorems on null(H_-) and null(H_+)):
// Z_f = orthonormal span{Phi, S_z Phi} (in null(H_-) for a ground state),
// S_z Phi dropped when (numerically) parallel to Phi or zero, plus the part
// of S_x Phi outside that span when it is numerically in null(H_-) (states
// symmetric under the rotation about x: antiferromagnetic or polar at
// p = q = 0; every f of a pair with omega != 0 is H_- g / omega, so any
// null(H_-) vector may be deflated);
// Z_g = {-i S_y Phi / |.|} when |H_+ z| / |z| < 1e-8 (in null(H_+)).
static bdg_status build_deflation(bdg_plan_t plan, cudaStream_t s) {
  const long long np = plan->grid.npts, n3 = 3 * np;
  std::vector<double2*> cols;
  double2* zf = nullptr;
  double2* zg = nullptr;
  BDG_CUDA_TRY(plan, cudaMalloc(&zf, sizeof(double2) * 3 * n3));
  BDG_CUDA_TRY(plan, cudaMalloc(&zg, sizeof(double2) * n3));
  plan->zf64 = (double*)zf;
  plan->zg64 = (double*)zg;
  k_build<<<blocks_for(np), 256, 0, s>>>(plan->phiv64, np, 1, zf);
  k_build<<<blocks_for(np), 256, 0, s>>>(plan->phiv64, np, 2, zf + n3);
  k_build<<<blocks_for(np), 256, 0, s>>>(plan->phiv64, np, 3, zg);
  BDG_CUDA_TRY(plan, cudaGetLastError());
  double nn1, nn2, d12;
  bdg_status st = dot_cols<double>(plan, zf, zf, n3, &nn1, s);
  if (st) return st;
  if (!(nn1 > 0)) return fail(plan, BDG_ERR_INVALID, "Phi is zero");
  st = dot_cols<double>(plan, zf + n3, zf + n3, n3, &nn2, s);
  if (st) return st;
  st = dot_cols<double>(plan, zf, zf + n3, n3, &d12, s);
  if (st) return st;
  // z1 = Phi / |Phi|
  BDG_CUDA_TRY(plan, scale_pairs<double>(zf, n3, n3, 1, nullptr, 1.0 / std::sqrt(nn1), s));
  d12 /= std::sqrt(nn1);
  const double r2 = nn2 - d12 * d12;  // |S_z Phi - (z1.S_z Phi) z1|^2
  int nzf = 1;
  if (nn2 > 1e-24 * nn1 && r2 > 1e-24 * nn2) {
    // z2 = (S_z Phi - d12 z1) / sqrt(r2), twice for accuracy
    for (int pass = 0; pass < 2; ++pass) {
      double d;
      st = dot_cols<double>(plan, zf, zf + n3, n3, &d, s);
      if (st) return st;
      double hC[4] = {-d, 0.0, 0.0, -d};  // update: z2 -= d * z1 (pair coefficients)
      st = ensure(plan, SLOT_SMALL, 64 * sizeof(double));
      if (st) return st;
      double* C = (double*)plan->scratch[SLOT_SMALL].ptr;
      BDG_CUDA_TRY(plan, cudaMemcpyAsync(C, hC, sizeof(hC), cudaMemcpyHostToDevice, s));
      PairBlock<double> A{zf, n3, n3, 1};
      BDG_CUDA_TRY(plan, update_pairs<double>(A, C, 2, 1.0, zf + n3, n3, 1, s));
      BDG_CUDA_TRY(plan, cudaStreamSynchronize(s));
    }
    double nz;
    st = dot_cols<double>(plan, zf + n3, zf + n3, n3, &nz, s);
    if (st) return st;
    BDG_CUDA_TRY(plan, scale_pairs<double>(zf + n3, n3, n3, 1, nullptr, 1.0 / std::sqrt(nz), s));
    nzf = 2;
  }
  {
    // S_x Phi in the next column: orthogonalized twice against Z_f, kept
    // when a direction of relative size > 1e-6 is left and |H_- z| < 1e-8
    double2* zc = zf + nzf * n3;
    k_build<<<blocks_for(np), 256, 0, s>>>(plan->phiv64, np, 4, zc);
    BDG_CUDA_TRY(plan, cudaGetLastError());
    double nsx;
    st = dot_cols<double>(plan, zc, zc, n3, &nsx, s);
    if (st) return st;
    if (nsx > 1e-24 * nn1) {
      for (int pass = 0; pass < 2; ++pass)
        for (int j = 0; j < nzf; ++j)
          if ((st = subtract_projection(plan, zf + j * n3, zc, n3, s))) return st;
      double nr;
      st = dot_cols<double>(plan, zc, zc, n3, &nr, s);
      if (st) return st;
      if (nr > 1e-12 * nsx) {
        BDG_CUDA_TRY(plan, scale_pairs<double>(zc, n3, n3, 1, nullptr, 1.0 / std::sqrt(nr), s));
        st = ensure(plan, SLOT_VEC_A, sizeof(double2) * 6 * np);
        if (st) return st;
        st = ensure(plan, SLOT_VEC_B, sizeof(double2) * 6 * np);
        if (st) return st;
        double2* x = (double2*)plan->scratch[SLOT_VEC_A].ptr;
        double2* y = (double2*)plan->scratch[SLOT_VEC_B].ptr;
        // H_- z is the g-part of the FG product of (0, z)
        BDG_CUDA_TRY(plan, cudaMemsetAsync(x, 0, sizeof(double2) * 6 * np, s));
        BDG_CUDA_TRY(plan, cudaMemcpyAsync(x + n3, zc, sizeof(double2) * n3, cudaMemcpyDeviceToDevice, s));
        st = apply_internal(plan, BDG_FG, BDG_C128, x, y, 1, s, nullptr);
        if (st) return st;
        double nh;
        st = dot_cols<double>(plan, y + n3, y + n3, n3, &nh, s);
        if (st) return st;
        if (std::sqrt(nh) < 1e-8) nzf++;
      }
    }
  }
  plan->nzf = nzf;
  // Z_g candidate: H_+ z via the FG product of (z, 0)
  double ny;
  st = dot_cols<double>(plan, zg, zg, n3, &ny, s);
  if (st) return st;
  plan->nzg = 0;
  if (ny > 1e-24 * nn1) {
    st = ensure(plan, SLOT_VEC_A, sizeof(double2) * 6 * np);
    if (st) return st;
    st = ensure(plan, SLOT_VEC_B, sizeof(double2) * 6 * np);
    if (st) return st;
    double2* x = (double2*)plan->scratch[SLOT_VEC_A].ptr;
    double2* y = (double2*)plan->scratch[SLOT_VEC_B].ptr;
    BDG_CUDA_TRY(plan, cudaMemsetAsync(x, 0, sizeof(double2) * 6 * np, s));
    BDG_CUDA_TRY(plan, cudaMemcpyAsync(x, zg, sizeof(double2) * n3, cudaMemcpyDeviceToDevice, s));
    st = apply_internal(plan, BDG_FG, BDG_C128, x, y, 1, s, nullptr);
    if (st) return st;
    double nh;
    st = dot_cols<double>(plan, y, y, n3, &nh, s);
    if (st) return st;
    if (std::sqrt(nh / ny) < 1e-8) {
      BDG_CUDA_TRY(plan, scale_pairs<double>(zg, n3, n3, 1, nullptr, 1.0 / std::sqrt(ny), s));
      plan->nzg = 1;
    }
  }
  // FP32 copies
  BDG_CUDA_TRY(plan, cudaMalloc(&plan->zf32, sizeof(float2) * 3 * n3));
  BDG_CUDA_TRY(plan, cudaMalloc(&plan->zg32, sizeof(float2) * n3));
  BDG_CUDA_TRY(plan, (convert_pairs<double, float>(zf, n3, (float2*)plan->zf32, n3, n3, 3, s)));
  BDG_CUDA_TRY(plan, (convert_pairs<double, float>(zg, n3, (float2*)plan->zg32, n3, n3, 1, s)));
  BDG_CUDA_TRY(plan, cudaStreamSynchronize(s));
  return BDG_OK;
}

static void free_plan(bdg_plan_t plan) {
  if (!plan) return;
  cudaFree(plan->phiv64);
  cudaFree(plan->phiv32);
  for (int a = 0; a < 3; ++a) {
    cudaFree(plan->tw64[a]);
    cudaFree(plan->tw32[a]);
  }
  cudaFree(plan->zf64);
  cudaFree(plan->zg64);
  cudaFree(plan->zf32);
  cudaFree(plan->zg32);
  for (auto& b : plan->scratch) cudaFree(b.ptr);
  delete plan;
}

}  // namespace bdg

using namespace bdg;

extern "C" {

bdg_status bdg_plan_create(bdg_plan_t* out, const bdg_params* p, const double* V, const double* phi,
                           void* stream) {
  if (!out) return fail(nullptr, BDG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  Grid g;
  std::string why;
  bdg_status st = validate(p, &g, &why);
  if (st) return fail(nullptr, st, why);
  if (!V || !phi) return fail(nullptr, BDG_ERR_INVALID, "V and phi must be host pointers");
  cudaStream_t s = (cudaStream_t)stream;
  bdg_plan_t plan = new (std::nothrow) bdg_plan_s();
  if (!plan) return fail(nullptr, BDG_ERR_NOMEM, "host allocation failed");
  plan->prm = *p;
  plan->grid = g;
  memset(&plan->stats, 0, sizeof(plan->stats));
  cudaGetDevice(&plan->device);
  const long long np = g.npts;
  std::vector<dquad> h64(np);
  std::vector<float4> h32(np);
  for (long long i = 0; i < np; ++i) {
    const double a = phi[i], b = phi[np + i], c = phi[2 * np + i], v = V[i];
    if (!(std::isfinite(a) && std::isfinite(b) && std::isfinite(c) && std::isfinite(v))) {
      free_plan(plan);
      return fail(nullptr, BDG_ERR_NAN, "phi or V holds NaN/Inf");
    }
    h64[i] = dquad{a, b, c, v};
    h32[i] = make_float4((float)a, (float)b, (float)c, (float)v);
  }
#define CREATE_TRY(call)                                                                     \
  do {                                                                                       \
    cudaError_t e__ = (call);                                                                \
    if (e__ != cudaSuccess) {                                                                \
      std::string m__ = std::string(#call) + ": " + cudaGetErrorString(e__);                 \
      free_plan(plan);                                                                       \
      return fail(nullptr, e__ == cudaErrorMemoryAllocation ? BDG_ERR_NOMEM : BDG_ERR_CUDA, m__); \
    }                                                                                        \
  } while (0)
  CREATE_TRY(cudaMalloc(&plan->phiv64, sizeof(dquad) * np));
  CREATE_TRY(cudaMalloc(&plan->phiv32, sizeof(float4) * np));
  CREATE_TRY(cudaMemcpyAsync(plan->phiv64, h64.data(), sizeof(dquad) * np, cudaMemcpyHostToDevice, s));
  CREATE_TRY(cudaMemcpyAsync(plan->phiv32, h32.data(), sizeof(float4) * np, cudaMemcpyHostToDevice, s));
  for (int a = 0; a < g.dim; ++a) {
    std::vector<double> re, im;
    twiddles(g.n[a], re, im);
    std::vector<double2> t64(g.n[a]);
    std::vector<float2> t32(g.n[a]);
    for (int r = 0; r < g.n[a]; ++r) {
      t64[r] = make_double2(re[r], im[r]);
      t32[r] = make_float2((float)re[r], (float)im[r]);
    }
    CREATE_TRY(cudaMalloc(&plan->tw64[a], sizeof(double2) * g.n[a]));
    CREATE_TRY(cudaMalloc(&plan->tw32[a], sizeof(float2) * g.n[a]));
    CREATE_TRY(cudaMemcpyAsync(plan->tw64[a], t64.data(), sizeof(double2) * g.n[a], cudaMemcpyHostToDevice, s));
    CREATE_TRY(cudaMemcpyAsync(plan->tw32[a], t32.data(), sizeof(float2) * g.n[a], cudaMemcpyHostToDevice, s));
  }
  CREATE_TRY(cudaStreamSynchronize(s));
#undef CREATE_TRY
  bool need_mu = false;
  for (int j = 0; j < 3; ++j) {
    plan->mu[j] = p->mu[j];
    if (std::isnan(p->mu[j])) need_mu = true;
    else if (!std::isfinite(p->mu[j])) {
      free_plan(plan);
      return fail(nullptr, BDG_ERR_INVALID, "mu must be finite or NaN");
    }
  }
  if (need_mu) {
    double mu[3];
    st = compute_mu(plan, s, mu);
    if (st) {
      std::string m = plan->err;
      free_plan(plan);
      return fail(nullptr, st, m);
    }
    for (int j = 0; j < 3; ++j)
      if (std::isnan(p->mu[j])) plan->mu[j] = mu[j];
  }
  st = build_deflation(plan, s);
  if (st) {
    std::string m = plan->err;
    free_plan(plan);
    return fail(nullptr, st, m);
  }
  plan->last_stream = stream;
  *out = plan;
  return BDG_OK;
}

bdg_status bdg_plan_destroy(bdg_plan_t plan) {
  if (!plan) return BDG_OK;
  cudaStreamSynchronize((cudaStream_t)plan->last_stream);
  free_plan(plan);
  return BDG_OK;
}

bdg_status bdg_plan_mu(bdg_plan_t plan, double* mu) {
  if (!plan || !mu) return fail(plan, BDG_ERR_INVALID, "plan and mu must be non-NULL");
  for (int j = 0; j < 3; ++j) mu[j] = plan->mu[j];
  return BDG_OK;
}

bdg_status bdg_apply(bdg_plan_t plan, int mode, int dtype, const void* x, void* y, int nvec,
                     void* stream) {
  if (!plan) return fail(nullptr, BDG_ERR_INVALID, "plan is NULL");
  if (mode != BDG_UV && mode != BDG_FG) return fail(plan, BDG_ERR_INVALID, "mode must be BDG_UV or BDG_FG");
  if (dtype != BDG_C128 && dtype != BDG_C64) return fail(plan, BDG_ERR_INVALID, "dtype must be BDG_C128 or BDG_C64");
  if (nvec < 0) return fail(plan, BDG_ERR_INVALID, "nvec < 0");
  if (nvec == 0) return BDG_OK;
  if (bdg_status sd = check_device(plan)) return sd;
  if (!x || !y) return fail(plan, BDG_ERR_INVALID, "x and y must be device pointers");
  const size_t esz = dtype == BDG_C128 ? 16 : 8;
  const size_t bytes = esz * 6 * (size_t)plan->grid.npts * (size_t)nvec;
  const char* xb = (const char*)x;
  const char* yb = (const char*)y;
  if (xb < yb + bytes && yb < xb + bytes) return fail(plan, BDG_ERR_INVALID, "x and y overlap");
  if (((uintptr_t)x | (uintptr_t)y) % esz) return fail(plan, BDG_ERR_INVALID, "x, y not aligned to the element size");
  plan->last_stream = stream;
  return apply_internal(plan, mode, dtype, x, y, nvec, (cudaStream_t)stream, nullptr);
}

const char* bdg_last_error(bdg_plan_t plan) {
  if (plan) return plan->err.empty() ? "no error" : plan->err.c_str();
  return thread_error();
}

bdg_status bdg_gram(int dtype, int engine, const void* A, long long lda, int ncol_a, const void* B, long long ldb,
                    int ncol_b, long long n, double* G, void* stream) {
  if (dtype != BDG_C64 && dtype != BDG_C128) return fail(nullptr, BDG_ERR_INVALID, "dtype must be BDG_C64 or BDG_C128");
  if (engine != BDG_GRAM_SIMT && engine != BDG_GRAM_TENSOR)
    return fail(nullptr, BDG_ERR_INVALID, "engine must be BDG_GRAM_SIMT or BDG_GRAM_TENSOR");
  if (ncol_a < 0 || ncol_b < 0 || n < 0) return fail(nullptr, BDG_ERR_INVALID, "negative size");
  if (ncol_a == 0 || ncol_b == 0) return BDG_OK;
  if (!G || (n > 0 && (!A || !B))) return fail(nullptr, BDG_ERR_INVALID, "A, B and G must be device pointers");
  if ((ncol_a > 1 && lda < n) || (ncol_b > 1 && ldb < n))
    return fail(nullptr, BDG_ERR_INVALID, "column stride below the column length");
  if (engine == BDG_GRAM_TENSOR && !gram_tc_supported(ncol_a, ncol_b))
    return fail(nullptr, BDG_ERR_UNSUPPORTED, "tensor-core Gram needs 2 ncol_b <= 160");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ws_bytes = gram_workspace_bytes(ncol_a, ncol_b, n > 0 ? n : 1);
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, ws_bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, BDG_ERR_NOMEM, "Gram workspace allocation failed");
  }
  cudaError_t e;
  if (dtype == BDG_C128) {
    PairBlock<double> a{(const double2*)A, lda, n, ncol_a}, b{(const double2*)B, ldb, n, ncol_b};
    e = engine == BDG_GRAM_TENSOR ? gram_pairs_tc<double>(a, b, G, ws, ws_bytes, s)
                                  : gram_pairs<double>(a, b, G, ws, ws_bytes, s, false);
  } else {
    PairBlock<float> a{(const float2*)A, lda, n, ncol_a}, b{(const float2*)B, ldb, n, ncol_b};
    e = engine == BDG_GRAM_TENSOR ? gram_pairs_tc<float>(a, b, G, ws, ws_bytes, s)
                                  : gram_pairs<float>(a, b, G, ws, ws_bytes, s, false);
  }
  const cudaError_t ef = cudaFreeAsync(ws, s);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) return fail(nullptr, BDG_ERR_CUDA, std::string("bdg_gram: ") + cudaGetErrorString(e));
  return BDG_OK;
}

bdg_status bdg_get_solve_stats(bdg_plan_t plan, bdg_solve_stats* st) {
  if (!plan || !st) return fail(plan, BDG_ERR_INVALID, "plan and st must be non-NULL");
  *st = plan->stats;
  return BDG_OK;
}

}  // extern "C"
