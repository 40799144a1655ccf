// Ground state on S_M (eq. groundDef) on the device, FP64.
//
// Phase 1, normalized gradient flow: with N(Phi) Phi the non-kinetic part of
// H Phi (eq. NLEP: trap, density, spin and Zeeman terms) and c = 1/tau +
// alpha, alpha >= max_x (V + (beta_n + |beta_s|) rho) + |p| + |q|,
//     (c - 1/2 Lap) Phi* = c Phi - N(Phi) Phi,   Phi <- P_SM(Phi*),
// the kinetic term implicit and diagonal in Fourier space (Section 3.1).
// Phase 2, inexact Newton on S_M: with the multipliers (mu + lambda S_z) of
// the least-squares fit H Phi ~ (mu + lambda S_z) Phi, solve
//     P H_+ P d = -P (H Phi - (mu + lambda S_z) Phi)
// by preconditioned CG on the tangent space {<Phi, d> = <S_z Phi, d> = 0}
// (P its projector, preconditioner P (c - 1/2 Lap)^-1 P), H_+ = A + B the
// Hessian of the Lagrangian (eqs. def_A + def_B at a real Phi), then
// Phi <- P_SM(Phi + d).  A Newton step that does not lower the residual
// hands back to 50 flow steps.
// Newton converges to any stationary point.  A converged state is therefore
// tested for negative curvature of the energy on S_M along the directions
// that move population between spin components; a saddle (e.g. the
// antiferromagnetic state when q > 0 makes the polar state lower) is left
// along that direction and the flow resumes (at most three times).
//
// P_SM scales the components, phi_j <- sigma_j phi_j, to mass 1 and
// magnetization M with sigma_1 sigma_-1 = sigma_0^2 (closed form).  The
// products H Phi and H_+ d come from the BdG product kernels of an internal
// plan whose (Phi, V) table is refreshed from the current iterate: with
// mu = 0 the FG product of (0, Phi) is H_- Phi = H Phi.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "blas.cuh"
#include "kdiag.cuh"
#include "plan.cuh"

namespace bdg {
namespace {

unsigned nblk(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b > 152 * 8 ? 152 * 8 : (b < 1 ? 1 : b));
}

// (phi_1, phi_0, phi_-1, V) table of the internal plan from the iterate
__global__ void k_gs_table(const double2* __restrict__ phi, const double* __restrict__ V, long long np,
                           dquad* __restrict__ t64, float4* __restrict__ t32) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
       i += (long long)gridDim.x * blockDim.x) {
    const double a = phi[i].x, b = phi[np + i].x, c = phi[2 * np + i].x, v = V[i];
    t64[i] = dquad{a, b, c, v};
    t32[i] = make_float4((float)a, (float)b, (float)c, (float)v);
  }
}

struct GsCoef {
  double beta_n, beta_s, p, q;
};

// rhs = c Phi - N(Phi) Phi.  For real Phi = (a, b, c3): F_x = sqrt2 b (a + c3),
// F_z = a^2 - c3^2, F_y = 0, and (F.S) Phi = (b^2 (a+c3) + F_z a, b (a+c3)^2,
// b^2 (a+c3) - F_z c3); the Zeeman term is diag(q - p, 0, q + p).
__global__ void k_gs_flow_rhs(const double2* __restrict__ phi, const double* __restrict__ V, long long np,
                              GsCoef k, double cst, double2* __restrict__ rhs) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
       i += (long long)gridDim.x * blockDim.x) {
    const double a = phi[i].x, b = phi[np + i].x, c = phi[2 * np + i].x;
    const double rho = a * a + b * b + c * c, fz = a * a - c * c, s = a + c;
    const double w = V[i] + k.beta_n * rho;
    const double n1 = w * a + k.beta_s * (b * b * s + fz * a) + (k.q - k.p) * a;
    const double n0 = w * b + k.beta_s * (b * s * s);
    const double nm = w * c + k.beta_s * (b * b * s - fz * c) + (k.q + k.p) * c;
    rhs[i] = make_double2(cst * a - n1, 0.0);
    rhs[np + i] = make_double2(cst * b - n0, 0.0);
    rhs[2 * np + i] = make_double2(cst * c - nm, 0.0);
  }
}

// atomic max of non-negative doubles through their bit patterns
__device__ void atomic_max_pos(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)blockDim.x / 32; ++q) m = fmax(m, red[q]);
  return m;
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)blockDim.x / 32; ++q) m += red[q];
  __syncthreads();
  return m;
}

// out[0] = max_x (V + (beta_n + |beta_s|) rho)
__global__ void k_gs_stab(const double2* __restrict__ phi, const double* __restrict__ V, long long np, double bsum,
                          double* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
       i += (long long)gridDim.x * blockDim.x) {
    const double a = phi[i].x, b = phi[np + i].x, c = phi[2 * np + i].x;
    m = fmax(m, V[i] + bsum * (a * a + b * b + c * c));
  }
  m = block_max(m, red);
  if (threadIdx.x == 0) atomic_max_pos(out, m);
}

// out[0] = max_{j,x} |Hphi_j - mu_j phi_j|
__global__ void k_gs_maxres(const double2* __restrict__ hphi, const double2* __restrict__ phi, long long np,
                            double mu0, double mu1, double mu2, double* out) {
  __shared__ double red[32];
  double m = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * np;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / np);
    const double mu = j == 0 ? mu0 : (j == 1 ? mu1 : mu2);
    m = fmax(m, fabs(hphi[e].x - mu * phi[e].x));
  }
  m = block_max(m, red);
  if (threadIdx.x == 0) atomic_max_pos(out, m);
}

// up to 8 dot products over len complex elements (real parts), as per-CTA
// partial sums out[q * gridDim.x + blockIdx.x] (summed in a fixed order on
// the host, so that the flow is reproducible run to run)
struct DotSet {
  const double2* a[8];
  const double2* b[8];
  int count;
};
__global__ void k_gs_dots(DotSet d, long long len, double* out) {
  __shared__ double red[32];
  for (int q = 0; q < d.count; ++q) {
    double s = 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (long long)gridDim.x * blockDim.x)
      s += d.a[q][e].x * d.b[q][e].x;
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[(long long)q * gridDim.x + blockIdx.x] = s;
  }
}

// y = a x + b y over len complex elements (real and imaginary parts alike)
__global__ void k_gs_axpby(long long len, double a, const double2* __restrict__ x, double b, double2* y) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < len;
       e += (long long)gridDim.x * blockDim.x) {
    const double2 u = x[e], v = y[e];
    y[e] = make_double2(a * u.x + b * v.x, a * u.y + b * v.y);
  }
}

// per-component scale phi_j *= s_j
__global__ void k_gs_scale3(double2* phi, long long np, double s0, double s1, double s2) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * np;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / np);
    const double s = j == 0 ? s0 : (j == 1 ? s1 : s2);
    phi[e].x *= s;
    phi[e].y *= s;
  }
}

// r_j = Hphi_j - m_j phi_j
__global__ void k_gs_resid(const double2* __restrict__ hphi, const double2* __restrict__ phi, long long np,
                           double m0, double m1, double m2, double2* __restrict__ r) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * np;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / np);
    const double m = j == 0 ? m0 : (j == 1 ? m1 : m2);
    r[e] = make_double2(hphi[e].x - m * phi[e].x, 0.0);
  }
}

// S_z Phi
// Directions that move population between the spin components of Phi = (a,
// b, c): kind 0: (0, (a + c) / sqrt2, 0) (from +-1 into 0), kind 1:
// (b, 0, b) / sqrt2 and kind 2: (b, 0, -b) / sqrt2 (from 0 into +-1).  At a
// stationary state that is not a minimum (e.g. the antiferromagnetic state
// (a, 0, a) when q > 0 makes the polar state lower) one of them has negative
// curvature.
__global__ void k_gs_transfer(const double2* __restrict__ phi, long long np, int kind, double2* __restrict__ out) {
  const double h = 0.70710678118654752440;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
       i += (long long)gridDim.x * blockDim.x) {
    const double a = phi[i].x, b = phi[np + i].x, c = phi[2 * np + i].x;
    double o0 = 0.0, o1 = 0.0, o2 = 0.0;
    if (kind == 0) o1 = h * (a + c);
    else if (kind == 1) { o0 = h * b; o2 = h * b; }
    else { o0 = h * b; o2 = -h * b; }
    out[i] = make_double2(o0, 0.0);
    out[np + i] = make_double2(o1, 0.0);
    out[2 * np + i] = make_double2(o2, 0.0);
  }
}

__global__ void k_gs_sz(const double2* __restrict__ phi, long long np, double2* __restrict__ out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * np;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / np);
    out[e] = j == 0 ? phi[e] : (j == 1 ? make_double2(0.0, 0.0) : make_double2(-phi[e].x, -phi[e].y));
  }
}

class GroundState {
 public:
  GroundState(bdg_plan_t plan, double M, cudaStream_t s) : plan_(plan), M_(M), s_(s) {
    np_ = plan->grid.npts;
    n3_ = 3 * np_;
    cell_ = 1.0;
    for (int a = 0; a < plan->grid.dim; ++a) cell_ *= plan->grid.len[a] / plan->grid.n[a];
    k_.beta_n = plan->prm.beta_n;
    k_.beta_s = plan->prm.beta_s;
    k_.p = plan->prm.p;
    k_.q = plan->prm.q;
  }
  ~GroundState() {
    for (void* p : bufs_) cudaFree(p);
  }

  bdg_status init(const double* V, const double* phi0) {
    bdg_status st;
    if ((st = alloc(&V_, sizeof(double) * np_)) || (st = alloc(&phi_, sizeof(double2) * n3_)) ||
        (st = alloc(&trial_, sizeof(double2) * n3_)) || (st = alloc(&hphi_, sizeof(double2) * n3_)) ||
        (st = alloc(&x6_, sizeof(double2) * 6 * np_)) || (st = alloc(&y6_, sizeof(double2) * 6 * np_)) ||
        (st = alloc(&z_[0], sizeof(double2) * n3_)) || (st = alloc(&z_[1], sizeof(double2) * n3_)) ||
        (st = alloc(&cx_, sizeof(double2) * n3_)) || (st = alloc(&cr_, sizeof(double2) * n3_)) ||
        (st = alloc(&cz_, sizeof(double2) * n3_)) || (st = alloc(&cp_, sizeof(double2) * n3_)) ||
        (st = alloc(&cap_, sizeof(double2) * n3_)) || (st = alloc(&dred_, sizeof(double) * 16)) ||
        (st = alloc(&dpart_, sizeof(double) * DPART)))
      return st;
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(V_, V, sizeof(double) * np_, cudaMemcpyHostToDevice, s_));
    std::vector<double2> h(n3_);
    for (long long e = 0; e < n3_; ++e) h[e] = make_double2(phi0[e], 0.0);
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(phi_, h.data(), sizeof(double2) * n3_, cudaMemcpyHostToDevice, s_));
    BDG_CUDA_TRY(plan_, cudaStreamSynchronize(s_));
    return project(phi_);
  }

  // the loop of phases 1 and 2; returns the residual through *res
  bdg_status run(double tol, int maxit, double* res, double mu[3], int* iters) {
    const double tau = 1.0, newton_start = 1e-3;
    int it = 0;
    bdg_status st = residual(phi_, res, mu);
    if (st) return st;
    double alpha = 0.0;
    if ((st = stab(phi_, &alpha))) return st;
    double c = 1.0 / tau + alpha;
    int phase = 1, flow_left = 0, restarts = 0, flow_only = 0;
    double last = INFINITY;
    while (it < maxit) {
      if (*res <= tol) {
        // a converged stationary state that is a saddle of the energy on S_M
        // is left along its negative-curvature direction and the flow resumes
        bool unstable = false;
        if (restarts >= 3) break;
        if ((st = stability(&unstable))) return st;
        if (!unstable) break;
        ++restarts;
        const double nphi = std::sqrt(dot1(phi_, phi_, &st));
        if (st) return st;
        k_gs_axpby<<<nblk(n3_), 256, 0, s_>>>(n3_, 1e-2 * nphi, cp_, 1.0, phi_);
        BDG_CUDA_TRY(plan_, cudaGetLastError());
        if ((st = project(phi_)) || (st = residual(phi_, res, mu))) return st;
        phase = 1;
        flow_left = 0;
        flow_only = 500;   // no Newton step until the unstable component has grown
        last = INFINITY;
        continue;
      }
      if (phase == 1 || flow_left > 0) {
        if ((st = flow_step(c))) return st;
        flow_left = flow_left > 0 ? flow_left - 1 : 0;
        ++it;
        if ((st = residual(phi_, res, mu))) return st;
        if (it % 50 == 0) {
          if ((st = stab(phi_, &alpha))) return st;
          c = 1.0 / tau + alpha;
          if (phase == 1 && flow_only == 0 && *res > 0.99 * last) phase = 2;
          last = *res;
        }
        const double mmax = std::max(std::fabs(mu[0]), std::max(std::fabs(mu[1]), std::fabs(mu[2])));
        if (flow_only > 0) {
          --flow_only;
          phase = 1;
        }
        if (phase == 1 && flow_only == 0 && *res < newton_start * (1.0 + mmax)) phase = 2;
      } else {
        int products = 0;
        if ((st = newton_step(c, &products))) return st;
        it += 1 + products;
        double rt, mt[3];
        if ((st = residual(trial_, &rt, mt))) return st;
        if (rt < *res) {
          BDG_CUDA_TRY(plan_, cudaMemcpyAsync(phi_, trial_, sizeof(double2) * n3_, cudaMemcpyDeviceToDevice, s_));
          *res = rt;
          for (int j = 0; j < 3; ++j) mu[j] = mt[j];
        } else {
          flow_left = 50;
        }
      }
      if (!std::isfinite(*res)) return fail(plan_, BDG_ERR_NAN, "ground state iteration produced NaN");
    }
    *iters = it;
    return BDG_OK;
  }

  bdg_status download(double* phi) {
    std::vector<double2> h(n3_);
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(h.data(), phi_, sizeof(double2) * n3_, cudaMemcpyDeviceToHost, s_));
    BDG_CUDA_TRY(plan_, cudaStreamSynchronize(s_));
    for (long long e = 0; e < n3_; ++e) phi[e] = h[e].x;
    return BDG_OK;
  }

 private:
  bdg_status alloc(void* pp, size_t bytes) {
    void** p = (void**)pp;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return fail(plan_, BDG_ERR_NOMEM, "ground state: device allocation failed");
    }
    bufs_.push_back(*p);
    return BDG_OK;
  }

  bdg_status dots(const DotSet& d, long long len, double* out) {
    const unsigned nb = nblk(len);
    if ((size_t)nb * 8 > DPART) return fail(plan_, BDG_ERR_INVALID, "ground state: reduction grid too large");
    k_gs_dots<<<nb, 256, 0, s_>>>(d, len, dpart_);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    hpart_.resize((size_t)nb * d.count);
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(hpart_.data(), dpart_, sizeof(double) * hpart_.size(), cudaMemcpyDeviceToHost, s_));
    BDG_CUDA_TRY(plan_, cudaStreamSynchronize(s_));
    for (int q = 0; q < d.count; ++q) {
      double t = 0.0;
      for (unsigned b = 0; b < nb; ++b) t += hpart_[(size_t)q * nb + b];
      out[q] = t;
    }
    return BDG_OK;
  }
  double2* comp(double2* v, int j) { return v + (long long)j * np_; }

  // P_SM: sum_j sigma_j^2 N_j = 1, sigma_1^2 N_1 - sigma_-1^2 N_-1 = M,
  // sigma_1 sigma_-1 = sigma_0^2, N_j = h^d |phi_j|^2
  bdg_status project(double2* phi) {
    DotSet d{};
    for (int j = 0; j < 3; ++j) {
      d.a[j] = comp(phi, j);
      d.b[j] = comp(phi, j);
    }
    d.count = 3;
    double N[3];
    bdg_status st = dots(d, np_, N);
    if (st) return st;
    for (int j = 0; j < 3; ++j) N[j] *= cell_;
    const double N1 = N[0], N0 = N[1], Nm = N[2], M = M_;
    const double sden = N0 + std::sqrt(M * M * N0 * N0 + 4.0 * (1.0 - M * M) * N1 * Nm);
    if (!(sden > 0)) return fail(plan_, BDG_ERR_INVALID, "ground state: spinor has no admissible component");
    const double s = (1.0 - M * M) / sden;
    double sig[3] = {0.0, std::sqrt(s), 0.0};
    if (N1 > 0) sig[0] = std::sqrt(std::max(1.0 + M - s * N0, 0.0) / (2.0 * N1));
    if (Nm > 0) sig[2] = std::sqrt(std::max(1.0 - M - s * N0, 0.0) / (2.0 * Nm));
    if (N1 == 0 && Nm == 0) sig[1] = 1.0 / std::sqrt(N0);
    k_gs_scale3<<<nblk(n3_), 256, 0, s_>>>(phi, np_, sig[0], sig[1], sig[2]);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    return BDG_OK;
  }

  // internal plan table <- phi; H phi into hphi_ (mu = 0)
  bdg_status hphi(const double2* phi) {
    k_gs_table<<<nblk(np_), 256, 0, s_>>>(phi, V_, np_, plan_->phiv64, plan_->phiv32);
    BDG_CUDA_TRY(plan_, cudaMemsetAsync(x6_, 0, sizeof(double2) * n3_, s_));
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(x6_ + n3_, phi, sizeof(double2) * n3_, cudaMemcpyDeviceToDevice, s_));
    const double zero[3] = {0.0, 0.0, 0.0};
    bdg_status st = apply_internal(plan_, BDG_FG, BDG_C128, x6_, y6_, 1, s_, zero);
    if (st) return st;
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(hphi_, y6_ + n3_, sizeof(double2) * n3_, cudaMemcpyDeviceToDevice, s_));
    return BDG_OK;
  }

  // max |H Phi - mu Phi| with mu by eq. chem-formula (vanishing components
  // filled from mu_1 + mu_-1 = 2 mu_0)
  bdg_status residual(double2* phi, double* res, double mu[3]) {
    bdg_status st = hphi(phi);
    if (st) return st;
    DotSet d{};
    for (int j = 0; j < 3; ++j) {
      d.a[j] = comp(phi, j);
      d.b[j] = comp(hphi_, j);
      d.a[3 + j] = comp(phi, j);
      d.b[3 + j] = comp(phi, j);
    }
    d.count = 6;
    double v[6];
    if ((st = dots(d, np_, v))) return st;
    bool z[3];
    const double tiny = 1e-20 * (v[3] + v[4] + v[5]);   // vanishing components, relative to |Phi|^2
    for (int j = 0; j < 3; ++j) {
      z[j] = v[3 + j] < tiny;
      mu[j] = z[j] ? NAN : v[j] / v[3 + j];
    }
    if (z[1] && !z[0] && !z[2]) mu[1] = 0.5 * (mu[0] + mu[2]);
    else if (z[0] && z[2] && !z[1]) mu[0] = mu[2] = mu[1];
    else if (z[0] && !z[2] && !z[1]) mu[0] = 2 * mu[1] - mu[2];
    else if (z[2] && !z[0] && !z[1]) mu[2] = 2 * mu[1] - mu[0];
    BDG_CUDA_TRY(plan_, cudaMemsetAsync(dred_, 0, sizeof(double), s_));
    k_gs_maxres<<<nblk(n3_), 256, 0, s_>>>(hphi_, phi, np_, mu[0], mu[1], mu[2], dred_);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(res, dred_, sizeof(double), cudaMemcpyDeviceToHost, s_));
    BDG_CUDA_TRY(plan_, cudaStreamSynchronize(s_));
    return BDG_OK;
  }

  bdg_status stab(const double2* phi, double* alpha) {
    BDG_CUDA_TRY(plan_, cudaMemsetAsync(dred_, 0, sizeof(double), s_));
    k_gs_stab<<<nblk(np_), 256, 0, s_>>>(phi, V_, np_, k_.beta_n + std::fabs(k_.beta_s), dred_);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(alpha, dred_, sizeof(double), cudaMemcpyDeviceToHost, s_));
    BDG_CUDA_TRY(plan_, cudaStreamSynchronize(s_));
    *alpha += std::fabs(k_.p) + std::fabs(k_.q);
    return BDG_OK;
  }

  // y = (c - 1/2 Lap)^-1 x on 3 planes
  bdg_status kinetic_inverse(const double2* x, double2* y, double c) {
    KdArgs<double> g;
    g.grid = &plan_->grid;
    g.x = x;
    g.y = y;
    g.nplanes = 3;
    for (int a = 0; a < 3; ++a) g.tw[a] = plan_->tw64[a];
    g.shift = c;
    g.scale = 0.5;
    g.stream = s_;
    BDG_CUDA_TRY(plan_, kdiag_launch<double>(g));
    return BDG_OK;
  }

  bdg_status flow_step(double c) {
    k_gs_flow_rhs<<<nblk(np_), 256, 0, s_>>>(phi_, V_, np_, k_, c, trial_);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    bdg_status st = kinetic_inverse(trial_, phi_, c);
    if (st) return st;
    return project(phi_);
  }

  // P v = v - sum_i z_i <z_i, v>  (weighted inner product; z_i weighted-orthonormal)
  bdg_status tangent(double2* v) {
    if (nz_ == 0) return BDG_OK;
    DotSet d{};
    for (int i = 0; i < nz_; ++i) {
      d.a[i] = z_[i];
      d.b[i] = v;
    }
    d.count = nz_;
    double c[2];
    bdg_status st = dots(d, n3_, c);
    if (st) return st;
    for (int i = 0; i < nz_; ++i) {
      k_gs_axpby<<<nblk(n3_), 256, 0, s_>>>(n3_, -c[i] * cell_, z_[i], 1.0, v);
      BDG_CUDA_TRY(plan_, cudaGetLastError());
    }
    return BDG_OK;
  }

  bdg_status hplus(const double2* v, double2* out, const double mu[3]) {
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(x6_, v, sizeof(double2) * n3_, cudaMemcpyDeviceToDevice, s_));
    BDG_CUDA_TRY(plan_, cudaMemsetAsync(x6_ + n3_, 0, sizeof(double2) * n3_, s_));
    bdg_status st = apply_internal(plan_, BDG_FG, BDG_C128, x6_, y6_, 1, s_, mu);
    if (st) return st;
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(out, y6_, sizeof(double2) * n3_, cudaMemcpyDeviceToDevice, s_));
    return BDG_OK;
  }

  double dot1(const double2* a, const double2* b, bdg_status* st) {
    DotSet d{};
    d.a[0] = a;
    d.b[0] = b;
    d.count = 1;
    double v = 0.0;
    *st = dots(d, n3_, &v);
    return v;
  }

  // Multipliers m3 = mu + lambda S_z of the least-squares fit H Phi ~
  // (mu + lambda S_z) Phi at phi_ and the weighted-orthonormal basis z_ of
  // span{Phi, S_z Phi} (the normal directions of S_M); hphi_ = H Phi.
  bdg_status tangent_setup(double m3[3]) {
    bdg_status st = hphi(phi_);
    if (st) return st;
    // multipliers: least squares of H Phi ~ (mu + lambda S_z) Phi
    k_gs_sz<<<nblk(n3_), 256, 0, s_>>>(phi_, np_, z_[1]);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    DotSet d{};
    d.a[0] = phi_; d.b[0] = phi_;
    d.a[1] = phi_; d.b[1] = z_[1];
    d.a[2] = z_[1]; d.b[2] = z_[1];
    d.a[3] = phi_; d.b[3] = hphi_;
    d.a[4] = z_[1]; d.b[4] = hphi_;
    d.count = 5;
    double g[5];
    if ((st = dots(d, n3_, g))) return st;
    double mu, lam;
    const double det = g[0] * g[2] - g[1] * g[1];
    if (g[2] < 1e-300 || !(std::fabs(det) > 1e-30 * g[0] * g[2])) {
      mu = g[3] / g[0];
      lam = 0.0;
    } else {
      mu = (g[3] * g[2] - g[1] * g[4]) / det;
      lam = (g[0] * g[4] - g[1] * g[3]) / det;
    }
    m3[0] = mu + lam;
    m3[1] = mu;
    m3[2] = mu - lam;
    // weighted-orthonormal basis of span{Phi, S_z Phi}
    nz_ = 0;
    {
      const double nphi = std::sqrt(cell_ * g[0]);
      BDG_CUDA_TRY(plan_, cudaMemcpyAsync(z_[0], phi_, sizeof(double2) * n3_, cudaMemcpyDeviceToDevice, s_));
      k_gs_axpby<<<nblk(n3_), 256, 0, s_>>>(n3_, 0.0, z_[0], 1.0 / nphi, z_[0]);
      nz_ = 1;
      // z2 = S_z Phi - z1 <z1, S_z Phi>
      const double c12 = cell_ * g[1] / nphi;
      k_gs_axpby<<<nblk(n3_), 256, 0, s_>>>(n3_, -c12, z_[0], 1.0, z_[1]);
      BDG_CUDA_TRY(plan_, cudaGetLastError());
      const double n2 = std::sqrt(std::max(cell_ * dot1(z_[1], z_[1], &st), 0.0));
      if (st) return st;
      if (n2 > 1e-10 * nphi) {
        k_gs_axpby<<<nblk(n3_), 256, 0, s_>>>(n3_, 0.0, z_[1], 1.0 / n2, z_[1]);
        BDG_CUDA_TRY(plan_, cudaGetLastError());
        nz_ = 2;
      }
    }
    return BDG_OK;
  }

  // Stability of a converged stationary state: the curvature
  // <d, P H_+ P d> / <d, d> of the energy on S_M along the population-transfer
  // directions (k_gs_transfer).  *unstable is set, and the unit direction of
  // most negative curvature left in cp_, when a curvature is below
  // -1e-9 (1 + max |mu|).
  bdg_status stability(bool* unstable) {
    *unstable = false;
    double m3[3];
    bdg_status st = tangent_setup(m3);
    if (st) return st;
    const double mmax = std::max(std::fabs(m3[0]), std::max(std::fabs(m3[1]), std::fabs(m3[2])));
    const double nphi = dot1(phi_, phi_, &st);
    if (st) return st;
    double best = -1e-9 * (1.0 + mmax);
    for (int kind = 0; kind < 3; ++kind) {
      k_gs_transfer<<<nblk(np_), 256, 0, s_>>>(phi_, np_, kind, cz_);
      BDG_CUDA_TRY(plan_, cudaGetLastError());
      if ((st = tangent(cz_))) return st;
      const double dd = dot1(cz_, cz_, &st);
      if (st) return st;
      if (!(dd > 1e-16 * nphi)) continue;
      if ((st = hplus(cz_, cap_, m3)) || (st = tangent(cap_))) return st;
      const double kappa = dot1(cz_, cap_, &st) / dd;
      if (st) return st;
      if (kappa < best) {
        best = kappa;
        *unstable = true;
        k_gs_axpby<<<nblk(n3_), 256, 0, s_>>>(n3_, 1.0 / std::sqrt(dd), cz_, 0.0, cp_);
        BDG_CUDA_TRY(plan_, cudaGetLastError());
      }
    }
    return BDG_OK;
  }

  // one inexact Newton step from phi_ into trial_; *products = H_+ products
  bdg_status newton_step(double c, int* products) {
    const double eta = 1e-2;
    const int maxcg = 500;
    *products = 0;
    double m3[3];
    bdg_status st = tangent_setup(m3);
    if (st) return st;
    // b = -P r, r = H Phi - (mu + lambda S_z) Phi;  CG on P H_+ P x = b
    k_gs_resid<<<nblk(n3_), 256, 0, s_>>>(hphi_, phi_, np_, m3[0], m3[1], m3[2], cr_);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    if ((st = tangent(cr_))) return st;
    k_gs_axpby<<<nblk(n3_), 256, 0, s_>>>(n3_, 0.0, cr_, -1.0, cr_);  // res = b
    BDG_CUDA_TRY(plan_, cudaMemsetAsync(cx_, 0, sizeof(double2) * n3_, s_));
    const double b0 = std::sqrt(dot1(cr_, cr_, &st));
    if (st) return st;
    // z = P T^-1 P res  (res already tangent)
    if ((st = kinetic_inverse(cr_, cz_, c)) || (st = tangent(cz_))) return st;
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(cp_, cz_, sizeof(double2) * n3_, cudaMemcpyDeviceToDevice, s_));
    double rz = dot1(cr_, cz_, &st);
    if (st) return st;
    for (int kcg = 0; kcg < maxcg && b0 > 0; ++kcg) {
      // Ap = P H_+ P p  (p is tangent)
      if ((st = hplus(cp_, cap_, m3)) || (st = tangent(cap_))) return st;
      ++*products;
      const double pap = dot1(cp_, cap_, &st);
      if (st) return st;
      if (!(pap > 0)) break;
      const double a = rz / pap;
      k_gs_axpby<<<nblk(n3_), 256, 0, s_>>>(n3_, a, cp_, 1.0, cx_);
      k_gs_axpby<<<nblk(n3_), 256, 0, s_>>>(n3_, -a, cap_, 1.0, cr_);
      BDG_CUDA_TRY(plan_, cudaGetLastError());
      const double rn = std::sqrt(dot1(cr_, cr_, &st));
      if (st) return st;
      if (rn <= eta * b0) break;
      if ((st = kinetic_inverse(cr_, cz_, c)) || (st = tangent(cz_))) return st;
      const double rz_new = dot1(cr_, cz_, &st);
      if (st) return st;
      k_gs_axpby<<<nblk(n3_), 256, 0, s_>>>(n3_, 1.0, cz_, rz_new / rz, cp_);
      BDG_CUDA_TRY(plan_, cudaGetLastError());
      rz = rz_new;
    }
    // trial = P_SM(Phi + x)
    BDG_CUDA_TRY(plan_, cudaMemcpyAsync(trial_, phi_, sizeof(double2) * n3_, cudaMemcpyDeviceToDevice, s_));
    k_gs_axpby<<<nblk(n3_), 256, 0, s_>>>(n3_, 1.0, cx_, 1.0, trial_);
    BDG_CUDA_TRY(plan_, cudaGetLastError());
    return project(trial_);
  }

  bdg_plan_t plan_;
  double M_;
  cudaStream_t s_;
  long long np_ = 0, n3_ = 0;
  double cell_ = 1.0;
  GsCoef k_{};
  std::vector<void*> bufs_;
  double* V_ = nullptr;
  double2 *phi_ = nullptr, *trial_ = nullptr, *hphi_ = nullptr, *x6_ = nullptr, *y6_ = nullptr;
  double2* z_[2] = {nullptr, nullptr};
  int nz_ = 0;
  double2 *cx_ = nullptr, *cr_ = nullptr, *cz_ = nullptr, *cp_ = nullptr, *cap_ = nullptr;
  double* dred_ = nullptr;
  static constexpr size_t DPART = 8 * 152 * 8;   // 8 sums x the largest reduction grid
  double* dpart_ = nullptr;
  std::vector<double> hpart_;
};

}  // namespace
}  // namespace bdg

using namespace bdg;

bdg_status bdg_ground_state(const bdg_params* p, double M, const double* V, const double* phi0, double tol,
                            int maxit, double* phi, double* mu, double* resid, int* iters, void* stream) {
  if (!p || !V || !phi0 || !phi || !mu) return fail(nullptr, BDG_ERR_INVALID, "NULL argument");
  if (!(std::fabs(M) < 1.0)) return fail(nullptr, BDG_ERR_INVALID, "magnetization must satisfy |M| < 1");
  if (!(tol > 0) || maxit < 0) return fail(nullptr, BDG_ERR_INVALID, "tol must be > 0 and maxit >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  // the internal plan: mu = 0 so that the FG product of (0, Phi) is H Phi
  bdg_params q = *p;
  q.mu[0] = q.mu[1] = q.mu[2] = 0.0;
  q.prec = BDG_FP64;
  bdg_plan_t plan = nullptr;
  bdg_status st = bdg_plan_create(&plan, &q, V, phi0, stream);
  if (st) return st;
  double res = INFINITY, m[3] = {0, 0, 0};
  int it = 0;
  {
    GroundState gs(plan, M, s);
    st = gs.init(V, phi0);
    if (!st) st = gs.run(tol, maxit, &res, m, &it);
    if (!st) st = gs.download(phi);
  }
  std::string err = st ? plan->err : std::string();
  bdg_plan_destroy(plan);
  if (st) return fail(nullptr, st, err);
  for (int j = 0; j < 3; ++j) mu[j] = m[j];
  if (resid) *resid = res;
  if (iters) *iters = it;
  if (!(res <= tol)) return fail(nullptr, BDG_ERR_NOT_CONVERGED, "ground state did not reach tol within maxit");
  return BDG_OK;
}
