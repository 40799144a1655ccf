// Perturbed densities of excitation modes (Section 4.2, the "2D Case"
// example): with one mode l kept in the wave-function ansatz eq. waveAssump,
//
//   n_j^l(x, t) = | phi_j(x) + eps ( u_j(x) e^{-i w t} + conj(v_j(x)) e^{i w t} ) |^2,
//
// j = 1, 0, -1 (the global phase e^{-i mu_j t} of the ansatz drops out of the
// modulus).  With u = ur + i ui, v = vr + i vi and (C, S) = eps (cos wt, sin wt)
// the bracket is
//
//   phi_j + [(ur + vr) C + (ui + vi) S] + i [(ui - vi) C + (vr - ur) S],
//
// so each grid point forms four sums per component once and then spends two
// multiply-adds per part and time.  One pass reads each mode's amplitudes
// once and writes every requested time: the kernel streams 6 complex values
// in and 3 nt reals out per point and mode.
#include <cmath>
#include <string>
#include <vector>

#include "plan.cuh"

namespace bdg {
namespace {

__device__ __forceinline__ void load_phi(const dquad* __restrict__ p, long long i, double* f) {
  const dquad q = p[i];
  f[0] = q.x;
  f[1] = q.y;
  f[2] = q.z;
}
__device__ __forceinline__ void load_phi(const float4* __restrict__ p, long long i, float* f) {
  const float4 q = p[i];
  f[0] = q.x;
  f[1] = q.y;
  f[2] = q.z;
}

// Phase tables of up to INLINE_PHASES entries travel as a kernel argument
// (no copy, no host wait); longer ones go through device scratch.
constexpr int INLINE_PHASES = 128;
template <typename C> struct InlinePhases { C v[INLINE_PHASES]; };

// blockIdx.y = mode l; a grid-stride loop over the points.  Entry l * nt + t
// of the phase table (ph, or inl when ph is NULL) holds
// (eps cos w_l t, eps sin w_l t), formed in FP64 and rounded to R (an FP32
// kernel that converted FP64 phases per point would keep the slow FP64 pipe
// busy); out is [nmode][nt][3][np].
template <typename R>
__global__ void __launch_bounds__(256) k_perturbed_density(long long np, int nt,
                                                           const typename CT<R>::T* __restrict__ uv,
                                                           const typename CT<R>::Q* __restrict__ phiv,
                                                           const typename CT<R>::T* __restrict__ ph,
                                                           const __grid_constant__ InlinePhases<typename CT<R>::T> inl,
                                                           R* __restrict__ out) {
  typedef typename CT<R>::T C;
  const long long l = blockIdx.y;
  const C* x = uv + l * 6 * np;
  const C* pl = ph ? ph + l * nt : nullptr;
  const int i0 = (int)l * nt;
  R* o = out + l * nt * 3 * np;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
       i += (long long)gridDim.x * blockDim.x) {
    R f[3], a[3], b[3], d[3], e[3];
    load_phi(phiv, i, f);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const C u = x[j * np + i], v = x[(3 + j) * np + i];
      a[j] = u.x + v.x;
      b[j] = u.y + v.y;
      d[j] = u.y - v.y;
      e[j] = v.x - u.x;
    }
    for (int t = 0; t < nt; ++t) {
      const C cs = pl ? pl[t] : inl.v[i0 + t];
      const R c = cs.x, s = cs.y;
      R* ot = o + (long long)t * 3 * np + i;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const R re = fma(a[j], c, b[j] * s);
        const R im = fma(d[j], c, e[j] * s);
        const R y = f[j] + re;
        ot[j * np] = fma(y, y, im * im);
      }
    }
  }
}

}  // namespace
}  // namespace bdg

using namespace bdg;

extern "C" bdg_status bdg_perturbed_density(bdg_plan_t plan, int dtype, const void* UV, int nmode,
                                            const double* omega, const double* times, int nt, double eps,
                                            void* out, void* stream) {
  if (!plan) return fail(nullptr, BDG_ERR_INVALID, "plan is NULL");
  if (dtype != BDG_C128 && dtype != BDG_C64) return fail(plan, BDG_ERR_INVALID, "dtype must be BDG_C128 or BDG_C64");
  if (nmode < 0 || nt < 0) return fail(plan, BDG_ERR_INVALID, "nmode and nt must be >= 0");
  if (nmode > 65535) return fail(plan, BDG_ERR_UNSUPPORTED, "at most 65535 modes per call");
  if (!std::isfinite(eps)) return fail(plan, BDG_ERR_INVALID, "eps is not finite");
  if (nmode == 0 || nt == 0) return BDG_OK;
  if (!UV || !out) return fail(plan, BDG_ERR_INVALID, "UV and out must be device pointers");
  if (!omega || !times) return fail(plan, BDG_ERR_INVALID, "omega and times must be host arrays");
  const long long np = plan->grid.npts;
  const size_t esz = dtype == BDG_C128 ? 16 : 8, rsz = esz / 2;
  const size_t in_bytes = esz * 6 * (size_t)np * (size_t)nmode;
  const size_t out_bytes = rsz * 3 * (size_t)np * (size_t)nt * (size_t)nmode;
  const char* ib = (const char*)UV;
  const char* ob = (const char*)out;
  if (ib < ob + out_bytes && ob < ib + in_bytes) return fail(plan, BDG_ERR_INVALID, "UV and out overlap");
  if ((uintptr_t)UV % esz || (uintptr_t)out % rsz)
    return fail(plan, BDG_ERR_INVALID, "UV or out not aligned to its element size");
  if (bdg_status sd = check_device(plan)) return sd;
  // phase table (eps cos w t, eps sin w t) in FP64 on the host
  std::vector<double2> tab((size_t)nmode * nt);
  for (int l = 0; l < nmode; ++l) {
    if (!std::isfinite(omega[l])) return fail(plan, BDG_ERR_INVALID, "omega[" + std::to_string(l) + "] is not finite");
    for (int t = 0; t < nt; ++t) {
      if (!std::isfinite(times[t])) return fail(plan, BDG_ERR_INVALID, "times[" + std::to_string(t) + "] is not finite");
      const double th = omega[l] * times[t];
      tab[(size_t)l * nt + t] = make_double2(eps * std::cos(th), eps * std::sin(th));
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const bool inline_tab = tab.size() <= (size_t)INLINE_PHASES;
  void* ph = nullptr;
  if (!inline_tab) {
    bdg_status st = ensure(plan, SLOT_PHASE, sizeof(double2) * tab.size());
    if (st) return st;
    ph = plan->scratch[SLOT_PHASE].ptr;
  }
  long long gx = (np + 255) / 256;
  const long long cap = 4 * 152 * 8 / nmode + 1;   // about four waves of 8 resident 256-thread CTAs per SM
  if (gx > cap) gx = cap;
  const dim3 grid((unsigned)gx, (unsigned)nmode);
  // pageable sources below: each copy returns once its table is staged, so
  // the host vectors may go out of scope
  if (dtype == BDG_C128) {
    InlinePhases<double2> inl = {};
    if (inline_tab) {
      for (size_t i = 0; i < tab.size(); ++i) inl.v[i] = tab[i];
    } else {
      BDG_CUDA_TRY(plan, cudaMemcpyAsync(ph, tab.data(), sizeof(double2) * tab.size(), cudaMemcpyHostToDevice, s));
    }
    k_perturbed_density<double><<<grid, 256, 0, s>>>(np, nt, (const double2*)UV, plan->phiv64, (const double2*)ph,
                                                     inl, (double*)out);
  } else {
    std::vector<float2> tab32(tab.size());
    for (size_t i = 0; i < tab.size(); ++i) tab32[i] = make_float2((float)tab[i].x, (float)tab[i].y);
    InlinePhases<float2> inl = {};
    if (inline_tab) {
      for (size_t i = 0; i < tab32.size(); ++i) inl.v[i] = tab32[i];
    } else {
      BDG_CUDA_TRY(plan, cudaMemcpyAsync(ph, tab32.data(), sizeof(float2) * tab32.size(), cudaMemcpyHostToDevice, s));
    }
    k_perturbed_density<float><<<grid, 256, 0, s>>>(np, nt, (const float2*)UV, plan->phiv32, (const float2*)ph,
                                                    inl, (float*)out);
  }
  BDG_CUDA_TRY(plan, cudaGetLastError());
  plan->last_stream = stream;
  return BDG_OK;
}
