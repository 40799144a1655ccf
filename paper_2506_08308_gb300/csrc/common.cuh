// Shared device/host definitions of the BdG library: complex helpers,
// error plumbing and the plan object.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "../../include/bdg.h"

namespace bdg {

// ---------------------------------------------------------------------------
// complex arithmetic on float2 / double2
// ---------------------------------------------------------------------------
// Q: four reals per grid node, (phi_1, phi_0, phi_-1, V).
struct __align__(32) dquad { double x, y, z, w; };
template <typename R> struct CT;
template <> struct CT<float> { typedef float2 T; typedef float4 Q; };
template <> struct CT<double> { typedef double2 T; typedef dquad Q; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

#define BDG_COMPLEX_OPS(T, R)                                                            \
  __host__ __device__ __forceinline__ T operator+(T a, T b) { return mk(a.x + b.x, a.y + b.y); } \
  __host__ __device__ __forceinline__ T operator-(T a, T b) { return mk(a.x - b.x, a.y - b.y); } \
  __host__ __device__ __forceinline__ T operator*(T a, R s) { return mk(a.x * s, a.y * s); }     \
  __host__ __device__ __forceinline__ T cmul(T a, T b) {                                 \
    return mk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));                      \
  }                                                                                      \
  __host__ __device__ __forceinline__ T cmulc(T a, T b) { /* a * conj(b) */              \
    return mk(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));                      \
  }                                                                                      \
  __host__ __device__ __forceinline__ T cfma(T a, R s, T acc) {                          \
    return mk(fma(a.x, s, acc.x), fma(a.y, s, acc.y));                                   \
  }
BDG_COMPLEX_OPS(float2, float)
BDG_COMPLEX_OPS(double2, double)
#undef BDG_COMPLEX_OPS

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_thread_error(const std::string& msg);
const char* thread_error();

// Raise the dynamic shared-memory limit of kernel `func` on the current
// device to at least `bytes`.  The limit only grows: host threads that
// launch the same kernel with different sizes (concurrent solves) never
// lower it under one another.  Thread-safe.
cudaError_t allow_dynamic_smem(const void* func, size_t bytes);

#define BDG_CUDA_TRY(plan, call)                                                       \
  do {                                                                                 \
    cudaError_t e__ = (call);                                                          \
    if (e__ != cudaSuccess) {                                                          \
      bdg::fail((plan), BDG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
      return BDG_ERR_CUDA;                                                             \
    }                                                                                  \
  } while (0)

// ---------------------------------------------------------------------------
// grid description shared by all kernels
// ---------------------------------------------------------------------------
struct Grid {
  int dim;
  int n[3];        // points per axis (axis 0 slowest)
  long long npts;  // product
  double len[3];   // hi - lo per axis
  double lo[3];
};

// Scalars of the pointwise coupling (eqs. def_A, def_B with the Zeeman
// diagonal) in the arithmetic precision R.
template <typename R> struct Coupling {
  R beta_n, beta_s;
  R d1, d0, dm;  // q - p - mu_1, -mu_0, q + p - mu_-1
};

// Scratch arenas are owned by the plan and reused across calls.
struct Buffer {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace bdg

struct bdg_plan_s {
  bdg_params prm;
  bdg::Grid grid;
  double mu[3];
  int device;
  // device data
  bdg::dquad* phiv64 = nullptr;   // (phi_1, phi_0, phi_-1, V) per node, FP64
  float4* phiv32 = nullptr;    // the same rounded to FP32
  double2* tw64[3] = {nullptr, nullptr, nullptr};  // W_N^r = exp(-2 pi i r / N), r < N
  float2* tw32[3] = {nullptr, nullptr, nullptr};
  // deflation bases (orthonormal columns, real, [ncol][3][N_p] FP64 and FP32)
  int nzf = 0, nzg = 0;
  double* zf64 = nullptr;
  double* zg64 = nullptr;
  float* zf32 = nullptr;
  float* zg32 = nullptr;
  bdg::Buffer scratch[9];   // indexed by ScratchSlot
  std::string err;
  bdg_solve_stats stats;
  void* last_stream = nullptr;
};

namespace bdg {
bdg_status fail(bdg_plan_t plan, bdg_status st, const std::string& msg);
bdg_status ensure(bdg_plan_t plan, int slot, size_t bytes);
// BDG_OK when the calling thread's current device is the plan's device; else
// BDG_ERR_INVALID (the plan's data would be read from another GPU).
bdg_status check_device(bdg_plan_t plan);
}  // namespace bdg
