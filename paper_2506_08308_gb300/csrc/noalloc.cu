// Chemical potentials of a plan's ground state without any device allocation.
//
// Who needs this: callers that must not allocate device memory at the time
// of the call -- for instance code running under a caching allocator or a
// memory budget that forbids implicit cudaMalloc, or a real-time loop where
// an allocation's implicit synchronization is not acceptable.  Everything
// else in the library draws its scratch from buffers it allocates on first
// use; this entry point instead works in one file-scope device array of
// fixed size, so it never calls cudaMalloc, cudaFree or an allocating
// library routine.
//
// The array (NOALLOC_BYTES, about 3.1 MB) lives in every GPU that loads the
// library until the process exits.  It holds the product's input and output
// vectors (one 6-field FP64 vector each) and the Gram partial sums, which
// bounds the grid to NOALLOC_MAX_NPTS points.  Every byte the computation
// reads from the array is written first within the same call, so nothing
// has to start at zero; the array keeps the last call's contents.  All calls
// share the one array: calls that overlap on the GPU (several streams,
// several host threads, several plans) race on it and must be serialized by
// the caller.
//
// The device address of the array is looked up once per device (with that
// device current) by cudaGetSymbolAddress on the first call made on that
// device; the first call on a device should therefore come before any
// stream capture on it.  The address is kept for the life of the process:
// after a cudaDeviceReset of that device it would be stale, so a process that
// resets a device must not call this entry point on it again.
#include <cmath>
#include <mutex>
#include <string>

#include "blas.cuh"
#include "plan.cuh"

namespace bdg {
namespace {

constexpr long long NOALLOC_MAX_NPTS = 16384;                                   // e.g. 128^2 or 16x32^2
constexpr size_t NOALLOC_VEC_BYTES = sizeof(double2) * 6 * NOALLOC_MAX_NPTS;   // one 6-field FP64 vector
constexpr size_t NOALLOC_AUX_OFFSET = 2 * NOALLOC_VEC_BYTES;                   // Gram partials and results
constexpr size_t NOALLOC_AUX_BYTES = 64 * 1024;
constexpr size_t NOALLOC_BYTES = NOALLOC_AUX_OFFSET + NOALLOC_AUX_BYTES;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_noalloc_mutex;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_noalloc_scratch on the current device (the host-side
// symbol is only a stand-in and must never reach a kernel).
bdg_status scratch_address(bdg_plan_t plan, unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(plan, BDG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(plan, BDG_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(plan, BDG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = (unsigned char*)g_noalloc_addr[dev];
  return BDG_OK;
}

// x = [0, 0, 0, phi_1, phi_0, phi_-1] (FG vector, imaginary parts zero)
__global__ void k_noalloc_fg_phi(const dquad* __restrict__ pv, long long np, double2* __restrict__ x) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
       i += (long long)gridDim.x * blockDim.x) {
    const dquad v = pv[i];
    x[i] = make_double2(0.0, 0.0);
    x[np + i] = make_double2(0.0, 0.0);
    x[2 * np + i] = make_double2(0.0, 0.0);
    x[3 * np + i] = make_double2(v.x, 0.0);
    x[4 * np + i] = make_double2(v.y, 0.0);
    x[5 * np + i] = make_double2(v.z, 0.0);
  }
}

}  // namespace
}  // namespace bdg

using namespace bdg;

extern "C" bdg_status bdg_chemical_potentials_noalloc(bdg_plan_t plan, double* mu, void* stream) {
  if (!plan) return fail(nullptr, BDG_ERR_INVALID, "plan is NULL");
  if (!mu) return fail(plan, BDG_ERR_INVALID, "mu must be a host pointer to 3 doubles");
  const long long np = plan->grid.npts;
  if (np > NOALLOC_MAX_NPTS)
    return fail(plan, BDG_ERR_UNSUPPORTED,
                "grid has " + std::to_string(np) + " points; the allocation-free path holds at most " +
                    std::to_string(NOALLOC_MAX_NPTS));
  if (bdg_status sd = check_device(plan)) return sd;
  unsigned char* base = nullptr;
  bdg_status st = scratch_address(plan, &base);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  double2* x = (double2*)base;
  double2* y = (double2*)(base + NOALLOC_VEC_BYTES);
  double* aux = (double*)(base + NOALLOC_AUX_OFFSET);
  double* G = aux;                          // 4 doubles: the 2 x 2 real Gram of one complex column pair
  void* ws = aux + 8;
  const size_t ws_bytes = NOALLOC_AUX_BYTES - 8 * sizeof(double);
  if (gram_workspace_bytes(1, 1, np) > ws_bytes) return fail(plan, BDG_ERR_UNSUPPORTED, "Gram workspace too small");
  // With mu = 0 the FG product of (0, Phi) is (H_- Phi) = H Phi (eq. NLEP).
  long long nb = (np + 255) / 256;
  if (nb > 1216) nb = 1216;
  k_noalloc_fg_phi<<<(unsigned)nb, 256, 0, s>>>(plan->phiv64, np, x);
  BDG_CUDA_TRY(plan, cudaGetLastError());
  const double zero[3] = {0.0, 0.0, 0.0};
  if ((st = apply_internal(plan, BDG_FG, BDG_C128, x, y, 1, s, zero))) return st;
  // mu_j = <phi_j, (H Phi)_j> / |phi_j|^2 (eq. chem-formula)
  double num[3], den[3];
  for (int j = 0; j < 3; ++j) {
    for (int which = 0; which < 2; ++which) {
      PairBlock<double> A{x + (3 + j) * np, np, np, 1};
      PairBlock<double> B{(which ? x : y) + (3 + j) * np, np, np, 1};
      BDG_CUDA_TRY(plan, gram_pairs<double>(A, B, G, ws, ws_bytes, s));
      double h[4];
      BDG_CUDA_TRY(plan, cudaMemcpyAsync(h, G, sizeof(h), cudaMemcpyDeviceToHost, s));
      BDG_CUDA_TRY(plan, cudaStreamSynchronize(s));
      (which ? den : num)[j] = h[0] + h[3];
    }
  }
  // components with |phi_j|^2 < 1e-20 |Phi|^2 take their mu from mu_1 + mu_-1 = 2 mu_0
  bool z[3];
  const double tiny = 1e-20 * (den[0] + den[1] + den[2]);
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
