// Inner preconditioned conjugate gradients for the search directions of the
// subspace iteration.
//
// For the unconverged Ritz pairs the directions are approximate solutions of
//   H_+ d_f = r_f   on the complement of Z_g = null(H_+),
//   H_- d_g = r_g   on the complement of Z_f = null(H_-),
// the exact preconditioner (H_+^-1, H_-^-1) of the trace-minimization
// principle of the linear-response problem (eq. lrep-d): with it the search
// space grows like block inverse iteration on H_- H_+.  A fixed number of PCG
// steps from zero, preconditioned by the kinetic operator
// T_sigma = IDFT (1/2 |mu|^2 + sigma)^-1 DFT and the deflation projector,
// approximate it.  The paper gives no preconditioner; the converged pairs do
// not depend on it.
//
// The block holds P complex columns of 6 N_p values (FG form): every complex
// column carries two real columns (real and imaginary parts) and every real
// column two independent systems (its f- and g-halves), so there are four CG
// recurrences per complex column, run in lockstep.  All scalars stay on the
// device; every reduction sums its partials in a fixed order, so the result
// does not depend on scheduling.  The arithmetic precision RI of the inner
// iteration is independent of the outer one: FP32 in the mixed solver (its
// products cost about a twentieth of FP64 ones on this part), FP64 in the
// plain FP64 solver.
#pragma once

#include <vector>

#include "common.cuh"

namespace bdg {

template <typename RI>
class InnerPCG {
 public:
  typedef typename CT<RI>::T T;
  // Device buffers for up to max_pairs complex columns; owned by the caller's
  // allocator through alloc(ptr, bytes) (returns nonzero on failure).
  template <typename Alloc>
  bdg_status init(bdg_plan_t plan, int max_pairs, Alloc&& alloc) {
    plan_ = plan;
    np_ = plan->grid.npts;
    vlen_ = 6 * np_;
    max_pairs_ = max_pairs;
    const size_t vb = sizeof(T) * (size_t)vlen_ * max_pairs;
    void* p = nullptr;
    for (int i = 0; i < 5; ++i) {
      if (alloc(&p, vb)) return fail(plan, BDG_ERR_NOMEM, "inner solver allocation failed");
      buf_[i] = (T*)p;
    }
    nchunk_ = chunks_for(vlen_);
    const size_t sb = sizeof(double) * ((size_t)max_pairs * nchunk_ * 8 * 2 + (size_t)max_pairs * 8 + 64);
    if (alloc(&p, sb)) return fail(plan, BDG_ERR_NOMEM, "inner solver allocation failed");
    part_ = (double*)p;
    zpart_ = part_ + (size_t)max_pairs * nchunk_ * 8;
    rz_ = zpart_ + (size_t)max_pairs * nchunk_ * 8;
    zf_ = (const T*)(sizeof(RI) == 8 ? (const void*)plan->zf64 : (const void*)plan->zf32);
    zg_ = (const T*)(sizeof(RI) == 8 ? (const void*)plan->zg64 : (const void*)plan->zg32);
    return BDG_OK;
  }

  // D (outer precision R, pairs complex columns, column stride 6 N_p) =
  // steps PCG steps on the systems above with right-hand sides Rin (same
  // layout; Rin may equal D).  sigma is the shift of T_sigma.
  //
  // The steps issue about ten launches each and take no host decision, so
  // on large grids a call repeated with the same buffers, block width,
  // steps and shift replays a CUDA graph captured on its second occurrence
  // (the first runs directly and sets every kernel's launch attributes).
  // A capture that fails falls back to direct launches.
  template <typename R>
  bdg_status run(const typename CT<R>::T* Rin, typename CT<R>::T* D, int pairs, int steps, double sigma,
                 cudaStream_t s);

  ~InnerPCG() { release_graphs(); }

  static int chunks_for(long long vlen) {
    long long c = (vlen + 8191) / 8192;   // about 8192 values per CTA and column
    if (c > 128) c = 128;
    return (int)(c < 1 ? 1 : c);
  }

 private:
  template <typename R>
  bdg_status run_direct(const typename CT<R>::T* Rin, typename CT<R>::T* D, int pairs, int steps, double sigma,
                        cudaStream_t s);
  void release_graphs();
  struct Graph {
    const void* rin;
    const void* d;
    int pairs, steps, rbytes;
    double sigma;
    cudaGraphExec_t exec;  // null until captured
    bool direct;           // capture failed: launch directly
  };
  std::vector<Graph> graphs_;
  cudaStream_t cap_ = nullptr;   // private stream the graphs are captured on
  bool use_graphs_ = true;

  bdg_status deflate_swapped(T* v, int pairs, cudaStream_t s);
  bdg_status dots(const T* a, const T* b, int pairs, cudaStream_t s);
  bdg_status precondition(const T* x, T* y, int pairs, double sigma, cudaStream_t s);

  bdg_plan_t plan_ = nullptr;
  long long np_ = 0, vlen_ = 0;
  int max_pairs_ = 0, nchunk_ = 1;
  T* buf_[5] = {};   // x, r, z, p, q
  double* part_ = nullptr;
  double* zpart_ = nullptr;
  double* rz_ = nullptr;   // [2][pairs][4]
  const T* zf_ = nullptr;
  const T* zg_ = nullptr;
};

}  // namespace bdg
