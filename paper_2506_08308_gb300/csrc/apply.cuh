// Launch interface of the BdG product kernels.
#pragma once

#include "common.cuh"

namespace bdg {

template <typename R>
struct ApplyArgs {
  const Grid* grid;
  const typename CT<R>::T* x;
  typename CT<R>::T* y;
  int nvec;
  int mode;                         // BDG_UV or BDG_FG
  const typename CT<R>::Q* phiv;    // (phi_1, phi_0, phi_-1, V) per node
  const typename CT<R>::T* tw[3];   // per-axis twiddles W_N^r
  R kscale[3];                      // 1/2 (2 pi / len_a)^2 / n_a per axis
  Coupling<R> cp;
};

template <typename R>
cudaError_t apply_launch(const ApplyArgs<R>& g, cudaStream_t s);

}  // namespace bdg
