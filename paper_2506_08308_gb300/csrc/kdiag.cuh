// Launch interface of the k-space diagonal operator (preconditioner and the
// implicit kinetic step of the ground-state flow).
#pragma once

#include "common.cuh"

namespace bdg {

template <typename R>
struct KdArgs {
  const Grid* grid;
  const typename CT<R>::T* x;       // nplanes planes of N_p complex values
  typename CT<R>::T* y;             // may equal x
  long long nplanes;
  const typename CT<R>::T* tw[3];   // per-axis twiddles
  double shift, scale;              // y = IDFT [1 / (shift + scale |mu|^2)] DFT x
  cudaStream_t stream;
};

template <typename R>
cudaError_t kdiag_launch(const KdArgs<R>& g);

}  // namespace bdg
