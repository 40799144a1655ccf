// FP64 instantiation of the BdG product kernels.
#include "apply_impl.cuh"

namespace bdg {
template cudaError_t apply_launch<double>(const ApplyArgs<double>&, cudaStream_t);
}  // namespace bdg
