// FP32 instantiation of the BdG product kernels.
#include "apply_impl.cuh"

namespace bdg {
template cudaError_t apply_launch<float>(const ApplyArgs<float>&, cudaStream_t);
}  // namespace bdg
