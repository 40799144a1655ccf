// FP32 instantiation of the k-space diagonal operator.
#include "kdiag_impl.cuh"

namespace bdg {
template cudaError_t kdiag_launch<float>(const KdArgs<float>&);
}  // namespace bdg
