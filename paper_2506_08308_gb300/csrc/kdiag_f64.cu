// FP64 instantiation of the k-space diagonal operator.
#include "kdiag_impl.cuh"

namespace bdg {
template cudaError_t kdiag_launch<double>(const KdArgs<double>&);
}  // namespace bdg
