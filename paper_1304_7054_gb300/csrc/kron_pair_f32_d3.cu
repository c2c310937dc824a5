// Instantiates the packed-pair FP32 kernels for float storage, 3-D operands.
#include "kron_pair.cuh"

namespace kron {
kron_status launch_pair_f32_d3(const KronDesc& d, cudaStream_t s) { return launch_pair_d<float, 3>(d, s); }
}  // namespace kron
