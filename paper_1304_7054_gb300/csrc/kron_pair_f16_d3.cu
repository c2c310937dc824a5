// Instantiates the packed-pair FP32 kernels for __half storage, 3-D operands.
#include "kron_pair.cuh"

namespace kron {
kron_status launch_pair_f16_d3(const KronDesc& d, cudaStream_t s) { return launch_pair_d<__half, 3>(d, s); }
}  // namespace kron
