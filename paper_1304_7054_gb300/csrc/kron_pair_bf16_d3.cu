// Instantiates the packed-pair FP32 kernels for __nv_bfloat16 storage, 3-D operands.
#include "kron_pair.cuh"

namespace kron {
kron_status launch_pair_bf16_d3(const KronDesc& d, cudaStream_t s) { return launch_pair_d<__nv_bfloat16, 3>(d, s); }
}  // namespace kron
