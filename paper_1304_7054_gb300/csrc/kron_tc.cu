// Tensor-core split-precision kernels (placeholder until implemented).
#include "kron_internal.h"

namespace kron {
kron_status launch_tc(const KronDesc&, cudaStream_t) { return KRON_ERR_NOT_SUPPORTED; }
}  // namespace kron
