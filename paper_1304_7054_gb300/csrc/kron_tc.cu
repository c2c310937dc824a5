// Entry of the split tensor path (KRON_COMPUTE_32F_BF16X3): the layouts it takes,
// then the 2-D or 3-D launchers (kron_tc2.cu, kron_tc3.cu; kernels in kron_tc.cuh).
#include "kron_internal.h"

namespace kron {

kron_status launch_tc2_any(const KronDesc& d, cudaStream_t st);
kron_status launch_tc3_any(const KronDesc& d, cudaStream_t st);

kron_status launch_tc(const KronDesc& d, cudaStream_t st) {
    // Contiguous square batches only (minimal leading dimensions, 16-byte aligned X).
    if (!d.contiguous || d.ye[0] != d.N || d.ye[1] != d.N || d.ye[2] != (d.D == 3 ? d.N : 1) ||
        (d.D == 2 ? (d.ldy != d.N || d.ldyp != (int64_t)d.N * d.N)
                  : (d.ldy != d.N || d.ldy2 != d.N * d.N || d.ldyp != (int64_t)d.N * d.N * d.N)))
        return KRON_ERR_NOT_SUPPORTED;
    if (d.io != KRON_R32F && d.io != KRON_R16BF && d.io != KRON_R16F) return KRON_ERR_NOT_SUPPORTED;
    return d.D == 2 ? launch_tc2_any(d, st) : launch_tc3_any(d, st);
}

}  // namespace kron
