// Arithmetic-peak probes of the CUDA-core units the contraction kernels run on.
//
// The contraction kernels of this library are bound either by HBM or by the
// FP32 (FP64) FMA pipe of the CUDA cores.  Their rooflines therefore need the
// FMA throughput the chip really sustains, not a data-sheet figure (the paper
// quotes its K20c peaks from the data sheet, Sec. 5).  Each probe kernel runs
// independent chains of one FMA form per thread, with operands in registers and
// nothing else in the loop, on every SM; the caller times one launch with CUDA
// events and divides the flop count returned here by the time.
#include "kron_device.cuh"
#include "kron_internal.h"
#include "kron_pair.cuh"

namespace kron {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;   // independent chains per thread: hides the FMA latency

// A value that no chain reaches from the seeds below; storing only when it is
// reached keeps the chains alive without writing memory.
__device__ unsigned g_kron_peak_sink;

__global__ void __launch_bounds__(kPeakThreads) peak_ffma2_kernel(int iters, float a, float b) {
    f2 acc[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) acc[c] = f2_pack(threadIdx.x + c, c - 0.5f * threadIdx.x);
    const f2 m = f2_pack(a, a), s = f2_pack(b, b);
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) acc[c] = ffma2(acc[c], m, s);
    }
    float r = 0.0f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) r += f2_lo(acc[c]) + f2_hi(acc[c]);
    if (__float_as_uint(r) == 0x7fbadbadu) g_kron_peak_sink = 1u;
}

__global__ void __launch_bounds__(kPeakThreads) peak_ffma_kernel(int iters, float a, float b) {
    float acc[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) acc[c] = threadIdx.x + c;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) acc[c] = __fmaf_rn(acc[c], a, b);
    }
    float r = 0.0f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) r += acc[c];
    if (__float_as_uint(r) == 0x7fbadbadu) g_kron_peak_sink = 1u;
}

__global__ void __launch_bounds__(kPeakThreads) peak_dfma_kernel(int iters, double a, double b) {
    double acc[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) acc[c] = threadIdx.x + c;
#pragma unroll 1
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int c = 0; c < kPeakChains; ++c) acc[c] = __fma_rn(acc[c], a, b);
    }
    double r = 0.0;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) r += acc[c];
    if (__double_as_longlong(r) == 0x7ff4badbadbadbadll) g_kron_peak_sink = 1u;
}

}  // namespace kron

using namespace kron;

extern "C" KRON_API kron_status kron_peak_probe(kron_stream_t stream, int unit, int iters, double* flops) {
    if (unit < 0 || unit > 2 || iters < 1 || iters > (1 << 24) || !flops) return KRON_ERR_INVALID_VALUE;
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    const void* fn = unit == 0 ? (const void*)peak_ffma2_kernel
                   : unit == 1 ? (const void*)peak_ffma_kernel : (const void*)peak_dfma_kernel;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPeakThreads, 0) != cudaSuccess || per_sm < 1)
        return KRON_ERR_CUDA;
    const int grid = per_sm * dev.sms;
    // a = 1 - 2^-20 and b = 2^-30 keep every chain finite and away from the sink value
    const float af = 0.99999905f, bf = 9.3132257e-10f;
    cudaStream_t s = (cudaStream_t)stream;
    if (unit == 0)
        peak_ffma2_kernel<<<grid, kPeakThreads, 0, s>>>(iters, af, bf);
    else if (unit == 1)
        peak_ffma_kernel<<<grid, kPeakThreads, 0, s>>>(iters, af, bf);
    else
        peak_dfma_kernel<<<grid, kPeakThreads, 0, s>>>(iters, (double)af, (double)bf);
    if (cudaGetLastError() != cudaSuccess) return KRON_ERR_CUDA;
    const double fma_per_thread = 4.0 * kPeakChains * (unit == 0 ? 2.0 : 1.0) * (double)iters;
    *flops = 2.0 * fma_per_thread * (double)grid * kPeakThreads;
    return KRON_OK;
}
