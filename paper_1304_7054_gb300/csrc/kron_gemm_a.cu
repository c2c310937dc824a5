// Batched GEMM with a varying first factor and a shared second one (TGEMM_A,
// Sec. 3):  C^p = alpha op(A^p) op(B) + beta C^p.  The 1-D product (TKRON1,
// Sec. 3) runs on the same kernel as the case m = 1: x^p is the one row of
// A^p and op(B) = op(A)^T.
//
// One thread computes row i of one C^p.  It loads row i of op(A^p) (k <= 16
// elements; with op = 'N' consecutive threads read consecutive rows, so every
// load instruction is coalesced), forms the n <= 16 outputs with op(B) in the
// kernel parameter bank -- pairs of output columns per packed fma.rn.f32x2,
// the coefficient pair (B[l, j], B[l, j+1]) a constant operand, as in the
// pair kernels -- and stores the outputs column by column (coalesced across
// threads again).  FP64 uses plain double FMAs.  The grid is persistent and
// walks rows p * m + i with a stride kept as (instances, rows) so that no
// division is needed inside the loop.  With op = 'N' and even strides a thread
// takes a pair of rows instead (see gemm_a_pair_kernel).
#include "kron_pair.cuh"

namespace kron {

namespace {

inline unsigned __float_as_uint_host(float v) {
    unsigned b;
    memcpy(&b, &v, sizeof(b));
    return b;
}

constexpr int kGaThreads = 256;
constexpr int kGaMaxK = 16;

template <typename T, int NN>
struct __align__(8) GemmAArgs {
    T b[kGaMaxK * NN];   // op(B), kGaMaxK x NN row-major, zero beyond k x n
    const void* A;
    void* C;
    int64_t lda2, ldc2, batch;
    int64_t step_p;      // grid stride = step_p instances + step_i rows
    int step_i;
    int lda, ldc, m, n, k, transa;
    int beta_zero, alpha_one;
    T alpha, beta;
};

// Storage type S, FP32 arithmetic in packed column pairs.
template <typename S, int NN>
__global__ void __launch_bounds__(kGaThreads) gemm_a_kernel(const __grid_constant__ GemmAArgs<float, NN> a) {
    const int64_t r0 = (int64_t)blockIdx.x * kGaThreads + threadIdx.x;
    int64_t p = r0 / a.m;
    int i = (int)(r0 - p * a.m);
    const f2* bp = reinterpret_cast<const f2*>(a.b);
    const S* A = static_cast<const S*>(a.A);
    S* C = static_cast<S*>(a.C);
    const int64_t astep = a.transa ? 1 : a.lda;
    while (p < a.batch) {
        const S* ar = A + p * a.lda2 + (a.transa ? (int64_t)a.lda * i : (int64_t)i);
        float x[kGaMaxK];
#pragma unroll
        for (int l = 0; l < kGaMaxK; ++l) x[l] = l < a.k ? load_cvt<float, S>(ar[astep * l]) : 0.f;
        f2 c[NN / 2];
        const f2 x0 = f2_pack(x[0], x[0]);
#pragma unroll
        for (int r = 0; r < NN / 2; ++r) c[r] = fmul2(bp[r], x0);
#pragma unroll
        for (int l = 1; l < kGaMaxK; ++l) {
            if (l < a.k) {
                const f2 xl = f2_pack(x[l], x[l]);
#pragma unroll
                for (int r = 0; r < NN / 2; ++r) c[r] = ffma2(bp[l * (NN / 2) + r], xl, c[r]);
            }
        }
        S* cr = C + p * a.ldc2 + i;
#pragma unroll
        for (int j = 0; j < NN; ++j) {
            if (j < a.n) {
                float v = (j & 1) ? f2_hi(c[j / 2]) : f2_lo(c[j / 2]);
                if (!a.alpha_one) v *= a.alpha;
                S* dst = cr + (int64_t)a.ldc * j;
                if (!a.beta_zero) v = fmaf(a.beta, load_cvt<float, S>(*dst), v);
                *dst = store_cvt<S, float>(v);
            }
        }
        i += a.step_i;
        p += a.step_p;
        if (i >= a.m) {
            i -= a.m;
            ++p;
        }
    }
}

// Pairs of rows (op = 'N', even m and strides): rows (i, i+1) of op(A^p) are
// adjacent in memory, so one thread loads both as a pair, multiplies them by
// the duplicated coefficient (B[l, j], B[l, j]) -- a constant operand -- and
// stores the two results of column j as a pair.  Half the address arithmetic
// of the one-row kernel and no operand duplication.
template <int NN>
struct __align__(8) GemmA2Args {
    f2 bd[kGaMaxK * NN];   // (B[l, j], B[l, j]) at l * NN + j, zero beyond k x n
    const void* A;
    void* C;
    int64_t lda2, ldc2, batch;
    int64_t step_p;        // grid stride = step_p instances + step_i row pairs
    int step_i;
    int lda, ldc, m2, n, k;
    int beta_zero, alpha_one;
    float alpha, beta;
};

template <typename S, int NN>
__global__ void __launch_bounds__(kGaThreads) gemm_a_pair_kernel(const __grid_constant__ GemmA2Args<NN> a) {
    const int64_t r0 = (int64_t)blockIdx.x * kGaThreads + threadIdx.x;
    int64_t p = r0 / a.m2;
    int i2 = (int)(r0 - p * a.m2);
    const S* A = static_cast<const S*>(a.A);
    S* C = static_cast<S*>(a.C);
    while (p < a.batch) {
        const S* ar = A + p * a.lda2 + 2 * i2;
        f2 x[kGaMaxK];
#pragma unroll
        for (int l = 0; l < kGaMaxK; ++l) x[l] = l < a.k ? load_pair<S>(ar + (int64_t)a.lda * l) : 0ull;
        f2 c[NN];
#pragma unroll
        for (int j = 0; j < NN; ++j) c[j] = fmul2(a.bd[j], x[0]);
#pragma unroll
        for (int l = 1; l < kGaMaxK; ++l) {
            if (l < a.k) {
#pragma unroll
                for (int j = 0; j < NN; ++j) c[j] = ffma2(a.bd[l * NN + j], x[l], c[j]);
            }
        }
        S* cr = C + p * a.ldc2 + 2 * i2;
        const f2 al = f2_pack(a.alpha, a.alpha), be = f2_pack(a.beta, a.beta);
#pragma unroll
        for (int j = 0; j < NN; ++j) {
            if (j < a.n) {
                f2 v = a.alpha_one ? c[j] : fmul2(c[j], al);
                S* dst = cr + (int64_t)a.ldc * j;
                if (!a.beta_zero) v = ffma2(be, load_pair<S>(dst), v);
                if constexpr (sizeof(S) == 4)
                    *reinterpret_cast<f2*>(dst) = v;
                else
                    *reinterpret_cast<unsigned*>(dst) = pack16<S>(v);
            }
        }
        i2 += a.step_i;
        p += a.step_p;
        if (i2 >= a.m2) {
            i2 -= a.m2;
            ++p;
        }
    }
}

template <typename S, int NN>
kron_status launch_ga_pair(const GemmADesc& g, cudaStream_t st) {
    GemmA2Args<NN> a;
    memset(&a, 0, sizeof(a));
    for (int l = 0; l < g.k; ++l)
        for (int j = 0; j < g.n; ++j) {
            const float v = (float)g.b[l * kGaMaxK + j];
            a.bd[l * NN + j] = ((f2)__float_as_uint_host(v) << 32) | (f2)__float_as_uint_host(v);
        }
    a.A = g.A;
    a.C = g.C;
    a.lda2 = g.lda2;
    a.ldc2 = g.ldc2;
    a.batch = g.batch;
    a.lda = g.lda;
    a.ldc = g.ldc;
    a.m2 = g.m / 2;
    a.n = g.n;
    a.k = g.k;
    a.alpha = (float)g.alpha;
    a.beta = (float)g.beta;
    a.alpha_one = g.alpha == 1.0;
    a.beta_zero = g.beta == 0.0;
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    auto kern = gemm_a_pair_kernel<S, NN>;
    const int64_t units = g.batch * a.m2;
    int64_t grid = g.grid;
    if (grid <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGaThreads, 0) != cudaSuccess)
            return KRON_ERR_CUDA;
        grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
    }
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, (units + kGaThreads - 1) / kGaThreads));
    const int64_t step = grid * kGaThreads;
    a.step_p = step / a.m2;
    a.step_i = (int)(step % a.m2);
    kern<<<(unsigned)grid, kGaThreads, 0, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

// Layouts the row-pair kernel takes: op = 'N', every row pair 2 * sizeof(S)-aligned.
bool ga_pair_ok(const GemmADesc& g) {
    if (g.io == KRON_R64F || g.transa || g.m % 2) return false;
    const size_t es = elem_size(g.io);
    return g.lda % 2 == 0 && g.lda2 % 2 == 0 && g.ldc % 2 == 0 && g.ldc2 % 2 == 0 &&
           (uintptr_t)g.A % (2 * es) == 0 && (uintptr_t)g.C % (2 * es) == 0;
}

template <int NN>
__global__ void __launch_bounds__(kGaThreads) gemm_a_kernel_f64(const __grid_constant__ GemmAArgs<double, NN> a) {
    const int64_t r0 = (int64_t)blockIdx.x * kGaThreads + threadIdx.x;
    int64_t p = r0 / a.m;
    int i = (int)(r0 - p * a.m);
    const double* A = static_cast<const double*>(a.A);
    double* C = static_cast<double*>(a.C);
    const int64_t astep = a.transa ? 1 : a.lda;
    while (p < a.batch) {
        const double* ar = A + p * a.lda2 + (a.transa ? (int64_t)a.lda * i : (int64_t)i);
        double x[kGaMaxK];
#pragma unroll
        for (int l = 0; l < kGaMaxK; ++l) x[l] = l < a.k ? ar[astep * l] : 0.0;
        double c[NN];
#pragma unroll
        for (int j = 0; j < NN; ++j) c[j] = a.b[j] * x[0];
#pragma unroll
        for (int l = 1; l < kGaMaxK; ++l) {
            if (l < a.k) {
#pragma unroll
                for (int j = 0; j < NN; ++j) c[j] = fma(a.b[l * NN + j], x[l], c[j]);
            }
        }
        double* cr = C + p * a.ldc2 + i;
#pragma unroll
        for (int j = 0; j < NN; ++j) {
            if (j < a.n) {
                double v = a.alpha_one ? c[j] : a.alpha * c[j];
                double* dst = cr + (int64_t)a.ldc * j;
                if (!a.beta_zero) v = fma(a.beta, *dst, v);
                *dst = v;
            }
        }
        i += a.step_i;
        p += a.step_p;
        if (i >= a.m) {
            i -= a.m;
            ++p;
        }
    }
}

template <typename T, int NN, typename Kern>
kron_status launch_ga(const GemmADesc& g, Kern kern, cudaStream_t st) {
    GemmAArgs<T, NN> a;
    memset(&a, 0, sizeof(a));
    for (int l = 0; l < g.k; ++l)
        for (int j = 0; j < g.n; ++j) a.b[l * NN + j] = (T)g.b[l * kGaMaxK + j];
    a.A = g.A;
    a.C = g.C;
    a.lda2 = g.lda2;
    a.ldc2 = g.ldc2;
    a.batch = g.batch;
    a.lda = g.lda;
    a.ldc = g.ldc;
    a.m = g.m;
    a.n = g.n;
    a.k = g.k;
    a.transa = g.transa;
    a.alpha = (T)g.alpha;
    a.beta = (T)g.beta;
    a.alpha_one = g.alpha == 1.0;
    a.beta_zero = g.beta == 0.0;
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    const int64_t rows = g.batch * g.m;
    int64_t grid = g.grid;
    if (grid <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGaThreads, 0) != cudaSuccess)
            return KRON_ERR_CUDA;
        grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
    }
    grid = std::min<int64_t>(grid, (rows + kGaThreads - 1) / kGaThreads);
    grid = std::max<int64_t>(grid, 1);
    const int64_t step = grid * kGaThreads;
    a.step_p = step / g.m;
    a.step_i = (int)(step % g.m);
    kern<<<(unsigned)grid, kGaThreads, 0, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

template <int NN>
kron_status launch_ga_nn(const GemmADesc& g, cudaStream_t st) {
    if (ga_pair_ok(g)) {
        switch (g.io) {
            case KRON_R32F: return launch_ga_pair<float, NN>(g, st);
            case KRON_R16BF: return launch_ga_pair<__nv_bfloat16, NN>(g, st);
            case KRON_R16F: return launch_ga_pair<__half, NN>(g, st);
            default: break;
        }
    }
    switch (g.io) {
        case KRON_R32F: return launch_ga<float, NN>(g, gemm_a_kernel<float, NN>, st);
        case KRON_R16BF: return launch_ga<float, NN>(g, gemm_a_kernel<__nv_bfloat16, NN>, st);
        case KRON_R16F: return launch_ga<float, NN>(g, gemm_a_kernel<__half, NN>, st);
        case KRON_R64F: return launch_ga<double, NN>(g, gemm_a_kernel_f64<NN>, st);
    }
    return KRON_ERR_INVALID_VALUE;
}

}  // namespace

kron_status launch_gemm_a(const GemmADesc& g, cudaStream_t st) {
    if (g.n < 1 || g.n > kGaMaxK || g.k < 1 || g.k > kGaMaxK || g.m < 1) return KRON_ERR_INVALID_VALUE;
    switch ((g.n + 1) / 2 * 2) {
        case 2: return launch_ga_nn<2>(g, st);
        case 4: return launch_ga_nn<4>(g, st);
        case 6: return launch_ga_nn<6>(g, st);
        case 8: return launch_ga_nn<8>(g, st);
        case 10: return launch_ga_nn<10>(g, st);
        case 12: return launch_ga_nn<12>(g, st);
        case 14: return launch_ga_nn<14>(g, st);
        case 16: return launch_ga_nn<16>(g, st);
    }
    return KRON_ERR_INVALID_VALUE;
}

}  // namespace kron
