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
// Staged kernel: operand bytes per tile (at least one instance) and tiles in flight
// per CTA; measured at m = 256, k = 16: two 16 KB instances per tile (one row pair
// per thread), three tiles (0.98 of the copy bandwidth; one instance per tile,
// half the threads idle: 0.85; deeper rings cost resident CTAs).
constexpr size_t kGaTileBytes = 32768;
constexpr int kGaRing = 3;

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

// Contiguous batches (lda = m, lda2 = m k, ldc = m, ldc2 = m n, A 16-byte aligned,
// m k a whole number of 16-byte units): the row-pair products of the kernel
// above, with the operands staged in shared memory.  Tiles of P instances
// arrive by one bulk copy each (TMA) in an NB-deep ring; a warp's lanes then
// read 64 consecutive rows of one column per access (conflict-free) and store
// their row pairs of C straight from registers (256 contiguous bytes per warp
// and column).  Plain loads of the same rows streamed at 0.91-0.93 of the copy
// bandwidth, the staged tiles at 0.98.
template <int NN>
struct __align__(8) GemmATArgs {
    f2 bd[kGaMaxK * NN];   // (B[l, j], B[l, j]) at l * NN + j, zero beyond k x n
    const void* A;
    void* C;
    int64_t batch;
    int m, n, k;
    int P, nstage;
    int beta_zero, alpha_one;
    float alpha, beta;
    unsigned* err;
};

template <typename S, int NN>
__global__ void __launch_bounds__(kGaThreads) gemm_a_tma_kernel(const __grid_constant__ GemmATArgs<NN> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    unsigned char* xbase = smem + 128;
    const int P = a.P, NB = a.nstage, m2 = a.m / 2;
    const int64_t inst = (int64_t)a.m * a.k;   // elements of one A^p
    const size_t tile_bytes = ((size_t)P * inst * sizeof(S) + 127) / 128 * 128;
    const int64_t ntiles = (a.batch + P - 1) / P;
    const int64_t grid = gridDim.x;
    const S* A = static_cast<const S*>(a.A);
    S* C = static_cast<S*>(a.C);
    uint64_t pol = 0;
    auto issue = [&](int s, int64_t tile) {
        const int64_t i0 = tile * P;
        const unsigned bytes = (unsigned)(min((int64_t)P, a.batch - i0) * inst * (int64_t)sizeof(S));
        mbar_arrive_expect_tx(&bars[s], bytes);
        bulk_g2s(xbase + s * tile_bytes, A + i0 * inst, bytes, &bars[s], pol);
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < NB; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
        pol = l2_evict_first_policy();
        for (int s = 0; s < NB; ++s)
            if (blockIdx.x + s * grid < ntiles) issue(s, blockIdx.x + s * grid);
    }
    __syncthreads();
    const f2 al = f2_pack(a.alpha, a.alpha), be = f2_pack(a.beta, a.beta);
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
        const int s = it % NB;
        const bool ok = mbar_wait_bounded(&bars[s], (unsigned)(it / NB) & 1u, a.err);
        if (__syncthreads_or(!ok)) {
            // wait (bounded) for the copies that may still be in flight, then give up
            if (threadIdx.x == 0)
                for (int j = it; j < it + NB; ++j)
                    if (blockIdx.x + (int64_t)j * grid < ntiles)
                        mbar_wait_bounded(&bars[j % NB], (unsigned)(j / NB) & 1u, a.err);
            return;
        }
        const S* xt = reinterpret_cast<const S*>(xbase + s * tile_bytes);
        const int64_t i0 = tile * P;
        const int cnt = (int)min((int64_t)P, a.batch - i0);
        for (int f = threadIdx.x; f < cnt * m2; f += kGaThreads) {
            const int q = f / m2, i2 = f - q * m2;
            const S* ar = xt + q * inst + 2 * i2;
            f2 x[kGaMaxK];
#pragma unroll
            for (int l = 0; l < kGaMaxK; ++l) x[l] = l < a.k ? load_pair<S>(ar + a.m * l) : 0ull;
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
            S* cr = C + (i0 + q) * (int64_t)a.m * a.n + 2 * i2;
#pragma unroll
            for (int j = 0; j < NN; ++j) {
                if (j < a.n) {
                    f2 v = a.alpha_one ? c[j] : fmul2(c[j], al);
                    S* dst = cr + (int64_t)a.m * j;
                    if (!a.beta_zero) v = ffma2(be, load_pair<S>(dst), v);
                    if constexpr (sizeof(S) == 4)
                        *reinterpret_cast<f2*>(dst) = v;
                    else
                        *reinterpret_cast<unsigned*>(dst) = pack16<S>(v);
                }
            }
        }
        __syncthreads();   // the tile's operands are read: its buffer can be refilled
        if (threadIdx.x == 0) {
            const int64_t next = tile + (int64_t)NB * grid;
            if (next < ntiles) {
                fence_proxy_async_smem();
                issue(s, next);
            }
        }
    }
}

template <typename S, int NN>
kron_status launch_ga_tma(const GemmADesc& g, cudaStream_t st) {
    GemmATArgs<NN> a;
    memset(&a, 0, sizeof(a));
    for (int l = 0; l < g.k; ++l)
        for (int j = 0; j < g.n; ++j) {
            const float v = (float)g.b[l * kGaMaxK + j];
            a.bd[l * NN + j] = ((f2)__float_as_uint_host(v) << 32) | (f2)__float_as_uint_host(v);
        }
    a.A = g.A;
    a.C = g.C;
    a.batch = g.batch;
    a.m = g.m;
    a.n = g.n;
    a.k = g.k;
    a.alpha = (float)g.alpha;
    a.beta = (float)g.beta;
    a.alpha_one = g.alpha == 1.0;
    a.beta_zero = g.beta == 0.0;
    a.err = device_error_word();
    if (!a.err) return KRON_ERR_CUDA;
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    const size_t inst_bytes = (size_t)g.m * g.k * sizeof(S);
    int P = (int)std::max<size_t>(1, kGaTileBytes / inst_bytes);
    int nb = kGaRing;
    auto smem_of = [&](int p, int n_b) { return 128 + (size_t)n_b * (((size_t)p * inst_bytes + 127) / 128 * 128); };
    while (P > 1 && smem_of(P, nb) > dev.smem_per_block_optin) --P;
    while (nb > 1 && smem_of(P, nb) > dev.smem_per_block_optin) --nb;
    const size_t smem = smem_of(P, nb);
    if (smem > dev.smem_per_block_optin || (size_t)P * inst_bytes >= (1u << 20)) return KRON_ERR_NOT_SUPPORTED;
    a.P = P;
    a.nstage = nb;
    auto kern = gemm_a_tma_kernel<S, NN>;
    if (!ensure_smem_optin((const void*)kern, smem)) return KRON_ERR_CUDA;
    const int64_t ntiles = (g.batch + P - 1) / P;
    int64_t grid = g.grid;
    if (grid <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGaThreads, smem) != cudaSuccess)
            return KRON_ERR_CUDA;
        grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
    }
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, ntiles));
    kern<<<(unsigned)grid, kGaThreads, smem, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

// Layouts the staged kernel takes: the row-pair layouts, packed (minimal leading
// dimensions), A 16-byte aligned and each A^p a whole number of 16-byte units.
bool ga_tma_ok(const GemmADesc& g) {
    const size_t es = elem_size(g.io);
    return g.lda == g.m && g.lda2 == (int64_t)g.m * g.k && g.ldc == g.m && g.ldc2 == (int64_t)g.m * g.n &&
           (uintptr_t)g.A % 16 == 0 && ((size_t)g.m * g.k * es) % 16 == 0;
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
    if (ga_pair_ok(g) && ga_tma_ok(g)) {
        kron_status r = KRON_ERR_NOT_SUPPORTED;
        switch (g.io) {
            case KRON_R32F: r = launch_ga_tma<float, NN>(g, st); break;
            case KRON_R16BF: r = launch_ga_tma<__nv_bfloat16, NN>(g, st); break;
            case KRON_R16F: r = launch_ga_tma<__half, NN>(g, st); break;
            default: break;
        }
        if (r != KRON_ERR_NOT_SUPPORTED) return r;
    }
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
