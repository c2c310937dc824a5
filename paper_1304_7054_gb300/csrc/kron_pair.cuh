// Packed-pair CUDA-core kernels: FP32 arithmetic, even N, contiguous batches.
//
// Same sum factorisation as the fiber kernels (paper Sec. 2.1, Algorithm 1's
// mode order with the intermediate kept on chip), but every FMA instruction is a
// packed two-lane `fma.rn.f32x2`, which halves the FMA issue slots per flop:
//
//  * "pair of fibers" stages: a thread owns two adjacent fibers (i, i+1) and
//    multiplies the pair (x_i[l], x_{i+1}[l]) -- one 64-bit shared load -- by the
//    duplicated coefficient (M[k,l], M[k,l]) held in the parameter bank;
//  * "pair of rows" last stage: a thread owns one mode-1 fiber and produces the
//    outputs (y[i], y[i+1]) from the natural coefficient pair (M[i,l], M[i+1,l])
//    times (x[l], x[l]); the output pairs are contiguous in Y, so the store is a
//    plain vector store.
//
//   2-D:  stage 1 (pairs of rows l, mode 2, component M2), stage 2 (mode 1, M1)
//   3-D:  stage A (pairs i, mode 3, M3), stage B (pairs i, mode 2, M2),
//         stage C (mode 1, M1)
#pragma once

#include <string.h>

#include "kron_device.cuh"
#include "kron_fiber.cuh"
#include "kron_internal.h"

namespace kron {

// Two adjacent storage elements as a float pair.
template <typename S> __device__ __forceinline__ f2 load_pair(const S* p);
template <> __device__ __forceinline__ f2 load_pair<float>(const float* p) {
    return *reinterpret_cast<const f2*>(p);
}
template <> __device__ __forceinline__ f2 load_pair<__nv_bfloat16>(const __nv_bfloat16* p) {
    const unsigned w = *reinterpret_cast<const unsigned*>(p);
    return f2_pack(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <> __device__ __forceinline__ f2 load_pair<__half>(const __half* p) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
    return f2_pack(v.x, v.y);
}


// y[k] = Md[k, :] . x for the two fibers packed in x (Md: duplicated coefficients).
template <int N>
__device__ __forceinline__ void contract_dup(const f2* __restrict__ Md, const f2 (&x)[N], f2 (&y)[N]) {
#pragma unroll
    for (int k = 0; k < N; ++k) y[k] = fmul2(Md[k], x[0]);
#pragma unroll
    for (int l = 1; l < N; ++l) {
#pragma unroll
        for (int k = 0; k < N; ++k) y[k] = ffma2(Md[k + N * l], x[l], y[k]);
    }
}

// (y[2r], y[2r+1]) = M[2r:2r+2, :] . x for one fiber (M column-major, as pairs).
template <int N>
__device__ __forceinline__ void contract_rows(const f2* __restrict__ Mp, const float (&x)[N], f2 (&y)[N / 2]) {
    const f2 x0 = f2_pack(x[0], x[0]);
#pragma unroll
    for (int r = 0; r < N / 2; ++r) y[r] = fmul2(Mp[r], x0);
#pragma unroll
    for (int l = 1; l < N; ++l) {
        const f2 xl = f2_pack(x[l], x[l]);
#pragma unroll
        for (int r = 0; r < N / 2; ++r) y[r] = ffma2(Mp[r + (N / 2) * l], xl, y[r]);
    }
}

// bar.red.or over the 128 threads of compute group g (named barrier 1 + g).  The
// barrier number is an immediate, so the kernel reserves five barriers, not all
// sixteen (a CTA that reserves every barrier limits how many CTAs an SM holds).
template <int ID>
__device__ __forceinline__ bool bar_or_128(bool v) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, 128, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((unsigned)v), "n"(ID)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ bool group_sync_or(bool v, int g) {
    switch (g) {
        case 0: return bar_or_128<1>(v);
        case 1: return bar_or_128<2>(v);
        case 2: return bar_or_128<3>(v);
        default: return bar_or_128<4>(v);
    }
}

template <int N, int D>
struct PairArgs {
    f2 da[N * N];                  // first stage component, duplicated (2-D: M2, 3-D: M3)
    f2 db[D == 3 ? N * N : 1];     // 3-D second stage component M2, duplicated
    float m1[N * N];               // last stage component M1, column-major (read as pairs)
    const void* X;
    void* Y;
    int64_t batch;
    int P;                         // instances per tile
    int nstage;                    // bulk-copy pipeline depth (>= 1)
    int beta_zero, alpha_one;
    float alpha, beta;
    unsigned* err;
    // Nonzero: the first operand wait of each CTA polls for at most this many
    // nanoseconds (failure-path test; read by the 2-D n = 16 FP32 kernel).
    unsigned long long first_wait_ns = 0;
};

template <int N, int D, int SB>
struct PairLayout {
    static_assert(N % 2 == 0, "pair kernels need an even N");
    static constexpr int NX = ipow(N, D);
    // 2-D operand tile: N = 16 instances are placed 272 floats apart (one bulk copy
    // each) so the two instances read by a half-warp use different banks.
    static constexpr bool XPAD = (D == 2 && N == 16);
    static constexpr int SX = XPAD ? 272 : NX;
    // W (2-D) / U (3-D): element (l, j, k, q) at l + SJ j + SK k + SQ q
    static constexpr int SJ = N + 2;
    static constexpr int SK = stride_mod32(SJ * (N - 1) + N, N);
    static constexpr int SQ = (D == 2) ? SK : SK * N;
    // T (3-D): element (i, j, k, q) at i + N j + ST k + STQ q.  With FP32 storage T
    // overwrites the operand tile in place (ST = N^2): every thread reads its two
    // fibers into registers before it writes the two output fibers at the same
    // addresses, and no other thread touches them.  That saves a buffer, so more
    // CTAs are resident; the tile is refilled after stage B instead of stage A.
    static constexpr bool TIN = (D == 3 && SB == 4);
    static constexpr int ST = TIN ? N * N : stride_mod32(N * N, N);
    static constexpr int STQ = ST * N;
    // 2-D: W double-buffered; 3-D: T in its own buffer unless it is in place
    static constexpr int EX1 = (D == 2) ? 2 * SQ : (TIN ? 0 : STQ);
    static constexpr int EX2 = (D == 2) ? 0 : SQ;
};

// Loads tile `tile` into `dst`; called by all 32 lanes of warp 0.
template <typename S, int N, int D>
__device__ __forceinline__ void pair_issue(const PairArgs<N, D>& a, void* dst, uint64_t* bar, int64_t tile,
                                           uint64_t pol) {
    using L = PairLayout<N, D, (int)sizeof(S)>;
    const int lane = threadIdx.x & 31;
    const int64_t inst0 = tile * a.P;
    const int cnt = (int)min((int64_t)a.P, a.batch - inst0);
    const S* src = static_cast<const S*>(a.X) + inst0 * L::NX;
    if constexpr (L::XPAD) {
        constexpr unsigned ib = L::NX * sizeof(S);
        if (lane == 0) mbar_arrive_expect_tx(bar, ib * (unsigned)cnt);
        __syncwarp();
        for (int q = lane; q < cnt; q += 32)
            bulk_g2s(static_cast<S*>(dst) + (size_t)q * L::SX, src + (size_t)q * L::NX, ib, bar, pol);
    } else {
        if (lane == 0) {
            const unsigned bytes = (unsigned)cnt * L::NX * (unsigned)sizeof(S);
            const unsigned b16 = bytes & ~15u;
            mbar_arrive_expect_tx(bar, b16);
            if (b16) bulk_g2s(dst, src, b16, bar, pol);
        }
    }
}

// Epilogue + store of one mode-1 fiber given as N/2 float pairs (contiguous in Y).
template <typename S, int N, int D>
__device__ __forceinline__ void pair_store(const PairArgs<N, D>& a, S* dst, f2 (&y)[N / 2]) {
    if (!a.alpha_one) {
        const f2 al = f2_pack(a.alpha, a.alpha);
#pragma unroll
        for (int r = 0; r < N / 2; ++r) y[r] = fmul2(y[r], al);
    }
    if (!a.beta_zero) {
        const f2 be = f2_pack(a.beta, a.beta);
#pragma unroll
        for (int r = 0; r < N / 2; ++r) y[r] = ffma2(be, load_pair<S>(dst + 2 * r), y[r]);
    }
    if constexpr (sizeof(S) == 4) {
        if constexpr (N % 4 == 0) {
#pragma unroll
            for (int c = 0; c < N / 4; ++c) {
                uint4 v = make_uint4((unsigned)y[2 * c], (unsigned)(y[2 * c] >> 32), (unsigned)y[2 * c + 1],
                                     (unsigned)(y[2 * c + 1] >> 32));
                __stcs(reinterpret_cast<uint4*>(dst) + c, v);
            }
        } else {
#pragma unroll
            for (int r = 0; r < N / 2; ++r)
                __stcs(reinterpret_cast<uint2*>(dst) + r, make_uint2((unsigned)y[r], (unsigned)(y[r] >> 32)));
        }
    } else {
        unsigned w[N / 2];
#pragma unroll
        for (int r = 0; r < N / 2; ++r) w[r] = pack16<S>(y[r]);
        if constexpr (N % 8 == 0) {
#pragma unroll
            for (int c = 0; c < N / 8; ++c)
                __stcs(reinterpret_cast<uint4*>(dst) + c, make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]));
        } else if constexpr (N % 4 == 0) {
#pragma unroll
            for (int c = 0; c < N / 4; ++c) __stcs(reinterpret_cast<uint2*>(dst) + c, make_uint2(w[2 * c], w[2 * c + 1]));
        } else {
#pragma unroll
            for (int r = 0; r < N / 2; ++r) __stcs(reinterpret_cast<unsigned*>(dst) + r, w[r]);
        }
    }
}

// N contiguous floats of an exchange buffer (8-byte aligned) into registers.
template <int N>
__device__ __forceinline__ void load_row(const float* src, float (&v)[N]) {
#pragma unroll
    for (int l = 0; l < N; l += 2) {
        const f2 p = *reinterpret_cast<const f2*>(src + l);
        v[l] = f2_lo(p);
        v[l + 1] = f2_hi(p);
    }
}

// Last contraction over F mode-1 fibers, two fibers per thread and iteration so
// that the shared loads of the second overlap the arithmetic of the first.
// fetch(f, x) loads fiber f into x and returns where its outputs go.
template <typename S, int N, int D, int NT, typename Fetch>
__device__ __forceinline__ void last_stage(const PairArgs<N, D>& a, int F, Fetch fetch) {
    const f2* m1p = reinterpret_cast<const f2*>(a.m1);
    for (int f = threadIdx.x; f < F; f += 2 * NT) {
        const bool two = f + NT < F;
        float x0[N], x1[N];
        S* d0 = fetch(f, x0);
        S* d1 = two ? fetch(f + NT, x1) : d0;
        if (!two) {
#pragma unroll
            for (int l = 0; l < N; ++l) x1[l] = x0[l];
        }
        f2 y0[N / 2], y1[N / 2];
        contract_rows<N>(m1p, x0, y0);
        contract_rows<N>(m1p, x1, y1);
        pair_store<S, N, D>(a, d0, y0);
        if (two) pair_store<S, N, D>(a, d1, y1);
    }
}

// FPS: fibers per step of the last contraction (1, or 2 for more instruction-level
// parallelism at the cost of registers).
template <typename S, int N, int D, int NT, int FPS>
__global__ void __launch_bounds__(NT) pair_kernel(const __grid_constant__ PairArgs<N, D> a) {
    using L = PairLayout<N, D, (int)sizeof(S)>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    const int P = a.P;
    const size_t xstage = round_up((size_t)P * L::SX * sizeof(S), 128);
    unsigned char* xbase = smem + 128;
    float* ex1 = reinterpret_cast<float*>(xbase + a.nstage * xstage);
    float* ex2 = ex1 + (size_t)P * L::EX1;
    const int tid = threadIdx.x;
    const int64_t ntiles = (a.batch + P - 1) / P;
    const int64_t grid = gridDim.x;
    const bool warp0 = tid < 32;
    uint64_t pol = 0;

    if (tid == 0) {
        for (int s = 0; s < a.nstage; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (warp0) {
        pol = l2_evict_first_policy();
        for (int s = 0; s < a.nstage; ++s) {
            const int64_t t = blockIdx.x + s * grid;
            if (t < ntiles) pair_issue<S, N, D>(a, xbase + s * xstage, &bars[s], t, pol);
        }
    }

    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
        const int s = it % a.nstage;
        S* xt = reinterpret_cast<S*>(xbase + s * xstage);
        const int64_t inst0 = tile * P;
        const int cnt = (int)min((int64_t)P, a.batch - inst0);
        bool ok = mbar_wait_bounded(&bars[s], (unsigned)(it / a.nstage) & 1u, a.err);
        if constexpr (!L::XPAD) {
            const unsigned bytes = (unsigned)cnt * L::NX * (unsigned)sizeof(S);
            const unsigned b16 = bytes & ~15u;
            if (bytes != b16) {   // ragged end of the batch: last bytes by hand
                const S* src = static_cast<const S*>(a.X) + inst0 * L::NX;
                for (int e = b16 / sizeof(S) + tid; e < cnt * L::NX; e += NT) xt[e] = src[e];
                __syncthreads();
            }
        }

        // ---- first contraction (pairs of fibers): operand tile -> ex1 ----------------
        if constexpr (D == 2) {
            const int F = cnt * (N / 2);
            for (int u = tid; u < F; u += NT) {
                const int q = u / (N / 2), l = 2 * (u - q * (N / 2));
                const S* xr = xt + q * L::SX + l;
                f2 x[N], w[N];
#pragma unroll
                for (int m = 0; m < N; ++m) x[m] = load_pair<S>(xr + N * m);
                contract_dup<N>(a.da, x, w);
                float* wr = ex1 + (it & 1) * (size_t)P * L::SQ + q * L::SQ + l;
#pragma unroll
                for (int j = 0; j < N; ++j) *reinterpret_cast<f2*>(wr + L::SJ * j) = w[j];
            }
        } else {
            const int F = cnt * (N * N / 2);
            for (int u = tid; u < F; u += NT) {
                const int q = u / (N * N / 2), r = u - q * (N * N / 2);
                const int i = 2 * (r % (N / 2)), j = r / (N / 2);
                const S* xr = xt + q * L::NX + i + N * j;
                f2 x[N], t[N];
#pragma unroll
                for (int p = 0; p < N; ++p) x[p] = load_pair<S>(xr + N * N * p);
                contract_dup<N>(a.da, x, t);
                float* tr = (L::TIN ? reinterpret_cast<float*>(xt) : ex1) + q * L::STQ + i + N * j;
#pragma unroll
                for (int k = 0; k < N; ++k) *reinterpret_cast<f2*>(tr + L::ST * k) = t[k];
            }
        }
        if (__syncthreads_or(!ok)) {
            if (warp0 && tid == 0) {
                for (int j = it; j < it + a.nstage; ++j)
                    if (blockIdx.x + (int64_t)j * grid < ntiles)
                        mbar_wait_bounded(&bars[j % a.nstage], (unsigned)(j / a.nstage) & 1u, a.err);
            }
            return;
        }
        if constexpr (!L::TIN) {
            if (warp0) {
                const int64_t next = tile + a.nstage * grid;
                if (next < ntiles) {
                    fence_proxy_async_smem();
                    pair_issue<S, N, D>(a, xt, &bars[s], next, pol);
                }
            }
        }

        S* Y = static_cast<S*>(a.Y);
        if constexpr (D == 2) {
            const f2* m1p = reinterpret_cast<const f2*>(a.m1);
            const float* wb = ex1 + (it & 1) * (size_t)P * L::SQ;
            const int F = cnt * N;
            if constexpr (FPS == 2) {
                last_stage<S, N, D, NT>(a, F, [&](int f, float (&w)[N]) {
                    const int q = f / N, j = f - q * N;
                    load_row<N>(wb + q * L::SQ + L::SJ * j, w);
                    return Y + (inst0 + q) * L::NX + N * j;
                });
            } else {
                for (int f = tid; f < F; f += NT) {
                    const int q = f / N, j = f - q * N;
                    float w[N];
                    load_row<N>(wb + q * L::SQ + L::SJ * j, w);
                    f2 y[N / 2];
                    contract_rows<N>(m1p, w, y);
                    pair_store<S, N, D>(a, Y + (inst0 + q) * L::NX + N * j, y);
                }
            }
            // W alternates between two buffers: the next tile's first stage writes the
            // other one, and the barrier after it orders this tile's reads before reuse.
        } else {
            const int F = cnt * (N * N / 2);
            for (int u = tid; u < F; u += NT) {
                const int q = u / (N * N / 2), r = u - q * (N * N / 2);
                const int i = 2 * (r % (N / 2)), k = r / (N / 2);
                const float* tr = (L::TIN ? reinterpret_cast<const float*>(xt) : ex1) + q * L::STQ + i + L::ST * k;
                f2 t[N], v[N];
#pragma unroll
                for (int m = 0; m < N; ++m) t[m] = *reinterpret_cast<const f2*>(tr + N * m);
                contract_dup<N>(a.db, t, v);
                float* ur = ex2 + q * L::SQ + i + L::SK * k;
#pragma unroll
                for (int j = 0; j < N; ++j) *reinterpret_cast<f2*>(ur + L::SJ * j) = v[j];
            }
            __syncthreads();
            if constexpr (L::TIN) {
                if (warp0) {   // T is consumed: the tile buffer takes the next operands
                    const int64_t next = tile + a.nstage * grid;
                    if (next < ntiles) {
                        fence_proxy_async_smem();
                        pair_issue<S, N, D>(a, xt, &bars[s], next, pol);
                    }
                }
            }
            const int F3 = cnt * N * N;
            if constexpr (FPS == 2) {   // two fibers per step: more ILP
                last_stage<S, N, D, NT>(a, F3, [&](int f, float (&u)[N]) {
                    const int q = f / (N * N), r = f - q * (N * N);
                    const int j = r % N, k = r / N;
                    load_row<N>(ex2 + q * L::SQ + L::SJ * j + L::SK * k, u);
                    return Y + (inst0 + q) * L::NX + N * j + N * N * k;
                });
            } else {                    // one fiber per step: fewer registers
                const f2* m1p = reinterpret_cast<const f2*>(a.m1);
                for (int f = tid; f < F3; f += NT) {
                    const int q = f / (N * N), r = f - q * (N * N);
                    const int j = r % N, k = r / N;
                    float u[N];
                    load_row<N>(ex2 + q * L::SQ + L::SJ * j + L::SK * k, u);
                    f2 y[N / 2];
                    contract_rows<N>(m1p, u, y);
                    pair_store<S, N, D>(a, Y + (inst0 + q) * L::NX + N * j + N * N * k, y);
                }
            }
            // ex2 is rewritten only after the next tile's first barrier.
        }
    }
}

template <typename S, int N, int D>
size_t pair_smem_bytes(int P, int nstage) {
    using L = PairLayout<N, D, (int)sizeof(S)>;
    return 128 + nstage * round_up((size_t)P * L::SX * sizeof(S), 128) + (size_t)P * (L::EX1 + L::EX2) * sizeof(float);
}

// Default tile: threads per CTA and instances per tile for each (N, kind), and
// fibers per step of the last contraction (two measured faster for 3-D n >= 14,
// one elsewhere).
template <int N, int D>
struct PairConfig {
    static constexpr int NT = 128;
    static constexpr int FPS = (D == 3 && N >= 14) ? 2 : 1;
    // about one unit of first-stage work per thread (3-D: rounded up, so that a
    // tile keeps every thread busy in the first stage, measured 1.2x faster at
    // n = 12 than rounding down to one instance; two units at n <= 8, where the
    // tuner's choices were 1.1x faster)
    static constexpr int P0 = (D == 2) ? (2 * NT) / N
                                       : (N <= 8 ? 2 : 1) * ((2 * NT + N * N - 1) / (N * N));
};

template <typename S, int N, int D>
kron_status launch_pair_n(const KronDesc& d, cudaStream_t st) {
    using L = PairLayout<N, D, (int)sizeof(S)>;
    constexpr int NT = PairConfig<N, D>::NT;
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    PairArgs<N, D> a;
    const double* first = (D == 2) ? d.m2 : d.m3;
    auto dup = [](double x) {
        const float v = (float)x;
        unsigned b;
        memcpy(&b, &v, sizeof(b));
        return ((f2)b << 32) | (f2)b;
    };
    for (int e = 0; e < N * N; ++e) {
        a.da[e] = dup(first[e]);
        if constexpr (D == 3) a.db[e] = dup(d.m2[e]);
        a.m1[e] = (float)d.m1[e];
    }
    if constexpr (D == 2) a.db[0] = 0;
    a.X = d.X;
    a.Y = d.Y;
    a.batch = d.batch;
    a.alpha = (float)d.alpha;
    a.beta = (float)d.beta;
    a.beta_zero = d.beta == 0.0;
    a.alpha_one = d.alpha == 1.0;
    a.err = device_error_word();
    if (!a.err) return KRON_ERR_CUDA;
    int P = d.P > 0 ? d.P : PairConfig<N, D>::P0;
    if (!L::XPAD) {
        int mult = 1;
        while ((mult * L::NX * sizeof(S)) % 16) ++mult;
        P = (P + mult - 1) / mult * mult;
    }
    // One stage in flight gives the most resident CTAs, which matters more than a
    // deeper pipeline (measured for both kinds).
    int nstage = d.nstage >= 1 ? d.nstage : 1;
    if (nstage > 8) nstage = 8;
    size_t smem = pair_smem_bytes<S, N, D>(P, nstage);
    while (nstage > 1 && smem > dev.smem_per_block_optin) smem = pair_smem_bytes<S, N, D>(P, --nstage);
    if (smem > dev.smem_per_block_optin) return KRON_ERR_NOT_SUPPORTED;
    a.P = P;
    a.nstage = nstage;
    const int fps = d.fps > 0 ? d.fps : PairConfig<N, D>::FPS;
    auto kern = fps == 2 ? pair_kernel<S, N, D, NT, 2> : pair_kernel<S, N, D, NT, 1>;
    if (!ensure_smem_optin((const void*)kern, smem)) return KRON_ERR_CUDA;
    const int64_t ntiles = (d.batch + P - 1) / P;
    int64_t grid = d.grid;
    if (grid <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem) != cudaSuccess) return KRON_ERR_CUDA;
        grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
    }
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, NT, smem, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

// Even N only; returns KRON_ERR_NOT_SUPPORTED for odd N (caller falls back).
template <typename S, int D>
kron_status launch_pair_d(const KronDesc& d, cudaStream_t st) {
    switch (d.N) {
        case 2: return launch_pair_n<S, 2, D>(d, st);
        case 4: return launch_pair_n<S, 4, D>(d, st);
        case 6: return launch_pair_n<S, 6, D>(d, st);
        case 8: return launch_pair_n<S, 8, D>(d, st);
        case 10: return launch_pair_n<S, 10, D>(d, st);
        case 12: return launch_pair_n<S, 12, D>(d, st);
        case 14: return launch_pair_n<S, 14, D>(d, st);
        case 16: return launch_pair_n<S, 16, D>(d, st);
        default: return KRON_ERR_NOT_SUPPORTED;
    }
}

}  // namespace kron
