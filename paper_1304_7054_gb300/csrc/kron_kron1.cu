// The 1-D product (TKRON1, Sec. 3) for FP32 and 16-bit storage:
//   y^p = alpha op(A) x^p + beta y^p,  op(A): ma x na (<= 16).
//
// One thread computes one instance.  x^p comes in with plain (L1-cached)
// loads, 16 bytes at a time when the layout allows it; the outputs are formed
// in pairs of rows (fma.rn.f32x2 with the coefficient pair (A[i,l], A[i+1,l])
// from the kernel parameter bank, op(A) zero-padded to N x N).  When the
// outputs of consecutive instances are packed (ldyp = ma) a warp writes its 32
// results into a shared-memory buffer and sends them out as one bulk copy
// (TMA), so L2 receives whole lines rather than the partial sectors of per-
// thread vector stores; two buffers per warp let the next results be formed
// while the copy drains.  Other layouts store from registers.
#include "kron_pair.cuh"

namespace kron {

namespace {

constexpr int kK1Threads = 256;
constexpr int kK1Warps = kK1Threads / 32;

template <int N>
struct Kron1Args {
    float m[N * N];      // op(A), N x N column-major (zero-padded), read as row pairs
    const void* X;
    void* Y;
    int64_t ldxp, ldyp, batch;
    int ma, na;
    int vec_x;           // x^p loads as 16-byte vectors
    int bulk_y;          // packed, 16-byte aligned outputs: staged + bulk-copied
    int beta_zero, alpha_one;
    float alpha, beta;
};

template <typename S, int V> struct VecOf;
template <> struct VecOf<float, 4> { using T = float4; };
template <> struct VecOf<__nv_bfloat16, 8> { using T = uint4; };
template <> struct VecOf<__half, 8> { using T = uint4; };

// Writes the ma results of one instance (row pairs y[r]) at dst in the storage
// type, with the widest shared-memory stores that ma allows: lanes write ma
// elements apart, and 8- or 16-byte stores cut the bank conflicts of that
// stride to at most 4-way.
template <typename S, int N>
__device__ __forceinline__ void stage_row(S* dst, const f2 (&y)[N / 2], int ma) {
    if constexpr (sizeof(S) == 4) {
        if (ma % 4 == 0) {
#pragma unroll
            for (int c = 0; c < N / 4; ++c)
                if (4 * c < ma)
                    *reinterpret_cast<uint4*>(dst + 4 * c) = make_uint4(
                        (unsigned)y[2 * c], (unsigned)(y[2 * c] >> 32), (unsigned)y[2 * c + 1], (unsigned)(y[2 * c + 1] >> 32));
            return;
        }
        if (ma % 2 == 0) {
#pragma unroll
            for (int r = 0; r < N / 2; ++r)
                if (2 * r < ma) *reinterpret_cast<f2*>(dst + 2 * r) = y[r];
            return;
        }
    } else {
        if (ma % 8 == 0) {
#pragma unroll
            for (int c = 0; c < N / 8; ++c)
                if (8 * c < ma)
                    *reinterpret_cast<uint4*>(dst + 8 * c) = make_uint4(pack16<S>(y[4 * c]), pack16<S>(y[4 * c + 1]),
                                                                        pack16<S>(y[4 * c + 2]), pack16<S>(y[4 * c + 3]));
            return;
        }
        if (ma % 2 == 0) {
#pragma unroll
            for (int r = 0; r < N / 2; ++r)
                if (2 * r < ma) *reinterpret_cast<unsigned*>(dst + 2 * r) = pack16<S>(y[r]);
            return;
        }
    }
#pragma unroll
    for (int r = 0; r < N / 2; ++r) {
        if (2 * r < ma) dst[2 * r] = store_cvt<S, float>(f2_lo(y[r]));
        if (2 * r + 1 < ma) dst[2 * r + 1] = store_cvt<S, float>(f2_hi(y[r]));
    }
}

template <typename S, int N>
__global__ void __launch_bounds__(kK1Threads) kron1_kernel(const __grid_constant__ Kron1Args<N> a) {
    constexpr int R = N / 2;                         // output row pairs
    constexpr int VE = 16 / (int)sizeof(S);          // elements per 16-byte vector
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    S* stage = reinterpret_cast<S*>(smem) + (size_t)warp * 2 * 32 * N;   // two buffers of 32 x N
    const S* X = static_cast<const S*>(a.X);
    S* Y = static_cast<S*>(a.Y);
    const f2* mp = reinterpret_cast<const f2*>(a.m);
    const int64_t nchunks = (a.batch + 31) / 32;
    const int64_t wstride = (int64_t)gridDim.x * kK1Warps;
    int buf = 0;
    for (int64_t ch = (int64_t)blockIdx.x * kK1Warps + warp; ch < nchunks; ch += wstride, buf ^= 1) {
        const int64_t p = ch * 32 + lane;
        const bool live = p < a.batch;
        float x[N];
#pragma unroll
        for (int l = 0; l < N; ++l) x[l] = 0.f;
        if (live) {
            const S* xp = X + p * a.ldxp;
            if (a.vec_x) {
#pragma unroll
                for (int c = 0; c < N / VE; ++c) {
                    if (c * VE < a.na) {
                        const typename VecOf<S, VE>::T v = *reinterpret_cast<const typename VecOf<S, VE>::T*>(xp + c * VE);
                        const S* e = reinterpret_cast<const S*>(&v);
#pragma unroll
                        for (int u = 0; u < VE; ++u) x[c * VE + u] = load_cvt<float, S>(e[u]);
                    }
                }
            } else {
#pragma unroll
                for (int l = 0; l < N; ++l)
                    if (l < a.na) x[l] = load_cvt<float, S>(xp[l]);
            }
        }
        f2 y[R];
        contract_rows<N>(mp, x, y);
        if (!a.alpha_one) {
            const f2 al = f2_pack(a.alpha, a.alpha);
#pragma unroll
            for (int r = 0; r < R; ++r) y[r] = fmul2(y[r], al);
        }
        S* yp = Y + p * a.ldyp;
        if (!a.beta_zero && live) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float b0 = 2 * r < a.ma ? load_cvt<float, S>(yp[2 * r]) : 0.f;
                const float b1 = 2 * r + 1 < a.ma ? load_cvt<float, S>(yp[2 * r + 1]) : 0.f;
                y[r] = ffma2(f2_pack(a.beta, a.beta), f2_pack(b0, b1), y[r]);
            }
        }
        const int64_t p0 = ch * 32;
        const int cnt = (int)min((int64_t)32, a.batch - p0);
        const unsigned bytes = (unsigned)cnt * a.ma * (unsigned)sizeof(S);
        if (a.bulk_y && bytes % 16 == 0) {
            // stage the warp's results (instance lane at lane * ma) and copy them out
            S* sb = stage + buf * 32 * N;
            if (lane == 0) bulk_wait_read_1();   // this buffer's previous copy (two chunks back) has left
            __syncwarp();
            if (live) stage_row<S, N>(sb + lane * a.ma, y, a.ma);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                bulk_s2g_hint(Y + p0 * a.ma, sb, bytes, l2_evict_first_policy());
                bulk_commit();
            }
        } else if (live) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (2 * r < a.ma) yp[2 * r] = store_cvt<S, float>(f2_lo(y[r]));
                if (2 * r + 1 < a.ma) yp[2 * r + 1] = store_cvt<S, float>(f2_hi(y[r]));
            }
        }
    }
    if (lane == 0) bulk_wait_all();
}

// FP32, n = 16, packed square vectors (ldxp = ldyp = 16), 16-byte aligned X and Y:
// tiles of P vectors arrive by one bulk copy each (TMA) in an NB-deep ring, each
// thread overwrites its own vector in place with its results, and the tile
// leaves by one bulk copy.  Lane i reads and writes the four 16-byte chunks of
// its vector starting at chunk (i >> 1) & 3, so the eight lanes of a quarter-
// warp (vectors 64 bytes apart) hit eight distinct 4-bank groups; the chunks are
// rotated back in registers (selects, no dynamic indexing).
// 16 KB tiles (one vector per thread) in a 6-deep ring: measured 1.1x the copy
// throughput of 32 KB tiles in a 3-deep ring (the same shared memory per CTA).
constexpr int kK1TileVecs = 256;
constexpr int kK1Ring = 6;

struct Kron1TArgs {
    Kron1Args<16> a;
    int tile;            // vectors per tile
    int nstage;
    unsigned* err;
};

// t[k] <- t[(k + DIR * rho) mod 4] for DIR = -1 (undo a read rotation) or +1.
template <int DIR>
__device__ __forceinline__ void rotate_chunks(float4 (&t)[4], int rho) {
    const bool r1 = rho & 1, r2 = rho & 2;
    float4 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 x = t[k], y = t[(k + DIR + 4) & 3];
        v[k] = make_float4(r1 ? y.x : x.x, r1 ? y.y : x.y, r1 ? y.z : x.z, r1 ? y.w : x.w);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 x = v[k], y = v[(k + 2) & 3];
        t[k] = make_float4(r2 ? y.x : x.x, r2 ? y.y : x.y, r2 ? y.z : x.z, r2 ? y.w : x.w);
    }
}

__global__ void __launch_bounds__(kK1Threads) kron1t_kernel(const __grid_constant__ Kron1TArgs ta) {
    const Kron1Args<16>& a = ta.a;
    constexpr int N = 16, R = 8;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    float* ring = reinterpret_cast<float*>(smem + 128);
    const int NB = ta.nstage;
    const int TV = ta.tile;   // vectors per tile
    const int64_t ntiles = (a.batch + TV - 1) / TV;
    const int64_t grid = gridDim.x;
    const float* X = static_cast<const float*>(a.X);
    float* Y = static_cast<float*>(a.Y);
    const f2* mp = reinterpret_cast<const f2*>(a.m);
    uint64_t pol = 0;
    auto count = [&](int64_t t) { return (unsigned)min((int64_t)TV, a.batch - t * TV); };
    auto issue = [&](int s, int64_t t) {
        const unsigned bytes = count(t) * N * 4u;
        mbar_arrive_expect_tx(&bars[s], bytes);
        bulk_g2s(ring + (size_t)s * TV * N, X + t * TV * N, bytes, &bars[s], pol);
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < NB; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
        pol = l2_evict_first_policy();
        for (int s = 0; s < NB; ++s)
            if (blockIdx.x + s * grid < ntiles) issue(s, blockIdx.x + s * grid);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, rho = (lane >> 1) & 3;
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
        const int s = it % NB;
        const bool ok = mbar_wait_bounded(&bars[s], (unsigned)(it / NB) & 1u, ta.err);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                for (int j = it; j < it + NB; ++j)
                    if (blockIdx.x + (int64_t)j * grid < ntiles)
                        mbar_wait_bounded(&bars[j % NB], (unsigned)(j / NB) & 1u, ta.err);
                bulk_wait_all();
            }
            return;
        }
        float* buf = ring + (size_t)s * TV * N;
        const int cnt = (int)count(tile);
        for (int q = threadIdx.x; q < cnt; q += kK1Threads) {
            float* v = buf + q * N;
            float4 t[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) t[c] = *reinterpret_cast<const float4*>(v + 4 * ((c + rho) & 3));
            rotate_chunks<-1>(t, rho);
            float x[N];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                x[4 * c] = t[c].x;
                x[4 * c + 1] = t[c].y;
                x[4 * c + 2] = t[c].z;
                x[4 * c + 3] = t[c].w;
            }
            f2 y[R];
            contract_rows<N>(mp, x, y);
            if (!a.alpha_one) {
                const f2 al = f2_pack(a.alpha, a.alpha);
#pragma unroll
                for (int r = 0; r < R; ++r) y[r] = fmul2(y[r], al);
            }
            if (!a.beta_zero) {
                const float* yp = Y + (tile * TV + q) * N;
                const f2 be = f2_pack(a.beta, a.beta);
#pragma unroll
                for (int r = 0; r < R; ++r) y[r] = ffma2(be, load_pair<float>(yp + 2 * r), y[r]);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
                t[c] = make_float4(f2_lo(y[2 * c]), f2_hi(y[2 * c]), f2_lo(y[2 * c + 1]), f2_hi(y[2 * c + 1]));
            rotate_chunks<1>(t, rho);
#pragma unroll
            for (int c = 0; c < 4; ++c) *reinterpret_cast<float4*>(v + 4 * ((c + rho) & 3)) = t[c];
        }
        fence_proxy_async_smem();   // results written: visible to the bulk store
        __syncthreads();
        if (threadIdx.x == 0) {
            bulk_s2g_hint(Y + tile * TV * N, buf, count(tile) * N * 4u, pol);
            bulk_commit();
            const int64_t next = tile + (int64_t)NB * grid;
            if (next < ntiles) {
                bulk_wait_read();   // the results have left the buffer
                issue(s, next);
            }
        }
    }
    if (threadIdx.x == 0) bulk_wait_all();
}

template <typename S, int N>
kron_status launch_k1(const GemmADesc& g, cudaStream_t st) {
    // g describes TKRON1 as TGEMM_A with m = 1: b[l * 16 + j] = op(A)(j, l).
    Kron1Args<N> a;
    memset(&a, 0, sizeof(a));
    for (int l = 0; l < g.k; ++l)
        for (int j = 0; j < g.n; ++j) a.m[j + N * l] = (float)g.b[l * 16 + j];
    a.X = g.A;
    a.Y = g.C;
    a.ldxp = g.lda2;
    a.ldyp = g.ldc2;
    a.batch = g.batch;
    a.ma = g.n;
    a.na = g.k;
    constexpr int VE = 16 / (int)sizeof(S);
    a.vec_x = (a.na % VE == 0) && ((uintptr_t)g.A % 16 == 0) && ((a.ldxp * (int64_t)sizeof(S)) % 16 == 0);
    a.bulk_y = (a.ldyp == a.ma) && ((uintptr_t)g.C % 16 == 0);
    a.alpha = (float)g.alpha;
    a.beta = (float)g.beta;
    a.alpha_one = g.alpha == 1.0;
    a.beta_zero = g.beta == 0.0;
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    if constexpr (N == 16 && sizeof(S) == 4) {
        if (a.ma == 16 && a.na == 16 && a.ldxp == 16 && a.ldyp == 16 && (uintptr_t)g.A % 16 == 0 &&
            (uintptr_t)g.C % 16 == 0) {
            Kron1TArgs ta;
            ta.a = a;
            ta.err = device_error_word();
            if (!ta.err) return KRON_ERR_CUDA;
            int nb = kK1Ring;
            ta.tile = kK1TileVecs;
            const int TV = ta.tile;
            auto smem_of = [&](int n_b) { return 128 + (size_t)n_b * TV * 16 * sizeof(float); };
            while (nb > 1 && smem_of(nb) > dev.smem_per_block_optin) --nb;
            const size_t smem = smem_of(nb);
            ta.nstage = nb;
            if (smem <= dev.smem_per_block_optin) {
                const void* kern = (const void*)kron1t_kernel;
                if (!ensure_smem_optin(kern, smem)) return KRON_ERR_CUDA;
                int per_sm = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kron1t_kernel, kK1Threads, smem) !=
                    cudaSuccess)
                    return KRON_ERR_CUDA;
                const int64_t ntiles = (g.batch + TV - 1) / TV;
                int64_t grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
                grid = std::max<int64_t>(1, std::min<int64_t>(grid, ntiles));
                void* args[] = {&ta};
                if (cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(kK1Threads), args, smem, st) != cudaSuccess)
                    return KRON_ERR_CUDA;
                return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
            }
        }
    }
    auto kern = kron1_kernel<S, N>;
    const size_t smem = (size_t)kK1Warps * 2 * 32 * N * sizeof(S);
    if (!ensure_smem_optin((const void*)kern, smem)) return KRON_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kK1Threads, smem) != cudaSuccess)
        return KRON_ERR_CUDA;
    const int64_t chunks = (g.batch + 31) / 32;
    int64_t grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
    grid = std::min<int64_t>(grid, (chunks + kK1Warps - 1) / kK1Warps);
    grid = std::max<int64_t>(grid, 1);
    kern<<<(unsigned)grid, kK1Threads, smem, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

template <typename S>
kron_status launch_k1_s(const GemmADesc& g, cudaStream_t st) {
    const int n = std::max(g.n, g.k);
    switch ((n + 1) / 2 * 2) {
        case 2: return launch_k1<S, 2>(g, st);
        case 4: return launch_k1<S, 4>(g, st);
        case 6: return launch_k1<S, 6>(g, st);
        case 8: return launch_k1<S, 8>(g, st);
        case 10: return launch_k1<S, 10>(g, st);
        case 12: return launch_k1<S, 12>(g, st);
        case 14: return launch_k1<S, 14>(g, st);
        case 16: return launch_k1<S, 16>(g, st);
    }
    return KRON_ERR_INVALID_VALUE;
}

}  // namespace

// TKRON1 given as TGEMM_A with m = 1 (see kron1_batched); FP64 storage is left
// to the TGEMM_A kernel (KRON_ERR_NOT_SUPPORTED here).
kron_status launch_kron1(const GemmADesc& g, cudaStream_t st) {
    if (g.m != 1 || g.transa != 0 || g.lda != 1 || g.ldc != 1) return KRON_ERR_NOT_SUPPORTED;
    switch (g.io) {
        case KRON_R32F: return launch_k1_s<float>(g, st);
        case KRON_R16BF: return launch_k1_s<__nv_bfloat16>(g, st);
        case KRON_R16F: return launch_k1_s<__half>(g, st);
        default: return KRON_ERR_NOT_SUPPORTED;
    }
}

}  // namespace kron
