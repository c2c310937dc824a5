// 2-D and 3-D FP32 kernels for odd n with all mode contractions done in place.
//
// The contractions are those of the other 3-D kernels (Sec. 2.1, the order of
// Algorithm 1 with the intermediates on chip): mode 3 with M3, mode 2 with M2,
// mode 1 with M1.  Every stage gives one thread one fiber: it reads the fiber
// into registers, forms the outputs in pairs of rows (fma.rn.f32x2 with the
// coefficient pair (M[r, l], M[r+1, l]) from the kernel parameter bank; the
// components are padded with a zero row to an even row count) and writes them
// back over the fiber's own words.  So the operand tile is the only on-chip
// storage, and:
//
//   instance q of a tile sits at word n^d q (packed), element (i, j, k) at
//   i + n j + n^2 k.  Stage A and B threads walk consecutive i (consecutive
//   words), stage C threads consecutive j (stride n, odd): every scalar shared
//   access of a warp touches distinct banks.  2-D runs stages B and C only.
//
// Tiles of P instances (P a multiple of 4, so a tile is a whole number of 16-byte
// chunks) arrive and leave as one bulk copy (TMA) each; one producer warp streams
// them through a ring of buffers (full / empty mbarriers).
#include <algorithm>

#include "kron_pair.cuh"

namespace kron {

namespace {

constexpr int kFiCompute = 128;                 // compute threads of one group (4 warps)
constexpr int kFiThreads = kFiCompute + 32;
constexpr int kFiMaxRing = 12;
constexpr int kFiMaxGroups = 4;
// 2-D: up to four compute groups share one CTA's ring (one CTA per SM); 3-D:
// one group per CTA, several CTAs per SM (the FMA-bound 3-D stages want the
// resident warps of more CTAs).
template <int D> constexpr int fi_max_threads() { return D == 2 ? kFiCompute * kFiMaxGroups + 32 : kFiThreads; }
template <int D> constexpr int fi_min_blocks() { return D == 2 ? 1 : 4; }

template <int N>
struct FiberIpArgs {
    static constexpr int R = (N + 1) / 2;   // output row pairs (last one padded)
    f2 m3[R * N], m2[R * N], m1[R * N];     // (M[2r, l], M[2r+1, l]) at r + R l (m3 unused in 2-D)
    const void* X;
    void* Y;
    int64_t batch;
    int P, nstage;
    int beta_zero, alpha_one;
    float alpha, beta;
    unsigned* err;
};

// y[r] = (M x)[2r, 2r+1] for one fiber x of length N.
template <int N>
__device__ __forceinline__ void contract_pairs(const f2* __restrict__ Mp, const float (&x)[N], f2 (&y)[(N + 1) / 2]) {
    constexpr int R = (N + 1) / 2;
    const f2 x0 = f2_pack(x[0], x[0]);
#pragma unroll
    for (int r = 0; r < R; ++r) y[r] = fmul2(Mp[r], x0);
#pragma unroll
    for (int l = 1; l < N; ++l) {
        const f2 xl = f2_pack(x[l], x[l]);
#pragma unroll
        for (int r = 0; r < R; ++r) y[r] = ffma2(Mp[r + R * l], xl, y[r]);
    }
}

// Reads the fiber at p with stride S, contracts it with M, writes it back.
template <int N, int S>
__device__ __forceinline__ void fiber_in_place(float* p, const f2* Mp) {
    float x[N];
#pragma unroll
    for (int l = 0; l < N; ++l) x[l] = p[S * l];
    f2 y[(N + 1) / 2];
    contract_pairs<N>(Mp, x, y);
#pragma unroll
    for (int r = 0; r < N; ++r) p[S * r] = (r & 1) ? f2_hi(y[r / 2]) : f2_lo(y[r / 2]);
}

template <int N, int D>
__global__ void __launch_bounds__(fi_max_threads<D>(), fi_min_blocks<D>())
fiberip_kernel(const __grid_constant__ FiberIpArgs<N> a, int G) {
    constexpr int NN = N * N, NX = D == 3 ? NN * N : NN;
    constexpr int NF = NX / N;   // fibers per instance and stage
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kFiMaxRing;
    float* ring = reinterpret_cast<float*>(smem + 256);
    const int NB = a.nstage, P = a.P;
    const int tile_words = P * NX;
    const int ncompute = kFiCompute * G;
    const int gidx = threadIdx.x / kFiCompute;
    const int tid = threadIdx.x - kFiCompute * gidx;   // thread within its compute group
    const int64_t ntiles = (a.batch + P - 1) / P;
    const int64_t grid = gridDim.x;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kFiCompute);
        }
        fence_barrier_init();
    }
    __syncthreads();

    if (threadIdx.x >= ncompute) {   // producer
        const int lane = threadIdx.x - ncompute;
        const uint64_t pol = l2_evict_first_policy();
        float* Y = static_cast<float*>(a.Y);
        const float* X = static_cast<const float*>(a.X);
        auto store_tile = [&](int s, int64_t t) {
            const int64_t i0 = t * P;
            const int c = (int)min((int64_t)P, a.batch - i0);
            // whole 16-byte chunks by bulk copy; a ragged last tile's tail is
            // stored by the compute threads
            const unsigned bytes = ((unsigned)c * NX * 4u) & ~15u;
            if (lane == 0 && bytes) bulk_s2g_hint(Y + i0 * NX, ring + s * tile_words, bytes, pol);
            bulk_commit();
        };
        int it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
            const int s = it % NB;
            if (it >= NB) {
                if (!mbar_wait_bounded(&empty[s], (unsigned)(it / NB - 1) & 1u, a.err)) {
                    bulk_wait_all();
                    return;
                }
                store_tile(s, tile - (int64_t)NB * grid);
                bulk_wait_read();
            }
            const int64_t i0 = tile * P;
            const int cnt = (int)min((int64_t)P, a.batch - i0);
            const unsigned bytes = ((unsigned)cnt * NX * 4u) & ~15u;   // the compute threads load the rest
            fence_proxy_async_smem();
            if (lane == 0) {
                mbar_arrive_expect_tx(&full[s], bytes);
                if (bytes) bulk_g2s(ring + s * tile_words, X + i0 * NX, bytes, &full[s], pol);
            }
        }
        for (int j = it > NB ? it - NB : 0; j < it; ++j) {
            if (!mbar_wait_bounded(&empty[j % NB], (unsigned)(j / NB) & 1u, a.err)) break;
            store_tile(j % NB, blockIdx.x + (int64_t)j * grid);
        }
        bulk_wait_all();
        return;
    }

    const float* X = static_cast<const float*>(a.X);
    float* Y = static_cast<float*>(a.Y);
    for (int it = gidx; blockIdx.x + (int64_t)it * grid < ntiles; it += G) {
        const int64_t tile = blockIdx.x + (int64_t)it * grid;
        const int s = it % NB;
        float* buf = ring + s * tile_words;
        const int64_t i0 = tile * P;
        const int cnt = (int)min((int64_t)P, a.batch - i0);
        const int nel = cnt * NX, nbulk = (int)((((unsigned)nel * 4u) & ~15u) / 4u);
        const bool ok = mbar_wait_bounded(&full[s], (unsigned)(it / NB) & 1u, a.err);
        if (nbulk != nel) {   // ragged last tile: the elements past the last 16-byte chunk
            for (int e = nbulk + tid; e < nel; e += kFiCompute) buf[e] = X[i0 * NX + e];
            group_sync_or(false, gidx);
        }
        if constexpr (D == 3) {
            // Stage A (mode 3): fibers (q, i, j), consecutive threads consecutive i.
#pragma unroll 1
            for (int u = tid; u < cnt * NN; u += kFiCompute) {
                const int q = u / NN, r = u - q * NN;
                fiber_in_place<N, NN>(buf + q * NX + r, a.m3);
            }
        }
        if (group_sync_or(!ok, gidx)) {
            if (tid == 0)
                for (int j = it; j < it + NB; ++j)
                    if (blockIdx.x + (int64_t)j * grid < ntiles)
                        mbar_wait_bounded(&full[j % NB], (unsigned)(j / NB) & 1u, a.err);
            return;
        }
        // Stage B (mode 2): fibers (q, i, k) (2-D: (q, i)).
#pragma unroll 1
        for (int u = tid; u < cnt * NF; u += kFiCompute) {
            const int q = u / NF, r = u - q * NF;
            const int i = r % N, k = r / N;
            fiber_in_place<N, N>(buf + q * NX + i + NN * k, a.m2);
        }
        group_sync_or(false, gidx);
        // Stage C (mode 1): fibers (q, j, k) (contiguous), with the epilogue.
#pragma unroll 1
        for (int u = tid; u < cnt * NF; u += kFiCompute) {
            const int q = u / NF, r = u - q * NF;
            float* p = buf + q * NX + N * r;
            float x[N];
#pragma unroll
            for (int l = 0; l < N; ++l) x[l] = p[l];
            f2 y[(N + 1) / 2];
            contract_pairs<N>(a.m1, x, y);
            const float* yg = Y + (i0 + q) * NX + N * r;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                float v = (i & 1) ? f2_hi(y[i / 2]) : f2_lo(y[i / 2]);
                if (!a.alpha_one) v *= a.alpha;
                if (!a.beta_zero) v = fmaf(a.beta, yg[i], v);
                p[i] = v;
            }
        }
        if (nbulk != nel) {   // ragged last tile: the tail the bulk copy leaves out
            group_sync_or(false, gidx);
            for (int e = nbulk + tid; e < nel; e += kFiCompute) Y[i0 * NX + e] = buf[e];
        }
        fence_proxy_async_smem();
        mbar_arrive(&empty[s]);
    }
}

template <int N, int D>
kron_status launch_fi_n(const KronDesc& d, cudaStream_t st) {
    constexpr int R = (N + 1) / 2;
    constexpr int NX = D == 3 ? N * N * N : N * N;
    // instances per tile: about 16-54 KB of operands, a multiple of 4
    constexpr int P0 = std::max(4, (6144 / NX) / 4 * 4);
    if (d.P > 0 && d.P % 4) return KRON_ERR_NOT_SUPPORTED;   // other tiles: fiber kernel
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    FiberIpArgs<N> a;
    memset(&a, 0, sizeof(a));
    auto pairs = [&](const double* m, f2* out) {
        for (int l = 0; l < N; ++l)
            for (int r = 0; r < R; ++r) {
                const float v0 = (float)m[2 * r + N * l];
                const float v1 = 2 * r + 1 < N ? (float)m[2 * r + 1 + N * l] : 0.f;
                unsigned b0, b1;
                memcpy(&b0, &v0, 4);
                memcpy(&b1, &v1, 4);
                out[r + R * l] = (f2)b0 | ((f2)b1 << 32);
            }
    };
    if constexpr (D == 3) pairs(d.m3, a.m3);
    pairs(d.m2, a.m2);
    pairs(d.m1, a.m1);
    a.X = d.X;
    a.Y = d.Y;
    a.batch = d.batch;
    a.alpha = (float)d.alpha;
    a.beta = (float)d.beta;
    a.beta_zero = d.beta == 0.0;
    a.alpha_one = d.alpha == 1.0;
    a.err = device_error_word();
    if (!a.err) return KRON_ERR_CUDA;
    a.P = d.P > 0 ? d.P : P0;
    // compute warps: 2-D four groups of four (one CTA per SM), 3-D one group
    const int W = d.warps > 0 ? d.warps : (D == 2 ? 16 : 4);
    const int G = W / 4;
    if (W % 4 || G < 1 || G > (D == 2 ? kFiMaxGroups : 1)) return KRON_ERR_NOT_SUPPORTED;
    // ring depth: measured two buffers per group; a multiple of the group count, so
    // that buffer it % NB passes from a group to itself (a parity wait cannot tell
    // phase u from phase u - 2)
    int nb = d.nstage >= 1 ? d.nstage : 2 * G;
    if (nb > kFiMaxRing) nb = kFiMaxRing;
    nb = nb < G ? G : nb / G * G;
    auto smem_of = [&](int n_b) { return 256 + (size_t)n_b * a.P * NX * sizeof(float); };
    size_t smem = smem_of(nb);
    while (nb > G && smem > dev.smem_per_block_optin) smem = smem_of(nb -= G);
    if (smem > dev.smem_per_block_optin) return KRON_ERR_NOT_SUPPORTED;
    a.nstage = nb;
    auto kern = fiberip_kernel<N, D>;
    if (!ensure_smem_optin((const void*)kern, smem)) return KRON_ERR_CUDA;
    const int64_t ntiles = (d.batch + a.P - 1) / a.P;
    int64_t grid = d.grid;
    if (grid <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFiCompute * G + 32, smem) != cudaSuccess)
            return KRON_ERR_CUDA;
        grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
    }
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, ntiles));
    kern<<<(unsigned)grid, kFiCompute * G + 32, smem, st>>>(a, G);
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

}  // namespace

// Odd n >= 3, 2-D or 3-D, FP32 storage and arithmetic, contiguous X and Y;
// tiles that are not a multiple of 4 instances (and other shapes) get
// KRON_ERR_NOT_SUPPORTED and are left to the fiber kernel.
template <int D>
kron_status launch_fi_d(const KronDesc& d, cudaStream_t st) {
    switch (d.N) {
        case 3: return launch_fi_n<3, D>(d, st);
        case 5: return launch_fi_n<5, D>(d, st);
        case 7: return launch_fi_n<7, D>(d, st);
        case 9: return launch_fi_n<9, D>(d, st);
        case 11: return launch_fi_n<11, D>(d, st);
        case 13: return launch_fi_n<13, D>(d, st);
        case 15: return launch_fi_n<15, D>(d, st);
        default: return KRON_ERR_NOT_SUPPORTED;
    }
}

kron_status launch_fiberip(const KronDesc& d, cudaStream_t st) {
    if (d.io != KRON_R32F || d.comp != KRON_COMPUTE_NATIVE || !d.contiguous || !d.ycontig)
        return KRON_ERR_NOT_SUPPORTED;
    return d.D == 3 ? launch_fi_d<3>(d, st) : launch_fi_d<2>(d, st);
}

}  // namespace kron
