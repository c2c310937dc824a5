// 2-D FP32 pair kernels for n = 2 mod 4 (n = 10, 14) with the mode exchange
// done in place.
//
// The two contractions are those of the generic pair kernel (Sec. 2.1, the
// 2-D case of Algorithm 1: mode 2 with M2 = op(A) as pairs of fibers, then
// mode 1 with M1 = op(B) as pairs of rows), with all on-chip traffic in the
// operand tile itself:
//
//  * The intermediate W = X M2^T overwrites the operand: a thread reads rows
//    (2u, 2u+1) of one instance into registers and writes rows (2u, 2u+1) of
//    W to the same words.  The second stage reads column j of W (no other
//    thread touches those words), and writes column j of Y back over it.
//  * A tile arrives and its results leave as one bulk copy (TMA) each, so L2
//    receives whole lines for Y (partial 8- or 16-byte stores from registers
//    reach it as partial sectors).
//  * n^2 = 4 mod 32 for n = 2 mod 4, so consecutive packed instances start 4
//    words apart in bank order.  Each group of 16 threads takes 8 consecutive
//    instances times 2 adjacent units (row pairs in the first stage, columns
//    in the second), so the eight-byte shared accesses of a half-warp cover
//    the 32 banks once: no bank conflicts.
//  * One producer warp streams tiles in and results out through a ring of
//    buffers (full / empty mbarriers); the four compute warps issue no global
//    memory access except the reads of Y that beta != 0 needs.
#include "kron_pair.cuh"

namespace kron {

namespace {

constexpr int kIpCompute = 128;               // compute threads of one group (4 warps)
constexpr int kIpThreads = kIpCompute + 32;   // + one producer warp
constexpr int kIpMaxRing = 12;
constexpr int kIpMaxGroups = 4;

template <int N>
struct IpLayout {
    static_assert(N % 4 == 2, "packed in-place layout: n = 2 mod 4");
    static constexpr int NX = N * N;
    static constexpr int G1 = (N / 2 + 1) / 2;   // 16-thread groups per 8 instances, stage 1
    static constexpr int G2 = N / 2;              // same, stage 2
    // default tile and ring depth (measured on the bench batches)
    static constexpr int P0 = N == 10 ? 48 : 40;
    // default ring depth and compute warps (measured: at n = 10 one CTA per SM
    // with four groups and an 8-deep ring streams best; at n = 14 the 31 KB tiles
    // leave room for one tile per group only, and six CTAs of one group with two
    // buffers each are faster)
    static constexpr int NB0 = N == 10 ? 8 : 2;
    static constexpr int W0 = N == 10 ? 16 : 4;
};

template <int N>
__device__ __forceinline__ void load_col(const float* p, float (&w)[N]) {
#pragma unroll
    for (int c = 0; c < N / 2; ++c) {
        const float2 v = *reinterpret_cast<const float2*>(p + 2 * c);
        w[2 * c] = v.x;
        w[2 * c + 1] = v.y;
    }
}

// A CTA holds G compute groups of four warps and one producer warp; group g
// takes the CTA's tiles it = g mod G from one shared ring, so one CTA per SM
// can keep a deep ring in flight while its groups work.
template <int N>
__global__ void __launch_bounds__(kIpCompute * kIpMaxGroups + 32, 1) pair2ip_kernel(const __grid_constant__ PairArgs<N, 2> a,
                                                                                     int G) {
    using L = IpLayout<N>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kIpMaxRing;
    float* ring = reinterpret_cast<float*>(smem + 256);
    const int NB = a.nstage;
    const int P = a.P;             // a multiple of 8
    const int QG = P >> 3;
    const int tile_words = P * L::NX;
    const int ncompute = kIpCompute * G;
    const int gidx = threadIdx.x / kIpCompute;
    const int tid = threadIdx.x - kIpCompute * gidx;   // thread within its group (producer: lane + 128)
    const int64_t ntiles = (a.batch + P - 1) / P;
    const int64_t grid = gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kIpCompute);
        }
        fence_barrier_init();
    }
    __syncthreads();

    if (threadIdx.x >= ncompute) {
        // Producer: tile `it` goes to buffer it % NB once the compute threads have
        // released that buffer's previous tile (it - NB), whose results they left
        // in the buffer: those are stored first.
        const int lane = threadIdx.x - ncompute;
        const uint64_t pol = l2_evict_first_policy();
        float* Y = static_cast<float*>(a.Y);
        const float* X = static_cast<const float*>(a.X);
        auto store_tile = [&](int s, int64_t t) {
            const int64_t i0 = t * P;
            const int c = (int)min((int64_t)P, a.batch - i0);
            if (lane == 0) bulk_s2g_hint(Y + i0 * L::NX, ring + s * tile_words, (unsigned)c * L::NX * 4u, pol);
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
                bulk_wait_read();   // the results have left the buffer
            }
            const int64_t inst0 = tile * P;
            const int cnt = (int)min((int64_t)P, a.batch - inst0);
            float* buf = ring + s * tile_words;
            // The compute threads' generic accesses to this buffer happen before their
            // arrival on empty[s]; order them before the bulk copies that overwrite it.
            fence_proxy_async_smem();
            if (lane == 0) mbar_arrive_expect_tx(&full[s], (unsigned)cnt * L::NX * 4u);
            __syncwarp();
            if (lane == 0) bulk_g2s(buf, X + inst0 * L::NX, (unsigned)cnt * L::NX * 4u, &full[s], pol);
        }
        for (int j = it > NB ? it - NB : 0; j < it; ++j) {   // the last tiles' results
            if (!mbar_wait_bounded(&empty[j % NB], (unsigned)(j / NB) & 1u, a.err)) break;
            store_tile(j % NB, blockIdx.x + (int64_t)j * grid);
        }
        bulk_wait_all();
        return;
    }

    const f2* m1p = reinterpret_cast<const f2*>(a.m1);
    const float* Y = static_cast<const float*>(a.Y);
    for (int it = gidx; blockIdx.x + (int64_t)it * grid < ntiles; it += G) {
        const int64_t tile = blockIdx.x + (int64_t)it * grid;
        const int s = it % NB;
        float* buf = ring + s * tile_words;
        const int64_t inst0 = tile * P;
        const int cnt = (int)min((int64_t)P, a.batch - inst0);
        const bool ok = mbar_wait_bounded(&full[s], (unsigned)(it / NB) & 1u, a.err);

        // Stage 1: rows (2u, 2u+1) of instance q times M2^T, written back in place.
#pragma unroll 1
        for (int f = tid; f < QG * L::G1 * 16; f += kIpCompute) {
            const int g = f >> 4, r = f & 15;
            const int q = 8 * (g % QG) + (r & 7), u = 2 * (g / QG) + (r >> 3);
            if (q < cnt && u < N / 2) {
                float* p = buf + L::NX * q + 2 * u;
                f2 x[N];
#pragma unroll
                for (int m = 0; m < N; ++m) x[m] = *reinterpret_cast<const f2*>(p + N * m);
                f2 w[N];
                contract_dup<N>(a.da, x, w);
#pragma unroll
                for (int j = 0; j < N; ++j) *reinterpret_cast<f2*>(p + N * j) = w[j];
            }
        }
        if (group_sync_or(!ok, gidx)) {
            // A copy did not land in time: wait (bounded) for the ones that may still
            // be in flight into this CTA's buffers, then give up.  The producer cannot
            // issue beyond tile it + NB - 1, whose buffer this iteration still holds.
            if (tid == 0)
                for (int j = it; j < it + NB; ++j)
                    if (blockIdx.x + (int64_t)j * grid < ntiles)
                        mbar_wait_bounded(&full[j % NB], (unsigned)(j / NB) & 1u, a.err);
            return;
        }

        // Stage 2: column j of W of instance q times M1 (pairs of output rows); the
        // results overwrite the column.
#pragma unroll 1
        for (int f = tid; f < QG * L::G2 * 16; f += kIpCompute) {
            const int g = f >> 4, r = f & 15;
            const int q = 8 * (g % QG) + (r & 7), j = 2 * (g / QG) + (r >> 3);
            if (q >= cnt) continue;
            float* wq = buf + L::NX * q + N * j;
            float w[N];
            load_col<N>(wq, w);
            f2 y[N / 2];
            contract_rows<N>(m1p, w, y);
            if (!a.alpha_one) {
                const f2 al = f2_pack(a.alpha, a.alpha);
#pragma unroll
                for (int k = 0; k < N / 2; ++k) y[k] = fmul2(y[k], al);
            }
            if (!a.beta_zero) {
                const float* yq = Y + (inst0 + q) * L::NX + N * j;
                const f2 be = f2_pack(a.beta, a.beta);
#pragma unroll
                for (int k = 0; k < N / 2; ++k) y[k] = ffma2(be, load_pair<float>(yq + 2 * k), y[k]);
            }
#pragma unroll
            for (int k = 0; k < N / 2; ++k) *reinterpret_cast<f2*>(wq + 2 * k) = y[k];
        }
        fence_proxy_async_smem();   // results written: visible to the bulk stores
        mbar_arrive(&empty[s]);
    }
}

template <int N>
size_t ip_smem_bytes(int P, int nb) {
    return 256 + (size_t)nb * P * IpLayout<N>::NX * sizeof(float);
}

template <int N>
kron_status launch_ip_n(const KronDesc& d, cudaStream_t st) {
    using L = IpLayout<N>;
    if (d.P > 0 && d.P % 8) return KRON_ERR_NOT_SUPPORTED;   // other tile sizes: generic pair kernel
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    PairArgs<N, 2> a;
    auto dup = [](double x) {
        const float v = (float)x;
        unsigned b;
        memcpy(&b, &v, sizeof(b));
        return ((f2)b << 32) | (f2)b;
    };
    for (int e = 0; e < N * N; ++e) {
        a.da[e] = dup(d.m2[e]);
        a.m1[e] = (float)d.m1[e];
    }
    a.db[0] = 0;
    a.X = d.X;
    a.Y = d.Y;
    a.batch = d.batch;
    a.alpha = (float)d.alpha;
    a.beta = (float)d.beta;
    a.beta_zero = d.beta == 0.0;
    a.alpha_one = d.alpha == 1.0;
    a.err = device_error_word();
    if (!a.err) return KRON_ERR_CUDA;
    const int P = d.P > 0 ? d.P : L::P0;
    const int W = d.warps > 0 ? d.warps : L::W0;
    const int G = W / 4;
    if (G < 1 || G > kIpMaxGroups || (W % 4)) return KRON_ERR_NOT_SUPPORTED;
    // The ring depth is a multiple of the number of groups, so that buffer it % NB
    // passes from a group to the same group (tile it - NB): a group then starts
    // its parity wait on a buffer only after its own previous use completed (a
    // parity wait cannot tell phase u from phase u - 2).
    int nb = d.nstage >= 1 ? d.nstage : (d.warps > 0 || d.P > 0 ? 2 * G : L::NB0);
    if (nb > kIpMaxRing) nb = kIpMaxRing;
    nb = nb < G ? G : nb / G * G;
    size_t smem = ip_smem_bytes<N>(P, nb);
    while (nb > G && smem > dev.smem_per_block_optin) smem = ip_smem_bytes<N>(P, nb -= G);
    if (smem > dev.smem_per_block_optin) return KRON_ERR_NOT_SUPPORTED;
    a.P = P;
    a.nstage = nb;
    auto kern = pair2ip_kernel<N>;
    if (!ensure_smem_optin((const void*)kern, smem)) return KRON_ERR_CUDA;
    const int threads = kIpCompute * G + 32;
    const int64_t ntiles = (d.batch + P - 1) / P;
    int64_t grid = d.grid;
    if (grid <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess)
            return KRON_ERR_CUDA;
        grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
    }
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, threads, smem, st>>>(a, G);
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

}  // namespace

// 2-D, n = 10 or 14, FP32 storage and arithmetic, contiguous X and Y; tile sizes
// that are not a multiple of 8 instances (and other shapes) get
// KRON_ERR_NOT_SUPPORTED and are left to the generic pair kernel.
kron_status launch_pair2ip(const KronDesc& d, cudaStream_t st) {
    if (d.D != 2 || d.io != KRON_R32F || d.comp != KRON_COMPUTE_NATIVE || !d.contiguous || !d.ycontig)
        return KRON_ERR_NOT_SUPPORTED;
    switch (d.N) {
        case 10: return launch_ip_n<10>(d, st);
        case 14: return launch_ip_n<14>(d, st);
        default: return KRON_ERR_NOT_SUPPORTED;
    }
}

}  // namespace kron
