// 3-D FP32 pair kernels (n = 16; n = 10, 14 further down) with all three mode
// contractions done in place in the operand tile.
//
// The contractions are those of the generic 3-D pair kernel (Sec. 2.1, the
// order of Algorithm 1 with the intermediates on chip): mode 3 with M3 and mode
// 2 with M2 as pairs of fibers (duplicated coefficients), then mode 1 with M1
// as pairs of output rows.  Each stage reads its fibers into registers and
// writes the results back over the same words, so one 16.3 KB buffer per
// instance is all the shared memory a tile needs (the generic kernel needs two
// extra exchange buffers):
//
//   element (i, j, k) of the instance sits at word i + 16 j + 260 k.
//   Planes arrive and leave as one 1 KB bulk copy (TMA) each; 260 words is a
//   multiple of 4 (16-byte aligned planes) and 4 mod 32, and with the thread
//   mappings below every shared access of every stage touches distinct banks:
//     stage A (mode 3): a half-warp = 8 row pairs x 2 columns j
//     stage B (mode 2): a half-warp = 2 row pairs x 8 planes k
//     stage C (mode 1): a quarter-warp = 2 columns j x 4 planes k (16-byte
//                       accesses of a whole fiber)
//   Results leave by bulk copy, so L2 receives whole lines.
//
// One producer warp streams instances in and results out through a ring of
// buffers (full / empty mbarriers); the four compute warps issue no global
// memory access except the reads of Y that beta != 0 needs.
#include <algorithm>

#include "kron_pair.cuh"

namespace kron {

namespace {

constexpr int kN = 16, kNX = 4096;
constexpr int kPlane = 260;                 // words between planes
constexpr int kInstWords = 16 * kPlane;     // one buffer
constexpr int kCompute = 128;
constexpr int kThreads = kCompute + 32;
constexpr int kMaxRing = 4;

__device__ __forceinline__ int at(int i, int j, int k) { return i + 16 * j + kPlane * k; }

__global__ void __launch_bounds__(kThreads) pair3ip_kernel(const __grid_constant__ PairArgs<kN, 3> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kMaxRing;
    float* ring = reinterpret_cast<float*>(smem + 128);
    const int NB = a.nstage;
    const int tid = threadIdx.x;
    const int64_t ntiles = a.batch;   // one instance per tile
    const int64_t grid = gridDim.x;

    if (tid == 0) {
        for (int s = 0; s < NB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kCompute);
        }
        fence_barrier_init();
    }
    __syncthreads();

    if (tid >= kCompute) {
        // Producer: instance `it` goes to buffer it % NB once the compute threads
        // have released the buffer's previous instance, whose results are stored
        // first (16 planes each way, one lane per plane).
        const int lane = tid - kCompute;
        const uint64_t pol = l2_evict_first_policy();
        float* Y = static_cast<float*>(a.Y);
        const float* X = static_cast<const float*>(a.X);
        auto store_inst = [&](int s, int64_t p) {
            if (lane < 16) bulk_s2g_hint(Y + p * kNX + 256 * lane, ring + s * kInstWords + kPlane * lane, 1024u, pol);
            bulk_commit();
        };
        int it = 0;
        for (int64_t p = blockIdx.x; p < ntiles; p += grid, ++it) {
            const int s = it % NB;
            if (it >= NB) {
                if (!mbar_wait_bounded(&empty[s], (unsigned)(it / NB - 1) & 1u, a.err)) {
                    bulk_wait_all();
                    return;
                }
                store_inst(s, p - (int64_t)NB * grid);
                bulk_wait_read();
            }
            fence_proxy_async_smem();
            if (lane == 0) mbar_arrive_expect_tx(&full[s], 16u * 1024u);
            __syncwarp();
            if (lane < 16)
                bulk_g2s(ring + s * kInstWords + kPlane * lane, X + p * kNX + 256 * lane, 1024u, &full[s], pol);
        }
        for (int j = it > NB ? it - NB : 0; j < it; ++j) {
            if (!mbar_wait_bounded(&empty[j % NB], (unsigned)(j / NB) & 1u, a.err)) break;
            store_inst(j % NB, blockIdx.x + (int64_t)j * grid);
        }
        bulk_wait_all();
        return;
    }

    const f2* m1p = reinterpret_cast<const f2*>(a.m1);
    const float* Yg = static_cast<const float*>(a.Y);
    int it = 0;
    for (int64_t p = blockIdx.x; p < ntiles; p += grid, ++it) {
        const int s = it % NB;
        float* buf = ring + s * kInstWords;
        const bool ok = mbar_wait_bounded(&full[s], (unsigned)(it / NB) & 1u, a.err);

        // Stage A (mode 3): rows (2ip, 2ip+1) of column j, all planes.
        {
            const int ip = tid & 7, j = tid >> 3;
            float* q = buf + at(2 * ip, j, 0);
            f2 x[kN], t[kN];
#pragma unroll
            for (int k = 0; k < kN; ++k) x[k] = *reinterpret_cast<const f2*>(q + kPlane * k);
            contract_dup<kN>(a.da, x, t);
#pragma unroll
            for (int k = 0; k < kN; ++k) *reinterpret_cast<f2*>(q + kPlane * k) = t[k];
        }
        if (compute_sync_or(!ok)) {
            // A copy did not land in time: wait (bounded) for the ones that may still
            // be in flight into this CTA's buffers, then give up.
            if (tid == 0)
                for (int j = it; j < it + NB; ++j)
                    if (blockIdx.x + (int64_t)j * grid < ntiles)
                        mbar_wait_bounded(&full[j % NB], (unsigned)(j / NB) & 1u, a.err);
            return;
        }
        // Stage B (mode 2): rows (2ip, 2ip+1) of plane k, all columns.
        {
            const int r = tid & 15, g = tid >> 4;
            const int ip = 2 * (g & 3) + (r >> 3), k = 8 * (g >> 2) + (r & 7);
            float* q = buf + at(2 * ip, 0, k);
            f2 x[kN], u[kN];
#pragma unroll
            for (int m = 0; m < kN; ++m) x[m] = *reinterpret_cast<const f2*>(q + 16 * m);
            contract_dup<kN>(a.db, x, u);
#pragma unroll
            for (int m = 0; m < kN; ++m) *reinterpret_cast<f2*>(q + 16 * m) = u[m];
        }
        compute_sync_or(false);
        // Stage C (mode 1): the fiber (:, j, k), as pairs of output rows.
#pragma unroll 1
        for (int f = tid; f < 256; f += kCompute) {
            const int qq = f & 7, g = f >> 3;
            const int j = 2 * (g & 7) + (qq >> 2), k = 4 * (g >> 3) + (qq & 3);
            float* q = buf + at(0, j, k);
            float w[kN];
#pragma unroll
            for (int c = 0; c < kN / 4; ++c) {
                const float4 v = *reinterpret_cast<const float4*>(q + 4 * c);
                w[4 * c] = v.x;
                w[4 * c + 1] = v.y;
                w[4 * c + 2] = v.z;
                w[4 * c + 3] = v.w;
            }
            f2 y[kN / 2];
            contract_rows<kN>(m1p, w, y);
            if (!a.alpha_one) {
                const f2 al = f2_pack(a.alpha, a.alpha);
#pragma unroll
                for (int r2 = 0; r2 < kN / 2; ++r2) y[r2] = fmul2(y[r2], al);
            }
            if (!a.beta_zero) {
                const float* yg = Yg + p * kNX + 16 * j + 256 * k;
                const f2 be = f2_pack(a.beta, a.beta);
#pragma unroll
                for (int r2 = 0; r2 < kN / 2; ++r2) y[r2] = ffma2(be, load_pair<float>(yg + 2 * r2), y[r2]);
            }
#pragma unroll
            for (int c = 0; c < kN / 4; ++c)
                *reinterpret_cast<uint4*>(q + 4 * c) = make_uint4(
                    (unsigned)y[2 * c], (unsigned)(y[2 * c] >> 32), (unsigned)y[2 * c + 1], (unsigned)(y[2 * c + 1] >> 32));
        }
        fence_proxy_async_smem();   // results written: visible to the bulk stores
        mbar_arrive(&empty[s]);
    }
}

size_t pair3ip_smem_bytes(int nb) { return 128 + (size_t)nb * kInstWords * sizeof(float); }

// ---------------------------------------------------------------------------
// n = 10, 14: the same three in-place stages on tiles of 4 packed instances
// (instance q at word n^3 q, element (i, j, k) at i + n j + n^2 k), one bulk
// copy per tile each way.  n^3 = 8 or 24 mod 32 for these n, so with the
// instance index fastest in every stage's thread mapping the four instances of
// a group land 8 banks apart; the model of the three access patterns (checked
// on the host) gives 1.18 (n = 10) and 1.13 (n = 14) times the conflict-free
// wavefront count, all of it in stage B.
// ---------------------------------------------------------------------------
constexpr int kPkP = 4;   // instances per tile

template <int N>
__global__ void __launch_bounds__(kThreads, 4) pair3pk_kernel(const __grid_constant__ PairArgs<N, 3> a) {
    constexpr int NX = N * N * N, H = N / 2;
    constexpr int UA = kPkP * H * N, UC = kPkP * N * N;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kMaxRing;
    float* ring = reinterpret_cast<float*>(smem + 128);
    const int NB = a.nstage;
    const int tid = threadIdx.x;
    const int64_t ntiles = (a.batch + kPkP - 1) / kPkP;
    const int64_t grid = gridDim.x;
    if (tid == 0) {
        for (int s = 0; s < NB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kCompute);
        }
        fence_barrier_init();
    }
    __syncthreads();

    if (tid >= kCompute) {   // producer
        const int lane = tid - kCompute;
        const uint64_t pol = l2_evict_first_policy();
        float* Y = static_cast<float*>(a.Y);
        const float* X = static_cast<const float*>(a.X);
        auto store_tile = [&](int s, int64_t t) {
            const int64_t i0 = t * kPkP;
            const int c = (int)min((int64_t)kPkP, a.batch - i0);
            if (lane == 0) bulk_s2g_hint(Y + i0 * NX, ring + s * kPkP * NX, (unsigned)c * NX * 4u, pol);
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
            const int64_t i0 = tile * kPkP;
            const int cnt = (int)min((int64_t)kPkP, a.batch - i0);
            fence_proxy_async_smem();
            if (lane == 0) {
                const unsigned bytes = (unsigned)cnt * NX * 4u;
                mbar_arrive_expect_tx(&full[s], bytes);
                bulk_g2s(ring + s * kPkP * NX, X + i0 * NX, bytes, &full[s], pol);
            }
        }
        for (int j = it > NB ? it - NB : 0; j < it; ++j) {
            if (!mbar_wait_bounded(&empty[j % NB], (unsigned)(j / NB) & 1u, a.err)) break;
            store_tile(j % NB, blockIdx.x + (int64_t)j * grid);
        }
        bulk_wait_all();
        return;
    }

    const f2* m1p = reinterpret_cast<const f2*>(a.m1);
    const float* Yg = static_cast<const float*>(a.Y);
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
        const int s = it % NB;
        float* buf = ring + s * kPkP * NX;
        const int64_t i0 = tile * kPkP;
        const int cnt = (int)min((int64_t)kPkP, a.batch - i0);
        const bool ok = mbar_wait_bounded(&full[s], (unsigned)(it / NB) & 1u, a.err);
        // Stage A (mode 3): rows (2ip, 2ip+1) of column j of instance q, all planes.
#pragma unroll 1
        for (int u = tid; u < UA; u += kCompute) {
            const int q = u % kPkP, ip = (u / kPkP) % H, j = u / (kPkP * H);
            if (q >= cnt) continue;
            float* p = buf + q * NX + 2 * ip + N * j;
            f2 x[N], t[N];
#pragma unroll
            for (int k = 0; k < N; ++k) x[k] = *reinterpret_cast<const f2*>(p + N * N * k);
            contract_dup<N>(a.da, x, t);
#pragma unroll
            for (int k = 0; k < N; ++k) *reinterpret_cast<f2*>(p + N * N * k) = t[k];
        }
        if (compute_sync_or(!ok)) {
            if (tid == 0)
                for (int j = it; j < it + NB; ++j)
                    if (blockIdx.x + (int64_t)j * grid < ntiles)
                        mbar_wait_bounded(&full[j % NB], (unsigned)(j / NB) & 1u, a.err);
            return;
        }
        // Stage B (mode 2): rows (2ip, 2ip+1) of plane k of instance q, all columns.
#pragma unroll 1
        for (int u = tid; u < UA; u += kCompute) {
            const int q = u % kPkP, ip = (u / kPkP) % H, k = u / (kPkP * H);
            if (q >= cnt) continue;
            float* p = buf + q * NX + 2 * ip + N * N * k;
            f2 x[N], v[N];
#pragma unroll
            for (int m = 0; m < N; ++m) x[m] = *reinterpret_cast<const f2*>(p + N * m);
            contract_dup<N>(a.db, x, v);
#pragma unroll
            for (int m = 0; m < N; ++m) *reinterpret_cast<f2*>(p + N * m) = v[m];
        }
        compute_sync_or(false);
        // Stage C (mode 1): the fiber (:, j, k) of instance q, as pairs of output rows.
#pragma unroll 1
        for (int f = tid; f < UC; f += kCompute) {
            const int q = f % kPkP, j = (f / kPkP) % N, k = f / (kPkP * N);
            if (q >= cnt) continue;
            float* p = buf + q * NX + N * j + N * N * k;
            float w[N];
#pragma unroll
            for (int c = 0; c < N / 2; ++c) {
                const float2 v = *reinterpret_cast<const float2*>(p + 2 * c);
                w[2 * c] = v.x;
                w[2 * c + 1] = v.y;
            }
            f2 y[N / 2];
            contract_rows<N>(m1p, w, y);
            if (!a.alpha_one) {
                const f2 al = f2_pack(a.alpha, a.alpha);
#pragma unroll
                for (int r2 = 0; r2 < N / 2; ++r2) y[r2] = fmul2(y[r2], al);
            }
            if (!a.beta_zero) {
                const float* yg = Yg + (i0 + q) * NX + N * j + N * N * k;
                const f2 be = f2_pack(a.beta, a.beta);
#pragma unroll
                for (int r2 = 0; r2 < N / 2; ++r2) y[r2] = ffma2(be, load_pair<float>(yg + 2 * r2), y[r2]);
            }
#pragma unroll
            for (int c = 0; c < N / 2; ++c) *reinterpret_cast<f2*>(p + 2 * c) = y[c];
        }
        fence_proxy_async_smem();
        mbar_arrive(&empty[s]);
    }
}

template <int N>
kron_status launch_pk_n(const KronDesc& d, cudaStream_t st) {
    if (d.P > 0 && d.P != kPkP) return KRON_ERR_NOT_SUPPORTED;   // other tiles: generic pair kernel
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    PairArgs<N, 3> a;
    auto dup = [](double x) {
        const float v = (float)x;
        unsigned b;
        memcpy(&b, &v, sizeof(b));
        return ((f2)b << 32) | (f2)b;
    };
    for (int e = 0; e < N * N; ++e) {
        a.da[e] = dup(d.m3[e]);
        a.db[e] = dup(d.m2[e]);
        a.m1[e] = (float)d.m1[e];
    }
    a.X = d.X;
    a.Y = d.Y;
    a.batch = d.batch;
    a.alpha = (float)d.alpha;
    a.beta = (float)d.beta;
    a.beta_zero = d.beta == 0.0;
    a.alpha_one = d.alpha == 1.0;
    a.err = device_error_word();
    if (!a.err) return KRON_ERR_CUDA;
    a.P = kPkP;
    // measured: two buffers at n = 10 (16 KB tiles), one at n = 14 (44 KB tiles,
    // where a second buffer costs resident CTAs)
    int nb = d.nstage >= 1 ? d.nstage : (N == 10 ? 2 : 1);
    if (nb > kMaxRing) nb = kMaxRing;
    auto smem_of = [](int n_b) { return 128 + (size_t)n_b * kPkP * N * N * N * sizeof(float); };
    size_t smem = smem_of(nb);
    while (nb > 1 && smem > dev.smem_per_block_optin) smem = smem_of(--nb);
    if (smem > dev.smem_per_block_optin) return KRON_ERR_NOT_SUPPORTED;
    a.nstage = nb;
    auto kern = pair3pk_kernel<N>;
    if (!ensure_smem_optin((const void*)kern, smem)) return KRON_ERR_CUDA;
    const int64_t ntiles = (d.batch + kPkP - 1) / kPkP;
    int64_t grid = d.grid;
    if (grid <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) != cudaSuccess)
            return KRON_ERR_CUDA;
        grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
    }
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, ntiles));
    kern<<<(unsigned)grid, kThreads, smem, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

}  // namespace

// 3-D FP32 storage and arithmetic, contiguous X and Y: n = 16 with one instance
// per tile, n = 10 and 14 with four (other tile sizes go to the generic pair
// kernel).
kron_status launch_pair3ip(const KronDesc& d, cudaStream_t st) {
    if (d.D != 3 || d.io != KRON_R32F || d.comp != KRON_COMPUTE_NATIVE || !d.contiguous || !d.ycontig)
        return KRON_ERR_NOT_SUPPORTED;
    if (d.N == 10) return launch_pk_n<10>(d, st);
    if (d.N == 14) return launch_pk_n<14>(d, st);
    if (d.N != kN || d.P > 1) return KRON_ERR_NOT_SUPPORTED;
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    PairArgs<kN, 3> a;
    auto dup = [](double x) {
        const float v = (float)x;
        unsigned b;
        memcpy(&b, &v, sizeof(b));
        return ((f2)b << 32) | (f2)b;
    };
    for (int e = 0; e < kN * kN; ++e) {
        a.da[e] = dup(d.m3[e]);
        a.db[e] = dup(d.m2[e]);
        a.m1[e] = (float)d.m1[e];
    }
    a.X = d.X;
    a.Y = d.Y;
    a.batch = d.batch;
    a.alpha = (float)d.alpha;
    a.beta = (float)d.beta;
    a.beta_zero = d.beta == 0.0;
    a.alpha_one = d.alpha == 1.0;
    a.err = device_error_word();
    if (!a.err) return KRON_ERR_CUDA;
    a.P = 1;
    int nb = d.nstage >= 1 ? d.nstage : 2;
    if (nb > kMaxRing) nb = kMaxRing;
    size_t smem = pair3ip_smem_bytes(nb);
    while (nb > 1 && smem > dev.smem_per_block_optin) smem = pair3ip_smem_bytes(--nb);
    a.nstage = nb;
    const void* kern = (const void*)pair3ip_kernel;
    if (!ensure_smem_optin(kern, smem)) return KRON_ERR_CUDA;
    int64_t grid = d.grid;
    if (grid <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair3ip_kernel, kThreads, smem) != cudaSuccess)
            return KRON_ERR_CUDA;
        grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
    }
    if (grid > d.batch) grid = d.batch;
    if (grid < 1) grid = 1;
    pair3ip_kernel<<<(unsigned)grid, kThreads, smem, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

}  // namespace kron
