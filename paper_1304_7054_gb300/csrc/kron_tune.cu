// Kernel-configuration table and autotuner for the fixed-size kernels.
//
// A configuration is (kernel body, instances per tile, bulk-copy pipeline
// depth, fibers per step of the last contraction, compute warps per CTA) for
// one (kind, n, storage type, compute mode).  kron_autotune_config times the
// candidates on the caller's buffers with CUDA events and keeps the fastest;
// the table can be persisted in a small text file named by the KRON_TUNE_CACHE
// environment variable (one line per entry: device-key kind n io comp P depth
// variant fps warps, the key being GPU name, SM count and driver version; a
// later line overrides an earlier one and all zeros mean the built-in default),
// read at first use.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "kron_internal.h"

namespace kron {

namespace {

using Key = std::tuple<int, int, int, int>;   // kind, n, io, comp
struct Entry { int P, nstage, variant, fps, warps; };

std::mutex g_mu;
std::map<Key, Entry> g_table;
bool g_loaded = false;

// Cache key of this GPU: name, SM count and driver version (a tuning result
// holds for one chip configuration and one driver).
std::string device_key() {
    int dev = 0, drv = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
    cudaDriverGetVersion(&drv);
    std::string s = prop.name;
    for (char& c : s)
        if (c == ' ') c = '_';
    return s + ":" + std::to_string(prop.multiProcessorCount) + ":" + std::to_string(drv);
}

void load_cache_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char* path = getenv("KRON_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    const std::string me = device_key();
    char line[512], name[256];
    while (fgets(line, sizeof(line), f)) {
        int kind, n, io, comp, P, ns, var = 0, fps = 0, warps = 0;
        const int got = sscanf(line, "%255s %d %d %d %d %d %d %d %d %d", name, &kind, &n, &io, &comp, &P, &ns, &var,
                               &fps, &warps);
        if (got < 7 || me != name) continue;
        if (P == 0 && ns == 0 && var == 0 && fps == 0 && warps == 0)
            g_table.erase(Key(kind, n, io, comp));   // a later tuning kept the default
        else
            g_table[Key(kind, n, io, comp)] = Entry{P, ns, var, fps, warps};
    }
    fclose(f);
}

void append_cache(const Key& k, const Entry& e) {
    const char* path = getenv("KRON_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %d %d %d %d\n", device_key().c_str(), std::get<0>(k), std::get<1>(k), std::get<2>(k),
            std::get<3>(k), e.P, e.nstage, e.variant, e.fps, e.warps);
    fclose(f);
}

bool real_io(kron_dtype io) { return io == KRON_R32F || io == KRON_R64F || io == KRON_R16BF || io == KRON_R16F; }

// Whether kernel body `variant` exists for (kind, n, io, comp) and takes tile size P.
bool variant_ok(int kind, int n, kron_dtype io, kron_compute comp, int variant, int P) {
    if (variant == KRON_VARIANT_AUTO) return true;
    if (kind == 2 && comp == KRON_COMPUTE_32F_BF16X3 && real_io(io) && io != KRON_R64F) {
        // 2-D split tensor bodies: one padded 16 x 16 tile per instance (in place:
        // the second product takes the first's accumulators), or instances
        // stacked along the MMA's N dimension through exchange rows (9 <= n <= 16)
        if (variant == KRON_VARIANT_IN_PLACE) return true;
        return variant == KRON_VARIANT_EXCHANGE && n >= 9;
    }
    if (comp != KRON_COMPUTE_NATIVE || !real_io(io)) return false;
    const bool f32 = io == KRON_R32F, half = io == KRON_R16BF || io == KRON_R16F;
    switch (variant) {
        case KRON_VARIANT_IN_PLACE:
            if (kind == 2 && n == 16 && f32) return P == 0 || P == 16 || P == 24 || P == 32 || P == 8;
            if (kind == 2 && n == 16 && half) return P == 0 || P == 16;
            if (!f32) return false;
            if (kind == 2 && (n == 10 || n == 14)) return P % 8 == 0;
            if (kind == 3 && n == 16) return P <= 1;
            if (kind == 3 && (n == 10 || n == 14)) return P == 0 || P == 4;
            if ((n & 1) && n >= 3) return P % 4 == 0;
            return false;
        case KRON_VARIANT_EXCHANGE: return (n % 2 == 0) && (f32 || half);
        case KRON_VARIANT_SCALAR: return true;
        default: return false;
    }
}

// Whether `warps` compute warps per CTA fit the body (0: its default): the FP32
// 2-D n = 16 in-place body (groups of P / 4 warps, at most 16) and the 3-D split
// tensor body (1, 2, 4 or 8 warps per instance).
bool warps_ok(int kind, int n, kron_dtype io, kron_compute comp, int variant, int P, int warps) {
    if (warps == 0) return true;
    if (kind == 3 && comp == KRON_COMPUTE_32F_BF16X3)   // warps sharing one instance
        return warps == 1 || warps == 2 || warps == 4 || warps == 8;
    if (kind == 2 && (n == 10 || n == 14 || ((n & 1) && n >= 3)) && io == KRON_R32F && comp == KRON_COMPUTE_NATIVE &&
        (variant == KRON_VARIANT_AUTO || variant == KRON_VARIANT_IN_PLACE))   // groups of four warps
        return warps % 4 == 0 && warps <= 16;
    if (kind != 2 || n != 16 || io != KRON_R32F || comp != KRON_COMPUTE_NATIVE) return false;
    if (variant != KRON_VARIANT_AUTO && variant != KRON_VARIANT_IN_PLACE) return false;
    const int g = (P > 0 ? P : kPair16TDefaultP) / 4;
    return warps <= kPair16TMaxWarps && warps % g == 0;
}

Entry entry_of(const kron_kernel_config& c) {
    return Entry{c.instances_per_tile, c.pipeline_depth, c.variant, c.fibers_per_step, c.compute_warps};
}
bool is_default(const Entry& e) { return !e.P && !e.nstage && !e.variant && !e.fps && !e.warps; }

// Stores e for key k (all zero: removes the entry, i.e. the built-in default).
void put_locked(const Key& k, const Entry& e) {
    if (is_default(e))
        g_table.erase(k);
    else
        g_table[k] = e;
}

}  // namespace

void apply_tile_config(KronDesc& d) {
    std::lock_guard<std::mutex> lock(g_mu);
    load_cache_locked();
    auto it = g_table.find(Key(d.D, d.N, (int)d.io, (int)d.comp));
    if (it != g_table.end()) {
        if (d.P <= 0) d.P = it->second.P;
        if (d.nstage < 0) d.nstage = it->second.nstage > 0 ? it->second.nstage : -1;
        d.variant = it->second.variant;
        d.fps = it->second.fps;
        d.warps = it->second.warps;
    }
}

void tune_cache_append(int kind, int n, kron_dtype io, kron_compute comp, int P, int nstage) {
    std::lock_guard<std::mutex> lock(g_mu);
    append_cache(Key(kind, n, (int)io, (int)comp), Entry{P, nstage, 0, 0, 0});
}

}  // namespace kron

using namespace kron;

extern "C" {

KRON_API kron_status kron_set_kernel_config(int kind, int n, kron_dtype io, kron_compute comp,
                                            const kron_kernel_config* c) {
    if (!c || (kind != 2 && kind != 3) || n < 1 || n > kMaxN || c->instances_per_tile < 0 ||
        c->instances_per_tile > 4096 || c->pipeline_depth < 0 || c->pipeline_depth > kPair16TMaxRing ||
        c->fibers_per_step < 0 || c->fibers_per_step > 2 || c->variant < 0 || c->variant > KRON_VARIANT_SCALAR ||
        c->compute_warps < 0 || c->compute_warps > kPair16TMaxWarps)
        return KRON_ERR_INVALID_VALUE;
    if (!variant_ok(kind, n, io, comp, c->variant, c->instances_per_tile) ||
        !warps_ok(kind, n, io, comp, c->variant, c->instances_per_tile, c->compute_warps))
        return KRON_ERR_NOT_SUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    load_cache_locked();
    put_locked(Key(kind, n, (int)io, (int)comp), entry_of(*c));
    return KRON_OK;
}

KRON_API kron_status kron_get_kernel_config(int kind, int n, kron_dtype io, kron_compute comp, kron_kernel_config* c) {
    if (!c) return KRON_ERR_INVALID_VALUE;
    std::lock_guard<std::mutex> lock(g_mu);
    load_cache_locked();
    auto it = g_table.find(Key(kind, n, (int)io, (int)comp));
    const Entry e = it == g_table.end() ? Entry{0, 0, 0, 0, 0} : it->second;
    c->variant = e.variant;
    c->instances_per_tile = e.P;
    c->pipeline_depth = e.nstage;
    c->fibers_per_step = e.fps;
    c->compute_warps = e.warps;
    return KRON_OK;
}

KRON_API kron_status kron_set_tile_config(int kind, int n, kron_dtype io, kron_compute comp, int instances_per_tile,
                                          int pipeline_depth) {
    if ((kind != 2 && kind != 3) || n < 1 || n > kMaxN || instances_per_tile < 0 || pipeline_depth < 0 ||
        pipeline_depth > 8 || instances_per_tile > 4096)
        return KRON_ERR_INVALID_VALUE;
    std::lock_guard<std::mutex> lock(g_mu);
    load_cache_locked();
    put_locked(Key(kind, n, (int)io, (int)comp), Entry{instances_per_tile, pipeline_depth, 0, 0, 0});
    return KRON_OK;
}

KRON_API kron_status kron_get_tile_config(int kind, int n, kron_dtype io, kron_compute comp,
                                          int* instances_per_tile, int* pipeline_depth) {
    if (!instances_per_tile || !pipeline_depth) return KRON_ERR_INVALID_VALUE;
    kron_kernel_config c;
    kron_get_kernel_config(kind, n, io, comp, &c);
    *instances_per_tile = c.instances_per_tile;
    *pipeline_depth = c.pipeline_depth;
    return KRON_OK;
}

KRON_API kron_status kron_autotune_config(kron_stream_t stream, int kind, int n, int64_t batch_count, const void* X,
                                          void* Y, kron_dtype io, kron_compute comp, kron_kernel_config* out) {
    if ((kind != 2 && kind != 3) || n < 1 || n > kMaxN || batch_count < 1 || !X || !Y) return KRON_ERR_INVALID_VALUE;
    cudaStream_t st = (cudaStream_t)stream;
    // Components do not change the timing; identity keeps the outputs finite.
    // Buffers hold (re, im) pairs so that they also serve complex storage.
    const bool dbl = io == KRON_R64F || io == KRON_C64F;
    const int w = is_complex(io) ? 2 : 1;
    double eye[2 * kMaxN * kMaxN] = {};
    float eyef[2 * kMaxN * kMaxN] = {};
    for (int i = 0; i < n; ++i) eye[w * (i + n * i)] = eyef[w * (i + n * i)] = 1.0f;
    const void* comp_ptr = dbl ? (const void*)eye : (const void*)eyef;
    const double one[2] = {1.0, 0.0}, zero[2] = {0.0, 0.0};
    const float onef[2] = {1.0f, 0.0f}, zerof[2] = {0.0f, 0.0f};
    const void* al = dbl ? (const void*)one : (const void*)onef;
    const void* be = dbl ? (const void*)zero : (const void*)zerof;
    auto run = [&]() -> kron_status {
        if (kind == 2)
            return kron2_batched(stream, 'N', 'N', 'N', n, n, n, n, batch_count, al, comp_ptr, n, comp_ptr, n, X, n,
                                 (int64_t)n * n, be, Y, n, (int64_t)n * n, io, comp);
        return kron3_batched(stream, 'N', 'N', 'N', n, n, n, n, n, n, batch_count, al, comp_ptr, n, comp_ptr, n,
                             comp_ptr, n, X, n, n * n, (int64_t)n * n * n, be, Y, n, n * n, (int64_t)n * n * n, io,
                             comp);
    };
    kron_kernel_config prev;
    kron_get_kernel_config(kind, n, io, comp, &prev);
    // Candidates: the built-in default first; then every body that exists for
    // this configuration with tiles of half, one, two and four times "one
    // fiber per thread" (the in-place bodies: their own tile shapes), pipeline
    // depths 1 and 2, and for the packed-pair bodies one or two fibers per step.
    std::vector<kron_kernel_config> cands;
    cands.push_back(kron_kernel_config{0, 0, 0, 0, 0});
    const int base = kind == 2 ? (256 + n - 1) / n : (256 + n * n - 1) / (n * n);
    for (int var = KRON_VARIANT_IN_PLACE; var <= KRON_VARIANT_SCALAR; ++var) {
        if (!variant_ok(kind, n, io, comp, var, 0) && var != KRON_VARIANT_IN_PLACE) continue;
        std::vector<int> tiles;
        if (var == KRON_VARIANT_IN_PLACE) {
            for (int P : {0, 4, 8, 12, 16, 24, 32})
                if (variant_ok(kind, n, io, comp, var, P) && (P == 0 || (n & 1) || (kind == 2 && n != 16)))
                    tiles.push_back(P);
        } else {
            for (int mul2 : {1, 2, 4, 8}) tiles.push_back(std::max(1, base * mul2 / 2));
        }
        for (int P : tiles)
            for (int ns : {1, 2})
                for (int fps : {1, 2}) {
                    if (fps == 2 && var != KRON_VARIANT_EXCHANGE) continue;
                    cands.push_back(kron_kernel_config{var, P, ns, var == KRON_VARIANT_EXCHANGE ? fps : 0, 0});
                }
    }
    if (kind == 2 && n == 16 && io == KRON_R32F && comp == KRON_COMPUTE_NATIVE) {
        // The tensor-copy in-place body: tile, ring depth and compute warps
        // (registers against shared memory: a deeper ring leaves room for
        // fewer resident warps).
        const int shapes[][3] = {{32, 5, 16}, {32, 4, 16}, {32, 3, 8}, {16, 8, 16}, {16, 6, 12},
                                 {16, 4, 8},  {24, 3, 12}, {24, 6, 12}, {8, 8, 8}};
        for (const auto& s : shapes) cands.push_back(kron_kernel_config{KRON_VARIANT_IN_PLACE, s[0], s[1], 0, s[2]});
    }
    if (comp != KRON_COMPUTE_NATIVE || !real_io(io)) {   // one body: tile and depth (2-D), warps (3-D)
        cands.resize(1);
        if (kind == 3 && comp == KRON_COMPUTE_32F_BF16X3) {
            for (int w : {1, 2, 4, 8}) cands.push_back(kron_kernel_config{0, 0, 0, 0, w});
        } else {
            if (kind == 2 && comp == KRON_COMPUTE_32F_BF16X3 && real_io(io)) {
                // the 2-D split tensor bodies (padded tile; stacked for 9 <= n <= 16):
                // tiles of half to four times "one instance per thread" and of 32-128
                // instances, one to three tiles in flight
                // (the stacked body also with one or two groups per warp step: fibers_per_step)
                for (int var : {(int)KRON_VARIANT_IN_PLACE, (int)KRON_VARIANT_EXCHANGE}) {
                    if (!variant_ok(kind, n, io, comp, var, 0)) continue;
                    for (int fps : {0, 1, 2}) {
                        if (fps && (var != KRON_VARIANT_EXCHANGE || n % 2)) continue;
                        for (int P : {0, base / 2, base, 2 * base, 4 * base, 32, 64, 128})
                            for (int ns : {1, 2, 3})
                                if (P > 0 || ns == 1)
                                    cands.push_back(kron_kernel_config{var, P > 0 ? P : 0, P > 0 ? ns : 0, fps, 0});
                    }
                }
            } else {
                for (int mul2 : {1, 2, 4, 8})
                    for (int ns : {1, 2}) cands.push_back(kron_kernel_config{0, std::max(1, base * mul2 / 2), ns, 0, 0});
            }
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return KRON_ERR_CUDA;
    float best = 1e30f, t_default = 1e30f;
    kron_kernel_config best_c{0, 0, 0, 0, 0};
    kron_status rs = KRON_OK;
    for (const kron_kernel_config& c : cands) {
        {
            std::lock_guard<std::mutex> lock(g_mu);
            put_locked(Key(kind, n, (int)io, (int)comp), entry_of(c));
        }
        if (run() != KRON_OK) continue;   // not available at this size (e.g. shared memory)
        float t = 1e30f;
        for (int round = 0; round < 2; ++round) {
            cudaEventRecord(e0, st);
            for (int r = 0; r < 5; ++r) run();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rs = KRON_ERR_CUDA; break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            t = std::min(t, ms);
        }
        if (rs != KRON_OK) break;
        if (is_default(entry_of(c))) t_default = t;
        if (t < best) { best = t; best_c = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs != KRON_OK) {
        kron_set_kernel_config(kind, n, io, comp, &prev);
        return rs;
    }
    if (best > 0.98f * t_default) best_c = kron_kernel_config{0, 0, 0, 0, 0};   // not clearly better: keep the default
    {
        std::lock_guard<std::mutex> lock(g_mu);
        const Entry e = entry_of(best_c);
        put_locked(Key(kind, n, (int)io, (int)comp), e);
        append_cache(Key(kind, n, (int)io, (int)comp), e);   // all zero records "default kept"
    }
    if (out) *out = best_c;
    return KRON_OK;
}

KRON_API kron_status kron_autotune(kron_stream_t stream, int kind, int n, int64_t batch_count, const void* X, void* Y,
                                   kron_dtype io, kron_compute comp, int* instances_per_tile, int* pipeline_depth) {
    kron_kernel_config c;
    const kron_status r = kron_autotune_config(stream, kind, n, batch_count, X, Y, io, comp, &c);
    if (r != KRON_OK) return r;
    if (instances_per_tile) *instances_per_tile = c.instances_per_tile;
    if (pipeline_depth) *pipeline_depth = c.pipeline_depth;
    return KRON_OK;
}

}  // extern "C"
