// mg_tune.cu - tile-variant table and the autotuner that fills it.
//
// The FP32 stencil kernels (k_down: sweeps + residual + full weighting, k_up:
// cubic prolongation + correction + sweeps) are compiled in several tile
// shapes (64, 32, 16 or 8 rows of 64 points; one or two spline midpoints per
// prolongation work item).  Which one is fastest depends on the grid size:
// a 2048^2 level has enough 64-row tiles to fill 152 SMs, while a 256^2 level
// has 16 of them; there smaller tiles shorten each block's chain of
// dependent phases, which bounds the kernel's time when SMs sit idle.  All variants give
// bit-identical results, so the table only decides speed.
//
// The table is process-wide, keyed by (kernel kind, grid size, sweep count).
// Entries come from built-in defaults (op-level timings on GB300, see
// default_variant), from
// mg_autotune (CUDA-event timings of every variant on a context's own level
// buffers), or from a cache file that earlier autotuning wrote.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "mg_internal.cuh"
#include "mg_tune.cuh"

namespace mg {

namespace {

using Key = std::tuple<int, int, int>;  // kind, n, nu
std::mutex g_mu;
std::map<Key, int> g_table;
std::atomic<unsigned> g_epoch{1};

int default_variant(int kind, int n, int nu) {
    (void)nu;
    // op-level timings on GB300 (nu = 2): 64-row tiles from 1024^2, 32-row
    // tiles at 512^2, and below that 8-row tiles for the down kernel and
    // 16-row tiles for the up kernel, whose spline halo makes 8 rows dearer;
    // the up kernel's packed FP32x2 spline passes throughout
    if (kind == 0) return n >= 1024 ? 0 : (n == 512 ? 1 : 3);
    return kVariantPacked | (n >= 1024 ? 0 : (n == 512 ? 1 : 2));
}

std::string gpu_tag(int device) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string name(prop.name);
    for (char &ch : name)
        if (ch == ' ' || ch == '\t') ch = '_';
    // the trailing tag names the variant numbering (rows 64 >> (v & 3), bit 2 packed)
    return name + "/" + std::to_string(prop.multiProcessorCount) + "/v8";
}

}  // namespace

int tile_variant(int kind, int n, int nu) {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_table.find(Key(kind, n, nu));
    return it != g_table.end() ? it->second : default_variant(kind, n, nu);
}

void set_tile_variant(int kind, int n, int nu, int variant) {
    std::lock_guard<std::mutex> lock(g_mu);
    const Key k(kind, n, nu);
    auto it = g_table.find(k);
    const int old = it != g_table.end() ? it->second : default_variant(kind, n, nu);
    g_table[k] = variant;
    if (old != variant) g_epoch.fetch_add(1);
}

unsigned tune_epoch() { return g_epoch.load(); }

namespace {
std::atomic<int> g_overlap{-1};  // -1: not read from the environment yet
}

int launch_overlap_mode() {
    int v = g_overlap.load(std::memory_order_relaxed);
    if (v < 0) {
        const char *env = getenv("MG_LAUNCH_OVERLAP");
        v = (env && (env[0] == '1' || env[0] == '2')) ? env[0] - '0' : 0;
        int expect = -1;
        g_overlap.compare_exchange_strong(expect, v);
        v = g_overlap.load();
    }
    return v;
}

bool launch_overlap_enabled() { return launch_overlap_mode() != 0; }

namespace {
std::atomic<int> g_tma_tiles{0};
}

int tma_tiles_mode() { return g_tma_tiles.load(std::memory_order_relaxed); }

namespace {
std::atomic<int> g_coarse_cluster{1};
}

int coarse_cluster_mode() { return g_coarse_cluster.load(std::memory_order_relaxed); }

void set_coarse_cluster(int on) {
    const int old = g_coarse_cluster.exchange(on ? 1 : 0);
    if (old != (on ? 1 : 0)) g_epoch.fetch_add(1);
}

namespace {
std::atomic<int> g_fp64_x_pass{1};
}

int fp64_separate_x_pass_mode() { return g_fp64_x_pass.load(std::memory_order_relaxed); }

void set_fp64_separate_x_pass(int on) {
    const int old = g_fp64_x_pass.exchange(on ? 1 : 0);
    if (old != (on ? 1 : 0)) g_epoch.fetch_add(1);
}

namespace {
std::atomic<int> g_fused_update{1};
}

int fused_update_mode() { return g_fused_update.load(std::memory_order_relaxed); }

void set_fused_update(int on) {
    const int old = g_fused_update.exchange(on ? 1 : 0);
    if (old != (on ? 1 : 0)) g_epoch.fetch_add(1);
}

void set_tma_tiles(int on) {
    const int old = g_tma_tiles.exchange(on ? 1 : 0);
    if (old != (on ? 1 : 0)) g_epoch.fetch_add(1);
}

void set_launch_overlap(int mode) {
    const int old = launch_overlap_mode();
    g_overlap.store(mode);
    if (old != mode) g_epoch.fetch_add(1);
}

namespace {

// Mean time per launch of fn (min over three batches of ten, after warm-up).
template <typename Fn>
cudaError_t time_launches(Fn fn, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float *us) {
    for (int i = 0; i < 3; ++i) {
        cudaError_t e = fn();
        if (e != cudaSuccess) return e;
    }
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaError_t e = cudaEventRecord(e0, s);
        for (int i = 0; i < 10 && e == cudaSuccess; ++i) e = fn();
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) return e;
        best = ms < best ? ms : best;
    }
    *us = best * 100.0f;  // ms per 10 launches -> us per launch
    return cudaSuccess;
}

void read_cache(const char *path, const std::string &tag, std::map<Key, int> *out) {
    FILE *fp = fopen(path, "r");
    if (!fp) return;
    char line[512], gtag[256];
    while (fgets(line, sizeof line, fp)) {
        int kind, n, nu, v;
        float us;
        if (sscanf(line, "%255s %d %d %d %d %f", gtag, &kind, &n, &nu, &v, &us) == 6 && tag == gtag &&
            kind >= 0 && kind <= 1 && v >= 0 && v < kTileVariants)
            (*out)[Key(kind, n, nu)] = v;
    }
    fclose(fp);
}

}  // namespace

mg_status tune_levels(const TuneLevel *lv, int nlev, int nu1, int nu2, const FirTaps &taps, cudaStream_t s,
                      int device, const char *cache_path, int *n_timed, char *err, size_t errlen) {
    const std::string tag = gpu_tag(device);
    std::map<Key, int> cached;
    if (cache_path) read_cache(cache_path, tag, &cached);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    FILE *fp = nullptr;
    int timed = 0;
    for (int l = 0; l < nlev && ce == cudaSuccess; ++l) {
        const TuneLevel &L = lv[l];
        for (int kind = 0; kind < 2 && ce == cudaSuccess; ++kind) {
            const int nu = kind == 0 ? nu1 : nu2;
            auto hit = cached.find(Key(kind, L.n, nu));
            if (hit != cached.end()) {
                set_tile_variant(kind, L.n, nu, hit->second);
                continue;
            }
            int best_v = -1;
            float best_us = 1e30f;
            for (int v = 0; v < kTileVariants && ce == cudaSuccess; ++v) {
                if (kind == 0 && variant_runs(v) != 1) continue;  // k_down has no spline pass
                float us = 0.f;
                if (kind == 0)
                    ce = time_launches([&] { return launch_down<float>(L.x, L.t, L.b, L.n, nu, false, L.bc, s, v); },
                                       s, e0, e1, &us);
                else
                    ce = time_launches(
                        [&] { return launch_up<float>(L.t, L.x, L.b, L.xc, L.n, nu, taps, s, nullptr, v); }, s, e0,
                        e1, &us);
                if (ce == cudaSuccess && us < best_us) {
                    best_us = us;
                    best_v = v;
                }
            }
            if (ce != cudaSuccess) break;
            set_tile_variant(kind, L.n, nu, best_v);
            ++timed;
            if (cache_path) {
                if (!fp) fp = fopen(cache_path, "a");
                if (fp) fprintf(fp, "%s %d %d %d %d %.3f\n", tag.c_str(), kind, L.n, nu, best_v, best_us);
            }
        }
    }
    if (fp) fclose(fp);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (n_timed) *n_timed = timed;
    if (ce != cudaSuccess) {
        snprintf(err, errlen, "autotune: %s", cudaGetErrorString(ce));
        cudaGetLastError();
        return MG_ERR_CUDA;
    }
    return MG_OK;
}

}  // namespace mg
