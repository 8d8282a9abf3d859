// mg_api.cu - context, drivers and the C ABI declared in include/mg.h.
//
// The solve follows the V-cycle iteration of Algorithm 6 (Appendix A) with the
// stopping rule on the relative residual.  MIXED precision wraps FP32
// V-cycles in FP64 defect correction:
//     s = h^2 (f - mean f) - (4x - sum nbrs)    (FP64, = h^2 r; ||r|| = ||s|| / h^2)
//     if ||r|| / ||f - mean f|| <= tol: stop
//     e = V^m(0; float(s))                      (m FP32 V-cycles, scaled rhs)
//     x += e                                    (FP64)
// and the result is projected to zero mean at the end.  The only host
// synchronisation inside the loop is the read-back of the two residual sums.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <new>
#include <utility>
#include <type_traits>
#include <vector>

#include "mg_internal.cuh"
#include "mg_tune.cuh"
#include "mg_sr.cuh"

using namespace mg;

static thread_local char g_err[512] = "";

static void set_err(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

void mg::set_last_error(const char *msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

#define MG_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            set_err("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;               \
        }                                                                                    \
    } while (0)

#define MG_TRY(expr)                    \
    do {                                \
        mg_status s_ = (expr);          \
        if (s_ != MG_OK) return s_;     \
    } while (0)

namespace {

constexpr int kMaxLevels = 16;
constexpr size_t kAlign = 256;

// Per level: the iterate x, a second buffer t for the out-of-place tile
// passes (down: x -> t, up: t -> x), and the scaled right-hand side b.
struct Level {
    int n = 0;
    float *x32 = nullptr, *t32 = nullptr, *b32 = nullptr;
    double *x64 = nullptr, *t64 = nullptr, *b64 = nullptr;
};

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Closed-form pseudo-inverse of the scaled periodic operator 4I - shifts on an
// m x m grid: A~^+[p][q] = (1/m^2) sum_{k != 0} cos(2 pi k.(p - q) / m) / lam(k),
// lam(k) = 4 sin^2(pi kx / m) + 4 sin^2(pi ky / m)  (Fourier eigen-decomposition).
void coarse_pinv_host(int m, double *out) {
    const int Nc = m * m;
    const double PI = 3.14159265358979323846;
    // kernel depends only on the difference (di, dj) mod m
    double *kern = new double[Nc];
    for (int di = 0; di < m; ++di)
        for (int dj = 0; dj < m; ++dj) {
            double acc = 0.0;
            for (int ky = 0; ky < m; ++ky)
                for (int kx = 0; kx < m; ++kx) {
                    if (kx == 0 && ky == 0) continue;
                    const double sx = sin(PI * kx / m), sy = sin(PI * ky / m);
                    const double lam = 4.0 * (sx * sx + sy * sy);
                    acc += cos(2.0 * PI * (double)(kx * dj + ky * di) / m) / lam;
                }
            kern[di * m + dj] = acc / Nc;
        }
    for (int pi = 0; pi < m; ++pi)
        for (int pj = 0; pj < m; ++pj)
            for (int qi = 0; qi < m; ++qi)
                for (int qj = 0; qj < m; ++qj) {
                    const int di = (pi - qi + m) % m, dj = (pj - qj + m) % m;
                    out[(pi * m + pj) * Nc + qi * m + qj] = kern[di * m + dj];
                }
    delete[] kern;
}

bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// One instantiated solve graph: prologue (source sum, first residual, test),
// a WHILE node whose body runs one outer step (V-cycles, update, residual,
// test), and the zero-mean projection.  Keyed by the buffers and the
// prolongation it was recorded with.
struct SolveGraph {
    const double *f = nullptr;
    double *x = nullptr;
    int prolong = -1;
    double tol = 0.0;
    bool xzero = false;  // recorded for a cold start whose kernels do not read x
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long n_pro = 0, n_body = 0, n_epi = 0;  // kernels per part
    long long n_sr = 0;                         // kernels of one conditional SR correction
    long long n_cyc = 0;                        // kernels of one optional (conditional) V-cycle
    int adapt_max = 0;                          // optional cycles recorded: 2 .. adapt_max
    unsigned long long stamp = 0;               // last use (LRU)
    unsigned epoch = 0;                         // tile-variant table at recording
};
constexpr int kGraphCache = 4;

struct mg_ctx {
    int N = 0, levels = 0, coarsest = 0, device = 0;
    mg_precision prec = MG_PREC_MIXED;
    int nu1 = 2, nu2 = 2, max_cycles = 100, inner = 2;
    // adaptive inner cycles of mixed cubic solves: up to adapt_max V-cycles per
    // outer step, chosen from the residual with contraction rho (0: fixed `inner`)
    int adapt_max = 3;
    double rho = 0.06;
    bool zero_guess = false;  // solves start from x = 0 and do not read x (mg_set_zero_guess)
    cudaStream_t stream = nullptr;
    Level lv[kMaxLevels];
    void *h32_block = nullptr, *h64_block = nullptr;
    // scaled right-hand side h^2 (f - mu) of the finest level, FP64, written by
    // each solve's first outer residual (mixed contexts; FP64 ones use lv[0].b64)
    double *bsc64 = nullptr;
    int *ebt = nullptr;  // per residual task of the finest grid: bsc64's alignment exponent (N >= kResMinN)
    // the second FP64 iterate of a mixed solve whose outer steps fuse the
    // update with the next residual (N >= kResMinN): the steps alternate
    // between the solve's x and this buffer
    double *xalt = nullptr;
    // FP64 hierarchies: the coarse error of the level being prolonged, refined
    // along x once ((N/2) x N doubles; launch_refine_rows)
    double *xr64 = nullptr;
    float *ainv32 = nullptr;
    double *ainv64 = nullptr;
    FirTaps taps;
    // reductions: partials, counter, results [4 groups][kMaxSlots]
    double *red_partials = nullptr;
    unsigned *red_counter = nullptr;
    double *red_out = nullptr;
    double *host_out = nullptr;  // pinned mirror of red_out
    double *f_stage = nullptr, *x_stage = nullptr;
    SrState sr;
    SrWindows srw;  // windowed SR mosaic buffers (mg_op_sr_windowed)
    // views of sr's generator for the stages of the two-level SR prolongation
    // (stage j refines level j + 1 to level j)
    static constexpr int kSrStages = 8;
    SrState sr_stage[kSrStages];
    // graph execution
    bool use_graphs = true;
    ProlongPolicy policy = {1, 0, 0.0};  // SR on every V-cycle
    int *d_srflag = nullptr;             // device: the current V-cycle uses SR
    cudaStream_t cap_stream = nullptr;  // private stream used only for recording graphs
    DevState *dstate = nullptr, *hstate = nullptr;
    // 2D tensor maps of each FP32 level's x and b with the TMA-staged k_down
    // tile as box (levels of >= 128 points a side; tm_ok when encoded)
    CUtensorMap tm_x32[kMaxLevels], tm_b32[kMaxLevels];
    bool tm_ok[kMaxLevels] = {};
    SolveGraph graphs[kGraphCache];
    unsigned long long graph_clock = 0;
    // optional CUDA-event probe around one kernel kind (instrumentation)
    int probe_kind = 0, probe_cap = 0, probe_used = 0;
    cudaEvent_t *probe_ev = nullptr;
    double probe_bytes = 0.0;

    Reduction red(int group) const { return Reduction{red_partials, red_counter, red_out + group * kMaxSlots}; }
    double *out(int group) const { return red_out + group * kMaxSlots; }
};

enum { kGrpF = 0, kGrpR = 1, kGrpU = 2, kGrpX = 3 };
enum {
    kProbeNone = 0,
    kProbeDown = 1,
    kProbeUp = 2,
    kProbeResidual = 3,
    kProbeUpdate = 4,
    kProbeCoarse = 5,
    kProbeUpdateResidual = 6
};

// Algorithmic bytes of the coarse part of a V-cycle below level l0: 13 B per
// point for each tile kernel (down and up) of every tiled level, and the
// bottom kernel's read of b, read and write of x.
template <typename T>
static double coarse_bytes(const mg_ctx *c, int l0) {
    double by = 0.0;
    for (int l = l0; l < c->levels; ++l) {
        const double nn = (double)c->lv[l].n * c->lv[l].n;
        if (c->lv[l].n > bottom_max<T>()) {
            by += 2.0 * 13.0 * nn * sizeof(T) / 4.0;
        } else {
            by += 3.0 * nn * sizeof(T);
            break;
        }
    }
    return by;
}

static void probe_begin(mg_ctx *c, int kind) {
    if (c->probe_kind == kind && c->probe_used < c->probe_cap)
        cudaEventRecord(c->probe_ev[2 * c->probe_used], c->stream);
}
static void probe_end(mg_ctx *c, int kind, double bytes) {
    if (c->probe_kind == kind && c->probe_used < c->probe_cap) {
        cudaEventRecord(c->probe_ev[2 * c->probe_used + 1], c->stream);
        ++c->probe_used;
        c->probe_bytes += bytes;
    }
}
static void probe_free(mg_ctx *c) {
    for (int i = 0; i < 2 * c->probe_cap; ++i) cudaEventDestroy(c->probe_ev[i]);
    delete[] c->probe_ev;
    c->probe_ev = nullptr;
    c->probe_cap = c->probe_used = 0;
    c->probe_kind = kProbeNone;
    c->probe_bytes = 0.0;
}

static mg_status ensure_hierarchy(mg_ctx *c, bool fp64) {
    void *&blk = fp64 ? c->h64_block : c->h32_block;
    if (blk) return MG_OK;
    const size_t es = fp64 ? sizeof(double) : sizeof(float);
    size_t total = 0;
    for (int l = 0; l < c->levels; ++l) {
        const size_t nn = (size_t)c->lv[l].n * c->lv[l].n;
        total += 3 * align_up(nn * es);
    }
    const size_t bsc_off = total;
    if (!fp64) total += align_up((size_t)c->N * c->N * sizeof(double));
    const size_t ebt_off = total;
    const bool tasks = !fp64 && c->N >= kResMinN;
    if (tasks) total += align_up(res_tasks(c->N) * sizeof(int));
    const size_t xalt_off = total;
    if (tasks) total += align_up((size_t)c->N * c->N * sizeof(double));
    const size_t xr_off = total;
    const bool xr = fp64 && c->N >= 128;
    if (xr) total += align_up((size_t)c->N / 2 * c->N * sizeof(double));
    MG_CUDA(cudaMalloc(&blk, total));
    MG_CUDA(cudaMemsetAsync(blk, 0, total, c->stream));
    char *p = (char *)blk;
    for (int l = 0; l < c->levels; ++l) {
        const size_t nn = (size_t)c->lv[l].n * c->lv[l].n;
        const size_t bytes = align_up(nn * es);
        if (fp64) {
            c->lv[l].x64 = (double *)p;
            c->lv[l].t64 = (double *)(p + bytes);
            c->lv[l].b64 = (double *)(p + 2 * bytes);
        } else {
            c->lv[l].x32 = (float *)p;
            c->lv[l].t32 = (float *)(p + bytes);
            c->lv[l].b32 = (float *)(p + 2 * bytes);
        }
        p += 3 * bytes;
    }
    if (!fp64) c->bsc64 = (double *)((char *)blk + bsc_off);
    if (tasks) {
        c->ebt = (int *)((char *)blk + ebt_off);
        c->xalt = (double *)((char *)blk + xalt_off);
    }
    if (xr) c->xr64 = (double *)((char *)blk + xr_off);
    if (!fp64) {
        int bc = 0, br = 0;
        down_tma_box(2, &bc, &br);
        for (int l = 0; l < c->levels; ++l)
            c->tm_ok[l] = c->lv[l].n >= 128 && make_grid_map_f32(&c->tm_x32[l], c->lv[l].x32, c->lv[l].n, bc, br) &&
                          make_grid_map_f32(&c->tm_b32[l], c->lv[l].b32, c->lv[l].n, bc, br);
    }
    return MG_OK;
}

// Streaming multiprocessors of the current device (queried once).
static int num_sms() {
    static std::atomic<int> sms{0};
    int v = sms.load(std::memory_order_relaxed);
    if (v == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 152;
        }
        sms.store(v, std::memory_order_relaxed);
    }
    return v;
}

// Variant of a batched tile launch over ngrid grids of size sz: the table's
// choice while the launch's 32-row tiles would not fill the GPU once (small
// tiles shorten a lone grid's chain of dependent phases); beyond that the GPU
// is full and smaller tiles only add halo work, so at least 32 rows.
static int batch_variant(int kind, int sz, int nu, int ngrid) {
    int v = tile_variant(kind, sz, nu);
    if (variant_rows(v) < 32 && (long long)ngrid * variant_tiles(sz, 1) >= num_sms()) v = (v & kVariantPacked) | 1;
    return v;
}

// The finest level's scaled right-hand side buffer of a solve.
static double *scaled_rhs(mg_ctx *c, bool mixed) { return mixed ? c->bsc64 : c->lv[0].b64; }

// The outer residual of a solve on stream s.  The solve's first evaluation
// (first) sums (f - mu)^2 and stores b = h^2 (f - mu); later ones load b.
// Mixed solves of N >= kResMinN use the task-tiled kernel (b stored aligned).
static cudaError_t solve_residual(mg_ctx *c, const double *fd, const double *xd, bool mixed, bool first,
                                  double h2, cudaStream_t s, bool xzero = false) {
    const int N = c->N;
    if (mixed && N >= kResMinN)
        return launch_outer_residual_tasks(fd, xd, N, h2, c->out(kGrpF), 0.0, c->lv[0].b32, first,
                                           reinterpret_cast<long long *>(c->bsc64), c->ebt, c->red(kGrpR), s,
                                           xzero);
    if (xzero) return cudaErrorInvalidValue;
    return launch_outer_residual(fd, xd, N, h2, c->out(kGrpF), 0.0, mixed ? c->lv[0].b32 : nullptr, first,
                                 scaled_rhs(c, mixed), !first, c->red(kGrpR), s);
}

// Whether a solve fuses each outer step's update with the next residual.
static bool fused_update(const mg_ctx *c, bool mixed) { return mixed && c->N >= kResMinN && c->xalt && fused_update_mode(); }

// Whether a solve's kernels take the cold start themselves (mg_set_zero_guess
// with the fused outer step): the first residual and the first update treat
// x as zero without reading it, so x is neither zeroed nor copied in.
static bool kernels_take_zero(const mg_ctx *c, bool mixed) { return c->zero_guess && fused_update(c, mixed); }

// The update of outer step k (from 1) fused with the residual that follows
// it; step_dev (the graph's device step counter, k - 1 when the kernel runs)
// or else step_host = k - 1 selects which buffer of (xd, xalt) holds the
// step's x; with xzero step 0 starts from x = 0 without reading it.
static cudaError_t solve_update_residual(mg_ctx *c, double *xd, const int *step_dev, int step_host, bool xzero,
                                         double h2, cudaStream_t s) {
    return launch_update_residual_tasks(xd, c->xalt, step_dev, step_host, xzero, c->lv[0].x32, c->N, h2,
                                        c->lv[0].b32, reinterpret_cast<long long *>(c->bsc64), c->ebt,
                                        c->red(kGrpR), s);
}

template <typename T> static T *lvx(mg_ctx *c, int l);
template <typename T> static T *lvt(mg_ctx *c, int l);
template <typename T> static T *lvb(mg_ctx *c, int l);
template <> float *lvx<float>(mg_ctx *c, int l) { return c->lv[l].x32; }
template <> float *lvt<float>(mg_ctx *c, int l) { return c->lv[l].t32; }
template <> float *lvb<float>(mg_ctx *c, int l) { return c->lv[l].b32; }
template <> double *lvx<double>(mg_ctx *c, int l) { return c->lv[l].x64; }
template <> double *lvt<double>(mg_ctx *c, int l) { return c->lv[l].t64; }
template <> double *lvb<double>(mg_ctx *c, int l) { return c->lv[l].b64; }
template <typename T> static const T *ainv(mg_ctx *c);
template <> const float *ainv<float>(mg_ctx *c) { return c->ainv32; }
template <> const double *ainv<double>(mg_ctx *c) { return c->ainv64; }

// The down pass of level l (x -> t, restricted residual -> bc).  FP32 levels
// on 64-row tiles with V(2, .) take the TMA-staged kernel when TMA tiles are
// on (mg_set_tma_tiles) and the level's maps describe these buffers.
template <typename T>
static cudaError_t down_level(mg_ctx *c, int l, const T *x, T *t, const T *b, bool zero, T *bc, cudaStream_t s) {
    return launch_down<T>(x, t, b, c->lv[l].n, c->nu1, zero, bc, s);
}
template <>
cudaError_t down_level<float>(mg_ctx *c, int l, const float *x, float *t, const float *b, bool zero, float *bc,
                              cudaStream_t s) {
    const int n = c->lv[l].n;
    if (tma_tiles_mode() && c->tm_ok[l] && c->nu1 == 2 && x == c->lv[l].x32 && b == c->lv[l].b32 &&
        variant_rows(tile_variant(0, n, c->nu1)) == 64)
        return launch_down_tma(x, t, b, n, c->nu1, zero, bc, &c->tm_x32[l], &c->tm_b32[l], &c->dstate->tile_err, s);
    return launch_down<float>(x, t, b, n, c->nu1, zero, bc, s);
}

// One V(nu1, nu2) cycle on 4x - sum = b at level l (x = 0 on entry if zero);
// t is the level's second buffer, the result is left in x.
template <typename T>
static mg_status vcycle_rec(mg_ctx *c, int l, T *x, T *t, const T *b, bool zero) {
    const int n = c->lv[l].n;
    if (n <= bottom_max<T>()) {
        MG_CUDA(launch_bottom<T>(x, b, n, c->coarsest, c->nu1, c->nu2, zero, ainv<T>(c), c->taps,
                                 c->stream));
        return MG_OK;
    }
    T *xc = lvx<T>(c, l + 1), *tc = lvt<T>(c, l + 1), *bc = lvb<T>(c, l + 1);
    if constexpr (std::is_same<T, float>::value) {
        // the 128^2 level and the bottom solve below it as one cluster launch
        if (coarse_cluster_mode() && l > 0 && zero && n == 128 && c->lv[l + 1].n <= bottom_max<T>() &&
            c->nu1 == 2 && c->nu2 == 2) {
            MG_CUDA(launch_coarse_cluster(x, t, b, xc, bc, c->coarsest, 2, 2, ainv<T>(c), c->taps, c->stream));
            return MG_OK;
        }
    }
    const double nn = (double)n * n * sizeof(T);
    if (l == 0) probe_begin(c, kProbeDown);
    MG_CUDA(down_level<T>(c, l, x, t, b, zero, bc, c->stream));
    if (l == 0) probe_end(c, kProbeDown, nn * ((zero ? 0 : 1) + 1 + 1 + 0.25));
    if (l == 0) probe_begin(c, kProbeCoarse);
    MG_TRY(vcycle_rec<T>(c, l + 1, xc, tc, bc, true));
    if (l == 0) probe_end(c, kProbeCoarse, coarse_bytes<T>(c, 1));
    if (l == 0) probe_begin(c, kProbeUp);
    const T *xr = nullptr;
    if constexpr (std::is_same<T, double>::value) {
        // the x pass of the prolongation once for the level, not per tile
        if (c->xr64 && fp64_separate_x_pass_mode()) {
            MG_CUDA(launch_refine_rows(xc, c->xr64, n, c->taps, c->stream));
            xr = c->xr64;
        }
    }
    MG_CUDA(launch_up<T>(t, x, b, xc, n, c->nu2, c->taps, c->stream, nullptr, -1, nullptr, xr));
    if (l == 0) probe_end(c, kProbeUp, nn * (2 + (c->nu2 > 0 ? 1 : 0) + 0.25));
    return MG_OK;
}

// Top-level FP32 V-cycle with the chosen prolongation at the finest transition.
static mg_status vcycle32_top(mg_ctx *c, bool zero, mg_prolong prolong) {
    float *x = c->lv[0].x32, *t = c->lv[0].t32, *b = c->lv[0].b32;
    if (prolong == MG_PROLONG_SR && c->levels > 1 && c->lv[0].n > kBottomMax) {
        float *xc = c->lv[1].x32, *tc = c->lv[1].t32, *bc = c->lv[1].b32;
        const double nn = (double)c->lv[0].n * c->lv[0].n * sizeof(float);
        probe_begin(c, kProbeDown);
        MG_CUDA(down_level<float>(c, 0, x, t, b, zero, bc, c->stream));
        probe_end(c, kProbeDown, nn * ((zero ? 0 : 1) + 1 + 1 + 0.25));
        probe_begin(c, kProbeCoarse);
        MG_TRY(vcycle_rec<float>(c, 1, xc, tc, bc, true));
        probe_end(c, kProbeCoarse, coarse_bytes<float>(c, 1));
        // generator correction s * G(e_c / s) on the fine grid, then the cubic
        // part, the correction and the post-smoothing in one up pass
        MG_TRY(sr_correction(&c->sr, xc, c->lv[1].n, c->stream, g_err, sizeof g_err));
        probe_begin(c, kProbeUp);
        MG_CUDA(launch_up<float>(t, x, b, xc, c->lv[0].n, c->nu2, c->taps, c->stream, c->sr.fine_out));
        probe_end(c, kProbeUp, nn * (3 + (c->nu2 > 0 ? 1 : 0) + 0.25));
        return MG_OK;
    }
    return vcycle_rec<float>(c, 0, x, t, b, zero);
}

// Device views of f and x for a call; host buffers are staged into the
// context's device copies.  zero_x: x is output only (a solve from x = 0): a
// host x is not copied in and the device copy, or a device x, is zeroed.
static mg_status resolve_io(mg_ctx *c, const double *f, double *x, const double **fd, double **xd,
                            bool *staged, bool zero_x = false, bool kernels_zero = false) {
    const size_t bytes = (size_t)c->N * c->N * sizeof(double);
    const bool fdev = is_device_pointer(f), xdev = is_device_pointer(x);
    *staged = !xdev;
    // with kernels_zero the solve's kernels take x = 0 without reading x
    zero_x = zero_x && !kernels_zero;
    const bool copy_x = !zero_x && !kernels_zero;
    if (fdev && xdev) {
        *fd = f;
        *xd = x;
        if (zero_x) MG_CUDA(cudaMemsetAsync(x, 0, bytes, c->stream));
        return MG_OK;
    }
    if (!c->f_stage) MG_CUDA(cudaMalloc(&c->f_stage, bytes));
    if (!c->x_stage) MG_CUDA(cudaMalloc(&c->x_stage, bytes));
    if (fdev) {
        *fd = f;
    } else {
        MG_CUDA(cudaMemcpyAsync(c->f_stage, f, bytes, cudaMemcpyHostToDevice, c->stream));
        *fd = c->f_stage;
    }
    if (xdev) {
        *xd = x;
        if (zero_x) MG_CUDA(cudaMemsetAsync(x, 0, bytes, c->stream));
    } else {
        if (zero_x) MG_CUDA(cudaMemsetAsync(c->x_stage, 0, bytes, c->stream));
        else if (copy_x) MG_CUDA(cudaMemcpyAsync(c->x_stage, x, bytes, cudaMemcpyHostToDevice, c->stream));
        *xd = c->x_stage;
    }
    return MG_OK;
}

static mg_status check_common(mg_ctx *c, const double *f, double *x, mg_prolong prolong) {
    if (!c || !f || !x) {
        set_err("null context or pointer");
        return MG_ERR_INVALID_ARG;
    }
    if (prolong != MG_PROLONG_CUBIC && prolong != MG_PROLONG_SR) {
        set_err("unknown prolongation %d", (int)prolong);
        return MG_ERR_INVALID_ARG;
    }
    if (prolong == MG_PROLONG_SR) {
        if (!c->sr.loaded) {
            set_err("SR prolongation requested but no generator weights are loaded");
            return MG_ERR_NO_WEIGHTS;
        }
        if (c->prec != MG_PREC_MIXED) {
            set_err("SR prolongation runs inside the FP32 V-cycle (MG_PREC_MIXED only)");
            return MG_ERR_INVALID_ARG;
        }
    }
    MG_CUDA(cudaSetDevice(c->device));
    return MG_OK;
}

static void drop_graphs(mg_ctx *c) {
    for (SolveGraph &g : c->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        g = SolveGraph();
    }
}

// Record the solve of A x = f for fixed buffers as one graph.  All launches go
// to the private capture stream; on any failure the capture is ended and the
// partial graph destroyed.
// One FP32 V-cycle whose top prolongation the policy chooses, recorded into
// the graph `body` that stream s is capturing: down, the coarse levels, the
// policy kernel, an IF node holding the SR correction, up (which adds the
// correction only when the policy chose SR).  Capture continues after the IF
// node on return.  *n_sr = kernels inside the IF body.
static mg_status record_policy_vcycle(mg_ctx *c, bool zero, int k, cudaGraph_t body, cudaGraphConditionalHandle h,
                                      cudaStream_t s, long long *n_sr) {
    const int n = c->lv[0].n;
    float *x = c->lv[0].x32, *t = c->lv[0].t32, *b = c->lv[0].b32;
    float *xc = c->lv[1].x32, *tc = c->lv[1].t32, *bc = c->lv[1].b32;
    MG_CUDA(down_level<float>(c, 0, x, t, b, zero, bc, s));
    MG_TRY(vcycle_rec<float>(c, 1, xc, tc, bc, true));
    MG_CUDA(launch_policy(c->dstate, k, c->policy, c->d_srflag, h, s));
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    MG_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
    std::vector<cudaGraphNode_t> tail(deps, deps + ndeps);
    MG_CUDA(cudaStreamEndCapture(s, &body));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t ifn;
    MG_CUDA(cudaGraphAddNode(&ifn, body, tail.data(), nullptr, tail.size(), &cp));
    cudaGraph_t ifbody = cp.conditional.phGraph_out[0];
    MG_CUDA(cudaStreamBeginCaptureToGraph(s, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const long long l0 = (long long)launches_total();
    mg_status st = sr_correction(&c->sr, xc, c->lv[1].n, s, g_err, sizeof g_err);
    *n_sr = (long long)launches_total() - l0;
    cudaError_t e = cudaStreamEndCapture(s, &ifbody);
    MG_TRY(st);
    MG_CUDA(e);
    MG_CUDA(cudaStreamBeginCaptureToGraph(s, body, &ifn, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    MG_CUDA(launch_up<float>(t, x, b, xc, n, c->nu2, c->taps, s, c->sr.fine_out, -1, c->d_srflag));
    return MG_OK;
}

static mg_status record_solve_graph(mg_ctx *c, const double *fd, double *xd, mg_prolong prolong,
                                    double tol, SolveGraph *out) {
    const bool mixed = c->prec == MG_PREC_MIXED;
    const int N = c->N;
    const double N2 = (double)N * N;
    const double h = 2.0 * 3.14159265358979323846 / N, h2 = h * h;
    const bool use_policy_ = mixed && prolong == MG_PROLONG_SR && c->levels > 1 && c->lv[0].n > kBottomMax;
    const bool adaptive = mixed && !use_policy_ && c->rho > 0.0 && c->adapt_max > 1;
    const int step = mixed ? (adaptive ? c->adapt_max : c->inner) : 1;
    const double rho = adaptive ? c->rho : 0.0;
    CycleHandles ifh{};
    long long n_cyc = 0;
    cudaStream_t user_stream = c->stream;
    cudaStream_t s = c->cap_stream;
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle handle;
    bool capturing = false;
    mg_status st = MG_OK;
    long long n_pro = 0, n_body = 0, n_epi = 0, n_sr = 0;
    const bool use_policy = mixed && prolong == MG_PROLONG_SR && c->levels > 1 && c->lv[0].n > kBottomMax;
    const bool fuse = fused_update(c, mixed);
    const bool xz = kernels_take_zero(c, mixed);  // cold start: x is not read
    auto fail = [&](cudaError_t e, const char *what) {
        set_err("graph recording (%s) failed: %s", what, cudaGetErrorString(e));
        st = MG_ERR_CUDA;
    };
    c->stream = s;  // the V-cycle helpers launch on c->stream
    do {
        cudaError_t e = cudaGraphCreate(&g, 0);
        if (e != cudaSuccess) { fail(e, "create"); break; }
        e = cudaGraphConditionalHandleCreate(&handle, g, 0, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) { fail(e, "conditional handle"); break; }
        for (int k = 2; adaptive && k <= step && e == cudaSuccess; ++k)
            e = cudaGraphConditionalHandleCreate(&ifh.h[k - 2], g, 0, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) { fail(e, "cycle handles"); break; }
        // prologue
        long long l0 = (long long)launches_total();
        e = cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { fail(e, "begin prologue"); break; }
        capturing = true;
        e = launch_source_sum(fd, N, c->red(kGrpF), s);
        // the first residual also stores the scaled right-hand side b = h^2 (f - mu)
        if (e == cudaSuccess) e = solve_residual(c, fd, xd, mixed, true, h2, s, xz);
        if (e == cudaSuccess)
            e = launch_check(c->dstate, c->out(kGrpR), nullptr, c->out(kGrpF), N2, h2, tol, step,
                             c->max_cycles, true, handle, s, rho, ifh);
        if (e != cudaSuccess) { fail(e, "prologue"); break; }
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
        if (e != cudaSuccess) { fail(e, "capture info"); break; }
        std::vector<cudaGraphNode_t> tail(deps, deps + ndeps);
        e = cudaStreamEndCapture(s, &g);
        capturing = false;
        if (e != cudaSuccess) { fail(e, "end prologue"); break; }
        n_pro = (long long)launches_total() - l0;
        // WHILE node: one outer step per iteration
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cond;
        e = cudaGraphAddNode(&cond, g, tail.data(), nullptr, tail.size(), &cp);
        if (e != cudaSuccess) { fail(e, "while node"); break; }
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        l0 = (long long)launches_total();
        e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { fail(e, "begin body"); break; }
        capturing = true;
        if (use_policy) {
            // one conditional handle per IF node (a handle serves a single node)
            for (int k = 0; k < c->inner && st == MG_OK; ++k) {
                cudaGraphConditionalHandle ih;
                e = cudaGraphConditionalHandleCreate(&ih, body, 0, cudaGraphCondAssignDefault);
                if (e != cudaSuccess) break;
                st = record_policy_vcycle(c, k == 0, k, body, ih, s, &n_sr);
            }
            if (e != cudaSuccess) { fail(e, "if handle"); break; }
            if (st != MG_OK) break;
            if (!fuse) e = launch_update(xd, c->lv[0].x32, N, c->red(kGrpU), s);
        } else if (adaptive) {
            // V-cycle 1 always; V-cycles 2 .. step each behind an IF node
            st = vcycle32_top(c, true, prolong);
            for (int k = 2; k <= step && st == MG_OK && e == cudaSuccess; ++k) {
                cudaStreamCaptureStatus cs2;
                const cudaGraphNode_t *d2 = nullptr;
                size_t nd2 = 0;
                e = cudaStreamGetCaptureInfo(s, &cs2, nullptr, nullptr, &d2, nullptr, &nd2);
                if (e != cudaSuccess) break;
                std::vector<cudaGraphNode_t> t2(d2, d2 + nd2);
                e = cudaStreamEndCapture(s, &body);
                if (e != cudaSuccess) break;
                cudaGraphNodeParams ip = {};
                ip.type = cudaGraphNodeTypeConditional;
                ip.conditional.handle = ifh.h[k - 2];
                ip.conditional.type = cudaGraphCondTypeIf;
                ip.conditional.size = 1;
                cudaGraphNode_t ifn;
                e = cudaGraphAddNode(&ifn, body, t2.data(), nullptr, t2.size(), &ip);
                if (e != cudaSuccess) break;
                cudaGraph_t ib = ip.conditional.phGraph_out[0];
                e = cudaStreamBeginCaptureToGraph(s, ib, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) break;
                const long long lc = (long long)launches_total();
                st = vcycle32_top(c, false, prolong);
                n_cyc = (long long)launches_total() - lc;
                cudaError_t e2 = cudaStreamEndCapture(s, &ib);
                if (st != MG_OK) break;
                e = e2;
                if (e != cudaSuccess) break;
                e = cudaStreamBeginCaptureToGraph(s, body, &ifn, nullptr, 1, cudaStreamCaptureModeThreadLocal);
            }
            if (st != MG_OK) break;
            if (e != cudaSuccess) { fail(e, "optional cycles"); break; }
            if (!fuse) e = launch_update(xd, c->lv[0].x32, N, c->red(kGrpU), s);
        } else if (mixed) {
            for (int k = 0; k < c->inner && st == MG_OK; ++k) st = vcycle32_top(c, k == 0, prolong);
            if (st != MG_OK) break;
            if (!fuse) e = launch_update(xd, c->lv[0].x32, N, c->red(kGrpU), s);
        } else {
            st = vcycle_rec<double>(c, 0, xd, c->lv[0].t64, c->lv[0].b64, false);
            if (st != MG_OK) break;
        }
        // the fused form reads the step counter before k_check advances it
        if (e == cudaSuccess)
            e = fuse ? solve_update_residual(c, xd, &c->dstate->outer, 0, xz, h2, s)
                     : solve_residual(c, fd, xd, mixed, false, h2, s);
        if (e == cudaSuccess)
            e = launch_check(c->dstate, c->out(kGrpR),
                             mixed ? (fuse ? c->out(kGrpR) + 1 : c->out(kGrpU)) : nullptr, c->out(kGrpF), N2, h2,
                             tol, step, c->max_cycles, false, handle, s, rho, ifh);
        if (e != cudaSuccess) { fail(e, "body"); break; }
        e = cudaStreamEndCapture(s, &body);
        capturing = false;
        if (e != cudaSuccess) { fail(e, "end body"); break; }
        n_body = (long long)launches_total() - l0;
        // epilogue: zero-mean projection (or zero for a constant source)
        l0 = (long long)launches_total();
        e = cudaStreamBeginCaptureToGraph(s, g, &cond, nullptr, 1, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { fail(e, "begin epilogue"); break; }
        capturing = true;
        // after k outer steps of the fused form, x is in xalt when k is odd
        // (on a cold start with no outer step run, x is zero and not read)
        e = launch_sum(xd, N, c->red(kGrpX), s, fuse ? c->xalt : nullptr, fuse ? &c->dstate->outer : nullptr, xz);
        if (e == cudaSuccess)
            e = launch_project(xd, N, c->out(kGrpX), s, &c->dstate->zero_source, fuse ? c->xalt : nullptr,
                               fuse ? &c->dstate->outer : nullptr, xz);
        if (e != cudaSuccess) { fail(e, "epilogue"); break; }
        e = cudaStreamEndCapture(s, &g);
        capturing = false;
        if (e != cudaSuccess) { fail(e, "end epilogue"); break; }
        n_epi = (long long)launches_total() - l0;
        e = cudaGraphInstantiate(&out->exec, g, 0);
        if (e != cudaSuccess) { fail(e, "instantiate"); break; }
    } while (false);
    c->stream = user_stream;
    count_launches(-(n_pro + n_body + n_epi));  // recording is not execution
    if (capturing) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(s, &junk);
        if (junk && junk != g) cudaGraphDestroy(junk);
    }
    if (st != MG_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        out->exec = nullptr;
        return st;
    }
    out->graph = g;
    out->f = fd;
    out->x = xd;
    out->prolong = (int)prolong;
    out->tol = tol;
    out->n_pro = n_pro;
    out->n_body = n_body;
    out->n_epi = n_epi;
    out->n_sr = n_sr;
    out->n_cyc = n_cyc;
    out->adapt_max = adaptive ? step : 0;
    return MG_OK;
}

static mg_status get_solve_graph(mg_ctx *c, const double *fd, double *xd, mg_prolong prolong, double tol,
                                 SolveGraph **out) {
    SolveGraph *lru = &c->graphs[0];
    const bool xz = kernels_take_zero(c, c->prec == MG_PREC_MIXED);
    for (SolveGraph &g : c->graphs) {
        if (g.exec && g.f == fd && g.x == xd && g.prolong == (int)prolong && g.tol == tol && g.xzero == xz &&
            g.epoch == tune_epoch()) {
            g.stamp = ++c->graph_clock;
            *out = &g;
            return MG_OK;
        }
        if (!g.exec || g.stamp < lru->stamp) lru = &g;
    }
    if (lru->exec) cudaGraphExecDestroy(lru->exec);
    if (lru->graph) cudaGraphDestroy(lru->graph);
    *lru = SolveGraph();
    const unsigned epoch = tune_epoch();
    MG_TRY(record_solve_graph(c, fd, xd, prolong, tol, lru));
    lru->epoch = epoch;
    lru->xzero = xz;
    lru->stamp = ++c->graph_clock;
    *out = lru;
    return MG_OK;
}


// ---------------------------------------------------------------------------
// Batched solves: one graph for B right-hand sides of (possibly) different
// sizes.  A V-cycle of the whole batch is a down launch per grid size from the
// largest to 128^2 (every right-hand side with a level of that size takes
// part), one bottom launch (a block per right-hand side), and an up launch per
// size back up; the FP64 outer steps, the convergence tests and the projection
// are one launch each.  Converged right-hand sides drop out through an active
// mask; the WHILE node runs until none is active.
// ---------------------------------------------------------------------------
struct BatchLaunch {
    int kind;    // 0 down, 1 up, 2 bottom
    size_t off;  // table offset (entries of TileGrid / BottomGrid)
    int ngrid;
    int nblocks;
    int variant;  // tile variant (down / up)
    int size = 0;  // grid size (down / up)
};

struct BatchPlan {
    std::vector<mg_ctx *> ctxs;
    std::vector<const double *> f;
    std::vector<double *> x;
    double tol = 0.0;
    int B = 0, device = -1;
    mg_prolong prolong = MG_PROLONG_CUBIC;
    // SR prolongation: one generator batch per grid size whose right-hand
    // sides end in an SR transition (their finest coarse grid >= 128)
    std::vector<SrBatch> srb;
    std::vector<int> sr_size;  // fine grid size of srb[i]
    uint64_t srb_hash = 0;     // weights the plan was recorded with
    void *dmem = nullptr;
    RhsDesc *d_rhs = nullptr;
    TileGrid *d_tiles = nullptr;
    BottomGrid *d_bottom = nullptr;
    DevState *d_state = nullptr, *h_state = nullptr;
    int *d_active = nullptr;
    double *d_partials = nullptr, *d_out = nullptr;  // out: 4 groups x [B][kMaxSlots]
    unsigned *d_counters = nullptr;
    int rhs_blocks = 0;
    std::vector<BatchLaunch> cyc[2];  // [0] first inner cycle (zero start), [1] the others
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long n_pro = 0, n_body = 0, n_epi = 0;
    long long n_cyc = 0;   // kernels of one optional (conditional) batch V-cycle
    int adapt_max = 0;     // adaptive inner cycles: optional cycles 2 .. adapt_max recorded
    int *d_bm = nullptr;   // [0] next step's V-cycles, [1] V-cycles run (adaptive)
    int h_bm[2] = {0, 0};
    unsigned epoch = 0;
    // every right-hand side's outer step fuses the update with the next
    // residual on its context's iterate pair (x, xalt)
    bool fused = false;
    BatchRed red(int g) const { return BatchRed{d_partials, d_counters, d_out + (size_t)g * B * kMaxSlots}; }
    double *out(int g) const { return d_out + (size_t)g * B * kMaxSlots; }
};

static std::mutex g_batch_mutex;
static BatchPlan *g_batch = nullptr;

static void batch_free(BatchPlan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap) cudaStreamDestroy(p->cap);
    cudaFree(p->dmem);
    cudaFreeHost(p->h_state);
    for (SrBatch &b : p->srb) sr_batch_free(&b);
    delete p;
}

static mg_status batch_build(BatchPlan *p) {
    mg_ctx *c0 = p->ctxs[0];
    const int B = p->B;
    FirTaps taps;
    fir_taps_host(&taps);
    // right-hand-side descriptors and the level plan
    std::vector<RhsDesc> rhs(B);
    int blk = 0, maxN = 0;
    for (int r = 0; r < B; ++r) {
        mg_ctx *c = p->ctxs[r];
        const int n = c->N;
        const double h = 2.0 * 3.14159265358979323846 / n;
        int nblk = (int)(((size_t)n * n) / 16384);
        nblk = nblk < 1 ? 1 : (nblk > kRedBlocks ? kRedBlocks : nblk);
        rhs[r] = RhsDesc{p->f[r], p->x[r], c->lv[0].b32, c->lv[0].x32, c->bsc64, c->ebt, n, blk, nblk, r, 0, 0,
                         h * h};
        blk += nblk;
        maxN = n > maxN ? n : maxN;
    }
    p->rhs_blocks = blk;
    p->fused = fused_update_mode() != 0;
    for (int r = 0; r < B; ++r) p->fused = p->fused && rhs[r].n >= kResMinN && p->ctxs[r]->xalt;
    if (p->fused)
        for (int r = 0; r < B; ++r) rhs[r].xalt = p->ctxs[r]->xalt;
    // SR groups: right-hand sides of one fine size whose coarse grid the
    // generator takes (>= 128, a multiple of 128); smaller ones stay cubic
    std::vector<int> sr_group(B, -1), sr_index(B, -1);
    if (p->prolong == MG_PROLONG_SR) {
        for (int sz = maxN; sz >= 2 * kSrMinCoarse; sz >>= 1) {
            std::vector<const float *> ecs;
            for (int r = 0; r < B; ++r) {
                mg_ctx *c = p->ctxs[r];
                if (c->N == sz && c->levels > 1 && c->lv[0].n > kBottomMax) {
                    sr_group[r] = (int)p->srb.size();
                    sr_index[r] = (int)ecs.size();
                    ecs.push_back(c->lv[1].x32);
                    rhs[r].sr = 1;
                }
            }
            if (ecs.empty()) continue;
            p->srb.emplace_back();
            p->sr_size.push_back(sz);
            MG_TRY(sr_batch_prepare(&p->srb.back(), (int)ecs.size(), sz / 2, ecs.data(), g_err, sizeof g_err));
        }
    }
    std::vector<TileGrid> tiles;
    std::vector<BottomGrid> bottoms;
    for (int v = 0; v < 2; ++v) {
        const bool first = v == 0;
        p->cyc[v].clear();
        auto grids_of = [&](int sz) {
            int g = 0;
            for (int r = 0; r < B; ++r)
                for (int l = 0; l + 1 < p->ctxs[r]->levels; ++l) g += p->ctxs[r]->lv[l].n == sz;
            return g;
        };
        for (int sz = maxN; sz > kBottomMax; sz >>= 1) {  // down sweeps
            BatchLaunch L{0, tiles.size(), 0, 0, batch_variant(0, sz, c0->nu1, grids_of(sz)), sz};
            for (int r = 0; r < B; ++r) {
                mg_ctx *c = p->ctxs[r];
                for (int l = 0; l + 1 < c->levels; ++l)
                    if (c->lv[l].n == sz) {
                        tiles.push_back(TileGrid{c->lv[l].x32, c->lv[l].t32, c->lv[l].b32, c->lv[l + 1].b32, sz,
                                                 (l > 0 || first) ? 1 : 0, L.nblocks, r});
                        L.nblocks += variant_tiles(sz, L.variant);
                        ++L.ngrid;
                    }
            }
            if (L.ngrid) p->cyc[v].push_back(L);
        }
        {  // bottom
            BatchLaunch L{2, bottoms.size(), 0, 0, 0};
            for (int r = 0; r < B; ++r) {
                mg_ctx *c = p->ctxs[r];
                int l = 0;
                while (c->lv[l].n > kBottomMax) ++l;
                bottoms.push_back(BottomGrid{c->lv[l].x32, c->lv[l].b32, c->ainv32, c->lv[l].n, c->levels - l,
                                             (l > 0 || first) ? 1 : 0, r});
                ++L.ngrid;
            }
            L.nblocks = L.ngrid;
            p->cyc[v].push_back(L);
        }
        for (int sz = 2 * kBottomMax; sz <= maxN; sz <<= 1) {  // up sweeps
            BatchLaunch L{1, tiles.size(), 0, 0, batch_variant(1, sz, c0->nu2, grids_of(sz)), sz};
            for (int r = 0; r < B; ++r) {
                mg_ctx *c = p->ctxs[r];
                for (int l = 0; l + 1 < c->levels; ++l)
                    if (c->lv[l].n == sz) {
                        TileGrid t{c->lv[l].t32, c->lv[l].x32, c->lv[l].b32, c->lv[l + 1].x32, sz, 0, L.nblocks, r};
                        if (l == 0 && sr_group[r] >= 0)
                            t.extra = p->srb[sr_group[r]].fine_out + (size_t)sr_index[r] * sz * sz;
                        tiles.push_back(t);
                        L.nblocks += variant_tiles(sz, L.variant);
                        ++L.ngrid;
                    }
            }
            if (L.ngrid) p->cyc[v].push_back(L);
        }
    }
    // one device block for every table and buffer
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t o_rhs = 0, o_tiles = o_rhs + al(sizeof(RhsDesc) * B);
    const size_t o_bot = o_tiles + al(sizeof(TileGrid) * (tiles.size() + 1));
    const size_t o_state = o_bot + al(sizeof(BottomGrid) * bottoms.size());
    const size_t o_active = o_state + al(sizeof(DevState) * B);
    const size_t o_part = o_active + al(sizeof(int) * B);
    const size_t o_out = o_part + al(sizeof(double) * kMaxSlots * blk);
    const size_t o_cnt = o_out + al(sizeof(double) * 4 * B * kMaxSlots);
    const size_t o_bm = o_cnt + al(sizeof(unsigned) * B);
    const size_t total = o_bm + al(2 * sizeof(int));
    MG_CUDA(cudaMalloc(&p->dmem, total));
    char *d = (char *)p->dmem;
    p->d_rhs = (RhsDesc *)(d + o_rhs);
    p->d_tiles = (TileGrid *)(d + o_tiles);
    p->d_bottom = (BottomGrid *)(d + o_bot);
    p->d_state = (DevState *)(d + o_state);
    p->d_active = (int *)(d + o_active);
    p->d_partials = (double *)(d + o_part);
    p->d_out = (double *)(d + o_out);
    p->d_counters = (unsigned *)(d + o_cnt);
    p->d_bm = (int *)(d + o_bm);
    for (TileGrid &t : tiles)  // SR is skipped for a right-hand side once it has fallen back
        if (t.extra) t.extra_off = &p->d_state[t.rhs].fallback;
    MG_CUDA(cudaMemset(p->dmem, 0, total));
    MG_CUDA(cudaMemcpy(p->d_rhs, rhs.data(), sizeof(RhsDesc) * B, cudaMemcpyHostToDevice));
    if (!tiles.empty())
        MG_CUDA(cudaMemcpy(p->d_tiles, tiles.data(), sizeof(TileGrid) * tiles.size(), cudaMemcpyHostToDevice));
    MG_CUDA(cudaMemcpy(p->d_bottom, bottoms.data(), sizeof(BottomGrid) * bottoms.size(), cudaMemcpyHostToDevice));
    MG_CUDA(cudaMallocHost(&p->h_state, sizeof(DevState) * B));
    MG_CUDA(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));

    // record: prologue, WHILE(outer step), epilogue
    cudaStream_t s = p->cap;
    // SR batches keep the fixed count of V-cycles per outer step (as SR solves do)
    const bool adaptive = p->prolong == MG_PROLONG_CUBIC && c0->rho > 0.0 && c0->adapt_max > 1;
    const int step = adaptive ? c0->adapt_max : c0->inner;
    const double rho = adaptive ? c0->rho : 0.0;
    p->adapt_max = adaptive ? step : 0;
    cudaGraphConditionalHandle handle;
    CycleHandles ifh{};
    MG_CUDA(cudaGraphCreate(&p->graph, 0));
    MG_CUDA(cudaGraphConditionalHandleCreate(&handle, p->graph, 0, cudaGraphCondAssignDefault));
    for (int k = 2; adaptive && k <= step; ++k)
        MG_CUDA(cudaGraphConditionalHandleCreate(&ifh.h[k - 2], p->graph, 0, cudaGraphCondAssignDefault));
    bool capturing = false;
    cudaError_t e = cudaSuccess;
    auto run_cycle = [&](int v) {
        for (const BatchLaunch &L : p->cyc[v]) {
            if (e != cudaSuccess) return;
            if (L.kind == 0)
                e = launch_down_batched(p->d_tiles + L.off, L.ngrid, L.nblocks, c0->nu1, p->d_active, s,
                                        L.variant);
            else if (L.kind == 1) {
                // the generator's correction for the right-hand sides whose finest grid is this size
                for (size_t g = 0; g < p->srb.size() && e == cudaSuccess; ++g)
                    if (p->sr_size[g] == L.size &&
                        sr_batch_correction(&p->srb[g], &c0->sr, s, g_err, sizeof g_err) != MG_OK)
                        e = cudaErrorLaunchFailure;
                if (e == cudaSuccess)
                    e = launch_up_batched(p->d_tiles + L.off, L.ngrid, L.nblocks, c0->nu2, p->d_active, taps, s,
                                          L.variant);
            }
            else
                e = launch_bottom_batched(p->d_bottom + L.off, L.ngrid, c0->nu1, c0->nu2, p->d_active, taps, s);
        }
    };
    long long l0 = (long long)launches_total();
    do {
        e = cudaStreamBeginCaptureToGraph(s, p->graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        capturing = true;
        e = launch_sum_batched(p->d_rhs, B, blk, false, p->red(kGrpF), s);
        if (e == cudaSuccess)
            e = launch_outer_residual_batched(p->d_rhs, B, blk, p->out(kGrpF), true, true, nullptr, p->red(kGrpR), s);
        if (e == cudaSuccess)
            e = launch_check_batched(p->d_state, p->d_rhs, B, p->out(kGrpR), nullptr, p->out(kGrpF), p->tol, step,
                                     c0->max_cycles, true, p->d_active, handle, true, s, rho, ifh, p->d_bm);
        if (e != cudaSuccess) break;
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
        if (e != cudaSuccess) break;
        std::vector<cudaGraphNode_t> tail(deps, deps + ndeps);
        e = cudaStreamEndCapture(s, &p->graph);
        capturing = false;
        if (e != cudaSuccess) break;
        p->n_pro = (long long)launches_total() - l0;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cond;
        e = cudaGraphAddNode(&cond, p->graph, tail.data(), nullptr, tail.size(), &cp);
        if (e != cudaSuccess) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        l0 = (long long)launches_total();
        e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        capturing = true;
        if (adaptive) {
            run_cycle(0);
            for (int k = 2; k <= step && e == cudaSuccess; ++k) {  // optional cycles behind IF nodes
                cudaStreamCaptureStatus cs2;
                const cudaGraphNode_t *d2 = nullptr;
                size_t nd2 = 0;
                e = cudaStreamGetCaptureInfo(s, &cs2, nullptr, nullptr, &d2, nullptr, &nd2);
                if (e != cudaSuccess) break;
                std::vector<cudaGraphNode_t> t2(d2, d2 + nd2);
                e = cudaStreamEndCapture(s, &body);
                capturing = false;
                if (e != cudaSuccess) break;
                cudaGraphNodeParams ip = {};
                ip.type = cudaGraphNodeTypeConditional;
                ip.conditional.handle = ifh.h[k - 2];
                ip.conditional.type = cudaGraphCondTypeIf;
                ip.conditional.size = 1;
                cudaGraphNode_t ifn;
                e = cudaGraphAddNode(&ifn, body, t2.data(), nullptr, t2.size(), &ip);
                if (e != cudaSuccess) break;
                cudaGraph_t ib = ip.conditional.phGraph_out[0];
                e = cudaStreamBeginCaptureToGraph(s, ib, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess) break;
                capturing = true;
                const long long lc = (long long)launches_total();
                run_cycle(1);
                p->n_cyc = (long long)launches_total() - lc;
                cudaError_t e2 = cudaStreamEndCapture(s, &ib);
                capturing = false;
                if (e == cudaSuccess) e = e2;
                if (e != cudaSuccess) break;
                e = cudaStreamBeginCaptureToGraph(s, body, &ifn, nullptr, 1, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) capturing = true;
            }
        } else {
            for (int k = 0; k < step; ++k) run_cycle(k == 0 ? 0 : 1);
        }
        if (p->fused) {
            // each right-hand side's step count is read before k_check_b advances it
            if (e == cudaSuccess)
                e = launch_update_residual_batched(p->d_rhs, B, blk, p->d_state, p->d_active, p->red(kGrpR), s);
        } else {
            if (e == cudaSuccess) e = launch_update_batched(p->d_rhs, B, blk, p->d_active, p->red(kGrpU), s);
            if (e == cudaSuccess)
                e = launch_outer_residual_batched(p->d_rhs, B, blk, p->out(kGrpF), false, false, p->d_active,
                                                  p->red(kGrpR), s);
        }
        // (the fused form leaves each sum of e^2 beside its residual's)
        if (e == cudaSuccess)
            e = launch_check_batched(p->d_state, p->d_rhs, B, p->out(kGrpR),
                                     p->fused ? p->out(kGrpR) + 1 : p->out(kGrpU), p->out(kGrpF), p->tol, step,
                                     c0->max_cycles, false, p->d_active, handle, true, s, rho, ifh, p->d_bm);
        if (e != cudaSuccess) break;
        e = cudaStreamEndCapture(s, &body);
        capturing = false;
        if (e != cudaSuccess) break;
        p->n_body = (long long)launches_total() - l0;
        l0 = (long long)launches_total();
        e = cudaStreamBeginCaptureToGraph(s, p->graph, &cond, nullptr, 1, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        capturing = true;
        e = launch_sum_batched(p->d_rhs, B, blk, true, p->red(kGrpX), s, p->fused ? p->d_state : nullptr);
        if (e == cudaSuccess)
            e = launch_project_batched(p->d_rhs, B, blk, p->out(kGrpX), p->d_state, s, p->fused);
        if (e != cudaSuccess) break;
        e = cudaStreamEndCapture(s, &p->graph);
        capturing = false;
        if (e != cudaSuccess) break;
        p->n_epi = (long long)launches_total() - l0;
        e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    } while (false);
    count_launches(-(p->n_pro + p->n_body + p->n_epi));
    if (capturing) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(s, &junk);
        if (junk && junk != p->graph) cudaGraphDestroy(junk);
    }
    if (e != cudaSuccess) {
        set_err("batched graph recording failed: %s", cudaGetErrorString(e));
        cudaGetLastError();
        return MG_ERR_CUDA;
    }
    return MG_OK;
}

// Drop the cached batch graph if it refers to context c (destroyed or changed).
static void batch_forget(mg_ctx *c) {
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    if (!g_batch) return;
    for (mg_ctx *q : g_batch->ctxs)
        if (q == c) {
            batch_free(g_batch);
            g_batch = nullptr;
            return;
        }
}

// All contexts mixed precision with equal cycle options on one device, all
// buffers on the device, and the cubic prolongation or the SR one with the
// same generator weights in every context: the batched graph applies.
static bool batch_eligible(mg_ctx *const *ctxs, const double *const *f, double *const *x, int B,
                           mg_prolong prolong) {
    if (B < 1 || (prolong != MG_PROLONG_CUBIC && prolong != MG_PROLONG_SR)) return false;
    mg_ctx *c0 = ctxs[0];
    if (!c0 || c0->prec != MG_PREC_MIXED || c0->probe_kind != kProbeNone) return false;
    if (prolong == MG_PROLONG_SR) {  // every context holds the same generator weights
        for (int r = 0; r < B; ++r)
            if (!ctxs[r] || !ctxs[r]->sr.loaded || ctxs[r]->sr.hash != c0->sr.hash) return false;
    }
    for (int r = 0; r < B; ++r) {
        mg_ctx *c = ctxs[r];
        if (!c || !f[r] || !x[r] || c->prec != MG_PREC_MIXED || c->nu1 != c0->nu1 || c->nu2 != c0->nu2 ||
            c->inner != c0->inner || c->max_cycles != c0->max_cycles || c->device != c0->device ||
            c->adapt_max != c0->adapt_max || c->rho != c0->rho ||
            !is_device_pointer(f[r]) || !is_device_pointer(x[r]))
            return false;
        for (int q = 0; q < r; ++q)
            if (ctxs[q] == c || x[q] == x[r]) return false;  // each context and x once
    }
    return true;
}

static mg_status solve_batched_graph(mg_ctx *const *ctxs, const double *const *f, double *const *x, int B,
                                     double tol, mg_prolong prolong, mg_solve_info *infos) {
    const auto t0 = std::chrono::steady_clock::now();
    mg_ctx *c0 = ctxs[0];
    MG_CUDA(cudaSetDevice(c0->device));
    for (int r = 0; r < B; ++r) MG_TRY(ensure_hierarchy(ctxs[r], false));
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    BatchPlan *p = g_batch;
    bool same = p && p->B == B && p->tol == tol && p->device == c0->device && p->epoch == tune_epoch() &&
                p->prolong == prolong && (prolong == MG_PROLONG_CUBIC || p->srb_hash == c0->sr.hash);
    for (int r = 0; same && r < B; ++r)
        same = p->ctxs[r] == ctxs[r] && p->f[r] == f[r] && p->x[r] == x[r];
    if (!same) {
        batch_free(g_batch);
        g_batch = nullptr;
        p = new BatchPlan();
        p->B = B;
        p->tol = tol;
        p->device = c0->device;
        p->prolong = prolong;
        p->srb_hash = prolong == MG_PROLONG_SR ? c0->sr.hash : 0;
        p->ctxs.assign(ctxs, ctxs + B);
        p->f.assign(f, f + B);
        p->x.assign(x, x + B);
        p->epoch = tune_epoch();
        mg_status st = batch_build(p);
        if (st != MG_OK) {
            batch_free(p);
            return st;
        }
        g_batch = p;
    }
    cudaStream_t s = c0->stream;
    const bool sr = !p->srb.empty();
    int sr_flag = 0;
    if (sr) MG_CUDA(cudaMemsetAsync(c0->sr.err, 0, sizeof(int), s));
    MG_CUDA(cudaGraphLaunch(p->exec, s));
    MG_CUDA(cudaMemcpyAsync(p->h_state, p->d_state, sizeof(DevState) * B, cudaMemcpyDeviceToHost, s));
    if (sr) MG_CUDA(cudaMemcpyAsync(&sr_flag, c0->sr.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (p->adapt_max > 0) MG_CUDA(cudaMemcpyAsync(p->h_bm, p->d_bm, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    int outer_max = 0;
    mg_status worst = MG_OK;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int r = 0; r < B; ++r) {
        const DevState &ds = p->h_state[r];
        outer_max = ds.outer > outer_max ? ds.outer : outer_max;
        if (ds.status != MG_OK && worst == MG_OK) worst = (mg_status)ds.status;
        if (infos) {
            infos[r].outer_iters = ds.outer;
            infos[r].vcycles = ds.cycles;
            infos[r].rel_residual = ds.rel;
            infos[r].removed_mean = ds.mu;
            infos[r].update_norm = ds.unorm;
            infos[r].time_ms = ms;
            infos[r].prolong_used = ds.sr_used > 0 ? MG_PROLONG_SR : MG_PROLONG_CUBIC;
            infos[r].sr_fallback = ds.fallback;
            infos[r].sr_cycles = ds.sr_used;
        }
    }
    if (p->adapt_max > 0)  // optional V-cycles ran only in the steps that chose them
        count_launches(p->n_pro + (long long)outer_max * p->n_body -
                       ((long long)outer_max * p->adapt_max - p->h_bm[1]) * p->n_cyc + p->n_epi);
    else
        count_launches(p->n_pro + (long long)outer_max * p->n_body + p->n_epi);
    if (sr_flag) {
        set_err("a bounded wait in the tensor-core convolution timed out (batched SR)");
        return MG_ERR_TIMEOUT;
    }
    if (worst == MG_ERR_NONFINITE) set_err("non-finite residual in a batched right-hand side");
    if (worst == MG_ERR_NOT_CONVERGED) set_err("a batched right-hand side did not converge");
    return worst;
}

// ---------------------------------------------------------------------------
// Continuous-batching server.  Requests wait in a FIFO until a slot (a
// resident level hierarchy plus FP64 f and x of the request's size) and the
// device-memory budget allow admission.  Every tick runs one outer step of
// defect correction for every admitted request as batched launches (new
// requests start with their first residual, the others continue), then
// retires the requests that converged: zero-mean projection, the solution
// copied to the caller's buffer and kept as the warm start of the request's
// stream.  Requests therefore join and leave the batch between ticks while
// the others keep going.
// ---------------------------------------------------------------------------
constexpr int kServerSlots = 1024;

struct ServerSlot {
    mg_ctx *ctx = nullptr;
    int N = 0;
    double *f = nullptr, *x = nullptr;
    size_t bytes = 0;
    bool busy = false, first = false;
    long long req = -1;
    int stream_id = -1;
    double *x_out = nullptr;
    double t_submit = 0.0, t_admit = 0.0;
    // adaptive inner cycles: what the host knows of this request's progress
    int m_last = 0;          // V-cycles of its last outer step
    int cycles_run = 0;      // V-cycles scheduled so far
    int nrel = 0;            // relative residuals seen (start of each of its ticks)
    double rel1 = 0.0, rel2 = 0.0;  // the last two of them (rel1 newest)
    int m2 = 0;              // V-cycles between rel2 and rel1
};
struct ServerRequest {
    long long id;
    int stream_id, N;
    const double *f;
    double *x_out;
    double t_submit;
};

struct mg_server {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0, used = 0;
    int nu1 = 2, nu2 = 2, inner = 2, max_cycles = 100;
    bool adaptive = false;  // inner_cycles = 0 at creation: per-slot adaptive V-cycles
    int m_max = 3;
    double rho = 0.06;
    double tol = 1e-10;
    std::vector<ServerSlot> slots;
    std::vector<ServerRequest> queue;  // FIFO
    size_t qhead = 0;
    std::vector<std::pair<long long, double *>> warm;  // key = stream_id * 2^20 + N -> last solution
    std::vector<mg_server_result> done;
    size_t dhead = 0;
    long long next_id = 0;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    // device state and tables
    void *dmem = nullptr;
    DevState *d_state = nullptr;
    int *d_active = nullptr;
    double *d_out = nullptr, *d_partials = nullptr;
    unsigned *d_counters = nullptr;
    char *d_tab = nullptr, *h_tab = nullptr;  // tables, pinned staging
    size_t tab_bytes = 0;
    DevState *h_state = nullptr;
    int *h_active = nullptr;
    FirTaps taps;
    BatchRed red(int g) const { return BatchRed{d_partials, d_counters, d_out + (size_t)g * kServerSlots * kMaxSlots}; }
    double *out(int g) const { return d_out + (size_t)g * kServerSlots * kMaxSlots; }
};

static size_t server_slot_bytes(int N) {
    size_t b = 3ull * N * N * sizeof(double);  // f, x, scaled right-hand side
    if (N >= kResMinN) b += res_tasks(N) * sizeof(int);
    for (int n = N; n >= 8; n >>= 1) b += 3ull * n * n * sizeof(float);
    return b;
}

static int server_levels(int N) {
    int l = 1;
    for (int n = N; n > 8; n >>= 1) ++l;
    return l;
}

static double *server_warm(mg_server *sv, int stream_id, int N, bool create) {
    const long long key = (long long)stream_id * (1ll << 20) + N;
    for (auto &w : sv->warm)
        if (w.first == key) return w.second;
    if (!create) return nullptr;
    double *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * N * N) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    sv->used += sizeof(double) * N * N;
    sv->warm.push_back({key, buf});
    return buf;
}

static void server_free_slot(mg_server *sv, size_t k) {
    ServerSlot &sl = sv->slots[k];
    cudaFree(sl.f);
    cudaFree(sl.x);
    mg_destroy(sl.ctx);
    sv->used -= sl.bytes;
    sl = ServerSlot();
}

// Free idle hierarchies of other sizes, least recently used first, until
// `need` more bytes fit the budget.  Slot indices never move (the device
// state is indexed by them); a freed entry is reused by later admissions.
static bool server_make_room(mg_server *sv, size_t need, int N) {
    while (sv->used + need > sv->budget) {
        long long best = -1;
        double oldest = 0.0;
        for (size_t k = 0; k < sv->slots.size(); ++k) {
            const ServerSlot &sl = sv->slots[k];
            if (sl.ctx && !sl.busy && sl.N != N && (best < 0 || sl.t_admit < oldest)) {
                best = (long long)k;
                oldest = sl.t_admit;
            }
        }
        if (best < 0) return false;
        server_free_slot(sv, (size_t)best);
    }
    return true;
}

// Admit queued requests in FIFO order while a slot and the budget allow.
static mg_status server_admit(mg_server *sv) {
    while (sv->qhead < sv->queue.size()) {
        const ServerRequest &rq = sv->queue[sv->qhead];
        int sid = -1, empty = -1;
        for (size_t k = 0; k < sv->slots.size(); ++k) {
            const ServerSlot &sl = sv->slots[k];
            if (sl.ctx && !sl.busy && sl.N == rq.N) {
                sid = (int)k;
                break;
            }
            if (!sl.ctx && empty < 0) empty = (int)k;
        }
        if (sid < 0) {
            const size_t need = server_slot_bytes(rq.N);
            if (sv->used + need > sv->budget) server_make_room(sv, need, rq.N);
            if (empty < 0) {  // make_room may have freed an entry
                for (size_t k = 0; k < sv->slots.size() && empty < 0; ++k)
                    if (!sv->slots[k].ctx) empty = (int)k;
            }
            if (empty < 0 || sv->used + need > sv->budget) break;
            ServerSlot sl;
            MG_TRY(mg_setup(server_levels(rq.N), rq.N, &sl.ctx));
            sl.ctx->nu1 = sv->nu1;
            sl.ctx->nu2 = sv->nu2;
            sl.ctx->inner = sv->inner;
            sl.ctx->max_cycles = sv->max_cycles;
            sl.ctx->stream = sv->stream;
            mg_status st = ensure_hierarchy(sl.ctx, false);
            if (st == MG_OK && cudaMalloc(&sl.f, sizeof(double) * rq.N * rq.N) != cudaSuccess) st = MG_ERR_OOM;
            if (st == MG_OK && cudaMalloc(&sl.x, sizeof(double) * rq.N * rq.N) != cudaSuccess) st = MG_ERR_OOM;
            if (st != MG_OK) {
                cudaGetLastError();
                cudaFree(sl.f);
                cudaFree(sl.x);
                mg_destroy(sl.ctx);
                if (st == MG_ERR_OOM) break;  // wait for memory to free up
                return st;
            }
            sl.N = rq.N;
            sl.bytes = need;
            sv->used += need;
            sv->slots[empty] = sl;
            sid = empty;
        }
        ServerSlot &sl = sv->slots[sid];
        const size_t bytes = sizeof(double) * rq.N * rq.N;
        MG_CUDA(cudaMemcpyAsync(sl.f, rq.f, bytes, cudaMemcpyDefault, sv->stream));
        const double *w = server_warm(sv, rq.stream_id, rq.N, false);
        if (w)
            MG_CUDA(cudaMemcpyAsync(sl.x, w, bytes, cudaMemcpyDeviceToDevice, sv->stream));
        else
            MG_CUDA(cudaMemsetAsync(sl.x, 0, bytes, sv->stream));
        sl.busy = true;
        sl.first = true;
        sl.req = rq.id;
        sl.stream_id = rq.stream_id;
        sl.x_out = rq.x_out;
        sl.t_submit = rq.t_submit;
        sl.t_admit = sv->now_ms();
        sl.m_last = sl.cycles_run = sl.nrel = sl.m2 = 0;
        sl.rel1 = sl.rel2 = 0.0;
        ++sv->qhead;
    }
    if (sv->qhead == sv->queue.size()) {
        sv->queue.clear();
        sv->qhead = 0;
    }
    return MG_OK;
}

// Tables for one tick live in one staging block: [RhsDesc x n][first-slot
// RhsDesc x nf][TileGrid ...][BottomGrid ...]; offsets in bytes.
struct TickPlan {
    std::vector<RhsDesc> rhs, firsts, dones;
    std::vector<TileGrid> tiles;
    std::vector<BottomGrid> bottoms;
    std::vector<BatchLaunch> cyc[kMaxAdaptive > 2 ? kMaxAdaptive : 2];  // see plan_cycles
    int blk = 0, blk_first = 0, blk_done = 0;
};

static void plan_rhs(std::vector<RhsDesc> &v, int &blk, const ServerSlot &sl, int sid) {
    const int n = sl.N;
    const double h = 2.0 * 3.14159265358979323846 / n;
    int nblk = (int)(((size_t)n * n) / 16384);
    nblk = nblk < 1 ? 1 : (nblk > kRedBlocks ? kRedBlocks : nblk);
    v.push_back(RhsDesc{sl.f, sl.x, sl.ctx->lv[0].b32, sl.ctx->lv[0].x32, sl.ctx->bsc64, sl.ctx->ebt, n, blk, nblk, sid,
                        sl.first ? 1 : 0,
                        sl.first ? 0 : sl.m_last, h * h});
    blk += nblk;
}

// Tables of the tick's V-cycles.  Adaptive: table k serves V-cycle k (0-based)
// and holds the slots with m[slot] > k.  Fixed count: table 0 serves the first
// V-cycle and table 1 all later ones (every slot runs all of them).  The first
// V-cycle starts the finest level from zero.
static void plan_cycles(mg_server *sv, TickPlan &tp, const std::vector<int> &sids, const std::vector<int> &m) {
    int maxN = 0, maxm = 0;
    for (int sid : sids) {
        maxN = sv->slots[sid].N > maxN ? sv->slots[sid].N : maxN;
        maxm = m[sid] > maxm ? m[sid] : maxm;
    }
    const int ntab = sv->adaptive ? maxm : (maxm > 1 ? 2 : 1);
    for (int v = 0; v < ntab; ++v) {
        const bool first = v == 0;
        auto grids_of = [&](int sz) {
            int g = 0;
            for (int sid : sids) {
                if (m[sid] <= v) continue;
                const mg_ctx *c = sv->slots[sid].ctx;
                for (int l = 0; l + 1 < c->levels; ++l) g += c->lv[l].n == sz;
            }
            return g;
        };
        for (int sz = maxN; sz > kBottomMax; sz >>= 1) {
            BatchLaunch L{0, tp.tiles.size(), 0, 0, batch_variant(0, sz, sv->nu1, grids_of(sz))};
            for (int sid : sids) {
                if (m[sid] <= v) continue;
                mg_ctx *c = sv->slots[sid].ctx;
                for (int l = 0; l + 1 < c->levels; ++l)
                    if (c->lv[l].n == sz) {
                        tp.tiles.push_back(TileGrid{c->lv[l].x32, c->lv[l].t32, c->lv[l].b32, c->lv[l + 1].b32, sz,
                                                    (l > 0 || first) ? 1 : 0, L.nblocks, sid});
                        L.nblocks += variant_tiles(sz, L.variant);
                        ++L.ngrid;
                    }
            }
            if (L.ngrid) tp.cyc[v].push_back(L);
        }
        BatchLaunch Lb{2, tp.bottoms.size(), 0, 0, 0};
        for (int sid : sids) {
            if (m[sid] <= v) continue;
            mg_ctx *c = sv->slots[sid].ctx;
            int l = 0;
            while (c->lv[l].n > kBottomMax) ++l;
            tp.bottoms.push_back(BottomGrid{c->lv[l].x32, c->lv[l].b32, c->ainv32, c->lv[l].n, c->levels - l,
                                            (l > 0 || first) ? 1 : 0, sid});
            ++Lb.ngrid;
        }
        Lb.nblocks = Lb.ngrid;
        if (Lb.ngrid) tp.cyc[v].push_back(Lb);
        for (int sz = 2 * kBottomMax; sz <= maxN; sz <<= 1) {
            BatchLaunch L{1, tp.tiles.size(), 0, 0, batch_variant(1, sz, sv->nu2, grids_of(sz))};
            for (int sid : sids) {
                if (m[sid] <= v) continue;
                mg_ctx *c = sv->slots[sid].ctx;
                for (int l = 0; l + 1 < c->levels; ++l)
                    if (c->lv[l].n == sz) {
                        tp.tiles.push_back(TileGrid{c->lv[l].t32, c->lv[l].x32, c->lv[l].b32, c->lv[l + 1].x32, sz, 0,
                                                    L.nblocks, sid});
                        L.nblocks += variant_tiles(sz, L.variant);
                        ++L.ngrid;
                    }
            }
            if (L.ngrid) tp.cyc[v].push_back(L);
        }
    }
}

// V-cycles of a slot's next outer step.  Fixed: the server's count.  Adaptive:
// the rule of single solves, applied to the relative residual the slot is
// predicted to have now (its latest residual times the contraction it showed
// over its previous step, or rho, to the power of its last step's V-cycles),
// capped by the cycles it has left.  Only the slot's own history enters, so a
// request's schedule does not depend on the other requests in flight.
static int server_cycles(const mg_server *sv, const ServerSlot &sl) {
    if (!sv->adaptive) return sv->inner;
    int m = sv->m_max;
    if (!sl.first && sl.nrel >= 1) {
        double rho = sv->rho;
        if (sl.nrel >= 2 && sl.m2 > 0 && sl.rel2 > 0.0 && sl.rel1 > 0.0 && sl.rel1 < sl.rel2)
            rho = pow(sl.rel1 / sl.rel2, 1.0 / sl.m2);
        double pred = sl.rel1;
        for (int k = 0; k < sl.m_last; ++k) pred *= rho;
        m = adaptive_cycles(pred, sv->tol, sv->rho, sv->m_max);
    }
    const int left = sv->max_cycles - sl.cycles_run;
    return m < left ? (m > 0 ? m : 1) : (left > 0 ? left : 1);
}

// Copy the plan's tables to the device in one transfer; returns device pointers.
static mg_status upload_plan(mg_server *sv, const TickPlan &tp, RhsDesc **d_rhs, RhsDesc **d_first,
                             TileGrid **d_tiles, BottomGrid **d_bottom) {
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t o1 = al(sizeof(RhsDesc) * tp.rhs.size());
    const size_t o2 = o1 + al(sizeof(RhsDesc) * (tp.firsts.size() + 1));
    const size_t o3 = o2 + al(sizeof(TileGrid) * (tp.tiles.size() + 1));
    const size_t total = o3 + al(sizeof(BottomGrid) * (tp.bottoms.size() + 1));
    if (total > sv->tab_bytes) {
        cudaFree(sv->d_tab);
        cudaFreeHost(sv->h_tab);
        sv->d_tab = nullptr;
        sv->h_tab = nullptr;
        MG_CUDA(cudaMalloc(&sv->d_tab, 2 * total));
        MG_CUDA(cudaMallocHost(&sv->h_tab, 2 * total));
        sv->tab_bytes = 2 * total;
    }
    memcpy(sv->h_tab, tp.rhs.data(), sizeof(RhsDesc) * tp.rhs.size());
    memcpy(sv->h_tab + o1, tp.firsts.data(), sizeof(RhsDesc) * tp.firsts.size());
    memcpy(sv->h_tab + o2, tp.tiles.data(), sizeof(TileGrid) * tp.tiles.size());
    memcpy(sv->h_tab + o3, tp.bottoms.data(), sizeof(BottomGrid) * tp.bottoms.size());
    MG_CUDA(cudaMemcpyAsync(sv->d_tab, sv->h_tab, total, cudaMemcpyHostToDevice, sv->stream));
    *d_rhs = (RhsDesc *)sv->d_tab;
    *d_first = (RhsDesc *)(sv->d_tab + o1);
    *d_tiles = (TileGrid *)(sv->d_tab + o2);
    *d_bottom = (BottomGrid *)(sv->d_tab + o3);
    return MG_OK;
}

static mg_status server_tick(mg_server *sv, int *n_active, int *n_queued, int *n_done) {
    MG_CUDA(cudaSetDevice(sv->device));
    MG_TRY(server_admit(sv));
    cudaStream_t s = sv->stream;
    TickPlan tp;
    std::vector<int> sids;
    for (size_t k = 0; k < sv->slots.size(); ++k)
        if (sv->slots[k].busy) {
            sids.push_back((int)k);
            plan_rhs(tp.rhs, tp.blk, sv->slots[k], (int)k);
            if (sv->slots[k].first) plan_rhs(tp.firsts, tp.blk_first, sv->slots[k], (int)k);
        }
    int finished = 0;
    if (!sids.empty()) {
        std::vector<int> m(sv->slots.size(), 0);
        for (int sid : sids) m[sid] = server_cycles(sv, sv->slots[sid]);
        plan_cycles(sv, tp, sids, m);
        RhsDesc *d_rhs, *d_first;
        TileGrid *d_tiles;
        BottomGrid *d_bottom;
        MG_TRY(upload_plan(sv, tp, &d_rhs, &d_first, &d_tiles, &d_bottom));
        const int nr = (int)tp.rhs.size();
        if (!tp.firsts.empty())
            MG_CUDA(launch_sum_batched(d_first, (int)tp.firsts.size(), tp.blk_first, false, sv->red(kGrpF), s));
        MG_CUDA(launch_outer_residual_batched(d_rhs, nr, tp.blk, sv->out(kGrpF), true, false, nullptr,
                                              sv->red(kGrpR), s));
        MG_CUDA(launch_check_batched(sv->d_state, d_rhs, nr, sv->out(kGrpR), sv->out(kGrpU), sv->out(kGrpF), sv->tol,
                                     sv->adaptive ? 1 : sv->inner, sv->max_cycles, false, sv->d_active,
                                     cudaGraphConditionalHandle(), false, s));
        const int ncyc = sv->adaptive ? sv->m_max : sv->inner;
        for (int k = 0; k < ncyc; ++k)
            for (const BatchLaunch &L : tp.cyc[sv->adaptive ? k : (k == 0 ? 0 : 1)]) {
                if (L.kind == 0)
                    MG_CUDA(launch_down_batched(d_tiles + L.off, L.ngrid, L.nblocks, sv->nu1, sv->d_active, s,
                                                L.variant));
                else if (L.kind == 1)
                    MG_CUDA(launch_up_batched(d_tiles + L.off, L.ngrid, L.nblocks, sv->nu2, sv->d_active, sv->taps,
                                              s, L.variant));
                else
                    MG_CUDA(launch_bottom_batched(d_bottom + L.off, L.ngrid, sv->nu1, sv->nu2, sv->d_active, sv->taps, s));
            }
        MG_CUDA(launch_update_batched(d_rhs, nr, tp.blk, sv->d_active, sv->red(kGrpU), s));
        const int ns = sids.back() + 1;
        MG_CUDA(cudaMemcpyAsync(sv->h_state, sv->d_state, sizeof(DevState) * ns, cudaMemcpyDeviceToHost, s));
        MG_CUDA(cudaMemcpyAsync(sv->h_active, sv->d_active, sizeof(int) * ns, cudaMemcpyDeviceToHost, s));
        MG_CUDA(cudaStreamSynchronize(s));
        // retire: projection, result out, warm start kept
        std::vector<int> retire;
        for (int sid : sids) {
            ServerSlot &sl = sv->slots[sid];
            // bookkeeping of the adaptive rule: the residual at this tick's start
            sl.rel2 = sl.rel1;
            sl.m2 = sl.m_last;
            sl.rel1 = sv->h_state[sid].rel;
            sl.nrel += 1;
            sl.m_last = m[sid];
            sl.cycles_run += m[sid];
            sl.first = false;
            if (!sv->h_active[sid]) retire.push_back(sid);
        }
        if (!retire.empty()) {
            TickPlan rp;
            for (int sid : retire) plan_rhs(rp.rhs, rp.blk, sv->slots[sid], sid);
            RhsDesc *d_r, *d_f;
            TileGrid *d_t;
            BottomGrid *d_b;
            MG_TRY(upload_plan(sv, rp, &d_r, &d_f, &d_t, &d_b));
            MG_CUDA(launch_sum_batched(d_r, (int)rp.rhs.size(), rp.blk, true, sv->red(kGrpX), s));
            MG_CUDA(launch_project_batched(d_r, (int)rp.rhs.size(), rp.blk, sv->out(kGrpX), sv->d_state, s));
            for (int sid : retire) {
                ServerSlot &sl = sv->slots[sid];
                const size_t bytes = sizeof(double) * sl.N * sl.N;
                if (sl.x_out) MG_CUDA(cudaMemcpyAsync(sl.x_out, sl.x, bytes, cudaMemcpyDefault, s));
                if (sl.stream_id >= 0) {
                    double *w = server_warm(sv, sl.stream_id, sl.N, true);
                    if (w) MG_CUDA(cudaMemcpyAsync(w, sl.x, bytes, cudaMemcpyDeviceToDevice, s));
                }
            }
            MG_CUDA(cudaStreamSynchronize(s));
            const double t_fin = sv->now_ms();
            for (int sid : retire) {
                ServerSlot &sl = sv->slots[sid];
                const DevState &ds = sv->h_state[sid];
                mg_server_result d;
                d.request_id = sl.req;
                d.stream_id = sl.stream_id;
                d.N = sl.N;
                d.status = (mg_status)ds.status;
                d.t_submit_ms = sl.t_submit;
                d.t_admit_ms = sl.t_admit;
                d.t_finish_ms = t_fin;
                d.info.outer_iters = ds.outer;
                d.info.vcycles = ds.cycles;
                d.info.rel_residual = ds.rel;
                d.info.removed_mean = ds.mu;
                d.info.update_norm = ds.unorm;
                d.info.time_ms = t_fin - sl.t_submit;
                d.info.prolong_used = MG_PROLONG_CUBIC;
                d.info.sr_fallback = 0;
                d.info.sr_cycles = 0;
                sv->done.push_back(d);
                sl.busy = false;
                sl.req = -1;
                ++finished;
            }
        }
    }
    int active = 0;
    for (const ServerSlot &sl : sv->slots) active += sl.busy ? 1 : 0;
    if (n_active) *n_active = active;
    if (n_queued) *n_queued = (int)(sv->queue.size() - sv->qhead);
    if (n_done) *n_done = finished;
    return MG_OK;
}

extern "C" {

const char *mg_status_string(mg_status s) {
    switch (s) {
        case MG_OK: return "MG_OK";
        case MG_ERR_INVALID_ARG: return "MG_ERR_INVALID_ARG";
        case MG_ERR_OOM: return "MG_ERR_OOM";
        case MG_ERR_CUDA: return "MG_ERR_CUDA";
        case MG_ERR_NOT_CONVERGED: return "MG_ERR_NOT_CONVERGED";
        case MG_ERR_TIMEOUT: return "MG_ERR_TIMEOUT";
        case MG_ERR_NO_WEIGHTS: return "MG_ERR_NO_WEIGHTS";
        case MG_ERR_BAD_WEIGHTS: return "MG_ERR_BAD_WEIGHTS";
        case MG_ERR_NONFINITE: return "MG_ERR_NONFINITE";
    }
    return "MG_ERR_UNKNOWN";
}

const char *mg_last_error(void) { return g_err; }

void mg_destroy(mg_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    batch_forget(c);
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->h32_block);
    cudaFree(c->h64_block);
    cudaFree(c->ainv32);
    cudaFree(c->d_srflag);
    cudaFree(c->ainv64);
    cudaFree(c->red_partials);
    cudaFree(c->red_counter);
    cudaFree(c->red_out);
    cudaFreeHost(c->host_out);
    cudaFree(c->f_stage);
    cudaFree(c->x_stage);
    for (SrState &v : c->sr_stage) sr_free(&v);
    sr_free(&c->sr);
    sr_windows_free(&c->srw);
    probe_free(c);
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    cudaFree(c->dstate);
    cudaFreeHost(c->hstate);
    delete c;
}

mg_status mg_setup(int levels, int N, mg_ctx **out) {
    if (!out) {
        set_err("out is NULL");
        return MG_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!is_pow2(N) || N < 8 || N > 16384 || levels < 1 || levels > kMaxLevels) {
        set_err("N=%d must be a power of two in [8, 16384], levels=%d in [1, %d]", N, levels, kMaxLevels);
        return MG_ERR_INVALID_ARG;
    }
    const int coarsest = N >> (levels - 1);
    if (coarsest < 4 || coarsest > 16 || (coarsest << (levels - 1)) != N) {
        set_err("coarsest grid N >> (levels-1) = %d must be 4, 8 or 16", coarsest);
        return MG_ERR_INVALID_ARG;
    }
    mg_ctx *c = new (std::nothrow) mg_ctx();
    if (!c) return MG_ERR_OOM;
    c->N = N;
    c->levels = levels;
    c->coarsest = coarsest;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        set_err("no CUDA device: %s", cudaGetErrorString(cudaGetLastError()));
        delete c;
        return MG_ERR_CUDA;
    }
    for (int l = 0; l < levels; ++l) c->lv[l].n = N >> l;
    fir_taps_host(&c->taps);
    auto fail = [&](mg_status s) {
        mg_destroy(c);
        return s;
    };
    const int Nc = coarsest * coarsest;
    double *h = new double[(size_t)Nc * Nc];
    float *hf = new float[(size_t)Nc * Nc];
    coarse_pinv_host(coarsest, h);
    for (int i = 0; i < Nc * Nc; ++i) hf[i] = (float)h[i];
    cudaError_t e = cudaMalloc(&c->ainv64, sizeof(double) * Nc * Nc);
    if (e == cudaSuccess) e = cudaMalloc(&c->ainv32, sizeof(float) * Nc * Nc);
    if (e == cudaSuccess) e = cudaMemcpy(c->ainv64, h, sizeof(double) * Nc * Nc, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->ainv32, hf, sizeof(float) * Nc * Nc, cudaMemcpyHostToDevice);
    delete[] h;
    delete[] hf;
    if (e == cudaSuccess) e = cudaMalloc(&c->red_partials, sizeof(double) * kMaxSlots * kRedStride);
    if (e == cudaSuccess) e = cudaMalloc(&c->red_counter, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->red_counter, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&c->red_out, sizeof(double) * 4 * kMaxSlots);
    if (e == cudaSuccess) e = cudaMemset(c->red_out, 0, sizeof(double) * 4 * kMaxSlots);
    if (e == cudaSuccess) e = cudaMallocHost(&c->host_out, sizeof(double) * 4 * kMaxSlots);
    if (e == cudaSuccess) e = cudaMalloc(&c->dstate, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMemset(c->dstate, 0, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost(&c->hstate, sizeof(DevState));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = prepare_kernels();
    if (e != cudaSuccess) {
        set_err("mg_setup: %s", cudaGetErrorString(e));
        return fail(e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA);
    }
    *out = c;
    return MG_OK;
}

mg_status mg_set_options(mg_ctx *c, mg_precision prec, int nu_pre, int nu_post, int max_cycles,
                         void *stream) {
    if (!c || (prec != MG_PREC_FP64 && prec != MG_PREC_MIXED) || nu_pre < 0 || nu_pre > 4 ||
        nu_post < 0 || nu_post > 4 || max_cycles < 1) {
        set_err("invalid options (precision %d, nu %d/%d, max_cycles %d)", (int)prec, nu_pre, nu_post,
                max_cycles);
        return MG_ERR_INVALID_ARG;
    }
    if (prec != c->prec || nu_pre != c->nu1 || nu_post != c->nu2 || max_cycles != c->max_cycles) {
        drop_graphs(c);
        batch_forget(c);
    }
    c->prec = prec;
    c->nu1 = nu_pre;
    c->nu2 = nu_post;
    c->max_cycles = max_cycles;
    c->stream = (cudaStream_t)stream;
    return MG_OK;
}

mg_status mg_set_adaptive_cycles(mg_ctx *c, int m_max, double rho) {
    if (!c || m_max < 1 || m_max > kMaxAdaptive || !(rho >= 0.0 && rho < 1.0)) {
        set_err("adaptive cycles: m_max in [1, %d], rho in [0, 1)", kMaxAdaptive);
        return MG_ERR_INVALID_ARG;
    }
    if (m_max != c->adapt_max || rho != c->rho) {
        drop_graphs(c);
        batch_forget(c);
    }
    c->adapt_max = m_max;
    c->rho = rho;
    return MG_OK;
}

mg_status mg_set_inner_cycles(mg_ctx *c, int inner) {
    if (!c || inner < 1 || inner > 16) {
        set_err("inner_cycles must be in [1, 16]");
        return MG_ERR_INVALID_ARG;
    }
    if (inner != c->inner || c->rho != 0.0) {
        drop_graphs(c);
        batch_forget(c);
    }
    c->inner = inner;
    c->rho = 0.0;  // a fixed count: adaptive inner cycles off
    return MG_OK;
}

mg_status mg_load_prolong_weights(mg_ctx *c, const void *blob, size_t bytes) {
    if (!c || !blob) {
        set_err("null context or blob");
        return MG_ERR_INVALID_ARG;
    }
    MG_CUDA(cudaSetDevice(c->device));
    drop_graphs(c);
    return sr_load(&c->sr, blob, bytes, g_err, sizeof g_err);
}

mg_status mg_solve(mg_ctx *c, const double *f, double *x, double tol, mg_prolong prolong,
                   mg_solve_info *info) {
    const auto t0 = std::chrono::steady_clock::now();
    MG_TRY(check_common(c, f, x, prolong));
    if (!(tol >= 0.0)) {
        set_err("tol must be >= 0");
        return MG_ERR_INVALID_ARG;
    }
    const bool mixed = c->prec == MG_PREC_MIXED;
    MG_TRY(ensure_hierarchy(c, !mixed));
    if (prolong == MG_PROLONG_SR && c->levels > 1 && c->lv[0].n > kBottomMax) {
        MG_TRY(sr_prepare(&c->sr, c->lv[1].n, g_err, sizeof g_err));
        if (!c->d_srflag) MG_CUDA(cudaMalloc(&c->d_srflag, sizeof(int)));
    }
    const double *fd;
    double *xd;
    bool staged;
    const bool xz = kernels_take_zero(c, mixed);
    MG_TRY(resolve_io(c, f, x, &fd, &xd, &staged, c->zero_guess, xz));
    const int N = c->N;
    const double N2 = (double)N * N;
    const double h = 2.0 * 3.14159265358979323846 / N, h2 = h * h;
    cudaStream_t s = c->stream;

    if (c->use_graphs && c->probe_kind == kProbeNone) {
        // the whole solve as one graph launch; the loop runs on the device
        SolveGraph *sg = nullptr;
        MG_TRY(get_solve_graph(c, fd, xd, prolong, tol, &sg));
        MG_CUDA(cudaGraphLaunch(sg->exec, s));
        MG_CUDA(cudaMemcpyAsync(c->hstate, c->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        if (staged) MG_CUDA(cudaMemcpyAsync(x, xd, sizeof(double) * N * N, cudaMemcpyDeviceToHost, s));
        MG_CUDA(cudaStreamSynchronize(s));
        const DevState &ds = *c->hstate;
        // the SR kernels of a conditional node run only for the V-cycles that used SR
        if (sg->adapt_max > 0)  // optional V-cycles run only when chosen
            count_launches(sg->n_pro + (long long)ds.outer * sg->n_body -
                           ((long long)ds.outer * sg->adapt_max - ds.cycles) * sg->n_cyc + sg->n_epi);
        else
            count_launches(sg->n_pro + (long long)ds.outer * (sg->n_body - (long long)c->inner * sg->n_sr) +
                           (long long)ds.sr_used * sg->n_sr + sg->n_epi);
        if (ds.tile_err) {
            MG_CUDA(cudaMemsetAsync(&c->dstate->tile_err, 0, sizeof(int), s));
            set_err("a TMA tile load of k_down timed out");
            return MG_ERR_TIMEOUT;
        }
        mg_status gst = (mg_status)ds.status;
        if (gst == MG_ERR_NONFINITE) set_err("non-finite residual (NaN or Inf in f or x)");
        if (gst == MG_ERR_NOT_CONVERGED)
            set_err("not converged: rel residual %.3e after %d V-cycles", ds.rel, ds.cycles);
        if (info) {
            info->outer_iters = ds.outer;
            info->vcycles = ds.cycles;
            info->rel_residual = ds.rel;
            info->removed_mean = ds.mu;
            info->update_norm = ds.unorm;
            const bool policy = sg->n_sr > 0;
            info->sr_cycles = policy ? ds.sr_used : (prolong == MG_PROLONG_SR ? ds.cycles : 0);
            info->prolong_used = info->sr_cycles > 0 ? MG_PROLONG_SR : MG_PROLONG_CUBIC;
            info->sr_fallback = policy ? ds.fallback : 0;
            info->time_ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
        return gst;
    }

    MG_CUDA(launch_source_sum(fd, N, c->red(kGrpF), s));

    mg_status st = MG_OK;
    int cycles = 0, outer = 0;
    double fnorm = 0.0, rel = INFINITY, mu = 0.0;
    bool first = true;
    // the prolongation policy, decided on the host with the same rule as k_policy
    const bool use_policy = mixed && prolong == MG_PROLONG_SR && c->levels > 1 && c->lv[0].n > kBottomMax;
    const bool adaptive = mixed && !use_policy && c->rho > 0.0 && c->adapt_max > 1;
    const bool fuse = fused_update(c, mixed);
    int sr_used = 0;
    bool sr_step = false, fallback = false;
    double rel_prev = 0.0;
    for (;;) {
        if (first || !fuse) {
            probe_begin(c, kProbeResidual);
            // the first residual computes and stores b = h^2 (f - mu), later ones load it
            MG_CUDA(solve_residual(c, fd, xd, mixed, first, h2, s, first && xz));
            // read f 8 (b 8 later), x 8 unless a cold start's kernels skip it; write b 8 (first), s 4
            probe_end(c, kProbeResidual, N2 * ((first ? 24.0 : 16.0) - (first && xz ? 8.0 : 0.0) + (mixed ? 4.0 : 0.0)));
        } else {
            // the update of the outer step just run, fused with this residual:
            // x + e (12 bytes a point in, 8 out; a cold start's first step
            // does not read x), b (8 in), the float residual (4 out)
            probe_begin(c, kProbeUpdateResidual);
            MG_CUDA(solve_update_residual(c, xd, nullptr, outer - 1, xz, h2, s));
            probe_end(c, kProbeUpdateResidual, N2 * (xz && outer == 1 ? 24.0 : 32.0));
        }
        MG_CUDA(cudaMemcpyAsync(c->host_out, c->red_out, sizeof(double) * 2 * kMaxSlots,
                                cudaMemcpyDeviceToHost, s));
        MG_CUDA(cudaStreamSynchronize(s));
        if (first) {
            mu = c->host_out[kGrpF * kMaxSlots] / N2;
            fnorm = sqrt(c->host_out[kGrpR * kMaxSlots + 1]);
            first = false;
        }
        const double rnorm = sqrt(c->host_out[kGrpR * kMaxSlots]) / h2;
        if (!isfinite(rnorm) || !isfinite(fnorm)) {
            set_err("non-finite residual (NaN or Inf in f or x)");
            st = MG_ERR_NONFINITE;
            break;
        }
        if (fnorm == 0.0) {  // constant source: the zero-mean solution is 0
            MG_CUDA(cudaMemsetAsync(xd, 0, sizeof(double) * N * N, s));
            rel = 0.0;
            break;
        }
        rel = rnorm / fnorm;
        if (outer > 0 && sr_step && !(rel <= kSrMinReduction * rel_prev)) fallback = true;
        sr_step = false;
        rel_prev = rel;
        if (rel <= tol) break;
        // the same rule as k_check: the V-cycles of this outer step
        const int need = adaptive ? 1 : (mixed ? c->inner : 1);
        if (cycles + need > c->max_cycles) {
            set_err("not converged: rel residual %.3e after %d V-cycles", rel, cycles);
            st = MG_ERR_NOT_CONVERGED;
            break;
        }
        int m_step = mixed ? c->inner : 1;
        if (adaptive) {
            m_step = adaptive_cycles(rel, tol, c->rho, c->adapt_max);
            if (m_step > c->max_cycles - cycles) m_step = c->max_cycles - cycles;
        }
        if (mixed) {
            for (int k = 0; k < m_step; ++k, ++cycles) {
                mg_prolong pk = prolong;
                if (use_policy) {
                    const bool sr = policy_use_sr(c->policy, cycles + 1, rel, true, fallback);
                    pk = sr ? MG_PROLONG_SR : MG_PROLONG_CUBIC;
                    if (sr) {
                        ++sr_used;
                        sr_step = true;
                    }
                } else if (prolong == MG_PROLONG_SR) {
                    ++sr_used;
                }
                MG_TRY(vcycle32_top(c, k == 0, pk));
            }
            if (!fuse) {
                probe_begin(c, kProbeUpdate);
                MG_CUDA(launch_update(xd, c->lv[0].x32, N, c->red(kGrpU), s));
                probe_end(c, kProbeUpdate, N2 * 20.0);
            }
        } else {
            MG_TRY(vcycle_rec<double>(c, 0, xd, c->lv[0].t64, c->lv[0].b64, false));
            ++cycles;
        }
        ++outer;
    }
    // the fused form leaves x in xalt after an odd number of outer steps; a
    // cold start that ran none has not written x
    const double *x_last = (fuse && (outer & 1)) ? c->xalt : nullptr;
    if (xz && outer == 0) MG_CUDA(cudaMemsetAsync(xd, 0, sizeof(double) * N * N, s));
    if (st == MG_OK || st == MG_ERR_NOT_CONVERGED) {
        MG_CUDA(launch_sum(xd, N, c->red(kGrpX), s, x_last));
        MG_CUDA(launch_project(xd, N, c->out(kGrpX), s, nullptr, x_last));
    } else if (x_last) {
        MG_CUDA(cudaMemcpyAsync(xd, x_last, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, s));
    }
    if (staged) MG_CUDA(cudaMemcpyAsync(x, xd, sizeof(double) * N * N, cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaMemcpyAsync(c->host_out, c->red_out, sizeof(double) * 4 * kMaxSlots,
                            cudaMemcpyDeviceToHost, s));
    int tile_err = 0;
    if (tma_tiles_mode()) MG_CUDA(cudaMemcpyAsync(&tile_err, &c->dstate->tile_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    if (tile_err) {
        MG_CUDA(cudaMemsetAsync(&c->dstate->tile_err, 0, sizeof(int), s));
        set_err("a TMA tile load of k_down timed out");
        return MG_ERR_TIMEOUT;
    }
    if (info) {
        info->outer_iters = outer;
        info->vcycles = cycles;
        info->rel_residual = rel;
        info->removed_mean = mu;
        info->update_norm =
            mixed && outer > 0 ? sqrt(c->host_out[fuse ? kGrpR * kMaxSlots + 1 : kGrpU * kMaxSlots]) : 0.0;
        info->sr_cycles = sr_used;
        info->prolong_used = sr_used > 0 ? MG_PROLONG_SR : MG_PROLONG_CUBIC;
        info->sr_fallback = fallback ? 1 : 0;
        info->time_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return st;
}

// One FP32 two-level cycle on A e = s (s in the finest level's b32, e from
// zero): nu red-black sweeps, the residual restricted by 2^k (full weighting
// k times), ncs sweeps of the coarse correction equation from zero, the
// coarse correction interpolated back by 2^k with the cubic spline and added.
// Returns the buffer holding e.
static mg_status two_level_cycle32(mg_ctx *c, int k, int nu, int ncs, bool sr, float **e_out) {
    cudaStream_t s = c->stream;
    float *src = c->lv[0].x32, *dst = c->lv[0].t32;
    int left = nu;
    bool first = true;
    do {  // fine sweeps in passes of <= 4; the last pass restricts its residual to level 1
        const int m = left < 4 ? left : 4;
        MG_CUDA(launch_down<float>(src, dst, c->lv[0].b32, c->lv[0].n, m, first, c->lv[1].b32, s));
        std::swap(src, dst);
        left -= m;
        first = false;
    } while (left > 0);
    for (int l = 1; l < k; ++l)  // restrict the residual on down to level k (e = 0 there)
        MG_CUDA(launch_down<float>(c->lv[l].x32, c->lv[l].t32, c->lv[l].b32, c->lv[l].n, 0, true,
                                   c->lv[l + 1].b32, s));
    float *cs = c->lv[k].x32, *cd = c->lv[k].t32;
    left = ncs;
    first = true;
    do {  // coarse sweeps from zero (their restriction to level k + 1 is not used)
        const int m = left < 4 ? left : 4;
        MG_CUDA(launch_down<float>(cs, cd, c->lv[k].b32, c->lv[k].n, m, first, c->lv[k + 1].b32, s));
        std::swap(cs, cd);
        left -= m;
        first = false;
    } while (left > 0);
    if (!sr) {
        // B-spline coefficients of the coarse correction (rows into cd, then columns back into cs)
        MG_CUDA(launch_bspline_coef(cs, cd, c->lv[k].n, 0, s));
        MG_CUDA(launch_bspline_coef(cd, cs, c->lv[k].n, 1, s));
        MG_CUDA(launch_prolong_factor(src, cs, c->lv[0].n, k, s));
        *e_out = src;
        return MG_OK;
    }
    // SR prolongation by 2^k: k stages, each the cubic spline by 2 plus the
    // generator's correction s G(e / s) (the generator applied repeatedly, as
    // Algorithm 5 applies it twice); levels k - 1 .. 1 hold the intermediate
    // corrections, the last stage adds to the smoothed fine iterate
    const float *e = cs;
    for (int j = k - 1; j >= 0; --j) {
        SrState *v = &c->sr_stage[j];
        MG_TRY(sr_correction(v, e, c->lv[j + 1].n, s, g_err, sizeof g_err));
        const int nj = c->lv[j].n;
        if (j > 0) {
            MG_CUDA(cudaMemsetAsync(c->lv[j].x32, 0, sizeof(float) * nj * nj, s));
            MG_CUDA(launch_up<float>(c->lv[j].x32, c->lv[j].t32, c->lv[j].b32, e, nj, 0, c->taps, s, v->fine_out));
            e = c->lv[j].t32;
        } else {
            MG_CUDA(launch_up<float>(src, dst, c->lv[0].b32, e, nj, 0, c->taps, s, v->fine_out));
        }
    }
    *e_out = dst;
    return MG_OK;
}

mg_status mg_two_level_solve(mg_ctx *c, const double *f, double *x, double tol, int coarsen_log2, int nu_smooth,
                             int coarse_sweeps, int max_cycles, mg_prolong prolong, mg_solve_info *info) {
    const auto t0 = std::chrono::steady_clock::now();
    MG_TRY(check_common(c, f, x, prolong));
    const int k = coarsen_log2;
    if (c->prec != MG_PREC_MIXED || k < 1 || k + 2 > c->levels || (c->N >> k) < 64 || nu_smooth < 0 ||
        nu_smooth > 64 || coarse_sweeps < 1 || coarse_sweeps > 64 || max_cycles < 1 || !(tol > 0.0)) {
        set_err("two-level solve: mixed precision; 1 <= coarsen_log2 with levels >= coarsen_log2 + 2 and "
                "N >> coarsen_log2 >= 64; 0 <= nu_smooth <= 64; 1 <= coarse_sweeps <= 64; max_cycles >= 1; tol > 0");
        return MG_ERR_INVALID_ARG;
    }
    const bool sr_on = prolong == MG_PROLONG_SR;
    if (sr_on && (k > mg_ctx::kSrStages || (c->N >> k) < 128)) {
        set_err("two-level SR prolongation: coarsen_log2 <= %d and N >> coarsen_log2 >= 128 (the generator's "
                "smallest grid)", mg_ctx::kSrStages);
        return MG_ERR_INVALID_ARG;
    }
    MG_TRY(ensure_hierarchy(c, false));
    if (sr_on) {
        for (int j = 0; j < k; ++j) MG_TRY(sr_view(&c->sr_stage[j], &c->sr, c->lv[j + 1].n, g_err, sizeof g_err));
        MG_CUDA(cudaMemsetAsync(c->sr.err, 0, sizeof(int), c->stream));  // the convolutions' bounded waits
    }
    const double *fd;
    double *xd;
    bool staged;
    MG_TRY(resolve_io(c, f, x, &fd, &xd, &staged, c->zero_guess));
    const int N = c->N;
    const double N2 = (double)N * N;
    const double h = 2.0 * 3.14159265358979323846 / N, h2 = h * h;
    cudaStream_t s = c->stream;
    MG_CUDA(launch_source_sum(fd, N, c->red(kGrpF), s));
    mg_status st = MG_OK;
    int cycles = 0, sr_used = 0;
    double fnorm = 0.0, rel = INFINITY, rel_prev = INFINITY, mu = 0.0;
    bool first = true, sr_last = false, fallback = false;
    for (;;) {  // FP64 defect correction, one FP32 two-level cycle per outer step
        MG_CUDA(solve_residual(c, fd, xd, true, first, h2, s));
        MG_CUDA(cudaMemcpyAsync(c->host_out, c->red_out, sizeof(double) * 2 * kMaxSlots, cudaMemcpyDeviceToHost, s));
        MG_CUDA(cudaStreamSynchronize(s));
        if (first) {
            mu = c->host_out[kGrpF * kMaxSlots] / N2;
            fnorm = sqrt(c->host_out[kGrpR * kMaxSlots + 1]);
            first = false;
        }
        const double rnorm = sqrt(c->host_out[kGrpR * kMaxSlots]) / h2;
        if (!isfinite(rnorm) || !isfinite(fnorm)) {
            set_err("non-finite residual (NaN or Inf in f or x)");
            st = MG_ERR_NONFINITE;
            break;
        }
        if (fnorm == 0.0) {
            MG_CUDA(cudaMemsetAsync(xd, 0, sizeof(double) * N * N, s));
            rel = 0.0;
            break;
        }
        rel = rnorm / fnorm;
        // an SR cycle that did not reduce the residual turns SR off for the rest
        if (sr_last && !(rel < rel_prev)) fallback = true;
        if (rel <= tol) break;
        if (cycles >= max_cycles) {
            set_err("not converged: rel residual %.3e after %d two-level cycles", rel, cycles);
            st = MG_ERR_NOT_CONVERGED;
            break;
        }
        // the context's policy (N_GAN alternation, S_thres switch) picks the operator
        sr_last = sr_on && policy_use_sr(c->policy, cycles + 1, rel, true, fallback);
        sr_used += sr_last ? 1 : 0;
        rel_prev = rel;
        float *e = nullptr;
        MG_TRY(two_level_cycle32(c, k, nu_smooth, coarse_sweeps, sr_last, &e));
        MG_CUDA(launch_update(xd, e, N, c->red(kGrpU), s));
        ++cycles;
    }
    if (st == MG_OK || st == MG_ERR_NOT_CONVERGED) {
        MG_CUDA(launch_sum(xd, N, c->red(kGrpX), s));
        MG_CUDA(launch_project(xd, N, c->out(kGrpX), s));
    }
    if (staged) MG_CUDA(cudaMemcpyAsync(x, xd, sizeof(double) * N * N, cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaMemcpyAsync(c->host_out, c->red_out, sizeof(double) * 4 * kMaxSlots, cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    if (sr_on) {
        int flag = 0;
        MG_CUDA(cudaMemcpy(&flag, c->sr.err, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) {
            set_err("SR generator: a bounded wait in the tensor-core convolution expired");
            st = MG_ERR_TIMEOUT;
        }
    }
    if (info) {
        info->outer_iters = cycles;
        info->vcycles = cycles;
        info->rel_residual = rel;
        info->removed_mean = mu;
        info->update_norm = cycles > 0 ? sqrt(c->host_out[kGrpU * kMaxSlots]) : 0.0;
        info->sr_cycles = sr_used;
        info->prolong_used = sr_used > 0 ? MG_PROLONG_SR : MG_PROLONG_CUBIC;
        info->sr_fallback = fallback ? 1 : 0;
        info->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return st;
}

mg_status mg_vcycle(mg_ctx *c, const double *f, double *x, mg_prolong prolong) {
    MG_TRY(check_common(c, f, x, prolong));
    const bool mixed = c->prec == MG_PREC_MIXED;
    MG_TRY(ensure_hierarchy(c, !mixed));
    if (prolong == MG_PROLONG_SR && c->levels > 1 && c->lv[0].n > kBottomMax)
        MG_TRY(sr_prepare(&c->sr, c->lv[1].n, g_err, sizeof g_err));
    const double *fd;
    double *xd;
    bool staged;
    MG_TRY(resolve_io(c, f, x, &fd, &xd, &staged));
    const int N = c->N;
    const double h = 2.0 * 3.14159265358979323846 / N, h2 = h * h;
    cudaStream_t s = c->stream;
    MG_CUDA(launch_source_sum(fd, N, c->red(kGrpF), s));
    if (mixed) {
        MG_CUDA(launch_outer_residual(fd, xd, N, h2, c->out(kGrpF), 0.0, c->lv[0].b32, false, nullptr, false,
                                      c->red(kGrpR), s));
        MG_TRY(vcycle32_top(c, true, prolong));
        MG_CUDA(launch_update(xd, c->lv[0].x32, N, c->red(kGrpU), s));
    } else {
        MG_CUDA(launch_scaled_rhs(fd, N, h2, c->out(kGrpF), c->lv[0].b64, s));
        MG_TRY(vcycle_rec<double>(c, 0, xd, c->lv[0].t64, c->lv[0].b64, false));
    }
    if (staged) MG_CUDA(cudaMemcpyAsync(x, xd, sizeof(double) * N * N, cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    return MG_OK;
}

mg_status mg_solve_batched(mg_ctx *const *ctxs, const double *const *f, double *const *x, int B,
                           double tol, mg_prolong prolong, mg_solve_info *infos) {
    if (!ctxs || !f || !x || B < 0 || !(tol >= 0.0)) {
        set_err("null batch arrays or bad tolerance");
        return MG_ERR_INVALID_ARG;
    }
    if (B == 0) return MG_OK;
    if (batch_eligible(ctxs, f, x, B, prolong)) return solve_batched_graph(ctxs, f, x, B, tol, prolong, infos);
    mg_status worst = MG_OK;
    for (int k = 0; k < B; ++k) {
        mg_status s = mg_solve(ctxs[k], f[k], x[k], tol, prolong, infos ? &infos[k] : nullptr);
        if (s != MG_OK && worst == MG_OK) worst = s;
        if (s != MG_OK && s != MG_ERR_NOT_CONVERGED) return s;
    }
    return worst;
}

unsigned long long mg_kernel_launches(void) { return launches_total(); }

mg_status mg_set_prolong_policy(mg_ctx *c, double n_gan, double s_thres) {
    if (!c || !(n_gan > 0.0) || !(s_thres >= 0.0) || (std::isfinite(n_gan) && n_gan < 1.0 && n_gan * 1e6 < 1.0)) {
        set_err("n_gan must be > 0 (INFINITY: SR only) and >= 1e-6, s_thres >= 0");
        return MG_ERR_INVALID_ARG;
    }
    ProlongPolicy p;
    if (!std::isfinite(n_gan)) {
        p = ProlongPolicy{1, 0, s_thres};
    } else if (n_gan >= 1.0) {
        p = ProlongPolicy{1, (int)std::lround(n_gan), s_thres};
    } else {
        p = ProlongPolicy{0, (int)std::lround(1.0 / n_gan), s_thres};
    }
    if (p.first_sr != c->policy.first_sr || p.period != c->policy.period || p.s_thres != c->policy.s_thres)
        drop_graphs(c);
    c->policy = p;
    return MG_OK;
}

mg_status mg_set_graph_execution(mg_ctx *c, int enable) {
    if (!c) {
        set_err("null context");
        return MG_ERR_INVALID_ARG;
    }
    c->use_graphs = enable != 0;
    return MG_OK;
}

mg_status mg_autotune(mg_ctx *c, const char *cache_path, int *n_timed) {
    if (n_timed) *n_timed = 0;
    if (!c) {
        set_err("null context");
        return MG_ERR_INVALID_ARG;
    }
    MG_CUDA(cudaSetDevice(c->device));
    MG_TRY(ensure_hierarchy(c, false));
    std::vector<TuneLevel> lv;
    for (int l = 0; l + 1 < c->levels; ++l)
        if (c->lv[l].n > bottom_max<float>())
            lv.push_back(TuneLevel{c->lv[l].n, c->lv[l].x32, c->lv[l].t32, c->lv[l].b32, c->lv[l + 1].b32,
                                   c->lv[l + 1].x32});
    char err[256] = {0};
    mg_status st = tune_levels(lv.data(), (int)lv.size(), c->nu1, c->nu2, c->taps, c->stream, c->device,
                               cache_path, n_timed, err, sizeof err);
    if (st != MG_OK) set_err("%s", err);
    return st;
}

mg_status mg_set_launch_overlap(int enable) {
    if (enable < 0 || enable > 2) {
        set_err("launch overlap mode %d: 0 (off), 1 (every kernel) or 2 (grids of <= %d blocks)", enable,
                kOverlapMaxBlocks);
        return MG_ERR_INVALID_ARG;
    }
    set_launch_overlap(enable);
    return MG_OK;
}

int mg_get_launch_overlap(void) { return launch_overlap_mode(); }

mg_status mg_set_zero_guess(mg_ctx *c, int on) {
    if (!c || (on != 0 && on != 1)) {
        set_err("null context or zero-guess flag not 0 / 1");
        return MG_ERR_INVALID_ARG;
    }
    c->zero_guess = on != 0;
    return MG_OK;
}

mg_status mg_set_coarse_cluster(int on) {
    if (on != 0 && on != 1) {
        set_err("coarse cluster: 0 (separate launches) or 1 (one cluster launch)");
        return MG_ERR_INVALID_ARG;
    }
    set_coarse_cluster(on);
    return MG_OK;
}

int mg_get_coarse_cluster(void) { return coarse_cluster_mode(); }

mg_status mg_set_fp64_separate_x_pass(int on) {
    if (on != 0 && on != 1) {
        set_err("FP64 x pass: 0 (per tile) or 1 (once per level)");
        return MG_ERR_INVALID_ARG;
    }
    set_fp64_separate_x_pass(on);
    return MG_OK;
}

int mg_get_fp64_separate_x_pass(void) { return fp64_separate_x_pass_mode(); }

mg_status mg_set_fused_update(int on) {
    if (on != 0 && on != 1) {
        set_err("fused update: 0 (separate update and residual) or 1 (one fused launch)");
        return MG_ERR_INVALID_ARG;
    }
    set_fused_update(on);
    return MG_OK;
}

int mg_get_fused_update(void) { return fused_update_mode(); }

mg_status mg_set_tma_tiles(int on) {
    if (on != 0 && on != 1) {
        set_err("TMA tiles: 0 (vector loads) or 1 (TMA-staged interior tiles)");
        return MG_ERR_INVALID_ARG;
    }
    set_tma_tiles(on);
    return MG_OK;
}

int mg_get_tma_tiles(void) { return tma_tiles_mode(); }

mg_status mg_get_tile_variant(int kind, int n, int nu, int *variant) {
    if (!variant || kind < 0 || kind > 1 || !is_pow2(n) || n < 128 || nu < 0 || nu > 4) {
        set_err("invalid tile-variant query");
        return MG_ERR_INVALID_ARG;
    }
    *variant = tile_variant(kind, n, nu);
    return MG_OK;
}

mg_status mg_set_tile_variant(int kind, int n, int nu, int variant) {
    if (kind < 0 || kind > 1 || !is_pow2(n) || n < 128 || nu < 0 || nu > 4 || variant < 0 ||
        variant >= kTileVariants || (kind == 0 && variant_runs(variant) != 1)) {
        set_err("invalid tile variant (kind 0|1, n a power of two >= 128, nu 0..4, variant 0..%d; "
                "k_down takes 0..%d)", kTileVariants - 1, kVariantPacked - 1);
        return MG_ERR_INVALID_ARG;
    }
    set_tile_variant(kind, n, nu, variant);
    return MG_OK;
}

mg_status mg_probe_kernel(mg_ctx *c, int kind, int capacity) {
    if (!c || kind < kProbeNone || kind > kProbeUpdateResidual || capacity < 0 || capacity > 4096) {
        set_err("invalid probe request");
        return MG_ERR_INVALID_ARG;
    }
    MG_CUDA(cudaSetDevice(c->device));
    probe_free(c);
    if (kind == kProbeNone || capacity == 0) return MG_OK;
    c->probe_ev = new cudaEvent_t[2 * capacity];
    for (int i = 0; i < 2 * capacity; ++i) {
        cudaError_t e = cudaEventCreate(&c->probe_ev[i]);
        if (e != cudaSuccess) {
            c->probe_cap = i / 2;
            for (int k = 2 * c->probe_cap; k < i; ++k) cudaEventDestroy(c->probe_ev[k]);
            probe_free(c);
            MG_CUDA(e);
        }
    }
    c->probe_cap = capacity;
    c->probe_kind = kind;
    return MG_OK;
}

mg_status mg_probe_read(mg_ctx *c, int *launches, double *total_ms, double *bytes) {
    if (!c) {
        set_err("null context");
        return MG_ERR_INVALID_ARG;
    }
    MG_CUDA(cudaSetDevice(c->device));
    MG_CUDA(cudaStreamSynchronize(c->stream));
    double tot = 0.0;
    for (int i = 0; i < c->probe_used; ++i) {
        float ms = 0.f;
        MG_CUDA(cudaEventElapsedTime(&ms, c->probe_ev[2 * i], c->probe_ev[2 * i + 1]));
        tot += ms;
    }
    if (launches) *launches = c->probe_used;
    if (total_ms) *total_ms = tot;
    if (bytes) *bytes = c->probe_bytes;
    c->probe_used = 0;
    c->probe_bytes = 0.0;
    return MG_OK;
}


mg_status mg_server_create(size_t hbm_budget_bytes, int nu_pre, int nu_post, int inner_cycles, int max_cycles,
                           double tol, void *cuda_stream, mg_server **out) {
    if (out) *out = nullptr;
    if (!out || nu_pre < 0 || nu_pre > 4 || nu_post < 0 || nu_post > 4 || inner_cycles < 0 || inner_cycles > 16 ||
        max_cycles < 1 || !(tol >= 0.0)) {
        set_err("invalid server options");
        return MG_ERR_INVALID_ARG;
    }
    *out = nullptr;
    mg_server *sv = new (std::nothrow) mg_server();
    if (!sv) return MG_ERR_OOM;
    MG_CUDA(cudaGetDevice(&sv->device));
    sv->stream = (cudaStream_t)cuda_stream;
    sv->budget = hbm_budget_bytes;
    sv->nu1 = nu_pre;
    sv->nu2 = nu_post;
    sv->inner = inner_cycles > 0 ? inner_cycles : 2;
    sv->adaptive = inner_cycles == 0;
    sv->max_cycles = max_cycles;
    sv->tol = tol;
    sv->slots.resize(kServerSlots);
    fir_taps_host(&sv->taps);
    auto al = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t o_state = 0, o_act = al(sizeof(DevState) * kServerSlots);
    const size_t o_out = o_act + al(sizeof(int) * kServerSlots);
    const size_t o_cnt = o_out + al(sizeof(double) * 4 * kServerSlots * kMaxSlots);
    const size_t o_part = o_cnt + al(sizeof(unsigned) * kServerSlots);
    const size_t total = o_part + al(sizeof(double) * kMaxSlots * (size_t)kServerSlots * kRedBlocks);
    cudaError_t e = cudaMalloc(&sv->dmem, total);
    if (e == cudaSuccess) e = cudaMemset(sv->dmem, 0, total);
    if (e == cudaSuccess) e = cudaMallocHost(&sv->h_state, sizeof(DevState) * kServerSlots);
    if (e == cudaSuccess) e = cudaMallocHost(&sv->h_active, sizeof(int) * kServerSlots);
    if (e != cudaSuccess) {
        set_err("server setup: %s", cudaGetErrorString(e));
        mg_server_destroy(sv);
        return MG_ERR_OOM;
    }
    char *d = (char *)sv->dmem;
    sv->d_state = (DevState *)(d + o_state);
    sv->d_active = (int *)(d + o_act);
    sv->d_out = (double *)(d + o_out);
    sv->d_counters = (unsigned *)(d + o_cnt);
    sv->d_partials = (double *)(d + o_part);
    sv->used = total;
    *out = sv;
    return MG_OK;
}

mg_status mg_server_submit(mg_server *sv, int stream_id, int N, const double *f, double *x_out,
                           long long *request_id) {
    if (!sv || !f || !is_pow2(N) || N < 8 || N > 16384) {
        set_err("invalid request (N a power of two in [8, 16384], f not null)");
        return MG_ERR_INVALID_ARG;
    }
    if (server_slot_bytes(N) > sv->budget) {
        set_err("a %d^2 request needs more than the server's memory budget", N);
        return MG_ERR_OOM;
    }
    ServerRequest rq{sv->next_id++, stream_id, N, f, x_out, sv->now_ms()};
    sv->queue.push_back(rq);
    if (request_id) *request_id = rq.id;
    return MG_OK;
}

mg_status mg_server_tick(mg_server *sv, int *n_active, int *n_queued, int *n_done) {
    if (!sv) {
        set_err("null server");
        return MG_ERR_INVALID_ARG;
    }
    return server_tick(sv, n_active, n_queued, n_done);
}

mg_status mg_server_poll(mg_server *sv, mg_server_result *result, int *got) {
    if (!sv || !got || !result) {
        set_err("null server or output");
        return MG_ERR_INVALID_ARG;
    }
    *got = 0;
    if (sv->dhead < sv->done.size()) {
        *result = sv->done[sv->dhead++];
        *got = 1;
        if (sv->dhead == sv->done.size()) {
            sv->done.clear();
            sv->dhead = 0;
        }
    }
    return MG_OK;
}

void mg_server_destroy(mg_server *sv) {
    if (!sv) return;
    cudaSetDevice(sv->device);
    if (sv->stream) cudaStreamSynchronize(sv->stream);
    for (size_t k = 0; k < sv->slots.size(); ++k)
        if (sv->slots[k].ctx) server_free_slot(sv, k);
    for (auto &w : sv->warm) cudaFree(w.second);
    cudaFree(sv->dmem);
    cudaFree(sv->d_tab);
    cudaFreeHost(sv->h_tab);
    cudaFreeHost(sv->h_state);
    cudaFreeHost(sv->h_active);
    delete sv;
}

// ---------------------------------------------------------------------------
// Operator-level entry points
// ---------------------------------------------------------------------------
static mg_status op_check(int dtype, int n, int min_n) {
    if ((dtype != 0 && dtype != 1) || !is_pow2(n) || n < min_n || n > 16384) {
        set_err("invalid dtype %d or size %d", dtype, n);
        return MG_ERR_INVALID_ARG;
    }
    return MG_OK;
}

mg_status mg_op_down(int dtype, int n, const void *x, void *x_out, const void *b, int nu,
                     int zero_init, void *bc, void *stream) {
    MG_TRY(op_check(dtype, n, 64));
    if (!x || !x_out || x == x_out || !b || !bc || nu < 0 || nu > 4) {
        set_err("invalid arguments (x and x_out must be distinct)");
        return MG_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == 0)
        MG_CUDA(launch_down<double>((const double *)x, (double *)x_out, (const double *)b, n, nu,
                                    zero_init != 0, (double *)bc, s));
    else
        MG_CUDA(launch_down<float>((const float *)x, (float *)x_out, (const float *)b, n, nu,
                                   zero_init != 0, (float *)bc, s));
    return MG_OK;
}

mg_status mg_op_up(int dtype, int n, const void *x, void *x_out, const void *b, const void *ec, int nu,
                   void *stream) {
    MG_TRY(op_check(dtype, n, 64));
    if (!x || !x_out || x == x_out || !b || !ec || nu < 0 || nu > 4) {
        set_err("invalid arguments (x and x_out must be distinct)");
        return MG_ERR_INVALID_ARG;
    }
    FirTaps taps;
    fir_taps_host(&taps);
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == 0)
        MG_CUDA(launch_up<double>((const double *)x, (double *)x_out, (const double *)b,
                                  (const double *)ec, n, nu, taps, s));
    else
        MG_CUDA(launch_up<float>((const float *)x, (float *)x_out, (const float *)b,
                                 (const float *)ec, n, nu, taps, s));
    return MG_OK;
}

mg_status mg_op_vcycle(int dtype, int n, int coarsest, void *x, const void *b, int nu1, int nu2,
                       int zero_init, void *stream) {
    MG_TRY(op_check(dtype, n, 4));
    const int nmax = dtype == 0 ? bottom_max<double>() : bottom_max<float>();
    if (n > nmax || !is_pow2(coarsest) || coarsest < 4 || coarsest > 16 || coarsest > n ||
        !x || !b || nu1 < 0 || nu1 > 4 || nu2 < 0 || nu2 > 4) {
        set_err("invalid arguments (n <= %d for this dtype, coarsest 4..16)", nmax);
        return MG_ERR_INVALID_ARG;
    }
    const int Nc = coarsest * coarsest;
    double *h = new double[(size_t)Nc * Nc];
    coarse_pinv_host(coarsest, h);
    void *d = nullptr;
    const size_t es = dtype == 0 ? sizeof(double) : sizeof(float);
    cudaError_t e = cudaMalloc(&d, es * Nc * Nc);
    if (e == cudaSuccess) {
        if (dtype == 0) {
            e = cudaMemcpy(d, h, es * Nc * Nc, cudaMemcpyHostToDevice);
        } else {
            float *hf = new float[(size_t)Nc * Nc];
            for (int i = 0; i < Nc * Nc; ++i) hf[i] = (float)h[i];
            e = cudaMemcpy(d, hf, es * Nc * Nc, cudaMemcpyHostToDevice);
            delete[] hf;
        }
    }
    delete[] h;
    FirTaps taps;
    fir_taps_host(&taps);
    cudaStream_t s = (cudaStream_t)stream;
    if (e == cudaSuccess) {
        if (dtype == 0)
            e = launch_bottom<double>((double *)x, (const double *)b, n, coarsest, nu1, nu2, zero_init != 0,
                                      (const double *)d, taps, s);
        else
            e = launch_bottom<float>((float *)x, (const float *)b, n, coarsest, nu1, nu2, zero_init != 0,
                                     (const float *)d, taps, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    MG_CUDA(e);
    return MG_OK;
}

mg_status mg_op_sr_conv(int mode, int H, int W, const void *in, const void *skip, const void *w_packed,
                        const float *bias, const float *prelu, void *out, void *stream) {
    if (!in || !w_packed || !bias || !out) {
        set_err("null pointer");
        return MG_ERR_INVALID_ARG;
    }
    return sr_conv_layer(mode, H, W, in, skip, w_packed, bias, prelu, out, (cudaStream_t)stream, g_err,
                         sizeof g_err);
}

mg_status mg_op_sr_generator(mg_ctx *c, const float *ec, int nc, float *out) {
    if (!c || !ec || !out) {
        set_err("null pointer");
        return MG_ERR_INVALID_ARG;
    }
    MG_CUDA(cudaSetDevice(c->device));
    MG_TRY(sr_prepare(&c->sr, nc, g_err, sizeof g_err));
    MG_CUDA(cudaMemsetAsync(c->sr.err, 0, sizeof(int), c->stream));
    MG_TRY(sr_correction(&c->sr, ec, nc, c->stream, g_err, sizeof g_err));
    MG_CUDA(cudaMemcpyAsync(out, c->sr.fine_out, sizeof(float) * 4 * nc * nc, cudaMemcpyDeviceToDevice, c->stream));
    int flag = 0;
    MG_CUDA(cudaMemcpyAsync(&flag, c->sr.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(cudaStreamSynchronize(c->stream));
    if (flag) {
        set_err("a bounded wait in the tensor-core convolution timed out");
        return MG_ERR_TIMEOUT;
    }
    return MG_OK;
}

mg_status mg_op_sr_layer(mg_ctx *c, int layer, int nc, const void *in, const void *skip, float *s, void *out) {
    if (!c) {
        set_err("null context");
        return MG_ERR_INVALID_ARG;
    }
    MG_CUDA(cudaSetDevice(c->device));
    return sr_layer(&c->sr, layer, nc, in, skip, s, out, c->stream, g_err, sizeof g_err);
}

mg_status mg_op_sr_windowed(mg_ctx *c, const float *ec, int nc, double p_min, double p_max, float *out) {
    if (!c || !ec || !out) {
        set_err("null pointer");
        return MG_ERR_INVALID_ARG;
    }
    if (!(p_min > 0.0) || !(p_max > p_min) || !std::isfinite(p_max)) {
        set_err("normalisation interval [%g, %g] must satisfy 0 < p_min < p_max", p_min, p_max);
        return MG_ERR_INVALID_ARG;
    }
    if (!c->sr.loaded) {
        set_err("no generator weights loaded");
        return MG_ERR_NO_WEIGHTS;
    }
    MG_CUDA(cudaSetDevice(c->device));
    MG_TRY(sr_windows_prepare(&c->srw, nc, g_err, sizeof g_err));
    MG_CUDA(cudaMemsetAsync(c->sr.err, 0, sizeof(int), c->stream));
    MG_TRY(sr_windowed(&c->srw, &c->sr, ec, nc, p_min, p_max, out, c->stream, g_err, sizeof g_err));
    int flag = 0;
    MG_CUDA(cudaMemcpyAsync(&flag, c->sr.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MG_CUDA(cudaStreamSynchronize(c->stream));
    if (flag) {
        set_err("a bounded wait in the tensor-core convolution timed out");
        return MG_ERR_TIMEOUT;
    }
    return MG_OK;
}

mg_status mg_op_outer_residual(int n, const double *f, const double *x, double mu, float *s32,
                               double *out, void *stream) {
    MG_TRY(op_check(0, n, 4));
    if (!f || !x || !out) {
        set_err("invalid arguments");
        return MG_ERR_INVALID_ARG;
    }
    double *partials = nullptr;
    unsigned *counter = nullptr;
    long long *bint = nullptr;
    int *ebt = nullptr;
    const bool tasks = s32 && n >= kResMinN;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMalloc(&partials, sizeof(double) * kMaxSlots * kRedStride);
    if (e == cudaSuccess) e = cudaMalloc(&counter, sizeof(unsigned));
    if (e == cudaSuccess && tasks) e = cudaMalloc(&bint, sizeof(long long) * n * n);
    if (e == cudaSuccess && tasks) e = cudaMalloc(&ebt, sizeof(int) * res_tasks(n));
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
    const double h = 2.0 * 3.14159265358979323846 / n;
    if (e == cudaSuccess)
        e = tasks ? launch_outer_residual_tasks(f, x, n, h * h, nullptr, mu, s32, true, bint, ebt,
                                                Reduction{partials, counter, out}, s)
                  : launch_outer_residual(f, x, n, h * h, nullptr, mu, s32, true, nullptr, false,
                                          Reduction{partials, counter, out}, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(partials);
    cudaFree(counter);
    cudaFree(bint);
    cudaFree(ebt);
    MG_CUDA(e);
    return MG_OK;
}

mg_status mg_op_convert(int dir, size_t count, const void *in, void *out, void *stream) {
    if ((dir != 0 && dir != 1) || (count && (!in || !out))) {
        set_err("invalid conversion request");
        return MG_ERR_INVALID_ARG;
    }
    if (count == 0) return MG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    MG_CUDA(launch_convert(dir, count, in, out, s));
    MG_CUDA(cudaStreamSynchronize(s));
    return MG_OK;
}

}  // extern "C"
