// mg_internal.cuh - shared definitions of the multigrid kernels and host driver.
//
// Conventions (all kernels): grids are row-major n x n, n a power of two,
// index i*n + j.  Right-hand sides are stored scaled, b = h^2 * rhs, so one
// Gauss-Seidel update reads x <- (b + sum of 4 neighbours) / 4 and the scaled
// residual is s = b - (4x - sum) = h^2 r.  Restriction of s to the n/2 grid
// yields the next scaled right-hand side directly: b_c = 4 * FW(s) because
// h_c^2 = 4 h^2.  The inner V-cycle therefore carries no mesh width at all.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mg.h"

namespace mg {

// ----------------------------------------------------------------------------
// Periodic cubic-spline midpoint filter (Sec. 2.2, "bivariate spline").
//
// For a periodic line v, the interpolating cubic spline's value halfway
// between nodes I and I+1 is sum_k g_k (v[I+k] + v[I+1-k]), k = 1, 2, ...
// From the B-spline form of the spline (prefilter 6 / (z + 4 + 1/z), midpoint
// weights (1, 23, 23, 1) / 48) the symbol of the midpoint filter is
//   G(w) = (1 + e^{iw}) (11 + cos w) / (8 (2 + cos w)),
// whose taps are g_1 = (10 - 3 sqrt 3) / 8 and g_k = 3 sqrt3 a^{k-1} (1 + a) / 8
// for k >= 2, with a = sqrt 3 - 2 (|a| = 0.268).  The taps decay
// geometrically; truncating after L taps leaves an error below
// 0.13 * 0.268^(L-2) of the largest coarse value: L = 14 (1.8e-8) is below
// float rounding and L = 28 (9e-17) below double rounding.
// ----------------------------------------------------------------------------
constexpr int kFirF32 = 14;
constexpr int kFirF64 = 28;

struct FirTaps {
    double d[kFirF64];  // g_1 .. g_L in double
    float f[kFirF64];   // the same, rounded to float (first kFirF32 used)
};

void fir_taps_host(FirTaps *t);  // fills the closed-form taps

template <typename T> struct Prec;
template <> struct Prec<float> {
    static constexpr int L = kFirF32;
    using vec = float4;
    static constexpr int VW = 4;
    static __device__ __forceinline__ float tap(const FirTaps &t, int k) { return t.f[k - 1]; }
};
template <> struct Prec<double> {
    static constexpr int L = kFirF64;
    using vec = double2;
    static constexpr int VW = 2;
    static __device__ __forceinline__ double tap(const FirTaps &t, int k) { return t.d[k - 1]; }
};

// ----------------------------------------------------------------------------
// Precision conversions on the integer pipe.  GB300 issues FP64 instructions
// (which include the hardware conversions between float and double) at a
// small fraction of its FP32 rate, and the outer kernels' few FP64 operations
// are their bottleneck; these conversions use integer instructions instead, from the
// IEEE 754 binary32 / binary64 layouts (1 sign bit; 8 / 11 exponent bits with
// bias 127 / 1023; 23 / 52 fraction bits).  Both handle every input on the
// integer pipe (a fallback to the hardware conversion would be evaluated by
// every lane of a warp and occupy the FP64 pipe); a GPU test compares them
// bit for bit with the hardware conversions.
// ----------------------------------------------------------------------------
// float -> double is exact for every input, so all classes are handled here
// (a fallback to the hardware conversion would be evaluated by every lane and
// occupy the FP64 pipe).  Normal: re-bias the exponent by 1023 - 127 = 896 and
// widen the fraction by 29 bits.  Subnormal m * 2^-149 with leading bit p:
// exponent field p + 874, fraction m shifted so that bit p lands on bit 52.
// Infinity and NaN: exponent field 0x7ff, NaNs quieted (fraction bit 51).
__device__ __forceinline__ double f32_to_f64(float v) {
    const unsigned u = __float_as_uint(v);
    const unsigned ex = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    unsigned long long body = ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)m << 29);
    if (ex == 0u) {
        const int lz = __clz(m);  // m == 0: lz = 32 and the result is a signed zero
        body = m ? (((unsigned long long)(905 - lz) << 52) |
                    (((unsigned long long)m << (21 + lz)) & 0x000fffffffffffffull))
                 : 0ull;
    } else if (ex == 0xffu) {
        body = (0x7ffull << 52) | ((unsigned long long)m << 29) | (m ? (1ull << 51) : 0ull);
    }
    return __longlong_as_double((long long)(sign | body));
}

// double -> float, round to nearest even, for every input on the integer pipe.
// Normal results: keep the top 23 of the 52 fraction bits and round on the 29
// dropped; a carry out of the fraction bumps the exponent, which is the
// correctly rounded result (infinity past the top).  Subnormal results (value
// below 2^-126): the 53-bit significand scaled to units of 2^-149 and rounded
// (a carry into bit 23 is the smallest normal).  Infinity and NaN keep their
// class (NaNs quieted).
__device__ __forceinline__ float f64_to_f32_rn(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32);
    const unsigned sign = hi & 0x80000000u;
    const int e64 = (int)((hi >> 20) & 0x7ffu);
    const int ex = e64 - 896;  // binary32 biased exponent of a normal result
    if (ex >= 1 && ex < 0xff) {
        const unsigned frac = (unsigned)((b >> 29) & 0x7fffffu);  // top 23 of the 52 fraction bits
        const unsigned rest = (unsigned)(b & 0x1fffffffu);         // the 29 bits dropped
        unsigned u = sign | ((unsigned)ex << 23) | frac;
        const unsigned half = 0x10000000u;
        u += (rest > half || (rest == half && (frac & 1u))) ? 1u : 0u;
        return __uint_as_float(u);
    }
    const unsigned long long m52 = b & 0x000fffffffffffffull;
    if (e64 == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m52 ? (0x00400000u | (unsigned)(m52 >> 29)) : 0u));
    if (ex >= 0xff) return __uint_as_float(sign | 0x7f800000u);  // overflow
    if (e64 == 0) return __uint_as_float(sign);                  // binary64 subnormals round to zero
    const unsigned long long mant = (1ull << 52) | m52;
    const int sh = 926 - e64;  // >= 30
    unsigned long long q = 0ull;
    if (sh < 64) {
        q = mant >> sh;
        const unsigned long long r = mant - (q << sh), half = 1ull << (sh - 1);
        q += (r > half || (r == half && (q & 1ull))) ? 1ull : 0ull;
    }
    return __uint_as_float(sign | (unsigned)q);
}

// ----------------------------------------------------------------------------
// Exact outer residual on the integer pipe.  The scaled residual
// s = b - 4x + xN + xS + xW + xE of six binary64 operands is summed exactly in
// a 64-bit integer and rounded once to binary32 (nearest, ties to even), the
// precision the inner V-cycles take it in.  Each operand's 53-bit significand
// is aligned so that the largest operand's leading bit sits at bit 59 (the
// centre's exponent is raised by 2 for the factor 4, which is exact) and the
// others are shifted right by their exponent difference; six such terms stay
// below 2^63.  Only bits more than 59 places below the largest operand's
// leading bit are dropped, so before the final rounding the sum is within
// 6 * 2^-59 of the largest operand: tighter than any evaluation of the same
// sum in binary64 arithmetic, whose every addition may err by 2^-53 of its
// result.  An infinite or NaN operand gives NaN.
// ----------------------------------------------------------------------------
struct ExactOperand {
    unsigned long long m;  // significand, hidden bit included
    int e;                 // biased exponent (1 for zeros and subnormals) plus log2 of the factor
    unsigned neg;          // sign of the term
    bool special;          // infinity or NaN
};

__device__ __forceinline__ ExactOperand exact_operand(double v, int log2_factor, unsigned negate) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(u >> 32);
    const int ef = (int)((hi >> 20) & 0x7ffu);
    ExactOperand o;
    o.m = (u & 0x000fffffffffffffull) | (ef ? (1ull << 52) : 0ull);
    o.e = (ef ? ef : 1) + log2_factor;
    o.neg = (hi >> 31) ^ negate;
    o.special = ef == 0x7ff;
    return o;
}

// The operand's significand in units of 2^(emax - 1082), truncated, signed.
__device__ __forceinline__ long long exact_term(const ExactOperand &o, int emax) {
    const int d = min(emax - o.e, 63);
    const long long a = (long long)((o.m << 7) >> d);
    return o.neg ? -a : a;
}

// The binary32 nearest to acc * 2^(emax - 1082).
__device__ __forceinline__ float exact_to_f32(long long acc, int emax) {
    if (acc == 0) return 0.0f;
    const unsigned sign = acc < 0 ? 0x80000000u : 0u;
    const unsigned long long a = acc < 0 ? (unsigned long long)(-acc) : (unsigned long long)acc;
    const int t = 63 - __clzll((long long)a);  // a in [2^t, 2^(t+1))
    int bf = t + emax - 955;                     // biased binary32 exponent of the value
    // bits to drop: down to a 24-bit significand, or to units of 2^-149 (subnormal)
    const int sh = bf >= 1 ? t - 23 : 933 - emax;
    unsigned long long q;
    if (sh <= 0) {
        q = a << (-sh);
    } else if (sh >= 64) {
        q = 0ull;  // a < 2^63: below half a unit
    } else {
        q = a >> sh;
        const unsigned long long r = a - (q << sh), half = 1ull << (sh - 1);
        q += (r > half || (r == half && (q & 1ull))) ? 1ull : 0ull;
    }
    if (bf < 1) return __uint_as_float(sign | (unsigned)q);  // a carry into bit 23 is the smallest normal
    if (q >> 24) {
        q >>= 1;
        ++bf;
    }
    if (bf >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((unsigned)bf << 23) | ((unsigned)q & 0x7fffffu));
}

__device__ __forceinline__ float residual_exact_f32(double b, double x, double xn, double xs, double xw,
                                                    double xe) {
    const ExactOperand o0 = exact_operand(b, 0, 0u), o1 = exact_operand(x, 2, 1u), o2 = exact_operand(xn, 0, 0u),
                       o3 = exact_operand(xs, 0, 0u), o4 = exact_operand(xw, 0, 0u), o5 = exact_operand(xe, 0, 0u);
    if (o0.special | o1.special | o2.special | o3.special | o4.special | o5.special) return __uint_as_float(0x7fc00000u);
    const int emax = max(max(max(o0.e, o1.e), max(o2.e, o3.e)), max(o4.e, o5.e));
    const long long acc = ((exact_term(o0, emax) + exact_term(o1, emax)) + (exact_term(o2, emax) + exact_term(o3, emax))) +
                          (exact_term(o4, emax) + exact_term(o5, emax));
    return exact_to_f32(acc, emax);
}

// ----------------------------------------------------------------------------
// Deterministic two-stage reductions: each block writes one partial (fixed
// order inside the block), the last block to finish sums the partials in
// index order and resets the arrival counter.  `nslot` independent sums.
// ----------------------------------------------------------------------------
// Sum of squares of float values, kept per thread as an unevaluated pair
// hi + lo of floats: each square is split exactly (v * v = p + e, e from an
// FMA) and each addition to hi is made exact by Knuth's TwoSum, its rounding
// error going to lo with e.  hi + lo equals the exact sum up to the roundings
// of the lo additions (relative error below n^2 2^-48 for n terms): an FP64-
// grade sum at FP32 instruction cost (the FP64 pipe runs at 1/64 of the FP32
// rate).  The _rn intrinsics keep the compiler from contracting p into an FMA.
struct SqSum {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float p = __fmul_rn(v, v);
        const float e = __fmaf_rn(v, v, -p);
        const float s = __fadd_rn(hi, p);
        const float bp = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

constexpr int kRedBlocks = 304;  // 2 blocks per SM on 152 SMs (4 measured slower for the FP64 kernels)
constexpr int kRedStride = 1216;  // capacity of a Reduction's partials: blocks of one launch
constexpr int kWideBlocks = 608;  // 4 blocks per SM: the update (latency-bound)
constexpr int kResBlocks = 456;   // 3 blocks per SM: the steady task-tiled residual (<= 85 registers)
constexpr int kRedThreads = 256;
constexpr int kMaxSlots = 4;

struct Reduction {
    double *partials;   // [kMaxSlots][kRedStride]
    unsigned *counter;  // 1 arrival counter
    double *out;        // [kMaxSlots] final sums
};

// sum over the block; result valid in thread 0.  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) s += sh[w];
    }
    return s;
}

// Store this block's partials (thread 0 holds vals) and let the last block
// finish the reduction.  Must be called by all threads of the block.
template <int NS>
__device__ __forceinline__ void reduce_finish(const Reduction &red, const double (&vals)[NS],
                                              double *sh) {
    __shared__ bool am_last;
    if (threadIdx.x == 0) {
        for (int k = 0; k < NS; ++k) red.partials[k * kRedStride + blockIdx.x] = vals[k];
        __threadfence();
        const unsigned ticket = atomicAdd(red.counter, 1u);
        am_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    for (int k = 0; k < NS; ++k) {
        double v = 0.0;
        // fixed assignment of partials to threads, then a fixed-order tree
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
            v += ((volatile double *)red.partials)[k * kRedStride + i];
        v = block_sum(v, sh);
        if (threadIdx.x == 0) red.out[k] = v;
    }
    if (threadIdx.x == 0) *red.counter = 0u;
}

// ----------------------------------------------------------------------------
// Batched execution: many right-hand sides of different sizes in one launch.
// A tile launch covers every grid of its table; block b belongs to the last
// grid whose first tile is <= b.  Blocks of a right-hand side whose active
// flag is 0 return at once.
// ----------------------------------------------------------------------------
struct TileGrid {
    const void *x;  // input iterate
    void *xout;     // output iterate
    const void *b;  // scaled right-hand side
    void *aux;      // down: coarse right-hand side (written); up: coarse error (read)
    int n;          // grid size
    int zero;       // down: the input iterate is taken as zero
    int tile0;      // first block of this grid in the launch
    int rhs;        // right-hand side index
    const void *extra = nullptr;     // up: fine-grid additive correction (the SR term) or null
    const int *extra_off = nullptr;  // up: the correction is skipped while *extra_off != 0 (SR dropped)
};
struct BottomGrid {  // one block each
    void *x;
    const void *b;
    const void *ainv;  // coarsest pseudo-inverse
    int n, nlev, zero, rhs;
};
struct RhsDesc {  // outer kernels: blocks [blk0, blk0 + nblk) serve this right-hand side
    const double *f;
    double *x;
    float *s32;      // float residual (inner right-hand side)
    const float *e;  // inner correction
    double *bsc;     // scaled right-hand side h^2 (f - mu), written by its first residual
                     // (n >= kResMinN: as aligned int64 per residual task, see k_outer_residual_t)
    int *ebt;        // per residual task: the exponent bsc's integers are aligned to
    int n, blk0, nblk;
    int slot;        // index of its persistent state, sums and active flag
    int first;       // this step is its first residual evaluation
    int m_prev;      // V-cycles it ran in the previous outer step (0: the launch's common count)
    double h2;
    int sr = 0;      // its finest transition adds the SR correction (batched SR solves)
    // the second FP64 iterate of a batch whose outer steps fuse the update with
    // the next residual (launch_update_residual_batched); null otherwise
    double *xalt = nullptr;
};
struct BatchRed {
    double *partials;   // [blocks][kMaxSlots]
    unsigned *counters; // [slots]
    double *out;        // [slots][kMaxSlots]
};

// ----------------------------------------------------------------------------
// FP32 tile-kernel variants: bit 0 set = 32 rows per tile (else 64), bit 1
// set = the prolongation's spline passes on float2 pairs with packed FP32x2
// instructions (two rows / two columns per work item; else one midpoint per
// work item in scalar arithmetic).  Tiles are 64
// columns wide.  All variants give bit-identical results; the process-wide
// table below (mg_tune.cu) holds the one to use for each (kernel kind: 0 down
// / 1 up, grid size, sweep count), from built-in defaults or mg_autotune.
// ----------------------------------------------------------------------------
// Tile variant v: tiles of 64 >> (v & 3) rows (64, 32, 16 or 8) by 64 columns;
// bit 2 set: the spline passes on pairs of rows / columns (packed FP32x2).
constexpr int kTileVariants = 8;
constexpr int kVariantPacked = 4;
__host__ __device__ constexpr int variant_rows(int v) { return 64 >> (v & 3); }
__host__ __device__ constexpr int variant_runs(int v) { return (v & kVariantPacked) ? 2 : 1; }
inline int variant_tiles(int n, int v) { return (n / 64) * (n / variant_rows(v)); }
int tile_variant(int kind, int n, int nu);
void set_tile_variant(int kind, int n, int nu, int variant);
// Incremented whenever a table entry changes (recorded graphs re-record).
unsigned tune_epoch();
// Programmatic dependent launch of the path's kernels (process-wide, off by
// default; the environment variable MG_LAUNCH_OVERLAP=1 starts it on).  On
// GB300 it measured slower: a 2048^2 mixed solve took 1.96 ms with it and
// 1.73 ms without.
// Programmatic dependent launch: 0 off, 1 every kernel, 2 the kernels whose
// grid has at most kOverlapMaxBlocks blocks (at most about one wave: the
// coarse levels, the bottom solve, the outer and convergence kernels), where
// launch latency is a large part of a kernel's time.
constexpr int kOverlapMaxBlocks = 304;
int launch_overlap_mode();
// 1: single-solve FP32 k_down launches on 64-row tiles stage interior tiles by TMA
int tma_tiles_mode();
void set_tma_tiles(int on);
// box (columns, rows) of a TMA-staged k_down tile with nu sweeps
void down_tma_box(int nu, int *cols, int *rows);
// k_down (nu = 2, 64-row tiles) with interior tiles staged by TMA from the 2D
// maps tmx (of x; may be null with zero_init) and tmb (of b), boxes down_tma_box;
// err: device flag set when a bounded wait runs out
cudaError_t launch_down_tma(const float *x, float *xout, const float *b, int n, int nu, bool zero_init, float *bc,
                            const CUtensorMap *tmx, const CUtensorMap *tmb, int *err, cudaStream_t s);
// the 128^2 level's down pass, the bottom V-cycle (levels <= 64^2 to the
// coarsest) and the 128^2 level's up pass in one 8-CTA cluster launch
// (V(2,2), the level's x = 0 on entry); bits of the three separate launches
cudaError_t launch_coarse_cluster(float *x, float *t, const float *b, float *xb, float *bb, int coarsest, int nu1,
                                  int nu2, const float *ainv, const FirTaps &taps, cudaStream_t s);
// 1: single solves run the coarse tail (128^2 and below) as one cluster launch
int coarse_cluster_mode();
void set_coarse_cluster(int on);
// 1: single mixed solves fuse each outer step's update with the next residual
// (launch_update_residual_tasks) on a pair of FP64 iterates
int fused_update_mode();
void set_fused_update(int on);
// 1: FP64 V-cycles refine each level's coarse error along x once
// (launch_refine_rows) before k_up, instead of per tile
int fp64_separate_x_pass_mode();
void set_fp64_separate_x_pass(int on);
// 2D tensor map of an n x n FP32 grid with boxes of cols x rows (false if the
// driver's encoder is unavailable or rejects the map)
bool make_grid_map_f32(CUtensorMap *m, void *base, int n, int cols, int rows);
bool launch_overlap_enabled();
void set_launch_overlap(int mode);

// ----------------------------------------------------------------------------
// Host-side launchers (defined in mg_kernels.cu); all return cudaError_t.
// ----------------------------------------------------------------------------
// xout = nu sweeps of x (x = 0 if zero_init); bc = 4 FW(b - (4 xout - sum)).  x != xout.
// variant: a tile variant, or -1 for the table's choice (FP64 kernels have one shape).
template <typename T>
cudaError_t launch_down(const T *x, T *xout, const T *b, int n, int nu, bool zero_init, T *bc,
                        cudaStream_t s, int variant = -1);
// xout = nu sweeps of (x + P ec + extra); extra is a fine-grid additive
// correction or null.  x != xout.
// extra_flag (device, may be null): extra is added only when *extra_flag != 0.
template <typename T>
cudaError_t launch_up(const T *x, T *xout, const T *b, const T *ec, int n, int nu,
                      const FirTaps &taps, cudaStream_t s, const T *extra = nullptr, int variant = -1,
                      const int *extra_flag = nullptr, const T *xr = nullptr);
// The prolongation's x pass on its own (FP64): xr[I][2J] = ec[I][J], xr[I][2J+1]
// = the row pass's midpoint, for the (n/2) x (n/2) coarse error ec; xr is
// (n/2) x n.  launch_up<double> with xr loads these rows instead of refining
// them per tile (bit-identical).  n a power of two >= 128.
cudaError_t launch_refine_rows(const double *ec, double *xr, int n, const FirTaps &taps, cudaStream_t s);
template <typename T>
cudaError_t launch_bottom(T *x, const T *b, int n, int coarsest, int nu1, int nu2, bool zero_init,
                          const T *ainv, const FirTaps &taps, cudaStream_t s);
// Grids up to bottom_max<T>() squared run the bottom kernel (one block, the
// whole V-cycle below in shared memory).  One SM is slower than the tile
// kernels on the whole GPU from 128^2 up, so the limit is 64 for both types
// (the kernel itself fits 128^2 in FP32).
constexpr int kBottomMax = 64;  // the FP32 limit (batched solves and the server are FP32)
template <typename T> constexpr int bottom_max() { return 64; }

// Set the message mg_last_error() returns on the calling thread.
void set_last_error(const char *msg);

// Process-wide count of kernels this library has launched (instrumentation).
// Launches recorded into a CUDA graph are taken back after capture and
// counted again for every replay.
void count_launches(long long k);
unsigned long long launches_total();

// Set the shared-memory attributes of every tile kernel on the current device
// (called once per context, so that later launches, including those recorded
// into graphs, need no attribute calls).
cudaError_t prepare_kernels();

// Device-side state of one solve, advanced by k_check (graph execution).
struct DevState {
    int cycles;       // V-cycles run
    int outer;        // outer steps (loop iterations) run
    int status;       // MG_OK, MG_ERR_NOT_CONVERGED or MG_ERR_NONFINITE
    int zero_source;  // f is constant: the zero-mean solution is 0
    double fnorm;     // ||f - mean f||_2
    double rel;       // last relative residual
    double unorm;     // ||e||_2 of the last update
    double mu;        // mean of f
    int sr_used;      // V-cycles that used the SR prolongation
    int sr_step;      // the current outer step used it
    int fallback;     // SR stopped for this solve (an outer step with SR did not halve the residual)
    int m_next;       // V-cycles of the next outer step (adaptive inner cycles)
    double rel_prev;  // relative residual before the current outer step
    int tile_err;     // a TMA tile load's bounded wait ran out (set by k_down_tma)
};

// Prolongation policy of a solve with the SR prolongation (the hybrid
// operator choice of Sec. 4.2 and Algorithm 6).  n_gan >= 1: n_gan SR cycles
// per cubic cycle (first = SR); n_gan < 1: 1/n_gan cubic cycles per SR cycle
// (first = cubic); period = 0 means the first operator only.  Once the
// relative residual of the latest outer step is <= s_thres (> 0), the second
// operator is used from then on.  V-cycle i (1-based, counted over the solve)
// uses the first operator when i mod (period + 1) != 0.
struct ProlongPolicy {
    int first_sr;   // first operator is SR (1) or cubic (0)
    int period;     // consecutive first-operator cycles, 0 = no second operator by count
    double s_thres;
};
__host__ __device__ inline bool policy_use_sr(const ProlongPolicy &p, int i, double rel, bool have_rel,
                                              bool fallback) {
    if (fallback) return false;
    const bool switched = p.s_thres > 0.0 && have_rel && rel <= p.s_thres;
    const bool first = !switched && (p.period == 0 || i % (p.period + 1) != 0);
    return first ? p.first_sr != 0 : p.first_sr == 0;
}
// An outer step that used SR must reduce the relative residual by at least
// this factor, else SR is dropped for the rest of the solve.
constexpr double kSrMinReduction = 0.5;

// Decide V-cycle (st->cycles + k + 1) of the running solve on the device:
// *flag = use SR, the IF node's condition likewise, st->sr_used / sr_step.
cudaError_t launch_policy(DevState *st, int k, ProlongPolicy p, int *flag, cudaGraphConditionalHandle handle,
                          cudaStream_t s);

// Adaptive inner cycles: the V-cycles of the next outer step, the smallest
// m in [1, m_max] with rel * rho^m <= tol, rho the expected contraction per
// V-cycle.  Multiplications only, so host and device take the same decision.
__host__ __device__ inline int adaptive_cycles(double rel, double tol, double rho, int m_max) {
    double r = rel;
    int m = 0;
    do {
        r *= rho;
        ++m;
    } while (m < m_max && r > tol);
    return m;
}
constexpr int kMaxAdaptive = 4;  // optional cycles are IF nodes 2 .. kMaxAdaptive of a graph body

// Handles of the IF nodes around the optional V-cycles 2 .. m_max of an outer step.
struct CycleHandles {
    cudaGraphConditionalHandle h[kMaxAdaptive - 1];
};

// Convergence test of one outer step: reads the residual sums, updates the
// state and sets the graph's loop condition (1 = run another step).  With
// rho > 0 the step just run had st->m_next cycles and the next one gets
// adaptive_cycles(...) of them (IF handles 2 .. step set accordingly); with
// rho = 0 every step has `step` cycles.
cudaError_t launch_check(DevState *st, const double *rsum, const double *usum, const double *fsum,
                         double n2, double h2, double tol, int step, int max_cycles, bool first,
                         cudaGraphConditionalHandle handle, cudaStream_t s, double rho = 0.0,
                         CycleHandles ifh = CycleHandles{});

// batched forms (float tile kernels; outer kernels)
// every grid of one batched launch uses the same variant; nblocks = sum of variant_tiles
cudaError_t launch_down_batched(const TileGrid *tab, int ngrid, int nblocks, int nu, const int *active,
                                cudaStream_t s, int variant);
cudaError_t launch_up_batched(const TileGrid *tab, int ngrid, int nblocks, int nu, const int *active,
                              const FirTaps &taps, cudaStream_t s, int variant);
cudaError_t launch_bottom_batched(const BottomGrid *tab, int ngrid, int nu1, int nu2, const int *active,
                                  const FirTaps &taps, cudaStream_t s);
// sums of f (of_x = false) or of x (of_x = true) per right-hand side -> red.out[r][0]
// of_x with st: each right-hand side's x is read from its xalt when its slot's
// outer-step count is odd (a batch with the fused outer step)
cudaError_t launch_sum_batched(const RhsDesc *rd, int nrhs, int nblocks, bool of_x, BatchRed red,
                               cudaStream_t s, const DevState *st = nullptr);
// want_fnorm: the right-hand sides at their first residual (all with
// first_all, else those whose descriptor says first) compute b = h^2 (f - mu)
// in FP64, store it to bsc and sum (f - mu)^2; all others load b from bsc.
cudaError_t launch_outer_residual_batched(const RhsDesc *rd, int nrhs, int nblocks, const double *fsum,
                                          bool want_fnorm, bool first_all, const int *active, BatchRed red,
                                          cudaStream_t s);
cudaError_t launch_update_batched(const RhsDesc *rd, int nrhs, int nblocks, const int *active, BatchRed red,
                                  cudaStream_t s);
// fused: each right-hand side's last iterate is in its xalt when its slot's
// outer-step count is odd (the projection writes x)
cudaError_t launch_project_batched(const RhsDesc *rd, int nrhs, int nblocks, const double *xsum,
                                   const DevState *st, cudaStream_t s, bool fused = false);
// Batched launch_update_residual_tasks: every active right-hand side (n >=
// kResMinN, xalt set) takes x + e from one buffer of (x, xalt) to the other,
// by its slot's outer-step count (st[slot].outer, read before the check
// advances it), and its residual; out[slot][0] = the residual's sum of
// squares, out[slot][1] = that of e.
cudaError_t launch_update_residual_batched(const RhsDesc *rd, int nrhs, int nblocks, const DevState *st,
                                           const int *active, BatchRed red, cudaStream_t s);
// first: every entry is at its first residual (else each entry's own flag);
// use_handle: set the graph loop condition (inside a graph only)
// rho > 0: adaptive inner cycles (batch_m: [0] the next step's V-cycles, [1] total run; ifh: IF handles)
cudaError_t launch_check_batched(DevState *st, const RhsDesc *rd, int nrhs, const double *rsum,
                                 const double *usum, const double *fsum, double tol, int step, int max_cycles,
                                 bool first, int *active, cudaGraphConditionalHandle handle, bool use_handle,
                                 cudaStream_t s, double rho = 0.0, CycleHandles ifh = CycleHandles{},
                                 int *batch_m = nullptr);

cudaError_t launch_source_sum(const double *f, int n, Reduction red, cudaStream_t s);
cudaError_t launch_scaled_rhs(const double *f, int n, double h2, const double *f_sum,
                              double *b, cudaStream_t s);
// Cubic spline prolongation by 2^lgf in one step (the paper's two-level
// configuration).  Coefficients: c = the periodic cubic B-spline coefficients
// of the nc x nc coarse grid e, a truncated exact inverse of the B-spline
// collocation filter (1, 4, 1) / 6 along one axis (dir 0 rows, 1 columns):
// c_J = a_0 e_J + sum_{k=1..kBspTaps} a_k (e_{J+k} + e_{J-k}),
// a_k = sqrt(3) (sqrt(3) - 2)^k.  Prolongation: e_f(i, j) += the tensor
// cubic B-spline sum over the 4 x 4 coefficients around (i, j) / 2^lgf.
constexpr int kBspTaps = 14;  // |sqrt(3) - 2|^15 < 3e-9: below FP32 rounding
cudaError_t launch_bspline_coef(const float *e, float *c, int nc, int dir, cudaStream_t s);
cudaError_t launch_prolong_factor(float *ef, const float *c, int n, int lgf, cudaStream_t s);

// Task-tiled outer residual of mixed solves (grids of n >= kResMinN): each
// warp takes tasks of 32 columns x kResRows rows and aligns all of a task's
// operands to one exponent, the task's largest.  The first residual of a
// solve computes b = h^2 (f - mu) and stores it as int64 aligned to the
// task's largest b exponent (bint, with that exponent in ebt[task]); later
// residuals load it.  ebt holds res_tasks(n) entries.
constexpr int kResRows = 8;
constexpr int kResMinN = 32;
inline size_t res_tasks(int n) { return (size_t)(n / 32) * (size_t)(n / kResRows); }
// xzero (first only): x is zero (a cold start) and is not read.
cudaError_t launch_outer_residual_tasks(const double *f, const double *x, int n, double h2, const double *mu_sum,
                                        double mu_host, float *s32, bool first, long long *bint, int *ebt,
                                        Reduction red, cudaStream_t s, bool xzero = false);

// Scaled outer residual.  b = h^2 (f - mu) is computed from f in FP64 (and
// stored to bsc when bsc is given), or with load_b taken from bsc as an
// earlier call stored it; the stencil sum is exact (residual_exact_f32).
cudaError_t launch_outer_residual(const double *f, const double *x, int n, double h2,
                                  const double *mu_sum, double mu_host, float *s32,
                                  bool want_fnorm, double *bsc, bool load_b, Reduction red, cudaStream_t s);
cudaError_t launch_update(double *x, const float *e, int n, Reduction red, cudaStream_t s);
// An outer step's update fused with the next (steady) task-tiled residual:
// x_new = x_old + e into the other buffer of the pair (xa, xb), the residual
// of x_new into s32, out[0] = sum of its squares, out[1] = sum of e^2.  The
// outer step index k from 0 (*step_dev if non-null, else step_host) selects
// the source: xb when k is odd, else xa; with zero_first, step 0's source is
// zero and is not read.  x_new and the residual are bit for bit those of
// launch_update followed by launch_outer_residual_tasks(first = false).
cudaError_t launch_update_residual_tasks(double *xa, double *xb, const int *step_dev, int step_host, bool zero_first,
                                         const float *e, int n, double h2, float *s32, long long *bint, int *ebt,
                                         Reduction red, cudaStream_t s);
// x -= sum / n^2, or x = 0 where *zero_flag is set (zero_flag may be null);
// with alt given the values are read from alt (when par is null or *par is
// odd; par is a device pointer, read when the kernel runs); with zero_first
// (par required) the values are zero when *par == 0 and nothing is read.
cudaError_t launch_project(double *x, int n, const double *sum, cudaStream_t s, const int *zero_flag = nullptr,
                           const double *alt = nullptr, const int *par = nullptr, bool zero_first = false);
// the sum of x (of alt when alt is given and par is null or *par is odd; 0
// with zero_first when *par == 0)
cudaError_t launch_sum(const double *x, int n, Reduction red, cudaStream_t s, const double *alt = nullptr,
                       const int *par = nullptr, bool zero_first = false);
// out[i] = the integer-pipe conversion of in[i] (dir 0: double -> float, 1: float -> double)
cudaError_t launch_convert(int dir, size_t count, const void *in, void *out, cudaStream_t s);

}  // namespace mg
