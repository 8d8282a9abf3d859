// mg_kernels.cu - stencil kernels of the periodic multigrid V-cycle (sm_103a).
//
// Steps of Algorithm 6 (Appendix A) and Fig. 1a, fused into tile passes:
//   k_down   : nu red-black Gauss-Seidel sweeps + residual + full weighting
//              (relax, r = f - A p, restrict), one read of x and b, one write
//              of x and of the quarter-size coarse right-hand side.
//   k_up     : periodic cubic-spline prolongation of the coarse error (Sec. 2.2)
//              added to x, then nu sweeps; one read of x, b and the coarse
//              error, one write of x.
//   Both read x from one buffer and write the result to another: a block's
//   halo overlaps its neighbours' interiors, so an in-place update would let a
//   block of a later wave read values another block has already smoothed.
//   k_bottom : every level from <= 64 x 64 down to the coarsest grid in one
//              thread block, with all grids resident in shared memory and the
//              coarsest grid solved exactly by a pseudo-inverse matvec.
// Tiles are staged in shared memory with 16-byte vector loads; several
// Gauss-Seidel sweeps run on one staged tile (temporal blocking), the valid
// region shrinking by one point per half-sweep, so the halo is 2 per sweep.
// Within one colour every update reads only the other colour, so the fused
// sweeps give exactly the values of separate half-sweeps.
//
// Outer kernels (FP64 defect correction around FP32 V-cycles): source sum,
// scaled right-hand side, the residual of the FP64 iterate (summed exactly on
// the integer pipe) with norms and float conversion, FP64 solution update,
// zero-mean projection.  Sums are deterministic (fixed grid, fixed-order
// trees, last-block finish).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <type_traits>
#include <utility>

#include "mg_internal.cuh"
#include "mg_tc.cuh"

namespace mg {

static std::atomic<long long> g_launches{0};
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
unsigned long long launches_total() { return (unsigned long long)g_launches.load(std::memory_order_relaxed); }

void fir_taps_host(FirTaps *t) {
    const double s3 = sqrt(3.0), a = s3 - 2.0;
    t->d[0] = (10.0 - 3.0 * s3) / 8.0;
    double p = a;  // a^{k-1}
    for (int k = 2; k <= kFirF64; ++k) {
        t->d[k - 1] = 3.0 * s3 * p * (1.0 + a) / 8.0;
        p *= a;
    }
    for (int k = 0; k < kFirF64; ++k) t->f[k] = (float)t->d[k];
}

namespace {

constexpr int kThreads = 256;  // threads per tile block

// Programmatic dependent launch.  Every kernel of the path starts with
// pdl_enter(): griddepcontrol.wait blocks until the grids this one depends on
// have completed and their writes are visible.  A block signals its
// dependents implicitly when it exits, so the next kernel in the stream is
// launched once every block of this grid has finished its work (its launch
// then overlaps this grid's completion and memory flush) and never takes SM
// resources from blocks of this grid still waiting to run.  For a kernel
// launched without the attribute the wait returns at once.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Packed FP32x2 arithmetic (Blackwell): two IEEE round-to-nearest float
// operations per instruction, lane by lane the same bits as the scalar ones.
__device__ __forceinline__ unsigned long long f2_bits(float2 v) {
    unsigned long long u;
    memcpy(&u, &v, sizeof u);
    return u;
}
__device__ __forceinline__ float2 f2_from(unsigned long long u) {
    float2 v;
    memcpy(&v, &u, sizeof v);
    return v;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from(r);
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return f2_from(r);
}

// Launch k with the programmatic-stream-serialization attribute when launch
// overlap applies to it (mode 1, or mode 2 and a grid of at most
// kOverlapMaxBlocks blocks), else as a plain launch.
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    const int mode = launch_overlap_mode();
    if (mode == 1 || (mode == 2 && (size_t)grid.x * grid.y * grid.z <= (size_t)kOverlapMaxBlocks)) {
        cfg.attrs = at;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}


__host__ __device__ constexpr int round_up(int v, int m) { return (v + m - 1) / m * m; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Output tiles are TY x 64 points.  FP32 kernels come in variants (see
// variant_rows / variant_runs): 64, 32, 16 or 8 rows per tile, and NJ = 1 (scalar
// spline passes, one midpoint per work item) or NJ = 2 (the spline passes on
// float2 pairs of rows / columns with packed FP32x2 instructions).  Every
// variant computes the same values in the same order, so the choice only
// changes speed.  FP64 tiles are 32 x 64 with NJ = 1, to keep the staged tiles
// within shared memory.
constexpr int kTX = 64;
template <typename T> struct Fixed64;  // the FP64 shape
template <> struct Fixed64<double> {
    static constexpr int TY = 32, NJ = 1;
};

// Copy rows [r0, r0+R) x cols [c0, c0+C) of the periodic n x n grid g into
// shared memory s (pitch SP), with 16-byte vector loads.  c0 and C are
// multiples of the vector width.
template <typename T, int R, int C, int SP>
__device__ __forceinline__ void load_tile(T *__restrict__ s, const T *__restrict__ g, int n, int r0,
                                          int c0) {
    using V = typename Prec<T>::vec;
    constexpr int VW = Prec<T>::VW;
    constexpr int CV = C / VW;
    for (int idx = threadIdx.x; idx < R * CV; idx += blockDim.x) {
        const int rr = idx / CV, cv = idx - rr * CV;
        const int gr = (r0 + rr) & (n - 1), gc = (c0 + cv * VW) & (n - 1);
        const V v = __ldg(reinterpret_cast<const V *>(g + (size_t)gr * n + gc));
        *reinterpret_cast<V *>(s + rr * SP + cv * VW) = v;
    }
}

// ---------------------------------------------------------------------------
// Colour-split staging.  A staged R x C tile (C even) is held as two arrays,
// red and black, of R x CK entries (CK = C / 2): staged point (r, c) of
// colour q = (r + c) & 1 is entry r * CK + (c >> 1) of array q.  Tile
// origins and halos are even, so q is the point's red-black colour on the
// grid.  For a point (r, k) of colour q, with o = (r + q) & 1 and P the other
// colour's array, the neighbours are N = P[r-1][k], S = P[r+1][k],
// W = P[r][k-1+o], E = P[r][k+o]: unit stride across a warp, no bank
// conflicts, and no division in the index arithmetic.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void scatter_vec(float *red, float *black, int rr, int c, int CK, float4 v) {
    float2 a = make_float2(v.x, v.z), b2 = make_float2(v.y, v.w);
    const bool even = (rr & 1) == 0;  // c is a multiple of 4: parity of (rr + c) is rr's
    *reinterpret_cast<float2 *>(red + rr * CK + (c >> 1)) = even ? a : b2;
    *reinterpret_cast<float2 *>(black + rr * CK + (c >> 1)) = even ? b2 : a;
}
__device__ __forceinline__ void scatter_vec(double *red, double *black, int rr, int c, int CK, double2 v) {
    const bool even = (rr & 1) == 0;
    red[rr * CK + (c >> 1)] = even ? v.x : v.y;
    black[rr * CK + (c >> 1)] = even ? v.y : v.x;
}
__device__ __forceinline__ float4 gather_vec(const float *red, const float *black, int rr, int c, int CK) {
    const float2 r = *reinterpret_cast<const float2 *>(red + rr * CK + (c >> 1));
    const float2 b2 = *reinterpret_cast<const float2 *>(black + rr * CK + (c >> 1));
    return (rr & 1) == 0 ? make_float4(r.x, b2.x, r.y, b2.y) : make_float4(b2.x, r.x, b2.y, r.y);
}
__device__ __forceinline__ double2 gather_vec(const double *red, const double *black, int rr, int c, int CK) {
    const double r = red[rr * CK + (c >> 1)], b2 = black[rr * CK + (c >> 1)];
    return (rr & 1) == 0 ? make_double2(r, b2) : make_double2(b2, r);
}

// Load rows [r0, r0+R) x cols [c0, c0+C) of the periodic grid into a split tile.
template <typename T, int R, int C>
__device__ __forceinline__ void load_split(T *red, T *black, const T *__restrict__ g, int n, int r0,
                                           int c0) {
    using V = typename Prec<T>::vec;
    constexpr int VW = Prec<T>::VW;
    constexpr int CV = C / VW;
    for (int idx = threadIdx.x; idx < R * CV; idx += blockDim.x) {
        const int rr = idx / CV, cv = idx - rr * CV;
        const int gr = (r0 + rr) & (n - 1), gc = (c0 + cv * VW) & (n - 1);
        const V v = __ldg(reinterpret_cast<const V *>(g + (size_t)gr * n + gc));
        scatter_vec(red, black, rr, cv * VW, C / 2, v);
    }
}

// Two-phase tile loader: issue() starts every 16-byte load of the tile into
// registers (a thread's share, all independent, so their latencies overlap),
// scatter() writes them into the colour-split arrays.  Between the two a
// block can do other work with the loads in flight.
template <typename T, int R, int C, int NT = kThreads, bool COH = false>
struct SplitLoad {
    using V = typename Prec<T>::vec;
    static constexpr int VW = Prec<T>::VW, CV = C / VW, ITEMS = R * CV;
    static constexpr int PER = (ITEMS + NT - 1) / NT;
    V v[PER];
    __device__ __forceinline__ void issue(const T *__restrict__ g, int n, int r0, int c0) {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * NT;
            if (idx < ITEMS) {
                const int rr = idx / CV, cv = idx - rr * CV;
                const int gr = (r0 + rr) & (n - 1), gc = (c0 + cv * VW) & (n - 1);
                const V *src = reinterpret_cast<const V *>(g + (size_t)gr * n + gc);
                v[i] = COH ? __ldcg(src) : __ldg(src);
            }
        }
    }
    __device__ __forceinline__ void scatter(T *red, T *black) const {
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * NT;
            if (idx < ITEMS) {
                const int rr = idx / CV, cv = idx - rr * CV;
                scatter_vec(red, black, rr, cv * VW, C / 2, v[i]);
            }
        }
    }
};

// Store staged rows [r_s, r_s+TY) x cols [c_s, c_s+TX) of a split tile to
// global rows [gy, gy+TY) x cols [gx, gx+TX).
template <typename T, int TY, int TX, int C>
__device__ __forceinline__ void store_split(T *__restrict__ g, const T *red, const T *black, int n,
                                            int gy, int gx, int r_s, int c_s) {
    using V = typename Prec<T>::vec;
    constexpr int VW = Prec<T>::VW;
    constexpr int CV = TX / VW;
    for (int idx = threadIdx.x; idx < TY * CV; idx += blockDim.x) {
        const int rr = idx / CV, cv = idx - rr * CV;
        const V v = gather_vec(red, black, r_s + rr, c_s + cv * VW, C / 2);
        *reinterpret_cast<V *>(g + (size_t)(gy + rr) * n + gx + cv * VW) = v;
    }
}

// Rows of the remainder columns that one warp instruction can cover without
// shared-memory bank conflicts: the largest g <= 32 / kr for which the g rows'
// runs of kr elements (a row is ck elements of wb 4-byte words further on)
// fall into disjoint banks.
__host__ __device__ constexpr int strip_rem_rows(int ck, int kr, int wb) {
    int best = 1;
    for (int g = 2; g * kr <= 32; ++g) {
        bool ok = true;
        for (int a = 0; a < g && ok; ++a)
            for (int c = a + 1; c < g && ok; ++c) {
                const int d = ((c - a) * ck * wb) % 32;  // bank offset of row c against row a
                const int w = kr * wb;                   // banks a run of kr elements covers
                ok = d >= w && 32 - d >= w;
            }
        if (ok) best = g;
    }
    return best;
}

// Visit the points of colour q in staged rows [r_lo, r_hi), split columns
// [1, CK - 1), and call body(p, N, S, W, E) with the split index p = r * CK + k
// of each and its four neighbours (the other colour).  Columns 1 .. 32 go as
// vertical strips, one warp per block of consecutive rows, lane k - 1 walking
// down column k with N and the centre kept in registers: a warp's 32 lanes
// read 32 consecutive elements of one row, so no bank conflicts.  The
// remaining columns 33 .. CK - 2 go in groups of rows chosen so that one warp
// instruction's rows fall into disjoint banks (strip_rem_rows).
// Walk split column k down rows [ra, rb) (ra < rb), calling body for each
// point of colour q with N and the centre carried in registers.  Rows
// alternate which neighbour (west or east) sits in the same split column; the
// walk takes two rows per step with that alternation fixed at compile time,
// after one branch on the first row's parity.
template <int CK, typename T, typename Body>
__device__ __forceinline__ void strip_walk(const T *__restrict__ P, int ra, int rb, int k, int q, Body &body) {
    T pN = P[(ra - 1) * CK + k];
    T pC = P[ra * CK + k];
    auto row = [&](int r, auto odd) {
        constexpr int o = decltype(odd)::value;
        const T pS = P[(r + 1) * CK + k];
        const T side = P[r * CK + k - 1 + 2 * o];
        if constexpr (o) body(r * CK + k, pN, pS, pC, side);
        else body(r * CK + k, pN, pS, side, pC);
        pN = pC;
        pC = pS;
    };
    using O0 = std::integral_constant<int, 0>;
    using O1 = std::integral_constant<int, 1>;
    int r = ra;
    if (((ra + q) & 1) == 0) {
        for (; r + 1 < rb; r += 2) {
            row(r, O0{});
            row(r + 1, O1{});
        }
        if (r < rb) row(r, O0{});
    } else {
        for (; r + 1 < rb; r += 2) {
            row(r, O1{});
            row(r + 1, O0{});
        }
        if (r < rb) row(r, O1{});
    }
}

// Small tiles (a few rows per thread) are latency-bound rather than bound by
// shared-memory bandwidth; there the rows go as NSEG segments of KW = CK - 2
// consecutive threads each (warps may straddle two segments), which keeps the
// chain of dependent rows per thread shortest.
template <int CK, int NT = kThreads, typename T, typename Body>
__device__ __forceinline__ void colour_segments(const T *__restrict__ P, int r_lo, int r_hi, int q,
                                                Body body) {
    constexpr int KW = CK - 2;
    constexpr int NSEG = NT / KW;
    const int seg = threadIdx.x / KW;
    if (seg >= NSEG) return;
    const int k = 1 + (threadIdx.x - seg * KW);
    const int per = (r_hi - r_lo + NSEG - 1) / NSEG;
    const int ra = r_lo + seg * per;
    const int rb = min(r_hi, ra + per);
    if (ra >= rb) return;
    // per row parity (segments of one warp may start on rows of either parity,
    // so a parity branch would diverge)
    T pN = P[(ra - 1) * CK + k];
    T pC = P[ra * CK + k];
    for (int r = ra; r < rb; ++r) {
        const T pS = P[(r + 1) * CK + k];
        const int o = (r + q) & 1;
        const T side = P[r * CK + k - 1 + 2 * o];
        const T W = o ? pC : side;
        const T E = o ? side : pC;
        body(r * CK + k, pN, pS, W, E);
        pN = pC;
        pC = pS;
    }
}

template <int CK, bool STRIPS, int NT = kThreads, typename T, typename Body>
__device__ __forceinline__ void colour_strips(const T *__restrict__ P, int r_lo, int r_hi, int q,
                                              Body body) {
    if constexpr (!STRIPS) {
        colour_segments<CK, NT>(P, r_lo, r_hi, q, body);
        return;
    }
    constexpr int KW = CK - 2;
    constexpr int KM = KW < 32 ? KW : 32;  // columns of the strips
    constexpr int KR = KW - KM;            // remainder columns
    constexpr int NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rows = r_hi - r_lo;
    if (lane < KM) {
        const int per = (rows + NW - 1) / NW;
        const int ra = r_lo + warp * per;
        const int rb = min(r_hi, ra + per);
        const int k = 1 + lane;
        if (ra < rb) strip_walk<CK>(P, ra, rb, k, q, body);
    }
    if constexpr (KR > 0) {
        constexpr int RG = strip_rem_rows(CK, KR, (int)(sizeof(T) / 4));
        const int dr = lane / KR, k = KM + 1 + (lane - dr * KR);
        if (dr < RG) {
            for (int r = r_lo + warp * RG + dr; r < r_hi; r += NW * RG) {
                const T pN = P[(r - 1) * CK + k], pS = P[(r + 1) * CK + k], pC = P[r * CK + k];
                const int o = (r + q) & 1;
                const T side = P[r * CK + k - 1 + 2 * o];
                body(r * CK + k, pN, pS, o ? pC : side, o ? side : pC);
            }
        }
    }
}

// One Gauss-Seidel half-sweep of colour q: x <- (b + (((N + S) + W) + E)) / 4.
// X and B point at the red arrays; the black ones follow A entries later.
// STRIPS: the conflict-free strip mapping (tiles of >= 32 rows), else segments.
template <int CK, int A, bool STRIPS, int NT = kThreads, typename T>
__device__ __forceinline__ void half_sweep(T *X, const T *B, int r_lo, int r_hi, int q) {
    T *Xq = X + q * A;
    const T *Bq = B + q * A;
    colour_strips<CK, STRIPS, NT>(X + (q ^ 1) * A, r_lo, r_hi, q, [&](int p, T N, T S, T W, T E) {
        Xq[p] = (Bq[p] + (((N + S) + W) + E)) * T(0.25);
    });
}

// ---------------------------------------------------------------------------
// k_down: NU sweeps, residual, full-weighting restriction of one tile.
// ---------------------------------------------------------------------------
template <typename T, int NU, int TY_>
struct DownCfg {
    static constexpr int TY = TY_, TX = kTX;
    static constexpr int VW = Prec<T>::VW;
    static constexpr int H = 2 * NU + 2;           // logical halo (rows and cols)
    static constexpr int HX = round_up(H + 2, VW);  // staged column halo (>= H + 2: k >= 1)
    static constexpr int R = TY + 2 * H;
    static constexpr int C = TX + 2 * HX;
    static constexpr int CK = C / 2;
    static constexpr int A = R * CK + 16;  // one colour array (+16 entries: bank offset)
    static constexpr size_t smem = 4ull * A * sizeof(T);
};

// TMA staging of an interior k_down tile (FP32): one thread issues the tiled
// 2D copies of the b and x tiles (rows ty0 - H .., columns tx0 - HX .., the
// innermost coordinate a multiple of 4 floats) straight into the tile's
// colour-split regions, which a raw tile fits; every thread then reads its
// share of the raw rows into registers and, after a barrier, scatters them
// into the red and black arrays in place, as the vector-load path does from
// global memory.  The mbarrier sits just past the four arrays (the launch
// adds 16 bytes).  Tiles whose halo wraps around the periodic grid (a tiled
// copy does not wrap) and unaligned buffers return false and take the vector
// loads.  The wait is bounded; when it runs out, *err is set.
template <int NU, int TY_>
__device__ __forceinline__ bool tma_stage_tile(float *X, float *B, const void *tmx, const void *tmb, int n,
                                               int ty0, int tx0, bool zero, int *err) {
    using Cfg = DownCfg<float, NU, TY_>;
    constexpr int R = Cfg::R, C = Cfg::C, A = Cfg::A, H = Cfg::H, HX = Cfg::HX;
    static_assert(R * C <= 2 * A && (C * 4) % 16 == 0 && C <= 256 && R <= 256, "raw TMA tile");
    const bool interior = ty0 >= H && ty0 + TY_ + H <= n && tx0 >= HX && tx0 + Cfg::TX + HX <= n;
    const bool aligned = ((smem_u32(X) | smem_u32(B)) & 127u) == 0;
    if (!interior || !aligned || !tmb || (!zero && !tmx)) return false;
    uint64_t *bar = reinterpret_cast<uint64_t *>(X + 4 * A);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        mbar_expect_tx(bar, (zero ? 1u : 2u) * (uint32_t)(R * C * 4));
        tma_load_2d(B, tmb, bar, tx0 - HX, ty0 - H);
        if (!zero) tma_load_2d(X, tmx, bar, tx0 - HX, ty0 - H);
    }
    __syncthreads();
    if (!mbar_wait(bar, 0)) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        mbar_wait(bar, 0);  // once more, so no copy is left writing this block's tile
    }
    constexpr int CV = C / 4, ITEMS = R * CV, PER = (ITEMS + kThreads - 1) / kThreads;
    float4 vb[PER], vx[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = threadIdx.x + i * kThreads;
        if (idx < ITEMS) {
            const int rr = idx / CV, cv = idx - rr * CV;
            vb[i] = *reinterpret_cast<const float4 *>(B + rr * C + cv * 4);
            if (!zero) vx[i] = *reinterpret_cast<const float4 *>(X + rr * C + cv * 4);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = threadIdx.x + i * kThreads;
        if (idx < ITEMS) {
            const int rr = idx / CV, cv = idx - rr * CV;
            scatter_vec(B, B + A, rr, cv * 4, C / 2, vb[i]);
            if (!zero) scatter_vec(X, X + A, rr, cv * 4, C / 2, vx[i]);
        }
    }
    if (zero)
        for (int i = threadIdx.x; i < 2 * A; i += blockDim.x) X[i] = 0.f;
    return true;
}

template <typename T, int NU, int TY_, bool TMA = false, int NT = kThreads>
__device__ __forceinline__ void down_tile(const T *__restrict__ x, T *__restrict__ xout,
                                          const T *__restrict__ b, int n, T *__restrict__ bc,
                                          int ty0, int tx0, bool zero, const void *tmx = nullptr,
                                          const void *tmb = nullptr, int *err = nullptr) {
    using Cfg = DownCfg<T, NU, TY_>;
    constexpr int TY = Cfg::TY, TX = Cfg::TX, H = Cfg::H, HX = Cfg::HX, R = Cfg::R, C = Cfg::C,
                  CK = Cfg::CK, A = Cfg::A;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *X = reinterpret_cast<T *>(smem_raw);  // red at X, black at X + A
    T *B = X + 2 * A;                           // red at B, black at B + A

    bool staged = false;
    if constexpr (TMA) staged = tma_stage_tile<NU, TY_>(X, B, tmx, tmb, n, ty0, tx0, zero, err);
    if (!staged) {
        SplitLoad<T, R, C, NT> lb, lx;
        lb.issue(b, n, ty0 - H, tx0 - HX);
        if (!zero) lx.issue(x, n, ty0 - H, tx0 - HX);
        lb.scatter(B, B + A);
        if (zero) {
            for (int i = threadIdx.x; i < 2 * A; i += blockDim.x) X[i] = T(0);
        } else {
            lx.scatter(X, X + A);
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int s = 0; s < NU; ++s) {
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
            const int j = 2 * s + q + 1;  // valid region shrinks by one per half-sweep
            half_sweep<CK, A, (TY >= 32), NT>(X, B, j, R - j, q);
            __syncthreads();
        }
    }
    // scaled residual s = b - (4x - sum) over staged rows [H-1, H+TY+1), written over b
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
        const T *Xq = X + q * A;
        T *Bq = B + q * A;
        colour_strips<CK, (TY >= 32), NT>(X + (q ^ 1) * A, H - 1, H + TY + 1, q, [&](int p, T N, T S, T W, T E) {
            Bq[p] = Bq[p] - (T(4) * Xq[p] - (((N + S) + W) + E));
        });
    }
    __syncthreads();
    // full weighting at coarse (I, J) <-> fine (2I, 2J) (a red point);
    // times 4 because h_c^2 = 4 h^2
    const int nc = n >> 1;
    constexpr int CW = TX / 2;
    const T *Sr = B, *Sb = B + A;
    for (int idx = threadIdx.x; idx < (TY / 2) * CW; idx += blockDim.x) {
        const int I = idx / CW, J = idx - I * CW;
        const int r = H + 2 * I, k = (HX >> 1) + J;
        const int p = r * CK + k;
        const T edge = ((Sb[p - CK] + Sb[p + CK]) + Sb[p - 1]) + Sb[p];
        const T corner = ((Sr[p - CK - 1] + Sr[p - CK]) + Sr[p + CK - 1]) + Sr[p + CK];
        bc[(size_t)(ty0 / 2 + I) * nc + tx0 / 2 + J] = (T(4) * Sr[p] + T(2) * edge + corner) * T(0.25);
    }
    store_split<T, TY, TX, C>(xout, X, X + A, n, ty0, tx0, H, HX);
}

template <typename T, int NU, bool ZERO, int TY>
__global__ void __launch_bounds__(kThreads) k_down(const T *__restrict__ x, T *__restrict__ xout,
                                                   const T *__restrict__ b, int n,
                                                   T *__restrict__ bc) {
    pdl_enter();
    down_tile<T, NU, TY>(x, xout, b, n, bc, blockIdx.y * TY, blockIdx.x * kTX, ZERO);
}

// k_down on 64-row FP32 tiles with the interior tiles staged by TMA (tmx, tmb:
// 2D maps of x and b with boxes of the staged tile, C x R floats).
template <int NU, bool ZERO>
__global__ void __launch_bounds__(kThreads) k_down_tma(const __grid_constant__ CUtensorMap tmx,
                                                       const __grid_constant__ CUtensorMap tmb,
                                                       const float *__restrict__ x, float *__restrict__ xout,
                                                       const float *__restrict__ b, int n, float *__restrict__ bc,
                                                       int *err) {
    pdl_enter();
    down_tile<float, NU, 64, true>(x, xout, b, n, bc, blockIdx.y * 64, blockIdx.x * kTX, ZERO, &tmx, &tmb, err);
}

// Block of a batched tile launch: locate its grid (the last table entry whose
// first tile is <= blockIdx.x) and the tile's origin in that grid.
__device__ __forceinline__ int find_grid(const TileGrid *__restrict__ g, int ngrid) {
    int lo = 0, hi = ngrid - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g[mid].tile0 <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T, int NU, int TY>
__global__ void __launch_bounds__(kThreads) k_down_batched(const TileGrid *__restrict__ tab, int ngrid,
                                                           const int *__restrict__ active) {
    pdl_enter();
    const TileGrid t = tab[find_grid(tab, ngrid)];
    if (active && !active[t.rhs]) return;
    const int lt = (int)blockIdx.x - t.tile0, tpr = t.n / kTX;
    down_tile<T, NU, TY>((const T *)t.x, (T *)t.xout, (const T *)t.b, t.n, (T *)t.aux, (lt / tpr) * TY,
                         (lt % tpr) * kTX, t.zero != 0);
}

// ---------------------------------------------------------------------------
// k_up: x += P_cubic ec (+ extra), then NU sweeps, on one tile.
// ---------------------------------------------------------------------------
template <typename T, int NU, int TY_, int NJ_>
struct UpCfg {
    static constexpr int TY = TY_, TX = kTX, NJ = NJ_;
    static constexpr int VW = Prec<T>::VW;
    static constexpr int L = Prec<T>::L;
    static constexpr int H = 2 * NU;
    static constexpr int HX = round_up(H + 2, VW);
    static constexpr int R = TY + 2 * H;
    static constexpr int C = TX + 2 * HX;
    static constexpr int CK = C / 2;
    static constexpr int A = R * CK + 16;
    // coarse positions refined: J in [-H/2, TX/2 + H/2) (JW of them), I likewise (IW)
    static constexpr int JW = TX / 2 + H;
    static constexpr int IW = TY / 2 + H;
    // coarse tile: rows [I0 - CHY, I0 - CHY + CR), cols [J0 - CHX, J0 - CHX + CC)
    static constexpr int CHY = H / 2 + L - 1;
    static constexpr int CR = IW + 2 * L - 1;
    static constexpr int CHX = round_up(H / 2 + L - 1, VW);
    static constexpr int CXE = round_up(H / 2 + L, VW);
    static constexpr int CC = TX / 2 + CHX + CXE;
    static constexpr int FW = TX + 2 * H;  // fine columns refined, v in [-H, TX + H)
    static constexpr int CRP = (CR + 1) / 2;            // row pairs of the packed coarse tile
    // row pitch of the packed coarse tile in float2: 2 CCP = 8 (mod 32) 4-byte words,
    // so the row pass's remainder groups of rows fall into disjoint banks
    static constexpr int CCP = (CC + 15) / 16 * 16 + 4;
    static constexpr int U = cmax(2 * A, 2 * CRP * CCP);  // coarse tile, then b (after the row pass)
    static constexpr size_t smem = (2ull * A + U + (size_t)CR * FW) * sizeof(T);
    // with pre-refined rows (no coarse tile): x, b, then the refined rows
    static constexpr size_t smem_xr = (4ull * A + (size_t)CR * FW) * sizeof(T);
    static_assert(JW % NJ == 0 && IW % NJ == 0, "runs must tile the refined range");
};

// xr (optional, one-run tiles only): the coarse error already refined along x
// by k_refine_rows, (n/2) x n; the tile then loads its refined rows instead of
// running the row pass (the same values: the pass's arithmetic per midpoint).
template <typename T, int NU, int TY_, int NJ_, int NT = kThreads, bool COH = false>
__device__ __forceinline__ void up_tile(const T *__restrict__ x, T *__restrict__ xout,
                                        const T *__restrict__ b, const T *__restrict__ ec,
                                        const T *__restrict__ extra, int n, const FirTaps &taps, int ty0,
                                        int tx0, const T *__restrict__ xr = nullptr) {
    using Cfg = UpCfg<T, NU, TY_, NJ_>;
    constexpr int TY = Cfg::TY, TX = Cfg::TX, NJ = Cfg::NJ, H = Cfg::H, HX = Cfg::HX, R = Cfg::R,
                  C = Cfg::C, CK = Cfg::CK, A = Cfg::A, L = Cfg::L, JW = Cfg::JW, IW = Cfg::IW,
                  CHY = Cfg::CHY, CR = Cfg::CR, CHX = Cfg::CHX, CC = Cfg::CC, FW = Cfg::FW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *X = reinterpret_cast<T *>(smem_raw);  // red at X, black at X + A
    T *cs = X + 2 * A;                          // coarse tile [CR][CC] (row pass only)
    T *B = X + 2 * A;                           // b, loaded over cs after the row pass
    constexpr bool kXR = NJ == 1 && std::is_same<T, double>::value;  // pre-refined rows accepted
    const bool use_xr = kXR && xr != nullptr;
    T *rs = X + 2 * A + (use_xr ? 2 * A : Cfg::U);  // x-refined coarse rows [CR][FW]
    const int nc = n >> 1;

    if constexpr (std::is_same<T, float>::value && NJ == 2) {
        // Packed variant: both spline passes on float2 pairs with f32x2
        // instructions.  Row pass: the coarse tile is stored as row pairs,
        // cs2[rp][col] = (row 2rp, row 2rp + 1), so one 64-bit load feeds two
        // rows' midpoints; column pass: two adjacent fine columns of rs.
        constexpr int CRP = Cfg::CRP;
        float2 *cs2 = reinterpret_cast<float2 *>(cs);
        constexpr int CV = CC / 4, CITEMS = CRP * CV, CPER = (CITEMS + NT - 1) / NT;
        SplitLoad<T, R, C, NT, COH> lx;
        lx.issue(x, n, ty0 - H, tx0 - HX);
        float4 c0v[CPER], c1v[CPER];
#pragma unroll
        for (int i = 0; i < CPER; ++i) {
            const int idx = threadIdx.x + i * NT;
            if (idx < CITEMS) {
                const int rp = idx / CV, cv = idx - rp * CV;
                const int gr0 = (ty0 / 2 - CHY + 2 * rp) & (nc - 1), gr1 = (gr0 + 1) & (nc - 1);
                const int gc = (tx0 / 2 - CHX + 4 * cv) & (nc - 1);
                const float4 *s0 = reinterpret_cast<const float4 *>(ec + (size_t)gr0 * nc + gc);
                const float4 *s1 = reinterpret_cast<const float4 *>(ec + (size_t)gr1 * nc + gc);
                c0v[i] = COH ? __ldcg(s0) : __ldg(s0);
                c1v[i] = COH ? __ldcg(s1) : __ldg(s1);
            }
        }
        lx.scatter(X, X + A);
#pragma unroll
        for (int i = 0; i < CPER; ++i) {
            const int idx = threadIdx.x + i * NT;
            if (idx < CITEMS) {
                const int rp = idx / CV, cv = idx - rp * CV;
                float4 *dst = reinterpret_cast<float4 *>(cs2 + rp * Cfg::CCP + 4 * cv);
                dst[0] = make_float4(c0v[i].x, c1v[i].x, c0v[i].y, c1v[i].y);
                dst[1] = make_float4(c0v[i].z, c1v[i].z, c0v[i].w, c1v[i].w);
            }
        }
        float2 tp[L];
#pragma unroll
        for (int k = 1; k <= L; ++k) tp[k - 1] = make_float2(Prec<float>::tap(taps, k), Prec<float>::tap(taps, k));
        __syncthreads();
        SplitLoad<T, R, C, NT> lb;  // b arrives while the row pass runs
        if (NU > 0) lb.issue(b, n, ty0 - H, tx0 - HX);
        // Both spline passes map one warp instruction to one row of items (32
        // consecutive, conflict-free) and take each row's remaining items in
        // groups of rows whose runs fall into disjoint banks (strip_rem_rows).
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        constexpr int NWARP = NT / 32;
        auto row_item = [&](int rp, int jr) {
            const int J0 = -H / 2 + jr;
            const float2 *w = cs2 + rp * Cfg::CCP + CHX + J0;  // w[m] = rows (2rp, 2rp+1) at coarse col J0 + m
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = L; k >= 1; --k) acc = f2_fma(tp[k - 1], f2_add(w[k], w[1 - k]), acc);
            const float2 node = w[0];
            const int col = 2 * J0 + H;
            *reinterpret_cast<float2 *>(rs + (2 * rp) * FW + col) = make_float2(node.x, acc.x);
            if (2 * rp + 1 < CR) *reinterpret_cast<float2 *>(rs + (2 * rp + 1) * FW + col) = make_float2(node.y, acc.y);
        };
        {
            constexpr int JM = JW < 32 ? JW : 32, JR = JW - JM;
            if (lane < JM)
                for (int rp = warp; rp < CRP; rp += NWARP) row_item(rp, lane);
            if constexpr (JR > 0) {
                constexpr int RG = strip_rem_rows(Cfg::CCP, JR, 2);
                const int dr = lane / JR, jr = JM + (lane - dr * JR);
                if (dr < RG)
                    for (int rp = warp * RG + dr; rp < CRP; rp += NWARP * RG) row_item(rp, jr);
            }
        }
        __syncthreads();
        if (NU > 0) lb.scatter(B, B + A);
        constexpr int CP = FW / 2;
        // Column pass: an item refines two adjacent fine columns (2cp, 2cp + 1)
        // at the midpoints of RPI consecutive coarse rows I0 .. I0 + RPI - 1.
        // Each midpoint sums its taps k = L .. 1 in the order of the
        // one-midpoint form, w[k + i] + w[1 - k + i] for row I0 + i; the rows
        // share a rolling window (one step's w[k + i] is the next step's
        // w[k - 1 + (i + 1)], its w[2 - k + i] the next step's w[1 - (k - 1) + (i - 1)]),
        // so an item loads 2L + 2 RPI - 2 rows instead of 2L RPI.
        // four rows per item only where two-row items would need a second pass
        // of the block's threads (small tiles: the longer chain would cost more)
        constexpr int RPI = (IW % 4 == 0 && (IW / 2) * CP > NT) ? 4 : 2;
        static_assert(IW % RPI == 0, "column-pass items take RPI coarse rows");
        auto col_item = [&](int ip, int cp) {
            const int I0 = -H / 2 + RPI * ip;
            const float *w = rs + (CHY + I0) * FW + 2 * cp;  // w[m * FW]: refined row I0 + m
            auto ld = [&](int m) { return *reinterpret_cast<const float2 *>(w + m * FW); };
            float2 hi[RPI], lo[RPI], acc[RPI];
#pragma unroll
            for (int i = 0; i < RPI; ++i) {
                hi[i] = ld(L + i);
                lo[i] = ld(1 - L + i);
                acc[i] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int k = L; k >= 1; --k) {
#pragma unroll
                for (int i = 0; i < RPI; ++i) acc[i] = f2_fma(tp[k - 1], f2_add(hi[i], lo[i]), acc[i]);
                if (k > 1) {
#pragma unroll
                    for (int i = RPI - 1; i >= 1; --i) hi[i] = hi[i - 1];
                    hi[0] = ld(k - 1);
#pragma unroll
                    for (int i = 0; i + 1 < RPI; ++i) lo[i] = lo[i + 1];
                    lo[RPI - 1] = ld(RPI + 1 - k);
                }
            }
            // after the last step lo[i] = w[i]: the rows' nodes
#pragma unroll
            for (int i = 0; i < RPI; ++i) {
                const int u = 2 * (I0 + i), r = u + H;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int v = 2 * cp + h - H;
                    const int c = v + HX;
                    T ve = h ? lo[i].y : lo[i].x, vo = h ? acc[i].y : acc[i].x;
                    if (extra) {
                        const size_t gc = (size_t)((tx0 + v) & (n - 1));
                        ve += extra[(size_t)((ty0 + u) & (n - 1)) * n + gc];
                        vo += extra[(size_t)((ty0 + u + 1) & (n - 1)) * n + gc];
                    }
                    const int q = (r + c) & 1;
                    X[q * A + r * CK + (c >> 1)] += ve;
                    X[(q ^ 1) * A + (r + 1) * CK + (c >> 1)] += vo;
                }
            }
        };
        {
            constexpr int IP = IW / RPI;
            constexpr int CM = CP < 32 ? CP : 32, CRM = CP - CM;
            if (lane < CM)
                for (int ip = warp; ip < IP; ip += NWARP) col_item(ip, lane);
            if constexpr (CRM > 0) {
                // consecutive items are RPI refined rows (RPI FW / 2 float2) apart
                constexpr int RG = strip_rem_rows(RPI * FW / 2, CRM, 2);
                const int dr = lane / CRM, cp = CM + (lane - dr * CRM);
                if (dr < RG)
                    for (int ip = warp * RG + dr; ip < IP; ip += NWARP * RG) col_item(ip, cp);
            }
        }
        __syncthreads();
#pragma unroll 1
        for (int s = 0; s < NU; ++s) {
#pragma unroll 1
            for (int q = 0; q < 2; ++q) {
                const int j = 2 * s + q + 1;
                half_sweep<CK, A, (TY >= 32), NT>(X, B, j, R - j, q);
                __syncthreads();
            }
        }
        store_split<T, TY, TX, C>(xout, X, X + A, n, ty0, tx0, H, HX);
        return;
    }
    load_split<T, R, C>(X, X + A, x, n, ty0 - H, tx0 - HX);
    if constexpr (kXR) {
        if (use_xr) {
            // rs[cr][c] = xr[coarse row ty0 / 2 - CHY + cr][fine column tx0 - H + c]
            using V = typename Prec<T>::vec;
            constexpr int VW = Prec<T>::VW, FV = FW / VW;
            static_assert(FW % VW == 0 && H % VW == 0, "refined rows load as whole vectors");
            for (int idx = threadIdx.x; idx < CR * FV; idx += blockDim.x) {
                const int cr = idx / FV, cv = idx - cr * FV;
                const int gr = (ty0 / 2 - CHY + cr) & (nc - 1), gc = (tx0 - H + cv * VW) & (n - 1);
                *reinterpret_cast<V *>(rs + cr * FW + cv * VW) =
                    __ldg(reinterpret_cast<const V *>(xr + (size_t)gr * n + gc));
            }
        }
    }
    if (!use_xr) load_tile<T, CR, CC, CC>(cs, ec, nc, ty0 / 2 - CHY, tx0 / 2 - CHX);
    __syncthreads();

    // refine along x: coarse row cr, midpoints of J0..J0+NJ-1 (and the nodes)
    constexpr int NRUN = JW / NJ;
    for (int item = threadIdx.x; item < (use_xr ? 0 : CR * NRUN); item += blockDim.x) {
        const int cr = item / NRUN, jr = item - cr * NRUN;
        const int J0 = -H / 2 + jr * NJ;
        const T *w = cs + cr * CC + CHX + J0;  // w[m] = e_c[J0 + m]
        T *out = rs + cr * FW + 2 * J0 + H;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            T acc = T(0);
#pragma unroll
            for (int k = L; k >= 1; --k) acc += Prec<T>::tap(taps, k) * (w[j + k] + w[j + 1 - k]);
            out[2 * j] = w[j];
            out[2 * j + 1] = acc;
        }
    }
    __syncthreads();
    if (NU > 0) load_split<T, R, C>(B, B + A, b, n, ty0 - H, tx0 - HX);
    // refine along y and add: fine column v, rows 2I and 2I+1 for I in the run
    constexpr int NIRUN = IW / NJ;
    for (int item = threadIdx.x; item < FW * NIRUN; item += blockDim.x) {
        const int ir = item / FW, vv = item - ir * FW;
        const int I0 = -H / 2 + ir * NJ;
        const T *w = rs + (CHY + I0) * FW + vv;  // w[m * FW] = refined row I0 + m
        const int v = vv - H;
        const int c = v + HX;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            T acc = T(0);
#pragma unroll
            for (int k = L; k >= 1; --k)
                acc += Prec<T>::tap(taps, k) * (w[(j + k) * FW] + w[(j + 1 - k) * FW]);
            const int u = 2 * (I0 + j);
            T ve = w[j * FW], vo = acc;
            if (extra) {
                const size_t gc = (size_t)((tx0 + v) & (n - 1));
                ve += extra[(size_t)((ty0 + u) & (n - 1)) * n + gc];
                vo += extra[(size_t)((ty0 + u + 1) & (n - 1)) * n + gc];
            }
            const int r = u + H;
            const int q = (r + c) & 1;  // colour of (r, c); (r + 1, c) has the other
            X[q * A + r * CK + (c >> 1)] += ve;
            X[(q ^ 1) * A + (r + 1) * CK + (c >> 1)] += vo;
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int s = 0; s < NU; ++s) {
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
            const int j = 2 * s + q + 1;
            half_sweep<CK, A, (TY >= 32), NT>(X, B, j, R - j, q);
            __syncthreads();
        }
    }
    store_split<T, TY, TX, C>(xout, X, X + A, n, ty0, tx0, H, HX);
}

// extra_flag (may be null): the additive term is used only where *extra_flag != 0.
template <typename T, int NU, int TY, int NJ>
__global__ void __launch_bounds__(kThreads) k_up(const T *__restrict__ x, T *__restrict__ xout,
                                                 const T *__restrict__ b, const T *__restrict__ ec,
                                                 const T *__restrict__ extra, const int *__restrict__ extra_flag,
                                                 int n, FirTaps taps, const T *__restrict__ xr) {
    pdl_enter();
    const T *ex = (extra && (!extra_flag || *extra_flag)) ? extra : nullptr;
    up_tile<T, NU, TY, NJ>(x, xout, b, ec, ex, n, taps, blockIdx.y * TY, blockIdx.x * kTX, xr);
}

// The x pass of the cubic prolongation on its own (FP64 V-cycles): xr[I][2J]
// = ec[I][J] and xr[I][2J + 1] = the midpoint sum of k_up's row pass, for
// every coarse row I once (inside k_up a tile refines its rows plus the
// 2L - 1 halo rows its column pass reads, 3.75 times its own rows with the
// FP64 filter's L = 28 taps on 32-row tiles).  Blocks of kRefineJ threads
// take kRefineJ consecutive coarse columns of one row, staged with their
// taps' halo in shared memory.
constexpr int kRefineJ = 64;
template <typename T>
__global__ void __launch_bounds__(kRefineJ) k_refine_rows(const T *__restrict__ ec, T *__restrict__ xr, int n,
                                                          FirTaps taps) {
    pdl_enter();
    constexpr int L = Prec<T>::L, W = kRefineJ + 2 * L - 1;
    __shared__ T row[W];
    const int nc = n >> 1, I = blockIdx.y, J0 = blockIdx.x * kRefineJ;
    const T *er = ec + (size_t)I * nc;
    for (int i = threadIdx.x; i < W; i += kRefineJ) row[i] = er[(J0 - L + 1 + i) & (nc - 1)];
    __syncthreads();
    const int j = threadIdx.x;
    const T *w = row + j + L - 1;  // w[m] = ec[I][J0 + j + m]
    T acc = T(0);
#pragma unroll
    for (int k = L; k >= 1; --k) acc += Prec<T>::tap(taps, k) * (w[k] + w[1 - k]);
    T *out = xr + (size_t)I * n + 2 * (J0 + j);
    out[0] = w[0];
    out[1] = acc;
}

template <typename T, int NU, int TY, int NJ>
__global__ void __launch_bounds__(kThreads) k_up_batched(const TileGrid *__restrict__ tab, int ngrid,
                                                         const int *__restrict__ active, FirTaps taps) {
    pdl_enter();
    const TileGrid t = tab[find_grid(tab, ngrid)];
    if (active && !active[t.rhs]) return;
    const int lt = (int)blockIdx.x - t.tile0, tpr = t.n / kTX;
    const T *ex = (t.extra && !(t.extra_off && *t.extra_off)) ? (const T *)t.extra : nullptr;
    up_tile<T, NU, TY, NJ>((const T *)t.x, (T *)t.xout, (const T *)t.b, (const T *)t.aux, ex, t.n, taps,
                           (lt / tpr) * TY, (lt % tpr) * kTX);
}

// ---------------------------------------------------------------------------
// k_bottom: a whole V-cycle on grids <= 64 x 64, one block, shared memory.
// ---------------------------------------------------------------------------
constexpr int kBottomThreads = 1024;

// Runs.  On a level of m x m points (4 <= m <= 64) a thread holds a run: 4
// consecutive points of one row, m / 4 runs per row.  For m >= 16 the
// m^2 / 4 runs fill w = m^2 / 128 whole warps, warp g taking rows
// g, g + w, g + 2w, ...: w is even, so the rows of a warp share their parity
// and a half-sweep's colour choice is warp-uniform.  Smaller levels use
// lanes of warp 0.  The lanes of one row are adjacent, so the west and east
// neighbours of a run's end points come from the neighbouring lanes.
// log2 of a power of two (shifts instead of integer division by sizes
// known only at run time)
__device__ __forceinline__ int ilog2(int v) { return __ffs(v) - 1; }

struct RunMap {
    int row, c0;         // the run's row and first column
    int lane_w, lane_e;  // lanes holding the runs to the west and east (periodic)
    bool warp_on, on;    // the warp takes part; this lane holds a run
};

__device__ __forceinline__ RunMap run_map(int m) {
    const int tpr = m >> 2, runs = (m * m) >> 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    RunMap r;
    if (runs >= 64) {
        const int w = runs >> 5;
        r.warp_on = warp < w;
        r.on = r.warp_on;
        r.row = warp + (lane >> ilog2(tpr)) * w;
    } else {
        r.warp_on = warp == 0;
        r.on = warp == 0 && lane < runs;
        r.row = lane >> ilog2(tpr);
    }
    r.c0 = (lane & (tpr - 1)) << 2;
    const int base = lane & ~(tpr - 1);
    r.lane_w = base | ((lane - 1) & (tpr - 1));
    r.lane_e = base | ((lane + 1) & (tpr - 1));
    return r;
}

template <typename T> struct RunIO;
template <> struct RunIO<float> {
    static __device__ __forceinline__ void ld(const float *p, float (&v)[4]) {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        v[0] = a.x;
        v[1] = a.y;
        v[2] = a.z;
        v[3] = a.w;
    }
    static __device__ __forceinline__ void st(float *p, const float (&v)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct RunIO<double> {
    static __device__ __forceinline__ void ld(const double *p, double (&v)[4]) {
        const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = a.x;
        v[1] = a.y;
        v[2] = b.x;
        v[3] = b.y;
    }
    static __device__ __forceinline__ void st(double *p, const double (&v)[4]) {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
    }
};

// The other-colour neighbours of a run: north and south runs from shared
// memory, the points west and east of its ends from the neighbouring lanes.
// Called by whole warps (warp_on); lanes without a run get zeros.
template <typename T>
__device__ __forceinline__ void run_neighbours(const T *X, const T (&xr)[4], const RunMap &r, int m, T (&nr)[4],
                                               T (&sr)[4], T &wn, T &en) {
    if (r.on) {
        RunIO<T>::ld(X + ((r.row - 1) & (m - 1)) * m + r.c0, nr);
        RunIO<T>::ld(X + ((r.row + 1) & (m - 1)) * m + r.c0, sr);
    } else {
#pragma unroll
        for (int a = 0; a < 4; ++a) nr[a] = sr[a] = T(0);
    }
    wn = __shfl_sync(0xffffffffu, xr[3], r.lane_w);
    en = __shfl_sync(0xffffffffu, xr[0], r.lane_e);
}

// One Gauss-Seidel half-sweep of colour q over the level's runs,
// x <- (b + (((N + S) + W) + E)) / 4; the run (xr) stays in registers and is
// stored for the neighbours' next half-sweep.
template <typename T>
__device__ __forceinline__ void run_half_sweep(T *X, const T (&br)[4], T (&xr)[4], const RunMap &r, int m, int q) {
    if (r.warp_on) {
        T nr[4], sr[4], wn, en;
        run_neighbours(X, xr, r, m, nr, sr, wn, en);
        if (((r.row + q) & 1) == 0) {  // colour q at run positions 0 and 2
            xr[0] = (br[0] + (((nr[0] + sr[0]) + wn) + xr[1])) * T(0.25);
            xr[2] = (br[2] + (((nr[2] + sr[2]) + xr[1]) + xr[3])) * T(0.25);
        } else {  // at positions 1 and 3
            xr[1] = (br[1] + (((nr[1] + sr[1]) + xr[0]) + xr[2])) * T(0.25);
            xr[3] = (br[3] + (((nr[3] + sr[3]) + xr[2]) + en)) * T(0.25);
        }
        if (r.on) RunIO<T>::st(X + r.row * m + r.c0, xr);
    }
    __syncthreads();
}

// Midpoint J + 1/2 of a periodic coarse row E (mc points) by the cubic
// spline's FIR taps.
template <typename T>
__device__ __forceinline__ T spline_mid_row(const T *E, int J, int mc, const FirTaps &taps) {
    constexpr int L = Prec<T>::L;
    T acc = T(0);
#pragma unroll
    for (int k = L; k >= 1; --k)
        acc += Prec<T>::tap(taps, k) * (E[(J + k) & (mc - 1)] + E[(J + 1 - k) & (mc - 1)]);
    return acc;
}

// FP32 prolongation and correction of one bottom level: x (m x m) +=
// spline(E), E the coarse error (mc = m / 2 a side), S the m x mc scratch of
// row-refined coarse rows.  Each midpoint sums its taps in the same order as
// spline_mid_row (k = L down to 1), but a thread computes several midpoints
// from one window of loaded values: along x, 4 midpoints of a coarse row from
// 9 aligned 16-byte loads; along y, 4 odd fine rows of one column from
// 2L + 3 loads.  Ends with the level's x updated and a barrier.
__device__ __forceinline__ void bottom_prolong_f32(float *X, const float *E, float *S, int m,
                                                   const FirTaps &taps) {
    constexpr int L = Prec<float>::L;
    static_assert(L <= 16, "the x window holds 16 + 4 + 16 coarse values");
    const int mc = m >> 1, tid = threadIdx.x, nt = blockDim.x;
    // along x: item (I, J0), J0 a multiple of 4: coarse row I, midpoints
    // J0 + 1/2 .. J0 + 7/2; window w[p] = E[I][J0 - 16 + p], p < 36
    for (int t = tid; t < mc * (mc >> 2); t += nt) {
        const int I = t >> ilog2(mc >> 2), J0 = (t - I * (mc >> 2)) << 2;
        const float *Er = E + I * mc;
        float w[36];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float4 v = *reinterpret_cast<const float4 *>(Er + ((J0 - 16 + 4 * q) & (mc - 1)));
            w[4 * q] = v.x;
            w[4 * q + 1] = v.y;
            w[4 * q + 2] = v.z;
            w[4 * q + 3] = v.w;
        }
        float o[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float acc = 0.f;
#pragma unroll
            for (int k = L; k >= 1; --k) acc += Prec<float>::tap(taps, k) * (w[16 + i + k] + w[17 + i - k]);
            o[2 * i] = w[16 + i];
            o[2 * i + 1] = acc;
        }
        float *Sr = S + I * m + 2 * J0;
        *reinterpret_cast<float4 *>(Sr) = make_float4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<float4 *>(Sr + 4) = make_float4(o[4], o[5], o[6], o[7]);
    }
    __syncthreads();
    // along y: odd fine rows 2I + 1 (I = I0 .. I0 + 3) of column c from the
    // window v[q] = S[I0 + 1 - L + q][c]; even fine rows 2I take S row I
    const int nodd = m * (mc >> 2), neven = (m * m) >> 3;
    for (int t = tid; t < nodd + neven; t += nt) {
        if (t < nodd) {
            const int c = t & (m - 1), I0 = (t >> ilog2(m)) << 2;
            float v[2 * L + 3];
#pragma unroll
            for (int q = 0; q < 2 * L + 3; ++q) v[q] = S[((I0 + 1 - L + q) & (mc - 1)) * m + c];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float acc = 0.f;
#pragma unroll
                for (int k = L; k >= 1; --k) acc += Prec<float>::tap(taps, k) * (v[i + k + L - 1] + v[i - k + L]);
                float *xp = X + (2 * (I0 + i) + 1) * m + c;
                *xp = *xp + acc;
            }
        } else {
            const int e = t - nodd, row = (e >> ilog2(m >> 2)) << 1, c0 = (e - (row >> 1) * (m >> 2)) << 2;
            float xv[4], sv[4];
            RunIO<float>::ld(X + row * m + c0, xv);
            RunIO<float>::ld(S + (row >> 1) * m + c0, sv);
#pragma unroll
            for (int a = 0; a < 4; ++a) xv[a] += sv[a];
            RunIO<float>::st(X + row * m + c0, xv);
        }
    }
    __syncthreads();
}

// Shared-memory elements of a bottom solve of an n x n grid with nlev levels:
// x and b per level, n * n / 2 for the row-refined coarse grid of the
// prolongation and n * n for the residual that full weighting reads.
__host__ __device__ constexpr size_t bottom_elems(int n, int nlev) {
    size_t e = (size_t)n * n / 2 + (size_t)n * n;
    for (int l = 0; l < nlev; ++l) e += 2ull * (n >> l) * (n >> l);
    return e;
}

// A coarsest grid of at most this many points keeps its pseudo-inverse
// (Nc^2 entries) in shared memory, staged together with the finest level.
constexpr int kBottomAinvShared = 64;

__host__ __device__ constexpr size_t bottom_smem_elems(int n, int nlev) {
    const size_t nc = (size_t)(n >> (nlev - 1)) * (n >> (nlev - 1));
    return bottom_elems(n, nlev) + (nc <= (size_t)kBottomAinvShared ? nc * nc : 0);
}

// The largest bottom configuration: kBottomMax^2 over any level count that
// ends at a coarsest grid of at least 4^2.
constexpr size_t bottom_smem_max() {
    size_t best = 0;
    for (int l = 1; (kBottomMax >> (l - 1)) >= 4; ++l)
        best = bottom_smem_elems(kBottomMax, l) > best ? bottom_smem_elems(kBottomMax, l) : best;
    return best;
}


template <typename T>
__device__ __forceinline__ void bottom_body(T *__restrict__ x, const T *__restrict__ b, int n, int nlev,
                                            int nu1, int nu2, int zero_init, const T *__restrict__ ainv,
                                            const FirTaps &taps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *base = reinterpret_cast<T *>(smem_raw);
    // level l (m = n >> l points a side): x at X(l), b at X(l) + m^2; the levels
    // above it take 2 (n^2 + (n/2)^2 + ... + (2m)^2) = 8 (n^2 - m^2) / 3 elements
    auto X = [&](int l) { const int m = n >> l; return base + 8 * (n * n - m * m) / 3; };
    auto B = [&](int l) { const int m = n >> l; return base + 8 * (n * n - m * m) / 3 + m * m; };
    const int mlast = n >> (nlev - 1), Nc = mlast * mlast;
    T *S = base + 8 * (n * n - mlast * mlast) / 3 + 2 * mlast * mlast;  // n * n / 2: row-refined coarse rows
    T *R = S + n * n / 2;  // n * n: residual of the level being restricted
    T *Ash = R + n * n;    // Nc * Nc: the coarsest grid's pseudo-inverse (small coarsest grids)
    const bool a_sh = Nc <= kBottomAinvShared;
    const int tid = threadIdx.x, nt = blockDim.x;

    // Stage x, b and the pseudo-inverse with 16-byte loads, every load of a
    // thread issued before its stores; element by element when a pointer is
    // unaligned.
    constexpr int VW = Prec<T>::VW;
    using V = typename Prec<T>::vec;
    const bool aligned = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(b) |
                           reinterpret_cast<uintptr_t>(ainv)) & 15) == 0;
    if (aligned) {
        const int nx = (n * n) / VW, na = a_sh ? (Nc * Nc) / VW : 0;
        for (int i = tid; i < max(nx, na); i += nt) {
            V vx{}, vb{}, va{};
            if (i < nx) {
                if (!zero_init) vx = reinterpret_cast<const V *>(x)[i];
                vb = reinterpret_cast<const V *>(b)[i];
            }
            if (i < na) va = reinterpret_cast<const V *>(ainv)[i];
            if (i < nx) {
                reinterpret_cast<V *>(X(0))[i] = vx;
                reinterpret_cast<V *>(B(0))[i] = vb;
            }
            if (i < na) reinterpret_cast<V *>(Ash)[i] = va;
        }
    } else {
        for (int p = tid; p < n * n; p += nt) {
            X(0)[p] = zero_init ? T(0) : x[p];
            B(0)[p] = b[p];
        }
        if (a_sh)
            for (int p = tid; p < Nc * Nc; p += nt) Ash[p] = ainv[p];
    }
    __syncthreads();
    for (int l = 0; l + 1 < nlev; ++l) {
        const int m = n >> l, mc = m >> 1;
        const RunMap r = run_map(m);
        T xr[4] = {}, br[4] = {};
        if (r.on) {
            RunIO<T>::ld(X(l) + r.row * m + r.c0, xr);
            RunIO<T>::ld(B(l) + r.row * m + r.c0, br);
        }
        for (int s = 0; s < nu1; ++s) {
            run_half_sweep(X(l), br, xr, r, m, 0);
            run_half_sweep(X(l), br, xr, r, m, 1);
        }
        // scaled residual b - (4x - (((N + S) + W) + E))
        if (r.warp_on) {
            T nr[4], sr[4], wn, en;
            run_neighbours(X(l), xr, r, m, nr, sr, wn, en);
            const T w[4] = {wn, xr[0], xr[1], xr[2]}, e[4] = {xr[1], xr[2], xr[3], en};
            T rr[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) rr[a] = br[a] - (T(4) * xr[a] - (((nr[a] + sr[a]) + w[a]) + e[a]));
            if (r.on) RunIO<T>::st(R + r.row * m + r.c0, rr);
        }
        __syncthreads();
        // full weighting at coarse (I, J) <-> fine (2I, 2J), times 4 because
        // h_c^2 = 4 h^2; each coarse run reads fine rows 2I - 1 .. 2I + 1,
        // columns 2J0 - 1 .. 2J0 + 7
        const RunMap rc = run_map(mc);
        if (rc.on) {
            const int i = 2 * rc.row, j0 = 2 * rc.c0;
            T v[3][9];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const T *Rw = R + ((i - 1 + k) & (m - 1)) * m;
                T lo[4], hi[4];
                RunIO<T>::ld(Rw + j0, lo);
                RunIO<T>::ld(Rw + j0 + 4, hi);
                v[k][0] = Rw[(j0 - 1) & (m - 1)];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    v[k][1 + a] = lo[a];
                    v[k][5 + a] = hi[a];
                }
            }
            T bc[4];
            const T zero[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int jj = 1 + 2 * a;
                const T edge = ((v[0][jj] + v[2][jj]) + v[1][jj - 1]) + v[1][jj + 1];
                const T corner = ((v[0][jj - 1] + v[0][jj + 1]) + v[2][jj - 1]) + v[2][jj + 1];
                bc[a] = (T(4) * v[1][jj] + T(2) * edge + corner) * T(0.25);
            }
            RunIO<T>::st(B(l + 1) + rc.row * mc + rc.c0, bc);
            RunIO<T>::st(X(l + 1) + rc.row * mc + rc.c0, zero);
        }
        __syncthreads();
    }
    {   // coarsest grid: e = A~^+ b (the pseudo-inverse annihilates the mean).
        // tpo threads per output row take strided partial dot products (coalesced
        // loads, all issued in parallel), then a shuffle tree within the group.
        T *Xc = X(nlev - 1);
        const T *Bc = B(nlev - 1);
        const int tpo = min(32, nt >> ilog2(Nc));  // powers of two: groups never straddle a warp
        const int p = tid >> ilog2(tpo), lane = tid - p * tpo;
        T acc = T(0);
        if (p < Nc) {
            if (a_sh) {  // Nc <= 64 and tpo >= 16: at most 4 terms, from shared memory
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int q = lane + k * tpo;
                    if (q < Nc) acc += Ash[p * Nc + q] * Bc[q];
                }
            } else {
                for (int q = lane; q < Nc; q += tpo) acc += ainv[p * Nc + q] * Bc[q];
            }
        }
        for (int o = tpo >> 1; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, tpo);
        if (p < Nc && lane == 0) Xc[p] = acc;
        __syncthreads();
    }
    constexpr int L = Prec<T>::L;
    for (int l = nlev - 2; l >= 0; --l) {
        const int m = n >> l, mc = m >> 1;
        const T *E = X(l + 1);
        T xr[4] = {}, br[4] = {};
        const RunMap r = run_map(m);
        if constexpr (sizeof(T) == 4) {
            bottom_prolong_f32(X(l), E, S, m, taps);
            if (r.on) {
                RunIO<T>::ld(X(l) + r.row * m + r.c0, xr);
                RunIO<T>::ld(B(l) + r.row * m + r.c0, br);
            }
        } else {
            // refine coarse rows along x: runs of 4 fine columns j0 .. j0 + 3 of
            // coarse row I (coarse values at j0, j0 + 2, midpoints between)
            for (int t = tid; t < (m * m) >> 3; t += nt) {
                const int I = t >> ilog2(m >> 2), j0 = (t - I * (m >> 2)) << 2, J0 = j0 >> 1;
                const T *Er = E + I * mc;
                T o[4];
                o[0] = Er[J0];
                o[1] = spline_mid_row(Er, J0, mc, taps);
                o[2] = Er[J0 + 1];
                o[3] = spline_mid_row(Er, J0 + 1, mc, taps);
                RunIO<T>::st(S + I * m + j0, o);
            }
            __syncthreads();
            // refine along y and add to the level's x, in the level's runs
            if (r.on) {
                T val[4];
                if ((r.row & 1) == 0) {
                    RunIO<T>::ld(S + (r.row >> 1) * m + r.c0, val);
                } else {
                    const int I = r.row >> 1;
#pragma unroll
                    for (int a = 0; a < 4; ++a) val[a] = T(0);
#pragma unroll
                    for (int k = L; k >= 1; --k) {
                        T u[4], w[4];
                        RunIO<T>::ld(S + ((I + k) & (mc - 1)) * m + r.c0, u);
                        RunIO<T>::ld(S + ((I + 1 - k) & (mc - 1)) * m + r.c0, w);
#pragma unroll
                        for (int a = 0; a < 4; ++a) val[a] += Prec<T>::tap(taps, k) * (u[a] + w[a]);
                    }
                }
                RunIO<T>::ld(X(l) + r.row * m + r.c0, xr);
#pragma unroll
                for (int a = 0; a < 4; ++a) xr[a] += val[a];
                RunIO<T>::st(X(l) + r.row * m + r.c0, xr);
                RunIO<T>::ld(B(l) + r.row * m + r.c0, br);
            }
            __syncthreads();
        }
        for (int s = 0; s < nu2; ++s) {
            run_half_sweep(X(l), br, xr, r, m, 0);
            run_half_sweep(X(l), br, xr, r, m, 1);
        }
    }
    if (aligned) {
        for (int p = VW * tid; p < n * n; p += VW * nt)
            *reinterpret_cast<V *>(x + p) = *reinterpret_cast<const V *>(X(0) + p);
    } else {
        for (int p = tid; p < n * n; p += nt) x[p] = X(0)[p];
    }
}

template <typename T>
__global__ void __launch_bounds__(kBottomThreads) k_bottom(T *__restrict__ x, const T *__restrict__ b,
                                                           int n, int nlev, int nu1, int nu2,
                                                           int zero_init, const T *__restrict__ ainv,
                                                           FirTaps taps) {
    pdl_enter();
    bottom_body<T>(x, b, n, nlev, nu1, nu2, zero_init, ainv, taps);
}

// k_coarse_cluster: the down pass of the 128^2 level, the bottom V-cycle of
// the levels <= 64^2 and the up pass of the 128^2 level in one launch: a
// thread-block cluster of 8 CTAs of 1024 threads.  CTA r takes tile r of the
// 128^2 level (32 x 64 points, the tile functions of k_down / k_up with 1024
// threads; every point's arithmetic is theirs, so the results are the bits of
// the three separate launches), then CTA 0 runs the bottom V-cycle while the
// others wait, then every CTA prolongs, corrects and post-smooths its tile.
// The phases are ordered by the cluster's hardware barrier with release /
// acquire semantics, which also makes one phase's global writes visible to
// the next; the loads of data written inside the launch (the smoothed tile t
// and the bottom's correction xb) bypass the non-coherent read-only path.
constexpr int kCoarseCTAs = 8;
constexpr int kCoarseN = 128;  // the level above the bottom solve (64^2 and below)

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int NU1, int NU2>
__global__ void __cluster_dims__(kCoarseCTAs, 1, 1) __launch_bounds__(kBottomThreads)
    k_coarse_cluster(float *__restrict__ x, float *__restrict__ t, const float *__restrict__ b,
                     float *__restrict__ xb, float *__restrict__ bb, int nlev, const float *__restrict__ ainv,
                     FirTaps taps) {
    pdl_enter();
    constexpr int n = kCoarseN, TY = 32;
    constexpr int tpr = n / kTX;
    static_assert((n / TY) * tpr == kCoarseCTAs, "one tile per CTA");
    const int r = blockIdx.x;
    const int ty0 = (r / tpr) * TY, tx0 = (r % tpr) * kTX;
    down_tile<float, NU1, TY, false, kBottomThreads>(x, t, b, n, bb, ty0, tx0, true);
    cluster_barrier();
    if (r == 0) bottom_body<float>(xb, bb, n / 2, nlev, NU1, NU2, 1, ainv, taps);
    cluster_barrier();
    up_tile<float, NU2, TY, 2, kBottomThreads, true>(t, x, b, xb, nullptr, n, taps, ty0, tx0);
}

// one block per grid of the table
template <typename T>
__global__ void __launch_bounds__(kBottomThreads) k_bottom_batched(const BottomGrid *__restrict__ tab,
                                                                   int nu1, int nu2,
                                                                   const int *__restrict__ active,
                                                                   FirTaps taps) {
    pdl_enter();
    const BottomGrid g = tab[blockIdx.x];
    if (active && !active[g.rhs]) return;
    bottom_body<T>((T *)g.x, (const T *)g.b, g.n, g.nlev, nu1, nu2, g.zero, (const T *)g.ainv, taps);
}

// ---------------------------------------------------------------------------
// Outer kernels (FP64 data)
// ---------------------------------------------------------------------------
// The outer kernels are grid-stride loops over kRedBlocks x kRedThreads
// threads with kUnroll independent points per iteration (loads in flight).
constexpr int kUnroll = 4;

// The sums and the projection below read `alt` instead of their own array
// when par is null or *par is odd (the launchers pass alt = a when there is no
// alternative): a mixed solve whose fused update alternates a pair of FP64
// iterates sums and projects whichever holds the last one.  With zero_first
// and *par == 0 (no outer step ran on a cold start) the values are zero:
// pick_src returns null and nothing is read.
__device__ __forceinline__ const double *pick_src(const double *a, const double *alt, const int *par,
                                                  int zero_first) {
    if (par && zero_first && *par == 0) return nullptr;
    return (par ? (*par & 1) : 1) ? alt : a;
}

__global__ void __launch_bounds__(kRedThreads) k_sum(const double *a0, size_t N, Reduction red,
                                                     const double *alt, const int *par, int zero_first) {
    pdl_enter();
    const double *__restrict__ a = pick_src(a0, alt, par, zero_first);
    if (!a) N = 0;
    __shared__ double sh[32];
    double v = 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t p0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p0 < N; p0 += kUnroll * stride) {
        double t[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const size_t p = p0 + u * stride;
            t[u] = p < N ? a[p] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) v += t[u];
    }
    double vals[1] = {block_sum(v, sh)};
    reduce_finish<1>(red, vals, sh);
}

// The same sum on 16-byte-aligned data (N a multiple of 4): two 16-byte loads
// per thread and iteration, four groups in flight, so that enough loads are
// outstanding to cover the memory latency (the scalar form is latency-bound).
__global__ void __launch_bounds__(kRedThreads) k_sum_v(const double *a0, size_t N, Reduction red,
                                                       const double *alt, const int *par, int zero_first) {
    pdl_enter();
    const double *__restrict__ a = pick_src(a0, alt, par, zero_first);
    if (!a) N = 0;
    __shared__ double sh[32];
    double v = 0.0;
    const size_t G = N >> 1, stride = (size_t)gridDim.x * blockDim.x;
    const double2 *a2 = reinterpret_cast<const double2 *>(a);
    for (size_t g0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g0 < G; g0 += kUnroll * stride) {
        double2 t[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const size_t g = g0 + u * stride;
            t[u] = g < G ? a2[g] : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) v += t[u].x + t[u].y;
    }
    double vals[1] = {block_sum(v, sh)};
    reduce_finish<1>(red, vals, sh);
}

__global__ void __launch_bounds__(kRedThreads) k_scaled_rhs(const double *__restrict__ f, int n,
                                                            double h2, const double *__restrict__ fsum,
                                                            double *__restrict__ b) {
    pdl_enter();
    const size_t N = (size_t)n * n;
    const double mu = *fsum / (double)N;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x)
        b[p] = h2 * (f[p] - mu);
}

// residual_norm_note: the residual is exact before its rounding to float (the
// inner solve's input); its norm, which decides when to stop, is the 2-norm
// of those float values: each thread sums their squares exactly as a float
// pair (SqSum) and the block and grid sums run in FP64, so the norm carries
// the floats' rounding only (relative error <= 2^-24) and a relative residual
// of 1e-10 is known to ~7 digits.
//
// Scaled residual at point p = i * n + j of the periodic grid (n = 2^lg):
// s = b - (4 x - (x_N + x_S + x_W + x_E)), b = h^2 (f - mu), the stencil sum
// exact on the integer pipe (residual_exact_f32).  BMODE 0: b from f;
// 1: from f and stored to bsc; 2: loaded from bsc.  fc = f - mu (modes 0, 1).
template <int BMODE>
__device__ __forceinline__ float outer_point(const double *__restrict__ f, double *__restrict__ bsc,
                                             const double *__restrict__ x, size_t p, int n, int lg, double h2,
                                             double mu, double *fc) {
    const int i = (int)(p >> lg), j = (int)(p & (size_t)(n - 1));
    const size_t row = p - (size_t)j;
    const size_t up = (size_t)((i - 1) & (n - 1)) << lg, dn = (size_t)((i + 1) & (n - 1)) << lg;
    double b;
    if (BMODE == 2) {
        b = bsc[p];
        *fc = 0.0;
    } else {
        *fc = f[p] - mu;
        b = h2 * *fc;
        if (BMODE == 1) bsc[p] = b;
    }
    return residual_exact_f32(b, x[p], x[up + j], x[dn + j], x[row + ((j - 1) & (n - 1))],
                              x[row + ((j + 1) & (n - 1))]);
}

template <bool WRITE32, bool FNORM, int BMODE>
__global__ void __launch_bounds__(kRedThreads) k_outer_residual(
    const double *__restrict__ f, const double *__restrict__ x, int n, double h2,
    const double *__restrict__ fsum, double mu_host, float *__restrict__ s32, double *__restrict__ bsc,
    Reduction red) {
    pdl_enter();
    __shared__ double sh[32];
    const size_t N = (size_t)n * n;
    const int lg = __ffs(n) - 1;
    const double mu = fsum ? *fsum / (double)N : mu_host;
    SqSum ss;  // squares of the float residual (see residual_norm_note)
    double ff = 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t p0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p0 < N; p0 += 2 * stride) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const size_t p = p0 + u * stride;
            if (p < N) {
                double fc;
                const float sv = outer_point<BMODE>(f, bsc, x, p, n, lg, h2, mu, &fc);
                ss.add(sv);
                if (FNORM) ff += fc * fc;
                if (WRITE32) s32[p] = sv;
            }
        }
    }
    double vals[2];
    vals[0] = block_sum(ss.value(), sh);
    vals[1] = FNORM ? block_sum(ff, sh) : 0.0;
    reduce_finish<2>(red, vals, sh);
}

// ---------------------------------------------------------------------------
// Task-tiled outer residual (mixed solves).  A warp task is 32 columns (one per
// lane) x kResRows rows.  residual_exact_f32 aligns six operands per point;
// here each x value is aligned once, to the task's exponent
// E = max(largest x exponent + 2, largest b exponent), and reaches its four
// neighbours through registers (north, south) and shuffles (west, east; the
// task's two halo columns are held by lanes 0..kResRows-1 and 16..).  Every
// term is then a multiple of 2^(E - 1082): |b| < 2^60, |4x| and each
// neighbour < 2^58 (E >= x exponent + 2), so the int64 sum cannot overflow.
// Truncation leaves each x within one unit (4x within four) and b within two
// (its stored alignment, then the shift), under 10 units = 10 * 2^-59 of the
// task's largest operand in all; the sum is then rounded once to binary32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned hi_abs(double v) {
    return (unsigned)((unsigned long long)__double_as_longlong(v) >> 32) & 0x7fffffffu;
}

// v as a multiple of 2^(E - 1082), truncated toward zero (E >= v's biased exponent).
__device__ __forceinline__ long long align_to(double v, int E) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(u >> 32);
    const int ef = (int)((hi >> 20) & 0x7ffu);
    const unsigned long long m = (u & 0x000fffffffffffffull) | (ef ? (1ull << 52) : 0ull);
    const long long a = (long long)((m << 7) >> min(E - (ef ? ef : 1), 63));
    return (hi >> 31) ? -a : a;
}

// acc * 2^(E - 1082) rounded once to binary32.  The conversion rounds acc to
// 24 bits and the power-of-two scale (an exponent-field add) is exact while
// the result is a normal float; exact_to_f32 takes the other cases.  (The
// hardware int64 conversion runs on the FP64 pipe, which this kernel leaves
// mostly idle; the all-integer rounding measured slower, 26 -> 31 us, on the
// busier ALU pipe.)
__device__ __forceinline__ float aligned_to_f32(long long acc, int E) {
    const float v = __ll2float_rn(acc);
    const int ev = (int)((__float_as_uint(v) >> 23) & 0xffu);
    if (ev == 0) return 0.0f;  // acc == 0 (a nonzero integer converts to a normal float)
    const int k = E - 1082, er = ev + k;
    if (er >= 1 && er <= 254) return __uint_as_float(__float_as_uint(v) + ((unsigned)k << 23));
    return exact_to_f32(acc, E);
}

// UPD (steady residuals only): the task first applies the outer step's FP64
// update x + e to every value it loads (its own rows, the neighbour rows and
// the halo columns, by the addition the update kernel makes), stores its own
// rows to xo and sums their e^2 into ee; the residual is then that of x + e.
// XZERO: x is zero (a solve's cold start) and is not read.
template <bool FIRST, bool UPD = false, bool XZERO = false>
__device__ __forceinline__ void residual_task(int task, int n, int lg, const double *__restrict__ f, double mu,
                                              double h2, long long *__restrict__ bint, int *__restrict__ ebt,
                                              const double *__restrict__ x, float *__restrict__ s32, SqSum &ss,
                                              double &ff, const float *__restrict__ e = nullptr,
                                              double *__restrict__ xo = nullptr, SqSum *ee = nullptr) {
    static_assert(!(FIRST && UPD), "the first residual of a solve has no update");
    constexpr int R = kResRows;
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int strips = n >> 5;
    const int c0 = (task % strips) << 5, r0 = (task / strips) * R;
    const int c = c0 + lane;
    double xv[R + 2];  // rows r0 - 1 .. r0 + R of column c
#pragma unroll
    for (int k = 0; k < R + 2; ++k) xv[k] = XZERO ? 0.0 : x[((size_t)((r0 - 1 + k) & (n - 1)) << lg) + c];
    // halo columns: lane k < R holds x[r0 + k][c0 - 1], lane 16 + k holds x[r0 + k][c0 + 32]
    const int hk = lane & 15;
    double hv = 0.0;
    if (!XZERO && hk < R) hv = x[((size_t)(r0 + hk) << lg) + ((lane < 16 ? c0 - 1 : c0 + 32) & (n - 1))];
    if (UPD) {
        float ev[R + 2];
#pragma unroll
        for (int k = 0; k < R + 2; ++k) ev[k] = e[((size_t)((r0 - 1 + k) & (n - 1)) << lg) + c];
        float he = 0.f;
        if (hk < R) he = e[((size_t)(r0 + hk) << lg) + ((lane < 16 ? c0 - 1 : c0 + 32) & (n - 1))];
#pragma unroll
        for (int k = 0; k < R + 2; ++k) xv[k] = xv[k] + f32_to_f64(ev[k]);
        hv = hv + f32_to_f64(he);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            xo[((size_t)(r0 + k) << lg) + c] = xv[k + 1];
            ee->add(ev[k + 1]);
        }
    }
    long long bq[R];
    int eb;
    if (FIRST) {
        double bv[R];
        unsigned hb = 0u;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const double fc = f[((size_t)(r0 + k) << lg) + c] - mu;
            ff += fc * fc;
            bv[k] = h2 * fc;
            hb = max(hb, hi_abs(bv[k]));
        }
        eb = max((int)(__reduce_max_sync(kFull, hb) >> 20), 1);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            bq[k] = align_to(bv[k], eb);
            bint[((size_t)(r0 + k) << lg) + c] = bq[k];
        }
        if (lane == 0) ebt[task] = eb;
    } else {
        eb = ebt[task];
#pragma unroll
        for (int k = 0; k < R; ++k) bq[k] = bint[((size_t)(r0 + k) << lg) + c];
    }
    unsigned hx = hi_abs(hv);
#pragma unroll
    for (int k = 0; k < R + 2; ++k) hx = max(hx, hi_abs(xv[k]));
    const int ex = max((int)(__reduce_max_sync(kFull, hx) >> 20), 1);
    const bool special = ex == 0x7ff || eb == 0x7ff;  // an infinity or NaN in the task
    const int E = max(ex + 2, eb);
    const int bs = min(E - eb, 63);
    long long X[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) X[k] = align_to(xv[k], E);
    const long long H = align_to(hv, E);
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const long long C = X[k + 1];
        long long W = __shfl_up_sync(kFull, C, 1), Ea = __shfl_down_sync(kFull, C, 1);
        const long long hW = __shfl_sync(kFull, H, k), hE = __shfl_sync(kFull, H, 16 + k);
        if (lane == 0) W = hW;
        if (lane == 31) Ea = hE;
        const long long acc = ((bq[k] >> bs) - C * 4) + ((X[k] + X[k + 2]) + (W + Ea));
        const float sv = special ? __uint_as_float(0x7fc00000u) : aligned_to_f32(acc, E);
        ss.add(sv);
        s32[((size_t)(r0 + k) << lg) + c] = sv;
    }
}

// xzero (first residuals only): x is zero and is not read.
template <bool FIRST>
__global__ void __launch_bounds__(kRedThreads, FIRST ? 2 : 3) k_outer_residual_t(
    const double *__restrict__ f, const double *__restrict__ x, int n, double h2, const double *__restrict__ fsum,
    double mu_host, float *__restrict__ s32, long long *__restrict__ bint, int *__restrict__ ebt, Reduction red,
    int xzero) {
    pdl_enter();
    __shared__ double sh[32];
    const int lg = __ffs(n) - 1;
    const double mu = fsum ? *fsum / ((double)n * n) : mu_host;
    SqSum ss;  // squares of the float residual (see residual_norm_note)
    double ff = 0.0;
    const int ntask = (n >> 5) * (n / kResRows), wpb = blockDim.x >> 5;
    const int t0 = blockIdx.x * wpb + (int)(threadIdx.x >> 5), ts = gridDim.x * wpb;
    if (FIRST && xzero) {
        for (int t = t0; t < ntask; t += ts)
            residual_task<FIRST, false, FIRST>(t, n, lg, f, mu, h2, bint, ebt, x, s32, ss, ff);
    } else {
        for (int t = t0; t < ntask; t += ts) residual_task<FIRST>(t, n, lg, f, mu, h2, bint, ebt, x, s32, ss, ff);
    }
    double vals[2];
    vals[0] = block_sum(ss.value(), sh);
    vals[1] = FIRST ? block_sum(ff, sh) : 0.0;
    reduce_finish<2>(red, vals, sh);
}

// An outer step's FP64 update fused with the next outer residual (mixed
// solves of n >= kResMinN): x_new = x_old + e, written to the other buffer of
// the pair (xa, xb), and the task-tiled residual of x_new from the same loads,
// with out[0] = sum of the float residual's squares and out[1] = sum of e^2.
// Every task reads x_old and writes x_new in different buffers, so no task
// reads what another writes; each stored x_new and each residual is bit for
// bit that of k_update_v followed by k_outer_residual_t<false>.  The outer
// step index k (*step_dev, else step_host; from 0) selects the buffers: the
// source is xb when k is odd, else xa; with zero_first the source of step 0
// is zero (a solve's cold start) and is not read.
__global__ void __launch_bounds__(kRedThreads, 3) k_update_residual_t(
    double *xa, double *xb, const int *__restrict__ step_dev, int step_host, int zero_first,
    const float *__restrict__ e, int n, double h2, float *__restrict__ s32, long long *__restrict__ bint,
    int *__restrict__ ebt, Reduction red) {
    pdl_enter();
    __shared__ double sh[32];
    const int step = step_dev ? *step_dev : step_host;
    const double *__restrict__ x = (step & 1) ? xb : xa;
    double *__restrict__ xo = (step & 1) ? xa : xb;
    const int lg = __ffs(n) - 1;
    SqSum ss, ee;
    double ff = 0.0;
    const int ntask = (n >> 5) * (n / kResRows), wpb = blockDim.x >> 5;
    const int t0 = blockIdx.x * wpb + (int)(threadIdx.x >> 5), ts = gridDim.x * wpb;
    if (zero_first && step == 0) {
        for (int t = t0; t < ntask; t += ts)
            residual_task<false, true, true>(t, n, lg, nullptr, 0.0, h2, bint, ebt, x, s32, ss, ff, e, xo, &ee);
    } else {
        for (int t = t0; t < ntask; t += ts)
            residual_task<false, true>(t, n, lg, nullptr, 0.0, h2, bint, ebt, x, s32, ss, ff, e, xo, &ee);
    }
    double vals[2];
    vals[0] = block_sum(ss.value(), sh);
    vals[1] = block_sum(ee.value(), sh);
    reduce_finish<2>(red, vals, sh);
}

// x += e (FP64 update by the FP32 correction), sum e^2 -> out[0] (squares
// summed exactly per thread as a float pair, then in FP64 across threads).
__global__ void __launch_bounds__(kRedThreads) k_update(double *__restrict__ x,
                                                        const float *__restrict__ e, size_t N,
                                                        Reduction red) {
    pdl_enter();
    __shared__ double sh[32];
    SqSum ee;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t p0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p0 < N; p0 += kUnroll * stride) {
        float ev[kUnroll];
        double xv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const size_t p = p0 + u * stride;
            ev[u] = p < N ? e[p] : 0.f;
            xv[u] = p < N ? x[p] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const size_t p = p0 + u * stride;
            if (p < N) x[p] = xv[u] + f32_to_f64(ev[u]);
            ee.add(ev[u]);
        }
    }
    double vals[1] = {block_sum(ee.value(), sh)};
    reduce_finish<1>(red, vals, sh);
}

// The same update on 16-byte-aligned x and e, four points per 16-byte load of
// e (two loads of x), two groups in flight per thread.  N is a multiple of 4.
__global__ void __launch_bounds__(kRedThreads) k_update_v(double *__restrict__ x, const float *__restrict__ e,
                                                          size_t N, Reduction red) {
    pdl_enter();
    __shared__ double sh[32];
    SqSum ee;
    const size_t G = N >> 2, stride = (size_t)gridDim.x * blockDim.x;
    const float4 *e4 = reinterpret_cast<const float4 *>(e);
    double2 *x2 = reinterpret_cast<double2 *>(x);
    for (size_t g0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g0 < G; g0 += 2 * stride) {
        float4 ev[2];
        double2 xa[2], xb[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const size_t g = g0 + u * stride;
            if (g < G) {
                ev[u] = e4[g];
                xa[u] = x2[2 * g];
                xb[u] = x2[2 * g + 1];
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const size_t g = g0 + u * stride;
            if (g < G) {
                x2[2 * g] = make_double2(xa[u].x + f32_to_f64(ev[u].x), xa[u].y + f32_to_f64(ev[u].y));
                x2[2 * g + 1] = make_double2(xb[u].x + f32_to_f64(ev[u].z), xb[u].y + f32_to_f64(ev[u].w));
                ee.add(ev[u].x);
                ee.add(ev[u].y);
                ee.add(ev[u].z);
                ee.add(ev[u].w);
            }
        }
    }
    double vals[1] = {block_sum(ee.value(), sh)};
    reduce_finish<1>(red, vals, sh);
}

// ---------------------------------------------------------------------------
// Cubic spline prolongation by 2^lgf (two-level configuration)
// ---------------------------------------------------------------------------
struct BspTaps {
    float a[kBspTaps + 1];
};

// One axis of the B-spline coefficient filter (see launch_bspline_coef).
__global__ void __launch_bounds__(kRedThreads) k_bspline_coef(const float *__restrict__ e, float *__restrict__ c,
                                                              int nc, int dir, BspTaps taps) {
    pdl_enter();
    const int npt = nc * nc;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npt; p += gridDim.x * blockDim.x) {
        const int I = p / nc, J = p - I * nc;
        float acc = 0.f;
#pragma unroll
        for (int k = kBspTaps; k >= 1; --k) {
            const float u = dir == 0 ? e[I * nc + ((J + k) % nc)] : e[((I + k) % nc) * nc + J];
            const float w = dir == 0 ? e[I * nc + ((J - k) % nc + nc) % nc] : e[(((I - k) % nc + nc) % nc) * nc + J];
            acc = fmaf(taps.a[k], u + w, acc);
        }
        c[p] = fmaf(taps.a[0], e[p], acc);
    }
}

// ef(i, j) += sum_{a,b = 0..3} wy_a wx_b c(I - 1 + a, J - 1 + b), (I, J) = (i, j) >> lgf,
// w the uniform cubic B-spline weights at t = ((i, j) mod 2^lgf) / 2^lgf.
__global__ void __launch_bounds__(kRedThreads) k_prolong_factor(float *__restrict__ ef, const float *__restrict__ c,
                                                                int n, int lgf) {
    pdl_enter();
    const int nc = n >> lgf, lg = __ffs(n) - 1;
    const float inv = 1.0f / (float)(1 << lgf);
    const size_t npt = (size_t)n * n;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < npt; p += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(p >> lg), j = (int)(p & (size_t)(n - 1));
        const int I = i >> lgf, J = j >> lgf;
        float wy[4], wx[4];
        const float ty = (float)(i & ((1 << lgf) - 1)) * inv, tx = (float)(j & ((1 << lgf) - 1)) * inv;
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            const float t = d ? tx : ty, u = 1.f - t;
            float *w = d ? wx : wy;
            w[0] = u * u * u * (1.f / 6.f);
            w[1] = ((3.f * t - 6.f) * t * t + 4.f) * (1.f / 6.f);
            w[2] = (((-3.f * t + 3.f) * t + 3.f) * t + 1.f) * (1.f / 6.f);
            w[3] = t * t * t * (1.f / 6.f);
        }
        float v = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const float *row = c + (size_t)((I - 1 + a + nc) % nc) * nc;
            float r = 0.f;
#pragma unroll
            for (int b = 0; b < 4; ++b) r = fmaf(wx[b], row[(J - 1 + b + nc) % nc], r);
            v = fmaf(wy[a], r, v);
        }
        ef[p] += v;
    }
}

__global__ void k_convert(int dir, size_t count, const void *__restrict__ in, void *__restrict__ out) {
    pdl_enter();
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < count; p += (size_t)gridDim.x * blockDim.x) {
        if (dir == 0)
            ((float *)out)[p] = f64_to_f32_rn(((const double *)in)[p]);
        else
            ((double *)out)[p] = f32_to_f64(((const float *)in)[p]);
    }
}

__global__ void __launch_bounds__(kRedThreads) k_project(double *x, size_t N, const double *__restrict__ sum,
                                                         const int *__restrict__ zero_flag, const double *alt,
                                                         const int *par, int zero_first) {
    pdl_enter();
    const bool zero = zero_flag && *zero_flag;
    const double mu = *sum / (double)N;
    const double *src = pick_src(x, alt, par, zero_first);
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x)
        x[p] = zero ? 0.0 : (src ? src[p] : 0.0) - mu;
}

// The same projection on 16-byte-aligned x (N a multiple of 4), two 16-byte
// words per thread and iteration.
__global__ void __launch_bounds__(kRedThreads) k_project_v(double *x, size_t N, const double *__restrict__ sum,
                                                           const int *__restrict__ zero_flag, const double *alt,
                                                           const int *par, int zero_first) {
    pdl_enter();
    const bool zero = zero_flag && *zero_flag;
    const double mu = *sum / (double)N;
    double2 *x2 = reinterpret_cast<double2 *>(x);
    const double2 *s2 = reinterpret_cast<const double2 *>(pick_src(x, alt, par, zero_first));
    const size_t G = N >> 1, stride = (size_t)gridDim.x * blockDim.x;
    for (size_t g0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g0 < G; g0 += 2 * stride) {
        double2 t[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const size_t g = g0 + u * stride;
            if (g < G) t[u] = s2 ? s2[g] : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const size_t g = g0 + u * stride;
            if (g < G) x2[g] = zero ? make_double2(0.0, 0.0) : make_double2(t[u].x - mu, t[u].y - mu);
        }
    }
}

__global__ void k_check(DevState *st, const double *rsum, const double *usum, const double *fsum,
                        double n2, double h2, double tol, int step, int max_cycles, int first,
                        cudaGraphConditionalHandle handle, double rho, CycleHandles ifh) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (first) {
        st->fnorm = sqrt(rsum[1]);
        st->mu = fsum[0] / n2;
        st->cycles = 0;
        st->outer = 0;
        st->status = MG_OK;
        st->zero_source = 0;
        st->unorm = 0.0;
        st->sr_used = 0;
        st->sr_step = 0;
        st->fallback = 0;
    } else {
        st->cycles += rho > 0.0 ? st->m_next : step;
        st->outer += 1;
        if (usum) st->unorm = sqrt(usum[0]);
    }
    int m = step;
    const double rn = sqrt(rsum[0]) / h2, fn = st->fnorm;
    unsigned go = 0;
    if (!isfinite(rn) || !isfinite(fn)) {
        st->status = MG_ERR_NONFINITE;
        st->rel = rn / fn;
    } else if (fn == 0.0) {
        st->zero_source = 1;
        st->rel = 0.0;
    } else {
        const double rel = rn / fn;
        if (!first && st->sr_step && !(rel <= kSrMinReduction * st->rel_prev)) st->fallback = 1;
        st->sr_step = 0;
        st->rel_prev = rel;
        st->rel = rel;
        if (rel > tol) {
            if (rho > 0.0) {
                m = adaptive_cycles(rel, tol, rho, step);
                if (st->cycles + 1 <= max_cycles) {
                    go = 1;
                    if (m > max_cycles - st->cycles) m = max_cycles - st->cycles;
                } else {
                    st->status = MG_ERR_NOT_CONVERGED;
                }
            } else if (st->cycles + step <= max_cycles) {
                go = 1;
            } else {
                st->status = MG_ERR_NOT_CONVERGED;
            }
        }
    }
    st->m_next = m;
    if (rho > 0.0)
        for (int k = 2; k <= step && k <= kMaxAdaptive; ++k) cudaGraphSetConditional(ifh.h[k - 2], (go && m >= k) ? 1u : 0u);
    cudaGraphSetConditional(handle, go);
}

__global__ void k_policy(DevState *st, int k, ProlongPolicy p, int *flag, cudaGraphConditionalHandle handle) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const bool use = policy_use_sr(p, st->cycles + k + 1, st->rel, true, st->fallback != 0);
    *flag = use ? 1 : 0;
    if (use) {
        st->sr_used += 1;
        st->sr_step = 1;
    }
    cudaGraphSetConditional(handle, use ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Batched outer kernels: the blocks of right-hand side r are
// [blk0, blk0 + nblk); each right-hand side's sums finish in its last block.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_rhs(const RhsDesc *__restrict__ r, int nrhs) {
    int lo = 0, hi = nrhs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (r[mid].blk0 <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int NS>
__device__ __forceinline__ void batch_finish(const BatchRed &red, int slot, int blk0, int nblk,
                                             const double (&vals)[NS], double *sh) {
    const int rhs = slot;
    __shared__ bool am_last;
    if (threadIdx.x == 0) {
        for (int k = 0; k < NS; ++k) red.partials[(size_t)blockIdx.x * kMaxSlots + k] = vals[k];
        __threadfence();
        const unsigned ticket = atomicAdd(&red.counters[rhs], 1u);
        am_last = (ticket == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    for (int k = 0; k < NS; ++k) {
        double v = 0.0;
        for (int i = threadIdx.x; i < nblk; i += blockDim.x)
            v += ((volatile double *)red.partials)[(size_t)(blk0 + i) * kMaxSlots + k];
        v = block_sum(v, sh);
        if (threadIdx.x == 0) red.out[(size_t)rhs * kMaxSlots + k] = v;
    }
    if (threadIdx.x == 0) red.counters[rhs] = 0u;
}

// The x of a right-hand side of a batch with the fused outer step: its xalt
// after an odd number of outer steps (st non-null), else x.
__device__ __forceinline__ const double *batch_x(const RhsDesc &d, const DevState *st) {
    return (st && d.xalt && (st[d.slot].outer & 1)) ? d.xalt : d.x;
}

template <bool OF_X>
__global__ void __launch_bounds__(kRedThreads) k_sum_b(const RhsDesc *__restrict__ rd, int nrhs, BatchRed red,
                                                       const DevState *__restrict__ st) {
    pdl_enter();
    __shared__ double sh[32];
    const int r = find_rhs(rd, nrhs);
    const RhsDesc d = rd[r];
    const size_t N = (size_t)d.n * d.n;
    const double *a = OF_X ? batch_x(d, st) : d.f;
    double v = 0.0;
    for (size_t p = (size_t)(blockIdx.x - d.blk0) * blockDim.x + threadIdx.x; p < N; p += (size_t)d.nblk * blockDim.x)
        v += a[p];
    double vals[1] = {block_sum(v, sh)};
    batch_finish<1>(red, d.slot, d.blk0, d.nblk, vals, sh);
}

// One right-hand side's points of a batched outer residual (see outer_point).
template <int BMODE>
__device__ __forceinline__ void outer_rows_b(const RhsDesc &d, double mu, SqSum &ss, double &ff) {
    const int n = d.n, lg = __ffs(n) - 1;
    const size_t N = (size_t)n * n;
    const size_t stride = (size_t)d.nblk * blockDim.x;
    for (size_t p0 = (size_t)(blockIdx.x - d.blk0) * blockDim.x + threadIdx.x; p0 < N; p0 += 2 * stride) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const size_t p = p0 + u * stride;
            if (p < N) {
                double fc;
                const float sv = outer_point<BMODE>(d.f, d.bsc, d.x, p, n, lg, d.h2, mu, &fc);
                ss.add(sv);
                if (BMODE == 1) ff += fc * fc;
                d.s32[p] = sv;
            }
        }
    }
}

template <bool FNORM>
__global__ void __launch_bounds__(kRedThreads) k_outer_residual_b(const RhsDesc *__restrict__ rd, int nrhs,
                                                                  const double *__restrict__ fsum, int first_all,
                                                                  const int *__restrict__ active, BatchRed red) {
    pdl_enter();
    __shared__ double sh[32];
    const RhsDesc d = rd[find_rhs(rd, nrhs)];
    if (active && !active[d.slot]) return;
    const size_t N = (size_t)d.n * d.n;
    const double mu = fsum[(size_t)d.slot * kMaxSlots] / (double)N;
    SqSum ss;
    double ff = 0.0;
    const bool fresh = FNORM && (first_all || d.first);
    if (d.n >= kResMinN) {
        const int n = d.n, lg = __ffs(n) - 1, wpb = blockDim.x >> 5;
        const int ntask = (n >> 5) * (n / kResRows);
        long long *bint = reinterpret_cast<long long *>(d.bsc);
        for (int t = (blockIdx.x - d.blk0) * wpb + (int)(threadIdx.x >> 5); t < ntask; t += d.nblk * wpb) {
            if (fresh)
                residual_task<true>(t, n, lg, d.f, mu, d.h2, bint, d.ebt, d.x, d.s32, ss, ff);
            else
                residual_task<false>(t, n, lg, d.f, mu, d.h2, bint, d.ebt, d.x, d.s32, ss, ff);
        }
    } else if (fresh) {
        outer_rows_b<1>(d, mu, ss, ff);
    } else {
        outer_rows_b<2>(d, mu, ss, ff);
    }
    double vals[2];
    vals[0] = block_sum(ss.value(), sh);
    vals[1] = FNORM ? block_sum(ff, sh) : 0.0;
    batch_finish<2>(red, d.slot, d.blk0, d.nblk, vals, sh);
}

__global__ void __launch_bounds__(kRedThreads) k_update_b(const RhsDesc *__restrict__ rd, int nrhs,
                                                          const int *__restrict__ active, BatchRed red) {
    pdl_enter();
    __shared__ double sh[32];
    const RhsDesc d = rd[find_rhs(rd, nrhs)];
    if (active && !active[d.slot]) return;
    const size_t N = (size_t)d.n * d.n;
    SqSum ee;
    const size_t stride = (size_t)d.nblk * blockDim.x;
    for (size_t p0 = (size_t)(blockIdx.x - d.blk0) * blockDim.x + threadIdx.x; p0 < N; p0 += kUnroll * stride) {
        float ev[kUnroll];
        double xv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const size_t p = p0 + u * stride;
            ev[u] = p < N ? d.e[p] : 0.f;
            xv[u] = p < N ? d.x[p] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const size_t p = p0 + u * stride;
            if (p < N) d.x[p] = xv[u] + f32_to_f64(ev[u]);
            ee.add(ev[u]);
        }
    }
    double vals[1] = {block_sum(ee.value(), sh)};
    batch_finish<1>(red, d.slot, d.blk0, d.nblk, vals, sh);
}

__global__ void __launch_bounds__(kRedThreads) k_project_b(const RhsDesc *__restrict__ rd, int nrhs,
                                                           const double *__restrict__ xsum,
                                                           const DevState *__restrict__ st, int fused) {
    pdl_enter();
    const RhsDesc d = rd[find_rhs(rd, nrhs)];
    const size_t N = (size_t)d.n * d.n;
    const bool zero = st[d.slot].zero_source != 0;
    const double mu = xsum[(size_t)d.slot * kMaxSlots] / (double)N;
    const double *src = batch_x(d, fused ? st : nullptr);
    for (size_t p = (size_t)(blockIdx.x - d.blk0) * blockDim.x + threadIdx.x; p < N; p += (size_t)d.nblk * blockDim.x)
        d.x[p] = zero ? 0.0 : src[p] - mu;
}

// Batched k_update_residual_t: one right-hand side's blocks take its tasks;
// the slot's outer-step count selects the source of (x, xalt).
__global__ void __launch_bounds__(kRedThreads, 3) k_update_residual_b(const RhsDesc *__restrict__ rd, int nrhs,
                                                                      const DevState *__restrict__ st,
                                                                      const int *__restrict__ active, BatchRed red) {
    pdl_enter();
    __shared__ double sh[32];
    const RhsDesc d = rd[find_rhs(rd, nrhs)];
    if (active && !active[d.slot]) return;
    const int step = st[d.slot].outer;
    const double *__restrict__ x = (step & 1) ? d.xalt : d.x;
    double *__restrict__ xo = (step & 1) ? d.x : d.xalt;
    const int n = d.n, lg = __ffs(n) - 1, wpb = blockDim.x >> 5;
    const int ntask = (n >> 5) * (n / kResRows);
    long long *bint = reinterpret_cast<long long *>(d.bsc);
    SqSum ss, ee;
    double ff = 0.0;
    for (int t = (blockIdx.x - d.blk0) * wpb + (int)(threadIdx.x >> 5); t < ntask; t += d.nblk * wpb)
        residual_task<false, true>(t, n, lg, nullptr, 0.0, d.h2, bint, d.ebt, x, d.s32, ss, ff, d.e, xo, &ee);
    double vals[2];
    vals[0] = block_sum(ss.value(), sh);
    vals[1] = block_sum(ee.value(), sh);
    batch_finish<2>(red, d.slot, d.blk0, d.nblk, vals, sh);
}

// Convergence test of every listed right-hand side still active (or at its
// first residual); a graph loop continues while any is.  One block.
// With rho > 0 (adaptive inner cycles) the batch's next outer step runs m
// V-cycles, the largest adaptive_cycles(...) of its still-active right-hand
// sides, capped by the smallest cycle budget left among them; batch_m[0] holds
// the m of the step just run, batch_m[1] the V-cycles run so far.
__global__ void k_check_b(DevState *st, const RhsDesc *__restrict__ rd, int nrhs, const double *rsum,
                          const double *usum, const double *fsum, double tol, int step, int max_cycles,
                          int first_all, int *active, cudaGraphConditionalHandle handle, int use_handle,
                          double rho, CycleHandles ifh, int *batch_m) {
    pdl_enter();
    __shared__ int s_m, s_left;
    if (threadIdx.x == 0) {
        s_m = 1;
        s_left = max_cycles;
    }
    __syncthreads();
    const int m_prev = (rho > 0.0 && !first_all) ? batch_m[0] : step;
    int any = 0;
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
        const int slot = rd[r].slot;
        const bool first = first_all || rd[r].first;
        if (!first && !active[slot]) continue;
        DevState &s = st[slot];
        const double n2 = (double)rd[r].n * rd[r].n, h2 = rd[r].h2;
        const double *rs = rsum + (size_t)slot * kMaxSlots;
        if (first) {
            s.fnorm = sqrt(rs[1]);
            s.mu = fsum[(size_t)slot * kMaxSlots] / n2;
            s.cycles = 0;
            s.outer = 0;
            s.status = MG_OK;
            s.zero_source = 0;
            s.unorm = 0.0;
            s.sr_used = 0;
            s.sr_step = 0;
            s.fallback = 0;
            s.rel_prev = 0.0;
        } else {
            s.cycles += rd[r].m_prev > 0 ? rd[r].m_prev : m_prev;
            s.outer += 1;
            s.unorm = sqrt(usum[(size_t)slot * kMaxSlots]);
        }
        const double rn = sqrt(rs[0]) / h2, fn = s.fnorm;
        int go = 0;
        if (!isfinite(rn) || !isfinite(fn)) {
            s.status = MG_ERR_NONFINITE;
            s.rel = rn / fn;
        } else if (fn == 0.0) {
            s.zero_source = 1;
            s.rel = 0.0;
        } else {
            const double rel = rn / fn;
            // SR bookkeeping (batched SR solves; rd.sr = 0 otherwise): a step
            // that used SR and did not reduce the relative residual by
            // kSrMinReduction drops SR for the rest of this solve
            if (!first && s.sr_step) {
                s.sr_used += rd[r].m_prev > 0 ? rd[r].m_prev : m_prev;
                if (!(rel <= kSrMinReduction * s.rel_prev)) s.fallback = 1;
            }
            s.sr_step = (rd[r].sr && !s.fallback) ? 1 : 0;
            s.rel_prev = rel;
            s.rel = rel;
            if (rel > tol) {
                if (rho > 0.0) {
                    if (s.cycles + 1 <= max_cycles) {
                        go = 1;
                        atomicMax(&s_m, adaptive_cycles(rel, tol, rho, step));
                        atomicMin(&s_left, max_cycles - s.cycles);
                    } else {
                        s.status = MG_ERR_NOT_CONVERGED;
                    }
                } else if (s.cycles + step <= max_cycles) {
                    go = 1;
                } else {
                    s.status = MG_ERR_NOT_CONVERGED;
                }
            }
        }
        active[slot] = go;
        any |= go;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        if (rho > 0.0) {
            const int m = s_m < s_left ? s_m : s_left;
            batch_m[0] = m;
            if (first_all) batch_m[1] = 0;
            if (any) batch_m[1] += m;
            for (int k = 2; k <= step && k <= kMaxAdaptive; ++k)
                cudaGraphSetConditional(ifh.h[k - 2], (any && m >= k) ? 1u : 0u);
        }
        if (use_handle) cudaGraphSetConditional(handle, any ? 1u : 0u);
    }
}

template <typename KernelT>
cudaError_t set_smem(KernelT k, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// set_smem once per (kernel instantiation, device): `done` is that
// instantiation's bit mask of devices already configured.
template <typename KernelT>
cudaError_t set_smem_once(KernelT k, size_t bytes, std::atomic<unsigned> &done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned bit = dev < 32 ? (1u << dev) : 0u;
    if (bit && (done.load(std::memory_order_relaxed) & bit)) return cudaSuccess;
    e = set_smem(k, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_relaxed);
    return e;
}

template <typename T, int NU, bool ZERO, int TY>
cudaError_t down_impl(const T *x, T *xout, const T *b, int n, T *bc, cudaStream_t s) {
    using Cfg = DownCfg<T, NU, TY>;
    auto k = k_down<T, NU, ZERO, TY>;
    static std::atomic<unsigned> done{0};
    cudaError_t e = set_smem_once(k, Cfg::smem, done);
    if (e != cudaSuccess) return e;
    dim3 grid(n / Cfg::TX, n / Cfg::TY);
    {
        cudaError_t le_ = launch_kernel(k, grid, kThreads, Cfg::smem, s,
                                        x, xout, b, n, bc);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, int NU, int TY, int NJ>
cudaError_t up_impl(const T *x, T *xout, const T *b, const T *ec, const T *extra, const int *eflag, int n,
                    const FirTaps &taps, cudaStream_t s, const T *xr = nullptr) {
    using Cfg = UpCfg<T, NU, TY, NJ>;
    auto k = k_up<T, NU, TY, NJ>;
    static std::atomic<unsigned> done{0};
    cudaError_t e = set_smem_once(k, Cfg::smem, done);
    if (e != cudaSuccess) return e;
    dim3 grid(n / Cfg::TX, n / Cfg::TY);
    // pre-refined rows need no coarse tile: less shared memory, more blocks per SM
    const size_t smem = (NJ == 1 && std::is_same<T, double>::value && xr) ? Cfg::smem_xr : Cfg::smem;
    {
        cudaError_t le_ = launch_kernel(k, grid, kThreads, smem, s,
                                        x, xout, b, ec, extra, eflag, n, taps, xr);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, int NU, bool ZERO>
cudaError_t down_var(const T *x, T *xout, const T *b, int n, T *bc, cudaStream_t s, int variant) {
    if constexpr (std::is_same<T, double>::value) {
        return down_impl<T, NU, ZERO, Fixed64<double>::TY>(x, xout, b, n, bc, s);
    } else {
        switch (variant_rows(variant)) {
            case 8: return down_impl<T, NU, ZERO, 8>(x, xout, b, n, bc, s);
            case 16: return down_impl<T, NU, ZERO, 16>(x, xout, b, n, bc, s);
            case 32: return down_impl<T, NU, ZERO, 32>(x, xout, b, n, bc, s);
            default: return down_impl<T, NU, ZERO, 64>(x, xout, b, n, bc, s);
        }
    }
}

template <typename T, int NU>
cudaError_t up_var(const T *x, T *xout, const T *b, const T *ec, const T *extra, const int *eflag, int n,
                   const FirTaps &taps, cudaStream_t s, int variant, const T *xr) {
    if constexpr (std::is_same<T, double>::value) {
        return up_impl<T, NU, Fixed64<double>::TY, Fixed64<double>::NJ>(x, xout, b, ec, extra, eflag, n, taps, s,
                                                                        xr);
    } else {
#define MG_UP_ROWS(TYV)                                                                                  \
    case TYV:                                                                                            \
        return nj2 ? up_impl<T, NU, TYV, 2>(x, xout, b, ec, extra, eflag, n, taps, s)                   \
                   : up_impl<T, NU, TYV, 1>(x, xout, b, ec, extra, eflag, n, taps, s);
        const bool nj2 = variant_runs(variant) == 2;
        switch (variant_rows(variant)) {
            MG_UP_ROWS(8)
            MG_UP_ROWS(16)
            MG_UP_ROWS(32)
            default:
                return nj2 ? up_impl<T, NU, 64, 2>(x, xout, b, ec, extra, eflag, n, taps, s)
                           : up_impl<T, NU, 64, 1>(x, xout, b, ec, extra, eflag, n, taps, s);
        }
#undef MG_UP_ROWS
    }
}

}  // namespace

template <typename T>
cudaError_t launch_down(const T *x, T *xout, const T *b, int n, int nu, bool zero_init, T *bc,
                        cudaStream_t s, int variant) {
    if (n < 64 || x == xout || variant < -1 || variant >= kTileVariants) return cudaErrorInvalidValue;
    if (variant < 0) variant = tile_variant(0, n, nu);
#define MG_DOWN_CASE(NU)                                                                  \
    case NU:                                                                              \
        return zero_init ? down_var<T, NU, true>(x, xout, b, n, bc, s, variant)           \
                         : down_var<T, NU, false>(x, xout, b, n, bc, s, variant);
    switch (nu) {
        MG_DOWN_CASE(0)
        MG_DOWN_CASE(1)
        MG_DOWN_CASE(2)
        MG_DOWN_CASE(3)
        MG_DOWN_CASE(4)
        default: return cudaErrorInvalidValue;
    }
#undef MG_DOWN_CASE
}

// Box of the TMA-staged k_down tile (columns, rows) for sweeps nu.
void down_tma_box(int nu, int *cols, int *rows) {
    *cols = kTX + 2 * round_up(2 * nu + 4, 4);
    *rows = 64 + 2 * (2 * nu + 2);
}

cudaError_t launch_down_tma(const float *x, float *xout, const float *b, int n, int nu, bool zero_init, float *bc,
                            const CUtensorMap *tmx, const CUtensorMap *tmb, int *err, cudaStream_t s) {
    if (nu != 2 || n < 128 || x == xout || !tmb || !err) return cudaErrorInvalidValue;
    using Cfg = DownCfg<float, 2, 64>;
    const size_t smem = Cfg::smem + 16;
    auto k = zero_init ? k_down_tma<2, true> : k_down_tma<2, false>;
    static std::atomic<unsigned> done0{0}, done1{0};
    cudaError_t e = set_smem_once(k, smem, zero_init ? done1 : done0);
    if (e != cudaSuccess) return e;
    const CUtensorMap &mx = tmx ? *tmx : *tmb;  // x is not read with zero_init
    e = launch_kernel(k, dim3(n / kTX, n / 64), kThreads, smem, s, mx, *tmb, x, xout, b, n, bc, err);
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_up(const T *x, T *xout, const T *b, const T *ec, int n, int nu,
                      const FirTaps &taps, cudaStream_t s, const T *extra, int variant, const int *extra_flag,
                      const T *xr) {
    if (n < 64 || !ec || x == xout || variant < -1 || variant >= kTileVariants) return cudaErrorInvalidValue;
    if (xr && !std::is_same<T, double>::value) return cudaErrorInvalidValue;  // FP64 tiles only
    if (variant < 0) variant = tile_variant(1, n, nu);
    switch (nu) {
        case 0: return up_var<T, 0>(x, xout, b, ec, extra, extra_flag, n, taps, s, variant, xr);
        case 1: return up_var<T, 1>(x, xout, b, ec, extra, extra_flag, n, taps, s, variant, xr);
        case 2: return up_var<T, 2>(x, xout, b, ec, extra, extra_flag, n, taps, s, variant, xr);
        case 3: return up_var<T, 3>(x, xout, b, ec, extra, extra_flag, n, taps, s, variant, xr);
        case 4: return up_var<T, 4>(x, xout, b, ec, extra, extra_flag, n, taps, s, variant, xr);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_refine_rows(const double *ec, double *xr, int n, const FirTaps &taps, cudaStream_t s) {
    if (n < 2 * kRefineJ || (n & (n - 1)) || !ec || !xr) return cudaErrorInvalidValue;
    const cudaError_t e =
        launch_kernel(k_refine_rows<double>, dim3((n / 2) / kRefineJ, n / 2), kRefineJ, 0, s, ec, xr, n, taps);
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bottom(T *x, const T *b, int n, int coarsest, int nu1, int nu2, bool zero_init,
                          const T *ainv, const FirTaps &taps, cudaStream_t s) {
    if (n > bottom_max<T>() || coarsest < 4 || coarsest > n) return cudaErrorInvalidValue;
    int nlev = 0;
    for (int m = n; m >= coarsest; m >>= 1) ++nlev;
    if ((n >> (nlev - 1)) != coarsest || nlev > 8) return cudaErrorInvalidValue;
    const size_t smem = bottom_smem_elems(n, nlev) * sizeof(T);
    auto k = k_bottom<T>;
    static std::atomic<unsigned> done{0};
    cudaError_t e = set_smem_once(k, bottom_smem_max() * sizeof(T), done);
    if (e != cudaSuccess) return e;
    {
        cudaError_t le_ = launch_kernel(k, 1, kBottomThreads, smem, s,
                                        x, b, n, nlev, nu1, nu2, zero_init ? 1 : 0, ainv, taps);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_coarse_cluster(float *x, float *t, const float *b, float *xb, float *bb, int coarsest, int nu1,
                                  int nu2, const float *ainv, const FirTaps &taps, cudaStream_t s) {
    if (nu1 != 2 || nu2 != 2 || coarsest < 4 || coarsest > kCoarseN / 2) return cudaErrorInvalidValue;
    int nlev = 0;
    for (int m = kCoarseN / 2; m >= coarsest; m >>= 1) ++nlev;
    if (((kCoarseN / 2) >> (nlev - 1)) != coarsest || nlev > 8) return cudaErrorInvalidValue;
    size_t smem = bottom_smem_max() * sizeof(float);
    smem = std::max(smem, DownCfg<float, 2, 32>::smem);
    smem = std::max(smem, UpCfg<float, 2, 32, 2>::smem);
    auto k = k_coarse_cluster<2, 2>;
    static std::atomic<unsigned> done{0};
    cudaError_t e = set_smem_once(k, smem, done);
    if (e != cudaSuccess) return e;
    e = launch_kernel(k, kCoarseCTAs, kBottomThreads, smem, s, x, t, b, xb, bb, nlev, ainv, taps);
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_down<float>(const float *, float *, const float *, int, int, bool, float *,
                                        cudaStream_t, int);
template cudaError_t launch_down<double>(const double *, double *, const double *, int, int, bool,
                                         double *, cudaStream_t, int);
template cudaError_t launch_up<float>(const float *, float *, const float *, const float *, int, int,
                                      const FirTaps &, cudaStream_t, const float *, int, const int *,
                                      const float *);
template cudaError_t launch_up<double>(const double *, double *, const double *, const double *, int,
                                       int, const FirTaps &, cudaStream_t, const double *, int, const int *,
                                       const double *);
template cudaError_t launch_bottom<float>(float *, const float *, int, int, int, int, bool, const float *,
                                          const FirTaps &, cudaStream_t);
template cudaError_t launch_bottom<double>(double *, const double *, int, int, int, int, bool,
                                           const double *, const FirTaps &, cudaStream_t);

cudaError_t launch_sum(const double *x, int n, Reduction red, cudaStream_t s, const double *alt, const int *par,
                       bool zero_first) {
    if ((par && !alt) || (zero_first && !par)) return cudaErrorInvalidValue;
    {
        const size_t N = (size_t)n * n;
        const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(alt)) & 15) == 0 && N % 4 == 0;
        const double *alt_k = alt ? alt : x;
        const int zf = zero_first ? 1 : 0;
        cudaError_t le_ = vec ? launch_kernel(k_sum_v, kWideBlocks, kRedThreads, 0, s, x, N, red, alt_k, par, zf)
                              : launch_kernel(k_sum, kRedBlocks, kRedThreads, 0, s, x, N, red, alt_k, par, zf);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_source_sum(const double *f, int n, Reduction red, cudaStream_t s) {
    return launch_sum(f, n, red, s, nullptr, nullptr, false);
}
cudaError_t launch_scaled_rhs(const double *f, int n, double h2, const double *f_sum, double *b,
                              cudaStream_t s) {
    {
        cudaError_t le_ = launch_kernel(k_scaled_rhs, kRedBlocks, kRedThreads, 0, s,
                                        f, n, h2, f_sum, b);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}
namespace {
template <bool WRITE32, bool FNORM, int BMODE>
cudaError_t outer_residual_impl(const double *f, const double *x, int n, double h2, const double *mu_sum,
                                double mu_host, float *s32, double *bsc, Reduction red, cudaStream_t s) {
    return launch_kernel(k_outer_residual<WRITE32, FNORM, BMODE>, kRedBlocks, kRedThreads, 0, s, f, x, n, h2,
                         mu_sum, mu_host, s32, bsc, red);
}
template <bool WRITE32>
cudaError_t outer_residual_w(const double *f, const double *x, int n, double h2, const double *mu_sum,
                             double mu_host, float *s32, bool want_fnorm, double *bsc, bool load_b, Reduction red,
                             cudaStream_t s) {
    if (load_b) return outer_residual_impl<WRITE32, false, 2>(f, x, n, h2, mu_sum, mu_host, s32, bsc, red, s);
    if (want_fnorm)
        return bsc ? outer_residual_impl<WRITE32, true, 1>(f, x, n, h2, mu_sum, mu_host, s32, bsc, red, s)
                   : outer_residual_impl<WRITE32, true, 0>(f, x, n, h2, mu_sum, mu_host, s32, bsc, red, s);
    return bsc ? outer_residual_impl<WRITE32, false, 1>(f, x, n, h2, mu_sum, mu_host, s32, bsc, red, s)
               : outer_residual_impl<WRITE32, false, 0>(f, x, n, h2, mu_sum, mu_host, s32, bsc, red, s);
}
}  // namespace

cudaError_t launch_outer_residual(const double *f, const double *x, int n, double h2,
                                  const double *mu_sum, double mu_host, float *s32,
                                  bool want_fnorm, double *bsc, bool load_b, Reduction red, cudaStream_t s) {
    if (load_b && (!bsc || want_fnorm)) return cudaErrorInvalidValue;
    const cudaError_t e = s32 ? outer_residual_w<true>(f, x, n, h2, mu_sum, mu_host, s32, want_fnorm, bsc, load_b, red, s)
                              : outer_residual_w<false>(f, x, n, h2, mu_sum, mu_host, s32, want_fnorm, bsc, load_b, red, s);
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_outer_residual_tasks(const double *f, const double *x, int n, double h2, const double *mu_sum,
                                        double mu_host, float *s32, bool first, long long *bint, int *ebt,
                                        Reduction red, cudaStream_t s, bool xzero) {
    if (n < kResMinN || !s32 || !bint || !ebt || (xzero && !first)) return cudaErrorInvalidValue;
    const cudaError_t e =
        first ? launch_kernel(k_outer_residual_t<true>, kRedBlocks, kRedThreads, 0, s, f, x, n, h2, mu_sum, mu_host,
                              s32, bint, ebt, red, xzero ? 1 : 0)
              : launch_kernel(k_outer_residual_t<false>, kResBlocks, kRedThreads, 0, s, f, x, n, h2, mu_sum, mu_host,
                              s32, bint, ebt, red, 0);
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_update_residual_tasks(double *xa, double *xb, const int *step_dev, int step_host, bool zero_first,
                                         const float *e, int n, double h2, float *s32, long long *bint, int *ebt,
                                         Reduction red, cudaStream_t s) {
    if (n < kResMinN || !xa || !xb || xa == xb || !e || !s32 || !bint || !ebt || step_host < 0)
        return cudaErrorInvalidValue;
    const cudaError_t le = launch_kernel(k_update_residual_t, kResBlocks, kRedThreads, 0, s, xa, xb, step_dev,
                                         step_host, zero_first ? 1 : 0, e, n, h2, s32, bint, ebt, red);
    if (le != cudaSuccess) return le;
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_bspline_coef(const float *e, float *c, int nc, int dir, cudaStream_t s) {
    if (nc < 4 || (dir != 0 && dir != 1) || e == c) return cudaErrorInvalidValue;
    BspTaps t;
    const double z = 1.7320508075688772 - 2.0;  // sqrt(3) - 2, the B-spline filter's pole
    double a = 1.7320508075688772;
    for (int k = 0; k <= kBspTaps; ++k, a *= z) t.a[k] = (float)a;
    const int blocks = (nc * nc + kRedThreads - 1) / kRedThreads;
    {
        cudaError_t le_ = launch_kernel(k_bspline_coef, blocks < kRedBlocks ? blocks : kRedBlocks, kRedThreads, 0, s,
                                        e, c, nc, dir, t);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_prolong_factor(float *ef, const float *c, int n, int lgf, cudaStream_t s) {
    if (lgf < 1 || (n >> lgf) < 4) return cudaErrorInvalidValue;
    {
        cudaError_t le_ = launch_kernel(k_prolong_factor, kWideBlocks, kRedThreads, 0, s, ef, c, n, lgf);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_convert(int dir, size_t count, const void *in, void *out, cudaStream_t s) {
    {
        cudaError_t le_ = launch_kernel(k_convert, kRedBlocks, kRedThreads, 0, s,
                                        dir, count, in, out);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_update(double *x, const float *e, int n, Reduction red, cudaStream_t s) {
    const size_t N = (size_t)n * n;
    const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(e)) & 15u) == 0 && (N & 3u) == 0;
    {
        cudaError_t le_ = vec ? launch_kernel(k_update_v, kWideBlocks, kRedThreads, 0, s, x, e, N, red)
                              : launch_kernel(k_update, kRedBlocks, kRedThreads, 0, s, x, e, N, red);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_project(double *x, int n, const double *sum, cudaStream_t s, const int *zero_flag,
                           const double *alt, const int *par, bool zero_first) {
    if ((par && !alt) || (zero_first && !par)) return cudaErrorInvalidValue;
    {
        const size_t N = (size_t)n * n;
        const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(alt)) & 15) == 0 && N % 4 == 0;
        const double *alt_k = alt ? alt : x;
        const int zf = zero_first ? 1 : 0;
        cudaError_t le_ = vec ? launch_kernel(k_project_v, kWideBlocks, kRedThreads, 0, s, x, N, sum, zero_flag,
                                              alt_k, par, zf)
                              : launch_kernel(k_project, kRedBlocks, kRedThreads, 0, s, x, N, sum, zero_flag,
                                              alt_k, par, zf);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_check(DevState *st, const double *rsum, const double *usum, const double *fsum,
                         double n2, double h2, double tol, int step, int max_cycles, bool first,
                         cudaGraphConditionalHandle handle, cudaStream_t s, double rho, CycleHandles ifh) {
    {
        cudaError_t le_ = launch_kernel(k_check, 1, 32, 0, s,
                                        st, rsum, usum, fsum, n2, h2, tol, step, max_cycles, first ? 1 : 0, handle,
                                        rho, ifh);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}

namespace {
template <int NU, int TY>
cudaError_t down_batched_impl(const TileGrid *tab, int ngrid, int nblocks, const int *active, cudaStream_t s) {
    auto k = k_down_batched<float, NU, TY>;
    static std::atomic<unsigned> done{0};
    cudaError_t e = set_smem_once(k, DownCfg<float, NU, TY>::smem, done);
    if (e != cudaSuccess) return e;
    {
        cudaError_t le_ = launch_kernel(k, nblocks, kThreads, DownCfg<float, NU, TY>::smem, s,
                                        tab, ngrid, active);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}
template <int NU, int TY, int NJ>
cudaError_t up_batched_impl(const TileGrid *tab, int ngrid, int nblocks, const int *active, const FirTaps &taps,
                            cudaStream_t s) {
    auto k = k_up_batched<float, NU, TY, NJ>;
    static std::atomic<unsigned> done{0};
    cudaError_t e = set_smem_once(k, UpCfg<float, NU, TY, NJ>::smem, done);
    if (e != cudaSuccess) return e;
    {
        cudaError_t le_ = launch_kernel(k, nblocks, kThreads, UpCfg<float, NU, TY, NJ>::smem, s,
                                        tab, ngrid, active, taps);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}
template <int NU>
cudaError_t down_batched_var(const TileGrid *tab, int ngrid, int nblocks, const int *active, cudaStream_t s,
                             int variant) {
    switch (variant_rows(variant)) {
        case 8: return down_batched_impl<NU, 8>(tab, ngrid, nblocks, active, s);
        case 16: return down_batched_impl<NU, 16>(tab, ngrid, nblocks, active, s);
        case 32: return down_batched_impl<NU, 32>(tab, ngrid, nblocks, active, s);
        default: return down_batched_impl<NU, 64>(tab, ngrid, nblocks, active, s);
    }
}
template <int NU>
cudaError_t up_batched_var(const TileGrid *tab, int ngrid, int nblocks, const int *active, const FirTaps &taps,
                           cudaStream_t s, int variant) {
    const bool nj2 = variant_runs(variant) == 2;
    switch (variant_rows(variant)) {
        case 8: return nj2 ? up_batched_impl<NU, 8, 2>(tab, ngrid, nblocks, active, taps, s)
                           : up_batched_impl<NU, 8, 1>(tab, ngrid, nblocks, active, taps, s);
        case 16: return nj2 ? up_batched_impl<NU, 16, 2>(tab, ngrid, nblocks, active, taps, s)
                            : up_batched_impl<NU, 16, 1>(tab, ngrid, nblocks, active, taps, s);
        case 32: return nj2 ? up_batched_impl<NU, 32, 2>(tab, ngrid, nblocks, active, taps, s)
                            : up_batched_impl<NU, 32, 1>(tab, ngrid, nblocks, active, taps, s);
        default: return nj2 ? up_batched_impl<NU, 64, 2>(tab, ngrid, nblocks, active, taps, s)
                            : up_batched_impl<NU, 64, 1>(tab, ngrid, nblocks, active, taps, s);
    }
}
}  // namespace

cudaError_t launch_down_batched(const TileGrid *tab, int ngrid, int nblocks, int nu, const int *active,
                                cudaStream_t s, int variant) {
    if (variant < 0 || variant >= kTileVariants) return cudaErrorInvalidValue;
    switch (nu) {
        case 0: return down_batched_var<0>(tab, ngrid, nblocks, active, s, variant);
        case 1: return down_batched_var<1>(tab, ngrid, nblocks, active, s, variant);
        case 2: return down_batched_var<2>(tab, ngrid, nblocks, active, s, variant);
        case 3: return down_batched_var<3>(tab, ngrid, nblocks, active, s, variant);
        case 4: return down_batched_var<4>(tab, ngrid, nblocks, active, s, variant);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_up_batched(const TileGrid *tab, int ngrid, int nblocks, int nu, const int *active,
                              const FirTaps &taps, cudaStream_t s, int variant) {
    if (variant < 0 || variant >= kTileVariants) return cudaErrorInvalidValue;
    switch (nu) {
        case 0: return up_batched_var<0>(tab, ngrid, nblocks, active, taps, s, variant);
        case 1: return up_batched_var<1>(tab, ngrid, nblocks, active, taps, s, variant);
        case 2: return up_batched_var<2>(tab, ngrid, nblocks, active, taps, s, variant);
        case 3: return up_batched_var<3>(tab, ngrid, nblocks, active, taps, s, variant);
        case 4: return up_batched_var<4>(tab, ngrid, nblocks, active, taps, s, variant);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_bottom_batched(const BottomGrid *tab, int ngrid, int nu1, int nu2, const int *active,
                                  const FirTaps &taps, cudaStream_t s) {
    const size_t bytes = bottom_smem_max() * sizeof(float);  // every grid of the table fits
    static std::atomic<unsigned> done{0};
    cudaError_t e = set_smem_once(k_bottom_batched<float>, bytes, done);
    if (e != cudaSuccess) return e;
    {
        cudaError_t le_ = launch_kernel(k_bottom_batched<float>, ngrid, kBottomThreads, bytes, s,
                                        tab, nu1, nu2, active, taps);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sum_batched(const RhsDesc *rd, int nrhs, int nblocks, bool of_x, BatchRed red, cudaStream_t s,
                               const DevState *st) {
    if (of_x)
        {
            cudaError_t le_ = launch_kernel(k_sum_b<true>, nblocks, kRedThreads, 0, s,
                                            rd, nrhs, red, st);
            if (le_ != cudaSuccess) return le_;
        }
    else
        {
            cudaError_t le_ = launch_kernel(k_sum_b<false>, nblocks, kRedThreads, 0, s,
                                            rd, nrhs, red, (const DevState *)nullptr);
            if (le_ != cudaSuccess) return le_;
        }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_outer_residual_batched(const RhsDesc *rd, int nrhs, int nblocks, const double *fsum,
                                          bool want_fnorm, bool first_all, const int *active, BatchRed red,
                                          cudaStream_t s) {
    const int fa = first_all ? 1 : 0;
    if (want_fnorm)
        {
            cudaError_t le_ = launch_kernel(k_outer_residual_b<true>, nblocks, kRedThreads, 0, s,
                                            rd, nrhs, fsum, fa, active, red);
            if (le_ != cudaSuccess) return le_;
        }
    else
        {
            cudaError_t le_ = launch_kernel(k_outer_residual_b<false>, nblocks, kRedThreads, 0, s,
                                            rd, nrhs, fsum, fa, active, red);
            if (le_ != cudaSuccess) return le_;
        }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_update_batched(const RhsDesc *rd, int nrhs, int nblocks, const int *active, BatchRed red,
                                  cudaStream_t s) {
    {
        cudaError_t le_ = launch_kernel(k_update_b, nblocks, kRedThreads, 0, s,
                                        rd, nrhs, active, red);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_project_batched(const RhsDesc *rd, int nrhs, int nblocks, const double *xsum,
                                   const DevState *st, cudaStream_t s, bool fused) {
    {
        cudaError_t le_ = launch_kernel(k_project_b, nblocks, kRedThreads, 0, s,
                                        rd, nrhs, xsum, st, fused ? 1 : 0);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_update_residual_batched(const RhsDesc *rd, int nrhs, int nblocks, const DevState *st,
                                           const int *active, BatchRed red, cudaStream_t s) {
    if (!st) return cudaErrorInvalidValue;
    const cudaError_t e = launch_kernel(k_update_residual_b, nblocks, kRedThreads, 0, s, rd, nrhs, st, active, red);
    if (e != cudaSuccess) return e;
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_policy(DevState *st, int k, ProlongPolicy p, int *flag, cudaGraphConditionalHandle handle,
                          cudaStream_t s) {
    {
        cudaError_t le_ = launch_kernel(k_policy, 1, 32, 0, s, st, k, p, flag, handle);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_check_batched(DevState *st, const RhsDesc *rd, int nrhs, const double *rsum,
                                 const double *usum, const double *fsum, double tol, int step, int max_cycles,
                                 bool first, int *active, cudaGraphConditionalHandle handle, bool use_handle,
                                 cudaStream_t s, double rho, CycleHandles ifh, int *batch_m) {
    {
        cudaError_t le_ = launch_kernel(k_check_b, 1, 256, 0, s,
                                        st, rd, nrhs, rsum, usum, fsum, tol, step, max_cycles, first ? 1 : 0, active, handle, use_handle ? 1 : 0,
                                        rho, ifh, batch_m);
        if (le_ != cudaSuccess) return le_;
    }
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, int NU, int TY, int NJ>
static cudaError_t prepare_shape() {
    cudaError_t e = set_smem(k_down<T, NU, true, TY>, DownCfg<T, NU, TY>::smem);
    if (e == cudaSuccess) e = set_smem(k_down<T, NU, false, TY>, DownCfg<T, NU, TY>::smem);
    if (e == cudaSuccess) e = set_smem(k_up<T, NU, TY, NJ>, UpCfg<T, NU, TY, NJ>::smem);
    return e;
}

template <typename T, int NU>
static cudaError_t prepare_nu() {
    if constexpr (std::is_same<T, double>::value) {
        return prepare_shape<T, NU, Fixed64<double>::TY, Fixed64<double>::NJ>();
    } else {
        cudaError_t e = cudaSuccess;
        for (int v = 0; v < kTileVariants && e == cudaSuccess; ++v) {
            const int nj = variant_runs(v);
            switch (variant_rows(v)) {
                case 8: e = nj == 2 ? prepare_shape<T, NU, 8, 2>() : prepare_shape<T, NU, 8, 1>(); break;
                case 16: e = nj == 2 ? prepare_shape<T, NU, 16, 2>() : prepare_shape<T, NU, 16, 1>(); break;
                case 32: e = nj == 2 ? prepare_shape<T, NU, 32, 2>() : prepare_shape<T, NU, 32, 1>(); break;
                default: e = nj == 2 ? prepare_shape<T, NU, 64, 2>() : prepare_shape<T, NU, 64, 1>(); break;
            }
        }
        return e;
    }
}

template <typename T>
static cudaError_t prepare_type() {
    cudaError_t e = prepare_nu<T, 0>();
    if (e == cudaSuccess) e = prepare_nu<T, 1>();
    if (e == cudaSuccess) e = prepare_nu<T, 2>();
    if (e == cudaSuccess) e = prepare_nu<T, 3>();
    if (e == cudaSuccess) e = prepare_nu<T, 4>();
    // the bottom kernel's largest configuration
    if (e == cudaSuccess) e = set_smem(k_bottom<T>, bottom_smem_max() * sizeof(T));
    return e;
}

cudaError_t prepare_kernels() {
    cudaError_t e = prepare_type<float>();
    if (e == cudaSuccess) e = prepare_type<double>();
    return e;
}

}  // namespace mg
