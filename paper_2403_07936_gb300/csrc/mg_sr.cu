// mg_sr.cu - super-resolution prolongation: weight loading and generator
// kernels (Sec. 2.3, Fig. 1b; Sec. 3.1; Appendix A, Algorithm 5).
//
// The 64 -> 64 and 64 -> 256 convolutions run as implicit GEMMs on the
// tcgen05 tensor cores (BF16 operands, FP32 accumulation in tensor memory):
// for an output tile of 128 pixels of one row, D[pixel][co] = sum over the 9
// taps (dy, dx) and 64 input channels of In[row y+dy][pixel+dx][ci] *
// W[tap][co][ci].  A persistent block walks a vertical strip of rows: each
// input row is TMA-loaded once into a ring of six row slots and multiplied by
// the three dy taps at once (N = 192), accumulating into the TMEM slots of
// the three output rows it feeds (k_conv_tc below).  A staged row is stored
// as eight 8-channel planes of [pixel][8 channels] (no swizzle), so the
// x-shifted tap operands are descriptors offset by 16 * dx bytes into the
// staged row; the weights use the 128-byte swizzled K-major layout.  One
// warp issues the TMA loads, one thread the MMAs, and eight warps drain the
// finished accumulators (lane quarter x column half), and the bf16 results
// leave through a shared-memory stage and TMA stores.  Every wait on an mbarrier is bounded by a
// wall-clock limit and reports MG_ERR_TIMEOUT through a device flag.
// The 1 -> 64 and 64 -> 1 layers are too thin for tensor cores (K = 9 and
// N = 1) and run on the CUDA cores.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "mg_internal.cuh"
#include "mg_sr.cuh"
#include "mg_tc.cuh"

namespace mg {

namespace {

constexpr int C = kSrFeat;            // channels
constexpr int TM = 128;               // pixels per tile (one row segment)
constexpr int ROWPX = TM + 2;         // staged pixels per input row
constexpr int ROWBYTES = ROWPX * C * 2;
// one 8-channel plane of a staged row, [pixel][8 ch] (130 x 16 bytes), padded
// to a 128-byte multiple so that every TMA destination is 128-byte aligned
constexpr int PLANE = 2176;
constexpr int ROWSLOT = 8 * PLANE;    // 17 KiB slots, 1024-byte multiple
static_assert(PLANE >= ROWPX * 16 && PLANE % 128 == 0, "plane pitch");
constexpr int NSLOT = 4;              // ring of staged input rows (prefetch up to 4 rows ahead)
constexpr int WBYTES = 9 * C * C * 2;  // one layer's weights, 72 KiB
constexpr int TAPBYTES = C * C * 2;    // one tap: 64 rows (co) x 128 bytes (ci)
constexpr int DXBYTES = 3 * TAPBYTES;  // the three dy taps of one dx, 192 rows (dy, co) x 128 bytes
constexpr int TSLOTS = 8;              // 64-column FP32 accumulators in TMEM (one per output row)
constexpr int TMEM_COLS = TSLOTS * C;  // all 512 columns
// warp roles: 0 = TMA producer, 1 = MMA issuer, 2..9 = epilogue (lane quarter
// warp % 4, column half (warp - 2) / 4 of the 128 x 64 accumulator)
constexpr int EPI_WARPS = 8;
constexpr int CONV_THREADS = 32 * (2 + EPI_WARPS);
constexpr int STAGE = TM * C * 2;     // one output tile, 128 px x 128 B (epilogue staging)
constexpr int SKIPBUF = 3;            // residual-input tiles in flight (rows o .. o + 2)
// weights, row full / empty, accumulator full / empty, accumulators zeroed, MMAs done, skip tiles
constexpr int NBARS = 1 + 2 * NSLOT + 2 * TSLOTS + 1 + 1 + SKIPBUF;
constexpr int BAR_AREA = 512;
constexpr size_t CONV_SMEM =
    1024 + WBYTES + NSLOT * ROWSLOT + (2 + SKIPBUF) * STAGE + BAR_AREA + 2 * C * sizeof(float);
static_assert(NBARS * 8 + 16 <= BAR_AREA, "barrier area");
static_assert(CONV_SMEM <= 232448, "shared memory per block");

enum { MODE_PRELU = 0, MODE_RESID = 1, MODE_SHUFFLE = 2 };

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0,
                                            int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6, %7}], [%2];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];"
        ::"l"(map), "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, const void *src, int c0, int c1, int c2,
                                             int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];"
        ::"l"(map), "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Shared-memory matrix descriptors (K-major operands).
// B (weights): 128-byte swizzle, rows of 128 bytes, 8-row groups 1024 bytes
// apart, start on a 1024-byte boundary plus the 32-byte step of the K slice.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused when swizzled)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}
// A (activations): no swizzle, core matrices of 8 pixels x 16 bytes.  A staged
// row is 8 planes (one per 8 channels) of [pixel][8 ch]; consecutive pixels
// are 16 bytes apart, so 8-pixel core matrices are 128 bytes apart (stride
// offset) and the next 8 channels are one plane further (leading offset).  A
// view shifted by dx pixels simply starts 16 * dx bytes later.
__device__ __forceinline__ uint64_t sdesc_planes(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);   // start address
    d |= (uint64_t)(PLANE >> 4) << 16;          // leading byte offset: next 8 channels
    d |= (uint64_t)(128 >> 4) << 32;            // stride byte offset: next 8 pixels
    d |= (uint64_t)1 << 46;                     // descriptor version
    return d;                                   // layout type 0: no swizzle
}

// 32 lanes x 32 columns of zeros (the accumulator slot is reset for its next row).
__device__ __forceinline__ void tmem_zero32(uint32_t taddr) {
    const uint32_t z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
        "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};"
        ::"r"(taddr), "r"(z)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// Barrier `id` over `count` threads (the epilogue warps) returning the AND of
// every participant's predicate: a decision all of them take together.
__device__ __forceinline__ bool epi_bar_and(bool pred, int id, int count) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void epi_bar(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Store one pixel's 64 bf16 channels (8 x 16 bytes) at (y, x) of a padded
// H x W grid, and at every halo position that wraps onto it.
// With halo_only, the interior position is skipped.
__device__ __forceinline__ void store_px(__nv_bfloat16 *out, int H, int W, int y, int x, const uint4 *d,
                                         bool halo_only = false) {
    const int rows[2] = {y + 1, y == 0 ? H + 1 : (y == H - 1 ? 0 : -1)};
    const int cols[2] = {x + 1, x == 0 ? W + 1 : (x == W - 1 ? 0 : -1)};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        if (rows[a] < 0) continue;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            if (cols[b] < 0 || (halo_only && a == 0 && b == 0)) continue;
            uint4 *p = reinterpret_cast<uint4 *>(out + ((size_t)rows[a] * (W + 2) + cols[b]) * C);
#pragma unroll
            for (int i = 0; i < 8; ++i) p[i] = d[i];
        }
    }
}

// Store channels [32 half, 32 half + 32) of one pixel (4 x 16 bytes) at (y, x)
// of a padded H x W grid and at the halo positions that wrap onto it.  With
// halo_only, the interior position and the halo-row copy in the pixel's own
// column are skipped (the tile's TMA stores write those).
__device__ __forceinline__ void store_half_px(__nv_bfloat16 *out, int H, int W, int y, int x, int half,
                                              const uint4 *d, bool halo_only) {
    const int rows[2] = {y + 1, y == 0 ? H + 1 : (y == H - 1 ? 0 : -1)};
    const int cols[2] = {x + 1, x == 0 ? W + 1 : (x == W - 1 ? 0 : -1)};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        if (rows[a] < 0) continue;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            if (cols[b] < 0 || (halo_only && b == 0)) continue;
            uint4 *p = reinterpret_cast<uint4 *>(out + ((size_t)rows[a] * (W + 2) + cols[b]) * C + half * 32);
#pragma unroll
            for (int i = 0; i < 4; ++i) p[i] = d[i];
        }
    }
}

struct ConvArgs {
    const __nv_bfloat16 *skip;  // MODE_RESID: residual input (padded), else null
    __nv_bfloat16 *out;         // padded output (coarse, or fine for MODE_SHUFFLE)
    const float *bias;          // [groups][64]
    const float *prelu;         // [64] (MODE_PRELU, MODE_SHUFFLE)
    int H, W;                   // coarse grid; W a multiple of 128
    int layer;                  // weight layer of group 0
    int chunks;                 // row chunks per (group, column block) strip
    int rows_per_chunk;
    int *err;
    int imgs = 1;               // images stacked along y, each with its own halo
    int mosaic = 0;             // > 0: pixels with y or x = mosaic - 1 (mod mosaic) are window
                                // separators and their outputs are forced to zero
};

// ---------------------------------------------------------------------------
// k_conv_tc: persistent implicit-GEMM 3x3 convolution, 64 -> 64 channels per
// group, on tcgen05.  Block b handles strip b / chunks = (image, group,
// column block) and rows [chunk * rows_per_chunk, ...) of it.  A batch of
// equal-size images is stacked along y, each padded image (H + 2 rows, or
// 2H + 2 for the shuffle layer's output) after the previous one.
//
// The block walks its input rows once.  Input row i (padded row y_a + i)
// feeds output rows i, i - 1 and i - 2 through the taps dy = 0, 1, 2, so for
// each dx and each 16-channel slice one MMA with N = 192 multiplies the
// row's x-shifted pixels by the three dy taps' weights side by side (the
// weights are staged [dx][dy][co][ci]) into the accumulators of those three
// output rows, which sit side by side in TMEM: output row o owns the 64
// columns of slot (-o) mod 8, so rows i, i - 1, i - 2 own slots s, s + 1,
// s + 2.  Where that run wraps past slot 7 (two input rows of eight) the MMA
// splits into N = 128 + 64 or 64 + 128.  12 to 24 MMAs per input row instead
// of 36 of N = 64.  The epilogue drains a slot once its row's last input
// (dy = 2) is in, writes zeros back (every MMA accumulates: splitting off the
// first product of each row to overwrite its slot costs one more MMA per
// input row, which measured slower than the zero stores) and frees it; the
// two rows before the block's first output row (o = -2, -1) only collect
// partial sums and are drained without a store.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(CONV_THREADS, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_w,
              const __grid_constant__ CUtensorMap tm_out, const __grid_constant__ CUtensorMap tm_skip, ConvArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *wsm = sm;
    unsigned char *rows = sm + WBYTES;
    unsigned char *stage = rows + NSLOT * ROWSLOT;  // 2 x STAGE, 1024-byte aligned
    unsigned char *skipbuf = stage + 2 * STAGE;     // SKIPBUF x STAGE (residual layer)
    uint64_t *bars = reinterpret_cast<uint64_t *>(skipbuf + SKIPBUF * STAGE);
    uint64_t *wbar = bars, *full = bars + 1, *empty = full + NSLOT;
    uint64_t *tfull = empty + NSLOT, *tempty = tfull + TSLOTS, *tzero = tempty + TSLOTS, *mdone = tzero + 1;
    uint64_t *skipbar = mdone + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + NBARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + NBARS) + 1;
    float *s_bias = reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(bars) + BAR_AREA);  // [64] bias
    float *s_prelu = s_bias + C;                                                                     // [64] slopes

    const int NB = a.W / TM;
    const int strip = blockIdx.x / a.chunks, chunk = blockIdx.x - strip * a.chunks;
    const int per_img = (MODE == MODE_SHUFFLE ? 4 : 1) * NB;
    const int img = strip / per_img, gs = strip - img * per_img;
    const int g = gs / NB, cb = gs - g * NB;
    const int yin0 = img * (a.H + 2);  // first padded row of this image in the stacked input
    const size_t in_img = (size_t)img * (a.H + 2) * (a.W + 2) * C;
    const size_t out_img = MODE == MODE_SHUFFLE ? (size_t)img * (2 * a.H + 2) * (2 * a.W + 2) * C : in_img;
    const int y_a = chunk * a.rows_per_chunk;
    const int y_b = min(a.H, y_a + a.rows_per_chunk);
    if (y_a >= y_b) return;  // uniform across the block, before any barrier or TMEM use
    const int T = y_b - y_a;  // output rows; input rows y_a .. y_b + 1 (padded), i = 0 .. T + 1
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        mbar_init(wbar, 1);
        for (int s2 = 0; s2 < NSLOT; ++s2) {
            mbar_init(&full[s2], 1);
            mbar_init(&empty[s2], 1);
        }
        for (int b = 0; b < TSLOTS; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], EPI_WARPS);
        }
        mbar_init(tzero, EPI_WARPS);
        mbar_init(mdone, 1);
        for (int k = 0; k < SKIPBUF; ++k) mbar_init(&skipbar[k], 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tmem_slot, TMEM_COLS);
    if (threadIdx.x < C) {
        s_bias[threadIdx.x] = a.bias[g * C + threadIdx.x];
        s_prelu[threadIdx.x] = a.prelu ? a.prelu[threadIdx.x] : 0.f;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- producer: the weights ([dx][dy][co][ci]), then the ring of input rows
        if (lane == 0) {
            mbar_expect_tx(wbar, WBYTES);
            for (int dx = 0; dx < 3; ++dx) tma_load_5d(wsm + dx * DXBYTES, &tm_w, wbar, 0, 0, dx, 0, a.layer + g);
            int issued = 0;
            for (int i = 0; i < T + 2; ++i) {  // relative input row i = padded row y_a + i
                const int slot = i % NSLOT;
                if (i >= NSLOT && !mbar_wait(&empty[slot], ((i / NSLOT) - 1) & 1)) {
                    *abort_flag = 1;
                    break;
                }
                if (*abort_flag) break;
                mbar_expect_tx(&full[slot], ROWBYTES);
                for (int q = 0; q < 8; ++q)
                    tma_load_3d(rows + slot * ROWSLOT + q * PLANE, &tm_in, &full[slot], 8 * q, cb * TM, yin0 + y_a + i);
                issued = i + 1;
            }
            if (*abort_flag) {
                // wait (bounded) for the last load issued into each slot and the
                // weights, so no copy still writes this block's shared memory
                for (int i = issued - 1; i >= 0 && i >= issued - NSLOT; --i)
                    mbar_wait(&full[i % NSLOT], (i / NSLOT) & 1);
                mbar_wait(wbar, 0);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer ---------------------------------------------------------
        // Descriptors are formed once: every operand is a fixed byte offset from
        // the weight base or from the staged row, and the start address field of
        // a descriptor is that address / 16 (no carry: shared addresses stay
        // below 2^18), so each MMA costs two 64-bit adds.
        if (lane == 0) {
            bool ok = mbar_wait(tzero, 0) && mbar_wait(wbar, 0);
            const uint32_t rbase = smem_u32(rows);
            const uint64_t bd0 = sdesc_sw128(smem_u32(wsm));
            int si = 0;  // ring slot of input row i
            int i = 0;
            for (; ok && i < T + 2; ++i) {
                const int ts = (-i) & (TSLOTS - 1);  // accumulator slot of output row i
                // the slot's previous row (i - 8) must be drained and zeroed
                if (i >= TSLOTS - 2) ok = mbar_wait(&tempty[ts], ((i - (TSLOTS - 2)) >> 3) & 1);
                if (ok) ok = mbar_wait(&full[si], (i / NSLOT) & 1);
                if (!ok || *abort_flag) break;
                tc_fence_after();
                const uint64_t ad0 = sdesc_planes(rbase + (uint32_t)(si * ROWSLOT));
                const uint32_t d = tmem + (uint32_t)(ts * C);
#pragma unroll
                for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ad = ad0 + (uint64_t)(kk * (2 * PLANE / 16) + dx);
                        const uint64_t bd = bd0 + (uint64_t)(dx * (DXBYTES / 16) + kk * 2);
                        constexpr uint64_t B1 = TAPBYTES / 16, B2 = 2 * TAPBYTES / 16;  // dy = 1, 2 rows of B
                        if (ts <= TSLOTS - 3) {
                            mma_bf16<192, 1>(d, ad, bd);
                        } else if (ts == TSLOTS - 2) {  // rows i, i - 1 in slots 6, 7; row i - 2 in slot 0
                            mma_bf16<128, 1>(d, ad, bd);
                            mma_bf16<64, 1>(tmem, ad, bd + B2);
                        } else {  // row i in slot 7; rows i - 1, i - 2 in slots 0, 1
                            mma_bf16<64, 1>(d, ad, bd);
                            mma_bf16<128, 1>(tmem, ad, bd + B1);
                        }
                    }
                mma_commit(&tfull[(2 - i) & (TSLOTS - 1)]);  // output row i - 2 is complete
                mma_commit(&empty[si]);                      // input row i has no later reader
                si = si + 1 == NSLOT ? 0 : si + 1;
            }
            if (!ok) *abort_flag = 1;
            // every issued MMA completes before the block frees its TMEM
            mma_commit(mdone);
            mbar_wait(mdone, 0);
        }
    } else {
        // ---- epilogue: 8 warps drain the slot of output row o ----------------------
        const int e = warp - 2;
        const int quarter = warp & 3, half = e >> 2;
        const int j = quarter * 32 + lane;  // pixel of the tile
        const int x = cb * TM + j;
        const bool leader = (e == 0 && lane == 0);
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        // every slot starts at zero
        for (int b = 0; b < TSLOTS; ++b) tmem_zero32(tmem + (uint32_t)(b * C + half * 32) + lane_base);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tzero);
        // the residual layer's skip input (this block's output rows of the block
        // input) arrives by TMA, two rows ahead, in the output tile's swizzled layout
        if (MODE == MODE_RESID && leader)
            for (int k = 0; k < 2 && k < T; ++k) {
                mbar_expect_tx(&skipbar[k], STAGE);
                tma_load_3d(skipbuf + k * STAGE, &tm_skip, &skipbar[k], 0, cb * TM + 1, yin0 + y_a + k + 1);
            }
        for (int q = 0; q < T + 2; ++q) {  // output row o = q - 2 (o < 0: partial sums only)
            const int o = q - 2;
            const int ts = (2 - q) & (TSLOTS - 1);
            bool ok = true;
            if (lane == 0) {
                ok = mbar_wait(&tfull[ts], (q >> 3) & 1);
                if (MODE == MODE_RESID && o >= 0 && ok) ok = mbar_wait(&skipbar[o % SKIPBUF], (o / SKIPBUF) & 1);
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!epi_bar_and(ok && !*abort_flag, 1, 32 * EPI_WARPS)) {
                if (leader) *abort_flag = 1;
                break;
            }
            tc_fence_after();
            if (MODE == MODE_RESID && leader && o >= 0 && o + 2 < T) {
                // buffer (o + 2) % 3 last held row o - 1, whose readers are past the barrier above
                const int k = (o + 2) % SKIPBUF;
                mbar_expect_tx(&skipbar[k], STAGE);
                tma_load_3d(skipbuf + k * STAGE, &tm_skip, &skipbar[k], 0, cb * TM + 1, yin0 + y_a + o + 3);
            }
            const uint32_t taddr = tmem + (uint32_t)(ts * C + half * 32) + lane_base;
            float v[32];
            if (o >= 0) {
                tmem_ld32(taddr, v);
                tmem_wait_ld();
            }
            tmem_zero32(taddr);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[ts]);  // the slot may take row o + 8
            if (o < 0) continue;
            const int y = y_a + o;
            if (MODE == MODE_RESID) {
                const uint4 *sp = reinterpret_cast<const uint4 *>(skipbuf + (o % SKIPBUF) * STAGE + j * 128);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint4 qv = sp[(half * 4 + i) ^ (j & 7)];
                    const uint32_t w4[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w4[k]));
                        v[i * 8 + 2 * k] += f.x;
                        v[i * 8 + 2 * k + 1] += f.y;
                    }
                }
                fence_proxy_async();  // these reads come before the buffer's next TMA write
            }
            // a window separator of a mosaic stays zero (the windows' zero padding)
            const bool sep = a.mosaic > 0 && ((y % a.mosaic) == a.mosaic - 1 || (x % a.mosaic) == a.mosaic - 1);
            uint4 outv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t w4[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int c0 = i * 8 + 2 * k, cc = half * 32 + c0;
                    float v0 = v[c0] + s_bias[cc], v1 = v[c0 + 1] + s_bias[cc + 1];
                    if (MODE != MODE_RESID) {
                        v0 = v0 > 0.f ? v0 : s_prelu[cc] * v0;
                        v1 = v1 > 0.f ? v1 : s_prelu[cc + 1] * v1;
                    }
                    if (sep) v0 = v1 = 0.f;
                    const __nv_bfloat162 bb = __floats2bfloat162_rn(v0, v1);
                    w4[k] = *reinterpret_cast<const uint32_t *>(&bb);
                }
                outv[i] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
            // output geometry: the coarse grid, or for the pixel shuffle the fine
            // grid, where group g's pixel x lands at (2y + g / 2, 2x + g % 2)
            const int OH = MODE == MODE_SHUFFLE ? 2 * a.H : a.H, OW = MODE == MODE_SHUFFLE ? 2 * a.W : a.W;
            const int oy = MODE == MODE_SHUFFLE ? 2 * y + (g >> 1) : y;
            const int ox = MODE == MODE_SHUFFLE ? 2 * x + (g & 1) : x;
            const int yout0 = MODE == MODE_SHUFFLE ? img * (2 * a.H + 2) : yin0;
            // stage o & 1 was last read by the TMA store of row o - 2
            if (leader) bulk_wait_read1();
            epi_bar(2, 32 * EPI_WARPS);
            // 128-byte swizzled staging: 16-byte chunk i of pixel j at position i ^ (j & 7)
            uint4 *st = reinterpret_cast<uint4 *>(stage + (o & 1) * STAGE + j * 128);
#pragma unroll
            for (int i = 0; i < 4; ++i) st[(half * 4 + i) ^ (j & 7)] = outv[i];
            if (ox == 0 || ox == OW - 1) store_half_px(a.out + out_img, OH, OW, oy, ox, half, outv, true);
            fence_proxy_async();
            epi_bar(2, 32 * EPI_WARPS);
            if (leader) {
                const unsigned char *src = stage + (o & 1) * STAGE;
                if (MODE == MODE_SHUFFLE) {
                    // fine map (channels, x parity, x / 2, padded row) from padded column 1
                    tma_store_4d(&tm_out, src, 0, g & 1, cb * TM, yout0 + oy + 1);
                    if (oy == 0) tma_store_4d(&tm_out, src, 0, g & 1, cb * TM, yout0 + OH + 1);
                    if (oy == OH - 1) tma_store_4d(&tm_out, src, 0, g & 1, cb * TM, yout0);
                } else {
                    tma_store_3d(&tm_out, src, 0, cb * TM + 1, yout0 + oy + 1);
                    if (oy == 0) tma_store_3d(&tm_out, src, 0, cb * TM + 1, yout0 + OH + 1);
                    if (oy == OH - 1) tma_store_3d(&tm_out, src, 0, cb * TM + 1, yout0);
                }
                bulk_commit();
            }
        }
        if (leader) bulk_wait_all();  // tile stores complete
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) atomicExch(a.err, 1);
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// CUDA-core layers and helpers
// ---------------------------------------------------------------------------

// s = max |ec| (1 when ec = 0), deterministic two-stage reduction
__global__ void __launch_bounds__(kRedThreads) k_absmax(const float *__restrict__ ec, size_t N,
                                                        double *partials, unsigned *counter, float *s_out) {
    __shared__ double sh[32];
    __shared__ bool last;
    float m = 0.f;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(ec[p]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float bm = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) bm = fmaxf(bm, (float)sh[w]);
        partials[blockIdx.x] = bm;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {  // the last block takes the max of the partials, all threads at once
        __threadfence();
        float gm = 0.f;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            gm = fmaxf(gm, (float)((volatile double *)partials)[b]);
        for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_down_sync(0xffffffffu, gm, o));
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = gm;
        __syncthreads();
        if (threadIdx.x == 0) {
            float bm = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) bm = fmaxf(bm, (float)sh[w]);
            s_out[0] = bm > 0.f ? bm : 1.f;
            *counter = 0u;
        }
    }
}

// conv3x3 1 -> 64 of q = ec / s, + bias, PReLU, to padded bf16; one thread per
// pixel.  The block's 256 pixels (consecutive along rows) go through shared
// memory so that the interior stores are 16-byte words written by consecutive
// threads; the halo copies of edge pixels are written directly.
// wt: the layer's weights staged as [tap][64 channels] (tap 9 = bias, 10 =
// PReLU slope), read four channels per 16-byte broadcast load.
__device__ __forceinline__ void conv_in_px(const float *__restrict__ ec, int nc, float s, const float4 *wt, int y,
                                           int x, uint4 *outv, int swz) {
    float q[9];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx)
            q[ky * 3 + kx] = ec[(size_t)((y + ky - 1 + nc) & (nc - 1)) * nc + ((x + kx - 1 + nc) & (nc - 1))] / s;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float v[8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // channels 8i + 4h .. + 3
            const float4 b4 = wt[9 * (C / 4) + 2 * i + h];
            float acc[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const float4 w4 = wt[t * (C / 4) + 2 * i + h];
                acc[0] = fmaf(w4.x, q[t], acc[0]);
                acc[1] = fmaf(w4.y, q[t], acc[1]);
                acc[2] = fmaf(w4.z, q[t], acc[2]);
                acc[3] = fmaf(w4.w, q[t], acc[3]);
            }
            const float4 a4 = wt[10 * (C / 4) + 2 * i + h];
            v[4 * h + 0] = acc[0] > 0.f ? acc[0] : a4.x * acc[0];
            v[4 * h + 1] = acc[1] > 0.f ? acc[1] : a4.y * acc[1];
            v[4 * h + 2] = acc[2] > 0.f ? acc[2] : a4.z * acc[2];
            v[4 * h + 3] = acc[3] > 0.f ? acc[3] : a4.w * acc[3];
        }
        uint32_t w4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat162 bb = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
            w4[k] = *reinterpret_cast<const uint32_t *>(&bb);
        }
        outv[i ^ swz] = make_uint4(w4[0], w4[1], w4[2], w4[3]);  // straight to the staging row
    }
}

// Stage wpack (w[64][9], b[64], a[64]) as [tap][64] with the bias and the
// slopes as rows 9 and 10.
__device__ __forceinline__ void stage_in_weights(float *w, const float *__restrict__ wpack) {
    for (int i = threadIdx.x; i < C * 11; i += blockDim.x) {
        const int t = i / C, c = i - t * C;
        w[i] = t < 9 ? wpack[c * 9 + t] : wpack[C * 9 + (t - 9) * C + c];
    }
}

// The halo copies of this thread's edge pixel, read back from its staging row.
__device__ __forceinline__ void conv_in_halo(const uint4 *st, __nv_bfloat16 *__restrict__ out, int nc, int y,
                                             int x) {
    uint4 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = st[threadIdx.x * 8 + (i ^ (threadIdx.x & 7))];
    store_px(out, nc, nc, y, x, v, true);
}

// Write the block's 256 staged pixels (p0 .. p0 + 255 of an nc x nc grid, all
// valid) to their interior positions: 16-byte word k of the block = chunk
// k & 7 of pixel k >> 3 (staged with the chunk index XOR the pixel's low bits).
__device__ __forceinline__ void conv_in_flush(const uint4 *st, __nv_bfloat16 *__restrict__ out, int nc, int p0) {
    for (int k = threadIdx.x; k < 256 * 8; k += 256) {
        const int px = k >> 3, ch = k & 7;
        const int p = p0 + px, y = p / nc, x = p - y * nc;
        reinterpret_cast<uint4 *>(out + ((size_t)(y + 1) * (nc + 2) + (x + 1)) * C)[ch] = st[px * 8 + (ch ^ (px & 7))];
    }
}

__global__ void __launch_bounds__(256) k_conv_in(const float *__restrict__ ec, int nc,
                                                 const float *__restrict__ s_ptr,
                                                 const float *__restrict__ wpack,  // w[64][9], b[64], a[64]
                                                 __nv_bfloat16 *__restrict__ out) {
    __shared__ __align__(16) float w[C * 11];
    __shared__ uint4 st[256 * 8];
    stage_in_weights(w, wpack);
    __syncthreads();
    const int p0 = blockIdx.x * 256, p = p0 + threadIdx.x;  // nc * nc is a multiple of 256
    const int y = p / nc, x = p - y * nc;
    conv_in_px(ec, nc, *s_ptr, reinterpret_cast<const float4 *>(w), y, x, st + threadIdx.x * 8, threadIdx.x & 7);
    if (x == 0 || x == nc - 1 || y == 0 || y == nc - 1) conv_in_halo(st, out, nc, y, x);
    __syncthreads();
    conv_in_flush(st, out, nc, p0);
}

// conv3x3 64 -> 1 on the padded fine activation, + bias, times s:
// fine_out = s * G.  A block walks a strip of 32 output columns down
// OUT_ROWS rows with four warps, two output rows per step; the 34-pixel input
// rows it needs stream through a ring of six shared-memory rows (cp.async),
// the next step's two rows loading while the current step computes, so every
// input pixel is read from memory about once (1.06 times with the strip's
// halo columns).  A warp takes 16 outputs of one row with its lanes split over
// the channels (lane l holds channels 2l, 2l + 1: a pixel's 128 bytes are one
// conflict-free 32-word shared load); each staged pixel of the output row's
// three input rows is loaded once and feeds the three outputs it is a
// horizontal tap of, each output accumulating its even and odd channel sums
// as one packed FP32 pair; a transposing butterfly over the lanes then gives
// lanes 2j and 2j + 1 output j.
constexpr int OUT_W = 32;             // strip width (output columns)
constexpr int OUT_ROWS = 32;          // output rows per block
constexpr int OUT_RING = 6;           // staged input rows
constexpr int OUT_PX = OUT_W + 2;     // staged pixels per row
constexpr int OUT_THREADS = 128;

__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Stage padded input row py (pixels x0 .. x0 + 33 of a row of nf + 2) into ring slot py % OUT_RING.
__device__ __forceinline__ void out_stage_row(uint4 *ring, const __nv_bfloat16 *__restrict__ u, int nf, int py,
                                              int x0) {
    uint4 *dst = ring + (py % OUT_RING) * OUT_PX * 8;
    const uint4 *src = reinterpret_cast<const uint4 *>(u + ((size_t)py * (nf + 2) + x0) * C);
    for (int i = threadIdx.x; i < OUT_PX * 8; i += OUT_THREADS) cp_async16(dst + i, src + i);
}

// The 16 outputs (before bias and scale) of one output row segment: staged
// rows py .. py + 2 (ring), pixels c0 .. c0 + 17 of the staged rows.  Lanes
// 2j and 2j + 1 return output j.
__device__ __forceinline__ float out_row16(const uint4 *ring, int py, int c0, const unsigned long long (&wp)[9],
                                           int lane) {
    const uint32_t *t32 = reinterpret_cast<const uint32_t *>(ring);
    unsigned long long acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0ull;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const uint32_t *row = t32 + ((py + dy) % OUT_RING) * OUT_PX * 32;
#pragma unroll
        for (int xp = 0; xp < 18; ++xp) {
            const uint32_t v = row[(c0 + xp) * 32 + lane];
            const unsigned long long vv = (unsigned long long)(v << 16) | ((unsigned long long)(v & 0xffff0000u) << 32);
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int tx = xp - kx;
                if (tx >= 0 && tx < 16) acc[tx] = ffma2(wp[dy * 3 + kx], vv, acc[tx]);
            }
        }
    }
    float a[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = __uint_as_float((uint32_t)acc[j]) + __uint_as_float((uint32_t)(acc[j] >> 32));
    // lanes' bits 4 .. 1 select the output bits 3 .. 0; bit 0 pairs two lanes
#pragma unroll
    for (int off = 16, half = 8; off >= 2; off >>= 1, half >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? a[i] : a[i + half];
            const float keep = upper ? a[i + half] : a[i];
            a[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return a[0] + __shfl_xor_sync(0xffffffffu, a[0], 1);
}

// Block (bx, by [, image bz]): output columns bx * 32 .., rows by * OUT_ROWS ..
__device__ __forceinline__ void conv_out_strip(const __nv_bfloat16 *__restrict__ u, int nf,
                                               const float *__restrict__ wpack, float s,
                                               float *__restrict__ fine_out, uint4 *ring) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x0 = blockIdx.x * OUT_W, y0 = blockIdx.y * OUT_ROWS;
    unsigned long long wp[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) wp[t] = pack2(wpack[t * C + 2 * lane], wpack[t * C + 2 * lane + 1]);
    const float bias = wpack[9 * C];
    // output row y needs padded rows y .. y + 2; a step computes rows r, r + 1
    for (int p = 0; p < 4; ++p) out_stage_row(ring, u, nf, y0 + p, x0);
    cp_async_commit();
    for (int r = 0; r < OUT_ROWS; r += 2) {
        if (r + 2 < OUT_ROWS) {  // the next step's two new rows
            out_stage_row(ring, u, nf, y0 + r + 4, x0);
            out_stage_row(ring, u, nf, y0 + r + 5, x0);
        }
        cp_async_commit();
        cp_async_wait<1>();  // everything but the group just issued
        __syncthreads();
        const int ry = r + (w >> 1), c0 = (w & 1) * 16;
        const float g = out_row16(ring, y0 + ry, c0, wp, lane);
        if ((lane & 1) == 0) fine_out[(size_t)(y0 + ry) * nf + x0 + c0 + (lane >> 1)] = s * (g + bias);
        __syncthreads();  // the ring slots of rows r, r + 1 are free for the step after next
    }
    cp_async_wait<0>();
}

__global__ void __launch_bounds__(OUT_THREADS) k_conv_out(const __nv_bfloat16 *__restrict__ u, int nf,
                                                          const float *__restrict__ wpack,  // w[9][64], b
                                                          const float *__restrict__ s_ptr,
                                                          float *__restrict__ fine_out) {
    __shared__ uint4 ring[OUT_RING * OUT_PX * 8];
    conv_out_strip(u, nf, wpack, *s_ptr, fine_out, ring);
}

// Batched forms for a stack of equal-size images (image = blockIdx.y, or
// blockIdx.z for k_conv_out_b): the same per-pixel arithmetic as k_absmax,
// k_conv_in and k_conv_out, with each image's coarse error read through a
// pointer table and its own scale s[image].
__global__ void __launch_bounds__(1024) k_absmax_b(const float *const *__restrict__ ecs, int nc,
                                                   float *__restrict__ s_out) {
    __shared__ float sh[32];
    const float *ec = ecs[blockIdx.x];
    const size_t N = (size_t)nc * nc;
    float m = 0.f;
    for (size_t p = threadIdx.x; p < N; p += blockDim.x) m = fmaxf(m, fabsf(ec[p]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float bm = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) bm = fmaxf(bm, sh[w]);
        s_out[blockIdx.x] = bm > 0.f ? bm : 1.f;
    }
}

__global__ void __launch_bounds__(256) k_conv_in_b(const float *const *__restrict__ ecs, int nc,
                                                   const float *__restrict__ s_all,
                                                   const float *__restrict__ wpack, __nv_bfloat16 *__restrict__ out) {
    __shared__ __align__(16) float w[C * 11];
    __shared__ uint4 st[256 * 8];
    stage_in_weights(w, wpack);
    __syncthreads();
    const float *ec = ecs[blockIdx.y];
    __nv_bfloat16 *o = out + (size_t)blockIdx.y * (nc + 2) * (nc + 2) * C;
    const int p0 = blockIdx.x * 256, p = p0 + threadIdx.x;
    const int y = p / nc, x = p - y * nc;
    conv_in_px(ec, nc, s_all[blockIdx.y], reinterpret_cast<const float4 *>(w), y, x, st + threadIdx.x * 8,
               threadIdx.x & 7);
    if (x == 0 || x == nc - 1 || y == 0 || y == nc - 1) conv_in_halo(st, o, nc, y, x);
    __syncthreads();
    conv_in_flush(st, o, nc, p0);
}

__global__ void __launch_bounds__(OUT_THREADS) k_conv_out_b(const __nv_bfloat16 *__restrict__ u_all, int nf,
                                                            const float *__restrict__ wpack,
                                                            const float *__restrict__ s_all,
                                                            float *__restrict__ out_all) {
    __shared__ uint4 ring[OUT_RING * OUT_PX * 8];
    conv_out_strip(u_all + (size_t)blockIdx.z * (nf + 2) * (nf + 2) * C, nf, wpack, s_all[blockIdx.z],
                   out_all + (size_t)blockIdx.z * nf * nf, ring);
}

// ---------------------------------------------------------------------------
// Windowed SR (Sec. 3.1, Fig. 2; Appendix A, Algorithms 1-5).  The coarse
// field is normalised by the symmetric logarithm, cut into n_s x n_s = 6 x 6
// windows whose origins step by 2 (window (a, b) covers coarse rows
// 2a - 2 .. 2a + 3 and columns 2b - 2 .. 2b + 3, wrapped), each window is
// super-resolved on its own with zero padding, the central 2 x 2 coarse
// cells of each (4 x 4 fine points) are kept and stitched, and the result is
// mapped back through the inverse normalisation.  The windows are laid out
// as a mosaic: a 7 x 7 cell per window (6 x 6 values, one zero separator row
// and column), kWinPerRow windows per mosaic row.  The mosaic is periodic and
// ends in a separator, so its periodic halo and the separators give every
// window exactly the zero padding it would have alone, as long as every
// layer keeps the separators zero (ConvArgs::mosaic).
// ---------------------------------------------------------------------------
constexpr int kWinNs = 6, kWinCell = 7, kWinPerRow = 128;  // mosaic width 896, a multiple of TM

__device__ __forceinline__ float symlog_f(float p, float pmin, float pmax, float lmin, float inv_span) {
    if (p == 0.f) return 0.f;
    const float m = fminf(fmaxf(fabsf(p), pmin), pmax);
    return copysignf((log10f(m) - lmin) * inv_span, p);
}

// conv 1 -> 64 + PReLU of the normalised windows, one thread per mosaic pixel.
__global__ void __launch_bounds__(256) k_win_in(const float *__restrict__ ec, int nc, float pmin, float pmax,
                                                float lmin, float inv_span, const float *__restrict__ wpack,
                                                __nv_bfloat16 *__restrict__ out, int Hm, int Wm) {
    __shared__ float w[C * 9 + 2 * C];
    for (int i = threadIdx.x; i < C * 11; i += blockDim.x) w[i] = wpack[i];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Hm * Wm) return;
    const int y = p / Wm, x = p - y * Wm;
    const int r = y / kWinCell, i = y - r * kWinCell, k = x / kWinCell, j = x - k * kWinCell;
    uint4 outv[8];
    if (i < kWinNs && j < kWinNs) {
        const int half = nc >> 1;
        const int wi = r * kWinPerRow + k;
        const int a = wi / half, b = wi - a * half;
        float q[9];
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int li = i + ky - 1, lj = j + kx - 1;
                float v = 0.f;
                if (li >= 0 && li < kWinNs && lj >= 0 && lj < kWinNs)
                    v = symlog_f(ec[(size_t)((2 * a - 2 + li) & (nc - 1)) * nc + ((2 * b - 2 + lj) & (nc - 1))], pmin,
                                 pmax, lmin, inv_span);
                q[ky * 3 + kx] = v;
            }
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
            uint32_t w4[4];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                float v[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = ii * 8 + 2 * kk + h;
                    float acc = w[C * 9 + c];
#pragma unroll
                    for (int t = 0; t < 9; ++t) acc = fmaf(w[c * 9 + t], q[t], acc);
                    v[h] = acc > 0.f ? acc : w[C * 10 + c] * acc;
                }
                const __nv_bfloat162 bb = __floats2bfloat162_rn(v[0], v[1]);
                w4[kk] = *reinterpret_cast<const uint32_t *>(&bb);
            }
            outv[ii] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
    } else {
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) outv[ii] = make_uint4(0u, 0u, 0u, 0u);
    }
    store_px(out, Hm, Wm, y, x, outv);
}

// conv 64 -> 1 at the kept 4 x 4 fine points of every window, then the
// inverse normalisation: out[Y][X] (fine grid 2nc) for Y, X in window
// (Y / 4, X / 4)'s kept block.  One thread per fine point, 16 per window.
__global__ void __launch_bounds__(256) k_win_out(const __nv_bfloat16 *__restrict__ u, int Wmf,
                                                 const float *__restrict__ wpack, int nc, float lmin, float span,
                                                 float *__restrict__ out) {
    const int half = nc >> 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= half * half * 16) return;
    const int wi = t >> 4, o = t & 15, oy = o >> 2, ox = o & 3;
    const int a = wi / half, b = wi - a * half;
    const int r = wi / kWinPerRow, k = wi - r * kWinPerRow;
    const int yf = 2 * kWinCell * r + 4 + oy, xf = 2 * kWinCell * k + 4 + ox;  // mosaic fine pixel
    float acc = 0.f;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
            const uint4 *pp = reinterpret_cast<const uint4 *>(u + ((size_t)(yf + ky) * (Wmf + 2) + (xf + kx)) * C);
            const float *wt = wpack + (ky * 3 + kx) * C;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint4 q = pp[i];
                const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w4[kk]));
                    acc = fmaf(wt[i * 8 + 2 * kk], f.x, acc);
                    acc = fmaf(wt[i * 8 + 2 * kk + 1], f.y, acc);
                }
            }
        }
    const float g = acc + wpack[9 * C];
    const float mag = exp10f(lmin + fabsf(g) * span);
    out[(size_t)(4 * a + oy) * (2 * nc) + 4 * b + ox] = g > 0.f ? mag : (g < 0.f ? -mag : 0.f);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
constexpr char kMagic[8] = {'M', 'G', 'S', 'R', 'W', '0', '0', '1'};
constexpr size_t kHeader = 64;

size_t expected_params(int nf, int nb) {
    size_t n = (size_t)nf * 9 + nf + nf;                     // in.w, in.b, in.a
    n += (size_t)nb * (2 * ((size_t)nf * nf * 9 + nf) + nf);  // blocks
    n += (size_t)4 * nf * nf * 9 + 4 * nf + nf;              // up.w, up.b, up.a
    n += (size_t)nf * 9 + 1;                                 // out.w, out.b
    return n;
}

// bf16 round-to-nearest-even of a float (host)
uint16_t bf16_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    return (uint16_t)((u + 0x7FFFu + lsb) >> 16);
}
float bf16_value(float f) {
    const uint32_t u = (uint32_t)bf16_bits(f) << 16;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

}  // namespace

bool make_grid_map_f32(CUtensorMap *m, void *base, int n, int cols, int rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc || n < cols || n < rows) return false;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)n * 4};
    cuuint32_t box[2] = {(cuuint32_t)cols, (cuuint32_t)rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

// padded activation [H+2][W+2][64] bf16 as a 3D tensor (c, x, y); a box is
// one 8-channel plane of a staged row: 8 channels x 130 pixels x 1 row
bool make_act_map(CUtensorMap *m, void *base, int H, int W) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)(W + 2), (cuuint64_t)(H + 2)};
    cuuint64_t strides[2] = {(cuuint64_t)C * 2, (cuuint64_t)(W + 2) * C * 2};
    cuuint32_t box[3] = {8, (cuuint32_t)ROWPX, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// padded activation as the destination of a tile: box 64 channels x 128 pixels
// x 1 row, 128-byte swizzle (the epilogue stages the tile in that layout)
bool make_out_map(CUtensorMap *m, void *base, int H, int W) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)(W + 2), (cuuint64_t)(H + 2)};
    cuuint64_t strides[2] = {(cuuint64_t)C * 2, (cuuint64_t)(W + 2) * C * 2};
    cuuint32_t box[3] = {(cuuint32_t)C, (cuuint32_t)TM, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// packed weights [layers][9][64 co][64 ci] bf16 as a 4D tensor; box = one layer
// the padded fine activation of the pixel-shuffle layer as the destination of
// a tile: fine pixel X = 2 x2 + p of a row sits at padded column X + 1, so
// from padded column 1 the map is (64 channels, parity p, x2, padded row) and
// a box of 64 x 1 x 128 x 1 is the 128 pixels of one parity of one row,
// 128-byte swizzled; rows = padded fine rows of all stacked images
bool make_fine_map(CUtensorMap *m, void *base, int rows, int W) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[4] = {(cuuint64_t)C, 2, (cuuint64_t)W, (cuuint64_t)rows};
    cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)2 * C * 2, (cuuint64_t)(2 * W + 2) * C * 2};
    cuuint32_t box[4] = {(cuuint32_t)C, 1, (cuuint32_t)TM, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (char *)base + C * 2, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// packed weights [layers][9 taps = dy * 3 + dx][64 co][64 ci] bf16 as a 5D
// tensor (ci, co, dx, dy, layer); a box is one dx of one layer, all three dy:
// [dy][co][ci] = 192 rows of 128 bytes, 128-byte swizzled
bool make_w_map(CUtensorMap *m, void *base, int layers) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)C, 3, 3, (cuuint64_t)layers};
    cuuint64_t strides[4] = {(cuuint64_t)C * 2, (cuuint64_t)TAPBYTES, (cuuint64_t)3 * TAPBYTES,
                             (cuuint64_t)9 * TAPBYTES};
    cuuint32_t box[5] = {(cuuint32_t)C, (cuuint32_t)C, 1, 3, 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Opt the convolution kernels into their shared memory (current device).
cudaError_t prepare_conv() {
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc<MODE_PRELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)CONV_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_conv_tc<MODE_RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)CONV_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_conv_tc<MODE_SHUFFLE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)CONV_SMEM);
    return e;
}

template <int MODE>
// tm_out: the output activation map (make_out_map), or for MODE_SHUFFLE the
// fine map (make_fine_map); tm_skip: the residual input (make_out_map of the
// skip buffer) for MODE_RESID, any map otherwise (not read).
cudaError_t launch_conv(const CUtensorMap &tm_in, const CUtensorMap &tm_w, const CUtensorMap &tm_out,
                        const CUtensorMap &tm_skip, ConvArgs a, int groups, cudaStream_t s) {
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int strips = a.imgs * groups * (a.W / TM);
    int chunks = sms / strips;
    if (chunks < 1) chunks = 1;
    if (a.imgs > 1) {
        // many strips: the row split with the fewest waves x (rows + 2 halo rows) per block
        long long best = -1;
        for (int c = 1; c <= a.H; ++c) {
            const long long waves = ((long long)strips * c + sms - 1) / sms;
            const long long cost = waves * ((a.H + c - 1) / c + 2);
            if (best < 0 || cost < best) {
                best = cost;
                chunks = c;
            }
        }
    }
    if (chunks > a.H) chunks = a.H;
    a.rows_per_chunk = (a.H + chunks - 1) / chunks;
    a.chunks = chunks;
    k_conv_tc<MODE><<<strips * chunks, CONV_THREADS, CONV_SMEM, s>>>(tm_in, tm_w, tm_out, tm_skip, a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t ensure_buffers(SrState *st, int nc) {
    if (st->nc == nc && st->act[0]) return cudaSuccess;
    for (int i = 0; i < 3; ++i) {
        cudaFree(st->act[i]);
        st->act[i] = nullptr;
    }
    cudaFree(st->fine_act);
    cudaFree(st->fine_out);
    st->fine_act = nullptr;
    st->fine_out = nullptr;
    st->nc = 0;
    const size_t coarse = (size_t)(nc + 2) * (nc + 2) * C * 2;
    const size_t fine = (size_t)(2 * nc + 2) * (2 * nc + 2) * C * 2;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMalloc(&st->act[i], coarse);
    if (e == cudaSuccess) e = cudaMalloc(&st->fine_act, fine);
    if (e == cudaSuccess) e = cudaMalloc(&st->fine_out, sizeof(float) * 4 * nc * nc);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < 3; ++i)
        if (!make_act_map(&st->tm_act[i], st->act[i], nc, nc) || !make_out_map(&st->tm_out[i], st->act[i], nc, nc))
            return cudaErrorInvalidValue;
    if (!make_fine_map(&st->tm_fine, st->fine_act, 2 * nc + 2, nc)) return cudaErrorInvalidValue;
    st->nc = nc;
    return cudaSuccess;
}

}  // namespace

void sr_free(SrState *st) {
    if (st->view) {
        for (int i = 0; i < 3; ++i) cudaFree(st->act[i]);
        cudaFree(st->fine_act);
        cudaFree(st->fine_out);
        *st = SrState();
        return;
    }
    cudaFree(st->w_tc);
    cudaFree(st->bias_tc);
    cudaFree(st->prelu_blk);
    cudaFree(st->prelu_up);
    cudaFree(st->w_in);
    cudaFree(st->w_out);
    for (int i = 0; i < 3; ++i) cudaFree(st->act[i]);
    cudaFree(st->fine_act);
    cudaFree(st->fine_out);
    cudaFree(st->scal);
    cudaFree(st->red);
    cudaFree(st->red_counter);
    cudaFree(st->err);
    *st = SrState();
}

mg_status sr_load(SrState *st, const void *blob, size_t bytes, char *err, size_t errlen) {
    if (bytes < kHeader || memcmp(blob, kMagic, 8) != 0) {
        snprintf(err, errlen, "weight blob: bad magic or too short (%zu bytes)", bytes);
        return MG_ERR_BAD_WEIGHTS;
    }
    uint32_t hdr[3];
    memcpy(hdr, (const char *)blob + 8, sizeof hdr);
    const int nf = (int)hdr[0], nb = (int)hdr[1];
    const size_t np = hdr[2];
    if (nf != C || nb < 1 || nb > 32 || np != expected_params(nf, nb) || bytes != kHeader + np * sizeof(float)) {
        snprintf(err, errlen, "weight blob: n_feat=%d n_blocks=%d n_params=%zu bytes=%zu inconsistent", nf, nb, np,
                 bytes);
        return MG_ERR_BAD_WEIGHTS;
    }
    const float *p = (const float *)((const char *)blob + kHeader);
    for (size_t i = 0; i < np; ++i) {
        const float v = p[i];
        if (!(v == v) || v > 3.0e38f || v < -3.0e38f) {
            snprintf(err, errlen, "weight blob: non-finite parameter at %zu", i);
            return MG_ERR_BAD_WEIGHTS;
        }
    }
    // unpack in blob order
    const float *in_w = p, *in_b = in_w + C * 9, *in_a = in_b + C;
    const float *q = in_a + C;
    const int layers = 2 * nb + 4;
    std::vector<uint16_t> wtc((size_t)layers * 9 * C * C);
    std::vector<float> btc((size_t)layers * C), ablk((size_t)nb * C), aup(C), win(C * 11), wout(9 * C + 1);
    auto pack = [&](int layer, const float *w /*[co][ci][3][3]*/, int co_stride, int co_off) {
        // packed[layer][tap][co][ci] = w[co_src][ci][ky][kx]
        for (int t = 0; t < 9; ++t)
            for (int co = 0; co < C; ++co)
                for (int ci = 0; ci < C; ++ci) {
                    const int src = co * co_stride + co_off;
                    wtc[(((size_t)layer * 9 + t) * C + co) * C + ci] = bf16_bits(w[((size_t)src * C + ci) * 9 + t]);
                }
    };
    for (int k = 0; k < nb; ++k) {
        const float *w1 = q, *b1 = w1 + C * C * 9, *a1 = b1 + C, *w2 = a1 + C, *b2 = w2 + C * C * 9;
        pack(2 * k, w1, 1, 0);
        pack(2 * k + 1, w2, 1, 0);
        memcpy(&btc[(size_t)(2 * k) * C], b1, C * sizeof(float));
        memcpy(&btc[(size_t)(2 * k + 1) * C], b2, C * sizeof(float));
        memcpy(&ablk[(size_t)k * C], a1, C * sizeof(float));
        q = b2 + C;
    }
    const float *up_w = q, *up_b = up_w + 4 * C * C * 9, *up_a = up_b + 4 * C;
    const float *out_w = up_a + C, *out_b = out_w + C * 9;
    // pixel-shuffle group s holds output channels 4c + s, c = 0..63
    for (int s = 0; s < 4; ++s) {
        pack(2 * nb + s, up_w, 4, s);
        for (int c = 0; c < C; ++c) btc[(size_t)(2 * nb + s) * C + c] = up_b[4 * c + s];
    }
    memcpy(aup.data(), up_a, C * sizeof(float));
    for (int c = 0; c < C; ++c) {
        for (int t = 0; t < 9; ++t) win[c * 9 + t] = bf16_value(in_w[c * 9 + t]);
        win[C * 9 + c] = in_b[c];
        win[C * 10 + c] = in_a[c];
    }
    for (int t = 0; t < 9; ++t)
        for (int c = 0; c < C; ++c) wout[t * C + c] = bf16_value(out_w[c * 9 + t]);
    wout[9 * C] = out_b[0];

    sr_free(st);
    cudaError_t e = cudaMalloc(&st->w_tc, wtc.size() * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMemcpy(st->w_tc, wtc.data(), wtc.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&st->bias_tc, btc.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(st->bias_tc, btc.data(), btc.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&st->prelu_blk, ablk.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(st->prelu_blk, ablk.data(), ablk.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&st->prelu_up, C * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(st->prelu_up, aup.data(), C * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&st->w_in, win.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(st->w_in, win.data(), win.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&st->w_out, wout.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(st->w_out, wout.data(), wout.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&st->scal, 4 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&st->red, sizeof(double) * kRedBlocks);
    if (e == cudaSuccess) e = cudaMalloc(&st->red_counter, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(st->red_counter, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&st->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(st->err, 0, sizeof(int));
    if (e == cudaSuccess && !make_w_map(&st->tm_w, st->w_tc, layers)) e = cudaErrorInvalidValue;
    if (e != cudaSuccess) {
        snprintf(err, errlen, "weight upload: %s", cudaGetErrorString(e));
        sr_free(st);
        return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
    }
    st->n_feat = nf;
    st->n_blocks = nb;
    uint64_t hsh = 1469598103934665603ull;
    for (size_t i = 0; i < bytes; ++i) hsh = (hsh ^ ((const unsigned char *)blob)[i]) * 1099511628211ull;
    st->hash = hsh;
    st->loaded = true;
    return MG_OK;
}

mg_status sr_prepare(SrState *st, int nc, char *err, size_t errlen) {
    if (!st->loaded) {
        snprintf(err, errlen, "no generator weights loaded");
        return MG_ERR_NO_WEIGHTS;
    }
    if (nc < TM || nc % TM) {
        snprintf(err, errlen, "SR prolongation needs a coarse grid of at least %d (multiple of %d), got %d", TM, TM, nc);
        return MG_ERR_INVALID_ARG;
    }
    cudaError_t e = prepare_conv();
    if (e == cudaSuccess) e = ensure_buffers(st, nc);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "SR buffers for %d^2: %s", nc, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
    }
    return MG_OK;
}

mg_status sr_view(SrState *view, const SrState *st, int nc, char *err, size_t errlen) {
    if (!st->loaded || st->view) {
        snprintf(err, errlen, "no generator weights loaded");
        return MG_ERR_NO_WEIGHTS;
    }
    if (nc < TM || nc % TM) {
        snprintf(err, errlen, "SR prolongation needs a coarse grid of at least %d (multiple of %d), got %d", TM, TM, nc);
        return MG_ERR_INVALID_ARG;
    }
    // the view's own buffers survive; everything else is st's (refreshed on
    // every call, so reloaded weights are picked up)
    SrState v = *st;
    v.view = true;
    for (int i = 0; i < 3; ++i) {
        v.act[i] = view->act[i];
        v.tm_act[i] = view->tm_act[i];
        v.tm_out[i] = view->tm_out[i];
    }
    v.fine_act = view->fine_act;
    v.fine_out = view->fine_out;
    v.tm_fine = view->tm_fine;  // the view's own fine map (st's maps describe st's buffers)
    v.nc = view->view ? view->nc : 0;
    cudaError_t e = prepare_conv();
    if (e == cudaSuccess) e = ensure_buffers(&v, nc);
    *view = v;
    if (e != cudaSuccess) {
        snprintf(err, errlen, "SR buffers for %d^2: %s", nc, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
    }
    return MG_OK;
}

mg_status sr_correction(SrState *st, const float *ec, int nc, cudaStream_t s, char *err, size_t errlen) {
    if (!st->loaded || st->nc != nc) {
        snprintf(err, errlen, "SR generator not prepared for a %d^2 coarse grid", nc);
        return MG_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSuccess;
    const size_t N = (size_t)nc * nc;
    k_absmax<<<kRedBlocks, kRedThreads, 0, s>>>(ec, N, st->red, st->red_counter, st->scal);
    count_launches(1);
    k_conv_in<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(ec, nc, st->scal, st->w_in,
                                                        (__nv_bfloat16 *)st->act[0]);
    count_launches(1);
    e = cudaGetLastError();
    int cur = 0;
    const int nb = st->n_blocks;
    for (int k = 0; k < nb && e == cudaSuccess; ++k) {
        const int nxt = (cur + 1) % 3, tmp = (cur + 2) % 3;
        ConvArgs a1 = {nullptr, (__nv_bfloat16 *)st->act[tmp], st->bias_tc + (size_t)(2 * k) * C,
                       st->prelu_blk + (size_t)k * C, nc, nc, 2 * k, 0, 0, st->err};
        e = launch_conv<MODE_PRELU>(st->tm_act[cur], st->tm_w, st->tm_out[tmp], st->tm_out[cur], a1, 1, s);
        if (e != cudaSuccess) break;
        ConvArgs a2 = {(const __nv_bfloat16 *)st->act[cur], (__nv_bfloat16 *)st->act[nxt],
                       st->bias_tc + (size_t)(2 * k + 1) * C, nullptr, nc, nc, 2 * k + 1, 0, 0, st->err};
        e = launch_conv<MODE_RESID>(st->tm_act[tmp], st->tm_w, st->tm_out[nxt], st->tm_out[cur], a2, 1, s);
        cur = nxt;
    }
    if (e == cudaSuccess) {
        ConvArgs au = {nullptr, (__nv_bfloat16 *)st->fine_act, st->bias_tc + (size_t)(2 * nb) * C, st->prelu_up,
                       nc, nc, 2 * nb, 0, 0, st->err};
        e = launch_conv<MODE_SHUFFLE>(st->tm_act[cur], st->tm_w, st->tm_fine, st->tm_out[cur], au, 4, s);
    }
    if (e == cudaSuccess) {
        const int nf = 2 * nc;
        dim3 grid(nf / OUT_W, nf / OUT_ROWS);
        k_conv_out<<<grid, OUT_THREADS, 0, s>>>((const __nv_bfloat16 *)st->fine_act, nf, st->w_out, st->scal,
                                                  st->fine_out);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        snprintf(err, errlen, "SR generator launch: %s", cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    return MG_OK;
}

mg_status sr_layer(SrState *st, int layer, int nc, const void *in, const void *skip, float *s, void *out,
                   cudaStream_t strm, char *err, size_t errlen) {
    if (!st->loaded) {
        snprintf(err, errlen, "no generator weights loaded");
        return MG_ERR_NO_WEIGHTS;
    }
    const int nb = st->n_blocks;
    if (layer < 0 || layer > 2 * nb + 2 || nc < TM || nc % TM || !in || !out || !s ||
        (layer >= 1 && layer <= 2 * nb && layer % 2 == 0 && !skip)) {
        snprintf(err, errlen, "sr_layer: bad layer %d (0..%d), size %d (a multiple of %d) or null buffer", layer,
                 2 * nb + 2, nc, TM);
        return MG_ERR_INVALID_ARG;
    }
    cudaError_t e = prepare_conv();
    if (e == cudaSuccess) e = cudaMemsetAsync(st->err, 0, sizeof(int), strm);
    if (e == cudaSuccess && layer == 0) {
        const size_t N = (size_t)nc * nc;
        k_absmax<<<kRedBlocks, kRedThreads, 0, strm>>>((const float *)in, N, st->red, st->red_counter, s);
        count_launches(1);
        k_conv_in<<<(unsigned)((N + 255) / 256), 256, 0, strm>>>((const float *)in, nc, s, st->w_in,
                                                               (__nv_bfloat16 *)out);
        count_launches(1);
        e = cudaGetLastError();
    } else if (e == cudaSuccess && layer <= 2 * nb + 1) {
        const int l = layer - 1;  // weight layer (the pixel-shuffle groups follow the blocks)
        const int mode = layer == 2 * nb + 1 ? MODE_SHUFFLE : (l % 2 ? MODE_RESID : MODE_PRELU);
        CUtensorMap tin, tout, tskip;
        if (!make_act_map(&tin, const_cast<void *>(in), nc, nc) ||
            !(mode == MODE_SHUFFLE ? make_fine_map(&tout, out, 2 * nc + 2, nc) : make_out_map(&tout, out, nc, nc)) ||
            !make_out_map(&tskip, const_cast<void *>(mode == MODE_RESID ? skip : in), nc, nc)) {
            snprintf(err, errlen, "sr_layer: tensor map encoding failed");
            return MG_ERR_INVALID_ARG;
        }
        const float *prelu = mode == MODE_SHUFFLE ? st->prelu_up : st->prelu_blk + (size_t)(l / 2) * C;
        ConvArgs a = {mode == MODE_RESID ? (const __nv_bfloat16 *)skip : nullptr, (__nv_bfloat16 *)out,
                      st->bias_tc + (size_t)l * C, mode == MODE_RESID ? nullptr : prelu, nc, nc, l, 0, 0, st->err};
        if (mode == MODE_PRELU) e = launch_conv<MODE_PRELU>(tin, st->tm_w, tout, tskip, a, 1, strm);
        else if (mode == MODE_RESID) e = launch_conv<MODE_RESID>(tin, st->tm_w, tout, tskip, a, 1, strm);
        else e = launch_conv<MODE_SHUFFLE>(tin, st->tm_w, tout, tskip, a, 4, strm);
    } else if (e == cudaSuccess) {
        const int nf = 2 * nc;
        dim3 grid(nf / OUT_W, nf / OUT_ROWS);
        k_conv_out<<<grid, OUT_THREADS, 0, strm>>>((const __nv_bfloat16 *)in, nf, st->w_out, s, (float *)out);
        count_launches(1);
        e = cudaGetLastError();
    }
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, st->err, sizeof(int), cudaMemcpyDeviceToHost, strm);
    if (e == cudaSuccess) e = cudaStreamSynchronize(strm);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "sr_layer: %s", cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    if (flag) {
        snprintf(err, errlen, "sr_layer: a bounded wait in the tensor-core kernel timed out");
        return MG_ERR_TIMEOUT;
    }
    return MG_OK;
}

void sr_batch_free(SrBatch *b) {
    for (int i = 0; i < 3; ++i) cudaFree(b->act[i]);
    cudaFree(b->fine_act);
    cudaFree(b->fine_out);
    cudaFree(b->s);
    cudaFree(b->ecs);
    *b = SrBatch();
}

mg_status sr_batch_prepare(SrBatch *b, int imgs, int nc, const float *const *ecs, char *err, size_t errlen) {
    sr_batch_free(b);
    if (imgs < 1 || nc < TM || nc % TM) {
        snprintf(err, errlen, "batched SR: %d images of %d^2 (a multiple of %d) not supported", imgs, nc, TM);
        return MG_ERR_INVALID_ARG;
    }
    const size_t coarse = (size_t)imgs * (nc + 2) * (nc + 2) * C * 2;
    const size_t fine = (size_t)imgs * (2 * nc + 2) * (2 * nc + 2) * C * 2;
    cudaError_t e = prepare_conv();
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMalloc(&b->act[i], coarse);
    if (e == cudaSuccess) e = cudaMalloc(&b->fine_act, fine);
    if (e == cudaSuccess) e = cudaMalloc(&b->fine_out, sizeof(float) * imgs * 4 * (size_t)nc * nc);
    if (e == cudaSuccess) e = cudaMalloc(&b->s, sizeof(float) * imgs);
    if (e == cudaSuccess) e = cudaMalloc(&b->ecs, sizeof(float *) * imgs);
    if (e == cudaSuccess) e = cudaMemcpy(b->ecs, ecs, sizeof(float *) * imgs, cudaMemcpyHostToDevice);
    const int Hs = imgs * (nc + 2) - 2;  // the stack as one padded grid of Hs + 2 rows
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        if (!make_act_map(&b->tm_act[i], b->act[i], Hs, nc) || !make_out_map(&b->tm_out[i], b->act[i], Hs, nc))
            e = cudaErrorInvalidValue;
    if (e == cudaSuccess && !make_fine_map(&b->tm_fine, b->fine_act, imgs * (2 * nc + 2), nc)) e = cudaErrorInvalidValue;
    if (e != cudaSuccess) {
        snprintf(err, errlen, "batched SR buffers (%d x %d^2): %s", imgs, nc, cudaGetErrorString(e));
        sr_batch_free(b);
        return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
    }
    b->imgs = imgs;
    b->nc = nc;
    return MG_OK;
}

mg_status sr_batch_correction(SrBatch *b, const SrState *st, cudaStream_t s, char *err, size_t errlen) {
    if (!st->loaded || !b->imgs) {
        snprintf(err, errlen, "batched SR: no weights or no prepared batch");
        return MG_ERR_INVALID_ARG;
    }
    const int nc = b->nc, imgs = b->imgs, nb = st->n_blocks;
    k_absmax_b<<<imgs, 1024, 0, s>>>(b->ecs, nc, b->s);
    count_launches(1);
    k_conv_in_b<<<dim3((unsigned)(((size_t)nc * nc + 255) / 256), imgs), 256, 0, s>>>(b->ecs, nc, b->s, st->w_in,
                                                                                      (__nv_bfloat16 *)b->act[0]);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    int cur = 0;
    for (int k = 0; k < nb && e == cudaSuccess; ++k) {
        const int nxt = (cur + 1) % 3, tmp = (cur + 2) % 3;
        ConvArgs a1 = {nullptr, (__nv_bfloat16 *)b->act[tmp], st->bias_tc + (size_t)(2 * k) * C,
                       st->prelu_blk + (size_t)k * C, nc, nc, 2 * k, 0, 0, st->err, imgs};
        e = launch_conv<MODE_PRELU>(b->tm_act[cur], st->tm_w, b->tm_out[tmp], b->tm_out[cur], a1, 1, s);
        if (e != cudaSuccess) break;
        ConvArgs a2 = {(const __nv_bfloat16 *)b->act[cur], (__nv_bfloat16 *)b->act[nxt],
                       st->bias_tc + (size_t)(2 * k + 1) * C, nullptr, nc, nc, 2 * k + 1, 0, 0, st->err, imgs};
        e = launch_conv<MODE_RESID>(b->tm_act[tmp], st->tm_w, b->tm_out[nxt], b->tm_out[cur], a2, 1, s);
        cur = nxt;
    }
    if (e == cudaSuccess) {
        ConvArgs au = {nullptr, (__nv_bfloat16 *)b->fine_act, st->bias_tc + (size_t)(2 * nb) * C, st->prelu_up,
                       nc, nc, 2 * nb, 0, 0, st->err, imgs};
        e = launch_conv<MODE_SHUFFLE>(b->tm_act[cur], st->tm_w, b->tm_fine, b->tm_out[cur], au, 4, s);
    }
    if (e == cudaSuccess) {
        const int nf = 2 * nc;
        k_conv_out_b<<<dim3(nf / OUT_W, nf / OUT_ROWS, imgs), OUT_THREADS, 0, s>>>(
            (const __nv_bfloat16 *)b->fine_act, nf, st->w_out, b->s, b->fine_out);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        snprintf(err, errlen, "batched SR generator launch: %s", cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    return MG_OK;
}

void sr_windows_free(SrWindows *w) {
    for (int i = 0; i < 3; ++i) cudaFree(w->act[i]);
    cudaFree(w->fine_act);
    *w = SrWindows();
}

static int win_rows(int nc) { return (nc / 2) * (nc / 2) / kWinPerRow * kWinCell; }

mg_status sr_windows_prepare(SrWindows *w, int nc, char *err, size_t errlen) {
    if (nc < 32 || (nc & (nc - 1))) {
        snprintf(err, errlen, "windowed SR needs a power-of-two coarse grid of at least 32, got %d", nc);
        return MG_ERR_INVALID_ARG;
    }
    if (w->nc == nc && w->act[0]) return MG_OK;
    sr_windows_free(w);
    const int Hm = win_rows(nc), Wm = kWinPerRow * kWinCell;
    const size_t coarse = (size_t)(Hm + 2) * (Wm + 2) * C * 2;
    const size_t fine = (size_t)(2 * Hm + 2) * (2 * Wm + 2) * C * 2;
    cudaError_t e = prepare_conv();
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaMalloc(&w->act[i], coarse);
    if (e == cudaSuccess) e = cudaMalloc(&w->fine_act, fine);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        if (!make_act_map(&w->tm_act[i], w->act[i], Hm, Wm) || !make_out_map(&w->tm_out[i], w->act[i], Hm, Wm))
            e = cudaErrorInvalidValue;
    if (e == cudaSuccess && !make_fine_map(&w->tm_fine, w->fine_act, 2 * Hm + 2, Wm)) e = cudaErrorInvalidValue;
    if (e != cudaSuccess) {
        snprintf(err, errlen, "windowed SR buffers for %d^2: %s", nc, cudaGetErrorString(e));
        sr_windows_free(w);
        return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
    }
    w->nc = nc;
    w->Hm = Hm;
    w->Wm = Wm;
    return MG_OK;
}

mg_status sr_windowed(SrWindows *w, const SrState *st, const float *ec, int nc, double p_min, double p_max,
                      float *out, cudaStream_t s, char *err, size_t errlen) {
    if (!st->loaded || w->nc != nc) {
        snprintf(err, errlen, "windowed SR not prepared for a %d^2 coarse grid", nc);
        return MG_ERR_INVALID_ARG;
    }
    const double lmin = log10(p_min), lmax = log10(p_max);
    const int Hm = w->Hm, Wm = w->Wm, nb = st->n_blocks;
    k_win_in<<<(unsigned)(((size_t)Hm * Wm + 255) / 256), 256, 0, s>>>(
        ec, nc, (float)p_min, (float)p_max, (float)lmin, (float)(1.0 / (lmax - lmin)), st->w_in,
        (__nv_bfloat16 *)w->act[0], Hm, Wm);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    int cur = 0;
    for (int k = 0; k < nb && e == cudaSuccess; ++k) {
        const int nxt = (cur + 1) % 3, tmp = (cur + 2) % 3;
        ConvArgs a1 = {nullptr, (__nv_bfloat16 *)w->act[tmp], st->bias_tc + (size_t)(2 * k) * C,
                       st->prelu_blk + (size_t)k * C, Hm, Wm, 2 * k, 0, 0, st->err, 1, kWinCell};
        e = launch_conv<MODE_PRELU>(w->tm_act[cur], st->tm_w, w->tm_out[tmp], w->tm_out[cur], a1, 1, s);
        if (e != cudaSuccess) break;
        ConvArgs a2 = {(const __nv_bfloat16 *)w->act[cur], (__nv_bfloat16 *)w->act[nxt],
                       st->bias_tc + (size_t)(2 * k + 1) * C, nullptr, Hm, Wm, 2 * k + 1, 0, 0, st->err, 1, kWinCell};
        e = launch_conv<MODE_RESID>(w->tm_act[tmp], st->tm_w, w->tm_out[nxt], w->tm_out[cur], a2, 1, s);
        cur = nxt;
    }
    if (e == cudaSuccess) {
        ConvArgs au = {nullptr, (__nv_bfloat16 *)w->fine_act, st->bias_tc + (size_t)(2 * nb) * C, st->prelu_up,
                       Hm, Wm, 2 * nb, 0, 0, st->err, 1, kWinCell};
        e = launch_conv<MODE_SHUFFLE>(w->tm_act[cur], st->tm_w, w->tm_fine, w->tm_out[cur], au, 4, s);
    }
    if (e == cudaSuccess) {
        const size_t pts = (size_t)(nc / 2) * (nc / 2) * 16;
        k_win_out<<<(unsigned)((pts + 255) / 256), 256, 0, s>>>((const __nv_bfloat16 *)w->fine_act, 2 * Wm,
                                                               st->w_out, nc, (float)lmin, (float)(lmax - lmin), out);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        snprintf(err, errlen, "windowed SR launch: %s", cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    return MG_OK;
}

mg_status sr_conv_layer(int mode, int H, int W, const void *in, const void *skip, const void *w_packed,
                        const float *bias, const float *prelu, void *out, cudaStream_t s, char *err,
                        size_t errlen) {
    if (W < TM || W % TM || H < 1 || (mode != MODE_PRELU && mode != MODE_RESID && mode != MODE_SHUFFLE) ||
        (mode == MODE_RESID && !skip) || (mode != MODE_RESID && !prelu)) {
        snprintf(err, errlen, "sr_conv_layer: bad mode %d or size %dx%d (W a multiple of %d)", mode, H, W, TM);
        return MG_ERR_INVALID_ARG;
    }
    CUtensorMap tin, tw, tout, tskip;
    const int groups = mode == MODE_SHUFFLE ? 4 : 1;
    if (!make_act_map(&tin, const_cast<void *>(in), H, W) || !make_w_map(&tw, const_cast<void *>(w_packed), groups) ||
        !(mode == MODE_SHUFFLE ? make_fine_map(&tout, out, 2 * H + 2, W) : make_out_map(&tout, out, H, W)) ||
        !make_out_map(&tskip, const_cast<void *>(mode == MODE_RESID ? skip : in), H, W)) {
        snprintf(err, errlen, "sr_conv_layer: tensor map encoding failed");
        return MG_ERR_INVALID_ARG;
    }
    int *dflag = nullptr;
    cudaError_t e = prepare_conv();
    if (e == cudaSuccess) e = cudaMalloc(&dflag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(dflag, 0, sizeof(int), s);
    ConvArgs a = {(const __nv_bfloat16 *)skip, (__nv_bfloat16 *)out, bias, prelu, H, W, 0, 0, 0, dflag};
    if (e == cudaSuccess) {
        if (mode == MODE_PRELU) e = launch_conv<MODE_PRELU>(tin, tw, tout, tskip, a, 1, s);
        else if (mode == MODE_RESID) e = launch_conv<MODE_RESID>(tin, tw, tout, tskip, a, 1, s);
        else e = launch_conv<MODE_SHUFFLE>(tin, tw, tout, tskip, a, 4, s);
    }
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dflag);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "sr_conv_layer: %s", cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    if (flag) {
        snprintf(err, errlen, "sr_conv_layer: a bounded wait in the tensor-core kernel timed out");
        return MG_ERR_TIMEOUT;
    }
    return MG_OK;
}

}  // namespace mg
