// mg_train.cu - training of the SR generator on error pairs the solver
// produces (Sec. 2.3 and Sec. 3.2 of the paper train the generator on coarse /
// fine pressure pairs; here the pairs are the multigrid's own coarse-grid
// errors and fine-grid corrections).
//
// Model (the one the SR prolongation evaluates, see mg_sr.cuh):
//   x0 = PReLU(conv(q; 1 -> 64)),  x_{k+1} = x_k + conv(PReLU(conv(x_k)))  (k < nb),
//   u  = PReLU(shuffle(conv(x_nb; 64 -> 256))),  y = conv(u; 64 -> 1),
// every conv 3x3 with bias and circular padding, on a batch of periodic
// coarse fields q (H x W) and fine outputs y (2H x 2W).  Loss: the mean of
// mask * (y - t)^2 over the fine pixels.  Adam on FP32 master weights.
//
// The 64/256-channel convolutions are GEMMs in three forms: forward (K = 9
// taps x input channels), data gradient (the same with the taps mirrored and
// the weight's channel roles swapped) and weight gradient (K = pixels, split
// over fixed chunks and summed in chunk order, so results are
// deterministic).  They run on the tcgen05 tensor cores with BF16 operands
// and FP32 accumulation (k_conv_gemm_tc, k_conv_wgrad_tc; the default for
// rows of whole 128-pixel tiles), or in FP32 on the CUDA cores as implicit
// GEMMs over 64-pixel x 64-channel tiles (256 threads, 4 x 4 outputs per
// thread, K staged through shared memory 16 at a time).  The thin first and
// last layers, PReLU, the shuffle, the loss, the per-channel sums and Adam
// are FP32 CUDA-core kernels.  Activations are channels-last
// [batch][y][x][channel]; parameters, gradients and Adam moments are flat
// arrays in the weight-blob order of mg_load_prolong_weights.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include <cuda_bf16.h>

#include "mg_internal.cuh"
#include "mg_tc.cuh"

namespace mg {

namespace {

constexpr int F = 64;             // features
constexpr int TP = 64;            // pixels per GEMM tile
constexpr int KC = 16;            // K per shared-memory stage
constexpr int GT = 256;           // threads per GEMM block
constexpr int WCHUNK = 2048;      // pixels per weight-gradient partial (FP32 GEMM)
constexpr int WCHUNK_TC = 1024;   // pixels per weight-gradient partial (tensor cores)
constexpr int RCHUNK = 256;       // pixels per partial of the per-channel sums and thin-layer weight gradients
constexpr int RT = 256;           // threads of the small kernels

struct Geo {
    int H, W, lgH, lgW, B;  // coarse grid of one sample, batch
};

// Pixel p = (b * H + y) * W + x of an H x W periodic grid; neighbour at (dy, dx).
__device__ __forceinline__ int nbr(int p, int lgH, int lgW, int dy, int dx) {
    const int W = 1 << lgW, H = 1 << lgH;
    const int x = p & (W - 1), y = (p >> lgW) & (H - 1), base = p - (y << lgW) - x;
    return base + (((y + dy) & (H - 1)) << lgW) + ((x + dx) & (W - 1));
}

// ---------------------------------------------------------------------------
// Implicit-GEMM 3x3 convolution, forward or data gradient.
//   FWD : out[p][n] = sum_{tap, k} in[p + tap][k] * w[(n * CK + k) * 9 + tap]   (CK = in channels)
//   DGRAD: out[p][n] = sum_{tap, k} in[p - tap][k] * w[(k * CN + n) * 9 + tap]  (in = output grad,
//          CK = the layer's out channels, CN = the layer's in channels)
// Block: 64 pixels x 64 output channels (blockIdx.y picks the channel tile).
// Epilogue modes write either the raw sum (+ bias) or fused activations.
// ---------------------------------------------------------------------------
enum { EPI_RAW = 0, EPI_PRELU = 1, EPI_ADD = 2, EPI_SHUFFLE = 3 };

template <bool DGRAD, int CK, int CN, int EPI>
__global__ void __launch_bounds__(GT) k_conv_gemm(const float *__restrict__ in, const float *__restrict__ w,
                                                  const float *__restrict__ bias, const float *__restrict__ slope,
                                                  const float *__restrict__ skip, float *__restrict__ out,
                                                  float *__restrict__ out2, Geo g) {
    __shared__ __align__(16) float As[KC][TP + 4];
    __shared__ __align__(16) float Bs[KC][64 + 4];
    const int p0 = blockIdx.x * TP, n0 = blockIdx.y * 64;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;  // tx: pixel group, ty: channel group
    float acc[4][4] = {};
    for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        for (int k0 = 0; k0 < CK; k0 += KC) {
            {   // A: 64 pixels x 16 channels, one float4 per thread
                const int px = tid >> 2, kq = (tid & 3) * 4;
                const int q = DGRAD ? nbr(p0 + px, g.lgH, g.lgW, -dy, -dx) : nbr(p0 + px, g.lgH, g.lgW, dy, dx);
                const float4 v = *reinterpret_cast<const float4 *>(in + (size_t)q * CK + k0 + kq);
                As[kq + 0][px] = v.x;
                As[kq + 1][px] = v.y;
                As[kq + 2][px] = v.z;
                As[kq + 3][px] = v.w;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {  // B: 16 x 64
                const int e = tid + r * GT, kk = e >> 6, nn = e & 63;
                const int k = k0 + kk, n = n0 + nn;
                Bs[kk][nn] = DGRAD ? w[((size_t)k * CN + n) * 9 + tap] : w[((size_t)n * CK + k) * 9 + tap];
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
                const float4 a = *reinterpret_cast<const float4 *>(&As[kk][tx * 4]);
                const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][ty * 4]);
                const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
    constexpr int COUT = CN;  // output channels of this GEMM
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int p = p0 + tx * 4 + i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + ty * 4 + j;
            float v = acc[i][j] + (bias ? bias[n] : 0.f);
            if (EPI == EPI_RAW) {
                out[(size_t)p * COUT + n] = v;
            } else if (EPI == EPI_PRELU) {  // out = z, out2 = PReLU(z)
                out[(size_t)p * COUT + n] = v;
                out2[(size_t)p * COUT + n] = v > 0.f ? v : slope[n] * v;
            } else if (EPI == EPI_ADD) {    // out = skip + conv
                out[(size_t)p * COUT + n] = skip[(size_t)p * COUT + n] + v;
            } else {                        // EPI_SHUFFLE: out = z (coarse, 4F ch), out2 = PReLU at fine
                out[(size_t)p * COUT + n] = v;
                const int c = n >> 2, sy = (n >> 1) & 1, sx = n & 1;
                const int Wc = 1 << g.lgW, Hc = 1 << g.lgH;
                const int x = p & (Wc - 1), y = (p >> g.lgW) & (Hc - 1), b = p >> (g.lgW + g.lgH);
                const size_t pf = ((size_t)(b * 2 * Hc + 2 * y + sy) * (2 * Wc)) + 2 * x + sx;
                out2[pf * F + c] = v > 0.f ? v : slope[c] * v;
            }
        }
    }
}

// Weight gradient of a 3x3 conv: part[chunk][tap][n][k] = sum over the chunk's
// pixels p of dout[p][n] * in[p + tap][k]  (n < CN layer out channels, k < CK
// layer in channels).  Block: one tap, one 64-wide n tile, all 64 k.
template <int CK, int CN>
__global__ void __launch_bounds__(GT) k_conv_wgrad(const float *__restrict__ in, const float *__restrict__ dout,
                                                   float *__restrict__ part, Geo g, int npix) {
    __shared__ __align__(16) float As[KC][64 + 4];  // dout: [pixel][n]
    __shared__ __align__(16) float Bs[KC][64 + 4];  // in:   [pixel][k]
    const int tap = blockIdx.y, n0 = blockIdx.z * 64, chunk = blockIdx.x;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;  // tx: n group, ty: k group
    float acc[4][4] = {};
    const int pa = chunk * WCHUNK, pb = min(npix, pa + WCHUNK);
    for (int q0 = pa; q0 < pb; q0 += KC) {
        {
            const int px = tid >> 4, c4 = (tid & 15) * 4;
            const int p = q0 + px;
            const float4 a = *reinterpret_cast<const float4 *>(dout + (size_t)p * CN + n0 + c4);
            const int q = nbr(p, g.lgH, g.lgW, dy, dx);
            const float4 b = *reinterpret_cast<const float4 *>(in + (size_t)q * CK + c4);
            *reinterpret_cast<float4 *>(&As[px][c4]) = a;
            *reinterpret_cast<float4 *>(&Bs[px][c4]) = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[kk][tx * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][ty * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    float *dst = part + (((size_t)chunk * 9 + tap) * CN) * CK;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[(size_t)(n0 + tx * 4 + i) * CK + ty * 4 + j] = acc[i][j];
}

// ---------------------------------------------------------------------------
// Tensor-core (tcgen05) forms of the two GEMM kernels above: the same
// products and epilogues, with BF16 operands (the FP32 activations and the
// FP32 master weights rounded to nearest even) and FP32 accumulation in
// tensor memory.  Eight warps per block: all gather operands into shared
// memory, one thread issues the MMAs, and warp w drains TMEM lanes
// 32 (w mod 4) .. + 31 (the hardware's lane quarter of warp w), columns
// 32 (w / 4) .. + 31 of the 64-column accumulator.  Operands use the
// no-swizzle K-major layout (core matrices of 8 rows x 16 bytes).  Every
// mbarrier wait is bounded (kWaitNs) and reports through a device flag.
// ---------------------------------------------------------------------------
constexpr int TCM = 128;                 // pixels per block: one row segment (W a multiple of 128)
constexpr int TCN = 64;                  // output channels per block
constexpr int TC_THREADS = 256;
constexpr int TC_ROWPX = TCM + 2;        // staged pixels of an input row: x0 - 1 .. x0 + 128 (periodic)
// one 8-channel plane of a staged row, [pixel][8 ch]: 130 x 16 bytes padded to
// 2192 (548 words), so the 8 planes of one pixel fall into distinct banks
constexpr int TC_PLANE = 2192;
constexpr int TC_ABYTES = 8 * TC_PLANE;  // a staged row: 64 channels
constexpr int TC_BPLANE = TCN * 16 + 16; // 8 K values of the 64 weight rows (+16 bytes: distinct banks per plane)
constexpr int TC_BTAP = 8 * TC_BPLANE;   // one tap: 64 rows (n) x 64 k
constexpr int TC_STAGE = TC_ABYTES + 3 * TC_BTAP;
constexpr size_t TC_GEMM_SMEM = 128 + 2 * TC_STAGE + 64;
constexpr int TCW_APLANE = 128 * 16;     // weight gradient: 8 pixels of the 128 rows (tap, k)
constexpr int TCW_BPLANE = 64 * 16;      // 8 pixels of the 64 rows n
constexpr int TCW_STAGE = 8 * TCW_APLANE + 8 * TCW_BPLANE;
constexpr size_t TC_WGRAD_SMEM = 128 + 2 * TCW_STAGE + 64;
static_assert(TC_STAGE % 128 == 0 && TCW_STAGE % 128 == 0 && TC_PLANE % 16 == 0 && TC_BPLANE % 16 == 0,
              "stage and plane alignment");

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Forward / data gradient of a 3x3 conv (the GEMM of k_conv_gemm, same
// operand conventions, weights pre-packed as wp[tap][n][k] in bf16 with n
// over this GEMM's CN output channels and k over its CK inputs).  Block: 128
// pixels of one row x 64 output channels.  Stage (r, slice): input row
// y + r - 1 (periodic within the sample), channels [64 slice, 64 slice + 64),
// 130 pixels x0 - 1 .. x0 + 128 staged as eight planes, and the weights of the
// three taps that read that row; the MMA for column offset c (0..2) takes the
// staged row 16 c bytes in (pixel j of output m is m + c): forward tap
// (r, c), data gradient tap (2 - r, 2 - c) (the mirrored kernel).  Two stage
// buffers alternate, so the gather of stage s + 1 overlaps the MMAs of s.
template <bool DGRAD, int CK, int CN, int EPI>
__global__ void __launch_bounds__(TC_THREADS) k_conv_gemm_tc(const float *__restrict__ in,
                                                             const __nv_bfloat16 *__restrict__ wp,
                                                             const float *__restrict__ bias,
                                                             const float *__restrict__ slope,
                                                             const float *__restrict__ skip, float *__restrict__ out,
                                                             float *__restrict__ out2, Geo g, int *err) {
    extern __shared__ __align__(16) unsigned char tc_smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)tc_smem_raw + 127) & ~(uintptr_t)127);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * TC_STAGE);  // [2]: MMAs reading stage buffer b done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p0 = blockIdx.x * TCM, n0 = blockIdx.y * TCN;
    const int W = 1 << g.lgW, H = 1 << g.lgH;
    const int x0 = p0 & (W - 1), y = (p0 >> g.lgW) & (H - 1);
    const int sample0 = p0 - (y << g.lgW) - x0;  // first pixel of this sample
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tslot, TCN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    constexpr int KS = CK / 64, S = 3 * KS;
    bool ok = true;
    int committed = -1;
    for (int s = 0; s < S; ++s) {
        const int buf = s & 1, r = s / KS, ks = s - r * KS;
        unsigned char *A = sm + buf * TC_STAGE, *Bm = A + TC_ABYTES;
        if (s >= 2 && !mbar_wait(&bar[buf], ((s - 2) >> 1) & 1)) ok = false;
        if (ok) {
            const int ry = (y + r - 1) & (H - 1);
            const float *rowp = in + ((size_t)sample0 + ((size_t)ry << g.lgW)) * CK + ks * 64;
            // item (pixel j, plane q), q fastest: 8 lanes read one pixel's 256 contiguous bytes
            for (int i = tid; i < 8 * TC_ROWPX; i += TC_THREADS) {
                const int j = i >> 3, q = i & 7;
                const int x = (x0 - 1 + j) & (W - 1);
                const float4 *src = reinterpret_cast<const float4 *>(rowp + (size_t)x * CK + 8 * q);
                const float4 u = src[0], v = src[1];
                uint4 o;
                o.x = pack_bf16x2(u.x, u.y);
                o.y = pack_bf16x2(u.z, u.w);
                o.z = pack_bf16x2(v.x, v.y);
                o.w = pack_bf16x2(v.z, v.w);
                *reinterpret_cast<uint4 *>(A + q * TC_PLANE + j * 16) = o;
            }
            // item (tap c, row n, plane q), q fastest: 8 lanes read one weight row's 128 bytes
            for (int i = tid; i < 3 * 8 * TCN; i += TC_THREADS) {
                const int q = i & 7, rest = i >> 3, n = rest % TCN, c = rest / TCN;
                const int tap = DGRAD ? (2 - r) * 3 + (2 - c) : r * 3 + c;
                const uint4 v = *reinterpret_cast<const uint4 *>(wp + ((size_t)(tap * CN + n0 + n) * CK + ks * 64 + 8 * q));
                *reinterpret_cast<uint4 *>(Bm + c * TC_BTAP + q * TC_BPLANE + n * 16) = v;
            }
        }
        fence_proxy_async();
        ok = __syncthreads_and(ok) != 0;
        if (!ok) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(Bm);
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ad = sdesc_kmajor(a0 + 16 * c + kk * 2 * TC_PLANE, TC_PLANE, 128);
                    const uint64_t bd = sdesc_kmajor(b0 + c * TC_BTAP + kk * 2 * TC_BPLANE, TC_BPLANE, 128);
                    if (s == 0 && c == 0 && kk == 0) mma_bf16<TCN, 0>(tmem, ad, bd);
                    else mma_bf16<TCN, 1>(tmem, ad, bd);
                }
            mma_commit(&bar[buf]);
        }
        committed = s;
    }
    // the last commit covers every earlier MMA of this thread
    if (committed >= 0 && !mbar_wait(&bar[committed & 1], (committed >> 1) & 1)) ok = false;
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    if (ok) {
        constexpr int NH = TCN / 2;  // columns per warp
        float v[NH];
        const int quarter = warp & 3, nh = n0 + NH * (warp >> 2);  // this warp's pixels and first channel
        tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(NH * (warp >> 2)), v);
        tmem_wait_ld();
        const int p = p0 + 32 * quarter + lane;
#pragma unroll
        for (int j = 0; j < NH; ++j) v[j] += bias ? bias[nh + j] : 0.f;
        if (EPI == EPI_SHUFFLE) {
            const int Wc = W, Hc = H;
            const int x = p & (Wc - 1), yy = (p >> g.lgW) & (Hc - 1), b = p >> (g.lgW + g.lgH);
#pragma unroll
            for (int j = 0; j < NH; j += 4)
                *reinterpret_cast<float4 *>(out + (size_t)p * CN + nh + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
#pragma unroll
            for (int j = 0; j < NH; ++j) {
                const int n = nh + j, c = n >> 2, sy = (n >> 1) & 1, sx = n & 1;
                const size_t pf = ((size_t)(b * 2 * Hc + 2 * yy + sy) * (2 * Wc)) + 2 * x + sx;
                out2[pf * F + c] = v[j] > 0.f ? v[j] : slope[c] * v[j];
            }
        } else {
#pragma unroll
            for (int j = 0; j < NH; j += 4) {
                float4 o = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                if (EPI == EPI_ADD) {
                    const float4 k4 = *reinterpret_cast<const float4 *>(skip + (size_t)p * CN + nh + j);
                    o.x += k4.x;
                    o.y += k4.y;
                    o.z += k4.z;
                    o.w += k4.w;
                }
                *reinterpret_cast<float4 *>(out + (size_t)p * CN + nh + j) = o;
                if (EPI == EPI_PRELU) {
                    const float4 a4 = make_float4(o.x > 0.f ? o.x : slope[nh + j] * o.x,
                                                  o.y > 0.f ? o.y : slope[nh + j + 1] * o.y,
                                                  o.z > 0.f ? o.z : slope[nh + j + 2] * o.z,
                                                  o.w > 0.f ? o.w : slope[nh + j + 3] * o.w);
                    *reinterpret_cast<float4 *>(out2 + (size_t)p * CN + nh + j) = a4;
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCN);
}

// Weight gradient on the tensor cores: part[chunk][tap][n][k] = sum over the
// chunk's pixels p of dout[p][n] in[p + tap][k] (the partials k_conv_wgrad
// writes, summed by k_wgrad_reduce), for a layer with 64 input channels.
// Block: one chunk, a pair of taps (t0, t0 + 1; tap 9 is empty), 64 output
// channels.  D (128 x 64) has rows (tap of the pair, k) and columns n; K runs
// over the chunk's pixels, 64 per stage (64 consecutive pixels of one row):
// A[(t, k)][j] = in[p_j + tap_t][k] and B[n][j] = dout[p_j][n], transposed
// into K-major core matrices by the gathering threads (a warp's lanes read 32
// consecutive channels of one pixel and write 32 consecutive 16-byte rows).
template <int CN>
__global__ void __launch_bounds__(TC_THREADS) k_conv_wgrad_tc(const float *__restrict__ in,
                                                              const float *__restrict__ dout,
                                                              float *__restrict__ part, Geo g, int *err) {
    constexpr int CK = F;
    extern __shared__ __align__(16) unsigned char tc_smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)tc_smem_raw + 127) & ~(uintptr_t)127);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * TCW_STAGE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chunk = blockIdx.x, t0 = 2 * blockIdx.y, n0 = blockIdx.z * 64;
    const int W = 1 << g.lgW, H = 1 << g.lgH;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(tslot, 64);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    // this thread's A row m = tid & 127 = (tap of the pair, k), planes 4 (tid >> 7) .. + 3;
    // B row n = tid & 63, planes (tid >> 6) and (tid >> 6) + 4
    const int ma = tid & 127, qa = 4 * (tid >> 7);
    const int tap = t0 + (ma >> 6), ka = ma & 63, nb = tid & 63, qb = tid >> 6;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    constexpr int S = WCHUNK_TC / 64;
    bool ok = true;
    int committed = -1;
    for (int s = 0; s < S; ++s) {
        const int buf = s & 1;
        unsigned char *A = sm + buf * TCW_STAGE, *Bm = A + 8 * TCW_APLANE;
        if (s >= 2 && !mbar_wait(&bar[buf], ((s - 2) >> 1) & 1)) ok = false;
        if (ok) {
            const int pst = chunk * WCHUNK_TC + s * 64;  // 64 pixels of one row
            const int xs = pst & (W - 1), yr = (pst >> g.lgW) & (H - 1);
            const int smp = pst - (yr << g.lgW) - xs;
            if (tap < 9) {
                const float *rowp = in + ((size_t)smp + ((size_t)((yr + dy) & (H - 1)) << g.lgW)) * CK + ka;
#pragma unroll 2
                for (int q = qa; q < qa + 4; ++q) {
                    float v[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] = rowp[(size_t)((xs + 8 * q + i + dx) & (W - 1)) * CK];
                    uint4 o;
                    o.x = pack_bf16x2(v[0], v[1]);
                    o.y = pack_bf16x2(v[2], v[3]);
                    o.z = pack_bf16x2(v[4], v[5]);
                    o.w = pack_bf16x2(v[6], v[7]);
                    *reinterpret_cast<uint4 *>(A + q * TCW_APLANE + ma * 16) = o;
                }
            } else {
#pragma unroll
                for (int q = qa; q < qa + 4; ++q)
                    *reinterpret_cast<uint4 *>(A + q * TCW_APLANE + ma * 16) = make_uint4(0, 0, 0, 0);
            }
            const float *dp = dout + (size_t)pst * CN + n0 + nb;
#pragma unroll
            for (int i2 = 0; i2 < 2; ++i2) {
                const int q = qb + 4 * i2;
                float v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = dp[(size_t)(8 * q + i) * CN];
                uint4 o;
                o.x = pack_bf16x2(v[0], v[1]);
                o.y = pack_bf16x2(v[2], v[3]);
                o.z = pack_bf16x2(v[4], v[5]);
                o.w = pack_bf16x2(v[6], v[7]);
                *reinterpret_cast<uint4 *>(Bm + q * TCW_BPLANE + nb * 16) = o;
            }
        }
        fence_proxy_async();
        ok = __syncthreads_and(ok) != 0;
        if (!ok) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(Bm);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = sdesc_kmajor(a0 + kk * 2 * TCW_APLANE, TCW_APLANE, 128);
                const uint64_t bd = sdesc_kmajor(b0 + kk * 2 * TCW_BPLANE, TCW_BPLANE, 128);
                if (s == 0 && kk == 0) mma_bf16<64, 0>(tmem, ad, bd);
                else mma_bf16<64, 1>(tmem, ad, bd);
            }
            mma_commit(&bar[buf]);
        }
        committed = s;
    }
    if (committed >= 0 && !mbar_wait(&bar[committed & 1], (committed >> 1) & 1)) ok = false;
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    if (ok) {
        float v[32];
        const int quarter = warp & 3, nh = 32 * (warp >> 2);
        tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)nh, v);
        tmem_wait_ld();
        const int m = 32 * quarter + lane, tr = t0 + (m >> 6), k = m & 63;
        if (tr < 9) {
            float *dst = part + (((size_t)chunk * 9 + tr) * CN + n0 + nh) * CK + k;
#pragma unroll
            for (int n = 0; n < 32; ++n) dst[(size_t)n * CK] = v[n];
        }
    } else if (tid == 0) {
        atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 64);
}

// bf16 copies of one conv layer's weights w[(n CK + k) 9 + tap] (n < CN out,
// k < CK in) for the tensor-core GEMMs: wf[tap][n][k] (forward) and
// wd[tap][k][n] (data gradient, whose outputs are the layer's inputs).
__global__ void k_pack_tc(const float *__restrict__ w, int CN, int CK, __nv_bfloat16 *__restrict__ wf,
                          __nv_bfloat16 *__restrict__ wd) {
    const int total = 9 * CN * CK;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int tap = e / (CN * CK), rem = e - tap * CN * CK, n = rem / CK, k = rem - n * CK;
        const __nv_bfloat16 h = __float2bfloat16_rn(w[((size_t)n * CK + k) * 9 + tap]);
        wf[e] = h;
        wd[((size_t)tap * CK + k) * CN + n] = h;
    }
}

// grad[(n * CK + k) * 9 + tap] = sum over chunks (in order) of part[chunk][tap][n][k].
__global__ void k_wgrad_reduce(const float *__restrict__ part, float *__restrict__ grad, int CK, int CN,
                               int nchunk) {
    const int total = 9 * CN * CK;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int tap = e % 9, nk = e / 9, n = nk / CK, k = nk - n * CK;
        float s = 0.f;
        for (int c = 0; c < nchunk; ++c) s += part[(((size_t)c * 9 + tap) * CN + n) * CK + k];
        grad[e] = s;
    }
}

// Per-channel sums over pixels, two stages: part[block][c] then out[c].
// v(p, c) = a[p][c] * (mode 0: 1;  mode 1: z[p][c] <= 0 ? z[p][c] : 0).
// Block: pixels [blockIdx.x * RCHUNK, +RCHUNK); with C a multiple of 4 a
// thread takes 4 consecutive channels (16-byte loads) of every (256 / (C / 4))-th
// pixel, else one channel; the pixel lanes are then summed in lane order.
__global__ void k_chan_partial(const float *__restrict__ a, const float *__restrict__ z, int C, int npix,
                               int mode, float *__restrict__ part) {
    extern __shared__ float sh[];  // blockDim.x * 4 floats
    const int pa = blockIdx.x * RCHUNK, pb = min(npix, pa + RCHUNK);
    if ((C & 3) == 0) {
        const int Q = C >> 2, lanes = blockDim.x / Q;
        const int qd = threadIdx.x % Q, l = threadIdx.x / Q;
        float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (l < lanes) {
            for (int p = pa + l; p < pb; p += lanes) {
                float4 v = *reinterpret_cast<const float4 *>(a + (size_t)p * C + 4 * qd);
                if (mode != 0) {
                    const float4 zz = *reinterpret_cast<const float4 *>(z + (size_t)p * C + 4 * qd);
                    v.x = zz.x <= 0.f ? v.x * zz.x : 0.f;
                    v.y = zz.y <= 0.f ? v.y * zz.y : 0.f;
                    v.z = zz.z <= 0.f ? v.z * zz.z : 0.f;
                    v.w = zz.w <= 0.f ? v.w * zz.w : 0.f;
                }
                s4.x += v.x;
                s4.y += v.y;
                s4.z += v.z;
                s4.w += v.w;
            }
        }
        reinterpret_cast<float4 *>(sh)[threadIdx.x] = s4;
        __syncthreads();
        for (int c = threadIdx.x; c < C; c += blockDim.x) {
            float t = 0.f;
            for (int i = 0; i < lanes; ++i) t += sh[(i * Q + (c >> 2)) * 4 + (c & 3)];
            part[(size_t)blockIdx.x * C + c] = t;
        }
        return;
    }
    const int lanes = blockDim.x / C;
    const int c = threadIdx.x % C, l = threadIdx.x / C;
    float s = 0.f;
    for (int p = pa + l; p < pb; p += lanes) {
        const float v = a[(size_t)p * C + c];
        if (mode == 0) s += v;
        else {
            const float zz = z[(size_t)p * C + c];
            s += zz <= 0.f ? v * zz : 0.f;
        }
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    if (l == 0) {
        float t = 0.f;
        for (int i = 0; i < lanes; ++i) t += sh[i * C + c];
        part[(size_t)blockIdx.x * C + c] = t;
    }
}

// out[e] = sum over chunks of part[chunk][e] (e < m): a warp per element, its
// lanes summing chunks lane, lane + 32, ... in order, then a fixed shuffle
// tree (deterministic).
__global__ void k_sum_chunks(const float *__restrict__ part, int m, int nchunk, float *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < m; e += (gridDim.x * blockDim.x) >> 5) {
        float s = 0.f;
        for (int c = lane; c < nchunk; c += 32) s += part[(size_t)c * m + e];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[e] = s;
    }
}

// dz = da * PReLU'(z), elementwise over n values of C channels (in place allowed: dz may be da)
__global__ void k_prelu_back(const float *__restrict__ da, const float *__restrict__ z,
                             const float *__restrict__ slope, int C, size_t n, float *__restrict__ dz) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        dz[e] = z[e] > 0.f ? da[e] : slope[c] * da[e];
    }
}

// Fine gradient daf [fine pixel][F] -> coarse dzu [pixel][4F] through PReLU' and the shuffle.
// zf holds the fine pre-activation re-read from zu.
__global__ void k_shuffle_back(const float *__restrict__ daf, const float *__restrict__ zu,
                               const float *__restrict__ slope, float *__restrict__ dzu, Geo g, size_t npix) {
    const size_t n = npix * 4 * F;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int ch = (int)(e % (4 * F));
        const size_t p = e / (4 * F);
        const int c = ch >> 2, sy = (ch >> 1) & 1, sx = ch & 1;
        const int Wc = 1 << g.lgW, Hc = 1 << g.lgH;
        const int x = (int)(p & (Wc - 1)), y = (int)((p >> g.lgW) & (Hc - 1)), b = (int)(p >> (g.lgW + g.lgH));
        const size_t pf = ((size_t)(b * 2 * Hc + 2 * y + sy) * (2 * Wc)) + 2 * x + sx;
        const float z = zu[e], d = daf[pf * F + c];
        dzu[e] = z > 0.f ? d : slope[c] * d;
    }
}

// Slope gradient of the shuffled PReLU: part[block][c] = sum daf[pf][c] * zf[pf][c] over zf <= 0.
__global__ void k_shuffle_slope_partial(const float *__restrict__ daf, const float *__restrict__ zu, Geo g,
                                        int npix_f, float *__restrict__ part) {
    extern __shared__ float sh[];
    const int lanes = blockDim.x / F;
    const int c = threadIdx.x % F, l = threadIdx.x / F;
    const int pa = blockIdx.x * RCHUNK, pb = min(npix_f, pa + RCHUNK);
    const int Wf = 2 << g.lgW, Hf = 2 << g.lgH;
    float s = 0.f;
    for (int pf = pa + l; pf < pb; pf += lanes) {
        const int xf = pf & (Wf - 1), yf = (pf >> (g.lgW + 1)) & (Hf - 1), b = pf >> (g.lgW + g.lgH + 2);
        const int p = ((b << g.lgH) + (yf >> 1)) * (Wf >> 1) + (xf >> 1);
        const float z = zu[(size_t)p * 4 * F + 4 * c + 2 * (yf & 1) + (xf & 1)];
        s += z <= 0.f ? daf[(size_t)pf * F + c] * z : 0.f;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    if (l == 0) {
        float t = 0.f;
        for (int i = 0; i < lanes; ++i) t += sh[i * F + c];
        part[(size_t)blockIdx.x * F + c] = t;
    }
}

// First layer (1 -> F): z0[p][c] = b[c] + sum_tap w[c][tap] q[p + tap]; x0 = PReLU(z0).
__global__ void k_conv_in(const float *__restrict__ q, const float *__restrict__ w, const float *__restrict__ b,
                          const float *__restrict__ slope, float *__restrict__ z, float *__restrict__ a, Geo g,
                          size_t npix) {
    const size_t n = npix * F;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % F);
        const int p = (int)(e / F);
        float s = b[c];
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) s = fmaf(w[c * 9 + tap], q[nbr(p, g.lgH, g.lgW, tap / 3 - 1, tap % 3 - 1)], s);
        z[e] = s;
        a[e] = s > 0.f ? s : slope[c] * s;
    }
}

// Weight gradient of the first layer: part[chunk][c][tap] = sum dz[p][c] q[p + tap].
__global__ void k_conv_in_wgrad(const float *__restrict__ q, const float *__restrict__ dz, Geo g, int npix,
                                float *__restrict__ part) {
    // block: F channels x 4 lanes; pixel chunk blockIdx.x
    __shared__ float sh[4][F][9];
    const int c = threadIdx.x % F, l = threadIdx.x / F;
    const int pa = blockIdx.x * RCHUNK, pb = min(npix, pa + RCHUNK);
    float s[9] = {};
    for (int p = pa + l; p < pb; p += 4) {
        const float d = dz[(size_t)p * F + c];
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) s[tap] = fmaf(d, q[nbr(p, g.lgH, g.lgW, tap / 3 - 1, tap % 3 - 1)], s[tap]);
    }
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) sh[l][c][tap] = s[tap];
    __syncthreads();
    if (l == 0)
        for (int tap = 0; tap < 9; ++tap)
            part[((size_t)blockIdx.x * F + c) * 9 + tap] = ((sh[0][c][tap] + sh[1][c][tap]) + sh[2][c][tap]) + sh[3][c][tap];
}

// Last layer (F -> 1) at the fine grid: y[p] = b + sum_{tap, c} w[c][tap] u[p + tap][c].  Warp per pixel.
__global__ void k_conv_out(const float *__restrict__ u, const float *__restrict__ w, const float *__restrict__ b,
                           float *__restrict__ y, Geo gf, int npix_f) {
    const int lane = threadIdx.x & 31;
    for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < npix_f; p += (gridDim.x * blockDim.x) >> 5) {
        float s = 0.f;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int q = nbr(p, gf.lgH, gf.lgW, tap / 3 - 1, tap % 3 - 1);
            s = fmaf(w[lane * 9 + tap], u[(size_t)q * F + lane], s);
            s = fmaf(w[(lane + 32) * 9 + tap], u[(size_t)q * F + lane + 32], s);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) y[p] = s + b[0];
    }
}

// Loss and its gradient: dy = 2 mask (y - t) / count; part[block] = sum mask (y - t)^2.
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, const float *__restrict__ mask,
                      float inv_count, int n, float *__restrict__ dy, float *__restrict__ part) {
    __shared__ float sh[RT];
    float s = 0.f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float m = mask ? mask[p] : 1.f;
        const float d = m * (y[p] - t[p]);
        dy[p] = 2.f * d * inv_count;
        s = fmaf(d, y[p] - t[p], s);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Data gradient of the last layer: du[p][c] = sum_tap w[c][tap] dy[p - tap].
__global__ void k_conv_out_dgrad(const float *__restrict__ dy, const float *__restrict__ w,
                                 float *__restrict__ du, Geo gf, size_t npix_f) {
    const size_t n = npix_f * F;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % F);
        const int p = (int)(e / F);
        float s = 0.f;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) s = fmaf(w[c * 9 + tap], dy[nbr(p, gf.lgH, gf.lgW, 1 - tap / 3, 1 - tap % 3)], s);
        du[e] = s;
    }
}

// Weight gradient of the last layer: part[chunk][c][tap] = sum dy[p] u[p + tap][c].
__global__ void k_conv_out_wgrad(const float *__restrict__ u, const float *__restrict__ dy, Geo gf, int npix_f,
                                 float *__restrict__ part) {
    __shared__ float sh[4][F][9];
    const int c = threadIdx.x % F, l = threadIdx.x / F;
    const int pa = blockIdx.x * RCHUNK, pb = min(npix_f, pa + RCHUNK);
    float s[9] = {};
    for (int p = pa + l; p < pb; p += 4) {
        const float d = dy[p];
#pragma unroll
        for (int tap = 0; tap < 9; ++tap)
            s[tap] = fmaf(d, u[(size_t)nbr(p, gf.lgH, gf.lgW, tap / 3 - 1, tap % 3 - 1) * F + c], s[tap]);
    }
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) sh[l][c][tap] = s[tap];
    __syncthreads();
    if (l == 0)
        for (int tap = 0; tap < 9; ++tap)
            part[((size_t)blockIdx.x * F + c) * 9 + tap] = ((sh[0][c][tap] + sh[1][c][tap]) + sh[2][c][tap]) + sh[3][c][tap];
}


__global__ void k_add(float *__restrict__ a, const float *__restrict__ b, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        a[e] += b[e];
}

// Adam (Kingma and Ba, 2015) with bias correction folded into the step size.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, size_t n, float lr_t, float b1, float b2, float eps) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float me = b1 * m[e] + (1.f - b1) * ge;
        const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
        m[e] = me;
        v[e] = ve;
        p[e] -= lr_t * me / (sqrtf(ve) + eps);
    }
}

int grid_for(size_t n, int threads = RT) {
    size_t b = (n + threads - 1) / threads;
    return (int)(b < 4096 ? (b ? b : 1) : 4096);
}

}  // namespace

// ---------------------------------------------------------------------------
// Trainer state
// ---------------------------------------------------------------------------
struct Trainer {
    Geo g, gf;
    int nb = 8;
    int npix = 0, npix_f = 0, nchunk = 0, nchunk_tc = 0, nchunk_r = 0, nchunk_rf = 0;
    size_t nparam = 0;
    // parameter offsets (floats) in blob order
    size_t o_in_w, o_in_b, o_in_a, o_up_w, o_up_b, o_up_a, o_out_w, o_out_b;
    std::vector<size_t> o_w1, o_b1, o_a, o_w2, o_b2;
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    // activations
    float *z0 = nullptr;
    std::vector<float *> xs, z1, a1;  // xs[0..nb]
    float *zu = nullptr, *af = nullptr, *y = nullptr;
    // gradients
    float *dx = nullptr, *dx2 = nullptr, *da = nullptr, *dzu = nullptr, *daf = nullptr, *dy = nullptr;
    float *part = nullptr, *lpart = nullptr, *hloss = nullptr;
    // tensor-core GEMMs: bf16 copies of the 64/256-channel conv weights,
    // packed per step (forward wf, data gradient wd; offsets per layer)
    bool tc = false;
    __nv_bfloat16 *wf = nullptr, *wd = nullptr;
    std::vector<size_t> po_w1, po_w2;
    size_t po_up = 0;
    int *d_err = nullptr;  // set by a tensor-core kernel whose bounded wait ran out
    int steps = 0;
    float lr = 1e-4f, b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    std::vector<void *> allocs;
};

namespace {

size_t layout(Trainer *t) {
    size_t o = 0;
    t->o_in_w = o; o += F * 9;
    t->o_in_b = o; o += F;
    t->o_in_a = o; o += F;
    t->o_w1.resize(t->nb); t->o_b1.resize(t->nb); t->o_a.resize(t->nb); t->o_w2.resize(t->nb); t->o_b2.resize(t->nb);
    for (int k = 0; k < t->nb; ++k) {
        t->o_w1[k] = o; o += (size_t)F * F * 9;
        t->o_b1[k] = o; o += F;
        t->o_a[k] = o; o += F;
        t->o_w2[k] = o; o += (size_t)F * F * 9;
        t->o_b2[k] = o; o += F;
    }
    t->o_up_w = o; o += (size_t)4 * F * F * 9;
    t->o_up_b = o; o += 4 * F;
    t->o_up_a = o; o += F;
    t->o_out_w = o; o += F * 9;
    t->o_out_b = o; o += 1;
    return o;
}

cudaError_t talloc(Trainer *t, float **p, size_t n) {
    cudaError_t e = cudaMalloc(p, n * sizeof(float));
    if (e == cudaSuccess) t->allocs.push_back(*p);
    return e;
}

#define TR_CK(x)                              \
    do {                                      \
        cudaError_t e_ = (x);                 \
        if (e_ != cudaSuccess) return e_;     \
    } while (0)

// One conv GEMM (forward or data gradient): on the tensor cores from the
// packed bf16 weights wpk when the trainer uses them, else in FP32 from w.
template <bool DGRAD, int CK, int CN, int EPI>
cudaError_t gemm(Trainer *t, const float *in, const float *w, const __nv_bfloat16 *wpk, const float *bias,
                 const float *slope, const float *skip, float *out, float *out2, cudaStream_t s) {
    constexpr int NOUT = CN;
    if (t->tc) {
        auto k = k_conv_gemm_tc<DGRAD, CK, CN, EPI>;
        static std::atomic<bool> attr{false};
        if (!attr.load()) {
            TR_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_GEMM_SMEM));
            attr.store(true);
        }
        dim3 grid(t->npix / TCM, NOUT / TCN);
        k<<<grid, TC_THREADS, TC_GEMM_SMEM, s>>>(in, wpk, bias, slope, skip, out, out2, t->g, t->d_err);
        count_launches(1);
        return cudaGetLastError();
    }
    dim3 grid(t->npix / TP, NOUT / 64);
    k_conv_gemm<DGRAD, CK, CN, EPI><<<grid, GT, 0, s>>>(in, w, bias, slope, skip, out, out2, t->g);
    count_launches(1);
    return cudaGetLastError();
}

template <int CK, int CN>
cudaError_t wgrad(Trainer *t, const float *in, const float *dout, float *grad, cudaStream_t s) {
    if (t->tc) {
        static_assert(CK == F, "tensor-core weight gradient: 64 input channels");
        auto k = k_conv_wgrad_tc<CN>;
        static std::atomic<bool> attr{false};
        if (!attr.load()) {
            TR_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_WGRAD_SMEM));
            attr.store(true);
        }
        dim3 grid(t->nchunk_tc, 5, CN / 64);
        k<<<grid, TC_THREADS, TC_WGRAD_SMEM, s>>>(in, dout, t->part, t->g, t->d_err);
    } else {
        dim3 grid(t->nchunk, 9, CN / 64);
        k_conv_wgrad<CK, CN><<<grid, GT, 0, s>>>(in, dout, t->part, t->g, t->npix);
    }
    k_wgrad_reduce<<<grid_for((size_t)9 * CN * CK), RT, 0, s>>>(t->part, grad, CK, CN,
                                                                t->tc ? t->nchunk_tc : t->nchunk);
    count_launches(2);
    return cudaGetLastError();
}

// bf16 forward and data-gradient copies of every 64/256-channel conv layer
cudaError_t pack_weights(Trainer *t, cudaStream_t s) {
    const float *P = t->P;
    auto pack = [&](size_t o_w, size_t po, int CN, int CK) {
        k_pack_tc<<<grid_for((size_t)9 * CN * CK), RT, 0, s>>>(P + o_w, CN, CK, t->wf + po, t->wd + po);
        count_launches(1);
    };
    for (int k = 0; k < t->nb; ++k) {
        pack(t->o_w1[k], t->po_w1[k], F, F);
        pack(t->o_w2[k], t->po_w2[k], F, F);
    }
    pack(t->o_up_w, t->po_up, 4 * F, F);
    return cudaGetLastError();
}

// per-channel sum of a (mode 0) or slope gradient (mode 1) over the coarse pixels
cudaError_t chan_sum(Trainer *t, const float *a, const float *z, int C, int mode, float *out, cudaStream_t s) {
    k_chan_partial<<<t->nchunk_r, RT, 4 * RT * sizeof(float), s>>>(a, z, C, t->npix, mode, t->part);
    k_sum_chunks<<<grid_for((size_t)C * 32), RT, 0, s>>>(t->part, C, t->nchunk_r, out);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace

// Forward pass of the whole batch; q: [B][H][W].
cudaError_t train_forward(Trainer *t, const float *q, cudaStream_t s) {
    float *P = t->P;
    if (t->tc) TR_CK(pack_weights(t, s));
    k_conv_in<<<grid_for((size_t)t->npix * F), RT, 0, s>>>(q, P + t->o_in_w, P + t->o_in_b, P + t->o_in_a, t->z0,
                                                          t->xs[0], t->g, t->npix);
    count_launches(1);
    TR_CK(cudaGetLastError());
    for (int k = 0; k < t->nb; ++k) {
        TR_CK((gemm<false, F, F, EPI_PRELU>(t, t->xs[k], P + t->o_w1[k], t->wf + t->po_w1[k], P + t->o_b1[k],
                                            P + t->o_a[k], nullptr,
                                            t->z1[k], t->a1[k], s)));
        TR_CK((gemm<false, F, F, EPI_ADD>(t, t->a1[k], P + t->o_w2[k], t->wf + t->po_w2[k], P + t->o_b2[k], nullptr,
                                          t->xs[k],
                                          t->xs[k + 1], nullptr, s)));
    }
    TR_CK((gemm<false, F, 4 * F, EPI_SHUFFLE>(t, t->xs[t->nb], P + t->o_up_w, t->wf + t->po_up, P + t->o_up_b,
                                              P + t->o_up_a,
                                              nullptr, t->zu, t->af, s)));
    k_conv_out<<<grid_for((size_t)t->npix_f * 32), RT, 0, s>>>(t->af, P + t->o_out_w, P + t->o_out_b, t->y, t->gf,
                                                             t->npix_f);
    count_launches(1);
    return cudaGetLastError();
}

// Loss, gradient of every parameter into t->G (blob order); loss sum to t->lpart[0..].
cudaError_t train_backward(Trainer *t, const float *q, const float *target, const float *mask, float inv_count,
                           cudaStream_t s) {
    float *P = t->P, *G = t->G;
    const int nl = 256;
    k_mse<<<nl, RT, 0, s>>>(t->y, target, mask, inv_count, t->npix_f, t->dy, t->lpart);
    count_launches(1);
    TR_CK(cudaGetLastError());
    // last layer
    k_conv_out_wgrad<<<t->nchunk_rf, RT, 0, s>>>(t->af, t->dy, t->gf, t->npix_f, t->part);
    k_sum_chunks<<<grid_for((size_t)F * 9 * 32), RT, 0, s>>>(t->part, F * 9, t->nchunk_rf, G + t->o_out_w);
    count_launches(2);
    {   // out bias = sum dy: reuse the channel reduction with C = 1 over fine pixels
        k_chan_partial<<<t->nchunk_rf, RT, 4 * RT * sizeof(float), s>>>(t->dy, nullptr, 1, t->npix_f, 0, t->part);
        k_sum_chunks<<<1, RT, 0, s>>>(t->part, 1, t->nchunk_rf, G + t->o_out_b);
        count_launches(2);
    }
    k_conv_out_dgrad<<<grid_for((size_t)t->npix_f * F), RT, 0, s>>>(t->dy, P + t->o_out_w, t->daf, t->gf, t->npix_f);
    // up layer: slope gradient, then dzu through the shuffle and PReLU'
    k_shuffle_slope_partial<<<t->nchunk_rf, RT, RT * sizeof(float), s>>>(t->daf, t->zu, t->g, t->npix_f, t->part);
    k_sum_chunks<<<grid_for((size_t)F * 32), RT, 0, s>>>(t->part, F, t->nchunk_rf, G + t->o_up_a);
    k_shuffle_back<<<grid_for((size_t)t->npix * 4 * F), RT, 0, s>>>(t->daf, t->zu, P + t->o_up_a, t->dzu, t->g,
                                                                   t->npix);
    count_launches(4);
    TR_CK(cudaGetLastError());
    TR_CK((wgrad<F, 4 * F>(t, t->xs[t->nb], t->dzu, G + t->o_up_w, s)));
    TR_CK(chan_sum(t, t->dzu, nullptr, 4 * F, 0, G + t->o_up_b, s));
    TR_CK((gemm<true, 4 * F, F, EPI_RAW>(t, t->dzu, P + t->o_up_w, t->wd + t->po_up, nullptr, nullptr, nullptr, t->dx,
                                         nullptr, s)));
    // residual blocks, last to first; t->dx = gradient w.r.t. the block output
    for (int k = t->nb - 1; k >= 0; --k) {
        // conv2: input a1, output grad dx
        TR_CK((wgrad<F, F>(t, t->a1[k], t->dx, G + t->o_w2[k], s)));
        TR_CK(chan_sum(t, t->dx, nullptr, F, 0, G + t->o_b2[k], s));
        TR_CK((gemm<true, F, F, EPI_RAW>(t, t->dx, P + t->o_w2[k], t->wd + t->po_w2[k], nullptr, nullptr, nullptr,
                                         t->da, nullptr, s)));
        // PReLU: slope gradient, then da -> dz1 (in place)
        TR_CK(chan_sum(t, t->da, t->z1[k], F, 1, G + t->o_a[k], s));
        k_prelu_back<<<grid_for((size_t)t->npix * F), RT, 0, s>>>(t->da, t->z1[k], P + t->o_a[k], F,
                                                                (size_t)t->npix * F, t->da);
        count_launches(1);
        // conv1: input xs[k], output grad da (= dz1)
        TR_CK((wgrad<F, F>(t, t->xs[k], t->da, G + t->o_w1[k], s)));
        TR_CK(chan_sum(t, t->da, nullptr, F, 0, G + t->o_b1[k], s));
        TR_CK((gemm<true, F, F, EPI_RAW>(t, t->da, P + t->o_w1[k], t->wd + t->po_w1[k], nullptr, nullptr, nullptr,
                                         t->dx2, nullptr, s)));
        k_add<<<grid_for((size_t)t->npix * F), RT, 0, s>>>(t->dx, t->dx2, (size_t)t->npix * F);  // skip path
        count_launches(1);
        TR_CK(cudaGetLastError());
    }
    // first layer: PReLU then weights
    TR_CK(chan_sum(t, t->dx, t->z0, F, 1, G + t->o_in_a, s));
    k_prelu_back<<<grid_for((size_t)t->npix * F), RT, 0, s>>>(t->dx, t->z0, P + t->o_in_a, F, (size_t)t->npix * F,
                                                            t->dx);
    k_conv_in_wgrad<<<t->nchunk_r, RT, 0, s>>>(q, t->dx, t->g, t->npix, t->part);
    k_sum_chunks<<<grid_for((size_t)F * 9 * 32), RT, 0, s>>>(t->part, F * 9, t->nchunk_r, G + t->o_in_w);
    count_launches(3);
    TR_CK(chan_sum(t, t->dx, nullptr, F, 0, G + t->o_in_b, s));
    return cudaGetLastError();
}

}  // namespace mg

using mg::Trainer;

namespace {
thread_local char g_terr[256];
mg_status terr(mg_status st, const char *msg) {
    snprintf(g_terr, sizeof g_terr, "%s", msg);
    mg::set_last_error(g_terr);
    return st;
}
mg_status tcuda(cudaError_t e, const char *where) {
    snprintf(g_terr, sizeof g_terr, "%s: %s", where, cudaGetErrorString(e));
    cudaGetLastError();
    mg::set_last_error(g_terr);
    return MG_ERR_CUDA;
}
bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}
}  // namespace

struct mg_trainer : Trainer {};

// MG_ERR_TIMEOUT (and the flag cleared) when a tensor-core kernel's bounded
// wait ran out during the last pass; call after the pass has completed.
static mg_status trainer_check_flag(mg_trainer *t) {
    int f = 0;
    cudaError_t e = cudaMemcpy(&f, t->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return tcuda(e, "trainer status flag");
    if (f) {
        cudaMemset(t->d_err, 0, sizeof(int));
        return terr(MG_ERR_TIMEOUT, "a tensor-core training kernel timed out waiting for its MMAs");
    }
    return MG_OK;
}

extern "C" {

mg_status mg_trainer_create(int H, int W, int batch, const void *blob, size_t bytes, double lr,
                            mg_trainer **out) {
    if (out) *out = nullptr;
    if (!out || !blob || !pow2(H) || !pow2(W) || H < 8 || W < 8 || batch < 1 || !(lr > 0.0) ||
        ((size_t)batch * H * W) % 2048 != 0 || (size_t)batch * H * W > (1u << 24))
        return terr(MG_ERR_INVALID_ARG,
                    "mg_trainer_create: H, W powers of two >= 8, batch * H * W a multiple of 2048 "
                    "(at most 2^24), lr > 0, blob not null");
    const unsigned char *b = (const unsigned char *)blob;
    if (bytes < 64 || memcmp(b, "MGSRW001", 8) != 0) return terr(MG_ERR_BAD_WEIGHTS, "bad weight blob header");
    uint32_t nf, nbk, np;
    memcpy(&nf, b + 8, 4);
    memcpy(&nbk, b + 12, 4);
    memcpy(&np, b + 16, 4);
    mg_trainer *t = new (std::nothrow) mg_trainer();
    if (!t) return MG_ERR_OOM;
    t->nb = (int)nbk;
    const size_t n = mg::layout(t);
    if (nf != 64 || nbk < 1 || nbk > 32 || np != n || bytes != 64 + 4ull * n) {
        delete t;
        return terr(MG_ERR_BAD_WEIGHTS, "weight blob does not match the generator layout");
    }
    t->nparam = n;
    t->g = mg::Geo{H, W, ilog2(H), ilog2(W), batch};
    t->gf = mg::Geo{2 * H, 2 * W, ilog2(H) + 1, ilog2(W) + 1, batch};
    t->npix = batch * H * W;
    t->npix_f = 4 * t->npix;
    t->nchunk = t->npix / mg::WCHUNK;  // npix is a multiple of WCHUNK, so every chunk is full
    t->nchunk_tc = t->npix / mg::WCHUNK_TC;
    t->nchunk_r = t->npix / mg::RCHUNK;
    t->nchunk_rf = t->npix_f / mg::RCHUNK;
    t->lr = (float)lr;
    const size_t A = (size_t)t->npix * mg::F;
    cudaError_t e = cudaSuccess;
    auto al = [&](float **p, size_t cnt) {
        if (e == cudaSuccess) e = mg::talloc(t, p, cnt);
    };
    al(&t->P, n);
    al(&t->G, n);
    al(&t->M, n);
    al(&t->V, n);
    al(&t->z0, A);
    t->xs.assign(t->nb + 1, nullptr);
    t->z1.assign(t->nb, nullptr);
    t->a1.assign(t->nb, nullptr);
    for (int k = 0; k <= t->nb; ++k) al(&t->xs[k], A);
    for (int k = 0; k < t->nb; ++k) {
        al(&t->z1[k], A);
        al(&t->a1[k], A);
    }
    al(&t->zu, 4 * A);
    al(&t->af, 4 * A);
    al(&t->y, (size_t)t->npix_f);
    al(&t->dx, A);
    al(&t->dx2, A);
    al(&t->da, A);
    al(&t->dzu, 4 * A);
    al(&t->daf, 4 * A);
    al(&t->dy, (size_t)t->npix_f);
    al(&t->part, std::max({(size_t)t->nchunk_tc * 9 * 4 * mg::F * mg::F, (size_t)t->nchunk_rf * mg::F * 9,
                           (size_t)t->nchunk_r * 4 * mg::F}));
    al(&t->lpart, 512);
    // tensor-core GEMMs: the default whenever a coarse row holds whole
    // 128-pixel tiles (mg_trainer_set_tensor_cores switches them off)
    t->tc = (W % mg::TCM) == 0;
    size_t npk = 0;
    t->po_w1.assign(t->nb, 0);
    t->po_w2.assign(t->nb, 0);
    for (int k = 0; k < t->nb; ++k) {
        t->po_w1[k] = npk;
        npk += (size_t)9 * mg::F * mg::F;
        t->po_w2[k] = npk;
        npk += (size_t)9 * mg::F * mg::F;
    }
    t->po_up = npk;
    npk += (size_t)9 * 4 * mg::F * mg::F;
    auto alb = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) {
            e = cudaMalloc(p, bytes);
            if (e == cudaSuccess) t->allocs.push_back(*p);
        }
    };
    alb((void **)&t->wf, npk * sizeof(__nv_bfloat16));
    alb((void **)&t->wd, npk * sizeof(__nv_bfloat16));
    alb((void **)&t->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(t->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(t->P, b + 64, 4 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(t->M, 0, 4 * n);
    if (e == cudaSuccess) e = cudaMemset(t->V, 0, 4 * n);
    if (e == cudaSuccess) e = cudaMallocHost(&t->hloss, 256 * sizeof(float));
    if (e != cudaSuccess) {
        mg_trainer_destroy(t);
        return tcuda(e, "mg_trainer_create");
    }
    *out = t;
    return MG_OK;
}

mg_status mg_trainer_forward(mg_trainer *t, const float *q, float *y) {
    if (!t || !q || !y) return terr(MG_ERR_INVALID_ARG, "null trainer or pointer");
    cudaError_t e = mg::train_forward(t, q, 0);
    if (e == cudaSuccess) e = cudaMemcpy(y, t->y, sizeof(float) * t->npix_f, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) return tcuda(e, "mg_trainer_forward");
    return trainer_check_flag(t);
}

static mg_status trainer_grad(mg_trainer *t, const float *q, const float *target, const float *mask,
                              double *loss) {
    // normalise by the number of fine pixels the loss covers
    const float inv = 1.0f / (float)t->npix_f;
    cudaError_t e = mg::train_forward(t, q, 0);
    if (e == cudaSuccess) e = mg::train_backward(t, q, target, mask, inv, 0);
    if (e == cudaSuccess) e = cudaMemcpy(t->hloss, t->lpart, 256 * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return tcuda(e, "trainer gradient");
    mg_status fs = trainer_check_flag(t);
    if (fs != MG_OK) return fs;
    if (loss) {
        double s = 0.0;
        for (int i = 0; i < 256; ++i) s += t->hloss[i];
        *loss = s * inv;
    }
    return MG_OK;
}

mg_status mg_trainer_gradients(mg_trainer *t, const float *q, const float *target, const float *mask,
                               float *grad, double *loss) {
    if (!t || !q || !target || !grad) return terr(MG_ERR_INVALID_ARG, "null trainer or pointer");
    mg_status st = trainer_grad(t, q, target, mask, loss);
    if (st != MG_OK) return st;
    cudaError_t e = cudaMemcpy(grad, t->G, sizeof(float) * t->nparam, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) return tcuda(e, "mg_trainer_gradients");
    return MG_OK;
}

mg_status mg_trainer_step(mg_trainer *t, const float *q, const float *target, const float *mask, double *loss) {
    if (!t || !q || !target) return terr(MG_ERR_INVALID_ARG, "null trainer or pointer");
    mg_status st = trainer_grad(t, q, target, mask, loss);
    if (st != MG_OK) return st;
    t->steps += 1;
    const double bc1 = 1.0 - pow((double)t->b1, t->steps), bc2 = 1.0 - pow((double)t->b2, t->steps);
    const float lr_t = (float)(t->lr * sqrt(bc2) / bc1);
    mg::k_adam<<<mg::grid_for(t->nparam), mg::RT>>>(t->P, t->G, t->M, t->V, t->nparam, lr_t, t->b1, t->b2,
                                                    t->eps * (float)sqrt(bc2));
    mg::count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tcuda(e, "mg_trainer_step");
    return MG_OK;
}

mg_status mg_trainer_set_tensor_cores(mg_trainer *t, int on) {
    if (!t) return terr(MG_ERR_INVALID_ARG, "null trainer");
    if (on && (t->g.W % mg::TCM) != 0)
        return terr(MG_ERR_INVALID_ARG, "tensor-core training needs W a multiple of 128");
    t->tc = on != 0;
    return MG_OK;
}

mg_status mg_trainer_get_tensor_cores(mg_trainer *t, int *on) {
    if (!t || !on) return terr(MG_ERR_INVALID_ARG, "null trainer or pointer");
    *on = t->tc ? 1 : 0;
    return MG_OK;
}

mg_status mg_trainer_set_lr(mg_trainer *t, double lr) {
    if (!t || !(lr > 0.0)) return terr(MG_ERR_INVALID_ARG, "null trainer or lr <= 0");
    t->lr = (float)lr;
    return MG_OK;
}

mg_status mg_trainer_get_weights(mg_trainer *t, void *blob, size_t bytes) {
    if (!t || !blob || bytes != 64 + 4 * t->nparam) return terr(MG_ERR_INVALID_ARG, "blob size mismatch");
    unsigned char *b = (unsigned char *)blob;
    memset(b, 0, 64);
    memcpy(b, "MGSRW001", 8);
    const uint32_t nf = 64, nbk = (uint32_t)t->nb, np = (uint32_t)t->nparam;
    memcpy(b + 8, &nf, 4);
    memcpy(b + 12, &nbk, 4);
    memcpy(b + 16, &np, 4);
    cudaError_t e = cudaMemcpy(b + 64, t->P, 4 * t->nparam, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return tcuda(e, "mg_trainer_get_weights");
    return MG_OK;
}

void mg_trainer_destroy(mg_trainer *t) {
    if (!t) return;
    for (void *p : t->allocs) cudaFree(p);
    if (t->hloss) cudaFreeHost(t->hloss);
    delete t;
}

}  // extern "C"
