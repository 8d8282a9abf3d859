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
// Everything runs in FP32 on the CUDA cores.  The 64/256-channel
// convolutions are implicit GEMMs over 64-pixel x 64-channel tiles (256
// threads, 4 x 4 outputs per thread, K staged through shared memory 16 at a
// time): forward (K = 9 taps x input channels), data gradient (the same with
// the taps mirrored and the weight's channel roles swapped) and weight
// gradient (K = pixels, split over fixed chunks and summed in chunk order, so
// results are deterministic).  Activations are channels-last
// [batch][y][x][channel]; parameters, gradients and Adam moments are flat
// arrays in the weight-blob order of mg_load_prolong_weights.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "mg_internal.cuh"

namespace mg {

namespace {

constexpr int F = 64;             // features
constexpr int TP = 64;            // pixels per GEMM tile
constexpr int KC = 16;            // K per shared-memory stage
constexpr int GT = 256;           // threads per GEMM block
constexpr int WCHUNK = 2048;      // pixels per weight-gradient partial
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

// Per-channel sums over pixels, two stages: part[block][c] then out[c] (in block order).
// v(p, c) = a[p][c] * (mode 0: 1;  mode 1: z[p][c] <= 0 ? z[p][c] : 0)
__global__ void k_chan_partial(const float *__restrict__ a, const float *__restrict__ z, int C, int npix,
                               int mode, float *__restrict__ part) {
    // block: 256 threads = C channel lanes x (256 / C) pixel lanes; pixels [blockIdx.x * WCHUNK, +WCHUNK)
    extern __shared__ float sh[];
    const int lanes = blockDim.x / C;
    const int c = threadIdx.x % C, l = threadIdx.x / C;
    const int pa = blockIdx.x * WCHUNK, pb = min(npix, pa + WCHUNK);
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
__global__ void k_chan_reduce(const float *__restrict__ part, int C, int nblk, float *__restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * C + c];
    out[c] = s;
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
    const int pa = blockIdx.x * WCHUNK, pb = min(npix_f, pa + WCHUNK);
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
    const int pa = blockIdx.x * WCHUNK, pb = min(npix, pa + WCHUNK);
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
    const int pa = blockIdx.x * WCHUNK, pb = min(npix_f, pa + WCHUNK);
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

// Sum chunk partials laid out [chunk][m] into out[m] in chunk order.
__global__ void k_sum_chunks(const float *__restrict__ part, int m, int nchunk, float *__restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * m + e];
        out[e] = s;
    }
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
    int npix = 0, npix_f = 0, nchunk = 0, nchunk_f = 0;
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

template <bool DGRAD, int CK, int CN, int EPI>
cudaError_t gemm(Trainer *t, const float *in, const float *w, const float *bias, const float *slope,
                 const float *skip, float *out, float *out2, cudaStream_t s) {
    constexpr int NOUT = CN;
    dim3 grid(t->npix / TP, NOUT / 64);
    k_conv_gemm<DGRAD, CK, CN, EPI><<<grid, GT, 0, s>>>(in, w, bias, slope, skip, out, out2, t->g);
    count_launches(1);
    return cudaGetLastError();
}

template <int CK, int CN>
cudaError_t wgrad(Trainer *t, const float *in, const float *dout, float *grad, cudaStream_t s) {
    dim3 grid(t->nchunk, 9, CN / 64);
    k_conv_wgrad<CK, CN><<<grid, GT, 0, s>>>(in, dout, t->part, t->g, t->npix);
    k_wgrad_reduce<<<grid_for((size_t)9 * CN * CK), RT, 0, s>>>(t->part, grad, CK, CN, t->nchunk);
    count_launches(2);
    return cudaGetLastError();
}

// per-channel sum of a (mode 0) or slope gradient (mode 1) over the coarse pixels
cudaError_t chan_sum(Trainer *t, const float *a, const float *z, int C, int mode, float *out, cudaStream_t s) {
    k_chan_partial<<<t->nchunk, RT, RT * sizeof(float), s>>>(a, z, C, t->npix, mode, t->part);
    k_chan_reduce<<<(C + 63) / 64, 64, 0, s>>>(t->part, C, t->nchunk, out);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace

// Forward pass of the whole batch; q: [B][H][W].
cudaError_t train_forward(Trainer *t, const float *q, cudaStream_t s) {
    float *P = t->P;
    k_conv_in<<<grid_for((size_t)t->npix * F), RT, 0, s>>>(q, P + t->o_in_w, P + t->o_in_b, P + t->o_in_a, t->z0,
                                                          t->xs[0], t->g, t->npix);
    count_launches(1);
    TR_CK(cudaGetLastError());
    for (int k = 0; k < t->nb; ++k) {
        TR_CK((gemm<false, F, F, EPI_PRELU>(t, t->xs[k], P + t->o_w1[k], P + t->o_b1[k], P + t->o_a[k], nullptr,
                                            t->z1[k], t->a1[k], s)));
        TR_CK((gemm<false, F, F, EPI_ADD>(t, t->a1[k], P + t->o_w2[k], P + t->o_b2[k], nullptr, t->xs[k],
                                          t->xs[k + 1], nullptr, s)));
    }
    TR_CK((gemm<false, F, 4 * F, EPI_SHUFFLE>(t, t->xs[t->nb], P + t->o_up_w, P + t->o_up_b, P + t->o_up_a,
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
    k_conv_out_wgrad<<<t->nchunk_f, RT, 0, s>>>(t->af, t->dy, t->gf, t->npix_f, t->part);
    k_sum_chunks<<<grid_for(F * 9), RT, 0, s>>>(t->part, F * 9, t->nchunk_f, G + t->o_out_w);
    count_launches(2);
    {   // out bias = sum dy: reuse the channel reduction with C = 1 over fine pixels
        k_chan_partial<<<t->nchunk_f, RT, RT * sizeof(float), s>>>(t->dy, nullptr, 1, t->npix_f, 0, t->part);
        k_chan_reduce<<<1, 64, 0, s>>>(t->part, 1, t->nchunk_f, G + t->o_out_b);
        count_launches(2);
    }
    k_conv_out_dgrad<<<grid_for((size_t)t->npix_f * F), RT, 0, s>>>(t->dy, P + t->o_out_w, t->daf, t->gf, t->npix_f);
    // up layer: slope gradient, then dzu through the shuffle and PReLU'
    k_shuffle_slope_partial<<<t->nchunk_f, RT, RT * sizeof(float), s>>>(t->daf, t->zu, t->g, t->npix_f, t->part);
    k_chan_reduce<<<1, 64, 0, s>>>(t->part, F, t->nchunk_f, G + t->o_up_a);
    k_shuffle_back<<<grid_for((size_t)t->npix * 4 * F), RT, 0, s>>>(t->daf, t->zu, P + t->o_up_a, t->dzu, t->g,
                                                                   t->npix);
    count_launches(4);
    TR_CK(cudaGetLastError());
    TR_CK((wgrad<F, 4 * F>(t, t->xs[t->nb], t->dzu, G + t->o_up_w, s)));
    TR_CK(chan_sum(t, t->dzu, nullptr, 4 * F, 0, G + t->o_up_b, s));
    TR_CK((gemm<true, 4 * F, F, EPI_RAW>(t, t->dzu, P + t->o_up_w, nullptr, nullptr, nullptr, t->dx, nullptr, s)));
    // residual blocks, last to first; t->dx = gradient w.r.t. the block output
    for (int k = t->nb - 1; k >= 0; --k) {
        // conv2: input a1, output grad dx
        TR_CK((wgrad<F, F>(t, t->a1[k], t->dx, G + t->o_w2[k], s)));
        TR_CK(chan_sum(t, t->dx, nullptr, F, 0, G + t->o_b2[k], s));
        TR_CK((gemm<true, F, F, EPI_RAW>(t, t->dx, P + t->o_w2[k], nullptr, nullptr, nullptr, t->da, nullptr, s)));
        // PReLU: slope gradient, then da -> dz1 (in place)
        TR_CK(chan_sum(t, t->da, t->z1[k], F, 1, G + t->o_a[k], s));
        k_prelu_back<<<grid_for((size_t)t->npix * F), RT, 0, s>>>(t->da, t->z1[k], P + t->o_a[k], F,
                                                                (size_t)t->npix * F, t->da);
        count_launches(1);
        // conv1: input xs[k], output grad da (= dz1)
        TR_CK((wgrad<F, F>(t, t->xs[k], t->da, G + t->o_w1[k], s)));
        TR_CK(chan_sum(t, t->da, nullptr, F, 0, G + t->o_b1[k], s));
        TR_CK((gemm<true, F, F, EPI_RAW>(t, t->da, P + t->o_w1[k], nullptr, nullptr, nullptr, t->dx2, nullptr, s)));
        k_add<<<grid_for((size_t)t->npix * F), RT, 0, s>>>(t->dx, t->dx2, (size_t)t->npix * F);  // skip path
        count_launches(1);
        TR_CK(cudaGetLastError());
    }
    // first layer: PReLU then weights
    TR_CK(chan_sum(t, t->dx, t->z0, F, 1, G + t->o_in_a, s));
    k_prelu_back<<<grid_for((size_t)t->npix * F), RT, 0, s>>>(t->dx, t->z0, P + t->o_in_a, F, (size_t)t->npix * F,
                                                            t->dx);
    k_conv_in_wgrad<<<t->nchunk, RT, 0, s>>>(q, t->dx, t->g, t->npix, t->part);
    k_sum_chunks<<<grid_for(F * 9), RT, 0, s>>>(t->part, F * 9, t->nchunk, G + t->o_in_w);
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
    t->nchunk = (t->npix + mg::WCHUNK - 1) / mg::WCHUNK;
    t->nchunk_f = (t->npix_f + mg::WCHUNK - 1) / mg::WCHUNK;
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
    al(&t->part, std::max((size_t)t->nchunk * 9 * 4 * mg::F * mg::F, (size_t)t->nchunk_f * mg::F * 9));
    al(&t->lpart, 512);
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
    return MG_OK;
}

static mg_status trainer_grad(mg_trainer *t, const float *q, const float *target, const float *mask,
                              double *loss) {
    // normalise by the number of fine pixels the loss covers
    const float inv = 1.0f / (float)t->npix_f;
    cudaError_t e = mg::train_forward(t, q, 0);
    if (e == cudaSuccess) e = mg::train_backward(t, q, target, mask, inv, 0);
    if (e == cudaSuccess) e = cudaMemcpy(t->hloss, t->lpart, 256 * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return tcuda(e, "trainer gradient");
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
