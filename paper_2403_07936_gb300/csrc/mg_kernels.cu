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
// FP64 outer kernels (defect correction around FP32 V-cycles): source sum,
// scaled right-hand side, FP64 residual with norms and float conversion,
// solution update, zero-mean projection.  Sums are deterministic (fixed grid,
// fixed-order trees, last-block finish).
#include <math.h>

#include <atomic>

#include "mg_internal.cuh"

namespace mg {

static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
unsigned long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

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

constexpr int kTY = 32;        // tile rows
constexpr int kTX = 64;        // tile columns
constexpr int kThreads = 256;  // threads per tile block

__host__ __device__ constexpr int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Copy rows [r0, r0+R) x cols [c0, c0+C) of the periodic n x n grid g into
// shared memory s (pitch SP).  c0, C, SP are multiples of the vector width.
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

// Store the interior rows [r_s, r_s+TY) x cols [c_s, c_s+TX) of a staged tile
// to global rows [gy, gy+TY) x cols [gx, gx+TX).
template <typename T, int SP>
__device__ __forceinline__ void store_tile(T *__restrict__ g, const T *__restrict__ s, int n, int gy,
                                           int gx, int r_s, int c_s) {
    using V = typename Prec<T>::vec;
    constexpr int VW = Prec<T>::VW;
    constexpr int CV = kTX / VW;
    for (int idx = threadIdx.x; idx < kTY * CV; idx += blockDim.x) {
        const int rr = idx / CV, cv = idx - rr * CV;
        const V v = *reinterpret_cast<const V *>(s + (r_s + rr) * SP + c_s + cv * VW);
        *reinterpret_cast<V *>(g + (size_t)(gy + rr) * n + gx + cv * VW) = v;
    }
}

// One colour of Gauss-Seidel on the staged rows [r_lo, r_hi) x cols
// [c_lo, c_hi) (c_lo and the width even; staged parity equals global parity).
// x <- (b + ((x_N + x_S) + x_W) + x_E) / 4 for the points with (r+c)%2 == colour.
template <typename T, int SP>
__device__ __forceinline__ void half_sweep(T *__restrict__ xs, const T *__restrict__ bs, int r_lo,
                                           int r_hi, int c_lo, int c_hi, int colour) {
    const int W = (c_hi - c_lo) >> 1;
    const int total = (r_hi - r_lo) * W;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int rr = idx / W, k = idx - rr * W;
        const int r = r_lo + rr;
        const int c = c_lo + 2 * k + ((r + c_lo + colour) & 1);
        const int p = r * SP + c;
        const T nb = ((xs[p - SP] + xs[p + SP]) + xs[p - 1]) + xs[p + 1];
        xs[p] = (bs[p] + nb) * T(0.25);
    }
}

// ---------------------------------------------------------------------------
// k_down: NU sweeps, residual, full-weighting restriction of one tile.
// ---------------------------------------------------------------------------
template <typename T, int NU>
struct DownCfg {
    static constexpr int VW = Prec<T>::VW;
    static constexpr int H = 2 * NU + 2;             // logical halo (rows and cols)
    static constexpr int HX = round_up(H, VW);       // staged column halo
    static constexpr int R = kTY + 2 * H;
    static constexpr int C = kTX + 2 * HX;
    static constexpr int SP = C;
    static constexpr size_t smem = 2ull * R * SP * sizeof(T);
};

template <typename T, int NU, bool ZERO>
__global__ void __launch_bounds__(kThreads) k_down(const T *__restrict__ x, T *__restrict__ xout,
                                                   const T *__restrict__ b, int n,
                                                   T *__restrict__ bc) {
    using Cfg = DownCfg<T, NU>;
    constexpr int H = Cfg::H, HX = Cfg::HX, R = Cfg::R, C = Cfg::C, SP = Cfg::SP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    T *bs = xs + R * SP;
    const int ty0 = blockIdx.y * kTY, tx0 = blockIdx.x * kTX;

    load_tile<T, R, C, SP>(bs, b, n, ty0 - H, tx0 - HX);
    if (ZERO) {
        for (int i = threadIdx.x; i < R * SP; i += blockDim.x) xs[i] = T(0);
    } else {
        load_tile<T, R, C, SP>(xs, x, n, ty0 - H, tx0 - HX);
    }
    __syncthreads();

    // staged coordinates: logical (u, v) -> (u + H, v + HX)
    const int c_off = HX - H;
#pragma unroll 1
    for (int s = 0; s < NU; ++s) {
#pragma unroll 1
        for (int colour = 0; colour < 2; ++colour) {
            const int k = 2 * s + colour + 1;
            half_sweep<T, SP>(xs, bs, k, R - k, c_off + k, C - c_off - k, colour);
            __syncthreads();
        }
    }
    // scaled residual s = b - (4x - sum) on logical [-1, T+1), written over b
    constexpr int RW = kTX + 2;
    for (int idx = threadIdx.x; idx < (kTY + 2) * RW; idx += blockDim.x) {
        const int rr = idx / RW, cc = idx - rr * RW;
        const int p = (H - 1 + rr) * SP + (HX - 1 + cc);
        const T nb = ((xs[p - SP] + xs[p + SP]) + xs[p - 1]) + xs[p + 1];
        bs[p] = bs[p] - (T(4) * xs[p] - nb);
    }
    __syncthreads();
    // full weighting at coarse (I, J) <-> fine (2I, 2J); times 4 for h_c^2 = 4 h^2
    const int nc = n >> 1;
    constexpr int CW = kTX / 2;
    for (int idx = threadIdx.x; idx < (kTY / 2) * CW; idx += blockDim.x) {
        const int I = idx / CW, J = idx - I * CW;
        const int p = (H + 2 * I) * SP + (HX + 2 * J);
        const T edge = ((bs[p - SP] + bs[p + SP]) + bs[p - 1]) + bs[p + 1];
        const T corner = ((bs[p - SP - 1] + bs[p - SP + 1]) + bs[p + SP - 1]) + bs[p + SP + 1];
        bc[(size_t)(ty0 / 2 + I) * nc + tx0 / 2 + J] = (T(4) * bs[p] + T(2) * edge + corner) * T(0.25);
    }
    store_tile<T, SP>(xout, xs, n, ty0, tx0, H, HX);
}

// ---------------------------------------------------------------------------
// k_up: x += P_cubic ec, then NU sweeps, on one tile.
// ---------------------------------------------------------------------------
template <typename T, int NU>
struct UpCfg {
    static constexpr int VW = Prec<T>::VW;
    static constexpr int L = Prec<T>::L;
    static constexpr int H = 2 * NU;
    static constexpr int HX = round_up(H, VW);
    static constexpr int R = kTY + 2 * H;
    static constexpr int C = kTX + 2 * HX;
    static constexpr int SP = C;
    // coarse rows [I0 - CHY, I0 + TY/2 + H/2 + L), cols [J0 - CHX, J0 + TX/2 + CXE)
    static constexpr int CHY = H / 2 + L - 1;
    static constexpr int CR = kTY / 2 + CHY + H / 2 + L;
    static constexpr int CHX = round_up(H / 2 + L - 1, VW);
    static constexpr int CXE = round_up(H / 2 + L, VW);
    static constexpr int CC = kTX / 2 + CHX + CXE;
    static constexpr size_t smem = (2ull * R * SP + (size_t)CR * CC + (size_t)CR * SP) * sizeof(T);
};

template <typename T, int NU>
__global__ void __launch_bounds__(kThreads) k_up(const T *__restrict__ x, T *__restrict__ xout,
                                                 const T *__restrict__ b, const T *__restrict__ ec,
                                                 const T *__restrict__ extra, int n, FirTaps taps) {
    using Cfg = UpCfg<T, NU>;
    constexpr int H = Cfg::H, HX = Cfg::HX, R = Cfg::R, C = Cfg::C, SP = Cfg::SP, L = Cfg::L;
    constexpr int CHY = Cfg::CHY, CR = Cfg::CR, CHX = Cfg::CHX, CC = Cfg::CC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    T *bs = xs + R * SP;
    T *cs = bs + R * SP;   // coarse tile [CR][CC]
    T *rs = cs + CR * CC;  // row-refined coarse rows [CR][SP]
    const int ty0 = blockIdx.y * kTY, tx0 = blockIdx.x * kTX;
    const int nc = n >> 1;

    load_tile<T, R, C, SP>(xs, x, n, ty0 - H, tx0 - HX);
    if (NU > 0) load_tile<T, R, C, SP>(bs, b, n, ty0 - H, tx0 - HX);
    load_tile<T, CR, CC, CC>(cs, ec, nc, ty0 / 2 - CHY, tx0 / 2 - CHX);
    __syncthreads();

    // refine along x: fine logical column v in [-H, TX+H) for every coarse row
    constexpr int FW = kTX + 2 * H;
    for (int idx = threadIdx.x; idx < CR * FW; idx += blockDim.x) {
        const int cr = idx / FW, vv = idx - cr * FW;
        const int v = vv - H;
        const T *row = cs + cr * CC;
        T val;
        if ((v & 1) == 0) {
            val = row[CHX + (v >> 1)];
        } else {
            const int cb = CHX + ((v - 1) >> 1);
            T acc = T(0);
#pragma unroll
            for (int k = L; k >= 1; --k) acc += Prec<T>::tap(taps, k) * (row[cb + k] + row[cb + 1 - k]);
            val = acc;
        }
        rs[cr * SP + HX + v] = val;
    }
    __syncthreads();
    // refine along y and add: fine logical rows u in [-H, TY+H)
    constexpr int FH = kTY + 2 * H;
    for (int idx = threadIdx.x; idx < FH * FW; idx += blockDim.x) {
        const int uu = idx / FW, vv = idx - uu * FW;
        const int u = uu - H, v = vv - H;
        const int col = HX + v;
        T val;
        if ((u & 1) == 0) {
            val = rs[(CHY + (u >> 1)) * SP + col];
        } else {
            const int rb = CHY + ((u - 1) >> 1);
            T acc = T(0);
#pragma unroll
            for (int k = L; k >= 1; --k)
                acc += Prec<T>::tap(taps, k) * (rs[(rb + k) * SP + col] + rs[(rb + 1 - k) * SP + col]);
            val = acc;
        }
        if (extra) val += extra[(size_t)((ty0 + u) & (n - 1)) * n + ((tx0 + v) & (n - 1))];
        xs[(u + H) * SP + col] += val;
    }
    __syncthreads();
    const int c_off = HX - H;
#pragma unroll 1
    for (int s = 0; s < NU; ++s) {
#pragma unroll 1
        for (int colour = 0; colour < 2; ++colour) {
            const int k = 2 * s + colour + 1;
            half_sweep<T, SP>(xs, bs, k, R - k, c_off + k, C - c_off - k, colour);
            __syncthreads();
        }
    }
    store_tile<T, SP>(xout, xs, n, ty0, tx0, H, HX);
}

// ---------------------------------------------------------------------------
// k_bottom: a whole V-cycle on grids <= 64 x 64, one block, shared memory.
// ---------------------------------------------------------------------------
constexpr int kBottomThreads = 512;

template <typename T>
__device__ __forceinline__ void sweep_periodic(T *X, const T *B, int m, int colour) {
    const int half = (m * m) >> 1, hm = m >> 1;
    for (int idx = threadIdx.x; idx < half; idx += blockDim.x) {
        const int i = idx / hm, k = idx - i * hm;
        const int j = 2 * k + ((i + colour) & 1);
        const int im = (i - 1) & (m - 1), ip = (i + 1) & (m - 1);
        const int jm = (j - 1) & (m - 1), jp = (j + 1) & (m - 1);
        const T nb = ((X[im * m + j] + X[ip * m + j]) + X[i * m + jm]) + X[i * m + jp];
        X[i * m + j] = (B[i * m + j] + nb) * T(0.25);
    }
}

template <typename T>
__global__ void __launch_bounds__(kBottomThreads) k_bottom(T *__restrict__ x, const T *__restrict__ b,
                                                           int n, int nlev, int nu1, int nu2,
                                                           int zero_init, const T *__restrict__ ainv,
                                                           FirTaps taps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *base = reinterpret_cast<T *>(smem_raw);
    T *X[8], *B[8];
    int off = 0;
    for (int l = 0; l < nlev; ++l) {
        const int m = n >> l;
        X[l] = base + off;
        off += m * m;
        B[l] = base + off;
        off += m * m;
    }
    T *S = base + off;  // n*n scratch: residual, then row-refined coarse rows
    const int tid = threadIdx.x, nt = blockDim.x;

    for (int p = tid; p < n * n; p += nt) {
        X[0][p] = zero_init ? T(0) : x[p];
        B[0][p] = b[p];
    }
    __syncthreads();
    for (int l = 0; l + 1 < nlev; ++l) {
        const int m = n >> l, mc = m >> 1;
        for (int s = 0; s < nu1; ++s) {
            sweep_periodic(X[l], B[l], m, 0);
            __syncthreads();
            sweep_periodic(X[l], B[l], m, 1);
            __syncthreads();
        }
        for (int p = tid; p < m * m; p += nt) {
            const int i = p / m, j = p - i * m;
            const int im = (i - 1) & (m - 1), ip = (i + 1) & (m - 1);
            const int jm = (j - 1) & (m - 1), jp = (j + 1) & (m - 1);
            const T nb = ((X[l][im * m + j] + X[l][ip * m + j]) + X[l][i * m + jm]) + X[l][i * m + jp];
            S[p] = B[l][p] - (T(4) * X[l][p] - nb);
        }
        __syncthreads();
        for (int q = tid; q < mc * mc; q += nt) {
            const int I = q / mc, J = q - I * mc;
            const int i = 2 * I, j = 2 * J;
            const int im = (i - 1) & (m - 1), ip = (i + 1) & (m - 1);
            const int jm = (j - 1) & (m - 1), jp = (j + 1) & (m - 1);
            const T edge = ((S[im * m + j] + S[ip * m + j]) + S[i * m + jm]) + S[i * m + jp];
            const T corner = ((S[im * m + jm] + S[im * m + jp]) + S[ip * m + jm]) + S[ip * m + jp];
            B[l + 1][q] = (T(4) * S[i * m + j] + T(2) * edge + corner) * T(0.25);
            X[l + 1][q] = T(0);
        }
        __syncthreads();
    }
    {   // coarsest grid: e = A~^+ b (the pseudo-inverse annihilates the mean)
        const int mcst = n >> (nlev - 1), Nc = mcst * mcst;
        T *Xc = X[nlev - 1];
        const T *Bc = B[nlev - 1];
        for (int p = tid; p < Nc; p += nt) {
            T acc = T(0);
            for (int q = 0; q < Nc; ++q) acc += ainv[p * Nc + q] * Bc[q];
            Xc[p] = acc;
        }
        __syncthreads();
    }
    constexpr int L = Prec<T>::L;
    for (int l = nlev - 2; l >= 0; --l) {
        const int m = n >> l, mc = m >> 1;
        const T *E = X[l + 1];
        for (int p = tid; p < mc * m; p += nt) {  // refine coarse rows along x
            const int I = p / m, j = p - I * m;
            T val;
            if ((j & 1) == 0) {
                val = E[I * mc + (j >> 1)];
            } else {
                const int J = j >> 1;
                T acc = T(0);
#pragma unroll 4
                for (int k = L; k >= 1; --k)
                    acc += Prec<T>::tap(taps, k) *
                           (E[I * mc + ((J + k) & (mc - 1))] + E[I * mc + ((J + 1 - k) & (mc - 1))]);
                val = acc;
            }
            S[p] = val;
        }
        __syncthreads();
        for (int p = tid; p < m * m; p += nt) {  // refine along y and add
            const int i = p / m, j = p - i * m;
            T val;
            if ((i & 1) == 0) {
                val = S[(i >> 1) * m + j];
            } else {
                const int I = i >> 1;
                T acc = T(0);
#pragma unroll 4
                for (int k = L; k >= 1; --k)
                    acc += Prec<T>::tap(taps, k) *
                           (S[((I + k) & (mc - 1)) * m + j] + S[((I + 1 - k) & (mc - 1)) * m + j]);
                val = acc;
            }
            X[l][p] += val;
        }
        __syncthreads();
        for (int s = 0; s < nu2; ++s) {
            sweep_periodic(X[l], B[l], m, 0);
            __syncthreads();
            sweep_periodic(X[l], B[l], m, 1);
            __syncthreads();
        }
    }
    for (int p = tid; p < n * n; p += nt) x[p] = X[0][p];
}

// ---------------------------------------------------------------------------
// FP64 outer kernels
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kRedThreads) k_sum(const double *__restrict__ a, size_t N,
                                                     Reduction red) {
    __shared__ double sh[32];
    double v = 0.0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x)
        v += a[p];
    double vals[1] = {block_sum(v, sh)};
    reduce_finish<1>(red, vals, sh);
}

__global__ void __launch_bounds__(kRedThreads) k_scaled_rhs(const double *__restrict__ f, int n,
                                                            double h2, const double *__restrict__ fsum,
                                                            double *__restrict__ b) {
    const size_t N = (size_t)n * n;
    const double mu = *fsum / (double)N;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x)
        b[p] = h2 * (f[p] - mu);
}

template <bool WRITE32, bool FNORM>
__global__ void __launch_bounds__(kRedThreads) k_outer_residual(
    const double *__restrict__ f, const double *__restrict__ x, int n, double h2,
    const double *__restrict__ fsum, double mu_host, float *__restrict__ s32, Reduction red) {
    __shared__ double sh[32];
    const size_t N = (size_t)n * n;
    const double mu = fsum ? *fsum / (double)N : mu_host;
    double ss = 0.0, ff = 0.0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(p / n), j = (int)(p - (size_t)i * n);
        const int im = (i - 1) & (n - 1), ip = (i + 1) & (n - 1);
        const int jm = (j - 1) & (n - 1), jp = (j + 1) & (n - 1);
        const double nb = ((x[(size_t)im * n + j] + x[(size_t)ip * n + j]) + x[(size_t)i * n + jm]) +
                          x[(size_t)i * n + jp];
        const double fc = f[p] - mu;
        const double s = h2 * fc - (4.0 * x[p] - nb);
        ss += s * s;
        if (FNORM) ff += fc * fc;
        if (WRITE32) s32[p] = (float)s;
    }
    double vals[2];
    vals[0] = block_sum(ss, sh);
    vals[1] = FNORM ? block_sum(ff, sh) : 0.0;
    reduce_finish<2>(red, vals, sh);
}

__global__ void __launch_bounds__(kRedThreads) k_update(double *__restrict__ x,
                                                        const float *__restrict__ e, size_t N,
                                                        Reduction red) {
    __shared__ double sh[32];
    double ee = 0.0, xs = 0.0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        const double d = (double)e[p];
        const double xn = x[p] + d;
        x[p] = xn;
        ee += d * d;
        xs += xn;
    }
    double vals[2];
    vals[0] = block_sum(ee, sh);
    vals[1] = block_sum(xs, sh);
    reduce_finish<2>(red, vals, sh);
}

__global__ void __launch_bounds__(kRedThreads) k_project(double *__restrict__ x, size_t N,
                                                         const double *__restrict__ sum) {
    const double mu = *sum / (double)N;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x)
        x[p] -= mu;
}

template <typename KernelT>
cudaError_t set_smem(KernelT k, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int NU, bool ZERO>
cudaError_t down_impl(const T *x, T *xout, const T *b, int n, T *bc, cudaStream_t s) {
    using Cfg = DownCfg<T, NU>;
    auto k = k_down<T, NU, ZERO>;
    cudaError_t e = set_smem(k, Cfg::smem);
    if (e != cudaSuccess) return e;
    dim3 grid(n / kTX, n / kTY);
    k<<<grid, kThreads, Cfg::smem, s>>>(x, xout, b, n, bc);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, int NU>
cudaError_t up_impl(const T *x, T *xout, const T *b, const T *ec, const T *extra, int n,
                    const FirTaps &taps, cudaStream_t s) {
    using Cfg = UpCfg<T, NU>;
    auto k = k_up<T, NU>;
    cudaError_t e = set_smem(k, Cfg::smem);
    if (e != cudaSuccess) return e;
    dim3 grid(n / kTX, n / kTY);
    k<<<grid, kThreads, Cfg::smem, s>>>(x, xout, b, ec, extra, n, taps);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_down(const T *x, T *xout, const T *b, int n, int nu, bool zero_init, T *bc,
                        cudaStream_t s) {
    if (n < kTX || n % kTX || n % kTY || x == xout) return cudaErrorInvalidValue;
#define MG_DOWN_CASE(NU)                                                                  \
    case NU:                                                                              \
        return zero_init ? down_impl<T, NU, true>(x, xout, b, n, bc, s)                   \
                         : down_impl<T, NU, false>(x, xout, b, n, bc, s);
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

template <typename T>
cudaError_t launch_up(const T *x, T *xout, const T *b, const T *ec, int n, int nu,
                      const FirTaps &taps, cudaStream_t s, const T *extra) {
    if (n < kTX || n % kTX || n % kTY || !ec || x == xout) return cudaErrorInvalidValue;
    switch (nu) {
        case 0: return up_impl<T, 0>(x, xout, b, ec, extra, n, taps, s);
        case 1: return up_impl<T, 1>(x, xout, b, ec, extra, n, taps, s);
        case 2: return up_impl<T, 2>(x, xout, b, ec, extra, n, taps, s);
        case 3: return up_impl<T, 3>(x, xout, b, ec, extra, n, taps, s);
        case 4: return up_impl<T, 4>(x, xout, b, ec, extra, n, taps, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_bottom(T *x, const T *b, int n, int coarsest, int nu1, int nu2, bool zero_init,
                          const T *ainv, const FirTaps &taps, cudaStream_t s) {
    if (n > kBottomMax || coarsest < 4 || coarsest > n) return cudaErrorInvalidValue;
    int nlev = 0;
    size_t elems = 0;
    for (int m = n; m >= coarsest; m >>= 1) {
        elems += 2ull * m * m;
        ++nlev;
    }
    if ((n >> (nlev - 1)) != coarsest || nlev > 8) return cudaErrorInvalidValue;
    elems += (size_t)n * n;
    const size_t smem = elems * sizeof(T);
    auto k = k_bottom<T>;
    cudaError_t e = set_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<1, kBottomThreads, smem, s>>>(x, b, n, nlev, nu1, nu2, zero_init ? 1 : 0, ainv, taps);
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_down<float>(const float *, float *, const float *, int, int, bool, float *,
                                        cudaStream_t);
template cudaError_t launch_down<double>(const double *, double *, const double *, int, int, bool,
                                         double *, cudaStream_t);
template cudaError_t launch_up<float>(const float *, float *, const float *, const float *, int, int,
                                      const FirTaps &, cudaStream_t, const float *);
template cudaError_t launch_up<double>(const double *, double *, const double *, const double *, int,
                                       int, const FirTaps &, cudaStream_t, const double *);
template cudaError_t launch_bottom<float>(float *, const float *, int, int, int, int, bool, const float *,
                                          const FirTaps &, cudaStream_t);
template cudaError_t launch_bottom<double>(double *, const double *, int, int, int, int, bool,
                                           const double *, const FirTaps &, cudaStream_t);

cudaError_t launch_source_sum(const double *f, int n, Reduction red, cudaStream_t s) {
    k_sum<<<kRedBlocks, kRedThreads, 0, s>>>(f, (size_t)n * n, red);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_sum(const double *x, int n, Reduction red, cudaStream_t s) {
    return launch_source_sum(x, n, red, s);
}
cudaError_t launch_scaled_rhs(const double *f, int n, double h2, const double *f_sum, double *b,
                              cudaStream_t s) {
    k_scaled_rhs<<<kRedBlocks, kRedThreads, 0, s>>>(f, n, h2, f_sum, b);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_outer_residual(const double *f, const double *x, int n, double h2,
                                  const double *mu_sum, double mu_host, float *s32,
                                  bool want_fnorm, Reduction red, cudaStream_t s) {
    if (s32) {
        if (want_fnorm)
            k_outer_residual<true, true><<<kRedBlocks, kRedThreads, 0, s>>>(f, x, n, h2, mu_sum, mu_host, s32, red);
        else
            k_outer_residual<true, false><<<kRedBlocks, kRedThreads, 0, s>>>(f, x, n, h2, mu_sum, mu_host, s32, red);
    } else {
        if (want_fnorm)
            k_outer_residual<false, true><<<kRedBlocks, kRedThreads, 0, s>>>(f, x, n, h2, mu_sum, mu_host, s32, red);
        else
            k_outer_residual<false, false><<<kRedBlocks, kRedThreads, 0, s>>>(f, x, n, h2, mu_sum, mu_host, s32, red);
    }
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_update(double *x, const float *e, int n, Reduction red, cudaStream_t s) {
    k_update<<<kRedBlocks, kRedThreads, 0, s>>>(x, e, (size_t)n * n, red);
    count_launches(1);
    return cudaGetLastError();
}
cudaError_t launch_project(double *x, int n, const double *sum, cudaStream_t s) {
    k_project<<<kRedBlocks, kRedThreads, 0, s>>>(x, (size_t)n * n, sum);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace mg
