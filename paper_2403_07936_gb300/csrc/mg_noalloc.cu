// mg_noalloc.cu - a V-cycle entry point that performs no device allocation.
//
// mg_op_vcycle allocates device memory on every call for the dense
// pseudo-inverse of the coarsest-grid operator.  Some callers cannot do that:
// cudaMalloc implicitly synchronises the whole device, which a caller that
// steps a simulation at a fixed rate cannot afford in its loop, and a
// process whose framework allocator has already reserved nearly all device
// memory sees cudaMalloc fail even when the framework holds free blocks.
// mg_op_vcycle_static serves them: the pseudo-inverse is built on the device
// into the file-scope array below, which every GPU that loads this library
// keeps until the process exits.
//
// Scratch: kStaticPinvEntries doubles (512 KiB), enough for a coarsest grid of
// up to 16 x 16 points (a 256 x 256 matrix); larger grids are rejected.  All
// calls share the one array and each call rewrites it on the caller's stream,
// so calls that overlap on the GPU (different streams, no ordering) race.
// The array's address is looked up once per device and kept for the process;
// after a cudaDeviceReset the module is loaded anew and that address is stale,
// so this entry point must not be used across a device reset.
#include <stdio.h>

#include <mutex>

#include "mg_internal.cuh"

namespace mg {
namespace {

constexpr int kStaticCoarsestMax = 16;
constexpr int kStaticPinvEntries = (kStaticCoarsestMax * kStaticCoarsestMax) *
                                   (kStaticCoarsestMax * kStaticCoarsestMax);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_pinv[kStaticPinvEntries];

// Device address of g_static_pinv on each device, looked up once per device.
std::mutex g_setup_mutex;
void *g_pinv_addr[kMaxDevices] = {};

// Closed-form pseudo-inverse of the scaled periodic operator 4I - shifts on an
// m x m grid: entry (p, q) = (1/m^2) sum_{k != 0} cos(2 pi k.(p - q) / m) / lam(k),
// lam(k) = 4 sin^2(pi kx / m) + 4 sin^2(pi ky / m).  One thread per entry.
// Each block first tabulates lam(k) (m^2 <= 256 values) and cos(2 pi j / m)
// (m <= 16 values) in shared memory, so an entry costs table reads, FP64
// divisions and additions instead of three transcendental calls per term.
template <typename T>
__global__ void k_build_pinv(T *__restrict__ out, int m) {
    __shared__ double lam[kStaticCoarsestMax * kStaticCoarsestMax];
    __shared__ double cosv[kStaticCoarsestMax];
    const int Nc = m * m;
    for (int k = threadIdx.x; k < Nc; k += blockDim.x) {
        const int ky = k / m, kx = k - ky * m;
        const double sx = sinpi((double)kx / m), sy = sinpi((double)ky / m);
        lam[k] = 4.0 * (sx * sx + sy * sy);
    }
    for (int j = threadIdx.x; j < m; j += blockDim.x) cosv[j] = cospi(2.0 * j / m);
    __syncthreads();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Nc * Nc) return;
    const int P = e / Nc, Q = e - P * Nc;
    const int di = ((P / m) - (Q / m) + m) % m;
    const int dj = ((P % m) - (Q % m) + m) % m;
    double acc = 0.0;
    for (int ky = 0; ky < m; ++ky)
        for (int kx = 0; kx < m; ++kx) {
            if (kx == 0 && ky == 0) continue;
            acc += cosv[(kx * dj + ky * di) % m] / lam[ky * m + kx];
        }
    out[e] = (T)(acc / Nc);
}

// The array's device address on the current device.  It is looked up again
// on every call made outside stream capture (the lookup allocates nothing, and
// a context reset reloads the module at another address); a call on a
// capturing stream takes the address cached by the last uncaptured call.
mg_status static_scratch(void **addr, cudaStream_t s, char *err, size_t errlen) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        snprintf(err, errlen, "mg_op_vcycle_static: no usable current device (%s)",
                 cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;  // unknown: keep the cached address
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_pinv_addr[dev] || cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_pinv);
        if (e != cudaSuccess || !p) {
            snprintf(err, errlen, "mg_op_vcycle_static: cudaGetSymbolAddress failed on device %d: %s",
                     dev, cudaGetErrorString(e));
            return MG_ERR_CUDA;
        }
        g_pinv_addr[dev] = p;
    }
    *addr = g_pinv_addr[dev];
    return MG_OK;
}

template <typename T>
cudaError_t run(T *x, const T *b, int n, int coarsest, int nu1, int nu2, bool zero_init, T *pinv,
                cudaStream_t s) {
    const int entries = coarsest * coarsest * coarsest * coarsest;
    k_build_pinv<T><<<(entries + 255) / 256, 256, 0, s>>>(pinv, coarsest);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    FirTaps taps;
    fir_taps_host(&taps);
    return launch_bottom<T>(x, b, n, coarsest, nu1, nu2, zero_init, pinv, taps, s);
}

}  // namespace
}  // namespace mg

// Largest grid this entry point accepts (both dtypes).
constexpr int kStaticMax = 64;

extern "C" mg_status mg_op_vcycle_static(int dtype, int n, int coarsest, void *x, const void *b,
                                         int nu1, int nu2, int zero_init, void *stream) {
    thread_local static char err[256];
    auto fail = [&](mg_status st) {
        mg::set_last_error(err);
        return st;
    };
    if ((dtype != 0 && dtype != 1) || n < 4 || n > kStaticMax || (n & (n - 1)) ||
        coarsest < 4 || coarsest > mg::kStaticCoarsestMax || (coarsest & (coarsest - 1)) ||
        coarsest > n || !x || !b || nu1 < 0 || nu1 > 4 || nu2 < 0 || nu2 > 4) {
        snprintf(err, sizeof err,
                 "mg_op_vcycle_static: need n a power of two in [4, %d], coarsest a power of two in "
                 "[4, min(n, %d)] (static scratch of %d doubles), 0 <= nu <= 4, non-null x and b; "
                 "got n=%d coarsest=%d",
                 kStaticMax, mg::kStaticCoarsestMax, mg::kStaticPinvEntries, n, coarsest);
        return fail(MG_ERR_INVALID_ARG);
    }
    cudaStream_t s = (cudaStream_t)stream;
    void *pinv = nullptr;
    mg_status st = mg::static_scratch(&pinv, s, err, sizeof err);
    if (st != MG_OK) return fail(st);
    cudaError_t e = dtype == 0
        ? mg::run<double>((double *)x, (const double *)b, n, coarsest, nu1, nu2, zero_init != 0,
                          (double *)pinv, s)
        : mg::run<float>((float *)x, (const float *)b, n, coarsest, nu1, nu2, zero_init != 0,
                         (float *)pinv, s);
    if (e != cudaSuccess) {
        snprintf(err, sizeof err, "mg_op_vcycle_static: launch failed: %s", cudaGetErrorString(e));
        return fail(MG_ERR_CUDA);
    }
    return MG_OK;
}
