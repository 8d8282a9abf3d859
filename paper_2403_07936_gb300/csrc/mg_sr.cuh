// mg_sr.cuh - super-resolution (SR) prolongation state and entry points.
//
// The SR prolongation (Sec. 2.3, Fig. 1b; Sec. 3.1; Appendix A, Algorithm 5)
// adds a learned correction s * G(e_c / s), s = max|e_c|, to the cubic-spline
// interpolant of the coarse error e_c.  G is a convolutional generator:
// conv3x3 1->64 + PReLU, residual blocks [conv3x3 64->64, PReLU, conv3x3
// 64->64, + skip], conv3x3 64->256, pixel-shuffle x2, PReLU, conv3x3 64->1,
// all with circular padding.
//
// Activations are bf16, channels-last (64 channels = 128 bytes per pixel),
// stored with a one-pixel periodic halo: an H x W grid occupies
// (H + 2) x (W + 2) pixels, pixel (y, x) at padded (y + 1, x + 1), and the
// halo rows/columns hold the wrapped neighbours.  Every 3x3 window is then a
// plain rectangle, which is what the TMA tile loads of the tensor-core
// convolution read.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/mg.h"

namespace mg {

constexpr int kSrFeat = 64;
constexpr int kSrMinCoarse = 128;  // coarse grids the generator takes: multiples of 128

struct SrState {
    bool loaded = false;
    bool view = false;  // shares another state's weights and scratch scalars (sr_view)
    int n_feat = 0, n_blocks = 0;
    uint64_t hash = 0;  // FNV-1a of the loaded blob (equal weights in a batch)
    // weights (device): tensor-core layers packed bf16 [layer][tap][co][ci],
    // layers = 2 * n_blocks + 4 (the 4 pixel-shuffle groups of conv 64->256)
    void *w_tc = nullptr;
    float *bias_tc = nullptr;   // [layers][64]
    float *prelu_blk = nullptr; // [n_blocks][64]
    float *prelu_up = nullptr;  // [64]
    float *w_in = nullptr;      // [64][9], bias [64], prelu [64]  (in one array)
    float *w_out = nullptr;     // [9][64] then bias [1]
    // buffers sized for coarse grid nc (reallocated when nc changes)
    int nc = 0;
    void *act[3] = {nullptr, nullptr, nullptr};  // padded coarse activations
    void *fine_act = nullptr;                    // padded fine activation (after shuffle)
    float *fine_out = nullptr;                   // s * G(e_c / s), fine grid (unpadded)
    float *scal = nullptr;                       // device scalars: [0] = s
    double *red = nullptr;                       // reduction partials
    unsigned *red_counter = nullptr;
    int *err = nullptr;                          // device error flag (bounded waits)
    CUtensorMap tm_act[3];  // activation buffers as convolution inputs (row planes)
    CUtensorMap tm_out[3];  // the same buffers as destinations of output tiles
    CUtensorMap tm_fine;    // fine_act as the destination of the pixel-shuffle layer
    CUtensorMap tm_w;
};

// SR generator buffers for a batch of `imgs` equal-size coarse errors (the
// finest transitions of several right-hand sides of one size): activations of
// all images stacked along y, each padded image after the previous one, so a
// single launch per layer serves the whole batch.  Weights come from an
// SrState at run time.
struct SrBatch {
    int imgs = 0, nc = 0;
    void *act[3] = {nullptr, nullptr, nullptr};
    void *fine_act = nullptr;
    float *fine_out = nullptr;  // [imgs][2nc][2nc]: s_i G(e_i / s_i)
    float *s = nullptr;         // [imgs]
    const float **ecs = nullptr;  // [imgs] device pointers to the coarse errors (device table)
    CUtensorMap tm_act[3];
    CUtensorMap tm_out[3];
    CUtensorMap tm_fine;
};
// Allocate for imgs coarse errors of nc x nc at the device addresses ecs[]
// (host array of device pointers; copied).  Outside any stream capture.
mg_status sr_batch_prepare(SrBatch *b, int imgs, int nc, const float *const *ecs, char *err, size_t errlen);
// b->fine_out[i] = s_i G(e_i / s_i), s_i = max|e_i|, with st's weights
// (asynchronous on stream; capturable).
mg_status sr_batch_correction(SrBatch *b, const SrState *st, cudaStream_t stream, char *err, size_t errlen);
void sr_batch_free(SrBatch *b);

// Windowed SR (Sec. 3.1, Fig. 2; Algorithms 1-5): mosaic buffers for the
// (nc/2)^2 windows of an nc x nc coarse field (see mg_sr.cu).
struct SrWindows {
    int nc = 0, Hm = 0, Wm = 0;  // coarse grid; mosaic rows and columns
    void *act[3] = {nullptr, nullptr, nullptr};
    void *fine_act = nullptr;
    CUtensorMap tm_act[3];
    CUtensorMap tm_out[3];
    CUtensorMap tm_fine;
};
// Allocate for coarse grids of nc (a power of two >= 32); outside capture.
mg_status sr_windows_prepare(SrWindows *w, int nc, char *err, size_t errlen);
// out (2nc x 2nc, device) = the windowed SR prolongation of ec with st's
// weights and the normalisation interval [p_min, p_max] (asynchronous).
mg_status sr_windowed(SrWindows *w, const SrState *st, const float *ec, int nc, double p_min, double p_max,
                      float *out, cudaStream_t stream, char *err, size_t errlen);
void sr_windows_free(SrWindows *w);

// Parse and copy a weight blob (layout in mg.h).  Errors go to err.
mg_status sr_load(SrState *st, const void *blob, size_t bytes, char *err, size_t errlen);
// Allocate the activation buffers and tensor maps for coarse grids of size nc
// (outside any stream capture).
mg_status sr_prepare(SrState *st, int nc, char *err, size_t errlen);
// Compute s * G(e_c / s) for the coarse error ec (nc x nc) into st->fine_out
// (asynchronous on stream; sr_prepare must have run for nc).
mg_status sr_correction(SrState *st, const float *ec, int nc, cudaStream_t stream, char *err,
                        size_t errlen);
// Point view at st's weights and scratch scalars, with activation and output
// buffers of its own for coarse grids of size nc (kept while nc is unchanged),
// so that one generator runs at several grid sizes without reallocating.
// Outside any stream capture; a view is used on st's stream only.
mg_status sr_view(SrState *view, const SrState *st, int nc, char *err, size_t errlen);
// Free a state; a view frees only its own buffers.
void sr_free(SrState *st);

// One layer of the loaded generator on caller buffers (verification; the
// kernels and weights of sr_correction): layer 0 = s = max|ec| into *s, then
// conv 1 -> 64 + PReLU of ec / s; 1 .. 2 n_blocks = the block convolutions
// (odd: + PReLU; even: + skip); 2 n_blocks + 1 = conv 64 -> 256, shuffle,
// PReLU; 2 n_blocks + 2 = s * conv 64 -> 1 of the padded fine activation.
// Synchronous on stream.
mg_status sr_layer(SrState *st, int layer, int nc, const void *in, const void *skip, float *s, void *out,
                   cudaStream_t stream, char *err, size_t errlen);

// One tensor-core convolution layer on padded bf16 activations (verification).
mg_status sr_conv_layer(int mode, int H, int W, const void *in, const void *skip, const void *w_packed,
                        const float *bias, const float *prelu, void *out, cudaStream_t stream,
                        char *err, size_t errlen);

}  // namespace mg
