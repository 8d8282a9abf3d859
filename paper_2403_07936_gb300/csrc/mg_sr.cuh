// mg_sr.cuh - super-resolution (SR) prolongation state and entry points.
//
// The SR prolongation (Sec. 2.3, Fig. 1b; Sec. 3.1; Appendix A, Algorithm 5)
// adds a learned correction s * G(e_c / s), s = max|e_c|, to the cubic-spline
// interpolant of the coarse error e_c.  G is a convolutional generator:
// conv3x3 1->64 + PReLU, residual blocks [conv3x3 64->64, PReLU, conv3x3
// 64->64, + skip], conv3x3 64->256, pixel-shuffle x2, PReLU, conv3x3 64->1,
// all with circular padding.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/mg.h"

namespace mg {

struct SrState {
    bool loaded = false;
    int n_feat = 0, n_blocks = 0;
    size_t n_params = 0;
    float *params = nullptr;   // all parameters, float, blob order (device)
    void *packed = nullptr;    // tensor-core weight tiles (device)
    size_t packed_bytes = 0;
    float *fine_out = nullptr; // s * G(e_c / s) on the fine grid (device)
    int fine_n = 0;
    void *act = nullptr;       // activation buffers (device)
    size_t act_bytes = 0;
    double *scal = nullptr;    // device scalars: input scale
};

// Parse and copy a weight blob (layout in mg.h).  Errors go to err.
mg_status sr_load(SrState *st, const void *blob, size_t bytes, char *err, size_t errlen);
// Compute s * G(e_c / s) for the coarse error ec (nc x nc) into st->fine_out.
mg_status sr_correction(SrState *st, const float *ec, int nc, cudaStream_t stream, char *err,
                        size_t errlen);
void sr_free(SrState *st);

}  // namespace mg
