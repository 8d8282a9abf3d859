// mg_sr.cu - super-resolution prolongation: weight loading and generator.
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "mg_sr.cuh"

namespace mg {

namespace {
constexpr char kMagic[8] = {'M', 'G', 'S', 'R', 'W', '0', '0', '1'};
constexpr size_t kHeader = 64;

size_t expected_params(int nf, int nb) {
    size_t n = (size_t)nf * 9 + nf + nf;                     // in.w, in.b, in.a
    n += (size_t)nb * (2 * ((size_t)nf * nf * 9 + nf) + nf);  // blocks
    n += (size_t)4 * nf * nf * 9 + 4 * nf + nf;              // up.w, up.b, up.a
    n += (size_t)nf * 9 + 1;                                 // out.w, out.b
    return n;
}
}  // namespace

void sr_free(SrState *st) {
    cudaFree(st->params);
    cudaFree(st->packed);
    cudaFree(st->fine_out);
    cudaFree(st->act);
    cudaFree(st->scal);
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
    if (nf != 64 || nb < 1 || nb > 32 || np != expected_params(nf, nb) ||
        bytes != kHeader + np * sizeof(float)) {
        snprintf(err, errlen, "weight blob: n_feat=%d n_blocks=%d n_params=%zu bytes=%zu inconsistent",
                 nf, nb, np, bytes);
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
    sr_free(st);
    cudaError_t e = cudaMalloc(&st->params, np * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(st->params, p, np * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "weight upload: %s", cudaGetErrorString(e));
        sr_free(st);
        return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
    }
    st->n_feat = nf;
    st->n_blocks = nb;
    st->n_params = np;
    st->loaded = true;
    return MG_OK;
}

mg_status sr_correction(SrState *st, const float *ec, int nc, cudaStream_t stream, char *err,
                        size_t errlen) {
    (void)st;
    (void)ec;
    (void)nc;
    (void)stream;
    snprintf(err, errlen, "SR generator kernels are not available in this build");
    return MG_ERR_INVALID_ARG;
}

}  // namespace mg
