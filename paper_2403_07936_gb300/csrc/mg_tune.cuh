// mg_tune.cuh - the autotuner's entry point (table accessors are in
// mg_internal.cuh).
#pragma once

#include <stddef.h>

#include "mg_internal.cuh"

namespace mg {

// One tile level of a context: x, t (ping-pong partner of x) and b at size n,
// and the next coarser level's b (restriction target) and x (prolongation
// source).  The buffers are overwritten.
struct TuneLevel {
    int n;
    float *x, *t, *b, *bc, *xc;
};

// Time every tile variant of k_down (nu1 sweeps) and k_up (nu2 sweeps) on each
// level, set the table to the fastest, and (if cache_path is not null) take
// entries for this GPU from the cache file instead of timing, appending new
// measurements to it.  *n_timed = table entries measured (not from the cache).
mg_status tune_levels(const TuneLevel *lv, int nlev, int nu1, int nu2, const FirTaps &taps, cudaStream_t s,
                      int device, const char *cache_path, int *n_timed, char *err, size_t errlen);

}  // namespace mg
