/*
 * hts_profile.h -- measurement utilities of the HT-reduction library.  These entry points
 * have no counterpart in the paper: they exist so that a benchmark can time every kernel of a
 * call with CUDA events on the stream the kernel runs on, and can measure the FP64
 * arithmetic peak of the device it runs on.
 */
#ifndef HTS_PROFILE_H
#define HTS_PROFILE_H

#include "hts.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Kernel classes reported by the profiler. */
enum {
    HTS_K_GENERATE = 0,     /* near-diagonal chase (stage 2 generate phase) */
    HTS_K_APPLY_RIGHT = 1,  /* delayed right updates of A and B (stage 2) */
    HTS_K_APPLY_LEFT = 2,   /* delayed left updates of A and B (stage 2) */
    HTS_K_UTIL = 3,         /* identity initialisation, final zeroing */
    HTS_K_STAGE1 = 4,       /* stage 0 / stage 1 kernels */
    HTS_K_APPLY_QZ = 5,     /* delayed right updates of Q and Z (stage 2, side stream) */
    HTS_K_BATCH = 6,        /* batched reduction of many small pencils */
    HTS_K_FORM_U = 7,       /* block formation: reflector products per block (stage 2) */
    HTS_K_EMU_RIGHT = 8,    /* emulated-FP64 delayed right updates of A and B (stage 2) */
    HTS_K_EMU_LEFT = 9,     /* emulated-FP64 delayed left updates of A and B (stage 2) */
    HTS_K_EMU_QZ = 10,      /* emulated-FP64 delayed updates of Q and Z (stage 2, side stream) */
    HTS_K_UPDATE = 11,      /* look-ahead update launch: a group's A / B updates and the previous
                               group's Q / Z update, beside the next group's chase (stage 2) */
    HTS_K_NKINDS = 12
};

typedef struct {
    int launches;      /* launches recorded */
    double ms;         /* summed CUDA-event durations of those launches */
    double flops;      /* algorithmic floating-point operations (4 per element and reflector) */
    double bytes;      /* algorithmic DRAM bytes (each touched element read and written once) */
    double mma_flops;  /* BF16 tensor-core flops issued (emulated-FP64 kernels; 0 elsewhere) */
} hts_kernel_profile;

/* Start recording: preallocates 2 * max_launches CUDA events on the context's device (do
 * this outside any timed region).  Subsequent calls on ctx record an event pair around every
 * kernel launch until max_launches is reached.  HTS_ERR_ARG for bad arguments,
 * HTS_ERR_CUDA if the events cannot be created. */
hts_status hts_profile_begin(hts_ctx *ctx, int max_launches);

/* Stop recording: waits for the last recorded event, sums the durations per kernel class
 * into out[0 .. HTS_K_NKINDS-1] and releases the events.  *dropped (may be NULL) receives the
 * number of launches that did not fit into the pool. */
hts_status hts_profile_end(hts_ctx *ctx, hts_kernel_profile out[HTS_K_NKINDS], int *dropped);

/* Number of chase steps (r <= 16) whose opposite-reflector direction failed the checks of the
 * column elimination (residual above 2^-44 max|block| max|z|, or a pivot outside 2^+-960) and
 * was recomputed from the RQ of the B block, counted on the device since the context was
 * created or since the previous call of this function.  Waits for `stream` first.  Steps forced
 * onto the RQ by HTS_FLAG_TEST_DIRECT_RQ are not counted. */
hts_status hts_fallback_count(hts_ctx *ctx, void *stream, long long *count);

/* Measure the FP64 fused multiply-add throughput of the current device (TFLOP/s, 2 flops per
 * FMA) with a short kernel on `stream`; blocks until it finishes. */
hts_status hts_probe_fp64_peak(void *stream, double *tflops);

#ifdef __cplusplus
}
#endif

#endif /* HTS_PROFILE_H */
