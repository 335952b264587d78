/*
 * pylom_probe.h -- measurement support for the roofline of the binary64
 * path (no counterpart in the paper).
 *
 * The FP64 POD path runs its dense contractions on the FP64 tensor pipe
 * (mma.sync.m8n8k4.f64) and its panel/tree work on scalar FP64 FMA.  These
 * probes time each instruction stream alone on the current device so the
 * benchmark can state the denominator of its FP64 roofline as a measured
 * figure.
 */
#ifndef PYLOM_PROBE_H
#define PYLOM_PROBE_H

#include <stdint.h>

#include "pylom.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Runs a throughput loop of independent FP64 MMAs (kind 0: mma.sync
 * m8n8k4 f64), FP64 FMAs (kind 1) or FP32 FMAs (kind 2) over every SM of
 * the current device on
 * `stream`, synchronises, and writes to HOST memory the achieved TFLOP/s.
 * scratch: device buffer of >= pylom_probe_scratch_bytes() bytes (results
 * are stored there so the loop is not optimised away). */
size_t pylom_probe_scratch_bytes(void);
pylom_status pylom_probe_fp64_peak(int kind, void* scratch, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PYLOM_PROBE_H */
