/*
 * nk_probe.h -- machine probes of libnk: the peak rates that the kernels'
 * roofline fractions divide by, measured on the GPU the library runs on.
 *
 * The paper has no counterpart: it reports no kernel throughput.  These
 * calls exist so that a fraction such as "achieved FP32 operations / peak"
 * divides by a rate measured on this GPU rather than one derived from unit
 * counts.  Each call allocates its own scratch (cudaMalloc), launches a
 * warm-up and then one timed kernel on `stream` (CUDA events), synchronises,
 * frees its scratch and returns the rate.  No clock, power or other device
 * setting is read or changed.
 */
#ifndef NK_PROBE_H
#define NK_PROBE_H

#include <stdint.h>

#include "nk.h"

#ifdef __cplusplus
extern "C" {
#endif

enum {
  NK_PROBE_FP32_FMA = 0, /* independent FP32 FMA chains on every SM: lane-FMAs/s */
  NK_PROBE_FP64_FMA = 1, /* the same in FP64: lane-FMAs/s */
  NK_PROBE_L2_READ = 2,  /* reads of an L2-resident buffer (work = bytes, <= 64 MB), bypassing L1: bytes/s */
  NK_PROBE_HBM_READ = 3  /* reads of a buffer larger than L2 (work = bytes, >= 512 MB): bytes/s */
};

/* Runs probe `which` with `work` (FMA probes: iterations of 8 chains per
 * thread, 0 = default; read probes: buffer bytes, 0 = default) and returns
 * the rate in *rate (per second) and the timed kernel's duration in *ms.
 * NK_ERR_INVALID_ARG for an unknown probe or a size outside its range;
 * NK_ERR_NO_MEMORY / NK_ERR_CUDA from the allocation or launch. */
nk_status nk_probe(int which, int64_t work, double* rate, double* ms, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NK_PROBE_H */
