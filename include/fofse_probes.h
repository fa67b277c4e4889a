/*
 * fofse_probes.h -- measurement probes of the GB300 FOFSE library, built into
 * their own library (libfofse_probes.so) beside libfofse.so; the benchmark
 * uses them to measure the rates the kernels' rooflines are quoted against.
 * They have no counterpart in the paper and compute nothing of the method.
 *
 * Each probe launches `ctas` blocks of 1024 threads doing `rounds` rounds on
 * `stream` (a cudaStream_t passed as void*) and returns the work queued:
 *   fofse_probe_smem   *bytes loaded from shared memory (16 B per thread and
 *                      load, consecutive lanes consecutive 16 B: no bank
 *                      conflicts)
 *   fofse_probe_fma    *fmas FP32 fused multiply-adds (lanes)
 *   fofse_probe_dfma   *fmas FP64 fused multiply-adds (lanes)
 * d_sink: device buffer of ctas x 1024 floats (doubles for the FP64 probe),
 * caller-owned; it keeps the work from being optimised away and is in
 * practice never written.  The caller times the launch (CUDA events).
 * Returns FOFSE_OK once queued, FOFSE_E_ARG for non-positive sizes or NULL
 * pointers (nothing launched), FOFSE_E_CUDA if the launch failed (the CUDA
 * error is then left for cudaGetLastError).
 */
#ifndef FOFSE_PROBES_H_
#define FOFSE_PROBES_H_

#include "fofse.h"

#ifdef __cplusplus
extern "C" {
#endif

fofse_status fofse_probe_smem(int ctas, int rounds, float* d_sink, double* bytes, void* stream);
fofse_status fofse_probe_fma(int ctas, int rounds, float* d_sink, double* fmas, void* stream);
fofse_status fofse_probe_dfma(int ctas, int rounds, double* d_sink, double* fmas, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FOFSE_PROBES_H_ */
