/*
 * ddg_probe.h - FMA throughput probe of libddg.so.
 *
 * Measures the FP32 and FP64 fused multiply-add rates the GPU reaches, the
 * ALU peaks against which the GNN kernel (FP32, Section III-B, Eqs. 18-22)
 * and the Krylov kernels (FP64, Algorithm 1) are measured.  No passage of the
 * paper corresponds to this call; it exists for measurement.
 */
#ifndef DDG_PROBE_H
#define DDG_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Runs independent FMA chains on every SM of CUDA device `device` (8 CTAs of
 * 256 threads per SM, 8 chains per thread, values kept in registers), one
 * warm-up launch and one timed launch per precision on a stream of its own,
 * and writes the rates in TFLOP/s (2 FLOP per FMA) to *fp32_tflops and
 * *fp64_tflops.  Takes about 15 ms and 2.4 MB of device memory on a B300,
 * which it frees before returning.  The GPU's clock at the time sets the
 * result; the call changes no GPU setting.  Errors: DDG_INVALID_ARG (NULL
 * output, no such device), DDG_CUDA_ERROR. */
int32_t ddg_probe_fma_peaks(int32_t device, double *fp32_tflops, double *fp64_tflops);

#ifdef __cplusplus
}
#endif

#endif /* DDG_PROBE_H */
