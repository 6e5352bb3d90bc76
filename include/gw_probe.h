/*
 * gw_probe.h -- measurement helper of the benchmark (no counterpart in the paper).
 *
 * The roofline of the FP64 kernels needs the GPU's dense FP64 FMA rate, which the
 * measured-peaks file of this machine does not list.  gw_fp_peak measures it on
 * the given device with independent FMA chains (8 per thread, no memory traffic
 * in the loop) and reports TFLOP/s counting an FMA as two flops.
 */
#ifndef GW_PROBE_H
#define GW_PROBE_H

#include "gw.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Measures dense FP64 and FP32 FMA throughput on `device` (allocates and frees a
 * small output buffer; synchronizes the device).  Outputs may be NULL. */
gw_status gw_fp_peak(int device, double* fp64_tflops, double* fp32_tflops);

#ifdef __cplusplus
}
#endif
#endif /* GW_PROBE_H */
