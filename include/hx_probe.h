/*
 * hx_probe.h -- measurement support of the benchmark (not part of the
 * solver): the FP64 and FP32 fused-multiply-add throughput of the current
 * GPU, the denominators of the ALU roofline that the residual kernels are
 * reported against.  The paper has no counterpart; it quotes its GPUs'
 * nominal FP64 rates (Sec. 3, Table 1), this measures the GPU at hand.
 * Built as libhx_probe.so beside libhx.so.
 */
#ifndef HX_PROBE_H
#define HX_PROBE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { HX_PROBE_OK = 0, HX_PROBE_ERR_INVALID_ARG = -1, HX_PROBE_ERR_CUDA = -6 };

/* Times one launch (after a warm-up launch) of independent FMA chains that
 * fill every SM of the current device at full occupancy, in FP64 and in
 * FP32, with CUDA events on the legacy default stream; writes the achieved
 * TFLOP/s (2 flops per FMA) to *fp64_tflops and *fp32_tflops, and, when ms
 * is not NULL, the two launch times in ms to ms[0], ms[1].  Each launch takes
 * about 0.1 s on a GB300.  Allocates and frees one small device buffer.
 * Returns HX_PROBE_OK, HX_PROBE_ERR_INVALID_ARG (null outputs) or
 * HX_PROBE_ERR_CUDA. */
int hx_probe_fma_peaks(double* fp64_tflops, double* fp32_tflops, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* HX_PROBE_H */
