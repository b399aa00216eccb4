/*
 * gl_peaks.h -- C-ABI of libglpeaks.so: measured non-tensor throughput of one
 * GPU, the denominators of the light-curve kernels' ALU rooflines.
 *
 * The paper has no counterpart (it quotes only the FP32:FP64 ratio of the card it
 * ran on, Sec. 2); the light-curve path is bound by plain FP32 and FP64
 * arithmetic, so its roofline needs the rates of those pipes on this GPU, taken
 * the way a kernel sees them rather than from unit counts.
 *
 * Each probe launches a grid of 8 x 256-thread CTAs per SM whose threads run
 * independent dependency chains of one instruction kind (enough chains per
 * thread to cover the pipe's latency), times it with CUDA events on a private
 * stream after one untimed launch, and keeps the best of `repeats` launches.
 * Results depend on the SM clock at the time; callers sample it alongside.
 *
 * All functions return 0, -1 for a bad argument, or -3 for a CUDA failure.  They
 * use the given device (cudaSetDevice) and allocate 4 bytes of device memory per
 * call (freed before returning).
 */
#ifndef GL_PEAKS_H
#define GL_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

#define GLP_FFMA 0   /* FP32 fused multiply-add (fma.rn.f32), 2 flops each */
#define GLP_DFMA 1   /* FP64 fused multiply-add (fma.rn.f64), 2 flops each */
#define GLP_MUFU 2   /* FP32 approximate reciprocal square root (rsqrt.approx.f32), 1 op each */

/* Throughput of instruction kind `kind` on CUDA device `device`:
 *   *flops_per_s  floating-point operations per second (FMA counted as 2, MUFU as 1)
 *   *best_ms      duration of the fastest timed launch (ms)
 *   *ops          operations per launch
 * repeats: timed launches, 1 .. 100. */
int glp_measure(int device, int kind, int repeats, double *flops_per_s, double *best_ms,
                double *ops);

#ifdef __cplusplus
}
#endif

#endif /* GL_PEAKS_H */
