/*
 * mmpc_peaks.h -- measured throughput of the FP32 pipes the solve kernels
 * are bound by.
 *
 * The fused AM kernels do no dense contraction on the tensor cores and move
 * almost nothing through HBM: their roofline is the issue rate of FP32
 * arithmetic on the CUDA cores (the element-wise updates of Eqs. split_v,
 * split_alpha_o and split_alpha_a and the basis contractions of Eqs.
 * lin_solve_xy_2 and lin_solve_psi_2, all FP32).  mmpc_measure_peaks times
 * three saturating kernels on the current device -- dependent chains of
 * scalar FFMA, of packed f32x2 FFMA2 (two lanes of work per instruction) and
 * of MUFU rsqrt, 8 independent chains per thread, 8 CTAs of 256 threads per
 * SM -- and reports the best of `reps` runs of each, so that a roofline can
 * be stated against a measured peak beside the one derived from unit counts
 * and clocks.
 *
 * Conventions as in mmpc.h: the call is synchronous (it waits for its own
 * kernels), allocates and frees its own small device buffer, and returns
 * MMPC_OK or MMPC_ERR_INVALID_ARG (out NULL, reps < 1) or MMPC_ERR_CUDA.
 */
#ifndef MMPC_PEAKS_H
#define MMPC_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double ffma;    /* scalar FFMA: FP32 lane operations per second (an FMA counts 1) */
    double ffma2;   /* packed FFMA2: FP32 lane operations per second (2 per lane and instruction) */
    double rsqrt;   /* MUFU rsqrt: operations per second */
    double ms_ffma, ms_ffma2, ms_rsqrt;  /* best kernel durations, CUDA events */
    int sms;        /* SMs of the device */
    int clock_khz;  /* the device's maximum SM clock (cudaDevAttrClockRate) */
} mmpc_peaks;

int mmpc_measure_peaks(mmpc_peaks* out, int reps, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MMPC_PEAKS_H */
