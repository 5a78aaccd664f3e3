/*
 * ns_peaks.h -- FMA throughput probe of libns_peaks.so (measurement only).
 *
 * Not part of the method: the paper's solver is graded against HBM bandwidth
 * where memory binds, and against the GPU's own FP32 / FP64 fused
 * multiply-add rate where arithmetic binds (the FP64 comparators); this probe
 * measures those two rates.
 */
#ifndef NS_PEAKS_H
#define NS_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* Runs the probe once on cuda_stream (a cudaStream_t; NULL = legacy default
 * stream): `blocks` CTAs of 256 threads, each thread 8 independent chains of
 * `iters` dependent FMAs (FP64 when fp64 != 0, else FP32).  *ms (host)
 * receives the kernel's CUDA-event time, *flops (host) the floating-point
 * operations performed (2 per FMA).  Returns 0, or the CUDA error code
 * (cudaErrorInvalidValue for blocks < 1, iters < 1 or a null output). */
int nsp_fma_probe(int fp64, int blocks, int iters, void *cuda_stream, float *ms, double *flops);

#ifdef __cplusplus
}
#endif

#endif /* NS_PEAKS_H */
