// FMA throughput probe (measurement only, not part of the stepper): the
// FP32 and FP64 arithmetic ceilings the stencil and solver kernels are graded
// against where HBM does not bind.  Every thread runs NCHAIN independent
// chains x <- x * a + b of `iters` fused multiply-adds each (2 flops per FMA);
// the chains converge to b / (1 - a) = 1, so no value overflows or turns
// subnormal.  Timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>

namespace {

template <typename T, int NCHAIN>
__global__ void __launch_bounds__(256) k_fma_chains(T* __restrict__ sink, int iters, T a, T b) {
    T x[NCHAIN];
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) x[c] = T(1) + T(0.001) * T(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < NCHAIN; ++c) s += x[c];
    // never true (the chains sit near 1): keeps them live without a store
    if (s < T(-1)) sink[blockIdx.x] = s;
}

constexpr int kChains = 8;

}  // namespace

extern "C" {

// Runs the probe once on `cuda_stream` (a cudaStream_t, NULL = legacy default
// stream) with blocks x 256 threads; *ms receives the kernel time and *flops
// the floating-point operations it performed.  fp64 != 0 selects double.
// Returns 0 on success, else the CUDA error code.
int nsp_fma_probe(int fp64, int blocks, int iters, void* cuda_stream, float* ms, double* flops) {
    if (blocks < 1 || iters < 1 || !ms || !flops) return (int)cudaErrorInvalidValue;
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaEvent_t e0, e1;
    cudaError_t err = cudaEventCreate(&e0);
    if (err != cudaSuccess) return (int)err;
    err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        cudaEventDestroy(e0);
        return (int)err;
    }
    cudaEventRecord(e0, st);
    if (fp64)
        k_fma_chains<double, kChains><<<blocks, 256, 0, st>>>(nullptr, iters, 0.999, 0.001);
    else
        k_fma_chains<float, kChains><<<blocks, 256, 0, st>>>(nullptr, iters, 0.999f, 0.001f);
    err = cudaGetLastError();
    cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *flops = 2.0 * kChains * (double)iters * 256.0 * (double)blocks;
    return (int)err;
}

}  // extern "C"
