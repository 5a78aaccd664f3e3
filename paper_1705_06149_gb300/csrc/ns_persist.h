// Host interface of the persistent pressure solve (ns_persist.cu): one
// cooperative launch runs a whole multigrid-preconditioned BiCGStab solve of
// the pressure equation L p = b (Section 2) -- the start, every iteration with
// its two V-cycles, the FP32+refine outer corrections and the loop decisions
// -- for a small batch of states, with a grid-wide barrier between phases
// instead of a kernel boundary.  It serves the latency-bound batch-1 solves of
// Parareal's coarse propagator, where a launched kernel costs several
// microseconds whatever its size.
#pragma once

#include <cuda_runtime.h>

#include "ns_mg.cuh"

namespace nsk {

// A persistent CTA: PERSIST_GROUPS groups of NTHREADS threads (32 x 4 x 8),
// each running the cell kernels' CTAs of a phase.
constexpr int PERSIST_GROUPS = 8;
constexpr int PERSIST_THREADS = NTHREADS * PERSIST_GROUPS;
// Grid barrier words: the arrival count and, a cache line away so that the
// waiting CTAs' polls do not contend with the arrivals, the generation.
constexpr int PERSIST_BAR_GEN = 32;
constexpr int PERSIST_BAR_WORDS = 64;

// Everything one persistent solve reads: the same arguments the launched
// kernels of the solve take.
template <typename T>
struct PSolve {
    MgPlan plan;
    MgBuf<T> mb;
    FFBuf ff;                 // FP32+refine: the float-float iterate and residual
    SliceCtl* ctl;
    double* part_div;         // partial sums of b (the right side's fluid mean)
    double* part_mg;
    double* b;                // right side (the FP64 start removes its mean in place)
    const double* p_in;       // warm start (FP64); null: the extrapolated one
    const double* p_prev;     // FP64: the extrapolated warm start 2 p^n - p^(n-1)
    LoopCount* loopc;
    unsigned* bar;            // grid barrier: [0] arrivals, [PERSIST_BAR_GEN] generation
    int* err;                 // set to 1 when a barrier wait gave up
    long long spin_ns;        // longest wait at one barrier, nanoseconds
    double otol2, itol2, tol2;
    int maxit, max_outer, n_fluid, batch;
    unsigned cap;             // hard cap on loop bodies (as the graph loops)
};

// Largest dynamic shared memory a persistent launch takes (the one-CTA
// levels stay within 48 KB).
constexpr int PERSIST_MAX_DYN_SMEM = 64 * 1024;

// Sets the kernels' dynamic shared memory limit to PERSIST_MAX_DYN_SMEM (a
// fixed value, so grids created later never lower it).
cudaError_t persist_prepare();

// Persistent CTAs that fit on one SM (0: the solve cannot run persistently).
int persist_blocks_per_sm(bool fp32, size_t smem);

// Launches the solve on `grid` CTAs of PERSIST_THREADS threads with `smem`
// bytes of dynamic shared memory (the one-CTA multigrid levels) on stream st.
cudaError_t persist_solve_launch(const PSolve<float>& a, int grid, size_t smem, cudaStream_t st);
cudaError_t persist_solve_launch(const PSolve<double>& a, int grid, size_t smem, cudaStream_t st);

}  // namespace nsk
