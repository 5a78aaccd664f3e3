// Persistent pressure solve: a whole multigrid-preconditioned BiCGStab solve
// (Section 2 names BiCGStab; the V-cycle preconditioner and the FP32 inner /
// FP64-accurate outer refinement are those of ns_mg.cuh) in one cooperative
// launch.  Every phase is the body of the kernel the stream and graph paths
// launch for it: this file compiles ns_mg.cuh with its kernels turned into
// inlined device functions whose block index is a virtual one, so each
// persistent CTA runs the phase's CTAs as its eight 128-thread groups and a
// grid-wide barrier takes the place of the kernel boundary.  The arithmetic,
// the per-CTA partial sums and the fixed order of every reduction are those of
// the launched kernels, so the results are bit-identical to theirs.
//
// Every wait at a barrier is bounded (spin_ns of the global timer): a CTA that
// gives up sets the error flag, and every CTA that sees the flag returns, so a
// missing CTA ends the launch with an error the host reads instead of a hang.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

// every CTA runs eight 128-thread groups (ns_device.cuh)
#define NS_PERSISTENT_GROUPS 8

// The virtual block index the kernel bodies below read as blockIdx: one slot
// per 128-thread group of the CTA (threadIdx.z), written before each body.
namespace nsk {
struct VBlock {
    unsigned x, y, z;
};
__shared__ VBlock g_pvb[8];
__device__ __forceinline__ VBlock persist_vblock() { return g_pvb[threadIdx.z]; }
}  // namespace nsk

#pragma push_macro("__global__")
#pragma push_macro("__launch_bounds__")
#pragma push_macro("__grid_constant__")
#undef __global__
#define __global__ __device__ __forceinline__
#undef __launch_bounds__
#define __launch_bounds__(...)
#undef __grid_constant__
#define __grid_constant__
#define blockIdx (::nsk::persist_vblock())
#include "ns_mg.cuh"
#undef blockIdx
#pragma pop_macro("__grid_constant__")
#pragma pop_macro("__launch_bounds__")
#pragma pop_macro("__global__")

#include "ns_persist.h"

namespace nsk {

static_assert(NSUB == PERSIST_GROUPS && NSUB == 8, "one virtual-block slot per group");

namespace {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

__device__ __forceinline__ bool first_thread() {
    return threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;
}

// Grid-wide barrier (all CTAs of the cooperative launch).  Thread 0 of each
// CTA makes the CTA's writes visible (fence), arrives at bar[0] and polls the
// generation bar[PERSIST_BAR_GEN] (a cache line away) until it moves on; the
// last arrival resets the count and releases the next generation.  A wait
// longer than spin_ns, or an error flag set by another CTA, ends the wait;
// returns false then.
__device__ __noinline__ bool grid_sync(unsigned* bar, int* err, long long spin_ns) {
    __shared__ int ok;
    __syncthreads();
    if (first_thread()) {
        unsigned* gen_p = bar + PERSIST_BAR_GEN;
        const unsigned gen = ld_acquire_u32(gen_p);
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        int good = 1;
        if (arrived == gridDim.x) {
            bar[0] = 0u;
            st_release_u32(gen_p, gen + 1u);
        } else {
            const long long t0 = global_ns();
            unsigned polls = 0;
            while (ld_relaxed_u32(gen_p) == gen) {
                if ((++polls & 63u) == 0u) {
                    if (ld_relaxed_i32(err) != 0) {
                        good = 0;
                        break;
                    }
                    if (global_ns() - t0 > spin_ns) {
                        atomicExch(err, 1);
                        good = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        ok = good && ld_relaxed_i32(err) == 0;
    }
    __syncthreads();
    return ok != 0;
}

// Runs `body` for the nvx x batch virtual CTAs of a phase: group z of CTA b
// takes the virtual CTAs z * gridDim.x + b, then + 8 gridDim.x, ..., so a
// phase with fewer virtual CTAs than groups still spreads over every SM.
template <typename F>
__device__ __forceinline__ void phase(int nvx, int batch, F&& body) {
    const int groups = (int)gridDim.x * NSUB;
    const int total = nvx * batch;
    for (int v = (int)threadIdx.z * (int)gridDim.x + (int)blockIdx.x; v < total; v += groups) {
        if (threadIdx.x == 0 && threadIdx.y == 0)
            g_pvb[threadIdx.z] = VBlock{(unsigned)(v % nvx), (unsigned)(v / nvx), 0u};
        sub_sync();
        body();
        sub_sync();
    }
}

}  // namespace
}  // namespace nsk

namespace nsk {
namespace {

// The one-CTA levels: CTA s (< batch) runs the state s with all its threads.
template <typename T>
__device__ __forceinline__ void block_levels(const PSolve<T>& a, const T* in, const T* in_odd,
                                             T* out) {
    if ((int)blockIdx.x < a.batch) {
        if (threadIdx.x == 0 && threadIdx.y == 0)
            g_pvb[threadIdx.z] = VBlock{blockIdx.x, 0u, 0u};
        __syncthreads();
        mg_block_levels<T>(a.plan, a.ctl, in, in_odd, out, blockIdx.x);
        __syncthreads();
    }
}

#define NS_PSYNC() \
    if (!grid_sync(a.bar, a.err, a.spin_ns)) return false

// One application of the V-cycle, phase for phase the launches of the host's
// mg_apply (the same kernel choice per level).
template <typename T, int MODE>
__device__ bool p_mg_apply(const PSolve<T>& a, const MgBuf<T>& mb, T* src, T* src_odd, T* dst) {
    const MgPlan& P = a.plan;
    const int lc = P.lc, B = a.batch;
    const Lev& L0 = P.lev[0];
    if (lc > 0 && L0.fcode == nullptr && L0.n[0] % 2 == 0) {
        const int pbx = (L0.n[0] + 63) / 64;
        phase(pbx * L0.by * L0.bz, B,
              [&] { k_mg_src_pair<T, MODE>(L0, mb, a.ctl, nullptr, dst, pbx); });
    } else if (lc > 0) {
        phase(L0.ctas, B, [&] { k_mg_src<T, MODE, true>(L0, mb, a.ctl, nullptr, dst); });
    } else {
        phase(L0.ctas, B, [&] { k_mg_src<T, MODE, false>(L0, mb, a.ctl, nullptr, dst); });
    }
    NS_PSYNC();
    for (int l = 0; l < lc; ++l) {
        const T* bsrc = l == 0 ? src : mb.B[l];
        const T* bsrc_odd = l == 0 ? src_odd : nullptr;
        const T* ysrc = l == 0 ? dst : mb.Yl[l];
        phase(P.lev[l].rctas, B, [&] {
            k_mg_restrict<T>(P.lev[l], P.lev[l + 1], a.ctl, bsrc, bsrc_odd, ysrc, mb.B[l + 1]);
        });
        NS_PSYNC();
        if (l + 1 < lc) {
            const Lev& Ls = P.lev[l + 1];
            if (Ls.fcode == nullptr && Ls.n[0] % 2 == 0) {
                const int pbx = (Ls.n[0] + 63) / 64;
                phase(pbx * Ls.by * Ls.bz, B, [&] {
                    k_mg_src_pair<T, SRC_ARR>(Ls, mb, a.ctl, mb.B[l + 1], mb.Yl[l + 1], pbx);
                });
            } else {
                phase(Ls.ctas, B, [&] {
                    k_mg_src<T, SRC_ARR, true>(Ls, mb, a.ctl, mb.B[l + 1], mb.Yl[l + 1]);
                });
            }
            NS_PSYNC();
        }
    }
    block_levels<T>(a, lc == 0 ? src : mb.B[lc], lc == 0 ? src_odd : nullptr,
                    lc == 0 ? dst : mb.Yl[lc]);
    NS_PSYNC();
    for (int l = lc - 1; l >= 0; --l) {
        T* y = l == 0 ? dst : mb.Yl[l];
        const Lev& L = P.lev[l];
        if (L.fcode == nullptr) {
            const int pbx = (L.n[0] + 63) / 64;
            phase(pbx * L.by * L.bz, B, [&] {
                k_mg_prolong_pair<T>(L, P.lev[l + 1], a.ctl, y, mb.Yl[l + 1], pbx);
            });
        } else {
            phase(L.ctas, B,
                  [&] { k_mg_prolong<T>(L, P.lev[l + 1], a.ctl, y, mb.Yl[l + 1]); });
        }
        NS_PSYNC();
    }
    return true;
}

// One preconditioned BiCGStab iteration, as the host's mg_iteration.
template <typename T>
__device__ bool p_mg_iteration(const PSolve<T>& a, double tol2, int zero_start) {
    const MgBuf<T>& mb = a.mb;
    const Lev& L0 = a.plan.lev[0];
    const int B = a.batch;
    const bool pair = L0.fcode == nullptr && L0.n[0] % 2 == 0;
    const int pbx = (L0.n[0] + 63) / 64;
    const int pctas = pbx * L0.by * L0.bz;
    if (!p_mg_apply<T, SRC_P>(a, mb, mb.P[0], mb.P[1], mb.Y)) return false;
    if (pair)
        phase(pctas, B, [&] { k_mg_lapdot_pair<T, 0>(L0, mb, a.ctl, a.part_mg, pbx, pctas); });
    else
        phase(L0.ctas, B, [&] { k_mg_lapdot_v<T>(L0, mb, a.ctl, a.part_mg); });
    NS_PSYNC();
    if (!p_mg_apply<T, SRC_S>(a, mb, mb.S, nullptr, mb.Z)) return false;
    if (pair)
        phase(pctas, B, [&] { k_mg_lapdot_pair<T, 1>(L0, mb, a.ctl, a.part_mg, pbx, pctas); });
    else
        phase(L0.ctas, B, [&] { k_mg_lapdot_t<T>(L0, mb, a.ctl, a.part_mg); });
    NS_PSYNC();
    if (pair)
        phase(pctas, B, [&] {
            k_mg_update_pair<T>(L0, mb, a.ctl, a.part_mg, tol2, a.maxit, zero_start, pbx, pctas);
        });
    else
        phase(L0.ctas, B,
              [&] { k_mg_update<T>(L0, mb, a.ctl, a.part_mg, tol2, a.maxit, zero_start); });
    NS_PSYNC();
    return true;
}

// End of a solve, as the exit of the graph loops' condition kernel: loop
// counts, the sticky failure bits and the per-state totals.
template <typename T>
__device__ void p_finish(const PSolve<T>& a, unsigned count, bool outer) {
    if (blockIdx.x != 0 || !first_thread()) return;
    a.loopc->inner = count;
    a.loopc->inner_total += count;
    for (int s = 0; s < a.batch; ++s) {
        SliceCtl* c = a.ctl + s;
        if (outer) {
            if (c->o_status == OS_NONFINITE) c->fail |= 2;
            else if (c->o_status != OS_DONE) c->fail |= 1;
            c->total_outer += c->o_steps;
        } else {
            if (c->status == ST_NONFINITE) c->fail |= 2;
            else if (c->status != ST_CONV) c->fail |= 1;
        }
        c->total_solves += 1;
    }
}

// Does any state still iterate (FP64) / refine (FP32+refine)?  Read by every
// thread after a barrier, so every CTA takes the same decision.
template <typename T>
__device__ __forceinline__ bool p_any(const PSolve<T>& a, bool outer) {
    bool any = false;
    for (int s = 0; s < a.batch; ++s) {
        const SliceCtl* c = a.ctl + s;
        any = any || (outer ? __ldcg(&c->o_status) == OS_REFINE : __ldcg(&c->status) == ST_ITER);
    }
    return any;
}

// FP32 inner iterations inside float-float refinement: the start, then one
// loop whose body is an inner iteration followed by the outer correction of
// every state whose inner solve has ended (the graph-resident form).
__device__ bool p_solve(const PSolve<float>& a) {
    const Lev& L0 = a.plan.lev[0];
    const int B = a.batch;
    if (a.p_in)
        phase(L0.ctas, B, [&] {
            k_mg_refine_init_ff<true>(L0, a.mb, a.ctl, a.part_div, a.n_fluid, a.b, a.p_in, a.ff,
                                      a.part_mg, a.otol2, a.itol2, a.maxit);
        });
    else
        phase(L0.ctas, B, [&] {
            k_mg_refine_init_ff<false>(L0, a.mb, a.ctl, a.part_div, a.n_fluid, a.b, nullptr,
                                       a.ff, a.part_mg, a.otol2, a.itol2, a.maxit);
        });
    NS_PSYNC();
    unsigned count = 0;
    while (p_any(a, true) && count < a.cap) {
        if (!p_mg_iteration<float>(a, a.itol2, 1)) return false;
        phase(L0.ctas, B, [&] {
            k_mg_refine_update_ff(L0, a.mb, a.ctl, a.ff, a.n_fluid, a.part_mg, a.otol2, a.itol2,
                                  a.maxit, a.max_outer, 1);
        });
        NS_PSYNC();
        ++count;
    }
    p_finish(a, count, true);
    return true;
}

// FP64: the warm start, then iterations while any state iterates.
__device__ bool p_solve(const PSolve<double>& a) {
    const Lev& L0 = a.plan.lev[0];
    const int B = a.batch;
    const double* x0 = a.p_in ? a.p_in : a.p_prev;
    phase(L0.ctas, B, [&] {
        k_mg_init_warm<double>(L0, a.mb, a.ctl, a.part_div, a.n_fluid, a.b, x0, a.part_mg,
                               a.tol2, a.maxit);
    });
    NS_PSYNC();
    unsigned count = 0;
    while (p_any(a, false) && count < a.cap) {
        if (!p_mg_iteration<double>(a, a.tol2, 0)) return false;
        ++count;
    }
    p_finish(a, count, false);
    return true;
}

#undef NS_PSYNC

}  // namespace

template <typename T>
__global__ void __launch_bounds__(PERSIST_THREADS, 1)
    k_persist_solve(const __grid_constant__ PSolve<T> a) {
    p_solve(a);
}

cudaError_t persist_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_persist_solve<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         PERSIST_MAX_DYN_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_persist_solve<double>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 PERSIST_MAX_DYN_SMEM);
    return e;
}

int persist_blocks_per_sm(bool fp32, size_t smem) {
    int n = 0;
    const cudaError_t e =
        fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persist_solve<float>,
                                                            PERSIST_THREADS, smem)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_persist_solve<double>,
                                                            PERSIST_THREADS, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <typename T>
static cudaError_t launch_coop(const PSolve<T>& a, int grid, size_t smem, cudaStream_t st) {
    PSolve<T> arg = a;
    void* params[] = {&arg};
    return cudaLaunchCooperativeKernel((const void*)k_persist_solve<T>, dim3(grid),
                                       dim3(TX, TY, NSUB), params, smem, st);
}

cudaError_t persist_solve_launch(const PSolve<float>& a, int grid, size_t smem, cudaStream_t st) {
    return launch_coop(a, grid, smem, st);
}

cudaError_t persist_solve_launch(const PSolve<double>& a, int grid, size_t smem,
                                 cudaStream_t st) {
    return launch_coop(a, grid, smem, st);
}

}  // namespace nsk
