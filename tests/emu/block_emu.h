// Host emulation of one CTA of the one-CTA multigrid kernel (test support).
//
// The kernel's source, taken verbatim from csrc/ns_mg.cuh by the test, is
// compiled as host C++ with the CUDA keywords below: every thread of the CTA
// is a std::thread, __syncthreads() is a barrier over all of them, and a warp
// shuffle is an exchange through a per-warp buffer between two barriers over
// the warp's 32 threads.  Shared memory is one heap block of exactly the size
// the library requests, so AddressSanitizer reports any access outside it.
#pragma once
#include <algorithm>
#include <atomic>
#include <barrier>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

using std::max;
using std::min;

#define __device__
#define __global__
#define __forceinline__ inline
#define __launch_bounds__(x)
#define __restrict__
#define __align__(x)
#define __grid_constant__
#define NS_PERSISTENT_GROUPS 1
// the kernels' dependent-launch wait: nothing to wait for on the host
#define NS_HOST_EMULATION 1
inline void pdl_wait() {}

struct EmuDim3 {
    unsigned x = 0, y = 0, z = 0;
};
thread_local EmuDim3 threadIdx, blockIdx;
// unset extents are 1, as in a launch (a 1-D CTA has blockDim.y = blockDim.z = 1)
EmuDim3 blockDim{0, 1, 1}, gridDim{0, 1, 1};

std::barrier<>* emu_cta_barrier;
std::barrier<>* emu_warp_barrier[32];
unsigned char* emu_smem;

inline void __syncthreads() { emu_cta_barrier->arrive_and_wait(); }

template <typename T>
inline T __shfl_sync(unsigned, T v, int src) {
    static T buf[32][32];
    const int lane = (int)threadIdx.x % 32, w = (int)threadIdx.x / 32;
    buf[w][lane] = v;
    emu_warp_barrier[w]->arrive_and_wait();
    const T r = buf[w][src];
    emu_warp_barrier[w]->arrive_and_wait();
    return r;
}

// IEEE single-precision reciprocal, rounded to nearest (as __frcp_rn)
inline float __frcp_rn(float x) { return 1.0f / x; }
inline float __fdividef(float a, float b) { return a / b; }

// --- further device primitives used by the grid-wide multigrid kernels ------
// (CTAs of a grid run one after another, so "global" atomics and fences only
// need to be ordinary operations; a CTA's static shared arrays are the
// function-local statics that __shared__ becomes)
#define __shared__ static
struct float2 {
    float x, y;
};
struct double2 {
    double x, y;
};
template <typename T>
inline T __shfl_xor_sync(unsigned, T v, int mask) {
    static T buf[32][32];
    const int lane = (int)(threadIdx.y * 32 + threadIdx.x) % 32;
    const int w = (int)(threadIdx.y * 32 + threadIdx.x) / 32;
    buf[w][lane] = v;
    emu_warp_barrier[w]->arrive_and_wait();
    const T r = buf[w][lane ^ mask];
    emu_warp_barrier[w]->arrive_and_wait();
    return r;
}
inline void __threadfence() { std::atomic_thread_fence(std::memory_order_seq_cst); }
template <typename T>
inline T __ldcg(const T* p) { return *p; }
inline int __popc(unsigned x) { return __builtin_popcount(x); }
using std::isfinite;
inline unsigned atomicAdd(unsigned* p, unsigned v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
template <typename T>
inline T __shfl_up_sync(unsigned, T v, int delta) {
    static T buf[32][32];
    const int t = (int)(threadIdx.y * 32 + threadIdx.x);
    const int lane = t % 32, w = t / 32;
    buf[w][lane] = v;
    emu_warp_barrier[w]->arrive_and_wait();
    const T r = lane >= delta ? buf[w][lane - delta] : v;
    emu_warp_barrier[w]->arrive_and_wait();
    return r;
}
inline unsigned long long atomicMax(unsigned long long* p, unsigned long long v) {
    unsigned long long old = *p;
    while (old < v && !__atomic_compare_exchange_n(p, &old, v, false, __ATOMIC_SEQ_CST,
                                                   __ATOMIC_SEQ_CST)) {
    }
    return old;
}
inline long long __double_as_longlong(double x) {
    long long r;
    std::memcpy(&r, &x, sizeof r);
    return r;
}
struct float3 {
    float x, y, z;
};
inline double atomicAdd(double* p, double v) {
    return std::atomic_ref<double>(*p).fetch_add(v);
}
inline bool __any_sync(unsigned, bool v) {
    static bool buf[32][32];
    const int t = (int)(threadIdx.y * 32 + threadIdx.x);
    const int lane = t % 32, w = t / 32;
    buf[w][lane] = v;
    emu_warp_barrier[w]->arrive_and_wait();
    bool r = false;
    for (int q = 0; q < 32; ++q) r = r || buf[w][q];
    emu_warp_barrier[w]->arrive_and_wait();
    return r;
}
