// Host emulation of one thread-block cluster of the cluster multigrid kernel
// (test support).
//
// The kernel's source, taken verbatim from csrc/ns_mg.cuh and
// csrc/ns_mg_cluster.cuh by the test, is compiled as host C++ with the CUDA
// keywords below: every thread of every CTA is a std::thread,
// __syncthreads() is a barrier over the threads of the caller's CTA, the
// cluster barrier one over all threads of the cluster, and a cluster-mapped
// address is the same offset in the other CTA's shared-memory block.  Each
// CTA's shared memory is its own heap block of exactly the size the library
// requests, so AddressSanitizer reports any access outside it.
#pragma once
#include <algorithm>
#include <barrier>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <optional>
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
#define NS_HOST_EMULATION 1
inline void pdl_wait() {}

struct EmuDim3 {
    unsigned x = 0, y = 0, z = 0;
};
thread_local EmuDim3 threadIdx, blockIdx;
EmuDim3 blockDim{0, 1, 1}, gridDim{0, 1, 1};

// per thread: its CTA's barrier, shared memory and rank in the cluster
thread_local std::barrier<>* emu_cta_barrier;
thread_local unsigned char* emu_smem;
thread_local int emu_rank;
thread_local std::optional<std::barrier<>::arrival_token> emu_token;
// the cluster: its barrier and every CTA's shared memory
std::barrier<>* emu_cl_barrier;
std::vector<unsigned char*> emu_cl_smem;
// warps of rank 0 (the only CTA that shuffles: the rank-0 levels)
std::barrier<>* emu_warp_barrier[32];

inline void __syncthreads() { emu_cta_barrier->arrive_and_wait(); }
// a barrier over the caller's warp (only rank 0's warps use the warp barriers)
inline void __syncwarp() { emu_warp_barrier[threadIdx.x / 32]->arrive_and_wait(); }

inline unsigned cl_rank() { return (unsigned)emu_rank; }
inline void cl_sync() { emu_cl_barrier->arrive_and_wait(); }
inline void cl_arrive() { emu_token.emplace(emu_cl_barrier->arrive()); }
inline void cl_wait() {
    emu_cl_barrier->wait(std::move(*emu_token));
    emu_token.reset();
}
template <typename T>
inline T* cl_map(T* p, unsigned rank) {
    const std::ptrdiff_t off = reinterpret_cast<unsigned char*>(p) - emu_smem;
    return reinterpret_cast<T*>(emu_cl_smem.at(rank) + off);
}

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

struct float2 {
    float x, y;
};
struct float4 {
    float x, y, z, w;
};
struct double2 {
    double x, y;
};

// IEEE single-precision reciprocal, rounded to nearest (as __frcp_rn)
inline float __frcp_rn(float x) { return 1.0f / x; }
inline float __fdividef(float a, float b) { return a / b; }
