// Device-side building blocks of the batched MAC-grid projection stepper:
// grid geometry, boundary (ghost) rules, the SMART face value, the masked
// 7-point Laplacian and deterministic per-state reductions.
//
// Discretisation (Croce, Ruprecht & Krause, Section 2): uniform Cartesian
// staggered mesh, forward-Euler Chorin-Temam projection, central differences
// for diffusion and the pressure gradient, SMART (bounded QUICK) upwinding for
// the conservative convective fluxes, homogeneous Neumann pressure conditions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nsk {

enum { BC_WALL = 0, BC_PERIODIC = 1, BC_SLIP = 2 };

// CTA shape of every cell/face kernel: TX x TY threads, each thread marching
// over `tz` cells along z.
constexpr int TX = 32;
constexpr int TY = 4;
constexpr int NTHREADS = TX * TY;
constexpr int NWARPS = NTHREADS / 32;
// Groups of NTHREADS threads (threadIdx.z) that one CTA runs as separate
// cell-kernel CTAs: 1 for the launched kernels; the persistent solver's
// translation unit defines NS_PERSISTENT_GROUPS (1024-thread CTAs).
#ifndef NS_PERSISTENT_GROUPS
#define NS_PERSISTENT_GROUPS 1
#endif
constexpr int NSUB = NS_PERSISTENT_GROUPS;

// The calling thread's group (0 in the launched kernels).
__device__ __forceinline__ int sub_id() { return NSUB > 1 ? (int)threadIdx.z : 0; }

#ifndef NS_HOST_EMULATION
// First statement of every kernel of the solve and step sequence.  With a
// programmatic dependency on the previous kernel (the coarse chain's graph
// edges), this kernel's CTAs may become resident before that kernel ends:
// they wait here for its completion and memory, then allow the next kernel
// to start launching (it fires once every CTA of this grid has passed this
// point, so a waiting successor never holds the slots this grid's later CTAs
// need).  Without such a dependency both instructions return at once.
__device__ __forceinline__ void pdl_wait() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
#endif

// Barrier over the NTHREADS threads of a (sub-)CTA: __syncthreads in the
// launched kernels, one named barrier per group in the persistent solver.
__device__ __forceinline__ void sub_sync() {
#if defined(__CUDA_ARCH__) && NS_PERSISTENT_GROUPS > 1
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.z), "r"(NTHREADS) : "memory");
#else
    __syncthreads();
#endif
}

struct Geo {
    int n[3];            // cells per axis
    int bc[3];           // BC_* per axis
    int ext[3][3];       // ext[c][d]: stored positions of velocity component c along axis d
    long long cnt[4];    // elements of u, v, w, p in one state
    double h[3], ih[3], ih2[3];
    double inv_re, u_lid;
    int tz;              // cells per thread along z
    int bx, by, bz, ctas;      // cell kernels: CTA tiles per state
    int fbx, fby, fbz, fctas;  // face kernels: CTA tiles over (n+1) per axis
    int n_fluid;         // fluid cells per state
    const uint8_t* solid;  // device cell mask (1 = solid), nullptr without obstacles
    float fih[3], fih2[3], finv_re;  // FP32 copies (no FP64 conversions in FP32 kernels)
    int pty, ptz;        // predictor tile: 32 x pty x ptz cells
};

// h^-1, h^-2 and 1/Re in the kernel's precision
template <typename T> __device__ __forceinline__ T g_ih(const Geo& g, int d);
template <> __device__ __forceinline__ float g_ih<float>(const Geo& g, int d) { return g.fih[d]; }
template <> __device__ __forceinline__ double g_ih<double>(const Geo& g, int d) { return g.ih[d]; }
template <typename T> __device__ __forceinline__ T g_ih2(const Geo& g, int d);
template <> __device__ __forceinline__ float g_ih2<float>(const Geo& g, int d) { return g.fih2[d]; }
template <> __device__ __forceinline__ double g_ih2<double>(const Geo& g, int d) { return g.ih2[d]; }
template <typename T> __device__ __forceinline__ T g_inv_re(const Geo& g);
template <> __device__ __forceinline__ float g_inv_re<float>(const Geo& g) { return g.finv_re; }
template <> __device__ __forceinline__ double g_inv_re<double>(const Geo& g) { return g.inv_re; }

__device__ __forceinline__ int tid_flat() { return threadIdx.y * TX + threadIdx.x; }

__device__ __forceinline__ void tile_origin(const Geo& g, int cta, int bx, int by, int& i, int& j,
                                            int& k0) {
    int tx = cta % bx;
    int r = cta / bx;
    int ty = r % by;
    int tzb = r / by;
    i = tx * TX + threadIdx.x;
    j = ty * TY + threadIdx.y;
    k0 = tzb * g.tz;
}

__device__ __forceinline__ long long vindex(const Geo& g, int c, int i, int j, int k) {
    return ((long long)k * g.ext[c][1] + j) * g.ext[c][0] + i;
}

__device__ __forceinline__ long long cindex(const Geo& g, int i, int j, int k) {
    return ((long long)k * g.n[1] + j) * g.n[0] + i;
}

// Value of velocity component c at (i,j,k), up to two positions outside the
// stored range.  Ghost rules per axis d:
//   periodic                  wrap;
//   normal component (d == c) odd reflection about the wall face (value 0 there);
//   tangential, wall          2*u_wall - mirror (u_wall = u_lid for u on y = ly);
//   tangential, slip          +mirror.
template <typename T>
__device__ __forceinline__ void ghost_axis(const Geo& g, int c, int d, int& x, T& sign, T& add) {
    const int e = g.ext[c][d];
    if (x >= 0 && x < e) return;
    const int n = g.n[d];
    if (g.bc[d] == BC_PERIODIC) {
        x = x < 0 ? x + e : x - e;
    } else if (d == c) {
        x = x < 0 ? -x : 2 * n - x;
        sign = -sign;
    } else {
        const bool hi = x >= e;
        x = hi ? 2 * n - 1 - x : -x - 1;
        if (g.bc[d] == BC_WALL) {
            sign = -sign;
            if (c == 0 && d == 1 && hi) add = T(2.0 * g.u_lid);
        }
    }
}

template <typename T>
__device__ __forceinline__ T vel(const Geo& g, int c, const T* __restrict__ a, int i, int j,
                                 int k) {
    int q[3] = {i, j, k};
    T sign = T(1);
    T add = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) ghost_axis(g, c, d, q[d], sign, add);
    return add + sign * a[vindex(g, c, q[0], q[1], q[2])];
}

// SMART face value from far-upwind U, upwind C and downwind D node values,
// written without a division: with cc = C-U, dd = D-U the normalised variable
// is cc/dd, and the face value U + f(cc/dd)*dd is
//   C                         if cc/dd is outside [0,1] (first-order upwind),
//   U + 3 cc                  on [0, 1/6],
//   U + 3/4 cc + 3/8 dd       on [1/6, 5/6] (QUICK),
//   D                         on [5/6, 1];
// a flat far field (dd == 0) takes C.
template <typename T>
__device__ __forceinline__ T smart_face(T U, T C, T D) {
    const T dd = D - U;
    const T cc = C - U;
    if (dd == T(0)) return C;
    const T a = dd > T(0) ? cc : -cc;
    const T b = fabs(dd);
    if (a < T(0) || a > b) return C;
    if (T(6) * a <= b) return U + T(3) * cc;
    if (T(6) * a <= T(5) * b) return U + T(0.75) * cc + T(0.375) * dd;
    return D;
}

// Convective flux uf * phi_face through a face between node values b (lower
// index) and f (higher index); bb lies behind b and ff in front of f.
template <typename T>
__device__ __forceinline__ T smart_flux(T uf, T bb, T b, T f, T ff) {
    if (uf > T(0)) return uf * smart_face(bb, b, f);
    if (uf < T(0)) return uf * smart_face(ff, f, b);
    return T(0);
}

// The same flux without branches (for warps whose faces take different
// SMART branches): pick the upwind triple, evaluate every branch, select.
// uf = 0 gives 0 as above (the face value is finite).
template <typename T>
__device__ __forceinline__ T smart_flux_sel(T uf, T bb, T b, T f, T ff) {
    const bool pos = uf > T(0);
    const T U = pos ? bb : ff;
    const T C = pos ? b : f;
    const T D = pos ? f : b;
    const T dd = D - U;
    const T cc = C - U;
    const T a = dd > T(0) ? cc : -cc;
    const T bd = fabs(dd);
    const T quick = fma(T(0.75), cc, fma(T(0.375), dd, U));
    const T steep = fma(T(3), cc, U);
    T phi = (T(6) * a <= bd) ? steep : ((T(6) * a <= T(5) * bd) ? quick : D);
    phi = (dd == T(0) || a < T(0) || a > bd) ? C : phi;
    return uf * phi;
}

__device__ __forceinline__ bool cell_solid(const Geo& g, int i, int j, int k) {
    return g.solid != nullptr && g.solid[cindex(g, i, j, k)] != 0;
}

// 7-point Laplacian at cell (i,j,k) of the field returned by val(i,j,k), with
// the value at the cell already in vc.  Wall faces are dropped (homogeneous
// Neumann); periodic axes wrap.  Terms are added axis by axis, the high face
// before the low face.
// With solid cells, a face next to a solid is dropped like a wall face and a
// solid cell's own row is zero.
template <typename T, typename F>
__device__ __forceinline__ T lap_cell(const Geo& g, const F& val, int i, int j, int k, T vc) {
    T s = T(0);
    const int c[3] = {i, j, k};
    if (g.solid != nullptr && cell_solid(g, i, j, k)) return s;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int n = g.n[d];
        const T w = g_ih2<T>(g, d);
        int hi[3] = {c[0], c[1], c[2]};
        int lo[3] = {c[0], c[1], c[2]};
        bool has_hi, has_lo;
        if (g.bc[d] == BC_PERIODIC) {
            hi[d] = c[d] + 1 == n ? 0 : c[d] + 1;
            lo[d] = c[d] == 0 ? n - 1 : c[d] - 1;
            has_hi = has_lo = true;
        } else {
            hi[d] = c[d] + 1;
            lo[d] = c[d] - 1;
            has_hi = hi[d] < n;
            has_lo = lo[d] >= 0;
        }
        if (g.solid != nullptr) {
            has_hi = has_hi && !cell_solid(g, hi[0], hi[1], hi[2]);
            has_lo = has_lo && !cell_solid(g, lo[0], lo[1], lo[2]);
        }
        if (has_hi) s += (val(hi[0], hi[1], hi[2]) - vc) * w;
        if (has_lo) s -= (vc - val(lo[0], lo[1], lo[2])) * w;
    }
    return s;
}

// Is the stored face of component c at f a face that moves fluid: not a
// wall-normal boundary face and, with solids, both neighbouring cells fluid.
__device__ __forceinline__ bool face_active_dev(const Geo& g, int c, const int f[3]) {
    const int n = g.n[c];
    if (g.bc[c] != BC_PERIODIC && (f[c] == 0 || f[c] == n)) return false;
    if (g.solid == nullptr) return true;
    int lo[3] = {f[0], f[1], f[2]};
    lo[c] = f[c] == 0 ? n - 1 : f[c] - 1;  // periodic wrap (walls have f[c] >= 1 here)
    int hi[3] = {f[0], f[1], f[2]};
    hi[c] = f[c] == n ? 0 : f[c];
    return !cell_solid(g, lo[0], lo[1], lo[2]) && !cell_solid(g, hi[0], hi[1], hi[2]);
}

// Is the stored face of component c at q (in range) inside a solid: both
// neighbouring cells along c solid (a wall face is not).
__device__ __forceinline__ bool face_in_solid_dev(const Geo& g, int c, const int q[3]) {
    const int n = g.n[c];
    int lo[3] = {q[0], q[1], q[2]}, hi[3] = {q[0], q[1], q[2]};
    if (g.bc[c] == BC_PERIODIC) {
        lo[c] = q[c] == 0 ? n - 1 : q[c] - 1;
        hi[c] = q[c] == n ? 0 : q[c];
    } else {
        if (q[c] == 0 || q[c] == n) return false;
        lo[c] = q[c] - 1;
        hi[c] = q[c];
    }
    return cell_solid(g, lo[0], lo[1], lo[2]) && cell_solid(g, hi[0], hi[1], hi[2]);
}

// Sum of NV per-thread values over the CTA; the result is valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sm_all[NSUB][NV][NWARPS];
    double(&sm)[NV][NWARPS] = sm_all[sub_id()];
    const int t = tid_flat();
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    }
    sub_sync();
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) sm[q][warp] = v[q];
    }
    sub_sync();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double x = lane < NWARPS ? sm[q][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            v[q] = x;
        }
    }
}

// Deterministic sum of the per-CTA partials [ctas][NV] of one state, computed
// by every CTA that needs it (same order in every CTA), broadcast to all
// threads of the CTA.
template <int NV>
__device__ __forceinline__ void reduce_partials(const double* __restrict__ part, int ctas,
                                                double (&out)[NV]) {
    __shared__ double bc_all[NSUB][NV];
    double(&bc)[NV] = bc_all[sub_id()];
    // each thread sums the CTAs t, t + NTHREADS, ... in that order, loading a
    // batch of them before adding so that the batch's reads overlap
    constexpr int UB = NV <= 3 ? 4 : 2;
    double v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = 0.0;
    for (int c0 = tid_flat(); c0 < ctas; c0 += UB * NTHREADS) {
        double buf[UB][NV];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int c = c0 + u * NTHREADS;
#pragma unroll
            for (int q = 0; q < NV; ++q) buf[u][q] = c < ctas ? part[(long long)c * NV + q] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            if (c0 + u * NTHREADS < ctas) {
#pragma unroll
                for (int q = 0; q < NV; ++q) v[q] += buf[u][q];
            }
        }
    }
    block_sum<NV>(v);
    if (tid_flat() == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) bc[q] = v[q];
    }
    sub_sync();
#pragma unroll
    for (int q = 0; q < NV; ++q) out[q] = bc[q];
    sub_sync();
}

template <int NV>
__device__ __forceinline__ void write_partials(double (&v)[NV], double* __restrict__ part) {
    block_sum<NV>(v);
    if (tid_flat() == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) part[q] = v[q];
    }
}

}  // namespace nsk
