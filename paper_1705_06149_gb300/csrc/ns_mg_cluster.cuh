// The coarse levels of the multigrid V-cycle that preconditions the pressure
// solve (the Poisson equation of Section 2) on a thread-block cluster: one
// cluster of C CTAs per state runs, in one launch, everything below the
// finest level's restriction -- the work that otherwise takes three short
// grid-level launches per coarse level plus the one-CTA kernel.
//
// The operator is the V(2,0) cycle of the one-CTA and grid-level kernels:
// per level two damped-Jacobi sweeps from zero, the residual, its restriction
// to the mean of the 8 children, the coarsest level's sweeps, and on the way
// up the trilinear prolongation added to the iterate.
//
// Levels J .. R-1 ("slab levels", every x extent a multiple of 4) are held in
// z slabs with a halo plane below and above: split over the C CTAs (owners
// = C, an even number of planes per CTA, so a slab restricts into the CTA's
// own coarse slab), or -- once a level is small or no longer splits -- whole
// in rank 0 (owners = 1).  A thread works on x quads (4 cells, one 16-byte
// shared-memory access) of one (y, z) row, so a 7-point stencil at 4 cells
// takes 8 accesses.  A level takes two phases down: the second Jacobi sweep
// (the first, y1 = w b / d, comes with the right side), then per coarse cell
// the residual of its 8 children, their mean and the coarse y1; and one
// phase up, the prolongation.  A value a neighbouring owner needs is written
// straight into its halo plane (distributed shared memory); a cluster barrier
// (a CTA barrier on a rank-0 level) publishes it.  Levels R .. nlev-1 (the
// coarsest level, and any level whose x extent is not a multiple of 4) run in
// rank 0 as the one-CTA kernel runs them (mg_block_core).
#pragma once

#include "ns_mg.cuh"

namespace nsk {

constexpr int MG_CL_THREADS = 512;
constexpr int MG_CL_MAX_CTAS = 8;       // the portable cluster size
constexpr long long MG_CL_SMALL = 512;  // slab levels at or below this size: rank 0 alone

// A slab level's constants, computed on the host so that a phase starts
// without an integer division: extents, plane size, x quads per row, planes
// per owner; the work items of the sweep / prolongation (x quads of the
// planes' rows) and of the restriction (x quads of row pairs) with the
// threads per item group (nt / items, 0 with more items than threads); the
// FP32 reciprocals of the item counts and of the quads per row, by which a
// thread index or an item divides exactly (its + 1/2 stays below 2^22).
struct ClLevC {
    int nx, ny, nz, P, nq, pz;
    int nit, git, nrt, grt;
    float rit, rrt, rnq;
    int px, py, pzp;
};

struct ClPlan {
    int J;  // first level (its right side comes from global memory, its result goes there)
    int R;  // first level of the one-CTA core in rank 0 (J < R)
    int C;  // CTAs per cluster
    int own[MG_MAX_LEVELS];  // owners of a slab level: C (split) or 1 (rank 0)
    // shared-memory offsets in elements: the Jacobi weight tables (27 per
    // level, after copies of both plans at the start of shared memory); a
    // slab level's right side B, first iterate Y and second iterate Y2
    // (planes per owner + 2 each); a core level's B and Y (one per cell)
    long long otab;
    long long ob[MG_MAX_LEVELS], oy[MG_MAX_LEVELS], oy2[MG_MAX_LEVELS];
    ClLevC lc[MG_MAX_LEVELS];  // the slab levels' constants
};

// Byte offsets of the plan copies in shared memory.
constexpr size_t CL_OFF_CP = (sizeof(MgPlan) + 15) / 16 * 16;
constexpr size_t CL_HEAD = CL_OFF_CP + (sizeof(ClPlan) + 15) / 16 * 16;

// Elements rounded up so that the next shared-memory array starts 16-byte
// aligned.
inline size_t cl_align(size_t elems, size_t elem) {
    const size_t per = 16 / elem;
    return (elems + per - 1) / per * per;
}

// The cluster plan for clusters of C CTAs (host).  R: the first level from 1
// on whose x extent is not a multiple of 4, or the coarsest level.  The slab
// levels from J on are split over the C CTAs while they have more than
// MG_CL_SMALL cells and a z extent divisible by 2C, then held by rank 0.  J:
// the finest level from 1 on (at most P.lc, whose buffers exist) that splits
// and whose arrays fit max_bytes of shared memory.  The core levels must fit
// the one-CTA core (MG_BLOCK_PER_THREAD cells per thread).  Returns false
// where there is no such plan; else fills Q and the bytes it takes.
inline bool cl_plan(const MgPlan& P, int C, int nt, size_t elem, size_t max_bytes, ClPlan& Q,
                    size_t& bytes) {
    const int nl = P.nlev;
    int R = nl - 1;
    for (int m = 1; m < nl - 1; ++m)
        if (P.lev[m].n[0] % 4 != 0) {
            R = m;
            break;
        }
    if (R < 2 || P.lev[R].cells > (long long)MG_BLOCK_PER_THREAD * MG_CL_THREADS) return false;
    auto splits = [&](int m) {
        return P.lev[m].cells > MG_CL_SMALL && P.lev[m].n[2] % (2 * C) == 0;
    };
    for (int J = 1; J < R && J <= P.lc; ++J) {
        if (!splits(J)) continue;
        ClPlan q{};
        q.J = J;
        q.R = R;
        q.C = C;
        q.otab = (long long)(CL_HEAD / elem);
        size_t o = cl_align(CL_HEAD / elem + 27 * MG_MAX_LEVELS, elem);
        bool split = true;
        for (int m = J; m < R; ++m) {
            const Lev& L = P.lev[m];
            split = split && splits(m);
            q.own[m] = split ? C : 1;
            ClLevC& c = q.lc[m];
            c.nx = L.n[0];
            c.ny = L.n[1];
            c.nz = L.n[2];
            c.P = c.nx * c.ny;
            c.nq = c.nx / 4;
            c.pz = c.nz / q.own[m];
            c.nit = c.nq * c.ny;
            c.git = c.nit <= nt ? nt / c.nit : 0;
            c.nrt = c.nq * (c.ny / 2);
            c.grt = c.nrt <= nt ? nt / c.nrt : 0;
            c.rit = 1.0f / (float)c.nit;
            c.rrt = 1.0f / (float)c.nrt;
            c.rnq = 1.0f / (float)c.nq;
            c.px = L.bc[0] == BC_PERIODIC;
            c.py = L.bc[1] == BC_PERIODIC;
            c.pzp = L.bc[2] == BC_PERIODIC;
            const size_t slab =
                cl_align((size_t)(L.n[2] / q.own[m] + 2) * L.n[0] * L.n[1], elem);
            q.ob[m] = (long long)o;
            q.oy[m] = (long long)(o + slab);
            q.oy2[m] = (long long)(o + 2 * slab);
            o += 3 * slab;
        }
        for (int m = R; m < nl; ++m) {
            const size_t n = cl_align((size_t)P.lev[m].cells, elem);
            q.ob[m] = (long long)o;
            q.oy[m] = (long long)(o + n);
            o += 2 * n;
        }
        if (o * elem > max_bytes) continue;
        Q = q;
        bytes = o * elem;
        return true;
    }
    return false;
}

#ifndef NS_HOST_EMULATION
// This CTA's rank in its cluster.
__device__ __forceinline__ unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Cluster-wide barrier: the shared-memory writes of every CTA (to its own or
// to another CTA's shared memory) before it are visible to all after it.
__device__ __forceinline__ void cl_sync() {
    asm volatile(
        "barrier.cluster.arrive.release.aligned;\n\t"
        "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The two halves of a cluster barrier, for one whose wait comes later.
__device__ __forceinline__ void cl_arrive() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cl_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The generic address of the same shared-memory location in CTA `rank`.
template <typename T>
__device__ __forceinline__ T* cl_map(T* p, unsigned rank) {
    unsigned long long a = reinterpret_cast<unsigned long long>(p), b;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(b) : "l"(a), "r"(rank));
    return reinterpret_cast<T*>(b);
}
#endif

// Four consecutive x cells (16-byte aligned in FP32, two 16-byte halves in
// FP64) and pairs of them.
template <typename T>
struct Q4 {
    T v[4];
};

template <typename T> __device__ __forceinline__ Q4<T> q4_ld(const T* p);
template <> __device__ __forceinline__ Q4<float> q4_ld<float>(const float* p) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    return Q4<float>{{a.x, a.y, a.z, a.w}};
}
template <> __device__ __forceinline__ Q4<double> q4_ld<double>(const double* p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    return Q4<double>{{a.x, a.y, b.x, b.y}};
}
template <typename T> __device__ __forceinline__ void q4_st(T* p, const Q4<T>& q);
template <> __device__ __forceinline__ void q4_st<float>(float* p, const Q4<float>& q) {
    *reinterpret_cast<float4*>(p) = float4{q.v[0], q.v[1], q.v[2], q.v[3]};
}
template <> __device__ __forceinline__ void q4_st<double>(double* p, const Q4<double>& q) {
    reinterpret_cast<double2*>(p)[0] = double2{q.v[0], q.v[1]};
    reinterpret_cast<double2*>(p)[1] = double2{q.v[2], q.v[3]};
}
template <typename T> __device__ __forceinline__ void q2_ld(const T* p, T& a, T& b);
template <> __device__ __forceinline__ void q2_ld<float>(const float* p, float& a, float& b) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    a = v.x;
    b = v.y;
}
template <> __device__ __forceinline__ void q2_ld<double>(const double* p, double& a, double& b) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    a = v.x;
    b = v.y;
}
template <typename T> __device__ __forceinline__ void q2_st(T* p, T a, T b);
template <> __device__ __forceinline__ void q2_st<float>(float* p, float a, float b) {
    *reinterpret_cast<float2*>(p) = float2{a, b};
}
template <> __device__ __forceinline__ void q2_st<double>(double* p, double a, double b) {
    *reinterpret_cast<double2*>(p) = double2{a, b};
}

// Class of a coordinate for the Jacobi weight: 0 the first cell, 1 an inner
// cell, 2 the last cell (1 along a periodic axis).  A cell's weight w / diag
// is the entry cx + 3 cy + 9 cz of its level's table.
__device__ __forceinline__ int cl_cls(int x, int n, bool per) {
    return per ? 1 : (x == 0 ? 0 : (x + 1 == n ? 2 : 1));
}

// The table entry of class c of level L: the diagonal summed as diag_at sums
// it, the weight as blk_wd forms it.
template <typename T>
__device__ __forceinline__ T cl_wd_entry(const Lev& L, int c, T w) {
    const int cls[3] = {c % 3, (c / 3) % 3, c / 9};
    T d = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T wa = lw<T>(L, a);
        if (L.bc[a] == BC_PERIODIC) {
            d -= T(2) * wa;
        } else {
            if (cls[a] != 0) d -= wa;
            if (cls[a] != 2) d -= wa;
        }
    }
    return -neg_over<T>(w, d);
}

// A slab level as CTA r sees it: the plan's constants, the first plane r
// holds, whether it holds planes.
struct ClLev {
    int nx, ny, nz, P, nq, pz, k0;
    int nit, git, nrt, grt;
    float rit, rrt, rnq;
    bool px, py, pzp, held;
};

__device__ __forceinline__ ClLev cl_lev(const ClLevC& c, int owners, int r) {
    ClLev v;
    v.nx = c.nx;
    v.ny = c.ny;
    v.nz = c.nz;
    v.P = c.P;
    v.nq = c.nq;
    v.pz = c.pz;
    v.k0 = owners > 1 ? r * c.pz : 0;
    v.nit = c.nit;
    v.git = c.git;
    v.nrt = c.nrt;
    v.grt = c.grt;
    v.rit = c.rit;
    v.rrt = c.rrt;
    v.rnq = c.rnq;
    v.px = c.px != 0;
    v.py = c.py != 0;
    v.pzp = c.pzp != 0;
    v.held = owners > 1 || r == 0;
    return v;
}

// Exact floor(x / d) for 0 <= x, x + 1/2 < 2^22, with rd = fl32(1 / d): the
// product's relative error is below 2^-23 and x / d lies at least 1/(2d)
// from the next integer.
__device__ __forceinline__ int cl_div(int x, float rd) { return (int)((float(x) + 0.5f) * rd); }

// Where the first and the last plane of an owner's slab go besides the slab
// itself: the halo plane of the owner below / above (across a periodic seam
// too), or across a wall the owner's own halo plane (a copy of the boundary
// plane, so the z face term there is exactly 0).  local: the array's start
// in this CTA's shared memory; vo: the owner's view; lo / hi: generic
// addresses of the planes to write into.
template <typename T>
__device__ __forceinline__ void cl_halo_dst(T* local, const ClLev& vo, int owners, int owner,
                                            T*& lo, T*& hi) {
    const int rl = owners > 1 ? (owner > 0 ? owner - 1 : owners - 1) : owner;
    const int ru = owners > 1 ? (owner + 1 < owners ? owner + 1 : 0) : owner;
    const int top = (vo.pz + 1) * vo.P;
    lo = (vo.k0 > 0 || vo.pzp) ? cl_map(local + top, (unsigned)rl) : cl_map(local, (unsigned)owner);
    hi = (vo.k0 + vo.pz < vo.nz || vo.pzp) ? cl_map(local, (unsigned)ru)
                                           : cl_map(local + top, (unsigned)owner);
}

// The x neighbours of a quad's first and last cell (offsets from the first
// cell): clamped to the cell across a wall, wrapped across a periodic seam.
__device__ __forceinline__ void cl_qx(const ClLev& v, int a, int& lx, int& hx) {
    lx = a > 0 ? -1 : (v.px ? v.nx - 1 : 0);
    hx = a + 1 < v.nq ? 4 : (v.px ? 4 - v.nx : 3);
}

// The y neighbour rows of row j (offsets): clamped / wrapped.
__device__ __forceinline__ void cl_qy(const ClLev& v, int j, int& ly, int& hy) {
    ly = j > 0 ? -v.nx : (v.py ? (v.ny - 1) * v.nx : 0);
    hy = j + 1 < v.ny ? v.nx : (v.py ? -(v.ny - 1) * v.nx : 0);
}

// L a at the quad starting at slab index q (4 cells, values c): face terms
// in blk_lap's order, the x neighbours inside the quad from the quad itself.
template <typename T>
__device__ __forceinline__ Q4<T> cl_lap4(const T* a, int q, int lx, int hx, int ly, int hy,
                                         int P, T w0, T w1, T w2, const Q4<T>& c) {
    const Q4<T> ym = q4_ld(a + q + ly), yp = q4_ld(a + q + hy);
    const Q4<T> zm = q4_ld(a + q - P), zp = q4_ld(a + q + P);
    const T xl = a[q + lx], xh = a[q + hx];
    Q4<T> s;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const T vc = c.v[e];
        const T xm = e > 0 ? c.v[e - 1] : xl;
        const T xp = e < 3 ? c.v[e + 1] : xh;
        T u = T(0);
        u += (xp - vc) * w0;
        u -= (vc - xm) * w0;
        u += (yp.v[e] - vc) * w1;
        u -= (vc - ym.v[e]) * w1;
        u += (zp.v[e] - vc) * w2;
        u -= (vc - zm.v[e]) * w2;
        s.v[e] = u;
    }
    return s;
}

// The weights of a quad's 4 cells on row j, z class cz, from the table wd.
template <typename T>
__device__ __forceinline__ Q4<T> cl_wd4(const T* wd, const ClLev& v, int a, int j, int cz) {
    const int base = 3 * cl_cls(j, v.ny, v.py) + 9 * cz;
    Q4<T> w;
#pragma unroll
    for (int e = 0; e < 4; ++e) w.v[e] = wd[cl_cls(4 * a + e, v.nx, v.px) + base];
    return w;
}

// Work items of a level (x quads or x pairs of rows) spread over the CTA's
// threads: with n <= nt items, G = nt / n threads share an item, taking the
// planes g, g + G, ...; else (G = 0) thread t takes the items t, t + nt, ...
// and every plane.
struct ClItems {
    int i0, is, p0, ps, n;
};

__device__ __forceinline__ ClItems cl_items(int n, int G, float rn, int t, int nt) {
    if (G > 0) {
        const int g = cl_div(t, rn);
        return g < G ? ClItems{t - g * n, n, g, G, n} : ClItems{n, n, 0, 1, n};
    }
    return ClItems{t, nt, 0, 1, n};
}

// Phase 1 of a slab level: y2 = y1 + w (b - L y1) / d on the slab, written to
// Y2 and its boundary planes to lo / hi.
template <typename T>
__device__ __forceinline__ void cl_sweep(const ClLev& v, const T* wd, const T* B, const T* Y,
                                         T* Y2, T* lo, T* hi, T w0, T w1, T w2, int t, int nt) {
    const ClItems it = cl_items(v.nit, v.git, v.rit, t, nt);
    for (int item = it.i0; item < it.n; item += it.is) {
        const int j = cl_div(item, v.rnq), a = item - j * v.nq;
        const int xy = j * v.nx + 4 * a;
        int lx, hx, ly, hy;
        cl_qx(v, a, lx, hx);
        cl_qy(v, j, ly, hy);
        for (int lp0 = it.p0; lp0 < v.pz; lp0 += it.ps) {
            const int q = (lp0 + 1) * v.P + xy;
            const Q4<T> c = q4_ld(Y + q), b = q4_ld(B + q);
            const Q4<T> l = cl_lap4<T>(Y, q, lx, hx, ly, hy, v.P, w0, w1, w2, c);
            const Q4<T> wq = cl_wd4<T>(wd, v, a, j, cl_cls(v.k0 + lp0, v.nz, v.pzp));
            Q4<T> y2;
#pragma unroll
            for (int e = 0; e < 4; ++e) y2.v[e] = c.v[e] + wq.v[e] * (b.v[e] - l.v[e]);
            q4_st(Y2 + q, y2);
            if (lp0 == 0) q4_st(lo + xy, y2);
            if (lp0 == v.pz - 1) q4_st(hi + xy, y2);
        }
    }
}

// Phase 2 of a slab level: per coarse x pair (2a, 2a+1) of coarse row Jc and
// coarse plane Kc0 + K, the residual b - L y2 of the 16 children and each
// coarse cell's mean of its 8 (summed in the one-CTA kernel's order dz, dy,
// dx).  To a slab level (vc: its owner's view): the coarse right side into
// Bc's slab, the coarse y1 into Yc's slab and its boundary planes to lo / hi.
// To the core's first level: the right side alone into Bc (global index).
template <typename T>
__device__ __forceinline__ void cl_restrict(const ClLev& v, const ClLev& vc, const T* wdc,
                                            const T* B, const T* Y2, T* Bc, T* Yc, T* lo, T* hi,
                                            bool to_slab, T w0, T w1, T w2, int t, int nt) {
    const int ncx = v.nx >> 1, pzc = v.pz >> 1, Kc0 = v.k0 >> 1;
    const int ncy = v.ny >> 1, Pc = ncx * ncy;
    const ClItems it = cl_items(v.nrt, v.grt, v.rrt, t, nt);
    for (int item = it.i0; item < it.n; item += it.is) {
        const int Jc = cl_div(item, v.rnq), a = item - Jc * v.nq;
        int lx, hx;
        cl_qx(v, a, lx, hx);
        int ly[2], hy[2];
        cl_qy(v, 2 * Jc, ly[0], hy[0]);
        cl_qy(v, 2 * Jc + 1, ly[1], hy[1]);
        const int xyc = Jc * ncx + 2 * a;
        for (int K = it.p0; K < pzc; K += it.ps) {
            T acc0 = T(0), acc1 = T(0);
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    const int q = (1 + 2 * K + dz) * v.P + (2 * Jc + dy) * v.nx + 4 * a;
                    const Q4<T> c = q4_ld(Y2 + q), b = q4_ld(B + q);
                    const Q4<T> l = cl_lap4<T>(Y2, q, lx, hx, ly[dy], hy[dy], v.P, w0, w1, w2, c);
                    acc0 += b.v[0] - l.v[0];
                    acc0 += b.v[1] - l.v[1];
                    acc1 += b.v[2] - l.v[2];
                    acc1 += b.v[3] - l.v[3];
                }
            const T b0 = acc0 * T(0.125), b1 = acc1 * T(0.125);
            const int Kg = Kc0 + K;
            if (!to_slab) {
                q2_st(Bc + (long long)Kg * Pc + xyc, b0, b1);
                continue;
            }
            const int s = (Kg - vc.k0 + 1) * Pc + xyc;
            q2_st(Bc + s, b0, b1);
            const int base = 3 * cl_cls(Jc, ncy, vc.py) + 9 * cl_cls(Kg, vc.nz, vc.pzp);
            const T y0 = wdc[cl_cls(2 * a, ncx, vc.px) + base] * b0;
            const T y1 = wdc[cl_cls(2 * a + 1, ncx, vc.px) + base] * b1;
            q2_st(Yc + s, y0, y1);
            if (Kg == vc.k0) q2_st(lo + xyc, y0, y1);
            if (Kg == vc.k0 + vc.pz - 1) q2_st(hi + xyc, y0, y1);
        }
    }
}

// Phase up of a slab level: y2 += the trilinear prolongation (tri_axis's
// weights, prolong_off's order) of the coarse correction e, whose plane z
// lies at e + slot(z) Pc, slot(z) = z + zoff, wrapped by nzw (0: no wrap).
// The result stays in Y2 (its boundary planes also to lo / hi when lo is
// given) or, with out given, goes to out.
template <typename T>
__device__ __forceinline__ void cl_prolong(const ClLev& v, const Lev& Lc, const T* e, int zoff,
                                           int nzw, T* Y2, T* lo, T* hi, T* out, int t, int nt) {
    const int ncx = Lc.n[0], ncy = Lc.n[1], nzc = Lc.n[2], Pc = ncx * ncy;
    const bool xper = Lc.bc[0] == BC_PERIODIC;
    const ClItems it = cl_items(v.nit, v.git, v.rit, t, nt);
    for (int item = it.i0; item < it.n; item += it.is) {
        const int j = cl_div(item, v.rnq), a = item - j * v.nq;
        const int xy = j * v.nx + 4 * a;
        // coarse x cells 2a-1 .. 2a+2 as offsets from 2a: clamped across a
        // wall, wrapped across a seam (fine cell 4a+c takes c0 = 2a + c/2 with
        // weight 3/4 and c1 = c0 -+ 1 with 1/4, as tri_axis gives)
        const int om = a > 0 ? -1 : (xper ? ncx - 1 : 0);
        const int op = 2 * a + 2 < ncx ? 2 : (xper ? 2 - ncx : 1);
        int y0, y1;
        T wy;
        tri_axis<T>(j, ncy, Lc.bc[1], y0, y1, wy);
        const T ay = T(1) - wy, ax = T(0.75), wx = T(0.25);
        for (int lp0 = it.p0; lp0 < v.pz; lp0 += it.ps) {
            const int k = v.k0 + lp0, q = (lp0 + 1) * v.P + xy;
            int z0, z1;
            T wz;
            tri_axis<T>(k, nzc, Lc.bc[2], z0, z1, wz);
            int s0 = z0 + zoff, s1 = z1 + zoff;
            if (nzw) {
                s0 += s0 < 0 ? nzw : (s0 >= nzw ? -nzw : 0);
                s1 += s1 < 0 ? nzw : (s1 >= nzw ? -nzw : 0);
            }
            // per coarse plane (z0, then z1): the bilinear values at the 4
            // cells from rows y0, y1 (coarse cells 2a-1 .. 2a+2 at slots 0 .. 3)
            T bl[2][4];
#pragma unroll
            for (int zz = 0; zz < 2; ++zz) {
                const T* p0 = e + (long long)(zz ? s1 : s0) * Pc + 2 * a;
                const T* r0 = p0 + y0 * ncx;
                const T* r1 = p0 + y1 * ncx;
                T c0[4], c1[4];
                c0[0] = r0[om];
                q2_ld(r0, c0[1], c0[2]);
                c0[3] = r0[op];
                c1[0] = r1[om];
                q2_ld(r1, c1[1], c1[2]);
                c1[3] = r1[op];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int i0 = 1 + c / 2, i1 = (c & 1) ? i0 + 1 : i0 - 1;
                    bl[zz][c] = ay * (ax * c0[i0] + wx * c0[i1]) + wy * (ax * c1[i0] + wx * c1[i1]);
                }
            }
            const T az = T(1) - wz;
            Q4<T> y2 = q4_ld(Y2 + q);
#pragma unroll
            for (int c = 0; c < 4; ++c) y2.v[c] = y2.v[c] + (az * bl[0][c] + wz * bl[1][c]);
            if (out) {
                q4_st(out + (long long)k * v.P + xy, y2);
            } else {
                q4_st(Y2 + q, y2);
                if (lo && lp0 == 0) q4_st(lo + xy, y2);
                if (lo && lp0 == v.pz - 1) q4_st(hi + xy, y2);
            }
        }
    }
}

// One V-cycle of levels cp.J .. nlev-1 for the right side `in` (global,
// level J) into `out` (global, level J), by the CTAs of one cluster, every
// thread taking part; the plans and the Jacobi weight tables wdt in shared
// memory.
template <typename T>
__device__ __forceinline__ void mg_cluster_levels(const MgPlan& plan, const ClPlan& cp,
                                                  const T* wdt, const T* __restrict__ in,
                                                  T* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int C = cp.C, J = cp.J, R = cp.R;
    const int r = (int)cl_rank();
    const int t = (int)threadIdx.x, nt = (int)blockDim.x;
    // every CTA of the cluster has started before the first remote write
    cl_arrive();
    {
        // level J (split): b and y1 = w b / d on the slab and its halo planes
        // from global memory; across a wall the halo plane repeats the
        // boundary plane's y1
        const ClLev v = cl_lev(cp.lc[J], C, r);
        const T* wd = wdt + 27 * J;
        T* B = sm + cp.ob[J];
        T* Y = sm + cp.oy[J];
        const ClItems it = cl_items(v.nit, v.git, v.rit, t, nt);
        for (int item = it.i0; item < it.n; item += it.is) {
            const int j = cl_div(item, v.rnq), a = item - j * v.nq;
            const int xy = j * v.nx + 4 * a;
#pragma unroll 2
            for (int lp = it.p0; lp < v.pz + 2; lp += it.ps) {
                int k = v.k0 + lp - 1;
                bool ghost = false;
                if (k < 0 || k >= v.nz) {
                    if (v.pzp) {
                        k = k < 0 ? k + v.nz : k - v.nz;
                    } else {
                        k = k < 0 ? 0 : v.nz - 1;
                        ghost = true;
                    }
                }
                const Q4<T> b = q4_ld(in + (long long)k * v.P + xy);
                if (!ghost) q4_st(B + lp * v.P + xy, b);
                const Q4<T> w = cl_wd4<T>(wd, v, a, j, cl_cls(k, v.nz, v.pzp));
                Q4<T> y;
#pragma unroll
                for (int e = 0; e < 4; ++e) y.v[e] = w.v[e] * b.v[e];
                q4_st(Y + lp * v.P + xy, y);
            }
        }
    }
    __syncthreads();
    cl_wait();
    // down through the slab levels: the split ones by the whole cluster
    // (cluster barriers), then rank 0's (CTA barriers; a rank-0 level of at
    // most 64 cells by warp 0 alone, with warp barriers)
    auto level_sync = [&](bool split, bool tiny) {
        if (split)
            cl_sync();
        else if (r == 0 && !tiny)
            __syncthreads();
        else if (r == 0 && t < 32)
            __syncwarp();
    };
    for (int m = J; m < R; ++m) {
        const int owners = cp.own[m];
        const bool split = owners > 1;
        const ClLev v = cl_lev(cp.lc[m], owners, r);
        // a level of at most 64 cells has at most 16 (quad, plane) items: the
        // CTA-wide grouping gives each its own thread of warp 0
        const bool tiny = !split && v.P * v.nz <= 64;
        const int ntl = tiny ? 32 : nt;
        const bool work = v.held && t < ntl;
        const Lev& L = plan.lev[m];
        const T w0 = lw<T>(L, 0), w1 = lw<T>(L, 1), w2 = lw<T>(L, 2);
        if (work) {
            T *lo, *hi;
            cl_halo_dst(sm + cp.oy2[m], v, owners, r, lo, hi);
            cl_sweep<T>(v, wdt + 27 * m, sm + cp.ob[m], sm + cp.oy[m], sm + cp.oy2[m], lo, hi,
                        w0, w1, w2, t, ntl);
        }
        level_sync(split, tiny);
        if (work) {
            const bool to_slab = m + 1 < R;
            const int oc = to_slab ? cp.own[m + 1] : 1;
            // the owner of this CTA's coarse planes: this CTA when the coarse
            // level splits too, else rank 0
            const unsigned dst = oc > 1 ? (unsigned)r : 0u;
            const ClLev vc = cl_lev(cp.lc[to_slab ? m + 1 : m], oc, (int)dst);
            T* Bc = cl_map(sm + cp.ob[m + 1], dst);
            T* Yc = nullptr;
            T *lo = nullptr, *hi = nullptr;
            if (to_slab) {
                Yc = cl_map(sm + cp.oy[m + 1], dst);
                cl_halo_dst(sm + cp.oy[m + 1], vc, oc, (int)dst, lo, hi);
            }
            cl_restrict<T>(v, vc, wdt + 27 * (m + 1), sm + cp.ob[m], sm + cp.oy2[m], Bc, Yc, lo,
                           hi, to_slab, w0, w1, w2, t, ntl);
        }
        level_sync(split, tiny);
    }
    if (r == 0) {
        // the core levels (the coarsest alone, when it has at most 32 cells:
        // warp 0 with register shuffles), then up through rank 0's slab
        // levels, each after the barrier its predecessor's writers need
        if (R == plan.nlev - 1 && plan.lev[R].cells <= 32) {
            if (t < 32) {
                __syncwarp();
                mg_coarsest_warp<T>(plan.lev[R], sm + cp.ob[R], sm + cp.oy[R], (unsigned)t,
                                    T(MG_OMEGA));
            }
        } else {
            __syncthreads();
            T* bq[MG_MAX_LEVELS];
            T* yq[MG_MAX_LEVELS];
            for (int m = R; m < plan.nlev; ++m) {
                bq[m] = sm + cp.ob[m];
                yq[m] = sm + cp.oy[m];
            }
            mg_block_core<T>(plan, R, bq, yq, (unsigned)t, (unsigned)nt);
        }
        int m = R - 1;
        for (; m >= J && cp.own[m] == 1; --m) {
            const ClLev v = cl_lev(cp.lc[m], 1, 0);
            const bool tiny = v.P * v.nz <= 64;
            const bool from_core = m + 1 == R;
            const T* e = from_core ? sm + cp.oy[R] : sm + cp.oy2[m + 1];
            if (tiny) {
                if (t < 32) {
                    __syncwarp();
                    cl_prolong<T>(v, plan.lev[m + 1], e, from_core ? 0 : 1, 0, sm + cp.oy2[m],
                                  nullptr, nullptr, m == J ? out : nullptr, t, 32);
                }
            } else {
                __syncthreads();
                cl_prolong<T>(v, plan.lev[m + 1], e, from_core ? 0 : 1, 0, sm + cp.oy2[m], nullptr,
                              nullptr, m == J ? out : nullptr, t, nt);
            }
        }
        __syncthreads();
        // the split level above reads the correction of the level below it
        // whole: a copy into every CTA, so that those reads stay local
        {
            const bool from_core = m + 1 == R;
            T* src = from_core ? sm + cp.oy[R] : sm + cp.oy2[m + 1];
            const Lev& Lb = plan.lev[m + 1];
            const long long n = from_core ? Lb.cells : (long long)(Lb.n[2] + 2) * Lb.n[0] * Lb.n[1];
            for (long long q = t; q < n; q += nt) {
                const T x = src[q];
                for (int rk = 1; rk < C; ++rk) *cl_map(src + q, (unsigned)rk) = x;
            }
        }
    }
    cl_sync();
    // up through the split levels
    for (int m = R - 1; m >= J; --m) {
        if (cp.own[m] == 1) continue;
        const ClLev v = cl_lev(cp.lc[m], C, r);
        const bool from_core = m + 1 == R;
        const bool from0 = from_core || cp.own[m + 1] == 1;
        // the coarse correction: rank 0's core level (slot z) or whole slab
        // level (slot z + 1), copied into this CTA, or this CTA's coarse slab
        // with its halo planes (slot z - Kc0 + 1, wrapped across a periodic
        // seam)
        const T* e = from_core ? sm + cp.oy[R] : sm + cp.oy2[m + 1];
        const int zoff = from_core ? 0 : (from0 ? 1 : 1 - v.k0 / 2);
        const int nzw = from0 ? 0 : plan.lev[m + 1].n[2];
        T *lo = nullptr, *hi = nullptr;
        if (m > J) cl_halo_dst(sm + cp.oy2[m], v, C, r, lo, hi);
        cl_prolong<T>(v, plan.lev[m + 1], e, zoff, nzw, sm + cp.oy2[m], lo, hi,
                      m == J ? out : nullptr, t, nt);
        // the next level up reads the halo planes just written; after level
        // J no CTA touches another's shared memory
        if (m > J) cl_sync();
    }
}

// One cluster of cp.C CTAs per state (blockIdx.y).  Each CTA copies both
// plans into the start of its shared memory (the level loops read them from
// there, not from the kernel parameters) and fills the Jacobi weight tables
// of the slab levels, then waits for the preceding kernel.
template <typename T>
__global__ void __launch_bounds__(MG_CL_THREADS)
    k_mg_cluster(const __grid_constant__ MgPlan plan, const __grid_constant__ ClPlan cp,
                 SliceCtl* __restrict__ ctl, const T* __restrict__ in, T* __restrict__ out) {
    // the prologue reads the kernel parameters only, so under a programmatic
    // dependency it runs before the wait for the preceding kernel
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = (int)threadIdx.x, nt = (int)blockDim.x;
    {
        const unsigned* a = reinterpret_cast<const unsigned*>(&plan);
        unsigned* d = reinterpret_cast<unsigned*>(smem_raw);
        for (int q = t; q < (int)(sizeof(MgPlan) / 4); q += nt) d[q] = a[q];
        const unsigned* b = reinterpret_cast<const unsigned*>(&cp);
        unsigned* e = reinterpret_cast<unsigned*>(smem_raw + CL_OFF_CP);
        for (int q = t; q < (int)(sizeof(ClPlan) / 4); q += nt) e[q] = b[q];
    }
    T* wdt = reinterpret_cast<T*>(smem_raw) + cp.otab;
    const T w = T(MG_OMEGA);
    for (int q = t; q < 27 * (cp.R - cp.J); q += nt) {
        const int m = cp.J + q / 27, c = q - (q / 27) * 27;
        wdt[27 * m + c] = cl_wd_entry<T>(plan.lev[m], c, w);
    }
    __syncthreads();
    pdl_wait();
    const long long s = blockIdx.y;
    // the whole cluster returns together: the flag is the state's
    if (ctl[s].status != ST_ITER) return;
    const MgPlan& sp = *reinterpret_cast<const MgPlan*>(smem_raw);
    const ClPlan& sc = *reinterpret_cast<const ClPlan*>(smem_raw + CL_OFF_CP);
    const long long cells = sp.lev[sc.J].cells;
    mg_cluster_levels<T>(sp, sc, wdt, in + s * cells, out + s * cells);
}

}  // namespace nsk
