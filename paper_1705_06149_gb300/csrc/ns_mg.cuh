// Multigrid-preconditioned BiCGStab for the pressure equation L p = b of the
// projection step (Section 2 names BiCGStab as the solver).  The Krylov
// iteration is BiCGStab with right preconditioning; the preconditioner is one
// geometric multigrid V-cycle on the cell-centred pressure grid:
//   - levels: the grid halved in every direction while all sizes are even and
//     >= 4; each level uses the same Neumann / periodic rules with doubled h;
//   - smoothing: two damped-Jacobi sweeps (weight 6/7) from zero before each
//     restriction, none after the correction (a V(2,0) cycle);
//   - restriction: mean of the 8 children; prolongation: trilinear
//     (weights 3/4 and 1/4 per direction, mirrored at walls, wrapped when
//     periodic);
//   - the small levels (<= MG_BLOCK_CELLS cells) run inside one CTA per state,
//     in shared memory; their coarsest level gets a fixed number of sweeps;
//   - with solid cells only the finest level carries them (faces into solids
//     dropped, Jacobi weight 0 and prolonged correction 0 in solid cells); the
//     coarse levels keep the obstacle-free operator.  The correction is then
//     cruder near obstacles but M stays a fixed linear map that keeps solid
//     cells at zero (4-5 iterations to 1e-4 on the 64^3 cavity with 8 boxes,
//     against 160 for plain BiCGStab).
// The V-cycle is a fixed linear operator, so BiCGStab's recurrences hold.
//
// Per-state reductions finish in the CTA that arrives last (a per-state
// counter): it sums the per-CTA partials in a fixed order and writes the
// scalars the next phase needs into SliceCtl, so no phase re-reduces.
#pragma once

#include "ns_kernels.cuh"

namespace nsk {

constexpr int MG_MAX_LEVELS = 14;
constexpr double MG_OMEGA = 6.0 / 7.0;
constexpr int MG_BLOCK_THREADS = 1024;
constexpr int MG_COARSEST_SWEEPS = 32;

// Per-cell face code of the finest level with solid cells: bit 2a (2a+1) set
// when the face to the lower (upper) neighbour along axis a joins two fluid
// cells; bit 6 set for a fluid cell.
constexpr unsigned FC_FLUID = 64u;

struct Lev {
    int n[3];
    int bc[3];
    const uint8_t* fcode;  // finest level with solid cells, else null
    double ih2[3];
    float fih2[3];  // FP32 copy
    float lih2[3];  // ih2 - fih2 (the FP32 remainder: fih2 + lih2 = ih2 to ~2^-48)
    long long cells;
    int tz, bx, by, bz, ctas;
    int rbx, rby, rctas;   // restriction tiling: 32 x 8 cells per CTA plane
};

template <typename T> __device__ __forceinline__ T lw(const Lev& L, int d);
template <> __device__ __forceinline__ float lw<float>(const Lev& L, int d) { return L.fih2[d]; }
template <> __device__ __forceinline__ double lw<double>(const Lev& L, int d) { return L.ih2[d]; }

// Neighbours of cell (i,j,k) along each axis as linear indices: clamped to the
// cell itself across a wall, wrapped across a periodic seam.  With a clamped
// neighbour the face term v[nb] - v[c] of the Laplacian is exactly zero, so
//   L v = sum_d w_d (v[hi_d] + v[lo_d] - 2 v[c])
// is the Neumann Laplacian for every cell, without branches.
struct Nbr {
    int c;
    int lo[3], hi[3];
};

__device__ __forceinline__ void axis_nbr(int x, int n, int bc, int& lo, int& hi, int& act) {
    if (bc == BC_PERIODIC) {
        lo = x == 0 ? n - 1 : x - 1;
        hi = x + 1 == n ? 0 : x + 1;
        act = 2;
    } else {
        lo = x > 0 ? x - 1 : x;
        hi = x + 1 < n ? x + 1 : x;
        act = (x > 0) + (x + 1 < n);
    }
}

// The x and y parts of a thread's neighbours, fixed along its march in z:
// the column's base index and the offsets to its x / y neighbours.
struct NbrXY {
    int base;
    int xl, xh, yl, yh;
};

__device__ __forceinline__ NbrXY make_nbr_xy(const Lev& L, int i, int j) {
    NbrXY q;
    int lo, hi, act;
    const int sy = L.n[0];
    q.base = j * sy + i;
    axis_nbr(i, L.n[0], L.bc[0], lo, hi, act);
    q.xl = lo - i;
    q.xh = hi - i;
    axis_nbr(j, L.n[1], L.bc[1], lo, hi, act);
    q.yl = (lo - j) * sy;
    q.yh = (hi - j) * sy;
    return q;
}

__device__ __forceinline__ Nbr nbr_at(const Lev& L, const NbrXY& q, int k) {
    Nbr b;
    const int sz = L.n[0] * L.n[1];
    b.c = k * sz + q.base;
    b.lo[0] = b.c + q.xl;
    b.hi[0] = b.c + q.xh;
    b.lo[1] = b.c + q.yl;
    b.hi[1] = b.c + q.yh;
    int lo, hi, act;
    axis_nbr(k, L.n[2], L.bc[2], lo, hi, act);
    b.lo[2] = b.c + (lo - k) * sz;
    b.hi[2] = b.c + (hi - k) * sz;
    if (L.fcode != nullptr) {
        // faces into solid cells (and every face of a solid cell) are dropped:
        // the neighbour is clamped to the cell itself, as at a wall
        const unsigned m = L.fcode[b.c];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!(m & (1u << (2 * a)))) b.lo[a] = b.c;
            if (!(m & (2u << (2 * a)))) b.hi[a] = b.c;
        }
    }
    return b;
}

__device__ __forceinline__ Nbr make_nbr(const Lev& L, int i, int j, int k) {
    return nbr_at(L, make_nbr_xy(L, i, j), k);
}

// Cell is fluid (always true without solid cells).
__device__ __forceinline__ bool lev_fluid(const Lev& L, int id) {
    return L.fcode == nullptr || (L.fcode[id] & FC_FLUID) != 0;
}

// The Laplacian from the cell value and its six neighbour values (x high,
// x low, y high, y low, z high, z low).
template <typename T>
__device__ __forceinline__ T lap7(const Lev& L, T xh, T xl, T yh, T yl, T zh, T zl, T vc) {
    const T two = T(2);
    return (xh + xl - two * vc) * lw<T>(L, 0) + (yh + yl - two * vc) * lw<T>(L, 1) +
           (zh + zl - two * vc) * lw<T>(L, 2);
}

template <typename T, typename F>
__device__ __forceinline__ T lap_nbr(const Lev& L, const Nbr& b, const F& val, T vc) {
    return lap7<T>(L, val(b.hi[0]), val(b.lo[0]), val(b.hi[1]), val(b.lo[1]), val(b.hi[2]),
                   val(b.lo[2]), vc);
}

// The 7-point values of a cell in registers: a thread's march in z loads a
// batch of MG_ZB cells before it computes any of them, so every load of the
// batch is in flight at once (the cells' arithmetic and the order of the
// per-thread sums along z are those of the plain march).
constexpr int MG_ZB = 4;

template <typename T>
struct Vals7 {
    T c, xh, xl, yh, yl, zh, zl;
};

template <typename T>
__device__ __forceinline__ Vals7<T> load7(const Nbr& b, const T* __restrict__ a) {
    return Vals7<T>{a[b.c], a[b.hi[0]], a[b.lo[0]], a[b.hi[1]], a[b.lo[1]], a[b.hi[2]],
                    a[b.lo[2]]};
}

template <typename T>
__device__ __forceinline__ T lap_vals(const Lev& L, const Vals7<T>& v) {
    return lap7<T>(L, v.xh, v.xl, v.yh, v.yl, v.zh, v.zl, v.c);
}

// Error-free transformations of FP32 arithmetic (Knuth's TwoSum; the exact
// product remainder by FMA), used to evaluate L e for an FP32 field e to about
// FP64 accuracy on the FP32 pipe.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// A float-float number hi + lo (|lo| <= ulp(hi) / 2 after normalisation):
// about 48 significant bits on the FP32 pipe.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_norm(float s, float e) {  // |s| >= |e|
    const float h = s + e;
    return FF{h, e - (h - s)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return ff_norm(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ FF ff_add_f(FF a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    return ff_norm(s, e + a.lo);
}
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }
__device__ __forceinline__ FF ff_from_double(double d) {
    const float h = float(d);
    return FF{h, float(d - double(h))};
}
__device__ __forceinline__ double ff_to_double(FF a) { return double(a.hi) + double(a.lo); }

// L e at a cell in float-float for FP32 e: per axis the second difference
// e_hi + e_lo - 2 e_c in float-float (exact), times the float-float weight
// (fih2 + lih2), summed in float-float.
__device__ __forceinline__ FF lap_ff6(const Lev& L, const float (&eh)[3], const float (&el)[3],
                                     float ec) {
    float acc_hi = 0.0f, acc_lo = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float t_hi, t_lo, u_hi, u_err;
        two_sum(eh[d], el[d], t_hi, t_lo);
        two_sum(t_hi, -2.0f * ec, u_hi, u_err);
        const float u_lo = t_lo + u_err;
        const float w_hi = L.fih2[d], w_lo = L.lih2[d];
        const float p_hi = u_hi * w_hi;
        const float p_err = fmaf(u_hi, w_hi, -p_hi);
        const float p_lo = p_err + (u_hi * w_lo + u_lo * w_hi);
        float s_hi, s_err;
        two_sum(acc_hi, p_hi, s_hi, s_err);
        acc_hi = s_hi;
        acc_lo += s_err + p_lo;
    }
    const float h = acc_hi + acc_lo;
    return FF{h, acc_lo - (h - acc_hi)};
}

// The same at a cell from its stencil neighbours' indices (values from e).
__device__ __forceinline__ FF lap_ff_pair(const Lev& L, const Nbr& nb, const float* e, float ec) {
    const float eh[3] = {e[nb.hi[0]], e[nb.hi[1]], e[nb.hi[2]]};
    const float el[3] = {e[nb.lo[0]], e[nb.lo[1]], e[nb.lo[2]]};
    return lap_ff6(L, eh, el, ec);
}

// The same from a cell's 7-point values.
__device__ __forceinline__ FF lap_ff_vals(const Lev& L, const Vals7<float>& v) {
    const float eh[3] = {v.xh, v.yh, v.zh};
    const float el[3] = {v.xl, v.yl, v.zl};
    return lap_ff6(L, eh, el, v.c);
}

// -w / d in the preconditioner (deterministic; the V-cycle only has to be a
// fixed linear operator, so FP32 uses the fast division)
template <typename T> __device__ __forceinline__ T neg_over(T a, T d);
template <> __device__ __forceinline__ float neg_over<float>(float a, float d) {
    return -__fdividef(a, d);
}
template <> __device__ __forceinline__ double neg_over<double>(double a, double d) {
    return -a / d;
}

// Jacobi weight w / diagonal of a masked cell from its face code (the
// diagonal is minus the sum of the active-face weights); 0 for a cell without
// active faces (solid).
template <typename T>
__device__ __forceinline__ T jacobi_code(const Lev& L, unsigned m, T w) {
    const T d = T(__popc(m & 3u)) * lw<T>(L, 0) + T(__popc(m & 12u)) * lw<T>(L, 1) +
                T(__popc(m & 48u)) * lw<T>(L, 2);
    return d != T(0) ? neg_over<T>(w, d) : T(0);
}

// Jacobi diagonal of the Neumann Laplacian at a cell: -sum_d w_d act_d.
template <typename T>
__device__ __forceinline__ T diag_axis(const Lev& L, int d, int x) {
    const int act = L.bc[d] == BC_PERIODIC ? 2 : (x > 0) + (x + 1 < L.n[d]);
    return T(act) * lw<T>(L, d);
}

struct MgPlan {
    int nlev;                 // levels in the hierarchy (grid + block)
    int lc;                   // first level handled by the block kernel
    int block_ok;             // 1: levels >= lc fit in one CTA's shared memory
    Lev lev[MG_MAX_LEVELS];
};

template <typename T>
struct MgBuf {
    T* x;      // solution / inner correction
    T* r;      // residual
    T* rhat;   // shadow residual
    T* P[2];   // search direction by parity
    T* V[2];   // L y by parity
    T* Y;      // M^-1 p
    T* Z;      // M^-1 s
    T* S;      // s = r - alpha v
    T* Tt;     // L z
    T* B[MG_MAX_LEVELS];   // restricted right sides, levels 1..lc
    T* Yl[MG_MAX_LEVELS];  // smoothed / corrected iterates, levels 1..lc
    unsigned int* counter; // per state: CTAs arrived
};

__device__ __forceinline__ int lindex(const Lev& L, int i, int j, int k) {
    return (k * L.n[1] + j) * L.n[0] + i;
}

// Jacobi diagonal of L at (i,j,k): minus the sum of the active-face weights.
template <typename T>
__device__ __forceinline__ T diag_at(const Lev& L, int i, int j, int k) {
    const int c[3] = {i, j, k};
    T d = T(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T w = lw<T>(L, a);
        if (L.bc[a] == BC_PERIODIC) {
            d -= T(2) * w;
        } else {
            if (c[a] > 0) d -= w;
            if (c[a] + 1 < L.n[a]) d -= w;
        }
    }
    return d;
}

__device__ __forceinline__ void lev_origin(const Lev& L, int cta, int& i, int& j, int& k0) {
    int tx = cta % L.bx;
    int r = cta / L.bx;
    int ty = r % L.by;
    int tzb = r / L.by;
    i = tx * TX + threadIdx.x;
    j = ty * TY + threadIdx.y;
    k0 = tzb * L.tz;
}

// Arrival at the per-state counter after this CTA's partials are written.
// Returns true in the last CTA of the state, which may then read all partials.
__device__ __forceinline__ bool arrive_last(unsigned int* counter, int ctas) {
    __shared__ int last_all[NSUB];
    int& last = last_all[sub_id()];
    __threadfence();
    sub_sync();
    if (tid_flat() == 0) {
        const unsigned int prev = atomicAdd(counter, 1u);
        last = prev + 1 == (unsigned int)ctas;
        if (last) *counter = 0u;  // every other CTA has arrived: reset for the next phase
    }
    sub_sync();
    const bool is_last = last != 0;
    if (is_last) __threadfence();
    return is_last;
}

// Fixed-order sum of [ctas][NV] partials, read through L2, in the last CTA.
// Each thread sums the CTAs t, t + NTHREADS, ... in that order; it loads a
// batch of them before adding, so the reads of the batch overlap (the last
// CTA's reduction is on the critical path of every solver phase).
template <int NV>
__device__ __forceinline__ void sum_partials_l2(const double* part, int ctas, double (&out)[NV]) {
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
            for (int q = 0; q < NV; ++q)
                buf[u][q] = c < ctas ? __ldcg(part + (long long)c * NV + q) : 0.0;
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
#pragma unroll
    for (int q = 0; q < NV; ++q) out[q] = v[q];  // valid in thread 0
}

// Sum over the CTA of per-thread values: a warp-shuffle tree in the values'
// own precision, then the warp sums in FP64 (valid in thread 0).  For FP32
// kernels this keeps the FP64 pipe out of the per-thread work.
template <typename A, int NV>
__device__ __forceinline__ void block_sum_mixed(A (&v)[NV], double (&out)[NV]) {
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
        for (int q = 0; q < NV; ++q) sm[q][warp] = double(v[q]);
    }
    sub_sync();
    if (t == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double x = 0.0;
            for (int w = 0; w < NWARPS; ++w) x += sm[q][w];
            out[q] = x;
        }
    }
}

// Sum over the CTA of per-warp FP64 values held by each warp's lane 0 (the
// other lanes' values are ignored), valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum_warps(const double (&v)[NV], double (&out)[NV]) {
    __shared__ double sw_all[NSUB][NV][NWARPS];
    double(&sm)[NV][NWARPS] = sw_all[sub_id()];
    const int t = tid_flat();
    const int lane = t & 31, warp = t >> 5;
    sub_sync();
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) sm[q][warp] = v[q];
    }
    sub_sync();
    if (t == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double x = 0.0;
            for (int w = 0; w < NWARPS; ++w) x += sm[q][w];
            out[q] = x;
        }
    }
}

// Writes this CTA's partials and returns whether it is the last CTA of the
// state; the last one then holds the state's totals in thread 0.
template <typename A, int NV>
__device__ __forceinline__ bool partials_arrive(A (&acc)[NV], double* part_state,
                                                unsigned int* counter, int ctas,
                                                double (&total)[NV]) {
    double blk[NV];
    block_sum_mixed<A, NV>(acc, blk);
    if (tid_flat() == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) part_state[(long long)blockIdx.x * NV + q] = blk[q];
    }
    if (!arrive_last(counter, ctas)) return false;
    sum_partials_l2<NV>(part_state, ctas, total);
    return true;
}

// Writes this CTA's partials (block-reduced) and returns whether it is last.
template <int NV>
__device__ __forceinline__ bool partials_and_arrive(double (&acc)[NV], double* part_state,
                                                    unsigned int* counter, int ctas,
                                                    double (&total)[NV]) {
    block_sum<NV>(acc);
    if (tid_flat() == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) part_state[(long long)blockIdx.x * NV + q] = acc[q];
    }
    if (!arrive_last(counter, ctas)) return false;
    sum_partials_l2<NV>(part_state, ctas, total);
    return true;
}

// ---------------------------------------------------------------------------
// level-0 sources and the pre-smoothing of a level
// ---------------------------------------------------------------------------

// Two consecutive values at an even index as one vector load (the arrays of
// every level that is restricted have even rows, planes and states).
template <typename T> struct Pair2;
template <> struct Pair2<float> { using type = float2; };
template <> struct Pair2<double> { using type = double2; };

template <typename T>
__device__ __forceinline__ void load_pair(const T* __restrict__ p, T& a, T& b) {
    const typename Pair2<T>::type v = *reinterpret_cast<const typename Pair2<T>::type*>(p);
    a = v.x;
    b = v.y;
}

enum { SRC_P = 0, SRC_S = 1, SRC_ARR = 2 };

// Parity of the iteration in progress (1 for the first): selects the
// ping-pong buffers of the search direction and of L y.  Every kernel of an
// iteration reads it from the state's control block, so a fixed launch
// sequence (a captured graph) serves odd and even iterations alike.
__device__ __forceinline__ int iter_parity(const SliceCtl* c) { return (c->it_cur + 1) & 1; }

// MODE SRC_P: p = r + beta (p_old - omega v_old) (p = r on a (re)start), stored.
// MODE SRC_S: s = r - alpha v, stored.
// MODE SRC_ARR: b = the level's restricted right side.
// PRE: also two Jacobi sweeps from zero on L y = b, stored in ydst:
//   y0 = w b / d,  y1 = y0 + w (b - L y0) / d.
template <typename T, int MODE, bool PRE>
__global__ void __launch_bounds__(NTHREADS)
    k_mg_src(Lev L, MgBuf<T> mb, SliceCtl* __restrict__ ctl, const T* __restrict__ barr,
             T* __restrict__ ydst) {
    pdl_wait();
    const long long s = blockIdx.y;
    const SliceCtl* c = ctl + s;
    if (c->status != ST_ITER) return;
    const int par = iter_parity(c);
    const long long off = s * L.cells;
    const T* __restrict__ r = mb.r + off;
    T* __restrict__ rh = mb.rhat + off;
    const T* __restrict__ po = mb.P[par ^ 1] + off;
    const T* __restrict__ vo = mb.V[par ^ 1] + off;
    T* __restrict__ pn = mb.P[par] + off;
    const T* __restrict__ vn = mb.V[par] + off;
    T* __restrict__ sv = mb.S + off;
    const T* __restrict__ ba = (MODE == SRC_ARR) ? barr + off : nullptr;
    T* __restrict__ y = PRE ? ydst + off : nullptr;
    const bool restart = c->restart != 0;
    const bool first = c->it_cur == 0;
    const T tb = T(c->beta), tw = T(c->omega), ta = T(c->alpha);
    auto srcq = [&](int q) -> T {
        if (MODE == SRC_P) return restart ? r[q] : r[q] + tb * (po[q] - tw * vo[q]);
        if (MODE == SRC_S) return r[q] - ta * vn[q];
        return ba[q];
    };
    int i, j, k0;
    lev_origin(L, blockIdx.x, i, j, k0);
    if (i >= L.n[0] || j >= L.n[1]) return;
    const int k1 = min(k0 + L.tz, L.n[2]);
    const T w = T(MG_OMEGA);
    // separable diagonal: x and y parts of this thread's cell and neighbours
    int il, ih_, jl, jh, act;
    axis_nbr(i, L.n[0], L.bc[0], il, ih_, act);
    axis_nbr(j, L.n[1], L.bc[1], jl, jh, act);
    const T dxc = diag_axis<T>(L, 0, i), dxl = diag_axis<T>(L, 0, il), dxh = diag_axis<T>(L, 0, ih_);
    const T dyc = diag_axis<T>(L, 1, j), dyl = diag_axis<T>(L, 1, jl), dyh = diag_axis<T>(L, 1, jh);
    // weights w / d where the cell and both z neighbours are interior in z
    // (the same expressions as the general case, evaluated once)
    const T dz2 = T(2) * lw<T>(L, 2);
    const T icI = neg_over<T>(w, dxc + dyc + dz2);
    const T icxhI = neg_over<T>(w, dxh + dyc + dz2), icxlI = neg_over<T>(w, dxl + dyc + dz2);
    const T icyhI = neg_over<T>(w, dxc + dyh + dz2), icylI = neg_over<T>(w, dxc + dyl + dz2);
    // the source at the z neighbour below and at the cell, carried along the
    // march (each value is computed once per thread, as the neighbours' are)
    const bool roll = PRE && L.fcode == nullptr;
    T zlo = T(0), zc = T(0);
    const NbrXY xy = make_nbr_xy(L, i, j);
    for (int k = k0; k < k1; ++k) {
        const Nbr nb = nbr_at(L, xy, k);
        const int id = nb.c;
        if (roll && k == k0) {
            zlo = srcq(nb.lo[2]);
            zc = srcq(id);
        }
        const T bc = roll ? zc : srcq(id);
        if (MODE == SRC_P) {
            pn[id] = bc;
            if (restart && !first) rh[id] = r[id];
        }
        if (MODE == SRC_S) sv[id] = bc;
        if (PRE && L.fcode != nullptr) {
            // masked finest level: per-cell diagonals from the face codes
            const uint8_t* fc = L.fcode;
            const T ic = jacobi_code<T>(L, fc[id], w);
            const T y0c = ic * bc;
            const T lap = (jacobi_code<T>(L, fc[nb.hi[0]], w) * srcq(nb.hi[0]) +
                           jacobi_code<T>(L, fc[nb.lo[0]], w) * srcq(nb.lo[0]) - T(2) * y0c) *
                              lw<T>(L, 0) +
                          (jacobi_code<T>(L, fc[nb.hi[1]], w) * srcq(nb.hi[1]) +
                           jacobi_code<T>(L, fc[nb.lo[1]], w) * srcq(nb.lo[1]) - T(2) * y0c) *
                              lw<T>(L, 1) +
                          (jacobi_code<T>(L, fc[nb.hi[2]], w) * srcq(nb.hi[2]) +
                           jacobi_code<T>(L, fc[nb.lo[2]], w) * srcq(nb.lo[2]) - T(2) * y0c) *
                              lw<T>(L, 2);
            y[id] = y0c + ic * (bc - lap);
        } else if (PRE) {
            const T zhi = srcq(nb.hi[2]);
            // y0 = w b / d at the cell and its neighbours (d = -(dx + dy + dz))
            T ic, icxh, icxl, icyh, icyl, iczh, iczl;
            if (L.bc[2] == BC_PERIODIC || (k >= 2 && k + 2 < L.n[2])) {
                ic = icI;
                icxh = icxhI;
                icxl = icxlI;
                icyh = icyhI;
                icyl = icylI;
                iczh = iczl = icI;
            } else {
                int kl, kh;
                axis_nbr(k, L.n[2], L.bc[2], kl, kh, act);
                const T dzc = diag_axis<T>(L, 2, k), dzl = diag_axis<T>(L, 2, kl),
                        dzh = diag_axis<T>(L, 2, kh);
                ic = neg_over<T>(w, dxc + dyc + dzc);
                icxh = neg_over<T>(w, dxh + dyc + dzc);
                icxl = neg_over<T>(w, dxl + dyc + dzc);
                icyh = neg_over<T>(w, dxc + dyh + dzc);
                icyl = neg_over<T>(w, dxc + dyl + dzc);
                iczh = neg_over<T>(w, dxc + dyc + dzh);
                iczl = neg_over<T>(w, dxc + dyc + dzl);
            }
            const T y0c = ic * bc;
            const T lap =
                (icxh * srcq(nb.hi[0]) + icxl * srcq(nb.lo[0]) - T(2) * y0c) * lw<T>(L, 0) +
                (icyh * srcq(nb.hi[1]) + icyl * srcq(nb.lo[1]) - T(2) * y0c) * lw<T>(L, 1) +
                (iczh * zhi + iczl * zlo - T(2) * y0c) * lw<T>(L, 2);
            y[id] = y0c + ic * (bc - lap);
            zlo = bc;
            zc = zhi;
        }
    }
}

// The same as k_mg_src<T, MODE, true> on a level without solid cells and with
// an even nx, a thread holding the x pair (i, i+1): the
// source values of the pair, of the rows beside it and of the plane above are
// evaluated once per pair from paired vector loads, those of the pair's x
// neighbours i-1 and i+2 singly, and the plane below and the pair itself are
// carried along the march.  Every cell's arithmetic is that of k_mg_src.
// Tiling: 32 x 4 threads cover 64 x 4 cells of a plane; pbx = ceil(nx / 64).
template <typename T, int MODE>
__global__ void __launch_bounds__(NTHREADS)
    k_mg_src_pair(Lev L, MgBuf<T> mb, SliceCtl* __restrict__ ctl, const T* __restrict__ barr,
                  T* __restrict__ ydst, int pbx) {
    pdl_wait();
    const long long s = blockIdx.y;
    const SliceCtl* c = ctl + s;
    if (c->status != ST_ITER) return;
    const int par = iter_parity(c);
    const long long off = s * L.cells;
    const T* __restrict__ r = mb.r + off;
    T* __restrict__ rh = mb.rhat + off;
    const T* __restrict__ po = mb.P[par ^ 1] + off;
    const T* __restrict__ vo = mb.V[par ^ 1] + off;
    T* __restrict__ pn = mb.P[par] + off;
    const T* __restrict__ vn = mb.V[par] + off;
    T* __restrict__ sv = mb.S + off;
    T* __restrict__ y = ydst + off;
    const T* __restrict__ ba = MODE == SRC_ARR ? barr + off : nullptr;
    const bool restart = c->restart != 0;
    const bool first = c->it_cur == 0;
    const T tb = T(c->beta), tw = T(c->omega), ta = T(c->alpha);
    auto src1 = [&](int q) -> T {
        if (MODE == SRC_ARR) return ba[q];
        if (MODE == SRC_P) return restart ? r[q] : r[q] + tb * (po[q] - tw * vo[q]);
        return r[q] - ta * vn[q];
    };
    auto src2 = [&](int q, T& a, T& b) {
        if (MODE == SRC_ARR) {
            load_pair<T>(ba + q, a, b);
            return;
        }
        T r0, r1;
        load_pair<T>(r + q, r0, r1);
        if (MODE == SRC_P) {
            if (restart) {
                a = r0;
                b = r1;
            } else {
                T p0, p1, v0, v1;
                load_pair<T>(po + q, p0, p1);
                load_pair<T>(vo + q, v0, v1);
                a = r0 + tb * (p0 - tw * v0);
                b = r1 + tb * (p1 - tw * v1);
            }
        } else {
            T v0, v1;
            load_pair<T>(vn + q, v0, v1);
            a = r0 - ta * v0;
            b = r1 - ta * v1;
        }
    };
    const int cta = blockIdx.x;
    const int tx = cta % pbx;
    const int rest = cta / pbx;
    const int i = tx * 64 + 2 * (int)threadIdx.x;
    const int j = (rest % L.by) * TY + (int)threadIdx.y;
    const int k0 = (rest / L.by) * L.tz;
    const int nx = L.n[0], nxy = L.n[0] * L.n[1];
    if (i >= nx || j >= L.n[1]) return;
    const int k1 = min(k0 + L.tz, L.n[2]);
    const T w = T(MG_OMEGA);
    // x neighbours of the two cells, the rows beside them, and the separable
    // diagonal parts (as k_mg_src evaluates them for each cell)
    int ila, iha, ilb, ihb, jl, jh, act;
    axis_nbr(i, nx, L.bc[0], ila, iha, act);
    axis_nbr(i + 1, nx, L.bc[0], ilb, ihb, act);
    axis_nbr(j, L.n[1], L.bc[1], jl, jh, act);
    const int ox_lo = ila - i, ox_hi = ihb - i;  // from cell i: x-low of i, x-high of i+1
    const int oy_lo = (jl - j) * nx, oy_hi = (jh - j) * nx;
    const T dxa = diag_axis<T>(L, 0, i), dxla = diag_axis<T>(L, 0, ila), dxha = diag_axis<T>(L, 0, iha);
    const T dxb = diag_axis<T>(L, 0, i + 1), dxlb = diag_axis<T>(L, 0, ilb),
            dxhb = diag_axis<T>(L, 0, ihb);
    const T dyc = diag_axis<T>(L, 1, j), dyl = diag_axis<T>(L, 1, jl), dyh = diag_axis<T>(L, 1, jh);
    const T dz2 = T(2) * lw<T>(L, 2);
    const T icIa = neg_over<T>(w, dxa + dyc + dz2), icIb = neg_over<T>(w, dxb + dyc + dz2);
    const T icxhIa = neg_over<T>(w, dxha + dyc + dz2), icxlIa = neg_over<T>(w, dxla + dyc + dz2);
    const T icxhIb = neg_over<T>(w, dxhb + dyc + dz2), icxlIb = neg_over<T>(w, dxlb + dyc + dz2);
    const T icyhIa = neg_over<T>(w, dxa + dyh + dz2), icylIa = neg_over<T>(w, dxa + dyl + dz2);
    const T icyhIb = neg_over<T>(w, dxb + dyh + dz2), icylIb = neg_over<T>(w, dxb + dyl + dz2);
    const T w0 = lw<T>(L, 0), w1 = lw<T>(L, 1), w2 = lw<T>(L, 2);
    // the source at the plane below and at the pair, carried along the march
    T zla, zlb, bca, bcb;
    {
        int kl, kh;
        axis_nbr(k0, L.n[2], L.bc[2], kl, kh, act);
        const int cq = k0 * nxy + j * nx + i;
        src2(cq + (kl - k0) * nxy, zla, zlb);
        src2(cq, bca, bcb);
    }
    for (int k = k0; k < k1; ++k) {
        int kl, kh;
        axis_nbr(k, L.n[2], L.bc[2], kl, kh, act);
        const int cq = k * nxy + j * nx + i;
        T zha, zhb, yla, ylb, yha, yhb;
        src2(cq + (kh - k) * nxy, zha, zhb);
        src2(cq + oy_lo, yla, ylb);
        src2(cq + oy_hi, yha, yhb);
        const T sxl = src1(cq + ox_lo), sxh = src1(cq + ox_hi);
        if (MODE == SRC_P) {
            reinterpret_cast<typename Pair2<T>::type*>(pn + cq)[0] = {bca, bcb};
            if (restart && !first) {
                T r0, r1;
                load_pair<T>(r + cq, r0, r1);
                reinterpret_cast<typename Pair2<T>::type*>(rh + cq)[0] = {r0, r1};
            }
        }
        if (MODE == SRC_S) reinterpret_cast<typename Pair2<T>::type*>(sv + cq)[0] = {bca, bcb};
        T ica, icxha, icxla, icyha, icyla, iczha, iczla;
        T icb, icxhb, icxlb, icyhb, icylb, iczhb, iczlb;
        if (L.bc[2] == BC_PERIODIC || (k >= 2 && k + 2 < L.n[2])) {
            ica = icIa;
            icxha = icxhIa;
            icxla = icxlIa;
            icyha = icyhIa;
            icyla = icylIa;
            iczha = iczla = icIa;
            icb = icIb;
            icxhb = icxhIb;
            icxlb = icxlIb;
            icyhb = icyhIb;
            icylb = icylIb;
            iczhb = iczlb = icIb;
        } else {
            const T dzc = diag_axis<T>(L, 2, k), dzl = diag_axis<T>(L, 2, kl),
                    dzh = diag_axis<T>(L, 2, kh);
            ica = neg_over<T>(w, dxa + dyc + dzc);
            icxha = neg_over<T>(w, dxha + dyc + dzc);
            icxla = neg_over<T>(w, dxla + dyc + dzc);
            icyha = neg_over<T>(w, dxa + dyh + dzc);
            icyla = neg_over<T>(w, dxa + dyl + dzc);
            iczha = neg_over<T>(w, dxa + dyc + dzh);
            iczla = neg_over<T>(w, dxa + dyc + dzl);
            icb = neg_over<T>(w, dxb + dyc + dzc);
            icxhb = neg_over<T>(w, dxhb + dyc + dzc);
            icxlb = neg_over<T>(w, dxlb + dyc + dzc);
            icyhb = neg_over<T>(w, dxb + dyh + dzc);
            icylb = neg_over<T>(w, dxb + dyl + dzc);
            iczhb = neg_over<T>(w, dxb + dyc + dzh);
            iczlb = neg_over<T>(w, dxb + dyc + dzl);
        }
        // cell i: x-high neighbour i+1 (bcb), x-low i-1 (sxl); cell i+1:
        // x-high i+2 (sxh), x-low i (bca)
        const T y0a = ica * bca, y0b = icb * bcb;
        const T lapa = (icxha * bcb + icxla * sxl - T(2) * y0a) * w0 +
                       (icyha * yha + icyla * yla - T(2) * y0a) * w1 +
                       (iczha * zha + iczla * zla - T(2) * y0a) * w2;
        const T lapb = (icxhb * sxh + icxlb * bca - T(2) * y0b) * w0 +
                       (icyhb * yhb + icylb * ylb - T(2) * y0b) * w1 +
                       (iczhb * zhb + iczlb * zlb - T(2) * y0b) * w2;
        reinterpret_cast<typename Pair2<T>::type*>(y + cq)[0] = {y0a + ica * (bca - lapa),
                                                                 y0b + icb * (bcb - lapb)};
        zla = bca;
        zlb = bcb;
        bca = zha;
        bcb = zhb;
    }
}

// Residual b - L y on level l, restricted (mean of the 8 children) to level l+1.
// b is bsrc, or with bsrc_odd given the one of the pair (bsrc, bsrc_odd) that
// the iteration's parity selects.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_mg_restrict(Lev L, Lev Lc, SliceCtl* __restrict__ ctl, const T* __restrict__ bsrc,
                  const T* __restrict__ bsrc_odd, const T* __restrict__ ysrc,
                  T* __restrict__ bdst) {
    pdl_wait();
    const long long s = blockIdx.y;
    if (ctl[s].status != ST_ITER) return;
    const T* __restrict__ b =
        (bsrc_odd != nullptr && iter_parity(ctl + s) ? bsrc_odd : bsrc) + s * L.cells;
    const T* __restrict__ y = ysrc + s * L.cells;
    T* __restrict__ bc = bdst + s * Lc.cells;
    // A thread holds the x pair (i, i+1) of a child octet, a warp 16 pairs of
    // two rows: the y pair of an octet is lanes (l, l^16), the z pair two
    // steps of the march, so the octet sums need no shared memory (sizes are
    // even on every level that is restricted, and tiles start at even indices)
    const int lane = threadIdx.x, warp = threadIdx.y;
    const int tx = blockIdx.x % L.rbx;
    const int rest = blockIdx.x / L.rbx;
    const int ty = rest % L.rby;
    const int i = tx * 32 + 2 * (lane & 15);
    const int j = ty * 8 + warp * 2 + (lane >> 4);
    const int k0 = (rest / L.rby) * L.tz;
    const bool in = i < L.n[0] && j < L.n[1];
    const int k1 = min(k0 + L.tz, L.n[2]);
    const int nx = L.n[0], nxy = L.n[0] * L.n[1];
    // neighbour offsets from cell i: its low x neighbour, the high x
    // neighbour of cell i+1 (its own low neighbour is i, the high one of i is
    // i+1), and the rows below / above (clamped at walls, wrapped when periodic)
    int lo, hi, act, xlo_i, xhi_i1, jl, jh;
    axis_nbr(i, nx, L.bc[0], xlo_i, hi, act);
    axis_nbr(i + 1, nx, L.bc[0], lo, xhi_i1, act);
    axis_nbr(j, L.n[1], L.bc[1], jl, jh, act);
    const int ox_lo = xlo_i - i, ox_hi = xhi_i1 - i;
    const int oy_lo = (jl - j) * nx, oy_hi = (jh - j) * nx;
    const bool masked = L.fcode != nullptr;
    const NbrXY xy0 = make_nbr_xy(L, i, j);
    const NbrXY xy1 = make_nbr_xy(L, i + 1, j);
    T accz = T(0);
    for (int kb = k0; kb < k1; kb += 2) {
        // the z pair's loads first, then its residuals and octet sums
        T r0[2], r1[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            r0[q] = T(0);
            r1[q] = T(0);
            const int k = kb + q;
            if (!in || k >= k1) continue;
            if (masked) {
                // solid cells: per-cell stencil arms from the face codes
                const Nbr n0 = nbr_at(L, xy0, k), n1 = nbr_at(L, xy1, k);
                r0[q] = b[n0.c] - lap_vals<T>(L, load7<T>(n0, y));
                r1[q] = b[n1.c] - lap_vals<T>(L, load7<T>(n1, y));
            } else {
                int kl, kh;
                axis_nbr(k, L.n[2], L.bc[2], kl, kh, act);
                const int c = k * nxy + j * nx + i;
                T y0, y1, yl0, yl1, yh0, yh1, zl0, zl1, zh0, zh1, b0, b1;
                load_pair<T>(y + c, y0, y1);
                load_pair<T>(y + c + oy_lo, yl0, yl1);
                load_pair<T>(y + c + oy_hi, yh0, yh1);
                load_pair<T>(y + c + (kl - k) * nxy, zl0, zl1);
                load_pair<T>(y + c + (kh - k) * nxy, zh0, zh1);
                load_pair<T>(b + c, b0, b1);
                const T xl0 = y[c + ox_lo], xh1 = y[c + ox_hi];
                r0[q] = b0 - lap7<T>(L, y1, xl0, yh0, yl0, zh0, zl0, y0);
                r1[q] = b1 - lap7<T>(L, xh1, y0, yh1, yl1, zh1, zl1, y1);
            }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int k = kb + q;
            if (k < k1) {  // the same for the whole CTA
                T res = r0[q] + r1[q];                         // x pair
                res += __shfl_xor_sync(0xffffffffu, res, 16);  // y pair
                accz += res;
                if ((k & 1) == 1) {  // z pair complete
                    if (in && lane < 16)
                        bc[lindex(Lc, i >> 1, j >> 1, k >> 1)] = accz * T(0.125);
                    accz = T(0);
                }
            }
        }
    }
}

// Trilinear prolongation of the coarse correction, added in place:
// y_l += P e_{l+1}.
template <typename T>
__device__ __forceinline__ void tri_axis(int f, int nc, int bc, int& c0, int& c1, T& w1) {
    c0 = f >> 1;
    const int nb = (f & 1) ? c0 + 1 : c0 - 1;
    w1 = T(0.25);
    if (nb < 0 || nb >= nc) {
        if (bc == BC_PERIODIC) {
            c1 = nb < 0 ? nb + nc : nb - nc;
        } else {
            c1 = c0;  // mirrored ghost equals the boundary cell
        }
    } else {
        c1 = nb;
    }
}

template <typename T>
__device__ __forceinline__ T prolong_at(const Lev& Lc, const T* e, int i, int j, int k) {
    int x0, x1, y0, y1, z0, z1;
    T wx, wy, wz;
    tri_axis<T>(i, Lc.n[0], Lc.bc[0], x0, x1, wx);
    tri_axis<T>(j, Lc.n[1], Lc.bc[1], y0, y1, wy);
    tri_axis<T>(k, Lc.n[2], Lc.bc[2], z0, z1, wz);
    const T ax = T(1) - wx, ay = T(1) - wy, az = T(1) - wz;
    auto E = [&](int a, int b, int c) { return e[lindex(Lc, a, b, c)]; };
    const T lo = ay * (ax * E(x0, y0, z0) + wx * E(x1, y0, z0)) +
                 wy * (ax * E(x0, y1, z0) + wx * E(x1, y1, z0));
    const T hi = ay * (ax * E(x0, y0, z1) + wx * E(x1, y0, z1)) +
                 wy * (ax * E(x0, y1, z1) + wx * E(x1, y1, z1));
    return az * lo + wz * hi;
}

// prolong_at with the coarse neighbours as offsets from the coarse cell (the
// same eight values in the same expression).
template <typename T>
__device__ __forceinline__ T prolong_off(const Lev& Lc, const T* e, int i, int j, int k) {
    int x0, x1, y0, y1, z0, z1;
    T wx, wy, wz;
    tri_axis<T>(i, Lc.n[0], Lc.bc[0], x0, x1, wx);
    tri_axis<T>(j, Lc.n[1], Lc.bc[1], y0, y1, wy);
    tri_axis<T>(k, Lc.n[2], Lc.bc[2], z0, z1, wz);
    const T ax = T(1) - wx, ay = T(1) - wy, az = T(1) - wz;
    const int cx = Lc.n[0], cxy = Lc.n[0] * Lc.n[1];
    const T* p = e + (z0 * Lc.n[1] + y0) * cx + x0;
    const int ox = x1 - x0, oy = (y1 - y0) * cx, oz = (z1 - z0) * cxy;
    const T lo = ay * (ax * p[0] + wx * p[ox]) + wy * (ax * p[oy] + wx * p[oy + ox]);
    const T hi = ay * (ax * p[oz] + wx * p[oz + ox]) + wy * (ax * p[oz + oy] + wx * p[oz + oy + ox]);
    return az * lo + wz * hi;
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_mg_prolong(Lev L, Lev Lc, SliceCtl* __restrict__ ctl, T* __restrict__ ydst,
                 const T* __restrict__ ecoarse) {
    pdl_wait();
    const long long s = blockIdx.y;
    if (ctl[s].status != ST_ITER) return;
    T* __restrict__ y = ydst + s * L.cells;
    const T* __restrict__ e = ecoarse + s * Lc.cells;
    int i, j, k0;
    lev_origin(L, blockIdx.x, i, j, k0);
    if (i >= L.n[0] || j >= L.n[1]) return;
    const int k1 = min(k0 + L.tz, L.n[2]);
    const int plane = L.n[0] * L.n[1];
    const int base = lindex(L, i, j, 0);
    // the x / y part of the trilinear weights is fixed for the thread's
    // column: bil(K) is the bilinear value of coarse plane K at the column,
    // the same expression prolong_at evaluates for each of its two planes
    int x0, x1, y0, y1;
    T wx, wy;
    tri_axis<T>(i, Lc.n[0], Lc.bc[0], x0, x1, wx);
    tri_axis<T>(j, Lc.n[1], Lc.bc[1], y0, y1, wy);
    const T ax = T(1) - wx, ay = T(1) - wy;
    const int cx = Lc.n[0], cplane = Lc.n[0] * Lc.n[1];
    const int o00 = y0 * cx + x0, o10 = y0 * cx + x1, o01 = y1 * cx + x0, o11 = y1 * cx + x1;
    auto bil = [&](int K) -> T {
        const T* __restrict__ pl = e + K * cplane;
        return ay * (ax * pl[o00] + wx * pl[o10]) + wy * (ax * pl[o01] + wx * pl[o11]);
    };
    // Fine cells 2K and 2K+1 lie in coarse cell K; along z the first takes
    // its second plane below K, the second above K (tri_axis: the cell itself
    // at a wall, wrapped when periodic).  Marching K upwards, the planes below
    // and at K are the previous pair's planes at and above: each plane is
    // interpolated once.  Tiles start at even k and levels that are
    // prolonged to have an even nz = 2 Lc.n[2].
    const T wz = T(0.25), az = T(1) - wz;
    const int nzc = Lc.n[2];
    const bool per = Lc.bc[2] == BC_PERIODIC;
    const int Ks = k0 >> 1;
    T bm = bil(Ks > 0 ? Ks - 1 : (per ? nzc - 1 : Ks));
    T bc = bil(Ks);
    constexpr int CH = 2 * MG_ZB;
    for (int kb = k0; kb < k1; kb += CH) {
        // the chunk's y values first, then the planes and the stores
        T yv[CH];
        bool fl[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int k = kb + q;
            fl[q] = k < k1 && lev_fluid(L, base + k * plane);
            if (fl[q]) yv[q] = y[base + k * plane];
        }
#pragma unroll
        for (int q = 0; q < CH; q += 2) {
            const int k = kb + q;
            if (k < k1) {
                const int K = k >> 1;
                const T bp = bil(K + 1 < nzc ? K + 1 : (per ? 0 : K));
                if (fl[q]) y[base + k * plane] = yv[q] + (az * bc + wz * bm);
                if (fl[q + 1]) y[base + (k + 1) * plane] = yv[q + 1] + (az * bc + wz * bp);
                bm = bc;
                bc = bp;
            }
        }
    }
}

// k_mg_prolong on a level without solid cells, a thread holding the x pair
// (i, i+1) (nx is even on every level prolonged to): both cells lie in coarse
// column i/2 and take their second x column on opposite sides, so a coarse
// plane costs six loads for the pair; the pair's y values move as one vector.
// Each cell's arithmetic is that of k_mg_prolong.  Tiling as k_mg_src_pair.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_mg_prolong_pair(Lev L, Lev Lc, SliceCtl* __restrict__ ctl, T* __restrict__ ydst,
                      const T* __restrict__ ecoarse, int pbx) {
    pdl_wait();
    const long long s = blockIdx.y;
    if (ctl[s].status != ST_ITER) return;
    T* __restrict__ y = ydst + s * L.cells;
    const T* __restrict__ e = ecoarse + s * Lc.cells;
    const int cta = blockIdx.x;
    const int tx = cta % pbx;
    const int rest = cta / pbx;
    const int i = tx * 64 + 2 * (int)threadIdx.x;
    const int j = (rest % L.by) * TY + (int)threadIdx.y;
    const int k0 = (rest / L.by) * L.tz;
    if (i >= L.n[0] || j >= L.n[1]) return;
    const int k1 = min(k0 + L.tz, L.n[2]);
    const int plane = L.n[0] * L.n[1];
    const int base = lindex(L, i, j, 0);
    int x0, x1a, x1b, y0, y1, xdup;
    T wxa, wxb, wy;
    tri_axis<T>(i, Lc.n[0], Lc.bc[0], x0, x1a, wxa);
    tri_axis<T>(i + 1, Lc.n[0], Lc.bc[0], xdup, x1b, wxb);
    tri_axis<T>(j, Lc.n[1], Lc.bc[1], y0, y1, wy);
    const T axa = T(1) - wxa, axb = T(1) - wxb, ay = T(1) - wy;
    const int cx = Lc.n[0], cplane = Lc.n[0] * Lc.n[1];
    const int r0 = y0 * cx, r1 = y1 * cx;
    // bilinear values of coarse plane K at the two columns
    auto bil = [&](int K, T& va, T& vb) {
        const T* __restrict__ pl = e + K * cplane;
        const T e00 = pl[r0 + x0], e01 = pl[r1 + x0];
        const T ea0 = pl[r0 + x1a], ea1 = pl[r1 + x1a];
        const T eb0 = pl[r0 + x1b], eb1 = pl[r1 + x1b];
        va = ay * (axa * e00 + wxa * ea0) + wy * (axa * e01 + wxa * ea1);
        vb = ay * (axb * e00 + wxb * eb0) + wy * (axb * e01 + wxb * eb1);
    };
    const T wz = T(0.25), az = T(1) - wz;
    const int nzc = Lc.n[2];
    const bool per = Lc.bc[2] == BC_PERIODIC;
    const int Ks = k0 >> 1;
    T bma, bmb, bca, bcb;
    bil(Ks > 0 ? Ks - 1 : (per ? nzc - 1 : Ks), bma, bmb);
    bil(Ks, bca, bcb);
    for (int k = k0; k < k1; k += 2) {
        const int K = k >> 1;
        T ya0, yb0, ya1 = T(0), yb1 = T(0), bpa, bpb;
        load_pair<T>(y + base + k * plane, ya0, yb0);
        if (k + 1 < k1) load_pair<T>(y + base + (k + 1) * plane, ya1, yb1);
        bil(K + 1 < nzc ? K + 1 : (per ? 0 : K), bpa, bpb);
        reinterpret_cast<typename Pair2<T>::type*>(y + base + k * plane)[0] = {
            ya0 + (az * bca + wz * bma), yb0 + (az * bcb + wz * bmb)};
        if (k + 1 < k1)
            reinterpret_cast<typename Pair2<T>::type*>(y + base + (k + 1) * plane)[0] = {
                ya1 + (az * bca + wz * bpa), yb1 + (az * bcb + wz * bpb)};
        bma = bca;
        bmb = bcb;
        bca = bpa;
        bcb = bpb;
    }
}

// ---------------------------------------------------------------------------
// the small levels in one CTA per state (shared memory)
// ---------------------------------------------------------------------------

// Cells per thread the one-CTA levels may hold (MG_BLOCK_THREADS threads).
constexpr int MG_BLOCK_PER_THREAD = 4;
constexpr int MG_BLOCK_MAX_CELLS = MG_BLOCK_THREADS * MG_BLOCK_PER_THREAD;

// (i, j, k) of linear index q on a one-CTA level.  The two divisions are
// floor((q + 1/2) * fl(1/d)) in FP32 with the correctly rounded reciprocal
// rd = fl(1/d) of the divisor d (nx, then nx * ny): with x = (q + 1/2) / d the
// product is within x 2^-23 <= 2^-11 / d of x (q < 4096 gives x d < 4096),
// while x lies at least 1/(2d) from an integer, so the truncation is exactly
// floor(q / d) for every q < 4096 and d <= 4096 (also checked exhaustively).
struct LevRcp {
    float rx, rxy;  // fl(1 / nx), fl(1 / (nx ny))
};

__device__ __forceinline__ LevRcp lev_rcp(const Lev& L) {
    return LevRcp{__frcp_rn(float(L.n[0])), __frcp_rn(float(L.n[0] * L.n[1]))};
}

__device__ __forceinline__ void lev_ijk(const Lev& L, const LevRcp& rc, unsigned q, int& i,
                                        int& j, int& k) {
    const int nx = L.n[0], nxy = L.n[0] * L.n[1];
    k = (int)((float(q) + 0.5f) * rc.rxy);
    const int r = (int)q - k * nxy;
    j = (int)((float(r) + 0.5f) * rc.rx);
    i = r - j * nx;
}

// A cell of a one-CTA level as one thread holds it across the phases of a
// level: its coordinates packed 10 bits per axis (every extent of a one-CTA
// level is at most 1024) and its Jacobi weight w / diag.
__device__ __forceinline__ int blk_pack(int i, int j, int k) { return i | (j << 10) | (k << 20); }

template <typename T>
__device__ __forceinline__ T blk_wd(const Lev& L, int pk, T w) {
    return -neg_over<T>(w, diag_at<T>(L, pk & 1023, (pk >> 10) & 1023, pk >> 20));
}

// The Neumann Laplacian of a one-CTA level at the packed cell pk (linear
// index q): per axis the high and the low face term, the neighbour wrapped
// across a periodic seam and clamped to the cell itself across a wall (that
// face term is then exactly 0: the wall face drops out of L).
template <typename T>
__device__ __forceinline__ T blk_lap(const Lev& L, int pk, int q, const T* a) {
    const int c[3] = {pk & 1023, (pk >> 10) & 1023, pk >> 20};
    const int st[3] = {1, L.n[0], L.n[0] * L.n[1]};
    const T vc = a[q];
    T s = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int n = L.n[d];
        const bool per = L.bc[d] == BC_PERIODIC;
        const int lo = c[d] > 0 ? -st[d] : (per ? (n - 1) * st[d] : 0);
        const int hi = c[d] + 1 < n ? st[d] : (per ? -(n - 1) * st[d] : 0);
        const T w = lw<T>(L, d);
        s += (a[q + hi] - vc) * w;
        s -= (vc - a[q + lo]) * w;
    }
    return s;
}

// Jacobi sweeps on the coarsest level: enough for its size (a 2^3 level
// needs few).
__device__ __forceinline__ int mg_coarsest_sweeps(const Lev& L) {
    const int nmax = max(L.n[0], max(L.n[1], L.n[2]));
    return min(MG_COARSEST_SWEEPS, 4 * ((nmax + 1) / 2) * 2);
}

// The coarsest level when it has at most 32 cells: y = mg_coarsest_sweeps
// damped-Jacobi sweeps from zero on L y = b by the 32 lanes of one warp (all
// of them call it), lane t holding cell t; the neighbours' iterates come by
// register shuffles, so the sweeps need no barrier (the same face terms as
// blk_lap, in its order).
template <typename T>
__device__ __forceinline__ void mg_coarsest_warp(const Lev& L, const T* b, T* y, unsigned lane,
                                                 T w) {
    const bool own = lane < (unsigned)L.cells;
    int c3[3] = {0, 0, 0};
    if (own) lev_ijk(L, lev_rcp(L), lane, c3[0], c3[1], c3[2]);
    const T wd = own ? blk_wd<T>(L, blk_pack(c3[0], c3[1], c3[2]), w) : T(0);
    const int st[3] = {1, L.n[0], L.n[0] * L.n[1]};
    int lo[3], hi[3];  // the neighbours' lanes
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int n = L.n[d];
        const bool per = L.bc[d] == BC_PERIODIC;
        lo[d] = (int)lane;
        hi[d] = (int)lane;
        if (own) {
            lo[d] += c3[d] > 0 ? -st[d] : (per ? (n - 1) * st[d] : 0);
            hi[d] += c3[d] + 1 < n ? st[d] : (per ? -(n - 1) * st[d] : 0);
        }
    }
    const T bv = own ? b[lane] : T(0);
    T v = T(0);
    const int sweeps = mg_coarsest_sweeps(L);
    for (int q = 0; q < sweeps; ++q) {
        const T vc = v;
        T sl = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const T vh = __shfl_sync(0xffffffffu, vc, hi[d]);
            const T vl = __shfl_sync(0xffffffffu, vc, lo[d]);
            const T wgt = lw<T>(L, d);
            sl += (vh - vc) * wgt;
            sl -= (vc - vl) * wgt;
        }
        v = vc + wd * (bv - sl);
    }
    if (own) y[lane] = v;
}

// V(2,0) cycle on the one-CTA levels lc .. nlev-1 held in shared memory: per
// level m the right side bq[m] and the iterate yq[m].  On entry bq[lc] holds
// the right side (visible to every thread); on exit yq[lc] holds the result
// (after a barrier).  Thread t of nt holds the cells t + c * nt
// (c < MG_BLOCK_PER_THREAD) of a level; their coordinates and Jacobi weights
// are computed once per level visit and kept in registers.  A Jacobi sweep
// stages its results in registers and writes them back after a barrier; the
// residual b - L y replaces b (a V(2,0) cycle does not need b again) and the
// restriction is the mean of its 8 children.
template <typename T>
__device__ __forceinline__ void mg_block_core(const MgPlan& plan, int lc, T* const* bq,
                                              T* const* yq, unsigned t, unsigned nt) {
    const int nl = plan.nlev;
    const T w = T(MG_OMEGA);
    // the first thread of this thread's warp: slot c of the warp holds cells
    // only if wt + c nt < cells, a warp-uniform test, so warps beyond a small
    // level's cells skip a slot's work instead of issuing it predicated off
    const unsigned wt = t & ~31u;
    // the thread's cells of level m: packed coordinates and Jacobi weights
    int pk[MG_BLOCK_PER_THREAD];
    T wd[MG_BLOCK_PER_THREAD];
    auto cells_of = [&](int m) {
        const Lev& L = plan.lev[m];
        const LevRcp rc = lev_rcp(L);
#pragma unroll
        for (int c = 0; c < MG_BLOCK_PER_THREAD; ++c) {
            const unsigned q = t + c * nt;
            pk[c] = 0;
            wd[c] = T(0);
            if (wt + c * nt < (unsigned)L.cells && q < (unsigned)L.cells) {
                int i, j, k;
                lev_ijk(L, rc, q, i, j, k);
                pk[c] = blk_pack(i, j, k);
                wd[c] = blk_wd<T>(L, pk[c], w);
            }
        }
    };
    // one Jacobi sweep y <- y + w (b - L y) / d over level m, in place
    auto sweep = [&](int m) {
        const unsigned cells = (unsigned)plan.lev[m].cells;
        T nv[MG_BLOCK_PER_THREAD];
#pragma unroll
        for (int c = 0; c < MG_BLOCK_PER_THREAD; ++c) {
            const unsigned q = t + c * nt;
            if (wt + c * nt < cells && q < cells)
                nv[c] = yq[m][q] + wd[c] * (bq[m][q] - blk_lap<T>(plan.lev[m], pk[c], (int)q, yq[m]));
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < MG_BLOCK_PER_THREAD; ++c) {
            const unsigned q = t + c * nt;
            if (wt + c * nt < cells && q < cells) yq[m][q] = nv[c];
        }
        __syncthreads();
    };
    // down: two Jacobi sweeps from zero, the residual, its restriction
    for (int m = lc; m < nl - 1; ++m) {
        const Lev& L = plan.lev[m];
        const Lev& Lc = plan.lev[m + 1];
        const unsigned cells = (unsigned)L.cells;
        cells_of(m);
#pragma unroll
        for (int c = 0; c < MG_BLOCK_PER_THREAD; ++c) {
            const unsigned q = t + c * nt;
            if (wt + c * nt < cells && q < cells) yq[m][q] = wd[c] * bq[m][q];
        }
        __syncthreads();
        sweep(m);
#pragma unroll
        for (int c = 0; c < MG_BLOCK_PER_THREAD; ++c) {
            const unsigned q = t + c * nt;
            if (wt + c * nt < cells && q < cells)
                bq[m][q] = bq[m][q] - blk_lap<T>(L, pk[c], (int)q, yq[m]);
        }
        __syncthreads();
        const LevRcp rcc = lev_rcp(Lc);
        for (unsigned q = t; q < (unsigned)Lc.cells; q += nt) {
            int I, J, K;
            lev_ijk(Lc, rcc, q, I, J, K);
            T acc = T(0);
            for (int dz = 0; dz < 2; ++dz)
                for (int dy = 0; dy < 2; ++dy)
                    for (int dx = 0; dx < 2; ++dx)
                        acc += bq[m][lindex(L, 2 * I + dx, 2 * J + dy, 2 * K + dz)];
            bq[m + 1][q] = acc * T(0.125);
        }
        __syncthreads();
    }
    // coarsest level: Jacobi sweeps from zero
    {
        const int m = nl - 1;
        const Lev& L = plan.lev[m];
        if (L.cells <= 32) {
            if (t < 32u) mg_coarsest_warp<T>(L, bq[m], yq[m], t, w);
            __syncthreads();
        } else {
            cells_of(m);
            for (unsigned q = t; q < (unsigned)L.cells; q += nt) yq[m][q] = T(0);
            __syncthreads();
            for (int q = 0; q < mg_coarsest_sweeps(L); ++q) sweep(m);
        }
    }
    // up: add the prolonged coarse correction
    for (int m = nl - 2; m >= lc; --m) {
        const Lev& L = plan.lev[m];
        const Lev& Lc = plan.lev[m + 1];
        const LevRcp rc = lev_rcp(L);
        for (unsigned q = t; q < (unsigned)L.cells; q += nt) {
            int i, j, k;
            lev_ijk(L, rc, q, i, j, k);
            yq[m][q] += prolong_off(Lc, yq[m + 1], i, j, k);
        }
        __syncthreads();
    }
}

// V(2,0) cycle on levels plan.lc .. nlev-1 for the right side `in` (global,
// level lc); writes the result to `out` (global, level lc), with the levels in
// shared memory (mg_block_core).
// The body, for state s, all threads of the CTA taking part (the persistent
// solver calls it with the plan held in its kernel parameters).
template <typename T>
__device__ __forceinline__ void mg_block_levels(const MgPlan& plan, SliceCtl* __restrict__ ctl,
                                                const T* __restrict__ in_even,
                                                const T* __restrict__ in_odd,
                                                T* __restrict__ out, long long s) {
    if (ctl[s].status != ST_ITER) return;
    // the input is in_even, or with in_odd given the parity's one of the pair
    const T* __restrict__ in = in_odd != nullptr && iter_parity(ctl + s) ? in_odd : in_even;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* __restrict__ sm = reinterpret_cast<T*>(smem_raw);
    const int lc = plan.lc, nl = plan.nlev;
    T* bq[MG_MAX_LEVELS];
    T* yq[MG_MAX_LEVELS];
    {
        long long o = 0;
        for (int m = lc; m < nl; ++m) {
            const long long n = plan.lev[m].cells;
            bq[m] = sm + o;
            yq[m] = sm + o + n;
            o += 2 * n;
        }
    }
    // flat thread index: the CTA is 1024 x 1 x 1 here, 32 x 4 x 8 in the
    // persistent solver
    const unsigned t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const unsigned nt = blockDim.x * blockDim.y * blockDim.z;
    {
        const Lev& L = plan.lev[lc];
        const T* __restrict__ src = in + s * L.cells;
        for (unsigned q = t; q < (unsigned)L.cells; q += nt) bq[lc][q] = src[q];
    }
    __syncthreads();
    mg_block_core<T>(plan, lc, bq, yq, t, nt);
    {
        const Lev& L = plan.lev[lc];
        T* __restrict__ dst = out + s * L.cells;
        for (unsigned q = t; q < (unsigned)L.cells; q += nt) dst[q] = yq[lc][q];
    }
}

// One CTA per state (blockIdx.x); the plan stays in the kernel parameters.
template <typename T>
__global__ void __launch_bounds__(MG_BLOCK_THREADS)
    k_mg_block(const __grid_constant__ MgPlan plan, SliceCtl* __restrict__ ctl,
               const T* __restrict__ in_even, const T* __restrict__ in_odd,
               T* __restrict__ out) {
    pdl_wait();
    mg_block_levels<T>(plan, ctl, in_even, in_odd, out, blockIdx.x);
}

// ---------------------------------------------------------------------------
// BiCGStab phases around the preconditioner (level 0)
// ---------------------------------------------------------------------------

// v = L y, (r_hat, v); the last CTA sets alpha = rho / (r_hat, v).
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_mg_lapdot_v(Lev L, MgBuf<T> mb, SliceCtl* __restrict__ ctl, double* __restrict__ part) {
    pdl_wait();
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    if (c->status != ST_ITER) return;
    const int par = iter_parity(c);
    const long long off = s * L.cells;
    const T* __restrict__ y = mb.Y + off;
    const T* __restrict__ rh = mb.rhat + off;
    T* __restrict__ v = mb.V[par] + off;
    int i, j, k0;
    lev_origin(L, blockIdx.x, i, j, k0);
    T acc_t = T(0);
    if (i < L.n[0] && j < L.n[1]) {
        const int k1 = min(k0 + L.tz, L.n[2]);
        const NbrXY xy = make_nbr_xy(L, i, j);
        const int plane = L.n[0] * L.n[1];
        for (int kb = k0; kb < k1; kb += MG_ZB) {
            Vals7<T> yv[MG_ZB];
            T rq[MG_ZB];
#pragma unroll
            for (int q = 0; q < MG_ZB; ++q) {
                if (kb + q < k1) {
                    const Nbr nb = nbr_at(L, xy, kb + q);
                    yv[q] = load7<T>(nb, y);
                    rq[q] = rh[nb.c];
                }
            }
#pragma unroll
            for (int q = 0; q < MG_ZB; ++q) {
                if (kb + q < k1) {
                    const T lv = lap_vals<T>(L, yv[q]);
                    v[(kb + q) * plane + xy.base] = lv;
                    acc_t += rq[q] * lv;
                }
            }
        }
    }
    T acc[1] = {acc_t};
    double tot[1];
    if (partials_arrive<T, 1>(acc, part + s * L.ctas, mb.counter + s, L.ctas, tot) &&
        tid_flat() == 0)
        c->alpha = c->rho[0] / tot[0];
}

// t = L z, (t, s), (t, t); the last CTA sets omega = (t,s)/(t,t).
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_mg_lapdot_t(Lev L, MgBuf<T> mb, SliceCtl* __restrict__ ctl, double* __restrict__ part) {
    pdl_wait();
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    if (c->status != ST_ITER) return;
    const long long off = s * L.cells;
    const T* __restrict__ z = mb.Z + off;
    const T* __restrict__ sv = mb.S + off;
    T* __restrict__ t = mb.Tt + off;
    int i, j, k0;
    lev_origin(L, blockIdx.x, i, j, k0);
    T ts = T(0), tt = T(0);
    if (i < L.n[0] && j < L.n[1]) {
        const int k1 = min(k0 + L.tz, L.n[2]);
        const NbrXY xy = make_nbr_xy(L, i, j);
        const int plane = L.n[0] * L.n[1];
        for (int kb = k0; kb < k1; kb += MG_ZB) {
            Vals7<T> zv[MG_ZB];
            T sq[MG_ZB];
#pragma unroll
            for (int q = 0; q < MG_ZB; ++q) {
                if (kb + q < k1) {
                    const Nbr nb = nbr_at(L, xy, kb + q);
                    zv[q] = load7<T>(nb, z);
                    sq[q] = sv[nb.c];
                }
            }
#pragma unroll
            for (int q = 0; q < MG_ZB; ++q) {
                if (kb + q < k1) {
                    const T tv = lap_vals<T>(L, zv[q]);
                    t[(kb + q) * plane + xy.base] = tv;
                    ts += tv * sq[q];
                    tt += tv * tv;
                }
            }
        }
    }
    T acc[2] = {ts, tt};
    double tot[2];
    if (partials_arrive<T, 2>(acc, part + s * L.ctas * 2, mb.counter + s, L.ctas, tot) &&
        tid_flat() == 0)
        c->omega = tot[1] != 0.0 ? tot[0] / tot[1] : 0.0;
}

// k_mg_lapdot_v (WHICH 0: v = L y, (r_hat, v); the last CTA sets alpha) and
// k_mg_lapdot_t (WHICH 1: t = L z, (t, s), (t, t); the last CTA sets omega)
// on a level without solid cells and with an even nx, a thread holding the x
// pair (i, i+1): the pair, its rows beside and its plane above from paired
// loads, its x neighbours singly, the plane below and the pair itself carried
// along the march.  Each cell's Laplacian is that of lap_nbr.  Tiling as
// k_mg_src_pair (ctas = pbx * by * bz CTAs per state reduce their partials).
template <typename T, int WHICH>
__global__ void __launch_bounds__(NTHREADS)
    k_mg_lapdot_pair(Lev L, MgBuf<T> mb, SliceCtl* __restrict__ ctl, double* __restrict__ part,
                     int pbx, int ctas) {
    pdl_wait();
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    if (c->status != ST_ITER) return;
    const long long off = s * L.cells;
    const T* __restrict__ a;   // the operand: y or z
    const T* __restrict__ d;   // r_hat or s
    T* __restrict__ o;         // v or t
    if (WHICH == 0) {
        const int par = iter_parity(c);
        a = mb.Y + off;
        d = mb.rhat + off;
        o = mb.V[par] + off;
    } else {
        a = mb.Z + off;
        d = mb.S + off;
        o = mb.Tt + off;
    }
    const int cta = blockIdx.x;
    const int tx = cta % pbx;
    const int rest = cta / pbx;
    const int i = tx * 64 + 2 * (int)threadIdx.x;
    const int j = (rest % L.by) * TY + (int)threadIdx.y;
    const int k0 = (rest / L.by) * L.tz;
    const int nx = L.n[0], nxy = L.n[0] * L.n[1];
    T acc0 = T(0), acc1 = T(0);
    if (i < nx && j < L.n[1]) {
        const int k1 = min(k0 + L.tz, L.n[2]);
        int ila, iha, ilb, ihb, jl, jh, act;
        axis_nbr(i, nx, L.bc[0], ila, iha, act);
        axis_nbr(i + 1, nx, L.bc[0], ilb, ihb, act);
        axis_nbr(j, L.n[1], L.bc[1], jl, jh, act);
        const int ox_lo = ila - i, ox_hi = ihb - i;
        const int oy_lo = (jl - j) * nx, oy_hi = (jh - j) * nx;
        T zla, zlb, ca, cb;
        {
            int kl, kh;
            axis_nbr(k0, L.n[2], L.bc[2], kl, kh, act);
            const int cq = k0 * nxy + j * nx + i;
            load_pair<T>(a + cq + (kl - k0) * nxy, zla, zlb);
            load_pair<T>(a + cq, ca, cb);
        }
        for (int k = k0; k < k1; ++k) {
            int kl, kh;
            axis_nbr(k, L.n[2], L.bc[2], kl, kh, act);
            const int cq = k * nxy + j * nx + i;
            T zha, zhb, yla, ylb, yha, yhb, da, db;
            load_pair<T>(a + cq + (kh - k) * nxy, zha, zhb);
            load_pair<T>(a + cq + oy_lo, yla, ylb);
            load_pair<T>(a + cq + oy_hi, yha, yhb);
            load_pair<T>(d + cq, da, db);
            const T xla = a[cq + ox_lo], xhb = a[cq + ox_hi];
            // cell i: x-high i+1 (cb), x-low i-1; cell i+1: x-high i+2, x-low i (ca)
            const T la = lap7<T>(L, cb, xla, yha, yla, zha, zla, ca);
            const T lb = lap7<T>(L, xhb, ca, yhb, ylb, zhb, zlb, cb);
            reinterpret_cast<typename Pair2<T>::type*>(o + cq)[0] = {la, lb};
            if (WHICH == 0) {
                acc0 += da * la;
                acc0 += db * lb;
            } else {
                acc0 += la * da;
                acc1 += la * la;
                acc0 += lb * db;
                acc1 += lb * lb;
            }
            zla = ca;
            zlb = cb;
            ca = zha;
            cb = zhb;
        }
    }
    if (WHICH == 0) {
        T acc[1] = {acc0};
        double tot[1];
        if (partials_arrive<T, 1>(acc, part + s * ctas, mb.counter + s, ctas, tot) &&
            tid_flat() == 0)
            c->alpha = c->rho[0] / tot[0];
    } else {
        T acc[2] = {acc0, acc1};
        double tot[2];
        if (partials_arrive<T, 2>(acc, part + s * ctas * 2, mb.counter + s, ctas, tot) &&
            tid_flat() == 0)
            c->omega = tot[1] != 0.0 ? tot[0] / tot[1] : 0.0;
    }
}

// FP32+refine: the squared relative tolerance of the next inner solve.  The
// outer residual must fall from o_rr to otol2 o_bb; an inner solve that
// reduces its residual by f leaves about f^2 o_rr, so the inner solve needs
// no more than a reduction whose square is otol2 o_bb / o_rr; it aims a
// factor 2 (4 in squares) below that, for the rounding of the FP32
// correction.  The tolerance is the looser of that and itol2, so the last
// outer step of a solve stops as soon as the target is in reach instead of
// always reducing by itol, and no inner solve is asked for more than itol.
__device__ __forceinline__ double inner_tol2(double otol2, double o_bb, double o_rr,
                                             double itol2) {
    return fmax(itol2, 0.25 * otol2 * o_bb / o_rr);
}

// Decision after an iteration (or after a start), in the last CTA:
// convergence on (r, r) <= tol2 bb (tol2_in bb when the state's inner solve
// set a looser one), the iteration limit, or the next beta.
__device__ __forceinline__ void bicg_decide(SliceCtl* c, double rho_new, double rr, double sx,
                                            double tol2, int maxit) {
    const int it = c->it_cur;
    c->rr = rr;
    c->sx = sx;
    if (!isfinite(rr) || !isfinite(rho_new)) {
        c->status = ST_NONFINITE;
        return;
    }
    if (rr <= fmax(tol2, c->tol2_in) * c->bb) {
        c->status = ST_CONV;
        return;
    }
    if (it >= maxit) {
        c->status = ST_MAXIT;
        return;
    }
    const bool restart = it == 0 || rho_new == 0.0 || c->omega == 0.0;
    if (restart) {
        c->beta = 0.0;
        c->rho[0] = rr;  // the shadow residual becomes r
    } else {
        c->beta = (rho_new / c->rho[0]) * (c->alpha / c->omega);
        c->rho[0] = rho_new;
    }
    c->restart = restart ? 1 : 0;
    c->status = ST_ITER;
}

// x += alpha y + omega z (x = alpha y + omega z on the first iteration of a
// solve that starts from zero); r = s - omega t; (r_hat, r), (r, r), sum x.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_mg_update(Lev L, MgBuf<T> mb, SliceCtl* __restrict__ ctl, double* __restrict__ part,
                double tol2, int maxit, int zero_start) {
    pdl_wait();
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    if (c->status != ST_ITER) return;
    const long long off = s * L.cells;
    T* __restrict__ x = mb.x + off;
    T* __restrict__ r = mb.r + off;
    const T* __restrict__ rh = mb.rhat + off;
    const T* __restrict__ y = mb.Y + off;
    const T* __restrict__ z = mb.Z + off;
    const T* __restrict__ sv = mb.S + off;
    const T* __restrict__ t = mb.Tt + off;
    const T ta = T(c->alpha), tw = T(c->omega);
    const bool fresh = zero_start && c->it_cur == 0;
    int i, j, k0;
    lev_origin(L, blockIdx.x, i, j, k0);
    T a0 = T(0), a1 = T(0), a2 = T(0);
    if (i < L.n[0] && j < L.n[1]) {
        const int k1 = min(k0 + L.tz, L.n[2]);
        const int plane = L.n[0] * L.n[1];
        const int base = lindex(L, i, j, 0);
        for (int kb = k0; kb < k1; kb += MG_ZB) {
            T xo[MG_ZB], yv[MG_ZB], zv[MG_ZB], sq[MG_ZB], tq[MG_ZB], rq[MG_ZB];
#pragma unroll
            for (int q = 0; q < MG_ZB; ++q) {
                if (kb + q < k1) {
                    const int id = base + (kb + q) * plane;
                    xo[q] = fresh ? T(0) : x[id];
                    yv[q] = y[id];
                    zv[q] = z[id];
                    sq[q] = sv[id];
                    tq[q] = t[id];
                    rq[q] = rh[id];
                }
            }
#pragma unroll
            for (int q = 0; q < MG_ZB; ++q) {
                if (kb + q < k1) {
                    const int id = base + (kb + q) * plane;
                    const T xv = xo[q] + (ta * yv[q] + tw * zv[q]);
                    const T rv = sq[q] - tw * tq[q];
                    x[id] = xv;
                    r[id] = rv;
                    a0 += rq[q] * rv;
                    a1 += rv * rv;
                    a2 += xv;
                }
            }
        }
    }
    T acc[3] = {a0, a1, a2};
    double tot[3];
    if (partials_arrive<T, 3>(acc, part + s * L.ctas * 3, mb.counter + s, L.ctas, tot) &&
        tid_flat() == 0) {
        c->it_cur += 1;
        c->total_iters += 1;
        bicg_decide(c, tot[0], tot[1], tot[2], tol2, maxit);
    }
}

// k_mg_update on a level without solid cells and with an even nx, a thread
// holding the x pair (i, i+1): the six vectors and the two results move as
// paired vector loads and stores, two z steps of loads in flight before their
// arithmetic.  Each cell's arithmetic is that of k_mg_update; the per-thread
// sums take the pair's cells in x order.  Tiling as k_mg_src_pair (ctas =
// pbx * by * bz CTAs per state reduce their partials).
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_mg_update_pair(Lev L, MgBuf<T> mb, SliceCtl* __restrict__ ctl, double* __restrict__ part,
                     double tol2, int maxit, int zero_start, int pbx, int ctas) {
    pdl_wait();
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    if (c->status != ST_ITER) return;
    const long long off = s * L.cells;
    T* __restrict__ x = mb.x + off;
    T* __restrict__ r = mb.r + off;
    const T* __restrict__ rh = mb.rhat + off;
    const T* __restrict__ y = mb.Y + off;
    const T* __restrict__ z = mb.Z + off;
    const T* __restrict__ sv = mb.S + off;
    const T* __restrict__ t = mb.Tt + off;
    const T ta = T(c->alpha), tw = T(c->omega);
    const bool fresh = zero_start && c->it_cur == 0;
    const int cta = blockIdx.x;
    const int tx = cta % pbx;
    const int rest = cta / pbx;
    const int i = tx * 64 + 2 * (int)threadIdx.x;
    const int j = (rest % L.by) * TY + (int)threadIdx.y;
    const int k0 = (rest / L.by) * L.tz;
    T a0 = T(0), a1 = T(0), a2 = T(0);
    if (i < L.n[0] && j < L.n[1]) {
        const int k1 = min(k0 + L.tz, L.n[2]);
        const int plane = L.n[0] * L.n[1];
        const int base = lindex(L, i, j, 0);
        constexpr int ZB = 2;
        for (int kb = k0; kb < k1; kb += ZB) {
            T xo[ZB][2], yv[ZB][2], zv[ZB][2], sq[ZB][2], tq[ZB][2], rq[ZB][2];
#pragma unroll
            for (int q = 0; q < ZB; ++q) {
                if (kb + q < k1) {
                    const int id = base + (kb + q) * plane;
                    if (fresh) {
                        xo[q][0] = T(0);
                        xo[q][1] = T(0);
                    } else {
                        load_pair<T>(x + id, xo[q][0], xo[q][1]);
                    }
                    load_pair<T>(y + id, yv[q][0], yv[q][1]);
                    load_pair<T>(z + id, zv[q][0], zv[q][1]);
                    load_pair<T>(sv + id, sq[q][0], sq[q][1]);
                    load_pair<T>(t + id, tq[q][0], tq[q][1]);
                    load_pair<T>(rh + id, rq[q][0], rq[q][1]);
                }
            }
#pragma unroll
            for (int q = 0; q < ZB; ++q) {
                if (kb + q < k1) {
                    const int id = base + (kb + q) * plane;
                    T xv[2], rv[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        xv[h] = xo[q][h] + (ta * yv[q][h] + tw * zv[q][h]);
                        rv[h] = sq[q][h] - tw * tq[q][h];
                        a0 += rq[q][h] * rv[h];
                        a1 += rv[h] * rv[h];
                        a2 += xv[h];
                    }
                    reinterpret_cast<typename Pair2<T>::type*>(x + id)[0] = {xv[0], xv[1]};
                    reinterpret_cast<typename Pair2<T>::type*>(r + id)[0] = {rv[0], rv[1]};
                }
            }
        }
    }
    T acc[3] = {a0, a1, a2};
    double tot[3];
    if (partials_arrive<T, 3>(acc, part + s * ctas * 3, mb.counter + s, ctas, tot) &&
        tid_flat() == 0) {
        c->it_cur += 1;
        c->total_iters += 1;
        bicg_decide(c, tot[0], tot[1], tot[2], tol2, maxit);
    }
}

// FP64 start from a warm x0 (p^n, or the extrapolated 2 p^n - p^(n-1) the
// previous correction wrote): b <- b - mean(b); x = x0; r = b - L x0;
// r_hat = r; the last CTA sets bb, rho and the first decision.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_mg_init_warm(Lev L, MgBuf<T> mb, SliceCtl* __restrict__ ctl,
                   const double* __restrict__ part_b, int nfluid, T* __restrict__ bvec,
                   const T* __restrict__ x0, double* __restrict__ part, double tol2,
                   int maxit) {
    pdl_wait();
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    double sb[1];
    reduce_partials<1>(part_b + s * L.ctas, L.ctas, sb);
    const T mean = T(sb[0] / nfluid);
    const long long off = s * L.cells;
    T* __restrict__ b = bvec + off;
    const T* __restrict__ xs = x0 + off;
    T* __restrict__ x = mb.x + off;
    T* __restrict__ r = mb.r + off;
    T* __restrict__ rh = mb.rhat + off;
    int i, j, k0;
    lev_origin(L, blockIdx.x, i, j, k0);
    T a0 = T(0), a1 = T(0), a2 = T(0);
    if (i < L.n[0] && j < L.n[1]) {
        const int k1 = min(k0 + L.tz, L.n[2]);
        auto xq = [&](int q) -> T { return xs[q]; };
        const NbrXY xy = make_nbr_xy(L, i, j);
        for (int k = k0; k < k1; ++k) {
            const Nbr nb = nbr_at(L, xy, k);
            const int id = nb.c;
            const T bv = lev_fluid(L, id) ? b[id] - mean : T(0);
            const T xc = xq(id);
            const T rv = bv - lap_nbr(L, nb, xq, xc);
            b[id] = bv;
            x[id] = xc;
            r[id] = rv;
            rh[id] = rv;
            a0 += rv * rv;
            a1 += xc;
            a2 += bv * bv;
        }
    }
    double acc[3] = {double(a0), double(a1), double(a2)};
    double tot[3];
    if (partials_and_arrive<3>(acc, part + s * L.ctas * 3, mb.counter + s, L.ctas, tot) &&
        tid_flat() == 0) {
        c->it_cur = 0;
        c->bb = tot[2];
        c->omega = 1.0;
        c->alpha = 1.0;
        c->p_final = 0;
        bicg_decide(c, tot[0], tot[0], tot[1], tol2, maxit);
    }
}

// ---------------------------------------------------------------------------
// FP32 inner iterations inside float-float iterative refinement: the pressure
// iterate p, the outer residual r and the warm starts are held as hi + lo
// FP32 pairs (about 48 significant bits), so the refinement runs on the FP32
// pipe -- GB300's FP64 rate is a small fraction of its FP32 rate.  The outer
// target (relative residual 1e-10) and the FP64 pressure the caller receives
// are unaffected by the 48-bit precision.
// ---------------------------------------------------------------------------

// Sum of squares of FP32 values accumulated in FP32 without losing the tiny
// ones: values below 2^-60 are squared after scaling by 2^64 into a second
// sum (so squares down to about 1e-76 count), combined in FP64.
struct SqAcc {
    float big = 0.0f, small = 0.0f;
    __device__ __forceinline__ void add(float x) {
        if (fabsf(x) >= 0x1p-60f) {
            big = fmaf(x, x, big);
        } else {
            const float y = x * 0x1p64f;
            small = fmaf(y, y, small);
        }
    }
    __device__ __forceinline__ double total() const {
        return double(big) + double(small) * 0x1p-128;
    }
};

// Power of two that brings a residual of squared norm rr over `cells` cells to
// an RMS of order one (1 for a zero residual): the inner FP32 solve works on
// the scaled residual, so its dot products neither underflow nor overflow
// however far the refinement has driven the residual down.
__device__ __forceinline__ double pow2_scale(double rr, long long cells) {
    if (!(rr > 0.0) || !isfinite(rr)) return 1.0;
    const int e = ilogb(sqrt(rr / double(cells)));
    return ldexp(1.0, -max(-100, min(100, e)));
}

// CTA partials of NF FP32 sums (warp trees in FP32) and NX float-float sums
// (converted to FP64 per thread, FP64 trees), FP64 across warps and CTAs;
// returns whether this CTA arrived last, which then holds the state's totals
// (the float-float ones last) in thread 0.
template <int NF, int NX>
__device__ __forceinline__ bool partials_arrive_ff(float (&v)[NF], const FF (&x)[NX],
                                                   double* part_state, unsigned int* counter,
                                                   int ctas, double (&total)[NF + NX]) {
    constexpr int NV = NF + NX;
    double bf[NF], bx[NX], dx[NX];
    // the float-float sums: a warp tree in float-float arithmetic (the FP32
    // pipe), each warp's sum converted to FP64 once, then summed over warps
    // in FP64 (lane 0's value; the other lanes add zeros)
    const int lane = tid_flat() & 31;
#pragma unroll
    for (int q = 0; q < NX; ++q) {
        FF a = x[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const FF b{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
            a = ff_add(a, b);
        }
        dx[q] = lane == 0 ? ff_to_double(a) : 0.0;
    }
    block_sum_mixed<float, NF>(v, bf);
    block_sum_warps<NX>(dx, bx);
    if (tid_flat() == 0) {
#pragma unroll
        for (int q = 0; q < NF; ++q) part_state[(long long)blockIdx.x * NV + q] = bf[q];
#pragma unroll
        for (int q = 0; q < NX; ++q) part_state[(long long)blockIdx.x * NV + NF + q] = bx[q];
    }
    if (!arrive_last(counter, ctas)) return false;
    sum_partials_l2<NV>(part_state, ctas, total);
    return true;
}

struct FFBuf {
    float *p_hi, *p_lo;   // the iterate
    float *r_hi, *r_lo;   // the outer residual b - L p
    float *w_hi, *w_lo;   // the next solve's warm start 2 p^n - p^(n-1)
    float *q_hi, *q_lo;   // the last gauged pressure p^n
};

// Start: b <- b - mean(b); p = the warm start (FROM64: the FP64 pressure p_in,
// which also becomes q; else w); r = b - L p; r32 = r_hat = r.hi.  The last
// CTA tests the outer residual and starts the inner solve (from e = 0) where
// it is not yet small enough.
template <bool FROM64>
__global__ void __launch_bounds__(NTHREADS)
    k_mg_refine_init_ff(Lev L, MgBuf<float> mb, SliceCtl* __restrict__ ctl,
                        const double* __restrict__ part_b, int nfluid,
                        const double* __restrict__ bvec, const double* __restrict__ p_in,
                        FFBuf f, double* __restrict__ part, double otol2, double itol2,
                        int maxit) {
    pdl_wait();
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    double sb[1];
    reduce_partials<1>(part_b + s * L.ctas, L.ctas, sb);
    const double mean = sb[0] / nfluid;
    const long long off = s * L.cells;
    const double* __restrict__ b = bvec + off;
    const double* __restrict__ ps = FROM64 ? p_in + off : nullptr;
    float* __restrict__ r = mb.r + off;
    float* __restrict__ rh = mb.rhat + off;
    int i, j, k0;
    lev_origin(L, blockIdx.x, i, j, k0);
    SqAcc arr, abb;
    FF sp{0.0f, 0.0f}, sr{0.0f, 0.0f};
    if (!FROM64 && i < L.n[0] && j < L.n[1]) {
        // the warm start w in float-float: a batch of MG_ZB cells' loads (b,
        // the 7-point values of both parts of w) before their arithmetic
        const int k1 = min(k0 + L.tz, L.n[2]);
        const NbrXY xy = make_nbr_xy(L, i, j);
        const float* __restrict__ wh = f.w_hi + off;
        const float* __restrict__ wl = f.w_lo + off;
        for (int kb = k0; kb < k1; kb += MG_ZB) {
            Vals7<float> hv[MG_ZB], lv[MG_ZB];
            double bb[MG_ZB];
            int ids[MG_ZB];
            bool fl[MG_ZB];
#pragma unroll
            for (int u = 0; u < MG_ZB; ++u) {
                if (kb + u < k1) {
                    const Nbr nb = nbr_at(L, xy, kb + u);
                    ids[u] = nb.c;
                    fl[u] = lev_fluid(L, nb.c);
                    bb[u] = b[nb.c];
                    hv[u] = load7<float>(nb, wh);
                    lv[u] = load7<float>(nb, wl);
                }
            }
#pragma unroll
            for (int u = 0; u < MG_ZB; ++u) {
                if (kb + u < k1) {
                    const int id = ids[u];
                    const double bv = fl[u] ? bb[u] - mean : 0.0;
                    const FF p0{hv[u].c, lv[u].c};
                    const FF lp = ff_add_f(lap_ff_vals(L, hv[u]), lap_vals<float>(L, lv[u]));
                    const FF res = ff_add(ff_from_double(bv), ff_neg(lp));
                    f.p_hi[off + id] = p0.hi;
                    f.p_lo[off + id] = p0.lo;
                    f.r_hi[off + id] = res.hi;
                    f.r_lo[off + id] = res.lo;
                    r[id] = res.hi;
                    rh[id] = res.hi;
                    arr.add(res.hi);
                    abb.add(float(bv));
                    sp = ff_add(sp, p0);
                    sr = ff_add(sr, res);
                }
            }
        }
    }
    if (FROM64 && i < L.n[0] && j < L.n[1]) {
        const int k1 = min(k0 + L.tz, L.n[2]);
        const NbrXY xy = make_nbr_xy(L, i, j);
        for (int k = k0; k < k1; ++k) {
            const Nbr nb = nbr_at(L, xy, k);
            const int id = nb.c;
            const bool fl = lev_fluid(L, id);
            const double bv = fl ? b[id] - mean : 0.0;
            FF p0, res;
            if (FROM64) {
                auto pq = [&](int q) -> double { return ps[q]; };
                const double pc = ps[id];
                res = ff_from_double(bv - lap_nbr(L, nb, pq, pc));
                p0 = ff_from_double(pc);
                f.q_hi[off + id] = p0.hi;
                f.q_lo[off + id] = p0.lo;
            } else {
                const float* __restrict__ wh = f.w_hi + off;
                const float* __restrict__ wl = f.w_lo + off;
                p0 = FF{wh[id], wl[id]};
                auto lq = [&](int q) -> float { return wl[q]; };
                const FF lp = ff_add_f(lap_ff_pair(L, nb, wh, p0.hi), lap_nbr(L, nb, lq, p0.lo));
                res = ff_add(ff_from_double(bv), ff_neg(lp));
            }
            f.p_hi[off + id] = p0.hi;
            f.p_lo[off + id] = p0.lo;
            f.r_hi[off + id] = res.hi;
            f.r_lo[off + id] = res.lo;
            r[id] = res.hi;
            rh[id] = res.hi;
            arr.add(res.hi);
            abb.add(float(bv));
            sp = ff_add(sp, p0);
            sr = ff_add(sr, res);
        }
    }
    float acc[4] = {arr.big, arr.small, abb.big, abb.small};
    const FF ffs[2] = {sp, sr};
    double t6[6];
    if (partials_arrive_ff<4, 2>(acc, ffs, part + s * L.ctas * 6, mb.counter + s, L.ctas, t6) &&
        tid_flat() == 0) {
        const double tot[3] = {t6[0] + t6[1] * 0x1p-128, t6[2] + t6[3] * 0x1p-128, t6[4]};
        const FF rmean = ff_from_double(t6[5] / nfluid);
        c->rmean_hi = rmean.hi;
        c->rmean_lo = rmean.lo;
        c->o_bb = tot[1];
        c->o_rr = tot[0];
        c->o_steps = 0;
        c->p_final = 0;
        c->sx = tot[2];
        c->o_scale = 1.0;
        c->o_funs = 1.0f;
        c->o_fsc = float(pow2_scale(tot[0], L.cells));
        const FF mean = ff_from_double(tot[2] / nfluid);
        c->mean_hi = mean.hi;
        c->mean_lo = mean.lo;
        if (!isfinite(tot[0])) {
            c->o_status = OS_NONFINITE;
            c->status = ST_IDLE;
        } else if (tot[0] <= otol2 * tot[1]) {
            c->o_status = OS_DONE;
            c->status = ST_IDLE;
        } else {
            c->o_status = OS_REFINE;
            c->it_cur = 0;
            c->bb = tot[0];
            c->omega = 1.0;
            c->alpha = 1.0;
            c->tol2_in = inner_tol2(otol2, tot[1], tot[0], itol2);
            bicg_decide(c, tot[0], tot[0], 0.0, itol2, maxit);
        }
    }
}

// Outer correction: p += e; r -= L e (L e of the FP32 correction in
// float-float); r32 = r_hat = r.hi.  The last CTA tests the outer residual and
// restarts the inner solve, or stops (converged / out of outer steps).
__global__ void __launch_bounds__(NTHREADS)
    k_mg_refine_update_ff(Lev L, MgBuf<float> mb, SliceCtl* __restrict__ ctl, FFBuf f,
                          int nfluid, double* __restrict__ part, double otol2, double itol2,
                          int maxit, int max_outer, int skip_iterating) {
    pdl_wait();
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    if (c->o_status != OS_REFINE) return;
    // graph-resident loop: a state whose inner solve is still running waits
    if (skip_iterating && c->status == ST_ITER) return;
    const bool bad = c->status == ST_NONFINITE;
    const long long off = s * L.cells;
    const float* __restrict__ e = mb.x + off;
    float* __restrict__ r = mb.r + off;
    float* __restrict__ rh = mb.rhat + off;
    // e carries the scale of the inner solve's right side; the next right
    // side is scaled by the previous residual's norm (all CTAs read both
    // before the last one updates them)
    const float unscale = c->o_funs;
    const float fsc = c->o_fsc;
    // the previous residual's fluid mean, taken out of the new one: the
    // residual of the singular (Neumann / periodic) problem must stay in the
    // range of L, or its rounding-made mean, which no correction can remove,
    // becomes the inner solve's floor once the residual is small
    const FF neg_rmean{-c->rmean_hi, -c->rmean_lo};
    int i, j, k0;
    lev_origin(L, blockIdx.x, i, j, k0);
    SqAcc arr;
    FF sp{0.0f, 0.0f}, sr{0.0f, 0.0f};
    if (!bad && i < L.n[0] && j < L.n[1]) {
        const int k1 = min(k0 + L.tz, L.n[2]);
        const NbrXY xy = make_nbr_xy(L, i, j);
        const int plane = L.n[0] * L.n[1];
        for (int kb = k0; kb < k1; kb += MG_ZB) {
            // the batch's loads first (e on the 7 points, the float-float
            // iterate and residual), then its arithmetic and stores
            Vals7<float> ev[MG_ZB];
            FF po[MG_ZB], ro[MG_ZB];
            bool fl[MG_ZB];
#pragma unroll
            for (int u = 0; u < MG_ZB; ++u) {
                if (kb + u < k1) {
                    const Nbr nb = nbr_at(L, xy, kb + u);
                    const long long q = off + nb.c;
                    ev[u] = load7<float>(nb, e);
                    po[u] = FF{f.p_hi[q], f.p_lo[q]};
                    ro[u] = FF{f.r_hi[q], f.r_lo[q]};
                    fl[u] = lev_fluid(L, nb.c);
                }
            }
#pragma unroll
            for (int u = 0; u < MG_ZB; ++u) {
                if (kb + u < k1) {
                    const int id = (kb + u) * plane + xy.base;
                    const long long q = off + id;
                    const float ec = ev[u].c;
                    const FF le = lap_ff_vals(L, ev[u]);
                    const FF pn = ff_add_f(po[u], ec * unscale);
                    FF rn = ff_add(ro[u], FF{-le.hi * unscale, -le.lo * unscale});
                    if (fl[u]) rn = ff_add(rn, neg_rmean);
                    f.p_hi[q] = pn.hi;
                    f.p_lo[q] = pn.lo;
                    f.r_hi[q] = rn.hi;
                    f.r_lo[q] = rn.lo;
                    r[id] = rn.hi * fsc;
                    rh[id] = rn.hi * fsc;
                    arr.add(rn.hi);
                    sp = ff_add(sp, pn);
                    sr = ff_add(sr, rn);
                }
            }
        }
    }
    float acc[2] = {arr.big, arr.small};
    const FF ffs[2] = {sp, sr};
    double t4[4];
    if (partials_arrive_ff<2, 2>(acc, ffs, part + s * L.ctas * 4, mb.counter + s, L.ctas, t4) &&
        tid_flat() == 0) {
        const double tot[2] = {t4[0] + t4[1] * 0x1p-128, t4[2]};
        const FF rmean = ff_from_double(t4[3] / nfluid);
        c->rmean_hi = rmean.hi;
        c->rmean_lo = rmean.lo;
        const double sc_next = double(fsc);
        c->o_steps += 1;
        c->o_rr = tot[0];
        c->sx = tot[1];
        c->p_final = 0;
        c->o_funs = 1.0f / fsc;
        c->o_fsc = float(pow2_scale(tot[0], L.cells));
        const FF mean = ff_from_double(tot[1] / nfluid);
        c->mean_hi = mean.hi;
        c->mean_lo = mean.lo;
        if (bad || !isfinite(tot[0])) {
            c->o_status = OS_NONFINITE;
            c->status = ST_IDLE;
        } else if (tot[0] <= otol2 * c->o_bb) {
            c->o_status = OS_DONE;
            c->status = ST_IDLE;
        } else if (c->o_steps >= max_outer) {
            c->o_status = OS_FAIL;
            c->status = ST_IDLE;
        } else {
            const double rr = tot[0] * sc_next * sc_next;  // of the scaled right side
            c->o_scale = sc_next;
            c->it_cur = 0;
            c->bb = rr;
            c->omega = 1.0;
            c->alpha = 1.0;
            c->tol2_in = inner_tol2(otol2, c->o_bb, tot[0], itol2);
            bicg_decide(c, rr, rr, 0.0, itol2, maxit);
        }
    }
}

// Velocity correction u += increment - dt G p (INCR) or u = F* - dt G p, with
// p = the float-float iterate: the difference of neighbouring values taken
// in float from both parts, times dt_ih = dt / h per axis.  Cells: p_out =
// p - mean (FP64; the mean the last refinement kernel left); with keep, the
// next warm start w = 2 (p - mean) - q and q = p - mean (float-float).
template <bool INCR>
__global__ void __launch_bounds__(NTHREADS)
    k_correct_ff(Geo g, const SliceCtl* __restrict__ ctl, const float* fu, const float* fv,
                 const float* fw, float* u, float* v, float* w, FFBuf f,
                 double* __restrict__ p_out, float3 dt_ih, int keep) {
    pdl_wait();
    const long long s = blockIdx.y;
    const SliceCtl* c = ctl + s;
    const long long off = s * g.cnt[3];
    const float* __restrict__ ph = f.p_hi + off;
    const float* __restrict__ pl = f.p_lo + off;
    const FF mean{c->mean_hi, c->mean_lo};
    const float* f3[3] = {fu + s * g.cnt[0], fv + s * g.cnt[1], fw + s * g.cnt[2]};
    float* o3[3] = {u + s * g.cnt[0], v + s * g.cnt[1], w + s * g.cnt[2]};
    const float dtih[3] = {dt_ih.x, dt_ih.y, dt_ih.z};
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.fbx, g.fby, i, j, k0);
    const int k1 = min(k0 + g.tz, g.n[2] + 1);
    // a batch of CF_ZB planes' loads (F*, u, the pressure pairs on both sides
    // of every active face, the cell's q) before their arithmetic, so the
    // loads of the batch are in flight together; the arithmetic is the
    // plane-by-plane march's
    constexpr int CF_ZB = 4;
    for (int kb = k0; kb < k1; kb += CF_ZB) {
        float fa[CF_ZB][3], oa[CF_ZB][3], hb[CF_ZB][3], lb[CF_ZB][3];
        float ha[CF_ZB], la[CF_ZB], qh[CF_ZB], ql[CF_ZB];
        bool act[CF_ZB][3];
#pragma unroll
        for (int z = 0; z < CF_ZB; ++z) {
            const int k = kb + z;
            if (k >= k1) break;
            const int q3[3] = {i, j, k};
            bool any = false;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                act[z][d] = false;
                if (i < g.ext[d][0] && j < g.ext[d][1] && k < g.ext[d][2] &&
                    face_active_dev(g, d, q3)) {
                    act[z][d] = true;
                    any = true;
                    const long long id = vindex(g, d, i, j, k);
                    int lo[3] = {i, j, k};
                    lo[d] = q3[d] == 0 ? g.n[d] - 1 : q3[d] - 1;
                    const int bq = cindex(g, lo[0], lo[1], lo[2]);
                    fa[z][d] = f3[d][id];
                    if (INCR) oa[z][d] = o3[d][id];
                    hb[z][d] = ph[bq];
                    lb[z][d] = pl[bq];
                }
            }
            // an active face has its cell (i, j, k) in the grid
            if (any || (i < g.n[0] && j < g.n[1] && k < g.n[2])) {
                const int id = cindex(g, i, j, k);
                ha[z] = ph[id];
                la[z] = pl[id];
                if (keep && i < g.n[0] && j < g.n[1] && k < g.n[2]) {
                    qh[z] = f.q_hi[off + id];
                    ql[z] = f.q_lo[off + id];
                }
            }
        }
#pragma unroll
        for (int z = 0; z < CF_ZB; ++z) {
            const int k = kb + z;
            if (k >= k1) break;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (i < g.ext[d][0] && j < g.ext[d][1] && k < g.ext[d][2]) {
                    const long long id = vindex(g, d, i, j, k);
                    if (!act[z][d]) {
                        o3[d][id] = 0.0f;
                    } else {
                        const float dgp = ((ha[z] - hb[z][d]) + (la[z] - lb[z][d])) * dtih[d];
                        if (INCR)
                            o3[d][id] = oa[z][d] + (fa[z][d] - dgp);
                        else
                            o3[d][id] = fa[z][d] - dgp;
                    }
                }
            }
            if (i < g.n[0] && j < g.n[1] && k < g.n[2]) {
                const int id = cindex(g, i, j, k);
                const bool sol = cell_solid(g, i, j, k);
                const FF pg = sol ? FF{0.0f, 0.0f} : ff_add(FF{ha[z], la[z]}, ff_neg(mean));
                if (p_out) p_out[off + id] = ff_to_double(pg);
                if (keep) {
                    const FF q{qh[z], ql[z]};
                    const FF wn = ff_add(FF{2.0f * pg.hi, 2.0f * pg.lo}, ff_neg(q));
                    f.w_hi[off + id] = wn.hi;
                    f.w_lo[off + id] = wn.lo;
                    f.q_hi[off + id] = pg.hi;
                    f.q_lo[off + id] = pg.lo;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// graph-resident solves: loop control of the conditional while nodes
// ---------------------------------------------------------------------------

// Iterations / refinement steps of the current solve (one solve per grid at a
// time), for the hard caps that end every captured loop whatever the flags.
struct LoopCount {
    unsigned inner;                  // loop bodies run in the current solve
    unsigned pad;
    unsigned long long inner_total;  // loop bodies run (all solves)
};

enum {
    LC_FP64_START = 0,    // after the FP64 start
    LC_FP64_ITER = 1,     // end of an FP64 iteration
    LC_REFINE_START = 2,  // after the FP32+refine start
    LC_REFINE_ITER = 3    // end of an FP32+refine loop body
};

// One warp reads the flags of every state and sets the condition of the loop
// that follows (1: run the body again).  FP64: while any state iterates.
// FP32+refine: one loop whose body is an inner iteration followed by the
// outer correction of the states whose inner solve has ended, while any state
// is still refining -- every state goes through the same sequence of inner
// iterations and corrections as with the host's nested loops, so the result
// is the same.  A loop also stops once its body count reaches its cap (the
// solver's own limits end it earlier).  When the solve ends, states that did
// not converge get a sticky failure bit.
__global__ void __launch_bounds__(32)
    k_loop_cond(SliceCtl* __restrict__ ctl, int batch, LoopCount* __restrict__ lc,
                cudaGraphConditionalHandle h, int mode, unsigned cap) {
    pdl_wait();
    const int lane = threadIdx.x;
    bool iter = false, refine = false;
    for (int s = lane; s < batch; s += 32) {
        iter |= ctl[s].status == ST_ITER;
        refine |= ctl[s].o_status == OS_REFINE;
    }
    iter = __any_sync(0xffffffffu, iter);
    refine = __any_sync(0xffffffffu, refine);
    unsigned count = 0;
    if (lane == 0) {
        if (mode == LC_FP64_START || mode == LC_REFINE_START) lc->inner = 0;
        if (mode == LC_FP64_ITER || mode == LC_REFINE_ITER) {
            lc->inner += 1;
            lc->inner_total += 1;
        }
        count = lc->inner;
    }
    count = __shfl_sync(0xffffffffu, count, 0);
    const bool outer = mode == LC_REFINE_START || mode == LC_REFINE_ITER;
    const bool go = (outer ? refine : iter) && count < cap;
    if (lane == 0) cudaGraphSetConditional(h, go ? 1u : 0u);
    if (go) return;
    for (int s = lane; s < batch; s += 32) {
        SliceCtl* c = ctl + s;
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

}  // namespace nsk
