// Kernels of one forward-Euler Chorin-Temam projection step on the MAC grid
// (Croce, Ruprecht & Krause, Section 2) for a batch of independent states,
// the BiCGStab pressure solve (FP64, or FP32 inner iterations inside an FP64
// iterative refinement), and the Parareal update of Eq. 6.
//
// Every kernel runs one CTA per (tile, state): blockIdx.y is the state and
// blockIdx.x the tile inside it, so the per-state reductions (dot products,
// means) are sums over a fixed set of CTAs in a fixed order, independent of the
// batch size.  Per-state Krylov scalars live in SliceCtl; partial sums of each
// phase are reduced redundantly by every CTA of the next phase, so one
// iteration needs three launches and no host round trip.
#pragma once

#include "ns_device.cuh"

namespace nsk {

enum { ST_ITER = 0, ST_CONV = 1, ST_MAXIT = 2, ST_NONFINITE = 3, ST_IDLE = 4 };
enum { OS_REFINE = 0, OS_DONE = 1, OS_FAIL = 2, OS_NONFINITE = 3 };

struct SliceCtl {
    int status;        // ST_*: state of the current Krylov solve
    int it_cur;        // iterations completed (written by phase C / init)
    int it_next;       // iteration in progress (written by phase A)
    int restart;       // phase A restarted the recurrence (p := r)
    double rho[2];     // (r_hat, r) of the last two iterations, by parity
    double alpha, omega;
    double bb;         // ||b||^2 of the current solve
    double rr;         // ||r||^2 when the solve stopped
    double sx;         // sum of the solution over the state when the solve stopped
    int o_status;      // OS_*: FP32+refine outer loop
    int o_steps;       // outer corrections applied
    int p_final;       // FP32+refine: p64 buffer holding the result
    int fail;          // graph-resident solves: sticky bits, 1 not converged, 2 non-finite
    double o_bb, o_rr;
    long long total_iters;  // Krylov iterations accumulated over solves
    double beta;       // multigrid path: beta of the next iteration
    long long total_outer;  // graph-resident solves: refinement steps accumulated
    long long total_solves; // graph-resident solves: solves finished
    double o_scale;    // FP32+refine: power of two the inner solve's right side carries
    float o_funs;      // FP32+refine: 1 / that scale, for the next outer correction
    float o_fsc;       // FP32+refine: the scale the next correction gives its right side
    float mean_hi, mean_lo;  // FP32+refine: the fluid mean of the iterate, float-float
    float rmean_hi, rmean_lo;  // FP32+refine: the fluid mean of the outer residual
    double tol2_in;    // FP32+refine: squared relative tolerance of the inner solve in
                       // progress, when looser than the launch's (else 0)
};

template <typename T>
struct KBuf {       // Krylov vectors of all states, [batch][cells]
    T* x;           // solution (FP64 mode) / inner correction e (FP32 mode)
    T* r;           // residual (FP32 mode: the outer residual r32 in place)
    T* rhat;        // shadow residual
    T* P[2];        // search direction, ping-pong by iteration parity
    T* V[2];        // L P, ping-pong by iteration parity
    T* t;           // L s
};

// ---------------------------------------------------------------------------
// predictor  F* = u + dt (Re^-1 lap u - div(u u))
// ---------------------------------------------------------------------------

// Tiled predictor: a CTA of PT_X x PT_Y x PT_Z cells stages u, v, w on its
// tile and a halo of two positions (ghost values applied while staging), then
// evaluates every face of the tile from shared memory with constant strides.
// Faces owned by the tile: the low face of each of its cells along each
// component's axis, plus the high wall face of the last cell of the domain.
// The tile is PT_X x PY x PZ cells (PT_X x PY threads); the default is
// 32 x 8 x 4, and the tile autotuner chooses among the instantiated shapes.
constexpr int PT_X = 32, PT_Y = 8, PT_Z = 4;
constexpr int PT_THREADS = PT_X * PT_Y;
constexpr int PH = 2;  // halo
constexpr int PS_X = PT_X + 2 * PH, PS_Y = PT_Y + 2 * PH, PS_Z = PT_Z + 2 * PH;
constexpr int PS_N = PS_X * PS_Y * PS_Z;

// Staged elements of one component for a PT_X x PY x PZ tile.
template <int PY, int PZ>
constexpr int ptile_elems() {
    return (PT_X + 2 * PH) * (PY + 2 * PH) * (PZ + 2 * PH);
}

template <typename T, bool INCR, int PY = PT_Y, int PZ = PT_Z>
__global__ void __launch_bounds__(PT_X * PY)
    k_predict_tile(Geo g, const T* __restrict__ u, const T* __restrict__ v,
                   const T* __restrict__ w, T* __restrict__ fu, T* __restrict__ fv,
                   T* __restrict__ fw, double dt, int tbx, int tby) {
    pdl_wait();
    constexpr int PT_Y = PY, PT_Z = PZ;
    constexpr int PT_THREADS = PT_X * PY;
    constexpr int PS_Y = PY + 2 * PH, PS_Z = PZ + 2 * PH;
    constexpr int PS_N = PS_X * PS_Y * PS_Z;
    extern __shared__ __align__(16) unsigned char psm_raw[];
    T* sm = reinterpret_cast<T*>(psm_raw);  // [3][PS_Z][PS_Y][PS_X]
    const long long s = blockIdx.y;
    const T* vel3[3] = {u + s * g.cnt[0], v + s * g.cnt[1], w + s * g.cnt[2]};
    T* out[3] = {fu + s * g.cnt[0], fv + s * g.cnt[1], fw + s * g.cnt[2]};
    const int cta = blockIdx.x;
    const int i0 = (cta % tbx) * PT_X;
    const int j0 = ((cta / tbx) % tby) * PT_Y;
    const int k0 = (cta / (tbx * tby)) * PT_Z;
    const int t = threadIdx.x;
    // Stage positions (i0-2 .. i0+PT_X+1) etc. of every component, ghost
    // values applied (the rules act on each axis separately).  The z part of
    // the rules is the same for the whole CTA and the x / y part is fixed per
    // plane position, so each is evaluated once; every element then costs a
    // load and at most a multiply-add.
    constexpr int PLANE = PS_X * PS_Y;
    constexpr int PER = (PLANE + PT_THREADS - 1) / PT_THREADS;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int e0 = g.ext[c][0], e1 = g.ext[c][1], e2 = g.ext[c][2];
        const long long plane = (long long)e1 * e0;
        long long zoff[PS_Z];
        T zsign[PS_Z];
        bool zghost[PS_Z], znear[PS_Z];
#pragma unroll
        for (int z = 0; z < PS_Z; ++z) {
            const int gk = k0 - PH + z;
            int qk = gk;
            T sg = T(1), ad = T(0);
            ghost_axis(g, c, 2, qk, sg, ad);
            zoff[z] = qk * plane;
            zsign[z] = sg;
            zghost[z] = gk < 0 || gk >= e2;
            znear[z] = gk >= -PH && gk < e2 + PH;
        }
#pragma unroll
        for (int h = 0; h < PER; ++h) {
            const int pq = t + h * PT_THREADS;
            if (pq >= PLANE) break;
            const int x = pq % PS_X, y = pq / PS_X;
            const int gi = i0 - PH + x, gj = j0 - PH + y;
            int qi = gi, qj = gj;
            T sxy = T(1), add = T(0);
            ghost_axis(g, c, 0, qi, sxy, add);
            ghost_axis(g, c, 1, qj, sxy, add);
            const bool xy_ghost = gi < 0 || gj < 0 || gi >= e0 || gj >= e1;
            // only positions up to two beyond the stored range are ever read
            const bool xy_near = gi >= -PH && gj >= -PH && gi < e0 + PH && gj < e1 + PH;
            const T* __restrict__ a = vel3[c] + (long long)qj * e0 + qi;
            T* dst = sm + c * PS_N + pq;
#pragma unroll
            for (int z = 0; z < PS_Z; ++z) {
                T val = T(0);
                if (xy_near && znear[z]) {
                    const T st = a[zoff[z]];
                    // stored values as they are (wall-normal boundary faces
                    // are stored as 0); ghosts = add + sign * mirror
                    val = (xy_ghost || zghost[z]) ? add + (sxy * zsign[z]) * st : st;
                }
                dst[z * PLANE] = val;
            }
        }
    }
    __syncthreads();
    const T tdt = T(dt), inv_re = g_inv_re<T>(g);
    constexpr int strd[3] = {1, PS_X, PS_X * PS_Y};
    // Each thread owns the column (x, y) = (lane, warp) of the tile and marches
    // its PT_Z cells in z.  A face flux is evaluated once: the flux entering
    // cell x across its low x face is the one lane x-1 computed for its high
    // face (a shuffle), and the low z face flux is the high one of the cell
    // below (carried along the march); only y fluxes are evaluated on both
    // faces.  The operands are the same values either way, so the fluxes are
    // identical to evaluating every face from both sides.
    const int x = t % PT_X, y = t / PT_X;
    const unsigned lane = t & 31u;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T* sc = sm + c * PS_N;
        const int sc_c = strd[c];
        // transport velocity at the high face of direction d of the cell at o
        auto up_at = [&](int d, int o) -> T {
            const int sd = strd[d];
            if (d == c) return T(0.5) * (sc[o] + sc[o + sd]);
            const T* sdc = sm + d * PS_N;
            return T(0.5) * (sdc[o - sc_c + sd] + sdc[o + sd]);
        };
        T fz_lo = T(0);
        for (int z = 0; z < PT_Z; ++z) {
            const int o = ((z + PH) * PS_Y + (y + PH)) * PS_X + (x + PH);
            T conv = T(0), diff = T(0);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int sd = strd[d];
                const T a0 = sc[o - 2 * sd], a1 = sc[o - sd], a2 = sc[o], a3 = sc[o + sd],
                        a4 = sc[o + 2 * sd];
                const T fp = smart_flux_sel(up_at(d, o), a1, a2, a3, a4);
                T fm;
                if (d == 0) {
                    fm = __shfl_up_sync(0xffffffffu, fp, 1);
                    if (lane == 0) fm = smart_flux_sel(up_at(0, o - 1), a0, a1, a2, a3);
                } else if (d == 1 || z == 0) {
                    fm = smart_flux_sel(up_at(d, o - sd), a0, a1, a2, a3);
                } else {
                    fm = fz_lo;
                }
                if (d == 2) fz_lo = fp;
                conv += (fp - fm) * g_ih<T>(g, d);
                diff += (a3 - T(2) * a2 + a1) * g_ih2<T>(g, d);
            }
            const int f[3] = {i0 + x, j0 + y, k0 + z};
            if (f[0] >= g.n[0] || f[1] >= g.n[1] || f[2] >= g.n[2]) continue;
            const long long id = vindex(g, c, f[0], f[1], f[2]);
            // the high wall face of the last cell along c is inactive: zero it
            if (g.bc[c] != BC_PERIODIC && f[c] == g.n[c] - 1) {
                int h3[3] = {f[0], f[1], f[2]};
                h3[c] += 1;
                out[c][vindex(g, c, h3[0], h3[1], h3[2])] = T(0);
            }
            if (!(g.bc[c] == BC_PERIODIC || f[c] > 0)) {
                out[c][id] = T(0);
                continue;
            }
            const T incr = tdt * (inv_re * diff - conv);
            out[c][id] = INCR ? incr : sc[o] + incr;
        }
    }
}

// ---------------------------------------------------------------------------
// predictor with solid cells: one thread per face, stencil arms that stop at
// walls and solid surfaces
// ---------------------------------------------------------------------------

// Value of component c at offset m (|m| <= 2) from face f along axis d, as f's
// stencil arm sees it: stored values up to the first interface (an inactive
// face for the normal arm; a position past a wall or inside a solid for a
// tangential arm), reflected across it beyond -- odd about the interface face
// (normal), 2 u_wall - mirror (tangential; u_wall = 0 at solids, +mirror at a
// slip wall).
template <typename T>
__device__ __forceinline__ T arm_value_dev(const Geo& g, int c, const T* a, const int f[3], int d,
                                           int m) {
    if (m == 0) return a[vindex(g, c, f[0], f[1], f[2])];
    const int sg = m > 0 ? 1 : -1;
    const int am = m > 0 ? m : -m;
    const int n = g.ext[c][d];
    for (int s = 1; s <= am; ++s) {
        int q[3] = {f[0], f[1], f[2]};
        q[d] += sg * s;
        if (g.bc[d] == BC_PERIODIC) q[d] = q[d] < 0 ? q[d] + n : (q[d] >= n ? q[d] - n : q[d]);
        if (c == d) {
            if (q[d] < 0 || q[d] >= n) break;
            if (!face_active_dev(g, c, q)) {
                if (s == am) return T(0);
                int r[3] = {f[0], f[1], f[2]};
                r[d] += sg * (2 * s - am);
                return -vel(g, c, a, r[0], r[1], r[2]);
            }
        } else {
            const bool outside = q[d] < 0 || q[d] >= n;
            if (outside || face_in_solid_dev(g, c, q)) {
                int r[3] = {f[0], f[1], f[2]};
                r[d] += sg * (2 * s - 1 - am);
                const T mirror = vel(g, c, a, r[0], r[1], r[2]);
                if (outside) {
                    if (g.bc[d] == BC_SLIP) return mirror;
                    const bool hi = q[d] >= n;
                    const T uw = (c == 0 && d == 1 && hi) ? T(g.u_lid) : T(0);
                    return T(2) * uw - mirror;
                }
                return -mirror;
            }
        }
    }
    int q[3] = {f[0], f[1], f[2]};
    q[d] += m;
    return vel(g, c, a, q[0], q[1], q[2]);
}

template <typename T, bool INCR>
__global__ void __launch_bounds__(NTHREADS)
    k_predict_masked(Geo g, const T* __restrict__ u, const T* __restrict__ v,
                     const T* __restrict__ w, T* __restrict__ fu, T* __restrict__ fv,
                     T* __restrict__ fw, double dt) {
    pdl_wait();
    const long long s = blockIdx.y;
    const T* vel3[3] = {u + s * g.cnt[0], v + s * g.cnt[1], w + s * g.cnt[2]};
    T* out[3] = {fu + s * g.cnt[0], fv + s * g.cnt[1], fw + s * g.cnt[2]};
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.fbx, g.fby, i, j, k0);
    const int k1 = min(k0 + g.tz, g.n[2] + 1);
    const T tdt = T(dt);
    for (int k = k0; k < k1; ++k) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (!(i < g.ext[c][0] && j < g.ext[c][1] && k < g.ext[c][2])) continue;
            const int f[3] = {i, j, k};
            const long long id = vindex(g, c, i, j, k);
            if (!face_active_dev(g, c, f)) {
                out[c][id] = T(0);
                continue;
            }
            T conv = T(0), diff = T(0);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                T a[5];
#pragma unroll
                for (int m = 0; m < 5; ++m) a[m] = arm_value_dev(g, c, vel3[c], f, d, m - 2);
                T up, um;
                if (d == c) {
                    up = T(0.5) * (a[2] + a[3]);
                    um = T(0.5) * (a[1] + a[2]);
                } else {
                    int q0[3] = {f[0], f[1], f[2]};
                    int q1[3] = {f[0], f[1], f[2]};
                    q0[c] = f[c] - 1;
                    q0[d] = f[d] + 1;
                    q1[d] = f[d] + 1;
                    up = T(0.5) * (vel(g, d, vel3[d], q0[0], q0[1], q0[2]) +
                                   vel(g, d, vel3[d], q1[0], q1[1], q1[2]));
                    q0[d] = f[d];
                    q1[d] = f[d];
                    um = T(0.5) * (vel(g, d, vel3[d], q0[0], q0[1], q0[2]) +
                                   vel(g, d, vel3[d], q1[0], q1[1], q1[2]));
                }
                const T fp = smart_flux(up, a[1], a[2], a[3], a[4]);
                const T fm = smart_flux(um, a[0], a[1], a[2], a[3]);
                conv += (fp - fm) * g_ih<T>(g, d);
                diff += (a[3] - T(2) * a[2] + a[1]) * g_ih2<T>(g, d);
            }
            const T incr = tdt * (g_inv_re<T>(g) * diff - conv);
            out[c][id] = INCR ? incr : vel3[c][id] + incr;
        }
    }
}

// ---------------------------------------------------------------------------
// b = D F* / dt, per-CTA partial sums of b (for the fluid mean)
// ---------------------------------------------------------------------------

// With u, v, w non-null (the increment form's first step) the divergence is
// that of (u + F*) -- F* then holds the increment -- each part differenced
// exactly in FP64.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_divergence(Geo g, const T* __restrict__ fu, const T* __restrict__ fv,
                 const T* __restrict__ fw, const T* __restrict__ u, const T* __restrict__ v,
                 const T* __restrict__ w, double* __restrict__ b, double* __restrict__ part,
                 double inv_dt) {
    pdl_wait();
    const long long s = blockIdx.y;
    fu += s * g.cnt[0];
    fv += s * g.cnt[1];
    fw += s * g.cnt[2];
    const bool with_u = u != nullptr;
    if (with_u) {
        u += s * g.cnt[0];
        v += s * g.cnt[1];
        w += s * g.cnt[2];
    }
    b += s * g.cnt[3];
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.bx, g.by, i, j, k0);
    double acc[1] = {0.0};
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + g.tz, g.n[2]);
        const int ip = (g.bc[0] == BC_PERIODIC && i + 1 == g.n[0]) ? 0 : i + 1;
        const int jp = (g.bc[1] == BC_PERIODIC && j + 1 == g.n[1]) ? 0 : j + 1;
        // a batch of DIV_ZB cells' face values is loaded before any of them
        // is differenced, so the loads of the batch are in flight together
        constexpr int DIV_ZB = 4;
        for (int kb = k0; kb < k1; kb += DIV_ZB) {
            T fa[DIV_ZB][6];
#pragma unroll
            for (int z = 0; z < DIV_ZB; ++z) {
                const int k = kb + z;
                if (k < k1) {
                    const int kp = (g.bc[2] == BC_PERIODIC && k + 1 == g.n[2]) ? 0 : k + 1;
                    fa[z][0] = fu[vindex(g, 0, ip, j, k)];
                    fa[z][1] = fu[vindex(g, 0, i, j, k)];
                    fa[z][2] = fv[vindex(g, 1, i, jp, k)];
                    fa[z][3] = fv[vindex(g, 1, i, j, k)];
                    fa[z][4] = fw[vindex(g, 2, i, j, kp)];
                    fa[z][5] = fw[vindex(g, 2, i, j, k)];
                }
            }
#pragma unroll
            for (int z = 0; z < DIV_ZB; ++z) {
                const int k = kb + z;
                if (k >= k1) break;
                const int kp = (g.bc[2] == BC_PERIODIC && k + 1 == g.n[2]) ? 0 : k + 1;
                // D of the stored F* (or increment) in the storage precision; in
                // FP32 this is the increment, whose differences carry no
                // cancellation against u
                T dt_ = (fa[z][0] - fa[z][1]) * g_ih<T>(g, 0);
                dt_ += (fa[z][2] - fa[z][3]) * g_ih<T>(g, 1);
                dt_ += (fa[z][4] - fa[z][5]) * g_ih<T>(g, 2);
                double dv = double(dt_);
                if (with_u) {
                    // the stored u itself: differences taken exactly in FP64
                    double du =
                        (double(u[vindex(g, 0, ip, j, k)]) - double(u[vindex(g, 0, i, j, k)])) *
                        g.ih[0];
                    du += (double(v[vindex(g, 1, i, jp, k)]) - double(v[vindex(g, 1, i, j, k)])) *
                          g.ih[1];
                    du += (double(w[vindex(g, 2, i, j, kp)]) - double(w[vindex(g, 2, i, j, k)])) *
                          g.ih[2];
                    dv += du;
                }
                const double bv = cell_solid(g, i, j, k) ? 0.0 : dv * inv_dt;
                b[cindex(g, i, j, k)] = bv;
                acc[0] += bv;
            }
        }
    }
    write_partials<1>(acc, part + (s * g.ctas + blockIdx.x));
}

// partial sums of a cell field (for the mean of a caller-supplied right side)
static __global__ void __launch_bounds__(NTHREADS)
    k_sum_cells(Geo g, const double* __restrict__ x, double* __restrict__ part) {
    const long long s = blockIdx.y;
    x += s * g.cnt[3];
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.bx, g.by, i, j, k0);
    double acc[1] = {0.0};
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + g.tz, g.n[2]);
        for (int k = k0; k < k1; ++k) acc[0] += x[cindex(g, i, j, k)];
    }
    write_partials<1>(acc, part + (s * g.ctas + blockIdx.x));
}

// ---------------------------------------------------------------------------
// BiCGStab (van der Vorst), three phases per iteration
// ---------------------------------------------------------------------------

// Start of a solve with a warm start x0 (FP64 mode): b <- b - mean(b);
// x = x0; r = b - L x0; r_hat = r.  Partials: (r_hat,r), (r,r), sum x, (b,b).
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_bicg_init_warm(Geo g, KBuf<T> kb, SliceCtl* __restrict__ ctl,
                     const double* __restrict__ part_b, T* __restrict__ bvec,
                     const T* __restrict__ x0, double* __restrict__ part_c) {
    const long long s = blockIdx.y;
    double sb[1];
    reduce_partials<1>(part_b + s * g.ctas, g.ctas, sb);
    const T mean = T(sb[0] / g.n_fluid);
    const long long off = s * g.cnt[3];
    T* b = bvec + off;
    const T* xs = x0 + off;
    T* x = kb.x + off;
    T* r = kb.r + off;
    T* rh = kb.rhat + off;
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.bx, g.by, i, j, k0);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + g.tz, g.n[2]);
        auto xv = [&](int a, int bb, int c) { return xs[cindex(g, a, bb, c)]; };
        for (int k = k0; k < k1; ++k) {
            const long long id = cindex(g, i, j, k);
            const bool sol = cell_solid(g, i, j, k);
            const T bv = sol ? T(0) : b[id] - mean;
            const T xc = sol ? T(0) : xs[id];
            const T rv = bv - lap_cell(g, xv, i, j, k, xc);
            b[id] = bv;
            x[id] = xc;
            r[id] = rv;
            rh[id] = rv;
            acc[1] += double(rv) * double(rv);
            acc[2] += double(xc);
            acc[3] += double(bv) * double(bv);
        }
    }
    acc[0] = acc[1];
    write_partials<4>(acc, part_c + (s * g.ctas + blockIdx.x) * 4);
    if (blockIdx.x == 0 && tid_flat() == 0) {
        SliceCtl* c = ctl + s;
        c->status = ST_ITER;
        c->it_cur = 0;
        c->it_next = 0;
        c->omega = 1.0;
        c->alpha = 1.0;
    }
}

// Phase A of iteration i (parity par = i & 1): convergence test on the
// residual of iteration i-1, then p = r + beta (p - omega v) (or p = r on a
// (re)start), v = L p.  Partial: (r_hat, v).
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_bicg_A(Geo g, KBuf<T> kb, SliceCtl* __restrict__ ctl, const double* __restrict__ part_c,
             double* __restrict__ part_a, double tol2, int maxit, int par) {
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    if (c->status != ST_ITER) return;
    double red[4];
    reduce_partials<4>(part_c + s * g.ctas * 4, g.ctas, red);
    const int done = c->it_cur;
    const int it = done + 1;
    double rho = red[0];
    const double rr = red[1];
    const double bb = it == 1 ? red[3] : c->bb;
    const bool lead = blockIdx.x == 0 && tid_flat() == 0;
    if (!isfinite(rr) || !isfinite(rho)) {
        if (lead) {
            c->status = ST_NONFINITE;
            c->rr = rr;
        }
        return;
    }
    if (rr <= tol2 * bb) {
        if (lead) {
            c->status = ST_CONV;
            c->rr = rr;
            c->sx = red[2];
            if (it == 1) c->bb = bb;
        }
        return;
    }
    if (done >= maxit) {
        if (lead) {
            c->status = ST_MAXIT;
            c->rr = rr;
            if (it == 1) c->bb = bb;
        }
        return;
    }
    const bool restart = it == 1 || rho == 0.0 || c->omega == 0.0;
    double beta = 0.0;
    if (restart)
        rho = rr;
    else
        beta = (rho / c->rho[par ^ 1]) * (c->alpha / c->omega);
    if (lead) {
        c->rho[par] = rho;
        c->it_next = it;
        c->restart = restart ? 1 : 0;
        if (it == 1) c->bb = bb;
    }
    const T tb = T(beta), tw = T(c->omega);
    const long long off = s * g.cnt[3];
    const T* r = kb.r + off;
    T* rh = kb.rhat + off;
    const T* po = kb.P[par ^ 1] + off;
    const T* vo = kb.V[par ^ 1] + off;
    T* pn = kb.P[par] + off;
    T* vn = kb.V[par] + off;
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.bx, g.by, i, j, k0);
    double acc[1] = {0.0};
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + g.tz, g.n[2]);
        auto pnew = [&](int a, int b, int cc) {
            const long long q = cindex(g, a, b, cc);
            return restart ? r[q] : r[q] + tb * (po[q] - tw * vo[q]);
        };
        for (int k = k0; k < k1; ++k) {
            const long long id = cindex(g, i, j, k);
            const T pc = pnew(i, j, k);
            const T lv = lap_cell(g, pnew, i, j, k, pc);
            pn[id] = pc;
            vn[id] = lv;
            T rhv;
            if (restart && it > 1) {
                rhv = r[id];
                rh[id] = rhv;
            } else {
                rhv = restart ? r[id] : rh[id];
            }
            acc[0] += double(rhv * lv);
        }
    }
    write_partials<1>(acc, part_a + (s * g.ctas + blockIdx.x));
}

// Phase B: alpha = rho / (r_hat, v); s = r - alpha v; t = L s.
// Partials: (t, s), (t, t).
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_bicg_B(Geo g, KBuf<T> kb, SliceCtl* __restrict__ ctl, const double* __restrict__ part_a,
             double* __restrict__ part_b, int par) {
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    if (c->status != ST_ITER) return;
    double red[1];
    reduce_partials<1>(part_a + s * g.ctas, g.ctas, red);
    const double alpha = c->rho[par] / red[0];
    if (blockIdx.x == 0 && tid_flat() == 0) c->alpha = alpha;
    const T ta = T(alpha);
    const long long off = s * g.cnt[3];
    const T* r = kb.r + off;
    const T* vn = kb.V[par] + off;
    T* t = kb.t + off;
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.bx, g.by, i, j, k0);
    double acc[2] = {0.0, 0.0};
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + g.tz, g.n[2]);
        auto sv = [&](int a, int b, int cc) {
            const long long q = cindex(g, a, b, cc);
            return r[q] - ta * vn[q];
        };
        for (int k = k0; k < k1; ++k) {
            const long long id = cindex(g, i, j, k);
            const T sc = sv(i, j, k);
            const T tv = lap_cell(g, sv, i, j, k, sc);
            t[id] = tv;
            acc[0] += double(tv * sc);
            acc[1] += double(tv * tv);
        }
    }
    write_partials<2>(acc, part_b + (s * g.ctas + blockIdx.x) * 2);
}

// Phase C: omega = (t,s)/(t,t); x += alpha p + omega s; r = s - omega t.
// Partials: (r_hat, r), (r, r), sum x.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_bicg_C(Geo g, KBuf<T> kb, SliceCtl* __restrict__ ctl, const double* __restrict__ part_b,
             double* __restrict__ part_c, int par) {
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    if (c->status != ST_ITER) return;
    double red[2];
    reduce_partials<2>(part_b + s * g.ctas * 2, g.ctas, red);
    const double omega = red[1] != 0.0 ? red[0] / red[1] : 0.0;
    const double alpha = c->alpha;
    if (blockIdx.x == 0 && tid_flat() == 0) {
        c->omega = omega;
        c->it_cur = c->it_next;
        c->total_iters += 1;
    }
    const T ta = T(alpha), tw = T(omega);
    const long long off = s * g.cnt[3];
    T* x = kb.x + off;
    T* r = kb.r + off;
    const T* rh = kb.rhat + off;
    const T* pn = kb.P[par] + off;
    const T* vn = kb.V[par] + off;
    const T* t = kb.t + off;
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.bx, g.by, i, j, k0);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + g.tz, g.n[2]);
        for (int k = k0; k < k1; ++k) {
            const long long id = cindex(g, i, j, k);
            const T sc = r[id] - ta * vn[id];
            const T xv = x[id] + (ta * pn[id] + tw * sc);
            const T rv = sc - tw * t[id];
            x[id] = xv;
            r[id] = rv;
            acc[0] += double(rh[id] * rv);
            acc[1] += double(rv * rv);
            acc[2] += double(xv);
        }
    }
    write_partials<4>(acc, part_c + (s * g.ctas + blockIdx.x) * 4);
}

// ---------------------------------------------------------------------------
// FP32 storage + FP64 iterative refinement of the pressure solve
// ---------------------------------------------------------------------------

// Outer start: b <- b - mean(b) (FP64); p64 = p; r64 = b - L p (FP64);
// r32 = float(r64).  Partials: (r,r), (b,b), sum p.
static __global__ void __launch_bounds__(NTHREADS)
    k_refine_init(Geo g, SliceCtl* __restrict__ ctl, const double* __restrict__ part_b,
                  double* __restrict__ bvec, const double* __restrict__ p_in,
                  double* __restrict__ p64, float* __restrict__ r32, double* __restrict__ part_r) {
    const long long s = blockIdx.y;
    double sb[1];
    reduce_partials<1>(part_b + s * g.ctas, g.ctas, sb);
    const double mean = sb[0] / g.n_fluid;
    const long long off = s * g.cnt[3];
    double* b = bvec + off;
    const double* ps = p_in + off;
    double* pd = p64 + off;
    float* r = r32 + off;
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.bx, g.by, i, j, k0);
    double acc[3] = {0.0, 0.0, 0.0};
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + g.tz, g.n[2]);
        auto pv = [&](int a, int bb, int c) { return ps[cindex(g, a, bb, c)]; };
        for (int k = k0; k < k1; ++k) {
            const long long id = cindex(g, i, j, k);
            const bool sol = cell_solid(g, i, j, k);
            const double bv = sol ? 0.0 : b[id] - mean;
            const double pc = sol ? 0.0 : ps[id];
            const double rv = bv - lap_cell(g, pv, i, j, k, pc);
            b[id] = bv;
            pd[id] = pc;
            r[id] = float(rv);
            acc[0] += rv * rv;
            acc[1] += bv * bv;
            acc[2] += pc;
        }
    }
    write_partials<3>(acc, part_r + (s * g.ctas + blockIdx.x) * 3);
    if (blockIdx.x == 0 && tid_flat() == 0) {
        SliceCtl* c = ctl + s;
        c->o_status = OS_REFINE;
        c->o_steps = 0;
        c->p_final = 0;
        c->status = ST_IDLE;
    }
}

// Outer convergence test for outer step m, then the start of the inner FP32
// solve of L e = r32 from e = 0: r_hat = r32, e = 0.
static __global__ void __launch_bounds__(NTHREADS)
    k_inner_init(Geo g, KBuf<float> kb, SliceCtl* __restrict__ ctl,
                 const double* __restrict__ part_r, double* __restrict__ part_c, double tol2,
                 int m, int max_outer) {
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    if (c->o_status != OS_REFINE) return;
    double red[3];
    reduce_partials<3>(part_r + s * g.ctas * 3, g.ctas, red);
    const double rr = red[0];
    const double bb = m == 0 ? red[1] : c->o_bb;
    const bool lead = blockIdx.x == 0 && tid_flat() == 0;
    if (!isfinite(rr)) {
        if (lead) {
            c->o_status = OS_NONFINITE;
            c->o_rr = rr;
            c->status = ST_IDLE;
        }
        return;
    }
    if (rr <= tol2 * bb) {
        if (lead) {
            c->o_status = OS_DONE;
            c->o_rr = rr;
            c->o_bb = bb;
            c->p_final = m & 1;
            c->sx = red[2];
            c->status = ST_IDLE;
        }
        return;
    }
    if (m >= max_outer) {
        if (lead) {
            c->o_status = OS_FAIL;
            c->o_rr = rr;
            c->o_bb = bb;
            c->status = ST_IDLE;
        }
        return;
    }
    const long long off = s * g.cnt[3];
    const float* r = kb.r + off;
    float* rh = kb.rhat + off;
    float* e = kb.x + off;
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.bx, g.by, i, j, k0);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + g.tz, g.n[2]);
        for (int k = k0; k < k1; ++k) {
            const long long id = cindex(g, i, j, k);
            const float rv = r[id];
            rh[id] = rv;
            e[id] = 0.0f;
            acc[1] += double(rv) * double(rv);
        }
    }
    acc[0] = acc[1];
    acc[3] = acc[1];
    write_partials<4>(acc, part_c + (s * g.ctas + blockIdx.x) * 4);
    if (lead) {
        c->status = ST_ITER;
        c->it_cur = 0;
        c->it_next = 0;
        c->omega = 1.0;
        c->alpha = 1.0;
        c->o_steps = m;
        if (m == 0) c->o_bb = bb;
    }
}

// Outer correction: p_new = p_old + e (FP64); r64 = b - L p_new (FP64, p_new
// recomputed at the neighbours); r32 = float(r64).  Partials: (r,r), 0, sum p.
static __global__ void __launch_bounds__(NTHREADS)
    k_refine_update(Geo g, SliceCtl* __restrict__ ctl, const double* __restrict__ bvec,
                    const double* __restrict__ p_old, double* __restrict__ p_new,
                    const float* __restrict__ e_in, float* __restrict__ r32,
                    double* __restrict__ part_r) {
    const long long s = blockIdx.y;
    SliceCtl* c = ctl + s;
    if (c->o_status != OS_REFINE) return;
    if (c->status == ST_NONFINITE) {
        if (blockIdx.x == 0 && tid_flat() == 0) c->o_status = OS_NONFINITE;
        return;
    }
    // a converged inner solve, or one stopped at its iteration limit, still
    // improves p; the outer residual test decides when to stop
    const long long off = s * g.cnt[3];
    const double* b = bvec + off;
    const double* po = p_old + off;
    double* pn = p_new + off;
    const float* e = e_in + off;
    float* r = r32 + off;
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.bx, g.by, i, j, k0);
    double acc[3] = {0.0, 0.0, 0.0};
    if (i < g.n[0] && j < g.n[1]) {
        const int k1 = min(k0 + g.tz, g.n[2]);
        auto pv = [&](int a, int bb, int cc) {
            const long long q = cindex(g, a, bb, cc);
            return po[q] + double(e[q]);
        };
        for (int k = k0; k < k1; ++k) {
            const long long id = cindex(g, i, j, k);
            const double pc = pv(i, j, k);
            const double rv = b[id] - lap_cell(g, pv, i, j, k, pc);
            pn[id] = pc;
            r[id] = float(rv);
            acc[0] += rv * rv;
            acc[2] += pc;
        }
    }
    write_partials<3>(acc, part_r + (s * g.ctas + blockIdx.x) * 3);
}

// ---------------------------------------------------------------------------
// velocity correction u = F* - dt G p and the gauged pressure p - mean(p)
// ---------------------------------------------------------------------------

// x0/x1 select the solution buffer of each state: FP64 mode passes the same
// pointer twice; FP32+refine passes p64[0], p64[1] and the state's
// SliceCtl.p_final picks one.  fs == vel is allowed (in-place projection).
// INCR = false: u = F* - dt G p.  INCR = true: fs holds the increment F* - u
// and u = u + (increment - dt G p).
template <typename T, bool INCR>
__global__ void __launch_bounds__(NTHREADS)
    k_correct(Geo g, const SliceCtl* __restrict__ ctl, const T* fu, const T* fv, const T* fw,
              T* u, T* v, T* w, const double* __restrict__ x0, const double* __restrict__ x1,
              double* __restrict__ p_out, double dt, double* __restrict__ p_keep = nullptr) {
    pdl_wait();
    const long long s = blockIdx.y;
    const SliceCtl* c = ctl + s;
    const double* x = (c->p_final ? x1 : x0) + s * g.cnt[3];
    const double mean = c->sx / g.n_fluid;
    const T* f3[3] = {fu + s * g.cnt[0], fv + s * g.cnt[1], fw + s * g.cnt[2]};
    T* o3[3] = {u + s * g.cnt[0], v + s * g.cnt[1], w + s * g.cnt[2]};
    const double dtih[3] = {dt * g.ih[0], dt * g.ih[1], dt * g.ih[2]};
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.fbx, g.fby, i, j, k0);
    const int k1 = min(k0 + g.tz, g.n[2] + 1);
    for (int k = k0; k < k1; ++k) {
        const int q[3] = {i, j, k};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (i < g.ext[d][0] && j < g.ext[d][1] && k < g.ext[d][2]) {
                const long long id = vindex(g, d, i, j, k);
                const bool active = face_active_dev(g, d, q);
                if (!active) {
                    o3[d][id] = T(0);
                } else {
                    int lo[3] = {i, j, k};
                    lo[d] = q[d] == 0 ? g.n[d] - 1 : q[d] - 1;
                    // dt (G p) in FP64 (dt / h folded into one factor); in the
                    // increment form u + (increment - dt G p) is rounded once
                    const double dgp =
                        (x[cindex(g, i, j, k)] - x[cindex(g, lo[0], lo[1], lo[2])]) * dtih[d];
                    if (INCR)
                        o3[d][id] = o3[d][id] + (f3[d][id] - T(dgp));
                    else
                        o3[d][id] = f3[d][id] - T(dgp);
                }
            }
        }
        if (p_out && i < g.n[0] && j < g.n[1] && k < g.n[2]) {
            const long long id = cindex(g, i, j, k);
            const double pn = cell_solid(g, i, j, k) ? 0.0 : x[id] - mean;
            // p_keep (optional) receives the next solve's warm start, the
            // linear extrapolation 2 p^(n+1) - p^n
            if (p_keep) p_keep[s * g.cnt[3] + id] = 2.0 * pn - p_out[s * g.cnt[3] + id];
            p_out[s * g.cnt[3] + id] = pn;
        }
    }
}

// ---------------------------------------------------------------------------
// Parareal update (Eq. 6): y_next = F + (G_new - G_old), G_old <- G_new,
// defect = max |y_next - y_next_previous| (FP64, atomic max on the bits of a
// non-negative double, so the result does not depend on the order).
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(256)
    k_parareal_update(long long n, const T* __restrict__ fy, const T* __restrict__ gnew,
                      T* __restrict__ gold, T* __restrict__ y, unsigned long long* defect) {
    pdl_wait();
    double dmax = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const T gn = gnew[q];
        const T nv = fy[q] + (gn - gold[q]);
        const double d = fabs(double(nv) - double(y[q]));
        dmax = (d > dmax || d != d) ? d : dmax;
        y[q] = nv;
        gold[q] = gn;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double other = __shfl_xor_sync(0xffffffffu, dmax, o);
        dmax = (other > dmax || other != other) ? other : dmax;
    }
    if ((threadIdx.x & 31) == 0)
        atomicMax(defect, (unsigned long long)__double_as_longlong(dmax));
}

}  // namespace nsk
