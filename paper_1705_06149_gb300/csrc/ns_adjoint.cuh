// Discrete adjoint of the fine step (Section 2 discretisation), for the
// gradient of J = 1/2 sum over active faces of component^2 hx hy hz.
//
// One step is u+ = P(u + dt R(u; u_lid)), P = I - G L^-1 D (the projection,
// symmetric since D = -G^T), R = Re^-1 lap_h u - div_h(u u) with SMART faces.
// Its adjoint maps lambda = dJ/du+ to
//   mu = P lambda,   dJ/du = mu + dt (dR/du)^T mu,   dJ/du_lid += dt (dR/du_lid)^T mu.
// (dR/du)^T mu is gathered: every stored value sums the derivatives of the
// stencil terms that read it (directly, or through the ghost rule of a wall
// reading it as a mirror), each interface flux weighted by the difference of
// mu on its two faces.  Every output is written by one thread in a fixed
// order, so the gradient does not depend on scheduling.  SMART takes the
// branch the forward kernel took (the same division-free comparisons); a
// flux with zero transporting velocity takes the derivative of its
// left-upwind form.  T = double (FP64 grids) or float (FP32 storage; the lid
// derivative and J are summed in FP64).
#pragma once

#include "ns_kernels.cuh"

namespace nsk {

// partial derivatives of smart_face(U, C, D), branch by branch
template <typename T>
__device__ __forceinline__ void smart_partials(T U, T C, T D, T& dU, T& dC, T& dD) {
    dU = dC = dD = T(0);
    const T dd = D - U;
    const T cc = C - U;
    if (dd == T(0)) {
        dC = T(1);
        return;
    }
    const T a = dd > T(0) ? cc : -cc;
    const T b = fabs(dd);
    if (a < T(0) || a > b) {
        dC = T(1);
    } else if (T(6) * a <= b) {
        dU = T(-2);
        dC = T(3);
    } else if (T(6) * a <= T(5) * b) {
        dU = T(-0.125);
        dC = T(0.75);
        dD = T(0.375);
    } else {
        dD = T(1);
    }
}

// flux uf * phi between b (lower) and f (higher): d/d uf and d/d (bb, b, f, ff)
template <typename T>
__device__ __forceinline__ void flux_partials(T uf, T bb, T b, T f, T ff, T& duf, T (&d4)[4]) {
    T dU, dC, dD;
    d4[0] = d4[1] = d4[2] = d4[3] = T(0);
    if (uf < T(0)) {
        duf = smart_face(ff, f, b);
        smart_partials(ff, f, b, dU, dC, dD);
        d4[3] = uf * dU;
        d4[2] = uf * dC;
        d4[1] = uf * dD;
    } else {
        duf = smart_face(bb, b, f);
        smart_partials(bb, b, f, dU, dC, dD);
        d4[0] = uf * dU;
        d4[1] = uf * dC;
        d4[2] = uf * dD;
    }
}

// mu of component c at f (f[d] may lie outside the stored range along d):
// wrapped along a periodic axis, zero outside the stored range and on
// inactive (wall-normal boundary) faces.
template <typename T>
__device__ __forceinline__ T adj_mu_at(const Geo& g, int c, const T* __restrict__ mu, int d,
                                       const int f[3]) {
    int q[3] = {f[0], f[1], f[2]};
    const int e = g.ext[c][d];
    if (q[d] < 0 || q[d] >= e) {
        if (g.bc[d] != BC_PERIODIC) return T(0);
        q[d] = q[d] < 0 ? q[d] + e : q[d] - e;
    }
    const bool active = g.bc[c] == BC_PERIODIC || (q[c] > 0 && q[c] < g.n[c]);
    return active ? mu[vindex(g, c, q[0], q[1], q[2])] : T(0);
}

// Is p an interface of component c along d that a forward flux is evaluated
// at (between positions p and p+1)?  Periodic axes wrap p.  Normal
// component: between the active faces 1..n-1 and their neighbours (0..n-1);
// tangential: -1..n-1 (the edges on the walls included).
__device__ __forceinline__ bool adj_iface(const Geo& g, int c, int d, int& p) {
    if (g.bc[d] == BC_PERIODIC) {
        const int e = g.ext[c][d];
        p = p < 0 ? p + e : (p >= e ? p - e : p);
        return true;
    }
    return d == c ? (p >= 0 && p <= g.n[d] - 1) : (p >= -1 && p <= g.n[d] - 1);
}

// Derivatives of the forward flux of component c through the interface
// between f and f + e_d (f[d] = p): with respect to its transporting
// velocity (duf) and to the four values at f - e_d .. f + 2 e_d (d4).
template <typename T>
__device__ __forceinline__ void adj_iface_flux(const Geo& g, int c, int d,
                                               const T* const (&vel3)[3], const int f[3],
                                               T& duf, T (&d4)[4]) {
    T a[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int r[3] = {f[0], f[1], f[2]};
        r[d] += q - 1;
        a[q] = vel(g, c, vel3[c], r[0], r[1], r[2]);
    }
    T uf;
    if (d == c) {
        uf = T(0.5) * (a[1] + a[2]);
    } else {
        int q0[3] = {f[0], f[1], f[2]};
        int q1[3] = {f[0], f[1], f[2]};
        q0[c] -= 1;
        q0[d] += 1;
        q1[d] += 1;
        uf = T(0.5) * (vel(g, d, vel3[d], q0[0], q0[1], q0[2]) +
                       vel(g, d, vel3[d], q1[0], q1[1], q1[2]));
    }
    flux_partials(uf, a[0], a[1], a[2], a[3], duf, d4);
}

// (dR/du)^T mu at the stored value t of component c, and its share of
// (dR/du_lid)^T mu (returned in dl).
template <typename T>
__device__ __forceinline__ T adj_gather(const Geo& g, int c, const int t[3],
                                        const T* const (&vel3)[3], const T* const (&mu3)[3],
                                        double& dl) {
    T acc = T(0);
    const T inv_re = g_inv_re<T>(g);
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
        const T ih = g_ih<T>(g, d), ih2 = g_ih2<T>(g, d);
        const int n = g.n[d], x = t[d];
        // the positions whose value is t's: t itself and the ghosts that
        // mirror it (sign, and the lid's coefficient in the ghost value)
        int r[3];
        T sg[3];
        T lid[3];
        int nim = 0;
        r[nim] = x;
        sg[nim] = T(1);
        lid[nim++] = T(0);
        if (g.bc[d] != BC_PERIODIC) {
            if (d == c) {
                if (x >= 1 && x <= 2) {
                    r[nim] = -x;
                    sg[nim] = T(-1);
                    lid[nim++] = T(0);
                }
                if (x >= n - 2 && x <= n - 1 && x >= 0) {
                    r[nim] = 2 * n - x;
                    sg[nim] = T(-1);
                    lid[nim++] = T(0);
                }
            } else {
                const T s = g.bc[d] == BC_SLIP ? T(1) : T(-1);
                if (x <= 1) {
                    r[nim] = -x - 1;
                    sg[nim] = s;
                    lid[nim++] = T(0);
                }
                if (x >= n - 2) {
                    r[nim] = 2 * n - 1 - x;
                    sg[nim] = s;
                    lid[nim++] = (g.bc[d] == BC_WALL && c == 0 && d == 1) ? T(2) : T(0);
                }
            }
        }
#pragma unroll 1
        for (int m = 0; m < nim; ++m) {
            int f[3] = {t[0], t[1], t[2]};
            // diffusion Re^-1 (a3 - 2 a2 + a1) / h^2 of the faces r+1, r, r-1
            T sd = T(0);
#pragma unroll
            for (int o = -1; o <= 1; ++o) {
                f[d] = r[m] + o;
                sd += (o == 0 ? T(-2) : T(1)) * adj_mu_at(g, c, mu3[c], d, f);
            }
            T tot = inv_re * ih2 * sd;
            // convection -(F(p) - F(p-1)) / h: the interfaces p = r - k that
            // read r in role k (k = -1: far upwind below, 0, 1, 2)
#pragma unroll 1
            for (int k = -1; k <= 2; ++k) {
                int p = r[m] - k;
                if (!adj_iface(g, c, d, p)) continue;
                f[d] = p + 1;
                const T hi = adj_mu_at(g, c, mu3[c], d, f);
                f[d] = p;
                const T lo = adj_mu_at(g, c, mu3[c], d, f);
                const T nu = (hi - lo) * ih;
                if (nu == T(0)) continue;
                T duf, d4[4];
                adj_iface_flux(g, c, d, vel3, f, duf, d4);
                T w = d4[k + 1];
                if (d == c && (k == 0 || k == 1)) w += T(0.5) * duf;
                tot += nu * w;
            }
            acc += sg[m] * tot;
            dl += double(lid[m]) * double(tot);
        }
    }
    // t as the transporting velocity of the other components' fluxes along
    // its own axis: the interfaces of faces t - e_c and t - e_c + e_c2
#pragma unroll 1
    for (int c2 = 0; c2 < 3; ++c2) {
        if (c2 == c) continue;
        const int d = c;
        const T ih = g_ih<T>(g, d);
#pragma unroll 1
        for (int cand = 0; cand < 2; ++cand) {
            int f[3] = {t[0], t[1], t[2]};
            int p = f[d] - 1;
            if (!adj_iface(g, c2, d, p)) continue;
            f[d] = p;
            if (cand) {
                f[c2] += 1;
                if (f[c2] >= g.ext[c2][c2]) {
                    if (g.bc[c2] != BC_PERIODIC) continue;
                    f[c2] -= g.ext[c2][c2];
                }
            }
            int fh[3] = {f[0], f[1], f[2]};
            fh[d] += 1;
            const T nu = (adj_mu_at(g, c2, mu3[c2], d, fh) - adj_mu_at(g, c2, mu3[c2], d, f)) * ih;
            if (nu == T(0)) continue;
            T duf, d4[4];
            adj_iface_flux(g, c2, d, vel3, f, duf, d4);
            acc += T(0.5) * nu * duf;
        }
    }
    return acc;
}

// out = (dR/du)^T mu for every state of the batch (blockIdx.y), every stored
// value written once, component blockIdx.z; each thread gathers ADJ_TZ
// positions along z of a 32 x 4 column tile (the gather is latency-bound, so
// the launch spreads over many CTAs).  Per-CTA partial sums of
// (dR/du_lid)^T mu go to part_lid[state][component][cta] (summed in a fixed
// order by k_adj_sum).
constexpr int ADJ_TZ = 2;

template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_adj_rhs(Geo g, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ w,
              const T* __restrict__ mu_u, const T* __restrict__ mu_v, const T* __restrict__ mu_w,
              T* __restrict__ ou, T* __restrict__ ov, T* __restrict__ ow,
              double* __restrict__ part_lid) {
    const long long s = blockIdx.y;
    const int c = blockIdx.z;
    const T* const vel3[3] = {u + s * g.cnt[0], v + s * g.cnt[1], w + s * g.cnt[2]};
    const T* const mu3[3] = {mu_u + s * g.cnt[0], mu_v + s * g.cnt[1], mu_w + s * g.cnt[2]};
    T* const out = (c == 0 ? ou : (c == 1 ? ov : ow)) + s * g.cnt[c];
    const int cta = blockIdx.x;
    const int i = (cta % g.fbx) * TX + (int)threadIdx.x;
    const int r = cta / g.fbx;
    const int j = (r % g.fby) * TY + (int)threadIdx.y;
    const int k0 = (r / g.fby) * ADJ_TZ;
    const int k1 = min(k0 + ADJ_TZ, g.ext[c][2]);
    double dl = 0.0;
    if (i < g.ext[c][0] && j < g.ext[c][1]) {
        for (int k = k0; k < k1; ++k) {
            const int t[3] = {i, j, k};
            out[vindex(g, c, i, j, k)] = adj_gather(g, c, t, vel3, mu3, dl);
        }
    }
    double v1[1] = {dl};
    write_partials<1>(v1, part_lid + (s * 3 + c) * (long long)gridDim.x + blockIdx.x);
}

// out[s] (+)= sum of part[s][0..n-1] in order, one thread per state.
__global__ void __launch_bounds__(32)
    k_adj_sum(const double* __restrict__ part, int n, int batch, double* __restrict__ out,
              int add) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= batch) return;
    double acc = 0.0;
    for (int q = 0; q < n; ++q) acc += part[(long long)s * n + q];
    out[s] = add ? out[s] + acc : acc;
}

// lambda = mu + dt * acc on active faces, 0 elsewhere; acc is zeroed for reuse.
template <typename T>
__global__ void __launch_bounds__(256)
    k_adj_finish(Geo g, int c, long long n_total, const T* __restrict__ mu,
                 T* __restrict__ acc, T* __restrict__ lam, double dt) {
    const T tdt = T(dt);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n_total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long local = q % g.cnt[c];
        const int i = int(local % g.ext[c][0]);
        const int j = int((local / g.ext[c][0]) % g.ext[c][1]);
        const int k = int(local / ((long long)g.ext[c][0] * g.ext[c][1]));
        const int f[3] = {i, j, k};
        const bool active = g.bc[c] == BC_PERIODIC || (f[c] > 0 && f[c] < g.n[c]);
        lam[q] = active ? mu[q] + tdt * acc[q] : T(0);
        acc[q] = T(0);
    }
}

// lambda = u * vol on active faces (0 elsewhere; skipped when lam is null)
// and the per-CTA partial sums of J = 1/2 sum u^2 vol in part[state][cta]
// (blockIdx.y = state; the CTAs of the three components at offsets
// c * gridDim.x).
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
    k_adj_terminal(Geo g, int c, const T* __restrict__ u, T* __restrict__ lam,
                   double* __restrict__ part, double vol) {
    const long long s = blockIdx.y;
    const long long per = g.cnt[c];
    const T* us = u + s * per;
    T* ls = lam ? lam + s * per : nullptr;
    const T tvol = T(vol);
    double acc = 0.0;
    for (long long q = blockIdx.x * (long long)NTHREADS + tid_flat(); q < per;
         q += (long long)gridDim.x * NTHREADS) {
        const int i = int(q % g.ext[c][0]);
        const int j = int((q / g.ext[c][0]) % g.ext[c][1]);
        const int k = int(q / ((long long)g.ext[c][0] * g.ext[c][1]));
        const int f[3] = {i, j, k};
        const bool active = g.bc[c] == BC_PERIODIC || (f[c] > 0 && f[c] < g.n[c]);
        const T x = active ? us[q] : T(0);
        if (ls) ls[q] = x * tvol;
        acc += 0.5 * double(x) * double(x) * vol;
    }
    double v1[1] = {acc};
    write_partials<1>(v1, part + s * 3LL * gridDim.x + (long long)c * gridDim.x + blockIdx.x);
}

}  // namespace nsk
