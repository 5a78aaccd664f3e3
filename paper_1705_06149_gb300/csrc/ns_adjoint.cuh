// Discrete adjoint of the fine step (Section 2 discretisation), for the
// gradient of J = 1/2 sum over active faces of component^2 hx hy hz.
//
// One step is u+ = P(u + dt R(u; u_lid)), P = I - G L^-1 D (the projection,
// symmetric since D = -G^T), R = Re^-1 lap_h u - div_h(u u) with SMART faces.
// Its adjoint maps lambda = dJ/du+ to
//   mu = P lambda,   dJ/du = mu + dt (dR/du)^T mu,   dJ/du_lid += dt (dR/du_lid)^T mu.
// (dR/du)^T mu is formed by differentiating every stencil term of R with
// respect to the stored values (and the lid speed) it reads, and adding the
// products into the output with FP64 atomics.  SMART takes the branch the
// forward kernel took (the same division-free comparisons); a flux with zero
// transporting velocity takes the derivative of its left-upwind form.
#pragma once

#include "ns_kernels.cuh"

namespace nsk {

// value of component c at (i,j,k) = sign * a[idx] + lid * u_lid
struct VSrc {
    long long idx;
    double sign;
    double lid;
};

__device__ __forceinline__ VSrc vel_src(const Geo& g, int c, int i, int j, int k) {
    int q[3] = {i, j, k};
    double sign = 1.0, lid = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int e = g.ext[c][d];
        int x = q[d];
        if (x < 0 || x >= e) {
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
                    if (c == 0 && d == 1 && hi) lid = 2.0;
                }
            }
            q[d] = x;
        }
    }
    VSrc r;
    r.idx = vindex(g, c, q[0], q[1], q[2]);
    r.sign = sign;
    r.lid = lid;
    return r;
}

// partial derivatives of smart_face(U, C, D), branch by branch
__device__ __forceinline__ void smart_partials(double U, double C, double D, double& dU,
                                               double& dC, double& dD) {
    dU = dC = dD = 0.0;
    const double dd = D - U;
    const double cc = C - U;
    if (dd == 0.0) {
        dC = 1.0;
        return;
    }
    const double a = dd > 0.0 ? cc : -cc;
    const double b = fabs(dd);
    if (a < 0.0 || a > b) {
        dC = 1.0;
    } else if (6.0 * a <= b) {
        dU = -2.0;
        dC = 3.0;
    } else if (6.0 * a <= 5.0 * b) {
        dU = -0.125;
        dC = 0.75;
        dD = 0.375;
    } else {
        dD = 1.0;
    }
}

// flux uf * phi between b (lower) and f (higher): d/d uf and d/d (bb, b, f, ff)
__device__ __forceinline__ void flux_partials(double uf, double bb, double b, double f,
                                              double ff, double& duf, double (&d4)[4]) {
    double dU, dC, dD;
    d4[0] = d4[1] = d4[2] = d4[3] = 0.0;
    if (uf < 0.0) {
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

__device__ __forceinline__ void adj_scatter(double* const* out, int c, const VSrc& s, double w,
                                            double& dlid) {
    if (w != 0.0) atomicAdd(out[c] + s.idx, s.sign * w);
    dlid += s.lid * w;
}

// out += (dR/du)^T mu for every state of the batch; dlid[s] += (dR/du_lid)^T mu.
__global__ void __launch_bounds__(NTHREADS)
    k_adj_rhs(Geo g, const double* __restrict__ u, const double* __restrict__ v,
              const double* __restrict__ w, const double* __restrict__ mu_u,
              const double* __restrict__ mu_v, const double* __restrict__ mu_w, double* ou,
              double* ov, double* ow, double* __restrict__ dlid) {
    const long long s = blockIdx.y;
    const double* vel3[3] = {u + s * g.cnt[0], v + s * g.cnt[1], w + s * g.cnt[2]};
    const double* mu3[3] = {mu_u + s * g.cnt[0], mu_v + s * g.cnt[1], mu_w + s * g.cnt[2]};
    double* out[3] = {ou + s * g.cnt[0], ov + s * g.cnt[1], ow + s * g.cnt[2]};
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.fbx, g.fby, i, j, k0);
    const int k1 = min(k0 + g.tz, g.n[2] + 1);
    double dl = 0.0;
    for (int k = k0; k < k1; ++k) {
        for (int c = 0; c < 3; ++c) {
            if (!(i < g.ext[c][0] && j < g.ext[c][1] && k < g.ext[c][2])) continue;
            const int f[3] = {i, j, k};
            const bool active = g.bc[c] == BC_PERIODIC || (f[c] > 0 && f[c] < g.n[c]);
            if (!active) continue;
            const double m = mu3[c][vindex(g, c, i, j, k)];
            if (m == 0.0) continue;
            for (int d = 0; d < 3; ++d) {
                VSrc sa[5];
                double a[5];
                for (int q = 0; q < 5; ++q) {
                    int p3[3] = {f[0], f[1], f[2]};
                    p3[d] += q - 2;
                    sa[q] = vel_src(g, c, p3[0], p3[1], p3[2]);
                    a[q] = vel(g, c, vel3[c], p3[0], p3[1], p3[2]);
                }
                // diffusion Re^-1 (a3 - 2 a2 + a1) / h^2
                const double wd = g.inv_re * g.ih2[d] * m;
                adj_scatter(out, c, sa[3], wd, dl);
                adj_scatter(out, c, sa[2], -2.0 * wd, dl);
                adj_scatter(out, c, sa[1], wd, dl);
                // convection -(Fp - Fm) / h
                double up, um;
                VSrc tp[2], tm[2];
                int tc;
                if (d == c) {
                    tc = c;
                    tp[0] = sa[2];
                    tp[1] = sa[3];
                    tm[0] = sa[1];
                    tm[1] = sa[2];
                    up = 0.5 * (a[2] + a[3]);
                    um = 0.5 * (a[1] + a[2]);
                } else {
                    tc = d;
                    int q0[3] = {f[0], f[1], f[2]};
                    int q1[3] = {f[0], f[1], f[2]};
                    q0[c] = f[c] - 1;
                    q0[d] = f[d] + 1;
                    q1[d] = f[d] + 1;
                    tp[0] = vel_src(g, d, q0[0], q0[1], q0[2]);
                    tp[1] = vel_src(g, d, q1[0], q1[1], q1[2]);
                    up = 0.5 * (vel(g, d, vel3[d], q0[0], q0[1], q0[2]) +
                                vel(g, d, vel3[d], q1[0], q1[1], q1[2]));
                    q0[d] = f[d];
                    q1[d] = f[d];
                    tm[0] = vel_src(g, d, q0[0], q0[1], q0[2]);
                    tm[1] = vel_src(g, d, q1[0], q1[1], q1[2]);
                    um = 0.5 * (vel(g, d, vel3[d], q0[0], q0[1], q0[2]) +
                                vel(g, d, vel3[d], q1[0], q1[1], q1[2]));
                }
                double dup, dum, dp[4], dm[4];
                flux_partials(up, a[1], a[2], a[3], a[4], dup, dp);
                flux_partials(um, a[0], a[1], a[2], a[3], dum, dm);
                const double wc = -m * g.ih[d];
                for (int q = 0; q < 4; ++q) {
                    adj_scatter(out, c, sa[q + 1], wc * dp[q], dl);
                    adj_scatter(out, c, sa[q], -wc * dm[q], dl);
                }
                for (int q = 0; q < 2; ++q) {
                    adj_scatter(out, tc, tp[q], 0.5 * wc * dup, dl);
                    adj_scatter(out, tc, tm[q], -0.5 * wc * dum, dl);
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) dl += __shfl_xor_sync(0xffffffffu, dl, o);
    if ((threadIdx.x & 31) == 0 && dl != 0.0) atomicAdd(dlid + s, dl);
}

// lambda = mu + dt * acc on active faces, 0 elsewhere; acc is zeroed for reuse.
__global__ void __launch_bounds__(256)
    k_adj_finish(Geo g, int c, long long n_total, const double* __restrict__ mu,
                 double* __restrict__ acc, double* __restrict__ lam, double dt) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n_total;
         q += (long long)gridDim.x * blockDim.x) {
        const long long local = q % g.cnt[c];
        const int i = int(local % g.ext[c][0]);
        const int j = int((local / g.ext[c][0]) % g.ext[c][1]);
        const int k = int(local / ((long long)g.ext[c][0] * g.ext[c][1]));
        const int f[3] = {i, j, k};
        const bool active = g.bc[c] == BC_PERIODIC || (f[c] > 0 && f[c] < g.n[c]);
        lam[q] = active ? mu[q] + dt * acc[q] : 0.0;
        acc[q] = 0.0;
    }
}

// lambda = u * vol on active faces (0 elsewhere) and J[s] += 1/2 sum u^2 vol
// (blockIdx.y = state; one atomic per warp).
__global__ void __launch_bounds__(256)
    k_adj_terminal(Geo g, int c, const double* __restrict__ u, double* __restrict__ lam,
                   double* __restrict__ J, double vol) {
    const long long s = blockIdx.y;
    const long long per = g.cnt[c];
    const double* us = u + s * per;
    double* ls = lam + s * per;
    double acc = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < per;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = int(q % g.ext[c][0]);
        const int j = int((q / g.ext[c][0]) % g.ext[c][1]);
        const int k = int(q / ((long long)g.ext[c][0] * g.ext[c][1]));
        const int f[3] = {i, j, k};
        const bool active = g.bc[c] == BC_PERIODIC || (f[c] > 0 && f[c] < g.n[c]);
        const double x = active ? us[q] : 0.0;
        ls[q] = x * vol;
        acc += 0.5 * x * x * vol;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(J + s, acc);
}

}  // namespace nsk
