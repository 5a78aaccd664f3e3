/*
 * ns_oracle.c -- plain FP64 CPU oracle for the projection time-stepper of
 * Croce, Ruprecht & Krause, "Parallel-in-Space-and-Time Simulation of the
 * Three-Dimensional, Unsteady Navier-Stokes Equations for Incompressible Flow"
 * (arXiv 1705.06149), Section 2.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct reference the
 * CUDA library is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * What it computes (Section 2 of the paper, readings where the paper is silent
 * are listed in the design notes):
 *   - incompressible Navier-Stokes, dimensionless, parameter Re (Eq. 1);
 *   - uniform Cartesian staggered (MAC) mesh: u on x-faces, v on y-faces,
 *     w on z-faces, p at cell centres;
 *   - Chorin-Temam projection with first-order forward Euler in time;
 *   - second-order central differences for diffusion and the pressure gradient;
 *   - convection in conservative form, face values from the SMART bounded-QUICK
 *     upwind scheme (Gaskell & Lau's normalised-variable map);
 *   - pressure Poisson equation solved with BiCGStab (van der Vorst).
 *
 * Array layout (x fastest), one state:
 *   u [nz][ny][nx+1]   (nx faces along a periodic x axis)
 *   v [nz][ny+1][nx]
 *   w [nz+1][ny][nx]
 *   p [nz][ny][nx]
 * Wall-normal boundary faces are stored and are identically zero.
 *
 * Boundary rules (ghost values of a velocity component along one axis d):
 *   wall, normal component  : reflected with a sign change about the wall face
 *                             (value at the wall is zero);
 *   wall, tangential        : ghost = 2*u_wall - mirror  (u_wall = lid speed for
 *                             u on the top face y = ly, zero elsewhere);
 *   slip, tangential        : ghost = +mirror;  slip, normal: as a wall;
 *   periodic                : wrap.
 * The pressure uses homogeneous Neumann conditions: faces on walls are dropped
 * from the Laplacian.  Solid cells (obstacles) drop their faces the same way.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OG_WALL 0
#define OG_PERIODIC 1
#define OG_SLIP 2

#define OG_OK 0
#define OG_ERR_ARG 1
#define OG_ERR_NOT_CONVERGED 4
#define OG_ERR_NONFINITE 5

typedef struct {
    int nx, ny, nz;
    double lx, ly, lz;
    double re;          /* Reynolds number; re <= 0 means inviscid (1/Re = 0) */
    double u_lid;       /* tangential speed of the top face y = ly, along +x   */
    int bc[3];          /* per axis: OG_WALL, OG_PERIODIC or OG_SLIP            */
    const uint8_t *solid; /* nz*ny*nx cell mask (1 = solid) or NULL            */
} og_grid;

/* ------------------------------------------------------------------------- */
/* geometry helpers                                                           */
/* ------------------------------------------------------------------------- */

static int ncell(const og_grid *g, int d) { return d == 0 ? g->nx : (d == 1 ? g->ny : g->nz); }
static double hstep(const og_grid *g, int d)
{
    return d == 0 ? g->lx / g->nx : (d == 1 ? g->ly / g->ny : g->lz / g->nz);
}

/* number of stored positions of velocity component c along axis d */
static int npos(const og_grid *g, int c, int d)
{
    int n = ncell(g, d);
    if (c == d && g->bc[d] != OG_PERIODIC) return n + 1;
    return n;
}

int og_count(const og_grid *g, int c) /* c = 0,1,2 velocity; 3 pressure */
{
    if (c == 3) return g->nx * g->ny * g->nz;
    return npos(g, c, 0) * npos(g, c, 1) * npos(g, c, 2);
}

static long vidx(const og_grid *g, int c, int i, int j, int k)
{
    return ((long)k * npos(g, c, 1) + j) * npos(g, c, 0) + i;
}

static long cidx(const og_grid *g, int i, int j, int k)
{
    return ((long)k * g->ny + j) * g->nx + i;
}

static int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

static int is_solid(const og_grid *g, int i, int j, int k)
{
    if (!g->solid) return 0;
    return g->solid[cidx(g, i, j, k)] != 0;
}

/* Is the face of component d at stored index (i,j,k) a face that moves fluid?
 * A face is active when it is not a wall-normal boundary face and both cells
 * next to it are fluid. */
static int face_active(const og_grid *g, int d, int i, int j, int k)
{
    int idx[3] = {i, j, k};
    int n = ncell(g, d);
    if (g->bc[d] != OG_PERIODIC && (idx[d] == 0 || idx[d] == n)) return 0;
    if (g->solid) {
        int lo[3] = {i, j, k};
        lo[d] = (g->bc[d] == OG_PERIODIC) ? wrap(idx[d] - 1, n) : idx[d] - 1;
        int hi[3] = {i, j, k};
        hi[d] = (g->bc[d] == OG_PERIODIC) ? wrap(idx[d], n) : idx[d];
        if (is_solid(g, lo[0], lo[1], lo[2]) || is_solid(g, hi[0], hi[1], hi[2])) return 0;
    }
    return 1;
}

/* Wall speed of component c on the wall at the end 'side' (0 low, 1 high) of
 * axis d.  Only the lid (top face y = ly) moves, along +x. */
static double wall_speed(const og_grid *g, int c, int d, int side)
{
    return (c == 0 && d == 1 && side == 1) ? g->u_lid : 0.0;
}

/* Value of velocity component c at index (i,j,k), which may lie up to two
 * positions outside the stored range along at most one axis. */
static double vget(const og_grid *g, int c, const double *a, int i, int j, int k)
{
    int idx[3] = {i, j, k};
    int out_axis = -1;
    for (int d = 0; d < 3; d++) {
        int n = npos(g, c, d);
        if (idx[d] < 0 || idx[d] >= n) {
            if (g->bc[d] == OG_PERIODIC) {
                idx[d] = wrap(idx[d], n);
            } else {
                if (out_axis >= 0) abort(); /* corners are never read */
                out_axis = d;
            }
        }
    }
    if (out_axis < 0) return a[vidx(g, c, idx[0], idx[1], idx[2])];
    int d = out_axis;
    int n = ncell(g, d);
    int side = idx[d] < 0 ? 0 : 1;
    if (c == d) {
        /* normal component: faces 0..n, wall faces hold 0; odd reflection */
        int m = side == 0 ? -idx[d] : 2 * n - idx[d];
        idx[d] = m;
        return -a[vidx(g, c, idx[0], idx[1], idx[2])];
    }
    /* tangential component: cells 0..n-1, wall halfway between -1 and 0 */
    int m = side == 0 ? -idx[d] - 1 : 2 * n - 1 - idx[d];
    idx[d] = m;
    double mirror = a[vidx(g, c, idx[0], idx[1], idx[2])];
    if (g->bc[d] == OG_SLIP) return mirror;
    return 2.0 * wall_speed(g, c, d, side) - mirror;
}

/* vget for the tests that pin the ghost rules by hand values: the value of
 * velocity component c (0 u, 1 v, 2 w) of field a at (i,j,k), up to two
 * positions outside the stored range along one axis. */
double og_vget(const og_grid *g, int c, const double *a, int i, int j, int k)
{
    return vget(g, c, a, i, j, k);
}

static double pget(const og_grid *g, const double *p, int i, int j, int k)
{
    int idx[3] = {i, j, k};
    for (int d = 0; d < 3; d++)
        if (g->bc[d] == OG_PERIODIC) idx[d] = wrap(idx[d], ncell(g, d));
    return p[cidx(g, idx[0], idx[1], idx[2])];
}

/* ------------------------------------------------------------------------- */
/* SMART (Gaskell & Lau 1988): normalised-variable face value                  */
/* ------------------------------------------------------------------------- */

/* Face value from the far-upwind (U), upwind (C) and downwind (D) node values.
 * phi_hat = (C-U)/(D-U); the face value in normalised form is
 *   3 phi_hat            on [0, 1/6]
 *   3/4 phi_hat + 3/8    on [1/6, 5/6]   (QUICK)
 *   1                    on [5/6, 1]
 *   phi_hat              otherwise       (first-order upwind)
 * With D == U the profile is flat (or an extremum) and the face takes C. */
double og_smart(double U, double C, double D)
{
    if (D == U) return C;
    double ph = (C - U) / (D - U);
    double pf;
    if (ph < 0.0 || ph > 1.0) pf = ph;
    else if (ph <= 1.0 / 6.0) pf = 3.0 * ph;
    else if (ph <= 5.0 / 6.0) pf = 0.75 * ph + 0.375;
    else pf = 1.0;
    return U + pf * (D - U);
}

/* Convective flux through a face whose transporting velocity is Uf, between
 * node values b (behind, lower index) and f (front, higher index); bb is the
 * node behind b and ff the node in front of f. */
static double smart_flux(double Uf, double bb, double b, double f, double ff)
{
    if (Uf > 0.0) return Uf * og_smart(bb, b, f);
    if (Uf < 0.0) return Uf * og_smart(ff, f, b);
    return 0.0;
}

/* ------------------------------------------------------------------------- */
/* predictor:  F* = u + dt (Re^-1 lap(u) - div(u u))                           */
/* ------------------------------------------------------------------------- */

/* The adjoint does not take solid cells (the forward does). */
static int solid_arms_unsupported(const og_grid *g)
{
    return g->solid != NULL;
}

/* Is the stored face of component c at (i,j,k) (in range) inside a solid,
 * i.e. are both cells next to it along axis c solid? */
static int face_in_solid(const og_grid *g, int c, const int q[3])
{
    int n = ncell(g, c);
    int lo[3] = {q[0], q[1], q[2]}, hi[3] = {q[0], q[1], q[2]};
    lo[c] = q[c] - 1;
    hi[c] = q[c];
    if (g->bc[c] == OG_PERIODIC) {
        lo[c] = wrap(lo[c], n);
        hi[c] = wrap(hi[c], n);
    } else if (lo[c] < 0 || hi[c] >= n) {
        return 0; /* a wall face */
    }
    return is_solid(g, lo[0], lo[1], lo[2]) && is_solid(g, hi[0], hi[1], hi[2]);
}

/* Value of component c at offset m (|m| <= 2) from face f along axis d, as
 * seen by f's stencil arm when the grid has solid cells: stored values up to
 * the first interface the arm meets, reflected across it beyond.
 *   normal arm (d == c): the first inactive face (a wall face or a face on a
 *     solid surface, value 0) is the interface; beyond it the arm takes the
 *     odd reflection about that face.
 *   tangential arm (d != c): the first position past a wall or inside a solid
 *     starts the ghost region; ghost = 2 u_wall - mirror (u_wall = 0 at
 *     solids, the lid speed at the lid; +mirror at a slip wall).
 * Without an interface within |m| positions the plain vget value is used. */
static double arm_value(const og_grid *g, int c, const double *a, const int f[3], int d, int m)
{
    if (m == 0) return a[vidx(g, c, f[0], f[1], f[2])];
    int sg = m > 0 ? 1 : -1;
    int am = m > 0 ? m : -m;
    for (int s = 1; s <= am; s++) {
        int q[3] = {f[0], f[1], f[2]};
        q[d] += sg * s;
        int n = npos(g, c, d);
        if (g->bc[d] == OG_PERIODIC) q[d] = wrap(q[d], n);
        if (c == d) {
            if (q[d] < 0 || q[d] >= n) break; /* cannot happen before a wall face */
            if (!face_active(g, c, q[0], q[1], q[2])) {
                if (s == am) return 0.0;
                /* s < am: reflect the remaining offset about this face */
                int r[3] = {f[0], f[1], f[2]};
                r[d] += sg * (2 * s - am);
                if (g->bc[d] == OG_PERIODIC) r[d] = wrap(r[d], n);
                return -a[vidx(g, c, r[0], r[1], r[2])];
            }
        } else {
            int outside = q[d] < 0 || q[d] >= n;
            if (outside || face_in_solid(g, c, q)) {
                /* interface between offsets s-1 and s; mirror of offset am
                 * (offset -1 when s = 1 and am = 2: read through the wall rules) */
                int r[3] = {f[0], f[1], f[2]};
                r[d] += sg * (2 * s - 1 - am);
                double mirror = vget(g, c, a, r[0], r[1], r[2]);
                if (outside) {
                    if (g->bc[d] == OG_SLIP) return mirror;
                    return 2.0 * wall_speed(g, c, d, q[d] < 0 ? 0 : 1) - mirror;
                }
                return -mirror;
            }
        }
    }
    int q[3] = {f[0], f[1], f[2]};
    q[d] += m;
    return vget(g, c, a, q[0], q[1], q[2]);
}

/* conv and diff of component c at face (i,j,k) of state (u,v,w) */
static void rhs_terms(const og_grid *g, int c, const double *const vel[3],
                      int i, int j, int k, double *conv_out, double *diff_out)
{
    double conv = 0.0, diff = 0.0;
    int f[3] = {i, j, k};
    for (int d = 0; d < 3; d++) {
        double h = hstep(g, d);
        double a[5];
        for (int m = -2; m <= 2; m++) {
            if (g->solid) {
                a[m + 2] = arm_value(g, c, vel[c], f, d, m);
            } else {
                int q[3] = {f[0], f[1], f[2]};
                q[d] += m;
                a[m + 2] = vget(g, c, vel[c], q[0], q[1], q[2]);
            }
        }
        double Up, Um;
        if (d == c) {
            /* fluxes at the cell centres on either side of the face */
            Up = 0.5 * (a[2] + a[3]);
            Um = 0.5 * (a[1] + a[2]);
        } else {
            /* fluxes at the cell edges: component d averaged over the two
             * positions of the face along axis c */
            int q0[3] = {f[0], f[1], f[2]};
            int q1[3] = {f[0], f[1], f[2]};
            q0[c] = f[c] - 1;
            q1[c] = f[c];
            q0[d] = f[d] + 1;
            q1[d] = f[d] + 1;
            Up = 0.5 * (vget(g, d, vel[d], q0[0], q0[1], q0[2]) +
                        vget(g, d, vel[d], q1[0], q1[1], q1[2]));
            q0[d] = f[d];
            q1[d] = f[d];
            Um = 0.5 * (vget(g, d, vel[d], q0[0], q0[1], q0[2]) +
                        vget(g, d, vel[d], q1[0], q1[1], q1[2]));
        }
        double Fp = smart_flux(Up, a[1], a[2], a[3], a[4]);
        double Fm = smart_flux(Um, a[0], a[1], a[2], a[3]);
        conv += (Fp - Fm) / h;
        diff += (a[3] - 2.0 * a[2] + a[1]) / (h * h);
    }
    *conv_out = conv;
    *diff_out = diff;
}

/* Split right-hand side for tests: conv = div(u u) and diff = lap(u) on every
 * active face of every component (zero elsewhere). */
int og_rhs(const og_grid *g, const double *u, const double *v, const double *w,
           double *cu, double *cv, double *cw, double *du, double *dv, double *dw)
{
    const double *vel[3] = {u, v, w};
    double *co[3] = {cu, cv, cw};
    double *di[3] = {du, dv, dw};
    for (int c = 0; c < 3; c++)
        for (int k = 0; k < npos(g, c, 2); k++)
            for (int j = 0; j < npos(g, c, 1); j++)
                for (int i = 0; i < npos(g, c, 0); i++) {
                    long id = vidx(g, c, i, j, k);
                    if (!face_active(g, c, i, j, k)) {
                        co[c][id] = 0.0;
                        di[c][id] = 0.0;
                        continue;
                    }
                    rhs_terms(g, c, vel, i, j, k, &co[c][id], &di[c][id]);
                }
    return OG_OK;
}

int og_predict(const og_grid *g, const double *u, const double *v, const double *w,
               double dt, double *fu, double *fv, double *fw)
{
    const double *vel[3] = {u, v, w};
    double *out[3] = {fu, fv, fw};
    double inv_re = g->re > 0.0 ? 1.0 / g->re : 0.0;
    for (int c = 0; c < 3; c++)
        for (int k = 0; k < npos(g, c, 2); k++)
            for (int j = 0; j < npos(g, c, 1); j++)
                for (int i = 0; i < npos(g, c, 0); i++) {
                    long id = vidx(g, c, i, j, k);
                    if (!face_active(g, c, i, j, k)) {
                        out[c][id] = 0.0;
                        continue;
                    }
                    double conv, diff;
                    rhs_terms(g, c, vel, i, j, k, &conv, &diff);
                    out[c][id] = vel[c][id] + dt * (inv_re * diff - conv);
                }
    return OG_OK;
}

/* ------------------------------------------------------------------------- */
/* discrete divergence D, gradient G and Laplacian L = D G                    */
/* ------------------------------------------------------------------------- */

static double face_val(const og_grid *g, int d, const double *a, int i, int j, int k)
{
    int idx[3] = {i, j, k};
    if (g->bc[d] == OG_PERIODIC) idx[d] = wrap(idx[d], ncell(g, d));
    return a[vidx(g, d, idx[0], idx[1], idx[2])];
}

/* div[c] = sum_d (a_d(c + 1/2 e_d) - a_d(c - 1/2 e_d)) / h_d; zero in solids */
void og_divergence(const og_grid *g, const double *u, const double *v, const double *w,
                   double *div)
{
    const double *vel[3] = {u, v, w};
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                double s = 0.0;
                if (!is_solid(g, i, j, k)) {
                    for (int d = 0; d < 3; d++) {
                        int hi[3] = {i, j, k};
                        hi[d] += 1;
                        s += (face_val(g, d, vel[d], hi[0], hi[1], hi[2]) -
                              face_val(g, d, vel[d], i, j, k)) / hstep(g, d);
                    }
                }
                div[cidx(g, i, j, k)] = s;
            }
}

/* Lp[c] = sum_d [a+ (p(c+e_d) - p(c)) - a- (p(c) - p(c-e_d))] / h_d^2, where a+-
 * is 1 for an active face and 0 for a wall/solid face (homogeneous Neumann). */
void og_laplacian(const og_grid *g, const double *p, double *lp)
{
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                double s = 0.0;
                if (!is_solid(g, i, j, k)) {
                    double pc = p[cidx(g, i, j, k)];
                    for (int d = 0; d < 3; d++) {
                        double h2 = hstep(g, d) * hstep(g, d);
                        int hi[3] = {i, j, k}, lo[3] = {i, j, k};
                        hi[d] += 1;
                        lo[d] -= 1;
                        if (face_active(g, d, hi[0], hi[1], hi[2]))
                            s += (pget(g, p, hi[0], hi[1], hi[2]) - pc) / h2;
                        if (face_active(g, d, i, j, k))
                            s -= (pc - pget(g, p, lo[0], lo[1], lo[2])) / h2;
                    }
                }
                lp[cidx(g, i, j, k)] = s;
            }
}

/* a_d(face) -= scale * (p(c) - p(c - e_d)) / h_d on active faces; inactive
 * faces are set to zero. */
static void sub_gradient(const og_grid *g, double scale, const double *p,
                         double *u, double *v, double *w)
{
    double *vel[3] = {u, v, w};
    for (int d = 0; d < 3; d++)
        for (int k = 0; k < npos(g, d, 2); k++)
            for (int j = 0; j < npos(g, d, 1); j++)
                for (int i = 0; i < npos(g, d, 0); i++) {
                    long id = vidx(g, d, i, j, k);
                    if (!face_active(g, d, i, j, k)) {
                        vel[d][id] = 0.0;
                        continue;
                    }
                    int lo[3] = {i, j, k};
                    lo[d] -= 1;
                    double gp = (pget(g, p, i, j, k) - pget(g, p, lo[0], lo[1], lo[2])) /
                                hstep(g, d);
                    vel[d][id] -= scale * gp;
                }
}

/* gradient of p on every face of every component (zero on inactive faces) */
void og_gradient(const og_grid *g, const double *p, double *gu, double *gv, double *gw)
{
    double *vel[3] = {gu, gv, gw};
    for (int d = 0; d < 3; d++) memset(vel[d], 0, sizeof(double) * og_count(g, d));
    sub_gradient(g, -1.0, p, gu, gv, gw);
}

/* ------------------------------------------------------------------------- */
/* gauge: mean over fluid cells                                              */
/* ------------------------------------------------------------------------- */

double og_fluid_mean(const og_grid *g, const double *x)
{
    double s = 0.0;
    long n = 0;
    for (long c = 0; c < (long)g->nx * g->ny * g->nz; c++) {
        if (g->solid && g->solid[c]) continue;
        s += x[c];
        n++;
    }
    return n ? s / (double)n : 0.0;
}

static void remove_mean(const og_grid *g, double *x)
{
    double m = og_fluid_mean(g, x);
    for (long c = 0; c < (long)g->nx * g->ny * g->nz; c++)
        x[c] = (g->solid && g->solid[c]) ? 0.0 : x[c] - m;
}

static double dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* ------------------------------------------------------------------------- */
/* the Laplacian as a table, for the iterative solver                         */
/* ------------------------------------------------------------------------- */

/* The same operator as og_laplacian, with the neighbour index and face
 * activity looked up once per solve instead of once per application.  The
 * arithmetic (order of the terms and the divisions by h^2) is the same. */
typedef struct {
    long n;
    long *nb;        /* [n][6]: neighbour cell (lo,hi) per axis, or -1 (inactive face) */
    double h2[3];
    uint8_t *solid;  /* [n] */
} og_stencil;

static void stencil_build(const og_grid *g, og_stencil *st)
{
    st->n = (long)g->nx * g->ny * g->nz;
    st->nb = malloc(sizeof(long) * 6 * st->n);
    st->solid = malloc(st->n);
    for (int d = 0; d < 3; d++) st->h2[d] = hstep(g, d) * hstep(g, d);
    for (int k = 0; k < g->nz; k++)
        for (int j = 0; j < g->ny; j++)
            for (int i = 0; i < g->nx; i++) {
                long c = cidx(g, i, j, k);
                st->solid[c] = (uint8_t)is_solid(g, i, j, k);
                for (int d = 0; d < 3; d++) {
                    int hi[3] = {i, j, k}, lo[3] = {i, j, k};
                    hi[d] += 1;
                    lo[d] -= 1;
                    for (int side = 0; side < 2; side++) {
                        int *q = side ? hi : lo;
                        int fa = side ? face_active(g, d, hi[0], hi[1], hi[2])
                                      : face_active(g, d, i, j, k);
                        long nbi = -1;
                        if (fa) {
                            int r[3] = {q[0], q[1], q[2]};
                            for (int e = 0; e < 3; e++)
                                if (g->bc[e] == OG_PERIODIC) r[e] = wrap(r[e], ncell(g, e));
                            nbi = cidx(g, r[0], r[1], r[2]);
                        }
                        st->nb[6 * c + 2 * d + side] = nbi;
                    }
                }
            }
}

static void stencil_free(og_stencil *st)
{
    free(st->nb);
    free(st->solid);
}

static void stencil_apply(const og_stencil *st, const double *p, double *lp)
{
    for (long c = 0; c < st->n; c++) {
        double s = 0.0;
        if (!st->solid[c]) {
            double pc = p[c];
            for (int d = 0; d < 3; d++) {
                long hi = st->nb[6 * c + 2 * d + 1], lo = st->nb[6 * c + 2 * d];
                if (hi >= 0) s += (p[hi] - pc) / st->h2[d];
                if (lo >= 0) s -= (pc - p[lo]) / st->h2[d];
            }
        }
        lp[c] = s;
    }
}

/* ------------------------------------------------------------------------- */
/* BiCGStab (van der Vorst 1992) for L x = b, warm start from x               */
/* ------------------------------------------------------------------------- */

/* Stops when ||b - L x||_2 (recursively updated residual) <= rtol ||b||_2.
 * The shadow residual is the initial residual; it is reset to the current
 * residual whenever rho or omega becomes exactly zero.  Returns OG_OK,
 * OG_ERR_NOT_CONVERGED after maxit iterations, or OG_ERR_NONFINITE. */
int og_bicgstab(const og_grid *g, const double *b, double *x, double rtol, int maxit,
                int *iters, double *rel_res)
{
    long n = (long)g->nx * g->ny * g->nz;
    double *r = malloc(sizeof(double) * n), *rh = malloc(sizeof(double) * n);
    double *pv = calloc(n, sizeof(double)), *vv = calloc(n, sizeof(double));
    double *s = malloc(sizeof(double) * n), *t = malloc(sizeof(double) * n);
    int status = OG_ERR_NOT_CONVERGED;
    int it = 0;
    double bnorm = sqrt(dot(n, b, b));
    double rnorm;
    og_stencil L;
    stencil_build(g, &L);

    stencil_apply(&L, x, r);
    for (long i = 0; i < n; i++) r[i] = b[i] - r[i];
    memcpy(rh, r, sizeof(double) * n);
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    rnorm = sqrt(dot(n, r, r));
    for (;;) {
        if (!isfinite(rnorm)) { status = OG_ERR_NONFINITE; break; }
        if (rnorm <= rtol * bnorm) { status = OG_OK; break; }
        if (it >= maxit) { status = OG_ERR_NOT_CONVERGED; break; }
        double rho_new = dot(n, rh, r);
        double beta;
        if (rho_new == 0.0 || omega == 0.0 || it == 0) {
            /* (re)start: shadow residual := current residual, p := r */
            if (it > 0) {
                memcpy(rh, r, sizeof(double) * n);
                rho_new = dot(n, rh, r);
            }
            for (long i = 0; i < n; i++) pv[i] = r[i];
        } else {
            beta = (rho_new / rho) * (alpha / omega);
            for (long i = 0; i < n; i++) pv[i] = r[i] + beta * (pv[i] - omega * vv[i]);
        }
        rho = rho_new;
        stencil_apply(&L, pv, vv);
        alpha = rho / dot(n, rh, vv);
        for (long i = 0; i < n; i++) s[i] = r[i] - alpha * vv[i];
        stencil_apply(&L, s, t);
        double tt = dot(n, t, t);
        omega = tt != 0.0 ? dot(n, t, s) / tt : 0.0;
        for (long i = 0; i < n; i++) {
            x[i] += alpha * pv[i] + omega * s[i];
            r[i] = s[i] - omega * t[i];
        }
        it++;
        rnorm = sqrt(dot(n, r, r));
    }
    if (iters) *iters = it;
    if (rel_res) *rel_res = bnorm > 0.0 ? rnorm / bnorm : rnorm;
    free(r); free(rh); free(pv); free(vv); free(s); free(t);
    stencil_free(&L);
    return status;
}

/* Solve L p = b for the pure-Neumann problem: b is first projected onto the
 * range of L (fluid mean removed), p is returned with zero fluid mean. */
int og_poisson(const og_grid *g, const double *b_in, double *p, double rtol, int maxit,
               int *iters, double *rel_res)
{
    long n = (long)g->nx * g->ny * g->nz;
    double *b = malloc(sizeof(double) * n);
    memcpy(b, b_in, sizeof(double) * n);
    remove_mean(g, b);
    int st = og_bicgstab(g, b, p, rtol, maxit, iters, rel_res);
    remove_mean(g, p);
    free(b);
    return st;
}

/* ------------------------------------------------------------------------- */
/* one forward-Euler Chorin-Temam step, and the projection on its own        */
/* ------------------------------------------------------------------------- */

/* u^{n+1} = F* - dt G p^{n+1},  L p^{n+1} = D F* / dt,  F* from og_predict.
 * (u, v, w, p) are updated in place; p is the warm start of the solve. */
int og_step(const og_grid *g, double *u, double *v, double *w, double *p, double dt,
            double rtol, int maxit, int *iters)
{
    long nu = og_count(g, 0), nv = og_count(g, 1), nw = og_count(g, 2);
    long n = og_count(g, 3);
    double *fu = malloc(sizeof(double) * nu), *fv = malloc(sizeof(double) * nv);
    double *fw = malloc(sizeof(double) * nw), *b = malloc(sizeof(double) * n);
    int st = og_predict(g, u, v, w, dt, fu, fv, fw);
    if (st == OG_OK) {
        og_divergence(g, fu, fv, fw, b);
        for (long c = 0; c < n; c++) b[c] /= dt;
        st = og_poisson(g, b, p, rtol, maxit, iters, NULL);
        memcpy(u, fu, sizeof(double) * nu);
        memcpy(v, fv, sizeof(double) * nv);
        memcpy(w, fw, sizeof(double) * nw);
        sub_gradient(g, dt, p, u, v, w);
    }
    free(fu); free(fv); free(fw); free(b);
    return st;
}

/* nsteps steps; iters (may be NULL) receives the Poisson iteration counts */
int og_run(const og_grid *g, double *u, double *v, double *w, double *p, double dt,
           int nsteps, double rtol, int maxit, int *iters)
{
    for (int s = 0; s < nsteps; s++) {
        int st = og_step(g, u, v, w, p, dt, rtol, maxit, iters ? iters + s : NULL);
        if (st != OG_OK) return st;
    }
    return OG_OK;
}

/* Independent states advanced by the same number of steps: the fine sweep of
 * Parareal over all time slices (each slice on its own thread when OpenMP is
 * enabled).  Pointers are arrays of nb state pointers. */
int og_run_batch(const og_grid *g, int nb, double **u, double **v, double **w, double **p,
                 double dt, int nsteps, double rtol, int maxit)
{
    int worst = OG_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < nb; b++) {
        int st = og_run(g, u[b], v[b], w[b], p[b], dt, nsteps, rtol, maxit, NULL);
        if (st != OG_OK) {
#pragma omp critical
            worst = st;
        }
    }
    return worst;
}

int og_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Projection on its own: x <- x - G phi with L phi = D x; phi is returned. */
int og_project(const og_grid *g, double *u, double *v, double *w, double *phi, double rtol,
               int maxit, int *iters)
{
    long n = og_count(g, 3);
    double *b = malloc(sizeof(double) * n);
    og_divergence(g, u, v, w, b);
    memset(phi, 0, sizeof(double) * n);
    int st = og_poisson(g, b, phi, rtol, maxit, iters, NULL);
    sub_gradient(g, 1.0, phi, u, v, w);
    free(b);
    return st;
}

/* ------------------------------------------------------------------------- */
/* discrete adjoint of the fine step (reverse mode, exact pressure solve)     */
/* ------------------------------------------------------------------------- */

/* One step is u+ = P(u + dt R(u; u_lid)) with P = I - G L^-1 D (the
 * projection, symmetric because D = -G^T on the MAC grid) and
 * R = Re^-1 lap_h u - div_h(u u) (SMART faces), both reading ghost values that
 * depend on the interior values and on the lid speed.  The adjoint of the step
 * maps lambda (= dJ/du+) to (dJ/du, dJ/du_lid):
 *   mu = P lambda;   dJ/du = mu + dt (dR/du)^T mu;   dJ/du_lid += dt (dR/du_lid)^T mu.
 * (dR/du)^T mu is formed by differentiating every stencil term of R with
 * respect to the stored values it reads and scattering; where the SMART map
 * switches branches the derivative of the branch the forward took is used,
 * and a flux with zero transporting velocity takes the derivative of its
 * left-upwind form. */

/* Where vget's value comes from: value = sign * a[idx] + lid * u_lid
 * (idx < 0: a constant, e.g. nothing stored). */
typedef struct { long idx; double sign; double lid; } og_src;

static og_src vsrc(const og_grid *g, int c, int i, int j, int k)
{
    og_src r = {-1, 0.0, 0.0};
    int idx[3] = {i, j, k};
    int out_axis = -1;
    for (int d = 0; d < 3; d++) {
        int n = npos(g, c, d);
        if (idx[d] < 0 || idx[d] >= n) {
            if (g->bc[d] == OG_PERIODIC) {
                idx[d] = wrap(idx[d], n);
            } else {
                if (out_axis >= 0) abort();
                out_axis = d;
            }
        }
    }
    if (out_axis < 0) {
        r.idx = vidx(g, c, idx[0], idx[1], idx[2]);
        r.sign = 1.0;
        return r;
    }
    int d = out_axis;
    int n = ncell(g, d);
    int side = idx[d] < 0 ? 0 : 1;
    if (c == d) {
        idx[d] = side == 0 ? -idx[d] : 2 * n - idx[d];
        r.idx = vidx(g, c, idx[0], idx[1], idx[2]);
        r.sign = -1.0;
        return r;
    }
    idx[d] = side == 0 ? -idx[d] - 1 : 2 * n - 1 - idx[d];
    r.idx = vidx(g, c, idx[0], idx[1], idx[2]);
    if (g->bc[d] == OG_SLIP) {
        r.sign = 1.0;
        return r;
    }
    r.sign = -1.0;
    r.lid = (c == 0 && d == 1 && side == 1) ? 2.0 : 0.0;
    return r;
}

/* partial derivatives of og_smart(U, C, D) with respect to U, C, D, on the
 * branch og_smart takes */
static void smart_partials(double U, double C, double D, double *dU, double *dC, double *dD)
{
    *dU = 0.0;
    *dC = 0.0;
    *dD = 0.0;
    if (D == U) { *dC = 1.0; return; }
    double ph = (C - U) / (D - U);
    if (ph < 0.0 || ph > 1.0) { *dC = 1.0; }
    else if (ph <= 1.0 / 6.0) { *dU = -2.0; *dC = 3.0; }        /* U + 3 (C - U)   */
    else if (ph <= 5.0 / 6.0) { *dU = -0.125; *dC = 0.75; *dD = 0.375; } /* QUICK */
    else { *dD = 1.0; }
}

/* flux Uf * phi through the face between b and f (bb behind b, ff in front of
 * f); derivatives with respect to Uf and the four node values */
static void smart_flux_partials(double Uf, double bb, double b, double f, double ff,
                                double *dUf, double d4[4])
{
    double dU, dC, dD;
    d4[0] = d4[1] = d4[2] = d4[3] = 0.0;
    if (Uf < 0.0) {
        /* upwind from the front: (U, C, D) = (ff, f, b) */
        *dUf = og_smart(ff, f, b);
        smart_partials(ff, f, b, &dU, &dC, &dD);
        d4[3] = Uf * dU;
        d4[2] = Uf * dC;
        d4[1] = Uf * dD;
    } else {
        /* Uf > 0, and Uf == 0 takes the same (left-upwind) form */
        *dUf = og_smart(bb, b, f);
        smart_partials(bb, b, f, &dU, &dC, &dD);
        d4[0] = Uf * dU;
        d4[1] = Uf * dC;
        d4[2] = Uf * dD;
    }
}

static void scatter(double *out[3], int c, og_src s, double w, double *dlid)
{
    if (s.idx >= 0) out[c][s.idx] += s.sign * w;
    *dlid += s.lid * w;
}

/* out = (dR/du)^T mu on every stored face (inactive faces get whatever the
 * scatter gives; callers zero them), dlid = (dR/du_lid)^T mu. */
int og_rhs_adjoint(const og_grid *g, const double *u, const double *v, const double *w,
                   const double *mu_u, const double *mu_v, const double *mu_w, double *ou,
                   double *ov, double *ow, double *dlid)
{
    if (solid_arms_unsupported(g)) return OG_ERR_ARG;
    const double *vel[3] = {u, v, w};
    const double *mu[3] = {mu_u, mu_v, mu_w};
    double *out[3] = {ou, ov, ow};
    double inv_re = g->re > 0.0 ? 1.0 / g->re : 0.0;
    for (int c = 0; c < 3; c++) memset(out[c], 0, sizeof(double) * og_count(g, c));
    *dlid = 0.0;
    for (int c = 0; c < 3; c++)
        for (int k = 0; k < npos(g, c, 2); k++)
            for (int j = 0; j < npos(g, c, 1); j++)
                for (int i = 0; i < npos(g, c, 0); i++) {
                    if (!face_active(g, c, i, j, k)) continue;
                    double m = mu[c][vidx(g, c, i, j, k)];
                    if (m == 0.0) continue;
                    int f[3] = {i, j, k};
                    for (int d = 0; d < 3; d++) {
                        double h = hstep(g, d);
                        og_src sa[5];
                        double a[5];
                        for (int q = -2; q <= 2; q++) {
                            int p3[3] = {f[0], f[1], f[2]};
                            p3[d] += q;
                            sa[q + 2] = vsrc(g, c, p3[0], p3[1], p3[2]);
                            a[q + 2] = vget(g, c, vel[c], p3[0], p3[1], p3[2]);
                        }
                        /* diffusion: Re^-1 (a3 - 2 a2 + a1) / h^2 */
                        double wd = inv_re / (h * h) * m;
                        scatter(out, c, sa[3], wd, dlid);
                        scatter(out, c, sa[2], -2.0 * wd, dlid);
                        scatter(out, c, sa[1], wd, dlid);
                        /* convection: -(Fp - Fm) / h */
                        double Up, Um;
                        og_src tp[2], tm[2];
                        int tcomp;
                        if (d == c) {
                            tcomp = c;
                            tp[0] = sa[2]; tp[1] = sa[3];
                            tm[0] = sa[1]; tm[1] = sa[2];
                            Up = 0.5 * (a[2] + a[3]);
                            Um = 0.5 * (a[1] + a[2]);
                        } else {
                            tcomp = d;
                            int q0[3] = {f[0], f[1], f[2]};
                            int q1[3] = {f[0], f[1], f[2]};
                            q0[c] = f[c] - 1;
                            q0[d] = f[d] + 1;
                            q1[d] = f[d] + 1;
                            tp[0] = vsrc(g, d, q0[0], q0[1], q0[2]);
                            tp[1] = vsrc(g, d, q1[0], q1[1], q1[2]);
                            Up = 0.5 * (vget(g, d, vel[d], q0[0], q0[1], q0[2]) +
                                        vget(g, d, vel[d], q1[0], q1[1], q1[2]));
                            q0[d] = f[d];
                            q1[d] = f[d];
                            tm[0] = vsrc(g, d, q0[0], q0[1], q0[2]);
                            tm[1] = vsrc(g, d, q1[0], q1[1], q1[2]);
                            Um = 0.5 * (vget(g, d, vel[d], q0[0], q0[1], q0[2]) +
                                        vget(g, d, vel[d], q1[0], q1[1], q1[2]));
                        }
                        double dUp, dUm, dp[4], dm[4];
                        smart_flux_partials(Up, a[1], a[2], a[3], a[4], &dUp, dp);
                        smart_flux_partials(Um, a[0], a[1], a[2], a[3], &dUm, dm);
                        double wc = -m / h;
                        /* d(Fp)/d(nodes a1..a4) and d(Fm)/d(nodes a0..a3) */
                        for (int q = 0; q < 4; q++) {
                            scatter(out, c, sa[q + 1], wc * dp[q], dlid);
                            scatter(out, c, sa[q], -wc * dm[q], dlid);
                        }
                        /* transporting velocities, each the mean of two values */
                        for (int q = 0; q < 2; q++) {
                            scatter(out, tcomp, tp[q], 0.5 * wc * dUp, dlid);
                            scatter(out, tcomp, tm[q], -0.5 * wc * dUm, dlid);
                        }
                    }
                }
    return OG_OK;
}

/* Gradient of J = 1/2 sum over active faces of component^2 * hx*hy*hz at the
 * end of nsteps fine steps from (u0, p0), with respect to every active face of
 * u0 (inactive faces get 0) and to the lid speed.  The forward states are kept
 * in memory (no checkpointing in the oracle).  p0 is only the warm start. */
int og_adjoint(const og_grid *g, const double *u0, const double *v0, const double *w0,
               const double *p0, double dt, int nsteps, double rtol, int maxit, double *J,
               double *gu, double *gv, double *gw, double *dJ_dlid)
{
    long nc[4];
    for (int c = 0; c < 4; c++) nc[c] = og_count(g, c);
    long per = nc[0] + nc[1] + nc[2];
    double *hist = malloc(sizeof(double) * per * (nsteps + 1));
    double *p = malloc(sizeof(double) * nc[3]);
    double *phi = malloc(sizeof(double) * nc[3]);
    double *mu[3], *tmp[3];
    for (int c = 0; c < 3; c++) {
        mu[c] = malloc(sizeof(double) * nc[c]);
        tmp[c] = malloc(sizeof(double) * nc[c]);
    }
    double vol = hstep(g, 0) * hstep(g, 1) * hstep(g, 2);
    int st = OG_OK;
    memcpy(hist, u0, sizeof(double) * nc[0]);
    memcpy(hist + nc[0], v0, sizeof(double) * nc[1]);
    memcpy(hist + nc[0] + nc[1], w0, sizeof(double) * nc[2]);
    memcpy(p, p0, sizeof(double) * nc[3]);
    for (int n = 0; n < nsteps && st == OG_OK; n++) {
        double *cur = hist + (long)(n + 1) * per;
        memcpy(cur, hist + (long)n * per, sizeof(double) * per);
        st = og_step(g, cur, cur + nc[0], cur + nc[0] + nc[1], p, dt, rtol, maxit, NULL);
    }
    if (st == OG_OK) {
        /* J and lambda = dJ/du^N */
        double *uN = hist + (long)nsteps * per;
        double Jv = 0.0;
        double *lam[3] = {gu, gv, gw};
        long off = 0;
        for (int c = 0; c < 3; c++) {
            for (int k = 0; k < npos(g, c, 2); k++)
                for (int j = 0; j < npos(g, c, 1); j++)
                    for (int i = 0; i < npos(g, c, 0); i++) {
                        long id = vidx(g, c, i, j, k);
                        double x = face_active(g, c, i, j, k) ? uN[off + id] : 0.0;
                        Jv += 0.5 * x * x * vol;
                        lam[c][id] = x * vol;
                    }
            off += nc[c];
        }
        *J = Jv;
        double dl = 0.0;
        for (int n = nsteps - 1; n >= 0 && st == OG_OK; n--) {
            /* mu = P lambda */
            for (int c = 0; c < 3; c++) memcpy(mu[c], lam[c], sizeof(double) * nc[c]);
            st = og_project(g, mu[0], mu[1], mu[2], phi, rtol, maxit, NULL);
            if (st != OG_OK) break;
            double *un = hist + (long)n * per;
            double dstep;
            st = og_rhs_adjoint(g, un, un + nc[0], un + nc[0] + nc[1], mu[0], mu[1], mu[2],
                                tmp[0], tmp[1], tmp[2], &dstep);
            dl += dt * dstep;
            for (int c = 0; c < 3; c++)
                for (int k = 0; k < npos(g, c, 2); k++)
                    for (int j = 0; j < npos(g, c, 1); j++)
                        for (int i = 0; i < npos(g, c, 0); i++) {
                            long id = vidx(g, c, i, j, k);
                            lam[c][id] = face_active(g, c, i, j, k)
                                             ? mu[c][id] + dt * tmp[c][id]
                                             : 0.0;
                        }
        }
        *dJ_dlid = dl;
    }
    free(hist); free(p); free(phi);
    for (int c = 0; c < 3; c++) { free(mu[c]); free(tmp[c]); }
    return st;
}
