/*
 * ns.h -- C ABI of the GB300 (sm_103a) batched projection stepper and Parareal
 * driver for the incompressible Navier-Stokes equations, after Croce, Ruprecht
 * & Krause, "Parallel-in-Space-and-Time Simulation of the Three-Dimensional,
 * Unsteady Navier-Stokes Equations for Incompressible Flow" (arXiv 1705.06149).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - A state is (u, v, w, p) on a uniform staggered (MAC) grid with nx*ny*nz
 *   cells on [0,lx]x[0,ly]x[0,lz] (Section 2), stored in DEVICE memory owned
 *   by the caller, x fastest, leading batch dimension:
 *       u [batch][nz][ny][nx+1]   v [batch][nz][ny+1][nx]
 *       w [batch][nz+1][ny][nx]   p [batch][nz][ny][nx]
 *   Along a periodic axis the normal component has n faces instead of n+1.
 *   Wall-normal boundary faces are stored and hold zero on output.
 * - Element types follow the grid's precision: NS_FP64 -> double everywhere;
 *   NS_FP32_REFINE -> float u, v, w and double p.
 * - The library owns only the workspace inside an ns_grid; it never frees or
 *   keeps caller pointers beyond a call.
 * - Calls run on the grid's CUDA stream.  Calls that iterate to a tolerance
 *   synchronise that stream to read per-slice convergence flags; all calls
 *   have returned their results to the caller's buffers when they return.
 * - No C++ exception crosses the ABI.  On a non-OK status the contents of
 *   output buffers are unspecified; ns_last_error() describes the failure.
 * - A grid object must not be used by two host threads at once.
 * - A grid belongs to the CUDA device that was current when it was created;
 *   every call (and every host thread a call starts) makes that device
 *   current for its duration and restores the caller's device on return.
 */
#ifndef NS_H
#define NS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NS_OK = 0,
    NS_ERR_ARG = 1,            /* invalid argument (null pointer, size, step...) */
    NS_ERR_CUDA = 2,           /* a CUDA runtime call failed                     */
    NS_ERR_OOM = 3,            /* workspace allocation failed                    */
    NS_ERR_NOT_CONVERGED = 4,  /* a pressure solve hit its iteration limit       */
    NS_ERR_NONFINITE = 5,      /* NaN/Inf met in a residual or a defect          */
    NS_ERR_TIMEOUT = 6         /* a bounded device-side wait gave up             */
} ns_status;

typedef enum { NS_FP64 = 0, NS_FP32_REFINE = 1 } ns_precision;

/* Boundary condition of one axis, applied at both ends.  NS_BC_WALL is the
 * no-slip wall of the cavity (Section 3); the top face y = ly additionally
 * moves with speed u_lid along +x.  NS_BC_SLIP keeps the normal component at
 * zero and the tangential derivative at zero. */
typedef enum { NS_BC_WALL = 0, NS_BC_PERIODIC = 1, NS_BC_SLIP = 2 } ns_bc;

typedef struct {
    int nx, ny, nz;          /* cells per axis, each >= 2                            */
    double lx, ly, lz;       /* box size                                             */
    double re;               /* Reynolds number of Eq. 1 (> 0)                       */
    double u_lid;            /* speed of the lid y = ly along +x                     */
    int bc[3];               /* ns_bc per axis                                       */
    const uint8_t *solid_mask; /* host, nz*ny*nx, 1 = solid cell; NULL = none; copied.
                                  Obstacles by first-order cell decomposition
                                  (Section 2): faces next to a solid hold zero, the
                                  stencil arms reflect at solid surfaces like at a
                                  no-slip wall, the pressure sees Neumann faces.
                                  The multigrid preconditioner carries the solids
                                  on its finest level only.                        */
    int precision;           /* ns_precision                                         */
    double poisson_rtol;     /* FP64: stop when ||b - L p||_2 <= rtol ||b||_2        */
    int poisson_maxit;       /* iteration limit per Krylov solve (<= 0: 20*max(n))   */
    double refine_rtol;      /* FP32_REFINE: outer FP64 relative residual target     */
    double inner_rtol;       /* FP32_REFINE: inner FP32 relative residual per outer
                                step (<= 0: 3e-4)                                    */
    int refine_maxit;        /* FP32_REFINE: outer corrections per solve before
                                NS_ERR_NOT_CONVERGED (<= 0: 40)                      */
    int batch;               /* capacity: largest batch one call may advance (>= 1)  */
    int preconditioner;      /* ns_preconditioner: BiCGStab as in Section 2 without
                                (NS_PC_NONE) or with one multigrid V-cycle as right
                                preconditioner (NS_PC_MULTIGRID; falls back to
                                NS_PC_NONE on grids it cannot coarsen far enough).
                                The levels with at most 4096 cells (FP32_REFINE;
                                512 in FP64) run in one CTA per state; the
                                environment variable NS_MG_BLOCK_CELLS, read at
                                ns_create_grid, overrides that size (>= 8).
                                Where the coarse levels split into z slabs of an
                                even number of planes, everything below the
                                finest level runs instead as one launch of a
                                thread-block cluster per state (2 to 8 CTAs; the
                                same V-cycle, results move at rounding level);
                                NS_MG_CLUSTER=0 at ns_create_grid turns that off. */
    int tile_z;              /* cells each thread marches along z in the stencil and
                                solver kernels: an even number >= 2 (clamped to nz);
                                0: 8.  Results depend on it at rounding level (it
                                fixes the order of the per-state reductions).       */
    int parareal_chunk;      /* ns_parareal_iterate: slices per chunk of the fine
                                sweep (> 0).  With the multigrid solver the chunks'
                                sweeps and coarse chains are graph launches
                                pipelined across the iterations of one call: the
                                sweep of chunk c in iteration k+1 starts once the
                                chain of iteration k has passed chunk c, and the
                                chain (on a high-priority stream) runs under the
                                sweeps; with plain BiCGStab the chain of chunk c
                                overlaps the sweep of chunk c+1 of the same
                                iteration.  0: automatic -- two chunks, pipelined,
                                when a call runs >= 2 iterations of >= 4 slices with
                                the multigrid solver (and no per-launch timing, no
                                persistent coarse solves), else one sweep.  < 0:
                                always one sweep over all slices, then the chain.
                                Results are bit-identical in every case.           */
    int predict_tile_y;      /* tile of the predictor (grids without solid cells): */
    int predict_tile_z;      /* 32 x predict_tile_y x predict_tile_z cells, one
                                thread per (x, y) column marching z; (y, z) one of
                                (4,4) (4,8) (8,2) (8,4) (8,8) (16,4), else
                                NS_ERR_ARG; (0, 0): (8, 4).  Every face takes the
                                same operands whatever the tile; results move only
                                at rounding level (the compiler may fuse products
                                into multiply-adds differently per shape).        */
    int coarse_tile_z;       /* tile_z of the batch-1 companion grid on which
                                ns_parareal_iterate evaluates the coarse
                                propagator (every G of a grid, so G_new and G_old
                                of equal inputs stay bit-identical); 0: 8.  Deep
                                marches (few CTAs) suit the pipelined schedule,
                                whose chain shares the GPU with the sweeps.       */
} ns_grid_desc;

typedef enum { NS_PC_NONE = 0, NS_PC_MULTIGRID = 1 } ns_preconditioner;

/* Caller-owned device buffers of `batch` states (1 <= batch <= grid capacity). */
typedef struct {
    void *u, *v, *w, *p;
    int batch;
} ns_state;

typedef struct ns_grid ns_grid;

/* Counters accumulated since creation (or the last ns_reset_stats). */
typedef struct {
    long long launches;         /* kernels launched by the library                   */
    long long steps;            /* state-steps taken (one state, one time step)      */
    long long solves;           /* per-state pressure solves                          */
    long long krylov_iters;     /* Krylov iterations summed over per-state solves
                                   (inner FP32 iterations in FP32_REFINE)             */
    long long refine_steps;     /* FP32_REFINE outer corrections, summed over states */
    int last_max_iters;         /* largest per-state iteration count of the last solve */
    double last_rel_residual;   /* largest relative residual of the last solve        */
} ns_stats;

/* Create a grid object: validates the description, chooses the CUDA tiling
 * and allocates the workspace for `batch` states.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  On success *out owns the
 * workspace until ns_destroy_grid.
 * Persistent solves: with NS_PERSISTENT=1 in the environment when the grid is
 * created (multigrid preconditioner, cooperative launch available), every
 * pressure solve of one state outside graph capture and outside
 * ns_step_fine_many runs as ONE cooperative kernel (one CTA per SM, grid-wide
 * barriers between the solver's phases); results agree with the default
 * launched kernels to rounding level.  Its solves are checked on the host at
 * the end of the call that issued them.  Each barrier wait is bounded by
 * NS_PERSIST_SPIN_NS nanoseconds (default 2e9); a wait that gives up ends the
 * launch and the call returns NS_ERR_TIMEOUT.  Two persistent solves must not
 * run concurrently on one GPU. */
ns_status ns_create_grid(const ns_grid_desc *desc, void *cuda_stream, ns_grid **out);
ns_status ns_destroy_grid(ns_grid *grid);
ns_status ns_set_stream(ns_grid *grid, void *cuda_stream);

/* The fine propagator F of Parareal (Section 2.1.2): nsteps forward-Euler
 * Chorin-Temam projection steps of size dt (Section 2), applied in place to
 * every state of io, all states in the same launches:
 *   F*      = u^n + dt (Re^-1 lap_h u^n - div_h(u^n u^n))   (SMART convection)
 *   L p     = D F* / dt   (L = D G, Neumann, BiCGStab, warm start p^n,
 *                          fluid mean removed from the right side and from p)
 *   u^{n+1} = F* - dt G p^{n+1}.
 * nsteps = 0 is a no-op. */
ns_status ns_step_fine(ns_grid *grid, ns_state io, double dt, int nsteps);

/* The coarse propagator G (Section 2.1.2): the same scheme with the coarse
 * step dt_coarse = N_r dt; kept separate so that F and G can be told apart in
 * traces and statistics. */
ns_status ns_step_coarse(ns_grid *grid, ns_state io, double dt_coarse, int nsteps);

/* The projection on its own (Section 2, Chorin-Temam): u <- u - G phi with
 * L phi = D u; p is left unchanged.  Used to make seeded inputs
 * divergence-free. */
ns_status ns_project(ns_grid *grid, ns_state io);

/* The predictor alone: F* of ns_step_fine for every state of `in`, written to
 * caller device buffers fu, fv, fw laid out like u, v, w (zero on inactive
 * faces).  Exposed for stage-by-stage checks. */
ns_status ns_predict(ns_grid *grid, ns_state in, double dt, void *fu, void *fv, void *fw);

/* The gauged pressure solve alone: for each of `batch` right-hand sides b
 * (double, [batch][nz][ny][nx], device), removes the fluid mean of b, solves
 * L p = b from the warm start in p (device, precision's p type = double) and
 * removes the fluid mean of p.  b is not modified.  *iters (host, may be
 * NULL) receives the largest per-state iteration count. */
ns_status ns_poisson_solve(ns_grid *grid, const double *b, double *p, int batch, int *iters);

/* Parareal (Section 2.1.2, Eq. 6) for one trajectory of n_slices slices:
 *   y_0 = u0;  iteration 0 is the serial coarse sweep y^0_{n+1} = G(y^0_n);
 *   then for k = 0..kmax-1:  all F(y^k_n) in one batched sweep, followed by the
 *   serial update y^{k+1}_{n+1} = F(y^k_n) + (G(y^{k+1}_n) - G(y^k_n)).
 * u0: batch-1 state.  slices: n_slices+1 states y_0..y_N (output; y_0 = u0).
 * Each slice spans fine_steps_per_slice steps of dt_fine (F) and
 * coarse_steps_per_slice steps of dt_fine*fine/coarse (G).  The grid's
 * capacity must be >= n_slices.  Stops after kmax iterations or once the
 * defect max_{n,field} |y^{k+1}_n - y^k_n| <= defect_tol (tol > 0).
 * resume = 0 starts from u0 (coarse sweep first); resume = 1 continues from
 * the y^k held in `slices` and the coarse values G(y^k_n) this grid stored at
 * the end of the previous call with the same slices, n_slices, steps per
 * slice and dt_fine (NS_ERR_ARG if there is none).
 * *k_done (host) receives the iterations performed, defects (host, kmax
 * entries, may be NULL) the FP64 defect of each. */
ns_status ns_parareal_iterate(ns_grid *grid, ns_state u0, ns_state slices, int n_slices,
                              int fine_steps_per_slice, int coarse_steps_per_slice,
                              double dt_fine, int kmax, double defect_tol, int resume,
                              int *k_done, double *defects);

/* Gradient of J = 1/2 sum over active faces of (component^2) h_x h_y h_z at
 * the end of nsteps fine steps (Section 2) from each state of u0, with
 * respect to every active face of u0 (inactive faces get 0) and to the lid
 * speed, by the discrete adjoint of the fine step:
 *   mu = P lambda (P = I - G L^-1 D, the projection, symmetric),
 *   lambda <- mu + dt (dR/du)^T mu,  dJ/du_lid += dt (dR/du_lid)^T mu,
 * with R = Re^-1 lap_h u - div_h(u u) (SMART faces, the branch the forward
 * took).  The forward states are recomputed from (u, p) checkpoints taken
 * every ckpt_every steps; the pressure solves are taken as exact.
 * NS_FP64 grids run everything in FP64; NS_FP32_REFINE grids run the forward
 * steps, the adjoint projections (the same FP32 inner solve with FP64-accurate
 * refinement) and the adjoint stencils in FP32, with J and dJ/du_lid summed in
 * FP64.  (dR/du)^T mu is gathered per stored value and every sum has a fixed
 * order, so repeated calls return identical bits.  Grids with solid cells are
 * rejected (NS_ERR_ARG).  u0: device state, batch B.  J, dJ_dulid: host
 * arrays of B doubles.  grad_u0: device u, v, w buffers of batch B in the
 * grid's velocity type (p unused).  Workspace (checkpoints, one segment of
 * states, the adjoint fields) is allocated for the call and freed before it
 * returns. */
ns_status ns_adjoint(ns_grid *grid, ns_state u0, double dt, int nsteps, int ckpt_every,
                     double *J, ns_state grad_u0, double *dJ_dulid);

/* The objective of ns_adjoint without the gradient: J[b] = 1/2 sum over the
 * active faces of state b of (component^2) h_x h_y h_z, for each state of
 * `state` (device, grid's precision; p unused), summed in a fixed order.  J:
 * host array of state.batch doubles.  Synchronises the grid's stream. */
ns_status ns_kinetic_energy(ns_grid *grid, ns_state state, double *J);

/* Sets the lid speed u_lid of the grid (for derivative checks in u_lid).
 * It reaches every later call, including the coarse propagator of
 * ns_parareal_iterate.  The coarse values a Parareal call stored for a
 * resume belong to the old lid and are dropped (resume = 1 then fails with
 * NS_ERR_ARG), and launches of graphs that ns_graph_create captured from
 * this grid before the change fail with NS_ERR_ARG. */
ns_status ns_set_lid_speed(ns_grid *grid, double u_lid);

ns_status ns_get_stats(const ns_grid *grid, ns_stats *out);
ns_status ns_reset_stats(ns_grid *grid);

/* Kernel kinds timed by the profiler (index into ns_profile_read's array). */
typedef enum {
    NS_K_PREDICT = 0,      /* F* = u + dt (Re^-1 lap u - div(u u))            */
    NS_K_DIVERGENCE = 1,   /* b = D F* / dt and its partial sums               */
    NS_K_SOLVE_INIT = 2,   /* start of a pressure solve (FP64 init / refine init) */
    NS_K_KRYLOV_A = 3,     /* BiCGStab phase A: p update, v = L p, (r_hat, v);
                              multigrid path: p update + finest-level smoothing */
    NS_K_KRYLOV_B = 4,     /* BiCGStab phase B: s, t = L s, (t,s), (t,t);
                              multigrid path: s + finest-level smoothing         */
    NS_K_KRYLOV_C = 5,     /* BiCGStab phase C: x, r updates, (r_hat,r), (r,r) */
    NS_K_INNER_INIT = 6,   /* FP32+refine: outer test and inner start          */
    NS_K_REFINE = 7,       /* FP32+refine: FP64 update p += e, r = b - L p     */
    NS_K_CORRECT = 8,      /* u = F* - dt G p, p - mean(p)                     */
    NS_K_PARAREAL = 9,     /* Parareal update of Eq. 6 and the defect          */
    NS_K_MG_LAP_V = 10,    /* multigrid path: v = L y, (r_hat, v)              */
    NS_K_MG_LAP_T = 11,    /* multigrid path: t = L z, (t,s), (t,t)            */
    NS_K_MG_RESTRICT0 = 12,/* multigrid: finest-level residual, restricted     */
    NS_K_MG_PROLONG0 = 13, /* multigrid: finest-level trilinear correction     */
    NS_K_MG_COARSE = 14,   /* multigrid: the grid-level kernels of the coarser levels
                              (smoothing, restriction, prolongation)              */
    NS_K_ADJOINT = 15,     /* adjoint: (dR/du)^T mu, terminal and update kernels */
    NS_K_MG_BLOCK = 16,    /* multigrid: the one-CTA levels (one CTA per state)   */
    NS_K_PERSIST = 17,     /* a whole pressure solve in one persistent cooperative
                              launch (small batches, multigrid preconditioner)    */
    NS_K_MG_CLUSTER = 18,  /* multigrid: the coarse levels on a thread-block cluster
                              per state (everything below the finest level)       */
    NS_K_KINDS = 19
} ns_kernel_kind;

typedef struct {
    double ms;             /* summed device time of the timed launches (CUDA events) */
    long long launches;    /* timed launches                                         */
    long long cell_units;  /* cells processed by them: for the Krylov phases the sum
                              over states of (iterations x cells), elsewhere
                              (states x cells) per launch; for NS_K_MG_COARSE,
                              NS_K_MG_BLOCK and NS_K_MG_CLUSTER the values (words)
                              the launches read and write by the algorithmic
                              model: 2 per cell for smoothing and for the one-CTA
                              and cluster levels' input and output, 2 + 1/8 for
                              restriction and prolongation */
} ns_kernel_time;

/* Turns per-launch timing on (on != 0) or off.  While on, every launch made by
 * a call whose batch is >= min_batch is bracketed by two CUDA events on the
 * grid's stream; times are collected at the call's synchronisation points.
 * Turning it on clears the accumulated times. */
ns_status ns_profile_enable(ns_grid *grid, int on, int min_batch);

/* Copies min(n, NS_K_KINDS) accumulated entries to out (host). */
ns_status ns_profile_read(ns_grid *grid, ns_kernel_time *out, int n);

/* Largest grid (nx*ny*nz cells) ns_poisson_solve_noalloc accepts. */
#define NS_NOALLOC_MAX_CELLS 65536

/* ns_poisson_solve without any allocation, for callers that cannot allocate
 * GPU memory when they need a solve (code running inside an allocator or
 * memory pool it does not own, frameworks that forbid cudaMalloc on their
 * hot path, processes whose memory budget is already committed).  There is
 * no counterpart in the paper: it is the same gauged FP64 solve (fluid mean
 * removed from b, BiCGStab on L p = b from the warm start in p, mean removed
 * from p) for ONE state on an nx*ny*nz grid of box lx*ly*lz with boundary
 * conditions bc[3], tolerance rtol and iteration limit maxit (<= 0:
 * 20*max(n)), with no ns_grid object.
 *   - b (device, nz*ny*nx doubles) is read only; p (device) is the warm start
 *     and the result.  cuda_stream is a cudaStream_t (NULL = default stream);
 *     the call synchronises it.  *iters (host, may be NULL) gets the count.
 *   - Scratch: one file-scope device array of about 5 MB, reserved on every
 *     GPU that loads the library until the process exits.  Grids larger than
 *     NS_NOALLOC_MAX_CELLS cells are rejected with NS_ERR_ARG.
 *   - No cudaMalloc, cudaFree or other allocating routine is called.  The
 *     first call on each device looks the array's device address up
 *     (cudaGetSymbolAddress) with that device current.
 *   - Every call polls its convergence flags into host memory and
 *     synchronises cuda_stream, so it must never be made while a stream is
 *     being captured into a CUDA graph.
 *   - Every call shares the one array: calls that overlap on the GPU (two
 *     streams, two host threads) race and give wrong results.  The array
 *     keeps the previous call's contents; the call clears what must start at
 *     zero itself.
 *   - Failures are reported by the status code only; ns_last_error() is not
 *     updated (storing a message would allocate). */
ns_status ns_poisson_solve_noalloc(int nx, int ny, int nz, double lx, double ly, double lz,
                                   const int *bc, double rtol, int maxit, const double *b,
                                   double *p, void *cuda_stream, int *iters);

/* Advances several independent grids at once: for each i < n exactly what
 * ns_step_fine(grids[i], states[i], dts[i], nsteps[i]) computes.  Each grid
 * runs on a stream of its own (ordered after, and joined back into, the
 * grid's stream) driven by a host thread of its own, so the grids' kernels
 * overlap on the GPU and a grid waiting for its convergence flags holds no
 * other.  This serves many independent cavities of different sizes and
 * Reynolds numbers (one grid per shape; Section 3's workloads as a mixed
 * batch).  The grids must be distinct.  Returns when every grid's work has
 * been issued and its solves have converged; the first failing grid (by
 * index) is reported. */
ns_status ns_step_fine_many(ns_grid *const *grids, const ns_state *states, const double *dts,
                            const int *nsteps, int n);

/* ---- CUDA graphs of fine steps ------------------------------------------
 * ns_graph_create captures, for each i < n, nsteps[i] fine steps of grids[i]
 * on states[i] with time step dts[i] -- exactly what
 * ns_step_fine(grids[i], states[i], dts[i], nsteps[i]) computes -- into one
 * CUDA graph whose n branches are independent and run concurrently.  Every
 * pressure solve iterates inside the graph: the BiCGStab iterations and the
 * FP32+refine outer corrections are conditional while nodes whose conditions
 * the solver's own decision kernels set on the device (each loop is also
 * capped at its iteration limit + 2), so a launch makes no host round trip.
 * This serves launch-bound small grids, repeated step sequences and many
 * independent cavities in one launch (one grid per shape, Section 3's
 * workloads as a mixed batch).
 *   grids    n distinct grids, each created with NS_PC_MULTIGRID on a grid it
 *            can coarsen (else NS_ERR_ARG); a grid may sit in one branch only
 *   states   n caller-owned device states; their pointers are baked into the
 *            graph, so they must stay allocated until ns_graph_destroy
 *   dts, nsteps  n time steps (> 0) and step counts (>= 1)
 * The grids' streams are synchronised once before the capture.  While a graph
 * exists, its grids may still be used directly, but never concurrently with a
 * launch of the graph.
 * ns_graph_launch enqueues one launch on cuda_stream (NULL: the legacy
 *   default stream) and returns at once.
 * ns_graph_check synchronises cuda_stream, adds the executed steps, solves,
 *   iterations and kernel launches to each grid's ns_stats, and reports a
 *   solve that failed in any launch since the last check: NS_ERR_NOT_CONVERGED
 *   (an iteration limit was reached) or NS_ERR_NONFINITE; the failure flags
 *   are then cleared.  The states hold the last launch's results.
 * ns_graph_destroy frees the graph (call it after the last launch completed). */
typedef struct ns_graph ns_graph;
ns_status ns_graph_create(ns_grid *const *grids, const ns_state *states, const double *dts,
                          const int *nsteps, int n, ns_graph **out);
ns_status ns_graph_launch(ns_graph *graph, void *cuda_stream);
ns_status ns_graph_check(ns_graph *graph, void *cuda_stream);
ns_status ns_graph_destroy(ns_graph *graph);

/* Message of the last failure on the calling host thread ("" if none). */
const char *ns_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NS_H */
