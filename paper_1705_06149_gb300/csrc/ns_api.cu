// C ABI (include/ns.h): grid objects, workspace, and the host-side drivers of
// the projection step, the pressure solves and Parareal.  All arithmetic runs
// in the kernels of ns_kernels.cuh; the host only sequences launches and reads
// the per-state convergence flags.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "ns.h"
#include "ns_adjoint.cuh"
#include "ns_mg.cuh"
#include "ns_mg_cluster.cuh"
#include "ns_persist.h"
#include "ns_pipeline.h"

using namespace nsk;

namespace {

thread_local std::string g_last_error;

ns_status fail(ns_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

#define NS_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(NS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define NS_TRY(expr)                         \
    do {                                     \
        ns_status s_ = (expr);               \
        if (s_ != NS_OK) return s_;          \
    } while (0)

constexpr int kMaxOuterDefault = 40;

// Makes `dev` the calling thread's current device for the guard's lifetime
// (host threads start on device 0; a grid's launches, copies and lazy
// allocations must all go to the device its memory lives on).
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

}  // namespace

struct ns_grid {
    ns_grid_desc d{};
    Geo geo{};
    cudaStream_t stream = nullptr;
    int device = 0;       // the CUDA device the grid's memory and streams live on
    long long gen = 0;    // bumped when a setting that captured graphs hold changes
    int cap = 0;
    bool fp32 = false;
    int maxit = 0;
    int max_outer = kMaxOuterDefault;  // FP32+refine: outer corrections per solve
    double inner_rtol = 3e-4;
    // workspace, [cap][...]
    void* fs[3] = {nullptr, nullptr, nullptr};  // F* (element type of the precision)
    double* b = nullptr;                        // right side of the pressure equation
    void* kv[8] = {};                           // Krylov vectors: x r rhat P0 P1 V0 V1 t
    double* p64[2] = {nullptr, nullptr};        // FP32+refine: FP64 pressure iterates
    // multigrid-preconditioned BiCGStab
    bool mg = false;
    MgPlan plan{};
    size_t mg_smem = 0;
    // the coarse levels on a thread-block cluster per state
    bool cl = false;
    ClPlan cplan{};
    size_t cl_smem = 0;
    void* mg_vec[3] = {};                       // Y, Z, S at level 0
    void* mg_B[MG_MAX_LEVELS] = {};             // restricted right sides, levels 1..lc
    void* mg_Y[MG_MAX_LEVELS] = {};             // level iterates, levels 1..lc
    unsigned int* counter = nullptr;            // per state: CTAs arrived
    double* p_prev = nullptr;                   // 2 p^n - p^(n-1): the next solve's warm start
    double* r64 = nullptr;                      // FP32+refine, plain solver: FP64 outer residual
    float* ffb[8] = {};                         // FP32+refine, multigrid: the float-float
                                                // iterate, residual, warm start, last p
    double* part_mg = nullptr;                  // [cap][ctas][4]
    double* part_div = nullptr;
    double* part_a = nullptr;
    double* part_b = nullptr;
    double* part_c = nullptr;
    double* part_r = nullptr;
    SliceCtl* ctl = nullptr;
    SliceCtl* h_ctl = nullptr;                  // pinned host mirror
    unsigned long long* d_defect = nullptr;
    unsigned long long* h_defect = nullptr;
    int iter_hint = 16;
    ns_stats stats{};
    // per-launch timing (ns_profile_enable)
    struct Prof {
        bool on = false;
        bool active = false;  // the current call is timed (batch >= min_batch)
        int min_batch = 1;
        int cap = 0;          // event pairs in the pool
        int n = 0;            // pairs recorded and not yet harvested
        std::vector<cudaEvent_t> ev;
        std::vector<int> kind;
        std::vector<long long> units;
        ns_kernel_time acc[NS_K_KINDS];
    } prof;
    // Parareal buffers (allocated on first use)
    void* pr_f[4] = {};
    void* pr_gold[4] = {};
    void* pr_g[4] = {};
    int pr_n = 0;
    const void* pr_slices_u = nullptr;
    bool pr_valid = false;
    // the slices and steps the stored coarse values belong to
    int pr_key_n = 0, pr_key_s = 0, pr_key_m = 0;
    double pr_key_dt = 0.0;
    // graph capture (ns_graph_create): while capturing, every launch goes to
    // `stream` (a capture stream) and the solver loops become conditional
    // while nodes whose bodies are captured on body_stream[0] / [1]
    bool capturing = false;
    cudaStream_t body_stream[2] = {nullptr, nullptr};
    std::vector<cudaGraph_t> cap_bodies;  // loop bodies of the capture in progress
    // the coarse chain's graph with programmatic dependencies between its
    // consecutive kernels (NS_CHAIN_PDL=0 in the environment at creation: off)
    bool chain_pdl = true;
    // the fine sweep's graphs: programmatic edges into the cluster V-cycle
    bool sweep_pdl = true;
    LoopCount* loopc = nullptr;
    long long cap_launches = 0;  // kernels captured so far
    // Parareal's coarse propagator: a batch-1 companion grid (this grid's
    // description, tiled for one state) on its own stream (ensure_chain)
    std::vector<uint8_t> mask_host;             // copy of the solid mask, for the companion
    ns_grid* chain = nullptr;
    cudaStream_t chain_stream = nullptr;
    std::vector<cudaEvent_t> pipe_ev;
    // the coarse chain of an iteration as one CUDA graph on the companion
    // (rebuilt when the slices, their count, the coarse steps or buffers change)
    cudaStream_t chain_cap[2] = {nullptr, nullptr};
    cudaGraph_t chain_graph = nullptr;
    cudaGraphExec_t chain_exec = nullptr;
    const void* chain_key_ys = nullptr;
    const void* chain_key_f = nullptr;
    int chain_key_n = 0, chain_key_m = 0;
    double chain_key_dt = 0.0;
    LoopCount chain_seen_lc{};
    SliceCtl chain_seen_ctl{};
    // persistent pressure solves (batch <= persist_max_batch, multigrid, not
    // while capturing): one cooperative launch per solve, checked on the host
    // only at the end of the call that issued them (or of the coarse chain)
    bool persist = false;
    int persist_grid = 0;            // CTAs of a persistent launch (one per SM)
    int persist_max_batch = 1;
    unsigned* pbar = nullptr;        // grid barrier words
    int* perr = nullptr;             // a barrier wait gave up
    long long spin_ns = 2000000000LL;
    int persist_pending = 0;         // solves issued since the last check
    int persist_batch = 0;
    bool defer = false;              // the caller checks the pending solves itself
    SliceCtl* psnap_ctl = nullptr;   // control blocks before the pending solves
    LoopCount* psnap_lc = nullptr;
    // the chain of each chunk of the chunked schedule as a graph of its own
    // the batched fine sweep of an iteration (S steps of the N slices in
    // pr_f) as one CUDA graph with device-resident solver loops (rebuilt when
    // N, S, dt or the settings change)
    cudaStream_t sweep_cap[2] = {nullptr, nullptr};
    cudaGraph_t sweep_graph = nullptr;
    cudaGraphExec_t sweep_exec = nullptr;
    int sweep_key_n = 0, sweep_key_s = 0;
    double sweep_key_dt = 0.0;
    LoopCount sweep_seen_lc{};
    std::vector<SliceCtl> sweep_seen_ctl;
    std::vector<cudaGraph_t> chunk_graph;
    std::vector<cudaGraphExec_t> chunk_exec;
    // what the chunks' chain graphs were captured for (their own key: the
    // whole-chain graph may since have been captured for other slices)
    int chunk_key = 0;
    const void* chunk_key_ys = nullptr;
    const void* chunk_key_f = nullptr;
    int chunk_key_n = 0, chunk_key_m = 0;
    double chunk_key_dt = 0.0;
    // the fine sweep of each chunk of the pipelined schedule (S steps of the
    // chunk's slices in pr_f) as a graph of its own
    std::vector<cudaGraph_t> swc_graph;
    std::vector<cudaGraphExec_t> swc_exec;
    int swc_key_chunk = 0, swc_key_n = 0, swc_key_s = 0;
    double swc_key_dt = 0.0;
    const void* swc_key_f = nullptr;
    // pinned host slots for the defects of the iterations of one call
    double* h_defects = nullptr;
    int h_defects_cap = 0;
    std::vector<void*> allocs;
};

namespace {

size_t elem_vel(const ns_grid* g) { return g->fp32 ? sizeof(float) : sizeof(double); }

ns_status dalloc(ns_grid* g, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(NS_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(bytes) +
                                    " bytes failed: " + cudaGetErrorString(e));
    }
    g->allocs.push_back(*p);
    return NS_OK;
}

void free_all(ns_grid* g) {
    for (cudaEvent_t e : g->prof.ev) cudaEventDestroy(e);
    g->prof.ev.clear();
    for (void* p : g->allocs) cudaFree(p);
    g->allocs.clear();
    if (g->h_ctl) cudaFreeHost(g->h_ctl);
    if (g->h_defect) cudaFreeHost(g->h_defect);
    if (g->h_defects) cudaFreeHost(g->h_defects);
    g->h_ctl = nullptr;
    g->h_defect = nullptr;
    g->h_defects = nullptr;
    g->h_defects_cap = 0;
}

int ceil_div(int a, int b) { return (a + b - 1) / b; }

void setup_geo(ns_grid* g) {
    Geo& G = g->geo;
    const ns_grid_desc& d = g->d;
    G.n[0] = d.nx;
    G.n[1] = d.ny;
    G.n[2] = d.nz;
    const double L[3] = {d.lx, d.ly, d.lz};
    for (int a = 0; a < 3; ++a) {
        G.bc[a] = d.bc[a];
        G.h[a] = L[a] / G.n[a];
        G.ih[a] = 1.0 / G.h[a];
        G.ih2[a] = 1.0 / (G.h[a] * G.h[a]);
    }
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a)
            G.ext[c][a] = G.n[a] + ((c == a && G.bc[a] != BC_PERIODIC) ? 1 : 0);
    for (int c = 0; c < 3; ++c)
        G.cnt[c] = (long long)G.ext[c][0] * G.ext[c][1] * G.ext[c][2];
    G.cnt[3] = (long long)G.n[0] * G.n[1] * G.n[2];
    G.inv_re = 1.0 / d.re;
    G.u_lid = d.u_lid;
    for (int a = 0; a < 3; ++a) {
        G.fih[a] = (float)G.ih[a];
        G.fih2[a] = (float)G.ih2[a];
    }
    G.finv_re = (float)G.inv_re;
    // cells per thread along z: fixed per grid (not per batch) so that every
    // state is reduced over the same CTAs whatever the batch size; an even
    // number so that the multigrid restriction pairs stay inside a CTA
    const int tz_want = d.tile_z > 0 ? std::max(2, d.tile_z & ~1) : 8;
    G.tz = std::min(tz_want, G.n[2]);
    G.bx = ceil_div(G.n[0], TX);
    G.by = ceil_div(G.n[1], TY);
    G.bz = ceil_div(G.n[2], G.tz);
    G.ctas = G.bx * G.by * G.bz;
    G.fbx = ceil_div(G.n[0] + 1, TX);
    G.fby = ceil_div(G.n[1] + 1, TY);
    G.fbz = ceil_div(G.n[2] + 1, G.tz);
    G.fctas = G.fbx * G.fby * G.fbz;
    G.n_fluid = G.n[0] * G.n[1] * G.n[2];
    const bool deflt = d.predict_tile_y == 0 && d.predict_tile_z == 0;
    G.pty = deflt ? PT_Y : d.predict_tile_y;
    G.ptz = deflt ? PT_Z : d.predict_tile_z;
}

// Face codes of the finest level with solid cells (FC_FLUID and one bit per
// face joining two fluid cells), by the same rules as the pressure operator.
std::vector<uint8_t> face_codes(const Geo& G, const uint8_t* solid) {
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
    std::vector<uint8_t> code((size_t)nx * ny * nz, 0);
    auto at = [&](int i, int j, int k) { return solid[((size_t)k * ny + j) * nx + i] == 0; };
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                if (!at(i, j, k)) continue;
                unsigned m = FC_FLUID;
                const int c[3] = {i, j, k};
                for (int a = 0; a < 3; ++a) {
                    for (int dir = 0; dir < 2; ++dir) {
                        int q[3] = {c[0], c[1], c[2]};
                        q[a] += dir ? 1 : -1;
                        if (q[a] < 0 || q[a] >= G.n[a]) {
                            if (G.bc[a] != BC_PERIODIC) continue;
                            q[a] = q[a] < 0 ? G.n[a] - 1 : 0;
                        }
                        if (at(q[0], q[1], q[2])) m |= 1u << (2 * a + dir);
                    }
                }
                code[((size_t)k * ny + j) * nx + i] = (uint8_t)m;
            }
    return code;
}

// Multigrid hierarchy: halve every size while all are even and >= 4; the
// levels from the first one with at most `block_cells` cells down run in one
// CTA per state.  Returns false when the hierarchy is not usable (the block
// levels would not fit in shared memory).
bool setup_mg(ns_grid* g, int block_cells, size_t elem, bool masked) {
    const Geo& G = g->geo;
    MgPlan& P = g->plan;
    P = MgPlan{};
    const int tz0 = G.tz;
    // every level marches tz0 cells per thread (the finest level's reduction
    // order depends on it; on the coarser levels, which reduce nothing, 2
    // cells per thread was measured slower in the batched sweep)
    auto fill = [](Lev& L, int tz) {
        L.cells = (long long)L.n[0] * L.n[1] * L.n[2];
        L.tz = std::min(std::max(tz, 2), L.n[2]);
        L.bx = ceil_div(L.n[0], TX);
        L.by = ceil_div(L.n[1], TY);
        L.bz = ceil_div(L.n[2], L.tz);
        L.ctas = L.bx * L.by * L.bz;
        L.rbx = ceil_div(L.n[0], 32);
        L.rby = ceil_div(L.n[1], 8);
        L.rctas = L.rbx * L.rby * L.bz;
    };
    Lev L0{};
    for (int a = 0; a < 3; ++a) {
        L0.n[a] = G.n[a];
        L0.bc[a] = G.bc[a];
        L0.ih2[a] = G.ih2[a];
        L0.fih2[a] = (float)G.ih2[a];
        L0.lih2[a] = (float)(G.ih2[a] - (double)L0.fih2[a]);
    }
    fill(L0, tz0);
    P.lev[0] = L0;
    P.nlev = 1;
    while (P.nlev < MG_MAX_LEVELS) {
        const Lev& L = P.lev[P.nlev - 1];
        bool ok = true;
        for (int a = 0; a < 3; ++a) ok = ok && L.n[a] % 2 == 0 && L.n[a] >= 4;
        if (!ok) break;
        Lev C{};
        for (int a = 0; a < 3; ++a) {
            C.n[a] = L.n[a] / 2;
            C.bc[a] = L.bc[a];
            C.ih2[a] = L.ih2[a] * 0.25;
            C.fih2[a] = (float)C.ih2[a];
            C.lih2[a] = (float)(C.ih2[a] - (double)C.fih2[a]);
        }
        fill(C, tz0);
        P.lev[P.nlev++] = C;
    }
    P.lc = P.nlev - 1;
    for (int m = 0; m < P.nlev; ++m)
        if (P.lev[m].cells <= block_cells) {
            P.lc = m;
            break;
        }
    if (masked) {
        // the solid cells live on the finest level only, which the one-CTA
        // block kernel does not handle
        if (P.nlev < 2) return false;
        P.lc = std::max(P.lc, 1);
    }
    size_t smem = 0;
    for (int m = P.lc; m < P.nlev; ++m) smem += 2 * (size_t)P.lev[m].cells * elem;
    g->mg_smem = smem;
    // the one-CTA levels: at most MG_BLOCK_PER_THREAD cells per thread, and
    // shared memory within 48 KB
    P.block_ok = P.lev[P.lc].cells <= MG_BLOCK_MAX_CELLS && smem <= 48 * 1024 ? 1 : 0;
    return P.block_ok != 0;
}

// Shared memory a cluster launch may take (one fixed limit for the kernel, so
// grids created later never lower it).
constexpr size_t MG_CL_MAX_SMEM = 200 * 1024;

// The cluster form of the V-cycle below the finest level (ns_mg_cluster.cuh):
// the largest cluster (8, 4 or 2 CTAs) whose clusters for `cap` states fit the
// device's SMs at one CTA each (else 2 CTAs) and that has a plan (cl_plan).
bool setup_cluster(ns_grid* g, size_t elem, int cap, int sms) {
    for (int C = MG_CL_MAX_CTAS; C >= 2; C /= 2) {
        if (C > 2 && (long long)cap * C > sms) continue;
        if (cl_plan(g->plan, C, MG_CL_THREADS, elem, MG_CL_MAX_SMEM, g->cplan, g->cl_smem)) return true;
    }
    return false;
}

// Launch configuration of the cluster kernel for `batch` states.
void cluster_config(const ns_grid* g, int batch, cudaLaunchConfig_t& cfg, cudaLaunchAttribute* at) {
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3(g->cplan.C, batch);
    cfg.blockDim = dim3(MG_CL_THREADS);
    cfg.dynamicSmemBytes = g->cl_smem;
    cfg.stream = g->stream;
    at[0] = cudaLaunchAttribute{};
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = g->cplan.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
}

// Whether the device runs the grid's cluster launch (its shared memory limit
// set, at least one cluster resident).
template <typename T>
bool cluster_ready(ns_grid* g) {
    if (cudaFuncSetAttribute(k_mg_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)MG_CL_MAX_SMEM) != cudaSuccess)
        return false;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    cluster_config(g, 1, cfg, at);
    int n = 0;
    return cudaOccupancyMaxActiveClusters(&n, k_mg_cluster<T>, &cfg) == cudaSuccess && n >= 1;
}

ns_status check_state(const ns_grid* g, const ns_state& s, const char* what) {
    if (!s.u || !s.v || !s.w || !s.p)
        return fail(NS_ERR_ARG, std::string(what) + ": null state pointer");
    if (s.batch < 1 || s.batch > g->cap)
        return fail(NS_ERR_ARG, std::string(what) + ": batch " + std::to_string(s.batch) +
                                    " outside [1, " + std::to_string(g->cap) + "]");
    return NS_OK;
}

template <typename T>
KBuf<T> kbuf(const ns_grid* g) {
    KBuf<T> k;
    k.x = (T*)g->kv[0];
    k.r = (T*)g->kv[1];
    k.rhat = (T*)g->kv[2];
    k.P[0] = (T*)g->kv[3];
    k.P[1] = (T*)g->kv[4];
    k.V[0] = (T*)g->kv[5];
    k.V[1] = (T*)g->kv[6];
    k.t = (T*)g->kv[7];
    return k;
}

dim3 block_dim() { return dim3(TX, TY, 1); }

// Accumulates the event pairs recorded so far; the stream must have been
// synchronised since the last one was recorded.
ns_status prof_harvest(ns_grid* g) {
    auto& P = g->prof;
    for (int q = 0; q < P.n; ++q) {
        float ms = 0.0f;
        NS_CUDA(cudaEventElapsedTime(&ms, P.ev[2 * q], P.ev[2 * q + 1]));
        ns_kernel_time& a = P.acc[P.kind[q]];
        a.ms += ms;
        a.launches += 1;
        a.cell_units += P.units[q];
    }
    P.n = 0;
    return NS_OK;
}

ns_status sync_stream(ns_grid* g) {
    NS_CUDA(cudaStreamSynchronize(g->stream));
    if (g->prof.n) NS_TRY(prof_harvest(g));
    return NS_OK;
}

void prof_begin(ns_grid* g, int kind, long long units) {
    auto& P = g->prof;
    if (g->capturing || !(P.on && P.active)) return;
    if (P.n == P.cap) {
        if (sync_stream(g) != NS_OK) return;
    }
    cudaEventRecord(P.ev[2 * P.n], g->stream);
    P.kind[P.n] = kind;
    P.units[P.n] = units;
}

void prof_end(ns_grid* g) {
    auto& P = g->prof;
    if (g->capturing) {
        g->cap_launches += 1;
        return;
    }
    g->stats.launches += 1;
    if (!(P.on && P.active)) return;
    cudaEventRecord(P.ev[2 * P.n + 1], g->stream);
    P.n += 1;
}

#define NS_LAUNCH(g, kind, units, ...)    \
    do {                                  \
        prof_begin((g), (kind), (units)); \
        __VA_ARGS__;                      \
        prof_end((g));                    \
    } while (0)

ns_status poll_ctl(ns_grid* g, int batch) {
    NS_CUDA(cudaMemcpyAsync(g->h_ctl, g->ctl, sizeof(SliceCtl) * batch, cudaMemcpyDeviceToHost,
                            g->stream));
    return sync_stream(g);
}

// Runs BiCGStab iterations (phases A, B, C) on every state whose status is
// ST_ITER until none is; the host polls the flags only near the expected
// iteration count, so most iterations are launched back to back.
template <typename T>
ns_status run_krylov(ns_grid* g, int batch, double rtol, int* max_iters, double* max_rel) {
    const Geo& G = g->geo;
    KBuf<T> kb = kbuf<T>(g);
    const dim3 grid(G.ctas, batch);
    const double tol2 = rtol * rtol;
    int next_poll = std::max(1, g->iter_hint - 2);
    int it = 1;
    for (;; ++it) {
        const int par = it & 1;
        NS_LAUNCH(g, NS_K_KRYLOV_A, 0,
                  k_bicg_A<T><<<grid, block_dim(), 0, g->stream>>>(G, kb, g->ctl, g->part_c,
                                                                   g->part_a, tol2, g->maxit, par));
        NS_LAUNCH(g, NS_K_KRYLOV_B, 0,
                  k_bicg_B<T><<<grid, block_dim(), 0, g->stream>>>(G, kb, g->ctl, g->part_a,
                                                                   g->part_b, par));
        NS_LAUNCH(g, NS_K_KRYLOV_C, 0,
                  k_bicg_C<T><<<grid, block_dim(), 0, g->stream>>>(G, kb, g->ctl, g->part_b,
                                                                   g->part_c, par));
        NS_CUDA(cudaGetLastError());
        if (it >= next_poll) {
            NS_TRY(poll_ctl(g, batch));
            bool any = false;
            for (int s = 0; s < batch; ++s) any |= g->h_ctl[s].status == ST_ITER;
            if (!any) break;
            if (it > g->maxit + 2) break;
            next_poll = it + std::max(2, it / 8);
        }
    }
    int mx = 0;
    double mr = 0.0;
    ns_status st = NS_OK;
    long long cell_iters = 0;
    for (int s = 0; s < batch; ++s) {
        const SliceCtl& c = g->h_ctl[s];
        if (c.status == ST_IDLE) continue;  // not part of this solve
        cell_iters += (long long)c.it_cur * G.cnt[3];
        mx = std::max(mx, c.it_cur);
        const double rel = c.bb > 0 ? std::sqrt(c.rr / c.bb) : std::sqrt(c.rr);
        mr = std::max(mr, rel);
        if (c.status == ST_NONFINITE)
            st = fail(NS_ERR_NONFINITE, "non-finite residual in the pressure solve");
        else if ((c.status == ST_MAXIT || c.status == ST_ITER) && st == NS_OK)
            st = fail(NS_ERR_NOT_CONVERGED,
                      "pressure solve reached its iteration limit (" + std::to_string(g->maxit) +
                          "), relative residual " + std::to_string(rel));
        g->stats.krylov_iters += c.it_cur;
    }
    if (g->prof.on && g->prof.active)
        for (int kind : {NS_K_KRYLOV_A, NS_K_KRYLOV_B, NS_K_KRYLOV_C})
            g->prof.acc[kind].cell_units += cell_iters;
    g->iter_hint = std::max(1, mx);
    if (max_iters) *max_iters = std::max(*max_iters, mx);
    if (max_rel) *max_rel = std::max(*max_rel, mr);
    return st;
}

template <typename T>
MgBuf<T> mgbuf(const ns_grid* g) {
    MgBuf<T> m{};
    m.x = (T*)g->kv[0];
    m.r = (T*)g->kv[1];
    m.rhat = (T*)g->kv[2];
    m.P[0] = (T*)g->kv[3];
    m.P[1] = (T*)g->kv[4];
    m.V[0] = (T*)g->kv[5];
    m.V[1] = (T*)g->kv[6];
    m.Tt = (T*)g->kv[7];
    m.Y = (T*)g->mg_vec[0];
    m.Z = (T*)g->mg_vec[1];
    m.S = (T*)g->mg_vec[2];
    for (int l = 0; l < MG_MAX_LEVELS; ++l) {
        m.B[l] = (T*)g->mg_B[l];
        m.Yl[l] = (T*)g->mg_Y[l];
    }
    m.counter = g->counter;
    return m;
}

// dt / h per axis, for the float-float correction
float3 dt_ih(const Geo& G, double dt) {
    return make_float3(float(dt * G.ih[0]), float(dt * G.ih[1]), float(dt * G.ih[2]));
}

FFBuf ffbuf(const ns_grid* g) {
    FFBuf f;
    f.p_hi = g->ffb[0];
    f.p_lo = g->ffb[1];
    f.r_hi = g->ffb[2];
    f.r_lo = g->ffb[3];
    f.w_hi = g->ffb[4];
    f.w_lo = g->ffb[5];
    f.q_hi = g->ffb[6];
    f.q_lo = g->ffb[7];
    return f;
}

// Start of an FP32+refine multigrid solve: from the FP64 pressure p_in, or
// (p_in null) from the extrapolated warm start the last correction wrote.
void launch_refine_init_ff(ns_grid* g, int batch, const double* p_in, double otol2,
                           double itol2) {
    const Lev& L0 = g->plan.lev[0];
    const dim3 grid(L0.ctas, batch), blk = block_dim();
    MgBuf<float> mb = mgbuf<float>(g);
    if (p_in)
        NS_LAUNCH(g, NS_K_SOLVE_INIT, L0.cells * batch,
                  k_mg_refine_init_ff<true><<<grid, blk, 0, g->stream>>>(
                      L0, mb, g->ctl, g->part_div, g->geo.n_fluid, g->b, p_in, ffbuf(g),
                      g->part_mg, otol2, itol2, g->maxit));
    else
        NS_LAUNCH(g, NS_K_SOLVE_INIT, L0.cells * batch,
                  k_mg_refine_init_ff<false><<<grid, blk, 0, g->stream>>>(
                      L0, mb, g->ctl, g->part_div, g->geo.n_fluid, g->b, nullptr, ffbuf(g),
                      g->part_mg, otol2, itol2, g->maxit));
}

// One application of the V-cycle to the level-0 vector the source kernel of
// the given mode writes (src, or for SRC_P the parity's one of src / src_odd),
// result in `dst`.
template <typename T, int MODE>
void mg_apply(ns_grid* g, int batch, MgBuf<T>& mb, T* src, T* src_odd, T* dst) {
    const MgPlan& P = g->plan;
    // the first level below the grid-level ones: the cluster kernel's top
    // level, else the first one-CTA level
    const int lc = g->cl ? g->cplan.J : P.lc;
    const dim3 blk = block_dim();
    const Lev& L0 = P.lev[0];
    if (lc > 0 && L0.fcode == nullptr && L0.n[0] % 2 == 0) {
        // x pairs per thread (no solid cells, even nx)
        const int pbx = ceil_div(L0.n[0], 64);
        NS_LAUNCH(g, MODE == SRC_P ? NS_K_KRYLOV_A : NS_K_KRYLOV_B, 0,
                  (k_mg_src_pair<T, MODE>
                   <<<dim3(pbx * L0.by * L0.bz, batch), blk, 0, g->stream>>>(
                       L0, mb, g->ctl, nullptr, dst, pbx)));
    } else if (lc > 0)
        NS_LAUNCH(g, MODE == SRC_P ? NS_K_KRYLOV_A : NS_K_KRYLOV_B, 0,
                  (k_mg_src<T, MODE, true><<<dim3(L0.ctas, batch), blk, 0, g->stream>>>(
                      L0, mb, g->ctl, nullptr, dst)));
    else
        NS_LAUNCH(g, MODE == SRC_P ? NS_K_KRYLOV_A : NS_K_KRYLOV_B, 0,
                  (k_mg_src<T, MODE, false><<<dim3(L0.ctas, batch), blk, 0, g->stream>>>(
                      L0, mb, g->ctl, nullptr, dst)));
    // NS_K_MG_COARSE and NS_K_MG_BLOCK count words moved (algorithmic model):
    // smoothing b -> y: 2 per cell; restriction b, y -> coarse b: 2 + 1/8;
    // prolongation y, coarse e -> y: 2 + 1/8; the one-CTA levels: the right
    // side in, the iterate out (2 per cell of the first one-CTA level)
    for (int l = 0; l < lc; ++l) {
        const T* bsrc = l == 0 ? src : mb.B[l];
        const T* bsrc_odd = l == 0 ? src_odd : nullptr;
        const T* ysrc = l == 0 ? dst : mb.Yl[l];
        const long long rwords = l == 0 ? 0 : (P.lev[l].cells * 17 / 8) * batch;
        NS_LAUNCH(g, l == 0 ? NS_K_MG_RESTRICT0 : NS_K_MG_COARSE, rwords,
                  k_mg_restrict<T><<<dim3(P.lev[l].rctas, batch), blk, 0, g->stream>>>(
                      P.lev[l], P.lev[l + 1], g->ctl, bsrc, bsrc_odd, ysrc, mb.B[l + 1]));
        if (l + 1 < lc) {
            const Lev& Ls = P.lev[l + 1];
            if (Ls.fcode == nullptr && Ls.n[0] % 2 == 0) {
                // x pairs per thread (a level that is restricted has an even nx)
                const int pbx = ceil_div(Ls.n[0], 64);
                NS_LAUNCH(g, NS_K_MG_COARSE, 2 * Ls.cells * batch,
                          (k_mg_src_pair<T, SRC_ARR>
                           <<<dim3(pbx * Ls.by * Ls.bz, batch), blk, 0, g->stream>>>(
                               Ls, mb, g->ctl, mb.B[l + 1], mb.Yl[l + 1], pbx)));
            } else {
                NS_LAUNCH(g, NS_K_MG_COARSE, 2 * Ls.cells * batch,
                          (k_mg_src<T, SRC_ARR, true>
                           <<<dim3(Ls.ctas, batch), blk, 0, g->stream>>>(
                               Ls, mb, g->ctl, mb.B[l + 1], mb.Yl[l + 1])));
            }
        }
    }
    if (g->cl) {
        // everything below the finest level: one cluster per state
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute at[1];
        cluster_config(g, batch, cfg, at);
        const T* bin = mb.B[lc];
        NS_LAUNCH(g, NS_K_MG_CLUSTER, 2 * P.lev[lc].cells * batch,
                  cudaLaunchKernelEx(&cfg, k_mg_cluster<T>, P, g->cplan, g->ctl, bin, mb.Yl[lc]));
    } else {
        T* bin = lc == 0 ? src : mb.B[lc];
        T* bin_odd = lc == 0 ? src_odd : nullptr;
        T* bout = lc == 0 ? dst : mb.Yl[lc];
        NS_LAUNCH(g, NS_K_MG_BLOCK, 2 * P.lev[lc].cells * batch,
                  k_mg_block<T><<<batch, MG_BLOCK_THREADS, g->mg_smem, g->stream>>>(
                      P, g->ctl, bin, bin_odd, bout));
    }
    for (int l = lc - 1; l >= 0; --l) {
        T* y = l == 0 ? dst : mb.Yl[l];
        const Lev& L = P.lev[l];
        const long long pwords = l == 0 ? 0 : (L.cells * 17 / 8) * batch;
        if (L.fcode == nullptr) {
            // x pairs per thread (no solid cells; nx is even on every level
            // prolonged to)
            const int pbx = ceil_div(L.n[0], 64);
            NS_LAUNCH(g, l == 0 ? NS_K_MG_PROLONG0 : NS_K_MG_COARSE, pwords,
                      k_mg_prolong_pair<T><<<dim3(pbx * L.by * L.bz, batch), blk, 0,
                                             g->stream>>>(L, P.lev[l + 1], g->ctl, y,
                                                          mb.Yl[l + 1], pbx));
        } else {
            NS_LAUNCH(g, l == 0 ? NS_K_MG_PROLONG0 : NS_K_MG_COARSE, pwords,
                      k_mg_prolong<T><<<dim3(L.ctas, batch), blk, 0, g->stream>>>(
                          L, P.lev[l + 1], g->ctl, y, mb.Yl[l + 1]));
        }
    }
}

// Preconditioned BiCGStab iterations on every state whose status is ST_ITER,
// until none is.  zero_start: the solve started from x = 0 (FP32 inner).
// One preconditioned BiCGStab iteration on every state still iterating: the
// same launch sequence for every iteration (the ping-pong parity is read from
// each state's control block), so it can also be captured as a loop body.
template <typename T>
ns_status mg_iteration(ns_grid* g, int batch, double tol2, int zero_start) {
    const Lev& L0 = g->plan.lev[0];
    MgBuf<T> mb = mgbuf<T>(g);
    const dim3 grid(L0.ctas, batch), blk = block_dim();
    // x pairs per thread where the level has no solid cells and an even nx
    const bool pair = L0.fcode == nullptr && L0.n[0] % 2 == 0;
    const int pbx = ceil_div(L0.n[0], 64);
    const int pctas = pbx * L0.by * L0.bz;
    const dim3 pgrid(pctas, batch);
    mg_apply<T, SRC_P>(g, batch, mb, mb.P[0], mb.P[1], mb.Y);
    if (pair)
        NS_LAUNCH(g, NS_K_MG_LAP_V, 0,
                  (k_mg_lapdot_pair<T, 0><<<pgrid, blk, 0, g->stream>>>(L0, mb, g->ctl,
                                                                       g->part_mg, pbx, pctas)));
    else
        NS_LAUNCH(g, NS_K_MG_LAP_V, 0,
                  k_mg_lapdot_v<T><<<grid, blk, 0, g->stream>>>(L0, mb, g->ctl, g->part_mg));
    mg_apply<T, SRC_S>(g, batch, mb, mb.S, nullptr, mb.Z);
    if (pair)
        NS_LAUNCH(g, NS_K_MG_LAP_T, 0,
                  (k_mg_lapdot_pair<T, 1><<<pgrid, blk, 0, g->stream>>>(L0, mb, g->ctl,
                                                                       g->part_mg, pbx, pctas)));
    else
        NS_LAUNCH(g, NS_K_MG_LAP_T, 0,
                  k_mg_lapdot_t<T><<<grid, blk, 0, g->stream>>>(L0, mb, g->ctl, g->part_mg));
    if (pair)
        NS_LAUNCH(g, NS_K_KRYLOV_C, 0,
                  (k_mg_update_pair<T><<<pgrid, blk, 0, g->stream>>>(
                      L0, mb, g->ctl, g->part_mg, tol2, g->maxit, zero_start, pbx, pctas)));
    else
        NS_LAUNCH(g, NS_K_KRYLOV_C, 0,
                  k_mg_update<T><<<grid, blk, 0, g->stream>>>(L0, mb, g->ctl, g->part_mg, tol2,
                                                               g->maxit, zero_start));
    NS_CUDA(cudaGetLastError());
    return NS_OK;
}

template <typename T>
ns_status run_mg(ns_grid* g, int batch, double rtol, int zero_start, int* max_iters,
                 double* max_rel) {
    const Lev& L0 = g->plan.lev[0];
    const double tol2 = rtol * rtol;
    int next_poll = std::max(1, g->iter_hint);
    for (int it = 1;; ++it) {
        NS_TRY(mg_iteration<T>(g, batch, tol2, zero_start));
        if (it >= next_poll) {
            NS_TRY(poll_ctl(g, batch));
            bool any = false;
            for (int s = 0; s < batch; ++s) any |= g->h_ctl[s].status == ST_ITER;
            if (!any) break;
            if (it > g->maxit + 2) break;
            next_poll = it + 1;
        }
    }
    int mx = 0;
    double mr = 0.0;
    ns_status st = NS_OK;
    long long cell_iters = 0;
    for (int s = 0; s < batch; ++s) {
        const SliceCtl& c = g->h_ctl[s];
        if (c.status == ST_IDLE) continue;
        cell_iters += (long long)c.it_cur * L0.cells;
        mx = std::max(mx, c.it_cur);
        const double rel = c.bb > 0 ? std::sqrt(c.rr / c.bb) : std::sqrt(c.rr);
        mr = std::max(mr, rel);
        if (c.status == ST_NONFINITE)
            st = fail(NS_ERR_NONFINITE, "non-finite residual in the pressure solve");
        else if ((c.status == ST_MAXIT || c.status == ST_ITER) && st == NS_OK)
            st = fail(NS_ERR_NOT_CONVERGED,
                      "pressure solve reached its iteration limit (" + std::to_string(g->maxit) +
                          "), relative residual " + std::to_string(rel));
        g->stats.krylov_iters += c.it_cur;
    }
    if (g->prof.on && g->prof.active) {
        // finest-level kernels: once per iteration (restrict/prolong twice)
        for (int kind : {NS_K_KRYLOV_A, NS_K_KRYLOV_B, NS_K_KRYLOV_C, NS_K_MG_LAP_V,
                         NS_K_MG_LAP_T})
            g->prof.acc[kind].cell_units += cell_iters;
        if (g->plan.lc > 0)
            for (int kind : {NS_K_MG_RESTRICT0, NS_K_MG_PROLONG0})
                g->prof.acc[kind].cell_units += 2 * cell_iters;
    }
    g->iter_hint = std::max(1, mx);
    if (max_iters) *max_iters = std::max(*max_iters, mx);
    if (max_rel) *max_rel = std::max(*max_rel, mr);
    return st;
}

// ---------------------------------------------------------------------------
// graph-resident solve: the same kernels, with the host's loops replaced by
// conditional while nodes whose conditions k_loop_cond sets on the device
// ---------------------------------------------------------------------------

ns_status capture_graph_of(cudaStream_t st, cudaGraph_t* graph, const cudaGraphNode_t** deps,
                           size_t* nd) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    NS_CUDA(cudaStreamGetCaptureInfo(st, &cs, nullptr, graph, deps, nullptr, nd));
    if (cs != cudaStreamCaptureStatusActive)
        return fail(NS_ERR_CUDA, "graph capture: stream is not capturing");
    return NS_OK;
}

ns_status make_handle(cudaStream_t st, cudaGraphConditionalHandle* h) {
    cudaGraph_t gr;
    const cudaGraphNode_t* deps;
    size_t nd;
    NS_TRY(capture_graph_of(st, &gr, &deps, &nd));
    NS_CUDA(cudaGraphConditionalHandleCreate(h, gr, 0u, 0u));
    return NS_OK;
}

ns_status loop_cond(ns_grid* g, int batch, cudaGraphConditionalHandle h, int mode, int cap) {
    k_loop_cond<<<1, 32, 0, g->stream>>>(g->ctl, batch, g->loopc, h, mode, (unsigned)cap);
    g->cap_launches += 1;
    NS_CUDA(cudaGetLastError());
    return NS_OK;
}

// Appends a while node (condition h) to the capture on g->stream and
// captures its body, launched by body() with g->stream = bst.
template <typename F>
ns_status add_while(ns_grid* g, cudaStream_t bst, cudaGraphConditionalHandle h, F&& body) {
    const cudaStream_t st = g->stream;
    cudaGraph_t gr;
    const cudaGraphNode_t* deps;
    size_t nd;
    NS_TRY(capture_graph_of(st, &gr, &deps, &nd));
    cudaGraphNodeParams prm{};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeWhile;
    prm.conditional.size = 1;
    cudaGraphNode_t node;
    NS_CUDA(cudaGraphAddNode(&node, gr, deps, nullptr, nd, &prm));
    g->cap_bodies.push_back(prm.conditional.phGraph_out[0]);
    NS_CUDA(cudaStreamBeginCaptureToGraph(bst, prm.conditional.phGraph_out[0], nullptr, nullptr,
                                          0, cudaStreamCaptureModeRelaxed));
    g->stream = bst;
    const ns_status sb = body();
    g->stream = st;
    cudaGraph_t out;
    const cudaError_t e = cudaStreamEndCapture(bst, &out);
    NS_TRY(sb);
    if (e != cudaSuccess)
        return fail(NS_ERR_CUDA, std::string("graph capture of a loop body: ") +
                                     cudaGetErrorString(e));
    NS_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1,
                                                cudaStreamSetCaptureDependencies));
    return NS_OK;
}

// Turns every plain dependency between two kernel nodes of `graph` into a
// programmatic one (the successor's CTAs may launch once every CTA of the
// predecessor passed its pdl_wait, and wait there for its completion); with
// only_into, just those into a kernel node of that function (or only_into2).
cudaError_t make_programmatic(cudaGraph_t graph, const void* only_into = nullptr,
                              const void* only_into2 = nullptr) {
    size_t n = 0;
    cudaError_t e = cudaGraphGetEdges(graph, nullptr, nullptr, nullptr, &n);
    if (e != cudaSuccess || n == 0) return e;
    std::vector<cudaGraphNode_t> from(n), to(n);
    std::vector<cudaGraphEdgeData> ed(n);
    e = cudaGraphGetEdges(graph, from.data(), to.data(), ed.data(), &n);
    if (e != cudaSuccess) return e;
    for (size_t q = 0; q < n; ++q) {
        cudaGraphNodeType tf, tt;
        if ((e = cudaGraphNodeGetType(from[q], &tf)) != cudaSuccess) return e;
        if ((e = cudaGraphNodeGetType(to[q], &tt)) != cudaSuccess) return e;
        if (tf != cudaGraphNodeTypeKernel || tt != cudaGraphNodeTypeKernel ||
            ed[q].type != cudaGraphDependencyTypeDefault || ed[q].from_port != 0)
            continue;
        if (only_into) {
            cudaKernelNodeParams kp{};
            if ((e = cudaGraphKernelNodeGetParams(to[q], &kp)) != cudaSuccess) return e;
            if (kp.func != only_into && kp.func != only_into2) continue;
        }
        if ((e = cudaGraphRemoveDependencies(graph, &from[q], &to[q], &ed[q], 1)) != cudaSuccess)
            return e;
        cudaGraphEdgeData pe{};
        pe.from_port = cudaGraphKernelNodePortProgrammatic;
        pe.type = cudaGraphDependencyTypeProgrammatic;
        if ((e = cudaGraphAddDependencies(graph, &from[q], &to[q], &pe, 1)) != cudaSuccess) {
            // put the plain dependency back: the graph stays correct
            cudaGraphAddDependencies(graph, &from[q], &to[q], &ed[q], 1);
            return e;
        }
    }
    return cudaSuccess;
}

// Captures the launches fn() issues on g->stream into an executable graph:
// the capture runs on `top`, the solver loops' bodies on `body`.  With
// `programmatic`, consecutive kernels (in the graph and in its loop bodies)
// get programmatic dependencies -- with `into_cluster_only` just the edges
// into the cluster V-cycle, whose CTAs then stage their plan while the
// restriction before them finishes; where the runtime refuses them the
// plain dependencies stay.
template <typename F>
ns_status capture_exec(ns_grid* g, cudaStream_t top, cudaStream_t body, F&& fn,
                       cudaGraph_t* graph_out, cudaGraphExec_t* exec_out,
                       bool programmatic = false, bool into_cluster_only = false) {
    *graph_out = nullptr;
    *exec_out = nullptr;
    g->cap_bodies.clear();
    NS_CUDA(cudaStreamBeginCapture(top, cudaStreamCaptureModeRelaxed));
    const cudaStream_t saved = g->stream;
    const bool prof_active = g->prof.active;
    g->stream = top;
    g->body_stream[0] = body;
    g->capturing = true;
    const ns_status st = fn();
    g->capturing = false;
    g->prof.active = prof_active;
    g->stream = saved;
    g->body_stream[0] = nullptr;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(top, &graph);
    if (st != NS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess)
        return fail(NS_ERR_CUDA, std::string("graph capture: cudaStreamEndCapture: ") +
                                     cudaGetErrorString(e));
    if (programmatic) {
        const void* k32 = into_cluster_only ? (const void*)k_mg_cluster<float> : nullptr;
        const void* k64 = into_cluster_only ? (const void*)k_mg_cluster<double> : nullptr;
        bool ok = make_programmatic(graph, k32, k64) == cudaSuccess;
        for (cudaGraph_t b : g->cap_bodies) ok = ok && make_programmatic(b, k32, k64) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
    g->cap_bodies.clear();
    cudaError_t ei = cudaGraphInstantiate(exec_out, graph, 0);
    if (ei != cudaSuccess && programmatic) {
        // the runtime refused the programmatic edges: capture again without
        cudaGetLastError();
        cudaGraphDestroy(graph);
        if (into_cluster_only)
            g->sweep_pdl = false;
        else
            g->chain_pdl = false;
        return capture_exec(g, top, body, std::forward<F>(fn), graph_out, exec_out, false);
    }
    if (ei != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(NS_ERR_CUDA, std::string("graph capture: cudaGraphInstantiate: ") +
                                     cudaGetErrorString(ei));
    }
    *graph_out = graph;
    return NS_OK;
}


// ---------------------------------------------------------------------------
// persistent solves: the whole solve in one cooperative launch (ns_persist.cu)
// ---------------------------------------------------------------------------

template <typename T>
PSolve<T> make_psolve(const ns_grid* g, int batch, const double* p_in) {
    PSolve<T> a{};
    a.plan = g->plan;
    a.mb = mgbuf<T>(g);
    if (g->fp32) a.ff = ffbuf(g);
    a.ctl = g->ctl;
    a.part_div = g->part_div;
    a.part_mg = g->part_mg;
    a.b = g->b;
    a.p_in = p_in;
    a.p_prev = g->p_prev;
    a.loopc = g->loopc;
    a.bar = g->pbar;
    a.err = g->perr;
    a.spin_ns = g->spin_ns;
    a.otol2 = g->d.refine_rtol * g->d.refine_rtol;
    a.itol2 = g->inner_rtol * g->inner_rtol;
    a.tol2 = g->d.poisson_rtol * g->d.poisson_rtol;
    a.maxit = g->maxit;
    a.max_outer = g->max_outer;
    a.n_fluid = g->geo.n_fluid;
    a.batch = batch;
    // the graph loops' caps: one body per inner iteration (+2), times the
    // outer corrections (+2) for FP32+refine
    a.cap = g->fp32 ? (unsigned)((g->maxit + 2) * (g->max_outer + 2)) : (unsigned)(g->maxit + 2);
    return a;
}

// Reads back what the pending persistent solves did: adds their solves,
// iterations and refinement steps to ns_stats and reports a solve that
// failed (sticky bits, then cleared) or a barrier wait that gave up.
ns_status persist_check(ns_grid* g) {
    if (g->persist_pending == 0) return NS_OK;
    const int B = g->persist_batch;
    g->persist_pending = 0;
    NS_TRY(sync_stream(g));
    std::vector<SliceCtl> now(B), before(B);
    int err = 0;
    NS_CUDA(cudaMemcpy(now.data(), g->ctl, sizeof(SliceCtl) * B, cudaMemcpyDeviceToHost));
    NS_CUDA(cudaMemcpy(before.data(), g->psnap_ctl, sizeof(SliceCtl) * B, cudaMemcpyDeviceToHost));
    NS_CUDA(cudaMemcpy(&err, g->perr, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        // the launch ended early: reset the barrier, the flag and the
        // per-state arrival counters for the next one
        NS_CUDA(cudaMemset(g->perr, 0, sizeof(int)));
        NS_CUDA(cudaMemset(g->pbar, 0, PERSIST_BAR_WORDS * sizeof(unsigned)));
        NS_CUDA(cudaMemset(g->counter, 0, sizeof(unsigned) * g->cap));
        return fail(NS_ERR_TIMEOUT, "persistent pressure solve: a grid-wide barrier wait gave up "
                                    "after " + std::to_string(g->spin_ns) + " ns");
    }
    ns_status result = NS_OK;
    int mx = 0;
    double mr = 0.0;
    for (int s = 0; s < B; ++s) {
        const SliceCtl& c = now[s];
        g->stats.solves += c.total_solves - before[s].total_solves;
        g->stats.krylov_iters += c.total_iters - before[s].total_iters;
        g->stats.refine_steps += c.total_outer - before[s].total_outer;
        mx = std::max(mx, c.it_cur);
        const double rel = g->fp32 ? (c.o_bb > 0 ? std::sqrt(c.o_rr / c.o_bb) : std::sqrt(c.o_rr))
                                   : (c.bb > 0 ? std::sqrt(c.rr / c.bb) : std::sqrt(c.rr));
        mr = std::max(mr, rel);
        if (c.fail && result == NS_OK)
            result = fail(c.fail & 2 ? NS_ERR_NONFINITE : NS_ERR_NOT_CONVERGED,
                          std::string("pressure solve of state ") + std::to_string(s) +
                              (c.fail & 2 ? " met a non-finite residual"
                                          : " did not reach its tolerance"));
        if (c.fail) {
            const int zero = 0;
            NS_CUDA(cudaMemcpy(&g->ctl[s].fail, &zero, sizeof(int), cudaMemcpyHostToDevice));
        }
    }
    g->stats.last_max_iters = mx;
    g->stats.last_rel_residual = mr;
    return result;
}

ns_status solve_pressure_persist(ns_grid* g, int batch, const double* p_in) {
    if (g->persist_pending && batch != g->persist_batch) NS_TRY(persist_check(g));
    if (g->persist_pending == 0) {
        // the totals before the solves, for persist_check
        NS_CUDA(cudaMemcpyAsync(g->psnap_ctl, g->ctl, sizeof(SliceCtl) * batch,
                                cudaMemcpyDeviceToDevice, g->stream));
        g->persist_batch = batch;
    }
    g->persist_pending += 1;
    const long long units = g->plan.lev[0].cells * batch;
    cudaError_t e = cudaSuccess;
    if (g->fp32) {
        const PSolve<float> a = make_psolve<float>(g, batch, p_in);
        NS_LAUNCH(g, NS_K_PERSIST, units,
                  e = persist_solve_launch(a, g->persist_grid, g->mg_smem, g->stream));
    } else {
        const PSolve<double> a = make_psolve<double>(g, batch, p_in);
        NS_LAUNCH(g, NS_K_PERSIST, units,
                  e = persist_solve_launch(a, g->persist_grid, g->mg_smem, g->stream));
    }
    if (e != cudaSuccess) {
        g->persist_pending -= 1;
        return fail(NS_ERR_CUDA, std::string("persistent pressure solve launch: ") +
                                     cudaGetErrorString(e));
    }
    return NS_OK;
}

// Checks the persistent solves a top-level call issued (unless its caller
// checks them later).
ns_status persist_settle(ns_grid* g) {
    if (g->defer || g->capturing) return NS_OK;
    return persist_check(g);
}

ns_status solve_pressure_mg_graph(ns_grid* g, int batch, const double* p_in) {
    const Lev& L0 = g->plan.lev[0];
    const dim3 grid(L0.ctas, batch), blk = block_dim();
    const int cap_inner = g->maxit + 2;
    const int cap_refine = (g->maxit + 2) * (g->max_outer + 2);
    if (!g->fp32) {
        MgBuf<double> mb = mgbuf<double>(g);
        const double tol2 = g->d.poisson_rtol * g->d.poisson_rtol;
        NS_LAUNCH(g, NS_K_SOLVE_INIT, 0,
                  k_mg_init_warm<double><<<grid, blk, 0, g->stream>>>(
                      L0, mb, g->ctl, g->part_div, g->geo.n_fluid, g->b,
                      p_in ? p_in : g->p_prev, g->part_mg, tol2, g->maxit));
        NS_CUDA(cudaGetLastError());
        cudaGraphConditionalHandle h;
        NS_TRY(make_handle(g->stream, &h));
        NS_TRY(loop_cond(g, batch, h, LC_FP64_START, cap_inner));
        return add_while(g, g->body_stream[0], h, [&]() -> ns_status {
            NS_TRY(mg_iteration<double>(g, batch, tol2, 0));
            return loop_cond(g, batch, h, LC_FP64_ITER, cap_inner);
        });
    }
    MgBuf<float> mb = mgbuf<float>(g);
    const double otol2 = g->d.refine_rtol * g->d.refine_rtol;
    const double itol2 = g->inner_rtol * g->inner_rtol;
    launch_refine_init_ff(g, batch, p_in, otol2, itol2);
    NS_CUDA(cudaGetLastError());
    // one loop: an inner iteration, then the outer correction of every state
    // whose inner solve has ended (k_loop_cond explains why this matches the
    // host's nested loops state by state)
    cudaGraphConditionalHandle h;
    NS_TRY(make_handle(g->stream, &h));
    NS_TRY(loop_cond(g, batch, h, LC_REFINE_START, cap_refine));
    return add_while(g, g->body_stream[0], h, [&]() -> ns_status {
        NS_TRY(mg_iteration<float>(g, batch, itol2, 1));
        NS_LAUNCH(g, NS_K_REFINE, 0,
                  k_mg_refine_update_ff<<<grid, blk, 0, g->stream>>>(
                      L0, mb, g->ctl, ffbuf(g), g->geo.n_fluid, g->part_mg, otol2, itol2,
                      g->maxit, g->max_outer, 1));
        NS_CUDA(cudaGetLastError());
        return loop_cond(g, batch, h, LC_REFINE_ITER, cap_refine);
    });
}

ns_status solve_pressure_mg(ns_grid* g, int batch, const double* p_in) {
    if (g->capturing) return solve_pressure_mg_graph(g, batch, p_in);
    if (g->persist && batch <= g->persist_max_batch) return solve_pressure_persist(g, batch, p_in);
    const Lev& L0 = g->plan.lev[0];
    const dim3 grid(L0.ctas, batch), blk = block_dim();
    int max_iters = 0;
    double max_rel = 0.0;
    if (!g->fp32) {
        MgBuf<double> mb = mgbuf<double>(g);
        const double tol2 = g->d.poisson_rtol * g->d.poisson_rtol;
        NS_LAUNCH(g, NS_K_SOLVE_INIT, L0.cells * batch,
                  k_mg_init_warm<double><<<grid, blk, 0, g->stream>>>(
                      L0, mb, g->ctl, g->part_div, g->geo.n_fluid, g->b,
                      p_in ? p_in : g->p_prev, g->part_mg, tol2, g->maxit));
        NS_CUDA(cudaGetLastError());
        NS_TRY(run_mg<double>(g, batch, g->d.poisson_rtol, 0, &max_iters, &max_rel));
    } else {
        MgBuf<float> mb = mgbuf<float>(g);
        const double otol2 = g->d.refine_rtol * g->d.refine_rtol;
        const double itol2 = g->inner_rtol * g->inner_rtol;
        launch_refine_init_ff(g, batch, p_in, otol2, itol2);
        NS_CUDA(cudaGetLastError());
        for (int m = 0;; ++m) {
            NS_TRY(poll_ctl(g, batch));
            bool any = false;
            for (int s = 0; s < batch; ++s) any |= g->h_ctl[s].o_status == OS_REFINE;
            if (!any || m > g->max_outer + 1) break;
            // an inner solve that stops at its iteration limit still improves
            // the outer residual; any other failure ends the solve
            ns_status st = run_mg<float>(g, batch, g->inner_rtol, 1, &max_iters, nullptr);
            if (st != NS_OK && st != NS_ERR_NOT_CONVERGED) return st;
            g_last_error.clear();
            NS_LAUNCH(g, NS_K_REFINE, L0.cells * batch,
                      k_mg_refine_update_ff<<<grid, blk, 0, g->stream>>>(
                          L0, mb, g->ctl, ffbuf(g), g->geo.n_fluid, g->part_mg, otol2, itol2,
                          g->maxit, g->max_outer, 0));
            NS_CUDA(cudaGetLastError());
        }
        for (int s = 0; s < batch; ++s) {
            const SliceCtl& c = g->h_ctl[s];
            const double rel = c.o_bb > 0 ? std::sqrt(c.o_rr / c.o_bb) : std::sqrt(c.o_rr);
            max_rel = std::max(max_rel, rel);
            g->stats.refine_steps += c.o_steps;
            if (c.o_status == OS_NONFINITE)
                return fail(NS_ERR_NONFINITE, "non-finite residual in the pressure solve");
            if (c.o_status != OS_DONE)
                return fail(NS_ERR_NOT_CONVERGED,
                            "iterative refinement did not reach refine_rtol (relative residual " +
                                std::to_string(rel) + ")");
        }
    }
    g->stats.solves += batch;
    g->stats.last_max_iters = max_iters;
    g->stats.last_rel_residual = max_rel;
    return NS_OK;
}

// Gauged pressure solve.  Input: g->b (double, [batch][cells]) and its partial
// sums in g->part_div; warm start p_in (double, device).  Result: the solution
// buffer of each state (FP64: kv x; FP32+refine: p64[p_final]) and its sum in
// SliceCtl.sx.
ns_status solve_pressure(ns_grid* g, int batch, const double* p_in) {
    if (g->mg) return solve_pressure_mg(g, batch, p_in);
    const Geo& G = g->geo;
    const dim3 grid(G.ctas, batch);
    int max_iters = 0;
    double max_rel = 0.0;
    if (!g->fp32) {
        KBuf<double> kb = kbuf<double>(g);
        NS_LAUNCH(g, NS_K_SOLVE_INIT, G.cnt[3] * batch,
                  k_bicg_init_warm<double><<<grid, block_dim(), 0, g->stream>>>(
                      G, kb, g->ctl, g->part_div, g->b, p_in, g->part_c));
        NS_CUDA(cudaGetLastError());
        NS_TRY(run_krylov<double>(g, batch, g->d.poisson_rtol, &max_iters, &max_rel));
    } else {
        KBuf<float> kb = kbuf<float>(g);
        NS_LAUNCH(g, NS_K_SOLVE_INIT, G.cnt[3] * batch,
                  k_refine_init<<<grid, block_dim(), 0, g->stream>>>(G, g->ctl, g->part_div, g->b,
                                                                     p_in, g->p64[0], kb.r,
                                                                     g->part_r));
        NS_CUDA(cudaGetLastError());
        const double tol2 = g->d.refine_rtol * g->d.refine_rtol;
        // outer corrections per state: one for every outer step that finds the
        // state still refining (SliceCtl.o_steps holds the index of the last
        // inner solve started, one less than the corrections applied)
        std::vector<int> corrections(batch, 0);
        int m = 0;
        for (;; ++m) {
            NS_LAUNCH(g, NS_K_INNER_INIT, G.cnt[3] * batch,
                      k_inner_init<<<grid, block_dim(), 0, g->stream>>>(
                          G, kb, g->ctl, g->part_r, g->part_c, tol2, m, g->max_outer));
            NS_CUDA(cudaGetLastError());
            NS_TRY(poll_ctl(g, batch));
            bool any = false;
            for (int s = 0; s < batch; ++s) {
                const bool refining = g->h_ctl[s].o_status == OS_REFINE;
                any |= refining;
                corrections[s] += refining ? 1 : 0;
            }
            if (!any) break;
            // a stalled inner solve still improves p (the outer test decides);
            // any other failure ends the solve
            ns_status st = run_krylov<float>(g, batch, g->inner_rtol, &max_iters, nullptr);
            if (st != NS_OK && st != NS_ERR_NOT_CONVERGED) return st;
            g_last_error.clear();
            NS_LAUNCH(g, NS_K_REFINE, G.cnt[3] * batch,
                      k_refine_update<<<grid, block_dim(), 0, g->stream>>>(
                          G, g->ctl, g->b, g->p64[m & 1], g->p64[(m + 1) & 1], kb.x, kb.r,
                          g->part_r));
            NS_CUDA(cudaGetLastError());
        }
        for (int s = 0; s < batch; ++s) {
            const SliceCtl& c = g->h_ctl[s];
            const double rel = c.o_bb > 0 ? std::sqrt(c.o_rr / c.o_bb) : std::sqrt(c.o_rr);
            max_rel = std::max(max_rel, rel);
            g->stats.refine_steps += corrections[s];
            if (c.o_status == OS_NONFINITE)
                return fail(NS_ERR_NONFINITE, "non-finite residual in the pressure solve");
            if (c.o_status != OS_DONE)
                return fail(NS_ERR_NOT_CONVERGED,
                            "iterative refinement did not reach refine_rtol (relative residual " +
                                std::to_string(rel) + ")");
        }
    }
    g->stats.solves += batch;
    g->stats.last_max_iters = max_iters;
    g->stats.last_rel_residual = max_rel;
    return NS_OK;
}

template <typename T, bool INCR>
void launch_predict(ns_grid* g, int batch, const T* u, const T* v, const T* w, T* fu, T* fv, T* fw,
                    double dt) {
    const Geo& G = g->geo;
    if (G.solid) {
        k_predict_masked<T, INCR><<<dim3(G.fctas, batch), block_dim(), 0, g->stream>>>(
            G, u, v, w, fu, fv, fw, dt);
        return;
    }
    auto go = [&](auto py_c, auto pz_c) {
        constexpr int PY = decltype(py_c)::value, PZ = decltype(pz_c)::value;
        const int tbx = ceil_div(G.n[0], PT_X), tby = ceil_div(G.n[1], PY),
                  tbz = ceil_div(G.n[2], PZ);
        const size_t smem = 3 * (size_t)ptile_elems<PY, PZ>() * sizeof(T);
        k_predict_tile<T, INCR, PY, PZ><<<dim3(tbx * tby * tbz, batch), PT_X * PY, smem,
                                          g->stream>>>(G, u, v, w, fu, fv, fw, dt, tbx, tby);
    };
    using I2 = std::integral_constant<int, 2>;
    using I4 = std::integral_constant<int, 4>;
    using I8 = std::integral_constant<int, 8>;
    using I16 = std::integral_constant<int, 16>;
    const int key = G.pty * 100 + G.ptz;
    switch (key) {
        case 404: go(I4{}, I4{}); break;
        case 408: go(I4{}, I8{}); break;
        case 802: go(I8{}, I2{}); break;
        case 808: go(I8{}, I8{}); break;
        case 1604: go(I16{}, I4{}); break;
        default: go(I8{}, I4{}); break;
    }
}

// Shared memory limit of the predictor instantiation the grid uses (a value
// fixed per instantiation, so grids never lower each other's).
template <typename T, bool INCR>
cudaError_t predict_smem_attr(int pty, int ptz) {
    auto set = [](auto py_c, auto pz_c) {
        constexpr int PY = decltype(py_c)::value, PZ = decltype(pz_c)::value;
        const int bytes = 3 * ptile_elems<PY, PZ>() * (int)sizeof(T);
        if (bytes <= 48 * 1024) return cudaSuccess;
        return cudaFuncSetAttribute(k_predict_tile<T, INCR, PY, PZ>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    using I2 = std::integral_constant<int, 2>;
    using I4 = std::integral_constant<int, 4>;
    using I8 = std::integral_constant<int, 8>;
    using I16 = std::integral_constant<int, 16>;
    switch (pty * 100 + ptz) {
        case 404: return set(I4{}, I4{});
        case 408: return set(I4{}, I8{});
        case 802: return set(I8{}, I2{});
        case 808: return set(I8{}, I8{});
        case 1604: return set(I16{}, I4{});
        default: return set(I8{}, I4{});
    }
}

bool predict_tile_ok(int y, int z) {
    const int key = y * 100 + z;
    return key == 404 || key == 408 || key == 802 || key == 804 || key == 808 || key == 1604;
}

// FP64 states take F* = u + dt RHS as in Section 2.  FP32 states take the
// increment form: the predictor stores dt RHS and the correction adds
// (dt RHS - dt G p) to u, so that the small increment is not lost against u
// in FP32 (F* = u + dt RHS rounded to FP32 would keep only its leading bits).  The first step of a call projects
// the whole u + dt RHS (b = D(u + dt RHS)/dt, each part differenced exactly);
// later steps start from the divergence-free result of the previous one and
// take b = D(dt RHS)/dt, which keeps FP32 rounding noise of the stored u out
// of the pressure.
template <typename T>
ns_status step_impl(ns_grid* g, const ns_state& io, double dt, int nsteps) {
    constexpr bool INCR = sizeof(T) == sizeof(float);
    const Geo& G = g->geo;
    const int B = io.batch;
    const dim3 gcell(G.ctas, B), gface(G.fctas, B);
    T* u = (T*)io.u;
    T* v = (T*)io.v;
    T* w = (T*)io.w;
    double* p = (double*)io.p;
    T* fu = (T*)g->fs[0];
    T* fv = (T*)g->fs[1];
    T* fw = (T*)g->fs[2];
    const double* x0 = g->fp32 ? g->p64[0] : (const double*)g->kv[0];
    const double* x1 = g->fp32 ? g->p64[1] : (const double*)g->kv[0];
    g->prof.active = B >= g->prof.min_batch;
    const long long cells = G.cnt[3] * B;
    for (int n = 0; n < nsteps; ++n) {
        NS_LAUNCH(g, NS_K_PREDICT, cells, launch_predict<T, INCR>(g, B, u, v, w, fu, fv, fw, dt));
        const bool with_u = INCR && n == 0;
        NS_LAUNCH(g, NS_K_DIVERGENCE, cells,
                  k_divergence<T><<<gcell, block_dim(), 0, g->stream>>>(
                      G, fu, fv, fw, with_u ? u : nullptr, with_u ? v : nullptr,
                      with_u ? w : nullptr, g->b, g->part_div, 1.0 / dt));
        NS_CUDA(cudaGetLastError());
        // multigrid path: from the second step of a call the solve starts from
        // 2 p^n - p^(n-1), which the previous correction wrote (null p_in)
        const bool extrap = g->mg && n > 0;
        NS_TRY(solve_pressure(g, B, extrap ? nullptr : p));
        const bool keep = g->mg && n + 1 < nsteps;
        if (INCR && g->mg)
            NS_LAUNCH(g, NS_K_CORRECT, cells,
                      k_correct_ff<INCR><<<gface, block_dim(), 0, g->stream>>>(
                          G, g->ctl, (const float*)fu, (const float*)fv, (const float*)fw,
                          (float*)u, (float*)v, (float*)w, ffbuf(g), p, dt_ih(G, dt),
                          keep ? 1 : 0));
        else
            NS_LAUNCH(g, NS_K_CORRECT, cells,
                      k_correct<T, INCR><<<gface, block_dim(), 0, g->stream>>>(
                          G, g->ctl, fu, fv, fw, u, v, w, x0, x1, p, dt,
                          keep ? g->p_prev : nullptr));
        NS_CUDA(cudaGetLastError());
        if (!g->capturing) g->stats.steps += B;
    }
    return persist_settle(g);
}

ns_status step_any(ns_grid* g, const ns_state& io, double dt, int nsteps, const char* what) {
    if (!g) return fail(NS_ERR_ARG, std::string(what) + ": null grid");
    const DeviceGuard dg(g->device);
    NS_TRY(check_state(g, io, what));
    if (!(dt > 0.0) || !std::isfinite(dt))
        return fail(NS_ERR_ARG, std::string(what) + ": dt must be positive and finite");
    if (nsteps < 0) return fail(NS_ERR_ARG, std::string(what) + ": nsteps < 0");
    if (nsteps == 0) return NS_OK;
    return g->fp32 ? step_impl<float>(g, io, dt, nsteps) : step_impl<double>(g, io, dt, nsteps);
}

template <typename T>
// u <- u - G phi with L phi = D u.  phi (device, [batch][cells], may be null):
// the warm start of the solve and, on return, the gauged phi; null: the solve
// starts from zero.
ns_status project_impl(ns_grid* g, const ns_state& io, double* phi = nullptr) {
    const Geo& G = g->geo;
    const int B = io.batch;
    const dim3 gcell(G.ctas, B), gface(G.fctas, B);
    T* u = (T*)io.u;
    T* v = (T*)io.v;
    T* w = (T*)io.w;
    g->prof.active = B >= g->prof.min_batch;
    NS_LAUNCH(g, NS_K_DIVERGENCE, G.cnt[3] * B,
              k_divergence<T><<<gcell, block_dim(), 0, g->stream>>>(
                  G, u, v, w, nullptr, nullptr, nullptr, g->b, g->part_div, 1.0));
    if (!phi) {
        // zero warm start: p64[1] is free scratch at this point in both precisions
        NS_CUDA(cudaMemsetAsync(g->p64[1], 0, sizeof(double) * G.cnt[3] * B, g->stream));
    }
    NS_CUDA(cudaGetLastError());
    NS_TRY(solve_pressure(g, B, phi ? phi : g->p64[1]));
    const double* x0 = g->fp32 ? g->p64[0] : (const double*)g->kv[0];
    const double* x1 = g->fp32 ? g->p64[1] : (const double*)g->kv[0];
    if (g->fp32 && g->mg)
        NS_LAUNCH(g, NS_K_CORRECT, G.cnt[3] * B,
                  k_correct_ff<false><<<gface, block_dim(), 0, g->stream>>>(
                      G, g->ctl, (const float*)u, (const float*)v, (const float*)w, (float*)u,
                      (float*)v, (float*)w, ffbuf(g), phi, dt_ih(G, 1.0), 0));
    else
        NS_LAUNCH(g, NS_K_CORRECT, G.cnt[3] * B,
                  k_correct<T, false><<<gface, block_dim(), 0, g->stream>>>(
                      G, g->ctl, u, v, w, u, v, w, x0, x1, phi, 1.0));
    NS_CUDA(cudaGetLastError());
    return persist_settle(g);
}

template <typename T>
ns_status copy_states(ns_grid* g, void* const dst[4], const void* const src[4], long long di,
                      long long si, long long count) {
    const Geo& G = g->geo;
    for (int c = 0; c < 4; ++c) {
        const size_t es = c == 3 ? sizeof(double) : sizeof(T);
        const size_t per = (size_t)G.cnt[c] * es;
        NS_CUDA(cudaMemcpyAsync((char*)dst[c] + di * per, (const char*)src[c] + si * per,
                                per * count, cudaMemcpyDeviceToDevice, g->stream));
    }
    return NS_OK;
}

template <typename T>
ns_status parareal_update(ns_grid* g, const void* const fy[4], const void* const gnew[4],
                          void* const gold[4], void* const y[4], long long fi, long long gi,
                          long long yi) {
    const Geo& G = g->geo;
    for (int c = 0; c < 4; ++c) {
        const long long n = G.cnt[c];
        const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
        if (c < 3) {
            NS_LAUNCH(g, NS_K_PARAREAL, n,
                      k_parareal_update<T><<<blocks, 256, 0, g->stream>>>(
                          n, (const T*)fy[c] + fi * n, (const T*)gnew[c] + 0,
                          (T*)gold[c] + gi * n, (T*)y[c] + yi * n, g->d_defect));
        } else {
            NS_LAUNCH(g, NS_K_PARAREAL, n,
                      k_parareal_update<double><<<blocks, 256, 0, g->stream>>>(
                          n, (const double*)fy[c] + fi * n, (const double*)gnew[c] + 0,
                          (double*)gold[c] + gi * n, (double*)y[c] + yi * n, g->d_defect));
        }
    }
    NS_CUDA(cudaGetLastError());
    return NS_OK;
}

// Kernels one preconditioned iteration launches (mg_apply twice + 3).
long long mg_iteration_launches(const ns_grid* g) {
    const int lc = g->plan.lc;
    const long long apply = 1 + lc + std::max(lc - 1, 0) + 1 + lc;
    return 2 * apply + 3;
}

// After graph launches that took `state_steps` state-steps in `step_groups`
// batched fine steps have completed on the first B states of the grid's
// workspace: adds the work the device counters show since `seen_*` to the
// grid's ns_stats (plus extra_launches kernels outside the steps) and reports
// (then clears) a failed solve.
ns_status account_graph(ns_grid* g, int B, long long state_steps, long long step_groups,
                        long long extra_launches, LoopCount& seen_lc, SliceCtl* seen_ctl,
                        const std::string& what) {
    LoopCount lc{};
    std::vector<SliceCtl> ctl(B);
    NS_CUDA(cudaMemcpy(&lc, g->loopc, sizeof(LoopCount), cudaMemcpyDeviceToHost));
    NS_CUDA(cudaMemcpy(ctl.data(), g->ctl, sizeof(SliceCtl) * B, cudaMemcpyDeviceToHost));
    const long long bodies = (long long)(lc.inner_total - seen_lc.inner_total);
    g->stats.steps += state_steps;
    // per step: predict, divergence, solve start, loop condition, correction;
    // per loop body: one iteration, (FP32) the outer correction, the condition
    g->stats.launches += step_groups * 5 +
                         bodies * (mg_iteration_launches(g) + (g->fp32 ? 2 : 1)) +
                         extra_launches;
    ns_status result = NS_OK;
    for (int s = 0; s < B; ++s) {
        const SliceCtl& a = ctl[s];
        const SliceCtl& b = seen_ctl[s];
        g->stats.solves += a.total_solves - b.total_solves;
        g->stats.krylov_iters += a.total_iters - b.total_iters;
        g->stats.refine_steps += a.total_outer - b.total_outer;
        if (a.fail && result == NS_OK)
            result = fail(a.fail & 2 ? NS_ERR_NONFINITE : NS_ERR_NOT_CONVERGED,
                          what + ": a pressure solve of state " + std::to_string(s) +
                              (a.fail & 2 ? " met a non-finite residual"
                                          : " did not reach its tolerance"));
        if (a.fail) {
            const int zero = 0;
            NS_CUDA(cudaMemcpy(&g->ctl[s].fail, &zero, sizeof(int), cudaMemcpyHostToDevice));
            ctl[s].fail = 0;
        }
        seen_ctl[s] = ctl[s];
    }
    seen_lc = lc;
    return result;
}

// The coarse propagator's grid: a batch-1 companion with this grid's
// description and its own march (coarse_tile_z, 8 cells per thread along z
// by default: few CTAs, which find room beside a concurrent sweep), on its
// own high-priority stream.  Every coarse evaluation of Parareal runs on it,
// so G_new and G_old of equal inputs are bit-identical.
ns_status ensure_chain(ns_grid* g) {
    if (g->chain) return NS_OK;
    ns_grid_desc d = g->d;
    d.batch = 1;
    d.parareal_chunk = 0;
    d.tile_z = g->d.coarse_tile_z > 0 ? g->d.coarse_tile_z : 8;
    d.solid_mask = g->mask_host.empty() ? nullptr : g->mask_host.data();
    int lo = 0, hi = 0;
    NS_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    NS_CUDA(cudaStreamCreateWithPriority(&g->chain_stream, cudaStreamNonBlocking, hi));
    NS_TRY(ns_create_grid(&d, g->chain_stream, &g->chain));
    if (g->pipe_ev.size() < 2) {
        for (int q = 0; q < 2; ++q) {
            cudaEvent_t e;
            NS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            g->pipe_ev.push_back(e);
        }
    }
    return NS_OK;
}

// Adds the companion's counters since `before` to this grid's.
void merge_chain_stats(ns_grid* g, const ns_stats& before) {
    const ns_stats& a = g->chain->stats;
    g->stats.launches += a.launches - before.launches;
    g->stats.steps += a.steps - before.steps;
    g->stats.solves += a.solves - before.solves;
    g->stats.krylov_iters += a.krylov_iters - before.krylov_iters;
    g->stats.refine_steps += a.refine_steps - before.refine_steps;
}

// Work on the companion's stream ordered after everything issued so far on
// this grid's stream (ev[0]); afterwards this grid's stream waits for it (ev[1]).
template <typename F>
ns_status on_chain(ns_grid* g, F&& fn) {
    ns_grid* h = g->chain;
    cudaEvent_t e0 = g->pipe_ev[0], e1 = g->pipe_ev[1];
    NS_CUDA(cudaEventRecord(e0, g->stream));
    NS_CUDA(cudaStreamWaitEvent(h->stream, e0, 0));
    const ns_stats before = h->stats;
    const ns_status st = fn(h);
    merge_chain_stats(g, before);
    NS_TRY(st);
    NS_CUDA(cudaEventRecord(e1, h->stream));
    NS_CUDA(cudaStreamWaitEvent(g->stream, e1, 0));
    return NS_OK;
}

// Captures (or reuses) the coarse chain of an iteration -- build() issues it
// on the companion -- as one executable graph.
template <typename F>
ns_status ensure_chain_graph(ns_grid* g, const void* ys, int N, int M, double dtc, F&& build) {
    if (g->chain_exec && g->chain_key_ys == ys && g->chain_key_f == g->pr_f[0] &&
        g->chain_key_n == N && g->chain_key_m == M && g->chain_key_dt == dtc)
        return NS_OK;
    if (g->chain_exec) cudaGraphExecDestroy(g->chain_exec);
    if (g->chain_graph) cudaGraphDestroy(g->chain_graph);
    g->chain_exec = nullptr;
    g->chain_graph = nullptr;
    for (cudaStream_t& cs : g->chain_cap)
        if (!cs) NS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    ns_grid* h = g->chain;
    NS_CUDA(cudaStreamSynchronize(h->stream));
    NS_TRY(capture_exec(h, g->chain_cap[0], g->chain_cap[1], build, &g->chain_graph,
                        &g->chain_exec, g->chain_pdl));
    g->chain_key_ys = ys;
    g->chain_key_f = g->pr_f[0];
    g->chain_key_n = N;
    g->chain_key_m = M;
    g->chain_key_dt = dtc;
    NS_CUDA(cudaMemcpy(&g->chain_seen_lc, h->loopc, sizeof(LoopCount), cudaMemcpyDeviceToHost));
    NS_CUDA(cudaMemcpy(&g->chain_seen_ctl, h->ctl, sizeof(SliceCtl), cudaMemcpyDeviceToHost));
    return NS_OK;
}

// One Parareal iteration with the fine sweep in chunks of `chunk` slices on
// this grid's stream (this thread) and the serial coarse chain with the
// update of Eq. 6 on the companion grid's stream (a second host thread).
// The chain takes slice n once the chunk holding n has been swept, and
// writes y_{n+1} only after the chunk holding n+1 has copied its inputs, so
// the chain of chunk c overlaps the sweep of chunk c+1.  Every state is
// computed by the same kernels as in the unchunked iteration (reductions do
// not depend on the batch, and the chain runs on the same companion), so the
// result is bit-identical.
template <typename T>
ns_status parareal_iteration_chunked(ns_grid* g, ns_state slices, int N, int S, int M,
                                     double dt, int chunk, double* defect) {
    const Geo& G = g->geo;
    const int C = (N + chunk - 1) / chunk;
    NS_TRY(ensure_chain(g));
    while ((int)g->pipe_ev.size() < 2 * C + 4) {
        cudaEvent_t e;
        NS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        g->pipe_ev.push_back(e);
    }
    ns_grid* h = g->chain;
    cudaEvent_t* ev_copied = g->pipe_ev.data() + 2;
    cudaEvent_t* ev_swept = g->pipe_ev.data() + 2 + C;
    cudaEvent_t ev_start = g->pipe_ev[2 * C + 2], ev_end = g->pipe_ev[2 * C + 3];
    void* ys[4] = {slices.u, slices.v, slices.w, slices.p};
    const double dtc = dt * S / M;
    // the chain's own coarse state buffer lives in this grid's pr_g
    ns_state gs{g->pr_g[0], g->pr_g[1], g->pr_g[2], g->pr_g[3], 1};
    NS_CUDA(cudaEventRecord(ev_start, g->stream));
    const ns_stats chain0 = h->stats;

    std::mutex mu;
    std::condition_variable cv;
    int copied = -1, swept = -1;  // last chunk whose event is recorded
    bool abort = false;
    ns_status st_chain = NS_OK;
    std::string err_chain;
    auto wait_for = [&](const int& what, int c) {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return what >= c || abort; });
        return !abort;
    };
    auto post = [&](int& what, int c) {
        {
            std::lock_guard<std::mutex> lk(mu);
            what = c;
        }
        cv.notify_all();
    };
    std::thread chain_thread([&]() {
        // a new host thread starts on device 0
        const DeviceGuard dg(g->device);
        auto run = [&]() -> ns_status {
            NS_CUDA(cudaStreamWaitEvent(h->stream, ev_start, 0));
            NS_CUDA(cudaMemsetAsync(h->d_defect, 0, sizeof(unsigned long long), h->stream));
            for (int c = 0; c < C; ++c) {
                if (!wait_for(swept, c)) return NS_OK;
                NS_CUDA(cudaStreamWaitEvent(h->stream, ev_swept[c], 0));
                if (c + 1 < C) {
                    if (!wait_for(copied, c + 1)) return NS_OK;
                    NS_CUDA(cudaStreamWaitEvent(h->stream, ev_copied[c + 1], 0));
                }
                const int n1 = std::min(N, (c + 1) * chunk);
                for (int n = c * chunk; n < n1; ++n) {
                    NS_TRY(copy_states<T>(h, g->pr_g, ys, 0, n, 1));
                    NS_TRY(step_impl<T>(h, gs, dtc, M));
                    NS_TRY(parareal_update<T>(h, g->pr_f, g->pr_g, g->pr_gold, ys, n, n, n + 1));
                }
            }
            NS_CUDA(cudaMemcpyAsync(h->h_defect, h->d_defect, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, h->stream));
            NS_CUDA(cudaEventRecord(ev_end, h->stream));
            return sync_stream(h);
        };
        st_chain = run();
        if (st_chain != NS_OK) {
            err_chain = g_last_error;
            std::lock_guard<std::mutex> lk(mu);
            abort = true;
        }
        cv.notify_all();
    });
    ns_status st = NS_OK;
    for (int c = 0; c < C && st == NS_OK; ++c) {
        const int n0 = c * chunk, m = std::min(N, n0 + chunk) - n0;
        {
            std::lock_guard<std::mutex> lk(mu);
            if (abort) break;
        }
        st = copy_states<T>(g, g->pr_f, ys, n0, n0, m);
        if (st == NS_OK && cudaEventRecord(ev_copied[c], g->stream) != cudaSuccess)
            st = fail(NS_ERR_CUDA, "chunked Parareal: event record failed");
        if (st != NS_OK) break;
        post(copied, c);
        ns_state fb{(char*)g->pr_f[0] + (size_t)n0 * G.cnt[0] * sizeof(T),
                    (char*)g->pr_f[1] + (size_t)n0 * G.cnt[1] * sizeof(T),
                    (char*)g->pr_f[2] + (size_t)n0 * G.cnt[2] * sizeof(T),
                    (char*)g->pr_f[3] + (size_t)n0 * G.cnt[3] * sizeof(double), m};
        st = step_impl<T>(g, fb, dt, S);
        if (st == NS_OK && cudaEventRecord(ev_swept[c], g->stream) != cudaSuccess)
            st = fail(NS_ERR_CUDA, "chunked Parareal: event record failed");
        if (st != NS_OK) break;
        post(swept, c);
    }
    if (st != NS_OK) {
        std::lock_guard<std::mutex> lk(mu);
        abort = true;
    }
    cv.notify_all();
    const std::string err_fine = g_last_error;
    chain_thread.join();
    // the slices are written by the chain: later work on this stream waits for it
    if (st == NS_OK && st_chain == NS_OK) {
        NS_CUDA(cudaStreamWaitEvent(g->stream, ev_end, 0));
        NS_TRY(sync_stream(g));
    } else {
        cudaStreamSynchronize(h->stream);
        cudaStreamSynchronize(g->stream);
    }
    // the chain's counters count as this grid's
    merge_chain_stats(g, chain0);
    if (st != NS_OK) return fail(st, err_fine);
    if (st_chain != NS_OK) return fail(st_chain, err_chain);
    std::memcpy(defect, h->h_defect, sizeof(double));
    return NS_OK;
}

// Drops the graphs of the whole sweep and of the chunks' sweeps (they share
// the capture streams and the accounting baseline).
void drop_sweep_graph(ns_grid* g) {
    if (g->sweep_exec) cudaGraphExecDestroy(g->sweep_exec);
    if (g->sweep_graph) cudaGraphDestroy(g->sweep_graph);
    g->sweep_exec = nullptr;
    g->sweep_graph = nullptr;
    for (cudaGraphExec_t e : g->swc_exec) cudaGraphExecDestroy(e);
    for (cudaGraph_t c : g->swc_graph) cudaGraphDestroy(c);
    g->swc_exec.clear();
    g->swc_graph.clear();
    g->swc_key_chunk = 0;
}

// The fine sweep F(y^k_n) of all N slices (S steps of dt, in place in pr_f)
// as one graph launch: captured on first use, then replayed; its solver
// loops are conditional while nodes, so no solve waits for the host.  The
// work is accounted (and failed solves reported) after the iteration's
// synchronisation by sweep_account.
template <typename T>
ns_status sweep_launch(ns_grid* g, int N, int S, double dt) {
    if (!(g->sweep_exec && g->sweep_key_n == N && g->sweep_key_s == S && g->sweep_key_dt == dt)) {
        drop_sweep_graph(g);
        for (cudaStream_t& cs : g->sweep_cap)
            if (!cs) NS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        NS_TRY(sync_stream(g));
        ns_state fb{g->pr_f[0], g->pr_f[1], g->pr_f[2], g->pr_f[3], N};
        NS_TRY(capture_exec(g, g->sweep_cap[0], g->sweep_cap[1],
                            [&]() -> ns_status { return step_impl<T>(g, fb, dt, S); },
                            &g->sweep_graph, &g->sweep_exec, g->sweep_pdl, true));
        g->sweep_key_n = N;
        g->sweep_key_s = S;
        g->sweep_key_dt = dt;
        g->sweep_seen_ctl.assign(N, SliceCtl{});
        NS_CUDA(cudaMemcpy(&g->sweep_seen_lc, g->loopc, sizeof(LoopCount),
                           cudaMemcpyDeviceToHost));
        NS_CUDA(cudaMemcpy(g->sweep_seen_ctl.data(), g->ctl, sizeof(SliceCtl) * N,
                           cudaMemcpyDeviceToHost));
    }
    NS_CUDA(cudaGraphLaunch(g->sweep_exec, g->stream));
    return NS_OK;
}

// The chain of each chunk of `chunk` slices (copy of y_n, M coarse steps, the
// update of Eq. 6 for every slice of the chunk) as a graph of its own on the
// companion, captured on first use.
template <typename T>
ns_status ensure_chunk_chains(ns_grid* g, ns_state slices, int N, int M, double dtc,
                              int chunk) {
    const int C = (N + chunk - 1) / chunk;
    ns_grid* h = g->chain;
    void* ys[4] = {slices.u, slices.v, slices.w, slices.p};
    ns_state gs{g->pr_g[0], g->pr_g[1], g->pr_g[2], g->pr_g[3], 1};
    if ((int)g->chunk_exec.size() == C && g->chunk_key == chunk && g->chunk_key_ys == ys[0] &&
        g->chunk_key_f == g->pr_f[0] && g->chunk_key_n == N && g->chunk_key_m == M &&
        g->chunk_key_dt == dtc)
        return NS_OK;
    for (cudaGraphExec_t e : g->chunk_exec) cudaGraphExecDestroy(e);
    for (cudaGraph_t c : g->chunk_graph) cudaGraphDestroy(c);
    g->chunk_exec.clear();
    g->chunk_graph.clear();
    g->chunk_key = 0;
    for (cudaStream_t& cs : g->chain_cap)
        if (!cs) NS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    NS_CUDA(cudaStreamSynchronize(h->stream));
    for (int c = 0; c < C; ++c) {
        cudaGraph_t gr;
        cudaGraphExec_t ex;
        const int n1 = std::min(N, (c + 1) * chunk);
        NS_TRY(capture_exec(
            h, g->chain_cap[0], g->chain_cap[1],
            [&]() -> ns_status {
                for (int n = c * chunk; n < n1; ++n) {
                    NS_TRY(copy_states<T>(h, g->pr_g, ys, 0, n, 1));
                    NS_TRY(step_impl<T>(h, gs, dtc, M));
                    NS_TRY(parareal_update<T>(h, g->pr_f, g->pr_g, g->pr_gold, ys, n, n, n + 1));
                }
                return NS_OK;
            },
            &gr, &ex, g->chain_pdl));
        g->chunk_graph.push_back(gr);
        g->chunk_exec.push_back(ex);
    }
    g->chunk_key = chunk;
    g->chunk_key_ys = ys[0];
    g->chunk_key_f = g->pr_f[0];
    g->chunk_key_n = N;
    g->chunk_key_m = M;
    g->chunk_key_dt = dtc;
    NS_CUDA(cudaMemcpy(&g->chain_seen_lc, h->loopc, sizeof(LoopCount), cudaMemcpyDeviceToHost));
    NS_CUDA(cudaMemcpy(&g->chain_seen_ctl, h->ctl, sizeof(SliceCtl), cudaMemcpyDeviceToHost));
    return NS_OK;
}

// The fine sweep of each chunk (S steps of dt of the chunk's slices, in
// place in pr_f) as a graph of its own, captured on first use.  Every chunk
// uses the first states of this grid's workspace, so the chunks' sweeps run
// one after another on this grid's stream.
template <typename T>
ns_status ensure_chunk_sweeps(ns_grid* g, int N, int S, double dt, int chunk) {
    const Geo& G = g->geo;
    const int C = (N + chunk - 1) / chunk;
    if ((int)g->swc_exec.size() == C && g->swc_key_chunk == chunk && g->swc_key_n == N &&
        g->swc_key_s == S && g->swc_key_dt == dt && g->swc_key_f == g->pr_f[0])
        return NS_OK;
    drop_sweep_graph(g);
    for (cudaStream_t& cs : g->sweep_cap)
        if (!cs) NS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    NS_TRY(sync_stream(g));
    for (int c = 0; c < C; ++c) {
        const int n0 = c * chunk, m = std::min(N, n0 + chunk) - n0;
        ns_state fb{(char*)g->pr_f[0] + (size_t)n0 * G.cnt[0] * sizeof(T),
                    (char*)g->pr_f[1] + (size_t)n0 * G.cnt[1] * sizeof(T),
                    (char*)g->pr_f[2] + (size_t)n0 * G.cnt[2] * sizeof(T),
                    (char*)g->pr_f[3] + (size_t)n0 * G.cnt[3] * sizeof(double), m};
        cudaGraph_t gr;
        cudaGraphExec_t ex;
        NS_TRY(capture_exec(g, g->sweep_cap[0], g->sweep_cap[1],
                            [&]() -> ns_status { return step_impl<T>(g, fb, dt, S); }, &gr,
                            &ex, g->sweep_pdl, true));
        g->swc_graph.push_back(gr);
        g->swc_exec.push_back(ex);
    }
    g->swc_key_chunk = chunk;
    g->swc_key_n = N;
    g->swc_key_s = S;
    g->swc_key_dt = dt;
    g->swc_key_f = g->pr_f[0];
    g->sweep_seen_ctl.assign(g->cap, SliceCtl{});
    NS_CUDA(cudaMemcpy(&g->sweep_seen_lc, g->loopc, sizeof(LoopCount), cudaMemcpyDeviceToHost));
    NS_CUDA(cudaMemcpy(g->sweep_seen_ctl.data(), g->ctl, sizeof(SliceCtl) * g->cap,
                       cudaMemcpyDeviceToHost));
    return NS_OK;
}

// Up to kmax Parareal iterations with the fine sweep in chunks of `chunk`
// slices, pipelined across iterations: the issue order of pipeline_issue
// (ns_pipeline.h), whose primitives are here the chunks' sweep graphs on this
// grid's stream, their chain graphs on the companion's high-priority stream,
// the copies of y into the F buffers, and one event per (kind, chunk).  The
// sweep of chunk 0 of the next iteration starts as soon as the chain has
// passed chunk 0, so the serial chain runs under the sweeps.  Every state is
// computed by the same kernels in the same order as in the unpipelined
// iteration (a slice's reductions do not depend on the batch), so results
// are bit-identical.  The work and any failed solve are read from the device
// counters after the call.
template <typename T>
ns_status parareal_pipelined(ns_grid* g, ns_state slices, int N, int S, int M, double dt,
                             int chunk, int kmax, double tol, int* k_out, double* defects) {
    const int C = (N + chunk - 1) / chunk;
    ns_grid* h = g->chain;
    void* ys[4] = {slices.u, slices.v, slices.w, slices.p};
    const double dtc = dt * S / M;
    NS_TRY(ensure_chunk_chains<T>(g, slices, N, M, dtc, chunk));
    NS_TRY(ensure_chunk_sweeps<T>(g, N, S, dt, chunk));
    while ((int)g->pipe_ev.size() < 2 + 3 * C + 2) {
        cudaEvent_t e;
        NS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        g->pipe_ev.push_back(e);
    }
    if (g->h_defects_cap < kmax) {
        if (g->h_defects) cudaFreeHost(g->h_defects);
        g->h_defects = nullptr;
        g->h_defects_cap = 0;
        NS_CUDA(cudaMallocHost((void**)&g->h_defects, sizeof(double) * kmax));
        g->h_defects_cap = kmax;
    }
    cudaEvent_t* ev = g->pipe_ev.data() + 2;  // [kind][chunk]: copied, swept, chained
    cudaEvent_t ev_start = ev[3 * C];  // ev[3 C + 1]: the last defect copied
    const ns_stats chain0 = h->stats;
    long long swept_states = 0, sweeps = 0;
    ns_status st_issue = NS_OK;
    // the primitives of pipeline_issue on this grid's and the companion's streams
    struct Ops {
        ns_grid *g, *h;
        cudaEvent_t* ev;
        int C, N, chunk;
        double tol;
        void* const* ys;
        long long *swept_states, *sweeps;
        ns_status* st;
        cudaStream_t stream(int s) const { return s == PS_SWEEP ? g->stream : h->stream; }
        bool ok(cudaError_t e, const char* what) {
            if (e == cudaSuccess) return true;
            *st = fail(NS_ERR_CUDA, std::string("pipelined Parareal: ") + what + ": " +
                                        cudaGetErrorString(e));
            return false;
        }
        bool wait(int s, int kind, int c) {
            return ok(cudaStreamWaitEvent(stream(s), ev[kind * C + c], 0), "event wait");
        }
        bool record(int s, int kind, int c) {
            return ok(cudaEventRecord(ev[kind * C + c], stream(s)), "event record");
        }
        bool copy_in(int c) {
            const int n0 = c * chunk, m = std::min(N, n0 + chunk) - n0;
            *st = copy_states<T>(g, g->pr_f, ys, n0, n0, m);
            return *st == NS_OK;
        }
        bool sweep(int c) {
            const int n0 = c * chunk, m = std::min(N, n0 + chunk) - n0;
            *swept_states += m;
            *sweeps += 1;
            return ok(cudaGraphLaunch(g->swc_exec[c], g->stream), "sweep graph launch");
        }
        bool defect_reset() {
            return ok(cudaMemsetAsync(h->d_defect, 0, sizeof(unsigned long long), h->stream),
                      "defect reset");
        }
        bool chain(int c) {
            return ok(cudaGraphLaunch(g->chunk_exec[c], h->stream), "chain graph launch");
        }
        bool defect_out(int k) {
            return ok(cudaMemcpyAsync(g->h_defects + k, h->d_defect, sizeof(double),
                                      cudaMemcpyDeviceToHost, h->stream),
                      "defect copy") &&
                   ok(cudaEventRecord(ev[3 * C + 1], h->stream), "event record");
        }
        int converged(int k) {
            if (!ok(cudaEventSynchronize(ev[3 * C + 1]), "defect wait")) return -1;
            const double dk = g->h_defects[k];
            return !std::isfinite(dk) || dk <= tol ? 1 : 0;
        }
    } ops{g, h, ev, C, N, chunk, tol, ys, &swept_states, &sweeps, &st_issue};
    int k = 0;
    if (cudaEventRecord(ev_start, g->stream) != cudaSuccess ||
        cudaStreamWaitEvent(h->stream, ev_start, 0) != cudaSuccess)
        st_issue = fail(NS_ERR_CUDA, "pipelined Parareal: event record failed");
    else {
        k = pipeline_issue(C, kmax, tol > 0.0, ops);
        if (k < 0) k = 0;
    }
    const std::string err_issue = g_last_error;
    // the slices are written by the chain: later work on this stream waits for it
    const cudaError_t e1 = cudaEventRecord(ev_start, h->stream);
    const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(g->stream, ev_start, 0) : e1;
    const cudaError_t e3 = cudaStreamSynchronize(g->stream);
    const cudaError_t e4 = cudaStreamSynchronize(h->stream);
    if (st_issue != NS_OK) return fail(st_issue, err_issue);
    for (cudaError_t e : {e2, e3, e4})
        if (e != cudaSuccess)
            return fail(NS_ERR_CUDA, std::string("pipelined Parareal: ") + cudaGetErrorString(e));
    // the work of every launch, and a failed solve, from the device counters
    const ns_status st_f = account_graph(g, std::min(N, chunk), swept_states * S, sweeps * S, 0,
                                        g->sweep_seen_lc, g->sweep_seen_ctl.data(),
                                        "ns_parareal_iterate (fine sweep)");
    const std::string err_f = g_last_error;
    const ns_status st_c = account_graph(h, 1, (long long)k * N * M, (long long)k * N * M,
                                        4LL * N * k, g->chain_seen_lc, &g->chain_seen_ctl,
                                        "ns_parareal_iterate");
    merge_chain_stats(g, chain0);
    if (st_f != NS_OK) return fail(st_f, err_f);
    NS_TRY(st_c);
    for (int i = 0; i < k; ++i) {
        if (defects) defects[i] = g->h_defects[i];
        if (!std::isfinite(g->h_defects[i])) {
            *k_out = i + 1;
            return fail(NS_ERR_NONFINITE, "non-finite Parareal defect");
        }
    }
    *k_out = k;
    return NS_OK;
}

template <typename T>
ns_status parareal_impl(ns_grid* g, ns_state u0, ns_state slices, int N, int S, int M,
                        double dt, int kmax, double tol, int resume, int* k_done,
                        double* defects) {
    const Geo& G = g->geo;
    if (!g->pr_f[0] || g->pr_n < N) {
        for (int c = 0; c < 4; ++c) {
            const size_t es = c == 3 ? sizeof(double) : sizeof(T);
            NS_TRY(dalloc(g, &g->pr_f[c], (size_t)G.cnt[c] * es * g->cap));
            NS_TRY(dalloc(g, &g->pr_gold[c], (size_t)G.cnt[c] * es * g->cap));
            NS_TRY(dalloc(g, &g->pr_g[c], (size_t)G.cnt[c] * es));
        }
        g->pr_n = g->cap;
        g->pr_valid = false;
    }
    void* ys[4] = {slices.u, slices.v, slices.w, slices.p};
    const void* u0s[4] = {u0.u, u0.v, u0.w, u0.p};
    const double dtc = dt * S / M;
    ns_state gs{g->pr_g[0], g->pr_g[1], g->pr_g[2], g->pr_g[3], 1};
    if (resume) {
        if (!g->pr_valid || g->pr_slices_u != slices.u || g->pr_n < N || g->pr_key_n != N ||
            g->pr_key_s != S || g->pr_key_m != M || g->pr_key_dt != dt)
            return fail(NS_ERR_ARG, "ns_parareal_iterate: resume=1 without stored coarse values "
                                    "for these slices, slice count, steps and dt");
    } else {
        // iteration 0: the serial coarse sweep y_{n+1} = G(y_n)
        NS_TRY(ensure_chain(g));
        NS_TRY(on_chain(g, [&](ns_grid* h) -> ns_status {
            // persistent solves: checked once, after the whole sweep
            h->defer = true;
            struct Undefer {
                ns_grid* h;
                ~Undefer() { h->defer = false; }
            } undefer{h};
            NS_TRY(copy_states<T>(h, ys, u0s, 0, 0, 1));
            for (int n = 0; n < N; ++n) {
                NS_TRY(copy_states<T>(h, ys, ys, n + 1, n, 1));
                ns_state one{(char*)slices.u + (size_t)(n + 1) * G.cnt[0] * sizeof(T),
                             (char*)slices.v + (size_t)(n + 1) * G.cnt[1] * sizeof(T),
                             (char*)slices.w + (size_t)(n + 1) * G.cnt[2] * sizeof(T),
                             (char*)slices.p + (size_t)(n + 1) * G.cnt[3] * sizeof(double), 1};
                NS_TRY(step_impl<T>(h, one, dtc, M));
                NS_TRY(copy_states<T>(h, g->pr_gold, ys, n, n + 1, 1));
            }
            h->defer = false;
            return persist_check(h);
        }));
    }
    g->pr_valid = false;
    const bool prof_sweep = g->prof.on && N >= g->prof.min_batch;
    int chunk = g->d.parareal_chunk > 0 ? g->d.parareal_chunk : 0;
    if (g->d.parareal_chunk == 0 && kmax >= 2 && N >= 4 && g->mg && !prof_sweep) {
        // automatic: two chunks pipelined across the call's iterations, where
        // both grids' graphs apply
        NS_TRY(ensure_chain(g));
        if (g->chain->mg && !g->chain->persist) chunk = (N + 1) / 2;
    }
    if (chunk > 0 && chunk < N && kmax > 0) {
        NS_TRY(ensure_chain(g));
        // chunks' sweeps and chains as graphs, pipelined across iterations
        // (per-launch timing, when on, needs the stream path's launches)
        if (g->mg && g->chain->mg && !prof_sweep) {
            int kd = 0;
            const ns_status st =
                parareal_pipelined<T>(g, slices, N, S, M, dt, chunk, kmax, tol, &kd, defects);
            if (k_done) *k_done = kd;
            NS_TRY(st);
            g->pr_valid = true;
            g->pr_slices_u = slices.u;
            g->pr_key_n = N;
            g->pr_key_s = S;
            g->pr_key_m = M;
            g->pr_key_dt = dt;
            return sync_stream(g);
        }
    }
    int k = 0;
    for (; k < kmax; ++k) {
        double dk;
        if (chunk > 0 && chunk < N) {
            NS_TRY(parareal_iteration_chunked<T>(g, slices, N, S, M, dt, chunk, &dk));
        } else {
            // F(y^k_n) for all n in one batched sweep: one graph launch with
            // the multigrid solver (per-launch timing, when on, needs the
            // stream path's launches)
            NS_TRY(copy_states<T>(g, g->pr_f, ys, 0, 0, N));
            const bool graphed = g->mg && !(g->prof.on && N >= g->prof.min_batch);
            if (graphed) {
                NS_TRY(sweep_launch<T>(g, N, S, dt));
            } else {
                ns_state fb{g->pr_f[0], g->pr_f[1], g->pr_f[2], g->pr_f[3], N};
                NS_TRY(step_impl<T>(g, fb, dt, S));
            }
            // serial coarse sweep with the update of Eq. 6, on the companion
            auto chain = [&](ns_grid* h) -> ns_status {
                NS_CUDA(cudaMemsetAsync(h->d_defect, 0, sizeof(unsigned long long), h->stream));
                for (int n = 0; n < N; ++n) {
                    NS_TRY(copy_states<T>(h, g->pr_g, ys, 0, n, 1));
                    NS_TRY(step_impl<T>(h, gs, dtc, M));
                    NS_TRY(parareal_update<T>(h, g->pr_f, g->pr_g, g->pr_gold, ys, n, n, n + 1));
                }
                return NS_OK;
            };
            NS_TRY(on_chain(g, [&](ns_grid* h) -> ns_status {
                if (!h->mg) {
                    NS_TRY(chain(h));
                } else if (h->persist) {
                    // every coarse solve is one persistent launch: the chain
                    // is issued directly and its solves checked at its end
                    h->defer = true;
                    const ns_status sc = chain(h);
                    h->defer = false;
                    if (sc != NS_OK) {
                        h->persist_pending = 0;
                        return sc;
                    }
                    NS_TRY(persist_check(h));
                } else {
                    // the whole chain is one graph launch: its solver loops
                    // run on the device, with no host round trip per solve
                    NS_TRY(ensure_chain_graph(g, slices.u, N, M, dtc, [&]() { return chain(h); }));
                    NS_CUDA(cudaGraphLaunch(g->chain_exec, h->stream));
                    NS_CUDA(cudaStreamSynchronize(h->stream));
                    // N x M coarse steps, plus the 4 update kernels per slice
                    NS_TRY(account_graph(h, 1, (long long)N * M, (long long)N * M, 4LL * N,
                                         g->chain_seen_lc,
                                         &g->chain_seen_ctl, "ns_parareal_iterate"));
                }
                NS_CUDA(cudaMemcpyAsync(h->h_defect, h->d_defect, sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, h->stream));
                return NS_OK;
            }));
            NS_TRY(sync_stream(g));
            if (graphed)
                NS_TRY(account_graph(g, N, (long long)N * S, S, 0, g->sweep_seen_lc,
                                     g->sweep_seen_ctl.data(),
                                     "ns_parareal_iterate (fine sweep)"));
            std::memcpy(&dk, g->chain->h_defect, sizeof(double));
        }
        if (defects) defects[k] = dk;
        if (!std::isfinite(dk)) {
            if (k_done) *k_done = k + 1;
            return fail(NS_ERR_NONFINITE, "non-finite Parareal defect");
        }
        if (tol > 0.0 && dk <= tol) {
            ++k;
            break;
        }
    }
    if (k_done) *k_done = k;
    g->pr_valid = true;
    g->pr_slices_u = slices.u;
    g->pr_key_n = N;
    g->pr_key_s = S;
    g->pr_key_m = M;
    g->pr_key_dt = dt;
    return sync_stream(g);
}

// Reverse mode through nsteps fine steps with checkpoints of (u, p) every
// ckpt_every steps: forward once storing checkpoints, then per segment (last
// first) recompute its states from the checkpoint and run the adjoint steps
// back through it.  T is the grid's velocity type: the FP32+refine grid runs
// the forward steps, the adjoint projections (its float-float refined solve)
// and the adjoint stencils in FP32, with J and dJ/du_lid summed in FP64.  All
// buffers are allocated for the call and freed after.
template <typename T>
ns_status adjoint_impl(ns_grid* g, const ns_state& u0, double dt, int N, int C, double* J,
                       const ns_state& grad, double* dlid_out) {
    const Geo& G = g->geo;
    const int B = u0.batch;
    const size_t nv[3] = {(size_t)G.cnt[0] * B, (size_t)G.cnt[1] * B, (size_t)G.cnt[2] * B};
    const size_t np = (size_t)G.cnt[3] * B;
    const size_t vel_elems = nv[0] + nv[1] + nv[2];
    const int nck = N > 0 ? (N + C - 1) / C : 0;
    const int seg_len = std::min(C, std::max(N, 1));
    const int tblocks = (int)std::min<long long>((std::max(G.cnt[0], std::max(G.cnt[1], G.cnt[2])) +
                                                  NTHREADS - 1) / NTHREADS, 512);
    std::vector<void*> mine;
    auto alloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        mine.push_back(p);
        return p;
    };
    auto release = [&]() {
        cudaStreamSynchronize(g->stream);
        for (void* p : mine) cudaFree(p);
        mine.clear();
    };
    T* cur = (T*)alloc(sizeof(T) * vel_elems);
    double* cur_p = (double*)alloc(sizeof(double) * np);
    T* ck = (T*)alloc(sizeof(T) * vel_elems * std::max(nck, 1));
    double* ck_p = (double*)alloc(sizeof(double) * np * std::max(nck, 1));
    T* seg = (T*)alloc(sizeof(T) * vel_elems * seg_len);
    T* lam = (T*)alloc(sizeof(T) * vel_elems);
    T* mu = (T*)alloc(sizeof(T) * vel_elems);
    T* acc = (T*)alloc(sizeof(T) * vel_elems);
    double* pmu = (double*)alloc(sizeof(double) * np);  // phi of the adjoint projections
    double* dJ = (double*)alloc(sizeof(double) * 2 * B);
    double* part_J = (double*)alloc(sizeof(double) * 3 * tblocks * B);
    // (dR/du)^T mu: 32 x 4 column tiles over the face extents, ADJ_TZ
    // positions along z per thread, one grid z-slice per component
    const int adj_ctas = G.fbx * G.fby * ceil_div(G.n[2] + 1, ADJ_TZ);
    double* part_lid = (double*)alloc(sizeof(double) * 3 * adj_ctas * B);
    if (mine.size() != 12) {
        release();
        return fail(NS_ERR_OOM, "ns_adjoint: workspace allocation failed");
    }
    auto vel_state = [&](T* base, double* p) {
        ns_state st{base, base + nv[0], base + nv[0] + nv[1], p, B};
        return st;
    };
    const void* src0[4] = {u0.u, u0.v, u0.w, u0.p};
    ns_state cs = vel_state(cur, cur_p);
    void* dst0[4] = {cs.u, cs.v, cs.w, cs.p};
    ns_status st = copy_states<T>(g, dst0, src0, 0, 0, B);
    NS_CUDA(cudaMemsetAsync(acc, 0, sizeof(T) * vel_elems, g->stream));
    NS_CUDA(cudaMemsetAsync(dJ, 0, sizeof(double) * 2 * B, g->stream));
    NS_CUDA(cudaMemsetAsync(pmu, 0, sizeof(double) * np, g->stream));
    auto copy = [&](void* dst, const void* src, size_t bytes, const char* what) {
        if (st == NS_OK && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice,
                                           g->stream) != cudaSuccess)
            st = fail(NS_ERR_CUDA, std::string("ns_adjoint: ") + what + " copy failed");
    };
    // forward with checkpoints
    for (int n = 0; n < N && st == NS_OK; ++n) {
        if (n % C == 0) {
            copy(ck + (size_t)(n / C) * vel_elems, cur, sizeof(T) * vel_elems, "checkpoint");
            copy(ck_p + (size_t)(n / C) * np, cur_p, sizeof(double) * np, "checkpoint");
        }
        if (st == NS_OK) st = step_impl<T>(g, cs, dt, 1);
    }
    // terminal adjoint and J (per-CTA partials, summed in a fixed order)
    const double vol = G.h[0] * G.h[1] * G.h[2];
    if (st == NS_OK) {
        for (int c = 0; c < 3; ++c) {
            const size_t off = c == 0 ? 0 : (c == 1 ? nv[0] : nv[0] + nv[1]);
            NS_LAUNCH(g, NS_K_ADJOINT, 0,
                      k_adj_terminal<T><<<dim3(tblocks, B), block_dim(), 0, g->stream>>>(
                          G, c, cur + off, lam + off, part_J, vol));
        }
        NS_LAUNCH(g, NS_K_ADJOINT, 0,
                  k_adj_sum<<<(B + 31) / 32, 32, 0, g->stream>>>(part_J, 3 * tblocks, B, dJ, 0));
        if (cudaGetLastError() != cudaSuccess) st = fail(NS_ERR_CUDA, "ns_adjoint: launch failed");
    }
    // reverse, segment by segment
    for (int sg = nck - 1; sg >= 0 && st == NS_OK; --sg) {
        const int n0 = sg * C, n1 = std::min(N, n0 + C);
        copy(cur, ck + (size_t)sg * vel_elems, sizeof(T) * vel_elems, "checkpoint");
        copy(cur_p, ck_p + (size_t)sg * np, sizeof(double) * np, "checkpoint");
        for (int n = n0; n < n1 && st == NS_OK; ++n) {
            copy(seg + (size_t)(n - n0) * vel_elems, cur, sizeof(T) * vel_elems, "segment");
            if (st == NS_OK && n + 1 < n1) st = step_impl<T>(g, cs, dt, 1);
        }
        for (int n = n1 - 1; n >= n0 && st == NS_OK; --n) {
            // mu = P lambda
            copy(mu, lam, sizeof(T) * vel_elems, "adjoint");
            if (st != NS_OK) break;
            // each adjoint projection starts from the previous one's phi
            st = project_impl<T>(g, vel_state(mu, pmu), pmu);
            if (st != NS_OK) break;
            // acc = (dR/du)^T mu at u^n, dJ/du_lid += dt (dR/du_lid)^T mu
            T* un = seg + (size_t)(n - n0) * vel_elems;
            NS_LAUNCH(g, NS_K_ADJOINT, 0,
                      k_adj_rhs<T><<<dim3(adj_ctas, B, 3), block_dim(), 0, g->stream>>>(
                          G, un, un + nv[0], un + nv[0] + nv[1], mu, mu + nv[0],
                          mu + nv[0] + nv[1], acc, acc + nv[0], acc + nv[0] + nv[1], part_lid));
            NS_LAUNCH(g, NS_K_ADJOINT, 0,
                      k_adj_sum<<<(B + 31) / 32, 32, 0, g->stream>>>(part_lid, 3 * adj_ctas, B,
                                                                    dJ + B, 1));
            // lambda = mu + dt acc (active faces); acc <- 0
            for (int c = 0; c < 3; ++c) {
                const size_t off = c == 0 ? 0 : (c == 1 ? nv[0] : nv[0] + nv[1]);
                const int blocks = (int)std::min<long long>(((long long)nv[c] + 255) / 256, 4096);
                NS_LAUNCH(g, NS_K_ADJOINT, 0,
                          k_adj_finish<T><<<blocks, 256, 0, g->stream>>>(
                              G, c, (long long)nv[c], mu + off, acc + off, lam + off, dt));
            }
            if (cudaGetLastError() != cudaSuccess)
                st = fail(NS_ERR_CUDA, "ns_adjoint: launch failed");
        }
    }
    if (st == NS_OK) {
        void* gd[3] = {grad.u, grad.v, grad.w};
        for (int c = 0; c < 3 && st == NS_OK; ++c) {
            const size_t off = c == 0 ? 0 : (c == 1 ? nv[0] : nv[0] + nv[1]);
            copy(gd[c], lam + off, sizeof(T) * nv[c], "gradient");
        }
        std::vector<double> h(2 * B);
        if (st == NS_OK &&
            (cudaMemcpyAsync(h.data(), dJ, sizeof(double) * 2 * B, cudaMemcpyDeviceToHost,
                             g->stream) != cudaSuccess ||
             cudaStreamSynchronize(g->stream) != cudaSuccess))
            st = fail(NS_ERR_CUDA, "ns_adjoint: result copy failed");
        if (st == NS_OK) {
            for (int b = 0; b < B; ++b) {
                J[b] = h[b];
                dlid_out[b] = dt * h[B + b];
            }
        }
    }
    release();
    return st;
}

}  // namespace

extern "C" {

const char* ns_last_error(void) { return g_last_error.c_str(); }

ns_status ns_create_grid(const ns_grid_desc* desc, void* cuda_stream, ns_grid** out) {
    g_last_error.clear();
    if (!desc || !out) return fail(NS_ERR_ARG, "ns_create_grid: null argument");
    *out = nullptr;
    const ns_grid_desc& d = *desc;
    if (d.nx < 2 || d.ny < 2 || d.nz < 2)
        return fail(NS_ERR_ARG, "ns_create_grid: every axis needs at least 2 cells");
    if ((long long)d.nx * d.ny * d.nz > (1LL << 31) - 1)
        return fail(NS_ERR_ARG, "ns_create_grid: more than 2^31-1 cells");
    if (!(d.lx > 0) || !(d.ly > 0) || !(d.lz > 0))
        return fail(NS_ERR_ARG, "ns_create_grid: box sizes must be positive");
    if (!(d.re > 0) || !std::isfinite(d.re))
        return fail(NS_ERR_ARG, "ns_create_grid: re must be positive and finite");
    if (!std::isfinite(d.u_lid)) return fail(NS_ERR_ARG, "ns_create_grid: u_lid not finite");
    for (int a = 0; a < 3; ++a)
        if (d.bc[a] != NS_BC_WALL && d.bc[a] != NS_BC_PERIODIC && d.bc[a] != NS_BC_SLIP)
            return fail(NS_ERR_ARG, "ns_create_grid: unknown boundary condition");
    if (d.precision != NS_FP64 && d.precision != NS_FP32_REFINE)
        return fail(NS_ERR_ARG, "ns_create_grid: unknown precision");
    if (!(d.poisson_rtol > 0) && d.precision == NS_FP64)
        return fail(NS_ERR_ARG, "ns_create_grid: poisson_rtol must be positive");
    if (d.precision == NS_FP32_REFINE && !(d.refine_rtol > 0))
        return fail(NS_ERR_ARG, "ns_create_grid: refine_rtol must be positive");
    if (d.batch < 1) return fail(NS_ERR_ARG, "ns_create_grid: batch must be >= 1");
    if (!(d.predict_tile_y == 0 && d.predict_tile_z == 0) &&
        !predict_tile_ok(d.predict_tile_y, d.predict_tile_z))
        return fail(NS_ERR_ARG, "ns_create_grid: unsupported predictor tile (" +
                                    std::to_string(d.predict_tile_y) + ", " +
                                    std::to_string(d.predict_tile_z) + ")");

    ns_grid* g = new (std::nothrow) ns_grid();
    if (!g) return fail(NS_ERR_OOM, "ns_create_grid: host allocation failed");
    g->d = d;
    g->d.solid_mask = nullptr;
    int n_solid = 0;
    if (d.solid_mask) {
        const long long nc = (long long)d.nx * d.ny * d.nz;
        g->mask_host.assign(d.solid_mask, d.solid_mask + nc);
        for (long long q = 0; q < nc; ++q) n_solid += d.solid_mask[q] != 0;
        if (n_solid == nc) {
            delete g;
            return fail(NS_ERR_ARG, "ns_create_grid: every cell is solid");
        }
    }
    g->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return fail(NS_ERR_CUDA, "ns_create_grid: cudaGetDevice failed");
    }
    g->cap = d.batch;
    g->fp32 = d.precision == NS_FP32_REFINE;
    g->maxit = d.poisson_maxit > 0 ? d.poisson_maxit : 20 * std::max(d.nx, std::max(d.ny, d.nz));
    g->inner_rtol = d.inner_rtol > 0 ? d.inner_rtol : 3e-4;
    g->max_outer = d.refine_maxit > 0 ? d.refine_maxit : kMaxOuterDefault;
    setup_geo(g);
    const Geo& G = g->geo;
    const size_t B = (size_t)g->cap;
    const size_t ncell = (size_t)G.cnt[3];
    const size_t ev = elem_vel(g);
    ns_status st = NS_OK;
    auto A = [&](void** p, size_t bytes) {
        if (st == NS_OK) st = dalloc(g, p, bytes);
    };
    for (int c = 0; c < 3; ++c) A(&g->fs[c], (size_t)G.cnt[c] * ev * B);
    A((void**)&g->b, ncell * sizeof(double) * B);
    for (int q = 0; q < 8; ++q) A(&g->kv[q], ncell * ev * B);
    A((void**)&g->p64[0], ncell * sizeof(double) * B);
    A((void**)&g->p64[1], ncell * sizeof(double) * B);
    const size_t nparts = (size_t)G.ctas * B;
    A((void**)&g->part_div, nparts * sizeof(double));
    A((void**)&g->part_a, nparts * sizeof(double));
    A((void**)&g->part_b, nparts * 2 * sizeof(double));
    A((void**)&g->part_c, nparts * 4 * sizeof(double));
    A((void**)&g->part_r, nparts * 3 * sizeof(double));
    A((void**)&g->ctl, sizeof(SliceCtl) * B);
    if (d.solid_mask && st == NS_OK) {
        // obstacles: a device copy of the cell mask
        void* m = nullptr;
        A(&m, ncell);
        if (st == NS_OK &&
            cudaMemcpy(m, d.solid_mask, ncell, cudaMemcpyHostToDevice) != cudaSuccess)
            st = fail(NS_ERR_CUDA, "ns_create_grid: mask copy failed");
        g->geo.solid = (const uint8_t*)m;
        g->geo.n_fluid = (int)(ncell - n_solid);
    }
    if (d.preconditioner == NS_PC_MULTIGRID && st == NS_OK) {
        // levels at or below this size run in one CTA per state (FP32: up to
        // 16^3, 37 KB of shared memory; FP64 keeps that one SM's share small,
        // its FP64 rate being low)
        const char* env = std::getenv("NS_MG_BLOCK_CELLS");
        const int block_cells = env ? std::max(8, std::atoi(env)) : (g->fp32 ? 4096 : 512);
        g->mg = setup_mg(g, block_cells, ev, d.solid_mask != nullptr);
        if (g->mg && d.solid_mask) {
            // solid cells enter the finest level through its face codes
            const std::vector<uint8_t> code = face_codes(g->geo, d.solid_mask);
            void* fc = nullptr;
            A(&fc, ncell);
            if (st == NS_OK &&
                cudaMemcpy(fc, code.data(), ncell, cudaMemcpyHostToDevice) != cudaSuccess)
                st = fail(NS_ERR_CUDA, "ns_create_grid: face-code copy failed");
            g->plan.lev[0].fcode = (const uint8_t*)fc;
        }
    }
    if (g->mg) {
        for (int q = 0; q < 3; ++q) A(&g->mg_vec[q], ncell * ev * B);
        for (int l = 1; l <= g->plan.lc; ++l) {
            A(&g->mg_B[l], (size_t)g->plan.lev[l].cells * ev * B);
            A(&g->mg_Y[l], (size_t)g->plan.lev[l].cells * ev * B);
        }
        A((void**)&g->counter, sizeof(unsigned int) * B);
        A((void**)&g->loopc, sizeof(LoopCount));
        A((void**)&g->p_prev, ncell * sizeof(double) * B);
        if (g->fp32)
            for (int q = 0; q < 8; ++q) A((void**)&g->ffb[q], ncell * sizeof(float) * B);
        A((void**)&g->part_mg, nparts * 6 * sizeof(double));
    }
    if (g->mg && st == NS_OK) {
        // the coarse levels on a thread-block cluster per state, where they
        // split into slabs (NS_MG_CLUSTER=0 turns it off)
        const char* ce = std::getenv("NS_MG_CLUSTER");
        int sms = 0;
        if (!(ce && std::atoi(ce) == 0) &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device) == cudaSuccess &&
            setup_cluster(g, ev, (int)B, sms))
            g->cl = g->fp32 ? cluster_ready<float>(g) : cluster_ready<double>(g);
        cudaGetLastError();
    }
    if (g->mg && st == NS_OK) {
        // persistent solves for small batches, on request (NS_PERSISTENT=1 in
        // the environment): one cooperative launch of one CTA per SM per
        // solve; NS_PERSIST_SPIN_NS bounds each barrier wait.  Measured on the
        // 64^3 coarse chain they are slower than the graph of launched
        // kernels (each phase costs a grid barrier on top of the same
        // memory-latency chain), so they are off by default.
        const char* env = std::getenv("NS_PERSISTENT");
        const bool want = env && std::atoi(env) != 0;
        int coop = 0, sms = 0;
        if (want &&
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device) == cudaSuccess &&
            coop &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device) == cudaSuccess &&
            persist_prepare() == cudaSuccess &&
            persist_blocks_per_sm(g->fp32, g->mg_smem) >= 1) {
            g->persist = true;
            g->persist_grid = sms;
        }
        cudaGetLastError();
        const char* pdl = std::getenv("NS_CHAIN_PDL");
        g->chain_pdl = !(pdl && std::atoi(pdl) == 0);
        const char* spin = std::getenv("NS_PERSIST_SPIN_NS");
        if (spin) g->spin_ns = std::max(1LL, std::atoll(spin));
        if (g->persist) {
            A((void**)&g->pbar, PERSIST_BAR_WORDS * sizeof(unsigned));
            A((void**)&g->perr, sizeof(int));
            A((void**)&g->psnap_ctl, sizeof(SliceCtl) * B);
            if (st == NS_OK && (cudaMemsetAsync(g->pbar, 0, PERSIST_BAR_WORDS * sizeof(unsigned),
                                                g->stream) !=
                                    cudaSuccess ||
                                cudaMemsetAsync(g->perr, 0, sizeof(int), g->stream) != cudaSuccess))
                st = fail(NS_ERR_CUDA, "ns_create_grid: memset failed");
        }
    }
    A((void**)&g->d_defect, sizeof(unsigned long long));
    if (st == NS_OK) {
        if (cudaMallocHost((void**)&g->h_ctl, sizeof(SliceCtl) * B) != cudaSuccess ||
            cudaMallocHost((void**)&g->h_defect, sizeof(unsigned long long)) != cudaSuccess) {
            cudaGetLastError();
            st = fail(NS_ERR_OOM, "ns_create_grid: pinned host allocation failed");
        }
    }
    if (st == NS_OK) {
        // zero once: P/V of the idle parity and the wall faces of F*
        for (int c = 0; c < 3; ++c)
            if (cudaMemsetAsync(g->fs[c], 0, (size_t)G.cnt[c] * ev * B, g->stream) != cudaSuccess)
                st = fail(NS_ERR_CUDA, "ns_create_grid: memset failed");
        for (int q = 0; q < 8 && st == NS_OK; ++q)
            if (cudaMemsetAsync(g->kv[q], 0, ncell * ev * B, g->stream) != cudaSuccess)
                st = fail(NS_ERR_CUDA, "ns_create_grid: memset failed");
        if (st == NS_OK &&
            cudaMemsetAsync(g->ctl, 0, sizeof(SliceCtl) * B, g->stream) != cudaSuccess)
            st = fail(NS_ERR_CUDA, "ns_create_grid: memset failed");
        if (st == NS_OK && g->loopc &&
            cudaMemsetAsync(g->loopc, 0, sizeof(LoopCount), g->stream) != cudaSuccess)
            st = fail(NS_ERR_CUDA, "ns_create_grid: memset failed");
        if (st == NS_OK) {
            const int py = g->geo.pty, pz = g->geo.ptz;
            const bool ok = g->fp32 ? (predict_smem_attr<float, false>(py, pz) == cudaSuccess &&
                                       predict_smem_attr<float, true>(py, pz) == cudaSuccess)
                                    : (predict_smem_attr<double, false>(py, pz) == cudaSuccess &&
                                       predict_smem_attr<double, true>(py, pz) == cudaSuccess);
            if (!ok) st = fail(NS_ERR_CUDA, "ns_create_grid: predictor shared memory attribute");
        }
        if (st == NS_OK && g->mg) {
            if (cudaMemsetAsync(g->counter, 0, sizeof(unsigned int) * B, g->stream) !=
                cudaSuccess)
                st = fail(NS_ERR_CUDA, "ns_create_grid: memset failed");
            for (int q = 0; q < 3 && st == NS_OK; ++q)
                if (cudaMemsetAsync(g->mg_vec[q], 0, ncell * ev * B, g->stream) != cudaSuccess)
                    st = fail(NS_ERR_CUDA, "ns_create_grid: memset failed");
            // k_mg_block's shared memory stays within the default 48 KB
            // (setup_mg): no function attribute, which is process-wide and
            // would be overwritten by every grid created later
        }
        if (st == NS_OK && cudaStreamSynchronize(g->stream) != cudaSuccess)
            st = fail(NS_ERR_CUDA, "ns_create_grid: stream synchronize failed");
    }
    if (st != NS_OK) {
        free_all(g);
        delete g;
        return st;
    }
    *out = g;
    return NS_OK;
}

ns_status ns_destroy_grid(ns_grid* grid) {
    if (!grid) return NS_OK;
    const DeviceGuard dg(grid->device);
    cudaStreamSynchronize(grid->stream);
    if (grid->chain_exec) cudaGraphExecDestroy(grid->chain_exec);
    if (grid->chain_graph) cudaGraphDestroy(grid->chain_graph);
    for (cudaGraphExec_t e : grid->chunk_exec) cudaGraphExecDestroy(e);
    for (cudaGraph_t c : grid->chunk_graph) cudaGraphDestroy(c);
    for (cudaStream_t cs : grid->chain_cap)
        if (cs) cudaStreamDestroy(cs);
    drop_sweep_graph(grid);
    for (cudaStream_t cs : grid->sweep_cap)
        if (cs) cudaStreamDestroy(cs);
    if (grid->chain) ns_destroy_grid(grid->chain);
    if (grid->chain_stream) cudaStreamDestroy(grid->chain_stream);
    for (cudaEvent_t e : grid->pipe_ev) cudaEventDestroy(e);
    grid->pipe_ev.clear();
    free_all(grid);
    delete grid;
    return NS_OK;
}

ns_status ns_set_stream(ns_grid* grid, void* cuda_stream) {
    if (!grid) return fail(NS_ERR_ARG, "ns_set_stream: null grid");
    grid->stream = (cudaStream_t)cuda_stream;
    return NS_OK;
}

ns_status ns_step_fine(ns_grid* grid, ns_state io, double dt, int nsteps) {
    g_last_error.clear();
    return step_any(grid, io, dt, nsteps, "ns_step_fine");
}

ns_status ns_step_coarse(ns_grid* grid, ns_state io, double dt_coarse, int nsteps) {
    g_last_error.clear();
    return step_any(grid, io, dt_coarse, nsteps, "ns_step_coarse");
}

ns_status ns_project(ns_grid* grid, ns_state io) {
    g_last_error.clear();
    if (!grid) return fail(NS_ERR_ARG, "ns_project: null grid");
    const DeviceGuard dg(grid->device);
    NS_TRY(check_state(grid, io, "ns_project"));
    ns_status st = grid->fp32 ? project_impl<float>(grid, io) : project_impl<double>(grid, io);
    if (st == NS_OK) NS_TRY(sync_stream(grid));
    return st;
}

ns_status ns_predict(ns_grid* grid, ns_state in, double dt, void* fu, void* fv, void* fw) {
    g_last_error.clear();
    if (!grid) return fail(NS_ERR_ARG, "ns_predict: null grid");
    const DeviceGuard dg(grid->device);
    NS_TRY(check_state(grid, in, "ns_predict"));
    if (!fu || !fv || !fw) return fail(NS_ERR_ARG, "ns_predict: null output pointer");
    if (!std::isfinite(dt)) return fail(NS_ERR_ARG, "ns_predict: dt not finite");
    const Geo& G = grid->geo;
    const dim3 gface(G.fctas, in.batch);
    grid->prof.active = in.batch >= grid->prof.min_batch;
    (void)gface;
    if (grid->fp32)
        NS_LAUNCH(grid, NS_K_PREDICT, G.cnt[3] * in.batch,
                  (launch_predict<float, false>(grid, in.batch, (const float*)in.u,
                                                (const float*)in.v, (const float*)in.w,
                                                (float*)fu, (float*)fv, (float*)fw, dt)));
    else
        NS_LAUNCH(grid, NS_K_PREDICT, G.cnt[3] * in.batch,
                  (launch_predict<double, false>(grid, in.batch, (const double*)in.u,
                                                 (const double*)in.v, (const double*)in.w,
                                                 (double*)fu, (double*)fv, (double*)fw, dt)));
    NS_CUDA(cudaGetLastError());
    NS_TRY(sync_stream(grid));
    return NS_OK;
}

ns_status ns_poisson_solve(ns_grid* grid, const double* b, double* p, int batch, int* iters) {
    g_last_error.clear();
    if (!grid) return fail(NS_ERR_ARG, "ns_poisson_solve: null grid");
    const DeviceGuard dg(grid->device);
    if (!b || !p) return fail(NS_ERR_ARG, "ns_poisson_solve: null pointer");
    if (batch < 1 || batch > grid->cap)
        return fail(NS_ERR_ARG, "ns_poisson_solve: batch outside [1, capacity]");
    const Geo& G = grid->geo;
    const dim3 gcell(G.ctas, batch), gface(G.fctas, batch);
    NS_CUDA(cudaMemcpyAsync(grid->b, b, sizeof(double) * G.cnt[3] * batch,
                            cudaMemcpyDeviceToDevice, grid->stream));
    grid->prof.active = batch >= grid->prof.min_batch;
    NS_LAUNCH(grid, NS_K_DIVERGENCE, G.cnt[3] * batch,
              k_sum_cells<<<gcell, block_dim(), 0, grid->stream>>>(G, grid->b, grid->part_div));
    NS_CUDA(cudaGetLastError());
    NS_TRY(solve_pressure(grid, batch, p));
    // write p - mean(p) back through the correction kernel's cell part, with
    // the face part pointed at the (unused) F* buffers
    const double* x0 = grid->fp32 ? grid->p64[0] : (const double*)grid->kv[0];
    const double* x1 = grid->fp32 ? grid->p64[1] : (const double*)grid->kv[0];
    if (grid->fp32 && grid->mg)
        NS_LAUNCH(grid, NS_K_CORRECT, G.cnt[3] * batch,
                  k_correct_ff<false><<<gface, block_dim(), 0, grid->stream>>>(
                      G, grid->ctl, (float*)grid->fs[0], (float*)grid->fs[1], (float*)grid->fs[2],
                      (float*)grid->fs[0], (float*)grid->fs[1], (float*)grid->fs[2], ffbuf(grid),
                      p, dt_ih(G, 0.0), 0));
    else if (grid->fp32)
        NS_LAUNCH(grid, NS_K_CORRECT, G.cnt[3] * batch,
                  k_correct<float, false><<<gface, block_dim(), 0, grid->stream>>>(
                      G, grid->ctl, (float*)grid->fs[0], (float*)grid->fs[1], (float*)grid->fs[2],
                      (float*)grid->fs[0], (float*)grid->fs[1], (float*)grid->fs[2], x0, x1, p,
                      0.0));
    else
        NS_LAUNCH(grid, NS_K_CORRECT, G.cnt[3] * batch,
                  k_correct<double, false><<<gface, block_dim(), 0, grid->stream>>>(
                      G, grid->ctl, (double*)grid->fs[0], (double*)grid->fs[1],
                      (double*)grid->fs[2], (double*)grid->fs[0], (double*)grid->fs[1],
                      (double*)grid->fs[2], x0, x1, p, 0.0));
    NS_CUDA(cudaGetLastError());
    NS_TRY(persist_settle(grid));
    NS_TRY(sync_stream(grid));
    if (iters) *iters = grid->stats.last_max_iters;
    return NS_OK;
}

ns_status ns_parareal_iterate(ns_grid* grid, ns_state u0, ns_state slices, int n_slices,
                              int fine_steps_per_slice, int coarse_steps_per_slice,
                              double dt_fine, int kmax, double defect_tol, int resume,
                              int* k_done, double* defects) {
    g_last_error.clear();
    if (k_done) *k_done = 0;
    if (!grid) return fail(NS_ERR_ARG, "ns_parareal_iterate: null grid");
    const DeviceGuard dg(grid->device);
    if (n_slices < 1 || n_slices > grid->cap)
        return fail(NS_ERR_ARG, "ns_parareal_iterate: n_slices outside [1, capacity]");
    if (u0.batch != 1) return fail(NS_ERR_ARG, "ns_parareal_iterate: u0 must hold one state");
    NS_TRY(check_state(grid, u0, "ns_parareal_iterate(u0)"));
    if (!slices.u || !slices.v || !slices.w || !slices.p || slices.batch != n_slices + 1)
        return fail(NS_ERR_ARG, "ns_parareal_iterate: slices must hold n_slices+1 states");
    if (fine_steps_per_slice < 1 || coarse_steps_per_slice < 1)
        return fail(NS_ERR_ARG, "ns_parareal_iterate: steps per slice must be >= 1");
    if (!(dt_fine > 0) || !std::isfinite(dt_fine))
        return fail(NS_ERR_ARG, "ns_parareal_iterate: dt_fine must be positive");
    if (kmax < 0) return fail(NS_ERR_ARG, "ns_parareal_iterate: kmax < 0");
    if (resume != 0 && resume != 1) return fail(NS_ERR_ARG, "ns_parareal_iterate: resume 0/1");
    ns_status st = grid->fp32
                       ? parareal_impl<float>(grid, u0, slices, n_slices, fine_steps_per_slice,
                                              coarse_steps_per_slice, dt_fine, kmax, defect_tol,
                                              resume, k_done, defects)
                       : parareal_impl<double>(grid, u0, slices, n_slices, fine_steps_per_slice,
                                               coarse_steps_per_slice, dt_fine, kmax, defect_tol,
                                               resume, k_done, defects);
    return st;
}

ns_status ns_adjoint(ns_grid* grid, ns_state u0, double dt, int nsteps, int ckpt_every, double* J,
                     ns_state grad_u0, double* dJ_dulid) {
    g_last_error.clear();
    if (!grid) return fail(NS_ERR_ARG, "ns_adjoint: null grid");
    const DeviceGuard dg(grid->device);
    NS_TRY(check_state(grid, u0, "ns_adjoint(u0)"));
    if (grid->geo.solid) return fail(NS_ERR_ARG, "ns_adjoint: grids with solid cells are not "
                                                 "supported");
    if (!grad_u0.u || !grad_u0.v || !grad_u0.w || grad_u0.batch != u0.batch)
        return fail(NS_ERR_ARG, "ns_adjoint: grad_u0 must hold u0.batch velocity fields");
    if (!J || !dJ_dulid) return fail(NS_ERR_ARG, "ns_adjoint: null J or dJ_dulid");
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0 || ckpt_every < 1)
        return fail(NS_ERR_ARG, "ns_adjoint: need dt > 0, nsteps >= 0, ckpt_every >= 1");
    return grid->fp32 ? adjoint_impl<float>(grid, u0, dt, nsteps, ckpt_every, J, grad_u0, dJ_dulid)
                      : adjoint_impl<double>(grid, u0, dt, nsteps, ckpt_every, J, grad_u0,
                                             dJ_dulid);
}

ns_status ns_kinetic_energy(ns_grid* grid, ns_state state, double* J) {
    g_last_error.clear();
    if (!grid) return fail(NS_ERR_ARG, "ns_kinetic_energy: null grid");
    const DeviceGuard dg(grid->device);
    if (!state.u || !state.v || !state.w || state.batch < 1)
        return fail(NS_ERR_ARG, "ns_kinetic_energy: null velocity or batch < 1");
    if (!J) return fail(NS_ERR_ARG, "ns_kinetic_energy: null J");
    const Geo& G = grid->geo;
    const int B = state.batch;
    const int tblocks = (int)std::min<long long>(
        (std::max(G.cnt[0], std::max(G.cnt[1], G.cnt[2])) + NTHREADS - 1) / NTHREADS, 512);
    double* part = nullptr;
    double* dJ = nullptr;
    if (cudaMalloc(&part, sizeof(double) * 3 * tblocks * B) != cudaSuccess ||
        cudaMalloc(&dJ, sizeof(double) * B) != cudaSuccess) {
        cudaGetLastError();
        if (part) cudaFree(part);
        return fail(NS_ERR_OOM, "ns_kinetic_energy: workspace allocation failed");
    }
    const double vol = G.h[0] * G.h[1] * G.h[2];
    const void* vel[3] = {state.u, state.v, state.w};
    for (int c = 0; c < 3; ++c) {
        if (grid->fp32)
            k_adj_terminal<float><<<dim3(tblocks, B), block_dim(), 0, grid->stream>>>(
                G, c, (const float*)vel[c], nullptr, part, vol);
        else
            k_adj_terminal<double><<<dim3(tblocks, B), block_dim(), 0, grid->stream>>>(
                G, c, (const double*)vel[c], nullptr, part, vol);
        grid->stats.launches += 1;
    }
    k_adj_sum<<<(B + 31) / 32, 32, 0, grid->stream>>>(part, 3 * tblocks, B, dJ, 0);
    grid->stats.launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(J, dJ, sizeof(double) * B, cudaMemcpyDeviceToHost, grid->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(grid->stream);
    cudaFree(part);
    cudaFree(dJ);
    if (e != cudaSuccess)
        return fail(NS_ERR_CUDA, std::string("ns_kinetic_energy: ") + cudaGetErrorString(e));
    return NS_OK;
}

ns_status ns_set_lid_speed(ns_grid* grid, double u_lid) {
    g_last_error.clear();
    if (!grid) return fail(NS_ERR_ARG, "ns_set_lid_speed: null grid");
    if (!std::isfinite(u_lid)) return fail(NS_ERR_ARG, "ns_set_lid_speed: u_lid not finite");
    grid->d.u_lid = u_lid;
    grid->geo.u_lid = u_lid;
    // the coarse propagator's companion grid and every graph captured from
    // this grid hold the description by value: update the companion, drop
    // the chain graphs (recaptured on next use), and invalidate the stored
    // coarse values G(y^k_n) of the old lid (a resume then needs a fresh
    // start) and the graphs of ns_graph_create (their launches then fail)
    const DeviceGuard dg(grid->device);
    if (grid->chain) {
        cudaStreamSynchronize(grid->chain->stream);
        grid->chain->d.u_lid = u_lid;
        grid->chain->geo.u_lid = u_lid;
        grid->chain->gen += 1;
    }
    if (grid->chain_exec) cudaGraphExecDestroy(grid->chain_exec);
    if (grid->chain_graph) cudaGraphDestroy(grid->chain_graph);
    grid->chain_exec = nullptr;
    grid->chain_graph = nullptr;
    for (cudaGraphExec_t e : grid->chunk_exec) cudaGraphExecDestroy(e);
    for (cudaGraph_t c : grid->chunk_graph) cudaGraphDestroy(c);
    grid->chunk_exec.clear();
    grid->chunk_graph.clear();
    drop_sweep_graph(grid);
    grid->pr_valid = false;
    grid->gen += 1;
    return NS_OK;
}

ns_status ns_profile_enable(ns_grid* grid, int on, int min_batch) {
    g_last_error.clear();
    if (!grid) return fail(NS_ERR_ARG, "ns_profile_enable: null grid");
    const DeviceGuard dg(grid->device);
    auto& P = grid->prof;
    if (on && P.cap == 0) {
        const int pairs = 8192;
        P.ev.resize(2 * pairs);
        for (auto& e : P.ev) NS_CUDA(cudaEventCreate(&e));
        P.kind.resize(pairs);
        P.units.resize(pairs);
        P.cap = pairs;
    }
    NS_TRY(sync_stream(grid));
    P.on = on != 0;
    P.min_batch = std::max(1, min_batch);
    P.n = 0;
    for (auto& a : P.acc) a = ns_kernel_time{};
    return NS_OK;
}

ns_status ns_profile_read(ns_grid* grid, ns_kernel_time* out, int n) {
    g_last_error.clear();
    if (!grid || !out) return fail(NS_ERR_ARG, "ns_profile_read: null argument");
    const DeviceGuard dg(grid->device);
    NS_TRY(sync_stream(grid));
    for (int q = 0; q < std::min<int>(n, NS_K_KINDS); ++q) out[q] = grid->prof.acc[q];
    return NS_OK;
}

ns_status ns_get_stats(const ns_grid* grid, ns_stats* out) {
    if (!grid || !out) return fail(NS_ERR_ARG, "ns_get_stats: null argument");
    *out = grid->stats;
    return NS_OK;
}

ns_status ns_reset_stats(ns_grid* grid) {
    if (!grid) return fail(NS_ERR_ARG, "ns_reset_stats: null argument");
    grid->stats = ns_stats{};
    return NS_OK;
}

ns_status ns_step_fine_many(ns_grid* const* grids, const ns_state* states, const double* dts,
                            const int* nsteps, int n) {
    if (!grids || !states || !dts || !nsteps || n < 1)
        return fail(NS_ERR_ARG, "ns_step_fine_many: null array or n < 1");
    for (int i = 0; i < n; ++i) {
        if (!grids[i]) return fail(NS_ERR_ARG, "ns_step_fine_many: null grid");
        for (int j = 0; j < i; ++j)
            if (grids[j] == grids[i])
                return fail(NS_ERR_ARG, "ns_step_fine_many: a grid appears twice");
    }
    std::vector<cudaStream_t> own(n, nullptr);
    std::vector<cudaStream_t> saved(n, nullptr);
    std::vector<cudaEvent_t> ev(2 * n, nullptr);
    ns_status st = NS_OK;
    for (int i = 0; i < n && st == NS_OK; ++i) {
        const DeviceGuard dg(grids[i]->device);
        if (cudaStreamCreateWithFlags(&own[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev[2 * i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev[2 * i + 1], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(ev[2 * i], grids[i]->stream) != cudaSuccess ||
            cudaStreamWaitEvent(own[i], ev[2 * i], 0) != cudaSuccess)
            st = fail(NS_ERR_CUDA, "ns_step_fine_many: stream setup failed");
    }
    std::vector<ns_status> res(n, NS_OK);
    std::vector<std::string> msg(n);
    if (st == NS_OK) {
        std::vector<std::thread> threads;
        // the grids' kernels overlap here: no persistent (cooperative) solves,
        // whose CTAs must all be resident at once
        std::vector<char> persist_saved(n);
        for (int i = 0; i < n; ++i) {
            saved[i] = grids[i]->stream;
            grids[i]->stream = own[i];
            persist_saved[i] = grids[i]->persist;
            const DeviceGuard dg(grids[i]->device);
            const ns_status sp = persist_check(grids[i]);
            if (sp != NS_OK && st == NS_OK) st = sp;
            grids[i]->persist = false;
        }
        for (int i = 0; i < n; ++i)
            threads.emplace_back([&, i]() {
                // a new host thread starts on device 0: step_any selects the grid's
                res[i] = step_any(grids[i], states[i], dts[i], nsteps[i], "ns_step_fine_many");
                if (res[i] != NS_OK) msg[i] = g_last_error;
            });
        for (auto& t : threads) t.join();
        for (int i = 0; i < n; ++i) {
            const DeviceGuard dg(grids[i]->device);
            grids[i]->persist = persist_saved[i] != 0;
            grids[i]->stream = saved[i];
            if (cudaEventRecord(ev[2 * i + 1], own[i]) != cudaSuccess ||
                cudaStreamWaitEvent(saved[i], ev[2 * i + 1], 0) != cudaSuccess)
                if (st == NS_OK) st = fail(NS_ERR_CUDA, "ns_step_fine_many: join failed");
        }
    }
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s2 : own)
        if (s2) cudaStreamDestroy(s2);
    if (st != NS_OK) return st;
    for (int i = 0; i < n; ++i)
        if (res[i] != NS_OK)
            return fail(res[i], msg[i] + " (grid " + std::to_string(i) + ")");
    return NS_OK;
}

// ---------------------------------------------------------------------------
// CUDA graphs of fine steps (several grids as concurrent branches)
// ---------------------------------------------------------------------------

struct ns_graph {
    // one executable graph per branch, each on its own stream: a launch forks
    // the branches from the caller's stream and joins them back
    std::vector<cudaGraph_t> graphs;
    std::vector<cudaGraphExec_t> execs;
    std::vector<ns_grid*> grids;
    std::vector<long long> gens;        // each grid's settings generation at capture
    std::vector<int> batch, nsteps;
    std::vector<cudaStream_t> streams;  // 2 per branch: top level, loop bodies
    std::vector<cudaEvent_t> events;    // per branch: done; last: fork
    std::vector<LoopCount> seen_loops;  // device loop totals at the last check
    std::vector<std::vector<SliceCtl>> seen_ctl;
    long long launched = 0;             // graph launches since the last check
};

namespace {

void graph_free(ns_graph* gr) {
    for (cudaGraphExec_t e : gr->execs) cudaGraphExecDestroy(e);
    for (cudaGraph_t g : gr->graphs) cudaGraphDestroy(g);
    for (cudaEvent_t e : gr->events) cudaEventDestroy(e);
    for (cudaStream_t s : gr->streams) cudaStreamDestroy(s);
    delete gr;
}

}  // namespace

ns_status ns_graph_create(ns_grid* const* grids, const ns_state* states, const double* dts,
                          const int* nsteps, int n, ns_graph** out) {
    if (!out) return fail(NS_ERR_ARG, "ns_graph_create: null output");
    *out = nullptr;
    if (!grids || !states || !dts || !nsteps || n < 1)
        return fail(NS_ERR_ARG, "ns_graph_create: null array or n < 1");
    for (int i = 0; i < n; ++i) {
        ns_grid* g = grids[i];
        if (!g) return fail(NS_ERR_ARG, "ns_graph_create: null grid");
        for (int j = 0; j < i; ++j)
            if (grids[j] == g)
                return fail(NS_ERR_ARG, "ns_graph_create: a grid appears in two branches");
        if (!g->mg)
            return fail(NS_ERR_ARG,
                        "ns_graph_create: graph-resident solves need the multigrid "
                        "preconditioner (branch " + std::to_string(i) + ")");
        NS_TRY(check_state(g, states[i], "ns_graph_create"));
        if (!(dts[i] > 0.0) || !std::isfinite(dts[i]) || nsteps[i] < 1)
            return fail(NS_ERR_ARG, "ns_graph_create: dt must be positive and nsteps >= 1");
    }
    ns_graph* gr = new (std::nothrow) ns_graph();
    if (!gr) return fail(NS_ERR_OOM, "ns_graph_create: out of host memory");
    auto bail = [&](ns_status st) {
        graph_free(gr);
        return st;
    };
    for (int i = 0; i < 2 * n; ++i) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(NS_ERR_CUDA, "ns_graph_create: stream creation failed"));
        gr->streams.push_back(s);
    }
    for (int i = 0; i < n + 1; ++i) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(NS_ERR_CUDA, "ns_graph_create: event creation failed"));
        gr->events.push_back(e);
    }
    // the branches must see the states as the caller's streams left them; a
    // grid in a graph no longer takes persistent solves (the graph's
    // accounting reads the same control-block totals)
    for (int i = 0; i < n; ++i) {
        const ns_status sp = persist_check(grids[i]);
        if (sp != NS_OK) return bail(sp);
        grids[i]->persist = false;
        if (cudaStreamSynchronize(grids[i]->stream) != cudaSuccess)
            return bail(fail(NS_ERR_CUDA, "ns_graph_create: stream synchronisation failed"));
    }
    for (int i = 0; i < n; ++i) {
        ns_grid* g = grids[i];
        cudaGraph_t graph;
        cudaGraphExec_t exec;
        const ns_status st = capture_exec(
            g, gr->streams[2 * i], gr->streams[2 * i + 1],
            [&]() -> ns_status {
                return g->fp32 ? step_impl<float>(g, states[i], dts[i], nsteps[i])
                               : step_impl<double>(g, states[i], dts[i], nsteps[i]);
            },
            &graph, &exec);
        if (st != NS_OK) return bail(st);
        gr->graphs.push_back(graph);
        gr->execs.push_back(exec);
        gr->grids.push_back(g);
        gr->gens.push_back(g->gen);
        gr->batch.push_back(states[i].batch);
        gr->nsteps.push_back(nsteps[i]);
        LoopCount lc{};
        std::vector<SliceCtl> ctl(states[i].batch);
        if (cudaMemcpy(&lc, g->loopc, sizeof(LoopCount), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(ctl.data(), g->ctl, sizeof(SliceCtl) * ctl.size(),
                       cudaMemcpyDeviceToHost) != cudaSuccess)
            return bail(fail(NS_ERR_CUDA, "ns_graph_create: reading the control blocks failed"));
        gr->seen_loops.push_back(lc);
        gr->seen_ctl.push_back(ctl);
    }
    *out = gr;
    return NS_OK;
}

ns_status ns_graph_launch(ns_graph* gr, void* cuda_stream) {
    if (!gr || gr->execs.empty()) return fail(NS_ERR_ARG, "ns_graph_launch: null graph");
    for (size_t i = 0; i < gr->grids.size(); ++i)
        if (gr->grids[i]->gen != gr->gens[i])
            return fail(NS_ERR_ARG, "ns_graph_launch: the lid speed of the grid of branch " +
                                        std::to_string(i) +
                                        " changed after the capture; create the graph again");
    const cudaStream_t cs = (cudaStream_t)cuda_stream;
    const size_t n = gr->execs.size();
    NS_CUDA(cudaEventRecord(gr->events[n], cs));
    for (size_t i = 0; i < n; ++i) {
        const cudaStream_t bs = gr->streams[2 * i];
        NS_CUDA(cudaStreamWaitEvent(bs, gr->events[n], 0));
        NS_CUDA(cudaGraphLaunch(gr->execs[i], bs));
        NS_CUDA(cudaEventRecord(gr->events[i], bs));
    }
    for (size_t i = 0; i < n; ++i) NS_CUDA(cudaStreamWaitEvent(cs, gr->events[i], 0));
    gr->launched += 1;
    return NS_OK;
}

ns_status ns_graph_check(ns_graph* gr, void* cuda_stream) {
    if (!gr) return fail(NS_ERR_ARG, "ns_graph_check: null graph");
    NS_CUDA(cudaStreamSynchronize((cudaStream_t)cuda_stream));
    ns_status result = NS_OK;
    std::string msg;
    for (size_t i = 0; i < gr->grids.size(); ++i) {
        const ns_status st = account_graph(
            gr->grids[i], gr->batch[i], gr->launched * gr->nsteps[i] * gr->batch[i],
            gr->launched * gr->nsteps[i], 0, gr->seen_loops[i],
            gr->seen_ctl[i].data(), "ns_graph_check: branch " + std::to_string(i));
        if (st != NS_OK && result == NS_OK) {
            result = st;
            msg = g_last_error;
        }
    }
    gr->launched = 0;
    return result == NS_OK ? NS_OK : fail(result, msg);
}

ns_status ns_graph_destroy(ns_graph* gr) {
    if (!gr) return NS_OK;
    for (cudaStream_t s : gr->streams) cudaStreamSynchronize(s);
    graph_free(gr);
    return NS_OK;
}

}  // extern "C"
