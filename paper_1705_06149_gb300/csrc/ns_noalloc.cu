// ns_poisson_solve_noalloc: the gauged FP64 pressure solve of ns_poisson_solve
// for one state, without any device or host allocation.
//
// Some callers cannot allocate GPU memory at the point where they need a solve:
// code running under a memory pool or allocator they do not control, inside a
// framework that forbids cudaMalloc between its own allocations, or in a
// process whose allocation budget is already spent.  This entry point serves
// them: its Krylov vectors, partial sums and control block live in one
// file-scope device array of fixed size, reserved on every GPU that loads the
// library for as long as the process runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "ns.h"
#include "ns_kernels.cuh"

using namespace nsk;

namespace {

constexpr long long kCells = NS_NOALLOC_MAX_CELLS;
constexpr int kCtas = 4096;  // CTA tiles of the largest accepted grid stay below this
constexpr int kVecs = 9;     // x, r, r_hat, P0, P1, V0, V1, t and a copy of b
constexpr long long kPartDoubles = 8LL * kCtas;  // divergence 1 + A 1 + B 2 + C 4
constexpr long long kDoubles = kVecs * kCells + kPartDoubles + 64;  // + the control block
constexpr int kMaxDevices = 64;

// The scratch.  In host code `g_scratch` is a host-side stand-in for the
// symbol, not a device address: the device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) double g_scratch[kDoubles];

std::mutex g_mutex;
double* g_base[kMaxDevices] = {};

// No message is stored (that would allocate): the status code is the report.
ns_status fail(ns_status st, const char*) { return st; }

// cells per thread along z and the tiling, as the grid object chooses them
void make_geo(Geo& G, int nx, int ny, int nz, const double L[3], const int bc[3]) {
    G = Geo{};
    G.n[0] = nx;
    G.n[1] = ny;
    G.n[2] = nz;
    for (int a = 0; a < 3; ++a) {
        G.bc[a] = bc[a];
        G.h[a] = L[a] / G.n[a];
        G.ih[a] = 1.0 / G.h[a];
        G.ih2[a] = 1.0 / (G.h[a] * G.h[a]);
    }
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a)
            G.ext[c][a] = G.n[a] + ((c == a && G.bc[a] != BC_PERIODIC) ? 1 : 0);
    for (int c = 0; c < 3; ++c) G.cnt[c] = (long long)G.ext[c][0] * G.ext[c][1] * G.ext[c][2];
    G.cnt[3] = (long long)nx * ny * nz;
    G.tz = std::min(8, nz);
    G.bx = (nx + TX - 1) / TX;
    G.by = (ny + TY - 1) / TY;
    G.bz = (nz + G.tz - 1) / G.tz;
    G.ctas = G.bx * G.by * G.bz;
    G.fbx = (nx + TX) / TX;
    G.fby = (ny + TY) / TY;
    G.fbz = (nz + G.tz) / G.tz;
    G.fctas = G.fbx * G.fby * G.fbz;
    G.n_fluid = nx * ny * nz;
}

// p = x - mean(x), the mean taken from the converged solve's sum
__global__ void __launch_bounds__(NTHREADS)
    k_noalloc_gauge(Geo g, const SliceCtl* __restrict__ ctl, const double* __restrict__ x,
                    double* __restrict__ p) {
    const double mean = ctl->sx / g.n_fluid;
    int i, j, k0;
    tile_origin(g, blockIdx.x, g.bx, g.by, i, j, k0);
    if (i >= g.n[0] || j >= g.n[1]) return;
    const int k1 = min(k0 + g.tz, g.n[2]);
    for (int k = k0; k < k1; ++k) {
        const long long id = cindex(g, i, j, k);
        p[id] = x[id] - mean;
    }
}

#define NA_CUDA(call)                                                   \
    do {                                                                \
        if ((call) != cudaSuccess) {                                    \
            cudaGetLastError();                                         \
            return fail(NS_ERR_CUDA, "ns_poisson_solve_noalloc: " #call \
                                     " failed");                        \
        }                                                               \
    } while (0)

}  // namespace

extern "C" ns_status ns_poisson_solve_noalloc(int nx, int ny, int nz, double lx, double ly,
                                              double lz, const int* bc, double rtol, int maxit,
                                              const double* b, double* p, void* cuda_stream,
                                              int* iters) {
    if (!bc || !b || !p) return fail(NS_ERR_ARG, "ns_poisson_solve_noalloc: null pointer");
    if (nx < 2 || ny < 2 || nz < 2)
        return fail(NS_ERR_ARG, "ns_poisson_solve_noalloc: every axis needs at least 2 cells");
    if ((long long)nx * ny * nz > kCells)
        return fail(NS_ERR_ARG,
                    "ns_poisson_solve_noalloc: grid exceeds NS_NOALLOC_MAX_CELLS cells");
    if (!(lx > 0) || !(ly > 0) || !(lz > 0) || !(rtol > 0) || !std::isfinite(rtol))
        return fail(NS_ERR_ARG, "ns_poisson_solve_noalloc: sizes and rtol must be positive");
    for (int a = 0; a < 3; ++a)
        if (bc[a] != NS_BC_WALL && bc[a] != NS_BC_PERIODIC && bc[a] != NS_BC_SLIP)
            return fail(NS_ERR_ARG, "ns_poisson_solve_noalloc: unknown boundary condition");
    const double L[3] = {lx, ly, lz};
    Geo G;
    make_geo(G, nx, ny, nz, L, bc);
    if (G.ctas > kCtas)
        return fail(NS_ERR_ARG, "ns_poisson_solve_noalloc: grid too thin for the scratch tiling");
    if (maxit <= 0) maxit = 20 * std::max(nx, std::max(ny, nz));

    // set-up, once per device, with that device current
    int dev = 0;
    NA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(NS_ERR_ARG, "device index out of range");
    double* base;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_base[dev]) {
            void* addr = nullptr;
            if (cudaGetSymbolAddress(&addr, g_scratch) != cudaSuccess || !addr) {
                cudaGetLastError();
                return fail(NS_ERR_CUDA,
                            "ns_poisson_solve_noalloc: cudaGetSymbolAddress failed");
            }
            g_base[dev] = static_cast<double*>(addr);
        }
        base = g_base[dev];
    }

    cudaStream_t st = (cudaStream_t)cuda_stream;
    const long long n = G.cnt[3];
    KBuf<double> kb;
    kb.x = base + 0 * kCells;
    kb.r = base + 1 * kCells;
    kb.rhat = base + 2 * kCells;
    kb.P[0] = base + 3 * kCells;
    kb.P[1] = base + 4 * kCells;
    kb.V[0] = base + 5 * kCells;
    kb.V[1] = base + 6 * kCells;
    kb.t = base + 7 * kCells;
    double* bcopy = base + 8 * kCells;
    double* part = base + kVecs * kCells;
    double* part_div = part;
    double* part_a = part + kCtas;
    double* part_b = part + 2LL * kCtas;
    double* part_c = part + 4LL * kCtas;
    SliceCtl* ctl = reinterpret_cast<SliceCtl*>(part + kPartDoubles);
    static_assert(sizeof(SliceCtl) <= 64 * sizeof(double), "control block does not fit");

    // the array keeps the previous call's contents: clear the control block,
    // and copy b so that the caller's b stays unmodified
    NA_CUDA(cudaMemsetAsync(ctl, 0, sizeof(SliceCtl), st));
    NA_CUDA(cudaMemcpyAsync(bcopy, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    const dim3 grid(G.ctas, 1), block(TX, TY, 1);
    k_sum_cells<<<grid, block, 0, st>>>(G, bcopy, part_div);
    k_bicg_init_warm<double><<<grid, block, 0, st>>>(G, kb, ctl, part_div, bcopy, p, part_c);
    NA_CUDA(cudaGetLastError());
    SliceCtl h{};
    const double tol2 = rtol * rtol;
    int next_poll = 8;
    for (int it = 1;; ++it) {
        const int par = it & 1;
        k_bicg_A<double><<<grid, block, 0, st>>>(G, kb, ctl, part_c, part_a, tol2, maxit, par);
        k_bicg_B<double><<<grid, block, 0, st>>>(G, kb, ctl, part_a, part_b, par);
        k_bicg_C<double><<<grid, block, 0, st>>>(G, kb, ctl, part_b, part_c, par);
        NA_CUDA(cudaGetLastError());
        if (it >= next_poll) {
            NA_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(SliceCtl), cudaMemcpyDeviceToHost, st));
            NA_CUDA(cudaStreamSynchronize(st));
            if (h.status != ST_ITER || it > maxit + 2) break;
            next_poll = it + std::max(2, it / 8);
        }
    }
    if (iters) *iters = h.it_cur;
    if (h.status == ST_NONFINITE)
        return fail(NS_ERR_NONFINITE, "ns_poisson_solve_noalloc: non-finite residual");
    if (h.status != ST_CONV)
        return fail(NS_ERR_NOT_CONVERGED, "ns_poisson_solve_noalloc: iteration limit reached");
    k_noalloc_gauge<<<grid, block, 0, st>>>(G, ctl, kb.x, p);
    NA_CUDA(cudaGetLastError());
    NA_CUDA(cudaStreamSynchronize(st));
    return NS_OK;
}
