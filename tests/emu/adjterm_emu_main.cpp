// Driver of the host emulation of the adjoint's terminal condition and
// finishing update (test support): k_adj_terminal (128-thread CTAs, per-CTA
// partial sums of J), k_adj_finish (256-thread CTAs) for each velocity
// component of `batch` states and k_adj_sum over the partials, FP64, grids
// smaller than the arrays (the grid-stride loops take several passes), every
// CTA as host threads.
//
// usage: adjterm_emu nx ny nz bcx bcy bcz batch vol dt in.bin out.bin
//   in.bin: for c = 0, 1, 2: u_c, mu_c, acc_c [batch][faces of c] (FP64).
//   out.bin: for c = 0, 1, 2: the terminal lambda_c, the finished lambda_c, acc_c
//   after the finish; then J [batch].

#include <functional>

// nt threads per CTA: 32 x (nt / 32) (the 128-thread kernels read
// threadIdx.y), or 256 x 1 when flat
static void launch(int gx, int gy, int nt, bool flat, const std::function<void()>& body) {
    blockDim.x = flat ? (unsigned)nt : 32u;
    blockDim.y = flat ? 1u : (unsigned)(nt / 32);
    gridDim.x = (unsigned)gx;
    gridDim.y = (unsigned)gy;
    for (int by = 0; by < gy; ++by)
        for (int bx = 0; bx < gx; ++bx) {
            std::barrier<> bar(nt);
            emu_cta_barrier = &bar;
            for (int w = 0; w < nt / 32; ++w) emu_warp_barrier[w] = new std::barrier<>(32);
            std::vector<std::thread> th;
            for (int t = 0; t < nt; ++t)
                th.emplace_back([&, t, bx, by]() {
                    threadIdx.x = flat ? (unsigned)t : (unsigned)(t % 32);
                    threadIdx.y = flat ? 0u : (unsigned)(t / 32);
                    blockIdx.x = (unsigned)bx;
                    blockIdx.y = (unsigned)by;
                    body();
                    emu_warp_barrier[t / 32]->arrive_and_drop();
                    bar.arrive_and_drop();
                });
            for (auto& x : th) x.join();
            for (int w = 0; w < nt / 32; ++w) delete emu_warp_barrier[w];
        }
}

int main(int argc, char** argv) {
    if (argc != 12) return 1;
    Geo G{};
    for (int a = 0; a < 3; ++a) {
        G.n[a] = atoi(argv[1 + a]);
        G.bc[a] = atoi(argv[4 + a]);
    }
    const int batch = atoi(argv[7]);
    const double vol = atof(argv[8]), dt = atof(argv[9]);
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a)
            G.ext[c][a] = G.n[a] + ((c == a && G.bc[a] != BC_PERIODIC) ? 1 : 0);
    for (int c = 0; c < 3; ++c) G.cnt[c] = (long long)G.ext[c][0] * G.ext[c][1] * G.ext[c][2];
    G.cnt[3] = (long long)G.n[0] * G.n[1] * G.n[2];
    FILE* f = fopen(argv[10], "rb");
    if (!f) return 3;
    std::vector<double> u[3], mu[3], acc[3];
    for (int c = 0; c < 3; ++c) {
        const size_t n = (size_t)batch * G.cnt[c];
        for (auto* v : {&u[c], &mu[c], &acc[c]}) {
            v->resize(n);
            if (fread(v->data(), 8, n, f) != n) return 4;
        }
    }
    fclose(f);
    FILE* out = fopen(argv[11], "wb");
    if (!out) return 5;
    std::vector<double> J((size_t)batch, 0.0);
    // the same CTA count for every component, about a third of the largest
    // component's faces per pass of the grid-stride loops
    long long most = std::max(G.cnt[0], std::max(G.cnt[1], G.cnt[2]));
    const int gx = (int)std::max<long long>(1, most / (3 * NTHREADS));
    std::vector<double> part((size_t)batch * 3 * gx, -7.0);
    for (int c = 0; c < 3; ++c) {
        const size_t n = (size_t)batch * G.cnt[c];
        std::vector<double> lam(n, -7.0), lam2(n, -7.0);
        launch(gx, batch, NTHREADS, false,
               [&] { k_adj_terminal<double>(G, c, u[c].data(), lam.data(), part.data(), vol); });
        const int gf = (int)std::max<long long>(1, (long long)n / (3 * 256));
        launch(gf, 1, 256, true, [&] {
            k_adj_finish<double>(G, c, (long long)n, mu[c].data(), acc[c].data(), lam2.data(), dt);
        });
        fwrite(lam.data(), 8, n, out);
        fwrite(lam2.data(), 8, n, out);
        fwrite(acc[c].data(), 8, n, out);
    }
    launch(1, 1, 32, true, [&] { k_adj_sum(part.data(), 3 * gx, batch, J.data(), 0); });
    fwrite(J.data(), 8, J.size(), out);
    fclose(out);
    return 0;
}
