// Driver of the host emulation of the adjoint right side (test support):
// k_adj_rhs, out = (dR/du)^T mu and the per-CTA partials of (dR/du_lid)^T mu
// for one state (the three components as grid z-slices), then k_adj_sum over
// the partials; every CTA as host threads.
// prec "d" runs the FP64 kernel, "f" the FP32 one on the inputs rounded to
// FP32.
//
// usage: adj_emu prec nx ny nz bcx bcy bcz re u_lid in.bin out.bin
//   in.bin: u, v, w, then mu_u, mu_v, mu_w (FP64); out.bin: the three adjoint
//   right sides, then dlid (FP64).

#include <functional>

static void launch(int gx, const std::function<void()>& body) {
    for (int bx = 0; bx < gx; ++bx) {
        std::barrier<> bar(NTHREADS);
        emu_cta_barrier = &bar;
        for (int w = 0; w < NWARPS; ++w) emu_warp_barrier[w] = new std::barrier<>(32);
        std::vector<std::thread> th;
        for (int t = 0; t < NTHREADS; ++t)
            th.emplace_back([&, t, bx]() {
                threadIdx.x = (unsigned)(t % TX);
                threadIdx.y = (unsigned)(t / TX);
                blockIdx.x = (unsigned)bx;
                blockIdx.y = 0;
                body();
                emu_warp_barrier[t / 32]->arrive_and_drop();
                bar.arrive_and_drop();
            });
        for (auto& x : th) x.join();
        for (int w = 0; w < NWARPS; ++w) delete emu_warp_barrier[w];
    }
}

template <typename T>
static int run(const Geo& G, const std::vector<double>& in, std::vector<double>& out,
               double& dlid) {
    const long long nv = G.cnt[0] + G.cnt[1] + G.cnt[2];
    std::vector<T> u(in.begin(), in.begin() + nv), mu(in.begin() + nv, in.end());
    std::vector<T> o(nv, T(-7));
    const int ctas = G.fbx * G.fby * ((G.n[2] + 1 + ADJ_TZ - 1) / ADJ_TZ);
    std::vector<double> part(3 * ctas, -7.0);
    gridDim.x = (unsigned)ctas;
    for (int c = 0; c < 3; ++c)
        launch(ctas, [&] {
            blockIdx.z = (unsigned)c;
            k_adj_rhs<T>(G, u.data(), u.data() + G.cnt[0], u.data() + G.cnt[0] + G.cnt[1],
                         mu.data(), mu.data() + G.cnt[0], mu.data() + G.cnt[0] + G.cnt[1],
                         o.data(), o.data() + G.cnt[0], o.data() + G.cnt[0] + G.cnt[1],
                         part.data());
        });
    blockDim.x = 32;
    blockDim.y = 1;
    threadIdx.x = 0;
    threadIdx.y = 0;
    blockIdx.x = 0;
    blockIdx.z = 0;
    k_adj_sum(part.data(), 3 * ctas, 1, &dlid, 0);
    out.assign(o.begin(), o.end());
    return 0;
}

int main(int argc, char** argv) {
    if (argc != 12) return 1;
    const char prec = argv[1][0];
    argv += 1;
    Geo G{};
    for (int a = 0; a < 3; ++a) {
        G.n[a] = atoi(argv[1 + a]);
        G.bc[a] = atoi(argv[4 + a]);
        G.h[a] = 1.0 / G.n[a];
        G.ih[a] = 1.0 / G.h[a];
        G.ih2[a] = 1.0 / (G.h[a] * G.h[a]);
        G.fih[a] = (float)G.ih[a];
        G.fih2[a] = (float)G.ih2[a];
    }
    G.inv_re = 1.0 / atof(argv[7]);
    G.finv_re = (float)G.inv_re;
    G.u_lid = atof(argv[8]);
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a)
            G.ext[c][a] = G.n[a] + ((c == a && G.bc[a] != BC_PERIODIC) ? 1 : 0);
    for (int c = 0; c < 3; ++c) G.cnt[c] = (long long)G.ext[c][0] * G.ext[c][1] * G.ext[c][2];
    G.cnt[3] = (long long)G.n[0] * G.n[1] * G.n[2];
    G.tz = std::min(8, G.n[2]);
    G.fbx = (G.n[0] + 1 + TX - 1) / TX;
    G.fby = (G.n[1] + 1 + TY - 1) / TY;
    G.fbz = (G.n[2] + 1 + G.tz - 1) / G.tz;
    G.fctas = G.fbx * G.fby * G.fbz;
    const long long nv = G.cnt[0] + G.cnt[1] + G.cnt[2];
    std::vector<double> in(2 * nv);
    FILE* f = fopen(argv[9], "rb");
    if (!f || fread(in.data(), 8, in.size(), f) != in.size()) return 3;
    fclose(f);
    std::vector<double> out;
    double dlid = 0.0;
    const int rc = prec == 'f' ? run<float>(G, in, out, dlid) : run<double>(G, in, out, dlid);
    if (rc) return rc;
    f = fopen(argv[10], "wb");
    if (!f) return 5;
    fwrite(out.data(), 8, out.size(), f);
    fwrite(&dlid, 8, 1, f);
    fclose(f);
    return 0;
}
