// Driver of the host emulation of the projection kernels (test support): the
// divergence of F* (k_divergence) and the velocity correction with the
// gauged pressure (k_correct), FP64, one state, every CTA as host threads.
//
// usage: proj_emu nx ny nz bcx bcy bcz dt in.bin solid.bin|- out.bin
//   in.bin: F* (u, v, w) and p (FP64, canonical layout) one after another;
//   out.bin: b, then the corrected u, v, w, then the gauged p.

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

int main(int argc, char** argv) {
    if (argc != 11) return 1;
    Geo G{};
    for (int a = 0; a < 3; ++a) {
        G.n[a] = atoi(argv[1 + a]);
        G.bc[a] = atoi(argv[4 + a]);
        G.h[a] = 1.0 / G.n[a];
        G.ih[a] = 1.0 / G.h[a];
        G.ih2[a] = 1.0 / (G.h[a] * G.h[a]);
        G.fih[a] = (float)G.ih[a];
    }
    const double dt = atof(argv[7]);
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a)
            G.ext[c][a] = G.n[a] + ((c == a && G.bc[a] != BC_PERIODIC) ? 1 : 0);
    for (int c = 0; c < 3; ++c) G.cnt[c] = (long long)G.ext[c][0] * G.ext[c][1] * G.ext[c][2];
    G.cnt[3] = (long long)G.n[0] * G.n[1] * G.n[2];
    G.inv_re = 1.0;
    G.tz = std::min(8, G.n[2]);
    G.bx = (G.n[0] + TX - 1) / TX;
    G.by = (G.n[1] + TY - 1) / TY;
    G.bz = (G.n[2] + G.tz - 1) / G.tz;
    G.ctas = G.bx * G.by * G.bz;
    G.fbx = (G.n[0] + 1 + TX - 1) / TX;
    G.fby = (G.n[1] + 1 + TY - 1) / TY;
    G.fbz = (G.n[2] + 1 + G.tz - 1) / G.tz;
    G.fctas = G.fbx * G.fby * G.fbz;
    const long long nv = G.cnt[0] + G.cnt[1] + G.cnt[2];
    std::vector<double> in(nv + G.cnt[3]);
    FILE* f = fopen(argv[8], "rb");
    if (!f || fread(in.data(), sizeof(double), in.size(), f) != in.size()) return 3;
    fclose(f);
    std::vector<uint8_t> mask;
    G.n_fluid = (int)G.cnt[3];
    if (strcmp(argv[9], "-") != 0) {
        mask.resize(G.cnt[3]);
        f = fopen(argv[9], "rb");
        if (!f || fread(mask.data(), 1, mask.size(), f) != mask.size()) return 4;
        fclose(f);
        G.solid = mask.data();
        for (uint8_t m : mask) G.n_fluid -= m ? 1 : 0;
    }
    const double* fu = in.data();
    const double* fv = fu + G.cnt[0];
    const double* fw = fv + G.cnt[1];
    const double* p = fw + G.cnt[2];
    std::vector<double> b(G.cnt[3], -12345.0), part((size_t)G.ctas, 0.0);
    launch(G.ctas, [&] {
        k_divergence<double>(G, fu, fv, fw, nullptr, nullptr, nullptr, b.data(), part.data(), 1.0 / dt);
    });
    double sb = 0.0, bsum = 0.0;
    for (double x : part) sb += x;
    for (double x : b) bsum += x;
    printf("partials %.17g %.17g", sb, bsum);
    // the FP32 storage: F* rounded to FP32, b as the float-float product
    std::vector<float> f32(in.begin(), in.begin() + nv);
    std::vector<double> b32(G.cnt[3], -12345.0), part32((size_t)G.ctas, 0.0);
    launch(G.ctas, [&] {
        k_divergence<float>(G, f32.data(), f32.data() + G.cnt[0], f32.data() + G.cnt[0] + G.cnt[1],
                            nullptr, nullptr, nullptr, b32.data(), part32.data(), 1.0 / dt);
    });
    double sb32 = 0.0, bsum32 = 0.0;
    for (double x : part32) sb32 += x;
    for (double x : b32) bsum32 += x;
    printf(" %.17g %.17g\n", sb32, bsum32);
    SliceCtl ctl{};
    ctl.p_final = 0;
    for (long long q = 0; q < G.cnt[3]; ++q)
        if (G.solid == nullptr || !G.solid[q]) ctl.sx += p[q];
    std::vector<double> vel(nv, -12345.0), pout(G.cnt[3], 0.0);
    double* u = vel.data();
    double* v = u + G.cnt[0];
    double* w = v + G.cnt[1];
    launch(G.fctas, [&] {
        k_correct<double, false>(G, &ctl, fu, fv, fw, u, v, w, p, nullptr, pout.data(), dt);
    });
    f = fopen(argv[10], "wb");
    if (!f || fwrite(b.data(), sizeof(double), b.size(), f) != b.size() ||
        fwrite(vel.data(), sizeof(double), vel.size(), f) != vel.size() ||
        fwrite(pout.data(), sizeof(double), pout.size(), f) != pout.size() ||
        fwrite(b32.data(), sizeof(double), b32.size(), f) != b32.size())
        return 5;
    fclose(f);
    return 0;
}
