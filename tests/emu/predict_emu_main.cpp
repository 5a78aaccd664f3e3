// Driver of the host emulation of the predictors (test support): sets up the
// grid geometry as the library does for the unit box, runs k_predict_tile (no
// solid cells) or k_predict_masked (with a cell mask) in FP64 for one state,
// every CTA as host threads, and writes F* (or its increment).
//
// usage: predict_emu nx ny nz bcx bcy bcz re u_lid dt incr in.bin solid.bin|- out.bin [py pz]
//   in.bin: u, v, w (FP64, canonical layout) one after another; py pz: the
//   tile of k_predict_tile (default 8 4).

#include <functional>
#include <type_traits>

static void launch(int gx, int threads, const std::function<void()>& body, bool flat = false) {
    for (int bx = 0; bx < gx; ++bx) {
        std::barrier<> bar(threads);
        emu_cta_barrier = &bar;
        const int warps = (threads + 31) / 32;
        for (int w = 0; w < warps; ++w) emu_warp_barrier[w] = new std::barrier<>(32);
        std::vector<std::thread> th;
        for (int t = 0; t < threads; ++t)
            th.emplace_back([&, t, bx]() {
                threadIdx.x = (unsigned)(!flat && threads == NTHREADS ? t % TX : t);
                threadIdx.y = (unsigned)(!flat && threads == NTHREADS ? t / TX : 0);
                blockIdx.x = (unsigned)bx;
                blockIdx.y = 0;
                body();
                emu_warp_barrier[t / 32]->arrive_and_drop();
                bar.arrive_and_drop();
            });
        for (auto& x : th) x.join();
        for (int w = 0; w < warps; ++w) delete emu_warp_barrier[w];
    }
}

int main(int argc, char** argv) {
    if (argc != 14 && argc != 16) return 1;
    Geo G{};
    for (int a = 0; a < 3; ++a) {
        G.n[a] = atoi(argv[1 + a]);
        G.bc[a] = atoi(argv[4 + a]);
        G.h[a] = 1.0 / G.n[a];
        G.ih[a] = 1.0 / G.h[a];
        G.ih2[a] = 1.0 / (G.h[a] * G.h[a]);
    }
    const double re = atof(argv[7]), dt = atof(argv[9]);
    const int incr = atoi(argv[10]);
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a)
            G.ext[c][a] = G.n[a] + ((c == a && G.bc[a] != BC_PERIODIC) ? 1 : 0);
    for (int c = 0; c < 3; ++c) G.cnt[c] = (long long)G.ext[c][0] * G.ext[c][1] * G.ext[c][2];
    G.cnt[3] = (long long)G.n[0] * G.n[1] * G.n[2];
    G.inv_re = 1.0 / re;
    G.u_lid = atof(argv[8]);
    for (int a = 0; a < 3; ++a) {
        G.fih[a] = (float)G.ih[a];
        G.fih2[a] = (float)G.ih2[a];
    }
    G.finv_re = (float)G.inv_re;
    G.tz = std::min(8, G.n[2]);
    G.bx = (G.n[0] + TX - 1) / TX;
    G.by = (G.n[1] + TY - 1) / TY;
    G.bz = (G.n[2] + G.tz - 1) / G.tz;
    G.ctas = G.bx * G.by * G.bz;
    G.fbx = (G.n[0] + 1 + TX - 1) / TX;
    G.fby = (G.n[1] + 1 + TY - 1) / TY;
    G.fbz = (G.n[2] + 1 + G.tz - 1) / G.tz;
    G.fctas = G.fbx * G.fby * G.fbz;
    G.n_fluid = (int)G.cnt[3];
    std::vector<double> in(G.cnt[0] + G.cnt[1] + G.cnt[2]);
    FILE* f = fopen(argv[11], "rb");
    if (!f || fread(in.data(), sizeof(double), in.size(), f) != in.size()) return 3;
    fclose(f);
    std::vector<uint8_t> mask;
    if (strcmp(argv[12], "-") != 0) {
        mask.resize(G.cnt[3]);
        f = fopen(argv[12], "rb");
        if (!f || fread(mask.data(), 1, mask.size(), f) != mask.size()) return 4;
        fclose(f);
        G.solid = mask.data();
    }
    const double* u = in.data();
    const double* v = u + G.cnt[0];
    const double* w = v + G.cnt[1];
    std::vector<double> out(in.size(), -12345.0);
    double* fu = out.data();
    double* fv = fu + G.cnt[0];
    double* fw = fv + G.cnt[1];
    if (G.solid == nullptr) {
        const int py = argc > 15 ? atoi(argv[14]) : PT_Y, pz = argc > 15 ? atoi(argv[15]) : PT_Z;
        auto run = [&](auto py_c, auto pz_c) {
            constexpr int PY = decltype(py_c)::value, PZ = decltype(pz_c)::value;
            const int tbx = (G.n[0] + PT_X - 1) / PT_X, tby = (G.n[1] + PY - 1) / PY,
                      tbz = (G.n[2] + PZ - 1) / PZ;
            std::vector<unsigned char> smem(3 * ptile_elems<PY, PZ>() * sizeof(double));
            emu_smem = smem.data();
            if (incr)
                launch(tbx * tby * tbz, PT_X * PY, [&] { k_predict_tile<double, true, PY, PZ>(G, u, v, w, fu, fv, fw, dt, tbx, tby); }, true);
            else
                launch(tbx * tby * tbz, PT_X * PY, [&] { k_predict_tile<double, false, PY, PZ>(G, u, v, w, fu, fv, fw, dt, tbx, tby); }, true);
        };
        using I2 = std::integral_constant<int, 2>;
        using I4 = std::integral_constant<int, 4>;
        using I8 = std::integral_constant<int, 8>;
        using I16 = std::integral_constant<int, 16>;
        switch (py * 100 + pz) {
            case 404: run(I4{}, I4{}); break;
            case 408: run(I4{}, I8{}); break;
            case 802: run(I8{}, I2{}); break;
            case 808: run(I8{}, I8{}); break;
            case 1604: run(I16{}, I4{}); break;
            default: run(I8{}, I4{}); break;
        }
    } else {
        if (incr)
            launch(G.fctas, NTHREADS, [&] { k_predict_masked<double, true>(G, u, v, w, fu, fv, fw, dt); });
        else
            launch(G.fctas, NTHREADS, [&] { k_predict_masked<double, false>(G, u, v, w, fu, fv, fw, dt); });
    }
    f = fopen(argv[13], "wb");
    if (!f || fwrite(out.data(), sizeof(double), out.size(), f) != out.size()) return 5;
    fclose(f);
    return 0;
}
