// Driver of the host emulation of the finest multigrid level with solid
// cells (test support): the two-sweep smoothing of a right side
// (k_mg_src<double, SRC_ARR, true>), the restriction of the residual
// (k_mg_restrict) and the prolongation (k_mg_prolong) on a level whose face
// codes mark the faces between fluid cells, FP64, one state, every CTA as
// host threads.
//
// usage: masked_emu nx ny nz bcx bcy bcz in.bin out.bin
//   in.bin: face codes [C] (bytes), then FP64: b [C], y [C], coarse e [C/8],
//   y_p [C];  out.bin (FP64): smoothed y [C], coarse right side [C/8],
//   y_p + P e [C].

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

static void fill_level(Lev& L, const int n[3], const int bc[3], double ih2_scale) {
    L = Lev{};
    for (int a = 0; a < 3; ++a) {
        L.n[a] = n[a];
        L.bc[a] = bc[a];
        L.ih2[a] = double(n[a]) * n[a] * ih2_scale;
        L.fih2[a] = (float)L.ih2[a];
        L.lih2[a] = (float)(L.ih2[a] - (double)L.fih2[a]);
    }
    L.cells = (long long)n[0] * n[1] * n[2];
    L.tz = std::min(8, n[2]);
    L.bx = (n[0] + TX - 1) / TX;
    L.by = (n[1] + TY - 1) / TY;
    L.bz = (n[2] + L.tz - 1) / L.tz;
    L.ctas = L.bx * L.by * L.bz;
    L.rbx = (n[0] + 31) / 32;
    L.rby = (n[1] + 7) / 8;
    L.rctas = L.rbx * L.rby * L.bz;
}

int main(int argc, char** argv) {
    if (argc != 9) return 1;
    const int n[3] = {atoi(argv[1]), atoi(argv[2]), atoi(argv[3])};
    const int bc[3] = {atoi(argv[4]), atoi(argv[5]), atoi(argv[6])};
    const int nc[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    Lev L, Lc;
    fill_level(L, n, bc, 1.0);
    fill_level(Lc, nc, bc, 0.25);
    const long long C = L.cells, Cc = Lc.cells;
    std::vector<uint8_t> code(C);
    std::vector<double> b(C), y(C), e(Cc), yp(C);
    FILE* f = fopen(argv[7], "rb");
    bool ok = f && fread(code.data(), 1, C, f) == (size_t)C && fread(b.data(), 8, C, f) == (size_t)C &&
              fread(y.data(), 8, C, f) == (size_t)C && fread(e.data(), 8, Cc, f) == (size_t)Cc &&
              fread(yp.data(), 8, C, f) == (size_t)C;
    if (f) fclose(f);
    if (!ok) return 3;
    L.fcode = code.data();
    SliceCtl ctl{};
    ctl.status = ST_ITER;
    ctl.it_cur = 1;
    // the Krylov vectors a SRC_ARR smoothing does not read still need storage
    std::vector<double> dummy((size_t)C * 12, 0.0);
    std::vector<unsigned> counter(1, 0u);
    MgBuf<double> mb{};
    double* dp = dummy.data();
    mb.x = dp;
    mb.r = dp + C;
    mb.rhat = dp + 2 * C;
    mb.P[0] = dp + 3 * C;
    mb.P[1] = dp + 4 * C;
    mb.V[0] = dp + 5 * C;
    mb.V[1] = dp + 6 * C;
    mb.Y = dp + 7 * C;
    mb.Z = dp + 8 * C;
    mb.S = dp + 9 * C;
    mb.Tt = dp + 10 * C;
    mb.counter = counter.data();
    std::vector<double> ys(C, -12345.0), bcoarse(Cc, -12345.0);
    launch(L.ctas, [&] { k_mg_src<double, SRC_ARR, true>(L, mb, &ctl, b.data(), ys.data()); });
    launch(L.rctas, [&] { k_mg_restrict<double>(L, Lc, &ctl, b.data(), nullptr, y.data(), bcoarse.data()); });
    launch(L.ctas, [&] { k_mg_prolong<double>(L, Lc, &ctl, yp.data(), e.data()); });
    f = fopen(argv[8], "wb");
    if (!f) return 5;
    fwrite(ys.data(), 8, C, f);
    fwrite(bcoarse.data(), 8, Cc, f);
    fwrite(yp.data(), 8, C, f);
    fclose(f);
    return 0;
}
