// Driver of the host emulation of the finest-level multigrid kernels (test
// support).  Every CTA of a grid runs as TX x TY std::threads (the CTAs one
// after another); a thread that leaves the kernel drops out of the CTA's and
// its warp's barriers, as an exited GPU thread does.  For one level without
// solid cells and two states it runs each x-pair kernel and the one-cell-per-
// thread kernel it stands in for on copies of the same seeded inputs, and
// prints one line per comparison: "name max_abs_diff scale" (the largest
// difference of the compared outputs and the largest magnitude among them).
//
// usage: pair_emu nx ny nz bcx bcy bcz tz

#include <functional>

static constexpr int EMU_B = 2;  // states

static void launch(int gx, int gy, const std::function<void()>& body) {
    for (int by = 0; by < gy; ++by)
        for (int bx = 0; bx < gx; ++bx) {
            std::barrier<> bar(NTHREADS);
            emu_cta_barrier = &bar;
            for (int w = 0; w < NWARPS; ++w) emu_warp_barrier[w] = new std::barrier<>(32);
            std::vector<std::thread> th;
            for (int t = 0; t < NTHREADS; ++t)
                th.emplace_back([&, t, bx, by]() {
                    threadIdx.x = (unsigned)(t % TX);
                    threadIdx.y = (unsigned)(t / TX);
                    blockIdx.x = (unsigned)bx;
                    blockIdx.y = (unsigned)by;
                    body();
                    emu_warp_barrier[t / 32]->arrive_and_drop();
                    bar.arrive_and_drop();
                });
            for (auto& x : th) x.join();
            for (int w = 0; w < NWARPS; ++w) delete emu_warp_barrier[w];
        }
}

static unsigned long long emu_rng = 88172645463325252ull;
static float rnd() {
    emu_rng ^= emu_rng << 13;
    emu_rng ^= emu_rng >> 7;
    emu_rng ^= emu_rng << 17;
    return (float)((emu_rng >> 11) * (1.0 / 9007199254740992.0)) - 0.5f;
}

static void fill_level(Lev& L, const int n[3], const int bc[3], int tz, double ih2_scale) {
    L = Lev{};
    for (int a = 0; a < 3; ++a) {
        L.n[a] = n[a];
        L.bc[a] = bc[a];
        L.ih2[a] = double(n[a]) * n[a] * ih2_scale;
        L.fih2[a] = (float)L.ih2[a];
        L.lih2[a] = (float)(L.ih2[a] - (double)L.fih2[a]);
    }
    L.cells = (long long)n[0] * n[1] * n[2];
    L.tz = std::min(std::max(tz, 2), n[2]);
    L.bx = (n[0] + TX - 1) / TX;
    L.by = (n[1] + TY - 1) / TY;
    L.bz = (n[2] + L.tz - 1) / L.tz;
    L.ctas = L.bx * L.by * L.bz;
    L.rbx = (n[0] + 31) / 32;
    L.rby = (n[1] + 7) / 8;
    L.rctas = L.rbx * L.rby * L.bz;
}

struct Bufs {
    std::vector<float> x, r, rhat, P0, P1, V0, V1, Y, Z, S, Tt, barr;
    std::vector<double> part;
    std::vector<unsigned> counter;
    std::vector<SliceCtl> ctl;
    MgBuf<float> mb() {
        MgBuf<float> m{};
        m.x = x.data();
        m.r = r.data();
        m.rhat = rhat.data();
        m.P[0] = P0.data();
        m.P[1] = P1.data();
        m.V[0] = V0.data();
        m.V[1] = V1.data();
        m.Y = Y.data();
        m.Z = Z.data();
        m.S = S.data();
        m.Tt = Tt.data();
        m.counter = counter.data();
        return m;
    }
};

static Bufs make_bufs(long long cells, int ctas, int restart, int it_cur) {
    Bufs b;
    for (auto* v : {&b.x, &b.r, &b.rhat, &b.P0, &b.P1, &b.V0, &b.V1, &b.Y, &b.Z, &b.S, &b.Tt,
                    &b.barr}) {
        v->resize((size_t)cells * EMU_B);
        for (auto& e : *v) e = rnd();
    }
    b.part.assign((size_t)ctas * EMU_B * 6, 0.0);
    b.counter.assign(EMU_B, 0u);
    b.ctl.assign(EMU_B, SliceCtl{});
    for (int s = 0; s < EMU_B; ++s) {
        SliceCtl& c = b.ctl[s];
        c.status = ST_ITER;
        c.it_cur = it_cur + s;  // the two states take opposite parities
        c.restart = restart;
        c.alpha = 0.7 + 0.1 * s;
        c.omega = 0.45 - 0.05 * s;
        c.beta = 0.3 + 0.02 * s;
        c.rho[0] = 1.7;
        c.bb = 1e30;  // no convergence decision
    }
    return b;
}

static void report(const char* name, const std::vector<float>& a, const std::vector<float>& b) {
    double d = 0.0, m = 0.0;
    for (size_t q = 0; q < a.size(); ++q) {
        d = std::max(d, (double)std::fabs(a[q] - b[q]));
        m = std::max(m, (double)std::fabs(a[q]));
    }
    printf("%s %.17g %.17g\n", name, d, m);
}

static void report_scalar(const char* name, double a, double b) {
    printf("%s %.17g %.17g\n", name, std::fabs(a - b), std::fabs(a));
}

int main(int argc, char** argv) {
    if (argc != 8) return 1;
    const int n[3] = {atoi(argv[1]), atoi(argv[2]), atoi(argv[3])};
    const int bc[3] = {atoi(argv[4]), atoi(argv[5]), atoi(argv[6])};
    const int tz = atoi(argv[7]);
    Lev L;
    fill_level(L, n, bc, tz, 1.0);
    const int pbx = (n[0] + 63) / 64;
    const int pctas = pbx * L.by * L.bz;
    const long long cells = L.cells;
    // BiCGStab phases A (fresh and restarted) and B, and the smoothing of a
    // coarse level's right side: y and the stored source
    for (int mode = 0; mode < 4; ++mode) {
        const int restart = mode == 1;
        Bufs a = make_bufs(cells, L.ctas, restart, 1), b = a;
        MgBuf<float> ma = a.mb(), mbb = b.mb();
        if (mode <= 1) {
            launch(L.ctas, EMU_B, [&] { k_mg_src<float, SRC_P, true>(L, ma, a.ctl.data(), nullptr, a.Y.data()); });
            launch(pctas, EMU_B, [&] { k_mg_src_pair<float, SRC_P>(L, mbb, b.ctl.data(), nullptr, b.Y.data(), pbx); });
        } else if (mode == 2) {
            launch(L.ctas, EMU_B, [&] { k_mg_src<float, SRC_S, true>(L, ma, a.ctl.data(), nullptr, a.Y.data()); });
            launch(pctas, EMU_B, [&] { k_mg_src_pair<float, SRC_S>(L, mbb, b.ctl.data(), nullptr, b.Y.data(), pbx); });
        } else {
            launch(L.ctas, EMU_B, [&] { k_mg_src<float, SRC_ARR, true>(L, ma, a.ctl.data(), a.barr.data(), a.Y.data()); });
            launch(pctas, EMU_B, [&] { k_mg_src_pair<float, SRC_ARR>(L, mbb, b.ctl.data(), b.barr.data(), b.Y.data(), pbx); });
        }
        char nm[64];
        snprintf(nm, sizeof nm, "src%d_y", mode);
        report(nm, a.Y, b.Y);
        snprintf(nm, sizeof nm, "src%d_p", mode);
        report(nm, a.P0, b.P0);
        snprintf(nm, sizeof nm, "src%d_p1", mode);
        report(nm, a.P1, b.P1);
        snprintf(nm, sizeof nm, "src%d_s", mode);
        report(nm, a.S, b.S);
        snprintf(nm, sizeof nm, "src%d_rhat", mode);
        report(nm, a.rhat, b.rhat);
    }
    // L y with (r_hat, v) and L z with (t, s), (t, t)
    {
        Bufs a = make_bufs(cells, std::max(L.ctas, pctas), 0, 1), b = a;
        MgBuf<float> ma = a.mb(), mbb = b.mb();
        launch(L.ctas, EMU_B, [&] { k_mg_lapdot_v<float>(L, ma, a.ctl.data(), a.part.data()); });
        launch(pctas, EMU_B, [&] { k_mg_lapdot_pair<float, 0>(L, mbb, b.ctl.data(), b.part.data(), pbx, pctas); });
        report("lapv_v0", a.V0, b.V0);
        report("lapv_v1", a.V1, b.V1);
        for (int s = 0; s < EMU_B; ++s) report_scalar("lapv_alpha", a.ctl[s].alpha, b.ctl[s].alpha);
        launch(L.ctas, EMU_B, [&] { k_mg_lapdot_t<float>(L, ma, a.ctl.data(), a.part.data()); });
        launch(pctas, EMU_B, [&] { k_mg_lapdot_pair<float, 1>(L, mbb, b.ctl.data(), b.part.data(), pbx, pctas); });
        report("lapt_t", a.Tt, b.Tt);
        for (int s = 0; s < EMU_B; ++s) report_scalar("lapt_omega", a.ctl[s].omega, b.ctl[s].omega);
    }
    // phase C: x, r and the three sums behind the convergence decision
    for (int zero = 0; zero < 2; ++zero) {
        Bufs a = make_bufs(cells, std::max(L.ctas, pctas), 0, 0), b = a;
        MgBuf<float> ma = a.mb(), mbb = b.mb();
        launch(L.ctas, EMU_B, [&] { k_mg_update<float>(L, ma, a.ctl.data(), a.part.data(), 1e-30, 100, zero); });
        launch(pctas, EMU_B, [&] { k_mg_update_pair<float>(L, mbb, b.ctl.data(), b.part.data(), 1e-30, 100, zero, pbx, pctas); });
        report(zero ? "upd0_x" : "upd_x", a.x, b.x);
        report(zero ? "upd0_r" : "upd_r", a.r, b.r);
        for (int s = 0; s < EMU_B; ++s) {
            report_scalar("upd_rr", a.ctl[s].rr, b.ctl[s].rr);
            report_scalar("upd_sx", a.ctl[s].sx, b.ctl[s].sx);
            report_scalar("upd_rho", a.ctl[s].rho[0], b.ctl[s].rho[0]);
        }
    }
    // prolongation from the next level (y += P e) and restriction to it
    {
        const int nc[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
        Lev Lc;
        fill_level(Lc, nc, bc, tz, 0.25);
        Bufs a = make_bufs(cells, L.ctas, 0, 1), b = a;
        std::vector<float> e((size_t)Lc.cells * EMU_B);
        for (auto& v : e) v = rnd();
        launch(L.ctas, EMU_B, [&] { k_mg_prolong<float>(L, Lc, a.ctl.data(), a.Y.data(), e.data()); });
        launch(pbx * L.by * L.bz, EMU_B, [&] { k_mg_prolong_pair<float>(L, Lc, b.ctl.data(), b.Y.data(), e.data(), pbx); });
        report("prolong_y", a.Y, b.Y);
        // restriction against a plain loop: the mean of the 8 children's b - L y
        std::vector<float> bcoarse((size_t)Lc.cells * EMU_B, -1.0f);
        launch(L.rctas, EMU_B, [&] { k_mg_restrict<float>(L, Lc, a.ctl.data(), a.r.data(), nullptr, a.Y.data(), bcoarse.data()); });
        std::vector<float> want(bcoarse.size());
        for (int s = 0; s < EMU_B; ++s)
            for (int K = 0; K < nc[2]; ++K)
                for (int J = 0; J < nc[1]; ++J)
                    for (int I = 0; I < nc[0]; ++I) {
                        double acc = 0.0;
                        for (int dz = 0; dz < 2; ++dz)
                            for (int dy = 0; dy < 2; ++dy)
                                for (int dx = 0; dx < 2; ++dx) {
                                    const int c3[3] = {2 * I + dx, 2 * J + dy, 2 * K + dz};
                                    const float* y = a.Y.data() + (size_t)s * cells;
                                    const int id = (c3[2] * n[1] + c3[1]) * n[0] + c3[0];
                                    double lap = 0.0;
                                    for (int d = 0; d < 3; ++d) {
                                        int lo, hi, act;
                                        axis_nbr(c3[d], n[d], bc[d], lo, hi, act);
                                        int ql[3] = {c3[0], c3[1], c3[2]}, qh[3] = {c3[0], c3[1], c3[2]};
                                        ql[d] = lo;
                                        qh[d] = hi;
                                        const int il = (ql[2] * n[1] + ql[1]) * n[0] + ql[0];
                                        const int ih = (qh[2] * n[1] + qh[1]) * n[0] + qh[0];
                                        lap += ((double)y[ih] + y[il] - 2.0 * y[id]) * L.fih2[d];
                                    }
                                    acc += a.r[(size_t)s * cells + id] - lap;
                                }
                        want[(size_t)s * Lc.cells + (K * nc[1] + J) * nc[0] + I] = (float)(acc * 0.125);
                    }
        report("restrict_b", want, bcoarse);
    }
    return 0;
}
