// Driver of the host emulation of the kernels that start and close a pressure
// solve (test support), one state, every CTA as host threads:
//   k_sum_cells       partial sums of the right side;
//   k_bicg_init_warm  FP64 BiCGStab start from a warm start;
//   k_refine_init     FP64 outer start of the FP32 + refinement solve;
//   k_inner_init      outer convergence test and the inner FP32 start;
//   k_refine_update   outer correction p += e, r = b - L p;
//   k_mg_init_warm    FP64 start of the multigrid-preconditioned solve.
//
// usage: start_emu nx ny nz bcx bcy bcz in.bin solid.bin|- out.bin
//   in.bin (C cells): b, x0, p, p_old [C each] FP64, then e [C] FP32;
//   solid.bin: the solid flags [C] (u8) and the face codes of the finest
//   multigrid level [C] (u8).
//   out.bin: FP64 b1 x r rhat | b2 p64 | FP32 r32 | FP32 rhat e | FP64 pnew |
//   FP32 r32 | FP64 b3 x r rhat.
//   stdout: "name value" lines (partial sums, SliceCtl fields).

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
static void put(FILE* f, const std::vector<T>& v) {
    fwrite(v.data(), sizeof(T), v.size(), f);
}

static double total(const std::vector<double>& part, int nv, int which) {
    double s = 0.0;
    for (size_t q = which; q < part.size(); q += nv) s += part[q];
    return s;
}

static void show(const char* name, double v) { printf("%s %.17g\n", name, v); }

static void show_ctl(const char* tag, const SliceCtl& c) {
    char nm[64];
    const std::pair<const char*, double> f[] = {
        {"status", c.status},     {"it_cur", c.it_cur}, {"it_next", c.it_next},
        {"omega", c.omega},       {"alpha", c.alpha},   {"o_status", c.o_status},
        {"o_steps", c.o_steps},   {"p_final", c.p_final}, {"o_bb", c.o_bb},
        {"o_rr", c.o_rr},         {"sx", c.sx},         {"rr", c.rr},
        {"bb", c.bb},             {"beta", c.beta},     {"rho0", c.rho[0]},
        {"restart", c.restart}};
    for (const auto& kv : f) {
        snprintf(nm, sizeof nm, "%s.%s", tag, kv.first);
        show(nm, kv.second);
    }
}

int main(int argc, char** argv) {
    if (argc != 10) return 1;
    Geo G{};
    Lev L{};
    for (int a = 0; a < 3; ++a) {
        G.n[a] = atoi(argv[1 + a]);
        G.bc[a] = atoi(argv[4 + a]);
        G.h[a] = 1.0 / G.n[a];
        G.ih[a] = 1.0 / G.h[a];
        G.ih2[a] = 1.0 / (G.h[a] * G.h[a]);
        L.n[a] = G.n[a];
        L.bc[a] = G.bc[a];
        L.ih2[a] = G.ih2[a];
        L.fih2[a] = (float)L.ih2[a];
        L.lih2[a] = (float)(L.ih2[a] - (double)L.fih2[a]);
    }
    for (int c = 0; c < 3; ++c)
        for (int a = 0; a < 3; ++a)
            G.ext[c][a] = G.n[a] + ((c == a && G.bc[a] != BC_PERIODIC) ? 1 : 0);
    for (int c = 0; c < 3; ++c) G.cnt[c] = (long long)G.ext[c][0] * G.ext[c][1] * G.ext[c][2];
    G.cnt[3] = (long long)G.n[0] * G.n[1] * G.n[2];
    G.tz = std::min(8, G.n[2]);
    G.bx = (G.n[0] + TX - 1) / TX;
    G.by = (G.n[1] + TY - 1) / TY;
    G.bz = (G.n[2] + G.tz - 1) / G.tz;
    G.ctas = G.bx * G.by * G.bz;
    G.n_fluid = (int)G.cnt[3];
    L.cells = G.cnt[3];
    L.tz = G.tz;
    L.bx = G.bx;
    L.by = G.by;
    L.bz = G.bz;
    L.ctas = G.ctas;
    L.rbx = (G.n[0] + 31) / 32;
    L.rby = (G.n[1] + 7) / 8;
    L.rctas = L.rbx * L.rby * L.bz;
    const long long C = G.cnt[3];
    std::vector<double> b(C), x0(C), p(C), pold(C);
    std::vector<float> e(C);
    FILE* f = fopen(argv[7], "rb");
    bool ok = f != nullptr;
    for (auto* v : {&b, &x0, &p, &pold}) ok = ok && fread(v->data(), 8, C, f) == (size_t)C;
    ok = ok && fread(e.data(), 4, C, f) == (size_t)C;
    if (f) fclose(f);
    if (!ok) return 3;
    std::vector<uint8_t> solid, code;
    if (strcmp(argv[8], "-") != 0) {
        solid.resize(C);
        code.resize(C);
        f = fopen(argv[8], "rb");
        ok = f && fread(solid.data(), 1, C, f) == (size_t)C && fread(code.data(), 1, C, f) == (size_t)C;
        if (f) fclose(f);
        if (!ok) return 4;
        G.solid = solid.data();
        L.fcode = code.data();
        for (uint8_t m : solid) G.n_fluid -= m ? 1 : 0;
    }
    FILE* out = fopen(argv[9], "wb");
    if (!out) return 5;
    const double tol2 = 1e-24;

    // partial sums of the right side
    std::vector<double> part_b((size_t)G.ctas, -1.0);
    launch(G.ctas, [&] { k_sum_cells(G, b.data(), part_b.data()); });
    show("sum_b", total(part_b, 1, 0));

    // FP64 BiCGStab start from x0
    {
        std::vector<double> b1 = b, x(C, -1.0), r(C, -1.0), rh(C, -1.0);
        std::vector<double> part((size_t)G.ctas * 4, -1.0);
        KBuf<double> kb{};
        kb.x = x.data();
        kb.r = r.data();
        kb.rhat = rh.data();
        SliceCtl ctl{};
        ctl.status = ST_IDLE;
        ctl.it_cur = ctl.it_next = 7;
        launch(G.ctas, [&] {
            k_bicg_init_warm<double>(G, kb, &ctl, part_b.data(), b1.data(), x0.data(), part.data());
        });
        for (auto* v : {&b1, &x, &r, &rh}) put(out, *v);
        for (int q = 0; q < 4; ++q) {
            char nm[32];
            snprintf(nm, sizeof nm, "init.part%d", q);
            show(nm, total(part, 4, q));
        }
        show_ctl("init", ctl);
    }

    // FP64 outer start of the refined solve, then the inner FP32 start
    std::vector<double> part_r((size_t)G.ctas * 3, -1.0);
    std::vector<float> r32(C, -1.0f);
    {
        std::vector<double> b2 = b, p64(C, -1.0);
        SliceCtl ctl{};
        ctl.status = ST_ITER;
        ctl.o_status = OS_FAIL;
        ctl.p_final = 1;
        launch(G.ctas, [&] {
            k_refine_init(G, &ctl, part_b.data(), b2.data(), p.data(), p64.data(), r32.data(),
                          part_r.data());
        });
        put(out, b2);
        put(out, p64);
        put(out, r32);
        for (int q = 0; q < 3; ++q) {
            char nm[32];
            snprintf(nm, sizeof nm, "rinit.part%d", q);
            show(nm, total(part_r, 3, q));
        }
        show_ctl("rinit", ctl);
    }
    {
        // m = 0, not converged: the inner start
        std::vector<float> rh(C, -1.0f), ev(C, -1.0f);
        std::vector<double> part((size_t)G.ctas * 4, -1.0);
        KBuf<float> kb{};
        kb.x = ev.data();
        kb.r = r32.data();
        kb.rhat = rh.data();
        SliceCtl ctl{};
        ctl.status = ST_IDLE;
        ctl.o_status = OS_REFINE;
        ctl.o_bb = -5.0;
        launch(G.ctas, [&] {
            k_inner_init(G, kb, &ctl, part_r.data(), part.data(), tol2, 0, 5);
        });
        put(out, rh);
        put(out, ev);
        for (int q = 0; q < 4; ++q) {
            char nm[32];
            snprintf(nm, sizeof nm, "inner.part%d", q);
            show(nm, total(part, 4, q));
        }
        show_ctl("inner", ctl);
        // m = 3 with a threshold the residual meets: converged, p_final = 1;
        // m = 5 = the outer limit: failure; both leave the vectors alone
        const int ms[2] = {3, 5};
        const double tols[2] = {1e30, tol2};
        const char* tags[2] = {"iconv", "ifail"};
        for (int t = 0; t < 2; ++t) {
            std::vector<float> rh2(C, -1.0f), e2(C, -1.0f);
            kb.x = e2.data();
            kb.rhat = rh2.data();
            SliceCtl c2{};
            c2.status = ST_CONV;
            c2.o_status = OS_REFINE;
            c2.o_bb = 2.0;
            launch(G.ctas, [&] {
                k_inner_init(G, kb, &c2, part_r.data(), part.data(), tols[t], ms[t], 5);
            });
            bool untouched = true;
            for (long long q = 0; q < C; ++q) untouched = untouched && rh2[q] == -1.0f && e2[q] == -1.0f;
            char nm[32];
            snprintf(nm, sizeof nm, "%s.untouched", tags[t]);
            show(nm, untouched ? 1.0 : 0.0);
            show_ctl(tags[t], c2);
        }
    }
    // outer correction p = p_old + e, r32 = float(b - L p)
    {
        std::vector<double> pn(C, -1.0), part((size_t)G.ctas * 3, -1.0);
        std::vector<float> r(C, -1.0f);
        SliceCtl ctl{};
        ctl.o_status = OS_REFINE;
        ctl.status = ST_CONV;
        launch(G.ctas, [&] {
            k_refine_update(G, &ctl, b.data(), pold.data(), pn.data(), e.data(), r.data(), part.data());
        });
        put(out, pn);
        put(out, r);
        for (int q = 0; q < 3; ++q) {
            char nm[32];
            snprintf(nm, sizeof nm, "rupd.part%d", q);
            show(nm, total(part, 3, q));
        }
        show_ctl("rupd", ctl);
    }
    // FP64 start of the multigrid-preconditioned solve (last-CTA decision)
    {
        std::vector<double> b3 = b, x(C, -1.0), r(C, -1.0), rh(C, -1.0);
        std::vector<double> part((size_t)L.ctas * 3, -1.0);
        std::vector<unsigned> counter(1, 0u);
        MgBuf<double> mb{};
        mb.x = x.data();
        mb.r = r.data();
        mb.rhat = rh.data();
        mb.counter = counter.data();
        SliceCtl ctl{};
        ctl.status = ST_IDLE;
        ctl.it_cur = 9;
        ctl.omega = 0.5;
        ctl.alpha = 0.25;
        ctl.p_final = 1;
        launch(L.ctas, [&] {
            k_mg_init_warm<double>(L, mb, &ctl, part_b.data(), G.n_fluid, b3.data(), x0.data(),
                                   part.data(), tol2, 50);
        });
        for (auto* v : {&b3, &x, &r, &rh}) put(out, *v);
        show("mginit.counter", counter[0]);
        show_ctl("mginit", ctl);
    }
    fclose(out);
    return 0;
}
