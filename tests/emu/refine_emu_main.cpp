// Driver of the host emulation of the float-float refinement kernels (test
// support): the start of a refined solve (k_mg_refine_init_ff from a warm
// start), an outer correction (k_mg_refine_update_ff) and the velocity
// correction with the float-float pressure (k_correct_ff), one state, every
// CTA as host threads.
//
// usage: refine_emu nx ny nz bcx bcy bcz lbox dt unscale fsc in.bin out.bin
//   lbox: the box length along every axis (h = lbox / n).
//   in.bin (cells C, faces Fu, Fv, Fw): b [C] FP64, then FP32: w_hi, w_lo, e, p_hi,
//   p_lo, r_hi, r_lo, q_hi, q_lo [C each], F*u [Fu], F*v [Fv], F*w [Fw], then
//   FP64: rmean, mean.
//   out.bin, FP32 unless noted: init p_hi p_lo r_hi r_lo r32 rhat; update p_hi
//   p_lo r_hi r_lo r32 rhat; correct u v w, p_out (FP64), w_hi w_lo q_hi q_lo;
//   then FP64, for the start and for the correction: o_bb, o_rr, bb, tol2_in,
//   status, o_status of the control block (the start with otol2 1e-4, the
//   correction with 1e-30; itol2 1e-8 both).

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

int main(int argc, char** argv) {
    if (argc != 13) return 1;
    const double lbox = atof(argv[7]);
    Geo G{};
    Lev L{};
    for (int a = 0; a < 3; ++a) {
        G.n[a] = atoi(argv[1 + a]);
        G.bc[a] = atoi(argv[4 + a]);
        G.h[a] = lbox / G.n[a];
        G.ih[a] = 1.0 / G.h[a];
        G.ih2[a] = 1.0 / (G.h[a] * G.h[a]);
        L.n[a] = G.n[a];
        L.bc[a] = G.bc[a];
        L.ih2[a] = G.ih2[a];
        L.fih2[a] = (float)L.ih2[a];
        L.lih2[a] = (float)(L.ih2[a] - (double)L.fih2[a]);
    }
    const double dt = atof(argv[8]);
    const float unscale = (float)atof(argv[9]), fsc = (float)atof(argv[10]);
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
    G.fbx = (G.n[0] + 1 + TX - 1) / TX;
    G.fby = (G.n[1] + 1 + TY - 1) / TY;
    G.fbz = (G.n[2] + 1 + G.tz - 1) / G.tz;
    G.fctas = G.fbx * G.fby * G.fbz;
    G.n_fluid = (int)G.cnt[3];
    L.cells = G.cnt[3];
    L.tz = G.tz;
    L.bx = G.bx;
    L.by = G.by;
    L.bz = G.bz;
    L.ctas = G.ctas;
    const long long C = G.cnt[3];
    FILE* f = fopen(argv[11], "rb");
    if (!f) return 3;
    std::vector<double> b(C);
    std::vector<float> wh(C), wl(C), e(C), ph(C), pl(C), rh(C), rl(C), qh(C), ql(C);
    std::vector<float> fs[3] = {std::vector<float>(G.cnt[0]), std::vector<float>(G.cnt[1]),
                                std::vector<float>(G.cnt[2])};
    double means[2];
    bool ok = fread(b.data(), 8, C, f) == (size_t)C;
    for (auto* v : {&wh, &wl, &e, &ph, &pl, &rh, &rl, &qh, &ql}) ok = ok && fread(v->data(), 4, C, f) == (size_t)C;
    for (auto& v : fs) ok = ok && fread(v.data(), 4, v.size(), f) == v.size();
    ok = ok && fread(means, 8, 2, f) == 2;
    fclose(f);
    if (!ok) return 4;
    FILE* out = fopen(argv[12], "wb");
    std::vector<double> decisions;
    auto keep = [&](const SliceCtl& c) {
        for (double v : {c.o_bb, c.o_rr, c.bb, c.tol2_in, (double)c.status, (double)c.o_status})
            decisions.push_back(v);
    };
    // start of a refined solve from the warm start w
    {
        std::vector<float> Ph(C), Pl(C), Rh(C), Rl(C), r32(C), rhat(C), x(C, 0.0f), Wh = wh, Wl = wl;
        std::vector<double> part_b((size_t)L.ctas, 0.0), part((size_t)L.ctas * 6, 0.0);
        for (double v : b) part_b[0] += v;
        std::vector<unsigned> counter(1, 0u);
        SliceCtl ctl{};
        MgBuf<float> mb{};
        mb.x = x.data();
        mb.r = r32.data();
        mb.rhat = rhat.data();
        mb.counter = counter.data();
        FFBuf fb{Ph.data(), Pl.data(), Rh.data(), Rl.data(), Wh.data(), Wl.data(), nullptr, nullptr};
        launch(L.ctas, [&] {
            k_mg_refine_init_ff<false>(L, mb, &ctl, part_b.data(), (int)C, b.data(), nullptr, fb,
                                       part.data(), 1e-4, 1e-8, 100);
        });
        for (auto* v : {&Ph, &Pl, &Rh, &Rl, &r32, &rhat}) put(out, *v);
        keep(ctl);
    }
    // one outer correction p += e / s, r -= L e / s (minus the residual's mean)
    {
        std::vector<float> Ph = ph, Pl = pl, Rh = rh, Rl = rl, r32(C), rhat(C), x = e;
        std::vector<double> part((size_t)L.ctas * 6, 0.0);
        std::vector<unsigned> counter(1, 0u);
        SliceCtl ctl{};
        ctl.o_status = OS_REFINE;
        ctl.status = ST_CONV;
        ctl.o_funs = unscale;
        ctl.o_fsc = fsc;
        const FF rm = ff_from_double(means[0]);
        ctl.rmean_hi = rm.hi;
        ctl.rmean_lo = rm.lo;
        ctl.o_bb = 1.0;
        MgBuf<float> mb{};
        mb.x = x.data();
        mb.r = r32.data();
        mb.rhat = rhat.data();
        mb.counter = counter.data();
        FFBuf fb{Ph.data(), Pl.data(), Rh.data(), Rl.data(), nullptr, nullptr, nullptr, nullptr};
        launch(L.ctas, [&] {
            k_mg_refine_update_ff(L, mb, &ctl, fb, (int)C, part.data(), 1e-30, 1e-8, 100, 40, 0);
        });
        for (auto* v : {&Ph, &Pl, &Rh, &Rl, &r32, &rhat}) put(out, *v);
        keep(ctl);
    }
    // velocity correction with the float-float pressure, gauged output, warm start
    {
        std::vector<float> Ph = ph, Pl = pl, Wh(C), Wl(C), Qh = qh, Ql = ql;
        std::vector<float> vel[3] = {std::vector<float>(G.cnt[0]), std::vector<float>(G.cnt[1]),
                                     std::vector<float>(G.cnt[2])};
        std::vector<double> pout(C, 0.0);
        SliceCtl ctl{};
        const FF m = ff_from_double(means[1]);
        ctl.mean_hi = m.hi;
        ctl.mean_lo = m.lo;
        FFBuf fb{Ph.data(), Pl.data(), nullptr, nullptr, Wh.data(), Wl.data(), Qh.data(), Ql.data()};
        const float3 dtih{(float)(dt * G.ih[0]), (float)(dt * G.ih[1]), (float)(dt * G.ih[2])};
        launch(G.fctas, [&] {
            k_correct_ff<false>(G, &ctl, fs[0].data(), fs[1].data(), fs[2].data(), vel[0].data(),
                                vel[1].data(), vel[2].data(), fb, pout.data(), dtih, 1);
        });
        for (auto& v : vel) put(out, v);
        put(out, pout);
        for (auto* v : {&Wh, &Wl, &Qh, &Ql}) put(out, *v);
    }
    put(out, decisions);
    fclose(out);
    return 0;
}
