// Driver of the host emulation of whole plain BiCGStab pressure solves (test
// support), one state, every CTA as host threads, the launch sequences of the
// library's host loops:
//   FP64:         k_sum_cells, k_bicg_init_warm, then k_bicg_A / B / C with
//                 parity it & 1 until the state stops iterating, then (without
//                 solid cells) the gauge k_noalloc_gauge;
//   FP32 + FP64 refinement: k_sum_cells, k_refine_init, then per outer step m
//                 k_inner_init, the FP32 phases A / B / C, k_refine_update
//                 into the other FP64 buffer.
//
// usage: krylov_emu nx ny nz bcx bcy bcz rtol maxit inner_rtol refine_rtol max_outer kmax
//                   in.bin solid.bin|- out.bin
//   kmax 0: the solves run to their ends; kmax > 0: exactly kmax iterations of
//   the FP64 solve and of the first inner solve, then one outer correction.
//   in.bin: b, x0 [cells each] FP64; solid.bin: the solid flags [cells] (u8).
//   out.bin, kmax 0: FP64 x, p (x minus its mean; zeros with solid cells), the
//   refined p; kmax > 0: FP64 x, r, then FP32 e, FP64 p_old + e, FP32 r32.
//   stdout: "name value" lines.

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

static void show(const char* name, double v) { printf("%s %.17g\n", name, v); }

template <typename T>
struct Vecs {
    std::vector<T> store;
    KBuf<T> kb{};
    explicit Vecs(long long C) : store((size_t)C * 8, T(-1)) {
        T* q = store.data();
        kb.x = q;
        kb.r = q + C;
        kb.rhat = q + 2 * C;
        kb.P[0] = q + 3 * C;
        kb.P[1] = q + 4 * C;
        kb.V[0] = q + 5 * C;
        kb.V[1] = q + 6 * C;
        kb.t = q + 7 * C;
    }
};

// the three phases per iteration until the state leaves ST_ITER (the host
// loops also stop a few iterations past the limit), or exactly kmax of them
template <typename T>
static int iterate(const Geo& G, KBuf<T> kb, SliceCtl& ctl, std::vector<double>& part_c,
                   double tol2, int maxit, int kmax) {
    std::vector<double> part_a((size_t)G.ctas, 0.0), part_b((size_t)G.ctas * 2, 0.0);
    int it = 1;
    for (;; ++it) {
        const int par = it & 1;
        launch(G.ctas, [&] {
            k_bicg_A<T>(G, kb, &ctl, part_c.data(), part_a.data(), tol2, maxit, par);
        });
        launch(G.ctas, [&] { k_bicg_B<T>(G, kb, &ctl, part_a.data(), part_b.data(), par); });
        launch(G.ctas, [&] { k_bicg_C<T>(G, kb, &ctl, part_b.data(), part_c.data(), par); });
        if (kmax > 0 ? it == kmax : (ctl.status != ST_ITER || it > maxit + 2)) break;
    }
    return it;
}

int main(int argc, char** argv) {
    if (argc != 16) return 1;
    Geo G{};
    for (int a = 0; a < 3; ++a) {
        G.n[a] = atoi(argv[1 + a]);
        G.bc[a] = atoi(argv[4 + a]);
        G.h[a] = 1.0 / G.n[a];
        G.ih[a] = 1.0 / G.h[a];
        G.ih2[a] = 1.0 / (G.h[a] * G.h[a]);
        G.fih2[a] = (float)G.ih2[a];  // the FP32 inner solves' weights
    }
    const double rtol = atof(argv[7]), inner_rtol = atof(argv[9]), refine_rtol = atof(argv[10]);
    const int maxit = atoi(argv[8]), max_outer = atoi(argv[11]), kmax = atoi(argv[12]);
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
    const long long C = G.cnt[3];
    std::vector<double> b(C), x0(C);
    FILE* f = fopen(argv[13], "rb");
    bool ok = f && fread(b.data(), 8, C, f) == (size_t)C && fread(x0.data(), 8, C, f) == (size_t)C;
    if (f) fclose(f);
    if (!ok) return 3;
    std::vector<uint8_t> solid;
    if (strcmp(argv[14], "-") != 0) {
        solid.resize(C);
        f = fopen(argv[14], "rb");
        ok = f && fread(solid.data(), 1, C, f) == (size_t)C;
        if (f) fclose(f);
        if (!ok) return 4;
        G.solid = solid.data();
        for (uint8_t m : solid) G.n_fluid -= m ? 1 : 0;
    }
    FILE* out = fopen(argv[15], "wb");
    if (!out) return 5;
    std::vector<double> part_div((size_t)G.ctas, 0.0);

    // FP64 solve
    {
        Vecs<double> v(C);
        std::vector<double> bc = b, part_c((size_t)G.ctas * 4, 0.0), p(C, 0.0);
        SliceCtl ctl{};
        launch(G.ctas, [&] { k_sum_cells(G, bc.data(), part_div.data()); });
        launch(G.ctas, [&] {
            k_bicg_init_warm<double>(G, v.kb, &ctl, part_div.data(), bc.data(), x0.data(),
                                     part_c.data());
        });
        const int launched = iterate<double>(G, v.kb, ctl, part_c, rtol * rtol, maxit, kmax);
        if (G.solid == nullptr && kmax == 0)
            launch(G.ctas, [&] { k_noalloc_gauge(G, &ctl, v.kb.x, p.data()); });
        fwrite(v.kb.x, 8, C, out);
        fwrite(kmax > 0 ? v.kb.r : p.data(), 8, C, out);
        show("fp64.status", ctl.status);
        show("fp64.iters", ctl.it_cur);
        show("fp64.launched", launched);
        show("fp64.total_iters", (double)ctl.total_iters);
        show("fp64.rr", ctl.rr);
        show("fp64.bb", ctl.bb);
        show("fp64.sx", ctl.sx);
        show("fp64.alpha", ctl.alpha);
        show("fp64.omega", ctl.omega);
        show("fp64.restart", ctl.restart);
    }
    // FP32 inner solves inside FP64 iterative refinement
    {
        Vecs<float> v(C);
        std::vector<double> bc = b, part_c((size_t)G.ctas * 4, 0.0), part_r((size_t)G.ctas * 3, 0.0);
        std::vector<double> p64[2] = {std::vector<double>(C, -1.0), std::vector<double>(C, -1.0)};
        SliceCtl ctl{};
        launch(G.ctas, [&] { k_sum_cells(G, bc.data(), part_div.data()); });
        launch(G.ctas, [&] {
            k_refine_init(G, &ctl, part_div.data(), bc.data(), x0.data(), p64[0].data(), v.kb.r,
                          part_r.data());
        });
        const double tol2 = refine_rtol * refine_rtol;
        int m = 0, inner_total = 0, corrections = 0;
        for (;; ++m) {
            launch(G.ctas, [&] {
                k_inner_init(G, v.kb, &ctl, part_r.data(), part_c.data(), tol2, m, max_outer);
            });
            if (ctl.o_status != OS_REFINE) break;
            corrections += 1;
            iterate<float>(G, v.kb, ctl, part_c, inner_rtol * inner_rtol, maxit, kmax);
            inner_total += ctl.it_cur;
            if (ctl.status == ST_NONFINITE) break;
            const std::vector<double>& po = p64[m & 1];
            std::vector<double>& pn = p64[(m + 1) & 1];
            launch(G.ctas, [&] {
                k_refine_update(G, &ctl, bc.data(), po.data(), pn.data(), v.kb.x, v.kb.r,
                                part_r.data());
            });
            if (kmax > 0) {  // one outer step: its inner iterate and the corrected p, r32
                fwrite(v.kb.x, 4, C, out);
                fwrite(pn.data(), 8, C, out);
                fwrite(v.kb.r, 4, C, out);
                show("ref.alpha", ctl.alpha);
                show("ref.omega", ctl.omega);
                break;
            }
        }
        if (kmax == 0) fwrite(p64[ctl.p_final].data(), 8, C, out);
        show("ref.o_status", ctl.o_status);
        show("ref.o_steps", ctl.o_steps);
        show("ref.m", m);
        show("ref.p_final", ctl.p_final);
        show("ref.o_rr", ctl.o_rr);
        show("ref.o_bb", ctl.o_bb);
        show("ref.sx", ctl.sx);
        show("ref.inner_total", inner_total);
        show("ref.corrections", corrections);
    }
    fclose(out);
    return 0;
}
