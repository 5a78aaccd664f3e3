// Driver of the host emulation of the loop-condition kernel of the
// graph-resident pressure solves (test support): k_loop_cond as one warp of
// host threads, the graph's conditional handle replaced by a variable.
//
// usage: loop_emu in.txt
//   in.txt: mode cap inner inner_total batch, then per state: status o_status
//   o_steps fail total_outer total_solves.
//   stdout: cond inner inner_total, then per state: fail total_outer total_solves.

int main(int argc, char** argv) {
    if (argc != 2) return 1;
    FILE* f = fopen(argv[1], "r");
    if (!f) return 2;
    int mode, batch;
    unsigned cap, inner;
    unsigned long long inner_total;
    if (fscanf(f, "%d %u %u %llu %d", &mode, &cap, &inner, &inner_total, &batch) != 5) return 3;
    std::vector<SliceCtl> ctl((size_t)batch);
    for (auto& c : ctl) {
        c = SliceCtl{};
        long long to, ts;
        if (fscanf(f, "%d %d %d %d %lld %lld", &c.status, &c.o_status, &c.o_steps, &c.fail, &to,
                   &ts) != 6)
            return 4;
        c.total_outer = to;
        c.total_solves = ts;
    }
    fclose(f);
    LoopCount lc{};
    lc.inner = inner;
    lc.inner_total = inner_total;
    std::barrier<> bar(32);
    emu_cta_barrier = &bar;
    emu_warp_barrier[0] = new std::barrier<>(32);
    std::vector<std::thread> th;
    for (int t = 0; t < 32; ++t)
        th.emplace_back([&, t]() {
            threadIdx.x = (unsigned)t;
            threadIdx.y = 0;
            blockIdx.x = blockIdx.y = 0;
            k_loop_cond(ctl.data(), batch, &lc, 7ull, mode, cap);
            emu_warp_barrier[0]->arrive_and_drop();
            bar.arrive_and_drop();
        });
    for (auto& x : th) x.join();
    delete emu_warp_barrier[0];
    printf("%u %u %llu\n", emu_cond, lc.inner, lc.inner_total);
    for (const auto& c : ctl) printf("%d %lld %lld\n", c.fail, c.total_outer, c.total_solves);
    return 0;
}
