// Driver of the cluster host emulation (test support): builds the multigrid
// plan of a grid as the library does (halve every extent while all are even
// and >= 4; the one-CTA levels from the first level with at most block_cells
// cells), the cluster plan for C CTAs (cl_plan), runs k_mg_cluster for one
// state on C x nt host threads, and writes the result.
//
// usage: cluster_emu T nx ny nz bcx bcy bcz C nt in.bin out.bin
//   T: f (float) or d (double); in.bin: the right side on the cluster's first
//   level J, x fastest ("-": print the plan only); prints "J R C nlev" and the
//   extents of levels J ..

template <typename T>
static int run(const int n0[3], const int bcs[3], int C, int nt, const char* fin,
               const char* fout) {
    MgPlan P{};
    Lev L0{};
    for (int a = 0; a < 3; ++a) {
        L0.n[a] = n0[a];
        L0.bc[a] = bcs[a];
        L0.ih2[a] = double(n0[a]) * n0[a];
        L0.fih2[a] = (float)L0.ih2[a];
        L0.lih2[a] = (float)(L0.ih2[a] - (double)L0.fih2[a]);
    }
    L0.cells = (long long)n0[0] * n0[1] * n0[2];
    P.lev[0] = L0;
    P.nlev = 1;
    while (P.nlev < MG_MAX_LEVELS) {
        const Lev& L = P.lev[P.nlev - 1];
        bool ok = true;
        for (int a = 0; a < 3; ++a) ok = ok && L.n[a] % 2 == 0 && L.n[a] >= 4;
        if (!ok) break;
        Lev Cl{};
        for (int a = 0; a < 3; ++a) {
            Cl.n[a] = L.n[a] / 2;
            Cl.bc[a] = L.bc[a];
            Cl.ih2[a] = L.ih2[a] * 0.25;
            Cl.fih2[a] = (float)Cl.ih2[a];
            Cl.lih2[a] = (float)(Cl.ih2[a] - (double)Cl.fih2[a]);
        }
        Cl.cells = (long long)Cl.n[0] * Cl.n[1] * Cl.n[2];
        P.lev[P.nlev++] = Cl;
    }
    const long long block_cells = sizeof(T) == 4 ? 4096 : 512;
    P.lc = P.nlev - 1;
    for (int m = 0; m < P.nlev; ++m)
        if (P.lev[m].cells <= block_cells) {
            P.lc = m;
            break;
        }
    ClPlan Q{};
    size_t bytes = 0;
    if (!cl_plan(P, C, nt, sizeof(T), 200 * 1024, Q, bytes)) {
        fprintf(stderr, "no cluster plan\n");
        return 5;
    }
    if ((long long)MG_BLOCK_PER_THREAD * nt < P.lev[Q.R].cells) {
        fprintf(stderr, "too few threads for the rank-0 levels\n");
        return 6;
    }
    auto print_plan = [&]() {
        printf("%d %d %d %d", Q.J, Q.R, Q.C, P.nlev);
        for (int m = Q.J; m < P.nlev; ++m)
            printf(" %d %d %d", P.lev[m].n[0], P.lev[m].n[1], P.lev[m].n[2]);
        printf("\n");
    };
    if (std::strcmp(fin, "-") == 0) {
        print_plan();
        return 0;
    }
    const Lev& LJ = P.lev[Q.J];
    std::vector<T> in(LJ.cells), out(LJ.cells, T(-12345));
    FILE* f = fopen(fin, "rb");
    if (!f || fread(in.data(), sizeof(T), in.size(), f) != in.size()) return 3;
    fclose(f);
    emu_cl_smem.assign(C, nullptr);
    // poison the blocks: a value read before it is written shows in the result
    for (int r = 0; r < C; ++r) {
        emu_cl_smem[r] = new unsigned char[bytes];
        std::vector<T> nan(bytes / sizeof(T), std::nan(""));
        std::memcpy(emu_cl_smem[r], nan.data(), nan.size() * sizeof(T));
    }
    SliceCtl ctl{};
    ctl.status = ST_ITER;
    blockDim.x = (unsigned)nt;
    gridDim.x = (unsigned)C;
    gridDim.y = 1;
    std::barrier<> cl_bar(C * nt);
    emu_cl_barrier = &cl_bar;
    std::vector<std::barrier<>*> cta(C);
    for (int r = 0; r < C; ++r) cta[r] = new std::barrier<>(nt);
    for (int w = 0; w < 32; ++w) emu_warp_barrier[w] = new std::barrier<>(32);
    std::vector<std::thread> th;
    for (int r = 0; r < C; ++r)
        for (int t = 0; t < nt; ++t)
            th.emplace_back([&, r, t]() {
                threadIdx.x = (unsigned)t;
                blockIdx.x = (unsigned)r;
                blockIdx.y = 0;
                emu_rank = r;
                emu_smem = emu_cl_smem[r];
                emu_cta_barrier = cta[r];
                k_mg_cluster<T>(P, Q, &ctl, in.data(), out.data());
            });
    for (auto& x : th) x.join();
    for (int r = 0; r < C; ++r) {
        delete[] emu_cl_smem[r];
        delete cta[r];
    }
    for (int w = 0; w < 32; ++w) delete emu_warp_barrier[w];
    f = fopen(fout, "wb");
    if (!f || fwrite(out.data(), sizeof(T), out.size(), f) != out.size()) return 4;
    fclose(f);
    print_plan();
    return 0;
}

int main(int argc, char** argv) {
    if (argc != 12) return 1;
    const int n0[3] = {atoi(argv[2]), atoi(argv[3]), atoi(argv[4])};
    const int bcs[3] = {atoi(argv[5]), atoi(argv[6]), atoi(argv[7])};
    const int C = atoi(argv[8]), nt = atoi(argv[9]);
    if (argv[1][0] == 'd') return run<double>(n0, bcs, C, nt, argv[10], argv[11]);
    return run<float>(n0, bcs, C, nt, argv[10], argv[11]);
}
