// Driver of the host emulation (test support): builds the multigrid plan of a
// grid as the library does (halve every extent while all are even and >= 4;
// the one-CTA levels start at the first level with at most block_cells
// cells), runs k_mg_block for one state on MG_BLOCK_THREADS host threads, and
// writes the result.
//
// usage: block_emu T nx ny nz bcx bcy bcz block_cells in.bin out.bin
//   T: f (float) or d (double); in.bin: the right side on the first one-CTA
//   level, x fastest; prints "lc nlev n0 n1 n2 ..." of the one-CTA levels.

template <typename T>
static int run(const int n0[3], const int bcs[3], int block_cells, const char* fin,
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
        Lev C{};
        for (int a = 0; a < 3; ++a) {
            C.n[a] = L.n[a] / 2;
            C.bc[a] = L.bc[a];
            C.ih2[a] = L.ih2[a] * 0.25;
            C.fih2[a] = (float)C.ih2[a];
            C.lih2[a] = (float)(C.ih2[a] - (double)C.fih2[a]);
        }
        C.cells = (long long)C.n[0] * C.n[1] * C.n[2];
        P.lev[P.nlev++] = C;
    }
    P.lc = P.nlev - 1;
    for (int m = 0; m < P.nlev; ++m)
        if (P.lev[m].cells <= block_cells) {
            P.lc = m;
            break;
        }
    const Lev& Lc = P.lev[P.lc];
    if (Lc.cells > MG_BLOCK_MAX_CELLS) {
        fprintf(stderr, "first one-CTA level has %lld cells\n", Lc.cells);
        return 2;
    }
    size_t smem = 0;
    for (int m = P.lc; m < P.nlev; ++m) smem += 2 * (size_t)P.lev[m].cells * sizeof(T);
    std::vector<T> in(Lc.cells), out(Lc.cells, T(-12345));
    FILE* f = fopen(fin, "rb");
    if (!f || fread(in.data(), sizeof(T), in.size(), f) != in.size()) return 3;
    fclose(f);
    emu_smem = new unsigned char[smem];
    SliceCtl ctl{};
    ctl.status = ST_ITER;
    blockDim.x = MG_BLOCK_THREADS;
    gridDim.x = 1;
    std::barrier<> bar(MG_BLOCK_THREADS);
    emu_cta_barrier = &bar;
    for (int w = 0; w < 32; ++w) emu_warp_barrier[w] = new std::barrier<>(32);
    std::vector<std::thread> th;
    for (int t = 0; t < MG_BLOCK_THREADS; ++t)
        th.emplace_back([&, t]() {
            threadIdx.x = (unsigned)t;
            blockIdx.x = 0;
            k_mg_block<T>(P, &ctl, in.data(), nullptr, out.data());
        });
    for (auto& x : th) x.join();
    delete[] emu_smem;
    for (int w = 0; w < 32; ++w) delete emu_warp_barrier[w];
    f = fopen(fout, "wb");
    if (!f || fwrite(out.data(), sizeof(T), out.size(), f) != out.size()) return 4;
    fclose(f);
    printf("%d %d", P.lc, P.nlev);
    for (int m = P.lc; m < P.nlev; ++m)
        printf(" %d %d %d", P.lev[m].n[0], P.lev[m].n[1], P.lev[m].n[2]);
    printf("\n");
    return 0;
}

int main(int argc, char** argv) {
    if (argc != 11) return 1;
    const int n0[3] = {atoi(argv[2]), atoi(argv[3]), atoi(argv[4])};
    const int bcs[3] = {atoi(argv[5]), atoi(argv[6]), atoi(argv[7])};
    const int block_cells = atoi(argv[8]);
    if (argv[1][0] == 'd') return run<double>(n0, bcs, block_cells, argv[9], argv[10]);
    return run<float>(n0, bcs, block_cells, argv[9], argv[10]);
}
