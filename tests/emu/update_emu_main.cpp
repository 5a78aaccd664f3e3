// Driver of the host emulation of the Parareal update kernel (test support):
// k_parareal_update in FP64 over n values with `blocks` CTAs of 256 threads
// (grid-stride loop), the CTAs one after another.
//
// usage: update_emu n blocks in.bin out.bin
//   in.bin: F, G_new, G_old, y (n doubles each); out.bin: y, G_old, defect.

#include <functional>

int main(int argc, char** argv) {
    if (argc != 5) return 1;
    const long long n = atoll(argv[1]);
    const int blocks = atoi(argv[2]);
    std::vector<double> in(4 * n);
    FILE* f = fopen(argv[3], "rb");
    if (!f || fread(in.data(), sizeof(double), in.size(), f) != in.size()) return 3;
    fclose(f);
    const double* fy = in.data();
    const double* gnew = fy + n;
    double* gold = in.data() + 2 * n;
    double* y = in.data() + 3 * n;
    unsigned long long defect = 0;
    blockDim.x = 256;
    gridDim.x = (unsigned)blocks;
    for (int bx = 0; bx < blocks; ++bx) {
        std::barrier<> bar(256);
        emu_cta_barrier = &bar;
        for (int w = 0; w < 8; ++w) emu_warp_barrier[w] = new std::barrier<>(32);
        std::vector<std::thread> th;
        for (int t = 0; t < 256; ++t)
            th.emplace_back([&, t, bx]() {
                threadIdx.x = (unsigned)t;
                threadIdx.y = 0;
                blockIdx.x = (unsigned)bx;
                k_parareal_update<double>(n, fy, gnew, gold, y, &defect);
                emu_warp_barrier[t / 32]->arrive_and_drop();
                bar.arrive_and_drop();
            });
        for (auto& x : th) x.join();
        for (int w = 0; w < 8; ++w) delete emu_warp_barrier[w];
    }
    double dfct;
    std::memcpy(&dfct, &defect, sizeof dfct);
    f = fopen(argv[4], "wb");
    if (!f || fwrite(y, sizeof(double), n, f) != (size_t)n ||
        fwrite(gold, sizeof(double), n, f) != (size_t)n || fwrite(&dfct, sizeof(double), 1, f) != 1)
        return 5;
    fclose(f);
    return 0;
}
