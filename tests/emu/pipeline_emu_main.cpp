// Driver of the pipelined Parareal issue order (test support): runs
// pipeline_issue from csrc/ns_pipeline.h with primitives that print what the
// library would issue, one line each:
//   wait <S|C> <kind> <chunk> | record <S|C> <kind> <chunk> | copy <chunk> |
//   sweep <chunk> | reset | chain <chunk> | out <k> | conv <k> <answer>
// then "issued <iterations>".
//
// usage: pipeline_emu C kmax check_defects stop
//   stop: with check_defects, the defect of iteration k meets the tolerance
//   once k + 1 >= stop (0: never).
#include <cstdio>
#include <cstdlib>

#include "ns_pipeline.h"

using namespace nsk;

struct Rec {
    int stop;
    static char s(int stream) { return stream == PS_SWEEP ? 'S' : 'C'; }
    bool wait(int st, int kind, int c) { return std::printf("wait %c %d %d\n", s(st), kind, c) > 0; }
    bool record(int st, int kind, int c) {
        return std::printf("record %c %d %d\n", s(st), kind, c) > 0;
    }
    bool copy_in(int c) { return std::printf("copy %d\n", c) > 0; }
    bool sweep(int c) { return std::printf("sweep %d\n", c) > 0; }
    bool defect_reset() { return std::printf("reset\n") > 0; }
    bool chain(int c) { return std::printf("chain %d\n", c) > 0; }
    bool defect_out(int k) { return std::printf("out %d\n", k) > 0; }
    int converged(int k) {
        const int d = stop > 0 && k + 1 >= stop ? 1 : 0;
        std::printf("conv %d %d\n", k, d);
        return d;
    }
};

int main(int argc, char** argv) {
    if (argc != 5) return 1;
    const int C = std::atoi(argv[1]), kmax = std::atoi(argv[2]);
    Rec r{std::atoi(argv[4])};
    const int k = pipeline_issue(C, kmax, std::atoi(argv[3]) != 0, r);
    std::printf("issued %d\n", k);
    return 0;
}
