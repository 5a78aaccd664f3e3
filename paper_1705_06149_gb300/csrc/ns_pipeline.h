// Issue order of Parareal iterations pipelined across iterations (host logic,
// no CUDA): the fine sweep of the slices in C chunks on one stream, the serial
// coarse chain with the update of Eq. 6 on another, ordered by events.
//
// SW(k, c), the sweep of chunk c in iteration k, copies y^{k-1} of the chunk's
// slices into the chunk's F buffers and sweeps them in place; CH(k, c), the
// chain of chunk c, reads those F values and y of the chunk's first slice and
// writes y of its other slices and of the next chunk's first slice.  Hence
//   SW(k, c) after CH(k-1, c)   (y^{k-1} written, the old F values consumed),
//   CH(k, c) after SW(k, c)     (the new F values),
//   CH(k, c) after SW(k, c+1)'s copy (it overwrites y of chunk c+1's first slice),
// and the chains of an iteration, like the sweeps, in chunk order on their
// stream.  An event wait takes the event's latest record at the time it is
// issued, so the host issues SW(k, c) before CH(k, c-1) and CH(k, c) before
// SW(k+1, c).  The sweep of chunk 0 of iteration k+1 is issued before the
// defect of iteration k is known (it writes only F buffers); with a defect
// tolerance the host reads each iteration's defect before it issues the next
// iteration's chains and later sweeps.
#pragma once

namespace nsk {

enum PipeStream { PS_SWEEP = 0, PS_CHAIN = 1 };
enum PipeEvent { PE_COPIED = 0, PE_SWEPT = 1, PE_CHAINED = 2 };

// P provides, each returning false on failure:
//   wait(stream, event, chunk), record(stream, event, chunk)  -- one event per (kind, chunk)
//   copy_in(chunk)        on PS_SWEEP: y of the chunk's slices -> its F buffers
//   sweep(chunk)          on PS_SWEEP: the chunk's fine sweep, in place
//   defect_reset()        on PS_CHAIN: the iteration's defect accumulator to 0
//   chain(chunk)          on PS_CHAIN: the chunk's coarse steps and updates
//   defect_out(k)         on PS_CHAIN: iteration k's defect to host slot k
//   converged(k) -> int   host: waits for slot k; 1 stop, 0 go on, -1 failure
// Returns the iterations whose chains were issued, or -1 on a failure.
template <class P>
int pipeline_issue(int C, int kmax, bool check_defects, P& p) {
    auto sweep = [&](int k, int c) -> bool {
        if (k > 0 && !p.wait(PS_SWEEP, PE_CHAINED, c)) return false;
        return p.copy_in(c) && p.record(PS_SWEEP, PE_COPIED, c) && p.sweep(c) &&
               p.record(PS_SWEEP, PE_SWEPT, c);
    };
    auto chain = [&](int k, int c) -> bool {
        if (!p.wait(PS_CHAIN, PE_SWEPT, c)) return false;
        if (c + 1 < C && !p.wait(PS_CHAIN, PE_COPIED, c + 1)) return false;
        if (c == 0 && !p.defect_reset()) return false;
        if (!p.chain(c) || !p.record(PS_CHAIN, PE_CHAINED, c)) return false;
        return c + 1 < C || p.defect_out(k);
    };
    if (kmax <= 0) return 0;
    if (!sweep(0, 0)) return -1;
    int k = 0;
    for (; k < kmax; ++k) {
        if (check_defects && k > 0) {
            const int d = p.converged(k - 1);
            if (d < 0) return -1;
            if (d > 0) break;
        }
        for (int c = 1; c < C; ++c)
            if (!sweep(k, c) || !chain(k, c - 1)) return -1;
        if (!chain(k, C - 1)) return -1;
        if (k + 1 < kmax && !sweep(k + 1, 0)) return -1;
    }
    return k;
}

}  // namespace nsk
