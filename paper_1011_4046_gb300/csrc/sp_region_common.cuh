// sp_region_common.cuh -- device helpers shared by the region kernels: the
// decode of a launch-global region id and the release of a finished
// region's successors (the manager's side of the work queue, paper Sec. 4).
#pragma once
#include "sp_device.cuh"

namespace sp {

__device__ __forceinline__ int wrap_axis(int p, int n)
{
    p += (p < 0) ? n : 0;
    p -= (p >= n) ? n : 0;
    return p;
}

// Region descriptor decoded from a launch-global region id.
struct RegionInfo {
    int sim, band, S, jl, j[3];
};

__device__ __forceinline__ int find_sim_in(const SimDev *sims, int n_sims, unsigned g)
{
    int lo = 0, hi = n_sims - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sims[mid].tile_base <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ RegionInfo decode_region(const SimDev *sims, int n_sims, int g)
{
    RegionInfo r;
    r.sim = find_sim_in(sims, n_sims, (unsigned)g);
    const SimDev &sd = sims[r.sim];
    const unsigned local = (unsigned)g - sd.tile_base;
    const unsigned per_band = 8u * (unsigned)sd.Jtot;
    r.band = (int)(local / per_band);
    const int rem = (int)(local - (unsigned)r.band * per_band);
    r.S = rem / sd.Jtot;
    r.jl = rem - r.S * sd.Jtot;
    r.j[0] = r.jl % sd.J[0];
    r.j[1] = (r.jl / sd.J[0]) % sd.J[1];
    r.j[2] = r.jl / (sd.J[0] * sd.J[1]);
    return r;
}

// One lane per successor: acq_rel decrement of its counter, push at zero.
// Called by the 32 lanes of one warp after the whole CTA finished the region.
// Ordering: the workers' surface writes precede (bar.sync, then a CTA-scope
// release/acquire of the done flag) lane 0's observation of the done flag;
// __syncwarp extends that to every lane, and each lane's GPU-scope acq_rel
// decrement (and the release store of a push) carries it to the successor's
// CTA, so no separate fence is needed.
static __device__ void release_successors(const RegionArgs &a, const SimDev &sd, const TablesDev &T, const RegionInfo &r,
                                   int lane, unsigned long long t_start, int g)
{
    __syncwarp();
    if (g == a.fault_drop) return;  // injected failure: completion is never reported downstream
    // successors: same band, then the next band's (an inverted pyramid's
    // 27), then with a single mailbox slot the next band's writers of this
    // region's mailbox; one lane each, in passes of 32
    const int n_same = T.type[r.S].n_same_succ;
    const int n_next = (r.S == kTypes - 1 && r.band + 1 < sd.nbands) ? kMaxNextSucc : 0;
    const int n_reuse = (sd.mb_reuse && r.band + 1 < sd.nbands) ? T.type[r.S].n_reuse : 0;
    const int n_all = n_same + n_next + n_reuse;
    for (int p = 0; p < n_all; p += 32) {
        const int i = p + lane;
        bool ready = false;
        int region = -1;
        if (i < n_all) {
            Succ su;
            int nb = r.band + 1;
            if (i < n_same) {
                su = T.type[r.S].same_succ[i];
                nb = r.band;
            } else if (i < n_same + n_next) {
                su = T.next_succ[(r.band + 1) & 1][i - n_same];
            } else {
                su = T.reuse[r.S * kMaxSameSucc + (i - n_same - n_next)];
            }
            int jc = 0, mul = 1;
            for (int d = 0; d < 3; ++d) {
                int v = r.j[d] + su.e[d];
                v += (v < 0) ? sd.J[d] : 0;
                v -= (v >= sd.J[d]) ? sd.J[d] : 0;
                jc += v * mul;
                mul *= sd.J[d];
            }
            const unsigned t = sd.tile_base + (unsigned)((nb * 8 + su.type) * sd.Jtot + jc);
            const int old = atom_add_acq_rel_gpu(a.counters + t, -1);
            ready = old == 1;
            region = (int)t;
        }
        // push the successors made ready here with one queue-tail atomic per
        // warp (every manager of the launch pushes at the same tail); the
        // learned ordering pushes them bucket by bucket
        for (int q = 0; q < (a.prio ? kBuckets : 1); ++q) {
            const bool mine = ready && (a.prio == nullptr || a.prio[region] == q);
            const unsigned m = __ballot_sync(0xffffffffu, mine);
            if (m == 0) continue;
            const int leader = __ffs((int)m) - 1;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(&a.ctl->tail, (unsigned)__popc(m));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (mine) st_release_gpu(a.queue + base + __popc(m & ((1u << lane) - 1u)), region);
        }
    }
    (void)t_start;
}

__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }


}  // namespace sp
