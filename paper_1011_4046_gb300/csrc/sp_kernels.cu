// sp_kernels.cu -- sm_103a kernels of the region-scheduled leapfrog.
//
//   reset_kernel   arms the dependency counters and seeds the ready queue
//   region_kernel  persistent: pops ready regions and evolves each on chip
//   sweep_kernel   monolithic whole-grid step (the comparator)
//   energy_*       FP64 energy of a stored state (deterministic reduction)
//   winding_kernel exact per-plaquette winding numbers and string counts
//
// All arithmetic of the evolution goes through sp::site_update (sp_update.h).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sp_device.cuh"
#include "sp_kernels.h"
#include "sp_region_common.cuh"

namespace sp {

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ int find_sim(const RegionArgs &a, unsigned g)
{
    int lo = 0, hi = a.n_sims - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (a.sims[mid].tile_base <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------ queue reset
// Region id of the t-th seed of the launch (t < n_seed): the seeds of a
// simulation are its first band-0 region ids (the types without same-band
// predecessors, which lead the type order).
__device__ __forceinline__ int seed_region(const RegionArgs &a, unsigned t)
{
    int lo = 0, hi = a.n_sims - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (a.sims[mid].seed_base <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return (int)(a.sims[lo].tile_base + (t - a.sims[lo].seed_base));
}

__global__ void reset_kernel(RegionArgs a)
{
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        a.ctl->head = 0;
        a.ctl->tail = a.n_seed;
        a.ctl->error = 0;
        a.ctl->error_info = 0;
        for (int b = 0; b < kBuckets; ++b) {
            a.ctl->bcount[b] = 0;
            a.ctl->bcursor[b] = 0;
        }
    }
    if (t >= a.total) return;
    const int s = find_sim(a, t);
    const SimDev &sd = a.sims[s];
    const TypeMeta *M = sd.tab->type;
    const unsigned local = t - sd.tile_base;
    const unsigned per_band = 8u * (unsigned)sd.Jtot;
    const unsigned band = local / per_band;
    const int S = (int)((local - band * per_band) / (unsigned)sd.Jtot);
    a.counters[t] = M[S].same_preds + (band > 0 ? M[S].prev_preds + (sd.mb_reuse ? M[S].reuse_preds : 0) : 0);
    // queue position t: the first n_seed positions hold the seeds (with the
    // learned ordering seed_kernel writes them, bucket by bucket)
    a.queue[t] = (t < a.n_seed && !a.prio) ? seed_region(a, t) : -1;
}

// Learned ordering: seeds per bucket (after reset_kernel zeroed the counts).
__global__ void seed_count_kernel(RegionArgs a)
{
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < a.n_seed) atomicAdd(&a.ctl->bcount[a.prio[seed_region(a, t)]], 1u);
}

// Learned ordering: the seeds in queue positions [0, n_seed),
// bucket 0 first (order within a bucket is immaterial).
__global__ void seed_kernel(RegionArgs a)
{
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_seed) return;
    const int v = seed_region(a, t);
    const int b = a.prio[v];
    unsigned base = 0;
    for (int q = 0; q < b; ++q) base += a.ctl->bcount[q];
    a.queue[base + atomicAdd(&a.ctl->bcursor[b], 1u)] = v;
}

// ------------------------------------------------------------ region kernel
// Warp-specialised persistent kernel.  Warp 0 is the manager (the paper's
// manager process, Sec. 4); the other NW threads are the worker that
// evolves one region at a time.
//
// Manager: while the workers evolve region R it waits (bounded) for the next
// queue position to be filled.  As soon as the workers report R done it hands
// them the next region and only then releases R's successors (GPU-scope fence,
// acq_rel decrements, push at zero), so the release overlaps the next
// region's work.  If the next region is not ready it releases R first (the
// next region may be one of R's successors).
//
// Worker shared memory, in order: two phi buffers (levels of alternating
// parity) of (B+2)^3 float2 for the region box plus its halo; one float4
// (pi, c) per own cell (B^3, slots permuted by pc_slot); the launch's tables
// (geometry and routing per region type); the band's level coefficients; the
// import lists.  The tables and import lists are copied once per launch and
// the simulation descriptor travels with the handoff, so no step of a region
// waits on a table read from global memory (export entries are read through
// L1, one level ahead).
//
// Copies: the band base and the band's coefficients are requested when the
// region starts (copy group 0), the sloped initial surface of level L
// (group L) at the start of level L-1, each landing directly in its final
// place (the level-L phi buffer, L & 1, and the (pi, c) array).  This is safe
// because the cells imported for level L lie outside everything levels L-2
// and L-1 read or write (checked on the host for every region type).  Before
// level k is computed a thread waits for groups 0..k-1.
//
// One worker barrier per level.  The face cells of level k-1 are exported
// after level k is computed, before the next barrier: they are read from the
// level-(k-1) buffer and from (pi, c) of cells outside A(k) (the planner checks
// this), while level k writes the other buffer and (pi, c) of A(k).  Their
// table entries are loaded into registers before the compute.
constexpr int kWorkerBarrier = 1;

static_assert(sizeof(SimDev) / 16 <= 32, "the manager warp copies a descriptor with one int4 per lane");

// Export entries of a level are loaded into registers before the compute of
// the next level (up to kExportPrefetch per worker thread); any remainder is
// read in batches.  Three cover the average level of base 16 with 256
// workers several times over; more cost registers and unrolled code for
// entries that rarely exist.
constexpr int kExportPrefetch = 3;
constexpr int kExportBatch = 4;
// Per worker count: independent cell updates in flight per thread (measured:
// one up to 128 workers, two for 256 and more; four were 3 % slower at base
// 16), and the CTAs per SM the registers are budgeted for.  64 and 128 workers
// serve base 8, whose small regions fit six and four CTAs per SM (an SM's
// throughput grows almost linearly with the regions it holds); 256 and more
// serve base 16, one CTA per SM.
__host__ __device__ constexpr int region_cells_per_step(int nw) { return nw <= 128 ? 1 : 2; }
__host__ __device__ constexpr int region_min_blocks(int nw) { return nw <= 64 ? 6 : nw <= 128 ? 4 : 1; }

__device__ __forceinline__ void export_one(int2 e, float2 *const *mb_of, const float2 *__restrict__ phi,
                                           const float4 *__restrict__ pc)
{
    float2 *mb = mb_of[(e.x >> 25) & 63];
    __stcg(mb + (e.y & 0xFFFF), phi[e.x & 0x1FFF]);
    if (e.x < 0) __stcg(reinterpret_cast<float4 *>(mb + ((unsigned)e.y >> 16)), pc[(e.x >> 13) & 0xFFF]);
}

template <int NW>
__device__ __forceinline__ void export_entries(const int2 *__restrict__ el, int ne, const int2 (&pre)[kExportPrefetch],
                                               float2 *const *mb_of, const float2 *__restrict__ phi,
                                               const float4 *__restrict__ pc, int wt)
{
#pragma unroll
    for (int u = 0; u < kExportPrefetch; ++u)
        if (wt + u * NW < ne) export_one(pre[u], mb_of, phi, pc);
    for (int base = wt + kExportPrefetch * NW; base < ne; base += kExportBatch * NW) {
        int2 e[kExportBatch];
#pragma unroll
        for (int u = 0; u < kExportBatch; ++u)
            if (base + u * NW < ne) e[u] = __ldg(el + base + u * NW);
#pragma unroll
        for (int u = 0; u < kExportBatch; ++u)
            if (base + u * NW < ne) export_one(e[u], mb_of, phi, pc);
    }
}

template <int NW>
__device__ __forceinline__ void prefetch_entries(const int2 *__restrict__ el, int ne, int2 (&pre)[kExportPrefetch],
                                                 int wt)
{
#pragma unroll
    for (int u = 0; u < kExportPrefetch; ++u)
        if (wt + u * NW < ne) pre[u] = __ldg(el + wt + u * NW);
}

// Sloped initial surface of one level: mailbox chunk -> its places in shared
// memory ((pi, c) and phi of full cells, phi of neighbour-only cells).  The
// lists are in shared memory; a full cell's phi index follows from its
// (pi, c) index.
template <int NW>
__device__ __forceinline__ void import_level(const float2 *__restrict__ mb, int nf, int np,
                                             const unsigned short *fl, const unsigned short *pl, float2 *dst,
                                             float4 *pc_s, int B, int P, int wt)
{
    const int lgB = 31 - __clz(B);  // B is a power of two (4, 8 or 16)
    for (int i = wt; i < nf; i += NW) {
        const int c = fl[i];
        const int pidx = (((c >> (2 * lgB)) + 1) * P + ((c >> lgB) & (B - 1)) + 1) * P + (c & (B - 1)) + 1;
        cp_async16(pc_s + pc_slot(c, lgB, B), mb + 2 * i);
        cp_async8(dst + pidx, mb + 2 * nf + i);
    }
    for (int i = wt; i < np; i += NW) cp_async8(dst + pl[i], mb + 3 * nf + i);
}

// The cells of level k are taken in 2x2x2 blocks (every extent of an active
// box is even): linear index j -> block m = j >> 3, counted z fastest, then x,
// then y (a = w0/2 and c = w2/2 blocks along x and z; rc = 1/c, ra = 1/a),
// and corner j & 7 of the block.  Eight consecutive threads then cover one
// block: a block pair along z spans all sixteen 8-byte bank pairs of a phi
// buffer (pitch B+2 = 2 mod 16 cells, plane pitch = 4 mod 16), and pc_slot
// gives the block's eight (pi, c) pairs eight different bank groups.
__device__ __forceinline__ void block_cell(int j, const Box3 &A, int a, int c, float rc, float ra, int &ux, int &uy,
                                           int &uz)
{
    const int m = j >> 3;
    const int r = fdiv(m, rc);   // m / c
    const int jj = fdiv(r, ra);  // r / a
    ux = A.lo[0] + 2 * (r - jj * a) + (j & 1);
    uy = A.lo[1] + 2 * jj + ((j >> 1) & 1);
    uz = A.lo[2] + 2 * (m - r * c) + ((j >> 2) & 1);
}

// Shared-memory slot of the (pi, c) pair of the cell at local u-coordinates.
__device__ __forceinline__ int pc_slot_of(int ux, int uy, int uz, int B)
{
    const int x = ux - 1, y = uy - 1, z = uz - 1;
    return (z * B + y) * B + (x ^ ((((y & 1) << 1) | ((z & 1) << 2)) & (B - 1)));
}

// One site of level k (linear index i, see block_cell).
__device__ __forceinline__ void evolve_cell(int i, const Box3 &A, int a, int c, float rc, float ra, int P, int PP,
                                            int B, const float2 *__restrict__ prev_buf, float2 *__restrict__ cur,
                                            float4 *__restrict__ pc_s, const LevelCoef &co, const PhysConst &q)
{
    int ux, uy, uz;
    block_cell(i, A, a, c, rc, ra, ux, uy, uz);
    const int pidx = (uz * P + uy) * P + ux;
    const int cidx = pc_slot_of(ux, uy, uz, B);
    const float4 pc = pc_s[cidx];
    float2 pi = make_float2(pc.x, pc.y), cc = make_float2(pc.z, pc.w);
    const float2 nphi = site_update(prev_buf[pidx], prev_buf[pidx - 1], prev_buf[pidx + 1], prev_buf[pidx - P],
                                    prev_buf[pidx + P], prev_buf[pidx - PP], prev_buf[pidx + PP], pi, cc, co, q);
    cur[pidx] = nphi;
    pc_s[cidx] = make_float4(pi.x, pi.y, cc.x, cc.y);
}

// U cells of level k, linear indices i, i + stride, ... (all < cnt): every
// input is loaded before any result is stored, so the U updates are
// independent instruction streams (the compiler cannot prove that a store to
// one cell's (pi, c) does not alias another cell's load).
template <int U>
__device__ __forceinline__ void evolve_cells(int i, int stride, const Box3 &A, int a, int cz, float rc, float ra,
                                             int P, int PP, int B, const float2 *__restrict__ prev_buf,
                                             float2 *__restrict__ cur, float4 *__restrict__ pc_s, const LevelCoef &co,
                                             const PhysConst &q)
{
    int pidx[U], cidx[U];
    float2 c[U], xm[U], xp[U], ym[U], yp[U], zm[U], zp[U];
    float4 pc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        int ux, uy, uz;
        block_cell(i + u * stride, A, a, cz, rc, ra, ux, uy, uz);
        pidx[u] = (uz * P + uy) * P + ux;
        cidx[u] = pc_slot_of(ux, uy, uz, B);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int p = pidx[u];
        c[u] = prev_buf[p];
        xm[u] = prev_buf[p - 1];
        xp[u] = prev_buf[p + 1];
        ym[u] = prev_buf[p - P];
        yp[u] = prev_buf[p + P];
        zm[u] = prev_buf[p - PP];
        zp[u] = prev_buf[p + PP];
        pc[u] = pc_s[cidx[u]];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        float2 pi = make_float2(pc[u].x, pc[u].y), cc = make_float2(pc[u].z, pc[u].w);
        c[u] = site_update(c[u], xm[u], xp[u], ym[u], yp[u], zm[u], zp[u], pi, cc, co, q);
        pc[u] = make_float4(pi.x, pi.y, cc.x, cc.y);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        cur[pidx[u]] = c[u];
        pc_s[cidx[u]] = pc[u];
    }
}

// The manager warp asks L2 for the next region's inputs while the worker is
// still on the current region: the band base (rows of its box in the state
// arrays, one request per 128-byte line) and the region's whole mailbox (all
// levels; the region is ready, so every chunk is written).  Prefetches of
// addresses inside the arrays never fault and change no data.  Used at base
// 16 (one region per SM: 7.95 -> 7.56 ms at 128^3); at base 8, with six CTAs
// per SM prefetching, it measured 10 % slower.
__device__ void prefetch_region_l2(const SimDev &sd, const TypeMeta &M, const RegionInfo &r, int lane)
{
    const int B = sd.B, H = sd.H;
    int gb[3];
    for (int d = 0; d < 3; ++d) gb[d] = (r.band & 1) * H + r.j[d] * B - (((r.S >> d) & 1) ? H + 1 : 1);
    const Box3 bp = M.base_phi;
    const int w1 = bp.hi[1] - bp.lo[1], rows = w1 * (bp.hi[2] - bp.lo[2]);
    const int nx = sd.n[0], ny = sd.n[1], nz = sd.n[2];
    for (int row = lane; row < rows; row += 32) {
        const int uy = bp.lo[1] + row % w1, uz = bp.lo[2] + row / w1;
        const long long rb = (long long)nx * (wrap_axis(gb[1] + uy, ny) + (long long)ny * wrap_axis(gb[2] + uz, nz));
        for (int ux = bp.lo[0]; ux < bp.hi[0] + 7; ux += 8) {  // every 8 cells and the last one
            const long long gi = rb + wrap_axis(gb[0] + min(ux, bp.hi[0] - 1), nx);
            prefetch_l2(sd.pc + gi);
            if (((ux - bp.lo[0]) & 15) == 0 || ux >= bp.hi[0] - 1) prefetch_l2(sd.phi + gi);
        }
    }
    const float2 *mb = sd.mbox + (long long)(r.band & 1) * sd.mb_slot + sd.mb_type_off[r.S] + (long long)r.jl * M.mb_size;
    for (int i = 16 * lane; i < M.mb_size; i += 16 * 32) prefetch_l2(mb + i);
}

// Manager warp: hand regions to the worker, release finished ones.
__device__ void manager_loop(const RegionArgs &a, const TablesDev *s_tabs, int *s_slot, SimDev *s_sd,
                             RegionInfo *s_ri, int *s_handoff, int *s_done, bool prefetch)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long limit = a.ctl->wait_limit_ns;
    int seq = 0;           // handoffs made
    int pending = -1;      // region handed at seq, not yet released
    RegionInfo pend_info = {};
    unsigned idx = 0;
    if (lane == 0) idx = atomicAdd(&a.ctl->head, 1u);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    int got = 0, v = -1;
    int prepared = 0;  // the next region's descriptor is in its handoff slot
    RegionInfo ni = pend_info;
    unsigned long long t0 = globaltimer_ns();
    unsigned long long t_progress = t0;  // last handoff or release
    for (unsigned spin = 0;; ++spin) {
        int done = 0;
        if (lane == 0) {
            if (!got) {
                if (idx >= a.total) {
                    got = 1;
                    v = -1;
                } else {
                    const int q = ld_acquire_gpu(a.queue + idx);
                    if (q >= 0) {
                        got = 1;
                        v = q;
                    } else if (ld_relaxed_gpu(&a.ctl->error) != 0) {
                        got = 1;
                        v = -2;
                    } else if ((spin & 15u) == 15u && globaltimer_ns() - t0 > limit) {
                        atomicCAS(&a.ctl->error, 0, kDevTimeout);
                        atomicExch(&a.ctl->error_info, (int)idx);
                        got = 1;
                        v = -2;
                    }
                }
            }
        }
        const int have = __shfl_sync(0xffffffffu, got, 0);
        const int next = __shfl_sync(0xffffffffu, v, 0);
        if (have && !prepared) {
            // while the worker is still busy: decode the next region and put it
            // and its simulation's descriptor into the free handoff slot
            if (next >= 0) {
                ni = decode_region(a.sims, a.n_sims, next);
                const int slot = (seq + 1) & 1;
                const int4 *src = reinterpret_cast<const int4 *>(a.sims + ni.sim);
                int4 *dst = reinterpret_cast<int4 *>(s_sd + slot);
                if (lane < (int)(sizeof(SimDev) / 16)) dst[lane] = src[lane];
                if (lane == 0) s_ri[slot] = ni;
                __syncwarp();
                if (prefetch) {
                    const SimDev &nsd = s_sd[slot];
                    prefetch_region_l2(nsd, s_tabs[nsd.tab_index].type[ni.S], ni, lane);
                }
            }
            prepared = 1;
        }
        if (lane == 0) done = ld_acquire_cta_shared(s_done) == seq;
        done = __shfl_sync(0xffffffffu, done, 0);
        if (done && have) {
            if (lane == 0) {
                s_slot[(seq + 1) & 1] = next;
                st_release_cta_shared(s_handoff, seq + 1);
            }
            ++seq;
            if (pending >= 0) {
                const SimDev &sd = a.sims[pend_info.sim];
                release_successors(a, sd, s_tabs[sd.tab_index], pend_info, lane, 0ull, pending);
            }
            pending = next;
            if (next < 0) break;
            pend_info = ni;
            prepared = 0;
            if (lane == 0) {
                got = 0;
                idx = atomicAdd(&a.ctl->head, 1u);
                t0 = globaltimer_ns();
                t_progress = t0;
            }
            continue;
        }
        if (done && pending >= 0) {
            // the next region is not ready yet: it may wait on this release
            const SimDev &sd = a.sims[pend_info.sim];
            release_successors(a, sd, s_tabs[sd.tab_index], pend_info, lane, 0ull, pending);
            pending = -1;
            if (lane == 0) t_progress = globaltimer_ns();
            continue;
        }
        // no handoff and no release for 4 wait limits: the worker is stuck;
        // record it and stop (the worker's own bounded wait then ends it too)
        int stuck = 0;
        if (lane == 0 && (spin & 15u) == 15u && globaltimer_ns() - t_progress > 4 * limit) {
            atomicCAS(&a.ctl->error, 0, kDevTimeout);
            stuck = 1;
        }
        if (__shfl_sync(0xffffffffu, stuck, 0)) break;
        if (!have) __nanosleep(32);  // waiting on the queue backs off; waiting on the worker polls shared memory
    }
}

// One instantiation per worker count NW, with the region base BB fixed at
// compile time (16: index arithmetic in shifts, stencil offsets as immediates;
// measured 1.5 % faster) or, for BB = 0, taken from the descriptor (bases 4
// and 8, whose several CTAs per SM favour the smaller code: the fixed-base
// build measured 1.4 % slower there).  A launch holds simulations of one base.
template <int NW, int BB>
__global__ void __launch_bounds__(NW + 32, region_min_blocks(NW)) region_kernel(RegionArgs a, int max_P_launch)
{
    const int max_P = BB ? BB + 2 : max_P_launch;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_slot[2], s_handoff, s_done;
    __shared__ SimDev s_sd[2];      // descriptor of the region handed over in each slot
    __shared__ RegionInfo s_ri[2];  // and the region, decoded
    __shared__ float2 *s_mb[64];  // consumer code (type | offset bits << 3) -> mailbox base
    const int tid = threadIdx.x;
    const int P3 = max_P * max_P * max_P, B3 = (max_P - 2) * (max_P - 2) * (max_P - 2);
    float2 *phi_buf0 = reinterpret_cast<float2 *>(smem_raw);
    float2 *phi_buf1 = phi_buf0 + P3;
    float4 *pc_s = reinterpret_cast<float4 *>(phi_buf1 + P3);
    TablesDev *s_tabs = reinterpret_cast<TablesDev *>(pc_s + B3);
    LevelCoef *s_coef = reinterpret_cast<LevelCoef *>(s_tabs + a.n_tabs);

    {  // the launch's tables and simulation descriptors, once
        const int4 *src = reinterpret_cast<const int4 *>(a.tabs);
        int4 *dst = reinterpret_cast<int4 *>(s_tabs);
        const int nt = a.n_tabs * (int)(sizeof(TablesDev) / 16);
        for (int i = tid; i < nt; i += NW + 32) dst[i] = src[i];
        if (tid == 0) {
            s_handoff = 0;
            s_done = 0;
        }
    }
    __syncthreads();
    unsigned short *s_imp = reinterpret_cast<unsigned short *>(s_coef + kMaxHDev);
    for (int t = 0; t < a.n_tabs; ++t) {  // every import list of the launch, once
        const int4 *src = reinterpret_cast<const int4 *>(s_tabs[t].imp);
        int4 *dst = reinterpret_cast<int4 *>(s_imp + s_tabs[t].imp_smem);
        for (int i = tid; i < s_tabs[t].imp_n / 8; i += NW + 32) dst[i] = src[i];
    }
    __syncthreads();
    if (tid < 32) {
        manager_loop(a, s_tabs, s_slot, s_sd, s_ri, &s_handoff, &s_done, BB == 16);
        return;
    }
    const int wt = tid - 32;  // worker thread index
    __shared__ int s_abort;
    for (int seq = 1;; ++seq) {
        if (wt == 0) {
            // bounded wait for the manager's handoff (a shared-memory poll: the
            // handoff normally follows within a microsecond)
            s_abort = 0;
            const unsigned long long t0 = globaltimer_ns(), limit = 8 * a.ctl->wait_limit_ns;
            for (unsigned spin = 0; ld_acquire_cta_shared(&s_handoff) < seq; ++spin) {
                if ((spin & 15u) == 15u && globaltimer_ns() - t0 > limit) {
                    atomicCAS(&a.ctl->error, 0, kDevTimeout);
                    s_abort = 1;
                    break;
                }
            }
        }
        named_barrier(kWorkerBarrier, NW);
        if (s_abort) break;
        const int g = s_slot[seq & 1];
        if (g < 0) break;
        if (a.trace && wt == 0) a.trace[2 * (size_t)g] = globaltimer_ns();

        const RegionInfo r = s_ri[seq & 1];  // decoded by the manager at the handoff
        const SimDev &sd = s_sd[seq & 1];
        const TablesDev &T = s_tabs[sd.tab_index];
        const TypeMeta &M = T.type[r.S];
        const int S = r.S, band = r.band, jl = r.jl;
        const int B = BB ? BB : sd.B, H = B / 2, P = B + 2, PP = P * P;  // sd.B == BB when BB is fixed
        int gbase[3];  // global coordinate of local u = 0 along each axis
        for (int d = 0; d < 3; ++d) gbase[d] = (band & 1) * H + r.j[d] * B - (((S >> d) & 1) ? H + 1 : 1);
        const int nx = sd.n[0], ny = sd.n[1], nz = sd.n[2];
        const long long nxy = (long long)nx * ny;
        const long long slot = (long long)(band & 1) * sd.mb_slot;
        if (wt < 64) {
            // mailbox of the consumer with this code, if the code names one
            const int Sc = wt & 7, eb = wt >> 3;
            int jc = 0, mul = 1;
            for (int d = 0; d < 3; ++d) {
                int v = r.j[d] + ((eb >> d) & 1);
                v -= (v >= sd.J[d]) ? sd.J[d] : 0;
                jc += v * mul;
                mul *= sd.J[d];
            }
            s_mb[wt] = sd.mbox + slot + sd.mb_type_off[Sc] + (long long)jc * T.type[Sc].mb_size;
        }

        // ---- group 0: the band base (tops of the previous band) + coefficients ----
        // Work units are (run of up to 4 cells along z, column), columns fastest:
        // every worker gets a similar share whatever the box's shape, and
        // consecutive threads read consecutive cells along x.
        {
            if (wt < H) cp_async16(s_coef + wt, sd.coef + band * H + wt);
            const Box3 bp = M.base_phi;
            const Box3 bc = M.base_pc;
            const int w0 = bp.hi[0] - bp.lo[0];
            const int ncol = M.base_cols, units = ncol * M.base_runs;
            for (int u = wt; u < units; u += NW) {
                const int run = fdiv(u, M.rcp_cols);
                const int i = u - run * ncol;
                const int t1 = fdiv(i, M.rcp_base[0]);
                const int ux = bp.lo[0] + i - t1 * w0;
                const int uy = bp.lo[1] + t1;
                const int oxy = (ux < bc.lo[0] || ux >= bc.hi[0]) + (uy < bc.lo[1] || uy >= bc.hi[1]);
                if (oxy > 1) continue;  // not a 7-point neighbour of A(1)
                const long long gxy =
                    (long long)wrap_axis(gbase[0] + ux, nx) + (long long)nx * wrap_axis(gbase[1] + uy, ny);
                const int z0 = bp.lo[2] + 4 * run, z1 = min(z0 + 4, bp.hi[2]);
                for (int uz = z0; uz < z1; ++uz) {
                    const int out = oxy + (uz < bc.lo[2] || uz >= bc.hi[2]);
                    if (out > 1) continue;
                    const long long gi = gxy + nxy * wrap_axis(gbase[2] + uz, nz);
                    cp_async8(phi_buf0 + (uz * P + uy) * P + ux, sd.phi + gi);
                    if (out == 0) cp_async16(pc_s + pc_slot_of(ux, uy, uz, B), sd.pc + gi);
                }
            }
            cp_async_commit();
        }
        // ---- sloped initial surface: level L lands as copy group L, issued one
        // level ahead (level 1 now, level k+1 at the start of level k) ----
        const float2 *mb_self = sd.mbox + slot + sd.mb_type_off[S] + (long long)jl * M.mb_size;
        const unsigned short *s_imp_t = s_imp + T.imp_smem;
        auto issue_level = [&](int L) {
            if (L <= H - 1) {
                const int nf = M.imp_full_n[L], np = M.imp_phi_n[L];
                if (nf + np > 0)
                    import_level<NW>(mb_self + M.mb_level_off[L], nf, np, s_imp_t + M.imp_full_off[L],
                                     s_imp_t + M.imp_phi_off[L], (L & 1) ? phi_buf1 : phi_buf0, pc_s, B, P, wt);
            }
            cp_async_commit();  // one group per level, empty or not
        };
        issue_level(1);

        const int nlev = M.levels;
        const PhysConst q = sd.q;
        int2 pre[kExportPrefetch];
        for (int k = 1; k <= nlev; ++k) {
            const float2 *__restrict__ prev_buf = (k & 1) ? phi_buf0 : phi_buf1;
            float2 *__restrict__ cur = (k & 1) ? phi_buf1 : phi_buf0;
            issue_level(k + 1);  // lands in buffer (k+1) & 1 outside what level k reads
            // export entries of level k-1, loaded now, used after the compute
            const int ne = k >= 2 ? M.exp_n[k - 1] : 0;
            const int2 *el = T.exp + (k >= 2 ? M.exp_off[k - 1] : 0);
            prefetch_entries<NW>(el, ne, pre, wt);
            cp_async_wait_pending(2);  // groups 0..k-1 (base, coefficients, levels < k) have landed
            named_barrier(kWorkerBarrier, NW);
            // ---- evolve the cells of level k, several independent cells per step ----
            const LevelCoef co = s_coef[k - 1];
            const Box3 A = M.active[k];
            const float rc = M.rcp_active[k][0], ra = M.rcp_active[k][1];
            const int w0 = A.hi[0] - A.lo[0], w2 = A.hi[2] - A.lo[2];
            const int cnt = w0 * (A.hi[1] - A.lo[1]) * w2;
            const int a = w0 >> 1, cz = w2 >> 1;  // 2x2x2 blocks along x and z
            int i = wt;
            constexpr int U = region_cells_per_step(NW);
            for (; i + (U - 1) * NW < cnt; i += U * NW)
                evolve_cells<U>(i, NW, A, a, cz, rc, ra, P, PP, B, prev_buf, cur, pc_s, co, q);
            for (; i < cnt; i += NW) evolve_cell(i, A, a, cz, rc, ra, P, PP, B, prev_buf, cur, pc_s, co, q);
            // ---- final surface of level k-1 (read-only data of level k-1) ----
            if (ne > 0) export_entries<NW>(el, ne, pre, s_mb, prev_buf, pc_s, wt);
        }
        const float2 *last = (nlev & 1) ? phi_buf1 : phi_buf0;
        if (nlev <= H - 1) {
            // ---- final surface of the last level ----
            const int ne = M.exp_n[nlev];
            const int2 *el = T.exp + M.exp_off[nlev];
            prefetch_entries<NW>(el, ne, pre, wt);
            named_barrier(kWorkerBarrier, NW);
            export_entries<NW>(el, ne, pre, s_mb, last, pc_s, wt);
        } else {
            named_barrier(kWorkerBarrier, NW);
            // ---- tops of the inverted pyramid: the next band's base ----
            const float rB = T.type[0].rcp_base[0];  // the pyramid's base box is B wide: 1/B
            for (int i = wt; i < B * B; i += NW) {
                const int t1 = fdiv(i, rB);
                const int ux = 1 + i - t1 * B;
                const int uy = 1 + t1;
                const long long gxy =
                    (long long)wrap_axis(gbase[0] + ux, nx) + (long long)nx * wrap_axis(gbase[1] + uy, ny);
                for (int uz = 1; uz <= B; ++uz) {
                    const long long gi = gxy + nxy * wrap_axis(gbase[2] + uz, nz);
                    __stcg(sd.phi + gi, last[(uz * P + uy) * P + ux]);
                    __stcg(sd.pc + gi, pc_s[pc_slot_of(ux, uy, uz, B)]);
                }
            }
        }
        named_barrier(kWorkerBarrier, NW);
        if (wt == 0) {
            if (a.trace) a.trace[2 * (size_t)g + 1] = globaltimer_ns();
            st_release_cta_shared(&s_done, seq);
        }
    }
}

// ------------------------------------------------------------ sweep kernel
// One level of the whole grid: block 32 x 8 over (x, y), each thread marches
// a chunk of z keeping phi(z-1), phi(z), phi(z+1) in registers; x and y
// neighbours come through L1.  48 bytes per site-update of HBM traffic.
__global__ void __launch_bounds__(256) sweep_kernel(const float2 *__restrict__ phi_in, float2 *__restrict__ phi_out,
                                                    float4 *__restrict__ pc, int nx, int ny, int nz, int zchunk,
                                                    const LevelCoef *__restrict__ coef, int lvl, PhysConst q)
{
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, nz);
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const LevelCoef co = coef[lvl];
    const long long plane = (long long)nx * ny;
    const int zb = z0 == 0 ? nz - 1 : z0 - 1;
    float2 zprev = phi_in[zb * plane + (long long)y * nx + x];
    float2 zcur = phi_in[z0 * plane + (long long)y * nx + x];
    for (int z = z0; z < z1; ++z) {
        const int zn = z == nz - 1 ? 0 : z + 1;
        const float2 znext = phi_in[zn * plane + (long long)y * nx + x];
        const long long zo = z * plane;
        const long long row = zo + (long long)y * nx;
        const float4 v = pc[row + x];
        float2 p = make_float2(v.x, v.y), cc = make_float2(v.z, v.w);
        const float2 out = site_update(zcur, phi_in[row + xm], phi_in[row + xp], phi_in[zo + (long long)ym * nx + x],
                                       phi_in[zo + (long long)yp * nx + x], zprev, znext, p, cc, co, q);
        phi_out[row + x] = out;
        pc[row + x] = make_float4(p.x, p.y, cc.x, cc.y);
        zprev = zcur;
        zcur = znext;
    }
}

// ------------------------------------------------------------ diagnostics
// Energy terms of a stored state in FP64: sum |pi|^2, sum over forward links
// |phi(x+e) - phi(x)|^2 / dx^2 and sum a^2 (lambda/2)(|phi|^2 - eta^2)^2.
// Each block reduces a fixed range of sites in a fixed tree order; the
// partials are then summed in block order: the result is deterministic.
constexpr int kDiagThreads = 256;

__global__ void __launch_bounds__(kDiagThreads)
    energy_partial_kernel(const float2 *__restrict__ phi, const float4 *__restrict__ pc, int nx, int ny, int nz,
                          double inv_dx2, double eta2, double half_lambda_a2, double *__restrict__ partial)
{
    __shared__ double red[3][kDiagThreads];
    const long long sites = (long long)nx * ny * nz;
    const long long per_block = (sites + gridDim.x - 1) / gridDim.x;
    const long long s0 = blockIdx.x * per_block;
    const long long s1 = min(s0 + per_block, sites);
    double kin = 0.0, grad = 0.0, pot = 0.0;
    for (long long s = s0 + threadIdx.x; s < s1; s += kDiagThreads) {
        const int x = (int)(s % nx);
        const int y = (int)((s / nx) % ny);
        const int z = (int)(s / ((long long)nx * ny));
        const float2 f = phi[s];
        const float4 v = pc[s];
        const double fr = f.x, fi = f.y;
        kin = __dadd_rn(kin, __dadd_rn(__dmul_rn((double)v.x, (double)v.x), __dmul_rn((double)v.y, (double)v.y)));
        const long long nb[3] = {s - x + (x == nx - 1 ? 0 : x + 1),
                                 s + (long long)((y == ny - 1 ? 0 : y + 1) - y) * nx,
                                 s + (long long)((z == nz - 1 ? 0 : z + 1) - z) * nx * ny};
        for (int k = 0; k < 3; ++k) {
            const float2 g = phi[nb[k]];
            const double dr = __dsub_rn((double)g.x, fr), di = __dsub_rn((double)g.y, fi);
            grad = __dadd_rn(grad, __dmul_rn(__dadd_rn(__dmul_rn(dr, dr), __dmul_rn(di, di)), inv_dx2));
        }
        const double m2 = __dsub_rn(__dadd_rn(__dmul_rn(fr, fr), __dmul_rn(fi, fi)), eta2);
        pot = __dadd_rn(pot, __dmul_rn(half_lambda_a2, __dmul_rn(m2, m2)));
    }
    red[0][threadIdx.x] = kin;
    red[1][threadIdx.x] = grad;
    red[2][threadIdx.x] = pot;
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = __dadd_rn(red[k][threadIdx.x], red[k][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) partial[3 * blockIdx.x + k] = red[k][0];
}

__global__ void energy_final_kernel(const double *__restrict__ partial, int nblocks, double *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < nblocks; ++b)
        for (int k = 0; k < 3; ++k) acc[k] = __dadd_rn(acc[k], partial[3 * b + k]);
    for (int k = 0; k < 3; ++k) out[k] = acc[k];
}

// Winding of the field around each plaquette: signed crossings of the
// positive real axis by the polygon phi(p0) phi(p1) phi(p2) phi(p3)
// (corners x, x+e_a, x+e_a+e_b, x+e_b; (a, b) = (k+1, k+2) mod 3).  An edge
// u -> v crossing upward counts +1 when cross(u, v) >= 0, downward -1 when
// cross(u, v) <= 0; a vertex on the axis counts as above it.  The products
// of FP32 inputs are exact in FP64, so the sign tests are exact.
__device__ __forceinline__ int crossing(float2 u, float2 v)
{
    const double cr = __dsub_rn(__dmul_rn((double)u.x, (double)v.y), __dmul_rn((double)u.y, (double)v.x));
    const bool ua = u.y >= 0.0f, va = v.y >= 0.0f;
    if (!ua && va) return cr >= 0.0 ? 1 : 0;
    if (ua && !va) return cr <= 0.0 ? -1 : 0;
    return 0;
}

__global__ void __launch_bounds__(kDiagThreads)
    winding_kernel(const float2 *__restrict__ phi, int nx, int ny, int nz, signed char *__restrict__ w,
                   unsigned long long *__restrict__ counts)
{
    // counts: [0..2] pierced plaquettes per normal axis, [3] sum |w|, [4..6] sum w (two's complement)
    __shared__ unsigned long long red[7];
    if (threadIdx.x < 7) red[threadIdx.x] = 0ull;
    __syncthreads();
    const long long sites = (long long)nx * ny * nz;
    unsigned long long loc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < sites;
         s += (long long)gridDim.x * blockDim.x) {
        const int c[3] = {(int)(s % nx), (int)((s / nx) % ny), (int)(s / ((long long)nx * ny))};
        const int n[3] = {nx, ny, nz};
        for (int k = 0; k < 3; ++k) {
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            int q1[3] = {c[0], c[1], c[2]}, q2[3] = {c[0], c[1], c[2]}, q3[3] = {c[0], c[1], c[2]};
            q1[a] = q1[a] + 1 == n[a] ? 0 : q1[a] + 1;
            q2[a] = q1[a];
            q2[b] = q2[b] + 1 == n[b] ? 0 : q2[b] + 1;
            q3[b] = q2[b];
            const float2 p0 = phi[s];
            const float2 p1 = phi[q1[0] + (long long)nx * (q1[1] + (long long)ny * q1[2])];
            const float2 p2 = phi[q2[0] + (long long)nx * (q2[1] + (long long)ny * q2[2])];
            const float2 p3 = phi[q3[0] + (long long)nx * (q3[1] + (long long)ny * q3[2])];
            const int tot = crossing(p0, p1) + crossing(p1, p2) + crossing(p2, p3) + crossing(p3, p0);
            if (w) w[k * sites + s] = (signed char)tot;
            if (tot != 0) {
                loc[k] += 1ull;
                loc[3] += (unsigned long long)(tot < 0 ? -tot : tot);
                loc[4 + k] += (unsigned long long)(long long)tot;
            }
        }
    }
    for (int k = 0; k < 7; ++k)
        if (loc[k]) atomicAdd(&red[k], loc[k]);
    __syncthreads();
    if (threadIdx.x < 7 && red[threadIdx.x]) atomicAdd(&counts[threadIdx.x], red[threadIdx.x]);
}

// ------------------------------------------------------------ launchers
// ------------------------------------------------------------ region features
// The 16 inputs of the region cost model, per region of a launch, from its
// descriptor and from the state at the start of the call (the footprint of
// the region's own cells, sampled on a 2 x 2 x 2 lattice):
//   0-2  inverted axes of the region type (x, y, z);  3  |S| / 3 (phase);
//   4    B / 16;  5  log2(sites) / 24;  6  nu / 2;  7  a^2 lambda at the band's
//   first level;  8  band / bands;  9  (4 band + |S|) / (4 bands);
//   10, 11  mean and max |phi|^2;  12  mean |pi|^2;  13  fraction of sampled
//   xy plaquettes with nonzero winding;  14  mean |phi(x+1) - phi(x)|^2 / dx^2;
//   15  the region's measured time in the previous traced call (us / 20), or 0.
// simf[s] = (B / 16, log2(sites) / 24, nu / 2, 0) of simulation s.
__global__ void __launch_bounds__(128) feature_kernel(RegionArgs a, const float4 *__restrict__ simf,
                                                      const unsigned long long *__restrict__ prev_trace,
                                                      float *__restrict__ X)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int)a.total) return;
    const RegionInfo r = decode_region(a.sims, a.n_sims, g);
    const SimDev &sd = a.sims[r.sim];
    const float4 sf = simf[r.sim];
    const int S = r.S, B = sd.B, H = sd.H, nb = sd.nbands;
    const int ns = (S & 1) + ((S >> 1) & 1) + ((S >> 2) & 1);
    float f[16];
    f[0] = (float)(S & 1);
    f[1] = (float)((S >> 1) & 1);
    f[2] = (float)((S >> 2) & 1);
    f[3] = ns / 3.0f;
    f[4] = sf.x;
    f[5] = sf.y;
    f[6] = sf.z;
    f[7] = sd.coef[r.band * H].m;
    f[8] = (float)r.band / (float)nb;
    f[9] = (float)(4 * r.band + ns) / (float)(4 * nb);
    int gb[3];
    for (int d = 0; d < 3; ++d) gb[d] = (r.band & 1) * H + r.j[d] * B - (((S >> d) & 1) ? H + 1 : 1);
    const int nx = sd.n[0], ny = sd.n[1], nz = sd.n[2];
    const int stride = B / 2;
    double sphi = 0.0, spi = 0.0, sgrad = 0.0;
    float mphi = 0.0f;
    int pierced = 0;
    for (int m = 0; m < 8; ++m) {
        const int x = wrap_axis(gb[0] + 1 + stride * (m & 1), nx);
        const int y = wrap_axis(gb[1] + 1 + stride * ((m >> 1) & 1), ny);
        const int z = wrap_axis(gb[2] + 1 + stride * (m >> 2), nz);
        const int x1 = x + 1 == nx ? 0 : x + 1, y1 = y + 1 == ny ? 0 : y + 1;
        const long long row = (long long)nx * (y + (long long)ny * z), row1 = (long long)nx * (y1 + (long long)ny * z);
        const float2 p0 = sd.phi[row + x], p1 = sd.phi[row + x1], p2 = sd.phi[row1 + x1], p3 = sd.phi[row1 + x];
        const float4 pc = sd.pc[row + x];
        const float a2 = p0.x * p0.x + p0.y * p0.y;
        sphi += a2;
        mphi = fmaxf(mphi, a2);
        spi += (double)(pc.x * pc.x + pc.y * pc.y);
        const float dx = p1.x - p0.x, dy = p1.y - p0.y;
        sgrad += (double)(dx * dx + dy * dy);
        pierced += (crossing(p0, p1) + crossing(p1, p2) + crossing(p2, p3) + crossing(p3, p0)) != 0;
    }
    f[10] = (float)(sphi / 8.0);
    f[11] = mphi;
    f[12] = (float)(spi / 8.0);
    f[13] = pierced / 8.0f;
    f[14] = (float)(sgrad / 8.0) * sd.q.inv_dx2;
    f[15] = 0.0f;
    if (prev_trace) {
        const unsigned long long t0 = prev_trace[2 * (size_t)g], t1 = prev_trace[2 * (size_t)g + 1];
        if (t1 > t0) f[15] = (float)((double)(t1 - t0) * 1e-3 / 20.0);
    }
    float4 *o = reinterpret_cast<float4 *>(X + 16 * (size_t)g);
    for (int q = 0; q < 4; ++q) o[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
}

cudaError_t launch_features(const RegionArgs &a, const float4 *simf, const unsigned long long *prev_trace, float *X,
                            cudaStream_t st)
{
    if (a.total == 0) return cudaSuccess;
    feature_kernel<<<(a.total + 127) / 128, 128, 0, st>>>(a, simf, prev_trace, X);
    return cudaGetLastError();
}

cudaError_t launch_reset(const RegionArgs &a, cudaStream_t st)
{
    const unsigned blocks = (a.total + 255) / 256;
    reset_kernel<<<blocks ? blocks : 1, 256, 0, st>>>(a);
    if (a.prio && a.n_seed > 0) {
        seed_count_kernel<<<(a.n_seed + 255) / 256, 256, 0, st>>>(a);
        seed_kernel<<<(a.n_seed + 255) / 256, 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <int NW, int BB>
static cudaError_t region_launch_t(const RegionArgs &a, int B, size_t smem, int grid, cudaStream_t st)
{
    cudaError_t e =
        cudaFuncSetAttribute(region_kernel<NW, BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    region_kernel<NW, BB><<<grid, NW + 32, smem, st>>>(a, B + 2);
    return cudaGetLastError();
}

template <int NW>
static cudaError_t region_launch_nw(const RegionArgs &a, int B, size_t smem, int grid, cudaStream_t st)
{
    switch (B) {
    case 4:
    case 8:
        return region_launch_t<NW, 0>(a, B, smem, grid, st);
    case 16:
        return region_launch_t<NW, 16>(a, B, smem, grid, st);
    default:
        return cudaErrorInvalidValue;
    }
}

template <int NW, int BB>
static cudaError_t region_occupancy_t(size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(region_kernel<NW, BB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, region_kernel<NW, BB>, NW + 32, smem);
}

template <int NW>
static cudaError_t region_occupancy_nw(int B, size_t smem, int *blocks_per_sm)
{
    switch (B) {
    case 4:
    case 8:
        return region_occupancy_t<NW, 0>(smem, blocks_per_sm);
    case 16:
        return region_occupancy_t<NW, 16>(smem, blocks_per_sm);
    default:
        return cudaErrorInvalidValue;
    }
}

size_t region_smem_bytes(int max_B, int n_tabs, int n_sims, int imp_units)
{
    (void)n_sims;  // descriptors travel with the handoff (static shared memory)
    const int P = max_B + 2;
    return (size_t)2 * P * P * P * sizeof(float2) + (size_t)max_B * max_B * max_B * sizeof(float4) +
           (size_t)n_tabs * sizeof(TablesDev) + kMaxHDev * sizeof(LevelCoef) +
           (size_t)imp_units * sizeof(unsigned short);
}

// threads = worker threads per CTA (the manager warp comes on top)
cudaError_t region_occupancy(int threads, int B, size_t smem, int *blocks_per_sm)
{
#define SP_OCC(NW)                                                                                               \
    case NW:                                                                                                     \
        return region_occupancy_nw<NW>(B, smem, blocks_per_sm);
    switch (threads) {
        SP_OCC(64)
        SP_OCC(128)
        SP_OCC(256)
        SP_OCC(320)
        SP_OCC(384)
        SP_OCC(480)
        SP_OCC(512)
        SP_OCC(768)
    default:
        return cudaErrorInvalidValue;
    }
#undef SP_OCC
}

cudaError_t launch_region(const RegionArgs &a, int threads, int max_B, size_t smem, int grid, cudaStream_t st)
{
    switch (threads) {
    case 64:
        return region_launch_nw<64>(a, max_B, smem, grid, st);
    case 128:
        return region_launch_nw<128>(a, max_B, smem, grid, st);
    case 256:
        return region_launch_nw<256>(a, max_B, smem, grid, st);
    case 320:
        return region_launch_nw<320>(a, max_B, smem, grid, st);
    case 384:
        return region_launch_nw<384>(a, max_B, smem, grid, st);
    case 480:
        return region_launch_nw<480>(a, max_B, smem, grid, st);
    case 512:
        return region_launch_nw<512>(a, max_B, smem, grid, st);
    case 768:
        return region_launch_nw<768>(a, max_B, smem, grid, st);
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sweep(const float2 *phi_in, float2 *phi_out, float4 *pc, const int n[3],
                         const LevelCoef *coef, int lvl, PhysConst q, cudaStream_t st)
{
    const int zchunk = 8;
    dim3 block(32, 8, 1);
    dim3 grid((n[0] + 31) / 32, (n[1] + 7) / 8, (n[2] + zchunk - 1) / zchunk);
    sweep_kernel<<<grid, block, 0, st>>>(phi_in, phi_out, pc, n[0], n[1], n[2], zchunk, coef, lvl, q);
    return cudaGetLastError();
}

int energy_blocks(const int n[3])
{
    const long long sites = (long long)n[0] * n[1] * n[2];
    long long b = (sites + 4095) / 4096;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

cudaError_t launch_energy(const float2 *phi, const float4 *pc, const int n[3], double inv_dx2, double eta2,
                          double half_lambda_a2, double *partial, double *out, cudaStream_t st)
{
    const int nb = energy_blocks(n);
    energy_partial_kernel<<<nb, kDiagThreads, 0, st>>>(phi, pc, n[0], n[1], n[2], inv_dx2, eta2, half_lambda_a2,
                                                        partial);
    energy_final_kernel<<<1, 32, 0, st>>>(partial, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_winding(const float2 *phi, const int n[3], signed char *w, unsigned long long *counts,
                           cudaStream_t st)
{
    const long long sites = (long long)n[0] * n[1] * n[2];
    long long b = (sites + kDiagThreads - 1) / kDiagThreads;
    if (b > 8192) b = 8192;
    winding_kernel<<<(int)b, kDiagThreads, 0, st>>>(phi, n[0], n[1], n[2], w, counts);
    return cudaGetLastError();
}

}  // namespace sp
