// sp_octant.cu -- the base-32 region kernel: one region of 32^3 cells and 16
// levels per thread-block cluster of 2 x 2 x 2 CTAs, one octant per CTA.
//
// A 32^3 region (its two phi levels, (pi, c) and import lists) does not fit
// one SM's shared memory, so the region is cut at its centre into eight
// octants (planner.h, OctTables).  In mirrored coordinates every octant's
// active cells at level k form the same corner box, so the eight CTAs do the
// same work at every level.  Each CTA keeps its octant (16^3 cells, phi with
// a one-cell halo) on chip for the whole region; the only exchange between
// them is the inner faces (the dist = 0 layer of phi) before every level:
// each face cell is written straight into the neighbour CTA's halo with an
// asynchronous distributed-shared-memory store that completes on the
// neighbour's mbarrier (st.async ... complete_tx), as soon as it is computed
// (or, for a face cell that entered as a sloped-surface import, as soon as
// that import has landed).  Everything else -- band base, sloped surfaces,
// final surfaces, band tops -- moves between HBM and the octant exactly as
// in the single-CTA kernel, with per-octant mailboxes.
//
// Work queue (paper Sec. 4): warp 0 of the cluster's first CTA is the
// manager.  It takes ready regions from the device queue, hands each one to
// the eight CTAs (descriptor and decoded region written into their shared
// memory, then a release store of the handoff counter), waits until all
// eight have reported the region done (remote release-adds on its counter),
// hands out the next one and releases the finished region's successors.
// Every wait is bounded (the grid's wait limit); a CTA that gives up records
// the error and leaves its loop, and the manager then hands every CTA the
// stop mark, so every CTA reaches the final cluster barrier.
//
// Safety of the direct halo stores (octant neighbours differ by one axis d):
// a CTA writes phi(k) into its neighbour's buffer k & 1 at u_d = 0 only
// during its own level k, i.e. after it received all of the neighbour's
// phi(k-1) face cells; the neighbour sends those only after computing them,
// and a face cell is computed after the only reads of the halo it needs
// (interior cells never read the halo).  So the neighbour has finished
// reading phi(k-2) from that halo.  Transfers of consecutive levels go to
// alternating mbarriers, so bytes of level k+1 can never complete level k.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sp_device.cuh"
#include "sp_kernels.h"
#include "sp_region_common.cuh"

namespace sp {

namespace {

constexpr int kOctNW = 384;         // worker threads per CTA (one manager warp on top)
constexpr int kOctBar = 1;          // named barrier of the workers
constexpr int kOctH = 16, kOctP = 18, kOctLgH = 4;
constexpr int kOctExpPrefetch = 3;  // export entries per thread loaded before the compute
constexpr int kOctExpBatch = 4;

__device__ __forceinline__ void oct_export_one(int2 e, float2 *const *mb_of, const float2 *__restrict__ phi,
                                               const float4 *__restrict__ pc)
{
    float2 *mb = mb_of[(e.x >> 25) & 63];
    __stcg(mb + (e.y & 0xFFFF), phi[e.x & 0x1FFF]);
    if (e.x < 0) __stcg(reinterpret_cast<float4 *>(mb + ((unsigned)e.y >> 16)), pc[(e.x >> 13) & 0xFFF]);
}

__device__ __forceinline__ void oct_exports(const int2 *__restrict__ el, int ne, const int2 (&pre)[kOctExpPrefetch],
                                            float2 *const *mb_of, const float2 *__restrict__ phi,
                                            const float4 *__restrict__ pc, int wt)
{
#pragma unroll
    for (int u = 0; u < kOctExpPrefetch; ++u)
        if (wt + u * kOctNW < ne) oct_export_one(pre[u], mb_of, phi, pc);
    for (int base = wt + kOctExpPrefetch * kOctNW; base < ne; base += kOctExpBatch * kOctNW) {
        int2 e[kOctExpBatch];
#pragma unroll
        for (int u = 0; u < kOctExpBatch; ++u)
            if (base + u * kOctNW < ne) e[u] = __ldg(el + base + u * kOctNW);
#pragma unroll
        for (int u = 0; u < kOctExpBatch; ++u)
            if (base + u * kOctNW < ne) oct_export_one(e[u], mb_of, phi, pc);
    }
}

__device__ __forceinline__ void oct_prefetch(const int2 *__restrict__ el, int ne, int2 (&pre)[kOctExpPrefetch],
                                             int wt)
{
#pragma unroll
    for (int u = 0; u < kOctExpPrefetch; ++u)
        if (wt + u * kOctNW < ne) pre[u] = __ldg(el + wt + u * kOctNW);
}

// phi index in the octant buffer of the own cell with (pi, c) index c
__device__ __forceinline__ int oct_pidx(int c)
{
    return (((c >> (2 * kOctLgH)) + 1) * kOctP + ((c >> kOctLgH) & (kOctH - 1)) + 1) * kOctP + (c & (kOctH - 1)) + 1;
}

// Manager (warp 0 of the cluster's CTA 0).  Stages region `next` as handoff
// number `seq` in the eight CTAs' shared memory: lane r writes CTA r's slot
// seq & 1 (the simulation descriptor, the decoded region and the region id).
// A slot is staged only after every CTA finished the region that last used
// it (handoff seq - 2), so staging runs while the CTAs still evolve region
// seq - 1; the handoff itself (oct_release) follows once all eight are done.
__device__ void oct_stage(const RegionArgs &a, int next, const RegionInfo &ni, int seq, int *s_slot, SimDev *s_sd,
                          RegionInfo *s_ri, int lane)
{
    const int slot = seq & 1;
    if (lane < 8) {
        if (next >= 0) {
            const int4 *src = reinterpret_cast<const int4 *>(a.sims + ni.sim);
            const unsigned dst = map_shared(s_sd + slot, (unsigned)lane);
            for (int i = 0; i < (int)(sizeof(SimDev) / 16); ++i) st_cluster_shared_int4(dst + 16u * i, src[i]);
            const int *ri = reinterpret_cast<const int *>(&ni);
            const unsigned rdst = map_shared(s_ri + slot, (unsigned)lane);
            for (int i = 0; i < (int)(sizeof(RegionInfo) / 4); ++i)
                asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(rdst + 4u * i), "r"(ri[i]) : "memory");
        }
        asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(map_shared(s_slot + slot, (unsigned)lane)), "r"(next)
                     : "memory");
    }
}

// Releases handoff number seq to the eight CTAs (lane r: CTA r, after its own
// staging stores, which the release orders before the counter).
__device__ void oct_release(int seq, int *s_handoff, int lane)
{
    if (lane < 8) st_release_cluster_shared(map_shared(s_handoff, (unsigned)lane), seq);
    __syncwarp();
}

__device__ void oct_manager(const RegionArgs &a, int *s_slot, SimDev *s_sd, RegionInfo *s_ri, int *s_handoff,
                            int *s_done_count)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long limit = a.ctl->wait_limit_ns;
    int seq = 0;          // handoffs made
    int pending = -1;     // region handed out as number seq, not yet released
    RegionInfo pend_info = {}, ni = {};
    unsigned idx = 0;
    if (lane == 0) idx = atomicAdd(&a.ctl->head, 1u);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    int got = 0, v = -1, staged = 0;
    unsigned long long t0 = globaltimer_ns(), t_progress = t0;
    for (unsigned spin = 0;; ++spin) {
        if (lane == 0 && !got) {
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
        const int have = __shfl_sync(0xffffffffu, got, 0);
        const int next = __shfl_sync(0xffffffffu, v, 0);
        if (have && !staged) {
            ni = RegionInfo{};
            if (next >= 0) ni = decode_region(a.sims, a.n_sims, next);
            oct_stage(a, next, ni, seq + 1, s_slot, s_sd, s_ri, lane);
            staged = 1;
        }
        int done = 0;
        if (lane == 0) done = ld_acquire_cluster_shared(s_done_count) >= 8 * seq;
        done = __shfl_sync(0xffffffffu, done, 0);
        if (done && have) {
            ++seq;
            oct_release(seq, s_handoff, lane);
            if (pending >= 0) {
                const SimDev &sd = a.sims[pend_info.sim];
                release_successors(a, sd, a.tabs[sd.tab_index], pend_info, lane, 0ull, pending);
            }
            pending = next;
            pend_info = ni;
            staged = 0;
            if (next < 0) break;
            if (lane == 0) {
                got = 0;
                idx = atomicAdd(&a.ctl->head, 1u);
                t0 = globaltimer_ns();
                t_progress = t0;
            }
            continue;
        }
        if (done && pending >= 0) {
            // all eight finished and the next region is not ready: it may wait on this release
            const SimDev &sd = a.sims[pend_info.sim];
            release_successors(a, sd, a.tabs[sd.tab_index], pend_info, lane, 0ull, pending);
            pending = -1;
            if (lane == 0) t_progress = globaltimer_ns();
            continue;
        }
        // no handoff and no release for four wait limits: a CTA is stuck; stop everyone
        int stuck = 0;
        if (lane == 0 && (spin & 15u) == 15u && globaltimer_ns() - t_progress > 4 * limit) {
            atomicCAS(&a.ctl->error, 0, kDevTimeout);
            stuck = 1;
        }
        if (__shfl_sync(0xffffffffu, stuck, 0)) {
            oct_stage(a, -2, RegionInfo{}, seq + 1, s_slot, s_sd, s_ri, lane);
            oct_release(seq + 1, s_handoff, lane);
            break;
        }
        if (!have) __nanosleep(32);
    }
}

// U cells of one level (independent instruction streams: every input is
// loaded before any result is stored).  A computed cell on an inner face
// (u_d = 1) inside the next level's box along the other axes goes straight
// to the neighbour along d.
template <int U>
__device__ __forceinline__ void oct_cells(const int (&ux)[U], const int (&uy)[U], const int (&uz)[U],
                                          const bool (&on)[U], const float2 *__restrict__ prev,
                                          float2 *__restrict__ cur, float4 *__restrict__ pc_s, const LevelCoef &co,
                                          const PhysConst &q, int wn0, int wn1, int wn2, unsigned rank,
                                          const unsigned (&xb)[3])
{
    constexpr int P = kOctP, PP = P * P, H = kOctH;
    int pidx[U], cidx[U];
    float2 c[U], xm[U], xp[U], ym[U], yp[U], zm[U], zp[U];
    float4 pc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        pidx[u] = (uz[u] * P + uy[u]) * P + ux[u];
        cidx[u] = ((uz[u] - 1) * H + (uy[u] - 1)) * H + (ux[u] - 1);
        if (on[u]) {
            const int p = pidx[u];
            c[u] = prev[p];
            xm[u] = prev[p - 1];
            xp[u] = prev[p + 1];
            ym[u] = prev[p - P];
            yp[u] = prev[p + P];
            zm[u] = prev[p - PP];
            zp[u] = prev[p + PP];
            pc[u] = pc_s[cidx[u]];
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (on[u]) {
            float2 pi = make_float2(pc[u].x, pc[u].y), cc = make_float2(pc[u].z, pc[u].w);
            c[u] = site_update(c[u], xm[u], xp[u], ym[u], yp[u], zm[u], zp[u], pi, cc, co, q);
            pc[u] = make_float4(pi.x, pi.y, cc.x, cc.y);
        }
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (on[u]) {
            cur[pidx[u]] = c[u];
            pc_s[cidx[u]] = pc[u];
            if (ux[u] == 1 && wn0 > 0 && uy[u] <= wn1 && uz[u] <= wn2)
                st_async_f2(map_shared(cur + pidx[u] - 1, rank ^ 1u), c[u], xb[0]);
            if (uy[u] == 1 && wn1 > 0 && ux[u] <= wn0 && uz[u] <= wn2)
                st_async_f2(map_shared(cur + pidx[u] - P, rank ^ 2u), c[u], xb[1]);
            if (uz[u] == 1 && wn2 > 0 && ux[u] <= wn0 && uy[u] <= wn1)
                st_async_f2(map_shared(cur + pidx[u] - PP, rank ^ 4u), c[u], xb[2]);
        }
}

// Cell i of level k in face-first order: the x slab (ux = 1, w1 x w2 cells),
// the y slab (uy = 1, ux >= 2), the z slab (uz = 1, ux, uy >= 2); with
// interior = true, cell i of the interior (ux, uy, uz >= 2).
__device__ __forceinline__ void oct_decode(int i, bool interior, int w0, int w1, int w2, const float (&rf)[3],
                                           int &ux, int &uy, int &uz)
{
    if (interior) {
        const int t = fdiv(i, rf[1]);
        ux = 2 + i - t * (w0 - 1);
        const int t2 = fdiv(t, rf[2]);
        uy = 2 + t - t2 * (w1 - 1);
        uz = 2 + t2;
        return;
    }
    const int nX = w1 * w2, nY = (w0 - 1) * w2;
    if (i < nX) {
        const int t = fdiv(i, rf[0]);
        ux = 1;
        uy = 1 + i - t * w1;
        uz = 1 + t;
    } else if (i < nX + nY) {
        const int j = i - nX, t = fdiv(j, rf[1]);
        ux = 2 + j - t * (w0 - 1);
        uy = 1;
        uz = 1 + t;
    } else {
        const int j = i - nX - nY, t = fdiv(j, rf[1]);
        ux = 2 + j - t * (w0 - 1);
        uy = 2 + t;
        uz = 1;
    }
}

}  // namespace

__global__ void __launch_bounds__(kOctNW + 32, 1) region_oct_kernel(RegionArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_slot[2], s_handoff, s_done_count, s_abort, s_xpar;
    __shared__ SimDev s_sd[2];
    __shared__ RegionInfo s_ri[2];
    __shared__ float2 *s_mb[64];  // consumer code (type | G << 3) -> octant mailbox base
    __shared__ __align__(8) unsigned long long s_xbar[2];
    constexpr int P = kOctP, PP = P * P, P3 = P * P * P, H = kOctH;
    const int tid = threadIdx.x;
    const unsigned rank = cluster_ctarank();  // octant: bit d set = upper half along axis d
    float2 *phi_buf[2];
    phi_buf[0] = reinterpret_cast<float2 *>(smem_raw);
    phi_buf[1] = phi_buf[0] + P3;
    float4 *pc_s = reinterpret_cast<float4 *>(phi_buf[1] + P3);
    TablesOct *s_to = reinterpret_cast<TablesOct *>(pc_s + H * H * H);
    LevelCoef *s_coef = reinterpret_cast<LevelCoef *>(s_to + 1);
    unsigned short *s_imp = reinterpret_cast<unsigned short *>(s_coef + kMaxHOct);
    int *s_face = nullptr;  // set once the tables are in shared memory
    {
        const int4 *src = reinterpret_cast<const int4 *>(a.sims[0].oct);  // one base per launch
        int4 *dst = reinterpret_cast<int4 *>(s_to);
        for (int i = tid; i < (int)(sizeof(TablesOct) / 16); i += kOctNW + 32) dst[i] = src[i];
    }
    if (tid == 0) {
        s_handoff = 0;
        s_done_count = 0;
        s_abort = 0;
        mbar_init(&s_xbar[0], 1);
        mbar_init(&s_xbar[1], 1);
        fence_mbar_init_cluster();
    }
    __syncthreads();
    s_face = reinterpret_cast<int *>(s_imp + s_to->imp_n);
    {
        const int4 *src = reinterpret_cast<const int4 *>(s_to->imp);
        int4 *dst = reinterpret_cast<int4 *>(s_imp);
        for (int i = tid; i < s_to->imp_n / 8; i += kOctNW + 32) dst[i] = src[i];
        const int4 *fsrc = reinterpret_cast<const int4 *>(s_to->face);
        int4 *fdst = reinterpret_cast<int4 *>(s_face);
        for (int i = tid; i < s_to->face_total / 4; i += kOctNW + 32) fdst[i] = fsrc[i];
    }
    __syncthreads();
    cluster_barrier();  // every CTA's mbarriers exist before any remote store

    if (tid < 32) {
        if (rank == 0) oct_manager(a, s_slot, s_sd, s_ri, &s_handoff, &s_done_count);
    } else {
        const int wt = tid - 32;
        const int2 *exp_all = s_to->exp;
        const int *face_all = s_face;
        unsigned xph[2] = {0u, 0u};  // wt 0: parity of each exchange mbarrier's current phase
        const unsigned xbar_remote[3][2] = {
            {map_shared(&s_xbar[0], rank ^ 1u), map_shared(&s_xbar[1], rank ^ 1u)},
            {map_shared(&s_xbar[0], rank ^ 2u), map_shared(&s_xbar[1], rank ^ 2u)},
            {map_shared(&s_xbar[0], rank ^ 4u), map_shared(&s_xbar[1], rank ^ 4u)}};
        const unsigned done_remote = map_shared(&s_done_count, 0u);
        for (int seq = 1;; ++seq) {
            if (wt == 0) {
                const unsigned long long t0 = globaltimer_ns(), limit = 8 * a.ctl->wait_limit_ns;
                for (unsigned spin = 0; ld_acquire_cluster_shared(&s_handoff) < seq; ++spin) {
                    if ((spin & 15u) == 15u && globaltimer_ns() - t0 > limit) {
                        atomicCAS(&a.ctl->error, 0, kDevTimeout);
                        s_abort = 1;
                        break;
                    }
                }
            }
            named_barrier(kOctBar, kOctNW);
            if (s_abort) break;
            const int g = s_slot[seq & 1];
            if (g < 0) break;
            if (a.trace && wt == 0 && rank == 0) a.trace[2 * (size_t)g] = globaltimer_ns();
            const RegionInfo r = s_ri[seq & 1];
            const SimDev &sd = s_sd[seq & 1];
            const OctTypeMeta &M = s_to->type[r.S];
            const int S = r.S, band = r.band, B = 2 * H;
            const int nx = sd.n[0], ny = sd.n[1], nz = sd.n[2];
            const long long nxy = (long long)nx * ny;
            // global coordinate of buffer coordinate u along axis d: base[d] + sgn[d] u
            int base[3], sgn[3];
            for (int d = 0; d < 3; ++d) {
                const int C = (band & 1) * H + r.j[d] * B + (((S >> d) & 1) ? 0 : H);
                const int up = (rank >> d) & 1;
                base[d] = up ? C - 1 : C;
                sgn[d] = up ? 1 : -1;
            }
            auto gx = [&](int d, int u, int n) { return wrap_axis(base[d] + sgn[d] * u, n); };
            const long long slot_off = (long long)(band & 1) * sd.mb_slot;
            if (wt < 64) {
                // mailbox of the consumer with code (Sc | G << 3): octant rank ^ G, one
                // position further along the flipped axes where rank's bit equals G's
                const int Sc = wt & 7, G = wt >> 3;
                const int F = Sc ^ S, step = F & ~((int)rank ^ G) & 7;
                int jc = 0, mul = 1;
                for (int d = 0; d < 3; ++d) {
                    int v = r.j[d] + ((step >> d) & 1);
                    v -= (v >= sd.J[d]) ? sd.J[d] : 0;
                    jc += v * mul;
                    mul *= sd.J[d];
                }
                s_mb[wt] = sd.mbox + slot_off + sd.mb_type_off[Sc] +
                           ((long long)jc * 8 + (int)(rank ^ (unsigned)G)) * s_to->type[Sc].mb_size;
            }
            // ---- group 0: band base + coefficients ----
            {
                if (wt < H) cp_async16(s_coef + wt, sd.coef + band * H + wt);
                const Box3 bp = M.base_phi, bc = M.base_pc;
                const int w0 = bp.hi[0] - bp.lo[0], ncol = M.base_cols, units = ncol * M.base_runs;
                for (int u = wt; u < units; u += kOctNW) {
                    const int run = fdiv(u, M.rcp_cols);
                    const int i = u - run * ncol;
                    const int t1 = fdiv(i, M.rcp_base0);
                    const int ux = bp.lo[0] + i - t1 * w0, uy = bp.lo[1] + t1;
                    const int oxy = (ux < bc.lo[0] || ux >= bc.hi[0]) + (uy < bc.lo[1] || uy >= bc.hi[1]);
                    if (oxy > 1) continue;  // not a 7-point neighbour of the level-1 box
                    const long long gxy = (long long)gx(0, ux, nx) + (long long)nx * gx(1, uy, ny);
                    const int z0 = bp.lo[2] + 4 * run, z1 = min(z0 + 4, bp.hi[2]);
                    for (int uz = z0; uz < z1; ++uz) {
                        const int out = oxy + (uz < bc.lo[2] || uz >= bc.hi[2]);
                        if (out > 1) continue;
                        const long long gi = gxy + nxy * gx(2, uz, nz);
                        cp_async8(phi_buf[0] + (uz * P + uy) * P + ux, sd.phi + gi);
                        if (out == 0) cp_async16(pc_s + ((uz - 1) * H + (uy - 1)) * H + (ux - 1), sd.pc + gi);
                    }
                }
                cp_async_commit();
            }
            const float2 *mb_self =
                sd.mbox + slot_off + sd.mb_type_off[S] + ((long long)r.jl * 8 + (int)rank) * M.mb_size;
            auto issue_level = [&](int L) {
                if (L <= H - 1) {
                    const int nf = M.imp_full_n[L], np = M.imp_phi_n[L];
                    const float2 *mb = mb_self + M.mb_level_off[L];
                    const unsigned short *fl = s_imp + M.imp_full_off[L], *pl = s_imp + M.imp_phi_off[L];
                    float2 *dst = phi_buf[L & 1];
                    for (int i = wt; i < nf; i += kOctNW) {
                        const int c = fl[i];
                        cp_async16(pc_s + c, mb + 2 * i);
                        cp_async8(dst + oct_pidx(c), mb + 2 * nf + i);
                    }
                    for (int i = wt; i < np; i += kOctNW) cp_async8(dst + pl[i], mb + 3 * nf + i);
                }
                cp_async_commit();  // one group per level, empty or not
            };
            issue_level(1);

            const int nlev = M.levels;
            const PhysConst q = sd.q;
            int2 pre[kOctExpPrefetch];
            bool aborted = false;
            for (int k = 1; k <= nlev; ++k) {
                const float2 *__restrict__ prev_buf = phi_buf[(k - 1) & 1];
                float2 *__restrict__ cur = phi_buf[k & 1];
                issue_level(k + 1);  // lands in buffer (k+1) & 1, outside what level k reads or writes
                const int ne = k >= 2 ? M.exp_n[k - 1] : 0;
                const int2 *el = exp_all + (k >= 2 ? M.exp_off[k - 1] : 0);
                oct_prefetch(el, ne, pre, wt);
                cp_async_wait_pending(1);  // groups 0..k: base, imports of levels < k and level k's
                if (k >= 2 && wt == 0) {
                    // the neighbours' inner faces of phi(k-1)
                    const int m = (k - 1) & 1;
                    mbar_arrive_expect_tx(&s_xbar[m], (unsigned)M.xbytes[k]);
                    const unsigned long long t0 = globaltimer_ns(), limit = a.ctl->wait_limit_ns;
                    for (unsigned spin = 0; !mbar_test_parity_cluster(&s_xbar[m], xph[m]); ++spin) {
                        if ((spin & 15u) == 15u && globaltimer_ns() - t0 > limit) {
                            atomicCAS(&a.ctl->error, 0, kDevTimeout);
                            s_abort = 1;
                            break;
                        }
                    }
                    s_xpar = (int)xph[m];
                    xph[m] ^= 1u;
                }
                named_barrier(kOctBar, kOctNW);
                if (s_abort) {
                    aborted = true;
                    break;
                }
                if (k >= 2) (void)mbar_test_parity_cluster(&s_xbar[(k - 1) & 1], (unsigned)s_xpar);  // acquire
                const unsigned char *wn = M.w[k + 1];  // next level's box (0: no next level)
                const int wn0 = wn[0], wn1 = wn[1], wn2 = wn[2];
                // ---- imported face cells of phi(k) to the neighbours ----
                if (k < nlev) {
                    const int nfc = M.face_n[k];
                    const int *fe = face_all + M.face_off[k];
                    for (int i = wt; i < nfc; i += kOctNW) {
                        const int e = fe[i];
                        const int pidx = e & 0xFFFF, mask = e >> 16;
                        const float2 v = cur[pidx];
                        if (mask & 1) st_async_f2(map_shared(cur + pidx - 1, rank ^ 1u), v, xbar_remote[0][k & 1]);
                        if (mask & 2) st_async_f2(map_shared(cur + pidx - P, rank ^ 2u), v, xbar_remote[1][k & 1]);
                        if (mask & 4) st_async_f2(map_shared(cur + pidx - PP, rank ^ 4u), v, xbar_remote[2][k & 1]);
                    }
                }
                // ---- evolve the corner box of level k: the inner-face cells first (each goes to
                // its neighbour as soon as it is computed), then the interior, while the faces travel ----
                {
                    const LevelCoef co = s_coef[k - 1];
                    const int w0 = M.w[k][0], w1 = M.w[k][1], w2 = M.w[k][2];
                    const float rf[3] = {M.rcp_f[k][0], M.rcp_f[k][1], M.rcp_f[k][2]};
                    const unsigned xb[3] = {xbar_remote[0][k & 1], xbar_remote[1][k & 1], xbar_remote[2][k & 1]};
                    const int n_face = w0 * w1 * w2 == 0 ? 0 : w1 * w2 + (w0 - 1) * w2 + (w0 - 1) * (w1 - 1);
                    const int n_int = (w0 - 1) * (w1 - 1) * (w2 - 1);
#pragma unroll 1
                    for (int pass = 0; pass < 2; ++pass) {
                        const int cnt = pass ? n_int : n_face;
                        for (int i = wt; i < cnt; i += 2 * kOctNW) {
                            int ux[2], uy[2], uz[2];
                            bool on[2];
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                const int iu = i + u * kOctNW;
                                on[u] = iu < cnt;
                                oct_decode(on[u] ? iu : i, pass == 1, w0, w1, w2, rf, ux[u], uy[u], uz[u]);
                            }
                            oct_cells<2>(ux, uy, uz, on, prev_buf, cur, pc_s, co, q, wn0, wn1, wn2, rank, xb);
                        }
                    }
                }
                // ---- final surface of level k-1 (read-only data of level k-1) ----
                if (ne > 0) oct_exports(el, ne, pre, s_mb, prev_buf, pc_s, wt);
            }
            if (aborted) break;
            const float2 *last = phi_buf[nlev & 1];
            if (nlev <= H - 1) {
                const int ne = M.exp_n[nlev];
                const int2 *el = exp_all + M.exp_off[nlev];
                oct_prefetch(el, ne, pre, wt);
                named_barrier(kOctBar, kOctNW);
                oct_exports(el, ne, pre, s_mb, last, pc_s, wt);
            } else {
                named_barrier(kOctBar, kOctNW);
                // ---- the octant's part of the inverted pyramid's top: the next band's base ----
                for (int i = wt; i < H * H; i += kOctNW) {
                    const int ux = 1 + (i & (H - 1)), uy = 1 + (i >> kOctLgH);
                    const long long gxy = (long long)gx(0, ux, nx) + (long long)nx * gx(1, uy, ny);
                    for (int uz = 1; uz <= H; ++uz) {
                        const long long gi = gxy + nxy * gx(2, uz, nz);
                        __stcg(sd.phi + gi, last[(uz * P + uy) * P + ux]);
                        __stcg(sd.pc + gi, pc_s[((uz - 1) * H + (uy - 1)) * H + (ux - 1)]);
                    }
                }
            }
            named_barrier(kOctBar, kOctNW);
            if (wt == 0) {
                if (a.trace && rank == 0) a.trace[2 * (size_t)g + 1] = globaltimer_ns();
                fence_acq_rel_gpu();  // this octant's surfaces, before the manager's GPU-scope release
                red_release_cluster_add(done_remote, 1);
            }
        }
    }
    __syncwarp();
    cluster_barrier();  // no CTA leaves while another may still write into its shared memory
}

size_t region_oct_smem_bytes(int imp_units, int face_units)
{
    return (size_t)2 * kOctP * kOctP * kOctP * sizeof(float2) + (size_t)kOctH * kOctH * kOctH * sizeof(float4) +
           sizeof(TablesOct) + kMaxHOct * sizeof(LevelCoef) + (size_t)imp_units * sizeof(unsigned short) +
           (size_t)face_units * sizeof(int);
}

static void oct_config(cudaLaunchConfig_t *cfg, cudaLaunchAttribute *at, size_t smem, int clusters, cudaStream_t st)
{
    *cfg = cudaLaunchConfig_t{};
    cfg->gridDim = dim3(8 * clusters, 1, 1);
    cfg->blockDim = dim3(kOctNW + 32, 1, 1);
    cfg->dynamicSmemBytes = smem;
    cfg->stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 8;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg->attrs = at;
    cfg->numAttrs = 1;
}

cudaError_t region_oct_clusters(size_t smem, int *clusters)
{
    cudaError_t e = cudaFuncSetAttribute(region_oct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    oct_config(&cfg, at, smem, 1, nullptr);
    return cudaOccupancyMaxActiveClusters(clusters, region_oct_kernel, &cfg);
}

cudaError_t launch_region_oct(const RegionArgs &a, size_t smem, int clusters, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(region_oct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    oct_config(&cfg, at, smem, clusters, st);
    return cudaLaunchKernelEx(&cfg, region_oct_kernel, a);
}

int region_oct_workers() { return kOctNW; }

}  // namespace sp
