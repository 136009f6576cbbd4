// sp_lattice.cu -- the persistent kernel of the 4-cube lattice regions
// (paper Sec. 2, Figs. 2-5; geometry, tables and the in-place data flow in
// lattice.h).
//
// Every region is a translate of one 4-cube of 16 s^4 site-updates over 4s
// levels, whose cells and halo fit a few tens of KB of shared memory (s = 4:
// 1278 phi slots in each of two parity buffers and 878 (pi, c) slots, 34.5
// KB; 44.4 KB with the row records and the entry ring), so several regions
// run on one SM, one per CTA (five at s = 4).  A region
//   1. waits until its four predecessors (layer L - 1) have reported done,
//   2. copies in the values it does not compute (cp.async: phi of the halo
//      and the whole state of cells entering the region), straight from the
//      state arrays, all at its start and in address order (every one is
//      final by then and stays in place until the region is done; lattice.h),
//      a phi value as the 16-byte pair of sites around it where the pair's
//      other slot may take it,
//   3. evolves level by level in shared memory (the site update of
//      sp_update.h), writing every value another region needs (a per-cell
//      flag of the tables) straight into the state arrays,
//   4. reports done with a release store of its layer number.
// The per-level cell lists and the import list (lattice.h) are the same for
// every region: a level's cell entries are copied into shared memory a level
// ahead (cp.async), so no table read waits on memory.  A cell's neighbours, its
// (pi, c) slot and its site index follow from its slot and one 16-byte
// per-row record in shared memory (byte offsets; the row's wrapped (y, z)
// index is refilled for each region), and the site's x follows from the x
// field of the entry, so a site index costs no branch and no table read.
//
// Regions are handed out by ticket in layer order (one atomic per region,
// taken a region ahead; the next region's predecessor flags are read early,
// relaxed, and one fence per region serves as the release of its writes and
// the acquire of those reads).  A ticket's predecessors hold smaller tickets, and
// a CTA holding a ticket is running or will run it next, so the waits always
// end; each is bounded anyway.  The manager of the paper (Sec. 4) is thus
// reduced to a counter and one flag per region.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.h"
#include "sp_device.cuh"
#include "sp_kernels.h"

namespace sp {

namespace {

// Per-row record in shared memory (16 bytes): byte offsets, from a cell's phi
// slot, of its y - 1 / y + 1 neighbours (dy: low / high 16 bits, signed) and
// z - 1 / z + 1 neighbours (dz); the byte offset of its (pi, c) slot minus
// 16 x its phi slot; and, for the region being evolved, the row's y + n1 z
// (both wrapped into the grid).
struct alignas(16) LatRow {
    int dy, dz, dpc;
    unsigned yz;
};

// Shared-memory layout of one region (bytes): (pi, c) slots, the two phi
// buffers (an even number of slots each, so that every even slot starts a
// 16-byte pair), the row records and a ring of two levels' cell entries
// (every cp.async16 destination on a 16-byte boundary).
struct LatSmem {
    size_t pc, ph0, ph1, row, ring, total;
    __host__ __device__ LatSmem(int n_slots, int n_foot, int W, int max_cell_n)
    {
        const size_t nb = 8 * (((size_t)n_slots + 1) & ~(size_t)1);
        pc = 0;
        ph0 = 16 * (size_t)n_foot;
        ph1 = ph0 + nb;
        row = ph1 + nb;
        ring = row + 16 * (size_t)W * W;
        total = ring + 2 * 4 * (size_t)max_cell_n;
    }
};

struct LatRegion {
    int sim, L, Labs, tau_b, k_lo, k_hi;
    int c[3];        // centre, cells
    unsigned t, j;   // ticket, region within the layer (all simulations)
    long long id;    // trace / fault-injection id
    int pred[4];     // predecessors' flag indices (-1: none)
};

// Decode ticket t (no waiting).  Returns false when the tickets are exhausted.
__device__ bool lat_decode(const LatArgs &a, unsigned t, int epoch, LatRegion *out)
{
    if (t >= a.total) return false;
    const unsigned li = t / a.per_layer_all;
    const unsigned j = t - li * a.per_layer_all;
    int sim = 0;
    while (sim + 1 < a.n_sims && (long long)j >= a.sims[sim + 1].region_base) ++sim;
    const LatSimDev &sd = a.sims[sim];
    const int idx = (int)((long long)j - sd.region_base);  // < 2^31 regions per layer of one simulation
    LatGeom g;
    g.s = a.s;
    g.M[0] = sd.M[0], g.M[1] = sd.M[1], g.M[2] = sd.M[2];
    const int L = lat_min_layer() + (int)li;
    int ctr[3];
    lat_centre(g, L, idx, ctr);
    LatRegion &r = *out;
    r.sim = sim;
    r.L = L;
    r.Labs = epoch + (int)li;
    r.tau_b = 1 + a.s * L;
    r.k_lo = r.tau_b < 1 ? 1 - r.tau_b : 0;
    r.k_hi = min(a.K - 1, a.T - r.tau_b);
    for (int d = 0; d < 3; ++d) r.c[d] = a.s * ctr[d];
    r.t = t;
    r.j = j;
    r.id = sd.trace_base + (long long)li * sd.per_layer + idx;
    const long long base = (long long)((r.Labs - 1) & 3) * a.per_layer_all + sd.region_base;
    for (int i = 0; i < 4; ++i) r.pred[i] = li > 0 ? (int)(base + lat_pred_of<int>(g, ctr, i)) : -1;
    return true;
}

// Control thread: bounded wait until every predecessor of r has reported done
// (acquire).  False (and the error word set) when a wait gave up or another
// CTA failed.
__device__ bool lat_wait(const LatArgs &a, const LatRegion &r)
{
    const int need = r.Labs - 1;
    const unsigned long long t0 = globaltimer_ns();
    const unsigned long long limit = a.ctl->wait_limit_ns;
    for (int i = 0; i < 4; ++i) {
        if (r.pred[i] < 0) continue;
        unsigned spins = 0;
        while (ld_acquire_gpu(a.flags + r.pred[i]) < need) {
            if ((++spins & 63u) == 0) {
                if (ld_relaxed_gpu(&a.ctl->error) != 0) return false;
                if (globaltimer_ns() - t0 > limit) {
                    if (atomicCAS(&a.ctl->error, 0, (int)kDevTimeout) == 0) a.ctl->error_info = (int)r.t;
                    return false;
                }
            }
            __nanosleep(100);
        }
    }
    return true;
}

// Site index of the cell of entry e in a row with wrapped index yz = y + n1 z:
// x = (centre x - 2s) + the entry's x field, wrapped once (branch-free;
// regions are narrower than the grid, so one wrap suffices).
__device__ __forceinline__ unsigned long long lat_site(uint32_t e, unsigned yz, int cx, int n0)
{
    int x = cx + lat_rx2s(e);
    x += x < 0 ? n0 : 0;
    x -= x >= n0 ? n0 : 0;
    return (unsigned long long)yz * (unsigned)n0 + (unsigned)x;
}

// A region's imports: the list of all of them (imp_all, in address order;
// entries (entry, import level)), loaded in batches, of which a thread loads
// lat_imp_batch entries before using any, so the entry reads overlap: with
// 128 workers 20 cover a whole region of edge 16 (2437 imports) in one round
// (measured at 240^3, 128 workers: 8, 16, 20, 24 entries 1.194e11,
// 1.220e11, 1.226e11, 1.221e11 site-updates/s); 160 and 192 workers keep 8
// (their register budget at 5 CTAs per SM, 56 registers, spills with more).
template <int NW>
__host__ __device__ constexpr int lat_imp_batch()
{
    return (NW == 160 || NW == 192) ? 8 : 20;
}

// One batch of import entries, i0 + u NW (padding: level ~0u).
template <int NW>
__device__ __forceinline__ void load_import_batch(uint2 (&ie)[lat_imp_batch<NW>()], const uint2 *__restrict__ imp_all,
                                                  int n, int i0)
{
#pragma unroll
    for (int u = 0; u < lat_imp_batch<NW>(); ++u)
        ie[u] = i0 + u * NW < n ? __ldg(imp_all + i0 + u * NW) : make_uint2(0u, ~0u);
}

// cp.async of one batch of imports of levels k_lo..k_hi: phi of one level
// into its buffer, and the (pi, c) of full imports.  pair_bit: a phi import
// whose entry has this bit (kLatImpPair for a region that loads nothing else
// into its phi buffers at its start, kLatImpPairRow for one cut by the call's
// first level, lattice.h) and whose slot and site have the same parity copies
// the aligned 16-byte site pair into the aligned slot pair (L2 only): the
// other slot of the pair then receives the same bytes any other load of it
// does, or is written by the region only at a later level, and an 8-byte copy
// would have to allocate in L1.
template <int NW>
__device__ __forceinline__ void issue_import_batch(const uint2 (&ie)[lat_imp_batch<NW>()], int k_lo, int k_hi, int cx,
                                                   int n0, const LatRow *s_row, char *pcb, char *ph0, char *ph1,
                                                   const float2 *g0, const float2 *g1, const float4 *gpc, uint32_t pair_bit)
{
#pragma unroll
    for (int u = 0; u < lat_imp_batch<NW>(); ++u) {
        if ((int)ie[u].y < k_lo || (int)ie[u].y > k_hi) continue;  // (also the padding, level ~0u)
        const uint32_t e = ie[u].x;
        const int sl = lat_slot(e), row = lat_row(e);
        const bool b = (e & kLatImpBuf) != 0;  // phi buffer (k - 1) & 1; g0 / g1 are its arrays
        const LatRow rr = s_row[row];
        const unsigned long long g = lat_site(e, rr.yz, cx, n0);
        char *dst = (b ? ph1 : ph0) + (sl << 3);
        const float2 *src = (b ? g1 : g0) + g;
        if ((e & pair_bit) && ((sl ^ (int)g) & 1) == 0)
            cp_async16(dst - ((sl & 1) << 3), src - (g & 1));
        else
            cp_async8(dst, src);
        if (e & kLatImpFull) cp_async16(pcb + (sl << 4) + rr.dpc, gpc + g);
    }
}

// cp.async of the cell entries of one level (16-byte chunks; lists are padded)
template <int NW>
__device__ __forceinline__ void copy_entries(uint32_t *ring, const uint32_t *__restrict__ tab, int off, int n)
{
    const int n4 = (n + 3) & ~3;
    for (int i = 4 * (int)threadIdx.x; i < n4; i += 4 * NW) cp_async16(ring + i, tab + off + i);
}

__device__ __forceinline__ float2 ld_f2(const char *base, int off) { return *reinterpret_cast<const float2 *>(base + off); }

// CTAs per SM the register budget is set for (shared memory allows 5 regions
// of edge 16 per SM, 2 of edge 20; measured at 240^3 with all imports at the
// region's start: 128 workers at 5 per SM 1.226e11 site-updates/s, 160 at 5
// per SM 1.204e11, 192 at 5 per SM (56 registers) 1.182e11, at 4 per SM
// (72 registers) 1.020e11).
template <int NW>
constexpr int lat_min_blocks()
{
    return NW <= 64 ? 8 : NW <= 192 ? 5 : NW <= 256 ? 2 : 1;
}

template <int NW>
__global__ void __launch_bounds__(NW, lat_min_blocks<NW>())
    lattice_kernel(const LatArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_cell_off[4 * kLatMaxS + 1], s_cell_n[4 * kLatMaxS];
    __shared__ LatRegion s_reg;
    __shared__ int s_stop;
    const int tid = threadIdx.x;
    const int R = 2 * a.s, W = 4 * a.s + 1, WW = W * W;
    const int max_cell_n = a.max_cell_n;
    const LatSmem L(a.n_slots, a.n_foot, W, max_cell_n);
    char *s_pcb = reinterpret_cast<char *>(smem + L.pc);
    char *s_ph0 = reinterpret_cast<char *>(smem + L.ph0);
    char *s_ph1 = reinterpret_cast<char *>(smem + L.ph1);
    LatRow *s_row = reinterpret_cast<LatRow *>(smem + L.row);
    uint32_t *s_ring = reinterpret_cast<uint32_t *>(smem + L.ring);
    const uint32_t *__restrict__ g_cell = a.cell;
    if (tid <= a.K) {
        s_cell_off[tid] = a.cell_off[tid];
        if (tid < a.K) s_cell_n[tid] = a.cell_n[tid];
    }
    for (int i = tid; i < WW; i += NW) {
        const uint64_t nb = a.row_nb[i];
        LatRow r;
        r.dy = (lat_dym(nb) * 8 & 0xffff) | (lat_dyp(nb) * 8) << 16;
        r.dz = (lat_dzm(nb) * 8 & 0xffff) | (lat_dzp(nb) * 8) << 16;
        r.dpc = a.row_pc[i] * 16;
        r.yz = 0;
        s_row[i] = r;
    }
    // The control thread is the last one: cells are dealt out from thread 0,
    // so it has the least evolution work at every level.  Its state: the next
    // ticket, and early (relaxed) reads of the flags of the region that
    // ticket names.
    const int ctl = NW - 1;
    unsigned next = 0;
    int epoch = 0;
    int fv[4] = {0, 0, 0, 0};
    bool early = false;
    if (tid == ctl) {
        epoch = *(volatile int *)&a.ctl->epoch;
        s_stop = 0;
        const unsigned t = atomicAdd(&a.ctl->head, 1u);
        if (!lat_decode(a, t, epoch, &s_reg) || !lat_wait(a, s_reg))
            s_stop = 1;
        else
            next = atomicAdd(&a.ctl->head, 1u);
    }
    __syncthreads();
    while (!s_stop) {
        const LatRegion r = s_reg;
        const LatSimDev &sdr = a.sims[r.sim];
        const int n0 = sdr.n[0], cx = r.c[0] - R;
        // the first batch of import entries (their loads overlap the row set-up)
        uint2 ie[lat_imp_batch<NW>()];
        load_import_batch<NW>(ie, a.imp_all, a.n_imp_all, tid);
        // the rows' wrapped y + n1 z for this region (row = (y + 2s) W + z + 2s)
        {
            const int n1 = sdr.n[1], n2 = sdr.n[2];
            const unsigned wdiv = lat_row_div(a.s);
            for (int i = tid; i < WW; i += NW) {
                const int y2s = lat_row_y2s(i, wdiv);
                int y = r.c[1] + y2s - R, z = r.c[2] + (i - y2s * W) - R;
                y += y < 0 ? n1 : 0;
                y -= y >= n1 ? n1 : 0;
                z += z < 0 ? n2 : 0;
                z -= z >= n2 ? n2 : 0;
                s_row[i].yz = (unsigned)y + (unsigned)n1 * (unsigned)z;
            }
        }
        const PhysConst q = sdr.q;
        const LevelCoef *__restrict__ coef = sdr.coef;
        float2 *const g_even = sdr.phi0;
        float2 *const g_odd = sdr.phi1;
        float4 *const gpc = sdr.pc;
        unsigned long long t_start = 0;
        if (tid == ctl && a.trace) t_start = globaltimer_ns();
        const int par0 = r.tau_b & 1;  // level k of the region is global parity par0 ^ (k & 1)
        __syncthreads();  // row indices written

        // a region cut by the call's first level: its own cells of level k_lo - 1, whole
        if (r.k_lo > 0) {
            const int kb = r.k_lo - 1;
            char *phb = (kb & 1) ? s_ph1 : s_ph0;
            const float2 *gp = (par0 ^ (kb & 1)) ? g_odd : g_even;
            const int off = s_cell_off[kb], n = s_cell_n[kb];
            for (int i = tid; i < n; i += NW) {
                const uint32_t e = __ldg(g_cell + off + i);
                const int sl = lat_slot(e), row = lat_row(e);
                const LatRow rr = s_row[row];
                const unsigned long long g = lat_site(e, rr.yz, cx, n0);
                cp_async8(phb + (sl << 3), gp + g);
                cp_async16(s_pcb + (sl << 4) + rr.dpc, gpc + g);
            }
        }
        copy_entries<NW>(s_ring + (r.k_lo & 1) * max_cell_n, g_cell, s_cell_off[r.k_lo], s_cell_n[r.k_lo]);
        // every import of the region's levels; buffer b holds values of local
        // levels of parity b, global parity par0 ^ b
        for (int i0 = tid;;) {
            issue_import_batch<NW>(ie, r.k_lo, r.k_hi, cx, n0, s_row, s_pcb, s_ph0, s_ph1, par0 ? g_odd : g_even,
                                   par0 ? g_even : g_odd, gpc, r.k_lo == 0 ? kLatImpPair : kLatImpPairRow);
            i0 += lat_imp_batch<NW>() * NW;
            if (i0 >= a.n_imp_all) break;
            load_import_batch<NW>(ie, a.imp_all, a.n_imp_all, i0);
        }
        LevelCoef co = coef[r.tau_b + r.k_lo - 1];
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        for (int k = r.k_lo; k <= r.k_hi; ++k) {
            const int odd = k & 1;
            const char *rd = odd ? s_ph0 : s_ph1;
            char *wr = odd ? s_ph1 : s_ph0;
            LevelCoef co_next = co;
            if (k < r.k_hi) {
                // the cell entries of level k + 1
                copy_entries<NW>(s_ring + ((k + 1) & 1) * max_cell_n, g_cell, s_cell_off[k + 1], s_cell_n[k + 1]);
                cp_async_commit();
                co_next = coef[r.tau_b + k];
            }
            if (tid == ctl && k == r.k_lo) {
                // every thread has copied the descriptor: decode the next
                // region into it and read its predecessors' flags early
                early = lat_decode(a, next, epoch, &s_reg);
                if (early)
                    for (int i = 0; i < 4; ++i)
                        fv[i] = s_reg.pred[i] >= 0 ? ld_relaxed_gpu(a.flags + s_reg.pred[i]) : 0x7fffffff;
            }
            float2 *gout = (par0 ^ odd) ? g_odd : g_even;
            const uint32_t exp_phi = k == r.k_hi ? ~0u : kLatExpPhi;  // the call's last level: export all
            const uint32_t exp_pc = k == r.k_hi ? ~0u : kLatExpPc;
            const int n = s_cell_n[k];
            const uint32_t *ent = s_ring + odd * max_cell_n;
#pragma unroll 1  // measured: unrolling 2, 3 or 4 cells per step is slower
            for (int i = tid; i < n; i += NW) {
                const uint32_t e = ent[i];
                const int sl = lat_slot(e), row = lat_row(e);
                const LatRow rr = s_row[row];
                const int own = sl << 3;
                const int pcoff = (sl << 4) + rr.dpc;
                const float4 v = *reinterpret_cast<const float4 *>(s_pcb + pcoff);
                float2 pi = make_float2(v.x, v.y), cc = make_float2(v.z, v.w);
                const float2 out = site_update(ld_f2(rd, own), ld_f2(rd, own - 8), ld_f2(rd, own + 8),
                                               ld_f2(rd, own + (int)(short)rr.dy), ld_f2(rd, own + (rr.dy >> 16)),
                                               ld_f2(rd, own + (int)(short)rr.dz), ld_f2(rd, own + (rr.dz >> 16)), pi,
                                               cc, co, q);
                *reinterpret_cast<float2 *>(wr + own) = out;
                const float4 pcv = make_float4(pi.x, pi.y, cc.x, cc.y);
                *reinterpret_cast<float4 *>(s_pcb + pcoff) = pcv;
                if (e & (exp_phi | exp_pc)) {
                    const unsigned long long g = lat_site(e, rr.yz, cx, n0);
                    if (e & exp_phi) __stcg(gout + g, out);  // L2 only: read by other SMs
                    if (e & exp_pc) __stcg(gpc + g, pcv);
                }
            }
            cp_async_wait_all();
            __syncthreads();
            co = co_next;
        }
        if (tid == ctl) {
            if (a.trace) {
                a.trace[2 * r.id] = t_start;
                a.trace[2 * r.id + 1] = globaltimer_ns();
            }
            // One fence: release of this region's writes (made before the
            // barrier above by every thread) to the flag store after it, and
            // acquire for the early flag reads before it.
            fence_acq_rel_gpu();
            if (r.id != a.fault_drop) st_relaxed_gpu(a.flags + (size_t)((r.Labs & 3) * a.per_layer_all) + r.j, r.Labs);
            if (!early) {
                s_stop = 1;
            } else {
                const int need = s_reg.Labs - 1;
                bool ready = true;
                for (int i = 0; i < 4; ++i) ready = ready && fv[i] >= need;
                if (!ready && !lat_wait(a, s_reg)) s_stop = 1;
                if (!s_stop) next = atomicAdd(&a.ctl->head, 1u);
            }
        }
        __syncthreads();
    }
}

// Before every lattice call: a fresh ticket counter and error word, and the
// call's layers numbered above every done flag written before.
__global__ void lattice_reset_kernel(Ctl *ctl, int layers)
{
    ctl->head = 0;
    ctl->error = 0;
    ctl->error_info = 0;
    lat_next_epoch(&ctl->last_layer, layers, &ctl->epoch);
}

template <int NW>
cudaError_t lattice_launch_t(const LatArgs &a, size_t smem, int grid, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(lattice_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    lattice_kernel<NW><<<grid, NW, smem, st>>>(a);
    return cudaGetLastError();
}

const void *lattice_fn(int threads)
{
    switch (threads) {
    case 64:
        return (const void *)lattice_kernel<64>;
    case 128:
        return (const void *)lattice_kernel<128>;
    case 192:
        return (const void *)lattice_kernel<192>;
    case 256:
        return (const void *)lattice_kernel<256>;
    case 512:
        return (const void *)lattice_kernel<512>;
    default:
        return nullptr;
    }
}

}  // namespace

size_t lattice_smem_bytes(int n_slots, int n_foot, int rb_side, int max_cell_n)
{
    return LatSmem(n_slots, n_foot, rb_side, max_cell_n).total;
}

bool lattice_valid_threads(int threads) { return lattice_fn(threads) != nullptr; }

cudaError_t lattice_occupancy(int threads, size_t smem, int *blocks_per_sm)
{
    *blocks_per_sm = 0;
    const void *f = lattice_fn(threads);
    if (!f) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, threads, smem);
}

cudaError_t launch_lattice_reset(Ctl *ctl, int layers, cudaStream_t st)
{
    lattice_reset_kernel<<<1, 1, 0, st>>>(ctl, layers);
    return cudaGetLastError();
}

cudaError_t launch_lattice(const LatArgs &a, int threads, size_t smem, int grid, cudaStream_t st)
{
    switch (threads) {
    case 64:
        return lattice_launch_t<64>(a, smem, grid, st);
    case 128:
        return lattice_launch_t<128>(a, smem, grid, st);
    case 192:
        return lattice_launch_t<192>(a, smem, grid, st);
    case 256:
        return lattice_launch_t<256>(a, smem, grid, st);
    case 512:
        return lattice_launch_t<512>(a, smem, grid, st);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace sp
