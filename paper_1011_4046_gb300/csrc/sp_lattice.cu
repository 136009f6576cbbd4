// sp_lattice.cu -- the persistent kernel of the 4-cube lattice regions
// (paper Sec. 2, Figs. 2-5; geometry, tables and the in-place data flow in
// lattice.h).
//
// Every region is a translate of one 4-cube of 16 s^4 site-updates over 4s
// levels, whose cells and halo fit a few tens of KB of shared memory (s = 4:
// 1225 phi slots in two parity buffers and 847 (pi, c) slots, 33 KB), so
// several regions run on one SM, one per CTA.  A region
//   1. waits until its four predecessors (layer L - 1) have reported done,
//   2. copies in the values it does not compute (cp.async, one level ahead of
//      the evolution: phi of the halo and the whole state of cells entering
//      the region), straight from the state arrays,
//   3. evolves level by level in shared memory (the site update of
//      sp_update.h), writing every value another region needs (a per-cell
//      flag of the tables) straight into the state arrays,
//   4. reports done with a release store of its layer number.
// Regions are handed out by ticket in layer order (one atomic per region,
// taken a region ahead).  A ticket's predecessors hold smaller tickets, and
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

struct LatRegion {
    int sim, L, Labs, tau_b, k_lo, k_hi;
    int c[3];        // centre, cells
    unsigned t, j;   // ticket, region within the layer (all simulations)
    long long id;    // trace / fault-injection id
};

__device__ __forceinline__ int sext10(unsigned v) { return ((int)(v & 1023u) ^ 512) - 512; }

__device__ __forceinline__ long long site_at(const LatSimDev &sd, const int c[3], unsigned rec, int R)
{
    int x = c[0] + (int)(rec & 31u) - R;
    int y = c[1] + (int)((rec >> 5) & 31u) - R;
    int z = c[2] + (int)((rec >> 10) & 31u) - R;
    x += x < 0 ? sd.n[0] : 0;
    x -= x >= sd.n[0] ? sd.n[0] : 0;
    y += y < 0 ? sd.n[1] : 0;
    y -= y >= sd.n[1] ? sd.n[1] : 0;
    z += z < 0 ? sd.n[2] : 0;
    z -= z >= sd.n[2] ? sd.n[2] : 0;
    return (long long)x + (long long)sd.n[0] * ((long long)y + (long long)sd.n[1] * z);
}

// Thread 0: decode ticket t and wait (bounded) for its predecessors.  Sets
// *stop when the tickets are exhausted or a wait gave up.
__device__ void lat_claim(const LatArgs &a, unsigned t, int epoch, LatRegion *out, int *stop)
{
    if (t >= a.total) {
        *stop = 1;
        return;
    }
    const unsigned li = t / a.per_layer_all;
    const unsigned j = t - li * a.per_layer_all;
    int sim = 0;
    while (sim + 1 < a.n_sims && (long long)j >= a.sims[sim + 1].region_base) ++sim;
    const LatSimDev &sd = a.sims[sim];
    const long long idx = (long long)j - sd.region_base;
    LatGeom g;
    g.s = a.s;
    g.M[0] = sd.M[0], g.M[1] = sd.M[1], g.M[2] = sd.M[2];
    const int L = lat_min_layer() + (int)li;
    int ctr[3];
    lat_centre(g, L, idx, ctr);
    LatRegion r;
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
    if (li > 0) {
        const unsigned long long t0 = globaltimer_ns();
        const unsigned long long limit = a.ctl->wait_limit_ns;
        const int need = r.Labs - 1;
        const int *fl = a.flags + (size_t)((need & 3) * a.per_layer_all) + sd.region_base;
        for (int i = 0; i < 4; ++i) {
            const int *f = fl + lat_pred(g, L, idx, i);
            unsigned spins = 0;
            while (ld_acquire_gpu(f) < need) {
                if ((++spins & 63u) == 0) {
                    if (ld_relaxed_gpu(&a.ctl->error) != 0) {
                        *stop = 1;
                        return;
                    }
                    if (globaltimer_ns() - t0 > limit) {
                        if (atomicCAS(&a.ctl->error, 0, (int)kDevTimeout) == 0) a.ctl->error_info = (int)t;
                        *stop = 1;
                        return;
                    }
                }
                __nanosleep(100);
            }
        }
    }
    *out = r;
}

// Copies (cp.async) of the values imported before level k: phi(k - 1) of the
// halo into phi buffer (k - 1) & 1, and (pi, c)(k - 1) of cells entering.
template <int NW>
__device__ __forceinline__ void lat_imports(const LatArgs &a, const LatSimDev &sd, const LatRegion &r, int k, int lo,
                                            int hi, float4 *s_pc, float2 *s_ph, const float2 *gphi, int R)
{
    for (int i = lo + (int)threadIdx.x; i < hi; i += NW) {
        const unsigned e = __ldg(a.imp + i);
        const unsigned sl = e & 0x7fffu;
        const unsigned rec = __ldg(a.slot_rec + sl);
        const long long g = site_at(sd, r.c, rec, R);
        cp_async8(s_ph + sl, gphi + g);
        if (e & kLatImpFull) cp_async16(s_pc + ((rec >> 15) & 0xfffu), sd.pc + g);
    }
}

constexpr int kLatMinBlocks = 6;

template <int NW>
__global__ void __launch_bounds__(NW, (NW <= 128 ? kLatMinBlocks : 2)) lattice_kernel(const LatArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_cell_off[4 * kLatMaxS + 1], s_imp_off[4 * kLatMaxS + 1];
    __shared__ LatRegion s_reg;
    __shared__ int s_stop;
    float4 *s_pc = reinterpret_cast<float4 *>(smem);
    float2 *s_ph0 = reinterpret_cast<float2 *>(smem + 16 * (size_t)a.n_foot);
    float2 *s_ph1 = s_ph0 + a.n_slots;
    const int tid = threadIdx.x;
    const int R = 2 * a.s;
    if (tid <= a.K) {
        s_cell_off[tid] = a.cell_off[tid];
        s_imp_off[tid] = a.imp_off[tid];
    }
    unsigned next = 0;
    int epoch = 0;
    if (tid == 0) {
        epoch = *(volatile int *)&a.ctl->epoch;
        s_stop = 0;
        next = atomicAdd(&a.ctl->head, 1u);
        lat_claim(a, next, epoch, &s_reg, &s_stop);
        if (!s_stop) next = atomicAdd(&a.ctl->head, 1u);
    }
    __syncthreads();
    while (!s_stop) {
        const LatRegion r = s_reg;
        const LatSimDev &sd = a.sims[r.sim];
        unsigned long long t_start = 0;
        if (tid == 0 && a.trace) t_start = globaltimer_ns();
        const PhysConst q = sd.q;
        float2 *const g_even = sd.phi0, *const g_odd = sd.phi1;
        const int par0 = r.tau_b & 1;  // level k of the region is global parity par0 ^ (k & 1)
        // a region cut by the call's first level: its own cells of level k_lo - 1, whole
        if (r.k_lo > 0) {
            const int kb = r.k_lo - 1;
            float2 *s_ph = (kb & 1) ? s_ph1 : s_ph0;
            const float2 *gp = (par0 ^ (kb & 1)) ? g_odd : g_even;
            for (int i = s_cell_off[kb] + tid; i < s_cell_off[kb + 1]; i += NW) {
                const unsigned long long e = __ldg(a.cell + i);
                const unsigned sl = (unsigned)e & 0xfffu;
                const long long g = site_at(sd, r.c, __ldg(a.slot_rec + sl), R);
                cp_async8(s_ph + sl, gp + g);
                cp_async16(s_pc + ((unsigned)(e >> 12) & 0xfffu), sd.pc + g);
            }
        }
        {
            const int kb = r.k_lo - 1;
            lat_imports<NW>(a, sd, r, r.k_lo, s_imp_off[r.k_lo], s_imp_off[r.k_lo + 1], s_pc, (kb & 1) ? s_ph1 : s_ph0,
                            (par0 ^ (kb & 1)) ? g_odd : g_even, R);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        for (int k = r.k_lo; k <= r.k_hi; ++k) {
            const int odd = k & 1;
            const float2 *rd = odd ? s_ph0 : s_ph1;
            float2 *wr = odd ? s_ph1 : s_ph0;
            if (k < r.k_hi) {  // next level's imports: values of level k, into buffer k & 1
                lat_imports<NW>(a, sd, r, k + 1, s_imp_off[k + 1], s_imp_off[k + 2], s_pc, wr, (par0 ^ odd) ? g_odd : g_even,
                                R);
                cp_async_commit();
            }
            const LevelCoef co = sd.coef[r.tau_b + k - 1];
            float2 *gout = (par0 ^ odd) ? g_odd : g_even;
            const bool all = k == r.k_hi;
            for (int i = s_cell_off[k] + tid; i < s_cell_off[k + 1]; i += NW) {
                const unsigned long long e = __ldg(a.cell + i);
                const int sl = (int)((unsigned)e & 0xfffu);
                const int pcx = (int)((unsigned)(e >> 12) & 0xfffu);
                const int ym = (int)(signed char)(unsigned char)(e >> 24);
                const int yp = (int)(signed char)(unsigned char)(e >> 32);
                const int zm = sext10((unsigned)(e >> 40));
                const int zp = sext10((unsigned)(e >> 50));
                const float4 v = s_pc[pcx];
                float2 pi = make_float2(v.x, v.y), cc = make_float2(v.z, v.w);
                const float2 out = site_update(rd[sl], rd[sl - 1], rd[sl + 1], rd[sl + ym], rd[sl + yp], rd[sl + zm],
                                               rd[sl + zp], pi, cc, co, q);
                wr[sl] = out;
                s_pc[pcx] = make_float4(pi.x, pi.y, cc.x, cc.y);
                const bool ephi = all || (e & kLatExpPhi), epc = all || (e & kLatExpPc);
                if (ephi || epc) {
                    const long long g = site_at(sd, r.c, __ldg(a.slot_rec + sl), R);
                    if (ephi) gout[g] = out;
                    if (epc) sd.pc[g] = make_float4(pi.x, pi.y, cc.x, cc.y);
                }
            }
            cp_async_wait_all();
            __syncthreads();
        }
        if (tid == 0) {
            if (a.trace) {
                a.trace[2 * r.id] = t_start;
                a.trace[2 * r.id + 1] = globaltimer_ns();
            }
            if (r.id != a.fault_drop) {
                fence_acq_rel_gpu();
                st_release_gpu(a.flags + (size_t)((r.Labs & 3) * a.per_layer_all) + r.j, r.Labs);
            }
            lat_claim(a, next, epoch, &s_reg, &s_stop);
            if (!s_stop) next = atomicAdd(&a.ctl->head, 1u);
        }
        __syncthreads();
    }
}

// Before every lattice call: a fresh ticket counter and error word, and the
// call's layers numbered last_layer + 1 .. last_layer + layers, above every
// done flag written before (the flags start at 0 and last_layer at 0).
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

}  // namespace

size_t lattice_smem_bytes(int n_slots, int n_foot) { return 16 * (size_t)n_foot + 16 * (size_t)n_slots; }

bool lattice_valid_threads(int threads) { return threads == 64 || threads == 128 || threads == 256; }

cudaError_t lattice_occupancy(int threads, size_t smem, int *blocks_per_sm)
{
    *blocks_per_sm = 0;
    const void *f = threads == 64 ? (const void *)lattice_kernel<64>
                    : threads == 128 ? (const void *)lattice_kernel<128>
                                     : (const void *)lattice_kernel<256>;
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
    case 256:
        return lattice_launch_t<256>(a, smem, grid, st);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace sp
