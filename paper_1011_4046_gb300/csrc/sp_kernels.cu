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

__device__ __forceinline__ int wrap_axis(int p, int n)
{
    p += (p < 0) ? n : 0;
    p -= (p >= n) ? n : 0;
    return p;
}

// ------------------------------------------------------------ queue reset
__global__ void reset_kernel(RegionArgs a)
{
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        a.ctl->head = 0;
        a.ctl->tail = a.n_seed;
        a.ctl->error = 0;
        a.ctl->error_info = 0;
        a.ctl->completed = 0;
    }
    if (t >= a.total) return;
    const int s = find_sim(a, t);
    const SimDev &sd = a.sims[s];
    const TablesDev *T = sd.tab;
    const unsigned local = t - sd.tile_base;
    const unsigned per_band = 8u * (unsigned)sd.Jtot;
    const unsigned band = local / per_band;
    const int S = (int)((local - band * per_band) / (unsigned)sd.Jtot);
    a.counters[t] = T->same_preds[S] + (band > 0 ? T->prev_preds[S] : 0);
    // queue position t: the first n_seed positions hold the band-0 pyramids
    int v = -1;
    if (t < a.n_seed) {
        int lo = 0, hi = a.n_sims - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (a.sims[mid].seed_base <= t)
                lo = mid;
            else
                hi = mid - 1;
        }
        v = (int)(a.sims[lo].tile_base + (t - a.sims[lo].seed_base));
    }
    a.queue[t] = v;
}

// ------------------------------------------------------------ queue pop
// Returns a region id, or -1 when the launch is out of work, or -2 on error.
// Every wait is bounded by ctl->wait_limit_ns.
__device__ int pop_region(const RegionArgs &a)
{
    const unsigned idx = atomicAdd(&a.ctl->head, 1u);
    if (idx >= a.total) return -1;
    const unsigned long long limit = a.ctl->wait_limit_ns;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned spin = 0;; ++spin) {
        int v = ld_acquire_gpu(a.queue + idx);
        if (v >= 0) return v;
        if (ld_relaxed_gpu(&a.ctl->error) != 0) return -2;
        if ((spin & 15u) == 15u && globaltimer_ns() - t0 > limit) {
            atomicCAS(&a.ctl->error, 0, kDevTimeout);
            atomicExch(&a.ctl->error_info, (int)idx);
            return -2;
        }
        __nanosleep(100);
    }
}

// ------------------------------------------------------------ region kernel
// Shared memory: two phi buffers (levels of alternating parity) of (B+2)^3
// float2 for the region box plus its halo, and one float4 (pi, c) per own
// cell (B^3).  Imports of level k land in the level-k phi buffer while level k
// is being computed (disjoint cells), so their latency hides behind the
// compute of that level.
template <int NT>
__global__ void __launch_bounds__(NT) region_kernel(RegionArgs a, int max_P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_region;
    const int tid = threadIdx.x;
    float2 *phi_buf0 = reinterpret_cast<float2 *>(smem_raw);
    float2 *phi_buf1 = phi_buf0 + max_P * max_P * max_P;
    float4 *pc_s = reinterpret_cast<float4 *>(phi_buf1 + max_P * max_P * max_P);

    for (;;) {
        __syncthreads();
        if (tid == 0) s_region = pop_region(a);
        __syncthreads();
        const int g = s_region;
        if (g < 0) break;
        unsigned long long t_start = 0;
        if (a.trace && tid == 0) t_start = globaltimer_ns();

        const int s = find_sim(a, (unsigned)g);
        const SimDev &sd = a.sims[s];
        const TablesDev *__restrict__ T = sd.tab;
        const int B = sd.B, H = sd.H, P = sd.P;
        const unsigned local = (unsigned)g - sd.tile_base;
        const unsigned per_band = 8u * (unsigned)sd.Jtot;
        const int band = (int)(local / per_band);
        const int rem = (int)(local - (unsigned)band * per_band);
        const int S = rem / sd.Jtot;
        const int jl = rem - S * sd.Jtot;
        int j[3];
        j[0] = jl % sd.J[0];
        j[1] = (jl / sd.J[0]) % sd.J[1];
        j[2] = jl / (sd.J[0] * sd.J[1]);
        const int o = (band & 1) * H;
        int gbase[3];  // global coordinate of local u = 0 along each axis
        for (int d = 0; d < 3; ++d) gbase[d] = o + j[d] * B - (((S >> d) & 1) ? H + 1 : 1);
        const int nx = sd.n[0], ny = sd.n[1], nz = sd.n[2];
        const long long slot = (long long)(band & 1) * sd.mb_slot;

        // ---- level 0: the band base (tops of the previous band) ----
        {
            const Box3 bp = T->base_phi[S];
            const Box3 bc = T->base_pc[S];
            const int w0 = bp.hi[0] - bp.lo[0], w1 = bp.hi[1] - bp.lo[1];
            const int cnt = w0 * w1 * (bp.hi[2] - bp.lo[2]);
            for (int i = tid; i < cnt; i += NT) {
                const int ux = bp.lo[0] + i % w0;
                const int t1 = i / w0;
                const int uy = bp.lo[1] + t1 % w1;
                const int uz = bp.lo[2] + t1 / w1;
                const int out = (ux < bc.lo[0] || ux >= bc.hi[0]) + (uy < bc.lo[1] || uy >= bc.hi[1]) +
                                (uz < bc.lo[2] || uz >= bc.hi[2]);
                if (out > 1) continue;  // not a 7-point neighbour of A(1)
                const int gx = wrap_axis(gbase[0] + ux, nx);
                const int gy = wrap_axis(gbase[1] + uy, ny);
                const int gz = wrap_axis(gbase[2] + uz, nz);
                const long long gi = (long long)gx + (long long)nx * ((long long)gy + (long long)ny * gz);
                const int pidx = (uz * P + uy) * P + ux;
                cp_async8(phi_buf0 + pidx, sd.phi + gi);
                if (out == 0) {
                    const int cidx = ((uz - 1) * B + (uy - 1)) * B + (ux - 1);
                    float2 *pc2 = reinterpret_cast<float2 *>(pc_s + cidx);
                    cp_async8(pc2, sd.pi + gi);
                    cp_async8(pc2 + 1, sd.c + gi);
                }
            }
            cp_async_commit();
            cp_async_wait_all();
            __syncthreads();
        }

        const int nlev = T->levels[S];
        const float2 *mb_self = sd.mbox + slot + sd.mb_type_off[S] + (long long)jl * T->mb_size[S];
        for (int k = 1; k <= nlev; ++k) {
            const float2 *__restrict__ prev = (k & 1) ? phi_buf0 : phi_buf1;
            float2 *__restrict__ cur = (k & 1) ? phi_buf1 : phi_buf0;
            // ---- sloped initial surface of level k (needed by level k+1) ----
            if (k <= H - 1 && S != 0) {
                const float2 *mb = mb_self + T->mb_level_off[S][k];
                const int nf = T->imp_full_n[S][k], np = T->imp_phi_n[S][k];
                const int *fl = T->imp_full + T->imp_full_off[S][k];
                const int *pl = T->imp_phi + T->imp_phi_off[S][k];
                for (int i = tid; i < nf; i += NT) {
                    const int e = __ldg(fl + i);
                    cp_async16(pc_s + (e >> 16), mb + 2 * i);
                    cp_async8(cur + (e & 0xFFFF), mb + 2 * nf + i);
                }
                for (int i = tid; i < np; i += NT) cp_async8(cur + __ldg(pl + i), mb + 3 * nf + i);
                cp_async_commit();
            }
            // ---- evolve the cells of level k ----
            {
                const LevelCoef co = sd.coef[band * H + k - 1];
                const PhysConst q = sd.q;
                const Box3 A = T->active[S][k];
                const int w0 = A.hi[0] - A.lo[0], w1 = A.hi[1] - A.lo[1];
                const int cnt = w0 * w1 * (A.hi[2] - A.lo[2]);
                const int PP = P * P;
                for (int i = tid; i < cnt; i += NT) {
                    const int ux = A.lo[0] + i % w0;
                    const int t1 = i / w0;
                    const int uy = A.lo[1] + t1 % w1;
                    const int uz = A.lo[2] + t1 / w1;
                    const int pidx = (uz * P + uy) * P + ux;
                    const int cidx = ((uz - 1) * B + (uy - 1)) * B + (ux - 1);
                    const float4 pc = pc_s[cidx];
                    float2 pi = make_float2(pc.x, pc.y), cc = make_float2(pc.z, pc.w);
                    const float2 nphi = site_update(prev[pidx], prev[pidx - 1], prev[pidx + 1], prev[pidx - P],
                                                    prev[pidx + P], prev[pidx - PP], prev[pidx + PP], pi, cc, co, q);
                    cur[pidx] = nphi;
                    pc_s[cidx] = make_float4(pi.x, pi.y, cc.x, cc.y);
                }
            }
            cp_async_wait_all();
            __syncthreads();
            // ---- final surfaces of level k: into the consumers' mailboxes ----
            if (k <= H - 1) {
                const int4 *el = T->exp + T->exp_off[S][k];
                const int ne = T->exp_n[S][k];
                for (int i = tid; i < ne; i += NT) {
                    const int4 e = __ldg(el + i);
                    const int Sc = e.y & 7;
                    int jc = 0, mul = 1;
                    for (int d = 0; d < 3; ++d) {
                        int v = j[d] + ((e.y >> (3 + d)) & 1);
                        v -= (v >= sd.J[d]) ? sd.J[d] : 0;
                        jc += v * mul;
                        mul *= sd.J[d];
                    }
                    float2 *mb = sd.mbox + slot + sd.mb_type_off[Sc] + (long long)jc * T->mb_size[Sc];
                    __stcg(mb + e.z, cur[e.x & 0xFFFF]);
                    if (e.w >= 0) __stcg(reinterpret_cast<float4 *>(mb + e.w), pc_s[(e.x >> 16) & 0xFFFF]);
                }
            }
            // ---- tops of the inverted pyramid: the next band's base ----
            if (k == H) {
                const int cnt = B * B * B;
                for (int i = tid; i < cnt; i += NT) {
                    const int ux = 1 + i % B;
                    const int uy = 1 + (i / B) % B;
                    const int uz = 1 + i / (B * B);
                    const int gx = wrap_axis(gbase[0] + ux, nx);
                    const int gy = wrap_axis(gbase[1] + uy, ny);
                    const int gz = wrap_axis(gbase[2] + uz, nz);
                    const long long gi = (long long)gx + (long long)nx * ((long long)gy + (long long)ny * gz);
                    const float4 pc = pc_s[i];
                    __stcg(sd.phi + gi, cur[(uz * P + uy) * P + ux]);
                    __stcg(sd.pi + gi, make_float2(pc.x, pc.y));
                    __stcg(sd.c + gi, make_float2(pc.z, pc.w));
                }
            }
            __syncthreads();
        }

        // ---- release successors (one lane per successor) ----
        if (tid < 32) {
            __threadfence();
            const int n_same = T->n_same_succ[S];
            const int n_next = (S == kTypes - 1 && band + 1 < sd.nbands) ? kMaxNextSucc : 0;
            if (tid < n_same + n_next) {
                Succ su;
                int nb;
                if (tid < n_same) {
                    su = T->same_succ[S][tid];
                    nb = band;
                } else {
                    su = T->next_succ[(band + 1) & 1][tid - n_same];
                    nb = band + 1;
                }
                int jc = 0, mul = 1;
                for (int d = 0; d < 3; ++d) {
                    int v = j[d] + su.e[d];
                    v += (v < 0) ? sd.J[d] : 0;
                    v -= (v >= sd.J[d]) ? sd.J[d] : 0;
                    jc += v * mul;
                    mul *= sd.J[d];
                }
                const unsigned t = sd.tile_base + (unsigned)((nb * 8 + su.type) * sd.Jtot + jc);
                const int old = atom_add_acq_rel_gpu(a.counters + t, -1);
                if (old == 1) {
                    const unsigned pos = atomicAdd(&a.ctl->tail, 1u);
                    st_release_gpu(a.queue + pos, (int)t);
                }
            }
            if (tid == 0) {
                atomicAdd(&a.ctl->completed, 1u);
                if (a.trace) {
                    a.trace[2 * (size_t)g] = t_start;
                    a.trace[2 * (size_t)g + 1] = globaltimer_ns();
                }
            }
        }
    }
}

// ------------------------------------------------------------ sweep kernel
// One level of the whole grid: block 32 x 8 over (x, y), each thread marches
// a chunk of z keeping phi(z-1), phi(z), phi(z+1) in registers; x and y
// neighbours come through L1.  48 bytes per site-update of HBM traffic.
__global__ void __launch_bounds__(256) sweep_kernel(const float2 *__restrict__ phi_in, float2 *__restrict__ phi_out,
                                                    float2 *__restrict__ pi, float2 *__restrict__ c, int nx, int ny,
                                                    int nz, int zchunk, const LevelCoef *__restrict__ coef, int lvl,
                                                    PhysConst q)
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
        float2 p = pi[row + x], cc = c[row + x];
        const float2 out = site_update(zcur, phi_in[row + xm], phi_in[row + xp], phi_in[zo + (long long)ym * nx + x],
                                       phi_in[zo + (long long)yp * nx + x], zprev, znext, p, cc, co, q);
        phi_out[row + x] = out;
        pi[row + x] = p;
        c[row + x] = cc;
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
    energy_partial_kernel(const float2 *__restrict__ phi, const float2 *__restrict__ pi, int nx, int ny, int nz,
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
        const float2 f = phi[s], v = pi[s];
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
cudaError_t launch_reset(const RegionArgs &a, cudaStream_t st)
{
    const unsigned blocks = (a.total + 255) / 256;
    reset_kernel<<<blocks ? blocks : 1, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <int NT>
static cudaError_t region_launch_t(const RegionArgs &a, int max_B, int grid, cudaStream_t st)
{
    const int P = max_B + 2;
    const size_t smem = (size_t)2 * P * P * P * sizeof(float2) + (size_t)max_B * max_B * max_B * sizeof(float4);
    cudaError_t e = cudaFuncSetAttribute(region_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    region_kernel<NT><<<grid, NT, smem, st>>>(a, P);
    return cudaGetLastError();
}

size_t region_smem_bytes(int max_B)
{
    const int P = max_B + 2;
    return (size_t)2 * P * P * P * sizeof(float2) + (size_t)max_B * max_B * max_B * sizeof(float4);
}

cudaError_t region_occupancy(int threads, int max_B, int *blocks_per_sm)
{
    const size_t smem = region_smem_bytes(max_B);
    cudaError_t e;
#define SP_OCC(NT)                                                                                               \
    case NT:                                                                                                     \
        e = cudaFuncSetAttribute(region_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
        if (e != cudaSuccess) return e;                                                                          \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, region_kernel<NT>, NT, smem);
    switch (threads) {
        SP_OCC(128)
        SP_OCC(256)
        SP_OCC(512)
        SP_OCC(1024)
    default:
        return cudaErrorInvalidValue;
    }
#undef SP_OCC
}

cudaError_t launch_region(const RegionArgs &a, int threads, int max_B, int grid, cudaStream_t st)
{
    switch (threads) {
    case 128:
        return region_launch_t<128>(a, max_B, grid, st);
    case 256:
        return region_launch_t<256>(a, max_B, grid, st);
    case 512:
        return region_launch_t<512>(a, max_B, grid, st);
    case 1024:
        return region_launch_t<1024>(a, max_B, grid, st);
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sweep(const float2 *phi_in, float2 *phi_out, float2 *pi, float2 *c, const int n[3],
                         const LevelCoef *coef, int lvl, PhysConst q, cudaStream_t st)
{
    const int zchunk = 8;
    dim3 block(32, 8, 1);
    dim3 grid((n[0] + 31) / 32, (n[1] + 7) / 8, (n[2] + zchunk - 1) / zchunk);
    sweep_kernel<<<grid, block, 0, st>>>(phi_in, phi_out, pi, c, n[0], n[1], n[2], zchunk, coef, lvl, q);
    return cudaGetLastError();
}

int energy_blocks(const int n[3])
{
    const long long sites = (long long)n[0] * n[1] * n[2];
    long long b = (sites + 4095) / 4096;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

cudaError_t launch_energy(const float2 *phi, const float2 *pi, const int n[3], double inv_dx2, double eta2,
                          double half_lambda_a2, double *partial, double *out, cudaStream_t st)
{
    const int nb = energy_blocks(n);
    energy_partial_kernel<<<nb, kDiagThreads, 0, st>>>(phi, pi, n[0], n[1], n[2], inv_dx2, eta2, half_lambda_a2,
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
