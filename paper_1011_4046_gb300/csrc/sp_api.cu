// sp_api.cu -- host side of the C ABI declared in include/sp.h.
//
// The host plans (planner.cpp), computes the per-level coefficient table in
// FP64 and rounds it to FP32 once, owns the work queue, mailboxes and
// diagnostics scratch, and launches the kernels of sp_kernels.cu.  Every
// site-update runs on the GPU; there is no host compute path.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "planner.h"
#include "sp.h"
#include "sp_device.cuh"
#include "sp_kernels.h"

namespace {

struct TablesOnDevice {
    sp::TileTables host;
    sp::TablesDev *d_struct = nullptr;
    int *d_imp_full = nullptr;
    int *d_imp_phi = nullptr;
    int4 *d_exp = nullptr;
};

struct SweepGraph {
    cudaGraphExec_t exec = nullptr;
    int sim = -1;
    int64_t steps = -1, first_local = -1;
    const void *coef = nullptr;
};

template <class T>
cudaError_t grow(T **p, size_t *cap, size_t need)
{
    if (*cap >= need && *p) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t n = std::max<size_t>(need, 1);
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e == cudaSuccess) *cap = n;
    return e;
}

double a_of(const sp_params &p, double tau)
{
    double ratio = tau / p.tau_ref;
    double nu_i = std::floor(p.nu);
    if (p.nu == nu_i && p.nu >= 0 && p.nu <= 16) {
        double a = 1.0;
        for (int i = 0; i < (int)nu_i; ++i) a *= ratio;
        return a;
    }
    return std::pow(ratio, p.nu);
}

// tau, a, friction d at a level (the same reading as the public header)
void level_physics(const sp_params &p, int64_t level, double *tau, double *a, double *d)
{
    bool damping = level < p.damp_steps;
    *tau = damping ? p.tau0 : p.tau0 + (double)(level - p.damp_steps) * p.dt;
    *a = a_of(p, *tau);
    *d = damping ? 1.0 : p.nu * p.dt / *tau;
}

sp::LevelCoef level_coef(const sp_params &p, int64_t level)
{
    double tau, a, d;
    level_physics(p, level, &tau, &a, &d);
    sp::LevelCoef c;
    c.c1 = (float)((1.0 - d) / (1.0 + d));
    c.c2 = (float)(p.dt / (1.0 + d));
    c.m = (float)(a * a * p.lambda);
    c.pad = 0.0f;
    return c;
}

sp::PhysConst phys_const(const sp_params &p)
{
    sp::PhysConst q;
    q.dt = (float)p.dt;
    q.inv_dx2 = (float)(1.0 / (p.dx * p.dx));
    q.eta2 = (float)(p.eta * p.eta);
    q.pad = 0.0f;
    return q;
}

bool stable(const sp_params &p, int64_t level)
{
    double tau, a, d;
    level_physics(p, level, &tau, &a, &d);
    double w2 = 12.0 / (p.dx * p.dx) + 2.0 * p.lambda * p.eta * p.eta * a * a;
    return p.dt * p.dt * w2 < 4.0;
}

int64_t sites_of(const sp_params &p) { return (int64_t)p.n[0] * p.n[1] * p.n[2]; }

}  // namespace

struct sp_grid {
    int n_sims = 0;
    std::vector<sp_params> p;
    std::vector<float2 *> phi, pi, c;
    bool owns_state = false;
    cudaStream_t stream = nullptr;
    int device = 0, sm_count = 0;
    std::vector<int64_t> level;
    // plan
    bool planned = false;
    int threads = 0, max_B = 0, ctas_per_sm = 0, grid = 0, order = 0;
    std::vector<int> B;
    std::map<int, TablesOnDevice> tables;
    std::vector<float2 *> mbox;
    std::vector<long long> mb_slot;
    std::vector<std::array<long long, sp::kTypes>> mb_type_off;
    // launch scratch
    int *d_counters = nullptr, *d_queue = nullptr;
    size_t cap_counters = 0, cap_queue = 0;
    sp::Ctl *d_ctl = nullptr;
    sp::SimDev *d_sims = nullptr;
    size_t cap_sims = 0;
    sp::LevelCoef *d_coef = nullptr;
    size_t cap_coef = 0;
    unsigned long long *d_trace = nullptr;
    size_t cap_trace = 0;
    float2 *d_tmp = nullptr;
    size_t cap_tmp = 0;
    double *d_epart = nullptr, *d_eout = nullptr;
    size_t cap_epart = 0;
    unsigned long long *d_wcount = nullptr;
    signed char *d_wind = nullptr;
    size_t cap_wind = 0;
    // last region launch
    std::vector<unsigned> last_tile_base, last_tiles;
    bool last_traced = false;
    SweepGraph sweep_graph;
    unsigned long long wait_limit_ns = 2000000000ull;
    // what is already on the device (uploads are skipped when unchanged)
    std::vector<sp::LevelCoef> up_coef;
    std::vector<sp::SimDev> up_sims;
    unsigned long long up_limit = 0;
};

namespace {

int cuda_err(cudaError_t e) { return e == cudaSuccess ? SP_OK : SP_ECUDA; }

int check_params(const sp_params &p)
{
    for (int d = 0; d < 3; ++d)
        if (p.n[d] < 4 || p.n[d] > (1 << 14)) return SP_EINVAL;
    if (!(p.dx > 0) || !(p.dt > 0) || !(p.lambda >= 0) || !(p.eta >= 0) || !(p.nu >= 0)) return SP_EINVAL;
    if (!(p.tau0 > 0) || !(p.tau_ref > 0) || p.damp_steps < 0 || p.reserved != 0) return SP_EINVAL;
    if (sites_of(p) > (int64_t)1 << 33) return SP_EINVAL;
    return SP_OK;
}

int build_device_tables(sp_grid *g, int B)
{
    if (g->tables.count(B)) return SP_OK;
    TablesOnDevice td;
    std::string err = sp::build_tables(B, &td.host);
    if (!err.empty()) return SP_EINVAL;
    const sp::TileTables &t = td.host;
    sp::TablesDev h;
    std::memset(&h, 0, sizeof h);
    h.B = t.B;
    h.H = t.H;
    h.P = t.P;
    for (int S = 0; S < sp::kTypes; ++S) {
        h.levels[S] = t.levels[S];
        for (int k = 0; k <= sp::kMaxH; ++k) h.active[S][k] = t.active[S][k];
        h.base_phi[S] = t.base_phi[S];
        h.base_pc[S] = t.base_pc[S];
        for (int L = 0; L < sp::kMaxH; ++L) {
            h.imp_full_off[S][L] = t.imp_full_off[S][L];
            h.imp_full_n[S][L] = t.imp_full_n[S][L];
            h.imp_phi_off[S][L] = t.imp_phi_off[S][L];
            h.imp_phi_n[S][L] = t.imp_phi_n[S][L];
            h.mb_level_off[S][L] = t.mb_level_off[S][L];
            h.exp_off[S][L] = t.exp_off[S][L];
            h.exp_n[S][L] = t.exp_n[S][L];
        }
        h.mb_size[S] = t.mb_size[S];
        h.same_preds[S] = t.same_preds[S];
        h.prev_preds[S] = t.prev_preds[S];
        h.n_same_succ[S] = (int)t.same_succ[S].size();
        for (size_t i = 0; i < t.same_succ[S].size(); ++i) h.same_succ[S][i] = t.same_succ[S][i];
    }
    for (int q = 0; q < 2; ++q)
        for (size_t i = 0; i < t.next_succ[q].size(); ++i) h.next_succ[q][i] = t.next_succ[q][i];
    cudaError_t e = cudaSuccess;
    auto up = [&](void **dst, const void *src, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess && bytes) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up((void **)&td.d_imp_full, t.imp_full.data(), t.imp_full.size() * sizeof(int));
    up((void **)&td.d_imp_phi, t.imp_phi.data(), t.imp_phi.size() * sizeof(int));
    up((void **)&td.d_exp, t.exp.data(), t.exp.size() * sizeof(sp::ExportEntry));
    h.imp_full = td.d_imp_full;
    h.imp_phi = td.d_imp_phi;
    h.exp = td.d_exp;
    up((void **)&td.d_struct, &h, sizeof h);
    if (e != cudaSuccess) {
        cudaFree(td.d_imp_full);
        cudaFree(td.d_imp_phi);
        cudaFree(td.d_exp);
        cudaFree(td.d_struct);
        return e == cudaErrorMemoryAllocation ? SP_ENOMEM : SP_ECUDA;
    }
    g->tables[B] = td;
    return SP_OK;
}

void free_plan(sp_grid *g)
{
    for (auto &kv : g->tables) {
        cudaFree(kv.second.d_imp_full);
        cudaFree(kv.second.d_imp_phi);
        cudaFree(kv.second.d_exp);
        cudaFree(kv.second.d_struct);
    }
    g->tables.clear();
    for (float2 *m : g->mbox) cudaFree(m);
    g->mbox.clear();
    g->planned = false;
}

int choose_B(const sp_params &p, int requested)
{
    auto ok = [&](int B) {
        for (int d = 0; d < 3; ++d)
            if (p.n[d] % B != 0 || p.n[d] / B < 2) return false;
        return true;
    };
    if (requested) return ok(requested) ? requested : -1;
    if (ok(16)) return 16;
    if (ok(8)) return 8;
    return -1;
}

int default_threads(int B) { return B <= 8 ? 128 : 512; }

// Pending device error of the last region launch -> SP code.
int collect_device_error(sp_grid *g)
{
    sp::Ctl ctl;
    cudaError_t e = cudaMemcpyAsync(&ctl, g->d_ctl, sizeof ctl, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return SP_ECUDA;
    if (ctl.error == sp::kDevTimeout) return SP_ETIMEOUT;
    if (ctl.error != 0) return SP_ECUDA;
    return SP_OK;
}

int sweep_steps(sp_grid *g, int s, int64_t nsteps, int64_t first_local, const sp::LevelCoef *d_coef_sim)
{
    if (nsteps <= 0) return SP_OK;
    const sp_params &p = g->p[s];
    const int64_t sites = sites_of(p);
    cudaError_t e = grow(&g->d_tmp, &g->cap_tmp, (size_t)sites);
    if (e != cudaSuccess) return SP_ENOMEM;
    const sp::PhysConst q = phys_const(p);
    float2 *a = g->phi[s], *b = g->d_tmp;
    for (int64_t k = 0; k < nsteps; ++k) {
        e = sp::launch_sweep(a, b, g->pi[s], g->c[s], p.n, d_coef_sim, (int)(first_local + k), q, g->stream);
        if (e != cudaSuccess) return SP_ECUDA;
        std::swap(a, b);
    }
    if (a != g->phi[s]) {
        e = cudaMemcpyAsync(g->phi[s], a, sites * sizeof(float2), cudaMemcpyDeviceToDevice, g->stream);
        if (e != cudaSuccess) return SP_ECUDA;
    }
    return SP_OK;
}

}  // namespace

extern "C" {

const char *sp_strerror(int code)
{
    switch (code) {
    case SP_OK:
        return "ok";
    case SP_EINVAL:
        return "invalid argument or call order";
    case SP_ENOMEM:
        return "out of memory";
    case SP_ECUDA:
        return "CUDA runtime error";
    case SP_EUNSTABLE:
        return "leapfrog stability bound dt^2 (12/dx^2 + 2 lambda eta^2 a^2) < 4 violated";
    case SP_ETIMEOUT:
        return "a bounded device wait gave up (no ready region in time)";
    case SP_ENONFINITE:
        return "non-finite field";
    case SP_EFAULT_INJECTED:
        return "host-injected region failure";
    case SP_ENOTPLANNED:
        return "sp_evolve called before sp_region_plan";
    default:
        return "unknown error";
    }
}

int sp_grid_create(const sp_params *p, int32_t n_sims, void *const *state_dev, void *cuda_stream, sp_grid **out)
{
    if (!p || !out || n_sims < 1 || n_sims > 4096) return SP_EINVAL;
    *out = nullptr;
    for (int s = 0; s < n_sims; ++s)
        if (check_params(p[s]) != SP_OK) return SP_EINVAL;
    sp_grid *g = new (std::nothrow) sp_grid();
    if (!g) return SP_ENOMEM;
    g->n_sims = n_sims;
    g->p.assign(p, p + n_sims);
    g->stream = (cudaStream_t)cuda_stream;
    g->level.assign(n_sims, 0);
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) {
        delete g;
        return SP_ECUDA;
    }
    g->owns_state = state_dev == nullptr;
    for (int s = 0; s < n_sims; ++s) {
        float2 *f[3] = {nullptr, nullptr, nullptr};
        if (state_dev) {
            for (int k = 0; k < 3; ++k) {
                f[k] = (float2 *)state_dev[3 * s + k];
                if (!f[k] || ((uintptr_t)f[k] & 7u)) {
                    delete g;
                    return SP_EINVAL;
                }
            }
        } else {
            const size_t bytes = (size_t)sites_of(p[s]) * sizeof(float2);
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
                e = cudaMalloc((void **)&f[k], bytes);
                if (e == cudaSuccess) e = cudaMemsetAsync(f[k], 0, bytes, g->stream);
            }
        }
        g->phi.push_back(f[0]);
        g->pi.push_back(f[1]);
        g->c.push_back(f[2]);
        if (e != cudaSuccess) {
            sp_destroy(g);
            return SP_ENOMEM;
        }
    }
    e = cudaMalloc((void **)&g->d_ctl, sizeof(sp::Ctl));
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_ctl, 0, sizeof(sp::Ctl), g->stream);
    if (e == cudaSuccess) e = cudaMalloc((void **)&g->d_eout, 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&g->d_wcount, 8 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        sp_destroy(g);
        return SP_ENOMEM;
    }
    *out = g;
    return SP_OK;
}

int sp_region_plan(sp_grid *g, int32_t base_B, int32_t block_shape, int32_t order, const char *model_path)
{
    (void)model_path;
    if (!g) return SP_EINVAL;
    if (base_B != 0 && (base_B % 2 != 0 || base_B < 4 || base_B > 16)) return SP_EINVAL;
    if (block_shape != 0 && block_shape != 128 && block_shape != 256 && block_shape != 512 && block_shape != 1024)
        return SP_EINVAL;
    if (order != SP_ORDER_STATIC && order != SP_ORDER_LEARNED) return SP_EINVAL;
    free_plan(g);
    g->B.assign(g->n_sims, 0);
    g->max_B = 0;
    for (int s = 0; s < g->n_sims; ++s) {
        int B = choose_B(g->p[s], base_B);
        if (B < 0) return SP_EINVAL;
        g->B[s] = B;
        g->max_B = std::max(g->max_B, B);
        int rc = build_device_tables(g, B);
        if (rc != SP_OK) return rc;
    }
    g->threads = block_shape ? block_shape : default_threads(g->max_B);
    if (sp::region_smem_bytes(g->max_B) > 227 * 1024) return SP_EINVAL;
    cudaError_t e = sp::region_occupancy(g->threads, g->max_B, &g->ctas_per_sm);
    if (e != cudaSuccess || g->ctas_per_sm < 1) return SP_EINVAL;
    g->grid = g->ctas_per_sm * g->sm_count;
    g->order = order;
    // mailbox ring: two band slots per simulation
    g->mb_slot.assign(g->n_sims, 0);
    g->mb_type_off.assign(g->n_sims, {});
    for (int s = 0; s < g->n_sims; ++s) {
        const sp::TileTables &t = g->tables[g->B[s]].host;
        long long J = 1;
        for (int d = 0; d < 3; ++d) J *= g->p[s].n[d] / g->B[s];
        long long off = 0;
        for (int S = 0; S < sp::kTypes; ++S) {
            g->mb_type_off[s][S] = off;
            off += J * t.mb_size[S];
        }
        g->mb_slot[s] = off;
        float2 *m = nullptr;
        e = cudaMalloc((void **)&m, std::max<size_t>(2 * off * sizeof(float2), 16));
        if (e != cudaSuccess) {
            free_plan(g);
            return SP_ENOMEM;
        }
        g->mbox.push_back(m);
    }
    g->planned = true;
    return SP_OK;
}

int sp_evolve(sp_grid *g, int64_t n_steps, uint32_t flags)
{
    if (!g || n_steps < 0) return SP_EINVAL;
    if (flags & ~(SP_ASYNC | SP_MONOLITHIC | SP_RESTART | SP_TRACE)) return SP_EINVAL;
    if (flags & SP_RESTART) std::fill(g->level.begin(), g->level.end(), 0);
    if (n_steps == 0) return SP_OK;
    const bool mono = (flags & SP_MONOLITHIC) != 0;
    if (!mono && !g->planned) return SP_ENOTPLANNED;
    for (int s = 0; s < g->n_sims; ++s)
        for (int64_t k = 0; k < n_steps; ++k)
            if (!stable(g->p[s], g->level[s] + k)) return SP_EUNSTABLE;

    // coefficient tables of this call, all simulations concatenated
    std::vector<sp::LevelCoef> coef((size_t)g->n_sims * n_steps);
    for (int s = 0; s < g->n_sims; ++s)
        for (int64_t k = 0; k < n_steps; ++k) coef[(size_t)s * n_steps + k] = level_coef(g->p[s], g->level[s] + k);
    cudaError_t e = cudaSuccess;
    if (coef.size() != g->up_coef.size() ||
        std::memcmp(coef.data(), g->up_coef.data(), coef.size() * sizeof(sp::LevelCoef)) != 0) {
        e = grow(&g->d_coef, &g->cap_coef, coef.size());
        if (e != cudaSuccess) return SP_ENOMEM;
        e = cudaMemcpyAsync(g->d_coef, coef.data(), coef.size() * sizeof(sp::LevelCoef), cudaMemcpyHostToDevice,
                            g->stream);
        if (e != cudaSuccess) return SP_ECUDA;
        g->up_coef = coef;
    }

    int rc = SP_OK;
    if (mono) {
        for (int s = 0; s < g->n_sims && rc == SP_OK; ++s)
            rc = sweep_steps(g, s, n_steps, 0, g->d_coef + (size_t)s * n_steps);
    } else {
        // whole bands as regions, in one persistent launch over all simulations
        std::vector<sp::SimDev> sims;
        std::vector<int> sim_of;
        unsigned total = 0, seeds = 0;
        g->last_tile_base.assign(g->n_sims, 0);
        g->last_tiles.assign(g->n_sims, 0);
        for (int s = 0; s < g->n_sims; ++s) {
            const int B = g->B[s], H = B / 2;
            const int64_t nb = n_steps / H;
            if (nb == 0) continue;
            const TablesOnDevice &td = g->tables[B];
            sp::SimDev d;
            std::memset(&d, 0, sizeof d);
            for (int k = 0; k < 3; ++k) {
                d.n[k] = g->p[s].n[k];
                d.J[k] = d.n[k] / B;
            }
            d.Jtot = d.J[0] * d.J[1] * d.J[2];
            d.B = B;
            d.H = H;
            d.P = B + 2;
            d.nbands = (int)nb;
            const unsigned long long tiles = (unsigned long long)nb * 8ull * (unsigned long long)d.Jtot;
            if ((unsigned long long)total + tiles > 0x7fffffffull) return SP_EINVAL;
            d.tile_base = total;
            d.tiles = (unsigned)tiles;
            d.seed_base = seeds;
            d.coef = g->d_coef + (size_t)s * n_steps;
            d.q = phys_const(g->p[s]);
            d.phi = g->phi[s];
            d.pi = g->pi[s];
            d.c = g->c[s];
            d.mbox = g->mbox[s];
            d.mb_slot = g->mb_slot[s];
            for (int S = 0; S < sp::kTypes; ++S) d.mb_type_off[S] = g->mb_type_off[s][S];
            d.tab = td.d_struct;
            g->last_tile_base[s] = total;
            g->last_tiles[s] = d.tiles;
            total += d.tiles;
            seeds += (unsigned)d.Jtot;
            sims.push_back(d);
            sim_of.push_back(s);
        }
        if (!sims.empty()) {
            e = grow(&g->d_sims, &g->cap_sims, sims.size());
            if (e == cudaSuccess) e = grow(&g->d_counters, &g->cap_counters, total);
            if (e == cudaSuccess) e = grow(&g->d_queue, &g->cap_queue, total);
            const bool trace = (flags & SP_TRACE) != 0;
            if (e == cudaSuccess && trace) e = grow(&g->d_trace, &g->cap_trace, 2 * (size_t)total);
            if (e != cudaSuccess) return SP_ENOMEM;
            if (sims.size() != g->up_sims.size() ||
                std::memcmp(sims.data(), g->up_sims.data(), sims.size() * sizeof(sp::SimDev)) != 0) {
                e = cudaMemcpyAsync(g->d_sims, sims.data(), sims.size() * sizeof(sp::SimDev),
                                    cudaMemcpyHostToDevice, g->stream);
                if (e != cudaSuccess) return SP_ECUDA;
                g->up_sims = sims;
            }
            if (g->up_limit != g->wait_limit_ns) {
                unsigned long long lim = g->wait_limit_ns;
                e = cudaMemcpyAsync(&g->d_ctl->wait_limit_ns, &lim, sizeof lim, cudaMemcpyHostToDevice, g->stream);
                if (e != cudaSuccess) return SP_ECUDA;
                g->up_limit = lim;
            }
            sp::RegionArgs a;
            a.sims = g->d_sims;
            a.n_sims = (int)sims.size();
            a.total = total;
            a.n_seed = seeds;
            a.counters = g->d_counters;
            a.queue = g->d_queue;
            a.ctl = g->d_ctl;
            a.trace = trace ? g->d_trace : nullptr;
            g->last_traced = trace;
            e = sp::launch_reset(a, g->stream);
            if (e == cudaSuccess) e = sp::launch_region(a, g->threads, g->max_B, g->grid, g->stream);
            if (e != cudaSuccess) return SP_ECUDA;
        }
        // remainder steps of each simulation: whole-grid steps, same arithmetic
        for (int s = 0; s < g->n_sims && rc == SP_OK; ++s) {
            const int H = g->B[s] / 2;
            const int64_t done = (n_steps / H) * H;
            rc = sweep_steps(g, s, n_steps - done, done, g->d_coef + (size_t)s * n_steps);
        }
    }
    if (rc != SP_OK) return rc;
    for (int s = 0; s < g->n_sims; ++s) g->level[s] += n_steps;
    if (flags & SP_ASYNC) return SP_OK;
    e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return SP_ECUDA;
    if (!mono) return collect_device_error(g);
    return SP_OK;
}

int sp_write_surface(sp_grid *g, int32_t sim, int32_t what, const void *src, size_t src_bytes, int32_t src_is_device)
{
    if (!g || sim < 0 || sim >= g->n_sims || !src || what != SP_SURF_STATE) return SP_EINVAL;
    const size_t bytes = (size_t)sites_of(g->p[sim]) * sizeof(float2);
    if (src_bytes < 3 * bytes) return SP_EINVAL;
    const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const char *b = (const char *)src;
    cudaError_t e = cudaMemcpyAsync(g->phi[sim], b, bytes, kind, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->pi[sim], b + bytes, bytes, kind, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->c[sim], b + 2 * bytes, bytes, kind, g->stream);
    return cuda_err(e);
}

int sp_read_surface(const sp_grid *gc, int32_t sim, int32_t what, void *dst, size_t dst_bytes, int32_t dst_is_device)
{
    sp_grid *g = const_cast<sp_grid *>(gc);
    if (!g || sim < 0 || sim >= g->n_sims || !dst) return SP_EINVAL;
    const sp_params &p = g->p[sim];
    const int64_t sites = sites_of(p);
    const cudaMemcpyKind to = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSuccess;
    if (g->planned && g->d_ctl) {
        int rc = collect_device_error(g);
        if (rc != SP_OK) return rc;
    }
    switch (what) {
    case SP_SURF_STATE: {
        const size_t bytes = (size_t)sites * sizeof(float2);
        if (dst_bytes < 3 * bytes) return SP_EINVAL;
        char *b = (char *)dst;
        e = cudaMemcpyAsync(b, g->phi[sim], bytes, to, g->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b + bytes, g->pi[sim], bytes, to, g->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b + 2 * bytes, g->c[sim], bytes, to, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        return cuda_err(e);
    }
    case SP_SURF_WINDING: {
        if (dst_bytes < (size_t)(3 * sites)) return SP_EINVAL;
        signed char *w = nullptr;
        if (dst_is_device) {
            w = (signed char *)dst;
        } else {
            e = grow(&g->d_wind, &g->cap_wind, (size_t)(3 * sites));
            if (e != cudaSuccess) return SP_ENOMEM;
            w = g->d_wind;
        }
        e = cudaMemsetAsync(g->d_wcount, 0, 8 * sizeof(unsigned long long), g->stream);
        if (e == cudaSuccess) e = sp::launch_winding(g->phi[sim], p.n, w, g->d_wcount, g->stream);
        if (e == cudaSuccess && !dst_is_device)
            e = cudaMemcpyAsync(dst, w, (size_t)(3 * sites), cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        return cuda_err(e);
    }
    case SP_SURF_DIAG: {
        if (dst_bytes < sizeof(sp_diag)) return SP_EINVAL;
        const int nb = sp::energy_blocks(p.n);
        e = grow(&g->d_epart, &g->cap_epart, (size_t)3 * nb);
        if (e != cudaSuccess) return SP_ENOMEM;
        double tau, a, d;
        level_physics(p, g->level[sim], &tau, &a, &d);
        e = sp::launch_energy(g->phi[sim], g->pi[sim], p.n, 1.0 / (p.dx * p.dx), p.eta * p.eta,
                              0.5 * p.lambda * a * a, g->d_epart, g->d_eout, g->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(g->d_wcount, 0, 8 * sizeof(unsigned long long), g->stream);
        if (e == cudaSuccess) e = sp::launch_winding(g->phi[sim], p.n, nullptr, g->d_wcount, g->stream);
        double en[3];
        unsigned long long wc[7];
        if (e == cudaSuccess) e = cudaMemcpyAsync(en, g->d_eout, sizeof en, cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(wc, g->d_wcount, sizeof wc, cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) return SP_ECUDA;
        sp_diag out;
        std::memset(&out, 0, sizeof out);
        out.level = g->level[sim];
        out.tau = tau;
        out.a = a;
        out.kinetic = en[0];
        out.gradient = en[1];
        out.potential = en[2];
        out.total = en[0] + en[1] + en[2];
        for (int k = 0; k < 3; ++k) {
            out.pierced[k] = (int64_t)wc[k];
            out.net_winding[k] = (int64_t)wc[4 + k];
        }
        out.abs_winding = (int64_t)wc[3];
        out.string_length = (double)(wc[0] + wc[1] + wc[2]) * p.dx;
        if (dst_is_device) e = cudaMemcpy(dst, &out, sizeof out, cudaMemcpyHostToDevice);
        else std::memcpy(dst, &out, sizeof out);
        return cuda_err(e);
    }
    case SP_SURF_PLAN: {
        if (dst_bytes < sizeof(sp_plan_info) || !g->planned) return SP_EINVAL;
        const sp::TileTables &t = g->tables[g->B[sim]].host;
        sp::PlanStats ps = sp::plan_stats(t, p.n);
        sp_plan_info info;
        std::memset(&info, 0, sizeof info);
        info.base_B = g->B[sim];
        info.threads = g->threads;
        info.ctas_per_sm = g->ctas_per_sm;
        info.grid = g->grid;
        info.regions_per_band = ps.regions_per_band;
        info.updates_per_band = ps.updates_per_band;
        info.bytes_read_per_band = ps.bytes_read_per_band;
        info.bytes_written_per_band = ps.bytes_written_per_band;
        info.bytes_per_update = ps.bytes_per_update;
        info.mailbox_bytes = 2 * g->mb_slot[sim] * (int64_t)sizeof(float2);
        if (dst_is_device) e = cudaMemcpy(dst, &info, sizeof info, cudaMemcpyHostToDevice);
        else std::memcpy(dst, &info, sizeof info);
        return cuda_err(e);
    }
    case SP_SURF_TRACE: {
        if (!g->last_traced || sim >= (int)g->last_tiles.size()) return SP_EINVAL;
        const size_t n = 2 * (size_t)g->last_tiles[sim];
        if (dst_bytes < n * sizeof(unsigned long long)) return SP_EINVAL;
        e = cudaMemcpyAsync(dst, g->d_trace + 2 * (size_t)g->last_tile_base[sim], n * sizeof(unsigned long long), to,
                            g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        return cuda_err(e);
    }
    default:
        return SP_EINVAL;
    }
}

int sp_destroy(sp_grid *g)
{
    if (!g) return SP_EINVAL;
    cudaStreamSynchronize(g->stream);
    free_plan(g);
    if (g->owns_state)
        for (int s = 0; s < (int)g->phi.size(); ++s) {
            cudaFree(g->phi[s]);
            cudaFree(g->pi[s]);
            cudaFree(g->c[s]);
        }
    cudaFree(g->d_counters);
    cudaFree(g->d_queue);
    cudaFree(g->d_ctl);
    cudaFree(g->d_sims);
    cudaFree(g->d_coef);
    cudaFree(g->d_trace);
    cudaFree(g->d_tmp);
    cudaFree(g->d_epart);
    cudaFree(g->d_eout);
    cudaFree(g->d_wcount);
    cudaFree(g->d_wind);
    if (g->sweep_graph.exec) cudaGraphExecDestroy(g->sweep_graph.exec);
    delete g;
    return SP_OK;
}

}  // extern "C"
