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

#include "lattice.h"

namespace sp {
cudaError_t model_buckets(const sp_model *m, const float *X, long long n, unsigned char *prio, cudaStream_t st);
}

namespace {

struct TablesOnDevice {
    sp::TileTables host;
    sp::TablesDev dev;             // host copy of the device descriptor
    // base 32: the octant tables of the cluster kernel (TablesDev then holds
    // the dependency pattern only)
    bool octant = false;
    sp::OctTables oct;
    sp::TablesOct oct_dev;
    sp::TablesOct *d_oct = nullptr;
    unsigned short *d_oimp = nullptr;
    int2 *d_oexp = nullptr;
    int *d_oface = nullptr;
    int64_t region_mb_size[sp::kTypes] = {0};  // float2 elements of one region's mailbox
    // band-0 regions of types 0 .. seed_types-1 have no predecessor and are
    // queued at reset (1 for bases of 8 and more: the pyramids; at base 4 every
    // type but the inverted pyramid computes one level and imports nothing)
    int seed_types = 1;
    sp::TablesDev *d_dev = nullptr;  // device copy (the only table of its launch)
    unsigned short *d_imp = nullptr;
    int2 *d_exp = nullptr;
    sp::Succ *d_reuse = nullptr;  // mailbox-reuse successors, kMaxSameSucc per type
};

// The 4-cube lattice tables of one size s (lattice.h) on the device.
struct LatOnDevice {
    sp::LatticeTables host;
    uint32_t *d_cell = nullptr;
    uint32_t *d_imp_all = nullptr;  // imp_all: pairs (entry, level)
    uint64_t *d_nb = nullptr;
    int32_t *d_pcoff = nullptr;
};

// One persistent launch per region base: simulations of the same base share a
// launch sized (shared memory, CTAs per SM) for that base alone.
struct GroupCfg {
    int B = 0, threads = 0, ctas_per_sm = 0, grid = 0;
    size_t smem = 0;
};

// A group's launch in one call.
struct GroupLaunch {
    GroupCfg cfg;
    sp::RegionArgs a;
    size_t sim_off = 0;  // first descriptor of the group in the call's array
    unsigned roff = 0;   // first region id of the group (trace, features, buckets)
};

constexpr int kMaxGroups = 4;  // distinct region bases of a plan (4, 8, 16)

struct SweepGraph {
    cudaGraphExec_t exec = nullptr;
    int sim = -1;
    int64_t steps = -1, first_local = -1;
    const void *coef = nullptr;
    const void *phi = nullptr, *tmp = nullptr;
};

// What the autotuner of the last sp_region_plan measured.
struct TuneReport {
    int autotuned = 0, candidates = 0, trial_steps = 0;
    double best_ms = 0.0, default_ms = 0.0;
};

// The region path of one sp_evolve call, captured once and replayed while the
// launch parameters stay the same (the key is every byte that the captured
// launches take by value).
struct RegionGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;
};

template <class T>
void append_key(std::vector<unsigned char> *key, const T &v)
{
    const unsigned char *b = reinterpret_cast<const unsigned char *>(&v);
    key->insert(key->end(), b, b + sizeof(T));
}

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
    std::vector<float2 *> phi;
    std::vector<float4 *> pc;  // (pi, c) interleaved
    bool owns_state = false;
    cudaStream_t stream = nullptr;
    int device = 0, sm_count = 0;
    std::vector<int64_t> level;
    // plan
    bool planned = false;
    int threads = 0, max_B = 0, order = 0;
    std::vector<int> B;
    std::map<int, TablesOnDevice> tables;
    std::vector<GroupCfg> groups;  // one per distinct base, largest first
    std::vector<float2 *> mbox;
    std::vector<long long> mb_slot;   // float2 offset of band slot 1 (0: one slot for every band)
    std::vector<long long> mb_elems;  // float2 elements per slot
    int mb_slots = 1;                 // SP_OPT_MAILBOX_SLOTS, applied by sp_region_plan
    int shape_opt = SP_SHAPE_SPLIT;   // SP_OPT_REGION_SHAPE, applied by sp_region_plan
    int shape = SP_SHAPE_SPLIT;       // of the current plan
    // lattice plans: tables by size s, phi at odd levels of a call per
    // simulation, done flags of every group ([4][regions per layer] each)
    std::map<int, LatOnDevice> lat;
    std::vector<float2 *> phi_odd;
    int *d_lat_flags = nullptr;
    std::vector<size_t> lat_flag_off;  // per group
    sp::LatSimDev *d_lsims = nullptr;
    size_t cap_lsims = 0;
    std::vector<sp::LatSimDev> up_lsims;
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
    RegionGraph region_graph;
    TuneReport tune;
    // learned ordering and cost-model features
    sp_model *model = nullptr;
    float *d_feat = nullptr;
    size_t cap_feat = 0;
    float4 *d_simf = nullptr;
    size_t cap_simf = 0;
    unsigned char *d_prio = nullptr;
    size_t cap_prio = 0;
    bool last_features = false;
    unsigned last_total = 0;
    unsigned trace_total = 0;    // regions of the last traced call (its trace is still in d_trace)
    bool prev_trace_ok = false;  // this call's features may read d_trace
    int use_graphs = 1;  // capture launch sequences on non-legacy streams
    unsigned long long wait_limit_ns = 2000000000ull;
    int fault_drop = -1;  // SP_OPT_FAULT_DROP_RELEASE
    // what is already on the device (uploads are skipped when unchanged)
    std::vector<sp::LevelCoef> up_coef;
    std::vector<sp::SimDev> up_sims;
    unsigned long long up_limit = 0;
    // CUDA events of the last SP_TIMING call: before reset, before region
    // kernel, after region kernel, after the remainder sweep
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool timed = false;
};

namespace {

int cuda_err(cudaError_t e) { return e == cudaSuccess ? SP_OK : SP_ECUDA; }

int check_params(const sp_params &p)
{
    for (int d = 0; d < 3; ++d)
        if (p.n[d] < 4 || p.n[d] > (1 << 14)) return SP_EINVAL;
    if (!(p.dx > 0) || !(p.dt > 0) || !(p.lambda >= 0) || !(p.eta >= 0) || !(p.nu >= 0)) return SP_EINVAL;
    if (!(p.tau0 > 0) || !(p.tau_ref > 0) || p.damp_steps < 0 || p.precision != SP_FP32_KAHAN) return SP_EINVAL;
    if (sites_of(p) > (int64_t)1 << 33) return SP_EINVAL;
    return SP_OK;
}

// The kernel splits a linear index i < w0 w1 w2 into (x, y, z) with
// sp::fdiv and FP32 reciprocals; check every quotient it will form.
bool decode_exact(const sp::Box3 *boxes, int last, const float (*rcp)[2])
{
    for (int k = 0; k <= last; ++k) {
        const sp::Box3 &b = boxes[k];
        const int w0 = b.hi[0] - b.lo[0], w1 = b.hi[1] - b.lo[1], w2 = b.hi[2] - b.lo[2];
        if (w0 <= 0 || w1 <= 0 || w2 <= 0) continue;
        for (int i = 0; i < w0 * w1 * w2; ++i) {
            const int t1 = sp::fdiv(i, rcp[k][0]);
            if (t1 != i / w0 || sp::fdiv(t1, rcp[k][1]) != t1 / w1) return false;
        }
    }
    return true;
}

// The same for the 2x2x2-block decode of the active boxes: block index
// m < (w0/2)(w1/2)(w2/2) -> (m / (w2/2)) / (w0/2); every extent must be even.
bool block_decode_exact(const sp::Box3 *boxes, int last, const float (*rcp)[2])
{
    for (int k = 0; k <= last; ++k) {
        const sp::Box3 &b = boxes[k];
        const int w0 = b.hi[0] - b.lo[0], w1 = b.hi[1] - b.lo[1], w2 = b.hi[2] - b.lo[2];
        if (w0 <= 0 || w1 <= 0 || w2 <= 0) continue;
        if ((w0 | w1 | w2) & 1) return false;
        const int a = w0 / 2, c = w2 / 2;
        for (int m = 0; m < a * (w1 / 2) * c; ++m) {
            const int r = sp::fdiv(m, rcp[k][0]);
            if (r != m / c || sp::fdiv(r, rcp[k][1]) != r / a) return false;
        }
    }
    return true;
}

// The dependency pattern of a base (same-band, next-band and mailbox-reuse
// successors, predecessor counts) into the device descriptor; geometry
// fields are left to the caller.
void fill_dag(const sp::TileTables &t, sp::TablesDev *h)
{
    for (int S = 0; S < sp::kTypes; ++S) {
        sp::TypeMeta &m = h->type[S];
        m.levels = t.levels[S];
        m.n_same_succ = (int)t.same_succ[S].size();
        m.same_preds = t.same_preds[S];
        m.prev_preds = t.prev_preds[S];
        m.n_reuse = (int)t.reuse_succ[S].size();
        m.reuse_preds = t.reuse_preds[S];
        for (size_t i = 0; i < t.same_succ[S].size(); ++i) m.same_succ[i] = t.same_succ[S][i];
    }
    for (int q = 0; q < 2; ++q)
        for (size_t i = 0; i < t.next_succ[q].size(); ++i) h->next_succ[q][i] = t.next_succ[q][i];
}

int upload_reuse(const sp::TileTables &t, sp::Succ **d_reuse)
{
    std::vector<sp::Succ> reuse((size_t)sp::kTypes * sp::kMaxSameSucc, sp::Succ{0, {0, 0, 0}});
    for (int S = 0; S < sp::kTypes; ++S) {
        if ((int)t.reuse_succ[S].size() > sp::kMaxSameSucc) return SP_EINVAL;
        for (size_t i = 0; i < t.reuse_succ[S].size(); ++i) reuse[(size_t)S * sp::kMaxSameSucc + i] = t.reuse_succ[S][i];
    }
    if (cudaMalloc((void **)d_reuse, reuse.size() * sizeof(sp::Succ)) != cudaSuccess) return SP_ENOMEM;
    if (cudaMemcpy(*d_reuse, reuse.data(), reuse.size() * sizeof(sp::Succ), cudaMemcpyHostToDevice) != cudaSuccess)
        return SP_ECUDA;
    return SP_OK;
}

// Base 32: the region's dependency pattern plus the octant tables of the
// cluster kernel, packed for the device (see sp_device.cuh, TablesOct).
int build_octant_device_tables(sp_grid *g, TablesOnDevice *tdp)
{
    TablesOnDevice &td = *tdp;
    const sp::TileTables &t = td.host;
    if (!sp::build_octant_tables(t, &td.oct).empty()) return SP_EINVAL;
    const sp::OctTables &o = td.oct;
    if (o.H != 16 || o.P != 18) return SP_EINVAL;  // the kernel's index packing and shifts
    td.octant = true;
    td.seed_types = 0;
    while (td.seed_types < sp::kTypes && t.same_preds[td.seed_types] == 0) ++td.seed_types;
    for (int S = td.seed_types; S < sp::kTypes; ++S)
        if (t.same_preds[S] == 0) return SP_EINVAL;
    if (td.seed_types == 0) return SP_EINVAL;
    std::memset(&td.dev, 0, sizeof td.dev);
    td.dev.B = t.B;
    td.dev.H = t.H;
    td.dev.P = t.P;
    fill_dag(t, &td.dev);
    sp::TablesOct &h = td.oct_dev;
    std::memset(&h, 0, sizeof h);
    h.B = o.B;
    h.H = o.H;
    h.P = o.P;
    std::vector<unsigned short> imp;
    for (int S = 0; S < sp::kTypes; ++S) {
        sp::OctTypeMeta &m = h.type[S];
        m.levels = o.levels[S];
        m.mb_size = o.mb_size[S];
        td.region_mb_size[S] = 8LL * o.mb_size[S];
        td.dev.type[S].mb_size = 8 * o.mb_size[S];
        m.base_phi = o.base_phi[S];
        m.base_pc = o.base_pc[S];
        const sp::Box3 &bp = o.base_phi[S];
        const int bw0 = bp.hi[0] - bp.lo[0], bw1 = bp.hi[1] - bp.lo[1], bw2 = bp.hi[2] - bp.lo[2];
        m.base_cols = bw0 * bw1;
        m.base_runs = (bw2 + 3) / 4;
        m.rcp_cols = 1.0f / (float)m.base_cols;
        m.rcp_base0 = 1.0f / (float)bw0;
        for (int u = 0; u < m.base_cols * m.base_runs; ++u) {  // the kernel's (run, column, row) split
            const int run = sp::fdiv(u, m.rcp_cols), i = u - run * m.base_cols;
            if (run != u / m.base_cols || sp::fdiv(i, m.rcp_base0) != i / bw0) return SP_EINVAL;
        }
        for (int k = 0; k < sp::kMaxHOct + 2; ++k) {
            int w[3];
            for (int d = 0; d < 3; ++d) {
                w[d] = k <= sp::kMaxH + 1 ? o.w[S][k][d] : 0;
                m.w[k][d] = (unsigned char)w[d];
            }
            m.rcp_w[k][0] = w[0] ? 1.0f / (float)w[0] : 0.0f;
            m.rcp_w[k][1] = w[1] ? 1.0f / (float)w[1] : 0.0f;
            const int fd[3] = {w[1], w[0] - 1, w[1] - 1};
            for (int q = 0; q < 3; ++q) m.rcp_f[k][q] = fd[q] > 0 ? 1.0f / (float)fd[q] : 0.0f;
            // the kernel's face-first decode: slabs x (w1 x w2), y ((w0-1) x w2), z ((w0-1) x (w1-1)),
            // then the interior ((w0-1) x (w1-1) x (w2-1))
            if (w[0] > 0 && w[1] > 0 && w[2] > 0) {
                for (int i = 0; i < w[1] * w[2]; ++i)
                    if (sp::fdiv(i, m.rcp_f[k][0]) != i / w[1]) return SP_EINVAL;
                if (w[0] > 1)
                    for (int i = 0; i < (w[0] - 1) * std::max(w[2], w[1]); ++i)
                        if (sp::fdiv(i, m.rcp_f[k][1]) != i / (w[0] - 1)) return SP_EINVAL;
                if (w[0] > 1 && w[1] > 1)
                    for (int i = 0; i < (w[0] - 1) * (w[1] - 1) * (w[2] - 1); ++i) {
                        const int t = sp::fdiv(i, m.rcp_f[k][1]);
                        if (t != i / (w[0] - 1) || sp::fdiv(t, m.rcp_f[k][2]) != t / (w[1] - 1)) return SP_EINVAL;
                    }
            }
            for (int i = 0; i < w[0] * w[1] * w[2]; ++i) {  // the kernel's decode of level k's cells
                const int t1 = sp::fdiv(i, m.rcp_w[k][0]);
                if (t1 != i / w[0] || sp::fdiv(t1, m.rcp_w[k][1]) != t1 / w[1]) return SP_EINVAL;
            }
            int64_t xb = 0;  // inner-face bytes received before level k (the faces of phi(k-1))
            if (k >= 2)
                for (int d = 0; d < 3; ++d)
                    if (w[d] > 0) xb += 8LL * w[(d + 1) % 3] * w[(d + 2) % 3];
            m.xbytes[k] = (int)xb;
        }
        for (int L = 0; L < sp::kMaxHOct; ++L) {
            m.mb_level_off[L] = o.mb_level_off[S][L];
            m.exp_off[L] = o.exp_off[S][L];
            m.exp_n[L] = o.exp_n[S][L];
            m.face_off[L] = o.face_imp_off[S][L];
            m.face_n[L] = o.face_imp_n[S][L];
            m.imp_full_n[L] = o.imp_full_n[S][L];
            m.imp_phi_n[L] = o.imp_phi_n[S][L];
            m.imp_full_off[L] = (int)imp.size();
            for (int i = 0; i < o.imp_full_n[S][L]; ++i) {
                const int e = o.imp_full[o.imp_full_off[S][L] + i], c = e >> 16;
                const int pidx = (((c >> 8) + 1) * 18 + ((c >> 4) & 15) + 1) * 18 + (c & 15) + 1;
                if (pidx != (e & 0xFFFF)) return SP_EINVAL;  // the kernel derives phi from (pi, c) by shifts
                imp.push_back((unsigned short)c);
            }
            m.imp_phi_off[L] = (int)imp.size();
            for (int i = 0; i < o.imp_phi_n[S][L]; ++i) imp.push_back((unsigned short)o.imp_phi[o.imp_phi_off[S][L] + i]);
        }
        if (o.mb_size[S] > 0xFFFF) return SP_EINVAL;
    }
    while (imp.size() % 8) imp.push_back(0);
    h.imp_n = (int)imp.size();
    std::vector<int2> ex(o.exp.size());
    for (size_t i = 0; i < o.exp.size(); ++i) {
        const sp::ExportEntry &e = o.exp[i];
        const int phi = e.src & 0xFFFF, pc = (e.src >> 16) & 0xFFFF, has_pc = e.dst_pc >= 0;
        if (phi >= 8192 || (has_pc && pc >= 4096) || e.dst_phi < 0 || e.dst_phi > 0xFFFF || e.dst_pc > 0xFFFF)
            return SP_EINVAL;
        ex[i].x = (int)((unsigned)phi | ((unsigned)(has_pc ? pc : 0) << 13) | ((unsigned)e.code << 25) |
                        ((unsigned)has_pc << 31));
        ex[i].y = (int)((unsigned)e.dst_phi | ((unsigned)(has_pc ? e.dst_pc : 0) << 16));
    }
    cudaError_t e = cudaSuccess;
    auto up = [&](void **dst, const void *src, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess && bytes) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up((void **)&td.d_oimp, imp.data(), imp.size() * sizeof(unsigned short));
    up((void **)&td.d_oexp, ex.data(), ex.size() * sizeof(int2));
    std::vector<int> face(o.face_imp);
    while (face.size() % 4) face.push_back(0);
    h.face_total = (int)face.size();
    up((void **)&td.d_oface, face.data(), face.size() * sizeof(int));
    h.imp = td.d_oimp;
    h.exp = td.d_oexp;
    h.face = td.d_oface;
    up((void **)&td.d_oct, &h, sizeof h);
    int rc = e == cudaSuccess ? upload_reuse(t, &td.d_reuse) : SP_OK;
    if (e != cudaSuccess || rc != SP_OK) {
        cudaFree(td.d_oimp);
        cudaFree(td.d_oexp);
        cudaFree(td.d_oface);
        cudaFree(td.d_oct);
        cudaFree(td.d_reuse);
        return e == cudaErrorMemoryAllocation || rc == SP_ENOMEM ? SP_ENOMEM : (rc != SP_OK ? rc : SP_ECUDA);
    }
    td.dev.reuse = td.d_reuse;
    g->tables[32] = td;
    return SP_OK;
}

int build_device_tables(sp_grid *g, int B)
{
    if (g->tables.count(B)) return SP_OK;
    TablesOnDevice td;
    std::string err = sp::build_tables(B, &td.host);
    if (!err.empty()) return SP_EINVAL;
    const sp::TileTables &t = td.host;
    if (B == 32) return build_octant_device_tables(g, &td);
    // the device tables and index packing serve bases up to 16
    if (t.P * t.P * t.P > 8192 || t.B * t.B * t.B > 4096 || t.H > sp::kMaxHDev) return SP_EINVAL;
    for (int S = 0; S < sp::kTypes; ++S) td.region_mb_size[S] = t.mb_size[S];
    // the seeds (band-0 regions without predecessors) must be the leading
    // region types: the queue reset takes the first Jtot * seed_types ids
    td.seed_types = 0;
    while (td.seed_types < sp::kTypes && t.same_preds[td.seed_types] == 0) ++td.seed_types;
    for (int S = td.seed_types; S < sp::kTypes; ++S)
        if (t.same_preds[S] == 0) return SP_EINVAL;
    if (td.seed_types == 0) return SP_EINVAL;
    sp::TablesDev &h = td.dev;
    std::memset(&h, 0, sizeof h);
    h.B = t.B;
    h.H = t.H;
    h.P = t.P;
    for (int S = 0; S < sp::kTypes; ++S) {
        sp::TypeMeta &m = h.type[S];
        m.levels = t.levels[S];
        m.mb_size = t.mb_size[S];
        m.n_same_succ = (int)t.same_succ[S].size();
        m.same_preds = t.same_preds[S];
        m.prev_preds = t.prev_preds[S];
        m.n_reuse = (int)t.reuse_succ[S].size();
        m.reuse_preds = t.reuse_preds[S];
        for (int k = 0; k <= sp::kMaxHDev; ++k) m.active[k] = t.active[S][k];
        m.base_phi = t.base_phi[S];
        m.base_pc = t.base_pc[S];
        for (int k = 0; k <= sp::kMaxHDev; ++k)
            for (int q = 0; q < 2; ++q) {
                const int d = q == 0 ? 2 : 0;  // blocks along z, then along x
                const int w = (t.active[S][k].hi[d] - t.active[S][k].lo[d]) / 2;
                m.rcp_active[k][q] = w > 0 ? 1.0f / (float)w : 0.0f;
            }
        for (int d = 0; d < 2; ++d) m.rcp_base[d] = 1.0f / (float)(t.base_phi[S].hi[d] - t.base_phi[S].lo[d]);
        {
            const sp::Box3 &bp = t.base_phi[S];
            m.base_cols = (bp.hi[0] - bp.lo[0]) * (bp.hi[1] - bp.lo[1]);
            m.base_runs = (bp.hi[2] - bp.lo[2] + 3) / 4;
            m.rcp_cols = 1.0f / (float)m.base_cols;
            for (int u = 0; u < m.base_cols * m.base_runs; ++u)  // the kernel's (run, column) split
                if (sp::fdiv(u, m.rcp_cols) != u / m.base_cols) return SP_EINVAL;
        }
        if (!block_decode_exact(m.active, t.H, m.rcp_active) || !decode_exact(&m.base_phi, 0, &m.rcp_base))
            return SP_EINVAL;
        for (int L = 0; L < sp::kMaxHDev; ++L) {
            m.mb_level_off[L] = t.mb_level_off[S][L];
            m.exp_off[L] = t.exp_off[S][L];
            m.exp_n[L] = t.exp_n[S][L];
            m.imp_full_n[L] = t.imp_full_n[S][L];
            m.imp_phi_n[L] = t.imp_phi_n[S][L];
        }
        for (size_t i = 0; i < t.same_succ[S].size(); ++i) m.same_succ[i] = t.same_succ[S][i];
    }
    for (int q = 0; q < 2; ++q)
        for (size_t i = 0; i < t.next_succ[q].size(); ++i) h.next_succ[q][i] = t.next_succ[q][i];
    // compact device tables (see sp_device.cuh for the packing)
    std::vector<unsigned short> imp;
    for (int S = 0; S < sp::kTypes; ++S)
        for (int L = 0; L < sp::kMaxHDev; ++L) {
            sp::TypeMeta &m = h.type[S];
            m.imp_full_off[L] = (int)imp.size();
            for (int i = 0; i < t.imp_full_n[S][L]; ++i)
                imp.push_back((unsigned short)(t.imp_full[t.imp_full_off[S][L] + i] >> 16));  // (pi, c) index
            m.imp_phi_off[L] = (int)imp.size();
            for (int i = 0; i < t.imp_phi_n[S][L]; ++i) imp.push_back((unsigned short)t.imp_phi[t.imp_phi_off[S][L] + i]);
        }
    while (imp.size() % 8) imp.push_back(0);
    h.imp_n = (int)imp.size();
    std::vector<int2> ex(t.exp.size());
    const int lgB = __builtin_ctz((unsigned)t.B);
    for (size_t i = 0; i < t.exp.size(); ++i) {
        const sp::ExportEntry &e = t.exp[i];
        const int phi = e.src & 0xFFFF, pc = (e.src >> 16) & 0xFFFF;
        const int has_pc = e.dst_pc >= 0;
        // both mailbox offsets must fit 16 bits, the (pi, c) one in float2 units
        if (e.dst_phi < 0 || e.dst_phi > 0xFFFF || e.dst_pc > 0xFFFF) return SP_EINVAL;
        ex[i].x = (int)((unsigned)phi | ((unsigned)(has_pc ? sp::pc_slot(pc, lgB, t.B) : 0) << 13) |
                        ((unsigned)e.code << 25) | ((unsigned)has_pc << 31));
        ex[i].y = (int)((unsigned)e.dst_phi | ((unsigned)(has_pc ? e.dst_pc : 0) << 16));
    }
    // the kernel re-derives the phi index of a full import from its (pi, c)
    // index with shifts (B a power of two): check the derivation against the
    // planner's tables
    for (size_t i = 0; i < t.imp_full.size(); ++i) {
        const int c = t.imp_full[i] >> 16, want = t.imp_full[i] & 0xFFFF;
        const int pidx = (((c >> (2 * lgB)) + 1) * t.P + ((c >> lgB) & (t.B - 1)) + 1) * t.P + (c & (t.B - 1)) + 1;
        if (pidx != want) return SP_EINVAL;
    }
    cudaError_t e = cudaSuccess;
    auto up = [&](void **dst, const void *src, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess && bytes) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    std::vector<sp::Succ> reuse((size_t)sp::kTypes * sp::kMaxSameSucc, sp::Succ{0, {0, 0, 0}});
    for (int S = 0; S < sp::kTypes; ++S) {
        if ((int)t.reuse_succ[S].size() > sp::kMaxSameSucc) return SP_EINVAL;
        for (size_t i = 0; i < t.reuse_succ[S].size(); ++i) reuse[(size_t)S * sp::kMaxSameSucc + i] = t.reuse_succ[S][i];
    }
    up((void **)&td.d_imp, imp.data(), imp.size() * sizeof(unsigned short));
    up((void **)&td.d_exp, ex.data(), ex.size() * sizeof(int2));
    up((void **)&td.d_reuse, reuse.data(), reuse.size() * sizeof(sp::Succ));
    h.imp = td.d_imp;
    h.exp = td.d_exp;
    h.reuse = td.d_reuse;
    if (e != cudaSuccess) {
        cudaFree(td.d_imp);
        cudaFree(td.d_exp);
        cudaFree(td.d_reuse);
        return e == cudaErrorMemoryAllocation ? SP_ENOMEM : SP_ECUDA;
    }
    g->tables[B] = td;
    return SP_OK;
}

// One contiguous device array of every table the plan uses; SimDev::tab_index
// picks the entry (the region kernel copies the array into shared memory).
int upload_tables(sp_grid *g)
{
    for (auto &kv : g->tables) {
        TablesOnDevice &td = kv.second;
        if (td.d_dev) continue;
        td.dev.imp_smem = 0;  // the only table of its launch: import lists at the start of the area
        cudaError_t e = cudaMalloc((void **)&td.d_dev, sizeof(sp::TablesDev));
        if (e == cudaSuccess) e = cudaMemcpy(td.d_dev, &td.dev, sizeof(sp::TablesDev), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return SP_ENOMEM;
    }
    return SP_OK;
}

void free_plan(sp_grid *g)
{
    for (auto &kv : g->tables) {
        cudaFree(kv.second.d_imp);
        cudaFree(kv.second.d_exp);
        cudaFree(kv.second.d_reuse);
        cudaFree(kv.second.d_dev);
        cudaFree(kv.second.d_oimp);
        cudaFree(kv.second.d_oexp);
        cudaFree(kv.second.d_oface);
        cudaFree(kv.second.d_oct);
    }
    g->tables.clear();
    g->groups.clear();
    for (float2 *m : g->mbox) cudaFree(m);
    g->mbox.clear();
    for (auto &kv : g->lat) {
        cudaFree(kv.second.d_cell);
        cudaFree(kv.second.d_imp_all);
        cudaFree(kv.second.d_nb);
        cudaFree(kv.second.d_pcoff);
    }
    g->lat.clear();
    for (float2 *f : g->phi_odd) cudaFree(f);
    g->phi_odd.clear();
    cudaFree(g->d_lat_flags);
    g->d_lat_flags = nullptr;
    g->lat_flag_off.clear();
    g->shape = SP_SHAPE_SPLIT;
    if (g->region_graph.exec) cudaGraphExecDestroy(g->region_graph.exec);
    g->region_graph.exec = nullptr;
    g->region_graph.key.clear();
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

int default_threads(int B) { return B <= 8 ? 64 : B == 32 ? sp::region_oct_workers() : 384; }

// Pending device error of the last region launch -> SP code.
int collect_device_error(sp_grid *g)
{
    sp::Ctl ctl[kMaxGroups];
    cudaError_t e = cudaMemcpyAsync(ctl, g->d_ctl, sizeof ctl, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return SP_ECUDA;
    for (const sp::Ctl &c : ctl)
        if (c.error == sp::kDevTimeout) return SP_ETIMEOUT;
    for (const sp::Ctl &c : ctl)
        if (c.error != 0) return SP_ECUDA;
    return SP_OK;
}

int enqueue_sweep(sp_grid *g, int s, int64_t nsteps, int64_t first_local, const sp::LevelCoef *d_coef_sim)
{
    const sp_params &p = g->p[s];
    const int64_t sites = sites_of(p);
    const sp::PhysConst q = phys_const(p);
    float2 *a = g->phi[s], *b = g->d_tmp;
    cudaError_t e = cudaSuccess;
    for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
        e = sp::launch_sweep(a, b, g->pc[s], p.n, d_coef_sim, (int)(first_local + k), q, g->stream);
        std::swap(a, b);
    }
    if (e == cudaSuccess && a != g->phi[s])
        e = cudaMemcpyAsync(g->phi[s], a, sites * sizeof(float2), cudaMemcpyDeviceToDevice, g->stream);
    return e == cudaSuccess ? SP_OK : SP_ECUDA;
}

// nsteps whole-grid steps of simulation s.  On a capturable stream the steps
// are recorded once into a CUDA graph (one node per step) and replayed while
// the call repeats with the same buffers and coefficients, which removes the
// per-launch gaps of the plain loop.
int sweep_steps(sp_grid *g, int s, int64_t nsteps, int64_t first_local, const sp::LevelCoef *d_coef_sim)
{
    if (nsteps <= 0) return SP_OK;
    const int64_t sites = sites_of(g->p[s]);
    cudaError_t e = grow(&g->d_tmp, &g->cap_tmp, (size_t)sites);
    if (e != cudaSuccess) return SP_ENOMEM;
    if (g->stream == nullptr) return enqueue_sweep(g, s, nsteps, first_local, d_coef_sim);
    SweepGraph &sg = g->sweep_graph;
    if (!(sg.exec && sg.sim == s && sg.steps == nsteps && sg.first_local == first_local && sg.coef == d_coef_sim &&
          sg.phi == g->phi[s] && sg.tmp == g->d_tmp)) {
        if (sg.exec) cudaGraphExecDestroy(sg.exec);
        sg.exec = nullptr;
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return SP_ECUDA;
        int rc = enqueue_sweep(g, s, nsteps, first_local, d_coef_sim);
        e = cudaStreamEndCapture(g->stream, &graph);
        if (rc != SP_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return SP_ECUDA;
        }
        e = cudaGraphInstantiate(&sg.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            sg.exec = nullptr;
            return SP_ECUDA;
        }
        sg.sim = s;
        sg.steps = nsteps;
        sg.first_local = first_local;
        sg.coef = d_coef_sim;
        sg.phi = g->phi[s];
        sg.tmp = g->d_tmp;
    }
    return cudaGraphLaunch(sg.exec, g->stream) == cudaSuccess ? SP_OK : SP_ECUDA;
}

// The launches of one region-path call: per region base, the cost-model
// features and buckets (when asked for), the queue reset and the persistent
// region kernel over its simulations' whole bands; then each simulation's
// remainder steps as whole-grid steps.  Timing events 1 and 2 bracket the
// region kernels.
int enqueue_region_call(sp_grid *g, const std::vector<GroupLaunch> &groups, int64_t n_steps, bool timing, bool feats,
                        bool capturing)
{
    cudaError_t e = cudaSuccess;
    auto mark = [&](cudaEvent_t ev) {
        if (e == cudaSuccess)
            e = capturing ? cudaEventRecordWithFlags(ev, g->stream, cudaEventRecordExternal)
                          : cudaEventRecord(ev, g->stream);
    };
    for (size_t gi = 0; gi < groups.size() && e == cudaSuccess; ++gi) {
        const GroupLaunch &gl = groups[gi];
        const sp::RegionArgs &a = gl.a;
        if (feats) {
            // the previous call's trace feeds feature 15 when it covered the same regions
            const unsigned long long *prev = g->prev_trace_ok ? g->d_trace + 2 * (size_t)gl.roff : nullptr;
            e = sp::launch_features(a, g->d_simf + gl.sim_off, prev, g->d_feat + (size_t)SP_MODEL_FEATURES * gl.roff,
                                    g->stream);
            if (e == cudaSuccess && a.prio)
                e = sp::model_buckets(g->model, g->d_feat + (size_t)SP_MODEL_FEATURES * gl.roff, a.total,
                                      g->d_prio + gl.roff, g->stream);
        }
        if (e == cudaSuccess) e = sp::launch_reset(a, g->stream);
        if (timing && gi == 0) mark(g->ev[1]);
        if (e == cudaSuccess)
            e = gl.cfg.B == 32 ? sp::launch_region_oct(a, gl.cfg.smem, gl.cfg.grid / 8, g->stream)
                               : sp::launch_region(a, gl.cfg.threads, gl.cfg.B, gl.cfg.smem, gl.cfg.grid, g->stream);
    }
    if (groups.empty() && timing) mark(g->ev[1]);
    if (timing) mark(g->ev[2]);
    if (e != cudaSuccess) return SP_ECUDA;
    for (int s = 0; s < g->n_sims; ++s) {
        const int H = g->B[s] / 2;
        const int64_t done = (n_steps / H) * H;
        if (n_steps - done <= 0) continue;
        const int rc = enqueue_sweep(g, s, n_steps - done, done, g->d_coef + (size_t)s * n_steps);
        if (rc != SP_OK) return rc;
    }
    return SP_OK;
}

// Runs the region-path call.  On a capturable stream the launch sequence is
// recorded once into a CUDA graph and replayed while every by-value launch
// parameter is unchanged, so a repeated call costs one graph launch.
int run_region_call(sp_grid *g, const std::vector<GroupLaunch> &groups, int64_t n_steps, bool timing, bool feats)
{
    if (g->stream == nullptr || !g->use_graphs) return enqueue_region_call(g, groups, n_steps, timing, feats, false);
    std::vector<unsigned char> key;
    append_key(&key, n_steps);
    append_key(&key, timing);
    append_key(&key, feats);
    append_key(&key, g->d_feat);
    append_key(&key, g->d_simf);
    append_key(&key, g->d_prio);
    append_key(&key, g->prev_trace_ok);
    append_key(&key, groups.size());
    for (const GroupLaunch &gl : groups) {
        append_key(&key, gl.a);
        append_key(&key, gl.cfg);
        append_key(&key, gl.sim_off);
        append_key(&key, gl.roff);
    }
    append_key(&key, g->d_tmp);
    append_key(&key, g->d_coef);
    for (int s = 0; s < g->n_sims; ++s) {
        append_key(&key, g->phi[s]);
        append_key(&key, g->pc[s]);
        append_key(&key, g->B[s]);
    }
    RegionGraph &rg = g->region_graph;
    if (!rg.exec || rg.key != key) {
        if (rg.exec) cudaGraphExecDestroy(rg.exec);
        rg.exec = nullptr;
        rg.key.clear();
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return SP_ECUDA;
        const int rc = enqueue_region_call(g, groups, n_steps, timing, feats, true);
        e = cudaStreamEndCapture(g->stream, &graph);
        if (rc != SP_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc != SP_OK ? rc : SP_ECUDA;
        }
        e = cudaGraphInstantiate(&rg.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            rg.exec = nullptr;
            return SP_ECUDA;
        }
        rg.key = key;
    }
    return cudaGraphLaunch(rg.exec, g->stream) == cudaSuccess ? SP_OK : SP_ECUDA;
}

// A lattice call: per group (lattice size), the reset (ticket counter, error
// word, layer epoch) and the persistent kernel over all its simulations'
// regions; then, for an odd step count, phi (left in the odd-level array)
// copied back to the caller's array.  Timing events 1 and 2 bracket the
// kernels.
struct LatLaunch {
    GroupCfg cfg;
    sp::LatArgs a;
};

int enqueue_lattice_call(sp_grid *g, const std::vector<LatLaunch> &launches, int64_t n_steps, bool timing,
                         bool capturing)
{
    cudaError_t e = cudaSuccess;
    auto mark = [&](cudaEvent_t ev) {
        if (e == cudaSuccess)
            e = capturing ? cudaEventRecordWithFlags(ev, g->stream, cudaEventRecordExternal)
                          : cudaEventRecord(ev, g->stream);
    };
    for (size_t i = 0; i < launches.size() && e == cudaSuccess; ++i) {
        const LatLaunch &l = launches[i];
        e = sp::launch_lattice_reset(l.a.ctl, l.a.Lcount, g->stream);
        if (timing && i == 0) mark(g->ev[1]);
        if (e == cudaSuccess) e = sp::launch_lattice(l.a, l.cfg.threads, l.cfg.smem, l.cfg.grid, g->stream);
    }
    if (launches.empty() && timing) mark(g->ev[1]);
    if (timing) mark(g->ev[2]);
    if (n_steps & 1)
        for (int s = 0; s < g->n_sims && e == cudaSuccess; ++s)
            e = cudaMemcpyAsync(g->phi[s], g->phi_odd[s], (size_t)sites_of(g->p[s]) * sizeof(float2),
                                cudaMemcpyDeviceToDevice, g->stream);
    return e == cudaSuccess ? SP_OK : SP_ECUDA;
}

int run_lattice_call(sp_grid *g, const std::vector<LatLaunch> &launches, int64_t n_steps, bool timing)
{
    if (g->stream == nullptr || !g->use_graphs) return enqueue_lattice_call(g, launches, n_steps, timing, false);
    std::vector<unsigned char> key;
    append_key(&key, (int)SP_SHAPE_LATTICE);
    append_key(&key, n_steps);
    append_key(&key, timing);
    append_key(&key, launches.size());
    for (const LatLaunch &l : launches) {
        append_key(&key, l.cfg);
        append_key(&key, l.a);
    }
    for (int s = 0; s < g->n_sims; ++s) {
        append_key(&key, g->phi[s]);
        append_key(&key, g->phi_odd[s]);
    }
    RegionGraph &rg = g->region_graph;
    if (!rg.exec || rg.key != key) {
        if (rg.exec) cudaGraphExecDestroy(rg.exec);
        rg.exec = nullptr;
        rg.key.clear();
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return SP_ECUDA;
        const int rc = enqueue_lattice_call(g, launches, n_steps, timing, true);
        e = cudaStreamEndCapture(g->stream, &graph);
        if (rc != SP_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc != SP_OK ? rc : SP_ECUDA;
        }
        e = cudaGraphInstantiate(&rg.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            rg.exec = nullptr;
            return SP_ECUDA;
        }
        rg.key = key;
    }
    return cudaGraphLaunch(rg.exec, g->stream) == cudaSuccess ? SP_OK : SP_ECUDA;
}

// The region path of sp_evolve for a lattice plan: every step count runs as
// regions (layers cut by the call's first and last levels).
int evolve_lattice(sp_grid *g, int64_t n_steps, bool trace, bool timing)
{
    if (n_steps > 0x3fffffffll) return SP_EINVAL;
    std::vector<sp::LatSimDev> sims;
    std::vector<LatLaunch> launches;
    std::vector<size_t> sim_off;
    long long trace_total = 0;
    g->last_tile_base.assign(g->n_sims, 0);
    g->last_tiles.assign(g->n_sims, 0);
    for (size_t gi = 0; gi < g->groups.size(); ++gi) {
        const GroupCfg &c = g->groups[gi];
        const int s = c.B / 4;
        const LatOnDevice &ld = g->lat.at(s);
        const sp::LatticeTables &t = ld.host;
        const int Lcount = sp::lat_layer_count(s, n_steps);
        LatLaunch l;
        l.cfg = c;
        sp::LatArgs &a = l.a;
        std::memset(&a, 0, sizeof a);  // padding too: the bytes are a graph key
        const size_t first = sims.size();
        long long per_layer_all = 0;
        for (int sim = 0; sim < g->n_sims; ++sim) {
            if (g->B[sim] != c.B) continue;
            sp::LatSimDev d;
            std::memset(&d, 0, sizeof d);
            for (int k = 0; k < 3; ++k) {
                d.n[k] = g->p[sim].n[k];
                d.M[k] = d.n[k] / c.B;
            }
            d.region_base = per_layer_all;
            d.per_layer = 4ll * d.M[0] * d.M[1] * d.M[2];
            d.coef = g->d_coef + (size_t)sim * n_steps;
            d.q = phys_const(g->p[sim]);
            d.phi0 = g->phi[sim];
            d.phi1 = g->phi_odd[sim];
            d.pc = g->pc[sim];
            d.trace_base = trace_total;
            g->last_tile_base[sim] = (unsigned)trace_total;
            g->last_tiles[sim] = (unsigned)(d.per_layer * Lcount);
            trace_total += d.per_layer * Lcount;
            per_layer_all += d.per_layer;
            sims.push_back(d);
        }
        if (per_layer_all == 0) continue;
        if (per_layer_all * Lcount > 0xfffffff0ll || trace_total > 0x7fffffffll) return SP_EINVAL;
        a.n_sims = (int)(sims.size() - first);
        a.s = s;
        a.K = t.K;
        a.T = (int)n_steps;
        a.n_slots = t.n_slots;
        a.n_foot = t.n_foot;
        a.Lcount = Lcount;
        a.per_layer_all = (unsigned)per_layer_all;
        a.total = (unsigned)(per_layer_all * Lcount);
        a.cell = ld.d_cell;
        a.imp_all = reinterpret_cast<const uint2 *>(ld.d_imp_all);
        a.n_imp_all = (int)(t.imp_all.size() / 2);
        a.row_nb = ld.d_nb;
        a.row_pc = ld.d_pcoff;
        a.max_cell_n = t.max_cell_n;
        a.flags = g->d_lat_flags + g->lat_flag_off[gi];
        a.ctl = g->d_ctl + gi;
        a.fault_drop = g->fault_drop;
        for (int k = 0; k <= t.K; ++k) {
            a.cell_off[k] = t.cell_off[k];
            if (k < t.K) a.cell_n[k] = t.cell_n[k];
        }
        sim_off.push_back(first);
        launches.push_back(l);
    }
    cudaError_t e = grow(&g->d_lsims, &g->cap_lsims, sims.size());
    if (e == cudaSuccess && trace) e = grow(&g->d_trace, &g->cap_trace, 2 * (size_t)trace_total);
    if (e != cudaSuccess) return SP_ENOMEM;
    for (size_t i = 0; i < launches.size(); ++i) {
        launches[i].a.sims = g->d_lsims + sim_off[i];
        launches[i].a.trace = trace ? g->d_trace : nullptr;
    }
    if (sims.size() != g->up_lsims.size() ||
        std::memcmp(sims.data(), g->up_lsims.data(), sims.size() * sizeof(sp::LatSimDev)) != 0) {
        e = cudaMemcpyAsync(g->d_lsims, sims.data(), sims.size() * sizeof(sp::LatSimDev), cudaMemcpyHostToDevice,
                            g->stream);
        if (e != cudaSuccess) return SP_ECUDA;
        g->up_lsims = sims;
    }
    if (g->up_limit != g->wait_limit_ns) {
        unsigned long long lim = g->wait_limit_ns;
        for (int i = 0; i < kMaxGroups && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(&g->d_ctl[i].wait_limit_ns, &lim, sizeof lim, cudaMemcpyHostToDevice, g->stream);
        if (e != cudaSuccess) return SP_ECUDA;
        g->up_limit = lim;
    }
    if (trace) g->trace_total = (unsigned)trace_total;
    g->last_traced = trace;
    g->last_features = false;
    g->last_total = (unsigned)trace_total;
    g->prev_trace_ok = false;
    return run_lattice_call(g, launches, n_steps, timing);
}

// Worker counts of the region kernel (every worker does every step).
bool valid_threads(int t)
{
    return t == 64 || t == 128 || t == 256 || t == 320 || t == 384 || t == 480 || t == 512 || t == 768;
}


// Builds the plan for fixed region bases (one per simulation) and worker
// count: threads = 0 gives every base its default; otherwise every base gets
// threads, or only the largest base when largest_only is set.
int plan_fixed(sp_grid *g, const std::vector<int> &Bs, int threads, int order, const char *model_path,
               bool largest_only = false)
{
    free_plan(g);
    if (g->model) sp_model_destroy(g->model);
    g->model = nullptr;
    if (order == SP_ORDER_LEARNED) {
        if (!model_path) return SP_EINVAL;
        const int rc = sp_model_load(model_path, g->stream, &g->model);
        if (rc != SP_OK) return rc;
    }
    g->B = Bs;
    g->max_B = 0;
    for (int s = 0; s < g->n_sims; ++s) {
        g->max_B = std::max(g->max_B, Bs[s]);
        int rc = build_device_tables(g, Bs[s]);
        if (rc != SP_OK) return rc;
    }
    int rct = upload_tables(g);
    if (rct != SP_OK) return rct;
    // one launch configuration per base, largest base first
    cudaError_t e = cudaSuccess;
    g->threads = threads;
    for (auto it = g->tables.rbegin(); it != g->tables.rend(); ++it) {
        GroupCfg c;
        c.B = it->first;
        if (it->second.octant) {
            // base 32: one region per 8-CTA cluster, as many clusters as fit
            c.threads = sp::region_oct_workers();
            c.smem = sp::region_oct_smem_bytes(it->second.oct_dev.imp_n, it->second.oct_dev.face_total);
            if (c.smem > 227 * 1024) return SP_EINVAL;
            int clusters = 0;
            e = sp::region_oct_clusters(c.smem, &clusters);
            if (e != cudaSuccess || clusters < 1) return SP_EINVAL;
            c.ctas_per_sm = 1;
            c.grid = 8 * clusters;
            g->groups.push_back(c);
            continue;
        }
        const bool mine = threads && (!largest_only || c.B == g->max_B);
        c.threads = mine ? threads : default_threads(c.B);
        int n_in = 0;
        for (int s = 0; s < g->n_sims; ++s) n_in += g->B[s] == c.B;
        c.smem = sp::region_smem_bytes(c.B, 1, n_in, it->second.dev.imp_n);
        if (c.smem > 227 * 1024) return SP_EINVAL;
        e = sp::region_occupancy(c.threads, c.B, c.smem, &c.ctas_per_sm);
        if (e != cudaSuccess || c.ctas_per_sm < 1) return SP_EINVAL;
        c.grid = c.ctas_per_sm * g->sm_count;
        g->groups.push_back(c);
    }
    if ((int)g->groups.size() > kMaxGroups) return SP_EINVAL;
    g->order = order;
    // mailboxes: one slot for every band (the default: half the memory of
    // the ring, measured as fast at bases 8 and 16; regions also wait for the
    // previous band's readers of the mailboxes they write), or a ring of two
    // band slots
    g->mb_slot.assign(g->n_sims, 0);
    g->mb_elems.assign(g->n_sims, 0);
    g->mb_type_off.assign(g->n_sims, {});
    for (int s = 0; s < g->n_sims; ++s) {
        const TablesOnDevice &td = g->tables[g->B[s]];
        long long J = 1;
        for (int d = 0; d < 3; ++d) J *= g->p[s].n[d] / g->B[s];
        long long off = 0;
        for (int S = 0; S < sp::kTypes; ++S) {
            g->mb_type_off[s][S] = off;
            off += J * td.region_mb_size[S];
        }
        const int slots = g->mb_slots;
        g->mb_elems[s] = off;
        g->mb_slot[s] = slots == 2 ? off : 0;
        const size_t bytes = std::max<size_t>((size_t)slots * off * sizeof(float2), 16);
        float2 *m = nullptr;
        e = cudaMalloc((void **)&m, bytes);
        if (e != cudaSuccess) {
            free_plan(g);
            return SP_ENOMEM;
        }
        g->mbox.push_back(m);
    }
    g->planned = true;
    return SP_OK;
}

// Lattice plans (SP_SHAPE_LATTICE): B = 4s per simulation.  Tables per
// distinct s, one launch configuration per s (largest first), the odd-level
// phi array of every simulation and the done flags of every group.
int choose_lattice_B(const sp_params &p, int requested)
{
    auto ok = [&](int B) {
        if (B < 4 || B > 4 * sp::kLatMaxS || B % 4) return false;
        for (int d = 0; d < 3; ++d)
            if (p.n[d] % B != 0) return false;
        return (long long)p.n[1] * p.n[2] <= 0xffffffffll;  // a row's y + n1 z is 32 bits
    };
    if (requested) return ok(requested) ? requested : -1;
    for (int B : {16, 8, 4})
        if (ok(B)) return B;
    return -1;
}

int plan_lattice(sp_grid *g, const std::vector<int> &Bs, int threads)
{
    free_plan(g);
    if (g->model) sp_model_destroy(g->model);
    g->model = nullptr;
    if (threads != 0 && !sp::lattice_valid_threads(threads)) return SP_EINVAL;
    g->B = Bs;
    g->max_B = 0;
    cudaError_t e = cudaSuccess;
    for (int sim = 0; sim < g->n_sims; ++sim) {
        g->max_B = std::max(g->max_B, Bs[sim]);
        const int s = Bs[sim] / 4;
        if (g->lat.count(s)) continue;
        LatOnDevice &ld = g->lat[s];
        if (!sp::build_lattice_tables(s, &ld.host).empty()) return SP_EINVAL;
        const sp::LatticeTables &t = ld.host;
        e = cudaMalloc((void **)&ld.d_cell, t.cell.size() * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&ld.d_imp_all, std::max<size_t>(t.imp_all.size(), 4) * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&ld.d_nb, t.row_nb.size() * sizeof(uint64_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&ld.d_pcoff, t.row_pc.size() * sizeof(int32_t));
        if (e == cudaSuccess)
            e = cudaMemcpy(ld.d_cell, t.cell.data(), t.cell.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !t.imp_all.empty())
            e = cudaMemcpy(ld.d_imp_all, t.imp_all.data(), t.imp_all.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(ld.d_nb, t.row_nb.data(), t.row_nb.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(ld.d_pcoff, t.row_pc.data(), t.row_pc.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_plan(g);
            return SP_ENOMEM;
        }
    }
    size_t flags = 0;
    for (auto it = g->lat.rbegin(); it != g->lat.rend(); ++it) {
        const sp::LatticeTables &t = it->second.host;
        GroupCfg c;
        c.B = 4 * it->first;
        // default (measured): 64 workers up to s = 2 (at most 76 cells a
        // level), 128 at s = 3 and 4, 256 at s = 5, 512 at s = 6
        const int s_lat = it->first;
        c.threads = threads ? threads : s_lat <= 2 ? 64 : s_lat <= 4 ? 128 : s_lat == 5 ? 256 : 512;
        c.smem = sp::lattice_smem_bytes(t.n_slots, t.n_foot, t.rb_side, t.max_cell_n);
        if (c.smem > 227 * 1024) return SP_EINVAL;
        e = sp::lattice_occupancy(c.threads, c.smem, &c.ctas_per_sm);
        if (e != cudaSuccess || c.ctas_per_sm < 1) return SP_EINVAL;
        c.grid = c.ctas_per_sm * g->sm_count;
        g->groups.push_back(c);
        g->lat_flag_off.push_back(flags);
        long long per_layer = 0;
        for (int sim = 0; sim < g->n_sims; ++sim)
            if (g->B[sim] == c.B) per_layer += 4ll * (g->p[sim].n[0] / c.B) * (g->p[sim].n[1] / c.B) * (g->p[sim].n[2] / c.B);
        if (per_layer > 0x7fffffffll) return SP_EINVAL;
        flags += 4 * (size_t)per_layer;
    }
    if ((int)g->groups.size() > kMaxGroups) return SP_EINVAL;
    e = cudaMalloc((void **)&g->d_lat_flags, std::max<size_t>(flags, 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_lat_flags, 0, std::max<size_t>(flags, 1) * sizeof(int), g->stream);
    for (int sim = 0; sim < g->n_sims && e == cudaSuccess; ++sim) {
        float2 *f = nullptr;
        e = cudaMalloc((void **)&f, (size_t)sites_of(g->p[sim]) * sizeof(float2));
        if (e == cudaSuccess) g->phi_odd.push_back(f);
    }
    if (e != cudaSuccess) {
        free_plan(g);
        return SP_ENOMEM;
    }
    g->order = SP_ORDER_STATIC;
    g->threads = threads;
    g->mb_slot.assign(g->n_sims, 0);
    g->mb_elems.assign(g->n_sims, 0);
    g->shape = SP_SHAPE_LATTICE;
    g->planned = true;
    return SP_OK;
}

// Side of a trial grid along one axis: the simulation's own side up to 128
// cells, else 128 (a multiple of 16 when the side is) or 120.
int trial_side(int n) { return n <= 128 ? n : (n % 16 == 0 ? 128 : 120); }

// Autotuner: times every candidate (region-base policy x worker count) on
// scratch copies of the simulations -- the state itself is not touched --
// and returns the fastest.  A candidate is timed by CUDA events around a
// 16-step region-path call (two bands at B = 16, four at B = 8), best of
// two after one warm-up call.  Simulations larger than 128 cells along an
// axis are timed on a 128^3-class trial grid holding the first sites of
// their state.
int autotune(sp_grid *g, int base_B, int block_shape, std::vector<int> *best_B, int *best_threads)
{
    std::vector<std::vector<int>> policies;
    if (base_B == SP_AUTOTUNE) {
        for (int pref : {8, 16, 32}) {
            std::vector<int> Bs(g->n_sims);
            bool ok = true;
            for (int s = 0; s < g->n_sims && ok; ++s) {
                Bs[s] = choose_B(g->p[s], pref);
                if (Bs[s] < 0 && pref > 16) Bs[s] = choose_B(g->p[s], 16);
                if (Bs[s] < 0) Bs[s] = choose_B(g->p[s], 8);
                ok = Bs[s] > 0;
            }
            if (ok && std::find(policies.begin(), policies.end(), Bs) == policies.end()) policies.push_back(Bs);
        }
    } else {
        std::vector<int> Bs(g->n_sims);
        for (int s = 0; s < g->n_sims; ++s) {
            Bs[s] = choose_B(g->p[s], base_B);
            if (Bs[s] < 0) return SP_EINVAL;
        }
        policies.push_back(Bs);
    }
    if (policies.empty()) return SP_EINVAL;

    // trial grids: copies (or leading parts) of each simulation's state
    std::vector<sp_params> tp = g->p;
    for (auto &p : tp) {
        for (int d = 0; d < 3; ++d) p.n[d] = trial_side(p.n[d]);
        p.damp_steps = 0;
    }
    sp_grid *t = nullptr;
    int rc = sp_grid_create(tp.data(), g->n_sims, nullptr, g->stream, &t);
    if (rc != SP_OK) return rc;
    t->mb_slots = g->mb_slots;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < g->n_sims && e == cudaSuccess; ++s) {
        const size_t sites = (size_t)sites_of(tp[s]);
        e = cudaMemcpyAsync(t->phi[s], g->phi[s], sites * sizeof(float2), cudaMemcpyDeviceToDevice, g->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(t->pc[s], g->pc[s], sites * sizeof(float4), cudaMemcpyDeviceToDevice, g->stream);
    }
    if (e != cudaSuccess) {
        sp_destroy(t);
        return SP_ECUDA;
    }
    constexpr int kTrialSteps = 16;
    float best = 0.0f;
    bool have = false;
    for (const auto &Bs : policies) {
        const int maxB = *std::max_element(Bs.begin(), Bs.end());
        std::vector<int> shapes;
        if (block_shape != SP_AUTOTUNE)
            shapes.push_back(block_shape ? block_shape : default_threads(maxB));
        else if (maxB <= 8)
            shapes = {64, 128};
        else
            shapes = {320, 384, 480};
        for (int nt : shapes) {
            rc = plan_fixed(t, Bs, nt, SP_ORDER_STATIC, nullptr, block_shape == SP_AUTOTUNE);
            if (rc == SP_EINVAL) continue;  // does not fit this device
            float ms = 0.0f;
            for (int rep = 0; rep < 3 && rc == SP_OK; ++rep) {
                rc = sp_evolve(t, kTrialSteps, SP_RESTART | SP_TIMING);
                float m = 0.0f;
                if (rc == SP_OK && cudaEventElapsedTime(&m, t->ev[0], t->ev[3]) != cudaSuccess) rc = SP_ECUDA;
                if (rep == 1 || (rep == 2 && m < ms)) ms = m;
            }
            if (rc != SP_OK) {
                sp_destroy(t);
                return rc;
            }
            ++g->tune.candidates;
            const bool is_default = Bs == policies.back() && nt == default_threads(maxB);
            if (is_default) g->tune.default_ms = ms;
            if (!have || ms < best) {
                best = ms;
                have = true;
                *best_B = Bs;
                *best_threads = nt;
            }
        }
    }
    sp_destroy(t);
    if (!have) return SP_EINVAL;
    g->tune.autotuned = 1;
    g->tune.best_ms = best;
    g->tune.trial_steps = kTrialSteps;
    return SP_OK;
}

// Autotuner of lattice plans: for every lattice size B = 4s that divides
// every side (and every worker count when block_shape is SP_AUTOTUNE), a
// scratch grid of the simulations cut to at most 128 cells per side (a
// multiple of B) runs 32-step calls from a copy of the current state; the
// candidate with the least time per site-update (best of two after a
// warm-up call) wins.
int autotune_lattice(sp_grid *g, int base_B, int block_shape, std::vector<int> *best_B, int *best_threads)
{
    std::vector<int> sizes;
    if (base_B == SP_AUTOTUNE) {
        for (int B = 8; B <= 4 * sp::kLatMaxS; B += 4) {
            bool ok = true;
            for (int s = 0; s < g->n_sims && ok; ++s) ok = choose_lattice_B(g->p[s], B) == B;
            if (ok) sizes.push_back(B);
        }
    } else {
        for (int s = 0; s < g->n_sims; ++s)
            if (choose_lattice_B(g->p[s], base_B) < 0) return SP_EINVAL;
        sizes.push_back(base_B ? base_B : 0);
    }
    if (sizes.empty()) return SP_EINVAL;
    const std::vector<int> shapes =
        block_shape == SP_AUTOTUNE ? std::vector<int>{64, 128, 192, 256, 512} : std::vector<int>{block_shape};
    constexpr int kTrialSteps = 32;
    double best = 0.0;
    bool have = false;
    for (int B : sizes) {
        std::vector<int> Bs(g->n_sims);
        std::vector<sp_params> tp = g->p;
        double updates = 0.0;
        for (int s = 0; s < g->n_sims; ++s) {
            Bs[s] = choose_lattice_B(g->p[s], B);
            for (int d = 0; d < 3; ++d)
                if (tp[s].n[d] > 128) tp[s].n[d] = (128 / Bs[s]) * Bs[s];
            tp[s].damp_steps = 0;
            updates += (double)sites_of(tp[s]) * kTrialSteps;
        }
        sp_grid *t = nullptr;
        int rc = sp_grid_create(tp.data(), g->n_sims, nullptr, g->stream, &t);
        if (rc != SP_OK) return rc;
        cudaError_t e = cudaSuccess;
        for (int s = 0; s < g->n_sims && e == cudaSuccess; ++s) {
            const size_t sites = (size_t)sites_of(tp[s]);
            e = cudaMemcpyAsync(t->phi[s], g->phi[s], sites * sizeof(float2), cudaMemcpyDeviceToDevice, g->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(t->pc[s], g->pc[s], sites * sizeof(float4), cudaMemcpyDeviceToDevice, g->stream);
        }
        if (e != cudaSuccess) {
            sp_destroy(t);
            return SP_ECUDA;
        }
        for (int nt : shapes) {
            rc = plan_lattice(t, Bs, nt);
            if (rc == SP_EINVAL) continue;  // does not fit this device
            float ms = 0.0f;
            for (int rep = 0; rep < 3 && rc == SP_OK; ++rep) {
                rc = sp_evolve(t, kTrialSteps, SP_RESTART | SP_TIMING);
                float m = 0.0f;
                if (rc == SP_OK && cudaEventElapsedTime(&m, t->ev[0], t->ev[3]) != cudaSuccess) rc = SP_ECUDA;
                if (rep == 1 || (rep == 2 && m < ms)) ms = m;
            }
            if (rc != SP_OK) {
                sp_destroy(t);
                return rc;
            }
            ++g->tune.candidates;
            const double per = ms / updates;
            if ((B == 16 || B == 0) && (nt == 128 || nt == 0)) g->tune.default_ms = ms;
            if (!have || per < best) {
                best = per;
                have = true;
                *best_B = Bs;
                *best_threads = nt;
                g->tune.best_ms = ms;
            }
        }
        sp_destroy(t);
    }
    if (!have) return SP_EINVAL;
    g->tune.autotuned = 1;
    g->tune.trial_steps = kTrialSteps;
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
    case SP_ESCRATCH:
        return "sp_sweep_noalloc: more than SP_NOALLOC_MAX_SITES (262144) sites or SP_NOALLOC_MAX_STEPS (8192) "
               "steps, the size of its fixed scratch";
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
        void *f[2] = {nullptr, nullptr};
        const size_t unit[2] = {sizeof(float2), sizeof(float4)};
        if (state_dev) {
            for (int k = 0; k < 2; ++k) {
                f[k] = state_dev[2 * s + k];
                if (!f[k] || ((uintptr_t)f[k] & (unit[k] - 1))) {
                    delete g;
                    return SP_EINVAL;
                }
            }
        } else {
            for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
                const size_t bytes = (size_t)sites_of(p[s]) * unit[k];
                e = cudaMalloc(&f[k], bytes);
                if (e == cudaSuccess) e = cudaMemsetAsync(f[k], 0, bytes, g->stream);
            }
        }
        g->phi.push_back((float2 *)f[0]);
        g->pc.push_back((float4 *)f[1]);
        if (e != cudaSuccess) {
            sp_destroy(g);
            return SP_ENOMEM;
        }
    }
    e = cudaMalloc((void **)&g->d_ctl, kMaxGroups * sizeof(sp::Ctl));
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_ctl, 0, kMaxGroups * sizeof(sp::Ctl), g->stream);
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
    if (!g) return SP_EINVAL;
    if (g->shape_opt == SP_SHAPE_LATTICE) {
        // congruent regions in a fixed topological (layer) order: nothing to learn
        if (order != SP_ORDER_STATIC) return SP_EINVAL;
        if (block_shape != 0 && block_shape != SP_AUTOTUNE && !sp::lattice_valid_threads(block_shape))
            return SP_EINVAL;
        g->tune = TuneReport();
        std::vector<int> Bs(g->n_sims);
        int threads = block_shape;
        if (base_B == SP_AUTOTUNE || block_shape == SP_AUTOTUNE) {
            const int rc = autotune_lattice(g, base_B, block_shape, &Bs, &threads);
            if (rc != SP_OK) return rc;
        } else {
            for (int s = 0; s < g->n_sims; ++s) {
                Bs[s] = choose_lattice_B(g->p[s], base_B);
                if (Bs[s] < 0) return SP_EINVAL;
            }
        }
        return plan_lattice(g, Bs, threads);
    }
    // bases are powers of two: the kernels decode cell indices with shifts
    if (base_B != 0 && base_B != SP_AUTOTUNE && base_B != 4 && base_B != 8 && base_B != 16 && base_B != 32)
        return SP_EINVAL;
    if (block_shape != 0 && block_shape != SP_AUTOTUNE && !valid_threads(block_shape)) return SP_EINVAL;
    if (order != SP_ORDER_STATIC && order != SP_ORDER_LEARNED) return SP_EINVAL;
    g->tune = TuneReport();
    std::vector<int> Bs(g->n_sims);
    int threads = block_shape;
    const bool tune_shape = block_shape == SP_AUTOTUNE;
    if (base_B == SP_AUTOTUNE || tune_shape) {
        const int rc = autotune(g, base_B, block_shape, &Bs, &threads);
        if (rc != SP_OK) return rc;
    } else {
        for (int s = 0; s < g->n_sims; ++s) {
            Bs[s] = choose_B(g->p[s], base_B);
            if (Bs[s] < 0) return SP_EINVAL;
        }
    }
    return plan_fixed(g, Bs, threads, order, model_path, tune_shape);
}

int sp_evolve(sp_grid *g, int64_t n_steps, uint32_t flags)
{
    if (!g || n_steps < 0) return SP_EINVAL;
    if (flags & ~(SP_ASYNC | SP_MONOLITHIC | SP_RESTART | SP_TRACE | SP_TIMING | SP_FEATURES)) return SP_EINVAL;
    const bool timing = (flags & SP_TIMING) != 0;
    if (timing && !g->ev[0])
        for (int i = 0; i < 4; ++i)
            if (cudaEventCreate(&g->ev[i]) != cudaSuccess) return SP_ECUDA;
    g->timed = false;
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
    if (timing) {
        e = cudaEventRecord(g->ev[0], g->stream);
        if (e == cudaSuccess && mono) e = cudaEventRecord(g->ev[1], g->stream);
        if (e == cudaSuccess && mono) e = cudaEventRecord(g->ev[2], g->stream);
        if (e != cudaSuccess) return SP_ECUDA;
    }
    if (mono) {
        for (int s = 0; s < g->n_sims && rc == SP_OK; ++s)
            rc = sweep_steps(g, s, n_steps, 0, g->d_coef + (size_t)s * n_steps);
    } else if (g->shape == SP_SHAPE_LATTICE) {
        if (flags & SP_FEATURES) return SP_EINVAL;  // congruent regions: no cost features
        rc = evolve_lattice(g, n_steps, (flags & SP_TRACE) != 0, timing);
    } else {
        // whole bands as regions: one persistent launch per region base over all
        // simulations of that base; region ids run on across the groups
        bool feats = false, prev_trace_ok = false;
        std::vector<sp::SimDev> sims;
        std::vector<int> sim_of;
        std::vector<GroupLaunch> launches;
        unsigned all_total = 0, max_total = 0;
        g->last_tile_base.assign(g->n_sims, 0);
        g->last_tiles.assign(g->n_sims, 0);
        const bool learned = g->order == SP_ORDER_LEARNED && g->model;
        const bool trace = (flags & SP_TRACE) != 0;
        feats = learned || (flags & SP_FEATURES) != 0;
        for (const GroupCfg &c : g->groups) {
            const int B = c.B, H = B / 2;
            const int64_t nb = n_steps / H;
            if (nb == 0) continue;
            GroupLaunch gl;
            gl.cfg = c;
            gl.sim_off = sims.size();
            gl.roff = all_total;
            unsigned total = 0, seeds = 0;
            for (int s = 0; s < g->n_sims; ++s) {
                if (g->B[s] != B) continue;
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
                if ((unsigned long long)all_total + total + tiles > 0x7fffffffull) return SP_EINVAL;
                d.tile_base = total;
                d.tiles = (unsigned)tiles;
                d.seed_base = seeds;
                d.coef = g->d_coef + (size_t)s * n_steps;
                d.q = phys_const(g->p[s]);
                d.phi = g->phi[s];
                d.pc = g->pc[s];
                d.mbox = g->mbox[s];
                d.mb_slot = g->mb_slot[s];
                d.mb_reuse = g->mb_slot[s] == 0;
                for (int S = 0; S < sp::kTypes; ++S) d.mb_type_off[S] = g->mb_type_off[s][S];
                d.tab = g->tables[B].d_dev;
                d.tab_index = 0;
                d.oct = g->tables[B].octant ? g->tables[B].d_oct : nullptr;
                g->last_tile_base[s] = all_total + total;
                g->last_tiles[s] = d.tiles;
                total += d.tiles;
                seeds += (unsigned)d.Jtot * (unsigned)g->tables[B].seed_types;
                sims.push_back(d);
                sim_of.push_back(s);
            }
            if (total == 0) continue;
            sp::RegionArgs &ra = gl.a;
            std::memset(&ra, 0, sizeof ra);  // padding too: the bytes are a graph key
            ra.tabs = g->tables[B].d_dev;
            ra.n_tabs = 1;
            ra.n_sims = (int)(sims.size() - gl.sim_off);
            ra.total = total;
            ra.n_seed = seeds;
            ra.ctl = g->d_ctl + launches.size();
            const long long fd = (long long)g->fault_drop - (long long)all_total;
            ra.fault_drop = (g->fault_drop >= 0 && fd >= 0 && fd < (long long)total) ? (int)fd : -1;
            launches.push_back(gl);
            all_total += total;
            max_total = std::max(max_total, total);
        }
        if (!launches.empty()) {
            e = grow(&g->d_sims, &g->cap_sims, sims.size());
            if (e == cudaSuccess) e = grow(&g->d_counters, &g->cap_counters, max_total);
            if (e == cudaSuccess) e = grow(&g->d_queue, &g->cap_queue, max_total);
            if (e == cudaSuccess && trace) e = grow(&g->d_trace, &g->cap_trace, 2 * (size_t)all_total);
            if (e == cudaSuccess && feats) e = grow(&g->d_feat, &g->cap_feat, (size_t)SP_MODEL_FEATURES * all_total);
            if (e == cudaSuccess && feats) e = grow(&g->d_simf, &g->cap_simf, sims.size());
            if (e == cudaSuccess && learned) e = grow(&g->d_prio, &g->cap_prio, (size_t)all_total);
            if (e != cudaSuccess) return SP_ENOMEM;
            for (GroupLaunch &gl : launches) {  // device addresses, now that the buffers exist
                gl.a.sims = g->d_sims + gl.sim_off;
                gl.a.counters = g->d_counters;
                gl.a.queue = g->d_queue;
                gl.a.trace = trace ? g->d_trace + 2 * (size_t)gl.roff : nullptr;
                gl.a.prio = learned ? g->d_prio + gl.roff : nullptr;
            }
            if (feats) {
                std::vector<float4> simf(sims.size());
                for (size_t i = 0; i < sims.size(); ++i) {
                    const sp_params &pp = g->p[sim_of[i]];
                    simf[i] = make_float4((float)g->B[sim_of[i]] / 16.0f, (float)(std::log2((double)sites_of(pp)) / 24.0),
                                          (float)(pp.nu / 2.0), 0.0f);
                }
                e = cudaMemcpyAsync(g->d_simf, simf.data(), simf.size() * sizeof(float4), cudaMemcpyHostToDevice,
                                    g->stream);
                if (e != cudaSuccess) return SP_ECUDA;
            }
            if (sims.size() != g->up_sims.size() ||
                std::memcmp(sims.data(), g->up_sims.data(), sims.size() * sizeof(sp::SimDev)) != 0) {
                e = cudaMemcpyAsync(g->d_sims, sims.data(), sims.size() * sizeof(sp::SimDev),
                                    cudaMemcpyHostToDevice, g->stream);
                if (e != cudaSuccess) return SP_ECUDA;
                g->up_sims = sims;
            }
            if (g->up_limit != g->wait_limit_ns) {
                unsigned long long lim = g->wait_limit_ns;
                for (int i = 0; i < kMaxGroups && e == cudaSuccess; ++i)
                    e = cudaMemcpyAsync(&g->d_ctl[i].wait_limit_ns, &lim, sizeof lim, cudaMemcpyHostToDevice,
                                        g->stream);
                if (e != cudaSuccess) return SP_ECUDA;
                g->up_limit = lim;
            }
            prev_trace_ok = g->trace_total == all_total;  // the trace buffer still holds a call of this layout
            if (trace) g->trace_total = all_total;
            g->last_traced = trace;
            g->last_features = feats;
            g->last_total = all_total;
        }
        // remainder steps of each simulation: whole-grid steps, same arithmetic
        for (int s = 0; s < g->n_sims; ++s) {
            const int H = g->B[s] / 2;
            const int64_t done = (n_steps / H) * H;
            if (n_steps - done > 0) {
                e = grow(&g->d_tmp, &g->cap_tmp, (size_t)sites_of(g->p[s]));
                if (e != cudaSuccess) return SP_ENOMEM;
            }
        }
        g->prev_trace_ok = prev_trace_ok;
        rc = run_region_call(g, launches, n_steps, timing, feats);
    }
    if (rc != SP_OK) return rc;
    if (timing) {
        e = cudaEventRecord(g->ev[3], g->stream);
        if (e != cudaSuccess) return SP_ECUDA;
        g->timed = true;
    }
    for (int s = 0; s < g->n_sims; ++s) g->level[s] += n_steps;
    if (flags & SP_ASYNC) return SP_OK;
    e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return SP_ECUDA;
    if (!mono) return collect_device_error(g);
    return SP_OK;
}

int sp_set_option(sp_grid *g, int32_t option, int64_t value)
{
    if (!g) return SP_EINVAL;
    switch (option) {
    case SP_OPT_WAIT_LIMIT_NS:
        if (value < 1000000 || value > 60000000000ll) return SP_EINVAL;
        g->wait_limit_ns = (unsigned long long)value;
        return SP_OK;
    case SP_OPT_FAULT_DROP_RELEASE:
        if (value < -1 || value > 0x7fffffffll) return SP_EINVAL;
        g->fault_drop = (int)value;
        return SP_OK;
    case SP_OPT_GRAPHS:
        if (value != 0 && value != 1) return SP_EINVAL;
        g->use_graphs = (int)value;
        return SP_OK;
    case SP_OPT_MAILBOX_SLOTS:
        if (value != 1 && value != 2) return SP_EINVAL;
        g->mb_slots = (int)value;
        return SP_OK;
    case SP_OPT_REGION_SHAPE:
        if (value != SP_SHAPE_SPLIT && value != SP_SHAPE_LATTICE) return SP_EINVAL;
        g->shape_opt = (int)value;
        return SP_OK;
    default:
        return SP_EINVAL;
    }
}

int sp_write_surface(sp_grid *g, int32_t sim, int32_t what, const void *src, size_t src_bytes, int32_t src_is_device)
{
    if (!g || sim < 0 || sim >= g->n_sims || !src) return SP_EINVAL;
    if (what == SP_SURF_LEVEL) {
        if (src_bytes < sizeof(int64_t) || src_is_device) return SP_EINVAL;
        int64_t level;
        std::memcpy(&level, src, sizeof level);
        if (level < 0) return SP_EINVAL;
        g->level[sim] = level;
        return SP_OK;
    }
    if (what != SP_SURF_STATE) return SP_EINVAL;
    const size_t sites = (size_t)sites_of(g->p[sim]);
    if (src_bytes < 24 * sites) return SP_EINVAL;
    const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const char *b = (const char *)src;
    cudaError_t e = cudaMemcpyAsync(g->phi[sim], b, 8 * sites, kind, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->pc[sim], b + 8 * sites, 16 * sites, kind, g->stream);
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
    case SP_SURF_LEVEL: {
        if (dst_bytes < sizeof(int64_t) || dst_is_device) return SP_EINVAL;
        const int64_t level = g->level[sim];
        std::memcpy(dst, &level, sizeof level);
        return SP_OK;
    }
    case SP_SURF_STATE: {
        if (dst_bytes < (size_t)(24 * sites)) return SP_EINVAL;
        char *b = (char *)dst;
        e = cudaMemcpyAsync(b, g->phi[sim], 8 * (size_t)sites, to, g->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b + 8 * (size_t)sites, g->pc[sim], 16 * (size_t)sites, to, g->stream);
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
        e = sp::launch_energy(g->phi[sim], g->pc[sim], p.n, 1.0 / (p.dx * p.dx), p.eta * p.eta,
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
        if (g->shape == SP_SHAPE_LATTICE) {
            const sp::LatticeTables &t = g->lat.at(g->B[sim] / 4).host;
            const int64_t per_layer = 4ll * (p.n[0] / g->B[sim]) * (p.n[1] / g->B[sim]) * (p.n[2] / g->B[sim]);
            sp_plan_info info;
            std::memset(&info, 0, sizeof info);
            info.base_B = g->B[sim];
            for (const GroupCfg &c : g->groups)
                if (c.B == g->B[sim]) {
                    info.threads = c.threads;
                    info.ctas_per_sm = c.ctas_per_sm;
                    info.grid = c.grid;
                }
            info.regions_per_band = per_layer;
            info.updates_per_band = per_layer * t.updates;
            info.bytes_read_per_band = per_layer * t.bytes_read;
            info.bytes_written_per_band = per_layer * t.bytes_written;
            info.bytes_per_update = (double)(t.bytes_read + t.bytes_written) / (double)t.updates;
            info.mailbox_slots = 0;
            info.mailbox_bytes = sites * (int64_t)sizeof(float2);
            info.region_shape = SP_SHAPE_LATTICE;
            info.autotuned = g->tune.autotuned;
            info.tune_candidates = g->tune.candidates;
            info.tune_best_ms = g->tune.best_ms;
            info.tune_default_ms = g->tune.default_ms;
            if (dst_is_device) e = cudaMemcpy(dst, &info, sizeof info, cudaMemcpyHostToDevice);
            else std::memcpy(dst, &info, sizeof info);
            return cuda_err(e);
        }
        const TablesOnDevice &td = g->tables[g->B[sim]];
        sp::PlanStats ps = sp::plan_stats(td.host, p.n);
        if (td.octant) {  // the cluster kernel moves the octant tables' traffic
            int64_t J = 1, upd = 0, rd = 0, wr = 0;
            for (int d = 0; d < 3; ++d) J *= p.n[d] / td.oct.B;
            for (int S = 0; S < sp::kTypes; ++S) {
                upd += td.oct.updates[S];
                rd += td.oct.bytes_read[S];
                wr += td.oct.bytes_written[S];
            }
            ps.bytes_read_per_band = J * rd;
            ps.bytes_written_per_band = J * wr;
            ps.bytes_per_update = (double)(rd + wr) / (double)upd;
        }
        sp_plan_info info;
        std::memset(&info, 0, sizeof info);
        info.base_B = g->B[sim];
        for (const GroupCfg &c : g->groups)
            if (c.B == g->B[sim]) {
                info.threads = c.threads;
                info.ctas_per_sm = c.ctas_per_sm;
                info.grid = c.grid;
            }
        info.regions_per_band = ps.regions_per_band;
        info.updates_per_band = ps.updates_per_band;
        info.bytes_read_per_band = ps.bytes_read_per_band;
        info.bytes_written_per_band = ps.bytes_written_per_band;
        info.bytes_per_update = ps.bytes_per_update;
        info.mailbox_slots = g->mb_slot[sim] ? 2 : 1;
        info.mailbox_bytes = info.mailbox_slots * g->mb_elems[sim] * (int64_t)sizeof(float2);
        info.autotuned = g->tune.autotuned;
        info.tune_candidates = g->tune.candidates;
        info.tune_best_ms = g->tune.best_ms;
        info.tune_default_ms = g->tune.default_ms;
        if (dst_is_device) e = cudaMemcpy(dst, &info, sizeof info, cudaMemcpyHostToDevice);
        else std::memcpy(dst, &info, sizeof info);
        return cuda_err(e);
    }
    case SP_SURF_FEATURES: {
        if (!g->last_features || sim >= (int)g->last_tiles.size()) return SP_EINVAL;
        const size_t bytes = (size_t)g->last_tiles[sim] * SP_MODEL_FEATURES * sizeof(float);
        if (dst_bytes < bytes) return SP_EINVAL;
        e = cudaMemcpyAsync(dst, g->d_feat + (size_t)g->last_tile_base[sim] * SP_MODEL_FEATURES, bytes,
                            dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        return cuda_err(e);
    }
    case SP_SURF_TIMING: {
        if (!g->timed || dst_bytes < 3 * sizeof(double) || dst_is_device) return SP_EINVAL;
        e = cudaEventSynchronize(g->ev[3]);
        float ms[3] = {0, 0, 0};
        for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&ms[i], g->ev[i], g->ev[i + 1]);
        if (e != cudaSuccess) return SP_ECUDA;
        double *o = (double *)dst;
        for (int i = 0; i < 3; ++i) o[i] = ms[i];
        return SP_OK;
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

int sp_lattice_call_bytes(int32_t B, int64_t n_steps, int64_t *updates, int64_t *bytes_read, int64_t *bytes_written)
{
    if (B < 4 || B > 4 * sp::kLatMaxS || B % 4 || n_steps < 1 || !updates || !bytes_read || !bytes_written)
        return SP_EINVAL;
    sp::LatticeTables t;
    if (!sp::build_lattice_tables(B / 4, &t).empty()) return SP_EINVAL;
    const sp::LatCallStats st = sp::lattice_call_stats(t, n_steps);
    *updates = st.updates;
    *bytes_read = st.bytes_read;
    *bytes_written = st.bytes_written;
    return SP_OK;
}

int sp_destroy(sp_grid *g)
{
    if (!g) return SP_EINVAL;
    cudaStreamSynchronize(g->stream);
    free_plan(g);
    if (g->owns_state) {
        for (float2 *f : g->phi) cudaFree(f);
        for (float4 *f : g->pc) cudaFree(f);
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
    cudaFree(g->d_feat);
    cudaFree(g->d_simf);
    cudaFree(g->d_prio);
    cudaFree(g->d_lsims);
    if (g->model) sp_model_destroy(g->model);
    if (g->sweep_graph.exec) cudaGraphExecDestroy(g->sweep_graph.exec);
    if (g->region_graph.exec) cudaGraphExecDestroy(g->region_graph.exec);
    for (int i = 0; i < 4; ++i)
        if (g->ev[i]) cudaEventDestroy(g->ev[i]);
    delete g;
    return SP_OK;
}

}  // extern "C"
