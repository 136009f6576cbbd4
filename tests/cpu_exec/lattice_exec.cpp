// lattice_exec.cpp -- TEST-ONLY CPU scaffold for the 4-cube lattice regions
// (lattice.h).  Compiled by the tests, never part of libsp.so.
//
// It runs the regions of one call one at a time, in the kernel's ticket
// order or a seeded random / last-ready-first topological order, with the
// data flow of the kernel: per-region shared-memory slots tagged with the
// level they hold (every read checks its tag), the next level's imports in
// flight while a level is computed (no cell of that level may touch their
// slots), exports straight into the in-place global arrays (phi in two
// parity buffers, (pi, c) in one).  Every global access is logged and then
// checked against the dependency DAG (each region after its four
// predecessors): the writes of one location form a chain of the DAG order,
// every read sees the value of its level written by an ancestor (or the
// call's initial state), and the next write of that location is made by the
// reader itself, later, or by a descendant.  The result can then be compared
// bit for bit with a whole-grid sweep using the same site update.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "lattice.h"
#include "sp_update.h"

using sp::f2;

namespace {

struct Call {
    sp::LatGeom g;
    int s, K, T, Lmin, Lcount, n[3];
    int64_t per_layer;
    int64_t sites() const { return (int64_t)n[0] * n[1] * n[2]; }
    int64_t regions() const { return (int64_t)Lcount * per_layer; }
    int layer(int64_t id) const { return Lmin + (int)(id / per_layer); }
};

struct Access {
    int64_t loc;   // phi: parity * sites + site; (pi, c): 2 * sites + site
    int32_t region, tau;
    bool write;
    int32_t order;  // position in the region's own program order (level)
};

int64_t site_of(const Call &c, const int a[3], int rx, int ry, int rz)
{
    const int s = c.s;
    const int x = sp::lat_wrap(s * a[0] + rx, c.n[0]);
    const int y = sp::lat_wrap(s * a[1] + ry, c.n[1]);
    const int z = sp::lat_wrap(s * a[2] + rz, c.n[2]);
    return x + (int64_t)c.n[0] * (y + (int64_t)c.n[1] * z);
}

std::string g_err;
// Planted mistakes (tests of the checks themselves): 1 = one phi buffer for
// both parities; 2 = the DAG without the edge n - e_1 -> n; 3 = pair imports
// (16-byte site pairs into slot pairs) whatever the pair bit says; 4 = a
// region cut by the call's first or last level loading every import of the
// whole region (no level filter).
int g_plant = 0;
bool err(const std::string &m)
{
    if (g_err.empty()) g_err = m;
    return false;
}

}  // namespace

extern "C" {

// Whole-grid sweep: nsteps levels with coef4[4 l .. 4 l + 3] for level l.
int lx_sweep(int nx, int ny, int nz, int nsteps, const float *coef4, float dt, float inv_dx2, float eta2, float *phi,
             float *pc)
{
    const int64_t sites = (int64_t)nx * ny * nz;
    std::vector<f2> a((size_t)sites), b((size_t)sites);
    std::memcpy(a.data(), phi, sites * 8);
    sp::PhysConst q = {dt, inv_dx2, eta2, 0.0f};
    for (int l = 0; l < nsteps; ++l) {
        const sp::LevelCoef co = {coef4[4 * l], coef4[4 * l + 1], coef4[4 * l + 2], 0.0f};
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    auto at = [&](int xx, int yy, int zz) {
                        xx = (xx + nx) % nx, yy = (yy + ny) % ny, zz = (zz + nz) % nz;
                        return a[xx + (int64_t)nx * (yy + (int64_t)ny * zz)];
                    };
                    const int64_t i = x + (int64_t)nx * (y + (int64_t)ny * z);
                    f2 p = {pc[4 * i], pc[4 * i + 1]}, c = {pc[4 * i + 2], pc[4 * i + 3]};
                    b[i] = sp::site_update(a[i], at(x - 1, y, z), at(x + 1, y, z), at(x, y - 1, z), at(x, y + 1, z),
                                           at(x, y, z - 1), at(x, y, z + 1), p, c, co, q);
                    pc[4 * i] = p.x, pc[4 * i + 1] = p.y, pc[4 * i + 2] = c.x, pc[4 * i + 3] = c.y;
                }
        std::swap(a, b);
    }
    std::memcpy(phi, a.data(), sites * 8);
    return 0;
}

// Runs one call of nsteps levels as lattice regions of size s.  mode 0: the
// kernel's ticket order (layer by layer); 1: seeded random ready region;
// 2: the most recently readied region first.  Returns 0, or -1 with msg.
// stats (optional, 6 int64): regions, race-checked reads, writes, site-updates
// of one region, bytes read and written from and to the state arrays.
int lx_run(int s, int nx, int ny, int nz, int nsteps, int mode, uint64_t order_seed, const float *coef4, float dt,
           float inv_dx2, float eta2, float *phi, float *pc, char *msg, int msglen, int64_t *stats)
{
    g_err.clear();
    auto finish = [&](int rc) {
        if (msg && msglen > 0) std::snprintf(msg, msglen, "%s", g_err.c_str());
        return rc;
    };
    sp::LatticeTables t;
    std::string e = sp::build_lattice_tables(s, &t);
    if (!e.empty()) return err(e), finish(-1);
    const int w = 4 * s;
    if (nx % w || ny % w || nz % w || nsteps < 1) return err("grid sides must be multiples of 4s"), finish(-1);
    Call c;
    c.s = s, c.K = t.K, c.T = nsteps, c.n[0] = nx, c.n[1] = ny, c.n[2] = nz;
    c.g.s = s, c.g.M[0] = nx / w, c.g.M[1] = ny / w, c.g.M[2] = nz / w;
    c.Lmin = sp::lat_min_layer();
    c.Lcount = sp::lat_layer_count(s, nsteps);
    c.per_layer = sp::lat_per_layer(c.g);
    const int64_t sites = c.sites(), nreg = c.regions();

    // global arrays with level tags
    std::vector<f2> P[2];
    std::vector<int> tagP[2];
    for (int p = 0; p < 2; ++p) P[p].assign((size_t)sites, {0.0f, 0.0f}), tagP[p].assign((size_t)sites, -1000000);
    std::memcpy(P[0].data(), phi, sites * 8);
    std::fill(tagP[0].begin(), tagP[0].end(), 0);
    std::vector<float> G(pc, pc + 4 * sites);
    std::vector<int> tagG((size_t)sites, 0);
    std::vector<int> computed((size_t)sites * nsteps, 0);
    std::vector<Access> log;
    log.reserve(1 << 20);
    const sp::PhysConst q = {dt, inv_dx2, eta2, 0.0f};

    // order
    std::vector<int> npred((size_t)nreg, 0);
    for (int64_t id = 0; id < nreg; ++id) npred[id] = c.layer(id) > c.Lmin ? (g_plant == 2 ? 3 : 4) : 0;
    std::vector<int64_t> order;
    if (mode == 0) {
        for (int64_t id = 0; id < nreg; ++id) order.push_back(id);
    } else {
        std::mt19937_64 rng(order_seed);
        std::vector<int64_t> ready;
        for (int64_t id = 0; id < nreg; ++id)
            if (npred[id] == 0) ready.push_back(id);
        std::vector<int> cnt = npred;
        while (!ready.empty()) {
            size_t pick = mode == 1 ? (size_t)(rng() % ready.size()) : ready.size() - 1;
            const int64_t id = ready[pick];
            ready[pick] = ready.back();
            ready.pop_back();
            order.push_back(id);
            const int L = c.layer(id);
            if (L + 1 >= c.Lmin + c.Lcount) continue;
            int a[3];
            sp::lat_centre(c.g, L, id % c.per_layer, a);
            for (int i = g_plant == 2 ? 1 : 0; i < 4; ++i) {
                int d[3], b[3];
                sp::lat_pred_shift(i, d);
                for (int k = 0; k < 3; ++k) b[k] = sp::lat_wrap(a[k] - d[k], 4 * c.g.M[k]);
                const int64_t sid = (int64_t)(L + 1 - c.Lmin) * c.per_layer + sp::lat_index<int64_t>(c.g, b);
                if (--cnt[sid] == 0) ready.push_back(sid);
            }
        }
        if ((int64_t)order.size() != nreg) return err("dependency DAG has a cycle"), finish(-1);
    }

    // decode checks: centre <-> index, predecessor <-> successor
    for (int64_t id = 0; id < nreg; ++id) {
        const int L = c.layer(id);
        int a[3];
        sp::lat_centre(c.g, L, id % c.per_layer, a);
        for (int k = 0; k < 3; ++k)
            if (a[k] < 0 || a[k] >= 4 * c.g.M[k] || ((a[k] - L) & 1)) return err("centre out of range"), finish(-1);
        if ((((a[0] + a[1] + a[2] + L) % 4) + 4) % 4 != 0) return err("centre off the layer's lattice"), finish(-1);
        if (sp::lat_index<int64_t>(c.g, a) != id % c.per_layer) return err("lat_index does not invert lat_centre"), finish(-1);
        if (sp::lat_index<int32_t>(c.g, a) != (int32_t)(id % c.per_layer)) return err("32-bit index differs"), finish(-1);
        int a32[3];
        sp::lat_centre(c.g, L, (int32_t)(id % c.per_layer), a32);
        if (a32[0] != a[0] || a32[1] != a[1] || a32[2] != a[2]) return err("32-bit centre differs"), finish(-1);
    }

    std::vector<f2> ps[2];
    std::vector<int> tps[2];
    std::vector<float> pcs;
    std::vector<int> tpc;
    auto slot_of = [&](uint32_t e) { return sp::lat_slot(e); };
    auto pc_of = [&](uint32_t e) { return sp::lat_slot(e) + t.row_pc[sp::lat_row(e)]; };

    for (int64_t id : order) {
        const int L = c.layer(id);
        int a[3];
        sp::lat_centre(c.g, L, id % c.per_layer, a);
        const int tau_b = 1 + s * L;
        const int k_lo = std::max(0, 1 - tau_b), k_hi = std::min(c.K - 1, nsteps - tau_b);
        if (k_lo > k_hi) return err("empty region in the call"), finish(-1);
        for (int p = 0; p < 2; ++p) ps[p].assign((t.n_slots + 1) & ~1, {0, 0}), tps[p].assign((t.n_slots + 1) & ~1, -999);
        pcs.assign(4 * (size_t)t.n_foot, 0.0f), tpc.assign(t.n_foot, -999);
        // value of local level k (global tau_b + k); pair: as the kernel does for a
        // region not cut by the call's first level, also copy the site pair's
        // other value into the slot pair's other slot (what the array holds now)
        auto load = [&](uint32_t en, bool full, int k, bool pair = false) {
            const int sl = slot_of(en);
            if (sl < 0 || sl >= t.n_slots) return err("slot out of range");
            int rx, ry, rz;
            t.offset_of(sl, sp::lat_row(en), &rx, &ry, &rz);
            const int64_t g = site_of(c, a, rx, ry, rz);
            const int tau = tau_b + k, par = g_plant == 1 ? 0 : tau & 1;
            if (tagP[par][g] != tau) return err("import of phi sees level " + std::to_string(tagP[par][g]) +
                                                " instead of " + std::to_string(tau));
            log.push_back({par * sites + g, (int32_t)id, tau, false, k + 1});
            ps[k & 1][sl] = P[par][g];
            tps[k & 1][sl] = k;
            // (planted mistake 3: the pair bit ignored)
            if (pair && ((en & (k_lo == 0 ? sp::kLatImpPair : sp::kLatImpPairRow)) || g_plant == 3) &&
                ((sl ^ (int)(g & 1)) & 1) == 0) {
                const int ps2 = sl ^ 1;
                const int64_t g2 = g ^ 1;  // the row's other site of the aligned pair (sides are even)
                if (ps2 >= (int)ps[k & 1].size()) return err("pair slot out of range");
                if (tps[k & 1][ps2] != -999 && !(tps[k & 1][ps2] == tagP[par][g2] - tau_b && ps[k & 1][ps2].x == P[par][g2].x &&
                                                  ps[k & 1][ps2].y == P[par][g2].y))
                    return err("pair copy overwrites a loaded slot with another value");
                ps[k & 1][ps2] = P[par][g2];
                tps[k & 1][ps2] = tagP[par][g2] - tau_b;
            }
            if (full) {
                const int pi = pc_of(en);
                if (pi < 0 || pi >= t.n_foot) return err("(pi, c) index out of range");
                if (tagG[g] != tau) return err("import of (pi, c) sees a wrong level");
                log.push_back({2 * sites + g, (int32_t)id, tau, false, k + 1});
                std::memcpy(&pcs[4 * pi], &G[4 * g], 16);
                tpc[pi] = k;
            }
            return true;
        };
        // cut region: its own cells of level k_lo - 1, whole, from the state at t0
        if (k_lo > 0)
            for (int i = t.cell_off[k_lo - 1]; i < t.cell_off[k_lo - 1] + t.cell_n[k_lo - 1]; ++i)
                if (!load(t.cell[i], true, k_lo - 1)) return finish(-1);
        // every import of the region's levels, at its start, in the kernel's
        // order (the one list of all imports, filtered by level)
        for (size_t i = 0; i + 1 < t.imp_all.size(); i += 2) {
            const uint32_t en = t.imp_all[i];
            const int kk = (int)t.imp_all[i + 1];
            if ((kk < k_lo || kk > k_hi) && g_plant != 4) continue;
            if (((en & sp::kLatImpBuf) != 0) != (((kk - 1) & 1) != 0)) return err("import buffer bit"), finish(-1);
            if (!load(en, (en & sp::kLatImpFull) != 0, kk - 1, true)) return finish(-1);
        }
        for (int k = k_lo; k <= k_hi; ++k) {
            const int tau = tau_b + k;
            const float *cf = coef4 + 4 * (tau - 1);
            const sp::LevelCoef co = {cf[0], cf[1], cf[2], 0.0f};
            const int rp = (k - 1) & 1, wp = k & 1;
            for (int i = t.cell_off[k]; i < t.cell_off[k] + t.cell_n[k]; ++i) {
                const uint32_t en = t.cell[i];
                const int sl = sp::lat_slot(en), pi = pc_of(en);
                const uint64_t rn = t.row_nb[sp::lat_row(en)];
                int rx, ry, rz;
                t.offset_of(sl, sp::lat_row(en), &rx, &ry, &rz);
                if (pi < 0 || pi >= t.n_foot) return err("(pi, c) index out of range"), finish(-1);
                const int nb[7] = {sl, sl - 1, sl + 1, sl + sp::lat_dym(rn), sl + sp::lat_dyp(rn), sl + sp::lat_dzm(rn),
                                   sl + sp::lat_dzp(rn)};
                for (int j = 0; j < 7; ++j) {
                    if (nb[j] < 0 || nb[j] >= t.n_slots) return err("neighbour slot out of range"), finish(-1);
                    if (tps[rp][nb[j]] != k - 1) return err("level " + std::to_string(k) + " reads a phi slot holding level " +
                                                            std::to_string(tps[rp][nb[j]])), finish(-1);
                }
                if (tpc[pi] != k - 1) return err("level reads a (pi, c) slot of a wrong level"), finish(-1);
                f2 p = {pcs[4 * pi], pcs[4 * pi + 1]}, cc = {pcs[4 * pi + 2], pcs[4 * pi + 3]};
                const f2 out = sp::site_update(ps[rp][nb[0]], ps[rp][nb[1]], ps[rp][nb[2]], ps[rp][nb[3]], ps[rp][nb[4]],
                                               ps[rp][nb[5]], ps[rp][nb[6]], p, cc, co, q);
                ps[wp][sl] = out, tps[wp][sl] = k;
                pcs[4 * pi] = p.x, pcs[4 * pi + 1] = p.y, pcs[4 * pi + 2] = cc.x, pcs[4 * pi + 3] = cc.y;
                tpc[pi] = k;
                const int64_t g = site_of(c, a, rx, ry, rz);
                if (++computed[(size_t)(tau - 1) * sites + g] != 1) return err("a site-update computed twice"), finish(-1);
                const bool cut_top = k == k_hi;
                if ((en & sp::kLatExpPhi) || cut_top) {
                    const int par = g_plant == 1 ? 0 : tau & 1;
                    P[par][g] = out, tagP[par][g] = tau;
                    log.push_back({par * sites + g, (int32_t)id, tau, true, k + 1});
                }
                if ((en & sp::kLatExpPc) || cut_top) {
                    G[4 * g] = p.x, G[4 * g + 1] = p.y, G[4 * g + 2] = cc.x, G[4 * g + 3] = cc.y;
                    tagG[g] = tau;
                    log.push_back({2 * sites + g, (int32_t)id, tau, true, k + 1});
                }
            }
        }
    }
    for (size_t i = 0; i < computed.size(); ++i)
        if (computed[i] != 1) return err("a site-update never computed"), finish(-1);
    for (int64_t g = 0; g < sites; ++g)
        if (tagP[g_plant == 1 ? 0 : nsteps & 1][g] != nsteps || tagG[g] != nsteps) return err("final state incomplete"), finish(-1);

    // race check against the DAG: reachability from every region (bitsets)
    const int64_t words = (nreg + 63) / 64;
    std::vector<uint64_t> reach((size_t)(nreg * words), 0);  // reach[u] = descendants of u (strict)
    for (int64_t u = nreg - 1; u >= 0; --u) {
        const int L = c.layer(u);
        if (L + 1 >= c.Lmin + c.Lcount) continue;
        int a[3];
        sp::lat_centre(c.g, L, u % c.per_layer, a);
        for (int i = g_plant == 2 ? 1 : 0; i < 4; ++i) {
            int d[3], b[3];
            sp::lat_pred_shift(i, d);
            for (int k = 0; k < 3; ++k) b[k] = sp::lat_wrap(a[k] - d[k], 4 * c.g.M[k]);
            const int64_t v = (int64_t)(L + 1 - c.Lmin) * c.per_layer + sp::lat_index<int64_t>(c.g, b);
            // v's predecessor i must be u
            if (sp::lat_pred(c.g, L + 1, v % c.per_layer, i) != u % c.per_layer) return err("pred/succ mismatch"), finish(-1);
            reach[u * words + v / 64] |= 1ull << (v % 64);
            for (int64_t k = 0; k < words; ++k) reach[u * words + k] |= reach[v * words + k];
        }
    }
    auto before = [&](int64_t u, int64_t v) { return (reach[u * words + v / 64] >> (v % 64)) & 1; };
    std::sort(log.begin(), log.end(), [](const Access &x, const Access &y) {
        if (x.loc != y.loc) return x.loc < y.loc;
        if (x.tau != y.tau) return x.tau < y.tau;
        return x.write > y.write;  // the write of a level before its reads
    });
    int64_t nreads = 0, nwrites = 0;
    for (size_t i = 0; i < log.size();) {
        size_t j = i;
        while (j < log.size() && log[j].loc == log[i].loc) ++j;
        // writes of this location in level order: a chain of the DAG order
        std::vector<const Access *> wr;
        for (size_t k = i; k < j; ++k)
            if (log[k].write) wr.push_back(&log[k]);
        nwrites += (int64_t)wr.size();
        for (size_t k = 1; k < wr.size(); ++k) {
            const Access *x = wr[k - 1], *y = wr[k];
            if (x->tau == y->tau) return err("two writes of one level to one location"), finish(-1);
            if (!(x->region == y->region ? x->order < y->order : before(x->region, y->region)))
                return err("writes of one location not ordered by the DAG"), finish(-1);
        }
        for (size_t k = i; k < j; ++k) {
            if (log[k].write) continue;
            ++nreads;
            const Access &r = log[k];
            const Access *src = nullptr, *next = nullptr;
            for (const Access *x : wr) {
                if (x->tau == r.tau) src = x;
                if (x->tau > r.tau && !next) next = x;
            }
            if (r.tau > 0) {
                if (!src) return err("a read of a value nobody wrote"), finish(-1);
                if (src->region == r.region || !before(src->region, r.region))
                    return err("a read not preceded by its writer"), finish(-1);
            }
            if (next && !(next->region == r.region ? next->order > r.order : before(r.region, next->region)))
                return err("a write may overtake a read of the previous value"), finish(-1);
        }
        i = j;
    }

    std::memcpy(phi, P[g_plant == 1 ? 0 : nsteps & 1].data(), sites * 8);
    std::memcpy(pc, G.data(), sites * 16);
    if (stats) {
        stats[0] = nreg, stats[1] = nreads, stats[2] = nwrites, stats[3] = (int64_t)t.updates;
        int64_t br = 0, bw = 0;
        for (const Access &x : log) {
            const int64_t b = x.loc >= 2 * sites ? 16 : 8;
            (x.write ? bw : br) += b;
        }
        stats[4] = br, stats[5] = bw;
    }
    return finish(0);
}

void lx_plant(int which) { g_plant = which; }

// Layer numbering of a sequence of calls (layers[i] layers each): the first
// number of every call, as the reset kernel computes it.
void lx_epochs(const int *layers, int n, int *first)
{
    int last = 0;
    for (int i = 0; i < n; ++i) sp::lat_next_epoch(&last, layers[i], &first[i]);
}

// Table statistics of size s: updates, phi slots, footprint cells, imports
// (full, phi), exports (phi, (pi, c)), bytes read, bytes written, largest
// level, (pi, c) slots, halo cells.
int lx_stats(int s, int64_t *out)
{
    sp::LatticeTables t;
    if (!sp::build_lattice_tables(s, &t).empty()) return -1;
    out[0] = t.updates, out[1] = t.n_slots, out[2] = t.foot_cells, out[3] = t.imports_full, out[4] = t.imports_phi;
    out[5] = t.exports_phi, out[6] = t.exports_pc, out[7] = t.bytes_read, out[8] = t.bytes_written;
    out[9] = t.max_level_cells, out[10] = t.n_foot, out[11] = t.halo_cells;
    return 0;
}

// Cells of level k of one region (local offsets), for the geometry pins.
int lx_level(int s, int k, int32_t *xyz, int max)
{
    sp::LatticeTables t;
    if (!sp::build_lattice_tables(s, &t).empty() || k < 0 || k >= t.K) return -1;
    const int n = t.cell_n[k];
    for (int i = 0; i < n && i < max; ++i) {
        const uint32_t e = t.cell[t.cell_off[k] + i];
        t.offset_of(sp::lat_slot(e), sp::lat_row(e), &xyz[3 * i], &xyz[3 * i + 1], &xyz[3 * i + 2]);
    }
    return n;
}

}  // extern "C"
