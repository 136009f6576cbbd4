// region_exec.cpp -- TEST-ONLY CPU scaffold for the region planner.
//
// Compiled by the tests (never part of libsp.so).  It takes the planner's
// tables exactly as the GPU kernel does and
//   * checks on a concrete periodic grid that every (site, level) is computed
//     by exactly one region, that every read of a region is produced by one
//     of its predecessors, and that no write can overtake a read it would
//     clobber (main arrays and the mailboxes: a ring of two band slots, or
//     one slot for every band), by reachability in the dependency DAG the
//     kernel releases;
//   * executes the regions one at a time in a seeded random topological
//     order with the same FP32 site update, so the result can be compared bit
//     for bit with a whole-grid CPU sweep.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "planner.h"
#include "sp_update.h"

using sp::f2;

namespace {

struct Grid {
    int n[3], J[3], Jtot, B, H, P, nbands;
    int64_t sites() const { return (int64_t)n[0] * n[1] * n[2]; }
    int64_t regions() const { return (int64_t)nbands * 8 * Jtot; }
    int64_t id(int band, int S, const int j[3]) const
    {
        return ((int64_t)band * 8 + S) * Jtot + j[0] + J[0] * (j[1] + J[1] * j[2]);
    }
    void decode(int64_t t, int *band, int *S, int j[3]) const
    {
        *band = (int)(t / (8 * Jtot));
        int64_t r = t % (8 * Jtot);
        *S = (int)(r / Jtot);
        int jl = (int)(r % Jtot);
        j[0] = jl % J[0];
        j[1] = (jl / J[0]) % J[1];
        j[2] = jl / (J[0] * J[1]);
    }
    int64_t site(const int p[3]) const { return p[0] + (int64_t)n[0] * (p[1] + (int64_t)n[1] * p[2]); }
};

int wrap(int p, int n) { return ((p % n) + n) % n; }

// ---- study: transitive reduction of the region DAG's pattern ----
// A pattern edge runs from (b, S, j) to (b + dband, T, j + d); par is the
// parity of band b + 1 an inverted pyramid's next-band edge belongs to (-1:
// every band).  The reduction drops, one edge at a time, every edge whose
// endpoints stay connected through the edges still kept, on a window of
// three bands and positions |j_d| <= R (a window path is a path of every
// periodic grid, so the reduction never drops an edge it cannot replace),
// and for both band parities.  With g_reduced set the executor releases and
// counts by the reduced pattern (one mailbox slot only: its next-band edges
// are implied through the mailbox-reuse edges).
struct PEdge {
    int S, dband, T, d[3], par;
    bool on;
};
bool g_reduced = false;
std::vector<PEdge> g_pattern;
int g_pattern_B = 0;

constexpr int kWinR = 3, kWinW = 2 * kWinR + 1;
int win_id(int b, int S, int x, int y, int z) { return (((b * 8 + S) * kWinW + z + kWinR) * kWinW + y + kWinR) * kWinW + x + kWinR; }

bool win_reach(const std::vector<PEdge> &es, int q, const PEdge &target, int skip)
{
    std::vector<char> seen(3 * 8 * kWinW * kWinW * kWinW, 0);
    std::vector<int> stack = {win_id(0, target.S, 0, 0, 0)};
    seen[stack[0]] = 1;
    const int goal = win_id(target.dband, target.T, target.d[0], target.d[1], target.d[2]);
    while (!stack.empty()) {
        const int u = stack.back();
        stack.pop_back();
        if (u == goal) return true;
        const int x = u % kWinW - kWinR, y = u / kWinW % kWinW - kWinR, z = u / (kWinW * kWinW) % kWinW - kWinR;
        const int S = u / (kWinW * kWinW * kWinW) % 8, b = u / (kWinW * kWinW * kWinW * 8);
        for (size_t k = 0; k < es.size(); ++k) {
            const PEdge &e = es[k];
            if (!e.on || (int)k == skip || e.S != S || b + e.dband > 2) continue;
            if (e.par >= 0 && e.par != ((q + b) & 1)) continue;  // band b + 1 has parity q + b
            const int a = x + e.d[0], bb = y + e.d[1], c = z + e.d[2];
            if (a < -kWinR || a > kWinR || bb < -kWinR || bb > kWinR || c < -kWinR || c > kWinR) continue;
            const int v = win_id(b + e.dband, e.T, a, bb, c);
            if (!seen[v]) {
                seen[v] = 1;
                stack.push_back(v);
            }
        }
    }
    return false;
}

std::vector<PEdge> reduced_pattern(const sp::TileTables &t)
{
    std::vector<PEdge> es;
    for (int S = 0; S < 8; ++S)
        for (const sp::Succ &s : t.same_succ[S]) es.push_back({S, 0, s.type, {s.e[0], s.e[1], s.e[2]}, -1, true});
    for (int q = 0; q < 2; ++q)
        for (const sp::Succ &s : t.next_succ[q]) es.push_back({7, 1, s.type, {s.e[0], s.e[1], s.e[2]}, q, true});
    for (int S = 0; S < 8; ++S)
        for (const sp::Succ &s : t.reuse_succ[S]) es.push_back({S, 1, s.type, {s.e[0], s.e[1], s.e[2]}, -1, true});
    for (size_t k = 0; k < es.size(); ++k) {
        bool implied = true;
        for (int q = 0; q < 2 && implied; ++q)
            if (es[k].par < 0 || es[k].par == q) implied = win_reach(es, q, es[k], (int)k);
        if (implied) es[k].on = false;
    }
    std::vector<PEdge> kept;
    for (const PEdge &e : es)
        if (e.on) kept.push_back(e);
    return kept;
}

const std::vector<PEdge> &pattern_for(const sp::TileTables &t)
{
    if (g_pattern_B != t.B) {
        g_pattern = reduced_pattern(t);
        g_pattern_B = t.B;
    }
    return g_pattern;
}

// successors exactly as the kernel releases them; reuse: with the
// mailbox-reuse edges of a single mailbox slot
std::vector<int64_t> successors(const sp::TileTables &t, const Grid &g, int64_t r, bool reuse)
{
    int band, S, j[3];
    g.decode(r, &band, &S, j);
    std::vector<int64_t> out;
    if (g_reduced && reuse) {
        for (const PEdge &e : pattern_for(t)) {
            if (e.S != S || band + e.dband >= g.nbands) continue;
            if (e.par >= 0 && e.par != ((band + 1) & 1)) continue;
            int jc[3];
            for (int d = 0; d < 3; ++d) jc[d] = wrap(j[d] + e.d[d], g.J[d]);
            out.push_back(g.id(band + e.dband, e.T, jc));
        }
        return out;
    }
    for (const sp::Succ &s : t.same_succ[S]) {
        int jc[3];
        for (int d = 0; d < 3; ++d) jc[d] = wrap(j[d] + s.e[d], g.J[d]);
        out.push_back(g.id(band, s.type, jc));
    }
    if (S == 7 && band + 1 < g.nbands)
        for (const sp::Succ &s : t.next_succ[(band + 1) & 1]) {
            int jc[3];
            for (int d = 0; d < 3; ++d) jc[d] = wrap(j[d] + s.e[d], g.J[d]);
            out.push_back(g.id(band + 1, s.type, jc));
        }
    if (reuse && band + 1 < g.nbands)
        for (const sp::Succ &s : t.reuse_succ[S]) {
            int jc[3];
            for (int d = 0; d < 3; ++d) jc[d] = wrap(j[d] + s.e[d], g.J[d]);
            out.push_back(g.id(band + 1, s.type, jc));
        }
    return out;
}

int initial_count(const sp::TileTables &t, int band, int S, bool reuse)
{
    if (g_reduced && reuse) {
        int n = 0;
        for (const PEdge &e : pattern_for(t))
            if (e.T == S && (e.dband == 0 || (band > 0 && (e.par < 0 || e.par == (band & 1))))) ++n;
        return n;
    }
    int n = t.same_preds[S];
    if (band > 0) n += t.prev_preds[S] + (reuse ? t.reuse_preds[S] : 0);
    return n;
}

// global coordinate of local u along axis d
int gcoord(const Grid &g, int band, int S, const int j[3], int d, int u)
{
    int o = (band & 1) * g.H;
    return wrap(o + j[d] * g.B + u - (sp::inverted(S, d) ? g.H + 1 : 1), g.n[d]);
}

bool setup(int B, const int n[3], int nbands, Grid *g, sp::TileTables *t, std::string *err)
{
    *err = sp::build_tables(B, t);
    if (!err->empty()) return false;
    g->B = B;
    g->H = B / 2;
    g->P = B + 2;
    g->nbands = nbands;
    g->Jtot = 1;
    for (int d = 0; d < 3; ++d) {
        g->n[d] = n[d];
        if (n[d] % B || n[d] / B < 2) {
            *err = "grid side not a multiple of B with at least 2 regions";
            return false;
        }
        g->J[d] = n[d] / B;
        g->Jtot *= g->J[d];
    }
    return true;
}

// ---- octant executor: a region as eight octants (the cluster kernel's data
// flow), level by level, with the inner faces exchanged between octants
// before every level and everything else taken from the octant tables.
// Buffers start as NaN, so any read the tables do not provide shows up as a
// mismatch with the sweep. ----
int run_octants(const Grid &g, const sp::TileTables &t, int nsteps, uint64_t order_seed, const sp::LevelCoef *coef,
                const sp::PhysConst &q, f2 *F, f2 *V, f2 *K, char *msg, int msglen, int slots)
{
    auto fail = [&](const std::string &m) {
        std::snprintf(msg, msglen, "%s", m.c_str());
        return 0;
    };
    sp::OctTables o;
    std::string err = sp::build_octant_tables(t, &o);
    if (!err.empty()) return fail(err);
    const int B = g.B, H = g.H, P = o.P, PP = P * P;
    const int64_t R = g.regions();
    std::vector<std::vector<f2>> mbox(2);
    std::vector<int64_t> type_off(8);
    int64_t slot = 0;
    for (int S = 0; S < 8; ++S) {
        type_off[S] = slot;
        slot += (int64_t)g.Jtot * 8 * o.mb_size[S];
    }
    for (auto &m : mbox) m.assign(slot, f2{NAN, NAN});
    std::vector<int> count(R);
    std::vector<int64_t> ready;
    for (int64_t r = 0; r < R; ++r) {
        int band, S, j[3];
        g.decode(r, &band, &S, j);
        count[r] = initial_count(t, band, S, slots == 1);
        if (count[r] == 0) ready.push_back(r);
    }
    std::mt19937_64 rng(order_seed);
    struct Oct {
        std::vector<f2> buf[2], pis, cs;
    };
    std::vector<Oct> oc(8);
    for (auto &x : oc) {
        x.buf[0].resize(P * P * P);
        x.buf[1].resize(P * P * P);
        x.pis.resize(H * H * H);
        x.cs.resize(H * H * H);
    }
    int64_t done = 0;
    while (!ready.empty()) {
        size_t pick = (size_t)(rng() % ready.size());
        int64_t r = ready[pick];
        ready[pick] = ready.back();
        ready.pop_back();
        int band, S, j[3];
        g.decode(r, &band, &S, j);
        int C[3];
        for (int d = 0; d < 3; ++d) C[d] = (band & 1) * H + j[d] * B + (sp::inverted(S, d) ? 0 : H);
        auto gsite = [&](int oi, const int u[3]) {
            int p[3];
            for (int d = 0; d < 3; ++d) {
                const int dist = u[d] - 1;
                p[d] = wrap(C[d] + (((oi >> d) & 1) ? dist : -1 - dist), g.n[d]);
            }
            return g.site(p);
        };
        std::vector<f2> &mb = mbox[slots == 2 ? band & 1 : 0];
        const int jl = j[0] + g.J[0] * (j[1] + g.J[1] * j[2]);
        for (int oi = 0; oi < 8; ++oi) {
            Oct &x = oc[oi];
            for (auto *v : {&x.buf[0], &x.buf[1], &x.pis, &x.cs}) std::fill(v->begin(), v->end(), f2{NAN, NAN});
            const sp::Box3 &bp = o.base_phi[S], &bc = o.base_pc[S];
            for (int uz = bp.lo[2]; uz < bp.hi[2]; ++uz)
                for (int uy = bp.lo[1]; uy < bp.hi[1]; ++uy)
                    for (int ux = bp.lo[0]; ux < bp.hi[0]; ++ux) {
                        const int out = (ux < bc.lo[0] || ux >= bc.hi[0]) + (uy < bc.lo[1] || uy >= bc.hi[1]) +
                                        (uz < bc.lo[2] || uz >= bc.hi[2]);
                        if (out > 1) continue;
                        const int u[3] = {ux, uy, uz};
                        const int64_t s = gsite(oi, u);
                        x.buf[0][(uz * P + uy) * P + ux] = F[s];
                        if (out == 0) {
                            const int ci = ((uz - 1) * H + (uy - 1)) * H + (ux - 1);
                            x.pis[ci] = V[s];
                            x.cs[ci] = K[s];
                        }
                    }
            // every sloped-surface import lands at region start (the kernel: one level ahead)
            const int64_t self = type_off[S] + ((int64_t)jl * 8 + oi) * o.mb_size[S];
            for (int L = 1; L <= H - 1; ++L) {
                std::vector<f2> &dst = x.buf[L & 1];
                const int64_t base = self + o.mb_level_off[S][L];
                const int nf = o.imp_full_n[S][L], np = o.imp_phi_n[S][L];
                for (int i = 0; i < nf; ++i) {
                    const int e = o.imp_full[o.imp_full_off[S][L] + i];
                    x.pis[e >> 16] = mb[base + 2 * i];
                    x.cs[e >> 16] = mb[base + 2 * i + 1];
                    dst[e & 0xFFFF] = mb[base + 2 * nf + i];
                }
                for (int i = 0; i < np; ++i) dst[o.imp_phi[o.imp_phi_off[S][L] + i]] = mb[base + 3 * nf + i];
            }
        }
        for (int k = 1; k <= o.levels[S]; ++k) {
            const int *w = o.w[S][k];
            // inner faces of phi(k-1) (level 1: the band base brought them)
            if (k >= 2)
                for (int oi = 0; oi < 8; ++oi)
                    for (int d = 0; d < 3; ++d) {
                        if (w[d] == 0) continue;
                        const int a = (d + 1) % 3, b = (d + 2) % 3;
                        const std::vector<f2> &src = oc[oi].buf[(k - 1) & 1];
                        std::vector<f2> &dst = oc[oi ^ (1 << d)].buf[(k - 1) & 1];
                        for (int ib = 1; ib <= w[b]; ++ib)
                            for (int ia = 1; ia <= w[a]; ++ia) {
                                int us[3], ud[3];
                                us[d] = 1;
                                ud[d] = 0;
                                us[a] = ud[a] = ia;
                                us[b] = ud[b] = ib;
                                dst[(ud[2] * P + ud[1]) * P + ud[0]] = src[(us[2] * P + us[1]) * P + us[0]];
                            }
                    }
            for (int oi = 0; oi < 8; ++oi) {
                Oct &x = oc[oi];
                const std::vector<f2> &prev = x.buf[(k - 1) & 1];
                std::vector<f2> &cur = x.buf[k & 1];
                for (int uz = 1; uz <= w[2]; ++uz)
                    for (int uy = 1; uy <= w[1]; ++uy)
                        for (int ux = 1; ux <= w[0]; ++ux) {
                            const int pi_ = (uz * P + uy) * P + ux;
                            const int ci = ((uz - 1) * H + (uy - 1)) * H + (ux - 1);
                            cur[pi_] = sp::site_update(prev[pi_], prev[pi_ - 1], prev[pi_ + 1], prev[pi_ - P],
                                                       prev[pi_ + P], prev[pi_ - PP], prev[pi_ + PP], x.pis[ci],
                                                       x.cs[ci], coef[band * H + k - 1], q);
                        }
                if (k <= H - 1)
                    for (int i = 0; i < o.exp_n[S][k]; ++i) {
                        const sp::ExportEntry &e = o.exp[o.exp_off[S][k] + i];
                        const int Sc = e.code & 7, Gm = (e.code >> 3) & 7, Fm = Sc ^ S;
                        // one further along a flipped axis where the producer's octant bit equals G's
                        const int step = Fm & ~(oi ^ Gm) & 7;
                        int jc[3];
                        for (int d = 0; d < 3; ++d) jc[d] = wrap(j[d] + ((step >> d) & 1), g.J[d]);
                        const int oc_ = oi ^ Gm;
                        const int64_t dst = type_off[Sc] +
                                            ((int64_t)(jc[0] + g.J[0] * (jc[1] + g.J[1] * jc[2])) * 8 + oc_) *
                                                o.mb_size[Sc];
                        mb[dst + e.dst_phi] = cur[e.src & 0xFFFF];
                        if (e.dst_pc >= 0) {
                            mb[dst + e.dst_pc] = x.pis[(e.src >> 16) & 0xFFFF];
                            mb[dst + e.dst_pc + 1] = x.cs[(e.src >> 16) & 0xFFFF];
                        }
                    }
                if (k == H)
                    for (int uz = 1; uz <= H; ++uz)
                        for (int uy = 1; uy <= H; ++uy)
                            for (int ux = 1; ux <= H; ++ux) {
                                const int u[3] = {ux, uy, uz};
                                const int64_t s = gsite(oi, u);
                                const int ci = ((uz - 1) * H + (uy - 1)) * H + (ux - 1);
                                F[s] = cur[(uz * P + uy) * P + ux];
                                V[s] = x.pis[ci];
                                K[s] = x.cs[ci];
                            }
            }
        }
        for (int64_t s : successors(t, g, r, slots == 1))
            if (--count[s] == 0) ready.push_back(s);
        ++done;
    }
    if (done != R) return fail("not every region ran");
    return 1;
}

}  // namespace

extern "C" {

// Structural checks on a concrete grid.  Returns 0 and fills msg on failure.
// slots: 2 (ring of two band slots), 1 (one slot, with the reuse edges), or
// -1 (one slot without them: a DAG the hazard check must reject).
int rx_check(int B, int nx, int ny, int nz, int nbands, char *msg, int msglen, int slots)
{
    int n[3] = {nx, ny, nz};
    Grid g;
    sp::TileTables t;
    std::string err;
    auto fail = [&](const std::string &m) {
        std::snprintf(msg, msglen, "%s", m.c_str());
        return 0;
    };
    if (!setup(B, n, nbands, &g, &t, &err)) return fail(err);
    if (slots != 1 && slots != 2 && slots != -1) return fail("slots must be 2, 1 or -1");
    const bool reuse = slots == 1;
    if (slots < 0) slots = 1;
    const int64_t R = g.regions(), sites = g.sites();

    // 1) exact cover: every (site, level) computed by exactly one region
    for (int band = 0; band < nbands; ++band)
        for (int k = 1; k <= g.H; ++k) {
            std::vector<int> cover(sites, 0);
            for (int S = 0; S < 8; ++S)
                for (int jl = 0; jl < g.Jtot; ++jl) {
                    int j[3] = {jl % g.J[0], (jl / g.J[0]) % g.J[1], jl / (g.J[0] * g.J[1])};
                    if (k > t.levels[S]) continue;
                    const sp::Box3 &A = t.active[S][k];
                    for (int uz = A.lo[2]; uz < A.hi[2]; ++uz)
                        for (int uy = A.lo[1]; uy < A.hi[1]; ++uy)
                            for (int ux = A.lo[0]; ux < A.hi[0]; ++ux) {
                                int p[3] = {gcoord(g, band, S, j, 0, ux), gcoord(g, band, S, j, 1, uy),
                                            gcoord(g, band, S, j, 2, uz)};
                                cover[g.site(p)]++;
                            }
                }
            for (int64_t s = 0; s < sites; ++s)
                if (cover[s] != 1) return fail("level not covered exactly once");
        }

    // 2) DAG: counters match the number of releasing predecessors; acyclic
    std::vector<std::vector<int64_t>> succ(R);
    std::vector<int> indeg(R, 0);
    for (int64_t r = 0; r < R; ++r) {
        succ[r] = successors(t, g, r, reuse);
        for (int64_t s : succ[r]) indeg[s]++;
    }
    for (int64_t r = 0; r < R; ++r) {
        int band, S, j[3];
        g.decode(r, &band, &S, j);
        if (indeg[r] != initial_count(t, band, S, reuse)) return fail("predecessor count differs from releases");
    }
    // reachability (descendants) by DFS from each region
    std::vector<std::vector<uint8_t>> reach(R, std::vector<uint8_t>(R, 0));
    for (int64_t r = 0; r < R; ++r) {
        std::vector<int64_t> stack = succ[r];
        while (!stack.empty()) {
            int64_t x = stack.back();
            stack.pop_back();
            if (x == r) return fail("cycle in the region DAG");
            if (reach[r][x]) continue;
            reach[r][x] = 1;
            for (int64_t y : succ[x]) stack.push_back(y);
        }
    }

    // 3) main-array hazards: the base read at band b must come from the band b-1
    //    writer (a predecessor) and precede the band-b writer of the same site
    std::vector<std::vector<int64_t>> top_writer(nbands, std::vector<int64_t>(sites, -1));
    for (int band = 0; band < nbands; ++band)
        for (int jl = 0; jl < g.Jtot; ++jl) {
            int j[3] = {jl % g.J[0], (jl / g.J[0]) % g.J[1], jl / (g.J[0] * g.J[1])};
            for (int uz = 1; uz <= B; ++uz)
                for (int uy = 1; uy <= B; ++uy)
                    for (int ux = 1; ux <= B; ++ux) {
                        int p[3] = {gcoord(g, band, 7, j, 0, ux), gcoord(g, band, 7, j, 1, uy),
                                    gcoord(g, band, 7, j, 2, uz)};
                        if (top_writer[band][g.site(p)] != -1) return fail("two tops write one site");
                        top_writer[band][g.site(p)] = g.id(band, 7, j);
                    }
        }
    for (int64_t r = 0; r < R; ++r) {
        int band, S, j[3];
        g.decode(r, &band, &S, j);
        const sp::Box3 &bp = t.base_phi[S], &bc = t.base_pc[S];
        for (int uz = bp.lo[2]; uz < bp.hi[2]; ++uz)
            for (int uy = bp.lo[1]; uy < bp.hi[1]; ++uy)
                for (int ux = bp.lo[0]; ux < bp.hi[0]; ++ux) {
                    int out = (ux < bc.lo[0] || ux >= bc.hi[0]) + (uy < bc.lo[1] || uy >= bc.hi[1]) +
                              (uz < bc.lo[2] || uz >= bc.hi[2]);
                    if (out > 1) continue;
                    int p[3] = {gcoord(g, band, S, j, 0, ux), gcoord(g, band, S, j, 1, uy),
                                gcoord(g, band, S, j, 2, uz)};
                    int64_t s = g.site(p);
                    if (band > 0) {
                        int64_t w = top_writer[band - 1][s];
                        if (w < 0 || !reach[w][r]) return fail("base read not produced by a predecessor");
                    }
                    int64_t w2 = top_writer[band][s];
                    if (w2 < 0) return fail("site without a band top");
                    if (w2 != r && !reach[r][w2]) return fail("band top may overwrite an unread base");
                }
    }

    // 4) mailbox hazards: writer of a mailbox word is a predecessor of its
    //    reader; the writers of the next band that uses the same slot (two
    //    bands later with a ring of two, the next band with one slot) are
    //    its descendants
    for (int64_t r = 0; r < R; ++r) {
        int band, S, j[3];
        g.decode(r, &band, &S, j);
        for (int L = 1; L < g.H; ++L) {
            const int *beg = t.exp.empty() ? nullptr : nullptr;
            (void)beg;
            for (int i = 0; i < t.exp_n[S][L]; ++i) {
                const sp::ExportEntry &e = t.exp[t.exp_off[S][L] + i];
                int jc[3];
                for (int d = 0; d < 3; ++d) jc[d] = wrap(j[d] + ((e.code >> (3 + d)) & 1), g.J[d]);
                const int64_t consumer = g.id(band, e.code & 7, jc);
                if (!reach[r][consumer]) return fail("mailbox writer is not a predecessor of its reader");
                if (band >= slots) {
                    const int64_t old_reader = g.id(band - slots, e.code & 7, jc);
                    if (!reach[old_reader][r]) return fail("mailbox slot reused before its reader finished");
                }
            }
        }
    }
    // 5) every mailbox word that is read has exactly one writer per band
    for (int Sc = 1; Sc < 8; ++Sc) {
        std::vector<int> hits(t.mb_size[Sc], 0);
        for (int Sp = 0; Sp < 8; ++Sp)
            for (int L = 1; L < g.H; ++L)
                for (int i = 0; i < t.exp_n[Sp][L]; ++i) {
                    const sp::ExportEntry &e = t.exp[t.exp_off[Sp][L] + i];
                    if ((e.code & 7) != Sc) continue;
                    hits[e.dst_phi]++;
                    if (e.dst_pc >= 0) {
                        hits[e.dst_pc]++;
                        hits[e.dst_pc + 1]++;
                    }
                }
        int64_t used = 0;
        for (int L = 1; L < g.H; ++L) used += 3LL * t.imp_full_n[Sc][L] + t.imp_phi_n[Sc][L];
        int64_t written = 0;
        for (int v : hits) {
            if (v > 1) return fail("mailbox word written twice");
            written += v;
        }
        if (written != used) return fail("mailbox words read but never written");
    }
    return 1;
}

// Runs nsteps levels (a multiple of H) on FP32 state arrays (float2 as
// interleaved floats).  mode 0: whole-grid sweep; mode 1: regions in a random
// topological order drawn from order_seed.  coef holds one LevelCoef per level.
int rx_run(int B, int nx, int ny, int nz, int nsteps, int mode, uint64_t order_seed, const float *coef4,
           float dt, float inv_dx2, float eta2, float *phi, float *pi, float *c, char *msg, int msglen, int slots)
{
    int n[3] = {nx, ny, nz};
    Grid g;
    sp::TileTables t;
    std::string err;
    auto fail = [&](const std::string &m) {
        std::snprintf(msg, msglen, "%s", m.c_str());
        return 0;
    };
    if (nsteps % (B / 2)) return fail("nsteps must be a multiple of B/2");
    if (!setup(B, n, nsteps / (B / 2), &g, &t, &err)) return fail(err);
    if (slots != 1 && slots != 2) return fail("slots must be 1 or 2");
    const sp::LevelCoef *coef = reinterpret_cast<const sp::LevelCoef *>(coef4);
    sp::PhysConst q{dt, inv_dx2, eta2, 0.0f};
    f2 *F = reinterpret_cast<f2 *>(phi), *V = reinterpret_cast<f2 *>(pi), *K = reinterpret_cast<f2 *>(c);
    const int64_t sites = g.sites();

    if (mode == 0) {
        std::vector<f2> nxt(sites);
        for (int lvl = 0; lvl < nsteps; ++lvl) {
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y)
                    for (int x = 0; x < nx; ++x) {
                        int p[3] = {x, y, z};
                        auto at = [&](int dx, int dy, int dz) {
                            int r[3] = {wrap(x + dx, nx), wrap(y + dy, ny), wrap(z + dz, nz)};
                            return F[g.site(r)];
                        };
                        int64_t s = g.site(p);
                        nxt[s] = sp::site_update(F[s], at(-1, 0, 0), at(1, 0, 0), at(0, -1, 0), at(0, 1, 0),
                                                 at(0, 0, -1), at(0, 0, 1), V[s], K[s], coef[lvl], q);
                    }
            std::memcpy(F, nxt.data(), sites * sizeof(f2));
        }
        return 1;
    }

    if (mode == 2) return run_octants(g, t, nsteps, order_seed, coef, q, F, V, K, msg, msglen, slots);

    // ---- region executor: the kernel's data flow, one region at a time ----
    const int P = g.P, H = g.H;
    const int64_t R = g.regions();
    std::vector<std::vector<f2>> mbox(2);
    std::vector<int64_t> type_off(8);
    int64_t slot = 0;
    for (int S = 0; S < 8; ++S) {
        type_off[S] = slot;
        slot += (int64_t)g.Jtot * t.mb_size[S];
    }
    for (auto &m : mbox) m.assign(slot, f2{NAN, NAN});
    std::vector<int> count(R);
    std::vector<int64_t> ready;
    for (int64_t r = 0; r < R; ++r) {
        int band, S, j[3];
        g.decode(r, &band, &S, j);
        count[r] = initial_count(t, band, S, slots == 1);
        if (count[r] == 0) ready.push_back(r);
    }
    std::mt19937_64 rng(order_seed);
    std::vector<f2> buf0(P * P * P), buf1(P * P * P);
    std::vector<f2> pis(B * B * B), cs(B * B * B);
    int64_t done = 0;
    while (!ready.empty()) {
        size_t pick = (size_t)(rng() % ready.size());
        int64_t r = ready[pick];
        ready[pick] = ready.back();
        ready.pop_back();
        int band, S, j[3];
        g.decode(r, &band, &S, j);
        std::fill(buf0.begin(), buf0.end(), f2{NAN, NAN});
        std::fill(buf1.begin(), buf1.end(), f2{NAN, NAN});
        std::fill(pis.begin(), pis.end(), f2{NAN, NAN});
        std::fill(cs.begin(), cs.end(), f2{NAN, NAN});
        auto gsite = [&](int ux, int uy, int uz) {
            int p[3] = {gcoord(g, band, S, j, 0, ux), gcoord(g, band, S, j, 1, uy), gcoord(g, band, S, j, 2, uz)};
            return g.site(p);
        };
        // base
        const sp::Box3 &bp = t.base_phi[S], &bc = t.base_pc[S];
        for (int uz = bp.lo[2]; uz < bp.hi[2]; ++uz)
            for (int uy = bp.lo[1]; uy < bp.hi[1]; ++uy)
                for (int ux = bp.lo[0]; ux < bp.hi[0]; ++ux) {
                    int out = (ux < bc.lo[0] || ux >= bc.hi[0]) + (uy < bc.lo[1] || uy >= bc.hi[1]) +
                              (uz < bc.lo[2] || uz >= bc.hi[2]);
                    if (out > 1) continue;
                    int64_t s = gsite(ux, uy, uz);
                    buf0[(uz * P + uy) * P + ux] = F[s];
                    if (out == 0) {
                        int ci = ((uz - 1) * B + (uy - 1)) * B + (ux - 1);
                        pis[ci] = V[s];
                        cs[ci] = K[s];
                    }
                }
        std::vector<f2> &mb = mbox[slots == 2 ? band & 1 : 0];
        const int64_t self = type_off[S] + (int64_t)(j[0] + g.J[0] * (j[1] + g.J[1] * j[2])) * t.mb_size[S];
        // every sloped-surface import of every level lands at region start, as
        // in the kernel: level k goes to the level-k phi buffer (k & 1)
        if (S != 0)
            for (int k = 1; k <= H - 1; ++k) {
                std::vector<f2> &dst = (k & 1) ? buf1 : buf0;
                const int64_t base = self + t.mb_level_off[S][k];
                const int nf = t.imp_full_n[S][k], np = t.imp_phi_n[S][k];
                for (int i = 0; i < nf; ++i) {
                    int e = t.imp_full[t.imp_full_off[S][k] + i];
                    pis[e >> 16] = mb[base + 2 * i];
                    cs[e >> 16] = mb[base + 2 * i + 1];
                    dst[e & 0xFFFF] = mb[base + 2 * nf + i];
                }
                for (int i = 0; i < np; ++i) dst[t.imp_phi[t.imp_phi_off[S][k] + i]] = mb[base + 3 * nf + i];
            }
        for (int k = 1; k <= t.levels[S]; ++k) {
            std::vector<f2> &prev = (k & 1) ? buf0 : buf1;
            std::vector<f2> &cur = (k & 1) ? buf1 : buf0;
            const sp::Box3 &A = t.active[S][k];
            const int PP = P * P;
            for (int uz = A.lo[2]; uz < A.hi[2]; ++uz)
                for (int uy = A.lo[1]; uy < A.hi[1]; ++uy)
                    for (int ux = A.lo[0]; ux < A.hi[0]; ++ux) {
                        int pi_ = (uz * P + uy) * P + ux;
                        int ci = ((uz - 1) * B + (uy - 1)) * B + (ux - 1);
                        cur[pi_] = sp::site_update(prev[pi_], prev[pi_ - 1], prev[pi_ + 1], prev[pi_ - P],
                                                   prev[pi_ + P], prev[pi_ - PP], prev[pi_ + PP], pis[ci], cs[ci],
                                                   coef[band * H + k - 1], q);
                    }
            if (k <= H - 1)
                for (int i = 0; i < t.exp_n[S][k]; ++i) {
                    const sp::ExportEntry &e = t.exp[t.exp_off[S][k] + i];
                    int jc[3];
                    for (int d = 0; d < 3; ++d) jc[d] = wrap(j[d] + ((e.code >> (3 + d)) & 1), g.J[d]);
                    const int Sc = e.code & 7;
                    const int64_t dst = type_off[Sc] + (int64_t)(jc[0] + g.J[0] * (jc[1] + g.J[1] * jc[2])) *
                                                           t.mb_size[Sc];
                    mb[dst + e.dst_phi] = cur[e.src & 0xFFFF];
                    if (e.dst_pc >= 0) {
                        mb[dst + e.dst_pc] = pis[(e.src >> 16) & 0xFFFF];
                        mb[dst + e.dst_pc + 1] = cs[(e.src >> 16) & 0xFFFF];
                    }
                }
            if (k == H)
                for (int uz = 1; uz <= B; ++uz)
                    for (int uy = 1; uy <= B; ++uy)
                        for (int ux = 1; ux <= B; ++ux) {
                            int64_t s = gsite(ux, uy, uz);
                            int ci = ((uz - 1) * B + (uy - 1)) * B + (ux - 1);
                            F[s] = cur[(uz * P + uy) * P + ux];
                            V[s] = pis[ci];
                            K[s] = cs[ci];
                        }
        }
        for (int64_t s : successors(t, g, r, slots == 1))
            if (--count[s] == 0) ready.push_back(s);
        ++done;
    }
    if (done != R) return fail("not every region ran");
    return 1;
}

// Study switch: release and count by the transitively reduced pattern (one
// mailbox slot only).  Returns the number of pattern edges kept for base B
// and fills kept_by_source[8] (edges leaving each region type) and
// kept_kind[3] (same-band, next-band, mailbox-reuse).
int rx_reduced_dag(int B, int on, int *kept_by_source, int *kept_kind)
{
    sp::TileTables t;
    if (!sp::build_tables(B, &t).empty()) return -1;
    g_reduced = on != 0;
    const std::vector<PEdge> &p = pattern_for(t);
    for (int S = 0; S < 8; ++S) kept_by_source[S] = 0;
    for (int k = 0; k < 3; ++k) kept_kind[k] = 0;
    for (const PEdge &e : p) {
        kept_by_source[e.S]++;
        kept_kind[e.dband == 0 ? 0 : (e.par >= 0 ? 1 : 2)]++;
    }
    return (int)p.size();
}

// Same-band successor types of a type-S region (with repeats, one per edge):
// returns their number and writes up to max of them to types.
int rx_same_succ(int B, int S, int *types, int max)
{
    sp::TileTables t;
    if (!sp::build_tables(B, &t).empty() || S < 0 || S > 7) return -1;
    int n = 0;
    for (const sp::Succ &e : t.same_succ[S]) {
        if (n < max) types[n] = e.type;
        ++n;
    }
    return n;
}

// Mailbox-reuse edges per region type: successors n_succ[S] (and how many of
// them go to pyramids, to_pyramid[S]) and predecessors preds[S].
int rx_reuse(int B, int *n_succ, int *to_pyramid, int *preds)
{
    sp::TileTables t;
    if (!sp::build_tables(B, &t).empty()) return 0;
    for (int S = 0; S < 8; ++S) {
        n_succ[S] = (int)t.reuse_succ[S].size();
        to_pyramid[S] = 0;
        for (const sp::Succ &e : t.reuse_succ[S]) to_pyramid[S] += e.type == 0;
        preds[S] = t.reuse_preds[S];
    }
    return 1;
}

// Traffic per update of the design for base B (for the byte-count test).
double rx_bytes_per_update(int B, int64_t *read_per_band_cell, int64_t *write_per_band_cell, int64_t *upd)
{
    sp::TileTables t;
    if (!sp::build_tables(B, &t).empty()) return -1.0;
    int64_t r = 0, w = 0, u = 0;
    for (int S = 0; S < 8; ++S) {
        r += t.bytes_read[S];
        w += t.bytes_written[S];
        u += t.updates[S];
    }
    *read_per_band_cell = r;
    *write_per_band_cell = w;
    *upd = u;
    return (double)(r + w) / (double)u;
}

// Region types without same-band predecessors: their count if they are the
// leading types 0 .. m-1 (what the GPU queue reset seeds), else -1.
int rx_seed_types(int B)
{
    sp::TileTables t;
    if (!sp::build_tables(B, &t).empty()) return -2;
    int m = 0;
    while (m < 8 && t.same_preds[m] == 0) ++m;
    for (int S = m; S < 8; ++S)
        if (t.same_preds[S] == 0) return -1;
    return m;
}

// Active u-box of region type S at level k (lo[3], hi[3]) and its level count,
// for the shared-memory bank test; returns -1 for a bad base.
int rx_active_box(int B, int S, int k, int32_t *lohi)
{
    sp::TileTables t;
    if (!sp::build_tables(B, &t).empty()) return -1;
    for (int d = 0; d < 3; ++d) {
        lohi[d] = t.active[S][k].lo[d];
        lohi[3 + d] = t.active[S][k].hi[d];
    }
    return t.levels[S];
}

}  // extern "C"

// Sizes of the octant tables of base B: out = {full imports, phi-only
// imports, export entries, face imports, largest octant mailbox (float2),
// site-updates, bytes read, bytes written (per steady-state band cell)}.
extern "C" int rx_octant_stats(int B, int64_t *out)
{
    sp::TileTables t;
    if (!sp::build_tables(B, &t).empty()) return 0;
    sp::OctTables o;
    if (!sp::build_octant_tables(t, &o).empty()) return 0;
    int64_t mb = 0, upd = 0, rd = 0, wr = 0;
    for (int S = 0; S < 8; ++S) {
        mb = std::max<int64_t>(mb, o.mb_size[S]);
        upd += o.updates[S];
        rd += o.bytes_read[S];
        wr += o.bytes_written[S];
    }
    const int64_t v[8] = {(int64_t)o.imp_full.size(), (int64_t)o.imp_phi.size(), (int64_t)o.exp.size(),
                          (int64_t)o.face_imp.size(), mb, upd, rd, wr};
    for (int i = 0; i < 8; ++i) out[i] = v[i];
    return 1;
}
