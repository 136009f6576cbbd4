// planner.cpp -- builds the split-tiling tables (see planner.h).
//
// Everything here is derived by enumerating cells: for each region type and
// level, which cells it computes, which cells it must receive (its initial
// surfaces), who computes those, and where they go.  The kernel follows the
// resulting lists; no geometry is hand-coded on the device.
#include "planner.h"

#include <algorithm>
#include <array>
#include <map>
#include <set>
#include <sstream>
#include <tuple>

namespace sp {

static int floor_div(int a, int b)
{
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

bool owner_1d(int r, int L, int B, int *delta)
{
    // Inverted piece I_m covers [m B - L, m B + L) and upright U_m covers
    // [m B + L, m B + B - L) at level L (offsets from c_j).
    int m = floor_div(r + L, B);
    int rr = r - m * B;  // in [-L, B - L)
    *delta = m;
    return rr < L;
}

namespace {

inline bool in_active_1d(bool inv, int r, int k, int B)
{
    return inv ? (r >= -k && r < k) : (r >= k && r < B - k);
}

inline bool in_active(int S, const int r[3], int k, int B)
{
    if (k <= 0) return false;
    for (int d = 0; d < 3; ++d)
        if (!in_active_1d(inverted(S, d), r[d], k, B)) return false;
    return true;
}

// 7-point neighbour of A(k) but not in A(k)
inline bool in_ring(int S, const int r[3], int k, int B)
{
    if (in_active(S, r, k, B)) return false;
    for (int d = 0; d < 3; ++d)
        for (int s = -1; s <= 1; s += 2) {
            int q[3] = {r[0], r[1], r[2]};
            q[d] += s;
            if (in_active(S, q, k, B)) return true;
        }
    return false;
}

inline int u_of(int S, int d, int r, int H) { return r + (inverted(S, d) ? H + 1 : 1); }

struct Idx {
    int phi, pc;
};

inline Idx index_of(int S, const int r[3], int B)
{
    int H = B / 2, P = B + 2;
    int u[3];
    for (int d = 0; d < 3; ++d) u[d] = u_of(S, d, r[d], H);
    Idx x;
    x.phi = (u[2] * P + u[1]) * P + u[0];
    bool own = true;
    for (int d = 0; d < 3; ++d) own = own && u[d] >= 1 && u[d] <= B;
    x.pc = own ? ((u[2] - 1) * B + (u[1] - 1)) * B + (u[0] - 1) : -1;
    return x;
}

inline bool in_u_box(int S, const int r[3], int B)
{
    int H = B / 2, P = B + 2;
    for (int d = 0; d < 3; ++d) {
        int u = u_of(S, d, r[d], H);
        if (u < 0 || u >= P) return false;
    }
    return true;
}

// Region DAG of two consecutive bands on a non-periodic window of positions
// |j_d| <= R around the origin: same-band edges, the inverted pyramids'
// next-band edges (next band of parity q) and the given mailbox-reuse edges
// (reuse[S] = (type, offset) list, one flag per entry).  Paths of the window
// are paths of every periodic grid, so a pair found ordered here is ordered
// there too; a pair the window misses is merely kept as an explicit edge.
struct BandPairDag {
    static constexpr int R = 3, W = 2 * R + 1;
    const TileTables &t;
    explicit BandPairDag(const TileTables &tt) : t(tt) {}
    static int id(int band, int S, int x, int y, int z) { return (((band * kTypes + S) * W + z + R) * W + y + R) * W + x + R; }
    // is (1, Sp, d) reachable from (0, S, 0), without pattern edge `skip`?
    bool ordered(int q, const std::vector<std::vector<char>> &on, int S, const Succ &to, int skip_S, int skip_i) const
    {
        std::vector<char> seen(2 * kTypes * W * W * W, 0);
        std::vector<int> stack = {id(0, S, 0, 0, 0)};
        seen[stack[0]] = 1;
        const int target = id(1, to.type, to.e[0], to.e[1], to.e[2]);
        auto push = [&](int band, int type, int x, int y, int z) {
            if (x < -R || x > R || y < -R || y > R || z < -R || z > R) return;
            const int v = id(band, type, x, y, z);
            if (!seen[v]) {
                seen[v] = 1;
                stack.push_back(v);
            }
        };
        while (!stack.empty()) {
            const int u = stack.back();
            stack.pop_back();
            if (u == target) return true;
            const int x = u % W - R, y = u / W % W - R, z = u / (W * W) % W - R;
            const int type = u / (W * W * W) % kTypes, band = u / (W * W * W * kTypes);
            for (const Succ &e : t.same_succ[type]) push(band, e.type, x + e.e[0], y + e.e[1], z + e.e[2]);
            if (band == 1) continue;
            if (type == kTypes - 1)
                for (const Succ &e : t.next_succ[q]) push(1, e.type, x + e.e[0], y + e.e[1], z + e.e[2]);
            for (size_t i = 0; i < t.reuse_succ[type].size(); ++i)
                if (on[type][i] && !(type == skip_S && (int)i == skip_i)) {
                    const Succ &e = t.reuse_succ[type][i];
                    push(1, e.type, x + e.e[0], y + e.e[1], z + e.e[2]);
                }
        }
        return false;
    }
};

// Drops the mailbox-reuse edges that the rest of the DAG already implies, for
// both parities of the next band: greedily, edges towards later-phase types
// first, each removal checked on the DAG as it stands, and the end result
// checked against every original pair (if that fails, nothing is dropped).
// From base 6 on, eight edges remain per band position: from the inverted
// pyramid of band b to the pyramids of band b+1 that do not build on its top,
// since every writer of band b+1 comes after those pyramids.
void prune_reuse(TileTables &t)
{
    BandPairDag dag(t);
    std::vector<std::vector<char>> on(kTypes);
    std::vector<std::pair<int, int>> order;
    for (int S = 0; S < kTypes; ++S) {
        on[S].assign(t.reuse_succ[S].size(), 1);
        for (size_t i = 0; i < t.reuse_succ[S].size(); ++i) order.push_back({S, (int)i});
    }
    std::stable_sort(order.begin(), order.end(), [&](const std::pair<int, int> &a, const std::pair<int, int> &b) {
        return __builtin_popcount(t.reuse_succ[a.first][a.second].type) >
               __builtin_popcount(t.reuse_succ[b.first][b.second].type);
    });
    for (const auto &o : order) {
        const Succ &e = t.reuse_succ[o.first][o.second];
        if (dag.ordered(0, on, o.first, e, o.first, o.second) && dag.ordered(1, on, o.first, e, o.first, o.second))
            on[o.first][o.second] = 0;
    }
    for (int S = 0; S < kTypes; ++S)
        for (const Succ &e : t.reuse_succ[S])
            for (int q = 0; q < 2; ++q)
                if (!dag.ordered(q, on, S, e, -1, -1)) return;  // keep every edge
    for (int S = 0; S < kTypes; ++S) {
        std::vector<Succ> kept;
        for (size_t i = 0; i < t.reuse_succ[S].size(); ++i)
            if (on[S][i]) kept.push_back(t.reuse_succ[S][i]);
        t.reuse_succ[S] = kept;
    }
}

}  // namespace

std::string build_tables(int B, TileTables *tp)
{
    TileTables &t = *tp;
    t = TileTables();
    if (B % 2 != 0 || B < 4 || B > kMaxB) return "base size B must be even and in [4, 32]";
    const int H = B / 2, P = B + 2;
    t.B = B;
    t.H = H;
    t.P = P;
    const int rlo = -H - 2, rhi = B + 2;  // enumeration range of offsets per axis

    for (int S = 0; S < kTypes; ++S) {
        t.levels[S] = (S == kTypes - 1) ? H : H - 1;
        for (int k = 0; k <= kMaxH; ++k)
            for (int d = 0; d < 3; ++d) {
                int lo, hi;
                if (k == 0 || k > H) {
                    lo = hi = 1;
                } else if (inverted(S, d)) {
                    lo = H - k + 1;
                    hi = H + k + 1;
                } else {
                    lo = k + 1;
                    hi = B - k + 1;
                }
                t.active[S][k].lo[d] = lo;
                t.active[S][k].hi[d] = hi;
            }
        for (int d = 0; d < 3; ++d) {
            bool inv = inverted(S, d);
            // phi: A(1) grown by one cell; pc: A(1)
            t.base_phi[S].lo[d] = inv ? H - 1 : 1;
            t.base_phi[S].hi[d] = inv ? H + 3 : B + 1;
            t.base_pc[S].lo[d] = inv ? H : 2;
            t.base_pc[S].hi[d] = inv ? H + 2 : B;
        }
    }

    // ---- sloped initial surfaces: imports per (consumer type, level) ----
    struct Exp {
        int producer, L;
        ExportEntry e;
    };
    std::vector<Exp> exports;
    std::set<std::tuple<int, int, int, int>> preds[kTypes];       // (S', dx, dy, dz)
    std::set<std::tuple<int, int, int, int>> succs[kTypes];       // (S, ex, ey, ez)
    int64_t imp_bytes[kTypes] = {0};
    for (int S = 0; S < kTypes; ++S) {
        int32_t off = 0;
        for (int L = 0; L < kMaxH; ++L) {
            t.imp_full_off[S][L] = (int32_t)t.imp_full.size();
            t.imp_phi_off[S][L] = (int32_t)t.imp_phi.size();
            t.imp_full_n[S][L] = t.imp_phi_n[S][L] = 0;
            t.mb_level_off[S][L] = off;
            if (L < 1 || L > H - 1) continue;
            std::vector<std::array<int, 3>> full, ring;
            for (int z = rlo; z < rhi; ++z)
                for (int y = rlo; y < rhi; ++y)
                    for (int x = rlo; x < rhi; ++x) {
                        int r[3] = {x, y, z};
                        if (in_active(S, r, L, B)) continue;
                        if (in_active(S, r, L + 1, B))
                            full.push_back({x, y, z});
                        else if (in_ring(S, r, L + 1, B))
                            ring.push_back({x, y, z});
                    }
            const int nf = (int)full.size(), np = (int)ring.size();
            t.imp_full_n[S][L] = nf;
            t.imp_phi_n[S][L] = np;
            imp_bytes[S] += 24LL * nf + 8LL * np;
            for (int kind = 0; kind < 2; ++kind) {
                const auto &cells = kind == 0 ? full : ring;
                for (int i = 0; i < (int)cells.size(); ++i) {
                    int r[3] = {cells[i][0], cells[i][1], cells[i][2]};
                    if (!in_u_box(S, r, B)) return "import cell outside the region's shared-memory box";
                    Idx ix = index_of(S, r, B);
                    if (kind == 0) {
                        if (ix.pc < 0) return "full-state import is not one of the region's own cells";
                        t.imp_full.push_back(ix.phi | (ix.pc << 16));
                    } else {
                        t.imp_phi.push_back(ix.phi);
                    }
                    // owner at level L in the same band
                    int Sp = 0, delta[3], rp[3];
                    for (int d = 0; d < 3; ++d) {
                        bool inv = owner_1d(r[d], L, B, &delta[d]);
                        if (inv) Sp |= 1 << d;
                        if (delta[d] < -1 || delta[d] > 0) return "import owner is not an adjacent region";
                        if (!inverted(S, d) && (inv || delta[d] != 0))
                            return "import along an upright axis comes from another region";
                        rp[d] = r[d] - delta[d] * B;
                    }
                    if ((Sp & ~S) != 0 || Sp == S) return "import owner type is not a proper subset";
                    if (!in_active(Sp, rp, L, B)) return "import owner does not compute the cell";
                    // the producer exports level L while it computes level L + 1, which
                    // rewrites (pi, c) of A(L + 1): a full-state export must lie outside it
                    if (kind == 0 && in_active(Sp, rp, L + 1, B))
                        return "full-state export cell is recomputed by the next level";
                    Idx px = index_of(Sp, rp, B);
                    if (px.pc < 0) return "producer cell outside its own box";
                    int ebits = 0;
                    for (int d = 0; d < 3; ++d)
                        if (delta[d] == -1) ebits |= 1 << d;
                    ExportEntry e;
                    e.src = px.phi | ((kind == 0 ? px.pc : 0xFFFF) << 16);
                    e.code = S | (ebits << 3);
                    e.dst_phi = kind == 0 ? off + 2 * nf + i : off + 3 * nf + i;
                    e.dst_pc = kind == 0 ? off + 2 * i : -1;
                    exports.push_back({Sp, L, e});
                    preds[S].insert({Sp, delta[0], delta[1], delta[2]});
                    succs[Sp].insert({S, -delta[0], -delta[1], -delta[2]});
                }
            }
            off += 3 * nf + np;
            off += off & 1;  // keep every chunk 16-byte aligned
        }
        t.mb_size[S] = off;
    }

    // ---- final surfaces: export lists per (producer type, level) ----
    std::stable_sort(exports.begin(), exports.end(), [](const Exp &a, const Exp &b) {
        if (a.producer != b.producer) return a.producer < b.producer;
        if (a.L != b.L) return a.L < b.L;
        if (a.e.code != b.e.code) return a.e.code < b.e.code;
        return a.e.dst_phi < b.e.dst_phi;
    });
    int64_t exp_bytes[kTypes] = {0};
    {
        size_t i = 0;
        for (int S = 0; S < kTypes; ++S)
            for (int L = 0; L < kMaxH; ++L) {
                t.exp_off[S][L] = (int32_t)t.exp.size();
                while (i < exports.size() && exports[i].producer == S && exports[i].L == L) {
                    t.exp.push_back(exports[i].e);
                    exp_bytes[S] += exports[i].e.dst_pc >= 0 ? 24 : 8;
                    ++i;
                }
                t.exp_n[S][L] = (int32_t)t.exp.size() - t.exp_off[S][L];
            }
        if (i != exports.size()) return "export bookkeeping mismatch";
    }

    // ---- band base: previous band's inverted-pyramid tops ----
    std::set<std::tuple<int, int, int, int>> nsucc[2];
    for (int S = 0; S < kTypes; ++S) {
        int64_t base_cells = 0;
        std::set<std::tuple<int, int, int>> own[2];
        for (int z = rlo; z < rhi; ++z)
            for (int y = rlo; y < rhi; ++y)
                for (int x = rlo; x < rhi; ++x) {
                    int r[3] = {x, y, z};
                    if (!in_active(S, r, 1, B) && !in_ring(S, r, 1, B)) continue;
                    ++base_cells;
                    for (int d = 0; d < 3; ++d) {
                        int u = u_of(S, d, r[d], H);
                        if (u < t.base_phi[S].lo[d] || u >= t.base_phi[S].hi[d]) return "base cell outside base box";
                    }
                    for (int q = 0; q < 2; ++q) {
                        // owner index offset i - j of T(xyz) in band b-1, band b offset parity q
                        int o[3];
                        for (int d = 0; d < 3; ++d) o[d] = q + floor_div(r[d], B);
                        own[q].insert({o[0], o[1], o[2]});
                        nsucc[q].insert({S, -o[0], -o[1], -o[2]});
                    }
                }
        if (own[0].size() != own[1].size()) return "previous-band predecessor count depends on parity";
        t.prev_preds[S] = (int32_t)own[0].size();
        t.same_preds[S] = (int32_t)preds[S].size();
        int expect_same = 1;
        for (int d = 0; d < 3; ++d) expect_same *= inverted(S, d) ? 3 : 1;
        if (t.same_preds[S] > expect_same - 1) return "more same-band predecessors than 3^|S| - 1";
        if (t.prev_preds[S] != (1 << __builtin_popcount(S))) return "previous-band predecessor count is not 2^|S|";
        for (auto &s : preds[S]) {
            Succ x;
            x.type = (int8_t)std::get<0>(s);
            x.e[0] = (int8_t)std::get<1>(s);
            x.e[1] = (int8_t)std::get<2>(s);
            x.e[2] = (int8_t)std::get<3>(s);
            t.reuse_succ[S].push_back(x);
        }
        for (auto &s : succs[S]) {
            Succ x;
            x.type = (int8_t)std::get<0>(s);
            x.e[0] = (int8_t)std::get<1>(s);
            x.e[1] = (int8_t)std::get<2>(s);
            x.e[2] = (int8_t)std::get<3>(s);
            t.same_succ[S].push_back(x);
        }
        t.updates[S] = 0;
        for (int k = 1; k <= t.levels[S]; ++k) t.updates[S] += t.active[S][k].volume();
        t.bytes_read[S] = 8 * base_cells + 16 * t.active[S][1].volume() + imp_bytes[S];
        t.bytes_written[S] = exp_bytes[S] + (S == kTypes - 1 ? 24LL * B * B * B : 0);
    }
    for (int q = 0; q < 2; ++q)
        for (auto &s : nsucc[q]) {
            Succ x;
            x.type = (int8_t)std::get<0>(s);
            x.e[0] = (int8_t)std::get<1>(s);
            x.e[1] = (int8_t)std::get<2>(s);
            x.e[2] = (int8_t)std::get<3>(s);
            t.next_succ[q].push_back(x);
        }
    if (t.same_succ[kTypes - 1].size() != 0) return "inverted pyramid has same-band successors";
    if ((int)t.next_succ[0].size() != kMaxNextSucc || (int)t.next_succ[1].size() != kMaxNextSucc)
        return "inverted pyramid does not have 27 next-band successors";
    for (int S = 0; S < kTypes; ++S)
        if ((int)t.same_succ[S].size() > kMaxSameSucc) return "too many same-band successors";
    // every same-band edge Sp -> S, mirrored one band later, is one reuse edge S -> Sp
    for (int Sp = 0; Sp < kTypes; ++Sp) {
        int n = 0;
        for (int S = 0; S < kTypes; ++S)
            for (const Succ &x : t.reuse_succ[S]) n += x.type == Sp;
        if (n != (int)t.same_succ[Sp].size()) return "mailbox-reuse edges do not mirror the same-band edges";
    }
    prune_reuse(t);
    for (int Sp = 0; Sp < kTypes; ++Sp) {
        t.reuse_preds[Sp] = 0;
        for (int S = 0; S < kTypes; ++S)
            for (const Succ &x : t.reuse_succ[S]) t.reuse_preds[Sp] += x.type == Sp;
    }

    // ---- exact cover of one period cell at every level ----
    for (int k = 1; k <= H; ++k) {
        int64_t v = 0;
        for (int S = 0; S < kTypes; ++S) v += t.active[S][k].volume();
        if (v != (int64_t)B * B * B) return "regions do not tile the period cell at some level";
    }

    // ---- the GPU kernel's copy schedule: the sloped surface of level L lands
    // (phi in buffer L & 1, (pi, c) in the region's array) while level L-1 is
    // computed and the final surface of level L-2 is exported, both from
    // that buffer; it must touch nothing they read or write ----
    auto in_box = [](const Box3 &b, int x, int y, int z) {
        return x >= b.lo[0] && x < b.hi[0] && y >= b.lo[1] && y < b.hi[1] && z >= b.lo[2] && z < b.hi[2];
    };
    for (int S = 0; S < kTypes; ++S)
        for (int L = 1; L <= H - 1; ++L) {
            const Box3 *A = t.active[S];
            auto phi_ok = [&](int q) {
                const int x = q % t.P, y = (q / t.P) % t.P, z = q / (t.P * t.P);
                if (L - 2 >= 1 && in_box(A[L - 2], x, y, z)) return false;  // written by L-2, exported after L-1
                if (L - 1 >= 1) {  // read by the 7-point stencil of level L-1
                    const int nb[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
                    for (const auto &o : nb)
                        if (in_box(A[L - 1], x + o[0], y + o[1], z + o[2])) return false;
                }
                return true;
            };
            for (int i = 0; i < t.imp_phi_n[S][L]; ++i)
                if (!phi_ok(t.imp_phi[t.imp_phi_off[S][L] + i])) return "a sloped-surface copy overtakes a level in flight";
            for (int i = 0; i < t.imp_full_n[S][L]; ++i) {
                const int e = t.imp_full[t.imp_full_off[S][L] + i];
                if (!phi_ok(e & 0xFFFF)) return "a sloped-surface copy overtakes a level in flight";
                const int c = e >> 16, x = c % B + 1, y = (c / B) % B + 1, z = c / (B * B) + 1;
                for (int k = std::max(1, L - 2); k <= L; ++k)
                    if (in_box(A[k], x, y, z)) return "a (pi, c) copy overtakes a level in flight";
            }
        }
    return std::string();
}

// ---------------------------------------------------------------- octants
namespace {

// offset from c_j of the cell at octant distance dist (upper octant) of a
// region of type S along axis d
inline int xrel_of(int S, int d, int dist, int H) { return dist + (inverted(S, d) ? 0 : H); }

// the octant's cells at level k: dist < w along every axis
inline int oct_width(int S, int d, int k, int H, int levels)
{
    if (k < 1 || k > levels) return 0;
    return inverted(S, d) ? k : H - k;
}

}  // namespace

std::string build_octant_tables(const TileTables &t, OctTables *op)
{
    OctTables &o = *op;
    o = OctTables();
    const int B = t.B, H = t.H, P = H + 2;
    if (B < 8 || B > kMaxB || B % 4 != 0) return "octant tables need B a multiple of 4 in [8, 32]";
    o.B = B;
    o.H = H;
    o.P = P;
    auto phi_index = [&](const int u[3]) { return (u[2] * P + u[1]) * P + u[0]; };
    auto pc_index = [&](const int dist[3]) { return (dist[2] * H + dist[1]) * H + dist[0]; };
    for (int S = 0; S < kTypes; ++S) {
        o.levels[S] = t.levels[S];
        for (int k = 0; k <= kMaxH + 1; ++k)
            for (int d = 0; d < 3; ++d) {
                const int w = oct_width(S, d, k, H, o.levels[S]);
                o.w[S][k][d] = w;
                o.active[S][k].lo[d] = 1;
                o.active[S][k].hi[d] = 1 + w;
            }
        for (int d = 0; d < 3; ++d) {
            const int w1 = o.w[S][1][d];
            o.base_phi[S].lo[d] = 0;        // the inner halo comes from the band base too
            o.base_phi[S].hi[d] = w1 + 2;
            o.base_pc[S].lo[d] = 1;
            o.base_pc[S].hi[d] = w1 + 1;
        }
        // the octant boxes are the region's active sets cut at the centre
        for (int k = 1; k <= o.levels[S]; ++k) {
            int64_t v = 1;
            for (int d = 0; d < 3; ++d) v *= o.w[S][k][d];
            if (8 * v != t.active[S][k].volume()) return "octant boxes do not split the region's level";
        }
    }

    struct Exp {
        int producer, L;
        ExportEntry e;
    };
    std::vector<Exp> exports;
    int64_t imp_bytes[kTypes] = {0};
    for (int S = 0; S < kTypes; ++S) {
        int32_t off = 0;
        for (int L = 0; L < kMaxH; ++L) {
            o.imp_full_off[S][L] = (int32_t)o.imp_full.size();
            o.imp_phi_off[S][L] = (int32_t)o.imp_phi.size();
            o.face_imp_off[S][L] = (int32_t)o.face_imp.size();
            o.imp_full_n[S][L] = o.imp_phi_n[S][L] = o.face_imp_n[S][L] = 0;
            o.mb_level_off[S][L] = off;
            if (L < 1 || L > H - 1) continue;
            std::vector<std::array<int, 3>> full, ring;
            for (int z = 0; z <= H; ++z)
                for (int y = 0; y <= H; ++y)
                    for (int x = 0; x <= H; ++x) {
                        const int dist[3] = {x, y, z};
                        int r[3];
                        for (int d = 0; d < 3; ++d) r[d] = xrel_of(S, d, dist[d], H);
                        if (in_active(S, r, L, B)) continue;
                        if (in_active(S, r, L + 1, B))
                            full.push_back({x, y, z});
                        else if (in_ring(S, r, L + 1, B))
                            ring.push_back({x, y, z});
                    }
            const int nf = (int)full.size(), np = (int)ring.size();
            o.imp_full_n[S][L] = nf;
            o.imp_phi_n[S][L] = np;
            imp_bytes[S] += 8 * (24LL * nf + 8LL * np);
            for (int kind = 0; kind < 2; ++kind) {
                const auto &cells = kind == 0 ? full : ring;
                for (int i = 0; i < (int)cells.size(); ++i) {
                    const int dist[3] = {cells[i][0], cells[i][1], cells[i][2]};
                    int u[3], r[3];
                    for (int d = 0; d < 3; ++d) {
                        u[d] = dist[d] + 1;
                        r[d] = xrel_of(S, d, dist[d], H);
                        if (u[d] >= P) return "octant import outside the octant's buffer";
                    }
                    if (kind == 0) {
                        for (int d = 0; d < 3; ++d)
                            if (dist[d] >= H) return "octant full import is not an octant cell";
                        o.imp_full.push_back(phi_index(u) | (pc_index(dist) << 16));
                        int mask = 0;
                        for (int d = 0; d < 3; ++d)
                            if (dist[d] == 0) mask |= 1 << d;
                        if (mask) o.face_imp.push_back(phi_index(u) | (mask << 16));
                    } else {
                        o.imp_phi.push_back(phi_index(u));
                    }
                    // the producer: owner at level L in the same band
                    int Sp = 0, delta[3], dp[3], gmask = 0;
                    for (int d = 0; d < 3; ++d) {
                        const bool inv = owner_1d(r[d], L, B, &delta[d]);
                        if (inv) Sp |= 1 << d;
                        const int rp = r[d] - delta[d] * B - (inv ? 0 : H);  // from the producer's centre
                        const int op_d = rp >= 0;
                        dp[d] = op_d ? rp : -1 - rp;
                        const bool flip = inverted(S, d) != inv;
                        // the consumer is the upper octant at position 0: every producer sits at
                        // position 0 too; along an axis of the same type it is the same octant,
                        // along a flipped one either (the outer halo of the last level comes
                        // from the upright neighbour's upper half, the rest from its lower one)
                        if (delta[d] != 0 || (!flip && op_d != 1))
                            return "octant import from an unexpected producer octant";
                        gmask |= (op_d ? 0 : 1) << d;
                        if (dp[d] < 0 || dp[d] >= H) return "octant producer cell outside its octant";
                    }
                    if ((Sp & ~S) != 0 || Sp == S) return "octant import owner type is not a proper subset";
                    int rpx[3];
                    for (int d = 0; d < 3; ++d) rpx[d] = r[d] - delta[d] * B;
                    if (!in_active(Sp, rpx, L, B)) return "octant import owner does not compute the cell";
                    if (kind == 0 && in_active(Sp, rpx, L + 1, B))
                        return "octant full-state export cell is recomputed by the next level";
                    int up[3];
                    for (int d = 0; d < 3; ++d) up[d] = dp[d] + 1;
                    ExportEntry e;
                    e.src = phi_index(up) | ((kind == 0 ? pc_index(dp) : 0xFFFF) << 16);
                    e.code = S | (gmask << 3);
                    e.dst_phi = kind == 0 ? off + 2 * nf + i : off + 3 * nf + i;
                    e.dst_pc = kind == 0 ? off + 2 * i : -1;
                    exports.push_back({Sp, L, e});
                }
            }
            o.face_imp_n[S][L] = (int32_t)o.face_imp.size() - o.face_imp_off[S][L];
            off += 3 * nf + np;
            off += off & 1;  // every chunk 16-byte aligned
        }
        o.mb_size[S] = off;
    }
    std::stable_sort(exports.begin(), exports.end(), [](const Exp &a, const Exp &b) {
        if (a.producer != b.producer) return a.producer < b.producer;
        if (a.L != b.L) return a.L < b.L;
        if (a.e.code != b.e.code) return a.e.code < b.e.code;
        return a.e.dst_phi < b.e.dst_phi;
    });
    int64_t exp_bytes[kTypes] = {0};
    {
        size_t i = 0;
        for (int S = 0; S < kTypes; ++S)
            for (int L = 0; L < kMaxH; ++L) {
                o.exp_off[S][L] = (int32_t)o.exp.size();
                while (i < exports.size() && exports[i].producer == S && exports[i].L == L) {
                    o.exp.push_back(exports[i].e);
                    exp_bytes[S] += 8 * (exports[i].e.dst_pc >= 0 ? 24 : 8);
                    ++i;
                }
                o.exp_n[S][L] = (int32_t)o.exp.size() - o.exp_off[S][L];
            }
        if (i != exports.size()) return "octant export bookkeeping mismatch";
    }

    // ---- inner-face exchange: before level L+1 every octant needs phi(L) on
    // the neighbour's dist = 0 face inside the level-(L+1) box along the other
    // axes; the neighbour holds it as a level-L cell or a level-L import ----
    for (int S = 0; S < kTypes; ++S)
        for (int L = 1; L < o.levels[S]; ++L)
            for (int d = 0; d < 3; ++d) {
                const int *w1 = o.w[S][L + 1], *w0 = o.w[S][L];
                if (w1[d] == 0) continue;
                const int a = (d + 1) % 3, b = (d + 2) % 3;
                int64_t want = (int64_t)w1[a] * w1[b], computed = 0, imported = 0;
                for (int ib = 0; ib < w1[b]; ++ib)
                    for (int ia = 0; ia < w1[a]; ++ia)
                        if (ia < w0[a] && ib < w0[b] && w0[d] > 0) ++computed;
                for (int i = 0; i < o.face_imp_n[S][L]; ++i)
                    if ((o.face_imp[o.face_imp_off[S][L] + i] >> 16) & (1 << d)) ++imported;
                if (computed + imported != want) return "inner-face exchange does not cover the neighbour's needs";
            }

    // ---- the kernel's copy schedule, as for whole regions: level L's sloped
    // surface lands one level ahead; it must touch nothing levels L-2 and L-1
    // read or write ----
    auto in_box = [](const Box3 &bx, int x, int y, int z) {
        return x >= bx.lo[0] && x < bx.hi[0] && y >= bx.lo[1] && y < bx.hi[1] && z >= bx.lo[2] && z < bx.hi[2];
    };
    for (int S = 0; S < kTypes; ++S)
        for (int L = 1; L <= H - 1; ++L) {
            const Box3 *A = o.active[S];
            auto phi_ok = [&](int q) {
                const int x = q % P, y = (q / P) % P, z = q / (P * P);
                if (x == 0 || y == 0 || z == 0) return false;  // the inner halo is the exchange's
                if (L - 2 >= 1 && in_box(A[L - 2], x, y, z)) return false;
                if (L - 1 >= 1) {
                    const int nb[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
                    for (const auto &v : nb)
                        if (in_box(A[L - 1], x + v[0], y + v[1], z + v[2])) return false;
                }
                return true;
            };
            for (int i = 0; i < o.imp_phi_n[S][L]; ++i)
                if (!phi_ok(o.imp_phi[o.imp_phi_off[S][L] + i])) return "an octant copy overtakes a level in flight";
            for (int i = 0; i < o.imp_full_n[S][L]; ++i) {
                const int e = o.imp_full[o.imp_full_off[S][L] + i];
                if (!phi_ok(e & 0xFFFF)) return "an octant copy overtakes a level in flight";
                const int c = e >> 16, x = c % H + 1, y = (c / H) % H + 1, z = c / (H * H) + 1;
                for (int k = std::max(1, L - 2); k <= L; ++k)
                    if (in_box(A[k], x, y, z)) return "an octant (pi, c) copy overtakes a level in flight";
            }
        }

    // ---- traffic and site-updates per region (eight octants) ----
    for (int S = 0; S < kTypes; ++S) {
        int64_t base_cells = 0, upd = 0;
        const Box3 &bp = o.base_phi[S], &bc = o.base_pc[S];
        for (int z = bp.lo[2]; z < bp.hi[2]; ++z)
            for (int y = bp.lo[1]; y < bp.hi[1]; ++y)
                for (int x = bp.lo[0]; x < bp.hi[0]; ++x) {
                    const int out = (x < bc.lo[0] || x >= bc.hi[0]) + (y < bc.lo[1] || y >= bc.hi[1]) +
                                    (z < bc.lo[2] || z >= bc.hi[2]);
                    base_cells += out <= 1;
                }
        for (int k = 1; k <= o.levels[S]; ++k) upd += 8 * o.active[S][k].volume();
        if (upd != t.updates[S]) return "octant site-updates differ from the region's";
        o.updates[S] = upd;
        o.bytes_read[S] = 8 * (8 * base_cells + 16 * o.active[S][1].volume()) + imp_bytes[S];
        o.bytes_written[S] = exp_bytes[S] + (S == kTypes - 1 ? 24LL * B * B * B : 0);
    }
    return std::string();
}

PlanStats plan_stats(const TileTables &t, const int n[3])
{
    PlanStats s{};
    int64_t J = 1;
    for (int d = 0; d < 3; ++d) J *= n[d] / t.B;
    s.regions_per_band = J * kTypes;
    int64_t upd = 0, rd = 0, wr = 0;
    for (int S = 0; S < kTypes; ++S) {
        upd += t.updates[S];
        rd += t.bytes_read[S];
        wr += t.bytes_written[S];
    }
    s.updates_per_band = J * upd;
    s.bytes_read_per_band = J * rd;
    s.bytes_written_per_band = J * wr;
    s.bytes_per_update = (double)(rd + wr) / (double)upd;
    s.bands = 0;
    return s;
}

}  // namespace sp
