// lattice.cpp -- tables of the 4-cube lattice regions (lattice.h): per-level
// cell lists, imports and export flags of one region, all regions being
// translates of it, with the checks that make them trustworthy.
#include "lattice.h"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <set>
#include <tuple>
#include <utility>

namespace sp {

namespace {

constexpr int kSig[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};

constexpr int kNb[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};

struct R3 {
    int x, y, z;
    bool operator<(const R3 &o) const
    {
        if (z != o.z) return z < o.z;
        if (y != o.y) return y < o.y;
        return x < o.x;
    }
    bool operator==(const R3 &o) const { return x == o.x && y == o.y && z == o.z; }
};

R3 add(R3 a, const int d[3]) { return {a.x + d[0], a.y + d[1], a.z + d[2]}; }

int dot(const int s[3], R3 r) { return s[0] * r.x + s[1] * r.y + s[2] * r.z; }

// Local level k and offset r of point (t, x) of the infinite lattice (forms
// f_i = t + sigma_i . x, region n_i = floor(f_i / 4s), bottom vertex of
// region n at t = s (n_1 + n_2 + n_3 + n_4)); used to locate producers.
void locate(int s, int t, R3 x, int *k, R3 *r)
{
    const int w = 4 * s;
    int n[4];
    for (int i = 0; i < 4; ++i) {
        const int f = t + dot(kSig[i], x);
        n[i] = f >= 0 ? f / w : -((-f + w - 1) / w);
    }
    const int L = n[0] + n[1] + n[2] + n[3];
    const R3 c = {s * (n[0] + n[1] - n[2] - n[3]), s * (n[0] - n[1] + n[2] - n[3]), s * (n[0] - n[1] - n[2] + n[3])};
    *k = t - s * L;
    *r = {x.x - c.x, x.y - c.y, x.z - c.z};
}

bool in_level(int s, int k, R3 r)
{
    if (k < 0 || k >= 4 * s) return false;
    for (int i = 0; i < 4; ++i) {
        const int v = dot(kSig[i], r);
        if (v < -k || v > 4 * s - 1 - k) return false;
    }
    return true;
}

std::string fail(const char *fmt, int a = 0, int b = 0, int c = 0)
{
    char buf[200];
    std::snprintf(buf, sizeof buf, fmt, a, b, c);
    return buf;
}

void pad4(std::vector<uint32_t> *v)
{
    while (v->size() % 4) v->push_back(0u);
}

}  // namespace

std::string build_lattice_tables(int s, LatticeTables *t)
{
    if (s < kLatMinS || s > kLatMaxS) return fail("lattice size s=%d outside [1, 6]", s);
    *t = LatticeTables();
    t->s = s;
    const int K = 4 * s;
    t->K = K;
    const int R = 2 * s;  // |r_d| <= 2s - 1 for cells, 2s for the halo

    // cells of every level, in row order (z, y, x)
    std::vector<std::vector<R3>> lev(K);
    std::vector<std::set<R3>> levset(K);
    for (int k = 0; k < K; ++k) {
        for (int z = -R; z <= R; ++z)
            for (int y = -R; y <= R; ++y)
                for (int x = -R; x <= R; ++x)
                    if (in_level(s, k, {x, y, z})) lev[k].push_back({x, y, z});
        levset[k] = std::set<R3>(lev[k].begin(), lev[k].end());
        t->updates += (int64_t)lev[k].size();
        t->max_level_cells = std::max(t->max_level_cells, (int)lev[k].size());
    }
    if (t->updates != 16ll * s * s * s * s) return fail("region holds %d site-updates, not 16 s^4", (int)t->updates);

    // footprint and halo; slots in rows (z, y), each row contiguous in x
    std::set<R3> foot, used;
    for (int k = 0; k < K; ++k)
        for (const R3 &r : lev[k]) {
            foot.insert(r);
            used.insert(r);
            for (const auto &d : kNb) used.insert(add(r, d));
        }
    for (const R3 &r : used)
        if (std::abs(r.x) > R || std::abs(r.y) > R || std::abs(r.z) > R) return fail("halo cell beyond |r| = 2s");
    std::map<std::pair<int, int>, std::pair<int, int>> rows;  // (z, y) -> x range
    for (const R3 &r : used) {
        auto key = std::make_pair(r.z, r.y);
        auto it = rows.find(key);
        if (it == rows.end())
            rows[key] = {r.x, r.x};
        else {
            it->second.first = std::min(it->second.first, r.x);
            it->second.second = std::max(it->second.second, r.x);
        }
    }
    t->rb_side = 4 * s + 1;
    const int W = t->rb_side;
    if (W * W > (int)kLatRowMask + 1) return fail("%d rows exceed the entries' row field", W * W);
    auto row_index = [&](int y, int z) { return (y + R) * W + z + R; };
    std::vector<int> row_base((size_t)W * W, 0);
    std::map<R3, int> slot, pcidx;
    // Bank-friendly layout: every phi slot and every (pi, c) index is
    // congruent to x + a y + b z mod 16, so that the neighbours of 16 cells
    // with distinct residues (one half-warp's 8-byte accesses) again have
    // distinct residues, and so do their (pi, c) slots mod 8 for each group of
    // eight lanes (16-byte accesses).  Rows are chained so that each starts on
    // its residue, taking the row that needs the least padding next; (a, b)
    // is the pair with the smallest shared-memory footprint.
    int bank_a = 0, bank_b = 0;
    auto residue = [&](int x, int y, int z) { return (((x + bank_a * y + bank_b * z) % 16) + 16) % 16; };
    auto chain = [&](const std::map<std::pair<int, int>, std::pair<int, int>> &rws, std::map<R3, int> *index,
                     const std::set<R3> *only, int *count, std::vector<int> *base) {
        std::vector<std::pair<std::pair<int, int>, std::pair<int, int>>> todo(rws.begin(), rws.end());
        std::vector<char> done(todo.size(), 0);
        int pos = 0;
        for (size_t placed = 0; placed < todo.size(); ++placed) {
            int pick = -1, best_gap = 16;
            for (size_t i = 0; i < todo.size() && best_gap > 0; ++i) {
                if (done[i]) continue;
                const int want = residue(todo[i].second.first, todo[i].first.second, todo[i].first.first);
                const int gap = ((want - pos % 16) + 16) % 16;
                if (gap < best_gap) best_gap = gap, pick = (int)i;
            }
            pos += best_gap;
            done[pick] = 1;
            const int z = todo[pick].first.first, y = todo[pick].first.second;
            const int xlo = todo[pick].second.first, xhi = todo[pick].second.second;
            if (base) (*base)[row_index(y, z)] = pos - xlo;
            if (index)
                for (int x = xlo; x <= xhi; ++x) {
                    const R3 r = {x, y, z};
                    if (!only || only->count(r)) (*index)[r] = pos + (x - xlo);
                }
            pos += xhi - xlo + 1;
        }
        *count = pos;
    };
    std::map<std::pair<int, int>, std::pair<int, int>> frows;  // footprint rows (z, y) -> x range
    for (const R3 &r : foot) {
        auto key = std::make_pair(r.z, r.y);
        auto it = frows.find(key);
        if (it == frows.end())
            frows[key] = {r.x, r.x};
        else {
            it->second.first = std::min(it->second.first, r.x);
            it->second.second = std::max(it->second.second, r.x);
        }
    }
    {
        int best = 1 << 30, ba = 0, bb = 0;
        for (int a = 0; a < 16; ++a)
            for (int b = 0; b < 16; ++b) {
                bank_a = a, bank_b = b;
                int n1 = 0, n2 = 0;
                chain(rows, nullptr, nullptr, &n1, nullptr);
                chain(frows, nullptr, nullptr, &n2, nullptr);
                if (16 * n1 + 16 * n2 < best) best = 16 * n1 + 16 * n2, ba = a, bb = b;
            }
        bank_a = ba, bank_b = bb;
    }
    int ns = 0, nf = 0;
    chain(rows, &slot, nullptr, &ns, &row_base);
    chain(frows, &pcidx, &foot, &nf, nullptr);
    t->bank_a = bank_a;
    t->bank_b = bank_b;
    for (const auto &e : slot)
        if (e.second % 16 != residue(e.first.x, e.first.y, e.first.z)) return fail("slot off its bank residue");
    for (const auto &e : pcidx)
        if (e.second % 16 != residue(e.first.x, e.first.y, e.first.z)) return fail("(pi, c) index off its bank residue");
    t->n_slots = ns;
    t->n_foot = nf;  // (pi, c) slots, padding included
    t->foot_cells = (int)foot.size();
    t->halo_cells = (int)(used.size() - foot.size());
    if (ns > 8192 || nf > 8192) return fail("%d slots exceed the kernel's 13-bit indices", ns);

    // per-row constants: neighbour steps, (pi, c) offset, row base and offset
    t->row_nb.assign((size_t)W * W, 0);
    t->row_xy.assign((size_t)W * W, 0);
    for (int y = -R; y <= R; ++y)
        for (int z = -R; z <= R; ++z) {
            const int i = row_index(y, z);
            if (row_base[i] < -32768 || row_base[i] > 32767) return fail("row base beyond 16 bits");
            t->row_xy[i] = (uint32_t)(uint16_t)(int16_t)row_base[i] | (uint32_t)(y + R) << 16 | (uint32_t)(z + R) << 21;
        }
    std::map<int, std::vector<int>> row_vals;  // row -> (dym, dyp, dzm, dzp, dpc), from its footprint cells
    for (const auto &e : pcidx) {
        const R3 &r = e.first;
        const int sl = slot.at(r);
        std::vector<int> v = {slot.at({r.x, r.y - 1, r.z}) - sl, slot.at({r.x, r.y + 1, r.z}) - sl,
                              slot.at({r.x, r.y, r.z - 1}) - sl, slot.at({r.x, r.y, r.z + 1}) - sl, e.second - sl};
        const int i = row_index(r.y, r.z);
        auto it = row_vals.find(i);
        if (it == row_vals.end())
            row_vals[i] = v;
        else if (it->second != v)
            return fail("neighbour steps or (pi, c) offset vary along a row");
    }
    t->row_pc.assign((size_t)W * W, 0);
    for (const auto &rv : row_vals) {
        const std::vector<int> &v = rv.second;
        for (int i = 0; i < 4; ++i)
            if (v[i] < -4096 || v[i] > 4095) return fail("neighbour step beyond 13 bits");
        t->row_nb[rv.first] = (uint64_t)(uint16_t)(int16_t)v[0] | (uint64_t)(uint16_t)(int16_t)v[1] << 16 |
                              (uint64_t)(uint16_t)(int16_t)v[2] << 32 | (uint64_t)(uint16_t)(int16_t)v[3] << 48;
        t->row_pc[rv.first] = v[4];
    }
    auto entry_of = [&](const R3 &r) {
        return (uint32_t)slot.at(r) | (uint32_t)row_index(r.y, r.z) << kLatRowShift |
               (uint32_t)(r.x + 2 * s) << kLatRxShift;
    };

    // Each level's cells in groups of 16 with distinct slot residues mod 16
    // (one half-warp), taken in row order with a cell deferred while its
    // residue is taken; within a group, residues 0..7 first (two groups of
    // eight lanes with distinct residues mod 8).
    for (int k = 0; k < K; ++k) {
        std::vector<R3> pool = lev[k], out;
        while (!pool.empty()) {
            std::vector<R3> lo, hi, rest;
            unsigned used = 0;
            for (const R3 &r : pool) {
                const int res = slot.at(r) % 16;
                if (lo.size() + hi.size() < 16 && !(used >> res & 1u)) {
                    used |= 1u << res;
                    (res < 8 ? lo : hi).push_back(r);
                } else {
                    rest.push_back(r);
                }
            }
            out.insert(out.end(), lo.begin(), lo.end());
            out.insert(out.end(), hi.begin(), hi.end());
            pool.swap(rest);
        }
        lev[k] = out;
    }

    // cell entries with export flags
    t->cell_off.assign(K + 1, 0);
    t->cell_n.assign(K, 0);
    for (int k = 0; k < K; ++k) {
        t->cell_off[k] = (int32_t)t->cell.size();
        for (const R3 &r : lev[k]) {
            for (const auto &d : kNb)
                if (!slot.count(add(r, d))) return fail("neighbour without a slot at level %d", k);
            const bool epc = !(k + 1 < K && levset[k + 1].count(r));
            // phi(k, r) is read at level k + 1 by r and its six neighbours
            bool ephi = epc;
            for (const auto &d : kNb)
                if (!(k + 1 < K && levset[k + 1].count(add(r, d)))) ephi = true;
            uint32_t e = entry_of(r);
            if (ephi) e |= kLatExpPhi, ++t->exports_phi;
            if (epc) e |= kLatExpPc, ++t->exports_pc;
            t->cell.push_back(e);
        }
        t->cell_n[k] = (int32_t)t->cell.size() - t->cell_off[k];
        pad4(&t->cell);
        t->max_cell_n = std::max(t->max_cell_n, (int)t->cell.size() - t->cell_off[k]);
    }
    t->cell_off[K] = (int32_t)t->cell.size();

    // imports before level k: full (cells entering), phi only (neighbours outside)
    t->imp_off.assign(K + 1, 0);
    t->imp_n.assign(K, 0);
    for (int k = 0; k < K; ++k) {
        t->imp_off[k] = (int32_t)t->imp.size();
        std::set<R3> full, phi;
        for (const R3 &r : lev[k]) {
            if (!(k > 0 && levset[k - 1].count(r))) full.insert(r);
            for (const auto &d : kNb) {
                const R3 q = add(r, d);
                if ((k > 0 && levset[k - 1].count(q)) || levset[k].count(q)) continue;
                phi.insert(q);
            }
        }
        std::vector<std::pair<int, uint32_t>> list;  // ascending slots
        const uint32_t buf = ((k - 1) & 1) ? kLatImpBuf : 0u;
        for (const R3 &r : full) list.push_back({slot.at(r), entry_of(r) | kLatImpFull | buf});
        for (const R3 &r : phi) list.push_back({slot.at(r), entry_of(r) | buf});
        std::sort(list.begin(), list.end());
        for (const auto &e : list) t->imp.push_back(e.second);
        t->imp_n[k] = (int32_t)list.size();
        pad4(&t->imp);
        t->max_imp_n = std::max(t->max_imp_n, (int)t->imp.size() - t->imp_off[k]);
        t->imports_full += (int64_t)full.size();
        t->imports_phi += (int64_t)phi.size();
    }
    t->imp_off[K] = (int32_t)t->imp.size();
    {
        // the pair bit: slot ^ 1 is x +- 1 of the same row, or never imported
        // into the same buffer
        std::map<int, R3> cell_of;
        for (const auto &kv : slot) cell_of[kv.second] = kv.first;
        std::set<std::pair<int, int>> imported;
        for (int k = 0; k < K; ++k)
            for (int i = t->imp_off[k]; i < t->imp_off[k] + t->imp_n[k]; ++i)
                imported.insert({lat_slot(t->imp[i]), (k - 1) & 1});
        for (int k = 0; k < K; ++k)
            for (int i = t->imp_off[k]; i < t->imp_off[k] + t->imp_n[k]; ++i) {
                const int sl = lat_slot(t->imp[i]), p = sl ^ 1;
                const R3 &c = cell_of.at(sl);
                auto q = cell_of.find(p);
                const bool same_row =
                    q != cell_of.end() && q->second.y == c.y && q->second.z == c.z && q->second.x - c.x == p - sl;
                if (same_row || !imported.count({p, (k - 1) & 1})) t->imp[i] |= kLatImpPair;
                if (same_row) t->imp[i] |= kLatImpPairRow;
            }
    }
    {
        // every import in one list: by buffer, then offset (z, y, x)
        std::vector<std::pair<std::tuple<int, int, int, int>, std::pair<uint32_t, uint32_t>>> all;
        for (int k = 0; k < K; ++k)
            for (int i = t->imp_off[k]; i < t->imp_off[k] + t->imp_n[k]; ++i) {
                const uint32_t e = t->imp[i];
                int rx, ry, rz;
                t->offset_of(lat_slot(e), lat_row(e), &rx, &ry, &rz);
                all.push_back({{(e & kLatImpBuf) ? 1 : 0, rz, ry, rx}, {e, (uint32_t)k}});
            }
        std::sort(all.begin(), all.end());
        for (const auto &x : all) t->imp_all.push_back(x.second.first), t->imp_all.push_back(x.second.second);
    }
    t->bytes_read = 24 * t->imports_full + 8 * t->imports_phi;
    t->bytes_written = 8 * t->exports_phi + 16 * t->exports_pc;

    // decode an entry as the kernel does: offset, neighbour slots, (pi, c) index
    auto decode = [&](uint32_t e, R3 *r, int nb[7], int *pc) {
        const int sl = lat_slot(e), row = lat_row(e);
        t->offset_of(sl, row, &r->x, &r->y, &r->z);
        const uint64_t v = t->row_nb[row];
        nb[0] = sl, nb[1] = sl - 1, nb[2] = sl + 1;
        nb[3] = sl + lat_dym(v), nb[4] = sl + lat_dyp(v), nb[5] = sl + lat_dzm(v), nb[6] = sl + lat_dzp(v);
        *pc = sl + t->row_pc[row];
    };

    // check 0: the row index divides by 4s + 1 as the kernel divides it, and
    // every entry's x field is its cell's x offset (plus 2s)
    for (int row = 0; row < W * W; ++row) {
        const uint32_t xy = t->row_xy[row];
        const int y2s = lat_row_y2s(row, lat_row_div(s));
        if (y2s != (int)((xy >> 16) & 31u) || row - y2s * W != (int)((xy >> 21) & 31u))
            return fail("row %d does not divide into its y and z", row);
    }
    for (int k = 0; k < K; ++k) {
        auto x_ok = [&](uint32_t e) {
            int rx, ry, rz;
            t->offset_of(lat_slot(e), lat_row(e), &rx, &ry, &rz);
            return lat_rx2s(e) == rx + 2 * s;
        };
        for (int i = t->cell_off[k]; i < t->cell_off[k] + t->cell_n[k]; ++i)
            if (!x_ok(t->cell[i])) return fail("cell entry with a wrong x field (level %d)", k);
        for (int i = t->imp_off[k]; i < t->imp_off[k] + t->imp_n[k]; ++i)
            if (!x_ok(t->imp[i])) return fail("import entry with a wrong x field (level %d)", k);
    }
    // check 1: entries decode to their cells, and every value level k reads
    // is computed at level k - 1 or imported before level k
    for (int k = 0; k < K; ++k) {
        std::set<int> have_phi, have_pc;
        if (k > 0)
            for (int i = t->cell_off[k - 1]; i < t->cell_off[k - 1] + t->cell_n[k - 1]; ++i) {
                R3 r;
                int nb[7], pc;
                decode(t->cell[i], &r, nb, &pc);
                have_phi.insert(nb[0]);
                have_pc.insert(pc);
            }
        for (int i = t->imp_off[k]; i < t->imp_off[k] + t->imp_n[k]; ++i) {
            R3 r;
            int nb[7], pc;
            decode(t->imp[i], &r, nb, &pc);
            if (slot.at(r) != nb[0]) return fail("import entry does not decode to its cell (level %d)", k);
            if (have_phi.count(nb[0])) return fail("level %d imports a value it already holds", k);
            have_phi.insert(nb[0]);
            if (t->imp[i] & kLatImpFull) {
                if (pc != pcidx.at(r)) return fail("full import with a wrong (pi, c) index");
                have_pc.insert(pc);
            }
        }
        int n = 0;
        for (int i = t->cell_off[k]; i < t->cell_off[k] + t->cell_n[k]; ++i, ++n) {
            R3 r;
            int nb[7], pc;
            decode(t->cell[i], &r, nb, &pc);
            if (!(r == lev[k][n]) || slot.at(r) != nb[0] || pc != pcidx.at(r))
                return fail("cell entry does not decode to its cell (level %d)", k);
            for (int d = 0; d < 6; ++d)
                if (nb[1 + d] != slot.at(add(r, kNb[d]))) return fail("neighbour slot wrong at level %d", k);
            if (!have_pc.count(pc) || !have_phi.count(nb[0])) return fail("level %d lacks a cell's own state", k);
            for (int d = 1; d < 7; ++d)
                if (!have_phi.count(nb[d])) return fail("level %d lacks a neighbour's phi", k);
        }
    }

    // check 1b: each (slot, phi buffer) is imported at most once, and no cell
    // computation writes it, or reads it, at a level before the import's (so
    // a region may load all its imports at its start)
    {
        std::map<std::pair<int, int>, int> imp_level;
        for (int k = 0; k < K; ++k)
            for (int i = t->imp_off[k]; i < t->imp_off[k] + t->imp_n[k]; ++i) {
                const auto key = std::make_pair(lat_slot(t->imp[i]), (k - 1) & 1);
                if (imp_level.count(key)) return fail("a slot of a phi buffer imported twice (level %d)", k);
                if (((t->imp[i] & kLatImpBuf) != 0) != (((k - 1) & 1) != 0)) return fail("import buffer bit wrong");
                imp_level[key] = k;
            }
        for (int k = 0; k < K; ++k)
            for (int i = t->cell_off[k]; i < t->cell_off[k] + t->cell_n[k]; ++i) {
                R3 r;
                int nb[7], pc;
                decode(t->cell[i], &r, nb, &pc);
                auto w = imp_level.find(std::make_pair(nb[0], k & 1));
                if (w != imp_level.end() && w->second > k) return fail("level %d writes a slot imported later", k);
                for (int d = 0; d < 7; ++d) {
                    auto q = imp_level.find(std::make_pair(nb[d], (k - 1) & 1));
                    if (q != imp_level.end() && q->second > k) return fail("level %d reads a slot imported later", k);
                }
            }
        if (t->imp_all.size() != 2 * (size_t)(t->imports_full + t->imports_phi)) return fail("import list incomplete");
    }
    // check 2: every import is exported by the region computing it.  Place
    // the region at the origin (centre 0, bottom vertex at t = 0); the value
    // imported before level k is at (k - 1, r).
    std::vector<std::map<R3, uint32_t>> entry(K);
    for (int k = 0; k < K; ++k)
        for (int i = t->cell_off[k]; i < t->cell_off[k] + t->cell_n[k]; ++i) {
            R3 r;
            int nb[7], pc;
            decode(t->cell[i], &r, nb, &pc);
            entry[k][r] = t->cell[i];
        }
    for (int k = 0; k < K; ++k)
        for (int i = t->imp_off[k]; i < t->imp_off[k] + t->imp_n[k]; ++i) {
            R3 r;
            int nb[7], pc;
            decode(t->imp[i], &r, nb, &pc);
            int kp;
            R3 rp;
            locate(s, k - 1, r, &kp, &rp);
            if (!in_level(s, kp, rp)) return fail("producer of an import at level %d not located", k);
            if (kp == k - 1 && rp == r) return fail("import at level %d is the region's own value", k);
            auto it = entry[kp].find(rp);
            if (it == entry[kp].end()) return fail("producer cell missing at level %d", kp);
            if (!(it->second & kLatExpPhi)) return fail("imported phi not exported (level %d)", k);
            if ((t->imp[i] & kLatImpFull) && !(it->second & kLatExpPc))
                return fail("imported (pi, c) not exported (level %d)", k);
        }
    // check 3: the local membership agrees with the lattice forms for every
    // point of the region placed at the origin
    for (int k = 0; k < K; ++k)
        for (const R3 &r : lev[k]) {
            int kp;
            R3 rp;
            locate(s, k, r, &kp, &rp);
            if (kp != k || !(rp == r)) return fail("cell of level %d belongs to another region", k);
        }
    return std::string();
}

LatCallStats lattice_call_stats(const LatticeTables &t, int64_t T)
{
    LatCallStats st;
    if (T < 1 || t.K == 0) return st;
    const int s = t.s, K = t.K, Lcount = lat_layer_count(s, T);
    for (int li = 0; li < Lcount; ++li) {
        const int L = lat_min_layer() + li;
        const int64_t tau_b = 1 + (int64_t)s * L;
        const int k_lo = tau_b < 1 ? (int)(1 - tau_b) : 0;
        const int k_hi = (int)std::min<int64_t>(K - 1, T - tau_b);
        if (k_lo > 0) st.bytes_read += 24 * (int64_t)t.cell_n[k_lo - 1];
        for (int k = k_lo; k <= k_hi; ++k) {
            st.updates += t.cell_n[k];
            for (int i = t.imp_off[k]; i < t.imp_off[k] + t.imp_n[k]; ++i)
                st.bytes_read += (t.imp[i] & kLatImpFull) ? 24 : 8;
            for (int i = t.cell_off[k]; i < t.cell_off[k] + t.cell_n[k]; ++i) {
                const uint32_t e = t.cell[i];
                const bool all = k == k_hi;
                if (all || (e & kLatExpPhi)) st.bytes_written += 8;
                if (all || (e & kLatExpPc)) st.bytes_written += 16;
            }
        }
    }
    return st;
}

}  // namespace sp
