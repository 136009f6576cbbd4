// lattice.cpp -- tables of the 4-cube lattice regions (lattice.h): per-level
// cell lists, imports and export flags of one region, all regions being
// translates of it, with the checks that make them trustworthy.
#include "lattice.h"

#include <algorithm>
#include <cstdlib>
#include <cstdio>
#include <map>
#include <set>

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

// Local level k (0 <= k < 4s) and offset r of point (t, x) of the infinite
// lattice (region forms f_i = t + sigma_i . x, region n_i = floor(f_i / 4s)),
// with the region's layer and centre; used to locate producers.
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
    std::map<R3, int> slot, pcidx;
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
    int ns = 0, nf = 0;
    for (const auto &row : rows)  // std::map: ascending (z, y)
        for (int x = row.second.first; x <= row.second.second; ++x) {
            const R3 r = {x, row.first.second, row.first.first};
            slot[r] = ns++;
            if (foot.count(r)) pcidx[r] = nf++;
        }
    t->n_slots = ns;
    t->n_foot = nf;
    if (ns > (1 << kLatCellSlotBits)) return fail("%d slots exceed 12-bit indices", ns);
    t->slot_rec.assign(ns, 0);
    for (const auto &e : slot) {
        const R3 &r = e.first;
        uint32_t rec = (uint32_t)(r.x + R) | (uint32_t)(r.y + R) << 5 | (uint32_t)(r.z + R) << 10;
        auto p = pcidx.find(r);
        if (p != pcidx.end()) rec |= (uint32_t)p->second << 15 | 1u << 27;
        t->slot_rec[e.second] = rec;
    }

    // cell entries with export flags
    t->cell_off.assign(K + 1, 0);
    for (int k = 0; k < K; ++k) {
        t->cell_off[k] = (int32_t)t->cell.size();
        for (const R3 &r : lev[k]) {
            const int sl = slot.at(r);
            const int ym = slot.at({r.x, r.y - 1, r.z}) - sl, yp = slot.at({r.x, r.y + 1, r.z}) - sl;
            const int zm = slot.at({r.x, r.y, r.z - 1}) - sl, zp = slot.at({r.x, r.y, r.z + 1}) - sl;
            if (ym < -128 || ym > 127 || yp < -128 || yp > 127) return fail("y slot step %d / %d beyond 8 bits", ym, yp);
            if (zm < -512 || zm > 511 || zp < -512 || zp > 511) return fail("z slot step %d / %d beyond 10 bits", zm, zp);
            if (slot.at({r.x - 1, r.y, r.z}) != sl - 1 || slot.at({r.x + 1, r.y, r.z}) != sl + 1)
                return fail("x neighbours of a cell are not adjacent slots");
            bool ephi = false;
            const bool epc = !(k + 1 < K && levset[k + 1].count(r));
            // phi(k, r) is read at level k + 1 by r and its six neighbours
            if (epc) ephi = true;
            for (const auto &d : kNb)
                if (!(k + 1 < K && levset[k + 1].count(add(r, d)))) ephi = true;
            uint64_t e = (uint64_t)sl | (uint64_t)pcidx.at(r) << 12 | (uint64_t)(uint8_t)(int8_t)ym << 24 |
                         (uint64_t)(uint8_t)(int8_t)yp << 32 | (uint64_t)(zm & 1023) << 40 | (uint64_t)(zp & 1023) << 50;
            if (ephi) e |= kLatExpPhi, ++t->exports_phi;
            if (epc) e |= kLatExpPc, ++t->exports_pc;
            t->cell.push_back(e);
        }
    }
    t->cell_off[K] = (int32_t)t->cell.size();

    // imports before level k: full (cells entering), phi only (neighbours outside)
    t->imp_off.assign(K + 1, 0);
    for (int k = 0; k < K; ++k) {
        t->imp_off[k] = (int32_t)t->imp.size();
        std::set<int> full, phi;
        for (const R3 &r : lev[k]) {
            if (!(k > 0 && levset[k - 1].count(r))) full.insert(slot.at(r));
            for (const auto &d : kNb) {
                const R3 q = add(r, d);
                if ((k > 0 && levset[k - 1].count(q)) || levset[k].count(q)) continue;
                phi.insert(slot.at(q));
            }
        }
        std::vector<uint16_t> list;
        for (int sl : full) list.push_back((uint16_t)(sl | kLatImpFull));
        for (int sl : phi) list.push_back((uint16_t)sl);
        std::sort(list.begin(), list.end(), [](uint16_t a, uint16_t b) { return (a & 0x7fff) < (b & 0x7fff); });
        t->imp.insert(t->imp.end(), list.begin(), list.end());
        t->imports_full += (int64_t)full.size();
        t->imports_phi += (int64_t)phi.size();
    }
    t->imp_off[K] = (int32_t)t->imp.size();
    t->bytes_read = 24 * t->imports_full + 8 * t->imports_phi;
    t->bytes_written = 8 * t->exports_phi + 16 * t->exports_pc;

    // check 1: every value level k reads is computed at level k - 1 or imported before level k
    std::map<R3, int> by_slot_r;
    for (const auto &e : slot) by_slot_r[e.first] = e.second;
    for (int k = 0; k < K; ++k) {
        std::set<int> have_phi, have_pc;
        if (k > 0)
            for (const R3 &r : lev[k - 1]) have_phi.insert(slot.at(r)), have_pc.insert(slot.at(r));
        for (int i = t->imp_off[k]; i < t->imp_off[k + 1]; ++i) {
            const int sl = t->imp[i] & 0x7fff;
            if (have_phi.count(sl)) return fail("level %d imports a value it already holds", k);
            have_phi.insert(sl);
            if (t->imp[i] & kLatImpFull) have_pc.insert(sl);
        }
        for (const R3 &r : lev[k]) {
            if (!have_pc.count(slot.at(r)) || !have_phi.count(slot.at(r))) return fail("level %d lacks a cell's own state", k);
            for (const auto &d : kNb)
                if (!have_phi.count(slot.at(add(r, d)))) return fail("level %d lacks a neighbour's phi", k);
        }
    }

    // check 2: every import is exported by the region computing it.  Place
    // the region at the origin (centre 0, bottom vertex at t = 0); the value
    // imported before level k is at (k - 1, r).
    std::vector<std::map<R3, uint64_t>> entry(K);
    for (int k = 0; k < K; ++k)
        for (int i = t->cell_off[k]; i < t->cell_off[k + 1]; ++i) {
            const uint32_t rec = t->slot_rec[t->cell[i] & 0xfff];
            entry[k][{(int)(rec & 31) - R, (int)(rec >> 5 & 31) - R, (int)(rec >> 10 & 31) - R}] = t->cell[i];
        }
    for (int k = 0; k < K; ++k)
        for (int i = t->imp_off[k]; i < t->imp_off[k + 1]; ++i) {
            const uint32_t rec = t->slot_rec[t->imp[i] & 0x7fff];
            const R3 r = {(int)(rec & 31) - R, (int)(rec >> 5 & 31) - R, (int)(rec >> 10 & 31) - R};
            int kp;
            R3 rp;
            locate(s, k - 1, r, &kp, &rp);
            if (!in_level(s, kp, rp)) return fail("producer of an import at level %d not located", k);
            if (kp == k - 1 && rp == r) return fail("import at level %d is the region's own value", k);
            auto it = entry[kp].find(rp);
            if (it == entry[kp].end()) return fail("producer cell missing at level %d", kp);
            if (!(it->second & kLatExpPhi)) return fail("imported phi not exported (level %d)", k);
            if ((t->imp[i] & kLatImpFull) && !(it->second & kLatExpPc)) return fail("imported (pi, c) not exported (level %d)", k);
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

}  // namespace sp
