// lattice.h -- the paper's own region geometry: a lattice of 4-cubes with
// time along the main diagonal (Sec. 2, Figs. 2-5), planned for in-place
// evolution of the state arrays.
//
// Geometry.  With the 7-point stencil, the value at (t, x) depends on
// (t-1, x) and (t-1, x +- e_d).  The four forms
//
//   f_i(t, x) = t + sigma_i . x,   sigma = (1,1,1), (1,-1,-1), (-1,1,-1), (-1,-1,1)
//
// change along such a dependency by 1 - sigma_i . d, which is 0, 1 or 2:
// none of them ever decreases.  So the cells with floor(f_i / 4s) = n_i
// (n in Z^4) form regions that read only from regions n' <= n (componentwise)
// and feed only regions n' >= n: each region has four initial faces
// (f_i = 4s n_i) and four final ones.  These are the paper's 4-cubes with the
// generators (+-1/2, +-1/2, +-1/2, 1/2) scaled by 4s; under the 7-point
// stencil's cone (one cell per step along every axis) their faces are
// characteristic as they are, with no rescaling of time.  A region holds
// 16 s^4 site-updates over 4s levels; all regions are translates of one
// another (one congruent type).  In local coordinates -- level k from the
// region's bottom vertex and cell offset r from its centre -- the region's
// cells at level k are
//
//   { r : -k <= sigma_i . r <= 4s - 1 - k  for i = 1..4 },
//
// a tetrahedron growing from one cell (k < s), an octahedron-like middle and
// a shrinking inverted tetrahedron (k >= 3s).
//
// Layers (Sec. 2, Fig. 2).  Region n starts at level s (n_1 + n_2 + n_3 + n_4)
// (its layer L times s) and has its centre at
//   s (n1 + n2 - n3 - n4, n1 - n2 + n3 - n4, n1 - n2 - n3 + n4).
// Regions of one layer start together; four layers are active at any level;
// region n's predecessors are n - e_i (layer L - 1, centres shifted by
// -s(1,1,1), s(-1,1,1), s(1,-1,1), s(1,1,-1)), its successors n + e_i.
// Dependencies that cross two or more faces at once (a corner or an edge)
// come from regions n - e_i - e_j ..., which precede n through the four face
// predecessors.
//
// Periodicity (Sec. 2.2).  On a periodic grid of sides N_d = 4 s M_d a
// centre is taken mod N_d; a layer then holds 4 M_x M_y M_z regions (the
// centres form a face-centred cubic lattice of cube side 4s).
//
// In-place state.  Regions read and write the state arrays themselves: phi at
// level t lives in buffer t mod 2 (two phi arrays), (pi, c) in one array.
// A region imports phi(t-1, y) and (pi, c)(t-1, y) it does not compute and
// exports every value some other region (or the end of the call) needs.
// This is race-free by the monotonicity above: a write that could clobber
// a read, phi(t+1, y) over phi(t-1, y) or (pi, c) at a later level over
// (pi, c)(t-1, y), is made by the reading region itself (later) or by one of
// its successors, and a value read is written by the reader's predecessor.
// Two regions of one layer may write phi(t, y) and read phi(t-1, y) at the
// same time: these sit in different buffers.  No mailbox is needed.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#if defined(__CUDACC__)
#define LAT_HD __host__ __device__ __forceinline__
#else
#define LAT_HD inline
#endif

namespace sp {

constexpr int kLatMinS = 1;
constexpr int kLatMaxS = 6;  // slot indices are 13 bits, coordinates 5 bits per axis

// Shared-memory phi slots are laid out in rows of constant (y, z), each
// contiguous in x: slot(r) = row_base(row) + rx with
// row = (ry + 2s) (4s + 1) + rz + 2s.  Rows are placed so that every slot,
// and every (pi, c) index, is congruent to rx + a ry + b rz mod 16 (a, b
// chosen per size): 16 cells with distinct residues then read their phi and
// all six neighbours without shared-memory bank conflicts, and groups of 8
// of them their (pi, c) too.  The x neighbours are slot - 1 and slot + 1; the
// y and z neighbours and the (pi, c) index follow from per-row constants:
//   row_nb (64 bits): slot(y - 1) - slot, slot(y + 1) - slot,
//     slot(z - 1) - slot, slot(z + 1) - slot (signed 16 bits each, low first);
//   row_pc (32 bits): pc - slot;
//   row_xy (32 bits): row_base (bits 0..15, signed) | (ry + 2s) << 16 |
//     (rz + 2s) << 21, for the cell's offset from the region's centre.
// Cell entry (32 bits), the per-level work list:
//   bits 0..12 slot; bits 13..22 row; bit 23 export phi at this level;
//   bit 24 export (pi, c) at this level; bits 25..29 the cell's x offset
//   from the region's centre plus 2s (so a site index needs no per-cell
//   table read beyond the row's).  Each level's list is ordered so
//   that every 16 consecutive entries have distinct slot residues mod 16,
//   the first and last 8 of them distinct residues mod 8.
// Import entry (32 bits): slot | row << 13 | full << 23 | ((k - 1) & 1) << 24 |
// (x offset + 2s) << 25 | pair << 30 | pair-row << 31, for an import before
// level k.  A full import loads
// phi(k-1) and (pi, c)(k-1) of a cell entering the region at level k; otherwise
// only phi(k-1) of a neighbour outside the region.
// Every value a region imports is final when the region starts (its producers
// are its ancestors, which are done) and stays in place until the region is
// done (whoever overwrites it depends on the region), and a region imports each
// (slot, phi buffer) at most once and touches that slot of that buffer only
// from the import's level on (the builder checks both), so a region may load
// all its imports at its start: imp_all holds them in one list, sorted by
// buffer and by offset from the centre (z, y, x: ascending addresses), each
// with its level, which regions cut by a call's first or last level filter.
// Every level's lists start on a 16-byte boundary (padded with zero entries
// to a multiple of four).
constexpr uint32_t kLatSlotMask = 0x1fffu;
constexpr int kLatRowShift = 13;
constexpr uint32_t kLatRowMask = 0x3ffu;
constexpr uint32_t kLatExpPhi = 1u << 23;
constexpr uint32_t kLatExpPc = 1u << 24;
constexpr uint32_t kLatImpFull = 1u << 23;
constexpr uint32_t kLatImpBuf = 1u << 24;  // the phi buffer ((k - 1) & 1) of the value
// Bit 30 of an import entry: the slot's pair partner (slot ^ 1) holds the
// neighbour in x of the same row, or is never imported into this buffer, so a
// region that loads nothing else into its phi buffers at its start may copy
// the aligned 16-byte site pair into the aligned slot pair when slot and
// site have the same parity.
constexpr uint32_t kLatImpPair = 1u << 30;
// Bit 31: the pair partner is the row's neighbour in x.  A region cut by the
// call's first level also loads its own cells of the level before its first
// from the state at its start; a pair copy whose partner is the row's
// neighbour writes the partner slot the same bytes any other load of it
// does, so such a region may copy the pairs with this bit.
constexpr uint32_t kLatImpPairRow = 1u << 31;
constexpr int kLatRxShift = 25;
constexpr uint32_t kLatRxMask = 0x1fu;  // 4s <= 24

LAT_HD int lat_slot(uint32_t e) { return (int)(e & kLatSlotMask); }
LAT_HD int lat_row(uint32_t e) { return (int)((e >> kLatRowShift) & kLatRowMask); }
LAT_HD int lat_dym(uint64_t nb) { return (int)(int16_t)(uint16_t)(nb & 0xffffu); }
LAT_HD int lat_dyp(uint64_t nb) { return (int)(int16_t)(uint16_t)((nb >> 16) & 0xffffu); }
LAT_HD int lat_dzm(uint64_t nb) { return (int)(int16_t)(uint16_t)((nb >> 32) & 0xffffu); }
LAT_HD int lat_dzp(uint64_t nb) { return (int)(int16_t)(uint16_t)((nb >> 48) & 0xffffu); }
LAT_HD int lat_row_base(uint32_t xy) { return (int)(int16_t)(xy & 0xffffu); }
// x offset from the region's centre, plus 2s
LAT_HD int lat_rx2s(uint32_t e) { return (int)((e >> kLatRxShift) & kLatRxMask); }
// A row index's y offset plus 2s, row / (4s + 1), by one multiply and shift:
// exact for every row index below (4s + 1)^2 with m = lat_row_div(s) (the
// table builder checks it); the z offset plus 2s is row - (4s + 1) y.
LAT_HD unsigned lat_row_div(int s) { return (65536u + 4u * (unsigned)s) / (4u * (unsigned)s + 1u); }
LAT_HD int lat_row_y2s(int row, unsigned m) { return (int)(((unsigned)row * m) >> 16); }

struct LatticeTables {
    int s = 0, K = 0;             // K = 4s levels per region
    int n_slots = 0, n_foot = 0;  // phi slots (footprint + halo), (pi, c) slots
    int rb_side = 0;              // 4s + 1: rows are indexed (ry + 2s) rb_side + rz + 2s
    std::vector<uint64_t> row_nb;   // rb_side^2
    std::vector<int32_t> row_pc;    // rb_side^2
    std::vector<uint32_t> row_xy;   // rb_side^2
    int bank_a = 0, bank_b = 0;     // slot residue rx + a ry + b rz mod 16
    std::vector<uint32_t> cell;     // level k: cell[cell_off[k] .. cell_off[k] + cell_n[k]), padded
    std::vector<int32_t> cell_off, cell_n;  // K + 1 offsets (multiples of 4), K counts
    std::vector<uint32_t> imp;      // before level k: imp[imp_off[k] .. imp_off[k] + imp_n[k]), padded
    std::vector<int32_t> imp_off, imp_n;
    std::vector<uint32_t> imp_all;  // pairs (entry, level k) of every import, address order
    int max_cell_n = 0, max_imp_n = 0;  // padded to multiples of 4
    // one whole region: site-updates, bytes read and written (this design)
    int64_t updates = 0, bytes_read = 0, bytes_written = 0;
    int64_t imports_full = 0, imports_phi = 0, exports_phi = 0, exports_pc = 0;
    int max_level_cells = 0;
    int foot_cells = 0, halo_cells = 0;  // footprint and halo cells (slots without padding)
    // offset of the cell in slot sl of row `row` from the region's centre
    void offset_of(int sl, int row, int *rx, int *ry, int *rz) const
    {
        const uint32_t xy = row_xy[row];
        *rx = sl - lat_row_base(xy);
        *ry = (int)((xy >> 16) & 31u) - 2 * s;
        *rz = (int)((xy >> 21) & 31u) - 2 * s;
    }
};

// Site-updates and bytes moved by one region column (one region position in
// every layer) of a call of T levels: regions cut by the call's first level
// also load their level-(k_lo - 1) cells whole (24 bytes each), regions cut by
// its last level export their top level's cells whole (24 bytes each; cells
// already flagged are not counted twice).  Every layer has the same number
// of regions, so bytes / updates is the call's bytes per site-update.
struct LatCallStats {
    int64_t updates = 0, bytes_read = 0, bytes_written = 0;
};
LatCallStats lattice_call_stats(const LatticeTables &t, int64_t T);

// Builds the tables of lattice size s (kLatMinS..kLatMaxS) and checks them:
// the cell count 16 s^4; that every value a level reads is in shared memory
// from the previous level or imported before it; that every import is
// exported by the region that computes it (located through the lattice);
// the packing ranges.  Returns an empty string on success.
std::string build_lattice_tables(int s, LatticeTables *t);

// ---- the regions of one call (host and device) ----
//
// A call advances levels t0 + 1 .. t0 + T.  The lattice is aligned to the
// call: layer L's regions start at relative level tau_b = 1 + s L (tau =
// t - t0), so layers L = -3 .. floor((T - 1) / s) intersect the call; the
// first three are cut by the call's first level and the last few by its
// last level.  A cut region computes its levels k_lo .. k_hi only: it loads
// its level-(k_lo - 1) cells whole from the state at t0, and at k_hi < 4s - 1
// exports the whole state of its level-k_hi cells (the state at t0 + T).
struct LatGeom {
    int s, M[3];  // N_d = 4 s M_d
};

LAT_HD int lat_layer_count(int s, int64_t T) { return (int)((T - 1) / s) + 4; }
LAT_HD int lat_min_layer() { return -3; }
LAT_HD int64_t lat_per_layer(const LatGeom &g) { return 4ll * g.M[0] * g.M[1] * g.M[2]; }

// Layer numbering across calls.  Done flags hold absolute layer numbers and
// are never cleared: a call of `layers` layers numbers them
// last + 1 .. last + layers (last: the largest number used before, 0
// initially, with flags starting at 0), so every wait of the call (for layer
// number >= its first + 1 ... ) is above every value a previous call wrote.
LAT_HD void lat_next_epoch(int *last, int layers, int *first)
{
    *first = *last + 1;
    *last += layers;
}

// Centre of region idx of layer L in units of s: a_d in [0, 4 M_d), all
// congruent to L mod 2, a_0 + a_1 + a_2 congruent to -L mod 4.  (I: the
// index type; the kernel uses 32-bit indices within one simulation.)
template <class I>
LAT_HD void lat_centre(const LatGeom &g, int L, I idx, int a[3])
{
    const int p = L & 1;
    const int q = ((-L - 3 * p) & 3) >> 1;  // parity of a'_0 + a'_1 + a'_2, a_d = 2 a'_d + p
    const I h = idx % (I)g.M[0];
    const I rest = idx / (I)g.M[0];
    const int b1 = (int)(rest % (I)(2 * g.M[1]));
    const int b2 = (int)(rest / (I)(2 * g.M[1]));
    const int b0 = 2 * (int)h + ((q + b1 + b2) & 1);
    a[0] = 2 * b0 + p;
    a[1] = 2 * b1 + p;
    a[2] = 2 * b2 + p;
}

// Inverse of lat_centre (a_d reduced mod 4 M_d by the caller).
template <class I>
LAT_HD I lat_index(const LatGeom &g, const int a[3])
{
    const int b0 = a[0] >> 1, b1 = a[1] >> 1, b2 = a[2] >> 1;
    return ((I)b2 * (I)(2 * g.M[1]) + (I)b1) * (I)g.M[0] + (I)(b0 >> 1);
}

// Centre shift (units of s) from a region to its predecessor n - e_i; the
// successor n + e_i is the opposite shift.
LAT_HD void lat_pred_shift(int i, int d[3])
{
    d[0] = (i == 0 || i == 1) ? -1 : 1;
    d[1] = (i == 0 || i == 2) ? -1 : 1;
    d[2] = (i == 0 || i == 3) ? -1 : 1;
}

LAT_HD int lat_wrap(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Index of the predecessor n - e_i of the region with centre a (layer L) in
// layer L - 1.
template <class I>
LAT_HD I lat_pred_of(const LatGeom &g, const int a[3], int i)
{
    int b[3], d[3];
    lat_pred_shift(i, d);
    for (int k = 0; k < 3; ++k) b[k] = lat_wrap(a[k] + d[k], 4 * g.M[k]);
    return lat_index<I>(g, b);
}

// Index of the predecessor n - e_i of region (L, idx) in layer L - 1.
template <class I>
LAT_HD I lat_pred(const LatGeom &g, int L, I idx, int i)
{
    int a[3];
    lat_centre(g, L, idx, a);
    return lat_pred_of<I>(g, a, i);
}

}  // namespace sp
