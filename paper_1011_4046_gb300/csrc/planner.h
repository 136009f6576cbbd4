// planner.h -- host-side region planner: split tiling of spacetime into
// causally closed regions, their dependency pattern and the tables that move
// surface data between them.
//
// Geometry (paper Sec. 2, Fig. 1 and Fig. 2).  The paper cuts spacetime by
// null surfaces into regions that take information only through initial
// surfaces and emit it only through final surfaces; in 1+1 dimensions these
// are the diamonds of its Fig. 1.  With the 7-point stencil information moves
// one cell per step along each axis, so along one axis a band of H = B/2 steps
// splits into
//
//   upright pyramids   U_j: cells [c_j + k, c_j + B - k)  at level k = 1..H
//   inverted pyramids  I_j: cells [c_j - k, c_j + k)      at level k = 1..H
//
// with c_j = o_b + j B and band offset o_b = (b mod 2) H.  A 3-D region is the
// product of one 1-D piece per axis: its type S is the set of axes along which
// it is inverted (8 types; S = {} is the pyramid, S = {x,y,z} the inverted
// pyramid, the rest are wedges).  At every level the 8 types tile the periodic
// grid exactly, and the tops of the inverted pyramids of band b are exactly
// the bases of the pyramids of band b+1 (the 1-D diamonds of Fig. 1).
//
// Dependencies.  A region of type S needs final-surface cells of regions of
// type S' strictly contained in S in the same band (its sloped initial
// surfaces) and the tops of the inverted pyramids of band b-1 (its base).  So
// a band runs in four phases |S| = 0, 1, 2, 3, the analogue of the four
// layers of regions active at any time in the paper's 4-cube lattice
// (Sec. 2, Fig. 2).  Periodicity is obtained by index wrap-around mod the
// number of regions per axis (Sec. 2.2).
//
// Local coordinates.  A region's cells and halo live in a (B+2)^3 box in
// shared memory; along axis d, u = r + 1 for an upright axis and
// u = r + H + 1 for an inverted axis, r being the offset from c_j.  (pi, c)
// are kept for the region's own B^3 cells only, index (u - 1) per axis.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace sp {

constexpr int kTypes = 8;
constexpr int kMaxB = 32;
constexpr int kMaxH = kMaxB / 2;
constexpr int kMaxSameSucc = 26;
constexpr int kMaxNextSucc = 27;

inline bool inverted(int S, int d) { return (S >> d) & 1; }

struct Box3 {
    int32_t lo[3], hi[3];  // half-open
    int64_t volume() const
    {
        int64_t v = 1;
        for (int d = 0; d < 3; ++d) v *= (hi[d] > lo[d] ? hi[d] - lo[d] : 0);
        return v;
    }
};

// One cell written by a producer into one consumer's mailbox.
struct ExportEntry {
    int32_t src;      // phi index | pc index << 16 (pc index 0xFFFF: phi only)
    int32_t code;     // consumer type | consumer offset bits << 3 (bit d: j_d + 1)
    int32_t dst_phi;  // float2 offset in the consumer's mailbox
    int32_t dst_pc;   // float2 offset of the (pi, c) pair, or -1
};

struct Succ {
    int8_t type, e[3];  // successor type and position offset (added to j)
};

// Everything the region kernel needs for one base size B.
struct TileTables {
    int B = 0, H = 0, P = 0;
    int32_t levels[kTypes];                    // levels computed by a region of type S
    Box3 active[kTypes][kMaxH + 1];            // u-box of the cells computed at level k
    Box3 base_phi[kTypes], base_pc[kTypes];    // u-boxes read from the band base
    // sloped initial surfaces (consumer side), level L = 1..H-1
    std::vector<int32_t> imp_full, imp_phi;
    int32_t imp_full_off[kTypes][kMaxH], imp_full_n[kTypes][kMaxH];
    int32_t imp_phi_off[kTypes][kMaxH], imp_phi_n[kTypes][kMaxH];
    int32_t mb_level_off[kTypes][kMaxH];       // float2 offset of level L's chunk
    int32_t mb_size[kTypes];                   // float2 elements per mailbox
    // final surfaces (producer side), level L = 1..H-1
    std::vector<ExportEntry> exp;
    int32_t exp_off[kTypes][kMaxH], exp_n[kTypes][kMaxH];
    // dependency pattern
    int32_t same_preds[kTypes], prev_preds[kTypes];
    std::vector<Succ> same_succ[kTypes];
    std::vector<Succ> next_succ[2];            // of an inverted pyramid, by parity of the next band
    // With one mailbox slot for all bands, region (b, S, j) must finish
    // before the band-(b+1) regions that write the same addresses (its
    // same-band predecessors' positions one band later) start.  These
    // mailbox-reuse edges (b+1, type, j + offset) are kept only where the
    // rest of the DAG does not already imply them; a region of type S' in
    // band b+1 has reuse_preds[S'] of them.
    std::vector<Succ> reuse_succ[kTypes];
    int32_t reuse_preds[kTypes];
    // traffic of this design per region, and site-updates per region
    int64_t bytes_read[kTypes], bytes_written[kTypes], updates[kTypes];
};

// Offsets of the 1-D owner of relative cell r at level L (1 <= L <= H) in
// the same band: returns true for an inverted piece, and its index offset.
bool owner_1d(int r, int L, int B, int *delta);

// One region split over a 2 x 2 x 2 cluster of CTAs, one octant each (the
// region's cells on one side of its centre along every axis; the centre is
// c_j for an inverted axis and c_j + H for an upright one).  Every octant is
// described in its own mirrored coordinates: dist = r for the upper half
// (r >= 0) and -1 - r for the lower one, so dist grows away from the centre
// and the octant's active cells at level k form the corner box
// dist < w(k) along each axis, w = k (inverted axis) or H - k (upright): the
// same box in all eight octants.  Buffer coordinate u = dist + 1 in
// [0, H + 2): u = 0 is the inner halo (the neighbouring octant's dist = 0
// layer, received from that CTA every level), u = H + 1 the outer halo.
//
// The tables below are those of the octant whose every dist equals r (the
// upper one along every axis); by the mirror symmetry they serve all eight.
// Imports are the region's imports that fall in the octant (the mailbox of a
// region is eight equal octant mailboxes, each laid out like the B <= 16
// ones).  An export entry names the consumer by its type and the set G of
// axes along which the consumer's octant differs from the producer's
// (consumer octant = producer octant ^ G).  Its position differs from the
// producer's only along the axes of F = (consumer type) ^ (producer type):
// there it is one further exactly when the producer's octant bit equals G's
// bit (producer upper and consumer lower octant, or, for the outer halo of
// the last level, producer lower and consumer lower).
struct OctTables {
    int B = 0, H = 0, P = 0;                   // P = H + 2 (buffer side)
    int32_t levels[kTypes];
    int32_t w[kTypes][kMaxH + 2][3];           // active widths at level k (0 = none)
    Box3 active[kTypes][kMaxH + 2];            // u-box [1, w + 1) of level k
    Box3 base_phi[kTypes], base_pc[kTypes];    // u-boxes read from the band base
    std::vector<int32_t> imp_full, imp_phi;    // (pc index << 16 | phi index), phi index
    int32_t imp_full_off[kTypes][kMaxH], imp_full_n[kTypes][kMaxH];
    int32_t imp_phi_off[kTypes][kMaxH], imp_phi_n[kTypes][kMaxH];
    int32_t mb_level_off[kTypes][kMaxH];       // float2 offset of level L's chunk in an octant mailbox
    int32_t mb_size[kTypes];                   // float2 elements per octant mailbox (16-byte multiple)
    // exports: code = consumer type | G << 3; dst offsets in the consumer octant's mailbox
    std::vector<ExportEntry> exp;
    int32_t exp_off[kTypes][kMaxH], exp_n[kTypes][kMaxH];
    // imported cells of level L on the inner faces (dist_d = 0 along some
    // axis d, inside the next level's box along the others): phi index | axis
    // mask << 16; the CTA sends them to its neighbours with its own face cells
    std::vector<int32_t> face_imp;
    int32_t face_imp_off[kTypes][kMaxH], face_imp_n[kTypes][kMaxH];
    // per region (all eight octants): traffic and site-updates
    int64_t bytes_read[kTypes], bytes_written[kTypes], updates[kTypes];
};

// Builds and self-checks the octant tables of base B (B a multiple of 4,
// 8 <= B <= 32) from the region tables t of the same base (its dependency
// pattern is the region's).  Returns an empty string on success.
std::string build_octant_tables(const TileTables &t, OctTables *o);

// Builds and self-checks the tables for base size B (even, 4 <= B <= 32).
// Returns an empty string on success or a description of the failed check.
std::string build_tables(int B, TileTables *t);

// Region counts and HBM traffic for a whole grid at base B.
struct PlanStats {
    int64_t regions_per_band, bands, updates_per_band;
    int64_t bytes_read_per_band, bytes_written_per_band;
    double bytes_per_update;
};
PlanStats plan_stats(const TileTables &t, const int n[3]);

}  // namespace sp
