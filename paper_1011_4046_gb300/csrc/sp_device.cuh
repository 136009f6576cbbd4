// sp_device.cuh -- device-side descriptors and PTX helpers shared by the
// kernels and the host API.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "planner.h"
#include "sp_update.h"

namespace sp {

// Levels per band the device tables hold: bases up to 16 (the kernels decode
// cell indices with shifts of at most 4 bits per axis).
constexpr int kMaxHDev = 8;

// Per-type geometry and routing of one base size (one block per region type,
// so a kernel can keep it in shared memory).
struct alignas(16) TypeMeta {
    int levels, mb_size, n_same_succ, same_preds;
    int prev_preds;
    // band-base copy in units of (column, run of up to 4 cells along z):
    // columns of the base box, runs per column, 1/columns in FP32
    int base_cols, base_runs;
    float rcp_cols;
    Box3 active[kMaxHDev + 1];
    Box3 base_phi, base_pc;
    // exact quotient decode (see fdiv below), reciprocals rounded to FP32:
    // of each active box, 1/(w2/2) and 1/(w0/2) (its cells are taken in
    // 2x2x2 blocks, see block_cell); of the base box, 1/w0 and 1/w1
    float rcp_active[kMaxHDev + 1][2];
    float rcp_base[2];
    int imp_full_off[kMaxHDev], imp_full_n[kMaxHDev];
    int imp_phi_off[kMaxHDev], imp_phi_n[kMaxHDev];
    int mb_level_off[kMaxHDev];
    int exp_off[kMaxHDev], exp_n[kMaxHDev];
    Succ same_succ[kMaxSameSucc];
    // one mailbox slot: mailbox-reuse successors (in TablesDev::reuse) and
    // predecessors of a region of this type in a band after the first
    int n_reuse, reuse_preds;
};

// Geometry and surface-routing tables for one base size, in device memory.
//
// Import lists are 16-bit: a full-state import holds the cell's (pi, c) index
// (its phi index follows from it), a neighbour-only import its phi index.
// All lists of one base size are copied into shared memory once per launch,
// at imp_smem (16-bit units) in the kernel's import area.
//
// Export entries are 8 bytes: x = phi index (13 bits) | (pi, c) shared-memory
// slot (pc_slot of the cell, 12 bits) << 13 | consumer code << 25 (6 bits) |
// has (pi, c) << 31, y = phi offset | (pi, c) offset << 16 in the consumer's
// mailbox (float2 units).  This packing needs (B+2)^3 <= 8192, B^3 <= 4096
// (B <= 16) and mailboxes of at most 65536 float2.
struct alignas(16) TablesDev {
    int B, H, P, pad;
    TypeMeta type[kTypes];
    Succ next_succ[2][kMaxNextSucc];
    int imp_n;      // 16-bit import entries of this base size (padded to 8)
    int imp_smem;   // their offset in the shared import area (16-bit units)
    // mailbox-reuse successors of a type-S region, reuse[S * kMaxSameSucc + i]
    // for i < n_reuse (used with a single mailbox slot), global memory
    const Succ *reuse;
    const unsigned short *imp;  // all import lists, global memory
    const int2 *exp;            // all export entries, global memory
};

// Levels per band of the octant (cluster) kernel: bases up to 32.
constexpr int kMaxHOct = 16;

// Geometry and routing of one region type for the cluster kernel, in the
// mirrored coordinates of one octant (planner.h, OctTables): buffer side
// P = H + 2, u = dist + 1.
struct alignas(16) OctTypeMeta {
    int levels, mb_size;        // levels; float2 elements of one octant mailbox
    int base_cols, base_runs;   // band-base copy in (column, run of up to 4 cells along z) units
    float rcp_cols, rcp_base0;  // 1 / columns, 1 / width of the base box along x
    int pad0, pad1;
    Box3 base_phi, base_pc;
    // widths of the active corner box at level k (0 = none) and the FP32
    // reciprocals of its extents along x and y (exact decode, fdiv)
    unsigned char w[kMaxHOct + 2][4];
    float rcp_w[kMaxHOct + 2][2];
    // face-first order of level k: 1 / w1, 1 / (w0 - 1), 1 / (w1 - 1) (0 where the width is 0)
    float rcp_f[kMaxHOct + 2][3];
    int pad2;
    int imp_full_off[kMaxHOct], imp_full_n[kMaxHOct];
    int imp_phi_off[kMaxHOct], imp_phi_n[kMaxHOct];
    int mb_level_off[kMaxHOct];
    int exp_off[kMaxHOct], exp_n[kMaxHOct];
    int face_off[kMaxHOct], face_n[kMaxHOct];
    int xbytes[kMaxHOct + 2];   // bytes of inner faces an octant receives before level k
};

// Everything the cluster kernel reads for one base (B = 32): per-type
// geometry (copied into shared memory once per launch), the 16-bit import
// lists (shared memory), the export entries and imported face cells
// (global memory, read through L1).  Export entry: x = phi index (13 bits) |
// (pi, c) index (12 bits) << 13 | consumer code (type | G << 3) << 25 |
// has (pi, c) << 31; y = phi offset | (pi, c) offset << 16 in the consumer
// octant's mailbox (float2 units).  Face entry: phi index | axis mask << 16.
struct alignas(16) TablesOct {
    int B, H, P, imp_n;
    OctTypeMeta type[kTypes];
    const unsigned short *imp;
    const int2 *exp;
    const int *face;  // all face entries (face_total, a multiple of 4), copied into shared memory
    int face_total, pad3;
};

// One simulation of a batch, as the persistent region kernel sees it.
struct alignas(16) SimDev {
    int n[3];
    int J[3];
    int Jtot;
    int B, H, P;
    int nbands;
    unsigned tile_base;   // global id of (band 0, type 0, j 0)
    unsigned tiles;       // nbands * 8 * Jtot
    unsigned seed_base;   // queue position of this sim's first ready region
    const LevelCoef *coef;  // coef[l] = coefficients of the l-th level of this call
    PhysConst q;
    float2 *phi;            // caller-owned state, x fastest: phi
    float4 *pc;             // and (pi.re, pi.im, c.re, c.im)
    float2 *mbox;           // mailboxes: a ring of 2 band slots, or 1 slot for every band
    long long mb_slot;      // float2 offset of band slot 1 (0 with a single slot)
    long long mb_type_off[kTypes];
    const TablesDev *tab;
    int tab_index;  // which of the launch's tables (RegionArgs::tabs) this is
    // 1: one mailbox slot for every band; a region also waits for the
    // previous band's readers of the mailboxes it writes (reuse edges)
    int mb_reuse;
    // base 32: the octant tables of the cluster kernel (the dependency
    // pattern stays in tab); nullptr otherwise
    const TablesOct *oct;
    long long pad_oct;
};

// Priority buckets of the learned ordering (bucket 0 is queued first).
constexpr int kBuckets = 4;

// Work-queue control block.  Every manager of the launch takes queue positions
// from head and pushes at tail (one atomic each per region), and polls error
// while it waits: the three sit in 128-byte lines of their own, so that the
// atomics on one do not queue behind those on another at the same L2 slice.
struct alignas(128) Ctl {
    unsigned int head;   // next queue position to pop
    unsigned int pad_head[31];
    unsigned int tail;   // next queue position to push
    unsigned int pad_tail[31];
    int error;           // first device error (0 = none)
    int error_info;
    unsigned long long wait_limit_ns;  // per-wait bound for every spin
    unsigned int bcount[kBuckets];     // learned ordering: band-0 seeds per bucket,
    unsigned int bcursor[kBuckets];    // and the next free position of each bucket's run
    // lattice launches: absolute number of the call's first layer, and the
    // last absolute layer number any call of this control block has used
    // (the reset kernel starts every call above it, so done flags, which
    // only grow, never need clearing)
    int epoch;
    int last_layer;
};

// One simulation of a lattice launch (4-cube regions, lattice.h).
struct alignas(16) LatSimDev {
    int n[3], M[3];             // sides, N_d = 4 s M_d
    long long region_base;      // first region of this simulation within a layer of the launch
    long long per_layer;        // 4 M_0 M_1 M_2
    const LevelCoef *coef;      // coef[tau - 1]: coefficients of relative level tau of this call
    PhysConst q;
    float2 *phi0, *phi1;        // phi at even / odd levels of the call (phi0: the caller's array)
    float4 *pc;                 // (pi, c), one array
    long long trace_base;       // trace / fault-injection id of this simulation's first region
};

// Launch arguments of the lattice kernel.  Regions are handed out by ticket
// in layer order; region t of the launch is region j = t mod per_layer_all
// of layer -3 + t / per_layer_all, j running over the simulations' regions
// in turn.  flags[(layer & 3) * per_layer_all + j] holds the absolute
// number of the last layer whose region j finished.
struct LatArgs {
    const LatSimDev *sims;
    int n_sims, s, K, T;
    int n_slots, n_foot, Lcount, pad0;
    long long fault_drop;            // region id (as in the trace) that never reports done (-1: none)
    unsigned per_layer_all, total;
    const uint32_t *cell;            // cell entries (lattice.h), all levels (16-byte aligned per level)
    const uint2 *imp_all;            // (entry, level) of every import of a region, address order
    const uint64_t *row_nb;          // (4s + 1)^2 row records: neighbour steps
    const int32_t *row_pc;           // (4s + 1)^2 row records: (pi, c) index - slot
    int max_cell_n, n_imp_all;       // longest level's cell list (padded); imports of a region
    int *flags;
    Ctl *ctl;
    unsigned long long *trace;       // optional (start, end) globaltimer per region: simulation by
                                     // simulation, layer by layer (trace_base + layer * per_layer + idx)
    int cell_off[4 * 6 + 1];  // per level (entries)
    int cell_n[4 * 6];
};

struct RegionArgs {
    const SimDev *sims;
    const TablesDev *tabs;  // the distinct tables of the launch, tabs[SimDev::tab_index]
    int n_tabs;
    int n_sims;
    unsigned total;  // regions in this launch
    unsigned n_seed; // regions ready at the start
    int *counters;   // unfinished predecessors per region
    int *queue;      // ready regions in release order (-1 = not yet pushed)
    Ctl *ctl;
    unsigned long long *trace;  // optional (start, end) globaltimer per region
    // Learned ordering: priority bucket of every region (0 first), or nullptr.
    // With it the seeds are queued bucket by bucket and the successors that
    // one finished region makes ready are pushed bucket by bucket.
    const unsigned char *prio;
    // Host-injected failure (failure-detection tests): the region with this
    // launch id finishes but never releases its successors; -1 = none.
    int fault_drop;
    int pad_;
};

static_assert(sizeof(TablesDev) % 16 == 0, "tables are copied in 16-byte units");
static_assert(sizeof(TablesOct) % 16 == 0, "octant tables are copied in 16-byte units");
static_assert(sizeof(SimDev) % 16 == 0, "descriptors are copied in 16-byte units");
static_assert(sizeof(LevelCoef) == 16, "coefficients are copied in 16-byte units");

enum DeviceError { kDevOk = 0, kDevTimeout = 1, kDevBadRegion = 2 };

#if defined(__CUDACC__)

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_acquire_gpu_u(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed_gpu_u(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_gpu(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acquire_cta_shared(const int *p)
{
    int v;
    unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.acquire.cta.shared.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_cta_shared(int *p, int v)
{
    unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("st.release.cta.shared.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Barrier among the nthreads threads (a multiple of 32) that use this id.
__device__ __forceinline__ void named_barrier(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Arrives at named barrier `id` without waiting (producer side of a
// producer / consumer pair; the consumers bar.sync with the same count).
__device__ __forceinline__ void named_arrive(int id, int nthreads)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_gpu(int *p, int v)
{
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int atom_add_acq_rel_gpu(int *p, int v)
{
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Asynchronous global -> shared copies (the copy engine of each SM; no
// register staging).  8-byte copies go through L1 (.ca is the only mode for
// that size); 16-byte copies bypass it (.cg).  The copies carry no compiler
// memory clobber, so independent loads may be scheduled around them; shared
// memory they write is read only after cp_async_wait_* (which has the
// clobber) and a barrier.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Waits until at most n of this thread's committed copy groups are pending.
__device__ __forceinline__ void cp_async_wait_pending(int n)
{
    switch (n) {
#define SP_WAIT_CASE(N)                                                     \
    case N:                                                                 \
        asm volatile("cp.async.wait_group " #N ";\n" ::: "memory");         \
        break;
        SP_WAIT_CASE(0) SP_WAIT_CASE(1) SP_WAIT_CASE(2) SP_WAIT_CASE(3) SP_WAIT_CASE(4) SP_WAIT_CASE(5)
        SP_WAIT_CASE(6) SP_WAIT_CASE(7) SP_WAIT_CASE(8) SP_WAIT_CASE(9) SP_WAIT_CASE(10) SP_WAIT_CASE(11)
        SP_WAIT_CASE(12) SP_WAIT_CASE(13) SP_WAIT_CASE(14) SP_WAIT_CASE(15)
#undef SP_WAIT_CASE
    default:
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
}

// ---- thread-block clusters: distributed shared memory and mbarriers ----
__device__ __forceinline__ unsigned cluster_ctarank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned map_shared(const void *p, unsigned rank)
{
    unsigned a = (unsigned)__cvta_generic_to_shared(p), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init_cluster()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// This thread's arrival on a local mbarrier, announcing `bytes` of
// asynchronous stores the current phase also waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    unsigned a = (unsigned)__cvta_generic_to_shared(bar);
    unsigned long long state;
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state)
                 : "r"(a), "r"(bytes)
                 : "memory");
    asm volatile("" ::"l"(state));
}

// One poll of the phase with parity `parity` (true once it completed);
// acquire at cluster scope, so the stores other CTAs made into this CTA's
// shared memory for that phase are visible to the caller.
__device__ __forceinline__ bool mbar_test_parity_cluster(unsigned long long *bar, unsigned parity)
{
    unsigned a = (unsigned)__cvta_generic_to_shared(bar), ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}

// 8-byte store into another CTA's shared memory (cluster address `raddr`)
// that completes as 8 bytes of transaction count on that CTA's mbarrier
// `rbar` (cluster address).
__device__ __forceinline__ void st_async_f2(unsigned raddr, float2 v, unsigned rbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "f"(v.x), "f"(v.y), "r"(rbar)
                 : "memory");
}

__device__ __forceinline__ void st_release_cluster_shared(unsigned raddr, int v)
{
    asm volatile("st.release.cluster.shared::cluster.s32 [%0], %1;" ::"r"(raddr), "r"(v) : "memory");
}

__device__ __forceinline__ void st_cluster_shared_int4(unsigned raddr, int4 v)
{
    asm volatile("st.shared::cluster.v4.s32 [%0], {%1, %2, %3, %4};" ::"r"(raddr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ int ld_acquire_cluster_shared(const int *p)
{
    int v;
    unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.acquire.cluster.shared::cta.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_cluster_add(unsigned raddr, int v)
{
    asm volatile("red.release.cluster.shared::cluster.add.s32 [%0], %1;" ::"r"(raddr), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

#endif

// floor(i / w) for 0 <= i < 2^20 and 1 <= w <= 64, from rcp = 1/w rounded to
// FP32: (i + 1/2) / w lies at least 1/(2w) away from an integer, and the two
// roundings (of 1/w and of the product) move it by at most about
// 2^-23 (i + 1/2) / w < 1/(2w), so truncation gives the exact quotient.  The
// host checks every (i, w) the tables use with the same operations.
#if defined(__CUDACC__)
__host__ __device__ __forceinline__
#else
inline
#endif
    int fdiv(int i, float rcp)
{
    return (int)(((float)i + 0.5f) * rcp);
}

// Shared-memory slot of the (pi, c) pair of local cell c = (z B + y) B + x
// (B a power of two, lgB = log2 B): bits 1 and 2 of x are flipped by the
// parities of y and z.  A row of cells keeps distinct banks (x is only
// permuted within its row), and so does a 2x2x2 block of cells, whose eight
// float4 slots are then eight different 16-byte bank groups.
#if defined(__CUDACC__)
__host__ __device__ __forceinline__
#else
inline
#endif
    int pc_slot(int c, int lgB, int B)
{
    return c ^ (((((c >> lgB) & 1) << 1) | (((c >> (2 * lgB)) & 1) << 2)) & (B - 1));
}

}  // namespace sp
