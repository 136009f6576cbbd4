// sp_device.cuh -- device-side descriptors and PTX helpers shared by the
// kernels and the host API.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "planner.h"
#include "sp_update.h"

namespace sp {

// Geometry and surface-routing tables for one base size, in device memory.
struct TablesDev {
    int B, H, P, pad;
    int levels[kTypes];
    Box3 active[kTypes][kMaxH + 1];
    Box3 base_phi[kTypes], base_pc[kTypes];
    int imp_full_off[kTypes][kMaxH], imp_full_n[kTypes][kMaxH];
    int imp_phi_off[kTypes][kMaxH], imp_phi_n[kTypes][kMaxH];
    int mb_level_off[kTypes][kMaxH];
    int mb_size[kTypes];
    int exp_off[kTypes][kMaxH], exp_n[kTypes][kMaxH];
    int same_preds[kTypes], prev_preds[kTypes];
    int n_same_succ[kTypes];
    Succ same_succ[kTypes][kMaxSameSucc];
    Succ next_succ[2][kMaxNextSucc];
    const int *imp_full;
    const int *imp_phi;
    const int4 *exp;
};

// One simulation of a batch, as the persistent region kernel sees it.
struct SimDev {
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
    float2 *phi, *pi, *c;   // caller-owned state, x fastest
    float2 *mbox;           // mailbox ring (2 band slots)
    long long mb_slot;      // float2 elements per band slot
    long long mb_type_off[kTypes];
    const TablesDev *tab;
};

// Work-queue control block.
struct Ctl {
    unsigned int head;   // next queue position to pop
    unsigned int tail;   // next queue position to push
    int error;           // first device error (0 = none)
    int error_info;
    unsigned long long wait_limit_ns;  // per-wait bound for every spin
    unsigned int completed;            // regions finished
    unsigned int pad;
};

struct RegionArgs {
    const SimDev *sims;
    int n_sims;
    unsigned total;  // regions in this launch
    unsigned n_seed; // regions ready at the start
    int *counters;   // unfinished predecessors per region
    int *queue;      // ready regions in release order (-1 = not yet pushed)
    Ctl *ctl;
    unsigned long long *trace;  // optional (start, end) globaltimer per region
};

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

__device__ __forceinline__ int ld_relaxed_gpu(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int atom_add_acq_rel_gpu(int *p, int v)
{
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Asynchronous global -> shared copies (the copy engine of each SM; no
// register staging).  8-byte copies go through L1 (.ca is the only mode for
// that size); 16-byte copies bypass it (.cg).
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

#endif

}  // namespace sp
