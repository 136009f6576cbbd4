// sp_noalloc.cu -- whole-grid evolution that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they want to
// advance a field: applications that hand out all device memory through
// their own fixed pools or arenas and forbid other allocations, plug-ins and
// callbacks that must not grow the process's device footprint, and code on a
// latency-critical path where an allocation (and the synchronisation it can
// imply) is not acceptable.  sp_sweep_noalloc serves them.  It runs
// the same whole-grid leapfrog steps as sp_evolve(..., SP_MONOLITHIC) with
// the same kernel and coefficients, so its results are bit-identical.  The
// only scratch it needs lives in this file: a phi ping-pong buffer and the
// per-level coefficients, both in file-scope device arrays of fixed size.
// Every GPU that loads the library holds these arrays until the process exits.
// The host side uses no heap either: the coefficients are computed in
// fixed-size chunks on the stack and reach the device as kernel arguments of
// a small fill kernel, so no host buffer has to outlive the call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "sp.h"
#include "sp_device.cuh"
#include "sp_kernels.h"

namespace {

constexpr int64_t kMaxSites = SP_NOALLOC_MAX_SITES;
constexpr int64_t kMaxSteps = SP_NOALLOC_MAX_STEPS;
constexpr int kMaxDevices = 64;

// The scratch.  In host code these names are host-side stand-ins, not device
// addresses: the device addresses come from cudaGetSymbolAddress below.
static __device__ __align__(256) float2 g_phi_scratch[kMaxSites];
static __device__ __align__(256) sp::LevelCoef g_coef_scratch[kMaxSteps];

// Coefficients handed to the device by value, kCoefChunk levels per launch
// (3.8 KB of kernel arguments, under the 4 KB that every launch accepts).
constexpr int kCoefChunk = 240;
struct CoefChunk {
    sp::LevelCoef c[kCoefChunk];
};

__global__ void fill_coef_kernel(CoefChunk chunk, int first, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) g_coef_scratch[first + i] = chunk.c[i];
}

struct ScratchAddr {
    float2 *phi = nullptr;
    sp::LevelCoef *coef = nullptr;
    bool ready = false;
};
ScratchAddr g_addr[kMaxDevices];
std::mutex g_addr_lock;

// Device addresses of the scratch on the current device, looked up once.
int scratch_for_current_device(ScratchAddr *out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SP_ECUDA;
    std::lock_guard<std::mutex> lock(g_addr_lock);
    ScratchAddr &a = g_addr[dev];
    if (!a.ready) {
        void *p = nullptr, *c = nullptr;
        if (cudaGetSymbolAddress(&p, g_phi_scratch) != cudaSuccess) return SP_ECUDA;
        if (cudaGetSymbolAddress(&c, g_coef_scratch) != cudaSuccess) return SP_ECUDA;
        a.phi = static_cast<float2 *>(p);
        a.coef = static_cast<sp::LevelCoef *>(c);
        a.ready = true;
    }
    *out = a;
    return SP_OK;
}

// Per-level coefficients, computed in FP64 and rounded to FP32 once (the same
// arithmetic as the grid path's table).
sp::LevelCoef level_coef(const sp_params &p, int64_t level, double *stiff)
{
    const bool damping = level < p.damp_steps;
    const double tau = damping ? p.tau0 : p.tau0 + (double)(level - p.damp_steps) * p.dt;
    const double ratio = tau / p.tau_ref;
    double a = 1.0;
    const double nu_i = std::floor(p.nu);
    if (p.nu == nu_i && p.nu >= 0 && p.nu <= 16)
        for (int i = 0; i < (int)nu_i; ++i) a *= ratio;
    else
        a = std::pow(ratio, p.nu);
    const double d = damping ? 1.0 : p.nu * p.dt / tau;
    sp::LevelCoef c;
    c.c1 = (float)((1.0 - d) / (1.0 + d));
    c.c2 = (float)(p.dt / (1.0 + d));
    c.m = (float)(a * a * p.lambda);
    c.pad = 0.0f;
    *stiff = p.dt * p.dt * (12.0 / (p.dx * p.dx) + 2.0 * p.lambda * p.eta * p.eta * a * a);
    return c;
}

}  // namespace

extern "C" int sp_sweep_noalloc(const sp_params *p, void *phi_dev, void *pic_dev, int64_t level0, int64_t n_steps,
                                void *cuda_stream)
{
    if (!p || !phi_dev || !pic_dev || level0 < 0 || n_steps < 0) return SP_EINVAL;
    if (((uintptr_t)phi_dev & 7u) || ((uintptr_t)pic_dev & 15u)) return SP_EINVAL;
    // each side bounded before the product is formed (no overflow), as in
    // sp_grid_create
    for (int d = 0; d < 3; ++d)
        if (p->n[d] < 4 || p->n[d] > (1 << 14)) return SP_EINVAL;
    if (!(p->dx > 0) || !(p->dt > 0) || !(p->lambda >= 0) || !(p->eta >= 0) || !(p->nu >= 0) || !(p->tau0 > 0) ||
        !(p->tau_ref > 0) || p->damp_steps < 0 || p->precision != SP_FP32_KAHAN)
        return SP_EINVAL;
    const int64_t sites = (int64_t)p->n[0] * p->n[1] * p->n[2];
    if (sites > kMaxSites || n_steps > kMaxSteps) return SP_ESCRATCH;
    if (n_steps == 0) return SP_OK;

    for (int64_t k = 0; k < n_steps; ++k) {  // every level stable before any work is enqueued
        double stiff = 0.0;
        level_coef(*p, level0 + k, &stiff);
        if (!(stiff < 4.0)) return SP_EUNSTABLE;
    }
    ScratchAddr s;
    int rc = scratch_for_current_device(&s);
    if (rc != SP_OK) return rc;

    cudaStream_t st = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSuccess;
    for (int64_t first = 0; first < n_steps && e == cudaSuccess; first += kCoefChunk) {
        const int count = (int)std::min<int64_t>(kCoefChunk, n_steps - first);
        CoefChunk chunk;
        double stiff = 0.0;
        for (int i = 0; i < kCoefChunk; ++i)
            chunk.c[i] = i < count ? level_coef(*p, level0 + first + i, &stiff) : sp::LevelCoef{0.0f, 0.0f, 0.0f, 0.0f};
        fill_coef_kernel<<<(count + 127) / 128, 128, 0, st>>>(chunk, (int)first, count);
        e = cudaGetLastError();
    }
    sp::PhysConst q;
    q.dt = (float)p->dt;
    q.inv_dx2 = (float)(1.0 / (p->dx * p->dx));
    q.eta2 = (float)(p->eta * p->eta);
    q.pad = 0.0f;
    float2 *phi = static_cast<float2 *>(phi_dev), *a = phi, *b = s.phi;
    float4 *pic = static_cast<float4 *>(pic_dev);
    for (int64_t k = 0; k < n_steps && e == cudaSuccess; ++k) {
        e = sp::launch_sweep(a, b, pic, p->n, s.coef, (int)k, q, st);
        float2 *t = a;
        a = b;
        b = t;
    }
    if (e == cudaSuccess && a != phi) e = cudaMemcpyAsync(phi, a, (size_t)sites * sizeof(float2), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? SP_OK : SP_ECUDA;
}
