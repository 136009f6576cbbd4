// sp_peaks.cu -- measured peaks of the on-chip resources the region kernel
// uses, for its roofline lines: shared-memory read bandwidth and FP32 FMA
// throughput of the whole device (HBM bandwidth is measured elsewhere).
//
// Shared memory: every thread of a full-occupancy grid reads eight distinct
// 16-byte words of a 32 KB shared array per step, a warp's 32 reads covering
// 512 consecutive bytes (four wavefronts, no bank conflict), folding them
// into an XOR so that no read can be dropped (the offsets differ, so no two
// reads of a step can be merged, and they move every step).  FP32: eight
// independent fused multiply-add chains per thread.  Both are timed with CUDA
// events around one launch after a warm-up launch; the result is written so
// the compiler must keep the work.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sp.h"

namespace {

constexpr int kPeakThreads = 1024;
constexpr int kSmemWords = 2048;  // float4 words: 32 KB per block

__global__ void __launch_bounds__(kPeakThreads) smem_read_kernel(int iters, unsigned *sink)
{
    __shared__ float4 buf[kSmemWords];
    for (int i = threadIdx.x; i < kSmemWords; i += kPeakThreads)
        buf[i] = make_float4((float)i, (float)(i + 1), (float)(i + 2), (float)(i + 3));
    __syncthreads();
    unsigned acc = 0;
    int idx = threadIdx.x;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float4 v = buf[(idx + u * (kSmemWords / 8)) & (kSmemWords - 1)];  // eight distinct words
            acc ^= __float_as_uint(v.x) ^ __float_as_uint(v.y) ^ __float_as_uint(v.z) ^ __float_as_uint(v.w);
        }
        idx = (idx + 32) & (kSmemWords - 1);
    }
    if (acc == 0x9e3779b9u) sink[blockIdx.x] = acc;  // practically never: keeps the reads alive
}

__global__ void __launch_bounds__(kPeakThreads) fma_kernel(int iters, float *sink)
{
    float a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = (float)(threadIdx.x + u);
    const float b = 0.999f, c = 1e-3f;
#pragma unroll 1
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = __fmaf_rn(a[u], b, c);
    float s = 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += a[u];
    if (s == 12345.678f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int sp_measure_peaks(void *cuda_stream, double *smem_gbs, double *fp32_tflops)
{
    if (!smem_gbs || !fp32_tflops) return SP_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smem_read_kernel, kPeakThreads, 0);
    if (e != cudaSuccess || sms < 1 || per_sm < 1) return SP_ECUDA;
    const int blocks = sms * per_sm;
    void *sink = nullptr;
    e = cudaMalloc(&sink, (size_t)blocks * sizeof(float));
    if (e != cudaSuccess) return SP_ENOMEM;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int smem_iters = 4096, fma_iters = 4096;
    float ms_smem = 0.0f, ms_fma = 0.0f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // warm-up, then timed
        smem_read_kernel<<<blocks, kPeakThreads, 0, st>>>(smem_iters, (unsigned *)sink);
        e = cudaEventRecord(t0, st);
        smem_read_kernel<<<blocks, kPeakThreads, 0, st>>>(smem_iters, (unsigned *)sink);
        if (e == cudaSuccess) e = cudaEventRecord(t1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_smem, t0, t1);
    }
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        fma_kernel<<<blocks, kPeakThreads, 0, st>>>(fma_iters, (float *)sink);
        e = cudaEventRecord(t0, st);
        fma_kernel<<<blocks, kPeakThreads, 0, st>>>(fma_iters, (float *)sink);
        if (e == cudaSuccess) e = cudaEventRecord(t1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_fma, t0, t1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(sink);
    if (e != cudaSuccess || ms_smem <= 0.0f || ms_fma <= 0.0f) return SP_ECUDA;
    const double threads = (double)blocks * kPeakThreads;
    *smem_gbs = threads * smem_iters * 8.0 * 16.0 / (ms_smem * 1e-3) / 1e9;
    *fp32_tflops = threads * fma_iters * 16.0 * 8.0 * 2.0 / (ms_fma * 1e-3) / 1e12;
    return SP_OK;
}
