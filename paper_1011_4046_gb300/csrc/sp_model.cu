// sp_model.cu -- the region cost model: a 16-64-64-1 ReLU network trained on
// measured region times, and the bucketing of a launch's regions by its
// predictions (the learned ordering of the device queue).
//
// The paper's manager issues regions so that expensive ones do not finish
// last (Sec. 4; uneven region costs, Sec. 6).  Here the network predicts the
// log of a region's time from 16 features (feature_kernel in sp_kernels.cu);
// regions go into one of four priority buckets and the persistent kernel pops
// the highest non-empty bucket first.  Only the schedule changes, never the
// arithmetic of a region, so results stay bit-identical.
//
// Kernels (FP32, hand-written):
//   mlp_forward_kernel  one thread per sample, parameters in shared memory;
//   mlp_bucket_kernel   forward + thresholds -> priority bucket per region;
//   mlp_grad_kernel     per block of <= 128 samples: forward, reverse pass and
//                       the block's sum of parameter gradients of the mean
//                       squared error, in a fixed order (deterministic);
//   grad_reduce_kernel  sums the blocks' partial gradients in block order;
//   adam_kernel         one Adam step per parameter (Kingma & Ba 2015).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "sp.h"
#include "sp_device.cuh"

namespace {

constexpr int kIn = 16, kHid = 64;
constexpr int kW1 = 0, kB1 = kW1 + kHid * kIn, kW2 = kB1 + kHid, kB2 = kW2 + kHid * kHid, kW3 = kB2 + kHid,
              kB3 = kW3 + kHid, kParams = kB3 + 1;
static_assert(kParams == SP_MODEL_PARAMS, "parameter count");
constexpr int kGradBlock = 128;   // samples per gradient block
constexpr int kPitch = kGradBlock + 1;  // sample-minor rows, padded against bank conflicts

__device__ __forceinline__ void load_params(float *s, const float *theta)
{
    for (int i = threadIdx.x; i < kParams; i += blockDim.x) s[i] = theta[i];
}

// Forward pass of one sample with the parameters in shared memory.
__device__ __forceinline__ float mlp_forward_one(const float *__restrict__ P, const float *__restrict__ x)
{
    float in[kIn];
#pragma unroll
    for (int i = 0; i < kIn; ++i) in[i] = x[i];
    float h1[kHid];
#pragma unroll
    for (int j = 0; j < kHid; ++j) {
        float z = P[kB1 + j];
#pragma unroll
        for (int i = 0; i < kIn; ++i) z = fmaf(P[kW1 + j * kIn + i], in[i], z);
        h1[j] = fmaxf(z, 0.0f);
    }
    float y = P[kB3];
    for (int j = 0; j < kHid; ++j) {
        float z = P[kB2 + j];
#pragma unroll
        for (int i = 0; i < kHid; ++i) z = fmaf(P[kW2 + j * kHid + i], h1[i], z);
        y = fmaf(P[kW3 + j], fmaxf(z, 0.0f), y);
    }
    return y;
}

__global__ void __launch_bounds__(128) mlp_forward_kernel(const float *__restrict__ theta, const float *__restrict__ X,
                                                          long long n, float *__restrict__ out)
{
    __shared__ float P[kParams];
    load_params(P, theta);
    __syncthreads();
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) out[s] = mlp_forward_one(P, X + kIn * s);
}

// Bucket of each region: 0 for a prediction >= thr[0] (most expensive), 1 for
// >= thr[1], 2 for >= thr[2], else 3.
__global__ void __launch_bounds__(128) mlp_bucket_kernel(const float *__restrict__ theta, const float *__restrict__ thr,
                                                         const float *__restrict__ X, long long n,
                                                         unsigned char *__restrict__ prio)
{
    __shared__ float P[kParams];
    load_params(P, theta);
    __syncthreads();
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float y = mlp_forward_one(P, X + kIn * s);
    prio[s] = (unsigned char)(y >= thr[0] ? 0 : (y >= thr[1] ? 1 : (y >= thr[2] ? 2 : 3)));
}

// Gradient of L = (1/n) sum (yhat - y)^2 over the samples idx[0..count) (or
// 0..count when idx is null), block b taking samples [128 b, 128 b + 128).
// partial[b][p] = block b's share of dL/dtheta_p; partial[b][kParams] = its
// share of L.  Shared memory: the parameters, then sample-minor arrays
// x[16], h1[64], h2[64], dL/dz1[64], dL/dz2[64], dL/dyhat, r^2/n.
__global__ void __launch_bounds__(kGradBlock) mlp_grad_kernel(const float *__restrict__ theta,
                                                              const float *__restrict__ X, const float *__restrict__ Y,
                                                              const int *__restrict__ idx, int count, float inv_n,
                                                              float *__restrict__ partial)
{
    extern __shared__ float sm[];
    float *P = sm;
    float *xs = P + kParams;
    float *h1s = xs + kIn * kPitch;
    float *h2s = h1s + kHid * kPitch;
    float *g1s = h2s + kHid * kPitch;
    float *g2s = g1s + kHid * kPitch;
    float *gos = g2s + kHid * kPitch;
    float *ls = gos + kPitch;
    load_params(P, theta);
    __syncthreads();
    const int t = threadIdx.x;
    const int k = blockIdx.x * kGradBlock + t;
    if (k < count) {
        const long long s = idx ? idx[k] : k;
        const float *x = X + kIn * s;
        float in[kIn];
#pragma unroll
        for (int i = 0; i < kIn; ++i) {
            in[i] = x[i];
            xs[i * kPitch + t] = in[i];
        }
        unsigned long long m1 = 0ull, m2 = 0ull;  // ReLU masks
        for (int j = 0; j < kHid; ++j) {
            float z = P[kB1 + j];
#pragma unroll
            for (int i = 0; i < kIn; ++i) z = fmaf(P[kW1 + j * kIn + i], in[i], z);
            if (z > 0.0f) m1 |= 1ull << j;
            h1s[j * kPitch + t] = fmaxf(z, 0.0f);
        }
        float yhat = P[kB3];
        for (int j = 0; j < kHid; ++j) {
            float z = P[kB2 + j];
            for (int i = 0; i < kHid; ++i) z = fmaf(P[kW2 + j * kHid + i], h1s[i * kPitch + t], z);
            if (z > 0.0f) m2 |= 1ull << j;
            const float h = fmaxf(z, 0.0f);
            h2s[j * kPitch + t] = h;
            yhat = fmaf(P[kW3 + j], h, yhat);
        }
        const float r = yhat - Y[s];
        const float go = 2.0f * r * inv_n;
        gos[t] = go;
        ls[t] = r * r * inv_n;
        for (int j = 0; j < kHid; ++j) g2s[j * kPitch + t] = ((m2 >> j) & 1ull) ? go * P[kW3 + j] : 0.0f;
        for (int i = 0; i < kHid; ++i) {
            float gh = 0.0f;
            for (int j = 0; j < kHid; ++j) gh = fmaf(P[kW2 + j * kHid + i], g2s[j * kPitch + t], gh);
            g1s[i * kPitch + t] = ((m1 >> i) & 1ull) ? gh : 0.0f;
        }
    } else {
        for (int i = 0; i < kIn; ++i) xs[i * kPitch + t] = 0.0f;
        for (int j = 0; j < kHid; ++j) {
            h1s[j * kPitch + t] = 0.0f;
            h2s[j * kPitch + t] = 0.0f;
            g1s[j * kPitch + t] = 0.0f;
            g2s[j * kPitch + t] = 0.0f;
        }
        gos[t] = 0.0f;
        ls[t] = 0.0f;
    }
    __syncthreads();
    float *out = partial + (size_t)blockIdx.x * (kParams + 1);
    for (int p = t; p <= kParams; p += kGradBlock) {
        const float *a, *b = nullptr;  // sum over samples of a[s] * b[s] (b null: of a[s])
        if (p < kB1) {
            a = g1s + (p / kIn) * kPitch;
            b = xs + (p % kIn) * kPitch;
        } else if (p < kW2) {
            a = g1s + (p - kB1) * kPitch;
        } else if (p < kB2) {
            a = g2s + ((p - kW2) / kHid) * kPitch;
            b = h1s + ((p - kW2) % kHid) * kPitch;
        } else if (p < kW3) {
            a = g2s + (p - kB2) * kPitch;
        } else if (p < kB3) {
            a = gos;
            b = h2s + (p - kW3) * kPitch;
        } else if (p == kB3) {
            a = gos;
        } else {
            a = ls;
        }
        float acc = 0.0f;
        if (b)
            for (int s = 0; s < kGradBlock; ++s) acc = fmaf(a[s], b[s], acc);
        else
            for (int s = 0; s < kGradBlock; ++s) acc += a[s];
        out[p] = acc;
    }
}

__global__ void grad_reduce_kernel(const float *__restrict__ partial, int blocks, float *__restrict__ grad,
                                   float *__restrict__ loss_out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kParams) return;
    float acc = 0.0f;
    for (int b = 0; b < blocks; ++b) acc += partial[(size_t)b * (kParams + 1) + p];
    if (p < kParams)
        grad[p] = acc;
    else if (loss_out)
        *loss_out = acc;
}

__global__ void adam_kernel(float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ grad, float lr, float beta1, float beta2, float eps, float c1,
                            float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kParams) return;
    const float g = grad[p];
    const float mp = beta1 * m[p] + (1.0f - beta1) * g;
    const float vp = beta2 * v[p] + (1.0f - beta2) * g * g;
    m[p] = mp;
    v[p] = vp;
    theta[p] -= lr * (mp * c1) / (sqrtf(vp * c2) + eps);
}

size_t grad_smem_bytes() { return sizeof(float) * (kParams + (kIn + 4 * kHid) * kPitch + 2 * kPitch); }

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) as a counter-based stream:
// output i of the stream at `seed` is mix(seed + (i + 1) * golden).
uint64_t splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double uniform01(uint64_t seed, uint64_t i) { return (double)(splitmix64(seed, i) >> 11) * 0x1.0p-53; }

}  // namespace

struct sp_model {
    cudaStream_t stream = nullptr;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *thr = nullptr;
    float *partial = nullptr;
    size_t cap_partial = 0;
    float *losses = nullptr;
    size_t cap_losses = 0;
    int *order = nullptr;
    size_t cap_order = 0;
    int64_t adam_t = 0;
    float thr_host[3] = {0.0f, 0.0f, 0.0f};
};

namespace {

template <class T>
cudaError_t grow_buf(T **p, size_t *cap, size_t need)
{
    if (*cap >= need && *p) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(need, 1) * sizeof(T));
    if (e == cudaSuccess) *cap = std::max<size_t>(need, 1);
    return e;
}

int upload_params(sp_model *m, const float *host)
{
    cudaError_t e = cudaMemcpyAsync(m->theta, host, kParams * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, kParams * sizeof(float), m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, kParams * sizeof(float), m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->thr, m->thr_host, 3 * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    m->adam_t = 0;
    return e == cudaSuccess ? SP_OK : SP_ECUDA;
}

// Gradient of the mean squared error over `count` samples into m->grad and
// the loss into *loss_dev (device, may be null).
int enqueue_grad(sp_model *m, const float *X, const float *Y, const int *idx, int count, float *loss_dev)
{
    const int blocks = (count + kGradBlock - 1) / kGradBlock;
    if (grow_buf(&m->partial, &m->cap_partial, (size_t)blocks * (kParams + 1)) != cudaSuccess) return SP_ENOMEM;
    const size_t smem = grad_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return SP_ECUDA;
    mlp_grad_kernel<<<blocks, kGradBlock, smem, m->stream>>>(m->theta, X, Y, idx, count, 1.0f / (float)count,
                                                              m->partial);
    grad_reduce_kernel<<<(kParams + 1 + 255) / 256, 256, 0, m->stream>>>(m->partial, blocks, m->grad, loss_dev);
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

}  // namespace

extern "C" {

int sp_model_create(uint64_t seed, void *cuda_stream, sp_model **out)
{
    if (!out) return SP_EINVAL;
    *out = nullptr;
    sp_model *m = new (std::nothrow) sp_model();
    if (!m) return SP_ENOMEM;
    m->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMalloc((void **)&m->theta, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->m, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->v, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->grad, kParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->thr, 3 * sizeof(float));
    if (e != cudaSuccess) {
        sp_model_destroy(m);
        return SP_ENOMEM;
    }
    // He-uniform weights: parameter k draws uniform k of the stream; a weight
    // of a layer with fan-in f is (2u - 1) sqrt(6 / f) in FP64, rounded once.
    std::vector<float> init(kParams, 0.0f);
    const int layer_off[3] = {kW1, kW2, kW3}, fan_in[3] = {kIn, kHid, kHid}, count[3] = {kHid * kIn, kHid * kHid, kHid};
    for (int l = 0; l < 3; ++l)
        for (int i = 0; i < count[l]; ++i) {
            const int k = layer_off[l] + i;
            init[k] = (float)((2.0 * uniform01(seed, (uint64_t)k) - 1.0) * std::sqrt(6.0 / fan_in[l]));
        }
    const int rc = upload_params(m, init.data());
    if (rc != SP_OK) {
        sp_model_destroy(m);
        return rc;
    }
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
        sp_model_destroy(m);
        return SP_ECUDA;
    }
    *out = m;
    return SP_OK;
}

int sp_model_destroy(sp_model *m)
{
    if (!m) return SP_EINVAL;
    cudaFree(m->theta);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->grad);
    cudaFree(m->thr);
    cudaFree(m->partial);
    cudaFree(m->losses);
    cudaFree(m->order);
    delete m;
    return SP_OK;
}

int sp_model_get_params(sp_model *m, float *params_host, float *thresholds_host)
{
    if (!m || !params_host) return SP_EINVAL;
    cudaError_t e = cudaMemcpyAsync(params_host, m->theta, kParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return SP_ECUDA;
    if (thresholds_host) std::memcpy(thresholds_host, m->thr_host, sizeof m->thr_host);
    return SP_OK;
}

int sp_model_set_params(sp_model *m, const float *params_host, const float *thresholds_host)
{
    if (!m || !params_host) return SP_EINVAL;
    if (thresholds_host) {
        if (!(thresholds_host[0] >= thresholds_host[1] && thresholds_host[1] >= thresholds_host[2])) return SP_EINVAL;
        std::memcpy(m->thr_host, thresholds_host, sizeof m->thr_host);
    }
    const int rc = upload_params(m, params_host);
    if (rc != SP_OK) return rc;
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? SP_OK : SP_ECUDA;
}

int sp_model_predict(sp_model *m, const float *x_dev, int64_t n, float *y_dev)
{
    if (!m || n < 0 || (n > 0 && (!x_dev || !y_dev))) return SP_EINVAL;
    if (n == 0) return SP_OK;
    mlp_forward_kernel<<<(unsigned)((n + 127) / 128), 128, 0, m->stream>>>(m->theta, x_dev, n, y_dev);
    if (cudaGetLastError() != cudaSuccess) return SP_ECUDA;
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? SP_OK : SP_ECUDA;
}

int sp_model_grad(sp_model *m, const float *x_dev, const float *y_dev, int64_t n, float *grad_host, double *loss)
{
    if (!m || n < 1 || n > (1 << 24) || !x_dev || !y_dev || !grad_host) return SP_EINVAL;
    if (grow_buf(&m->losses, &m->cap_losses, 1) != cudaSuccess) return SP_ENOMEM;
    int rc = enqueue_grad(m, x_dev, y_dev, nullptr, (int)n, m->losses);
    if (rc != SP_OK) return rc;
    float l = 0.0f;
    cudaError_t e = cudaMemcpyAsync(grad_host, m->grad, kParams * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, m->losses, sizeof l, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return SP_ECUDA;
    if (loss) *loss = l;
    return SP_OK;
}

int sp_model_adam_step(sp_model *m, const float *grad_host, float lr, float beta1, float beta2, float eps)
{
    if (!m || !grad_host || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return SP_EINVAL;
    cudaError_t e = cudaMemcpyAsync(m->grad, grad_host, kParams * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) return SP_ECUDA;
    ++m->adam_t;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)m->adam_t)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)m->adam_t)));
    adam_kernel<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->theta, m->m, m->v, m->grad, lr, beta1, beta2, eps,
                                                              c1, c2);
    if (cudaGetLastError() != cudaSuccess) return SP_ECUDA;
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? SP_OK : SP_ECUDA;
}

int sp_model_train(sp_model *m, const float *x_dev, const float *y_dev, int64_t n, int32_t epochs, int32_t batch,
                   float lr, uint64_t order_seed, const int32_t *order_host, float *losses_host)
{
    if (!m || !x_dev || !y_dev || n < 1 || n > (1 << 24) || epochs < 1 || batch < 1 || batch > (1 << 20) || !(lr > 0))
        return SP_EINVAL;
    const size_t total = (size_t)n * (size_t)epochs;
    std::vector<int> order(total);
    if (order_host) {
        for (size_t i = 0; i < total; ++i) {
            if (order_host[i] < 0 || order_host[i] >= n) return SP_EINVAL;
            order[i] = order_host[i];
        }
    } else {
        // epoch e: the stable argsort of uniforms 2^42 + e 2^32 + i of the stream
        std::vector<std::pair<double, int>> key((size_t)n);
        for (int ep = 0; ep < epochs; ++ep) {
            for (int64_t i = 0; i < n; ++i)
                key[(size_t)i] = {uniform01(order_seed, (1ull << 42) + ((uint64_t)ep << 32) + (uint64_t)i), (int)i};
            std::stable_sort(key.begin(), key.end(),
                             [](const std::pair<double, int> &a, const std::pair<double, int> &b) { return a.first < b.first; });
            for (int64_t i = 0; i < n; ++i) order[(size_t)ep * n + i] = key[(size_t)i].second;
        }
    }
    const int64_t per_epoch = (n + batch - 1) / batch;
    const size_t steps = (size_t)per_epoch * epochs;
    if (grow_buf(&m->order, &m->cap_order, total) != cudaSuccess) return SP_ENOMEM;
    if (grow_buf(&m->losses, &m->cap_losses, steps) != cudaSuccess) return SP_ENOMEM;
    cudaError_t e = cudaMemcpyAsync(m->order, order.data(), total * sizeof(int), cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) return SP_ECUDA;
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    size_t step = 0;
    for (int ep = 0; ep < epochs; ++ep)
        for (int64_t s0 = 0; s0 < n; s0 += batch, ++step) {
            const int count = (int)std::min<int64_t>(batch, n - s0);
            int rc = enqueue_grad(m, x_dev, y_dev, m->order + (size_t)ep * n + s0, count, m->losses + step);
            if (rc != SP_OK) return rc;
            ++m->adam_t;
            const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, (double)m->adam_t)));
            const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, (double)m->adam_t)));
            adam_kernel<<<(kParams + 255) / 256, 256, 0, m->stream>>>(m->theta, m->m, m->v, m->grad, lr, beta1, beta2,
                                                                      eps, c1, c2);
        }
    if (cudaGetLastError() != cudaSuccess) return SP_ECUDA;
    if (losses_host) {
        e = cudaMemcpyAsync(losses_host, m->losses, steps * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
        if (e != cudaSuccess) return SP_ECUDA;
    }
    // bucket thresholds: quartiles of the trained network's predictions on the training set
    std::vector<float> pred((size_t)n);
    float *d_pred = nullptr;
    if (cudaMalloc((void **)&d_pred, (size_t)n * sizeof(float)) != cudaSuccess) return SP_ENOMEM;
    mlp_forward_kernel<<<(unsigned)((n + 127) / 128), 128, 0, m->stream>>>(m->theta, x_dev, n, d_pred);
    e = cudaMemcpyAsync(pred.data(), d_pred, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    cudaFree(d_pred);
    if (e != cudaSuccess) return SP_ECUDA;
    std::sort(pred.begin(), pred.end());
    for (int q = 0; q < 3; ++q) m->thr_host[q] = pred[(size_t)((n - 1) * (3 - q) / 4)];
    e = cudaMemcpyAsync(m->thr, m->thr_host, 3 * sizeof(float), cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? SP_OK : SP_ECUDA;
}

// File: "SPMLP001", int32 parameter count, float params[count], float thresholds[3].
int sp_model_save(sp_model *m, const char *path)
{
    if (!m || !path) return SP_EINVAL;
    std::vector<float> p(kParams);
    int rc = sp_model_get_params(m, p.data(), nullptr);
    if (rc != SP_OK) return rc;
    FILE *f = std::fopen(path, "wb");
    if (!f) return SP_EINVAL;
    const int32_t cnt = kParams;
    bool ok = std::fwrite("SPMLP001", 1, 8, f) == 8 && std::fwrite(&cnt, sizeof cnt, 1, f) == 1 &&
              std::fwrite(p.data(), sizeof(float), kParams, f) == (size_t)kParams &&
              std::fwrite(m->thr_host, sizeof(float), 3, f) == 3;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SP_OK : SP_EINVAL;
}

int sp_model_load(const char *path, void *cuda_stream, sp_model **out)
{
    if (!path || !out) return SP_EINVAL;
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return SP_EINVAL;
    char magic[8];
    int32_t cnt = 0;
    std::vector<float> p(kParams);
    float thr[3];
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "SPMLP001", 8) == 0 &&
              std::fread(&cnt, sizeof cnt, 1, f) == 1 && cnt == kParams &&
              std::fread(p.data(), sizeof(float), kParams, f) == (size_t)kParams &&
              std::fread(thr, sizeof(float), 3, f) == 3;
    std::fclose(f);
    if (!ok) return SP_EINVAL;
    sp_model *m = nullptr;
    int rc = sp_model_create(0, cuda_stream, &m);
    if (rc != SP_OK) return rc;
    rc = sp_model_set_params(m, p.data(), thr);
    if (rc != SP_OK) {
        sp_model_destroy(m);
        return rc;
    }
    *out = m;
    return SP_OK;
}

}  // extern "C"

namespace sp {

// Priority bucket of every region of a launch from its features (used by
// sp_evolve with the learned ordering).
cudaError_t model_buckets(const sp_model *m, const float *X, long long n, unsigned char *prio, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    mlp_bucket_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(m->theta, m->thr, X, n, prio);
    return cudaGetLastError();
}

}  // namespace sp
