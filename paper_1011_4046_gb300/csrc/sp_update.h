// sp_update.h -- the FP32 site update shared by every GPU path.
//
// One leapfrog step of the complex string field at one lattice site,
//
//   F   = Lap7(phi) / dx^2 - m (|phi|^2 - eta^2) phi,      m = a_n^2 lambda
//   pi' = c1 pi + c2 F,                                     c1 = (1-d)/(1+d), c2 = dt/(1+d)
//   phi' = phi + dt pi'   (Kahan-compensated, carry c)
//
// with d_n = nu dt / tau_n (the friction term 2 (nu/tau) phi' of the model
// equation, time-centred).  The region kernel and the monolithic sweep both
// call this one function with the same per-level FP32 coefficients, and the
// library is compiled with -fmad=false: the only fused multiply-adds are the
// explicit ones below, so both paths round identically and the region
// decomposition is bit-exact against the sweep.  The order of the Laplacian
// sum is fixed: ((x- + x+) + (y- + y+)) + (z- + z+), then - 6 phi by one fma.
//
// The Kahan carry c holds the negated low-order part lost when dt*pi' was
// added to phi; keeping it per site (8 extra bytes) makes the FP32 position
// sum as accurate as an FP64 one over the run.
//
// On the GPU the real and imaginary parts go through the packed FP32 pipe
// (one f32x2 add, multiply or fused multiply-add for both lanes wherever they
// follow the same formula); each lane rounds as the scalar operation does,
// so the results are those of the scalar form, bit for bit.
#pragma once

#if defined(__CUDACC__)
#define SP_HD __host__ __device__ __forceinline__
#else
#include <cmath>
#define SP_HD inline
#endif

namespace sp {

struct f2 {
    float x, y;
};

SP_HD float fma_rn(float a, float b, float c)
{
#if defined(__CUDA_ARCH__)
    return __fmaf_rn(a, b, c);
#else
    return std::fmaf(a, b, c);
#endif
}

struct LevelCoef {
    float c1, c2, m, pad;
};

struct PhysConst {
    float dt, inv_dx2, eta2, pad;
};

// In: phi and its six neighbours at level n, pi at n-1/2, Kahan carry at n.
// Out: phi at n+1 (returned), pi at n+1/2 and the carry at n+1 (in place).
template <class V2>
SP_HD V2 site_update(V2 phi, V2 xm, V2 xp, V2 ym, V2 yp, V2 zm, V2 zp, V2 &pi, V2 &c,
                     const LevelCoef &k, const PhysConst &q)
{
    float sr = ((xm.x + xp.x) + (ym.x + yp.x)) + (zm.x + zp.x);
    float si = ((xm.y + xp.y) + (ym.y + yp.y)) + (zm.y + zp.y);
    float lr = fma_rn(-6.0f, phi.x, sr) * q.inv_dx2;
    float li = fma_rn(-6.0f, phi.y, si) * q.inv_dx2;
    float s = fma_rn(phi.x, phi.x, fma_rn(phi.y, phi.y, -q.eta2));
    float ms = k.m * s;
    float fr = fma_rn(-ms, phi.x, lr);
    float fi = fma_rn(-ms, phi.y, li);
    pi.x = fma_rn(k.c1, pi.x, k.c2 * fr);
    pi.y = fma_rn(k.c1, pi.y, k.c2 * fi);
    float yr = fma_rn(q.dt, pi.x, -c.x);
    float yi = fma_rn(q.dt, pi.y, -c.y);
    float tr = phi.x + yr;
    float ti = phi.y + yi;
    c.x = (tr - phi.x) - yr;
    c.y = (ti - phi.y) - yi;
    V2 out;
    out.x = tr;
    out.y = ti;
    return out;
}

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
// The packed form of the update above, for float2 on the device.
__device__ __forceinline__ float2 site_update(float2 phi, float2 xm, float2 xp, float2 ym, float2 yp, float2 zm,
                                              float2 zp, float2 &pi, float2 &c, const LevelCoef &k,
                                              const PhysConst &q)
{
    const float2 s = __fadd2_rn(__fadd2_rn(__fadd2_rn(xm, xp), __fadd2_rn(ym, yp)), __fadd2_rn(zm, zp));
    const float2 l = __fmul2_rn(__ffma2_rn(make_float2(-6.0f, -6.0f), phi, s), make_float2(q.inv_dx2, q.inv_dx2));
    const float s2 = fma_rn(phi.x, phi.x, fma_rn(phi.y, phi.y, -q.eta2));
    const float ms = k.m * s2;
    const float2 f = __ffma2_rn(make_float2(-ms, -ms), phi, l);
    pi = __ffma2_rn(make_float2(k.c1, k.c1), pi, __fmul2_rn(make_float2(k.c2, k.c2), f));
    const float2 y = __ffma2_rn(make_float2(q.dt, q.dt), pi, make_float2(-c.x, -c.y));
    const float2 t = __fadd2_rn(phi, y);
    c = __fadd2_rn(__fadd2_rn(t, make_float2(-phi.x, -phi.y)), make_float2(-y.x, -y.y));
    return t;
}
#endif

}  // namespace sp
