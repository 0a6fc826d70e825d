// FP32 complex helpers and the Fresnel reflection coefficients (Eq. fresnel-1/2
// of arXiv 2311.18558) with their derivatives, shared by the specular and the
// diffuse field kernels.
#pragma once
#include <cuda_runtime.h>

static __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
static __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
static __device__ __forceinline__ float2 cscale(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
// The hardware's approximate reciprocal and square root (PTX rcp.approx.ftz,
// sqrt.approx.ftz: a few units in the last place), several times cheaper than
// the correctly rounded forms and well inside the FP32 accuracy of the field
// chain.  Their arguments here are O(1e-3 .. 1e6), far from subnormals.
static __device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
static __device__ __forceinline__ float sqrt_fast(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Principal square root from |z|: sqrt(z) = t + j y/(2t) with t = sqrt((|z| + x)/2)
// for x >= 0, and the mirrored form for x < 0 (no cancellation either way).
// |z| of eta - sin^2 is O(1..1e3), so sqrt(x^2 + y^2) needs no scaling.
static __device__ __forceinline__ float2 csqrt(float2 z) {
    const float r = sqrt_fast(z.x * z.x + z.y * z.y);
    if (z.x >= 0.0f) {
        const float t = sqrt_fast(0.5f * (r + z.x));
        return make_float2(t, t > 0.0f ? z.y * rcp_fast(2.0f * t) : 0.0f);
    }
    const float t = sqrt_fast(0.5f * (r - z.x));
    return make_float2(fabsf(z.y) * rcp_fast(2.0f * t), copysignf(t, z.y));
}

// 1 / z = conj(z) / |z|^2 with one reciprocal (|z|^2 of the Fresnel denominators
// stays far from FP32 over- and underflow)
static __device__ __forceinline__ float2 crcp(float2 z) {
    const float inv = rcp_fast(z.x * z.x + z.y * z.y);
    return make_float2(z.x * inv, -z.y * inv);
}

// Fresnel coefficients (Eq. fresnel-1/2) and their derivatives w.r.t. eta, with
// s = sqrt(eta - sin^2 theta), c = cos theta, and p = 1 / (c + s),
// l = 1 / (eta c + s), 1 / s shared:
//   r_perp = (c - s) p,  r_par = (eta c - s) l,
//   d r_perp / d eta = -c p^2 / s,  d r_par / d eta = c (eta - 2 sin^2) l^2 / s.
template <bool GRAD>
static __device__ __forceinline__ void fresnel(float2 eta, float c, float2& rp, float2& rl, float2& drp, float2& drl) {
    const float s2 = fmaxf(0.0f, 1.0f - c * c);
    const float2 s = csqrt(make_float2(eta.x - s2, eta.y));
    const float2 ip = crcp(make_float2(c + s.x, s.y));
    rp = cmul(make_float2(c - s.x, -s.y), ip);
    const float2 ec = cscale(c, eta);
    const float2 il = crcp(cadd(ec, s));
    rl = cmul(make_float2(ec.x - s.x, ec.y - s.y), il);
    if (GRAD) {
        const float2 is = crcp(s);
        drp = cscale(-c, cmul(cmul(ip, ip), is));
        drl = cmul(cscale(c, make_float2(eta.x - 2.0f * s2, eta.y)), cmul(cmul(il, il), is));
    }
}

