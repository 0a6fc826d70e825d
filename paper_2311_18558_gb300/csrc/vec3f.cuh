// FP32 3-vectors and the bases of the per-path geometry records (theta/phi of a
// direction, the perpendicular of a plane of incidence), shared by the specular
// and the diffuse record kernels.
#pragma once
#include <cuda_runtime.h>

struct F3 {
    float x, y, z;
};
static __device__ __forceinline__ F3 f3(float x, float y, float z) { return F3{x, y, z}; }
static __device__ __forceinline__ F3 fsub(F3 a, F3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
static __device__ __forceinline__ F3 fscl(float s, F3 a) { return f3(s * a.x, s * a.y, s * a.z); }
static __device__ __forceinline__ float fdot(F3 a, F3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static __device__ __forceinline__ F3 fcross(F3 a, F3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static __device__ __forceinline__ F3 funit(F3 a) { return fscl(1.0f / sqrtf(fdot(a, a)), a); }

static __device__ __forceinline__ void sph_basis_f(F3 k, F3* th, F3* ph) {
    const float st = sqrtf(k.x * k.x + k.y * k.y);
    float cp = 1.0f, sp = 0.0f;
    if (st > 0.0f) {
        cp = k.x / st;
        sp = k.y / st;
    }
    *th = f3(k.z * cp, k.z * sp, -st);
    *ph = f3(-sp, cp, 0.0f);
}

// unit(k x n), or where k is (numerically) along n, `fb` made orthogonal to k
// (at such incidences every transverse basis gives the same field magnitude).
static __device__ __forceinline__ F3 perp_or_f(F3 k, F3 n, F3 fb) {
    const F3 c = fcross(k, n);
    if (fdot(c, c) > 1e-12f) return funit(c);
    return funit(fsub(fb, fscl(fdot(fb, k), k)));
}

