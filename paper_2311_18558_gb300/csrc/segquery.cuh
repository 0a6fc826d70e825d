// Exact segment and ray queries against the scene's BVH, shared by the diffuse
// (next-event estimation) and diffraction tracers: an FP32 prefilter whose error
// margins are bounded, and the FP64 watertight test (Woop, Benthin and Wald,
// JCGT 2013; triangles grown by DF_TRI_TOL, as the specular tracer and the
// oracle) wherever the prefilter cannot decide.  Included by one translation
// unit each (everything is in an unnamed namespace).
#pragma once

#include <cuda_runtime.h>

#include "rt_internal.cuh"

namespace {

constexpr double DF_TRI_TOL = 1e-9;    // relative growth of every triangle (as the specular tracer)
constexpr double DF_TIE_TOL = 1e-12;   // relative t-difference treated as a tie
constexpr int DF_STACK = 64;
constexpr int DF_MAX_VISITS = 1 << 20;

// ------------------------------------------------------------------ FP64 rays
struct Ray64 {
    double o[3], d[3];
    int kx, ky, kz;
    double Sx, Sy, Sz;
    float3 of, inv;   // FP32 origin and reciprocal direction for the box tests
};

// FP32 origin and reciprocal direction of the box tests.
__device__ __forceinline__ void ray64_init_box(Ray64& r) {
    r.of = make_float3((float)r.o[0], (float)r.o[1], (float)r.o[2]);
    float inv[3];
    for (int k = 0; k < 3; ++k) {
        const float dk = (float)r.d[k];
        inv[k] = 1.0f / (fabsf(dk) < 1e-30f ? copysignf(1e-30f, dk) : dk);
    }
    r.inv = make_float3(inv[0], inv[1], inv[2]);
}

// Axis permutation and shear of the FP64 watertight test.
__device__ __forceinline__ void ray64_init_shear(Ray64& r) {
    const double ax = fabs(r.d[0]), ay = fabs(r.d[1]), az = fabs(r.d[2]);
    int kz = 0;
    if (ay > ax) kz = 1;
    if (az > (kz == 0 ? ax : ay)) kz = 2;
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    if (r.d[kz] < 0.0) {
        const int s = kx;
        kx = ky;
        ky = s;
    }
    r.kx = kx;
    r.ky = ky;
    r.kz = kz;
    r.Sx = r.d[kx] / r.d[kz];
    r.Sy = r.d[ky] / r.d[kz];
    r.Sz = 1.0 / r.d[kz];
}

__device__ __forceinline__ void ray64_init(Ray64& r) {
    ray64_init_shear(r);
    ray64_init_box(r);
}

// Watertight ray/triangle test in FP64 (Woop, Benthin and Wald, JCGT 2013) with
// the scaled barycentrics allowed down to -DF_TRI_TOL (|U| + |V| + |W|); a ray in
// the triangle's plane misses.  On a hit returns true and t = T / det.
__device__ __forceinline__ bool tri_hit64(const Ray64& r, float4 p0, float4 p1, float4 p2, double& t) {
    const double A[3] = {(double)p0.x - r.o[0], (double)p0.y - r.o[1], (double)p0.z - r.o[2]};
    const double B[3] = {(double)p1.x - r.o[0], (double)p1.y - r.o[1], (double)p1.z - r.o[2]};
    const double C[3] = {(double)p2.x - r.o[0], (double)p2.y - r.o[1], (double)p2.z - r.o[2]};
    const double Ax = A[r.kx] - r.Sx * A[r.kz], Ay = A[r.ky] - r.Sy * A[r.kz];
    const double Bx = B[r.kx] - r.Sx * B[r.kz], By = B[r.ky] - r.Sy * B[r.kz];
    const double Cx = C[r.kx] - r.Sx * C[r.kz], Cy = C[r.ky] - r.Sy * C[r.kz];
    const double U = Cx * By - Cy * Bx, V = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
    const double m = DF_TRI_TOL * (fabs(U) + fabs(V) + fabs(W));
    if ((U < -m || V < -m || W < -m) && (U > m || V > m || W > m)) return false;
    const double det = U + V + W;
    if (!(fabs(det) > 3.0 * m)) return false;
    const double T = U * (r.Sz * A[r.kz]) + V * (r.Sz * B[r.kz]) + W * (r.Sz * C[r.kz]);
    t = T / det;
    return true;
}

// FP32 slab test of one child box over [tlo, thi] (boxes carry a 4e-6 diag pad,
// far above the rounding of the FP32 ray).
__device__ __forceinline__ bool box32(const Ray64& r, float lx, float ly, float lz, float hx, float hy, float hz,
                                      float tlo, float thi) {
    const float tx0 = (lx - r.of.x) * r.inv.x, tx1 = (hx - r.of.x) * r.inv.x;
    const float ty0 = (ly - r.of.y) * r.inv.y, ty1 = (hy - r.of.y) * r.inv.y;
    const float tz0 = (lz - r.of.z) * r.inv.z, tz1 = (hz - r.of.z) * r.inv.z;
    const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tlo));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), thi));
    return tn <= tf;
}

// BVH walk with a per-thread stack; leaf(first, count) returns true to stop.
// `thi` may be lowered by the leaf callback.  Visits are bounded.
template <typename Leaf>
__device__ __forceinline__ void walk(const BvhNode* __restrict__ nodes, const Ray64& r, float tlo, const float& thi,
                                     int32_t* status, Leaf&& leaf) {
    int stack[DF_STACK];
    int sp = 0, ref = 0, visits = 0;
    for (;;) {
        // descend until this lane holds a leaf, so that a warp's lanes test their
        // leaves together ("while-while" order; the nodes and their order per lane
        // are those of a one-node-per-step loop)
        while (ref >= 0) {
            if (++visits > DF_MAX_VISITS) {
                rt_set_status(status, RT_ERR_ITER_LIMIT);
                return;
            }
            const float4* np = reinterpret_cast<const float4*>(nodes + ref);
            const float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2);
            const int4 d = __ldg(reinterpret_cast<const int4*>(np + 3));
            const bool h0 = box32(r, a.x, a.y, a.z, a.w, b.x, b.y, tlo, thi);
            const bool h1 = box32(r, b.z, b.w, c.x, c.y, c.z, c.w, tlo, thi);
            if (h0 && h1) {
                if (sp >= DF_STACK) {
                    rt_set_status(status, RT_ERR_STACK_OVERFLOW);
                    return;
                }
                stack[sp++] = d.y;
                ref = d.x;
            } else if (h0 || h1) {
                ref = h0 ? d.x : d.y;
            } else {
                if (sp == 0) return;
                ref = stack[--sp];
            }
        }
        if (++visits > DF_MAX_VISITS) {
            rt_set_status(status, RT_ERR_ITER_LIMIT);
            return;
        }
        const int e = ~ref;
        if (leaf(e >> 3, (e & 7) + 1)) return;
        if (sp == 0) return;
        ref = stack[--sp];
    }
}

// FP32 upper end of a box interval that covers the FP64 parameter t.
__device__ __forceinline__ float up32(double t) { return __double2float_ru(t) * (1.0f + 1e-6f) + 1e-30f; }

// FP32 copy of a ray for the prefilter of the any-hit queries.
struct Ray32 {
    float o[3], d[3];
    int kx, ky, kz;
    float Sx, Sy, Sz;
};

__device__ __forceinline__ void ray32_set(float3 o, float3 d, Ray32& q) {
    q.o[0] = o.x;
    q.o[1] = o.y;
    q.o[2] = o.z;
    q.d[0] = d.x;
    q.d[1] = d.y;
    q.d[2] = d.z;
    const float ax = fabsf(q.d[0]), ay = fabsf(q.d[1]), az = fabsf(q.d[2]);
    int kz = 0;
    if (ay > ax) kz = 1;
    if (az > (kz == 0 ? ax : ay)) kz = 2;
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    if (q.d[kz] < 0.0f) {
        const int s = kx;
        kx = ky;
        ky = s;
    }
    q.kx = kx;
    q.ky = ky;
    q.kz = kz;
    q.Sx = q.d[kx] / q.d[kz];
    q.Sy = q.d[ky] / q.d[kz];
    q.Sz = 1.0f / q.d[kz];
}

// FP32 watertight test of a segment query: 0 = a miss of the FP64 test for
// certain, 1 = a hit of the FP64 test with tlo < t < thi for certain, 2 =
// undecided.  The FP32 ray differs from the FP64 one by the rounding of its
// origin and direction; with u = 2^-24 the sheared coordinates carry errors below
// 4u (M_v + M_o) (M_v = max over the vertices of |X_kx| + |X_ky| + |X_kz| (|S_x| + |S_y|),
// M_o the same of the origin), so the edge functions are off by less than
// 2u (4 L^2 + 16 (M_v + M_o) L) (L the largest sheared coordinate); the margin is
// that plus twice the FP64 test's growth DF_TRI_TOL (|U| + |V| + |W|).  The
// parameter t is trusted to 64u (M_v + M_o) / |d_kz| plus 1e-6.
struct Edge32 {
    float U, V, W, m;   // edge functions and their error margin
    float Akz, Bkz, Ckz, Mv, Mo;
};

__device__ __forceinline__ Edge32 edges32(const Ray32& r, float4 p0, float4 p1, float4 p2) {
    const float A[3] = {p0.x - r.o[0], p0.y - r.o[1], p0.z - r.o[2]};
    const float B[3] = {p1.x - r.o[0], p1.y - r.o[1], p1.z - r.o[2]};
    const float C[3] = {p2.x - r.o[0], p2.y - r.o[1], p2.z - r.o[2]};
    Edge32 e;
    e.Akz = A[r.kz];
    e.Bkz = B[r.kz];
    e.Ckz = C[r.kz];
    const float Ax = A[r.kx] - r.Sx * e.Akz, Ay = A[r.ky] - r.Sy * e.Akz;
    const float Bx = B[r.kx] - r.Sx * e.Bkz, By = B[r.ky] - r.Sy * e.Bkz;
    const float Cx = C[r.kx] - r.Sx * e.Ckz, Cy = C[r.ky] - r.Sy * e.Ckz;
    e.U = Cx * By - Cy * Bx;
    e.V = Ax * Cy - Ay * Cx;
    e.W = Bx * Ay - By * Ax;
    const float Sab = fabsf(r.Sx) + fabsf(r.Sy);
    e.Mv = fmaxf(fmaxf(fabsf(A[r.kx]) + fabsf(A[r.ky]) + fabsf(e.Akz) * Sab,
                       fabsf(B[r.kx]) + fabsf(B[r.ky]) + fabsf(e.Bkz) * Sab),
                 fabsf(C[r.kx]) + fabsf(C[r.ky]) + fabsf(e.Ckz) * Sab);
    e.Mo = fabsf(r.o[r.kx]) + fabsf(r.o[r.ky]) + fabsf(r.o[r.kz]) * Sab;
    const float L = fmaxf(fmaxf(fmaxf(fabsf(Ax), fabsf(Ay)), fmaxf(fabsf(Bx), fabsf(By))), fmaxf(fabsf(Cx), fabsf(Cy)));
    const float sum = fabsf(e.U) + fabsf(e.V) + fabsf(e.W);
    const float u = 5.9604645e-8f;
    e.m = 2.0f * u * (4.0f * L * L + 16.0f * (e.Mv + e.Mo) * L) + 2.0f * (float)DF_TRI_TOL * sum;
    return e;
}

// The line of the ray passes outside the triangle for certain (edge functions of
// both signs beyond the margin): the FP64 test misses too.
__device__ __forceinline__ bool certain_miss32(const Edge32& e) {
    return (e.U < -e.m || e.V < -e.m || e.W < -e.m) && (e.U > e.m || e.V > e.m || e.W > e.m);
}

__device__ __forceinline__ int tri_seg32(const Ray32& r, float4 p0, float4 p1, float4 p2, float tlo, float thi) {
    const Edge32 e = edges32(r, p0, p1, p2);
    if (certain_miss32(e)) return 0;
    const float m = e.m;
    const bool pos = e.U > m && e.V > m && e.W > m, neg = e.U < -m && e.V < -m && e.W < -m;
    if (!pos && !neg) return 2;
    const float u = 5.9604645e-8f;
    const float t = (e.U * e.Akz + e.V * e.Bkz + e.W * e.Ckz) * r.Sz / (e.U + e.V + e.W);
    const float tt = 64.0f * u * (e.Mv + e.Mo) * fabsf(r.Sz) + 1e-6f;
    if (t > tlo + tt && t < thi - tt) return 1;
    if (t < tlo - tt || t > thi + tt) return 0;
    return 2;
}

// Closest hit with t > tmin, skipping triangle `skip` (original ids): the
// smallest t, then among hits within DF_TIE_TOL of it the lowest triangle id.
// The FP64 test runs only on triangles that the FP32 edge test (q: the ray's
// FP32 copy) does not place outside for certain.
__device__ int closest_hit64(const BvhNode* __restrict__ nodes, const float4* __restrict__ tris, const Ray64& r,
                             const Ray32& q, double tmin, int skip, double& t_out, int32_t* status) {
    double bt = INFINITY;
    float thi = INFINITY;
    walk(nodes, r, (float)tmin * 0.5f, thi, status, [&](int first, int count) {
        for (int k = first; k < first + count; ++k) {
            const float4 p0 = __ldg(tris + 3 * k);
            if (__float_as_int(p0.w) == skip) continue;
            const float4 p1 = __ldg(tris + 3 * k + 1), p2 = __ldg(tris + 3 * k + 2);
            if (certain_miss32(edges32(q, p0, p1, p2))) continue;
            double t;
            if (!tri_hit64(r, p0, p1, p2, t)) continue;
            if (t > tmin && t < bt) {
                bt = t;
                thi = up32(bt + DF_TIE_TOL * bt);
            }
        }
        return false;
    });
    t_out = bt;
    if (!(bt < INFINITY)) return -1;
    const double tmax = bt + DF_TIE_TOL * bt;
    const float thi2 = up32(tmax);
    int best = -1;
    walk(nodes, r, (float)tmin * 0.5f, thi2, status, [&](int first, int count) {
        for (int k = first; k < first + count; ++k) {
            const float4 p0 = __ldg(tris + 3 * k);
            const int id = __float_as_int(p0.w);
            if (id == skip || (best >= 0 && id >= best)) continue;
            const float4 p1 = __ldg(tris + 3 * k + 1), p2 = __ldg(tris + 3 * k + 2);
            if (certain_miss32(edges32(q, p0, p1, p2))) continue;
            double t;
            if (!tri_hit64(r, p0, p1, p2, t)) continue;
            if (t > tmin && t <= tmax) best = id;
        }
        return false;
    });
    return best;
}

// Any hit with tlo < t < thi, skipping triangles `skip` and `skip2` and every
// triangle in the plane `pl0` or `pl1` (plane ids, the .w of a triangle's second
// vertex record) of a segment end, which the segment meets only at that end:
// FP32 prefilter, FP64 test only where the prefilter is undecided.
// The segment is origin + t d, t in (eps / |d|, 1 - eps / |d|); len2f is |d|^2
// from the FP32 direction (the FP32 bounds only), the FP64 |d| is formed from r.d;
// only r.o and r.d need to be set: the FP64 shear and bounds are formed the first
// time a triangle is undecided (most queries never need them).
__device__ bool any_hit_seg(const BvhNode* __restrict__ nodes, const float4* __restrict__ tris, Ray64& r,
                            float3 o32, float3 d32, float len2f, double eps, int skip, int32_t* status,
                            int skip2 = -1, int pl0 = -1, int pl1 = -1) {
    r.of = o32;
    {
        const float dk[3] = {d32.x, d32.y, d32.z};
        float inv[3];
        for (int k = 0; k < 3; ++k) inv[k] = 1.0f / (fabsf(dk[k]) < 1e-30f ? copysignf(1e-30f, dk[k]) : dk[k]);
        r.inv = make_float3(inv[0], inv[1], inv[2]);
    }
    Ray32 q;
    ray32_set(o32, d32, q);
    bool hit = false, fp64_ready = false;
    double tlo = 0.0, thi = 0.0;
    const float flo = (float)eps * rsqrtf(len2f), fthi = 1.0f - flo;
    const float fhi = fthi * (1.0f + 1e-6f) + 1e-30f;
    walk(nodes, r, flo * 0.5f, fhi, status, [&](int first, int count) {
        for (int k = first; k < first + count; ++k) {
            const float4 p0 = __ldg(tris + 3 * k);
            if (__float_as_int(p0.w) == skip || __float_as_int(p0.w) == skip2) continue;
            const float4 p1 = __ldg(tris + 3 * k + 1);
            const int pid = __float_as_int(p1.w);
            if (pid == pl0 || pid == pl1) continue;
            const float4 p2 = __ldg(tris + 3 * k + 2);
            const int c = tri_seg32(q, p0, p1, p2, flo, fthi);
            if (c == 0) continue;
            if (c == 1) {
                hit = true;
                return true;
            }
            if (!fp64_ready) {
                ray64_init_shear(r);
                const double len = sqrt(r.d[0] * r.d[0] + r.d[1] * r.d[1] + r.d[2] * r.d[2]);
                tlo = eps / len;
                thi = 1.0 - tlo;
                fp64_ready = true;
            }
            double t;
            if (!tri_hit64(r, p0, p1, p2, t)) continue;
            if (t > tlo && t < thi) {
                hit = true;
                return true;
            }
        }
        return false;
    });
    return hit;
}

}  // namespace
