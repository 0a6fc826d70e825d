// Specular path tracing on GB300 (Sec. II-F of arXiv 2311.18558):
//   1. SBR: Fibonacci rays bounce specularly over a software BVH in FP32; a ray
//      with any marginal FP32 decision is traced again in FP64;
//   2. dedup: every triangle-sequence prefix goes into an open-addressing hash
//      set, then the unique keys are sorted by (length, lexicographic);
//   3. image method over (candidate, receiver) pairs: FP32 prefilter with a
//      conservative margin; survivors are compacted into a queue;
//   4. per queued pair (dense): FP64 image-method confirmation, then visibility
//      of every segment (FP32 any-hit, FP64 recheck when marginal), recorded in
//      a (receiver x candidate) bitmask;
//   5. deterministic emission: per-receiver popcounts, scan, expansion in
//      candidate order, FP64 points, coplanar-duplicate rule.
//
// GB300 has very little FP64 throughput, and a warp-wide FP64 instruction costs
// the same with one active lane as with 32.  So FP64 work only runs on
// compacted lists (re-traced rays, queued pairs, emitted paths), and it avoids
// IEEE division and square root: reciprocals come from an FP32 seed refined by
// Newton-Raphson, hit tests compare t = T/det by cross-multiplication, and
// length tests compare squared lengths.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <vector>

#include "launch_dir.cuh"
#include "rt_internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;


// Programmatic dependent launch (sm_90 and later): a kernel launched with
// launch_pdl may be launched while the previous kernel of its stream finishes.
// Its first statement, pdl_entry, waits for that kernel's completion and memory
// (griddepcontrol.wait) before anything is read, then lets the next kernel
// launch (griddepcontrol.launch_dependents).  A dependent is launched only once
// every block of this kernel has started, so its waiting blocks never hold
// resources that this kernel's blocks still need.  Launched normally, the wait
// returns at once.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" :::);
}
constexpr int TRACE_THREADS = 128;
constexpr int REDO_THREADS = 32;
constexpr int REDO_BLOCKS_PER_SM = 16;
constexpr float SBR_MARGIN = 1e-3f;     // relative barycentric margin of the FP32 visibility passes
constexpr float PREFILTER_MARGIN = 1e-3f;
// Degenerate geometry: every triangle is closed and grown by TRI_TOL (relative
// barycentric), so a point or ray exactly on an edge shared by two triangles
// belongs to both whatever the rounding; hits whose t differ by at most TIE_TOL
// (relative) are ties, won by the lowest triangle index.
constexpr double TRI_TOL = 1e-9;
constexpr double TIE_TOL = 1e-12;

// ------------------------------------------------------------------ small vectors
template <typename T>
struct V3 {
    T x, y, z;
};
template <typename T>
__device__ __forceinline__ V3<T> mk(T x, T y, T z) { return V3<T>{x, y, z}; }
template <typename T>
__device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
template <typename T>
__device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
template <typename T>
__device__ __forceinline__ V3<T> operator*(T s, V3<T> a) { return mk(s * a.x, s * a.y, s * a.z); }
template <typename T>
__device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
__device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <typename T>
__device__ __forceinline__ T comp(V3<T> a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }
template <typename T>
__device__ __forceinline__ V3<T> from4(float4 v) { return mk((T)v.x, (T)v.y, (T)v.z); }

// 1/x in FP64 without the IEEE division: FP32 reciprocal as seed, then two
// Newton-Raphson steps r <- r + r (1 - x r), each doubling the correct bits
// (24 -> 48 -> full precision).  For the moderate |x| used here.
__device__ __forceinline__ double rcp64(double x) {
    double r = (double)__frcp_rn((float)x);
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

// ------------------------------------------------------------------ watertight ray
template <typename T>
struct WRay {
    V3<T> o, d;
    int kx, ky, kz;
    T Sx, Sy, Sz;
    float3 of, inv;   // FP32 origin and reciprocal direction for the slab tests
    float3 oinv;      // of * inv, so that a slab distance is one FMA: l * inv - oinv
};

template <typename T>
__device__ __forceinline__ T recip(T x);
template <>
__device__ __forceinline__ float recip<float>(float x) { return 1.0f / x; }
template <>
__device__ __forceinline__ double recip<double>(double x) { return rcp64(x); }

template <typename T>
__device__ __forceinline__ void wray_init(WRay<T>& r) {
    T ax = fabs(r.d.x), ay = fabs(r.d.y), az = fabs(r.d.z);
    int kz = 0;
    if (ay > ax) kz = 1;
    if (az > (kz == 0 ? ax : ay)) kz = 2;
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    T dz = comp(r.d, kz);
    if (dz < (T)0) {
        int s = kx;
        kx = ky;
        ky = s;
    }
    r.kx = kx;
    r.ky = ky;
    r.kz = kz;
    T iz = recip<T>(dz);
    r.Sx = comp(r.d, kx) * iz;
    r.Sy = comp(r.d, ky) * iz;
    r.Sz = iz;
    r.of = make_float3((float)r.o.x, (float)r.o.y, (float)r.o.z);
    float dx = (float)r.d.x, dy = (float)r.d.y, dzz = (float)r.d.z;
    r.inv = make_float3(1.0f / (fabsf(dx) < 1e-30f ? copysignf(1e-30f, dx) : dx),
                        1.0f / (fabsf(dy) < 1e-30f ? copysignf(1e-30f, dy) : dy),
                        1.0f / (fabsf(dzz) < 1e-30f ? copysignf(1e-30f, dzz) : dzz));
    r.oinv = make_float3(r.of.x * r.inv.x, r.of.y * r.inv.y, r.of.z * r.inv.z);
}

// Sheared edge functions U, V, W and scaled distance Tn of the watertight
// ray/triangle test (Woop, Benthin, Wald, JCGT 2013); t = Tn / (U + V + W).
template <typename T>
__device__ __forceinline__ void woop(const WRay<T>& r, float4 p0, float4 p1, float4 p2, T& U, T& V, T& W, T& Tn) {
    V3<T> A = from4<T>(p0) - r.o, B = from4<T>(p1) - r.o, C = from4<T>(p2) - r.o;
    T Akz = comp(A, r.kz), Bkz = comp(B, r.kz), Ckz = comp(C, r.kz);
    T Ax = comp(A, r.kx) - r.Sx * Akz, Ay = comp(A, r.ky) - r.Sy * Akz;
    T Bx = comp(B, r.kx) - r.Sx * Bkz, By = comp(B, r.ky) - r.Sy * Bkz;
    T Cx = comp(C, r.kx) - r.Sx * Ckz, Cy = comp(C, r.ky) - r.Sy * Ckz;
    U = Cx * By - Cy * Bx;
    V = Ax * Cy - Ay * Cx;
    W = Bx * Ay - By * Ax;
    Tn = (U * Akz + V * Bkz + W * Ckz) * r.Sz;
}

// FP32 test with an undecided band: 0 = miss, 1 = hit (t_out), 2 = undecided
// (an edge function within `margin` of zero relative to their total magnitude).
__device__ __forceinline__ int tri_test32(const WRay<float>& r, float4 p0, float4 p1, float4 p2, float& t_out) {
    float U, V, W, Tn;
    woop(r, p0, p1, p2, U, V, W, Tn);
    float m = SBR_MARGIN * (fabsf(U) + fabsf(V) + fabsf(W));
    bool pos = U > m && V > m && W > m;
    bool neg = U < -m && V < -m && W < -m;
    float det = U + V + W;
    if (pos || neg) {
        t_out = Tn / det;
        return 1;
    }
    if ((U < -m || V < -m || W < -m) && (U > m || V > m || W > m)) return 0;
    t_out = det != 0.0f ? Tn / det : 0.0f;
    return 2;
}

// tri_test32 for a ray of the FP32 SBR pass with a rigorous undecided band.
// Rounding part: with u = 2^-24 the translated and sheared coordinates carry
// errors below 3u (Mv + Mo), Mv = max over the vertices of |X_kx| + |X_ky| +
// |X_kz| (|S_x| + |S_y|) and Mo the same of the origin, so an edge function is
// off by at most u (4 L^2 + 12 (Mv + Mo) L), L = max |sheared x, y|; Mv is
// bounded here by 2 L + 2 (|S_x| + |S_y|) Z (|X_kx| <= L + |S_x| Z, Z the
// vertices' largest |X_kz|).  The launch ray is the FP64 ray's canonical FP32
// direction from the transmitter's FP32 rounding, which the origin term covers,
// and is tested with no drift.  A reflected ray has drifted from the FP64 ray
// of the final decision by at most Do (origin) and Dd (direction), 2-norm
// bounds from sbr_bounce: an origin shift Do moves a sheared vertex coordinate
// by Do (1 + |S_x|) <= 2 Do, a direction shift Dd moves S_x, S_y by at most
// 3.47 Dd (d_kz >= 1/sqrt 3) and so a sheared coordinate by 3.47 Dd (Z + Do);
// with sigma the sum, an edge function moves by at most 4 L sigma + 2 sigma^2.
// The margin is twice the sum of both parts plus the FP64 test's growth
// TRI_TOL (|U| + |V| + |W|), doubled.
__device__ __forceinline__ int tri_test32_dev(const WRay<float>& r, float4 p0, float4 p1, float4 p2, float Do,
                                              float Dd, float& t_out) {
    const V3<float> A = from4<float>(p0) - r.o, B = from4<float>(p1) - r.o, C = from4<float>(p2) - r.o;
    const float Akz = comp(A, r.kz), Bkz = comp(B, r.kz), Ckz = comp(C, r.kz);
    const float Akx = comp(A, r.kx), Aky = comp(A, r.ky), Bkx = comp(B, r.kx), Bky = comp(B, r.ky);
    const float Ckx = comp(C, r.kx), Cky = comp(C, r.ky);
    const float Ax = Akx - r.Sx * Akz, Ay = Aky - r.Sy * Akz;
    const float Bx = Bkx - r.Sx * Bkz, By = Bky - r.Sy * Bkz;
    const float Cx = Ckx - r.Sx * Ckz, Cy = Cky - r.Sy * Ckz;
    const float U = Cx * By - Cy * Bx, V = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
    const float L = fmaxf(fmaxf(fmaxf(fabsf(Ax), fabsf(Ay)), fmaxf(fabsf(Bx), fabsf(By))), fmaxf(fabsf(Cx), fabsf(Cy)));
    const float Z = fmaxf(fmaxf(fabsf(Akz), fabsf(Bkz)), fabsf(Ckz));
    const float Sab = fabsf(r.Sx) + fabsf(r.Sy);
    const float Mv = 2.0f * (L + Sab * Z);
    const float Mo = fabsf(comp(r.o, r.kx)) + fabsf(comp(r.o, r.ky)) + fabsf(comp(r.o, r.kz)) * Sab;
    const float sg = 2.0f * Do + 3.47f * Dd * (Z + Do);
    const float sum = fabsf(U) + fabsf(V) + fabsf(W);
    const float e = 1.01f * (5.9604645e-8f * (4.0f * L * L + 12.0f * (Mv + Mo) * L) + 4.0f * L * sg + 2.0f * sg * sg);
    const float m = 2.0f * e + 2.0f * (float)TRI_TOL * sum;
    const bool pos = U > m && V > m && W > m;
    const bool neg = U < -m && V < -m && W < -m;
    const float det = U + V + W;
    const float Tn = (U * Akz + V * Bkz + W * Ckz) * r.Sz;
    if (pos || neg) {
        t_out = Tn / det;
        return 1;
    }
    if ((U < -m || V < -m || W < -m) && (U > m || V > m || W > m)) return 0;
    t_out = det != 0.0f ? Tn / det : 0.0f;
    return 2;
}

// tri_test32 for the FP32 rounding rf of an FP64 ray r (the re-trace): rf's origin
// and direction differ from r's by one rounding each, so the margin is the
// rounding part of tri_test32_dev (whose origin term covers the origin's
// rounding) plus the direction's rounding.  That moves
// S_x, S_y by at most 2 sqrt(3) u (kz the largest component of a unit-length
// direction) and so a sheared vertex coordinate by 3.47 u Z, Z the vertices'
// largest |X_kz|, and an edge function by 4 L (3.47 u Z).  A robust hit also gets
// t_err, a bound on |t - tf| with t the exact hit distance along r: for a robust
// hit det = |U| + |V| + |W| = sum, each edge function is off by at most e (half
// the rounding part of the margin), a translated coordinate X_kz by
// u (|X_kz| + |o_kz|), so Tn = (U Akz + V Bkz + W Ckz) Sz is off by at most
// |Sz| (e (|Akz| + |Bkz| + |Ckz|) + 8 u sum (Z + |o_kz|)) + 6 u |Tn| (the
// roundings of the products and sums included), det by 3 e + 2 u sum, and
// t_err = (|dTn| + t |ddet|) / (sum - 3 e) + 2 u t.
__device__ __forceinline__ int tri_test32_exact(const WRay<float>& r, float4 p0, float4 p1, float4 p2,
                                                float& t_out, float& t_err) {
    const V3<float> A = from4<float>(p0) - r.o, B = from4<float>(p1) - r.o, C = from4<float>(p2) - r.o;
    const float Akz = comp(A, r.kz), Bkz = comp(B, r.kz), Ckz = comp(C, r.kz);
    const float Akx = comp(A, r.kx), Aky = comp(A, r.ky), Bkx = comp(B, r.kx), Bky = comp(B, r.ky);
    const float Ckx = comp(C, r.kx), Cky = comp(C, r.ky);
    const float Ax = Akx - r.Sx * Akz, Ay = Aky - r.Sy * Akz;
    const float Bx = Bkx - r.Sx * Bkz, By = Bky - r.Sy * Bkz;
    const float Cx = Ckx - r.Sx * Ckz, Cy = Cky - r.Sy * Ckz;
    const float U = Cx * By - Cy * Bx, V = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
    const float Sab = fabsf(r.Sx) + fabsf(r.Sy);
    const float Mv = fmaxf(fmaxf(fabsf(Akx) + fabsf(Aky) + fabsf(Akz) * Sab, fabsf(Bkx) + fabsf(Bky) + fabsf(Bkz) * Sab),
                           fabsf(Ckx) + fabsf(Cky) + fabsf(Ckz) * Sab);
    const float okz = fabsf(comp(r.o, r.kz));
    const float Mo = fabsf(comp(r.o, r.kx)) + fabsf(comp(r.o, r.ky)) + okz * Sab;
    const float L = fmaxf(fmaxf(fmaxf(fabsf(Ax), fabsf(Ay)), fmaxf(fabsf(Bx), fabsf(By))), fmaxf(fabsf(Cx), fabsf(Cy)));
    const float Z = fmaxf(fmaxf(fabsf(Akz), fabsf(Bkz)), fabsf(Ckz));
    const float u = 5.9604645e-8f;
    const float e = 1.01f * (u * (4.0f * L * L + 12.0f * (Mv + Mo) * L) + 4.0f * L * 3.47f * u * Z);
    const float sum = fabsf(U) + fabsf(V) + fabsf(W);
    const float m = 2.0f * e + 2.0f * (float)TRI_TOL * sum;
    const bool pos = U > m && V > m && W > m;
    const bool neg = U < -m && V < -m && W < -m;
    const float det = U + V + W;
    const float Tn = (U * Akz + V * Bkz + W * Ckz) * r.Sz;
    if (pos || neg) {
        t_out = Tn / det;
        const float dTn = fabsf(r.Sz) * (e * (fabsf(Akz) + fabsf(Bkz) + fabsf(Ckz)) + 8.0f * u * sum * (Z + okz)) +
                          6.0f * u * fabsf(Tn);
        const float ddet = 3.0f * e + 2.0f * u * sum;
        t_err = 1.01f * ((dTn + fabsf(t_out) * ddet) / (sum - 3.0f * e) + 2.0f * u * fabsf(t_out));
        return 1;
    }
    if ((U < -m || V < -m || W < -m) && (U > m || V > m || W > m)) return 0;
    t_out = det != 0.0f ? Tn / det : 0.0f;
    return 2;
}

// FP64 final decision: the triangle grown by TRI_TOL; a ray in its plane misses.
// On a hit returns true with det > 0 and t = Tn / det (not divided here).
__device__ __forceinline__ bool tri_test64(const WRay<double>& r, float4 p0, float4 p1, float4 p2, double& Tn,
                                           double& det) {
    double U, V, W;
    woop(r, p0, p1, p2, U, V, W, Tn);
    double mt = TRI_TOL * (fabs(U) + fabs(V) + fabs(W));
    if ((U < -mt || V < -mt || W < -mt) && (U > mt || V > mt || W > mt)) return false;
    det = U + V + W;
    if (!(fabs(det) > 3.0 * mt)) return false;
    if (det < 0.0) {
        det = -det;
        Tn = -Tn;
    }
    return true;
}

// Three-input FP32 min / max (sm_100 and later).
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Ray/box slab test over [tlo, thi]; a slab distance is l * inv - o * inv in one
// FMA (boxes carry a 4e-6 diag pad, far above this rounding).
template <typename R>
__device__ __forceinline__ bool slab(const R& r, float lx, float ly, float lz, float hx, float hy, float hz, float tlo,
                                     float thi, float& tn) {
    float tx0 = fmaf(lx, r.inv.x, -r.oinv.x), tx1 = fmaf(hx, r.inv.x, -r.oinv.x);
    float ty0 = fmaf(ly, r.inv.y, -r.oinv.y), ty1 = fmaf(hy, r.inv.y, -r.oinv.y);
    float tz0 = fmaf(lz, r.inv.z, -r.oinv.z), tz1 = fmaf(hz, r.inv.z, -r.oinv.z);
    tn = max3f(fminf(tx0, tx1), fminf(ty0, ty1), fmaxf(fminf(tz0, tz1), tlo));
    float tf = min3f(fmaxf(tx0, tx1), fmaxf(ty0, ty1), fminf(fmaxf(tz0, tz1), thi));
    return tn <= tf;
}


// Traversal of the two-child-box BVH with a per-thread stack in shared memory
// (stack[k * blockDim.x + threadIdx.x]), nearer child first.  `leaf(first,
// count)` tests the triangles of a leaf and returns true to stop; it may lower
// `thi`, the far end of the box tests.  Node visits are bounded.
template <int STACK = RT_STACK, typename R, typename Leaf>
__device__ __forceinline__ void traverse(const BvhNode* __restrict__ nodes, const R& r, float tlo, const float& thi,
                                         int* stack, int32_t* status, unsigned& nvis, Leaf&& leaf) {
    const int stride = blockDim.x;
    int sp = 0;
    int ref = 0;
    int visits = 0;
    for (;;) {
        // "while-while" order (Aila and Laine, High Performance Graphics 2009): a
        // lane descends through inner nodes until it holds a leaf, so that the
        // lanes of a warp test their leaves together instead of interleaving leaf
        // tests with node visits.  Each lane visits the same nodes in the same
        // order as a one-node-per-step loop.
        while (ref >= 0) {
            if (++visits > RT_MAX_VISITS) {
                rt_set_status(status, RT_ERR_ITER_LIMIT);
                return;
            }
            nvis++;
            const float4* np = reinterpret_cast<const float4*>(nodes + ref);
            float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2);
            int4 d = __ldg(reinterpret_cast<const int4*>(np + 3));
            float t0, t1;
            bool h0 = slab(r, a.x, a.y, a.z, a.w, b.x, b.y, tlo, thi, t0);
            bool h1 = slab(r, b.z, b.w, c.x, c.y, c.z, c.w, tlo, thi, t1);
            const int r0 = d.x, r1 = d.y;
            if (h0 && h1) {
                if (sp >= STACK) {
                    rt_set_status(status, RT_ERR_STACK_OVERFLOW);
                    return;
                }
                stack[sp * stride] = t0 <= t1 ? r1 : r0;
                sp++;
                ref = t0 <= t1 ? r0 : r1;
            } else if (h0 || h1) {
                ref = h0 ? r0 : r1;
            } else {
                if (sp == 0) return;
                sp--;
                ref = stack[sp * stride];
            }
        }
        if (++visits > RT_MAX_VISITS) {
            rt_set_status(status, RT_ERR_ITER_LIMIT);
            return;
        }
        const int e = ~ref;
        if (leaf(e >> 3, (e & 7) + 1)) return;
        if (sp == 0) return;
        sp--;
        ref = stack[sp * stride];
    }
}

// FP32 closest hit with t > tmin (skipping `skip` and every triangle in the
// plane `skip_plane` of the ray's start: the ray meets that plane only at
// t = 0, which no test takes as a hit): exact ties go to the lower triangle
// index; `und` is set if any decision that could matter was marginal.  The
// plane id of the hit (the .w of its second vertex record) is returned in
// `plane_out`.
template <int STACK = RT_STACK>
__device__ __forceinline__ int closest32(const BvhNode* __restrict__ nodes, const float4* __restrict__ tris,
                                         const WRay<float>& r, float tmin, int skip, int* stack, float& t_out,
                                         bool& und, int32_t* status, unsigned& nvis, unsigned& ntri,
                                         float Do, float Dd, int skip_plane, int& plane_out) {
    float tb = INFINITY, thi = INFINITY;
    int best = -1;
    traverse<STACK>(nodes, r, tmin * 0.5f, thi, stack, status, nvis, [&](int first, int count) {
        for (int k = first; k < first + count; ++k) {
            float4 p0 = __ldg(tris + 3 * k), p1 = __ldg(tris + 3 * k + 1), p2 = __ldg(tris + 3 * k + 2);
            int id = __float_as_int(p0.w);
            if (id == skip || __float_as_int(p1.w) == skip_plane) continue;
            ntri++;
            float th;
            int cls = tri_test32_dev(r, p0, p1, p2, Do, Dd, th);
            if (cls == 0) continue;
            if (cls == 2) {
                if (th > tmin * 0.5f && th < tb * 1.00001f) und = true;
                continue;
            }
            if (!(th > tmin)) {
                if (th > tmin * 0.1f) und = true;
                continue;
            }
            if (th < tmin * 10.0f) und = true;
            if (best >= 0 && fabsf(th - tb) <= 1e-4f * tb) und = true;
            if (th < tb || (th == tb && id < best)) {
                tb = th;
                best = id;
                plane_out = __float_as_int(p1.w);
                thi = tb * 1.00001f;
            }
        }
        return false;
    });
    t_out = tb;
    return best;
}

// FP32 any hit with tmin < t < tmax (skipping skip0, skip1 and every triangle
// in the plane pl0 or pl1 of a segment's end triangle: the segment meets that
// plane only at its end, at t = 0 or 1, outside (tmin, tmax) in exact arithmetic
// and in the FP64 test): true on a robust hit; `und` set if no robust hit was
// found but a marginal one might exist.  A triangle's plane id is the .w of
// its second vertex record.
template <int STACK = RT_STACK>
__device__ __forceinline__ bool any32(const BvhNode* __restrict__ nodes, const float4* __restrict__ tris,
                                     const WRay<float>& r, float tmin, float tmax, int skip0, int skip1, int pl0,
                                     int pl1, int* stack, bool& und, int32_t* status, unsigned& nvis,
                                     unsigned& ntri) {
    bool hit = false;
    const float thi = tmax * 1.00001f;
    traverse<STACK>(nodes, r, tmin * 0.5f, thi, stack, status, nvis, [&](int first, int count) {
        for (int k = first; k < first + count; ++k) {
            float4 p0 = __ldg(tris + 3 * k), p1 = __ldg(tris + 3 * k + 1), p2 = __ldg(tris + 3 * k + 2);
            int id = __float_as_int(p0.w);
            const int pid = __float_as_int(p1.w);
            if (id == skip0 || id == skip1 || pid == pl0 || pid == pl1) continue;
            ntri++;
            float th;
            int cls = tri_test32(r, p0, p1, p2, th);
            if (cls == 0) continue;
            if (cls == 2) {
                if (th > tmin * 0.5f && th < tmax * 1.00001f) und = true;
                continue;
            }
            if (!(th > tmin)) {
                if (th > tmin * 0.1f) und = true;
                continue;
            }
            if (th < tmax) {
                if (th < tmin * 10.0f || th > tmax - tmin * 9.0f) {
                    und = true;
                } else {
                    hit = true;
                    return true;
                }
            }
        }
        return false;
    });
    return hit;
}

// Closest hit of an FP64 ray, with final decisions in FP64: the smallest
// t = Tn/det (compared by cross-multiplication), then the lowest triangle index
// among the hits with t within TIE_TOL of it (independent of the visiting order).
// Every triangle first gets the FP32 test with its margin on the ray rounded to
// FP32 (rf); a robust FP32 miss is final, everything else gets the FP64 test,
// so the FP64 work is a few tests per query.  The tie pass runs only if two
// hits came within 1e-6 (relative) of each other.
__device__ int closest64_inline(const BvhNode* __restrict__ nodes, const float4* __restrict__ tris,
                                const WRay<double>& r, const WRay<float>& rf, double tmin, int skip, int* stack,
                                double& t_out, int32_t* status) {
    double bT = 0.0, bD = 1.0;
    bool have = false, near_tie = false;
    int best = -1;
    float thi = INFINITY;
    unsigned nv = 0;
    const float tminf = (float)tmin;
    traverse(nodes, rf, tminf * 0.5f, thi, stack, status, nv, [&](int first, int count) {
        for (int k = first; k < first + count; ++k) {
            float4 p0 = __ldg(tris + 3 * k), p1 = __ldg(tris + 3 * k + 1), p2 = __ldg(tris + 3 * k + 2);
            int id = __float_as_int(p0.w);
            if (id == skip) continue;
            float tf;
            if (tri_test32(rf, p0, p1, p2, tf) == 0) continue;
            double Tn, det;
            if (!tri_test64(r, p0, p1, p2, Tn, det)) continue;
            if (!(Tn > tmin * det)) continue;
            if (have && fabs(Tn * bD - bT * det) <= 1e-6 * bT * det) near_tie = true;
            if (!have || Tn * bD < bT * det || (Tn * bD == bT * det && id < best)) {
                bT = Tn;
                bD = det;
                best = id;
                have = true;
                thi = (float)(Tn * rcp64(det)) * 1.00001f + 1e-30f;
            }
        }
        return false;
    });
    if (!have) return -1;
    const double tb = bT * rcp64(bD);
    t_out = tb;
    if (!near_tie) return best;
    const double tmax = tb + TIE_TOL * tb;
    int low = 0x7fffffff;
    thi = (float)tmax * 1.00001f + 1e-30f;
    traverse(nodes, rf, tminf * 0.5f, thi, stack, status, nv, [&](int first, int count) {
        for (int k = first; k < first + count; ++k) {
            float4 p0 = __ldg(tris + 3 * k), p1 = __ldg(tris + 3 * k + 1), p2 = __ldg(tris + 3 * k + 2);
            int id = __float_as_int(p0.w);
            if (id == skip || id >= low) continue;
            float tf;
            if (tri_test32(rf, p0, p1, p2, tf) == 0) continue;
            double Tn, det;
            if (!tri_test64(r, p0, p1, p2, Tn, det)) continue;
            if (Tn > tmin * det && Tn <= tmax * det) low = id;
        }
        return false;
    });
    return low == 0x7fffffff ? best : low;
}

// The hit of a bounce whose triangle is known (a robust prefix bounce of the
// re-trace, or a closest hit decided in FP32 with error bounds): t where the FP64 ray meets the triangle's FP64 plane n.x = c,
// t = (c - n.o) / (n.d), a dozen FP64 operations instead of the full
// ray/triangle test (the FP64 pipe bounds this kernel).  False if the ray is
// (nearly) parallel to the plane or t <= tmin, which the caller treats as
// undecided.
__device__ __forceinline__ bool replay_plane(const double* __restrict__ tri_n64, int id, const WRay<double>& r,
                                             double tmin, double& t_out) {
    const double nx = tri_n64[4 * id], ny = tri_n64[4 * id + 1], nz = tri_n64[4 * id + 2], c = tri_n64[4 * id + 3];
    const double nd = nx * r.d.x + ny * r.d.y + nz * r.d.z;
    if (!(fabs(nd) > 1e-9)) return false;
    t_out = (c - (nx * r.o.x + ny * r.o.y + nz * r.o.z)) * rcp64(nd);
    return t_out > tmin;
}

// Same decisions as closest64_inline, with the FP64 work taken out of the
// divergent traversal.  An FP64 warp instruction costs the same with one active
// lane as with 32, so FP64 tests inside the traversal loop are paid on every
// step at which any lane sits at a leaf.  Here the FP32 traversal only collects
// the triangles whose FP32 test is not a robust miss (at most CAND_CAP, in
// `cand`, a per-thread list in shared memory with stride blockDim.x); a robust
// FP32 hit at t > 2 tmin lowers the far end of the box tests to t (1 + 1e-3) +
// 10 tmin, wider than the 1e-4 band in which the FP32 pass already treats two
// hits as a tie.  The FP64 tests then run
// over the list in one converged loop, and the tie pass over the same list
// (every hit within TIE_TOL of the best is in it).  A list overflow falls back to
// closest64_inline.
constexpr int CAND_CAP = 16;

__device__ int closest64(const BvhNode* __restrict__ nodes, const float4* __restrict__ tris, WRay<double>& r,
                         const WRay<float>& rf, const double* __restrict__ tri_n64, double tmin, int skip, int* stack,
                         int* cand, float* cand_t, float* cand_e, double& t_out, int32_t* status) {
    const int stride = blockDim.x;
    const float tminf = (float)tmin;
    float thi = INFINITY;
    int n = 0;
    unsigned nv = 0;
    traverse(nodes, rf, tminf * 0.5f, thi, stack, status, nv, [&](int first, int count) {
        for (int k = first; k < first + count; ++k) {
            float4 p0 = __ldg(tris + 3 * k), p1 = __ldg(tris + 3 * k + 1), p2 = __ldg(tris + 3 * k + 2);
            int id = __float_as_int(p0.w);
            if (id == skip) continue;
            float tf, te = 0.0f;
            int cls = tri_test32_exact(rf, p0, p1, p2, tf, te);
            if (cls == 0) continue;
            if (cls == 1) {
                if (tf - te > thi) continue;   // beyond a robust hit
                if (tf > tminf * 2.0f) thi = fminf(thi, tf * 1.001f + 10.0f * tminf + 4.0f * te);
            } else {
                // undecided (NaN: always goes to the FP64 test); te becomes a lower
                // bound of t over the whole triangle: a hit point is a convex
                // combination of the vertices, so t >= min_k (X_k - o).d / |d|^2.
                // The FP32 dots with rf differ from those with the FP64 ray by at
                // most 8 u (max_k |X_k - o|_1 + |o|_1) for a unit d (roundings of the
                // subtractions and products, and rf's own rounding of o and d)
                const V3<float> da = from4<float>(p0) - rf.o, db = from4<float>(p1) - rf.o, dc = from4<float>(p2) - rf.o;
                const float lo = fminf(fminf(dot(da, rf.d), dot(db, rf.d)), dot(dc, rf.d));
                const float R = fmaxf(fmaxf(fabsf(da.x) + fabsf(da.y) + fabsf(da.z), fabsf(db.x) + fabsf(db.y) + fabsf(db.z)),
                                      fabsf(dc.x) + fabsf(dc.y) + fabsf(dc.z)) +
                                fabsf(rf.o.x) + fabsf(rf.o.y) + fabsf(rf.o.z);
                te = (lo - 8.0f * 5.9604645e-8f * R) * (1.0f - 1e-6f) - 1e-30f;
                tf = __int_as_float(0x7fc00000);
            }
            if (n < CAND_CAP) {
                cand[n * stride] = k;
                cand_t[n * stride] = tf;
                cand_e[n * stride] = te;
            }
            n++;
        }
        return false;
    });
    if (n <= CAND_CAP) {
        // decided in FP32 when every candidate is a robust hit and the nearest one
        // beyond tmin is separated from tmin and from every other by more than
        // their error bounds: that triangle is the FP64 test's closest hit, and its
        // distance along r comes from its FP64 plane
        bool fast = true;
        int ib = -1;
        float tb = INFINITY, eb = 0.0f;
        for (int i = 0; i < n && fast; ++i) {
            const float t = cand_t[i * stride], te = cand_e[i * stride];
            if (t != t) continue;                             // undecided edge: checked below
            if (t - te > tminf) {
                if (t < tb) {
                    tb = t;
                    eb = te;
                    ib = i;
                }
            } else if (t + te >= tminf) fast = false;         // not clear of tmin
        }
        for (int i = 0; i < n && fast; ++i) {
            if (i == ib) continue;
            const float t = cand_t[i * stride], te = cand_e[i * stride];
            if (t != t) {
                // an undecided triangle only matters if some of it lies before the best
                if (!(ib >= 0 && te > tb + eb)) fast = false;
            } else if (ib >= 0 && t - te > tminf && !(t - te > tb + eb)) {
                fast = false;                                 // not clearly farther
            }
        }
        if (fast) {
            if (ib < 0) return -1;   // every candidate clearly before tmin
            const int k = cand[ib * stride];
            const int id = __float_as_int(__ldg(tris + 3 * k).w);
            double th;
            if (replay_plane(tri_n64, id, r, tmin, th)) {
                t_out = th;
                return id;
            }
        }
    }
    wray_init(r);   // the FP64 tests below need the ray's shear
    if (n > CAND_CAP) return closest64_inline(nodes, tris, r, rf, tmin, skip, stack, t_out, status);
    double bT = 0.0, bD = 1.0;
    bool have = false, near_tie = false;
    int best = -1;
    for (int i = 0; i < n; ++i) {
        // a robust hit beyond the final far end (NaN, undecided, compares false)
        if (cand_t[i * stride] - cand_e[i * stride] > thi) continue;
        const int k = cand[i * stride];
        float4 p0 = __ldg(tris + 3 * k), p1 = __ldg(tris + 3 * k + 1), p2 = __ldg(tris + 3 * k + 2);
        int id = __float_as_int(p0.w);
        double Tn, det;
        if (!tri_test64(r, p0, p1, p2, Tn, det)) continue;
        if (!(Tn > tmin * det)) continue;
        if (have && fabs(Tn * bD - bT * det) <= 1e-6 * bT * det) near_tie = true;
        if (!have || Tn * bD < bT * det || (Tn * bD == bT * det && id < best)) {
            bT = Tn;
            bD = det;
            best = id;
            have = true;
        }
    }
    if (!have) return -1;
    const double tb64 = bT * rcp64(bD);
    t_out = tb64;
    if (!near_tie) return best;
    const double tmax = tb64 + TIE_TOL * tb64;
    int low = 0x7fffffff;
    for (int i = 0; i < n; ++i) {
        if (cand_t[i * stride] - cand_e[i * stride] > thi) continue;
        const int k = cand[i * stride];
        float4 p0 = __ldg(tris + 3 * k), p1 = __ldg(tris + 3 * k + 1), p2 = __ldg(tris + 3 * k + 2);
        int id = __float_as_int(p0.w);
        if (id >= low) continue;
        double Tn, det;
        if (!tri_test64(r, p0, p1, p2, Tn, det)) continue;
        if (Tn > tmin * det && Tn <= tmax * det) low = id;
    }
    return low == 0x7fffffff ? best : low;
}

// Any hit with tmin < t < tmax of an FP64 ray (skipping skip0 and skip1),
// final decisions in FP64; robust FP32 misses on the rounded ray rf are final.
template <int STACK = RT_STACK>
__device__ bool any64_inline(const BvhNode* __restrict__ nodes, const float4* __restrict__ tris,
                             const WRay<double>& r, const WRay<float>& rf, double tmin, double tmax, int skip0,
                             int skip1, int* stack, int32_t* status) {
    bool hit = false;
    const float thi = (float)tmax * 1.00001f;
    unsigned nv = 0;
    traverse<STACK>(nodes, rf, (float)tmin * 0.5f, thi, stack, status, nv, [&](int first, int count) {
        for (int k = first; k < first + count; ++k) {
            float4 p0 = __ldg(tris + 3 * k), p1 = __ldg(tris + 3 * k + 1), p2 = __ldg(tris + 3 * k + 2);
            int id = __float_as_int(p0.w);
            if (id == skip0 || id == skip1) continue;
            float tf;
            if (tri_test32(rf, p0, p1, p2, tf) == 0) continue;
            double Tn, det;
            if (!tri_test64(r, p0, p1, p2, Tn, det)) continue;
            if (Tn > tmin * det && Tn < tmax * det) {
                hit = true;
                return true;
            }
        }
        return false;
    });
    return hit;
}

// any64_inline with the FP64 tests taken out of the traversal (as closest64):
// the FP32 traversal collects the triangles that are not a robust FP32 miss
// and whose FP32 t is not beyond tmax (1 + 1e-3) + 10 tmin (at most
// VIS_CAND_CAP, per-thread list in shared memory with stride blockDim.x); the
// FP64 tests run over the list afterwards.  A list overflow falls back to
// any64_inline.
constexpr int VIS_CAND_CAP = 8;

template <int STACK = RT_STACK>
__device__ bool any64(const BvhNode* __restrict__ nodes, const float4* __restrict__ tris, const WRay<double>& r,
                      const WRay<float>& rf, double tmin, double tmax, int skip0, int skip1, int* stack, int* cand,
                      int32_t* status) {
    const int stride = blockDim.x;
    const float thi = (float)tmax * 1.00001f;
    const float tcut = (float)tmax * 1.001f + 10.0f * (float)tmin;
    int n = 0;
    unsigned nv = 0;
    traverse<STACK>(nodes, rf, (float)tmin * 0.5f, thi, stack, status, nv, [&](int first, int count) {
        for (int k = first; k < first + count; ++k) {
            float4 p0 = __ldg(tris + 3 * k), p1 = __ldg(tris + 3 * k + 1), p2 = __ldg(tris + 3 * k + 2);
            int id = __float_as_int(p0.w);
            if (id == skip0 || id == skip1) continue;
            float tf;
            int cls = tri_test32(rf, p0, p1, p2, tf);
            if (cls == 0 || (cls == 1 && tf > tcut)) continue;
            if (n < VIS_CAND_CAP) cand[n * stride] = k;
            n++;
        }
        return false;
    });
    if (n > VIS_CAND_CAP) return any64_inline<STACK>(nodes, tris, r, rf, tmin, tmax, skip0, skip1, stack, status);
    for (int i = 0; i < n; ++i) {
        const int k = cand[i * stride];
        double Tn, det;
        if (!tri_test64(r, __ldg(tris + 3 * k), __ldg(tris + 3 * k + 1), __ldg(tris + 3 * k + 2), Tn, det)) continue;
        if (Tn > tmin * det && Tn < tmax * det) return true;
    }
    return false;
}

// ------------------------------------------------------------------ launch directions
// sincos_turn and launch_dir: launch_dir.cuh

// Processing order of the rays (the set of rays and every result are the same
// in any order).  Consecutive Fibonacci indices have nearby z but azimuths a
// golden angle apart, so a warp of consecutive rays diverges.  Instead the rays
// are taken in z-bands of B consecutive indices, and inside a band by azimuth:
// the azimuth fraction of ray i0 + k is (i0 G + k G) mod 2^32, i.e. the fractions
// of k G shifted by a constant, so every band's order is one fixed sorted list
// of k (by k G mod 2^32) rotated to start at the band's wrap point.
struct RaySched {
    int64_t n, band, full;
    const int32_t* order;
    const int32_t* wrap;
    const float* z;   // n entries: z of launch direction i
};

// j < n <= 2^31 - 1, so 32-bit division suffices.
__device__ __forceinline__ int64_t sched_ray(const RaySched& S, int64_t j) {
    if (S.band <= 0) return j;
    const uint32_t band = (uint32_t)S.band;
    const uint32_t b = (uint32_t)j / band;
    if ((int64_t)b >= S.full) return j;
    uint32_t pos = ((uint32_t)j - b * band) + (uint32_t)S.wrap[b];
    if (pos >= band) pos -= band;
    return (int64_t)b * S.band + S.order[pos];
}

// ------------------------------------------------------------------ hash set of keys
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    // 64-bit finaliser of SplitMix64 (Steele, Lea, Flood 2014)
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

__device__ __forceinline__ void hash_insert(unsigned long long* table, uint64_t mask, uint64_t key,
                                            unsigned long long* count, unsigned long long limit, int32_t* overflow) {
    if (*(volatile int32_t*)overflow) return;
    uint64_t h = mix64(key) & mask;
    for (uint64_t probe = 0; probe <= mask && probe < 4096; ++probe) {
        unsigned long long cur = table[h];
        if (cur == key) return;
        if (cur == 0ull) {
            unsigned long long prev = atomicCAS(table + h, 0ull, (unsigned long long)key);
            if (prev == 0ull) {
                unsigned long long c = atomicAdd(count, 1ull);
                if (c + 1 > limit) atomicExch(overflow, 1);
                return;
            }
            if (prev == key) return;
        }
        h = (h + 1) & mask;
    }
    atomicExch(overflow, 1);
}

struct SbrArgs {
    const BvhNode* nodes;
    const float4* tris;       // BVH order
    double tx, ty, tz;
    float3 txf;               // Tx rounded to FP32 (origin of the FP32 launch rays)
    int64_t n_rays;
    int depth;
    double eps;
    unsigned long long* table;
    uint64_t mask;
    unsigned long long* uniq;
    unsigned long long uniq_limit;
    int32_t* overflow;
    unsigned long long* next_ray;
    int64_t* redo;                  // re-trace list: ray | (undecided bounce << 32)
    uint64_t* redo_key;             // key of the robust prefix of each listed ray
    unsigned long long* redo_count;
    int64_t redo_cap;
    int32_t* status;
    unsigned long long* counters;   // optional instrumentation (slots 0..3)
    RaySched sched;
};

// Adds a per-thread count to a device counter (one atomic per warp).
__device__ __forceinline__ void warp_count(unsigned long long* c, unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(c, v);
}

// One specular bounce of the FP32 SBR ray at triangle id (plane record pl =
// FP32 unit normal n and n.v0): the hit point from the plane, o' = o + t d with
// t = (n.v0 - n.o) / (n.d), and the mirror direction d' = d - 2 (d.n) n
// (Sec. II-B).  Do and Dd bound the drift of the FP32 ray from the FP64 ray of
// the final decision, which reflects at its own plane hit about the FP64
// normal; with u = 2^-24 they grow as
//   Do' = 1.01 ((Do + t Dd + dN + 4u t) / (|n.d| - 4u) + u (|o|_1 + 4t)),
//   Dd' = Dd + 14u,
// dN = u (|n.v0| + 4 |o|_1 + |n.v0 - n.o|) and 4u bounding the roundings of
// the plane's numerator and of n.d (n one rounding off the FP64 normal), the
// first term the hit point's shift along the plane (an oblique projection of
// norm 1 / cos), the last the roundings of t (an approximate division, within
// 2 ulp) and of o + t d; the reflection is an isometry and adds the normal's
// rounding (4u) and its own (10u).  At an axis-aligned plane (two components
// of the unit normal zero, so the third is +-1 and n.v0 a vertex coordinate, in
// FP32 and in FP64 alike) both reflections are exact and n.d, n.o are exact:
// the direction's drift does not grow, and only the rounding of n.v0 - n.o
// remains in dN (an FP64 normal component below the FP32 range is absorbed by
// the 1 % slack).  Returns false if the ray meets the plane too obliquely for
// the bound (|n.d| <= 4u).
__device__ __forceinline__ bool sbr_bounce(WRay<float>& r, float4 pl, float& Do, float& Dd) {
    const float u = 5.9604645e-8f;
    const V3<float> n = mk(pl.x, pl.y, pl.z);
    const float N = pl.w - dot(n, r.o);
    const float Dn = dot(n, r.d);
    const bool axis = (int)(pl.x == 0.0f) + (int)(pl.y == 0.0f) + (int)(pl.z == 0.0f) == 2;
    const float eD = axis ? 0.0f : 4.0f * u;
    const float aD = fabsf(Dn) - 4.0f * u;
    if (!(aD > 0.0f)) return false;
    const float ts = __fdividef(N, Dn), t = fabsf(ts);
    const float o1 = fabsf(r.o.x) + fabsf(r.o.y) + fabsf(r.o.z);
    const float dN = axis ? u * fabsf(N) : u * (fabsf(pl.w) + 4.0f * o1 + fabsf(N));
    Do = 1.01f * ((Do + t * Dd + dN + eD * t) / aD + u * (o1 + 4.0f * t));
    if (!axis) Dd = Dd + 14.0f * u;
    const V3<float> p = r.o + ts * r.d;
    r.d = r.d - (2.0f * Dn) * n;
    r.o = p;
    wray_init(r);
    return true;
}

// Persistent SBR: every lane owns one ray; a lane whose ray ended takes the next
// ray index from a global counter (one atomic per warp refill), so warps stay
// full across bounces (warp-level compaction of the active rays).  One loop
// iteration = one closest-hit query per active lane.
template <int STACK>
__global__ void __launch_bounds__(TRACE_THREADS) k_sbr(SbrArgs A, const float4* __restrict__ tri_plane) {
    extern __shared__ int smem_stack[];
    int* stack = smem_stack + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int64_t ray = -1;
    bool done = false;
    int bounce = 0, prev = -1, prev_plane = -1;
    uint64_t key = 0;
    WRay<float> r;
    float Do = 0.0f, Dd = 0.0f;   // drift of the FP32 ray from the FP64 one (sbr_bounce)
    const float eps = (float)A.eps;
    unsigned long long c_vis = 0, c_tri = 0, c_q = 0;
    for (;;) {
        bool need = (ray < 0) && !done;
        unsigned m = __ballot_sync(FULL, need);
        if (m) {
            unsigned long long base = 0;
            int leader = __ffs(m) - 1;
            if (lane == leader) base = atomicAdd(A.next_ray, (unsigned long long)__popc(m));
            base = __shfl_sync(FULL, base, leader);
            if (need) {
                int64_t idx = (int64_t)(base + __popc(m & ((1u << lane) - 1)));
                if (idx < A.n_rays) {
                    idx = sched_ray(A.sched, idx);
                    ray = idx;
                    bounce = 0;
                    prev = -1;
                    prev_plane = -1;
                    key = 0;
                    float3 d = launch_dir(idx, __ldg(A.sched.z + idx));
                    r.o = mk(A.txf.x, A.txf.y, A.txf.z);
                    r.d = mk(d.x, d.y, d.z);
                    wray_init(r);
                    // the transmitter's rounding; the direction is the FP64 ray's
                    Do = 5.9604645e-8f * (fabsf(A.txf.x) + fabsf(A.txf.y) + fabsf(A.txf.z));
                    Dd = 0.0f;
                } else {
                    done = true;
                }
            }
        }
        if (__all_sync(FULL, done)) break;
        if (ray < 0) continue;
        float th;
        bool und = false;
        unsigned nv = 0, nt = 0;
        // the launch ray: its drift is the transmitter's rounding, which the test's
        // origin term covers, so it is tested with none
        int plane = -1;
        int id = closest32<STACK>(A.nodes, A.tris, r, eps, prev, stack, th, und, A.status, nv, nt,
                                  bounce == 0 ? 0.0f : Do, Dd, prev_plane, plane);
        c_vis += nv;
        c_tri += nt;
        c_q++;
        if (und) {
            unsigned long long slot = atomicAdd(A.redo_count, 1ull);
            if ((int64_t)slot < A.redo_cap) {
                A.redo[slot] = ray | ((int64_t)bounce << 32);
                A.redo_key[slot] = key;
            } else {
                atomicExch(A.overflow, 2);
            }
            ray = -1;
            continue;
        }
        if (id < 0) {
            ray = -1;
            continue;
        }
        key = rt_key_push(key, bounce, id);
        hash_insert(A.table, A.mask, key, A.uniq, A.uniq_limit, A.overflow);
        bounce++;
        if (bounce >= A.depth) {
            ray = -1;
            continue;
        }
        if (!sbr_bounce(r, __ldg(tri_plane + 3 * id), Do, Dd)) {
            // too oblique for the drift bound: the next bounce is decided in FP64
            unsigned long long slot = atomicAdd(A.redo_count, 1ull);
            if ((int64_t)slot < A.redo_cap) {
                A.redo[slot] = ray | ((int64_t)bounce << 32);
                A.redo_key[slot] = key;
            } else {
                atomicExch(A.overflow, 2);
            }
            ray = -1;
            continue;
        }
        prev = id;
        prev_plane = plane;
    }
    if (A.counters) {
        warp_count(A.counters + 0, c_vis);
        warp_count(A.counters + 1, c_tri);
        warp_count(A.counters + 2, c_q);
    }
}

// FP64 re-trace of the rays whose FP32 decisions were marginal (same rules,
// final decisions).  One warp per block spreads the few rays over all SMs.
// Inserts every prefix again; duplicates are harmless.
// Re-trace of a listed ray in FP64: the bounces before the one the FP32 pass
// left undecided were decided robustly, so their triangles (in the stored key)
// are replayed with one FP64 ray/triangle test each; the BVH search in
// mixed precision (closest64) starts at the undecided bounce.
__device__ __forceinline__ uint64_t key_prefix(uint64_t key, int b) {   // the fields of bounces < b
    return b <= 0 ? 0ull : key & (~0ull << (48 - 16 * (b - 1)));
}

__global__ void __launch_bounds__(REDO_THREADS) k_sbr_redo(SbrArgs A, const double* __restrict__ tri_n64,
                                                           const float4* __restrict__ tri_v) {
    pdl_entry();
    extern __shared__ int smem_stack[];
    int* stack = smem_stack + threadIdx.x;
    int* cand = smem_stack + RT_STACK * blockDim.x + threadIdx.x;
    float* cand_t = reinterpret_cast<float*>(smem_stack + (RT_STACK + CAND_CAP) * blockDim.x) + threadIdx.x;
    float* cand_e = reinterpret_cast<float*>(smem_stack + (RT_STACK + 2 * CAND_CAP) * blockDim.x) + threadIdx.x;
    unsigned long long n = *A.redo_count;
    if (n > (unsigned long long)A.redo_cap) n = A.redo_cap;
    if (A.counters && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(A.counters + 3, n);
    // few redo rays: spread them over all warps, rpw lanes per warp, so that more
    // warps hide the traversal latency and a warp carries fewer divergent rays
    const unsigned long long W = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long rpw = n < W ? 1ull : (n + W - 1) / W < 32ull ? (n + W - 1) / W : 32ull;
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (lane >= rpw) return;
    for (unsigned long long w = warp * rpw + lane; w < n; w += W * rpw) {
        const int64_t e = A.redo[w];
        const int64_t ray = e & 0xffffffffll;
        int b0 = (int)(e >> 32);
        uint64_t key = A.redo_key[w];
        float3 df = launch_dir(ray, __ldg(A.sched.z + ray));
        WRay<double> r;
        WRay<float> rf;
        r.o = mk(A.tx, A.ty, A.tz);
        r.d = mk((double)df.x, (double)df.y, (double)df.z);
        int prev = -1;
        for (int b = 0; b < A.depth; ++b) {
            double th;
            int id = -1;
            if (b < b0) {   // robust prefix: its triangle is known, t from its plane in FP64
                id = rt_key_tri(key, b);
                if (!replay_plane(tri_n64, id, r, A.eps, th)) {   // not expected: search from here on
                    b0 = b;
                    key = key_prefix(key, b);
                }
            }
            if (b >= b0) {
                rf.o = mk((float)r.o.x, (float)r.o.y, (float)r.o.z);
                rf.d = mk((float)r.d.x, (float)r.d.y, (float)r.d.z);
                wray_init(rf);
                id = closest64(A.nodes, A.tris, r, rf, tri_n64, A.eps, prev, stack, cand, cand_t, cand_e, th, A.status);
                if (id < 0) break;
                key = rt_key_push(key_prefix(key, b), b, id);
                hash_insert(A.table, A.mask, key, A.uniq, A.uniq_limit, A.overflow);
            }
            V3<double> nn = mk(tri_n64[4 * id], tri_n64[4 * id + 1], tri_n64[4 * id + 2]);
            V3<double> p = r.o + th * r.d;
            r.d = r.d - (2.0 * dot(r.d, nn)) * nn;
            r.o = p;
            prev = id;
        }
    }
}

// ------------------------------------------------------------------ compaction + sort
// Non-zero table entries into out (at most out_cap of them; the count keeps
// counting past it, which the host reads as an overflow).
__global__ void k_table_compact(const unsigned long long* __restrict__ table, uint64_t cap, uint64_t* out,
                                unsigned long long* count, uint64_t out_cap) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i - lane < cap;
         i += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long k = i < cap ? table[i] : 0ull;
        unsigned m = __ballot_sync(FULL, k != 0ull);
        if (!m) continue;
        unsigned long long base = 0;
        int leader = __ffs(m) - 1;
        if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
        base = __shfl_sync(FULL, base, leader);
        const unsigned long long slot = base + __popc(m & ((1u << lane) - 1));
        if (k && slot < out_cap) out[slot] = k;
    }
}

__device__ __forceinline__ bool key_less(uint64_t a, uint64_t b) {
    int da = rt_key_depth(a), db = rt_key_depth(b);
    return da < db || (da == db && a < b);
}

constexpr int SORT_BLOCK = 2048;   // elements per shared-memory bitonic block

// Full bitonic sort of each 2048-element chunk (stages k = 2..2048).
__global__ void k_bitonic_local(uint64_t* keys) {
    __shared__ uint64_t s[SORT_BLOCK];
    const uint64_t base = (uint64_t)blockIdx.x * SORT_BLOCK;
    for (int i = threadIdx.x; i < SORT_BLOCK; i += blockDim.x) s[i] = keys[base + i];
    __syncthreads();
    for (int k = 2; k <= SORT_BLOCK; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < SORT_BLOCK; i += blockDim.x) {
                int p = i ^ j;
                if (p > i) {
                    bool up = (((base + i) & k) == 0);
                    uint64_t x = s[i], y = s[p];
                    if (key_less(y, x) == up) {
                        s[i] = y;
                        s[p] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < SORT_BLOCK; i += blockDim.x) keys[base + i] = s[i];
}

// Stages j = 1024..1 of merge level k (k > 2048) inside each chunk.
__global__ void k_bitonic_merge_local(uint64_t* keys, uint64_t k) {
    __shared__ uint64_t s[SORT_BLOCK];
    const uint64_t base = (uint64_t)blockIdx.x * SORT_BLOCK;
    for (int i = threadIdx.x; i < SORT_BLOCK; i += blockDim.x) s[i] = keys[base + i];
    __syncthreads();
    for (int j = SORT_BLOCK >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < SORT_BLOCK; i += blockDim.x) {
            int p = i ^ j;
            if (p > i) {
                bool up = (((base + i) & k) == 0);
                uint64_t x = s[i], y = s[p];
                if (key_less(y, x) == up) {
                    s[i] = y;
                    s[p] = x;
                }
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < SORT_BLOCK; i += blockDim.x) keys[base + i] = s[i];
}

// Small sets (n <= RANK_SORT_MAX unique keys): rank of every key = the number of
// smaller keys, counted over all pairs spread across the grid (blockIdx.x: a
// tile of RANK_TILE keys staged in shared memory, blockIdx.y: the keys being
// ranked), then a scatter.  A bitonic network of a few thousand keys runs on
// one or two CTAs through ~66 barrier-separated steps; this runs in a few.
constexpr int RANK_SORT_MAX = 8192;
constexpr int RANK_TILE = 512;

// The order is key_less: depth first, then the key (left-aligned fields).  With
// every used field >= 1 (triangle id + 1), the key shifted right by its empty
// fields, v = key >> 16 (4 - depth), orders the same way as one unsigned number:
// a depth-q value is at least 2^(16 (q - 1)), above every depth-(q - 1) value, and
// within a depth the shift keeps the order.
__device__ __forceinline__ uint64_t rank_value(uint64_t key) {
    const int q = rt_key_depth(key);
    return q == 0 ? 0ull : key >> (16 * (4 - q));
}

// n: the number of keys, read from the compaction count (at most cap).
__global__ void k_rank_count(const uint64_t* __restrict__ keys, const unsigned long long* __restrict__ n_dev, int cap,
                             int* __restrict__ rank) {
    pdl_entry();
    __shared__ uint64_t sj[RANK_TILE];
    const int n = (int)min(*n_dev, (unsigned long long)cap);
    const int j0 = blockIdx.x * RANK_TILE;
    if (j0 >= n) return;
    for (int t = threadIdx.x; t < RANK_TILE; t += blockDim.x)
        sj[t] = j0 + t < n ? rank_value(keys[j0 + t]) : ~0ull;   // padding never counts as smaller
    __syncthreads();
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t v = rank_value(keys[i]);
    int c = 0;
#pragma unroll 8
    for (int t = 0; t < RANK_TILE; ++t) c += sj[t] < v ? 1 : 0;
    if (c) atomicAdd(rank + i, c);
}

__global__ void k_rank_scatter(const uint64_t* __restrict__ keys, const int* __restrict__ rank,
                               const unsigned long long* __restrict__ n_dev, int cap, uint64_t* __restrict__ out) {
    pdl_entry();
    const int n = (int)min(*n_dev, (unsigned long long)cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[rank[i]] = keys[i];
}

__global__ void k_bitonic_global(uint64_t* keys, uint64_t n, uint64_t j, uint64_t k) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t p = i ^ j;
        if (p > i) {
            bool up = ((i & k) == 0);
            uint64_t x = keys[i], y = keys[p];
            if (key_less(y, x) == up) {
                keys[i] = y;
                keys[p] = x;
            }
        }
    }
}

__global__ void k_fill_u64(uint64_t* p, uint64_t n, uint64_t v) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// ------------------------------------------------------------------ candidates
// The candidate list: the line of sight (key 0), then the sorted unique keys
// (n of them, read from the compaction count, at most cap); K = n + 1 is stored
// for the later kernels and the host.
__global__ void k_cand_keys(const uint64_t* __restrict__ sorted, const unsigned long long* __restrict__ n_dev,
                            int64_t cap, uint64_t* __restrict__ cand, int64_t* __restrict__ K_dev) {
    pdl_entry();
    const int64_t n = (int64_t)min(*n_dev, (unsigned long long)cap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        cand[i] = i == 0 ? 0ull : sorted[i - 1];
    if (blockIdx.x == 0 && threadIdx.x == 0) *K_dev = n + 1;
}

// Last-bounce frustum of a candidate (image method, Sec. II-F).  A receiver x
// completes the path only if the segment from x to the last image source I_q
// crosses the last triangle: x lies beyond the triangle's plane as seen from
// I_q, and inside the three planes through I_q and the triangle's edges.  Each
// plane is stored in FP32 as a unit normal and offset, f(x) = N.x + w with
// f >= 0 on the inside; F holds 4 such float4 and then (I_q, rho), plane-major
// with stride `stride`.  Everything is formed in FP32 with u = 2^-24:
//  * dI = n.(I_q - v0), the signed distance of I_q from the plane, to within
//    8u (|I_q|_1 + |n.v0|); the frustum is used only where |dI| is 8 times
//    that, so that its sign, which orients every plane, is exact
//    (det(v0 - I, v1 - I, v2 - I) = -dI |(v1 - v0) x (v2 - v0)| fixes the edge
//    planes' orientation too).
//  * an edge normal a_i x a_{i+1}, a_i = v_i - I_q, carries the roundings of
//    I_q and a_i (e_i = u (|I_q|_1 + |a_i|_1) per component) and of the cross
//    product, so its unit normal is off by at most
//    E_i = 2 (2 e_i |a_j|_1 + 2 e_j |a_i|_1 + 4 e_i e_j + 6 u |a_i|_1 |a_j|_1) / |N_i| + 5u,
//    which moves f_i(x) by E_i |x - I_q|.
//  * the grown triangle (barycentric >= -TRI_TOL): the crossing point p has
//    f_i(p) >= -TRI_TOL |v_opp - I_q|, and x = I_q + s (p - I_q) with
//    s <= |x - I_q| / |dI|, so f_i(x) >= -TRI_TOL max_v |v - I_q| / |dI| |x - I_q|.
// rho bounds the sum of the last two per unit |x - I_q| (with a factor 2 of
// room); the remaining roundings (of I_q, the offsets, the planes at a box) are
// below 10u of the magnitudes |x|_1, |I_q|_1, |w_0|, which the tile test's
// 1e-5 term covers.  The test is correct for any rho (at E >= 1 its margin
// exceeds every |f_i|); rho < 0 marks a candidate whose frustum is not used
// (no robust sign of dI, a degenerate edge, or rho > 0.5).
__device__ __forceinline__ void frustum_store(V3<double> I64, const float4* __restrict__ tri_v,
                                              const float4* __restrict__ tri_bary, int t, float4* F, int64_t stride,
                                              int64_t k) {
    const float u = 5.9604645e-8f;
    const V3<float> I = mk((float)I64.x, (float)I64.y, (float)I64.z);
    const float4 pl = __ldg(tri_bary + 3 * t);
    const V3<float> v[3] = {from4<float>(__ldg(tri_v + 3 * t)), from4<float>(__ldg(tri_v + 3 * t + 1)),
                            from4<float>(__ldg(tri_v + 3 * t + 2))};
    const float I1 = fabsf(I.x) + fabsf(I.y) + fabsf(I.z);
    const float dI = pl.x * I.x + pl.y * I.y + pl.z * I.z - pl.w;
    const float errdI = 8.0f * u * (I1 + fabsf(pl.w));
    float4 P[4];
    float rho = -1.0f;
    if (fabsf(dI) > 8.0f * errdI) {
        const float sg = dI > 0.0f ? -1.0f : 1.0f;   // f(I_q) < 0 for plane 0, f(v_opp) > 0 for the edges
        P[0] = make_float4(sg * pl.x, sg * pl.y, sg * pl.z, -sg * pl.w);
        const V3<float> a[3] = {v[0] - I, v[1] - I, v[2] - I};
        float a1[3], e[3], r2 = 0.0f, E = 0.0f;
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            a1[i] = fabsf(a[i].x) + fabsf(a[i].y) + fabsf(a[i].z);
            e[i] = u * (I1 + a1[i]);
            r2 = fmaxf(r2, dot(a[i], a[i]));
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int j = (i + 1) % 3;
            const V3<float> N = cross(a[i], a[j]);
            const float l2 = dot(N, N);
            if (!(l2 > 1e-30f && l2 < 1e30f)) ok = false;
            const float il = rsqrtf(l2);
            const float dN = 2.0f * e[i] * a1[j] + 2.0f * e[j] * a1[i] + 4.0f * e[i] * e[j] + 6.0f * u * a1[i] * a1[j];
            E = fmaxf(E, 2.0f * dN * il + 5.0f * u);
            const float s = sg * il;
            const V3<float> Nh = mk(s * N.x, s * N.y, s * N.z);
            P[i + 1] = make_float4(Nh.x, Nh.y, Nh.z, -dot(Nh, I));
        }
        if (ok) rho = 2.0f * (1.2f * (float)TRI_TOL * sqrtf(r2) / fabsf(dI) + E);
        if (!(rho <= 0.5f)) rho = -1.0f;   // a wider margin than that rejects almost nothing
    }
    for (int i = 0; i < 4; ++i) F[i * stride + k] = rho < 0.0f ? make_float4(0.0f, 0.0f, 0.0f, 0.0f) : P[i];
    F[4 * stride + k] = make_float4(I.x, I.y, I.z, rho);
}

// Per candidate: length q, triangles, and the image sources I_1..I_q of the
// transmitter (I_j = I_{j-1} - 2 ((I_{j-1} - a_j).n_j) n_j), FP64 and FP32.
// The arrays hold Kc slots (slot-major, stride Kc); the slots from *K_dev on are
// marked empty (depth -1) and produce no pairs.
__global__ void k_candidates(const uint64_t* __restrict__ keys, int64_t Kc, const int64_t* __restrict__ K_dev, int D,
                             double tx, double ty, double tz, const float4* __restrict__ tri_v,
                             const double* __restrict__ tri_n64, const float4* __restrict__ tri_bary,
                             int32_t* cand_depth, int32_t* cand_tri, double* img64, float4* img32, float4* frus) {
    pdl_entry();
    const int64_t K = *K_dev;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < Kc; k += (int64_t)gridDim.x * blockDim.x) {
        if (k >= K) {
            cand_depth[k] = -1;
            continue;
        }
        uint64_t key = keys[k];
        int q = rt_key_depth(key);
        cand_depth[k] = q;
        V3<double> I = mk(tx, ty, tz);
        for (int j = 0; j < D; ++j) {
            int t = j < q ? rt_key_tri(key, j) : -1;
            cand_tri[(int64_t)j * Kc + k] = t;
            if (t >= 0) {
                V3<double> n = mk(tri_n64[4 * t], tri_n64[4 * t + 1], tri_n64[4 * t + 2]);
                V3<double> a = from4<double>(__ldg(tri_v + 3 * t));
                I = I - (2.0 * dot(I - a, n)) * n;
            }
            double* o = img64 + ((int64_t)j * Kc + k) * 3;
            o[0] = I.x;
            o[1] = I.y;
            o[2] = I.z;
            img32[(int64_t)j * Kc + k] = make_float4((float)I.x, (float)I.y, (float)I.z, 0.0f);
            if (j == q - 1) frustum_store(I, tri_v, tri_bary, t, frus, Kc, k);
        }
    }
}

// Barycentric coordinates of p in triangle t from its FP64 planes
// lambda_0 = g0.p + h0, lambda_1 = g1.p + h1, lambda_2 = 1 - lambda_0 - lambda_1;
// inside means all >= -TRI_TOL.
__device__ __forceinline__ bool point_in_tri64(const double* __restrict__ bary64, int t, V3<double> p,
                                               double* minbary) {
    const double* g = bary64 + 8 * t;
    double l0 = fma(g[0], p.x, fma(g[1], p.y, fma(g[2], p.z, g[3])));
    double l1 = fma(g[4], p.x, fma(g[5], p.y, fma(g[6], p.z, g[7])));
    double l2 = 1.0 - l0 - l1;
    if (minbary) *minbary = fmin(l0, fmin(l1, l2));
    return l0 >= -TRI_TOL && l1 >= -TRI_TOL && l2 >= -TRI_TOL;
}

struct CandView {
    int64_t K;
    const int32_t* depth;
    const int32_t* tri;   // D x K
    const double* img64;  // D x K x 3
    const float4* img32;  // D x K
    const float4* frus;   // 5 x K: last-bounce frustum (frustum_store); set for the prefilter only
};

// Back-trace of candidate k from receiver position rx (image method, FP64):
// fills pts[0..q+1] = Tx, s_1..s_q, Rx and returns validity of the geometry
// (0 < u < 1, point in the grown triangle, every segment longer than eps).
__device__ __forceinline__ bool backtrace64(const CandView& C, int64_t k, int q, V3<double> tx, V3<double> rx,
                                            const float4* __restrict__ tri_v, const double* __restrict__ tri_n64,
                                            const double* __restrict__ bary64, double eps, V3<double>* pts,
                                            double* minbary) {
    pts[0] = tx;
    pts[q + 1] = rx;
    double mb = 1.0;
    for (int j = q; j >= 1; --j) {
        int t = C.tri[(int64_t)(j - 1) * C.K + k];
        const double* ip = C.img64 + ((int64_t)(j - 1) * C.K + k) * 3;
        V3<double> I = mk(ip[0], ip[1], ip[2]);
        V3<double> n = mk(tri_n64[4 * t], tri_n64[4 * t + 1], tri_n64[4 * t + 2]);
        V3<double> a = from4<double>(__ldg(tri_v + 3 * t));
        V3<double> from = pts[j + 1];
        V3<double> dir = I - from;
        double den = dot(n, dir);
        if (den == 0.0) return false;
        double u = dot(n, a - from) * rcp64(den);
        if (!(u > 0.0 && u < 1.0)) return false;
        V3<double> p = from + u * dir;
        double b;
        if (!point_in_tri64(bary64, t, p, &b)) return false;
        mb = fmin(mb, b);
        pts[j] = p;
    }
    const double eps2 = eps * eps;
    for (int j = 0; j <= q; ++j) {
        V3<double> d = pts[j + 1] - pts[j];
        if (!(dot(d, d) > eps2)) return false;
    }
    if (minbary) *minbary = mb;
    return true;
}

// One back-trace step of the FP32 prefilter (Sec. II-F image method): from P
// towards the image source I4 through the triangle with plane record pl and
// barycentric planes g0, g1.  0 = the pair is invalid by a clear margin, 1 = the
// step passes (P moves to the crossing point), 2 = undecided in FP32 (keep).
__device__ __forceinline__ int prefilter_step(V3<float>& P, float4 I4, float4 pl, float4 g0, float4 g1) {
    const float m = PREFILTER_MARGIN;
    V3<float> n = mk(pl.x, pl.y, pl.z);
    V3<float> dir = mk(I4.x, I4.y, I4.z) - P;
    float den = dot(n, dir);
    if (fabsf(den) < 1e-20f) return 2;
    // approximate division (a few ulp): far inside the prefilter's margin
    float u = __fdividef(pl.w - dot(n, P), den);
    if (u < -m || u > 1.0f + m) return 0;
    V3<float> s = P + u * dir;
    float l0 = g0.x * s.x + g0.y * s.y + g0.z * s.z + g0.w;
    float l1 = g1.x * s.x + g1.y * s.y + g1.z * s.z + g1.w;
    float l2 = 1.0f - l0 - l1;
    if (l0 < -m || l1 < -m || l2 < -m) return 0;
    P = s;
    return 1;
}

// FP32 prefilter of bounces j = q..1 of candidate k from P (the receiver, or
// the crossing point of bounce q + 1), as prefilter_step: 0 = invalid by a
// clear margin, 1 = every step passes, 2 = undecided in FP32.
__device__ __forceinline__ int prefilter32(const CandView& C, int64_t k, int q, V3<float> P,
                                          const float4* __restrict__ tri_bary) {
    for (int j = q; j >= 1; --j) {
        int t = C.tri[(int64_t)(j - 1) * C.K + k];
        float4 I4 = C.img32[(int64_t)(j - 1) * C.K + k];
        const int st = prefilter_step(P, I4, __ldg(tri_bary + 3 * t), __ldg(tri_bary + 3 * t + 1),
                                      __ldg(tri_bary + 3 * t + 2));
        if (st != 1) return st;
    }
    return 1;
}

// The FP32 back-trace of a queued pair (the prefilter's steps again, from the
// receiver R): the crossing points s_q..s_1 and segment j from s_j to s_{j+1}
// (s_0 = Tx, s_{q+1} = Rx), stored as origin with 1 / length in .w and vector.
// Returns the prefilter's verdict (0 invalid, 1 valid, 2 undecided in FP32);
// the segments are complete only for 1.
__device__ __forceinline__ int backtrace32(const CandView& C, int64_t k, int q, V3<float> R, float3 txf,
                                          const float4* __restrict__ tri_bary, unsigned long long w,
                                          unsigned long long qcap, float4* seg_o, float4* seg_d) {
    V3<float> next = R;
    for (int j = q; j >= 0; --j) {
        V3<float> P = mk(txf.x, txf.y, txf.z);
        if (j >= 1) {
            const int t = C.tri[(int64_t)(j - 1) * C.K + k];
            P = next;
            const int st = prefilter_step(P, C.img32[(int64_t)(j - 1) * C.K + k], __ldg(tri_bary + 3 * t),
                                          __ldg(tri_bary + 3 * t + 1), __ldg(tri_bary + 3 * t + 2));
            if (st != 1) return st;
        }
        const V3<float> d = next - P;
        seg_o[(size_t)j * qcap + w] = make_float4(P.x, P.y, P.z, rsqrtf(dot(d, d)));
        seg_d[(size_t)j * qcap + w] = make_float4(d.x, d.y, d.z, 0.0f);
        next = P;
    }
    return 1;
}

// The prefilter's queue of surviving (candidate, receiver) pairs.
struct PairSink {
    uint2* queue;
    unsigned long long* qcount;
    unsigned long long qcap;
    int32_t* overflow;
};

__device__ __forceinline__ float4 shfl4(float4 v, int src) {
    return make_float4(__shfl_sync(FULL, v.x, src), __shfl_sync(FULL, v.y, src), __shfl_sync(FULL, v.z, src),
                       __shfl_sync(FULL, v.w, src));
}

constexpr int PAIR_CC = 32;   // candidates per warp tile (receivers per tile: 32 lanes)
static_assert(PAIR_CC == 32, "one candidate per lane in the tile's frustum test");

// Order-preserving map of a float to an int and back, for warp min/max.
__device__ __forceinline__ int float_order(float x) {
    const int i = __float_as_int(x);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float order_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }
__device__ __forceinline__ float warp_minf(float x) { return order_float(__reduce_min_sync(FULL, float_order(x))); }
__device__ __forceinline__ float warp_maxf(float x) { return order_float(__reduce_max_sync(FULL, float_order(x))); }

// False only if no receiver in the box (centre c, half extents h) can complete
// candidate k's path through its last triangle (frustum_store): some plane's
// largest value over the box is below minus the margin, which covers the
// grown triangle (rho |x - I_q|) and the FP32 roundings of the planes, the
// receivers and the box (1e-5 of the magnitudes involved, far above them).
__device__ __forceinline__ bool frustum_pass(const float4* __restrict__ F, int64_t stride, int64_t k, float3 c,
                                             float3 h) {
    const float4 Ir = __ldg(F + 4 * stride + k);
    if (Ir.w < 0.0f) return true;
    const float hs = h.x + h.y + h.z;
    const float4 p0 = __ldg(F + k);
    const float m = 1e-5f * (fabsf(c.x) + fabsf(c.y) + fabsf(c.z) + hs + fabsf(Ir.x) + fabsf(Ir.y) + fabsf(Ir.z) +
                             fabsf(p0.w)) +
                    Ir.w * (fabsf(c.x - Ir.x) + fabsf(c.y - Ir.y) + fabsf(c.z - Ir.z) + hs);
    bool pass = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 P = i == 0 ? p0 : __ldg(F + i * stride + k);
        const float f = P.x * c.x + P.y * c.y + P.z * c.z + P.w + fabsf(P.x) * h.x + fabsf(P.y) * h.y + fabsf(P.z) * h.z;
        pass = pass && f >= -m;
    }
    return pass;
}

// One warp tile of the image-method prefilter: 32 receivers (one per lane, kept
// in registers) against up to PAIR_CC consecutive candidates.  First each lane
// tests one candidate's last-bounce frustum against the bounding box of the
// tile's receivers; only the candidates that pass are prefiltered per receiver
// (candidate data read once per warp and broadcast).  Survivors are appended to
// the queue as (global candidate, global receiver), one atomic per warp and
// candidate.
__device__ __forceinline__ void pairs_tile(const CandView& C, int64_t k0, int64_t k1, int64_t r_glob, bool r_ok,
                                           float3 rxf, const float4* __restrict__ tri_bary, const PairSink& S) {
    const int lane = threadIdx.x & 31;
    if (!__any_sync(FULL, r_ok)) return;
    const float inf = INFINITY;
    const float lx = warp_minf(r_ok ? rxf.x : inf), ly = warp_minf(r_ok ? rxf.y : inf),
                lz = warp_minf(r_ok ? rxf.z : inf);
    const float ux = warp_maxf(r_ok ? rxf.x : -inf), uy = warp_maxf(r_ok ? rxf.y : -inf),
                uz = warp_maxf(r_ok ? rxf.z : -inf);
    const float3 c = make_float3(0.5f * (lx + ux), 0.5f * (ly + uy), 0.5f * (lz + uz));
    const float3 h = make_float3(0.5f * (ux - lx), 0.5f * (uy - ly), 0.5f * (uz - lz));
    // lane l: candidate k0 + l, its frustum test and the data of its last bounce
    // (image source and the triangle's planes), broadcast below to the lanes
    bool want = false;
    int q_l = -1;
    float4 I_l = make_float4(0.0f, 0.0f, 0.0f, 0.0f), pl_l = I_l, g0_l = I_l, g1_l = I_l;
    if (k0 + lane < k1) {
        const int64_t k = k0 + lane;
        q_l = C.depth[k];
        want = q_l == 0 || (q_l > 0 && frustum_pass(C.frus, C.K, k, c, h));
        if (want && q_l > 0) {
            const int t = C.tri[(int64_t)(q_l - 1) * C.K + k];
            I_l = C.img32[(int64_t)(q_l - 1) * C.K + k];
            pl_l = __ldg(tri_bary + 3 * t);
            g0_l = __ldg(tri_bary + 3 * t + 1);
            g1_l = __ldg(tri_bary + 3 * t + 2);
        }
    }
    unsigned M = __ballot_sync(FULL, want);
    const V3<float> R = mk(rxf.x, rxf.y, rxf.z);
    while (M) {
        const int b = __ffs(M) - 1;
        M &= M - 1;
        const int64_t k = k0 + b;
        const int q = __shfl_sync(FULL, q_l, b);
        const float4 I4 = shfl4(I_l, b), pl = shfl4(pl_l, b), g0 = shfl4(g0_l, b), g1 = shfl4(g1_l, b);
        bool ok = r_ok;
        if (q > 0 && ok) {
            V3<float> P = R;
            int st = prefilter_step(P, I4, pl, g0, g1);
            if (st == 1 && q > 1) st = prefilter32(C, k, q - 1, P, tri_bary);
            ok = st != 0;
        }
        const unsigned m = __ballot_sync(FULL, ok);
        if (m) {
            unsigned long long base = 0;
            const int leader = __ffs(m) - 1;
            if (lane == leader) base = atomicAdd(S.qcount, (unsigned long long)__popc(m));
            base = __shfl_sync(FULL, base, leader);
            if (ok) {
                const unsigned long long slot = base + __popc(m & ((1u << lane) - 1));
                if (slot < S.qcap) S.queue[slot] = make_uint2((unsigned)k, (unsigned)r_glob);
                else atomicExch(S.overflow, 1);
            }
        }
    }
}

// Spatial order of the receivers for the image method's warp tiles (a tile's
// frustum test rejects more candidates when its 32 receivers are close): a
// counting sort, in one block of 1024 threads, by a coarse Morton cell of each
// receiver (4 bits per axis of its position in the receivers' bounding box,
// 4096 cells).  The order only decides which receivers share a tile, not any
// result; within a cell it follows the shared-memory atomics.  Positions are
// narrowed to FP32 with integer operations (truncation), which leaves the FP64
// unit of the one SM alone.
constexpr int RX_ORDER_MAX = 1 << 20;   // receivers of one sort (one block)
constexpr int RX_CELLS = 4096;

__device__ __forceinline__ float narrow_trunc(double v) {   // FP64 -> FP32 toward zero, normal range
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
    if (e <= 0) return 0.0f;
    const uint32_t f = (uint32_t)(b >> 32) & 0x80000000u;
    if (e >= 255) return __int_as_float((int)(f | 0x7f7fffffu));
    return __int_as_float((int)(f | ((uint32_t)e << 23) | (uint32_t)((b >> 29) & 0x7fffffu)));
}

__device__ __forceinline__ uint32_t morton_spread4(uint32_t x) {   // bits 0..3 to every third bit
    x &= 0xfu;
    return (x & 1u) | ((x & 2u) << 2) | ((x & 4u) << 4) | ((x & 8u) << 6);
}

// One block orders the receivers rx[0..R) into order[0..R) (indices into rx).
// Each thread holds up to RX_PER_THREAD receivers' positions and cells in
// registers, so the positions are read once; beyond that they are read again.
constexpr int RX_PER_THREAD = 8;

__device__ __forceinline__ void rx_order_block(const double* __restrict__ rx, int R, int32_t* order) {
    __shared__ int cnt[RX_CELLS];
    __shared__ float sbox[6][32];
    __shared__ int wsum[32];
    for (int c = threadIdx.x; c < RX_CELLS; c += blockDim.x) cnt[c] = 0;
    float px[RX_PER_THREAD][3];
#pragma unroll
    for (int k = 0; k < RX_PER_THREAD; ++k) {
        const int i = threadIdx.x + k * (int)blockDim.x;
#pragma unroll
        for (int c = 0; c < 3; ++c) px[k][c] = i < R ? narrow_trunc(rx[3 * (int64_t)i + c]) : 0.0f;
    }
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int k = 0; k < RX_PER_THREAD; ++k)
        if (threadIdx.x + k * (int)blockDim.x < R)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                lo[c] = fminf(lo[c], px[k][c]);
                hi[c] = fmaxf(hi[c], px[k][c]);
            }
    for (int i = threadIdx.x + RX_PER_THREAD * (int)blockDim.x; i < R; i += blockDim.x)
        for (int c = 0; c < 3; ++c) {
            const float v = narrow_trunc(rx[3 * (int64_t)i + c]);
            lo[c] = fminf(lo[c], v);
            hi[c] = fmaxf(hi[c], v);
        }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    for (int c = 0; c < 3; ++c) {
        lo[c] = warp_minf(lo[c]);
        hi[c] = warp_maxf(hi[c]);
        if (lane == 0) {
            sbox[c][wid] = lo[c];
            sbox[3 + c][wid] = hi[c];
        }
    }
    __syncthreads();
    float sc[3];
    for (int c = 0; c < 3; ++c) {
        lo[c] = warp_minf(lane < nw ? sbox[c][lane] : INFINITY);
        hi[c] = warp_maxf(lane < nw ? sbox[3 + c][lane] : -INFINITY);
        sc[c] = hi[c] > lo[c] ? 15.999f / (hi[c] - lo[c]) : 0.0f;
    }
    auto cell_of = [&](float x, float y, float z) {
        const float v[3] = {x, y, z};
        uint32_t m = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float q = fminf(fmaxf((v[c] - lo[c]) * sc[c], 0.0f), 15.0f);
            m |= morton_spread4((uint32_t)q) << c;
        }
        return (int)m;
    };
    auto cell_far = [&](int i) {
        return cell_of(narrow_trunc(rx[3 * (int64_t)i]), narrow_trunc(rx[3 * (int64_t)i + 1]),
                       narrow_trunc(rx[3 * (int64_t)i + 2]));
    };
    int myc[RX_PER_THREAD];
#pragma unroll
    for (int k = 0; k < RX_PER_THREAD; ++k) {
        myc[k] = cell_of(px[k][0], px[k][1], px[k][2]);
        if (threadIdx.x + k * (int)blockDim.x < R) atomicAdd(&cnt[myc[k]], 1);
    }
    for (int i = threadIdx.x + RX_PER_THREAD * (int)blockDim.x; i < R; i += blockDim.x) atomicAdd(&cnt[cell_far(i)], 1);
    __syncthreads();
    // exclusive scan of the cell counts: RX_CELLS / blockDim.x consecutive cells per thread
    const int per = RX_CELLS / (int)blockDim.x;
    int run = 0;
    for (int k = 0; k < per; ++k) run += cnt[threadIdx.x * per + k];
    int x = run;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int v = lane < nw ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int base = x - run + (wid > 0 ? wsum[wid - 1] : 0);
    for (int k = 0; k < per; ++k) {
        const int c = cnt[threadIdx.x * per + k];
        cnt[threadIdx.x * per + k] = base;   // the cell's next slot
        base += c;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RX_PER_THREAD; ++k) {
        const int i = threadIdx.x + k * (int)blockDim.x;
        if (i < R) order[atomicAdd(&cnt[myc[k]], 1)] = i;
    }
    for (int i = threadIdx.x + RX_PER_THREAD * (int)blockDim.x; i < R; i += blockDim.x)
        order[atomicAdd(&cnt[cell_far(i)], 1)] = i;
}

__global__ void __launch_bounds__(1024) k_rx_order(const double* __restrict__ rx, int R, int32_t* order) {
    rx_order_block(rx, R, order);
}

// One block per scene of a batch: order[rx_off[s] + j] = the scene-local index
// of its j-th receiver in tile order.
__global__ void __launch_bounds__(1024) k_rx_order_batch(const double* __restrict__ rx, const int64_t* rx_off,
                                                         int32_t* order) {
    const int64_t o = rx_off[blockIdx.x];
    rx_order_block(rx + 3 * o, (int)(rx_off[blockIdx.x + 1] - o), order + o);
}

struct PairArgs {
    CandView C;
    int R;
    const double* rx;
    const int32_t* order;   // tile order of the receivers (k_rx_order), or null: as given
    const float4* tri_bary;
    PairSink S;
};

// Image-method prefilter over all (candidate, receiver) pairs, FP32 only, in
// warp tiles (see pairs_tile).  The FP64 work happens on the dense queue.
__global__ void k_pairs(PairArgs A) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int64_t rt_n = (A.R + 31) / 32, kt_n = (A.C.K + PAIR_CC - 1) / PAIR_CC;
    const int64_t tiles = rt_n * kt_n;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp0; t < tiles; t += nwarps) {
        const int64_t kt = t / rt_n, rt = t - kt * rt_n;
        const int64_t rs = rt * 32 + lane;
        const bool r_ok = rs < A.R;
        const int64_t r = r_ok && A.order ? (int64_t)A.order[rs] : rs;
        float3 rxf = make_float3(0.0f, 0.0f, 0.0f);
        if (r_ok) rxf = make_float3((float)A.rx[3 * r], (float)A.rx[3 * r + 1], (float)A.rx[3 * r + 2]);
        const int64_t k0 = kt * PAIR_CC, k1 = min(A.C.K, k0 + PAIR_CC);
        pairs_tile(A.C, k0, k1, r, r_ok, rxf, A.tri_bary, A.S);
    }
}

struct VisArgs {
    CandView C;
    const double* rx;
    double tx, ty, tz;
    const BvhNode* nodes;
    const float4* bvh_tris;
    const float4* tri_v;
    const double* tri_n64;
    const double* bary64;
    const float4* tri_bary;   // FP32 plane records (FP32 back-trace)
    float3 txf;               // Tx rounded to FP32
    double eps;
    const uint2* queue;
    const unsigned long long* qcount;
    unsigned long long qcap;
    uint32_t* bits;
    int64_t words;   // words per receiver row
    int32_t* status;
    unsigned long long* counters;   // optional instrumentation (slots 4..6)
    int D;                          // max depth
    int32_t* seg_q;                 // qcap: depth of a confirmed pair, -1 otherwise
    float4* seg_o;                  // (D + 1) x qcap: segment origin (FP32), 1 / length in .w
    float4* seg_d;                  // (D + 1) x qcap: segment vector (FP32)
};

// Visibility in two launches.  k_backtrace: one thread per queued pair, the
// FP32 back-trace of the prefilter again, which stores the pair's FP32 segments
// and sets its bit (a pair undecided in FP32 is marked -2 and gets its
// segments from the FP64 points in k_segments).  k_segments: one thread per
// (pair, segment), segment-major so that the first segments of all pairs run
// before the second ones: any hit with eps < t*len < len - eps (end triangles
// excluded), FP32 first and FP64 for a marginal segment or a pair marked -2,
// whose FP64 image-method geometry is checked there; a blocked segment clears
// the pair's bit, and a segment whose pair is already cleared is skipped.  The
// FP64 image-method confirmation of the other pairs (0 < u < 1, the point in
// the grown triangle, segments longer than eps) runs in k_points on the dense
// list of the pairs left visible, where an invalid pair is dropped.
__global__ void __launch_bounds__(TRACE_THREADS) k_backtrace(VisArgs A) {
    pdl_entry();
    unsigned long long n = *A.qcount;
    if (n > A.qcap) n = A.qcap;
    for (unsigned long long w = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; w < n;
         w += (unsigned long long)gridDim.x * blockDim.x) {
        const uint2 e = A.queue[w];
        const int64_t k = e.x;
        const int r = (int)e.y;
        const int q = A.C.depth[k];
        const double* rp = A.rx + 3 * (int64_t)r;
        const int st = backtrace32(A.C, k, q, mk((float)rp[0], (float)rp[1], (float)rp[2]), A.txf, A.tri_bary, w,
                                   A.qcap, A.seg_o, A.seg_d);
        A.seg_q[w] = st == 1 ? q : st == 2 ? -2 : -1;
        if (st != 0) atomicOr(A.bits + (int64_t)r * A.words + (k >> 5), 1u << (k & 31));
    }
}

template <int STACK>
__global__ void __launch_bounds__(TRACE_THREADS) k_segments(VisArgs A) {
    pdl_entry();
    extern __shared__ int smem_stack[];
    int* stack = smem_stack + threadIdx.x;
    int* cand = smem_stack + STACK * blockDim.x + threadIdx.x;
    unsigned long long n = *A.qcount;
    if (n > A.qcap) n = A.qcap;
    const unsigned long long total = n * (unsigned long long)(A.D + 1);
    unsigned long long c_vis = 0, c_tri = 0, c_seg = 0;
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < total;
         t += (unsigned long long)gridDim.x * blockDim.x) {
        // segment index and pair: 32-bit division whenever the item count fits
        const int j = total <= 0xffffffffull ? (int)((unsigned)t / (unsigned)n) : (int)(t / n);
        const unsigned long long w = t - (unsigned long long)j * n;
        const int qs = A.seg_q[w];
        if (qs == -1) continue;
        uint2 e = A.queue[w];
        const int64_t k = e.x;
        const int r = (int)e.y;
        const int q = qs >= 0 ? qs : A.C.depth[k];
        if (q < j) continue;
        uint32_t* word = A.bits + (int64_t)r * A.words + (k >> 5);
        const uint32_t bit = 1u << (k & 31);
        if (!(*(volatile uint32_t*)word & bit)) continue;   // another segment already blocked it
        const int s0 = j >= 1 ? A.C.tri[(int64_t)(j - 1) * A.C.K + k] : -1;
        const int s1 = j + 1 <= q ? A.C.tri[(int64_t)j * A.C.K + k] : -1;
        const float epsf = (float)A.eps;
        WRay<float> rf;
        bool hit = false, und = true;
        if (qs >= 0) {
            const float4 o4 = A.seg_o[(size_t)j * A.qcap + w], d4 = A.seg_d[(size_t)j * A.qcap + w];
            rf.o = mk(o4.x, o4.y, o4.z);
            rf.d = mk(d4.x, d4.y, d4.z);
            wray_init(rf);
            und = false;
            unsigned nv = 0, nt = 0;
            const int pl0 = s0 >= 0 ? __float_as_int(__ldg(A.tri_v + 3 * s0 + 1).w) : -1;
            const int pl1 = s1 >= 0 ? __float_as_int(__ldg(A.tri_v + 3 * s1 + 1).w) : -1;
            hit = any32<STACK>(A.nodes, A.bvh_tris, rf, epsf * o4.w, 1.0f - epsf * o4.w, s0, s1, pl0, pl1, stack, und,
                        A.status, nv, nt);
            c_vis += nv;
            c_tri += nt;
            c_seg++;
        }
        if (!hit && und) {
            // marginal, or no FP32 segments: the segment from the FP64 points,
            // final decision in FP64 (a pair invalid in FP64 is cleared here)
            const double* rp = A.rx + 3 * (int64_t)r;
            V3<double> pts[RT_MAX_DEPTH + 2];
            if (!backtrace64(A.C, k, q, mk(A.tx, A.ty, A.tz), mk(rp[0], rp[1], rp[2]), A.tri_v, A.tri_n64, A.bary64,
                             A.eps, pts, nullptr)) {
                atomicAnd(word, ~bit);
                continue;
            }
            V3<double> d = pts[j + 1] - pts[j];
            double il = rsqrt(dot(d, d));
            WRay<double> rd;
            rd.o = pts[j];
            rd.d = d;
            wray_init(rd);
            if (qs < 0) {
                rf.o = mk((float)pts[j].x, (float)pts[j].y, (float)pts[j].z);
                rf.d = mk((float)d.x, (float)d.y, (float)d.z);
                wray_init(rf);
            }
            hit = any64<STACK>(A.nodes, A.bvh_tris, rd, rf, A.eps * il, 1.0 - A.eps * il, s0, s1, stack, cand, A.status);
        }
        if (hit) atomicAnd(word, ~bit);
    }
    if (A.counters) {
        // every thread of the block reaches this point (grid-stride loop above)
        warp_count(A.counters + 4, c_vis);
        warp_count(A.counters + 5, c_tri);
        warp_count(A.counters + 6, c_seg);
    }
}


// Per-receiver popcount of the validity bitmask (one warp per receiver).
__global__ void k_row_count(const uint32_t* __restrict__ bits, int R, int64_t words, int64_t* counts) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < R;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int64_t c = 0;
        for (int64_t w = lane; w < words; w += 32) c += __popc(bits[r * words + w]);
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(FULL, c, o);
        if (lane == 0) counts[r] = c;
    }
}

// Exclusive scan of n int64 counts into offsets[0..n] (single block).
__global__ void k_scan(const int64_t* __restrict__ counts, int n, int64_t* offsets) {
    pdl_entry();
    __shared__ int64_t wsum[32];
    const int T = blockDim.x;   // a multiple of 32, at most 1024
    const int per = (n + T - 1) / T;
    const int lo = threadIdx.x * per, hi = min(n, lo + per);
    // up to 8 counts per thread are loaded at once and kept (n <= 8 T)
    constexpr int KEEP = 8;
    int64_t v[KEEP];
#pragma unroll
    for (int k = 0; k < KEEP; ++k) v[k] = lo + k < hi ? counts[lo + k] : 0;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < KEEP; ++k) s += v[k];
    for (int i = lo + KEEP; i < hi; ++i) s += counts[i];
    // inclusive scan of the per-thread sums: within each warp by shuffles, then
    // over the warp totals by the first warp
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t v = lane < (T >> 5) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += y;
        }
        __syncwarp();
        wsum[lane] = v;
    }
    __syncthreads();
    int64_t run = x - s + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
    for (int k = 0; k < KEEP; ++k)
        if (lo + k < hi) {
            offsets[lo + k] = run;
            run += v[k];
        }
    for (int i = lo + KEEP; i < hi; ++i) {
        offsets[i] = run;
        run += counts[i];
    }
    if (threadIdx.x == T - 1) offsets[n] = run;
}

// Expansion of the bitmask into (receiver, candidate) pairs at their final
// positions, candidates in increasing order within a receiver (one warp each).
// Paths at or beyond cap are not written (the host reads offsets[R] > cap as an
// overflow and traces again with more room).
__global__ void k_expand(const uint32_t* __restrict__ bits, int R, int64_t words, const int64_t* __restrict__ offsets,
                         int32_t* path_rx, int32_t* path_cand, int64_t cap) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < R;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int64_t pos = offsets[r];
        for (int64_t w0 = 0; w0 < words; w0 += 32) {
            int64_t w = w0 + lane;
            uint32_t b = w < words ? bits[r * words + w] : 0u;
            int c = __popc(b);
            int incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                int v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            int64_t my = pos + incl - c;
            while (b) {
                int bit = __ffs(b) - 1;
                b &= b - 1;
                if (my < cap) {
                    path_rx[my] = (int32_t)r;
                    path_cand[my] = (int32_t)(w * 32 + bit);
                }
                my++;
            }
            pos += __shfl_sync(FULL, incl, 31);
        }
    }
}

// FP64 points of every emitted path, its triangle slots, and whether any
// reflection point lies on a triangle edge (input of the duplicate rule).  A
// path whose FP64 image-method geometry is invalid is dropped here (path_cand
// -1, bit cleared), before the duplicate rule and the final compaction.
// P: the number of emitted paths (*P_dev, at most cap), also the slot stride of tri_out.
__global__ void k_points(CandView C, const int64_t* __restrict__ P_dev, int64_t cap, int D,
                         const int32_t* __restrict__ path_rx,
                         int32_t* __restrict__ path_cand, const double* __restrict__ rx, double tx, double ty,
                         double tz, const float4* __restrict__ tri_v, const double* __restrict__ tri_n64,
                         const double* __restrict__ bary64, double eps, double* pts_out, int32_t* depth_out,
                         int32_t* rx_out, int32_t* tri_out, int32_t* edge_flag, uint32_t* bits, int64_t words) {
    pdl_entry();
    const int64_t P = min(*P_dev, cap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = path_cand[i];
        int r = path_rx[i];
        int q = C.depth[k];
        const double* rp = rx + 3 * (int64_t)r;
        V3<double> pts[RT_MAX_DEPTH + 2];
        double mb = 1.0;
        if (!backtrace64(C, k, q, mk(tx, ty, tz), mk(rp[0], rp[1], rp[2]), tri_v, tri_n64, bary64, eps, pts, &mb)) {
            // invalid in FP64 (the image-method confirmation): dropped like a duplicate
            path_cand[i] = -1;
            atomicAnd(bits + (int64_t)r * words + (k >> 5), ~(1u << (k & 31)));
            mb = 1.0;
            q = 0;
            pts[0] = pts[1] = mk(0.0, 0.0, 0.0);
        }
        for (int j = 0; j < D + 2; ++j) {
            V3<double> v = j <= q + 1 ? pts[j] : mk(0.0, 0.0, 0.0);
            double* o = pts_out + ((int64_t)i * (D + 2) + j) * 3;
            o[0] = v.x;
            o[1] = v.y;
            o[2] = v.z;
        }
        depth_out[i] = q;
        rx_out[i] = r;
        for (int j = 0; j < D; ++j) tri_out[(int64_t)j * P + i] = j < q ? C.tri[(int64_t)j * C.K + k] : -1;
        edge_flag[i] = (q > 0 && mb <= 1e-8) ? 1 : 0;
    }
}

// Coplanarity as in the duplicate rule: parallel unit normals (|n_t x n_u| <=
// 1e-9) and the vertex of u within 1e-9 diag of the plane of t.
__device__ __forceinline__ bool coplanar64(const double* __restrict__ tri_n64, const float4* __restrict__ tri_v, int t,
                                           int u, double diag) {
    if (t == u) return true;
    V3<double> a = mk(tri_n64[4 * t], tri_n64[4 * t + 1], tri_n64[4 * t + 2]);
    V3<double> b = mk(tri_n64[4 * u], tri_n64[4 * u + 1], tri_n64[4 * u + 2]);
    V3<double> c = cross(a, b);
    if (dot(c, c) > 1e-18) return false;
    double dt = dot(a, from4<double>(__ldg(tri_v + 3 * t)));
    double du = dot(a, from4<double>(__ldg(tri_v + 3 * u)));
    return fabs(dt - du) <= 1e-9 * diag;
}

// Coplanar-duplicate rule: a path with a reflection point on an edge is dropped
// if another path of its receiver, of equal length, has pairwise coplanar
// triangles, the same points (within 1e-9 diag) and a smaller triangle sequence.
__global__ void k_dedup(const int64_t* __restrict__ P_dev, int64_t cap, int D, const int64_t* __restrict__ rx_offsets,
                        const int32_t* __restrict__ path_rx,
                        int32_t* __restrict__ path_cand, const int32_t* __restrict__ depth,
                        const int32_t* __restrict__ tri, const double* __restrict__ pts,
                        const int32_t* __restrict__ edge_flag, const double* __restrict__ tri_n64,
                        const float4* __restrict__ tri_v, double diag, uint32_t* bits, int64_t words,
                        unsigned long long* drops) {
    pdl_entry();
    const int64_t P = min(*P_dev, cap);
    const double tol2 = (1e-9 * diag) * (1e-9 * diag);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        if (!edge_flag[i]) continue;
        int r = path_rx[i];
        int q = depth[i];
        for (int64_t j = rx_offsets[r]; j < rx_offsets[r + 1] && j < P; ++j) {
            if (j == i || !edge_flag[j] || depth[j] != q) continue;
            bool same = true;
            for (int b = 0; b < q && same; ++b)
                same = coplanar64(tri_n64, tri_v, tri[(int64_t)b * P + i], tri[(int64_t)b * P + j], diag);
            for (int b = 1; b <= q && same; ++b) {
                const double* pi = pts + ((int64_t)i * (D + 2) + b) * 3;
                const double* pj = pts + ((int64_t)j * (D + 2) + b) * 3;
                double dx = pi[0] - pj[0], dy = pi[1] - pj[1], dz = pi[2] - pj[2];
                same = dx * dx + dy * dy + dz * dz <= tol2;
            }
            if (!same) continue;
            bool less = false;
            for (int b = 0; b < q; ++b) {
                int ti = tri[(int64_t)b * P + i], tj = tri[(int64_t)b * P + j];
                if (ti != tj) {
                    less = tj < ti;
                    break;
                }
            }
            if (less) {
                int64_t k = path_cand[i];
                atomicAnd(bits + (int64_t)r * words + (k >> 5), ~(1u << (k & 31)));
                atomicAdd(drops, 1ull);
                path_cand[i] = -1;   // dropped (only this thread reads path_cand[i])
                break;
            }
        }
    }
}

// Copies the paths the duplicate rule kept (path_cand >= 0) into fresh arrays,
// one warp per receiver with a ballot prefix per 32 paths, so that the order
// within a receiver is kept and no path is re-derived.
// P = off[R] (the emitted paths, stride of tri) and Pn = off_n[R] (the kept ones,
// stride of tri_n) are read from device memory, both at most cap.
__global__ void k_compact_paths(int R, int D, int64_t cap, const int64_t* __restrict__ off,
                                const int64_t* __restrict__ off_n, const int32_t* __restrict__ path_cand,
                                const double* __restrict__ pts, const int32_t* __restrict__ depth,
                                const int32_t* __restrict__ rx, const int32_t* __restrict__ tri, double* __restrict__ pts_n,
                                int32_t* __restrict__ depth_n, int32_t* __restrict__ rx_n, int32_t* __restrict__ tri_n) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int64_t P = min(off[R], cap), Pn = min(off_n[R], cap);
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < R;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int64_t w = off_n[r];
        const int64_t o1 = off[r + 1];
        for (int64_t base = off[r]; base < o1; base += 32) {
            const int64_t i = base + lane;
            const bool keep = i < o1 && i < P && path_cand[i] >= 0;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const int64_t j = w + __popc(m & ((1u << lane) - 1u));
            if (keep && j < Pn) {
                for (int e = 0; e < (D + 2) * 3; ++e) pts_n[j * (D + 2) * 3 + e] = pts[i * (D + 2) * 3 + e];
                depth_n[j] = depth[i];
                rx_n[j] = rx[i];
                for (int b = 0; b < D; ++b) tri_n[(int64_t)b * Pn + j] = tri[(int64_t)b * P + i];
            }
            w += __popc(m);
        }
    }
}

// The counts and capacity flags of a pass, checked on the device before its
// records are formed.  meta = {kept paths (0 after an overflow, so that nothing
// reads the slots a cut-short pass may have left unwritten), candidates, overflow
// (0, 1, or 2 for the re-trace list)}.  In a trace that does not wait, an overflow
// also sets RT_ERR_CAPACITY in the status word.
__global__ void k_trace_check(const unsigned long long* __restrict__ tw, const int64_t* __restrict__ P_emit,
                              const int64_t* __restrict__ P_kept, int64_t ucap, int64_t pcap, int64_t* meta,
                              int32_t* status, int report) {
    pdl_entry();
    if (threadIdx.x != 0) return;
    const int32_t f1 = reinterpret_cast<const int32_t*>(tw + 8)[0];
    const int32_t f2 = reinterpret_cast<const int32_t*>(tw + 24)[0];
    const int64_t keys = (int64_t)tw[3];
    const bool ovf = f1 != 0 || f2 != 0 || keys > ucap || *P_emit > pcap;
    meta[0] = ovf ? 0 : min(*P_kept, pcap);
    meta[1] = min(keys, ucap) + 1;
    meta[2] = f1 == 2 ? 2 : (ovf ? 1 : 0);
    if (ovf && report) rt_set_status(status, RT_ERR_CAPACITY);
}

// After an overflowed pass (meta[2] != 0) the receiver offsets may point past the
// slots: every receiver is emptied, so that no later kernel reads beyond them.
__global__ void k_trace_guard(const int64_t* __restrict__ meta, int64_t* offsets, int R) {
    pdl_entry();
    if (meta[2] == 0) return;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= R; r += (int64_t)gridDim.x * blockDim.x)
        offsets[r] = 0;
}

inline int grid_for(rt_ctx* ctx, int64_t n, int threads, int per_sm = 8) {
    int64_t g = (n + threads - 1) / threads;
    int64_t cap = (int64_t)ctx->num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// A kernel launch with programmatic stream serialization (see pdl_entry, which
// every kernel launched this way calls first).  Errors are left to
// cudaGetLastError, as for the <<<>>> launches.
template <typename... KP, typename... Args>
void launch_pdl(void (*kern)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    static_assert(sizeof...(KP) == sizeof...(Args), "launch_pdl: argument count");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    (void)cudaLaunchKernelEx(&cfg, kern, static_cast<KP>(args)...);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host driver of the tracing pipeline.

// Builds (once per ray count) the band order of the coherent ray schedule.
static rt_status ray_schedule(rt_ctx* ctx, int64_t n, RaySched* out) {
    if (ctx->sched_n != n) {
        int64_t band = (int64_t)std::llround(8.0 * std::sqrt((double)n) / 32.0) * 32;
        band = std::max<int64_t>(32, std::min<int64_t>(band, 1 << 20));
        if (band > n) band = 0;
        const int64_t full = band > 0 ? n / band : 0;
        std::vector<int32_t> order(std::max<int64_t>(band, 1)), wrap(std::max<int64_t>(full, 1));
        if (band > 0) {
            std::vector<uint32_t> key(band);
            for (int64_t k = 0; k < band; ++k) {
                key[k] = (uint32_t)((uint64_t)k * 0x9E3779B9ull);
                order[k] = (int32_t)k;
            }
            std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
            std::vector<uint32_t> sk(band);
            for (int64_t j = 0; j < band; ++j) sk[j] = key[order[j]];
            for (int64_t b = 0; b < full; ++b) {
                // fractions of band b are (sk + c) mod 2^32: they wrap where sk >= 2^32 - c
                const uint32_t c = (uint32_t)((uint64_t)(b * band) * 0x9E3779B9ull);
                int64_t j = 0;
                if (c != 0) j = std::lower_bound(sk.begin(), sk.end(), (uint32_t)(0u - c)) - sk.begin();
                wrap[b] = (int32_t)(j == band ? 0 : j);
            }
        }
        // z of every launch direction, in FP64 as the definition states, once per N
        // (an FP64 division per ray inside the tracing kernel would cost a
        // full-warp FP64 sequence on every refill)
        std::vector<float> z(n);
        for (int64_t i = 0; i < n; ++i) z[i] = (float)(1.0 - (double)(2 * i + 1) / (double)n);
        if (ctx->d_sched_order) RT_CK(ctx, cudaFree(ctx->d_sched_order));
        if (ctx->d_sched_wrap) RT_CK(ctx, cudaFree(ctx->d_sched_wrap));
        if (ctx->d_sched_z) RT_CK(ctx, cudaFree(ctx->d_sched_z));
        ctx->d_sched_order = ctx->d_sched_wrap = nullptr;
        ctx->d_sched_z = nullptr;
        ctx->sched_n = 0;
        RT_CK(ctx, cudaMalloc((void**)&ctx->d_sched_order, order.size() * 4));
        RT_CK(ctx, cudaMalloc((void**)&ctx->d_sched_wrap, wrap.size() * 4));
        RT_CK(ctx, cudaMalloc((void**)&ctx->d_sched_z, z.size() * 4));
        RT_CK(ctx, cudaMemcpy(ctx->d_sched_order, order.data(), order.size() * 4, cudaMemcpyHostToDevice));
        RT_CK(ctx, cudaMemcpy(ctx->d_sched_wrap, wrap.data(), wrap.size() * 4, cudaMemcpyHostToDevice));
        RT_CK(ctx, cudaMemcpy(ctx->d_sched_z, z.data(), z.size() * 4, cudaMemcpyHostToDevice));
        ctx->sched_n = n;
        ctx->sched_band = band;
        ctx->sched_full = full;
    }
    *out = RaySched{ctx->sched_n, ctx->sched_band, ctx->sched_full, ctx->d_sched_order, ctx->d_sched_wrap,
                    ctx->d_sched_z};
    return RT_OK;
}

static bool stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// Stage events of the trace (profiling bit 0); none inside a stream capture.
static void mark(rt_ctx* ctx, int k) {
    if (k == 0) ctx->stage_pending = 0;   // a new trace: unread stage times of the last one are dropped
    if ((ctx->profile & 1) && !stream_capturing(ctx->stream)) cudaEventRecord(ctx->ev[k], ctx->stream);
}

struct Arena {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t n) {
        off = align_up(off, 256);
        T* p = reinterpret_cast<T*>(base + off);
        off += n * sizeof(T);
        return p;
    }
};

extern "C" __attribute__((visibility("default"))) rt_status rt_set_trace_async(rt_ctx* ctx, int32_t enable) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (enable != 0 && enable != 1) return rt_fail(ctx, RT_ERR_INVALID_ARG, "enable must be 0 or 1");
    ctx->trace_async = enable;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_paths_resolve(rt_paths* p) {
    if (!p) return RT_ERR_INVALID_ARG;
    if (!p->d_count) return RT_OK;
    rt_ctx* ctx = p->scene->ctx;
    int64_t* hp = ctx->h_pinned;
    RT_CK(ctx, cudaMemcpyAsync(hp, p->d_count, 3 * 8, cudaMemcpyDeviceToHost, p->stream));
    RT_CK(ctx, cudaStreamSynchronize(p->stream));
    if (hp[2] == 2) return rt_fail(ctx, RT_ERR_CAPACITY, "FP64 re-trace list overflow");
    if (hp[2]) return rt_fail(ctx, RT_ERR_CAPACITY, "a trace capacity overflowed: trace again with waiting on");
    p->P = hp[0];
    p->K = hp[1];
    p->d_count = nullptr;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_trace_paths(rt_ctx* ctx, const rt_scene* scene, const double* tx_host, const double* rx_dev,
                                    int32_t n_rx, int64_t n_rays, int32_t max_depth, rt_paths** out) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!scene || !tx_host || !rx_dev || !out) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    if (n_rx < 1 || n_rx > (1 << 24)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_rx out of range");
    if (n_rays < 1 || n_rays > 0x7fffffffLL) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_rays out of range");
    if (max_depth < 1 || max_depth > RT_MAX_DEPTH) return rt_fail(ctx, RT_ERR_INVALID_ARG, "max_depth must be 1..4");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(tx_host[c])) return rt_fail(ctx, RT_ERR_NUMERIC, "non-finite transmitter position");
    *out = nullptr;
    rt_scene* sc = const_cast<rt_scene*>(scene);
    cudaStream_t st = ctx->stream;
    const int D = max_depth;
    int32_t* status = rt_status_ptr(ctx);
    const size_t stack_bytes = (size_t)RT_STACK * TRACE_THREADS * sizeof(int);
    const size_t vis_bytes = (size_t)(RT_STACK + VIS_CAND_CAP) * TRACE_THREADS * sizeof(int);
    // inside a stream capture (a CUDA graph) the trace does not wait: its capacities
    // come from an earlier trace of the scene outside the capture
    const bool in_capture = stream_capturing(st);
    if (in_capture && (sc->uniq_hint == 0 || sc->paths_hint == 0))
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "a trace inside a stream capture needs an earlier trace of the scene");
    const bool async = ctx->trace_async || in_capture;

    // One pass of the whole pipeline with buffers sized from capacities (the hash
    // table, the unique candidates, the visibility queue and the paths: the scene
    // remembers the last counts), the counts of each stage read on the device by
    // the next; a single read-back at the end checks every capacity, and a pass
    // that overflowed one is run again with more room.
    const int64_t redo_cap = std::max<int64_t>(1 << 16, n_rays / 16);
    unsigned long long* tw = ctx->d_trace_words;   // 64 words, see rt_ctx
    unsigned long long* c1 = tw;                    // SBR: uniq, next_ray, redo_count, compacted keys
    int32_t* f1 = reinterpret_cast<int32_t*>(tw + 8);   // SBR flags: hash overflow (1), re-trace list (2)
    unsigned long long* c2 = tw + 16;               // visibility queue count, .., [4] duplicates dropped
    int32_t* f2 = reinterpret_cast<int32_t*>(tw + 24);  // queue overflow
    int64_t* K_dev = reinterpret_cast<int64_t*>(tw + 28);
    // the receivers' tile order for the image method (k_rx_order) depends only on
    // the receivers: it runs on the side stream, beside the SBR, and the image
    // method waits for it (inside a stream capture, a parallel branch)
    int32_t* rx_order = nullptr;
    if (n_rx > 32 && n_rx <= RX_ORDER_MAX) {
        if (ctx->rx_order_cap < n_rx && !in_capture) {
            if (ctx->d_rx_order) RT_CK(ctx, cudaFree(ctx->d_rx_order));
            ctx->d_rx_order = nullptr;
            ctx->rx_order_cap = 0;
            RT_CK(ctx, cudaMalloc((void**)&ctx->d_rx_order, (size_t)n_rx * sizeof(int32_t)));
            ctx->rx_order_cap = n_rx;
        }
        if (ctx->rx_order_cap >= n_rx) {   // (a capture with too small a buffer keeps the given order)
            RT_CK(ctx, cudaEventRecord(ctx->ev_fork, st));
            RT_CK(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
            k_rx_order<<<1, 1024, 0, ctx->side>>>(rx_dev, n_rx, ctx->d_rx_order);
            RT_COUNT(ctx);
            RT_CK(ctx, cudaEventRecord(ctx->ev_join, ctx->side));
            rx_order = ctx->d_rx_order;
        }
    }
    for (int attempt = 0;; ++attempt) {
        if (attempt >= 8) return rt_fail(ctx, RT_ERR_CAPACITY, "trace capacities did not converge");
        const size_t cap = sc->hash_cap;
        // unique keys: the last count with room, at most the table's limit
        int64_t ucap = std::max<int64_t>(1024, sc->uniq_hint + sc->uniq_hint / 8 + 256);
        ucap = std::min<int64_t>(ucap, (int64_t)(cap / 2));
        const bool rank_sort = ucap <= RANK_SORT_MAX;
        int64_t n_pad = SORT_BLOCK;
        while (n_pad < ucap) n_pad <<= 1;
        const int64_t Kc = ucap + 1;
        const int64_t words = (Kc + 31) / 32;
        const size_t qcap = sc->queue_cap;

        // ---------------- 1-2: SBR into the hash set
        const size_t need1 = cap * 8 + (size_t)n_pad * 8 + redo_cap * 16 + (size_t)RANK_SORT_MAX * 12 + 4096;
        void* base;
        rt_status s = rt_scratch(ctx, need1, &base);
        if (s != RT_OK) return s;
        Arena ar{(char*)base};
        unsigned long long* table = ar.take<unsigned long long>(cap);
        int64_t* redo = ar.take<int64_t>(redo_cap);
        uint64_t* redo_key = ar.take<uint64_t>(redo_cap);
        uint64_t* sorted = ar.take<uint64_t>(n_pad);
        uint64_t* unsorted = ar.take<uint64_t>(RANK_SORT_MAX);
        int* rank = ar.take<int>(RANK_SORT_MAX);
        mark(ctx, 0);
        RT_CK(ctx, cudaMemsetAsync(table, 0, cap * 8, st));
        RT_CK(ctx, cudaMemsetAsync(tw, 0, 64 * 8, st));
        SbrArgs A;
        A.nodes = sc->d_nodes;
        A.tris = sc->d_bvh_tris;
        A.tx = tx_host[0];
        A.ty = tx_host[1];
        A.tz = tx_host[2];
        A.txf = make_float3((float)tx_host[0], (float)tx_host[1], (float)tx_host[2]);
        A.n_rays = n_rays;
        A.depth = D;
        A.eps = sc->eps;
        A.table = table;
        A.mask = cap - 1;
        A.uniq = c1 + 0;
        A.uniq_limit = cap / 2;
        A.overflow = f1;
        A.next_ray = c1 + 1;
        A.redo = redo;
        A.redo_key = redo_key;
        A.redo_count = c1 + 2;
        A.redo_cap = redo_cap;
        A.status = status;
        A.counters = (ctx->profile & 2) ? ctx->d_counters : nullptr;
        {
            rt_status ss = ray_schedule(ctx, n_rays, &A.sched);
            if (ss != RT_OK) return ss;
        }
        int blocks = ctx->num_sms * ctx->tune_sbr_blocks_per_sm;
        mark(ctx, 6);
        // a stack of 32 entries when the scene's tree allows it: half the shared
        // memory per block, so more blocks of the latency-bound kernel per SM
        if (sc->bvh_depth <= 32)
            k_sbr<32><<<blocks, TRACE_THREADS, (size_t)32 * TRACE_THREADS * sizeof(int), st>>>(A, sc->d_tri_bary);
        else
            k_sbr<RT_STACK><<<blocks, TRACE_THREADS, stack_bytes, st>>>(A, sc->d_tri_bary);
        RT_COUNT(ctx);
        mark(ctx, 7);
        RT_CK_LAUNCH(ctx);
        launch_pdl(k_sbr_redo, ctx->num_sms * REDO_BLOCKS_PER_SM, REDO_THREADS, (size_t)(RT_STACK + 3 * CAND_CAP) * REDO_THREADS * sizeof(int), st, A, sc->d_tri_n64, sc->d_tri_v);
        RT_COUNT(ctx);
        mark(ctx, 1);
        RT_CK_LAUNCH(ctx);
        if (sc->uniq_hint == 0) {
            // the scene's first trace: learn the number of unique keys (later traces
            // size from the last count and do not wait here)
            RT_CK(ctx, cudaMemcpyAsync(ctx->h_pinned, c1, 8, cudaMemcpyDeviceToHost, st));
            RT_CK(ctx, cudaStreamSynchronize(st));
            sc->uniq_hint = std::max<int64_t>(1, ctx->h_pinned[0]);
            if (sc->uniq_hint > ucap && ucap < (int64_t)(cap / 2)) continue;
        }
        // ---------------- compact + sort (length, lexicographic), at most ucap keys
        if (rank_sort) {
            RT_CK(ctx, cudaMemsetAsync(rank, 0, (size_t)RANK_SORT_MAX * 4, st));
            launch_pdl(k_table_compact, grid_for(ctx, cap, 256, 16), 256, 0, st, table, cap, unsorted, c1 + 3, (uint64_t)ucap);
            RT_COUNT(ctx);
            const int n = (int)ucap;
            launch_pdl(k_rank_count, dim3((n + RANK_TILE - 1) / RANK_TILE, (n + 255) / 256), 256, 0, st, unsorted, c1 + 3, n,
                                                                                                 rank);
            RT_COUNT(ctx);
            launch_pdl(k_rank_scatter, grid_for(ctx, n, 256), 256, 0, st, unsorted, rank, c1 + 3, n, sorted);
            RT_COUNT(ctx);
        } else {
            k_fill_u64<<<grid_for(ctx, n_pad, 256), 256, 0, st>>>(sorted, n_pad, ~0ull); RT_COUNT(ctx);
            launch_pdl(k_table_compact, grid_for(ctx, cap, 256, 16), 256, 0, st, table, cap, sorted, c1 + 3, (uint64_t)ucap);
            RT_COUNT(ctx);
            k_bitonic_local<<<(unsigned)(n_pad / SORT_BLOCK), 1024, 0, st>>>(sorted); RT_COUNT(ctx);
            for (uint64_t k = 2 * SORT_BLOCK; k <= (uint64_t)n_pad; k <<= 1) {
                for (uint64_t j = k >> 1; j >= (uint64_t)SORT_BLOCK; j >>= 1) {
                    k_bitonic_global<<<grid_for(ctx, n_pad, 256, 16), 256, 0, st>>>(sorted, n_pad, j, k);
                    RT_COUNT(ctx);
                }
                k_bitonic_merge_local<<<(unsigned)(n_pad / SORT_BLOCK), 1024, 0, st>>>(sorted, k); RT_COUNT(ctx);
            }
        }
        RT_CK_LAUNCH(ctx);

        // ---------------- candidates (LoS first), Kc slots
        rt_paths* p = new rt_paths();
        p->scene = scene;
        p->stream = st;
        p->D = D;
        p->R = n_rx;
        auto fail = [&](rt_status e) {
            rt_paths_free(p);
            return e;
        };
#define TCK(call)                                                         \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return fail(rt_cuda_fail(ctx, _e, #call)); \
    } while (0)
        TCK(cudaMallocAsync((void**)&p->d_cand, Kc * 8, st));
        launch_pdl(k_cand_keys, grid_for(ctx, Kc, 256), 256, 0, st, sorted, c1 + 3, ucap, p->d_cand, K_dev); RT_COUNT(ctx);
        TCK(cudaGetLastError());

        // candidate arrays + visibility queue + bitmask: a fresh scratch layout (the
        // sorted keys above are consumed first, in stream order)
        const size_t need2 = Kc * 4 + (size_t)D * Kc * 4 + (size_t)D * Kc * 24 + (size_t)D * Kc * 16 + qcap * 8 +
                             (size_t)n_rx * words * 4 + (size_t)(n_rx + 1) * 8 * 2 + qcap * 4 +
                             2 * (size_t)(D + 1) * qcap * 16 + 5 * Kc * 16 + 20 * 256;
        s = rt_scratch(ctx, need2, &base);
        if (s != RT_OK) return fail(s);
        Arena ar2{(char*)base};
        int32_t* cand_depth = ar2.take<int32_t>(Kc);
        int32_t* cand_tri = ar2.take<int32_t>((size_t)D * Kc);
        double* img64 = ar2.take<double>((size_t)D * Kc * 3);
        float4* img32 = ar2.take<float4>((size_t)D * Kc);
        uint2* queue = ar2.take<uint2>(qcap);
        uint32_t* bits = ar2.take<uint32_t>((size_t)n_rx * words);
        int64_t* counts = ar2.take<int64_t>(n_rx + 1);
        int32_t* seg_q = ar2.take<int32_t>(qcap);
        float4* seg_o = ar2.take<float4>((size_t)(D + 1) * qcap);
        float4* seg_d = ar2.take<float4>((size_t)(D + 1) * qcap);
        float4* frus = ar2.take<float4>(5 * (size_t)Kc);
        TCK(cudaMemsetAsync(bits, 0, (size_t)n_rx * words * 4, st));
        launch_pdl(k_candidates, grid_for(ctx, Kc, 32, 32), 32, 0, st, p->d_cand, Kc, K_dev, D, tx_host[0], tx_host[1], tx_host[2],
                                                             sc->d_tri_v, sc->d_tri_n64, sc->d_tri_bary, cand_depth,
                                                             cand_tri, img64, img32, frus); RT_COUNT(ctx);
        TCK(cudaGetLastError());
        PairArgs PA{};
        PA.C = CandView{Kc, cand_depth, cand_tri, img64, img32, frus};
        PA.R = n_rx;
        PA.rx = rx_dev;
        PA.order = rx_order;
        if (rx_order) TCK(cudaStreamWaitEvent(st, ctx->ev_join, 0));   // the side stream's tile order
        PA.tri_bary = sc->d_tri_bary;
        PA.S = PairSink{queue, c2, qcap, f2};
        mark(ctx, 2);
        launch_pdl(k_pairs, grid_for(ctx, ((Kc + PAIR_CC - 1) / PAIR_CC) * ((n_rx + 31) / 32) * 32, 256,
                           ctx->tune_pairs_blocks_per_sm),
                  256, 0, st, PA); RT_COUNT(ctx);
        mark(ctx, 3);
        TCK(cudaGetLastError());
        VisArgs VA{};
        VA.C = PA.C;
        VA.rx = rx_dev;
        VA.tx = tx_host[0];
        VA.ty = tx_host[1];
        VA.tz = tx_host[2];
        VA.nodes = sc->d_nodes;
        VA.bvh_tris = sc->d_bvh_tris;
        VA.tri_v = sc->d_tri_v;
        VA.tri_n64 = sc->d_tri_n64;
        VA.bary64 = sc->d_tri_bary64;
        VA.tri_bary = sc->d_tri_bary;
        VA.txf = make_float3((float)tx_host[0], (float)tx_host[1], (float)tx_host[2]);
        VA.eps = sc->eps;
        VA.queue = queue;
        VA.qcount = c2;
        VA.qcap = qcap;
        VA.bits = bits;
        VA.words = words;
        VA.status = status;
        VA.counters = (ctx->profile & 2) ? ctx->d_counters : nullptr;
        VA.D = D;
        VA.seg_q = seg_q;
        VA.seg_o = seg_o;
        VA.seg_d = seg_d;
        launch_pdl(k_backtrace, ctx->num_sms * 8, TRACE_THREADS, 0, st, VA); RT_COUNT(ctx);
        TCK(cudaGetLastError());
        // a 32-entry traversal stack when the scene's tree allows it (as k_sbr): less
        // shared memory per block, so more of L1 holds the BVH
        if (sc->bvh_depth <= 32)
            launch_pdl(k_segments<32>, ctx->num_sms * ctx->tune_vis_blocks_per_sm, TRACE_THREADS,
                       (size_t)(32 + VIS_CAND_CAP) * TRACE_THREADS * sizeof(int), st, VA);
        else
            launch_pdl(k_segments<RT_STACK>, ctx->num_sms * ctx->tune_vis_blocks_per_sm, TRACE_THREADS, vis_bytes, st,
                       VA);
        RT_COUNT(ctx);
        mark(ctx, 4);
        TCK(cudaGetLastError());
        int64_t* off_e = nullptr;   // offsets of the emitted paths (before the duplicate rule)
        TCK(cudaMallocAsync((void**)&off_e, (size_t)(n_rx + 1) * 8, st));
        launch_pdl(k_row_count, grid_for(ctx, (int64_t)n_rx * 32, 256, 16), 256, 0, st, bits, n_rx, words, counts); RT_COUNT(ctx);
        launch_pdl(k_scan, 1, 1024, 0, st, counts, n_rx, off_e); RT_COUNT(ctx);
        TCK(cudaGetLastError());
        if (sc->paths_hint == 0) {
            // the scene's first trace: learn the number of emitted paths
            TCK(cudaMemcpyAsync(ctx->h_pinned, off_e + n_rx, 8, cudaMemcpyDeviceToHost, st));
            TCK(cudaStreamSynchronize(st));
            sc->paths_hint = std::max<int64_t>(1, ctx->h_pinned[0]);
        }
        const int64_t pcap = std::max<int64_t>(1024, sc->paths_hint + sc->paths_hint / 8 + 1024);

        // ---------------- emission (pcap slots), the duplicate rule, then the kept
        // paths compacted into the final arrays
        const size_t Pa = (size_t)pcap;
        int32_t* path_cand = nullptr;
        int32_t* edge = nullptr;
        char* tmp = nullptr;   // emitted paths before the duplicate rule
        RtCarve ct;
        const size_t t_pts = ct.take(Pa * (D + 2) * 3 * 8), t_depth = ct.take(Pa * 4), t_rx = ct.take(Pa * 4),
                     t_tri = ct.take(Pa * D * 4), t_cand = ct.take(Pa * 4), t_edge = ct.take(Pa * 4);
        TCK(cudaMallocAsync((void**)&tmp, ct.off, st));
        double* pts_e = reinterpret_cast<double*>(tmp + t_pts);
        int32_t* depth_e = reinterpret_cast<int32_t*>(tmp + t_depth);
        int32_t* rx_e = reinterpret_cast<int32_t*>(tmp + t_rx);
        int32_t* tri_e = reinterpret_cast<int32_t*>(tmp + t_tri);
        path_cand = reinterpret_cast<int32_t*>(tmp + t_cand);
        edge = reinterpret_cast<int32_t*>(tmp + t_edge);
        int64_t* meta = nullptr;
        {
            RtCarve c;
            const size_t o_pts = c.take(Pa * (D + 2) * 3 * 8), o_depth = c.take(Pa * 4), o_rx = c.take(Pa * 4),
                         o_tri = c.take(Pa * D * 4), o_meta = c.take(4 * 8);
            char* b = nullptr;
            TCK(cudaMallocAsync((void**)&b, c.off, st));
            p->d_block_geo = b;
            p->d_pts = reinterpret_cast<double*>(b + o_pts);
            p->d_depth = reinterpret_cast<int32_t*>(b + o_depth);
            p->d_rx = reinterpret_cast<int32_t*>(b + o_rx);
            p->d_tri = reinterpret_cast<int32_t*>(b + o_tri);
            meta = reinterpret_cast<int64_t*>(b + o_meta);
        }
        TCK(cudaMallocAsync((void**)&p->d_rx_offsets, (size_t)(n_rx + 1) * 8, st));
        const int64_t* P_e = off_e + n_rx;
        launch_pdl(k_expand, grid_for(ctx, (int64_t)n_rx * 32, 256, 16), 256, 0, st, bits, n_rx, words, off_e, rx_e, path_cand,
                                                                             pcap); RT_COUNT(ctx);
        CandView C{Kc, cand_depth, cand_tri, img64, img32};
        launch_pdl(k_points, grid_for(ctx, pcap, 32, 32), 32, 0, st, C, P_e, pcap, D, rx_e, path_cand, rx_dev, tx_host[0],
                                                           tx_host[1], tx_host[2], sc->d_tri_v, sc->d_tri_n64,
                                                           sc->d_tri_bary64, sc->eps, pts_e, depth_e, rx_e, tri_e, edge,
                                                           bits, words); RT_COUNT(ctx);
        launch_pdl(k_dedup, grid_for(ctx, pcap, 256), 256, 0, st, P_e, pcap, D, off_e, rx_e, path_cand, depth_e, tri_e, pts_e,
                                                          edge, sc->d_tri_n64, sc->d_tri_v, sc->diag, bits, words,
                                                          c2 + 4); RT_COUNT(ctx);
        launch_pdl(k_row_count, grid_for(ctx, (int64_t)n_rx * 32, 256, 16), 256, 0, st, bits, n_rx, words, counts); RT_COUNT(ctx);
        launch_pdl(k_scan, 1, 1024, 0, st, counts, n_rx, p->d_rx_offsets); RT_COUNT(ctx);
        launch_pdl(k_compact_paths, grid_for(ctx, (int64_t)n_rx * 32, 256, 16), 256, 0, st, n_rx, D, pcap, off_e, p->d_rx_offsets, path_cand, pts_e, depth_e, rx_e, tri_e, p->d_pts, p->d_depth,
            p->d_rx, p->d_tri); RT_COUNT(ctx);
        TCK(cudaGetLastError());
        launch_pdl(k_trace_check, 1, 32, 0, st, tw, off_e + n_rx, p->d_rx_offsets + n_rx, ucap, pcap, meta, status, async);
        RT_COUNT(ctx);
        launch_pdl(k_trace_guard, grid_for(ctx, n_rx + 1, 256), 256, 0, st, meta, p->d_rx_offsets, n_rx);
        RT_COUNT(ctx);
        TCK(cudaGetLastError());
        p->P = pcap;   // the slots of the record arrays; set to the count below
        rt_status rs = rt_launch_paths_records(ctx, p, meta);
        if (rs != RT_OK) return fail(rs);
        cudaFreeAsync(tmp, st);
        if (async) {
            // no read-back: the paths are counted on the device; the scene keeps its
            // capacities from the last trace that was read back
            cudaFreeAsync(off_e, st);
            p->K = Kc;
            p->d_count = meta;
            if ((ctx->profile & 1) && !in_capture) {
                TCK(cudaEventRecord(ctx->ev[5], st));
                ctx->stage_pending = 1;
            }
            *out = p;
            return RT_OK;
        }

        // ---------------- the one read-back: every count and capacity flag
        int64_t* hp = ctx->h_pinned;
        TCK(cudaMemcpyAsync(hp, tw, 32 * 8, cudaMemcpyDeviceToHost, st));
        TCK(cudaMemcpyAsync(hp + 32, off_e + n_rx, 8, cudaMemcpyDeviceToHost, st));
        TCK(cudaMemcpyAsync(hp + 33, p->d_rx_offsets + n_rx, 8, cudaMemcpyDeviceToHost, st));
        cudaFreeAsync(off_e, st);
        TCK(cudaStreamSynchronize(st));
        const int32_t ovf1 = reinterpret_cast<const int32_t*>(hp + 8)[0];
        const int64_t n_keys = hp[3];
        const int32_t ovf2 = reinterpret_cast<const int32_t*>(hp + 24)[0];
        const int64_t P_emit = hp[32], P_kept = hp[33];
        if (ovf1 == 2) return fail(rt_fail(ctx, RT_ERR_CAPACITY, "FP64 re-trace list overflow"));
        bool again = false;
        if (ovf1) {
            if (sc->hash_cap >= ((size_t)1 << 31)) return fail(rt_fail(ctx, RT_ERR_CAPACITY, "candidate hash table overflow"));
            sc->hash_cap *= 4;
            again = true;
        }
        if (n_keys > ucap) {
            sc->uniq_hint = n_keys;
            again = true;
        }
        if (ovf2) {
            sc->queue_cap *= 4;
            again = true;
        }
        if (P_emit > pcap) {
            sc->paths_hint = P_emit;
            again = true;
        }
        if (again) {
            rt_paths_free(p);
            continue;
        }
        sc->uniq_hint = n_keys;
        sc->paths_hint = P_emit;
        ctx->h_counters[7] += (n_keys + 1) * (int64_t)n_rx;
        p->K = n_keys + 1;
        p->P = P_kept;
        if (ctx->profile & 1) {
            // read out by rt_collect_stage_times: the trace itself does not wait
            TCK(cudaEventRecord(ctx->ev[5], st));
            ctx->stage_pending = 1;
        }
#undef TCK
        *out = p;
        return RT_OK;
    }
}

// ===========================================================================
// Batched tracing of many scenes (uneven sizes) in one pipeline.
//
// SBR runs as ONE persistent launch over the rays of all scenes: lanes refill
// from a global ray counter and find their scene by binary search in the
// prefix of per-scene ray counts, so warps stay full across scene boundaries
// and a small scene never leaves SMs idle.  Every later stage is likewise one
// launch over the concatenated (scene, candidate, receiver) index spaces.  The
// output is one paths object: receivers concatenated in scene order, triangle
// ids offset per scene into combined triangle tables.

namespace {

struct SceneDev {
    const BvhNode* nodes;
    const float4* bvh_tris;
    const float4* tri_v;
    const float4* tri_bary;
    const double* tri_n64;
    const double* bary64;
    double tx, ty, tz, eps;
    float3 txf;   // Tx rounded to FP32 (origin of the FP32 launch rays)
    int64_t n_rays;
    int32_t tri_off;
};

template <typename T>
__device__ __forceinline__ int find_seg(const T* __restrict__ off, int n, T idx) {   // last s with off[s] <= idx
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= idx) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct BatchSbr {
    const SceneDev* sd;
    const int64_t* ray_off;   // n + 1
    int n;
    int depth;
    unsigned long long* tables;   // n x cap
    uint64_t cap;
    unsigned long long* uniq;     // n
    unsigned long long uniq_limit;
    int32_t* overflow;
    unsigned long long* next_ray;
    int64_t* redo;                  // global ray | (undecided bounce << 32)
    uint64_t* redo_key;             // key of the robust prefix
    unsigned long long* redo_count;
    int64_t redo_cap;
    int32_t* status;
    int blocks_per_sm;
    unsigned long long* counters;   // optional instrumentation (slots 0..3)
    RaySched sched;
};

// Scene descriptor fields a lane needs on every bounce are loaded once, when the
// lane takes a ray, and kept in registers (lanes of one warp may hold rays of
// different scenes).
template <int STACK>
__global__ void __launch_bounds__(TRACE_THREADS, 6) k_sbr_batch(BatchSbr A) {
    extern __shared__ int smem_stack[];
    int* stack = smem_stack + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int64_t total = A.ray_off[A.n];
    int64_t ray = -1;
    bool done = false;
    int bounce = 0, prev = -1, prev_plane = -1;
    uint64_t key = 0;
    WRay<float> r;
    const BvhNode* nodes = nullptr;
    const float4* bvh_tris = nullptr;
    const float4* tri_plane = nullptr;   // the scene's plane records (sbr_bounce)
    unsigned long long* table = nullptr;
    unsigned long long* uniq = nullptr;
    float eps = 0.f;
    float Do = 0.0f, Dd = 0.0f;   // drift of the FP32 ray from the FP64 one (sbr_bounce)
    unsigned long long c_vis = 0, c_tri = 0, c_q = 0;
    for (;;) {
        bool need = (ray < 0) && !done;
        unsigned m = __ballot_sync(FULL, need);
        if (m) {
            unsigned long long base = 0;
            int leader = __ffs(m) - 1;
            if (lane == leader) base = atomicAdd(A.next_ray, (unsigned long long)__popc(m));
            base = __shfl_sync(FULL, base, leader);
            if (need) {
                int64_t idx = (int64_t)(base + __popc(m & ((1u << lane) - 1)));
                if (idx < total) {
                    const int s = find_seg(A.ray_off, A.n + 1, idx);
                    const SceneDev& d = A.sd[s];
                    const int64_t r0 = A.ray_off[s];
                    const int64_t local = sched_ray(A.sched, idx - r0);
                    ray = r0 + local;
                    bounce = 0;
                    prev = -1;
                    prev_plane = -1;
                    key = 0;
                    nodes = d.nodes;
                    bvh_tris = d.bvh_tris;
                    tri_plane = d.tri_bary;
                    eps = (float)d.eps;
                    table = A.tables + (uint64_t)s * A.cap;
                    uniq = A.uniq + s;
                    float3 dir = launch_dir(local, __ldg(A.sched.z + local));
                    r.o = mk(d.txf.x, d.txf.y, d.txf.z);
                    r.d = mk(dir.x, dir.y, dir.z);
                    wray_init(r);
                    Do = 5.9604645e-8f * (fabsf(d.txf.x) + fabsf(d.txf.y) + fabsf(d.txf.z));
                    Dd = 0.0f;
                } else {
                    done = true;
                }
            }
        }
        if (__all_sync(FULL, done)) break;
        if (ray < 0) continue;
        float th;
        bool und = false;
        unsigned nv = 0, nt = 0;
        int plane = -1;
        int id = closest32<STACK>(nodes, bvh_tris, r, eps, prev, stack, th, und, A.status, nv, nt,
                                  bounce == 0 ? 0.0f : Do, Dd, prev_plane, plane);
        c_vis += nv;
        c_tri += nt;
        c_q++;
        if (und) {
            unsigned long long slot = atomicAdd(A.redo_count, 1ull);
            if ((int64_t)slot < A.redo_cap) {
                A.redo[slot] = ray | ((int64_t)bounce << 32);
                A.redo_key[slot] = key;
            } else {
                atomicExch(A.overflow, 2);
            }
            ray = -1;
            continue;
        }
        if (id < 0) {
            ray = -1;
            continue;
        }
        key = rt_key_push(key, bounce, id);
        hash_insert(table, A.cap - 1, key, uniq, A.uniq_limit, A.overflow);
        bounce++;
        if (bounce >= A.depth) {
            ray = -1;
            continue;
        }
        if (!sbr_bounce(r, __ldg(tri_plane + 3 * id), Do, Dd)) {
            unsigned long long slot = atomicAdd(A.redo_count, 1ull);
            if ((int64_t)slot < A.redo_cap) {
                A.redo[slot] = ray | ((int64_t)bounce << 32);
                A.redo_key[slot] = key;
            } else {
                atomicExch(A.overflow, 2);
            }
            ray = -1;
            continue;
        }
        prev = id;
        prev_plane = plane;
    }
    if (A.counters) {
        warp_count(A.counters + 0, c_vis);
        warp_count(A.counters + 1, c_tri);
        warp_count(A.counters + 2, c_q);
    }
}

__global__ void __launch_bounds__(REDO_THREADS) k_sbr_redo_batch(BatchSbr A) {
    extern __shared__ int smem_stack[];
    int* stack = smem_stack + threadIdx.x;
    int* cand = smem_stack + RT_STACK * blockDim.x + threadIdx.x;
    float* cand_t = reinterpret_cast<float*>(smem_stack + (RT_STACK + CAND_CAP) * blockDim.x) + threadIdx.x;
    float* cand_e = reinterpret_cast<float*>(smem_stack + (RT_STACK + 2 * CAND_CAP) * blockDim.x) + threadIdx.x;
    unsigned long long n = *A.redo_count;
    if (n > (unsigned long long)A.redo_cap) n = A.redo_cap;
    if (A.counters && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(A.counters + 3, n);
    // few redo rays: spread them over all warps, rpw lanes per warp, so that more
    // warps hide the traversal latency and a warp carries fewer divergent rays
    const unsigned long long W = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long rpw = n < W ? 1ull : (n + W - 1) / W < 32ull ? (n + W - 1) / W : 32ull;
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (lane >= rpw) return;
    for (unsigned long long w = warp * rpw + lane; w < n; w += W * rpw) {
        const int64_t e = A.redo[w];
        const int64_t ray = e & 0xffffffffll;
        int b0 = (int)(e >> 32);
        uint64_t key = A.redo_key[w];
        int s = find_seg(A.ray_off, A.n + 1, ray);
        const SceneDev& d = A.sd[s];
        float3 df = launch_dir(ray - A.ray_off[s], __ldg(A.sched.z + (ray - A.ray_off[s])));
        WRay<double> r;
        WRay<float> rf;
        r.o = mk(d.tx, d.ty, d.tz);
        r.d = mk((double)df.x, (double)df.y, (double)df.z);
        int prev = -1;
        for (int b = 0; b < A.depth; ++b) {
            double th;
            int id = -1;
            if (b < b0) {   // robust prefix (as k_sbr_redo)
                id = rt_key_tri(key, b);
                if (!replay_plane(d.tri_n64, id, r, d.eps, th)) {
                    b0 = b;
                    key = key_prefix(key, b);
                }
            }
            if (b >= b0) {
                rf.o = mk((float)r.o.x, (float)r.o.y, (float)r.o.z);
                rf.d = mk((float)r.d.x, (float)r.d.y, (float)r.d.z);
                wray_init(rf);
                id = closest64(d.nodes, d.bvh_tris, r, rf, d.tri_n64, d.eps, prev, stack, cand, cand_t, cand_e, th,
                               A.status);
                if (id < 0) break;
                key = rt_key_push(key_prefix(key, b), b, id);
                hash_insert(A.tables + (uint64_t)s * A.cap, A.cap - 1, key, A.uniq + s, A.uniq_limit, A.overflow);
            }
            V3<double> nn = mk(d.tri_n64[4 * id], d.tri_n64[4 * id + 1], d.tri_n64[4 * id + 2]);
            V3<double> p = r.o + th * r.d;
            r.d = r.d - (2.0 * dot(r.d, nn)) * nn;
            r.o = p;
            prev = id;
        }
    }
}

// Unique keys of every scene's table into that scene's sort buffer (cap is a
// power of two >= 2^16, so a warp never spans two tables).
__global__ void k_table_compact_batch(const unsigned long long* __restrict__ tables, int n, uint64_t cap,
                                      uint64_t* out, uint64_t out_stride, unsigned long long* counts) {
    const int lane = threadIdx.x & 31;
    const uint64_t total = cap * (uint64_t)n;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i - lane < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long k = i < total ? tables[i] : 0ull;
        int s = (int)((i - lane) / cap);
        unsigned m = __ballot_sync(FULL, k != 0ull);
        if (!m) continue;
        unsigned long long base = 0;
        int leader = __ffs(m) - 1;
        if (lane == leader) base = atomicAdd(counts + s, (unsigned long long)__popc(m));
        base = __shfl_sync(FULL, base, leader);
        const unsigned long long slot = base + __popc(m & ((1u << lane) - 1));
        if (k && slot < out_stride) out[s * out_stride + slot] = k;   // beyond: counted, read as an overflow
    }
}

// The candidate list of every scene: LoS, then its sorted keys (at most the
// scene's slots minus one; the count comes from the compaction); K of each scene
// is stored in K_dev.
__global__ void k_cand_keys_batch(const uint64_t* __restrict__ sorted, uint64_t sort_stride,
                                  const unsigned long long* __restrict__ counts, const int64_t* __restrict__ cand_off,
                                  int n, uint64_t* __restrict__ cand, int64_t* __restrict__ K_dev) {
    const int64_t KT = cand_off[n];
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < KT; k += (int64_t)gridDim.x * blockDim.x) {
        const int s = find_seg(cand_off, n + 1, k);
        const int64_t local = k - cand_off[s];
        const int64_t ns = (int64_t)min(counts[s], (unsigned long long)(cand_off[s + 1] - cand_off[s] - 1));
        if (local == 0) {
            cand[k] = 0ull;
            K_dev[s] = ns + 1;
        } else if (local <= ns) {
            cand[k] = sorted[(uint64_t)s * sort_stride + (uint64_t)(local - 1)];
        }
    }
}

// Image sources of every candidate of every scene (global candidate index); the
// slots of a scene from its K_dev on are marked empty (depth -1).
__global__ void k_candidates_batch(const uint64_t* __restrict__ keys, int64_t K, int D, const SceneDev* sd,
                                   const int64_t* cand_off, int n, const int64_t* __restrict__ K_dev,
                                   int32_t* cand_depth, int32_t* cand_tri, double* img64, float4* img32,
                                   float4* frus) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
        const int sc = find_seg(cand_off, n + 1, k);
        if (k - cand_off[sc] >= K_dev[sc]) {
            cand_depth[k] = -1;
            continue;
        }
        const SceneDev& d = sd[sc];
        uint64_t key = keys[k];
        int q = rt_key_depth(key);
        cand_depth[k] = q;
        V3<double> I = mk(d.tx, d.ty, d.tz);
        for (int j = 0; j < D; ++j) {
            int t = j < q ? rt_key_tri(key, j) : -1;
            cand_tri[(int64_t)j * K + k] = t;
            if (t >= 0) {
                V3<double> nn = mk(d.tri_n64[4 * t], d.tri_n64[4 * t + 1], d.tri_n64[4 * t + 2]);
                V3<double> a = from4<double>(__ldg(d.tri_v + 3 * t));
                I = I - (2.0 * dot(I - a, nn)) * nn;
            }
            double* o = img64 + ((int64_t)j * K + k) * 3;
            o[0] = I.x;
            o[1] = I.y;
            o[2] = I.z;
            img32[(int64_t)j * K + k] = make_float4((float)I.x, (float)I.y, (float)I.z, 0.0f);
            if (j == q - 1) frustum_store(I, d.tri_v, d.tri_bary, t, frus, K, k);
        }
    }
}

struct BatchPairs {
    CandView C;   // global candidates
    const SceneDev* sd;
    const int64_t* tile_off;   // n + 1: prefix of warp tiles per scene
    const int64_t* cand_off;   // n + 1
    const int64_t* rx_off;     // n + 1
    int n;
    const double* rx;          // all receivers
    const int32_t* order;      // per scene, the tile order of its receivers (scene-local), or null
    PairSink S;
};

// Batched prefilter: warp tiles of every scene in one index space (the scene of
// a tile is found once per tile).
__global__ void k_pairs_batch(BatchPairs A) {
    const int lane = threadIdx.x & 31;
    const int64_t tiles = A.tile_off[A.n];
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp0; t < tiles; t += nwarps) {
        const int s = find_seg(A.tile_off, A.n + 1, t);
        const int64_t R = A.rx_off[s + 1] - A.rx_off[s];
        const int64_t K = A.cand_off[s + 1] - A.cand_off[s];
        const int64_t rt_n = (R + 31) / 32;
        const int64_t lt = t - A.tile_off[s];
        const int64_t kt = lt / rt_n, rt = lt - kt * rt_n;
        const int64_t rs = rt * 32 + lane;
        const bool r_ok = rs < R;
        const int64_t rg = A.rx_off[s] + (r_ok && A.order ? (int64_t)A.order[A.rx_off[s] + rs] : rs);
        float3 rxf = make_float3(0.0f, 0.0f, 0.0f);
        if (r_ok) rxf = make_float3((float)A.rx[3 * rg], (float)A.rx[3 * rg + 1], (float)A.rx[3 * rg + 2]);
        const int64_t k0 = A.cand_off[s] + kt * PAIR_CC, k1 = A.cand_off[s] + min(K, (kt + 1) * PAIR_CC);
        pairs_tile(A.C, k0, k1, rg, r_ok, rxf, A.sd[s].tri_bary, A.S);
    }
}

struct BatchVis {
    CandView C;
    const SceneDev* sd;
    const int64_t* cand_off;
    const int64_t* rx_off;
    const int64_t* bits_off;   // n + 1, in words
    int n;
    const double* rx;
    const uint2* queue;
    const unsigned long long* qcount;
    unsigned long long qcap;
    uint32_t* bits;
    int32_t* status;
    unsigned long long* counters;   // optional instrumentation (slots 4..6)
    int D;
    int32_t* seg_q;                 // as VisArgs
    float4* seg_o;
    float4* seg_d;
};

// k_backtrace / k_segments over the concatenated (scene, candidate, receiver)
// index spaces of a batch.
__global__ void __launch_bounds__(TRACE_THREADS) k_backtrace_batch(BatchVis A) {
    unsigned long long n = *A.qcount;
    if (n > A.qcap) n = A.qcap;
    for (unsigned long long w = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; w < n;
         w += (unsigned long long)gridDim.x * blockDim.x) {
        const uint2 e = A.queue[w];
        const int64_t kg = e.x, rg = e.y;
        const int s = find_seg(A.cand_off, A.n + 1, kg);
        const SceneDev& d = A.sd[s];
        const int q = A.C.depth[kg];
        const double* rp = A.rx + 3 * rg;
        const int st = backtrace32(A.C, kg, q, mk((float)rp[0], (float)rp[1], (float)rp[2]), d.txf, d.tri_bary, w,
                                   A.qcap, A.seg_o, A.seg_d);
        A.seg_q[w] = st == 1 ? q : st == 2 ? -2 : -1;
        if (st != 0) {
            const int64_t words = (A.cand_off[s + 1] - A.cand_off[s] + 31) / 32;
            const int64_t kl = kg - A.cand_off[s];
            atomicOr(A.bits + A.bits_off[s] + (rg - A.rx_off[s]) * words + (kl >> 5), 1u << (kl & 31));
        }
    }
}

template <int STACK>
__global__ void __launch_bounds__(TRACE_THREADS) k_segments_batch(BatchVis A) {
    extern __shared__ int smem_stack[];
    int* stack = smem_stack + threadIdx.x;
    int* cand = smem_stack + STACK * blockDim.x + threadIdx.x;
    unsigned long long n = *A.qcount;
    if (n > A.qcap) n = A.qcap;
    const unsigned long long total = n * (unsigned long long)(A.D + 1);
    unsigned long long c_vis = 0, c_tri = 0, c_seg = 0;
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < total;
         t += (unsigned long long)gridDim.x * blockDim.x) {
        // segment index and pair: 32-bit division whenever the item count fits
        const int j = total <= 0xffffffffull ? (int)((unsigned)t / (unsigned)n) : (int)(t / n);
        const unsigned long long w = t - (unsigned long long)j * n;
        const int qs = A.seg_q[w];
        if (qs == -1) continue;
        uint2 e = A.queue[w];
        const int64_t kg = e.x, rg = e.y;
        const int q = qs >= 0 ? qs : A.C.depth[kg];
        if (q < j) continue;
        const int s = find_seg(A.cand_off, A.n + 1, kg);
        const SceneDev& d = A.sd[s];
        const int64_t words = (A.cand_off[s + 1] - A.cand_off[s] + 31) / 32;
        const int64_t kl = kg - A.cand_off[s];
        uint32_t* word = A.bits + A.bits_off[s] + (rg - A.rx_off[s]) * words + (kl >> 5);
        const uint32_t bit = 1u << (kl & 31);
        if (!(*(volatile uint32_t*)word & bit)) continue;
        const int s0 = j >= 1 ? A.C.tri[(int64_t)(j - 1) * A.C.K + kg] : -1;
        const int s1 = j + 1 <= q ? A.C.tri[(int64_t)j * A.C.K + kg] : -1;
        const float epsf = (float)d.eps;
        WRay<float> rf;
        bool hit = false, und = true;
        if (qs >= 0) {
            const float4 o4 = A.seg_o[(size_t)j * A.qcap + w], d4 = A.seg_d[(size_t)j * A.qcap + w];
            rf.o = mk(o4.x, o4.y, o4.z);
            rf.d = mk(d4.x, d4.y, d4.z);
            wray_init(rf);
            und = false;
            unsigned nv = 0, nt = 0;
            const int pl0 = s0 >= 0 ? __float_as_int(__ldg(d.tri_v + 3 * s0 + 1).w) : -1;
            const int pl1 = s1 >= 0 ? __float_as_int(__ldg(d.tri_v + 3 * s1 + 1).w) : -1;
            hit = any32<STACK>(d.nodes, d.bvh_tris, rf, epsf * o4.w, 1.0f - epsf * o4.w, s0, s1, pl0, pl1, stack, und,
                        A.status, nv, nt);
            c_vis += nv;
            c_tri += nt;
            c_seg++;
        }
        if (!hit && und) {
            const double* rp = A.rx + 3 * rg;
            V3<double> pts[RT_MAX_DEPTH + 2];
            if (!backtrace64(A.C, kg, q, mk(d.tx, d.ty, d.tz), mk(rp[0], rp[1], rp[2]), d.tri_v, d.tri_n64, d.bary64,
                             d.eps, pts, nullptr)) {
                atomicAnd(word, ~bit);
                continue;
            }
            V3<double> dv = pts[j + 1] - pts[j];
            double il = rsqrt(dot(dv, dv));
            WRay<double> rd;
            rd.o = pts[j];
            rd.d = dv;
            wray_init(rd);
            if (qs < 0) {
                rf.o = mk((float)pts[j].x, (float)pts[j].y, (float)pts[j].z);
                rf.d = mk((float)dv.x, (float)dv.y, (float)dv.z);
                wray_init(rf);
            }
            hit = any64<STACK>(d.nodes, d.bvh_tris, rd, rf, d.eps * il, 1.0 - d.eps * il, s0, s1, stack, cand, A.status);
        }
        if (hit) atomicAnd(word, ~bit);
    }
    if (A.counters) {
        warp_count(A.counters + 4, c_vis);
        warp_count(A.counters + 5, c_tri);
        warp_count(A.counters + 6, c_seg);
    }
}


// Per-receiver popcount over all scenes (one warp per receiver).
__global__ void k_row_count_batch(const uint32_t* __restrict__ bits, const int64_t* rx_off, const int64_t* cand_off,
                                  const int64_t* bits_off, int n, int64_t* counts) {
    const int lane = threadIdx.x & 31;
    const int64_t R = rx_off[n];
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < R;
         g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int s = find_seg(rx_off, n + 1, g);
        const int64_t words = (cand_off[s + 1] - cand_off[s] + 31) / 32;
        const uint32_t* row = bits + bits_off[s] + (g - rx_off[s]) * words;
        int64_t c = 0;
        for (int64_t w = lane; w < words; w += 32) c += __popc(row[w]);
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(FULL, c, o);
        if (lane == 0) counts[g] = c;
    }
}

__global__ void k_expand_batch(const uint32_t* __restrict__ bits, const int64_t* rx_off, const int64_t* cand_off,
                               const int64_t* bits_off, int n, const int64_t* __restrict__ offsets, int32_t* path_rx,
                               int32_t* path_cand, int64_t cap) {
    const int lane = threadIdx.x & 31;
    const int64_t R = rx_off[n];
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < R;
         g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int s = find_seg(rx_off, n + 1, g);
        const int64_t words = (cand_off[s + 1] - cand_off[s] + 31) / 32;
        const uint32_t* row = bits + bits_off[s] + (g - rx_off[s]) * words;
        int64_t pos = offsets[g];
        for (int64_t w0 = 0; w0 < words; w0 += 32) {
            int64_t w = w0 + lane;
            uint32_t b = w < words ? row[w] : 0u;
            int c = __popc(b);
            int incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                int v = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += v;
            }
            int64_t my = pos + incl - c;
            while (b) {
                int bit = __ffs(b) - 1;
                b &= b - 1;
                if (my < cap) {
                    path_rx[my] = (int32_t)g;
                    path_cand[my] = (int32_t)(cand_off[s] + w * 32 + bit);
                }
                my++;
            }
            pos += __shfl_sync(FULL, incl, 31);
        }
    }
}

// FP64 points of every path; triangle slots carry global (offset) ids.
__global__ void k_points_batch(CandView C, const int64_t* __restrict__ P_dev, int64_t cap, int D, const SceneDev* sd,
                               const int64_t* cand_off, int n, const int32_t* __restrict__ path_rx,
                               int32_t* __restrict__ path_cand, const double* __restrict__ rx, double* pts_out,
                               int32_t* depth_out, int32_t* rx_out, int32_t* tri_out, int32_t* edge_flag,
                               uint32_t* bits, const int64_t* rx_off, const int64_t* bits_off) {
    const int64_t P = min(*P_dev, cap);   // also the slot stride of tri_out
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t kg = path_cand[i];
        int r = path_rx[i];
        const int s = find_seg(cand_off, n + 1, kg);
        const SceneDev& d = sd[s];
        int q = C.depth[kg];
        const double* rp = rx + 3 * (int64_t)r;
        V3<double> pts[RT_MAX_DEPTH + 2];
        double mb = 1.0;
        if (!backtrace64(C, kg, q, mk(d.tx, d.ty, d.tz), mk(rp[0], rp[1], rp[2]), d.tri_v, d.tri_n64, d.bary64, d.eps,
                         pts, &mb)) {
            // invalid in FP64: dropped like a duplicate (as k_points)
            path_cand[i] = -1;
            const int64_t words = (cand_off[s + 1] - cand_off[s] + 31) / 32;
            const int64_t kl = kg - cand_off[s];
            atomicAnd(bits + bits_off[s] + (r - rx_off[s]) * words + (kl >> 5), ~(1u << (kl & 31)));
            mb = 1.0;
            q = 0;
            pts[0] = pts[1] = mk(0.0, 0.0, 0.0);
        }
        for (int j = 0; j < D + 2; ++j) {
            V3<double> v = j <= q + 1 ? pts[j] : mk(0.0, 0.0, 0.0);
            double* o = pts_out + ((int64_t)i * (D + 2) + j) * 3;
            o[0] = v.x;
            o[1] = v.y;
            o[2] = v.z;
        }
        depth_out[i] = q;
        rx_out[i] = r;
        for (int j = 0; j < D; ++j)
            tri_out[(int64_t)j * P + i] = j < q ? C.tri[(int64_t)j * C.K + kg] + d.tri_off : -1;
        edge_flag[i] = (q > 0 && mb <= 1e-8) ? 1 : 0;
    }
}

// Duplicate rule over all scenes (global path, receiver, triangle and
// candidate indices; bits cleared in the scene's own bitmask layout).
__global__ void k_dedup_batch(const int64_t* __restrict__ P_dev, int64_t cap, int D,
                              const int64_t* __restrict__ path_off, const int32_t* __restrict__ path_rx,
                              int32_t* __restrict__ path_cand, const int32_t* __restrict__ depth,
                              const int32_t* __restrict__ tri, const double* __restrict__ pts,
                              const int32_t* __restrict__ edge_flag, const double* __restrict__ tri_n64,
                              const float4* __restrict__ tri_v, double diag, const int64_t* rx_off,
                              const int64_t* cand_off, const int64_t* bits_off, int n, uint32_t* bits,
                              unsigned long long* drops) {
    const int64_t P = min(*P_dev, cap);
    const double tol2 = (1e-9 * diag) * (1e-9 * diag);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        if (!edge_flag[i]) continue;
        int r = path_rx[i];
        int q = depth[i];
        for (int64_t j = path_off[r]; j < path_off[r + 1] && j < P; ++j) {
            if (j == i || !edge_flag[j] || depth[j] != q) continue;
            bool same = true;
            for (int b = 0; b < q && same; ++b)
                same = coplanar64(tri_n64, tri_v, tri[(int64_t)b * P + i], tri[(int64_t)b * P + j], diag);
            for (int b = 1; b <= q && same; ++b) {
                const double* pi = pts + ((int64_t)i * (D + 2) + b) * 3;
                const double* pj = pts + ((int64_t)j * (D + 2) + b) * 3;
                double dx = pi[0] - pj[0], dy = pi[1] - pj[1], dz = pi[2] - pj[2];
                same = dx * dx + dy * dy + dz * dz <= tol2;
            }
            if (!same) continue;
            bool less = false;
            for (int b = 0; b < q; ++b) {
                int ti = tri[(int64_t)b * P + i], tj = tri[(int64_t)b * P + j];
                if (ti != tj) {
                    less = tj < ti;
                    break;
                }
            }
            if (less) {
                int s = find_seg(rx_off, n + 1, (int64_t)r);
                const int64_t words = (cand_off[s + 1] - cand_off[s] + 31) / 32;
                const int64_t kl = path_cand[i] - cand_off[s];
                atomicAnd(bits + bits_off[s] + (r - rx_off[s]) * words + (kl >> 5), ~(1u << (kl & 31)));
                atomicAdd(drops, 1ull);
                path_cand[i] = -1;   // dropped (only this thread reads path_cand[i])
                break;
            }
        }
    }
}

// The counts and capacity flags of a batched pass (as k_trace_check): the scenes'
// unique keys against their slots, the emitted paths against the path slots.
__global__ void k_batch_check(const int32_t* __restrict__ f1, const int32_t* __restrict__ f2,
                              const unsigned long long* __restrict__ counts, const int64_t* __restrict__ cand_off, int n,
                              const int64_t* __restrict__ P_emit, const int64_t* __restrict__ P_kept, int64_t pcap,
                              int64_t* meta, int32_t* status, int report) {
    if (threadIdx.x != 0) return;
    bool ovf = f1[0] != 0 || f2[0] != 0 || *P_emit > pcap;
    int64_t K = 0;
    for (int s = 0; s < n; ++s) {
        const int64_t slots = cand_off[s + 1] - cand_off[s] - 1;
        if ((int64_t)counts[s] > slots) ovf = true;
        K += min((int64_t)counts[s], slots) + 1;
    }
    meta[0] = ovf ? 0 : min(*P_kept, pcap);
    meta[1] = K;
    meta[2] = f1[0] == 2 ? 2 : (ovf ? 1 : 0);
    if (ovf && report) rt_set_status(status, RT_ERR_CAPACITY);
}

}  // namespace

// Per-call metadata of a batch (scene descriptors, prefix arrays) written by
// kernels that carry it in their parameters, so that a captured batch keeps its
// own copy (no host buffer has to outlive the graph).
constexpr int META_SCENES = 16;
struct SceneChunk {
    int first, count;
    SceneDev sd[META_SCENES];
};
__global__ void k_put_scenes(SceneChunk c, SceneDev* out) {
    if ((int)threadIdx.x < c.count) out[c.first + threadIdx.x] = c.sd[threadIdx.x];
}
constexpr int META_I64 = 256;
struct I64Chunk {
    int first, count;
    int64_t v[META_I64];
};
__global__ void k_put_i64(I64Chunk c, int64_t* out) {
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) out[c.first + i] = c.v[i];
}

static rt_status put_scenes(rt_ctx* ctx, const std::vector<SceneDev>& h, SceneDev* d) {
    for (size_t f = 0; f < h.size(); f += META_SCENES) {
        SceneChunk c;
        c.first = (int)f;
        c.count = (int)std::min<size_t>(META_SCENES, h.size() - f);
        for (int i = 0; i < c.count; ++i) c.sd[i] = h[f + i];
        k_put_scenes<<<1, META_SCENES, 0, ctx->stream>>>(c, d);
        RT_COUNT(ctx);
    }
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

static rt_status put_i64(rt_ctx* ctx, const std::vector<int64_t>& h, int64_t* d) {
    for (size_t f = 0; f < h.size(); f += META_I64) {
        I64Chunk c;
        c.first = (int)f;
        c.count = (int)std::min<size_t>(META_I64, h.size() - f);
        for (int i = 0; i < c.count; ++i) c.v[i] = h[f + i];
        k_put_i64<<<1, 128, 0, ctx->stream>>>(c, d);
        RT_COUNT(ctx);
    }
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

// Combined triangle tables of a batch (triangle ids offset per scene), cached in
// the context for its last list of scenes (by serial number) and shared by
// reference with the paths objects that use them.
static rt_status batch_tables(rt_ctx* ctx, const rt_scene* const* scenes, int n, const std::vector<int64_t>& tri_off,
                              rt_scene** out) {
    std::vector<uint64_t> key(n);
    for (int s = 0; s < n; ++s) key[s] = scenes[s]->serial;
    if (ctx->batch_comb && ctx->batch_key == key) {
        *out = ctx->batch_comb;
        return RT_OK;
    }
    cudaStream_t st = ctx->stream;
    const int n_mat = scenes[0]->n_materials;
    rt_scene* comb = new rt_scene();
    comb->ctx = ctx;
    comb->owns_tables_only = true;
    comb->n_tris = (int)tri_off[n];
    comb->n_materials = n_mat;
    comb->diag = 0.0;
    for (int s = 0; s < n; ++s) comb->diag = std::max(comb->diag, scenes[s]->diag);
    comb->eps = 1e-6 * comb->diag;
    comb->refs = 1;   // the context cache
    cudaError_t e = cudaMalloc((void**)&comb->d_tri_n64, (size_t)tri_off[n] * 32);
    if (e == cudaSuccess) e = cudaMalloc((void**)&comb->d_tri_v, (size_t)tri_off[n] * 48);
    if (e == cudaSuccess) e = cudaMalloc((void**)&comb->d_tri_material, (size_t)tri_off[n] * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&comb->d_is_pec, (size_t)std::max(n_mat, 1));
    for (int s = 0; s < n && e == cudaSuccess; ++s) {
        const rt_scene* sc = scenes[s];
        e = cudaMemcpyAsync(comb->d_tri_n64 + 4 * tri_off[s], sc->d_tri_n64, (size_t)sc->n_tris * 32,
                            cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(comb->d_tri_v + 3 * tri_off[s], sc->d_tri_v, (size_t)sc->n_tris * 48,
                                cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(comb->d_tri_material + tri_off[s], sc->d_tri_material, (size_t)sc->n_tris * 4,
                                cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(comb->d_is_pec, scenes[0]->d_is_pec, n_mat, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        rt_scene_free(comb);
        return rt_cuda_fail(ctx, e, "batch triangle tables");
    }
    comb->h_is_pec = new uint8_t[std::max(n_mat, 1)];
    std::memcpy(comb->h_is_pec, scenes[0]->h_is_pec, n_mat);
    if (ctx->batch_comb && --ctx->batch_comb->refs == 0) {
        cudaStreamSynchronize(st);
        rt_scene_free(ctx->batch_comb);
    }
    ctx->batch_comb = comb;
    ctx->batch_key = key;
    *out = comb;
    return RT_OK;
}

// Batched trace with the structure of rt_trace_paths: capacities per scene (its
// last unique keys) and for the batch's paths (the last batch's count), counts
// read on the device, one read-back at the end (or none with rt_set_trace_async).
extern "C" __attribute__((visibility("default"))) rt_status rt_trace_batch(
    rt_ctx* ctx, const rt_scene* const* scenes, int32_t n_scenes, const double* tx_host, const double* rx_dev,
    const int32_t* rx_counts_host, int64_t n_rays, int32_t max_depth, rt_paths** out) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!scenes || !tx_host || !rx_dev || !rx_counts_host || !out) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    if (n_scenes < 1 || n_scenes > 256) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_scenes must be in [1, 256]");
    if (n_rays < 1 || n_rays > 0x7fffffffLL) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_rays out of range");
    if (max_depth < 1 || max_depth > RT_MAX_DEPTH) return rt_fail(ctx, RT_ERR_INVALID_ARG, "max_depth must be 1..4");
    const int n = n_scenes, D = max_depth;
    const int n_mat = scenes[0] ? scenes[0]->n_materials : 0;
    std::vector<int64_t> rx_off(n + 1, 0), ray_off(n + 1, 0), tri_off(n + 1, 0);
    for (int s = 0; s < n; ++s) {
        const rt_scene* sc = scenes[s];
        if (!sc || sc->owns_tables_only) return rt_fail(ctx, RT_ERR_INVALID_ARG, "scene %d is not a traceable scene", s);
        if (sc->n_materials != n_mat || std::memcmp(sc->h_is_pec, scenes[0]->h_is_pec, n_mat) != 0)
            return rt_fail(ctx, RT_ERR_INVALID_ARG, "scenes of a batch must share one material table");
        if (rx_counts_host[s] < 1) return rt_fail(ctx, RT_ERR_INVALID_ARG, "scene %d has no receivers", s);
        for (int c = 0; c < 3; ++c)
            if (!std::isfinite(tx_host[3 * s + c])) return rt_fail(ctx, RT_ERR_NUMERIC, "non-finite transmitter");
        rx_off[s + 1] = rx_off[s] + rx_counts_host[s];
        ray_off[s + 1] = ray_off[s] + n_rays;
        tri_off[s + 1] = tri_off[s] + sc->n_tris;
    }
    if (rx_off[n] > (1 << 24)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "more than 2^24 receivers in a batch");
    if (tri_off[n] > 0x7fffffff) return rt_fail(ctx, RT_ERR_INVALID_ARG, "too many triangles in a batch");
    *out = nullptr;
    cudaStream_t st = ctx->stream;
    int32_t* status = rt_status_ptr(ctx);
    const size_t stack_bytes = (size_t)RT_STACK * TRACE_THREADS * sizeof(int);
    const size_t vis_bytes = (size_t)(RT_STACK + VIS_CAND_CAP) * TRACE_THREADS * sizeof(int);
    const int64_t RT = rx_off[n];
    rt_scene* comb = nullptr;
    {
        rt_status sc0 = batch_tables(ctx, scenes, n, tri_off, &comb);
        if (sc0 != RT_OK) return sc0;
    }
    std::vector<SceneDev> hsd(n);
    for (int s = 0; s < n; ++s) {
        const rt_scene* sc = scenes[s];
        hsd[s] = SceneDev{sc->d_nodes, sc->d_bvh_tris, sc->d_tri_v, sc->d_tri_bary, sc->d_tri_n64, sc->d_tri_bary64,
                          tx_host[3 * s], tx_host[3 * s + 1], tx_host[3 * s + 2], sc->eps,
                          make_float3((float)tx_host[3 * s], (float)tx_host[3 * s + 1], (float)tx_host[3 * s + 2]),
                          n_rays, (int32_t)tri_off[s]};
    }
    unsigned long long* tw = ctx->d_trace_words;
    int32_t* f1 = reinterpret_cast<int32_t*>(tw + 8);      // SBR: hash overflow (1), re-trace list (2)
    unsigned long long* c2 = tw + 16;                       // visibility queue count, .., [4] duplicates
    int32_t* f2 = reinterpret_cast<int32_t*>(tw + 24);     // queue overflow
    unsigned long long* uniq_dev = tw + 64;                 // per scene: keys inserted
    unsigned long long* keys_dev = tw + 320;                // per scene: keys compacted
    int64_t* K_dev = reinterpret_cast<int64_t*>(tw + 576);  // per scene: candidates
    const int64_t redo_cap = std::max<int64_t>(1 << 16, ray_off[n] / 16);
    const bool in_capture = stream_capturing(st);
    if (in_capture) {
        bool known = ctx->batch_paths_hint > 0;
        for (int s = 0; s < n; ++s) known &= scenes[s]->uniq_hint > 0;
        if (!known) return rt_fail(ctx, RT_ERR_INVALID_ARG, "a batch trace inside a stream capture needs an earlier trace");
    }
    const bool async = ctx->trace_async || in_capture;
    for (int attempt = 0;; ++attempt) {
        if (attempt >= 8) return rt_fail(ctx, RT_ERR_CAPACITY, "batch trace capacities did not converge");
        size_t cap = 1u << 16;
        for (int s = 0; s < n; ++s) cap = std::max(cap, scenes[s]->hash_cap);
        std::vector<int64_t> ucap(n), cand_off(n + 1, 0), pair_off(n + 1, 0), bits_off(n + 1, 0);
        int64_t sort_cap = SORT_BLOCK;
        bool first = false;
        for (int s = 0; s < n; ++s) {
            const int64_t hint = scenes[s]->uniq_hint;
            first |= hint == 0;
            ucap[s] = std::min<int64_t>(std::max<int64_t>(1024, hint + hint / 8 + 256), (int64_t)(cap / 2));
            while (sort_cap < ucap[s]) sort_cap <<= 1;
            const int64_t K = ucap[s] + 1;
            cand_off[s + 1] = cand_off[s] + K;
            pair_off[s + 1] = pair_off[s] + ((K + PAIR_CC - 1) / PAIR_CC) * ((rx_off[s + 1] - rx_off[s] + 31) / 32);
            bits_off[s + 1] = bits_off[s] + ((K + 31) / 32) * (rx_off[s + 1] - rx_off[s]);
        }
        const int64_t KT = cand_off[n];
        if (KT > 0x7fffffffLL) return rt_fail(ctx, RT_ERR_CAPACITY, "more than 2^31 candidate slots in a batch");
        size_t qcap = 1u << 20;
        for (int s = 0; s < n; ++s) qcap = std::max(qcap, scenes[s]->queue_cap);

        rt_paths* p = new rt_paths();
        p->stream = st;
        p->D = D;
        p->R = (int)RT;
        p->n_scenes = n;
        p->scene = comb;
        p->owned_scene = comb;
        comb->refs++;
        p->h_scene_rx_off = new int64_t[n + 1];
        p->h_scene_tri_off = new int64_t[n + 1];
        for (int s = 0; s <= n; ++s) {
            p->h_scene_rx_off[s] = rx_off[s];
            p->h_scene_tri_off[s] = tri_off[s];
        }
        void* meta = nullptr;
        auto fail = [&](rt_status e) {
            if (meta) cudaFreeAsync(meta, st);
            rt_paths_free(p);
            return e;
        };
#define BCK(call)                                                         \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return fail(rt_cuda_fail(ctx, _e, #call)); \
    } while (0)
        // per-scene descriptors and the prefix arrays
        BCK(cudaMallocAsync(&meta, align_up(sizeof(SceneDev) * n, 64) + sizeof(int64_t) * 5 * (n + 1) + 256, st));
        SceneDev* d_sd = reinterpret_cast<SceneDev*>(meta);
        int64_t* d_offs = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(meta) + align_up(sizeof(SceneDev) * n, 64));
        int64_t* d_ray_off = d_offs;
        int64_t* d_rx_off = d_offs + (n + 1);
        int64_t* d_cand_off = d_offs + 2 * (n + 1);
        int64_t* d_pair_off = d_offs + 3 * (n + 1);
        int64_t* d_bits_off = d_offs + 4 * (n + 1);
        {
            rt_status sm = put_scenes(ctx, hsd, d_sd);
            std::vector<int64_t> offs;
            for (const auto* v : {&ray_off, &rx_off, &cand_off, &pair_off, &bits_off}) offs.insert(offs.end(), v->begin(), v->end());
            if (sm == RT_OK) sm = put_i64(ctx, offs, d_offs);
            if (sm != RT_OK) return fail(sm);
        }

        // ---------------- SBR over all scenes, one persistent launch (+ FP64 re-trace)
        size_t need1 = (size_t)n * cap * 8 + (size_t)n * sort_cap * 8 + redo_cap * 16 + 8 * 256;
        void* base;
        rt_status s0 = rt_scratch(ctx, need1, &base);
        if (s0 != RT_OK) return fail(s0);
        Arena ar{(char*)base};
        unsigned long long* tables = ar.take<unsigned long long>((size_t)n * cap);
        int64_t* redo = ar.take<int64_t>(redo_cap);
        uint64_t* redo_key = ar.take<uint64_t>(redo_cap);
        uint64_t* sorted = ar.take<uint64_t>((size_t)n * sort_cap);
        BCK(cudaMemsetAsync(tables, 0, (size_t)n * cap * 8, st));
        BCK(cudaMemsetAsync(tw, 0, RT_TRACE_WORDS * 8, st));
        BatchSbr A;
        A.sd = d_sd;
        A.ray_off = d_ray_off;
        A.n = n;
        A.depth = D;
        A.tables = tables;
        A.cap = cap;
        A.uniq = uniq_dev;
        A.uniq_limit = cap / 2;
        A.overflow = f1;
        A.next_ray = tw + 1;
        A.redo = redo;
        A.redo_key = redo_key;
        A.redo_count = tw + 2;
        A.redo_cap = redo_cap;
        A.status = status;
        A.counters = (ctx->profile & 2) ? ctx->d_counters : nullptr;
        {
            rt_status ss = ray_schedule(ctx, n_rays, &A.sched);
            if (ss != RT_OK) return fail(ss);
        }
        mark(ctx, 0);
        mark(ctx, 6);
        int depth_max = 0;   // the deepest tree of the batch sizes the traversal stack (as rt_trace_paths)
        for (int s2 = 0; s2 < n; ++s2) depth_max = std::max(depth_max, scenes[s2]->bvh_depth);
        if (depth_max <= 32)
            k_sbr_batch<32><<<ctx->num_sms * ctx->tune_sbr_blocks_per_sm, TRACE_THREADS,
                              (size_t)32 * TRACE_THREADS * sizeof(int), st>>>(A);
        else
            k_sbr_batch<RT_STACK><<<ctx->num_sms * ctx->tune_sbr_blocks_per_sm, TRACE_THREADS, stack_bytes, st>>>(A);
        RT_COUNT(ctx);
        mark(ctx, 7);
        BCK(cudaGetLastError());
        k_sbr_redo_batch<<<ctx->num_sms * REDO_BLOCKS_PER_SM, REDO_THREADS, (size_t)(RT_STACK + 3 * CAND_CAP) * REDO_THREADS * sizeof(int), st>>>(A);
        RT_COUNT(ctx);
        BCK(cudaGetLastError());
        mark(ctx, 1);
        if (first) {
            // some scene is traced for the first time: learn its unique keys
            int64_t* hp = ctx->h_pinned;
            BCK(cudaMemcpyAsync(hp, uniq_dev, 8 * n, cudaMemcpyDeviceToHost, st));
            BCK(cudaStreamSynchronize(st));
            bool grow = false;
            for (int s = 0; s < n; ++s) {
                rt_scene* sc = const_cast<rt_scene*>(scenes[s]);
                if (sc->uniq_hint == 0) sc->uniq_hint = std::max<int64_t>(1, hp[s]);
                grow |= hp[s] > ucap[s] && ucap[s] < (int64_t)(cap / 2);
            }
            if (grow) {
                cudaFreeAsync(meta, st);
                meta = nullptr;
                rt_paths_free(p);
                continue;
            }
        }
        // ---------------- keys of each scene sorted (length, lexicographic), at most its slots
        k_fill_u64<<<grid_for(ctx, (int64_t)n * sort_cap, 256), 256, 0, st>>>(sorted, (uint64_t)n * sort_cap, ~0ull);
        RT_COUNT(ctx);
        k_table_compact_batch<<<grid_for(ctx, (int64_t)n * cap, 256, 16), 256, 0, st>>>(tables, n, cap, sorted,
                                                                                        sort_cap, keys_dev);
        RT_COUNT(ctx);
        BCK(cudaGetLastError());
        for (int s = 0; s < n; ++s) {
            int64_t n_pad = SORT_BLOCK;
            while (n_pad < ucap[s]) n_pad <<= 1;
            uint64_t* keys = sorted + (size_t)s * sort_cap;
            k_bitonic_local<<<(unsigned)(n_pad / SORT_BLOCK), 1024, 0, st>>>(keys);
            RT_COUNT(ctx);
            for (uint64_t k = 2 * SORT_BLOCK; k <= (uint64_t)n_pad; k <<= 1) {
                for (uint64_t j = k >> 1; j >= (uint64_t)SORT_BLOCK; j >>= 1) {
                    k_bitonic_global<<<grid_for(ctx, n_pad, 256, 16), 256, 0, st>>>(keys, n_pad, j, k);
                    RT_COUNT(ctx);
                }
                k_bitonic_merge_local<<<(unsigned)(n_pad / SORT_BLOCK), 1024, 0, st>>>(keys, k);
                RT_COUNT(ctx);
            }
        }
        BCK(cudaGetLastError());

        // ---------------- candidates of all scenes (LoS first in each scene)
        BCK(cudaMallocAsync((void**)&p->d_cand, KT * 8, st));
        k_cand_keys_batch<<<grid_for(ctx, KT, 256), 256, 0, st>>>(sorted, (uint64_t)sort_cap, keys_dev, d_cand_off, n,
                                                                   p->d_cand, K_dev);
        RT_COUNT(ctx);
        size_t need2 = KT * 4 + (size_t)D * KT * 4 + (size_t)D * KT * 24 + (size_t)D * KT * 16 + qcap * 8 +
                       (size_t)bits_off[n] * 4 + (size_t)(RT + 1) * 8 * 2 + qcap * 4 +
                       2 * (size_t)(D + 1) * qcap * 16 + 5 * KT * 16 + (size_t)RT * 4 + 20 * 256;
        s0 = rt_scratch(ctx, need2, &base);
        if (s0 != RT_OK) return fail(s0);
        Arena ar2{(char*)base};
        int32_t* cand_depth = ar2.take<int32_t>(KT);
        int32_t* cand_tri = ar2.take<int32_t>((size_t)D * KT);
        double* img64 = ar2.take<double>((size_t)D * KT * 3);
        float4* img32 = ar2.take<float4>((size_t)D * KT);
        uint2* queue = ar2.take<uint2>(qcap);
        uint32_t* bits = ar2.take<uint32_t>((size_t)bits_off[n]);
        int64_t* counts = ar2.take<int64_t>(RT + 1);
        int32_t* seg_q = ar2.take<int32_t>(qcap);
        float4* seg_o = ar2.take<float4>((size_t)(D + 1) * qcap);
        float4* seg_d = ar2.take<float4>((size_t)(D + 1) * qcap);
        float4* frus = ar2.take<float4>(5 * (size_t)KT);
        int32_t* rx_order = ar2.take<int32_t>((size_t)RT);
        BCK(cudaMemsetAsync(bits, 0, (size_t)bits_off[n] * 4, st));
        k_rx_order_batch<<<n, 1024, 0, st>>>(rx_dev, d_rx_off, rx_order);
        RT_COUNT(ctx);
        k_candidates_batch<<<grid_for(ctx, KT, 32, 32), 32, 0, st>>>(p->d_cand, KT, D, d_sd, d_cand_off, n, K_dev,
                                                                    cand_depth, cand_tri, img64, img32, frus);
        RT_COUNT(ctx);
        BCK(cudaGetLastError());
        BatchPairs PA{};
        PA.C = CandView{KT, cand_depth, cand_tri, img64, img32, frus};
        PA.sd = d_sd;
        PA.tile_off = d_pair_off;
        PA.cand_off = d_cand_off;
        PA.rx_off = d_rx_off;
        PA.n = n;
        PA.rx = rx_dev;
        PA.order = rx_order;
        PA.S = PairSink{queue, c2, qcap, f2};
        mark(ctx, 2);
        k_pairs_batch<<<grid_for(ctx, pair_off[n] * 32, 256, ctx->tune_pairs_blocks_per_sm), 256, 0, st>>>(PA);
        RT_COUNT(ctx);
        BCK(cudaGetLastError());
        mark(ctx, 3);
        BatchVis VA{};
        VA.C = PA.C;
        VA.sd = d_sd;
        VA.cand_off = d_cand_off;
        VA.rx_off = d_rx_off;
        VA.bits_off = d_bits_off;
        VA.n = n;
        VA.rx = rx_dev;
        VA.queue = queue;
        VA.qcount = c2;
        VA.qcap = qcap;
        VA.bits = bits;
        VA.status = status;
        VA.counters = (ctx->profile & 2) ? ctx->d_counters : nullptr;
        VA.D = D;
        VA.seg_q = seg_q;
        VA.seg_o = seg_o;
        VA.seg_d = seg_d;
        k_backtrace_batch<<<ctx->num_sms * 8, TRACE_THREADS, 0, st>>>(VA);
        RT_COUNT(ctx);
        BCK(cudaGetLastError());
        if (depth_max <= 32)
            k_segments_batch<32><<<ctx->num_sms * ctx->tune_vis_blocks_per_sm, TRACE_THREADS,
                                   (size_t)(32 + VIS_CAND_CAP) * TRACE_THREADS * sizeof(int), st>>>(VA);
        else
            k_segments_batch<RT_STACK><<<ctx->num_sms * ctx->tune_vis_blocks_per_sm, TRACE_THREADS, vis_bytes, st>>>(VA);
        RT_COUNT(ctx);
        BCK(cudaGetLastError());
        mark(ctx, 4);

        // ---------------- emission over all receivers of all scenes (pcap slots),
        // the duplicate rule, the kept paths compacted
        int64_t* off_e = nullptr;
        BCK(cudaMallocAsync((void**)&off_e, (size_t)(RT + 1) * 8, st));
        k_row_count_batch<<<grid_for(ctx, RT * 32, 256, 16), 256, 0, st>>>(bits, d_rx_off, d_cand_off, d_bits_off, n,
                                                                          counts);
        RT_COUNT(ctx);
        k_scan<<<1, 1024, 0, st>>>(counts, (int)RT, off_e);
        RT_COUNT(ctx);
        BCK(cudaGetLastError());
        if (ctx->batch_paths_hint == 0) {
            BCK(cudaMemcpyAsync(ctx->h_pinned, off_e + RT, 8, cudaMemcpyDeviceToHost, st));
            BCK(cudaStreamSynchronize(st));
            ctx->batch_paths_hint = std::max<int64_t>(1, ctx->h_pinned[0]);
        }
        const int64_t pcap = std::max<int64_t>(1024, ctx->batch_paths_hint + ctx->batch_paths_hint / 8 + 1024);
        const size_t Pa = (size_t)pcap;
        char* tmp = nullptr;
        RtCarve ct;
        const size_t t_pts = ct.take(Pa * (D + 2) * 3 * 8), t_depth = ct.take(Pa * 4), t_rx = ct.take(Pa * 4),
                     t_tri = ct.take(Pa * D * 4), t_cand = ct.take(Pa * 4), t_edge = ct.take(Pa * 4);
        BCK(cudaMallocAsync((void**)&tmp, ct.off, st));
        double* pts_e = reinterpret_cast<double*>(tmp + t_pts);
        int32_t* depth_e = reinterpret_cast<int32_t*>(tmp + t_depth);
        int32_t* rx_e = reinterpret_cast<int32_t*>(tmp + t_rx);
        int32_t* tri_e = reinterpret_cast<int32_t*>(tmp + t_tri);
        int32_t* path_cand = reinterpret_cast<int32_t*>(tmp + t_cand);
        int32_t* edge = reinterpret_cast<int32_t*>(tmp + t_edge);
        int64_t* pmeta = nullptr;
        {
            RtCarve c;
            const size_t o_pts = c.take(Pa * (D + 2) * 3 * 8), o_depth = c.take(Pa * 4), o_rx = c.take(Pa * 4),
                         o_tri = c.take(Pa * D * 4), o_meta = c.take(4 * 8);
            char* b = nullptr;
            BCK(cudaMallocAsync((void**)&b, c.off, st));
            p->d_block_geo = b;
            p->d_pts = reinterpret_cast<double*>(b + o_pts);
            p->d_depth = reinterpret_cast<int32_t*>(b + o_depth);
            p->d_rx = reinterpret_cast<int32_t*>(b + o_rx);
            p->d_tri = reinterpret_cast<int32_t*>(b + o_tri);
            pmeta = reinterpret_cast<int64_t*>(b + o_meta);
        }
        BCK(cudaMallocAsync((void**)&p->d_rx_offsets, (size_t)(RT + 1) * 8, st));
        const int64_t* P_e = off_e + RT;
        k_expand_batch<<<grid_for(ctx, RT * 32, 256, 16), 256, 0, st>>>(bits, d_rx_off, d_cand_off, d_bits_off, n,
                                                                        off_e, rx_e, path_cand, pcap);
        RT_COUNT(ctx);
        CandView C{KT, cand_depth, cand_tri, img64, img32};
        k_points_batch<<<grid_for(ctx, pcap, 32, 32), 32, 0, st>>>(C, P_e, pcap, D, d_sd, d_cand_off, n, rx_e, path_cand,
                                                                 rx_dev, pts_e, depth_e, rx_e, tri_e, edge, bits,
                                                                 d_rx_off, d_bits_off);
        RT_COUNT(ctx);
        k_dedup_batch<<<grid_for(ctx, pcap, 256), 256, 0, st>>>(P_e, pcap, D, off_e, rx_e, path_cand, depth_e, tri_e,
                                                                pts_e, edge, comb->d_tri_n64, comb->d_tri_v, comb->diag,
                                                                d_rx_off, d_cand_off, d_bits_off, n, bits, c2 + 4);
        RT_COUNT(ctx);
        k_row_count_batch<<<grid_for(ctx, RT * 32, 256, 16), 256, 0, st>>>(bits, d_rx_off, d_cand_off, d_bits_off, n,
                                                                          counts);
        RT_COUNT(ctx);
        k_scan<<<1, 1024, 0, st>>>(counts, (int)RT, p->d_rx_offsets);
        RT_COUNT(ctx);
        k_compact_paths<<<grid_for(ctx, RT * 32, 256, 16), 256, 0, st>>>((int)RT, D, pcap, off_e, p->d_rx_offsets,
                                                                         path_cand, pts_e, depth_e, rx_e, tri_e,
                                                                         p->d_pts, p->d_depth, p->d_rx, p->d_tri);
        RT_COUNT(ctx);
        k_batch_check<<<1, 32, 0, st>>>(f1, f2, keys_dev, d_cand_off, n, P_e, p->d_rx_offsets + RT, pcap, pmeta, status,
                                        async);
        RT_COUNT(ctx);
        k_trace_guard<<<grid_for(ctx, RT + 1, 256), 256, 0, st>>>(pmeta, p->d_rx_offsets, (int)RT);
        RT_COUNT(ctx);
        BCK(cudaGetLastError());
        p->P = pcap;
        rt_status s1 = rt_launch_paths_records(ctx, p, pmeta);
        if (s1 != RT_OK) return fail(s1);
        cudaFreeAsync(tmp, st);
        cudaFreeAsync(meta, st);
        meta = nullptr;
        if (async) {
            cudaFreeAsync(off_e, st);
            p->K = KT;
            p->d_count = pmeta;
            if ((ctx->profile & 1) && !in_capture) {
                BCK(cudaEventRecord(ctx->ev[5], st));
                ctx->stage_pending = 1;
            }
            *out = p;
            return RT_OK;
        }
        // ---------------- the one read-back
        int64_t* hp = ctx->h_pinned;
        BCK(cudaMemcpyAsync(hp, pmeta, 3 * 8, cudaMemcpyDeviceToHost, st));
        BCK(cudaMemcpyAsync(hp + 4, off_e + RT, 8, cudaMemcpyDeviceToHost, st));
        BCK(cudaMemcpyAsync(hp + 8, tw + 8, 8, cudaMemcpyDeviceToHost, st));
        BCK(cudaMemcpyAsync(hp + 9, tw + 24, 8, cudaMemcpyDeviceToHost, st));
        BCK(cudaMemcpyAsync(hp + 16, keys_dev, 8 * n, cudaMemcpyDeviceToHost, st));
        cudaFreeAsync(off_e, st);
        BCK(cudaStreamSynchronize(st));
        const int32_t ovf1 = reinterpret_cast<const int32_t*>(hp + 8)[0];
        const int32_t ovf2 = reinterpret_cast<const int32_t*>(hp + 9)[0];
        const int64_t P_emit = hp[4];
        if (ovf1 == 2) return fail(rt_fail(ctx, RT_ERR_CAPACITY, "FP64 re-trace list overflow"));
        bool again = false;
        if (ovf1) {
            if (cap >= ((size_t)1 << 30)) return fail(rt_fail(ctx, RT_ERR_CAPACITY, "hash overflow"));
            for (int s = 0; s < n; ++s) const_cast<rt_scene*>(scenes[s])->hash_cap = cap * 4;
            again = true;
        }
        for (int s = 0; s < n; ++s) {
            rt_scene* sc = const_cast<rt_scene*>(scenes[s]);
            if (hp[16 + s] > ucap[s]) again = true;
            sc->uniq_hint = std::max<int64_t>(1, hp[16 + s]);
        }
        if (ovf2) {
            for (int s = 0; s < n; ++s) const_cast<rt_scene*>(scenes[s])->queue_cap = qcap * 4;
            again = true;
        }
        if (P_emit > pcap) again = true;
        ctx->batch_paths_hint = std::max<int64_t>(1, P_emit);
        if (again) {
            rt_paths_free(p);
            continue;
        }
        int64_t Ktot = 0;
        for (int s = 0; s < n; ++s) {
            Ktot += hp[16 + s] + 1;
            ctx->h_counters[7] += (hp[16 + s] + 1) * (rx_off[s + 1] - rx_off[s]);
        }
        p->K = Ktot;
        p->P = hp[0];
        if (ctx->profile & 1) {
            BCK(cudaEventRecord(ctx->ev[5], st));
            ctx->stage_pending = 1;
        }
#undef BCK
        *out = p;
        return RT_OK;
    }
}

// ===========================================================================
// Autotuner of the tracing launch shapes: coordinate descent over the blocks
// per SM of the SBR, image-method and visibility kernels, each timed by its own
// stage (CUDA events) on the caller's workload; results are cached per
// (device, triangles, scene size, rays, depth, receivers).
#include <map>
#include <mutex>
#include <string>

static std::map<std::string, std::array<int, 3>>& tune_cache() {
    static std::map<std::string, std::array<int, 3>> m;
    return m;
}
static std::mutex g_tune_mu;

extern "C" __attribute__((visibility("default"))) rt_status rt_set_tuning(rt_ctx* ctx, int32_t sbr_blocks_per_sm,
                                                                          int32_t pairs_blocks_per_sm,
                                                                          int32_t vis_blocks_per_sm) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (sbr_blocks_per_sm < 1 || sbr_blocks_per_sm > 64 || pairs_blocks_per_sm < 1 || pairs_blocks_per_sm > 64 ||
        vis_blocks_per_sm < 1 || vis_blocks_per_sm > 64)
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "blocks per SM must be in [1, 64]");
    ctx->tune_sbr_blocks_per_sm = sbr_blocks_per_sm;
    ctx->tune_pairs_blocks_per_sm = pairs_blocks_per_sm;
    ctx->tune_vis_blocks_per_sm = vis_blocks_per_sm;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_autotune_trace(
    rt_ctx* ctx, const rt_scene* scene, const double* tx_host, const double* rx_dev, int32_t n_rx, int64_t n_rays,
    int32_t max_depth, int32_t* chosen, double* best_ms) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!scene || !tx_host || !rx_dev || !chosen) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    cudaDeviceProp prop;
    RT_CK(ctx, cudaGetDeviceProperties(&prop, ctx->device));
    char key[512];
    snprintf(key, sizeof(key), "%s|%d|%.6e|%lld|%d|%d", prop.name, scene->n_tris, scene->diag, (long long)n_rays,
             max_depth, n_rx);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = tune_cache().find(key);
        if (it != tune_cache().end()) {
            for (int k = 0; k < 3; ++k) chosen[k] = it->second[k];
            if (best_ms) *best_ms = 0.0;
            return rt_set_tuning(ctx, chosen[0], chosen[1], chosen[2]);
        }
    }
    const int32_t saved_profile = ctx->profile;
    rt_status st = rt_set_profiling(ctx, 1);
    if (st != RT_OK) return st;
    // one trial: two traces, the better stage time counts
    auto trial = [&](int stage, double* ms_out) -> rt_status {
        double best = 1e30;
        for (int rep = 0; rep < 2; ++rep) {
            rt_paths* p = nullptr;
            rt_status s = rt_trace_paths(ctx, scene, tx_host, rx_dev, n_rx, n_rays, max_depth, &p);
            if (s != RT_OK) return s;
            rt_paths_free(p);
            s = rt_collect_stage_times(ctx);
            if (s != RT_OK) return s;
            best = std::min(best, ctx->stage_ms[stage]);
        }
        *ms_out = best;
        return RT_OK;
    };
    const int cand[3][5] = {{4, 6, 8, 12, 16}, {8, 16, 32, 64, 0}, {4, 8, 12, 16, 0}};
    const int stage_of[3] = {0, 2, 3};   // SBR, image method, visibility
    int cur[3] = {ctx->tune_sbr_blocks_per_sm, ctx->tune_pairs_blocks_per_sm, ctx->tune_vis_blocks_per_sm};
    double total = 0.0;
    for (int knob = 0; knob < 3; ++knob) {
        double best = 1e30;
        int best_v = cur[knob];
        for (int c = 0; c < 5 && cand[knob][c] > 0; ++c) {
            cur[knob] = cand[knob][c];
            st = rt_set_tuning(ctx, cur[0], cur[1], cur[2]);
            if (st != RT_OK) return st;
            double ms;
            st = trial(stage_of[knob], &ms);
            if (st != RT_OK) return st;
            if (ms < best) {
                best = ms;
                best_v = cur[knob];
            }
        }
        cur[knob] = best_v;
        total += best;
    }
    st = rt_set_tuning(ctx, cur[0], cur[1], cur[2]);
    rt_set_profiling(ctx, saved_profile);
    if (st != RT_OK) return st;
    for (int k = 0; k < 3; ++k) chosen[k] = cur[k];
    if (best_ms) *best_ms = total;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_cache()[key] = {cur[0], cur[1], cur[2]};
    return RT_OK;
}
