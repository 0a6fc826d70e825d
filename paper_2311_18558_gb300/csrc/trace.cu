// Specular path tracing on GB300 (Sec. II-F of arXiv 2311.18558):
//   1. SBR: Fibonacci rays bounce specularly over a software BVH (FP32, with an
//      FP64 re-trace of every ray whose FP32 decisions were marginal);
//   2. dedup: every triangle-sequence prefix goes into an open-addressing hash
//      set, then the unique keys are sorted by (length, lexicographic);
//   3. image method over (candidate, receiver) pairs: FP32 prefilter with a
//      conservative margin, FP64 confirmation of the survivors;
//   4. visibility of every segment of the surviving chains (FP32 any-hit,
//      FP64 recheck when marginal), recorded in a (receiver x candidate) bitmask;
//   5. deterministic emission: per-receiver popcounts, scan, expansion in
//      candidate order, FP64 points, coplanar-duplicate rule.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rt_internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TRACE_THREADS = 128;
constexpr float SBR_MARGIN = 1e-3f;     // relative barycentric margin of the FP32 passes
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

// ------------------------------------------------------------------ watertight ray
template <typename T>
struct WRay {
    V3<T> o, d;
    int kx, ky, kz;
    T Sx, Sy, Sz;
    float3 of, inv;   // FP32 origin and reciprocal direction for the slab tests
};

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
    r.Sx = comp(r.d, kx) / dz;
    r.Sy = comp(r.d, ky) / dz;
    r.Sz = (T)1 / dz;
    r.of = make_float3((float)r.o.x, (float)r.o.y, (float)r.o.z);
    float dx = (float)r.d.x, dy = (float)r.d.y, dzz = (float)r.d.z;
    r.inv = make_float3(1.0f / (fabsf(dx) < 1e-30f ? copysignf(1e-30f, dx) : dx),
                        1.0f / (fabsf(dy) < 1e-30f ? copysignf(1e-30f, dy) : dy),
                        1.0f / (fabsf(dzz) < 1e-30f ? copysignf(1e-30f, dzz) : dzz));
}

// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013) with a margin:
// returns 0 = miss, 1 = hit, 2 = undecided (some edge function lies within
// `margin` of zero relative to their total magnitude).  With margin 0 this is the
// final decision: the triangle grown by TRI_TOL, rays in its plane miss.
template <typename T>
__device__ __forceinline__ int tri_test(const WRay<T>& r, float4 p0, float4 p1, float4 p2, T margin, T& t_out) {
    V3<T> A = from4<T>(p0) - r.o, B = from4<T>(p1) - r.o, C = from4<T>(p2) - r.o;
    T Akz = comp(A, r.kz), Bkz = comp(B, r.kz), Ckz = comp(C, r.kz);
    T Ax = comp(A, r.kx) - r.Sx * Akz, Ay = comp(A, r.ky) - r.Sy * Akz;
    T Bx = comp(B, r.kx) - r.Sx * Bkz, By = comp(B, r.ky) - r.Sy * Bkz;
    T Cx = comp(C, r.kx) - r.Sx * Ckz, Cy = comp(C, r.ky) - r.Sy * Ckz;
    T U = Cx * By - Cy * Bx;
    T V = Ax * Cy - Ay * Cx;
    T W = Bx * Ay - By * Ax;
    T det = U + V + W;
    T Tn = U * (r.Sz * Akz) + V * (r.Sz * Bkz) + W * (r.Sz * Ckz);
    if (margin == (T)0) {
        // final decision (FP64): closed triangle grown by TRI_TOL
        T mt = (T)TRI_TOL * (fabs(U) + fabs(V) + fabs(W));
        if ((U < -mt || V < -mt || W < -mt) && (U > mt || V > mt || W > mt)) return 0;
        if (!(fabs(det) > (T)3 * mt)) return 0;
        t_out = Tn / det;
        return 1;
    }
    T m = margin * (fabs(U) + fabs(V) + fabs(W));
    bool pos = U > m && V > m && W > m;
    bool neg = U < -m && V < -m && W < -m;
    if (pos || neg) {
        t_out = Tn / det;
        return 1;
    }
    bool mixed = (U < -m || V < -m || W < -m) && (U > m || V > m || W > m);
    if (mixed) return 0;
    t_out = det != (T)0 ? Tn / det : (T)0;
    return 2;
}

__device__ __forceinline__ bool slab(const WRay<float>& r, float lx, float ly, float lz, float hx, float hy, float hz,
                                     float tlo, float thi, float& tn) {
    float tx0 = (lx - r.of.x) * r.inv.x, tx1 = (hx - r.of.x) * r.inv.x;
    float ty0 = (ly - r.of.y) * r.inv.y, ty1 = (hy - r.of.y) * r.inv.y;
    float tz0 = (lz - r.of.z) * r.inv.z, tz1 = (hz - r.of.z) * r.inv.z;
    tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tlo));
    float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), thi));
    return tn <= tf;
}
__device__ __forceinline__ bool slab(const WRay<double>& r, float lx, float ly, float lz, float hx, float hy, float hz,
                                     float tlo, float thi, float& tn) {
    float tx0 = (lx - r.of.x) * r.inv.x, tx1 = (hx - r.of.x) * r.inv.x;
    float ty0 = (ly - r.of.y) * r.inv.y, ty1 = (hy - r.of.y) * r.inv.y;
    float tz0 = (lz - r.of.z) * r.inv.z, tz1 = (hz - r.of.z) * r.inv.z;
    tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tlo));
    float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), thi));
    return tn <= tf;
}

__device__ __forceinline__ int leaf_ref(int first, int count) { return ~((first << 3) | (count - 1)); }

// Shared traversal over the two-child-box BVH with a per-thread stack in shared
// memory (stack[k * blockDim.x + threadIdx.x]).  mode 0: closest hit; mode 1:
// any hit.  Returns the BVH-order index of the hit (or -1); sets `undecided`
// when an FP32 decision was marginal and `t_out` to the hit distance.
template <typename T, int MODE>
__device__ int bvh_query(const BvhNode* __restrict__ nodes, const float4* __restrict__ tris, const WRay<T>& r,
                         T tmin, T tmax, int skip0, int skip1, T margin, int* stack, T& t_out, bool& undecided,
                         int32_t* status) {
    const int stride = blockDim.x;
    int sp = 0;
    int ref = 0;
    int best = -1, best_id = 0x7fffffff;
    T tb = tmax;
    const float tlo = (float)tmin * 0.5f;
    int visits = 0;
    for (;;) {
        if (++visits > RT_MAX_VISITS) {
            rt_set_status(status, RT_ERR_ITER_LIMIT);
            undecided = false;
            return -1;
        }
        if (ref >= 0) {
            const float4* np = reinterpret_cast<const float4*>(nodes + ref);
            float4 a = __ldg(np), b = __ldg(np + 1), c = __ldg(np + 2);
            int4 d = __ldg(reinterpret_cast<const int4*>(np + 3));
            float thi = (float)tb * 1.00001f + 1e-30f;
            float t0, t1;
            bool h0 = slab(r, a.x, a.y, a.z, a.w, b.x, b.y, tlo, thi, t0);
            bool h1 = slab(r, b.z, b.w, c.x, c.y, c.z, c.w, tlo, thi, t1);
            int r0 = d.z > 0 ? leaf_ref(d.x, d.z) : d.x;
            int r1 = d.w > 0 ? leaf_ref(d.y, d.w) : d.y;
            if (h0 && h1) {
                int nearr = t0 <= t1 ? r0 : r1, farr = t0 <= t1 ? r1 : r0;
                if (sp >= RT_STACK) {
                    rt_set_status(status, RT_ERR_STACK_OVERFLOW);
                    undecided = false;
                    return -1;
                }
                stack[sp * stride] = farr;
                sp++;
                ref = nearr;
                continue;
            }
            if (h0) {
                ref = r0;
                continue;
            }
            if (h1) {
                ref = r1;
                continue;
            }
        } else {
            int e = ~ref;
            int first = e >> 3, count = (e & 7) + 1;
            for (int k = first; k < first + count; ++k) {
                float4 p0 = __ldg(tris + 3 * k), p1 = __ldg(tris + 3 * k + 1), p2 = __ldg(tris + 3 * k + 2);
                int id = __float_as_int(p0.w);
                if (id == skip0 || id == skip1) continue;
                T th;
                int cls = tri_test<T>(r, p0, p1, p2, margin, th);
                if (cls == 0) continue;
                if (cls == 2) {
                    // undecided edge: only matters if the hit could be in range
                    if (th > tmin * (T)0.5 && th < tb * (T)1.00001) undecided = true;
                    continue;
                }
                if (!(th > tmin)) {
                    if (margin != (T)0 && th > tmin * (T)0.1) undecided = true;
                    continue;
                }
                if (MODE == 2) {
                    if (th <= tmax && id < best_id) {
                        best_id = id;
                        best = k;
                    }
                    continue;
                }
                if (MODE == 1) {
                    if (th < tmax) {
                        if (margin != (T)0 && (th < tmin * (T)10 || th > tmax - tmin * (T)9))
                            undecided = true;
                        else {
                            t_out = th;
                            return id;
                        }
                    }
                    continue;
                }
                if (margin != (T)0) {
                    if (th < tmin * (T)10) undecided = true;
                    if (best >= 0 && fabs(th - tb) <= (T)1e-4 * tb) undecided = true;
                }
                if (th < tb || (th == tb && id < best_id)) {
                    tb = th;
                    best = k;
                    best_id = id;
                }
            }
        }
        if (sp == 0) break;
        sp--;
        ref = stack[sp * stride];
    }
    t_out = tb;
    return MODE != 1 ? (best >= 0 ? best_id : -1) : -1;
}

// FP64 closest hit: the smallest t, then the lowest triangle index among the hits
// within TIE_TOL of it (independent of the visiting order).
__device__ int closest64(const BvhNode* __restrict__ nodes, const float4* __restrict__ tris, const WRay<double>& r,
                         double tmin, int skip, int* stack, double& t_out, int32_t* status) {
    bool und = false;
    double tb;
    int id = bvh_query<double, 0>(nodes, tris, r, tmin, (double)INFINITY, skip, -1, 0.0, stack, tb, und, status);
    if (id < 0) return -1;
    double t2;
    int id2 = bvh_query<double, 2>(nodes, tris, r, tmin, tb + TIE_TOL * tb, skip, -1, 0.0, stack, t2, und, status);
    t_out = tb;
    return id2 >= 0 ? id2 : id;
}

// ------------------------------------------------------------------ launch directions
// Fibonacci lattice (Gonzalez 2010), FP64 evaluated and rounded to FP32.
__device__ __forceinline__ float3 fib_dir(int64_t i, int64_t n) {
    const double g = 0.6180339887498948482;   // (sqrt(5) - 1) / 2
    double z = 1.0 - (2.0 * (double)i + 1.0) / (double)n;
    double rr = sqrt(fmax(0.0, 1.0 - z * z));
    double x = (double)i * g;
    double phi = 2.0 * RT_PI * (x - floor(x));
    double s, c;
    sincos(phi, &s, &c);
    return make_float3((float)(rr * c), (float)(rr * s), (float)z);
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
    int64_t n_rays;
    int depth;
    double eps;
    unsigned long long* table;
    uint64_t mask;
    unsigned long long* uniq;
    unsigned long long uniq_limit;
    int32_t* overflow;
    unsigned long long* next_ray;
    int64_t* redo;
    unsigned long long* redo_count;
    int64_t redo_cap;
    int32_t* status;
};

__device__ __forceinline__ float3 tri_normal_f(const float4* tris_orig, int id) {
    float4 p0 = __ldg(tris_orig + 3 * id), p1 = __ldg(tris_orig + 3 * id + 1), p2 = __ldg(tris_orig + 3 * id + 2);
    float ex = p1.x - p0.x, ey = p1.y - p0.y, ez = p1.z - p0.z;
    float fx = p2.x - p0.x, fy = p2.y - p0.y, fz = p2.z - p0.z;
    float nx = ey * fz - ez * fy, ny = ez * fx - ex * fz, nz = ex * fy - ey * fx;
    float inv = rsqrtf(nx * nx + ny * ny + nz * nz);
    return make_float3(nx * inv, ny * inv, nz * inv);
}

// Persistent SBR: every lane owns one ray; a lane whose ray ended takes the next
// ray index from a global counter (one atomic per warp refill), so warps stay
// full across bounces (warp-level compaction of the active rays).  One loop
// iteration = one closest-hit query per active lane.
__global__ void __launch_bounds__(TRACE_THREADS) k_sbr(SbrArgs A, const float4* __restrict__ tris_orig) {
    extern __shared__ int smem_stack[];
    int* stack = smem_stack + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int64_t ray = -1;
    bool done = false;
    int bounce = 0, prev = -1;
    uint64_t key = 0;
    WRay<float> r;
    const float eps = (float)A.eps;
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
                    ray = idx;
                    bounce = 0;
                    prev = -1;
                    key = 0;
                    float3 d = fib_dir(idx, A.n_rays);
                    r.o = mk((float)A.tx, (float)A.ty, (float)A.tz);
                    r.d = mk(d.x, d.y, d.z);
                    wray_init(r);
                } else {
                    done = true;
                }
            }
        }
        if (__all_sync(FULL, done)) break;
        if (ray < 0) continue;
        float th;
        bool und = false;
        int id = bvh_query<float, 0>(A.nodes, A.tris, r, eps, INFINITY, prev, -1, SBR_MARGIN, stack, th, und,
                                     A.status);
        if (und) {
            unsigned long long slot = atomicAdd(A.redo_count, 1ull);
            if ((int64_t)slot < A.redo_cap) A.redo[slot] = ray;
            else atomicExch(A.overflow, 2);
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
        float3 n = tri_normal_f(tris_orig, id);
        V3<float> nn = mk(n.x, n.y, n.z);
        V3<float> p = r.o + th * r.d;
        r.d = r.d - (2.0f * dot(r.d, nn)) * nn;
        r.o = p;
        wray_init(r);
        prev = id;
    }
}

// FP64 re-trace of the rays whose FP32 decisions were marginal (same rules, exact
// classification).  Inserts every prefix again; duplicates are harmless.
__global__ void __launch_bounds__(TRACE_THREADS) k_sbr_redo(SbrArgs A, const float4* __restrict__ tris_orig) {
    extern __shared__ int smem_stack[];
    int* stack = smem_stack + threadIdx.x;
    unsigned long long n = *A.redo_count;
    if (n > (unsigned long long)A.redo_cap) n = A.redo_cap;
    for (unsigned long long w = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; w < n;
         w += (unsigned long long)gridDim.x * blockDim.x) {
        int64_t ray = A.redo[w];
        float3 df = fib_dir(ray, A.n_rays);
        WRay<double> r;
        r.o = mk(A.tx, A.ty, A.tz);
        r.d = mk((double)df.x, (double)df.y, (double)df.z);
        wray_init(r);
        int prev = -1;
        uint64_t key = 0;
        for (int b = 0; b < A.depth; ++b) {
            double th;
            int id = closest64(A.nodes, A.tris, r, A.eps, prev, stack, th, A.status);
            if (id < 0) break;
            key = rt_key_push(key, b, id);
            hash_insert(A.table, A.mask, key, A.uniq, A.uniq_limit, A.overflow);
            float4 p0 = __ldg(tris_orig + 3 * id), p1 = __ldg(tris_orig + 3 * id + 1), p2 = __ldg(tris_orig + 3 * id + 2);
            V3<double> e1 = from4<double>(p1) - from4<double>(p0), e2 = from4<double>(p2) - from4<double>(p0);
            V3<double> nn = cross(e1, e2);
            nn = (1.0 / sqrt(dot(nn, nn))) * nn;
            V3<double> p = r.o + th * r.d;
            r.d = r.d - (2.0 * dot(r.d, nn)) * nn;
            r.o = p;
            wray_init(r);
            prev = id;
        }
    }
}

// ------------------------------------------------------------------ compaction + sort
__global__ void k_table_compact(const unsigned long long* __restrict__ table, uint64_t cap, uint64_t* out,
                                unsigned long long* count) {
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
        if (k) out[base + __popc(m & ((1u << lane) - 1))] = k;
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
// Per candidate: length q, triangles, and the image sources I_1..I_q of the
// transmitter (I_j = I_{j-1} - 2 ((I_{j-1} - a_j).n_j) n_j), FP64 and FP32.
__global__ void k_candidates(const uint64_t* __restrict__ keys, int64_t K, int D, double tx, double ty, double tz,
                             const float4* __restrict__ tri_v, const double* __restrict__ tri_n64, int32_t* cand_depth,
                             int32_t* cand_tri, double* img64, float4* img32) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K; k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t key = keys[k];
        int q = rt_key_depth(key);
        cand_depth[k] = q;
        V3<double> I = mk(tx, ty, tz);
        for (int j = 0; j < D; ++j) {
            int t = j < q ? rt_key_tri(key, j) : -1;
            cand_tri[(int64_t)j * K + k] = t;
            if (t >= 0) {
                V3<double> n = mk(tri_n64[4 * t], tri_n64[4 * t + 1], tri_n64[4 * t + 2]);
                V3<double> a = from4<double>(__ldg(tri_v + 3 * t));
                I = I - (2.0 * dot(I - a, n)) * n;
            }
            double* o = img64 + ((int64_t)j * K + k) * 3;
            o[0] = I.x;
            o[1] = I.y;
            o[2] = I.z;
            img32[(int64_t)j * K + k] = make_float4((float)I.x, (float)I.y, (float)I.z, 0.0f);
        }
    }
}

// Point-in-triangle test in FP64: the barycentric coordinates (edge functions
// along the normal over |n|^2) are >= -TRI_TOL.
__device__ __forceinline__ bool point_in_tri64(const float4* __restrict__ tri_v, int t, V3<double> p, double* minbary) {
    V3<double> a = from4<double>(__ldg(tri_v + 3 * t)), b = from4<double>(__ldg(tri_v + 3 * t + 1)),
               c = from4<double>(__ldg(tri_v + 3 * t + 2));
    V3<double> nn = cross(b - a, c - a);
    double e0 = dot(nn, cross(b - a, p - a));
    double e1 = dot(nn, cross(c - b, p - b));
    double e2 = dot(nn, cross(a - c, p - c));
    const double n2 = dot(nn, nn);
    e0 /= n2;
    e1 /= n2;
    e2 /= n2;
    if (minbary) *minbary = fmin(e0, fmin(e1, e2));
    return e0 >= -TRI_TOL && e1 >= -TRI_TOL && e2 >= -TRI_TOL;
}

struct CandView {
    int64_t K;
    const int32_t* depth;
    const int32_t* tri;   // D x K
    const double* img64;  // D x K x 3
    const float4* img32;  // D x K
};

// Back-trace of candidate k from receiver position rx (image method, FP64):
// fills pts[0..q+1] = Tx, s_1..s_q, Rx and returns validity of the geometry
// (0 < u < 1, closed triangle, every segment longer than eps).
__device__ __forceinline__ bool backtrace64(const CandView& C, int64_t k, int q, V3<double> tx, V3<double> rx,
                                            const float4* __restrict__ tri_v, const double* __restrict__ tri_n64,
                                            double eps, V3<double>* pts, double* minbary) {
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
        double u = dot(n, a - from) / den;
        if (!(u > 0.0 && u < 1.0)) return false;
        V3<double> p = from + u * dir;
        double b;
        if (!point_in_tri64(tri_v, t, p, &b)) return false;
        mb = fmin(mb, b);
        pts[j] = p;
    }
    for (int j = 0; j <= q; ++j) {
        V3<double> d = pts[j + 1] - pts[j];
        if (sqrt(dot(d, d)) <= eps) return false;
    }
    if (minbary) *minbary = mb;
    return true;
}

// FP32 prefilter of one (candidate, receiver) pair: false only if the pair is
// invalid by a clear margin.
__device__ __forceinline__ bool prefilter32(const CandView& C, int64_t k, int q, float3 rx,
                                           const float4* __restrict__ tri_bary) {
    const float m = PREFILTER_MARGIN;
    V3<float> P = mk(rx.x, rx.y, rx.z);
    for (int j = q; j >= 1; --j) {
        int t = C.tri[(int64_t)(j - 1) * C.K + k];
        float4 I4 = C.img32[(int64_t)(j - 1) * C.K + k];
        float4 pl = __ldg(tri_bary + 3 * t), g0 = __ldg(tri_bary + 3 * t + 1), g1 = __ldg(tri_bary + 3 * t + 2);
        V3<float> n = mk(pl.x, pl.y, pl.z);
        V3<float> dir = mk(I4.x, I4.y, I4.z) - P;
        float den = dot(n, dir);
        if (fabsf(den) < 1e-20f) return true;   // undecided in FP32
        float u = (pl.w - dot(n, P)) / den;
        if (u < -m || u > 1.0f + m) return false;
        V3<float> s = P + u * dir;
        float l0 = g0.x * s.x + g0.y * s.y + g0.z * s.z + g0.w;
        float l1 = g1.x * s.x + g1.y * s.y + g1.z * s.z + g1.w;
        float l2 = 1.0f - l0 - l1;
        if (l0 < -m || l1 < -m || l2 < -m) return false;
        P = s;
    }
    return true;
}

struct PairArgs {
    CandView C;
    int R;
    const double* rx;
    double tx, ty, tz;
    const float4* tri_v;
    const float4* tri_bary;
    const double* tri_n64;
    double eps;
    uint2* queue;
    unsigned long long* qcount;
    unsigned long long qcap;
    int32_t* overflow;
};

// Image method over all (candidate, receiver) pairs; lanes of a warp take
// consecutive receivers of the same candidate.  Survivors go to the visibility
// queue (one atomic per warp).
__global__ void k_pairs(PairArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t total = A.C.K * (int64_t)A.R;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p0 = blockIdx.x * (int64_t)blockDim.x; p0 < total; p0 += stride) {
        int64_t p = p0 + threadIdx.x;
        bool ok = false;
        int64_t k = 0;
        int r = 0;
        if (p < total) {
            k = p / A.R;
            r = (int)(p - k * A.R);
            int q = A.C.depth[k];
            const double* rp = A.rx + 3 * (int64_t)r;
            if (q == 0) {
                ok = true;
            } else if (prefilter32(A.C, k, q, make_float3((float)rp[0], (float)rp[1], (float)rp[2]), A.tri_bary)) {
                V3<double> pts[RT_MAX_DEPTH + 2];
                ok = backtrace64(A.C, k, q, mk(A.tx, A.ty, A.tz), mk(rp[0], rp[1], rp[2]), A.tri_v, A.tri_n64, A.eps,
                                 pts, nullptr);
            }
        }
        unsigned m = __ballot_sync(FULL, ok);
        if (m) {
            unsigned long long base = 0;
            int leader = __ffs(m) - 1;
            if (lane == leader) base = atomicAdd(A.qcount, (unsigned long long)__popc(m));
            base = __shfl_sync(FULL, base, leader);
            if (ok) {
                unsigned long long slot = base + __popc(m & ((1u << lane) - 1));
                if (slot < A.qcap) A.queue[slot] = make_uint2((unsigned)k, (unsigned)r);
                else atomicExch(A.overflow, 1);
            }
        }
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
    double eps;
    const uint2* queue;
    const unsigned long long* qcount;
    unsigned long long qcap;
    uint32_t* bits;
    int64_t words;   // words per receiver row
    int32_t* status;
};

// Visibility of every segment s_j -> s_{j+1} of a geometrically valid chain:
// any hit with eps < t*len < len - eps, excluding the end triangles.  FP32
// first, FP64 for marginal segments.  Valid pairs set their bit.
__global__ void __launch_bounds__(TRACE_THREADS) k_visibility(VisArgs A) {
    extern __shared__ int smem_stack[];
    int* stack = smem_stack + threadIdx.x;
    unsigned long long n = *A.qcount;
    if (n > A.qcap) n = A.qcap;
    for (unsigned long long w = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; w < n;
         w += (unsigned long long)gridDim.x * blockDim.x) {
        uint2 e = A.queue[w];
        int64_t k = e.x;
        int r = (int)e.y;
        int q = A.C.depth[k];
        const double* rp = A.rx + 3 * (int64_t)r;
        V3<double> pts[RT_MAX_DEPTH + 2];
        if (!backtrace64(A.C, k, q, mk(A.tx, A.ty, A.tz), mk(rp[0], rp[1], rp[2]), A.tri_v, A.tri_n64, A.eps, pts,
                         nullptr))
            continue;
        bool visible = true;
        for (int j = 0; j <= q && visible; ++j) {
            V3<double> d = pts[j + 1] - pts[j];
            double len = sqrt(dot(d, d));
            int s0 = j >= 1 ? A.C.tri[(int64_t)(j - 1) * A.C.K + k] : -1;
            int s1 = j + 1 <= q ? A.C.tri[(int64_t)j * A.C.K + k] : -1;
            double tlo = A.eps / len, thi = 1.0 - A.eps / len;
            WRay<float> rf;
            rf.o = mk((float)pts[j].x, (float)pts[j].y, (float)pts[j].z);
            rf.d = mk((float)d.x, (float)d.y, (float)d.z);
            wray_init(rf);
            float th;
            bool und = false;
            int hit = bvh_query<float, 1>(A.nodes, A.bvh_tris, rf, (float)tlo, (float)thi, s0, s1, SBR_MARGIN, stack,
                                          th, und, A.status);
            if (hit >= 0) {
                visible = false;
            } else if (und) {
                WRay<double> rd;
                rd.o = pts[j];
                rd.d = d;
                wray_init(rd);
                double t64;
                bool u2 = false;
                int h2 = bvh_query<double, 1>(A.nodes, A.bvh_tris, rd, tlo, thi, s0, s1, 0.0, stack, t64, u2, A.status);
                if (h2 >= 0) visible = false;
            }
        }
        if (visible) atomicOr(A.bits + (int64_t)r * A.words + (k >> 5), 1u << (k & 31));
    }
}

// Per-receiver popcount of the validity bitmask (one warp per receiver).
__global__ void k_row_count(const uint32_t* __restrict__ bits, int R, int64_t words, int64_t* counts) {
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
    __shared__ int64_t part[1024];
    const int T = blockDim.x;
    const int per = (n + T - 1) / T;
    const int lo = threadIdx.x * per, hi = min(n, lo + per);
    int64_t s = 0;
    for (int i = lo; i < hi; ++i) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        int64_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = threadIdx.x > 0 ? part[threadIdx.x - 1] : 0;
    for (int i = lo; i < hi; ++i) {
        offsets[i] = run;
        run += counts[i];
    }
    if (threadIdx.x == T - 1) offsets[n] = part[T - 1];
}

// Expansion of the bitmask into (receiver, candidate) pairs at their final
// positions, candidates in increasing order within a receiver (one warp each).
__global__ void k_expand(const uint32_t* __restrict__ bits, int R, int64_t words, const int64_t* __restrict__ offsets,
                         int32_t* path_rx, int32_t* path_cand) {
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
                path_rx[my] = (int32_t)r;
                path_cand[my] = (int32_t)(w * 32 + bit);
                my++;
            }
            pos += __shfl_sync(FULL, incl, 31);
        }
    }
}

// FP64 points of every emitted path, its triangle slots, and whether any
// reflection point lies on a triangle edge (input of the duplicate rule).
__global__ void k_points(CandView C, int64_t P, int D, const int32_t* __restrict__ path_rx,
                         const int32_t* __restrict__ path_cand, const double* __restrict__ rx, double tx, double ty,
                         double tz, const float4* __restrict__ tri_v, const double* __restrict__ tri_n64, double eps,
                         double* pts_out, int32_t* depth_out, int32_t* rx_out, int32_t* tri_out, int32_t* edge_flag,
                         int32_t* status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t k = path_cand[i];
        int r = path_rx[i];
        int q = C.depth[k];
        const double* rp = rx + 3 * (int64_t)r;
        V3<double> pts[RT_MAX_DEPTH + 2];
        double mb = 1.0;
        if (!backtrace64(C, k, q, mk(tx, ty, tz), mk(rp[0], rp[1], rp[2]), tri_v, tri_n64, eps, pts, &mb))
            rt_set_status(status, RT_ERR_NUMERIC);
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
    if (sqrt(dot(c, c)) > 1e-9) return false;
    double dt = dot(a, from4<double>(__ldg(tri_v + 3 * t)));
    double du = dot(a, from4<double>(__ldg(tri_v + 3 * u)));
    return fabs(dt - du) <= 1e-9 * diag;
}

// Coplanar-duplicate rule: a path with a reflection point on an edge is dropped
// if another path of its receiver, of equal length, has pairwise coplanar
// triangles, the same points (within 1e-9 diag) and a smaller triangle sequence.
__global__ void k_dedup(int64_t P, int D, const int64_t* __restrict__ rx_offsets, const int32_t* __restrict__ path_rx,
                        const int32_t* __restrict__ path_cand, const int32_t* __restrict__ depth,
                        const int32_t* __restrict__ tri, const double* __restrict__ pts,
                        const int32_t* __restrict__ edge_flag, const double* __restrict__ tri_n64,
                        const float4* __restrict__ tri_v, double diag, uint32_t* bits, int64_t words,
                        unsigned long long* drops) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        if (!edge_flag[i]) continue;
        int r = path_rx[i];
        int q = depth[i];
        for (int64_t j = rx_offsets[r]; j < rx_offsets[r + 1]; ++j) {
            if (j == i || !edge_flag[j] || depth[j] != q) continue;
            bool same = true;
            for (int b = 0; b < q && same; ++b) same = coplanar64(tri_n64, tri_v, tri[(int64_t)b * P + i], tri[(int64_t)b * P + j], diag);
            for (int b = 1; b <= q && same; ++b) {
                const double* pi = pts + ((int64_t)i * (D + 2) + b) * 3;
                const double* pj = pts + ((int64_t)j * (D + 2) + b) * 3;
                double dx = pi[0] - pj[0], dy = pi[1] - pj[1], dz = pi[2] - pj[2];
                same = sqrt(dx * dx + dy * dy + dz * dz) <= 1e-9 * diag;
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
                break;
            }
        }
    }
}

inline int grid_for(rt_ctx* ctx, int64_t n, int threads, int per_sm = 8) {
    int64_t g = (n + threads - 1) / threads;
    int64_t cap = (int64_t)ctx->num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

// ---------------------------------------------------------------------------
// Host driver of the tracing pipeline.

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

    // ---------------- 1-2: SBR into the hash set (grow and retry on overflow)
    const int64_t redo_cap = std::max<int64_t>(1 << 16, n_rays / 16);
    uint64_t* d_sorted = nullptr;
    int64_t n_uniq = 0;
    for (int attempt = 0;; ++attempt) {
        size_t cap = sc->hash_cap;
        const size_t sort_cap = std::max<size_t>(SORT_BLOCK, cap / 2);
        size_t need = cap * 8 + sort_cap * 8 + 256 * 8 + redo_cap * 8 + 4096;
        void* base;
        rt_status s = rt_scratch(ctx, need, &base);
        if (s != RT_OK) return s;
        Arena ar{(char*)base};
        unsigned long long* table = ar.take<unsigned long long>(cap);
        unsigned long long* counters = ar.take<unsigned long long>(8);   // uniq, next_ray, redo_count, compact
        int32_t* flags = ar.take<int32_t>(8);
        int64_t* redo = ar.take<int64_t>(redo_cap);
        uint64_t* sorted = ar.take<uint64_t>(sort_cap);
        RT_CK(ctx, cudaMemsetAsync(table, 0, cap * 8, st));
        RT_CK(ctx, cudaMemsetAsync(counters, 0, 8 * 8, st));
        RT_CK(ctx, cudaMemsetAsync(flags, 0, 8 * 4, st));
        SbrArgs A;
        A.nodes = sc->d_nodes;
        A.tris = sc->d_bvh_tris;
        A.tx = tx_host[0];
        A.ty = tx_host[1];
        A.tz = tx_host[2];
        A.n_rays = n_rays;
        A.depth = D;
        A.eps = sc->eps;
        A.table = table;
        A.mask = cap - 1;
        A.uniq = counters + 0;
        A.uniq_limit = cap / 2;
        A.overflow = flags;
        A.next_ray = counters + 1;
        A.redo = redo;
        A.redo_count = counters + 2;
        A.redo_cap = redo_cap;
        A.status = status;
        int blocks = ctx->num_sms * 8;
        k_sbr<<<blocks, TRACE_THREADS, stack_bytes, st>>>(A, sc->d_tri_v);
        RT_CK_LAUNCH(ctx);
        k_sbr_redo<<<ctx->num_sms * 2, TRACE_THREADS, stack_bytes, st>>>(A, sc->d_tri_v);
        RT_CK_LAUNCH(ctx);
        int64_t* hp = ctx->h_pinned;
        RT_CK(ctx, cudaMemcpyAsync(hp, counters, 8, cudaMemcpyDeviceToHost, st));
        RT_CK(ctx, cudaMemcpyAsync(hp + 1, flags, 4, cudaMemcpyDeviceToHost, st));
        RT_CK(ctx, cudaStreamSynchronize(st));
        n_uniq = hp[0];
        int32_t ovf = *(int32_t*)(hp + 1);
        if (ovf == 2) return rt_fail(ctx, RT_ERR_CAPACITY, "FP64 re-trace list overflow");
        if (ovf) {
            if (attempt >= 6 || sc->hash_cap >= ((size_t)1 << 31))
                return rt_fail(ctx, RT_ERR_CAPACITY, "candidate hash table overflow");
            sc->hash_cap *= 4;
            continue;
        }
        // ---------------- compact + sort (length, lexicographic)
        int64_t n_pad = SORT_BLOCK;
        while (n_pad < n_uniq) n_pad <<= 1;
        d_sorted = sorted;
        k_fill_u64<<<grid_for(ctx, n_pad, 256), 256, 0, st>>>(d_sorted, n_pad, ~0ull);
        k_table_compact<<<grid_for(ctx, cap, 256, 16), 256, 0, st>>>(table, cap, d_sorted, counters + 3);
        RT_CK_LAUNCH(ctx);
        k_bitonic_local<<<(unsigned)(n_pad / SORT_BLOCK), 1024, 0, st>>>(d_sorted);
        for (uint64_t k = 2 * SORT_BLOCK; k <= (uint64_t)n_pad; k <<= 1) {
            for (uint64_t j = k >> 1; j >= (uint64_t)SORT_BLOCK; j >>= 1)
                k_bitonic_global<<<grid_for(ctx, n_pad, 256, 16), 256, 0, st>>>(d_sorted, n_pad, j, k);
            k_bitonic_merge_local<<<(unsigned)(n_pad / SORT_BLOCK), 1024, 0, st>>>(d_sorted, k);
        }
        RT_CK_LAUNCH(ctx);
        break;
    }

    // ---------------- candidates (LoS first)
    const int64_t K = n_uniq + 1;
    rt_paths* p = new rt_paths();
    p->scene = scene;
    p->stream = st;
    p->D = D;
    p->R = n_rx;
    p->K = K;
    auto fail = [&](rt_status s) {
        rt_paths_free(p);
        return s;
    };
#define TCK(call)                                                         \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return fail(rt_cuda_fail(ctx, _e, #call)); \
    } while (0)
    TCK(cudaMallocAsync((void**)&p->d_cand, K * 8, st));
    TCK(cudaMemsetAsync(p->d_cand, 0, 8, st));
    if (n_uniq > 0) TCK(cudaMemcpyAsync(p->d_cand + 1, d_sorted, n_uniq * 8, cudaMemcpyDeviceToDevice, st));

    // candidate arrays + visibility queue + bitmask: a fresh scratch layout
    const int64_t words = (K + 31) / 32;
    int32_t* cand_depth = nullptr;
    int32_t* cand_tri = nullptr;
    double* img64 = nullptr;
    float4* img32 = nullptr;
    uint2* queue = nullptr;
    uint32_t* bits = nullptr;
    unsigned long long* counters = nullptr;
    int32_t* flags = nullptr;
    int64_t* counts = nullptr;
    for (int attempt = 0;; ++attempt) {
        size_t qcap = sc->queue_cap;
        size_t need = K * 4 + (size_t)D * K * 4 + (size_t)D * K * 24 + (size_t)D * K * 16 + qcap * 8 +
                      (size_t)n_rx * words * 4 + 64 * 8 + (size_t)(n_rx + 1) * 8 * 2 + 16 * 256;
        void* base;
        rt_status s = rt_scratch(ctx, need, &base);
        if (s != RT_OK) return fail(s);
        Arena ar{(char*)base};
        cand_depth = ar.take<int32_t>(K);
        cand_tri = ar.take<int32_t>((size_t)D * K);
        img64 = ar.take<double>((size_t)D * K * 3);
        img32 = ar.take<float4>((size_t)D * K);
        queue = ar.take<uint2>(qcap);
        bits = ar.take<uint32_t>((size_t)n_rx * words);
        counters = ar.take<unsigned long long>(8);
        flags = ar.take<int32_t>(8);
        counts = ar.take<int64_t>(n_rx + 1);
        TCK(cudaMemsetAsync(counters, 0, 64, st));
        TCK(cudaMemsetAsync(flags, 0, 32, st));
        TCK(cudaMemsetAsync(bits, 0, (size_t)n_rx * words * 4, st));
        k_candidates<<<grid_for(ctx, K, 256), 256, 0, st>>>(p->d_cand, K, D, tx_host[0], tx_host[1], tx_host[2],
                                                            sc->d_tri_v, sc->d_tri_n64, cand_depth, cand_tri, img64,
                                                            img32);
        TCK(cudaGetLastError());
        PairArgs PA;
        PA.C = CandView{K, cand_depth, cand_tri, img64, img32};
        PA.R = n_rx;
        PA.rx = rx_dev;
        PA.tx = tx_host[0];
        PA.ty = tx_host[1];
        PA.tz = tx_host[2];
        PA.tri_v = sc->d_tri_v;
        PA.tri_bary = sc->d_tri_bary;
        PA.tri_n64 = sc->d_tri_n64;
        PA.eps = sc->eps;
        PA.queue = queue;
        PA.qcount = counters;
        PA.qcap = qcap;
        PA.overflow = flags;
        k_pairs<<<grid_for(ctx, K * (int64_t)n_rx, 256, 16), 256, 0, st>>>(PA);
        TCK(cudaGetLastError());
        VisArgs VA;
        VA.C = PA.C;
        VA.rx = rx_dev;
        VA.tx = tx_host[0];
        VA.ty = tx_host[1];
        VA.tz = tx_host[2];
        VA.nodes = sc->d_nodes;
        VA.bvh_tris = sc->d_bvh_tris;
        VA.tri_v = sc->d_tri_v;
        VA.tri_n64 = sc->d_tri_n64;
        VA.eps = sc->eps;
        VA.queue = queue;
        VA.qcount = counters;
        VA.qcap = qcap;
        VA.bits = bits;
        VA.words = words;
        VA.status = status;
        k_visibility<<<ctx->num_sms * 8, TRACE_THREADS, stack_bytes, st>>>(VA);
        TCK(cudaGetLastError());
        int64_t* hp = ctx->h_pinned;
        TCK(cudaMemcpyAsync(hp, flags, 4, cudaMemcpyDeviceToHost, st));
        TCK(cudaStreamSynchronize(st));
        if (*(int32_t*)hp) {
            if (attempt >= 6) return fail(rt_fail(ctx, RT_ERR_CAPACITY, "visibility queue overflow"));
            sc->queue_cap *= 4;
            continue;
        }
        break;
    }

    // ---------------- emission (repeated once more if the duplicate rule drops paths)
    int32_t* path_rx = nullptr;
    int32_t* path_cand = nullptr;
    int32_t* edge = nullptr;
    for (int pass = 0;; ++pass) {
        k_row_count<<<grid_for(ctx, (int64_t)n_rx * 32, 256, 16), 256, 0, st>>>(bits, n_rx, words, counts);
        TCK(cudaGetLastError());
        if (!p->d_rx_offsets) TCK(cudaMallocAsync((void**)&p->d_rx_offsets, (size_t)(n_rx + 1) * 8, st));
        k_scan<<<1, 1024, 0, st>>>(counts, n_rx, p->d_rx_offsets);
        TCK(cudaGetLastError());
        int64_t* hp = ctx->h_pinned;
        TCK(cudaMemcpyAsync(hp, p->d_rx_offsets + n_rx, 8, cudaMemcpyDeviceToHost, st));
        TCK(cudaStreamSynchronize(st));
        const int64_t P = hp[0];
        p->P = P;
        if (pass > 0) {
            cudaFreeAsync(p->d_pts, st);
            cudaFreeAsync(p->d_depth, st);
            cudaFreeAsync(p->d_rx, st);
            cudaFreeAsync(p->d_tri, st);
            cudaFreeAsync(path_cand, st);
            cudaFreeAsync(edge, st);
        }
        const size_t Pa = std::max<int64_t>(P, 1);
        TCK(cudaMallocAsync((void**)&p->d_pts, Pa * (D + 2) * 3 * 8, st));
        TCK(cudaMallocAsync((void**)&p->d_depth, Pa * 4, st));
        TCK(cudaMallocAsync((void**)&p->d_rx, Pa * 4, st));
        TCK(cudaMallocAsync((void**)&p->d_tri, Pa * D * 4, st));
        TCK(cudaMallocAsync((void**)&path_cand, Pa * 4, st));
        TCK(cudaMallocAsync((void**)&edge, Pa * 4, st));
        path_rx = p->d_rx;
        if (P > 0) {
            k_expand<<<grid_for(ctx, (int64_t)n_rx * 32, 256, 16), 256, 0, st>>>(bits, n_rx, words, p->d_rx_offsets,
                                                                                 path_rx, path_cand);
            TCK(cudaGetLastError());
            CandView C{K, cand_depth, cand_tri, img64, img32};
            k_points<<<grid_for(ctx, P, 256), 256, 0, st>>>(C, P, D, path_rx, path_cand, rx_dev, tx_host[0], tx_host[1],
                                                             tx_host[2], sc->d_tri_v, sc->d_tri_n64, sc->eps, p->d_pts,
                                                             p->d_depth, p->d_rx, p->d_tri, edge, status);
            TCK(cudaGetLastError());
        }
        if (pass > 0 || P == 0) break;
        TCK(cudaMemsetAsync(counters + 4, 0, 8, st));
        k_dedup<<<grid_for(ctx, P, 256), 256, 0, st>>>(P, D, p->d_rx_offsets, path_rx, path_cand, p->d_depth,
                                                       p->d_tri, p->d_pts, edge, sc->d_tri_n64, sc->d_tri_v, sc->diag, bits, words,
                                                       counters + 4);
        TCK(cudaGetLastError());
        TCK(cudaMemcpyAsync(hp, counters + 4, 8, cudaMemcpyDeviceToHost, st));
        TCK(cudaStreamSynchronize(st));
        if (hp[0] == 0) break;
    }
    cudaFreeAsync(path_cand, st);
    cudaFreeAsync(edge, st);
    rt_status s = rt_launch_paths_records(ctx, p);
    if (s != RT_OK) return fail(s);
#undef TCK
    *out = p;
    return RT_OK;
}
