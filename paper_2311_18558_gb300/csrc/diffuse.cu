// Diffuse reflection (arXiv 2311.18558, Sec. II-D "Diffuse reflection",
// Eq. scattered_field), found by next-event estimation during shoot-and-bounce
// (Sec. II-F), with the trainable scattering pattern of Sec. III-C
// (Eq. trainable_scattering_pattern) and the specular share R = sqrt(1 - S^2)
// of Eq. specular_reflection.
//
// Tracing (once per geometry):
//   1. k_df_rays: every launch ray (canonical FP32 Fibonacci direction) bounces
//      specularly up to D times; closest hits are decided in FP64 (watertight
//      test, triangles grown by TRI_TOL, lowest index among hits within TIE_TOL),
//      and hit points and reflected directions are carried in FP64.  Every hit
//      s_j of ray i is a diffuse source with index i * D + (j - 1).
//   2. k_df_nee: one thread per (source, receiver): the receiver must be strictly
//      on the side of t_j's plane the ray came from and see s_j (FP64 any-hit
//      over (eps, len - eps), t_j excluded); visible pairs set a bit of a
//      (receiver x source) mask.
//   3. per-receiver popcounts, scans and an ordered expansion give the paths
//      grouped by receiver and ordered by (ray, j).
//   4. k_df_prefix forms, once per (ray, j), what all paths from s_j share (the
//      FP64 length up to s_j, the reflection bases of bounces 1..j);
//      k_df_records adds each path's last segment and scattered basis and writes
//      the FP32 records for the field kernels.
// Fields (every calibration step): the specular prefix as in the specular
// kernels (with R per bounce), then the diffuse bounce
//   |E_s| = sqrt(4 pi / N) S sqrt(f_s) |diag(r_perp, r_par) v|,
//   a = lambda / (4 pi) sqrt(g_T g_R) |E_s| / d_last (D_last[0,0] sqrt(1 - K_x)
//       + D_last[0,1] sqrt(K_x)),
// where v is the incident field at s_j in its incidence basis without the
// spherical spreading 1 / l_j, which cancels against cos(theta_i) dA = 4 pi l_j^2 / N
// (each ray samples the solid angle 4 pi / N).  The scattered polarisation
// [sqrt(1 - K_x) e^{j chi_1}, sqrt(K_x) e^{j chi_2}] (the phases per path, zero
// unless rt_set_diffuse_phases gave them) is taken in the basis
// e_perp = k_s x n / |k_s x n|, e_par = e_perp x k_s of the scattered direction.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "fresnel.cuh"
#include "vec3f.cuh"
#include "launch_dir.cuh"
#include "rt_internal.cuh"
#include "segquery.cuh"

namespace {

constexpr int DF_THREADS = 128;
constexpr int MAT_PEC = 1 << 30;       // PEC flag in the per-bounce material word (as the specular records)
constexpr float DF_PI = 3.14159265358979323846f;

int grid_of(const rt_ctx* ctx, int64_t n, int threads, int per_sm) {
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)ctx->num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

struct Scn {
    const BvhNode* nodes;
    const float4* tris;      // BVH order, original id in v0.w
    const double* n64;       // 4 per triangle: unit normal, n.v0
    const float4* plane32;   // 3 per triangle, the first = (unit normal, n.v0) in FP32
    double eps;
    const float4* tri_v;     // 3 per triangle (vertices; the plane id in the second record's .w)
};

__device__ __forceinline__ void load_n(const double* n64, int t, double n[3]) {
    n[0] = __ldg(n64 + 4 * t);
    n[1] = __ldg(n64 + 4 * t + 1);
    n[2] = __ldg(n64 + 4 * t + 2);
}

// ------------------------------------------------------------------ 1. rays
// Hits of ray i at bounce b: tri[b * N + i] (-1 after the ray escaped) and the
// FP64 point pt[(b * N + i) * 3 + c].  The point and the reflected direction use
// uncontracted FP64 operations, as the definition writes them.
__global__ void __launch_bounds__(DF_THREADS) k_df_rays(int64_t N, int D, double tx0, double tx1, double tx2,
                                                        const float* __restrict__ z, Scn S, int32_t* __restrict__ tri,
                                                        double* __restrict__ pt, float4* __restrict__ pt32, int R,
                                                        const double* __restrict__ rx, float4* __restrict__ rx32,
                                                        int32_t* status) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < R; q += (int64_t)gridDim.x * blockDim.x)
        rx32[q] = make_float4((float)rx[3 * q], (float)rx[3 * q + 1], (float)rx[3 * q + 2], 0.0f);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float3 f = launch_dir(i, __ldg(z + i));
        Ray64 r;
        r.o[0] = tx0;
        r.o[1] = tx1;
        r.o[2] = tx2;
        r.d[0] = f.x;
        r.d[1] = f.y;
        r.d[2] = f.z;
        int prev = -1;
        int b = 0;
        for (; b < D; ++b) {
            ray64_init(r);
            Ray32 q;
            ray32_set(make_float3((float)r.o[0], (float)r.o[1], (float)r.o[2]),
                      make_float3((float)r.d[0], (float)r.d[1], (float)r.d[2]), q);
            double th;
            const int t = closest_hit64(S.nodes, S.tris, r, q, S.eps, prev, th, status);
            if (t < 0) break;
            double p[3], n[3];
            for (int c = 0; c < 3; ++c) p[c] = __dadd_rn(r.o[c], __dmul_rn(th, r.d[c]));
            tri[(int64_t)b * N + i] = t;
            for (int c = 0; c < 3; ++c) pt[((int64_t)b * N + i) * 3 + c] = p[c];
            pt32[(int64_t)b * N + i] = make_float4((float)p[0], (float)p[1], (float)p[2], 0.0f);
            load_n(S.n64, t, n);
            const double dn = __dadd_rn(__dadd_rn(__dmul_rn(r.d[0], n[0]), __dmul_rn(r.d[1], n[1])),
                                        __dmul_rn(r.d[2], n[2]));
            const double dn2 = __dmul_rn(2.0, dn);
            for (int c = 0; c < 3; ++c) {
                r.d[c] = __dsub_rn(r.d[c], __dmul_rn(dn2, n[c]));
                r.o[c] = p[c];
            }
            prev = t;
        }
        for (; b < D; ++b) tri[(int64_t)b * N + i] = -1;
    }
}

// ------------------------------------------------------------------ 2. next-event estimation
// One (source, receiver) pair of the next-event estimation: source s = i D + b is
// hit b of launch ray i.
__device__ __forceinline__ void nee_pair(int64_t N, int b, int i, int s, int r, double tx0, double tx1, double tx2,
                                         const double* __restrict__ rx, const float4* __restrict__ rx32,
                                         const int32_t* __restrict__ tri, const double* __restrict__ pt,
                                         const float4* __restrict__ pt32, const Scn& S, uint32_t* __restrict__ mask,
                                         int64_t W, int32_t* status) {
    const int t = __ldg(tri + (int64_t)b * N + i);
    if (t < 0) return;
    // sides of the plane in FP32 (the FP32 copies are the rounded FP64 values; the
    // sign is certain when |side| exceeds 1e-6 (|x|_1 + |p|_1), far above the
    // rounding of the copies, the normal and the dot product), else in FP64
    const float4 pf = __ldg(pt32 + (int64_t)b * N + i);
    const float4 xf = __ldg(rx32 + r);
    const float4 vf = b == 0 ? make_float4((float)tx0, (float)tx1, (float)tx2, 0.0f)
                             : __ldg(pt32 + (int64_t)(b - 1) * N + i);
    const float4 nf = __ldg(S.plane32 + 3 * t);
    const float sr = (xf.x - pf.x) * nf.x + (xf.y - pf.y) * nf.y + (xf.z - pf.z) * nf.z;
    const float si = (vf.x - pf.x) * nf.x + (vf.y - pf.y) * nf.y + (vf.z - pf.z) * nf.z;
    const float ap = fabsf(pf.x) + fabsf(pf.y) + fabsf(pf.z);
    const float br = 1e-6f * (fabsf(xf.x) + fabsf(xf.y) + fabsf(xf.z) + ap);
    const float bi = 1e-6f * (fabsf(vf.x) + fabsf(vf.y) + fabsf(vf.z) + ap);
    double p[3], x[3];
    for (int c = 0; c < 3; ++c) {
        p[c] = __ldg(pt + ((int64_t)b * N + i) * 3 + c);
        x[c] = __ldg(rx + 3 * (int64_t)r + c);
    }
    if (fabsf(sr) > br && fabsf(si) > bi) {
        if ((sr > 0.0f) != (si > 0.0f)) return;
    } else {
        double pv[3], n[3];
        if (b == 0) {
            pv[0] = tx0;
            pv[1] = tx1;
            pv[2] = tx2;
        } else {
            for (int c = 0; c < 3; ++c) pv[c] = __ldg(pt + ((int64_t)(b - 1) * N + i) * 3 + c);
        }
        load_n(S.n64, t, n);
        const double side_in = (pv[0] - p[0]) * n[0] + (pv[1] - p[1]) * n[1] + (pv[2] - p[2]) * n[2];
        const double side_rx = (x[0] - p[0]) * n[0] + (x[1] - p[1]) * n[1] + (x[2] - p[2]) * n[2];
        if (!((side_in > 0.0 && side_rx > 0.0) || (side_in < 0.0 && side_rx < 0.0))) return;
    }
    Ray64 ray;
    for (int c = 0; c < 3; ++c) {
        ray.o[c] = p[c];
        ray.d[c] = x[c] - p[c];
    }
    const float3 o32 = make_float3(pf.x, pf.y, pf.z);
    const float3 d32 = make_float3((float)ray.d[0], (float)ray.d[1], (float)ray.d[2]);
    // |d| > eps decided in FP32 where the FP32 length (relative error below 1e-6)
    // is clear of eps^2 by 1e-5, else in FP64
    const float len2f = d32.x * d32.x + d32.y * d32.y + d32.z * d32.z;
    const float e2f = (float)(S.eps * S.eps);
    if (len2f < e2f * 0.99999f) return;
    if (!(len2f > e2f * 1.00001f)) {
        const double len2 = ray.d[0] * ray.d[0] + ray.d[1] * ray.d[1] + ray.d[2] * ray.d[2];
        if (!(len2 > S.eps * S.eps)) return;
    }
    // the source triangle's plane: the segment meets it only at its start
    const int pl = __float_as_int(__ldg(S.tri_v + 3 * t + 1).w);
    if (any_hit_seg(S.nodes, S.tris, ray, o32, d32, len2f, S.eps, t, status, -1, pl)) return;
    atomicOr(mask + (int64_t)r * W + (s >> 5), 1u << (s & 31));
}

// Pair index q = s * R + r (receivers fastest, so a warp shares its origin).
__global__ void __launch_bounds__(DF_THREADS) k_df_nee(int64_t N, int D, int R, double tx0, double tx1, double tx2,
                                                       const double* __restrict__ rx, const float4* __restrict__ rx32,
                                                       const int32_t* __restrict__ tri, const double* __restrict__ pt,
                                                       const float4* __restrict__ pt32, Scn S,
                                                       uint32_t* __restrict__ mask, int64_t W, int32_t* status) {
    // q = s R + r, advanced by the grid stride without a 64-bit division per pair
    // (s = i D + b < 2^31: n_rays max_depth < 2^31 is checked on the host)
    const int64_t total = N * D * (int64_t)R;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t q0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q0 >= total) return;
    int r = (int)(q0 % R);
    int64_t s = q0 / R;
    const int64_t ds = stride / R;
    const int dr = (int)(stride % R);
    for (int64_t q = q0; q < total; q += stride) {
        const int si = (int)s;
        const int i = si / D;
        const int b = si - i * D;
        nee_pair(N, b, i, si, r, tx0, tx1, tx2, rx, rx32, tri, pt, pt32, S, mask, W, status);
        s += ds;
        r += dr;
        if (r >= R) {
            r -= R;
            ++s;
        }
    }
}

// ------------------------------------------------------------------ 3. ordered emission
// One block per receiver: exclusive prefix of the word popcounts within the row
// (word_off) and the row total (cnt).
__global__ void k_df_row_scan(int64_t W, const uint32_t* __restrict__ mask, int32_t* __restrict__ word_off,
                              int64_t* __restrict__ cnt) {
    __shared__ int32_t warp_sum[32];
    __shared__ int64_t carry;
    const int r = blockIdx.x;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t base = 0; base < W; base += blockDim.x) {
        const int64_t w = base + threadIdx.x;
        const int v = w < W ? __popc(__ldg(mask + (int64_t)r * W + w)) : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int ws = lane < nw ? warp_sum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += y;
            }
            if (lane < nw) warp_sum[lane] = ws;
        }
        __syncthreads();
        const int before = (wid > 0 ? warp_sum[wid - 1] : 0) + x - v;
        if (w < W) word_off[(int64_t)r * W + w] = (int32_t)(carry + before);
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_sum[nw - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) cnt[r] = carry;
}

// Single block: rx_off[0] = 0, rx_off[r + 1] = rx_off[r] + cnt[r].
__global__ void k_df_offsets(int R, const int64_t* __restrict__ cnt, int64_t* __restrict__ off) {
    __shared__ int64_t warp_sum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) {
        carry = 0;
        off[0] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < R; base += blockDim.x) {
        const int r = base + threadIdx.x;
        const int64_t v = r < R ? cnt[r] : 0;
        int64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int64_t ws = lane < nw ? warp_sum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += y;
            }
            if (lane < nw) warp_sum[lane] = ws;
        }
        __syncthreads();
        const int64_t incl = (wid > 0 ? warp_sum[wid - 1] : 0) + x;
        if (r < R) off[r + 1] = carry + incl;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_sum[nw - 1];
        __syncthreads();
    }
}

__global__ void k_df_expand(int R, int64_t W, const uint32_t* __restrict__ mask, const int32_t* __restrict__ word_off,
                            const int64_t* __restrict__ rx_off, int32_t* __restrict__ out_rx,
                            int64_t* __restrict__ out_src) {
    const int64_t total = (int64_t)R * W;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        uint32_t bits = __ldg(mask + q);
        if (!bits) continue;
        const int r = (int)(q / W);
        const int64_t w = q - (int64_t)r * W;
        int64_t o = __ldg(rx_off + r) + __ldg(word_off + q);
        while (bits) {
            const int k = __ffs(bits) - 1;
            bits &= bits - 1;
            out_rx[o] = r;
            out_src[o] = w * 32 + k;
            ++o;
        }
    }
}

// ------------------------------------------------------------------ records
struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3(double x, double y, double z) { return D3{x, y, z}; }
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return d3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ double dotd(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

struct RecOut {
    int32_t* depth;
    int32_t* tri;      // D x P
    double* pts;       // P x (D + 2) x 3
    double* tau;
    float* len;        // d_last
    int2* mc;          // D x P
    float4* Dm;        // (D + 1) x P
    float4* dir;       // 2 x P
    float4* scat;      // P
};

// What every diffuse path of one (ray, diffuse bounce j) shares: the path up to the
// diffuse point is the ray's own, only the last segment goes to the receiver.
// Index s = ray * D + j - 1 (the source index of the emission).
struct __align__(16) DfPre {
    double ell;    // length of the j segments up to the diffuse point (FP64)
    double pad;
    float4 kin;    // direction of incidence at the diffuse point
    float4 n;      // unit normal there, facing the incident wave
    float4 ep;     // e_perp of the last reflection basis (the fallback of the scattered basis)
    float4 d0;     // direction of departure
};

// One thread per (ray, bounce): lengths in FP64, directions and the reflection bases
// of bounces 1..j in FP32 (the records are stored in FP32).  Dm and mc of bounce b
// go to pre_Dm / pre_mc[s * D + b - 1].
__global__ void k_df_prefix(int64_t N, int D, double tx0, double tx1, double tx2,
                            const int32_t* __restrict__ hit_tri, const double* __restrict__ hit_pt,
                            const double* __restrict__ n64, const int32_t* __restrict__ tri_material,
                            const uint8_t* __restrict__ is_pec, DfPre* __restrict__ pre,
                            float4* __restrict__ pre_Dm, int2* __restrict__ pre_mc) {
    const int64_t M = N * D;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < M; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ray = s / D;
        const int j = (int)(s - ray * D) + 1;
        if (hit_tri[(int64_t)(j - 1) * N + ray] < 0) continue;   // the ray escaped before bounce j
        D3 pts[RT_MAX_DEPTH + 1];
        pts[0] = d3(tx0, tx1, tx2);
        for (int b = 1; b <= j; ++b) {
            const double* q = hit_pt + ((int64_t)(b - 1) * N + ray) * 3;
            pts[b] = d3(q[0], q[1], q[2]);
        }
        F3 k[RT_MAX_DEPTH + 1];
        double ell = 0.0;
        for (int b = 1; b <= j; ++b) {
            const D3 dv = sub(pts[b], pts[b - 1]);
            const double db = sqrt(dotd(dv, dv));
            const float inv = 1.0f / (float)db;
            k[b] = f3((float)dv.x * inv, (float)dv.y * inv, (float)dv.z * inv);
            ell += db;
        }
        F3 out_p, out_q;
        sph_basis_f(k[1], &out_p, &out_q);
        F3 n = f3(0.0f, 0.0f, 0.0f), e_perp = n;
        for (int b = 1; b <= j; ++b) {
            const int t = hit_tri[(int64_t)(b - 1) * N + ray];
            n = f3((float)n64[4 * t], (float)n64[4 * t + 1], (float)n64[4 * t + 2]);
            if (fdot(k[b], n) > 0.0f) n = fscl(-1.0f, n);       // facing the incident wave
            const float cos_i = -fdot(k[b], n);
            e_perp = perp_or_f(k[b], n, out_p);
            const F3 in_q = fcross(e_perp, k[b]);
            pre_Dm[s * D + b - 1] =
                make_float4(fdot(e_perp, out_p), fdot(e_perp, out_q), fdot(in_q, out_p), fdot(in_q, out_q));
            const int mt = tri_material[t];
            pre_mc[s * D + b - 1] = make_int2(mt | (is_pec[mt] ? MAT_PEC : 0), __float_as_int(cos_i));
            if (b < j) {
                out_p = e_perp;
                out_q = fcross(e_perp, k[b + 1]);
            }
        }
        DfPre P;
        P.ell = ell;
        P.pad = 0.0;
        P.kin = make_float4(k[j].x, k[j].y, k[j].z, 0.0f);
        P.n = make_float4(n.x, n.y, n.z, 0.0f);
        P.ep = make_float4(e_perp.x, e_perp.y, e_perp.z, 0.0f);
        P.d0 = make_float4(k[1].x, k[1].y, k[1].z, 0.0f);
        pre[s] = P;
    }
}

// One thread per diffuse path: the shared part from its (ray, bounce) prefix, the
// last segment (diffuse point -> receiver) in FP64, the scattered basis in FP32.
// Blocks of DF_REC_THREADS take tiles of as many consecutive paths; the FP64 points
// of a tile (one row of (D + 2) x 3 per path) are staged in shared memory and
// written out as one contiguous, coalesced range.
constexpr int DF_REC_THREADS = 128;
__global__ void __launch_bounds__(DF_REC_THREADS) k_df_records(int64_t P, int64_t N, int D, double tx0, double tx1,
                                                               double tx2, const double* __restrict__ rx,
                                                               const int32_t* __restrict__ prx,
                                                               const int64_t* __restrict__ src,
                                                               const int32_t* __restrict__ hit_tri,
                                                               const double* __restrict__ hit_pt,
                                                               const DfPre* __restrict__ pre,
                                                               const float4* __restrict__ pre_Dm,
                                                               const int2* __restrict__ pre_mc, RecOut O) {
    constexpr double INV_C0 = 1.0 / RT_C0;
    __shared__ __align__(16) double sp[DF_REC_THREADS * (RT_MAX_DEPTH + 2) * 3];
    const int row = (D + 2) * 3;
    double* po = sp + threadIdx.x * row;
    for (int64_t i0 = (int64_t)blockIdx.x * DF_REC_THREADS; i0 < P; i0 += (int64_t)gridDim.x * DF_REC_THREADS) {
        const int64_t i = i0 + threadIdx.x;
        if (i < P) {
            const int s32 = (int)src[i];   // < n_rays max_depth < 2^31
            const int ray = s32 / D;
            const int j = s32 - ray * D + 1;
            const int64_t s = s32;
            const int r = prx[i];
            const DfPre Q = pre[s];
            po[0] = tx0;
            po[1] = tx1;
            po[2] = tx2;
            D3 last = d3(0.0, 0.0, 0.0);
            for (int b = 1; b <= j; ++b) {
                const double* q = hit_pt + ((int64_t)(b - 1) * N + ray) * 3;
                last = d3(q[0], q[1], q[2]);
                po[3 * b] = last.x;
                po[3 * b + 1] = last.y;
                po[3 * b + 2] = last.z;
            }
            const D3 pr = d3(rx[3 * (int64_t)r], rx[3 * (int64_t)r + 1], rx[3 * (int64_t)r + 2]);
            po[3 * (j + 1)] = pr.x;
            po[3 * (j + 1) + 1] = pr.y;
            po[3 * (j + 1) + 2] = pr.z;
            for (int c = 3 * (j + 2); c < row; ++c) po[c] = 0.0;
            O.depth[i] = j;
            for (int b = 0; b < D; ++b) O.tri[(int64_t)b * P + i] = b < j ? hit_tri[(int64_t)b * N + ray] : -1;
            const D3 dv = sub(pr, last);
            const double dl = sqrt(dotd(dv, dv));
            const float inv = 1.0f / (float)dl;
            const F3 ks = f3((float)dv.x * inv, (float)dv.y * inv, (float)dv.z * inv);
            O.tau[i] = (Q.ell + dl) * INV_C0;
            O.len[i] = (float)dl;
            for (int b = 0; b < j; ++b) {
                O.Dm[(int64_t)b * P + i] = pre_Dm[s * D + b];
                O.mc[(int64_t)b * P + i] = pre_mc[s * D + b];
            }
            for (int b = j; b < D; ++b) O.mc[(int64_t)b * P + i] = make_int2(0, 0);
            // diffuse bounce: pattern cosines and the scattered basis
            const F3 kin = f3(Q.kin.x, Q.kin.y, Q.kin.z);
            const F3 n = f3(Q.n.x, Q.n.y, Q.n.z);
            const F3 kr = fsub(kin, fscl(2.0f * fdot(kin, n), n));
            O.scat[i] = make_float4(fdot(ks, n), -fdot(kin, ks), fdot(kr, ks), (float)(1.0 / dl));
            const F3 sp_ = perp_or_f(ks, n, f3(Q.ep.x, Q.ep.y, Q.ep.z));
            const F3 sq = fcross(sp_, ks);
            F3 th, ph;
            sph_basis_f(fscl(-1.0f, ks), &th, &ph);
            O.Dm[(int64_t)j * P + i] = make_float4(fdot(th, sp_), fdot(th, sq), fdot(ph, sp_), fdot(ph, sq));
            O.dir[i] = Q.d0;
            O.dir[P + i] = make_float4(-ks.x, -ks.y, -ks.z, 0.0f);
        }
        __syncthreads();
        // the tile's points: rows of consecutive paths are contiguous in O.pts too;
        // i0 row doubles start on a 16-byte boundary (i0 is a multiple of 128)
        const int cnt = (int)(P - i0 < DF_REC_THREADS ? P - i0 : DF_REC_THREADS) * row;
        double2* dst = reinterpret_cast<double2*>(O.pts + i0 * row);
        const double2* s2 = reinterpret_cast<const double2*>(sp);
        for (int k = threadIdx.x; k < cnt / 2; k += DF_REC_THREADS) dst[k] = s2[k];
        if ((cnt & 1) && threadIdx.x == 0) O.pts[i0 * row + cnt - 1] = sp[cnt - 1];
        __syncthreads();
    }
}

// ------------------------------------------------------------------ scattering pattern
// One lobe exp(lambda c) / a(lambda, cos theta_i) evaluated as
// exp(lambda (c - 1)) / (a e^-lambda) so that nothing overflows; a is the smooth
// step s(t, cos theta_i) between the hemispherical integrals with the axis on the
// normal (U) and opposite it (L).  The parts that depend on lambda alone (t(lambda),
// e^t - 1, U e^-lambda, L e^-lambda and their derivatives) are formed once per
// material (LobeK); a path then needs three exponentials per lobe.
struct LobeK {
    float lam, t, e2, Uh, Lh, dt, dUh, dLh;
};

__device__ __forceinline__ LobeK lobe_prep(float lam) {
    LobeK k;
    const float q = expf(-lam);
    const float em = -expm1f(-lam);                       // 1 - e^-lambda
    const float k2 = 2.0f * DF_PI / lam;
    const float nn = (1.6988f * lam + 10.8438f) * lam;
    const float dn = (lam + 6.2201f) * lam + 10.2415f;
    k.lam = lam;
    k.t = sqrtf(lam) * nn / dn;
    k.e2 = expm1f(k.t);
    k.Uh = k2 * em;                                        // U e^-lambda
    k.Lh = k.Uh * q;                                       // L e^-lambda
    k.dt = k.t * (0.5f / lam + (3.3976f * lam + 10.8438f) / nn - (2.0f * lam + 6.2201f) / dn);
    k.dUh = -k.Uh / lam + k2 * q;
    k.dLh = -k.Lh / lam + k2 * (2.0f * q * q - q);
    return k;
}

// g = exp(lambda c) / a(lambda, ci); with dlog != nullptr also d log g / d lambda.
__device__ __forceinline__ float lobe_eval(const LobeK& k, float c, float ci, float* dlog) {
    const float e1 = expm1f(k.t * (1.0f + ci));
    const float e3 = expf(k.t * ci);
    const float Dd = k.e2 * (e3 + 1.0f);
    const float s = e1 / Dd;
    const float ah = s * k.Uh + (1.0f - s) * k.Lh;
    const float g = expf(k.lam * (c - 1.0f)) / ah;
    if (dlog) {
        const float dN = (1.0f + ci) * (e1 + 1.0f);
        const float dD = (k.e2 + 1.0f) * (e3 + 1.0f) + k.e2 * ci * e3;
        const float ds = (dN - s * dD) / Dd;
        const float dah = s * k.dUh + (1.0f - s) * k.dLh + (k.Uh - k.Lh) * ds * k.dt;
        *dlog = (c - 1.0f) - dah / ah;
    }
    return g;
}

// f_s of Eq. trainable_scattering_pattern; pr = [S, K_x, w_1, w_2, w_3, lambda_2,
// lambda_3, -], k2 / k3 the lambda-only parts of its two lobes; with df != nullptr
// also df/dw_1, df/dw_2, df/dw_3, df/dlambda_2, df/dlambda_3.
__device__ __forceinline__ float pattern(const float* pr, const LobeK& k2, const LobeK& k3, float4 geo, float ci,
                                         float* df) {
    float dl2, dl3;
    const float g2 = lobe_eval(k2, geo.y, ci, df ? &dl2 : nullptr);
    const float g3 = lobe_eval(k3, geo.z, ci, df ? &dl3 : nullptr);
    if (df) {
        df[0] = geo.x * (1.0f / DF_PI);
        df[1] = g2;
        df[2] = g3;
        df[3] = pr[3] * g2 * dl2;
        df[4] = pr[4] * g3 * dl3;
    }
    return pr[2] * (1.0f / DF_PI) * geo.x + pr[3] * g2 + pr[4] * g3;
}

// Per-material lobe table in shared memory (materials < DF_LOBE_TAB), else per path.
constexpr int DF_LOBE_TAB = 64;

__device__ __forceinline__ void lobe_table(LobeK (*tab)[2], const float* scat, int n_mat) {
    if (n_mat <= DF_LOBE_TAB) {
        for (int k = threadIdx.x; k < 2 * n_mat; k += blockDim.x) tab[k >> 1][k & 1] = lobe_prep(__ldg(scat + 8 * (k >> 1) + 5 + (k & 1)));
    }
    __syncthreads();
}

__device__ __forceinline__ void lobes_of(LobeK (*tab)[2], const float* prm, int mat, int n_mat, LobeK& k2, LobeK& k3) {
    if (n_mat <= DF_LOBE_TAB) {
        k2 = tab[mat][0];
        k3 = tab[mat][1];
    } else {
        k2 = lobe_prep(prm[5]);
        k3 = lobe_prep(prm[6]);
    }
}

// ------------------------------------------------------------------ fields
struct DfArgs {
    int64_t P;
    const int32_t* depth;
    const int2* mc;
    const float4* Dm;
    const float4* geo;       // (k_s.n, -k_i.k_s, k_r.k_s, 1/d_last)
    const float* eps;
    const float* sig;
    const float* scat;       // M x 8
    const float2* chi;       // per-path random phases (chi_1, chi_2), or null
    int n_mat;
    float inv_eps0w;
    float amp;               // lambda / (4 pi) sqrt(g_T g_R) sqrt(4 pi / N)
};

__device__ __forceinline__ void mat_params(const DfArgs& A, int2 m, float2& eta, bool& pec, int& mat, float& c) {
    pec = (m.x & MAT_PEC) != 0;
    mat = m.x & ~MAT_PEC;
    c = __int_as_float(m.y);
    eta = make_float2(__ldg(A.eps + mat), -__ldg(A.sig + mat) * A.inv_eps0w);
}

__device__ __forceinline__ float r_spec(float S) { return sqrtf(fmaxf(0.0f, 1.0f - S * S)); }

// Receiver projection of the scattered polarisation [c1 e^{j chi_1}, c2 e^{j chi_2}]
// through row 0 of D_last (chi = 0 without per-path phases).
__device__ __forceinline__ float2 pol_of(float4 Dl, float c1, float c2, const float2* __restrict__ chi, int64_t i) {
    if (!chi) return make_float2(Dl.x * c1 + Dl.y * c2, 0.0f);
    const float2 ch = __ldg(chi + i);
    float s1, k1, s2, k2;
    sincosf(ch.x, &s1, &k1);
    sincosf(ch.y, &s2, &k2);
    return make_float2(Dl.x * c1 * k1 + Dl.y * c2 * k2, Dl.x * c1 * s1 + Dl.y * c2 * s2);
}

__global__ void __launch_bounds__(256, 4) k_df_fwd(DfArgs A, float2* __restrict__ a, const double* __restrict__ tau_in,
                                                double* __restrict__ tau_out) {
    __shared__ LobeK s_lk[DF_LOBE_TAB][2];
    lobe_table(s_lk, A.scat, A.n_mat);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.P; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = A.depth[i];
        // the path's records first (independent loads in flight together)
        float4 Ds[RT_MAX_DEPTH];
        int2 mcs[RT_MAX_DEPTH];
#pragma unroll
        for (int b = 0; b < RT_MAX_DEPTH; ++b) {
            if (b < j) {
                Ds[b] = __ldg(A.Dm + (int64_t)b * A.P + i);
                mcs[b] = __ldg(A.mc + (int64_t)b * A.P + i);
            }
        }
        const float4 geo = __ldg(A.geo + i);
        const float4 Dl = __ldg(A.Dm + (int64_t)j * A.P + i);
        float2 E0 = make_float2(1.0f, 0.0f), E1 = make_float2(0.0f, 0.0f);
        float2 u0 = E0, u1 = E1;
        int mat = 0;
        float ci = 1.0f;
#pragma unroll
        for (int b = 0; b < RT_MAX_DEPTH; ++b) {
            if (b >= j) break;
            const float4 D = Ds[b];
            const float2 v0 = cadd(cscale(D.x, E0), cscale(D.y, E1));
            const float2 v1 = cadd(cscale(D.z, E0), cscale(D.w, E1));
            float2 eta, rp, rl, d0, d1;
            bool pec;
            mat_params(A, mcs[b], eta, pec, mat, ci);
            if (pec) {
                rp = make_float2(-1.0f, 0.0f);
                rl = make_float2(1.0f, 0.0f);
            } else {
                fresnel<false>(eta, ci, rp, rl, d0, d1);
            }
            u0 = cmul(rp, v0);
            u1 = cmul(rl, v1);
            if (b + 1 < j) {
                const float R = r_spec(__ldg(A.scat + 8 * mat));
                E0 = cscale(R, u0);
                E1 = cscale(R, u1);
            }
        }
        const float nu = sqrtf(u0.x * u0.x + u0.y * u0.y + u1.x * u1.x + u1.y * u1.y);
        const float* pr = A.scat + 8 * mat;
        float prm[8];
        for (int c = 0; c < 8; ++c) prm[c] = __ldg(pr + c);
        LobeK k2, k3;
        lobes_of(s_lk, prm, mat, A.n_mat, k2, k3);
        const float f = pattern(prm, k2, k3, geo, ci, nullptr);
        const float Kx = prm[1];
        const float2 pol = pol_of(Dl, sqrtf(fmaxf(0.0f, 1.0f - Kx)), sqrtf(fmaxf(0.0f, Kx)), A.chi, i);
        const float K = A.amp * prm[0] * sqrtf(fmaxf(f, 0.0f)) * nu * geo.w;
        a[i] = make_float2(K * pol.x, K * pol.y);
        if (tau_out) tau_out[i] = tau_in[i];
    }
}

// Adjoint: every quantity is real-valued in a (chi = 0), so dL/dtheta =
// Re(g) da/dtheta.  The field magnitude nu = |u| depends on eta of every bounce:
// with the row vector l = conj(u)^T / nu walked backwards through the chain,
// dnu/d eta_b = R_b l . diag(dr_perp, dr_par) v_b (holomorphic in eta), so
// dnu/d eps_r = Re(.) and dnu/d sigma = Im(.) / (eps0 omega).
// Per-material sums: with COLS > 0 (at most MAXM <= 8 materials, blocks of COLS
// threads) every thread owns a column of 9 x MAXM shared-memory accumulators
// (no atomics in the path loop; one block reduction at the end); otherwise
// shared-memory atomics (MAXM > 0) or global atomics.
template <int MAXM, int COLS>
__global__ void __launch_bounds__(256) k_df_bwd(DfArgs A, const float2* __restrict__ ga, float* __restrict__ geps,
                                                float* __restrict__ gsig, float* __restrict__ gscat, int n_mat) {
    __shared__ float acc[COLS > 0 ? 9 * MAXM * COLS : (MAXM > 0 ? MAXM * 9 : 1)];
    __shared__ LobeK s_lk[DF_LOBE_TAB][2];
    lobe_table(s_lk, A.scat, A.n_mat);
    if (COLS > 0) {
        for (int k = 0; k < 9 * MAXM; ++k) acc[k * COLS + threadIdx.x] = 0.0f;
    } else if (MAXM > 0) {
        for (int k = threadIdx.x; k < n_mat * 9; k += blockDim.x) acc[k] = 0.0f;
        __syncthreads();
    }
    auto add = [&](int m, int c, float v) {
        if (v == 0.0f) return;
        if (COLS > 0) {
            acc[(c * MAXM + m) * COLS + threadIdx.x] += v;
        } else if (MAXM > 0) {
            atomicAdd(&acc[m * 9 + c], v);
        } else if (c == 0) {
            if (geps) atomicAdd(geps + m, v);
        } else if (c == 1) {
            if (gsig) atomicAdd(gsig + m, v);
        } else if (gscat) {
            atomicAdd(gscat + 8 * m + (c - 2), v);
        }
    };
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.P; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 gc = ga[i];
        if (gc.x == 0.0f && gc.y == 0.0f) continue;
        const int j = A.depth[i];
        float2 v0s[RT_MAX_DEPTH], v1s[RT_MAX_DEPTH], rps[RT_MAX_DEPTH], rls[RT_MAX_DEPTH];
        float4 Ds[RT_MAX_DEPTH];
        int2 mcs[RT_MAX_DEPTH];
        int mats[RT_MAX_DEPTH];
        bool pecs[RT_MAX_DEPTH];
        float cis[RT_MAX_DEPTH], Rs[RT_MAX_DEPTH];
        // every record of the path first (independent loads in flight together),
        // then the chain
#pragma unroll
        for (int b = 0; b < RT_MAX_DEPTH; ++b) {
            if (b < j) {
                Ds[b] = __ldg(A.Dm + (int64_t)b * A.P + i);
                mcs[b] = __ldg(A.mc + (int64_t)b * A.P + i);
            }
        }
        const float4 geo = __ldg(A.geo + i);
        const float4 Dl = __ldg(A.Dm + (int64_t)j * A.P + i);
        float2 E0 = make_float2(1.0f, 0.0f), E1 = make_float2(0.0f, 0.0f), u0 = E0, u1 = E1;
        int md = 0;
        float ci_d = 1.0f;
#pragma unroll
        for (int b = 0; b < RT_MAX_DEPTH; ++b) {
            if (b >= j) break;
            const float4 D = Ds[b];
            const float2 v0 = cadd(cscale(D.x, E0), cscale(D.y, E1));
            const float2 v1 = cadd(cscale(D.z, E0), cscale(D.w, E1));
            float2 eta, rp, rl, d0, d1;
            mat_params(A, mcs[b], eta, pecs[b], mats[b], cis[b]);
            if (pecs[b]) {
                rp = make_float2(-1.0f, 0.0f);
                rl = make_float2(1.0f, 0.0f);
            } else {
                fresnel<false>(eta, cis[b], rp, rl, d0, d1);
            }
            v0s[b] = v0;
            v1s[b] = v1;
            rps[b] = rp;
            rls[b] = rl;
            u0 = cmul(rp, v0);
            u1 = cmul(rl, v1);
            Rs[b] = b + 1 < j ? r_spec(__ldg(A.scat + 8 * mats[b])) : 1.0f;
            E0 = cscale(Rs[b], u0);
            E1 = cscale(Rs[b], u1);
            if (b == j - 1) {
                md = mats[b];
                ci_d = cis[b];
            }
        }
        float prm[8];
        for (int c = 0; c < 8; ++c) prm[c] = __ldg(A.scat + 8 * md + c);
        const float nu = sqrtf(u0.x * u0.x + u0.y * u0.y + u1.x * u1.x + u1.y * u1.y);
        float df[5];
        LobeK k2, k3;
        lobes_of(s_lk, prm, md, A.n_mat, k2, k3);
        const float f = pattern(prm, k2, k3, geo, ci_d, df);
        const float sf = sqrtf(fmaxf(f, 0.0f));
        const float Kx = fminf(fmaxf(prm[1], 1e-12f), 1.0f - 1e-7f);
        const float sq1 = sqrtf(1.0f - Kx), sq2 = sqrtf(Kx);
        // a = K pol with K real: dL/dtheta = dK/dtheta Re(conj(g) pol) for every
        // parameter but K_x, whose derivative goes through pol
        const float2 pol = pol_of(Dl, sq1, sq2, A.chi, i);
        const float2 dpol = pol_of(Dl, -0.5f / sq1, 0.5f / sq2, A.chi, i);
        const float gpol = gc.x * pol.x + gc.y * pol.y;
        const float gdpol = gc.x * dpol.x + gc.y * dpol.y;
        const float C = A.amp * geo.w;
        const float S = prm[0];
        // diffuse material: S, K_x, pattern
        add(md, 2, gpol * C * sf * nu);
        add(md, 3, gdpol * C * S * sf * nu);
        if (f > 0.0f) {
            const float dAdf = gpol * C * S * nu * 0.5f / sf;
            for (int c = 0; c < 5; ++c) add(md, 4 + c, dAdf * df[c]);
        }
        if (!(nu > 0.0f)) continue;
        // reverse walk for d nu / d eta_b and d nu / d R_b
        const float dAnu = gpol * C * S * sf / nu;
        float2 l0 = make_float2(u0.x * dAnu, -u0.y * dAnu), l1 = make_float2(u1.x * dAnu, -u1.y * dAnu);
#pragma unroll
        for (int b = RT_MAX_DEPTH - 1; b >= 0; --b) {
            if (b > j - 1) continue;
            const float R = Rs[b];
            if (!pecs[b]) {
                float2 eta, rp, rl, d0, d1;
                bool pec;
                int mt;
                float c;
                mat_params(A, mcs[b], eta, pec, mt, c);
                fresnel<true>(eta, c, rp, rl, d0, d1);
                const float2 w = cscale(R, cadd(cmul(l0, cmul(d0, v0s[b])), cmul(l1, cmul(d1, v1s[b]))));
                add(mats[b], 0, w.x);
                add(mats[b], 1, w.y * A.inv_eps0w);
            }
            if (b + 1 < j) {
                const float2 h = cadd(cmul(l0, cmul(rps[b], v0s[b])), cmul(l1, cmul(rls[b], v1s[b])));
                const float S_b = __ldg(A.scat + 8 * mats[b]);
                if (R > 0.0f) add(mats[b], 2, h.x * (-S_b / R));
            }
            const float2 m0 = cscale(R, cmul(l0, rps[b])), m1 = cscale(R, cmul(l1, rls[b]));
            const float4 D = Ds[b];
            l0 = cadd(cscale(D.x, m0), cscale(D.z, m1));
            l1 = cadd(cscale(D.y, m0), cscale(D.w, m1));
        }
    }
    if (COLS > 0) {
        __syncthreads();
        const int lane = threadIdx.x & 31;
        for (int k = threadIdx.x >> 5; k < 9 * MAXM; k += COLS / 32) {
            const int c = k / MAXM, m = k - c * MAXM;
            if (m >= n_mat) continue;
            float v = 0.0f;
            for (int t = lane; t < COLS; t += 32) v += acc[k * COLS + t];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane != 0 || v == 0.0f) continue;
            if (c == 0) {
                if (geps) atomicAdd(geps + m, v);
            } else if (c == 1) {
                if (gsig) atomicAdd(gsig + m, v);
            } else if (gscat) {
                atomicAdd(gscat + 8 * m + (c - 2), v);
            }
        }
    } else if (MAXM > 0) {
        __syncthreads();
        for (int k = threadIdx.x; k < n_mat * 9; k += blockDim.x) {
            const float v = acc[k];
            if (v == 0.0f) continue;
            const int m = k / 9, c = k - 9 * m;
            if (c == 0) {
                if (geps) atomicAdd(geps + m, v);
            } else if (c == 1) {
                if (gsig) atomicAdd(gsig + m, v);
            } else if (gscat) {
                atomicAdd(gscat + 8 * m + (c - 2), v);
            }
        }
    }
}

// ------------------------------------------------------------------ specular share
__global__ void k_spec_reduce(int64_t P, const int32_t* __restrict__ depth, const int2* __restrict__ mc,
                              const float* __restrict__ scat, const float2* __restrict__ a, float2* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const int q = depth[i];
        float fac = 1.0f;
        for (int b = 0; b < q; ++b) fac *= r_spec(__ldg(scat + 8 * (__ldg(mc + (int64_t)b * P + i).x & ~MAT_PEC)));
        const float2 v = a[i];
        out[i] = make_float2(fac * v.x, fac * v.y);
    }
}

template <int MAXM>
__global__ void __launch_bounds__(256) k_spec_reduce_bwd(int64_t P, const int32_t* __restrict__ depth,
                                                         const int2* __restrict__ mc, const float* __restrict__ scat,
                                                         const float2* __restrict__ a_out, const float2* __restrict__ g,
                                                         float2* __restrict__ ga, float* __restrict__ gscat, int n_mat) {
    __shared__ float acc[MAXM > 0 ? MAXM : 1];
    if (MAXM > 0) {
        for (int k = threadIdx.x; k < n_mat; k += blockDim.x) acc[k] = 0.0f;
        __syncthreads();
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const int q = depth[i];
        float fac = 1.0f;
        for (int b = 0; b < q; ++b) fac *= r_spec(__ldg(scat + 8 * (__ldg(mc + (int64_t)b * P + i).x & ~MAT_PEC)));
        const float2 gi = g[i];
        if (ga) ga[i] = make_float2(fac * gi.x, fac * gi.y);
        if (!gscat) continue;
        const float2 ao = a_out[i];
        const float h = gi.x * ao.x + gi.y * ao.y;   // Re(conj(g) a_out) = fac dL/dfac
        if (h == 0.0f) continue;
        for (int b = 0; b < q; ++b) {
            const int m = __ldg(mc + (int64_t)b * P + i).x & ~MAT_PEC;
            const float S = __ldg(scat + 8 * m);
            const float R2 = fmaxf(1.0f - S * S, 1e-30f);
            const float v = h * (-S / R2);
            if (MAXM > 0) atomicAdd(&acc[m], v);
            else atomicAdd(gscat + 8 * m, v);
        }
    }
    if (MAXM > 0 && gscat) {
        __syncthreads();
        for (int k = threadIdx.x; k < n_mat; k += blockDim.x)
            if (acc[k] != 0.0f) atomicAdd(gscat + 8 * k, acc[k]);
    }
}

// ------------------------------------------------------------------ per-receiver merge / split
// The merged list holds receiver r's elements of list 1 then its elements of
// list 2, starting at S(r) = off1[r] + off2[r].  One thread per merged element
// (lanes on consecutive elements, so loads and stores coalesce); a thread finds
// the receiver of its first element by bisection on S and walks forward from
// there for its later ones (a grid stride later).
__device__ __forceinline__ int rx_of(int64_t i, int R, const int64_t* __restrict__ off1,
                                     const int64_t* __restrict__ off2) {
    int lo = 0, hi = R;   // S(lo) <= i < S(hi)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(off1 + mid) + __ldg(off2 + mid) <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <bool MERGE>
__global__ void __launch_bounds__(256) k_rx_perm(int R, const int64_t* __restrict__ off1,
                                                 const int64_t* __restrict__ off2, const uint64_t* __restrict__ a,
                                                 const uint64_t* __restrict__ b, uint64_t* __restrict__ x,
                                                 uint64_t* __restrict__ ya, uint64_t* __restrict__ yb,
                                                 int64_t* __restrict__ off_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (MERGE && off_out)
        for (int64_t q = g; q <= R; q += stride) off_out[q] = __ldg(off1 + q) + __ldg(off2 + q);
    const int64_t total = __ldg(off1 + R) + __ldg(off2 + R);
    if (g >= total) return;
    int r = rx_of(g, R, off1, off2);
    for (int64_t i = g; i < total; i += stride) {
        while (r + 1 < R && __ldg(off1 + r + 1) + __ldg(off2 + r + 1) <= i) ++r;
        const int64_t a0 = __ldg(off1 + r), b0 = __ldg(off2 + r);
        const int64_t k = i - (a0 + b0), n1 = __ldg(off1 + r + 1) - a0;
        if (MERGE) {
            x[i] = k < n1 ? a[a0 + k] : b[b0 + (k - n1)];
        } else {
            const uint64_t v = a[i];
            if (k < n1) {
                if (ya) ya[a0 + k] = v;
            } else if (yb) {
                yb[b0 + (k - n1)] = v;
            }
        }
    }
}

DfArgs make_df_args(const rt_paths* p, const float* eps, const float* sig, const float* scat, double freq,
                    float gtx, float grx) {
    DfArgs A;
    A.P = p->P;
    A.depth = p->d_depth;
    A.mc = p->d_mc;
    A.Dm = p->d_Dm;
    A.geo = p->d_scat;
    A.eps = eps;
    A.sig = sig;
    A.scat = scat;
    A.chi = p->d_chi;
    A.n_mat = p->scene->n_materials;
    A.inv_eps0w = (float)(1.0 / (RT_EPS0 * 2.0 * RT_PI * freq));
    A.amp = (float)(RT_C0 / freq / (4.0 * RT_PI) * std::sqrt((double)gtx * (double)grx) *
                    std::sqrt(4.0 * RT_PI / (double)p->n_rays));
    return A;
}

rt_status check_diffuse(rt_ctx* ctx, const rt_paths* p, const float* eps, const float* sig, const float* scat,
                        double freq, float gtx, float grx) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!p || !eps || !sig || !scat) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    if (p->kind != 1) return rt_fail(ctx, RT_ERR_INVALID_ARG, "not a diffuse paths object (rt_trace_diffuse)");
    if (!(freq > 0.0) || !std::isfinite(freq)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "freq_hz must be > 0");
    if (!(gtx > 0.0f) || !(grx > 0.0f) || !std::isfinite(gtx) || !std::isfinite(grx))
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "antenna gains must be > 0");
    return RT_OK;
}

}  // namespace

#define RT_EXPORT extern "C" __attribute__((visibility("default")))

RT_EXPORT rt_status rt_trace_diffuse(rt_ctx* ctx, const rt_scene* scene, const double* tx_host, const double* rx_dev,
                                     int32_t n_rx, int64_t n_rays, int32_t max_depth, rt_paths** out) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!scene || !tx_host || !rx_dev || !out) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    if (scene->owns_tables_only) return rt_fail(ctx, RT_ERR_INVALID_ARG, "scene has no BVH (batch tables)");
    if (n_rays < 1 || n_rays * max_depth > 2147483647LL || max_depth < 1 || max_depth > RT_MAX_DEPTH || n_rx < 1 ||
        n_rx > (1 << 24))
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "bad sizes");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(tx_host[c])) return rt_fail(ctx, RT_ERR_NUMERIC, "transmitter not finite");
    const int64_t N = n_rays, D = max_depth, R = n_rx;
    const int64_t W = (N * D + 31) / 32;
    if (R * W > (int64_t)1 << 31)
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_rx x n_rays x max_depth too large for the visibility mask");
    *out = nullptr;
    cudaStream_t st = ctx->stream;
    int32_t* status = rt_status_ptr(ctx);
    // launch z table (one FP64 division and subtraction per ray, rounded to FP32)
    std::vector<float> zh(N);
    for (int64_t i = 0; i < N; ++i) zh[i] = (float)(1.0 - (double)(2 * i + 1) / (double)N);
    float* z = nullptr;
    int32_t* hit_tri = nullptr;
    double* hit_pt = nullptr;
    float4* hit_pt32 = nullptr;
    float4* rx32 = nullptr;
    uint32_t* mask = nullptr;
    int32_t* word_off = nullptr;
    int64_t* cnt = nullptr;
    int64_t* src = nullptr;
    DfPre* pre = nullptr;
    float4* pre_Dm = nullptr;
    int2* pre_mc = nullptr;
    rt_paths* p = nullptr;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** d, size_t b) {
        if (e == cudaSuccess) e = cudaMallocAsync(d, b, st);
    };
    auto cleanup = [&]() {
        void* tmp[] = {z, hit_tri, hit_pt, hit_pt32, rx32, mask, word_off, cnt, src, pre, pre_Dm, pre_mc};
        for (void* q : tmp)
            if (q) cudaFreeAsync(q, st);
    };
    A((void**)&z, N * 4);
    A((void**)&hit_tri, N * D * 4);
    A((void**)&hit_pt, N * D * 3 * 8);
    A((void**)&hit_pt32, N * D * 16);
    A((void**)&rx32, R * 16);
    A((void**)&mask, R * W * 4);
    A((void**)&word_off, R * W * 4);
    A((void**)&cnt, R * 8);
    if (e == cudaSuccess) e = cudaMemcpyAsync(z, zh.data(), N * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(mask, 0, R * W * 4, st);
    if (e != cudaSuccess) {
        cleanup();
        return rt_cuda_fail(ctx, e, "diffuse trace buffers");
    }
    const Scn S{scene->d_nodes, scene->d_bvh_tris, scene->d_tri_n64, scene->d_tri_bary, scene->eps, scene->d_tri_v};
    k_df_rays<<<grid_of(ctx, std::max<int64_t>(N, R), DF_THREADS, 16), DF_THREADS, 0, st>>>(
        N, (int)D, tx_host[0], tx_host[1], tx_host[2], z, S, hit_tri, hit_pt, hit_pt32, (int)R, rx_dev, rx32,
        status); RT_COUNT(ctx);
    k_df_nee<<<grid_of(ctx, N * D * R, DF_THREADS, 16), DF_THREADS, 0, st>>>(
        N, (int)D, (int)R, tx_host[0], tx_host[1], tx_host[2], rx_dev, rx32, hit_tri, hit_pt, hit_pt32, S, mask, W,
        status); RT_COUNT(ctx);
    k_df_row_scan<<<(int)R, 256, 0, st>>>(W, mask, word_off, cnt); RT_COUNT(ctx);
    p = new rt_paths();
    p->scene = scene;
    p->stream = st;
    p->D = (int)D;
    p->R = (int)R;
    p->kind = 1;
    p->n_rays = N;
    A((void**)&p->d_rx_offsets, (R + 1) * 8);
    if (e == cudaSuccess) {
        k_df_offsets<<<1, 1024, 0, st>>>((int)R, cnt, p->d_rx_offsets); RT_COUNT(ctx);
        e = cudaGetLastError();
    }
    int64_t P = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_pinned, p->d_rx_offsets + R, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) P = *ctx->h_pinned;
    p->P = P;
    const size_t Pa = P > 0 ? (size_t)P : 1;
    A((void**)&src, Pa * 8);
    A((void**)&p->d_rx, Pa * 4);
    A((void**)&p->d_depth, Pa * 4);
    A((void**)&p->d_tri, Pa * D * 4);
    A((void**)&p->d_pts, Pa * (D + 2) * 3 * 8);
    A((void**)&p->d_tau, Pa * 8);
    A((void**)&p->d_len, Pa * 4);
    A((void**)&p->d_mc, Pa * D * 8);
    A((void**)&p->d_Dm, Pa * (D + 1) * 16);
    A((void**)&p->d_dir, Pa * 2 * 16);
    A((void**)&p->d_scat, Pa * 16);
    if (P > 0) {
        A((void**)&pre, N * D * sizeof(DfPre));
        A((void**)&pre_Dm, N * D * D * 16);
        A((void**)&pre_mc, N * D * D * 8);
    }
    if (e == cudaSuccess && P > 0) {
        k_df_expand<<<grid_of(ctx, R * W, 256, 8), 256, 0, st>>>((int)R, W, mask, word_off, p->d_rx_offsets, p->d_rx,
                                                                  src); RT_COUNT(ctx);
        RecOut O{p->d_depth, p->d_tri, p->d_pts, p->d_tau, p->d_len, p->d_mc, p->d_Dm, p->d_dir, p->d_scat};
        k_df_prefix<<<grid_of(ctx, N * D, 128, 16), 128, 0, st>>>(N, (int)D, tx_host[0], tx_host[1], tx_host[2], hit_tri,
                                                                  hit_pt, scene->d_tri_n64, scene->d_tri_material,
                                                                  scene->d_is_pec, pre, pre_Dm, pre_mc); RT_COUNT(ctx);
        k_df_records<<<grid_of(ctx, P, DF_REC_THREADS, 12), DF_REC_THREADS, 0, st>>>(
            P, N, (int)D, tx_host[0], tx_host[1], tx_host[2], rx_dev, p->d_rx, src, hit_tri, hit_pt, pre, pre_Dm, pre_mc,
            O);
        RT_COUNT(ctx);
        e = cudaGetLastError();
    }
    cleanup();
    if (e != cudaSuccess) {
        rt_paths_free(p);
        return rt_cuda_fail(ctx, e, "diffuse trace");
    }
    *out = p;
    return RT_OK;
}

RT_EXPORT rt_status rt_eval_fields_diffuse(rt_ctx* ctx, const rt_paths* paths, const float* eps_r_dev,
                                           const float* sigma_dev, const float* scat_dev, double freq_hz,
                                           float gain_tx, float gain_rx, void* a_dev, double* tau_dev) {
    rt_status s = check_diffuse(ctx, paths, eps_r_dev, sigma_dev, scat_dev, freq_hz, gain_tx, gain_rx);
    if (s != RT_OK) return s;
    if (!a_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null a_dev");
    if (paths->P == 0) return RT_OK;
    const DfArgs A = make_df_args(paths, eps_r_dev, sigma_dev, scat_dev, freq_hz, gain_tx, gain_rx);
    k_df_fwd<<<grid_of(ctx, paths->P, 256, 8), 256, 0, ctx->stream>>>(A, (float2*)a_dev, paths->d_tau, tau_dev);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

RT_EXPORT rt_status rt_eval_fields_diffuse_backward(rt_ctx* ctx, const rt_paths* paths, const float* eps_r_dev,
                                                    const float* sigma_dev, const float* scat_dev, double freq_hz,
                                                    float gain_tx, float gain_rx, const void* grad_a_dev,
                                                    float* grad_eps_r_dev, float* grad_sigma_dev,
                                                    float* grad_scat_dev) {
    rt_status s = check_diffuse(ctx, paths, eps_r_dev, sigma_dev, scat_dev, freq_hz, gain_tx, gain_rx);
    if (s != RT_OK) return s;
    if (!grad_a_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null grad_a_dev");
    if (paths->P == 0) return RT_OK;
    const DfArgs A = make_df_args(paths, eps_r_dev, sigma_dev, scat_dev, freq_hz, gain_tx, gain_rx);
    const int n_mat = paths->scene->n_materials;
    const float2* ga = (const float2*)grad_a_dev;
    if (n_mat <= 8)
        k_df_bwd<8, 128><<<grid_of(ctx, paths->P, 128, 12), 128, 0, ctx->stream>>>(A, ga, grad_eps_r_dev,
                                                                                   grad_sigma_dev, grad_scat_dev,
                                                                                   n_mat);
    else if (n_mat <= 64)
        k_df_bwd<64, 0><<<grid_of(ctx, paths->P, 256, 8), 256, 0, ctx->stream>>>(A, ga, grad_eps_r_dev,
                                                                                 grad_sigma_dev, grad_scat_dev, n_mat);
    else
        k_df_bwd<0, 0><<<grid_of(ctx, paths->P, 256, 8), 256, 0, ctx->stream>>>(A, ga, grad_eps_r_dev,
                                                                                grad_sigma_dev, grad_scat_dev, n_mat);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

RT_EXPORT rt_status rt_set_diffuse_phases(rt_ctx* ctx, rt_paths* paths, const float* chi_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!paths) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null paths");
    if (paths->kind != 1) return rt_fail(ctx, RT_ERR_INVALID_ARG, "not a diffuse paths object (rt_trace_diffuse)");
    paths->d_chi = reinterpret_cast<const float2*>(chi_dev);
    return RT_OK;
}

RT_EXPORT rt_status rt_specular_reduction(rt_ctx* ctx, const rt_paths* paths, const float* scat_dev, const void* a_dev,
                                          void* a_out_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!paths || !scat_dev || !a_dev || !a_out_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    if (paths->kind != 0) return rt_fail(ctx, RT_ERR_INVALID_ARG, "not a specular paths object");
    RT_REQUIRE_RESOLVED(ctx, paths);
    if (paths->P == 0) return RT_OK;
    k_spec_reduce<<<grid_of(ctx, paths->P, 256, 8), 256, 0, ctx->stream>>>(
        paths->P, paths->d_depth, paths->d_mc, scat_dev, (const float2*)a_dev, (float2*)a_out_dev); RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

RT_EXPORT rt_status rt_specular_reduction_backward(rt_ctx* ctx, const rt_paths* paths, const float* scat_dev,
                                                   const void* a_out_dev, const void* grad_out_dev, void* grad_a_dev,
                                                   float* grad_scat_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!paths || !scat_dev || !grad_out_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    if (grad_scat_dev && !a_out_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "grad_scat_dev needs a_out_dev");
    if (paths->kind != 0) return rt_fail(ctx, RT_ERR_INVALID_ARG, "not a specular paths object");
    RT_REQUIRE_RESOLVED(ctx, paths);
    if (paths->P == 0) return RT_OK;
    const int n_mat = paths->scene->n_materials;
    const int grid = grid_of(ctx, paths->P, 256, 8);
    if (n_mat <= 1024)
        k_spec_reduce_bwd<1024><<<grid, 256, 0, ctx->stream>>>(paths->P, paths->d_depth, paths->d_mc, scat_dev,
                                                               (const float2*)a_out_dev, (const float2*)grad_out_dev,
                                                               (float2*)grad_a_dev, grad_scat_dev, n_mat);
    else
        k_spec_reduce_bwd<0><<<grid, 256, 0, ctx->stream>>>(paths->P, paths->d_depth, paths->d_mc, scat_dev,
                                                            (const float2*)a_out_dev, (const float2*)grad_out_dev,
                                                            (float2*)grad_a_dev, grad_scat_dev, n_mat);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

RT_EXPORT rt_status rt_rx_merge(rt_ctx* ctx, int32_t n_rx, const int64_t* off1_dev, const int64_t* off2_dev,
                                const void* src1_dev, const void* src2_dev, void* dst_dev, int64_t* off_out_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (n_rx < 1 || !off1_dev || !off2_dev || !src1_dev || !src2_dev || !dst_dev)
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument or n_rx < 1");
    k_rx_perm<true><<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(n_rx, off1_dev, off2_dev, (const uint64_t*)src1_dev,
                                                               (const uint64_t*)src2_dev, (uint64_t*)dst_dev, nullptr,
                                                               nullptr, off_out_dev); RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

RT_EXPORT rt_status rt_rx_split(rt_ctx* ctx, int32_t n_rx, const int64_t* off1_dev, const int64_t* off2_dev,
                                const void* src_dev, void* dst1_dev, void* dst2_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (n_rx < 1 || !off1_dev || !off2_dev || !src_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument or n_rx < 1");
    k_rx_perm<false><<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(n_rx, off1_dev, off2_dev, (const uint64_t*)src_dev,
                                                                nullptr, nullptr, (uint64_t*)dst1_dev,
                                                                (uint64_t*)dst2_dev, nullptr); RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}
