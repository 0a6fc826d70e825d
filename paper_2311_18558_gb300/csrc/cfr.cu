// Discrete CFR of arXiv 2311.18558, Sec. II-A:
//   H[r, c] = sum_{i in r} a_i exp(-j 2 pi (f_0 + c df) tau_i),  c = 0..N-1,
// with f_0 = f_c - (N/2) df (column c holds subcarrier n = c - N/2), and its
// adjoint g_a[i] = sum_c g_H[r, c] conj(exp(-j 2 pi (f_0 + c df) tau_i)).
//
// Split-Vandermonde evaluation: write c = N2 c1 + c2 (N2 | 256, N1 = N / N2).
// Then exp(-j 2 pi c df tau) = A_i[c1] B_i[c2] with
//   A_i[c1] = exp(-j 2 pi N2 c1 u_i),  B_i[c2] = exp(-j 2 pi c2 u_i),  u_i = df tau_i,
// so a receiver needs N1 + N2 phasors per path instead of N, and the CFR is the
// complex product (N1 x P) . (P x N2) of c_i A_i[c1] with B_i[c2].
//
// Phase accuracy: the only FP64 work per path is reducing f_0 tau_i and u_i to
// their fractional parts (in cycles).  u is split as u_hi + u_lo with u_hi a
// multiple of 2^-12, so m u_hi is exact in FP32 for every integer m < 4096 and
// frac(m u_hi) + m u_lo carries ~1e-7 cycles of error; sin/cos(pi x) of the
// doubled phase then gives each phasor to FP32 accuracy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "rt_internal.cuh"

// Loss partials and the two counters (completed CTAs, next receiver) of the
// fused and tensor-core kernels (api.cu); the counters are zero between launches.
rt_status rt_cfr_fused_scratch(rt_ctx* ctx, int R, double** part, unsigned int** done);
// Counters (8 ints) and heavy-slot tables (6 ints per slot) of the split fused
// kernel, zeroed when first allocated, and the slots' rows (api.cu).
rt_status rt_cfr_split_scratch(rt_ctx* ctx, int R, size_t acc_bytes, int** ints, void** acc, float** deconv,
                               int** deconv_n);

namespace {

constexpr int CFR_THREADS = 256;
constexpr int CH = 32;   // paths per shared-memory chunk

struct PathPhase {
    float p0;     // frac(f_0 tau) in cycles
    float uhi;    // multiple of 2^-12, |uhi| <= 1/2
    float ulo;
};

// frac(x tau) of two doubles as a signed fixed-point fraction in units of 2^-64
// (value in [-1/2, 1/2)), from the exact 106-bit product of the significands:
// x tau = m_x m_t 2^(e_x + e_t - 2150) with biased exponents e, so the fraction
// scaled by 2^64 is the product shifted right by s = 2086 - e_x - e_t (left if s
// is negative; bits above 2^64 are whole cycles and drop out).  Integer
// arithmetic only: the FP64 units of this GPU issue at a small fraction of the
// integer rate.  Zeros and subnormals give 0 (|x tau| < 2^-1000 for any delay).
__device__ __forceinline__ int64_t frac_mul(double x, double tau) {
    const uint64_t bx = (uint64_t)__double_as_longlong(x), bt = (uint64_t)__double_as_longlong(tau);
    const int ex = (int)((bx >> 52) & 0x7ff), et = (int)((bt >> 52) & 0x7ff);
    if (ex == 0 || et == 0) return 0;
    const uint64_t frac_bits = (1ull << 52) - 1;
    const uint64_t mx = (bx & frac_bits) | (1ull << 52), mt = (bt & frac_bits) | (1ull << 52);
    const uint64_t lo = mx * mt, hi = __umul64hi(mx, mt);
    const int s = 2086 - ex - et;
    uint64_t f = 0;
    if (s >= 128) f = 0;
    else if (s >= 64) f = hi >> (s - 64);
    else if (s > 0) f = (hi << (64 - s)) | (lo >> s);
    else if (s > -64) f = lo << (-s);
    if ((bx ^ bt) >> 63) f = 0ull - f;   // frac(-y) = -frac(y)
    return (int64_t)f;
}

// fixed-point fraction (units 2^-64) to float, to FP32 precision
__device__ __forceinline__ float frac_to_float(int64_t f) { return (float)(int)(f >> 32) * 0x1p-32f; }

__device__ __forceinline__ PathPhase path_phase(double tau, double f0, double df) {
    PathPhase p;
    p.p0 = frac_to_float(frac_mul(f0, tau));
    // u = frac(df tau) = hi + lo with hi the nearest multiple of 2^-12
    const int64_t u = frac_mul(df, tau);
    const int64_t hi = (int64_t)(((uint64_t)u + (1ull << 51)) & ~((1ull << 52) - 1));
    p.uhi = (float)(int)(hi >> 52) * 0x1p-12f;
    p.ulo = (float)(int)((u - hi) >> 20) * 0x1p-44f;
    return p;
}

// exp(-j 2 pi phase(m)), phase(m) = frac(m u_hi) + m u_lo (+ extra)
__device__ __forceinline__ float2 phasor(const PathPhase& p, int m) {
    float x = (float)m * p.uhi;
    x = x - rintf(x);
    x = x + (float)m * p.ulo;
    float s, c;
    sincospif(2.0f * x, &s, &c);
    return make_float2(c, -s);
}

// As phasor(), with the hardware sine and cosine (absolute error about 4e-7 for
// arguments in [-pi, pi]): the tensor-core tables, whose operands are split
// into TF32 pairs and accumulated in FP32, stay within FP32 accuracy of H.
__device__ __forceinline__ float2 phasor_fast(const PathPhase& p, int m) {
    float x = (float)m * p.uhi;
    x = x - rintf(x);
    x = x + (float)m * p.ulo;
    float s, c;
    __sincosf(6.28318530717958647692f * x, &s, &c);
    return make_float2(c, -s);
}

__device__ __forceinline__ float2 base_phasor(const PathPhase& p) {
    float s, c;
    sincospif(2.0f * p.p0, &s, &c);
    return make_float2(c, -s);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

struct CfrShape {
    int N, N1, N2;
    double f0, df;
};

// Shared-memory tables of one chunk of n <= CH paths of a receiver:
//   sP[ii]            phase parameters of path ii
//   sA[ii N1 + c1]    A_i[c1]  = exp(-j 2 pi N2 c1 u_i)
//   sB[ii N2 + c2]    B_i[c2]  = exp(-j 2 pi c2 u_i)
//   sAc[ii N1 + c1]   c_i A_i[c1] with c_i = a_i exp(-j 2 pi f_0 tau_i)   (forward only)
struct Tables {
    PathPhase* sP;
    float2* sC;    // c_i = a_i exp(-j 2 pi f_0 tau_i) per path
    float2* sA;
    float2* sB;
    float2* sAc;   // reused as the partial sums of the adjoint
    float2* sF;    // factor phasors: per path A_lo[8], A_hi[NAH], B_lo[4], B_hi[4]
};

constexpr int NAL = 8, NBL = 4;   // low factors of c1 and c2

__device__ __forceinline__ int nah(const CfrShape& S) { return (S.N1 + NAL - 1) / NAL; }
__device__ __forceinline__ int nfac(const CfrShape& S) { return NAL + nah(S) + 2 * NBL; }

__device__ __forceinline__ Tables carve(const CfrShape& S, float4* smem4) {
    Tables T;
    T.sAc = reinterpret_cast<float2*>(smem4);
    T.sA = T.sAc + CH * S.N1;
    T.sB = T.sA + CH * S.N1;
    T.sF = T.sB + CH * S.N2;
    T.sC = T.sF + CH * nfac(S);
    T.sP = reinterpret_cast<PathPhase*>(T.sC + CH);
    return T;
}

__device__ __forceinline__ float2* carve_g(const CfrShape& S, float4* smem4) {   // N values after the tables
    Tables T = carve(S, smem4);
    return reinterpret_cast<float2*>(T.sP + CH + (CH & 1));
}

// Phasor tables of a chunk.  Each table entry is the product of two directly
// evaluated phasors: A_i[c1] = A_hi[c1 / 8] A_lo[c1 % 8] and
// B_i[c2] = B_hi[c2 / 4] B_lo[c2 % 4], which needs 8 + N1/8 + 8 sin/cos pairs per
// path instead of N1 + N2 (each factor carries ~1e-7 relative error).
__device__ __forceinline__ void build_tables(const CfrShape& S, int64_t base, int n, const float2* __restrict__ a,
                                             const double* __restrict__ tau, const Tables& T) {
    const int t = threadIdx.x;
    const int NAH = nah(S), NF = nfac(S);
    __syncthreads();
    if (t < n) {
        PathPhase p = path_phase(tau[base + t], S.f0, S.df);
        T.sP[t] = p;
        if (a) T.sC[t] = cmul(a[base + t], base_phasor(p));
    }
    __syncthreads();
    for (int e = t; e < n * NF; e += CFR_THREADS) {
        int ii = e / NF, k = e - ii * NF;
        int m;
        if (k < NAL) m = k * S.N2;                                    // A_lo: c1 = k
        else if (k < NAL + NAH) m = (k - NAL) * NAL * S.N2;           // A_hi: c1 = 8 (k - 8)
        else if (k < NAL + NAH + NBL) m = k - NAL - NAH;              // B_lo: c2 = k'
        else m = (k - NAL - NAH - NBL) * NBL;                         // B_hi: c2 = 4 k'
        T.sF[e] = phasor(T.sP[ii], m);
    }
    __syncthreads();
    for (int e = t; e < n * S.N2; e += CFR_THREADS) {
        int ii = e / S.N2, k = e - ii * S.N2;
        const float2* F = T.sF + ii * NF + NAL + NAH;
        T.sB[e] = cmul(F[NBL + k / NBL], F[k % NBL]);
    }
    for (int e = t; e < n * S.N1; e += CFR_THREADS) {
        int ii = e / S.N1, k = e - ii * S.N1;
        const float2* F = T.sF + ii * NF;
        float2 A = cmul(F[NAL + k / NAL], F[k % NAL]);
        T.sA[e] = A;
        if (a) T.sAc[e] = cmul(T.sC[ii], A);
    }
    __syncthreads();
}

// Forward CFR of one receiver into registers acc[OPT]: thread t owns columns
// c = t + 256 m (m < OPT); with N2 | 256 all of them share c2 = t % N2.
// Returns the number of chunks (the tables of the last chunk stay in place).
template <int OPT>
__device__ __forceinline__ int cfr_rx_forward(const CfrShape& S, int64_t i0, int64_t i1, const float2* __restrict__ a,
                                              const double* __restrict__ tau, const Tables& T, float2 (&acc)[OPT]) {
    const int t = threadIdx.x;
#pragma unroll
    for (int m = 0; m < OPT; ++m) acc[m] = make_float2(0.0f, 0.0f);
    const int c2 = t % S.N2;
    int c1[OPT];   // row of each owned column, computed once (no division in the loop)
#pragma unroll
    for (int m = 0; m < OPT; ++m) {
        int c = t + CFR_THREADS * m;
        c1[m] = c < S.N ? c / S.N2 : -1;
    }
    int chunks = 0;
    for (int64_t base = i0; base < i1; base += CH) {
        const int n = (int)min((int64_t)CH, i1 - base);
        build_tables(S, base, n, a, tau, T);
        chunks++;
        for (int ii = 0; ii < n; ++ii) {
            const float2 b = T.sB[ii * S.N2 + c2];
            const float2* row = T.sAc + ii * S.N1;
#pragma unroll
            for (int m = 0; m < OPT; ++m)
                if (c1[m] >= 0) cfma(acc[m], row[c1[m]], b);
        }
    }
    return chunks;
}

// Adjoint for one receiver given g_H in shared memory, stored transposed as
// sGt[c2 N1 + c1] (conflict-free for lanes with consecutive c1):
//   g_c[i] = sum_c1 conj(A_i[c1]) sum_c2 g[c1, c2] conj(B_i[c2]),  g_a[i] = conj(phi_i) g_c[i].
// The (path, c1) pairs of a chunk are spread over all threads (partial sums in
// shared memory), then one warp per path reduces its N1 partials with shuffles,
// so a receiver with few paths still keeps the whole CTA busy.  `reuse` = the
// tables of the only chunk are already in place.
__device__ __forceinline__ void cfr_rx_backward(const CfrShape& S, int64_t i0, int64_t i1,
                                                const double* __restrict__ tau, const float2* sGt, const Tables& T,
                                                bool reuse, float2* __restrict__ grad_a) {
    float2* part = T.sAc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t base = i0; base < i1; base += CH) {
        const int n = (int)min((int64_t)CH, i1 - base);
        if (!reuse) build_tables(S, base, n, nullptr, tau, T);
        __syncthreads();
        for (int e = threadIdx.x; e < n * S.N1; e += CFR_THREADS) {
            int ii = e / S.N1, c1 = e - ii * S.N1;
            const float2* B = T.sB + ii * S.N2;
            float2 inner = make_float2(0.0f, 0.0f);
            for (int k = 0; k < S.N2; ++k) {
                float2 gk = sGt[k * S.N1 + c1], bk = B[k];
                // inner += g * conj(B)
                inner.x = fmaf(gk.x, bk.x, fmaf(gk.y, bk.y, inner.x));
                inner.y = fmaf(gk.y, bk.x, fmaf(-gk.x, bk.y, inner.y));
            }
            part[e] = cmulc(inner, T.sA[e]);
        }
        __syncthreads();
        for (int ii = warp; ii < n; ii += CFR_THREADS / 32) {
            float2 acc = make_float2(0.0f, 0.0f);
            for (int c1 = lane; c1 < S.N1; c1 += 32) {
                float2 v = part[ii * S.N1 + c1];
                acc.x += v.x;
                acc.y += v.y;
            }
            for (int o = 16; o > 0; o >>= 1) {
                acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
            }
            if (lane == 0) grad_a[base + ii] = cmulc(acc, base_phasor(T.sP[ii]));
        }
        reuse = false;
    }
}

template <int OPT>
__global__ void __launch_bounds__(CFR_THREADS) k_cfr_fwd(CfrShape S, const int64_t* __restrict__ offs,
                                                         const float2* __restrict__ a, const double* __restrict__ tau,
                                                         float2* __restrict__ H) {
    extern __shared__ float4 smem4[];
    Tables T = carve(S, smem4);
    const int r = blockIdx.x;
    float2 acc[OPT];
    cfr_rx_forward<OPT>(S, offs[r], offs[r + 1], a, tau, T, acc);
#pragma unroll
    for (int m = 0; m < OPT; ++m) {
        int c = threadIdx.x + CFR_THREADS * m;
        if (c < S.N) H[(int64_t)r * S.N + c] = acc[m];
    }
}

__global__ void __launch_bounds__(CFR_THREADS) k_cfr_bwd(CfrShape S, const int64_t* __restrict__ offs,
                                                         const double* __restrict__ tau, const float2* __restrict__ gH,
                                                         float2* __restrict__ ga) {
    extern __shared__ float4 smem4[];
    Tables T = carve(S, smem4);
    float2* sG = carve_g(S, smem4);
    const int r = blockIdx.x;
    for (int c = threadIdx.x; c < S.N; c += CFR_THREADS) {
        int c1 = c / S.N2, c2 = c - c1 * S.N2;
        sG[c2 * S.N1 + c1] = gH[(int64_t)r * S.N + c];
    }
    cfr_rx_backward(S, offs[r], offs[r + 1], tau, sG, T, false, ga);
}

// Fused forward + power-MSE loss + adjoint for one receiver per CTA.  The loss
// partial of each receiver goes to part[r]; the last CTA to finish (counter)
// sums them in receiver order, so the loss is deterministic.
template <int OPT>
__global__ void __launch_bounds__(CFR_THREADS) k_cfr_fused(CfrShape S, const int64_t* __restrict__ offs, int R,
                                                           const float2* __restrict__ a, const double* __restrict__ tau,
                                                           const float* __restrict__ target, const float* __restrict__ w,
                                                           float* __restrict__ loss, float2* __restrict__ ga,
                                                           float2* __restrict__ H, double* __restrict__ part,
                                                           unsigned int* __restrict__ done) {
    extern __shared__ float4 smem4[];
    Tables T = carve(S, smem4);
    float2* sG = carve_g(S, smem4);
    __shared__ double red[CFR_THREADS / 32];
    __shared__ bool last;
    const int r = blockIdx.x;
    const int64_t i0 = offs[r], i1 = offs[r + 1];
    float2 acc[OPT];
    const int chunks = cfr_rx_forward<OPT>(S, i0, i1, a, tau, T, acc);
    const float wr = w[r];
    const float inv_rn = 1.0f / ((float)R * (float)S.N);
    double lsum = 0.0;
#pragma unroll
    for (int m = 0; m < OPT; ++m) {
        int c = threadIdx.x + CFR_THREADS * m;
        if (c < S.N) {
            float2 h = acc[m];
            if (H) H[(int64_t)r * S.N + c] = h;
            float e = h.x * h.x + h.y * h.y - target[(int64_t)r * S.N + c];
            float we = wr * e;
            lsum += (double)(we * we);
            float s = 4.0f * wr * wr * e * inv_rn;   // dL/dH = 4 w^2 (|H|^2 - P*) H / (R N)
            int c1 = c / S.N2, c2 = c - c1 * S.N2;
            sG[c2 * S.N1 + c1] = make_float2(s * h.x, s * h.y);   // transposed for the adjoint
        }
    }
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < CFR_THREADS / 32; ++k) s += red[k];
        part[r] = s;
        __threadfence();
        unsigned int prev = atomicAdd(done, 1u);
        last = (prev == (unsigned)R - 1);
    }
    cfr_rx_backward(S, i0, i1, tau, sG, T, chunks == 1, ga);
    __syncthreads();
    if (last) {
        __threadfence();
        double s = 0.0;
        for (int k = threadIdx.x; k < R; k += CFR_THREADS) s += ((volatile double*)part)[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int k = 0; k < CFR_THREADS / 32; ++k) tot += red[k];
            *loss = (float)(tot * (double)inv_rn);
            *done = 0u;   // ready for the next launch
        }
    }
}

// ===========================================================================
// Tensor-core path (tcgen05, kind::tf32, 3xTF32) for n_sub = 128 N2, N2 in
// {2, 4, 8, 16, 32}.  Split c = N2 c1 + c2 with N1 = 128 rows c1 (the MMA M),
// and carry the complex product in real form:
//   forward   D[c1][c2'] = sum_k A'[c1][k] B'[k][c2'],  D = [Re H | Im H]
//             A' = [Re Ac | Im Ac]  (128 x 2CP, Ac[c1][i] = c_i A_i[c1])
//             B' = [[Re B, Im B], [-Im B, Re B]]  (2CP x 2N2)
//   adjoint   Y[c1][i] = sum_c2 g[c1][c2] conj(B_i[c2]) as
//             Y' = [Re Y | Im Y] = G' Bc',  G' = [Re g | Im g]  (128 x 2N2),
//             Bc' = [[Re B^T, -Im B^T], [Im B^T, Re B^T]]  (2N2 x 2CP)
//             then g_c[i] = sum_c1 conj(A_i[c1]) Y[c1][i] (per thread, then a
//             transposed warp reduction over c1).
// Every FP32 operand x is split as hi = tf32(x), lo = tf32(x - hi) and each
// product accumulates hi.hi + hi.lo + lo.hi in FP32 (TMEM), which keeps FP32
// accuracy.  One CTA of 128 threads: thread m owns row c1 = m, i.e. TMEM lane m,
// so the loss epilogue and the adjoint reduction need no exchange of H.
// Operands live in shared memory in the no-swizzle K-major layout: 8-row x
// 16-byte core matrices, core (row block rb, k block kb) at rb * SBO + kb * 128.
// CTAs are persistent and take receivers from a counter.

constexpr int TC_THREADS = 128;
constexpr int TC_CP = 16;                 // paths per chunk (at most 32: one per lane in the adjoint reduction)
constexpr int TC_WAIT_LIMIT = 1 << 22;    // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte offset
// >> 4 (16-29), stride byte offset >> 4 (32-45), the fixed 0b001 at 46-48, no
// base offset, relative LBO, no swizzle (61-63 = 0).
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32
// (7-9 = 2, 10-12 = 2), both K-major, N >> 3 at 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Waits for the phase with the given parity to complete; false after
// TC_WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (int it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Stores 4 consecutive K elements (one core-matrix row) of row `row`, k block
// `kb`, split into hi and lo tiles.
__device__ __forceinline__ void put4(float* hi, float* lo, uint32_t sbo_floats, int row, int kb, float x0, float x1,
                                     float x2, float x3) {
    const int off = (row >> 3) * (int)sbo_floats + kb * 32 + (row & 7) * 4;
    const float h0 = tf32_rna(x0), h1 = tf32_rna(x1), h2 = tf32_rna(x2), h3 = tf32_rna(x3);
    *reinterpret_cast<float4*>(hi + off) = make_float4(h0, h1, h2, h3);
    *reinterpret_cast<float4*>(lo + off) =
        make_float4(tf32_rna(x0 - h0), tf32_rna(x1 - h1), tf32_rna(x2 - h2), tf32_rna(x3 - h3));
}

template <int N2>
struct TcDims {
    static constexpr int NB = 2 * N2 < 16 ? 16 : 2 * N2;   // forward MMA N (padded)
    static constexpr int KG = 2 * N2 < 8 ? 8 : 2 * N2;     // adjoint MMA K (padded)
    static constexpr int KA = 2 * TC_CP;                   // forward MMA K
    static constexpr int A_FLOATS = 128 * (KA > KG ? KA : KG);
    static constexpr int B_FLOATS = (NB * KA > 2 * TC_CP * KG) ? NB * KA : 2 * TC_CP * KG;
    static constexpr int NAH = 16, NAL = 8;                // A_i[c1] = Ah[c1 / 8] Al[c1 % 8]
    static constexpr int NF = NAH + NAL + N2;              // factor phasors per path
    // TMEM: the forward D at column 0 (NB columns), the adjoint's Y' (2 TC_CP
    // columns) from column Y_COL (32-column aligned); the allocation is the next
    // power of two, so that up to 512 / TMEM_COLS CTAs share an SM's TMEM
    static constexpr uint32_t Y_COL = NB < 32 ? 32 : NB;
    static constexpr uint32_t TMEM_COLS = Y_COL + 2 * TC_CP <= 64 ? 64 : 128;
};

// c_i A_i at c1 = 8k, per path (forward operand factors)
constexpr int TC_NFC = 16;

// Phasor tables of one chunk of TC_CP paths (two sets, so that the next chunk's
// tables are built while the current chunk's MMAs run).
struct TcTab {
    float2* tF;      // TC_CP x NF factor phasors
    float2* tFc;     // TC_CP x TC_NFC: c_i A_i at c1 = 8k (forward only)
    float2* tC;      // TC_CP: c_i = a_i exp(-j 2 pi f_0 tau_i) (forward only)
    PathPhase* tP;   // TC_CP phase data
};

template <int N2>
__host__ __device__ constexpr size_t tc_tab_bytes() {
    return (size_t)TC_CP * (TcDims<N2>::NF + TC_NFC) * 8 + (size_t)TC_CP * 8 + (size_t)TC_CP * sizeof(PathPhase);
}

// Phase data and c_i of a whole receiver, formed once when it has at most this
// many paths (one load latency per receiver instead of one per chunk).
constexpr int TC_PH_CAP = 128;

// Dynamic shared memory of the tensor-core kernel: A and B operand tiles (hi,
// lo), two sets of phasor tables, a reduction buffer and the receiver's phases.
template <int N2>
__host__ __device__ constexpr size_t tc_smem_bytes() {
    using T = TcDims<N2>;
    return (size_t)(2 * T::A_FLOATS + 2 * T::B_FLOATS) * 4 + 2 * tc_tab_bytes<N2>() + 4 * 32 * 8 +
           (size_t)TC_PH_CAP * (sizeof(PathPhase) + 8) + 64;
}

template <int N2>
__device__ __forceinline__ TcTab tc_tab(char* base) {
    TcTab t;
    t.tF = reinterpret_cast<float2*>(base);
    t.tFc = t.tF + TC_CP * TcDims<N2>::NF;
    t.tC = t.tFc + TC_CP * TC_NFC;
    t.tP = reinterpret_cast<PathPhase*>(t.tC + TC_CP);
    return t;
}

// Tables of chunk ch of a receiver's paths [i0, i0 + P): the chunk's paths
// [base, base + n), padded with zero phases (phasor 1, c = 0) up to n_pad (n
// itself for a direct receiver, else the next multiple of 8):
//   tP[ii], tC[ii] = a_i exp(-j 2 pi f_0 tau_i) (if a), tF[ii][0..16) = A_i at
//   c1 = 8k, tF[ii][16..24) = A_i at c1 = k, tF[ii][24..24+N2) = B_i[c2].
// With cP (the receiver's phases and c_i, formed at its start) the chunk's phase
// data come from there; else they are loaded and formed here.  The caller
// guarantees that no thread still reads tb; ends with a barrier.
template <int N2>
__device__ __forceinline__ void tc_tables(const CfrShape& S, int64_t i0, int P, int ch, bool direct,
                                          const float2* __restrict__ a, const double* __restrict__ tau,
                                          const TcTab& tb, const PathPhase* cP, const float2* cC) {
    using T = TcDims<N2>;
    const int t = threadIdx.x;
    const int64_t base = i0 + (int64_t)ch * TC_CP;
    const int n = min(TC_CP, P - ch * TC_CP);
    const int n_pad = direct ? n : (n + 7) & ~7;
    const PathPhase* srcP = tb.tP;
    const float2* srcC = tb.tC;
    if (cP) {
        srcP = cP + ch * TC_CP;
        srcC = cC + ch * TC_CP;
        if (t < n_pad) {
            tb.tP[t] = t < n ? srcP[t] : PathPhase{0.0f, 0.0f, 0.0f};
            tb.tC[t] = t < n && a ? srcC[t] : make_float2(0.0f, 0.0f);
        }
    } else {
        if (t < n_pad) {
            if (t < n) {
                PathPhase p = path_phase(tau[base + t], S.f0, S.df);
                tb.tP[t] = p;
                tb.tC[t] = a ? cmul(a[base + t], base_phasor(p)) : make_float2(0.0f, 0.0f);
            } else {
                tb.tP[t] = PathPhase{0.0f, 0.0f, 0.0f};
                tb.tC[t] = make_float2(0.0f, 0.0f);
            }
        }
        __syncthreads();
    }
    for (int e = t; e < n_pad * T::NF; e += TC_THREADS) {
        const int ii = e / T::NF, k = e - ii * T::NF;
        const int m = k < T::NAH ? k * T::NAL * N2 : k < T::NAH + T::NAL ? (k - T::NAH) * N2 : k - T::NAH - T::NAL;
        const PathPhase pp = ii < n ? srcP[ii] : PathPhase{0.0f, 0.0f, 0.0f};
        const float2 f = phasor_fast(pp, m);
        tb.tF[e] = f;
        if (a && k < T::NAH) tb.tFc[ii * TC_NFC + k] = ii < n ? cmul(srcC[ii], f) : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
}

__device__ __forceinline__ float2 tc_A(const float2* tF, int nf, int ii, int m) {   // A_i[c1 = m]
    return cmul(tF[ii * nf + (m >> 3)], tF[ii * nf + 16 + (m & 7)]);
}

// Receivers with many paths are split over CTAs (mode 3, the fused loss).  CTAs
// take receivers from a counter; a receiver of at most TC_SPLIT paths is
// processed whole, as in mode 2.  A receiver with more paths (the first
// TC_HEAVY_CAP of them met in a call; later ones stay whole) is deferred: the
// CTA that meets it clears its row of `acc` and its counters, then publishes it
// (pub = epoch + 1).  Every receiver counts as classified as soon as it is taken
// (a deferred one once published).  CTAs that find no receiver left work through
// the heavy list in segments of TC_SEG paths: they claim forward segments
// (per-receiver counter, cursor over the list); a forward segment adds its
// partial H to the row with float atomics (so H of a split receiver is summed in
// no fixed order); the CTA that finishes a receiver's last forward segment turns
// the row into dL/dH, writes the receiver's loss partial and raises `ready`.
// When every receiver is classified and every forward segment claimed, CTAs
// claim adjoint segments the same way and wait for `ready`.  Each wait (for
// classification, publication or `ready`) depends only on work that a running
// CTA took before, so it ends; all are bounded.  The last CTA sums the loss over
// all receivers in receiver order and advances the epoch.
constexpr int TC_SPLIT = 4096;
constexpr int TC_SEG = 1024;
constexpr int TC_HEAVY_CAP = 4096;

struct TcSplit {
    unsigned int* cnt = nullptr;       // [0] heavy receivers met, [1] forward cursor, [2] adjoint cursor,
                                       // [3] receivers classified, [4] call epoch (never reset)
    unsigned int* pub = nullptr;       // TC_HEAVY_CAP: epoch + 1 once the slot is published
    int* list = nullptr;               // TC_HEAVY_CAP: receiver of heavy slot h
    unsigned int* seg_next = nullptr;  // TC_HEAVY_CAP: next forward segment to claim
    unsigned int* adj_next = nullptr;  // TC_HEAVY_CAP: next adjoint segment to claim
    unsigned int* fwd_done = nullptr;  // TC_HEAVY_CAP: finished forward segments
    unsigned int* ready = nullptr;     // TC_HEAVY_CAP: dL/dH of the receiver is in acc
    float2* acc = nullptr;             // TC_HEAVY_CAP x 2N: oversampled grid of each heavy receiver
    const float* dec = nullptr;        // N: 1 / (M phi_hat(n)) per column (see below)
    int wait_limit = 1 << 22;          // polls of a wait on another CTA (rt_set_wait_limit)
};

// Heavy receivers use a non-uniform FFT instead of the dense product (the
// method of Barnett, Magland and af Klinteberg, "A parallel non-uniform fast
// Fourier transform library based on an exponential of semicircle kernel",
// SIAM J. Sci. Comput. 2019, written here from its mathematics):
//   H[c] = sum_i c'_i exp(-j 2 pi n x_i),  n = c - N/2,  c'_i = a_i exp(-j 2 pi f_c tau_i),
//   x_i = frac(df tau_i).
// Spreading: b[l] = sum_i c'_i phi((l - M x_i) 2 / W), l mod M, on a grid of
// M = 2N cells with phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1 (W cells
// wide); then B = FFT_-(b) and H[c] = B[n mod M] / (M phi_hat(n)) with
// M phi_hat(n) = W/2 int_{-1}^{1} phi(z) cos(pi n W z / M) dz (host quadrature).
// The adjoint is the transposed chain: g'[n] = g_H[c] / (M phi_hat(n)) placed at
// n mod M (zero elsewhere), b' = FFT_+(g'), and dL/dc'_i = sum_l phi(.) b'[l],
// dL/da_i = conj(exp(-j 2 pi f_c tau_i)) dL/dc'_i.  With W = 8 and beta = 2.3 W
// the kernel's aliasing error per entry is at most ~4e-7 of sum |c'_i| (a lone
// path); the errors of many paths partly cancel (~5e-9 of the sum for thousands).
constexpr int NU_W = 8;
constexpr float NU_BETA = 2.30f * NU_W;
constexpr double NU_BETA_D = 2.30 * NU_W;

__device__ __forceinline__ float es_phi(float z) {
    const float q = 1.0f - z * z;
    return q > 0.0f ? expf(NU_BETA * (sqrtf(q) - 1.0f)) : 0.0f;
}

// Path i in grid coordinates: the first cell l0 of its W-cell support, the FP32
// offset d0 = l0 - M x (in [-W/2, -W/2 + 1)), and the carrier phasor
// exp(-j 2 pi f_c tau).  The cell position is formed in FP64, so the phase error
// of any mode stays ~1e-7 rad.
__device__ __forceinline__ void nu_place(double tau, double fc, double df, int logM, int& l0, float& d0, float2& e) {
    float sn, cs;
    sincospif(-2.0f * frac_to_float(frac_mul(fc, tau)), &sn, &cs);
    e = make_float2(cs, sn);
    // x M = I + phi: I the cell (top logM bits of frac(df tau) in [0, 1)), phi the
    // remainder in [0, 1); l0 = ceil(x M - W/2) = I - W/2 + [phi > 0]
    const uint64_t x = (uint64_t)frac_mul(df, tau);
    const int I = (int)(x >> (64 - logM));
    const uint64_t phi = x << logM;
    const float phif = (float)(unsigned)(phi >> 40) * 0x1p-24f;
    l0 = I - NU_W / 2 + (phi != 0 ? 1 : 0);
    d0 = (phi != 0 ? 1.0f : 0.0f) - (float)(NU_W / 2) - phif;
}

// Bitonic sort of one value per lane across a full warp, ascending in key, the
// payload (d, c) travelling with its key.
__device__ __forceinline__ void warp_sort_by_key(int& key, float& d, float2& c, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int ok = __shfl_xor_sync(0xffffffffu, key, j);
            const float od = __shfl_xor_sync(0xffffffffu, d, j);
            const float ox = __shfl_xor_sync(0xffffffffu, c.x, j);
            const float oy = __shfl_xor_sync(0xffffffffu, c.y, j);
            // the lower lane of a pair keeps the smaller key in an ascending block
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            if (keep_min ? ok < key : ok > key) {
                key = ok;
                d = od;
                c = make_float2(ox, oy);
            }
        }
    }
}

// In-place radix-2 FFT of M = 2^logM complex values in shared memory by a CTA of
// TC_THREADS threads: X[k] = sum_l x[l] exp(sign j 2 pi k l / M).
__device__ void fft_smem(float2* x, int M, int logM, float sign) {
    for (int i = threadIdx.x; i < M; i += TC_THREADS) {
        const int j = (int)(__brev((unsigned)i) >> (32 - logM));
        if (i < j) {
            const float2 t = x[i];
            x[i] = x[j];
            x[j] = t;
        }
    }
    __syncthreads();
    for (int st = 1; st <= logM; ++st) {
        const int half = 1 << (st - 1);
        for (int b = threadIdx.x; b < M / 2; b += TC_THREADS) {
            const int pos = b & (half - 1);
            const int i0 = ((b >> (st - 1)) << st) + pos, i1 = i0 + half;
            float sn, cs;
            sincospif(sign * (float)pos / (float)half, &sn, &cs);
            const float2 v = x[i1], u = x[i0];
            const float2 t = make_float2(cs * v.x - sn * v.y, cs * v.y + sn * v.x);
            x[i0] = make_float2(u.x + t.x, u.y + t.y);
            x[i1] = make_float2(u.x - t.x, u.y - t.y);
        }
        __syncthreads();
    }
}

// Bounded wait of one thread until *flag reaches `want`; false after `limit` polls.
__device__ __forceinline__ bool wait_flag(const unsigned int* flag, unsigned int want, int limit) {
    for (int it = 0; it < limit; ++it) {
        if (*(volatile const unsigned int*)flag >= want) return true;
        __nanosleep(64);
    }
    return false;
}

// Receivers with at most TC_DIRECT paths skip the MMAs: each thread evaluates its
// row directly (N2 x n complex products), which is cheaper than building 128-row
// operand tiles for so few paths.
constexpr int TC_DIRECT = 8;

// MODE 0: forward (H out); 1: adjoint from g_H; 2: forward + power MSE + adjoint;
// 3, 4, 5: as 2, 0, 1 with receivers of many paths split over CTAs (TcSplit).
template <int N2, int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_cfr_tc(CfrShape S, const int64_t* __restrict__ offs, int R,
                                                       const float2* __restrict__ a, const double* __restrict__ tau,
                                                       const float* __restrict__ target, const float* __restrict__ w,
                                                       const float2* __restrict__ gH, float* __restrict__ loss,
                                                       float2* __restrict__ ga, float2* __restrict__ H,
                                                       double* __restrict__ part, unsigned int* __restrict__ ctr,
                                                       int32_t* __restrict__ status, TcSplit sp) {
    using T = TcDims<N2>;
    constexpr bool SPLIT = MODE >= 3;                  // receivers of many paths split over CTAs
    constexpr bool FWD = MODE != 1 && MODE != 5, BWD = MODE != 0 && MODE != 4;
    constexpr bool LOSS = MODE == 2 || MODE == 3;   // loss epilogue of whole receivers
    constexpr int LAST_PHASE = MODE == 4 ? 1 : 2;   // split work: 1 forward segments, 2 adjoint segments
    extern __shared__ float4 smem4[];
    float* A_hi = reinterpret_cast<float*>(smem4);
    float* A_lo = A_hi + T::A_FLOATS;
    float* B_hi = A_lo + T::A_FLOATS;
    float* B_lo = B_hi + T::B_FLOATS;
    char* tab_base = reinterpret_cast<char*>(B_lo + T::B_FLOATS);
    // table set k (k = chunk & 1), its pointers formed arithmetically
    auto tabset = [&](int k) { return tc_tab<N2>(tab_base + (size_t)(k & 1) * tc_tab_bytes<N2>()); };
    float2* tRed = reinterpret_cast<float2*>(tab_base + 2 * tc_tab_bytes<N2>());
    float2* rcC = tRed + 4 * 32;                                  // TC_PH_CAP: c_i of the receiver
    PathPhase* rcP = reinterpret_cast<PathPhase*>(rcC + TC_PH_CAP);   // TC_PH_CAP: its phase data
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_sh;
    __shared__ int s_r;
    __shared__ double s_red[TC_THREADS / 32];
    __shared__ bool s_last;
    __shared__ int s_kind, s_slot, s_nseg;
    __shared__ int64_t s_i0, s_i1;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t mb = smem_u32(&mbar);
    // mode 4: number of heavy receivers (fixed once mode 3 has finished); with
    // none, the CTA takes no TMEM and only joins the completion count
    if (tid == 0) mbar_init(mb, 1);
    __syncthreads();
    // mode 3: this call's epoch (only the last CTA advances it, at the very end)
    const unsigned int epoch = SPLIT ? __ldcg(sp.cnt + 4) : 0u;
    int phase = 0;   // mode 3, thread 0: 0 receivers, 1 heavy forward segments, 2 heavy adjoint segments
    if (warp == 0) tmem_alloc(smem_u32(&tmem_sh), T::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t parity = 0;
    bool ok = true;
    const float inv_rn = 1.0f / ((float)R * (float)S.N);
    const int m = tid;   // row c1 of this thread

    // one batch of MMAs issued by thread 0 once the operand tiles are written;
    // its completion arrives on the mbarrier, which mma_wait polls (bounded)
    auto mma_issue = [&](auto issue) {
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            issue();
            tc_commit(mb);
        }
    };
    auto mma_wait = [&]() -> bool {
        bool done = mbar_wait(mb, parity);
        parity ^= 1u;
        tc_fence_after();
        return __syncthreads_and(done) != 0;
    };

    for (;;) {
        __syncthreads();   // every thread has read s_r (and finished the previous receiver)
        if (tid == 0) {
            int kind = 0, slot = -1, nseg = 1, rr = R;
            int64_t a0 = 0, a1 = 0;
            if (SPLIT && phase == 0) {
                rr = (int)atomicAdd(ctr + 1, 1u);
                if (rr < R) {
                    a0 = offs[rr];
                    a1 = offs[rr + 1];
                    bool defer = false;
                    if (ok && a1 - a0 > TC_SPLIT) {
                        const int h = (int)atomicAdd(sp.cnt, 1u);
                        if (h < TC_HEAVY_CAP) {
                            kind = 3;   // deferred: published below, split later
                            slot = h;
                            defer = true;
                        }
                    }
                    if (!defer) atomicAdd(sp.cnt + 3, 1u);   // classified
                } else {
                    phase = MODE == 5 ? 2 : 1;
                }
            }
            if (SPLIT && phase > 0) {
                // heavy receivers: claim a forward segment; once the heavy list is final
                // and every forward segment claimed, an adjoint segment
                rr = R;
                for (int it = 0; it < sp.wait_limit && rr == R && phase <= LAST_PHASE; ++it) {
                    unsigned int* cur = sp.cnt + phase;
                    unsigned int* next = phase == 1 ? sp.seg_next : sp.adj_next;
                    const int h = (int)*(volatile unsigned int*)cur;
                    const int n_met = (int)min(*(volatile unsigned int*)sp.cnt, (unsigned int)TC_HEAVY_CAP);
                    if (h >= n_met) {
                        if (*(volatile unsigned int*)(sp.cnt + 3) < (unsigned int)R) {
                            __nanosleep(64);   // receivers still being classified: more may come
                            continue;
                        }
                        if ((int)min(*(volatile unsigned int*)sp.cnt, (unsigned int)TC_HEAVY_CAP) > h)
                            continue;   // appended while we looked
                        ++phase;
                        continue;
                    }
                    if (*(volatile unsigned int*)(sp.pub + h) != epoch + 1u) {
                        __nanosleep(64);   // being published by the CTA that met it
                        continue;
                    }
                    __threadfence();
                    const int rh = sp.list[h];
                    const int64_t b0 = offs[rh], b1 = offs[rh + 1];
                    const int g = (int)((b1 - b0 + TC_SEG - 1) / TC_SEG);
                    const int sg = (int)atomicAdd(next + h, 1u);
                    if (sg < g) {
                        rr = rh;
                        kind = phase;
                        slot = h;
                        nseg = g;
                        a0 = b0 + (int64_t)sg * TC_SEG;
                        a1 = min(b1, a0 + TC_SEG);
                        break;
                    }
                    atomicCAS(cur, (unsigned int)h, (unsigned int)h + 1u);
                }
                if (rr == R && phase <= LAST_PHASE) rt_set_status(status, RT_ERR_TIMEOUT);
            } else if (!SPLIT) {
                rr = (int)atomicAdd(ctr + 1, 1u);
                if (rr < R) {
                    a0 = offs[rr];
                    a1 = offs[rr + 1];
                }
            }
            s_r = rr;
            s_kind = kind;
            s_slot = slot;
            s_nseg = nseg;
            s_i0 = a0;
            s_i1 = a1;
        }
        __syncthreads();
        const int r = s_r;
        if (r >= R || !ok) break;
        const int kind = s_kind, slot = s_slot;
        const int64_t i0 = s_i0, i1 = s_i1;
        const int P = (int)(i1 - i0);
        if (SPLIT && kind == 3) {
            // a heavy receiver: clear its row and counters (mode 5: put the transformed
            // dL/dH in the row at once), then publish it
            const int M = 2 * S.N;
            float2* row = sp.acc + (int64_t)slot * M;
            if (MODE == 5) {
                float2* grid = reinterpret_cast<float2*>(A_hi);
                for (int l = tid; l < M; l += TC_THREADS) grid[l] = make_float2(0.0f, 0.0f);
                __syncthreads();
                for (int c = tid; c < S.N; c += TC_THREADS) {
                    const float2 g = gH[(int64_t)r * S.N + c];
                    const float dv = sp.dec[c];
                    grid[(c - S.N / 2) & (M - 1)] = make_float2(g.x * dv, g.y * dv);
                }
                __syncthreads();
                fft_smem(grid, M, 31 - __clz(M), 1.0f);
                for (int l = tid; l < M; l += TC_THREADS) row[l] = grid[l];
            } else {
                for (int l = tid; l < M; l += TC_THREADS) row[l] = make_float2(0.0f, 0.0f);
            }
            if (tid == 0) {
                sp.list[slot] = r;
                sp.seg_next[slot] = 0u;
                sp.adj_next[slot] = 0u;
                sp.fwd_done[slot] = 0u;
                sp.ready[slot] = MODE == 5 ? 1u : 0u;
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                atomicExch(sp.pub + slot, epoch + 1u);
                atomicAdd(sp.cnt + 3, 1u);   // classified
            }
            continue;
        }
        if (SPLIT && (kind == 1 || kind == 2)) {
            // a segment of a split receiver: non-uniform FFT on its grid row
            const int M = 2 * S.N, logM = 31 - __clz(M);
            const double fc = S.f0 + 0.5 * (double)S.N * S.df;
            float2* grid = reinterpret_cast<float2*>(A_hi);   // M values (fits in the operand tiles)
            float2* row = sp.acc + (int64_t)slot * M;
            if (kind == 1) {
                for (int l = tid; l < M; l += TC_THREADS) grid[l] = make_float2(0.0f, 0.0f);
                __syncthreads();
                // Delays cluster on a few cells of the grid, so per-path atomics
                // collide.  Each warp takes 32 consecutive paths, sorts them by
                // first cell l0 across its lanes, sums each run of equal l0 per
                // tap, and the run's first lane adds the 8 sums: the atomics of one
                // instruction then go to distinct cells.
                for (int64_t base = i0 + (tid & ~31); base < i1; base += TC_THREADS) {
                    const int64_t i = base + lane;
                    int key = 0x7fffffff;   // lanes past the segment sort last, add nothing
                    float d0 = 0.0f;
                    float2 cp = make_float2(0.0f, 0.0f);
                    if (i < i1) {
                        float2 e;
                        nu_place(tau[i], fc, S.df, logM, key, d0, e);
                        cp = cmul(a[i], e);
                    }
                    warp_sort_by_key(key, d0, cp, lane);
                    // same[s]: lane + s holds the same l0 (runs are contiguous)
                    unsigned same = 0u;
#pragma unroll
                    for (int b = 0; b < 5; ++b) {
                        const int ok = __shfl_down_sync(0xffffffffu, key, 1 << b);
                        if (lane + (1 << b) < 32 && ok == key) same |= 1u << b;
                    }
                    const int kp = __shfl_up_sync(0xffffffffu, key, 1);
                    const bool head = key != 0x7fffffff && (lane == 0 || kp != key);
#pragma unroll
                    for (int k = 0; k < NU_W; ++k) {
                        const float wk = es_phi((d0 + (float)k) * (2.0f / NU_W));
                        float vx = wk * cp.x, vy = wk * cp.y;
#pragma unroll
                        for (int b = 0; b < 5; ++b) {
                            const float ox = __shfl_down_sync(0xffffffffu, vx, 1 << b);
                            const float oy = __shfl_down_sync(0xffffffffu, vy, 1 << b);
                            if (same & (1u << b)) {
                                vx += ox;
                                vy += oy;
                            }
                        }
                        if (head) {
                            float2* gp = grid + ((key + k) & (M - 1));
                            atomicAdd(&gp->x, vx);
                            atomicAdd(&gp->y, vy);
                        }
                    }
                }
                __syncthreads();
                for (int l = tid; l < M; l += TC_THREADS) {
                    const float2 v = grid[l];
                    if (v.x != 0.0f) atomicAdd(&row[l].x, v.x);
                    if (v.y != 0.0f) atomicAdd(&row[l].y, v.y);
                }
                __threadfence();
                __syncthreads();
                if (tid == 0) s_last = atomicAdd(sp.fwd_done + slot, 1u) == (unsigned int)(s_nseg - 1);
                __syncthreads();
                if (!s_last) continue;
                // the last segment: H, the loss partial, then the adjoint grid b'
                __threadfence();
                for (int l = tid; l < M; l += TC_THREADS) grid[l] = __ldcg(row + l);
                __syncthreads();
                fft_smem(grid, M, logM, -1.0f);
                if (MODE == 4) {
                    for (int c = tid; c < S.N; c += TC_THREADS) {
                        const int idx = (c - S.N / 2) & (M - 1);
                        const float dv = sp.dec[c];
                        H[(int64_t)r * S.N + c] = make_float2(grid[idx].x * dv, grid[idx].y * dv);
                    }
                    continue;
                }
                const float wr = w[r];
                float lsum = 0.0f;   // FP32 within a receiver, FP64 across receivers
                for (int c = tid; c < S.N; c += TC_THREADS) {
                    const int idx = (c - S.N / 2) & (M - 1);
                    const float dv = sp.dec[c];
                    const float2 h = make_float2(grid[idx].x * dv, grid[idx].y * dv);
                    const float e = h.x * h.x + h.y * h.y - target[(int64_t)r * S.N + c];
                    const float we = wr * e;
                    lsum = fmaf(we, we, lsum);
                    const float sc = 4.0f * wr * wr * e * inv_rn * dv;
                    if (H) H[(int64_t)r * S.N + c] = h;
                    grid[idx] = make_float2(sc * h.x, sc * h.y);
                }
                for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
                if (lane == 0) s_red[warp] = lsum;
                __syncthreads();
                for (int l = S.N / 2 + tid; l < M - S.N / 2; l += TC_THREADS) grid[l] = make_float2(0.0f, 0.0f);
                __syncthreads();
                fft_smem(grid, M, logM, 1.0f);
                for (int l = tid; l < M; l += TC_THREADS) row[l] = grid[l];
                __threadfence();
                __syncthreads();
                if (tid == 0) {
                    part[r] = s_red[0] + s_red[1] + s_red[2] + s_red[3];
                    __threadfence();
                    atomicExch(sp.ready + slot, 1u);
                }
                continue;
            }
            // kind 2: dL/da of the segment's paths once the adjoint grid is ready
            if (tid == 0) s_last = wait_flag(sp.ready + slot, 1u, sp.wait_limit);
            __syncthreads();
            if (!s_last) {
                ok = false;
                break;
            }
            __threadfence();
            for (int l = tid; l < M; l += TC_THREADS) grid[l] = __ldcg(row + l);
            __syncthreads();
            for (int64_t i = i0 + tid; i < i1; i += TC_THREADS) {
                int l0;
                float d0;
                float2 e;
                nu_place(tau[i], fc, S.df, logM, l0, d0, e);
                float2 gc = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int k = 0; k < NU_W; ++k) {
                    const float wk = es_phi((d0 + (float)k) * (2.0f / NU_W));
                    const float2 v = grid[(l0 + k) & (M - 1)];
                    gc.x = fmaf(wk, v.x, gc.x);
                    gc.y = fmaf(wk, v.y, gc.y);
                }
                ga[i] = cmulc(gc, e);
            }
            continue;
        }
        const bool do_fwd = FWD;
        const bool direct = P <= TC_DIRECT;
        const int nch = (P + TC_CP - 1) / TC_CP;
        // the loss epilogue's target powers and weight, loaded now so that their
        // latency passes during the forward (N2 <= 8: a few registers)
        constexpr bool PREF = LOSS && N2 <= 8;
        float tgt[PREF ? N2 : 1];
        float wr_pref = 0.0f;
        if (PREF) {
            const int64_t hrow0 = (int64_t)r * S.N + (int64_t)m * N2;
#pragma unroll
            for (int c2 = 0; c2 < N2; ++c2) tgt[c2] = __ldg(target + hrow0 + c2);
            wr_pref = __ldg(w + r);
        }
        // a receiver of at most TC_PH_CAP paths: its phases and c_i once, all loads at once
        const bool cached = !direct && P <= TC_PH_CAP;
        if (cached) {
            for (int t = tid; t < P; t += TC_THREADS) {
                const PathPhase pp = path_phase(tau[i0 + t], S.f0, S.df);
                rcP[t] = pp;
                rcC[t] = do_fwd ? cmul(a[i0 + t], base_phasor(pp)) : make_float2(0.0f, 0.0f);
            }
            __syncthreads();
        }
        const PathPhase* cP = cached ? rcP : nullptr;
        float hre[N2], him[N2];
#pragma unroll
        for (int c2 = 0; c2 < N2; ++c2) hre[c2] = him[c2] = 0.0f;

        if (do_fwd && direct && P > 0) {
            const TcTab tb = tabset(0);
            tc_tables<N2>(S, i0, P, 0, true, a, tau, tb, cP, rcC);
            for (int ii = 0; ii < P; ++ii) {
                const float2 ac = cmul(tb.tFc[ii * TC_NFC + (m >> 3)], tb.tF[ii * T::NF + 16 + (m & 7)]);
                const float2* B = tb.tF + ii * T::NF + T::NAH + T::NAL;
#pragma unroll
                for (int c2 = 0; c2 < N2; ++c2) {
                    const float2 b = B[c2];
                    hre[c2] = fmaf(ac.x, b.x, fmaf(-ac.y, b.y, hre[c2]));
                    him[c2] = fmaf(ac.x, b.y, fmaf(ac.y, b.x, him[c2]));
                }
            }
        } else if (do_fwd && P > 0) {
            // Chunks in a software pipeline: the tables of chunk ch + 1 (with the
            // loads of its delays and coefficients) are built in the other table set
            // while the MMAs of chunk ch run; the operand tiles are rewritten only
            // after those MMAs have completed.
            tc_tables<N2>(S, i0, P, 0, false, a, tau, tabset(0), cP, rcC);
            bool first = true;
            for (int ch = 0; ch < nch && ok; ++ch) {
                const TcTab tb = tabset(ch);
                const int n = min(TC_CP, P - ch * TC_CP);
                const int n_pad = (n + 7) & ~7;   // the K steps issued cover paths [0, n_pad)
                // A' row m: k = i (Re Ac), k = CP + i (Im Ac)
                for (int i4 = 0; i4 < n_pad / 4; ++i4) {
                    float re[4], im[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ii = 4 * i4 + q;
                        float2 v = cmul(tb.tFc[ii * TC_NFC + (m >> 3)], tb.tF[ii * T::NF + 16 + (m & 7)]);
                        re[q] = v.x;
                        im[q] = v.y;
                    }
                    put4(A_hi, A_lo, (T::KA / 4) * 32, m, i4, re[0], re[1], re[2], re[3]);
                    put4(A_hi, A_lo, (T::KA / 4) * 32, m, TC_CP / 4 + i4, im[0], im[1], im[2], im[3]);
                }
                // B' (transposed, NB rows x KA): row c2' < N2: [Re B | -Im B], N2 <= c2' < 2N2: [Im B | Re B]
                const int nkb = n_pad / 4;   // k blocks per half
                for (int g = tid; g < 2 * N2 * 2 * nkb; g += TC_THREADS) {
                    const int row = g / (2 * nkb), kk = g - row * (2 * nkb);
                    const bool imhalf = kk >= nkb;
                    const int kb = imhalf ? TC_CP / 4 + (kk - nkb) : kk;
                    const int i0p = 4 * (imhalf ? kk - nkb : kk);
                    float x[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 b = tb.tF[(i0p + q) * T::NF + T::NAH + T::NAL + (row % N2)];
                        x[q] = row < N2 ? (imhalf ? -b.y : b.x) : (imhalf ? b.x : b.y);
                    }
                    put4(B_hi, B_lo, (T::KA / 4) * 32, row, kb, x[0], x[1], x[2], x[3]);
                }
                const bool acc0 = first;
                mma_issue([&]() {
                    const uint32_t idesc = tc_idesc(128, T::NB);
                    const uint32_t sbo = (T::KA / 4) * 128;
                    // K step s starts 256 bytes further: its descriptors are the base ones
                    // plus 16 s in the start-address field (addresses stay below 256 KB)
                    const uint64_t dah = tc_sdesc(smem_u32(A_hi), 128, sbo), dal = tc_sdesc(smem_u32(A_lo), 128, sbo);
                    const uint64_t dbh = tc_sdesc(smem_u32(B_hi), 128, sbo), dbl = tc_sdesc(smem_u32(B_lo), 128, sbo);
                    bool fst = acc0;
                    for (int s = 0; s < T::KA / 8; ++s) {
                        if (8 * (s % (TC_CP / 8)) >= n) continue;   // all-zero K step
                        const uint64_t o = (uint64_t)(16 * s);
                        tc_mma(tmem, dah + o, dbh + o, idesc, fst ? 0u : 1u);
                        tc_mma(tmem, dah + o, dbl + o, idesc, 1u);
                        tc_mma(tmem, dal + o, dbh + o, idesc, 1u);
                        fst = false;
                    }
                });
                if (ch + 1 < nch) tc_tables<N2>(S, i0, P, ch + 1, false, a, tau, tabset(ch + 1), cP, rcC);
                ok = mma_wait();
                first = false;
            }
            if (!ok) break;
            float v[T::NB];
#pragma unroll
            for (int c = 0; c < T::NB; c += 16) tmem_ld16(lane_base + (uint32_t)c, v + c);
            tmem_wait_ld();
            tc_fence_before();
#pragma unroll
            for (int c2 = 0; c2 < N2; ++c2) {
                hre[c2] = v[c2];
                him[c2] = v[N2 + c2];
            }
        }
        // ---- epilogue: H out, loss, g_H
        const int64_t hrow = (int64_t)r * S.N + (int64_t)m * N2;
        if (MODE == 0 || MODE == 4) {
#pragma unroll
            for (int c2 = 0; c2 < N2; ++c2) H[hrow + c2] = make_float2(hre[c2], him[c2]);
            continue;
        }
        float gre[N2], gim[N2];
        if (LOSS) {
            const float wr = PREF ? wr_pref : w[r];
            float lsum = 0.0f;   // FP32 within a receiver, FP64 across receivers
#pragma unroll
            for (int c2 = 0; c2 < N2; ++c2) {
                const float pt = PREF ? tgt[PREF ? c2 : 0] : target[hrow + c2];
                const float e = hre[c2] * hre[c2] + him[c2] * him[c2] - pt;
                const float we = wr * e;
                lsum = fmaf(we, we, lsum);
                const float s = 4.0f * wr * wr * e * inv_rn;   // dL/dH = 4 w^2 (|H|^2 - P*) H / (R N)
                gre[c2] = s * hre[c2];
                gim[c2] = s * him[c2];
                if (H) H[hrow + c2] = make_float2(hre[c2], him[c2]);
            }
            for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
            if (lane == 0) s_red[warp] = lsum;
        } else {
#pragma unroll
            for (int c2 = 0; c2 < N2; ++c2) {
                const float2 g = gH[hrow + c2];
                gre[c2] = g.x;
                gim[c2] = g.y;
            }
        }

        // ---- adjoint: Y[m][i] = sum_c2 g[m][c2] conj(B_i[c2]), then conj(A_i[m]) Y, reduced over m.
        // Chunks in reverse order.  After a forward the tables of the last two
        // chunks are still in place (chunk ch in set ch & 1); the tables of chunk
        // ch - 1 are built while the MMAs of chunk ch run.
        for (int ch = nch - 1; ch >= 0 && ok; --ch) {
            const TcTab tb = tabset(ch);
            const int64_t base = i0 + (int64_t)ch * TC_CP;
            const int n = min(TC_CP, P - ch * TC_CP);
            if (ch == nch - 1 && !do_fwd) tc_tables<N2>(S, i0, P, ch, direct, nullptr, tau, tb, cP, rcC);
            // the tables of chunk ch - 1 still in place from the forward
            const bool prev_kept = do_fwd && ch - 1 >= nch - 2;
            float vr[32], vi[32];
            if (direct) {
#pragma unroll
                for (int ii = 0; ii < 32; ++ii) {
                    float yr = 0.0f, yi = 0.0f;
                    if (ii < n) {
                        const float2* B = tb.tF + ii * T::NF + T::NAH + T::NAL;
#pragma unroll
                        for (int c2 = 0; c2 < N2; ++c2) {   // g conj(B)
                            const float2 b = B[c2];
                            yr = fmaf(gre[c2], b.x, fmaf(gim[c2], b.y, yr));
                            yi = fmaf(gim[c2], b.x, fmaf(-gre[c2], b.y, yi));
                        }
                    }
                    vr[ii] = yr;
                    vi[ii] = yi;
                }
            } else {
                const int n_pad = (n + 7) & ~7;
                if (ch == nch - 1) {
                    // G' (128 x KG), written once per receiver into the A tiles
#pragma unroll
                    for (int kb = 0; kb < T::KG / 4; ++kb) {
                        float x[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int k = 4 * kb + q;
                            x[q] = k < N2 ? gre[k % N2] : k < 2 * N2 ? gim[k % N2] : 0.0f;
                        }
                        put4(A_hi, A_lo, (T::KG / 4) * 32, m, kb, x[0], x[1], x[2], x[3]);
                    }
                }
                // Bc' (transposed, 2CP rows x KG): row i < CP: [Re B_i | Im B_i], row CP + i: [-Im B_i | Re B_i]
                for (int g = tid; g < 2 * n_pad * (T::KG / 4); g += TC_THREADS) {
                    const int rr = g / (T::KG / 4), kb = g - rr * (T::KG / 4);
                    const bool imrow = rr >= n_pad;
                    const int ii = imrow ? rr - n_pad : rr;
                    const int row = imrow ? TC_CP + ii : ii;
                    float x[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int k = 4 * kb + q;
                        float v = 0.0f;
                        if (k < 2 * N2) {
                            const float2 b = tb.tF[ii * T::NF + T::NAH + T::NAL + (k % N2)];
                            v = k < N2 ? (imrow ? -b.y : b.x) : (imrow ? b.x : b.y);
                        }
                        x[q] = v;
                    }
                    put4(B_hi, B_lo, (T::KG / 4) * 32, row, kb, x[0], x[1], x[2], x[3]);
                }
                mma_issue([&]() {
                    const uint32_t idesc = tc_idesc(128, 2 * TC_CP);
                    const uint32_t sbo = (T::KG / 4) * 128;
                    const uint64_t dah = tc_sdesc(smem_u32(A_hi), 128, sbo), dal = tc_sdesc(smem_u32(A_lo), 128, sbo);
                    const uint64_t dbh = tc_sdesc(smem_u32(B_hi), 128, sbo), dbl = tc_sdesc(smem_u32(B_lo), 128, sbo);
                    const uint32_t d = tmem + T::Y_COL;
                    for (int s = 0; s < T::KG / 8; ++s) {
                        const uint64_t o = (uint64_t)(16 * s);
                        tc_mma(d, dah + o, dbh + o, idesc, s > 0 ? 1u : 0u);
                        tc_mma(d, dah + o, dbl + o, idesc, 1u);
                        tc_mma(d, dal + o, dbh + o, idesc, 1u);
                    }
                });
                if (ch >= 1 && !prev_kept) tc_tables<N2>(S, i0, P, ch - 1, false, nullptr, tau, tabset(ch - 1), cP, rcC);
                ok = mma_wait();
                if (!ok) break;
#pragma unroll
                for (int c = 0; c < TC_CP; c += 16) {
                    tmem_ld16(lane_base + T::Y_COL + c, vr + c);
                    tmem_ld16(lane_base + T::Y_COL + TC_CP + c, vi + c);
                }
                tmem_wait_ld();
                tc_fence_before();
#pragma unroll
                for (int ii = TC_CP; ii < 32; ++ii) vr[ii] = vi[ii] = 0.0f;
            }
#pragma unroll
            for (int ii = 0; ii < 32; ++ii) {   // conj(A_i[m]) Y[m][i]
                float2 p = make_float2(0.0f, 0.0f);
                if (ii < n) p = cmulc(make_float2(vr[ii], vi[ii]), tc_A(tb.tF, T::NF, ii, m));
                vr[ii] = p.x;
                vi[ii] = p.y;
            }
            // transposed reduction: lane l ends with this warp's sum for path l (mod
            // 2 TOP); a direct receiver (at most TC_DIRECT paths) needs half the stages
            auto reduce = [&](auto top) {
                constexpr int TOP = decltype(top)::value;
#pragma unroll
                for (int o = TOP; o >= 1; o >>= 1) {
                    const bool up = (lane & o) != 0;
#pragma unroll
                    for (int j = 0; j < o; ++j) {
                        const float sr = up ? vr[j] : vr[j + o], si = up ? vi[j] : vi[j + o];
                        const float kr = up ? vr[j + o] : vr[j], ki = up ? vi[j + o] : vi[j];
                        vr[j] = kr + __shfl_xor_sync(0xffffffffu, sr, o);
                        vi[j] = ki + __shfl_xor_sync(0xffffffffu, si, o);
                    }
                }
#pragma unroll
                for (int o = 2 * TOP; o < 32; o <<= 1) {   // lanes l and l ^ o hold the same paths
                    vr[0] += __shfl_xor_sync(0xffffffffu, vr[0], o);
                    vi[0] += __shfl_xor_sync(0xffffffffu, vi[0], o);
                }
            };
            constexpr int RED_TOP = TC_CP > 16 ? 16 : TC_CP / 2;
            static_assert(TC_DIRECT % 2 == 0 && TC_DIRECT / 2 <= RED_TOP, "direct receivers use a shorter reduction");
            if (direct) reduce(std::integral_constant<int, TC_DIRECT / 2>());
            else reduce(std::integral_constant<int, RED_TOP>());
            tRed[warp * 32 + lane] = make_float2(vr[0], vi[0]);
            __syncthreads();
            if (warp == 0 && lane < n) {
                float2 s = tRed[lane];
#pragma unroll
                for (int k = 1; k < TC_THREADS / 32; ++k) {
                    s.x += tRed[k * 32 + lane].x;
                    s.y += tRed[k * 32 + lane].y;
                }
                ga[base + lane] = cmulc(s, base_phasor(tb.tP[lane]));
            }
        }
        if ((MODE == 2 || MODE == 3) && kind == 0) {
            __syncthreads();
            if (tid == 0) part[r] = s_red[0] + s_red[1] + s_red[2] + s_red[3];
        }
    }

    if (!ok) {
        rt_set_status(status, RT_ERR_TIMEOUT);
        mbar_wait(mb, parity ^ 1u);   // bounded: let an unfinished batch drain before TMEM goes
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, T::TMEM_COLS);
    // completion: the last CTA resets the counters and sums the loss over all
    // receivers in receiver order (mode 3: only if no receiver was deferred; mode 4
    // then does it)
    if (tid == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(ctr, 1u);
        s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (MODE == 2 || MODE == 3) {
            double s = 0.0;
            for (int k = tid; k < R; k += TC_THREADS) s += ((volatile double*)part)[k];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) s_red[warp] = s;
            __syncthreads();
            if (tid == 0) *loss = (float)((s_red[0] + s_red[1] + s_red[2] + s_red[3]) * (double)inv_rn);
        }
        if (tid == 0) {
            ctr[0] = 0u;
            ctr[1] = 0u;
            if (SPLIT) {
                sp.cnt[0] = 0u;
                sp.cnt[1] = 0u;
                sp.cnt[2] = 0u;
                sp.cnt[3] = 0u;
                sp.cnt[4] = epoch + 1u;
            }
        }
    }
}

// Tensor-core launch for n_sub = 128 N2; returns RT_ERR_UNSUPPORTED for other sizes.
template <int MODE>
rt_status launch_tc(rt_ctx* ctx, const CfrShape& S, const int64_t* offs, int R, const float2* a, const double* tau,
                    const float* target, const float* w, const float2* gH, float* loss, float2* ga, float2* H,
                    double* part, unsigned int* ctr, TcSplit sp = TcSplit()) {
    auto go = [&](auto n2) -> rt_status {
        constexpr int N2 = decltype(n2)::value;
        auto kern = k_cfr_tc<N2, MODE>;
        const size_t smem = tc_smem_bytes<N2>();
        RT_CK(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        RT_CK(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
        // resident CTAs per SM: shared memory (with the per-CTA reservation) and TMEM
        int smem_sm = 0, reserved = 0;
        RT_CK(ctx, cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
        RT_CK(ctx, cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, ctx->device));
        int per_sm = smem_sm / (int)(smem + 64 + (size_t)reserved);
        per_sm = std::max(1, std::min(per_sm, (int)(512 / TcDims<N2>::TMEM_COLS)));
        const int grid = std::max(1, MODE >= 3 ? ctx->num_sms * per_sm : std::min(R, ctx->num_sms * per_sm));
        kern<<<grid, TC_THREADS, smem, ctx->stream>>>(S, offs, R, a, tau, target, w, gH, loss, ga, H, part, ctr,
                                                       ctx->d_status, sp);
        RT_COUNT(ctx);
        RT_CK_LAUNCH(ctx);
        return RT_OK;
    };
    if (S.N1 * S.N2 != S.N) return RT_ERR_UNSUPPORTED;
    switch (S.N) {
        case 256: return go(std::integral_constant<int, 2>());
        case 512: return go(std::integral_constant<int, 4>());
        case 1024: return go(std::integral_constant<int, 8>());
        case 2048: return go(std::integral_constant<int, 16>());
        case 4096: return go(std::integral_constant<int, 32>());
        default: return RT_ERR_UNSUPPORTED;
    }
}

bool tc_supported(const rt_ctx* ctx, int n_sub) {
    return ctx->cfr_tensor_cores && (n_sub == 256 || n_sub == 512 || n_sub == 1024 || n_sub == 2048 || n_sub == 4096);
}

bool make_shape(int n_sub, double fc, double df, CfrShape& S) {
    if (n_sub < 1 || n_sub > 4096 || (n_sub > 1 && (n_sub & 1))) return false;
    S.N = n_sub;
    S.N2 = 1;
    while (S.N2 < 16 && n_sub % (S.N2 * 2) == 0) S.N2 *= 2;
    S.N1 = n_sub / S.N2;
    S.f0 = fc - (double)(n_sub / 2) * df;
    S.df = df;
    return true;
}

// sAc + sA (CH x N1 each), sB (CH x N2), factors (CH x (8 + N1/8 + 8)), sP
// (CH + padding), then optionally sG (N).
size_t fwd_smem(const CfrShape& S) {
    const size_t nf = 8 + (S.N1 + 7) / 8 + 8;
    return 2 * (size_t)CH * S.N1 * 8 + (size_t)CH * S.N2 * 8 + (size_t)CH * nf * 8 + (size_t)CH * 8 +
           (size_t)(CH + (CH & 1)) * sizeof(PathPhase) + 16;
}

template <typename F>
rt_status dispatch_opt(rt_ctx* ctx, int N, F&& f) {
    int opt = (N + CFR_THREADS - 1) / CFR_THREADS;
    if (opt <= 1) return f(std::integral_constant<int, 1>());
    if (opt <= 2) return f(std::integral_constant<int, 2>());
    if (opt <= 4) return f(std::integral_constant<int, 4>());
    if (opt <= 8) return f(std::integral_constant<int, 8>());
    return f(std::integral_constant<int, 16>());
}

}  // namespace

static rt_status check_cfr(rt_ctx* ctx, const int64_t* offs, int32_t n_rx, const double* tau, int32_t n_sub, double fc,
                           double df, CfrShape& S) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!offs || !tau) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null device pointer");
    if (n_rx < 1) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_rx must be >= 1");
    if (!(fc > 0.0) || !(df >= 0.0) || !std::isfinite(fc) || !std::isfinite(df))
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "frequencies must be finite, f_c > 0, df >= 0");
    if (!make_shape(n_sub, fc, df, S)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_sub must be 1 or even and <= 4096");
    return RT_OK;
}

template <typename K>
static rt_status set_smem(rt_ctx* ctx, K kernel, size_t bytes) {
    if (bytes > 48 * 1024) RT_CK(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return RT_OK;
}

// Scratch of the heavy-receiver split (modes 3 to 5) and the per-column factors
// 1 / (M phi_hat(n)) of its non-uniform FFT (made on the host when n_sub changes).
static rt_status split_setup(rt_ctx* ctx, int n_sub, TcSplit* sp) {
    int* ints = nullptr;
    void* acc = nullptr;
    float* dec = nullptr;
    int* dec_n = nullptr;
    rt_status s = rt_cfr_split_scratch(ctx, TC_HEAVY_CAP, (size_t)TC_HEAVY_CAP * 2 * (size_t)n_sub * sizeof(float2), &ints,
                             &acc, &dec, &dec_n);
    if (s != RT_OK) return s;
    if (*dec_n != n_sub) {
        // 1 / (M phi_hat(n)), M phi_hat(n) = W/2 int_{-1}^{1} phi(z) cos(pi n W z / M) dz
        // (Gauss-Legendre, 256 nodes by Newton iteration on P_256)
        const int Q = 256;
        std::vector<double> zq(Q), wq(Q);
        for (int i = 0; i < Q; ++i) {
            double z = std::cos(RT_PI * (i + 0.75) / (Q + 0.5)), dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = z;
                for (int k = 2; k <= Q; ++k) {
                    const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = Q * (z * p1 - p0) / (z * z - 1.0);
                const double dz = p1 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-15) break;
            }
            zq[i] = z;
            wq[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
        const int M = 2 * n_sub;
        std::vector<float> hd(n_sub);
        for (int c = 0; c < n_sub; ++c) {
            const double n = (double)(c - n_sub / 2);
            double acc_q = 0.0;
            for (int i = 0; i < Q; ++i)
                acc_q += wq[i] * std::exp(NU_BETA_D * (std::sqrt(1.0 - zq[i] * zq[i]) - 1.0)) *
                         std::cos(RT_PI * n * NU_W * zq[i] / M);
            hd[c] = (float)(1.0 / (0.5 * NU_W * acc_q));
        }
        RT_CK(ctx, cudaMemcpy(dec, hd.data(), n_sub * sizeof(float), cudaMemcpyHostToDevice));
        *dec_n = n_sub;
    }
    sp->cnt = reinterpret_cast<unsigned int*>(ints);   // zeroed with the tables, once per context
    sp->list = ints + 8;
    sp->seg_next = reinterpret_cast<unsigned int*>(sp->list + TC_HEAVY_CAP);
    sp->adj_next = sp->seg_next + TC_HEAVY_CAP;
    sp->fwd_done = sp->adj_next + TC_HEAVY_CAP;
    sp->ready = sp->fwd_done + TC_HEAVY_CAP;
    sp->pub = sp->ready + TC_HEAVY_CAP;
    sp->acc = static_cast<float2*>(acc);
    sp->dec = dec;
    sp->wait_limit = ctx->wait_limit > 0 ? ctx->wait_limit : TC_WAIT_LIMIT;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_cfr(rt_ctx* ctx, const int64_t* rx_offsets_dev, int32_t n_rx, const void* a_dev,
                            const double* tau_dev, double f_center_hz, double delta_f_hz, int32_t n_sub, void* H_dev) {
    CfrShape S;
    rt_status s = check_cfr(ctx, rx_offsets_dev, n_rx, tau_dev, n_sub, f_center_hz, delta_f_hz, S);
    if (s != RT_OK) return s;
    if (!a_dev || !H_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null device pointer");
    if (tc_supported(ctx, n_sub)) {
        double* part;
        unsigned int* ctr;
        s = rt_cfr_fused_scratch(ctx, n_rx, &part, &ctr);
        if (s != RT_OK) return s;
        TcSplit sp;
        s = split_setup(ctx, n_sub, &sp);
        if (s != RT_OK) return s;
        return launch_tc<4>(ctx, S, rx_offsets_dev, n_rx, (const float2*)a_dev, tau_dev, nullptr, nullptr, nullptr,
                            nullptr, nullptr, (float2*)H_dev, part, ctr, sp);
    }
    const size_t smem = fwd_smem(S);
    return dispatch_opt(ctx, S.N, [&](auto opt) -> rt_status {
        constexpr int O = decltype(opt)::value;
        rt_status e = set_smem(ctx, k_cfr_fwd<O>, smem);
        if (e != RT_OK) return e;
        k_cfr_fwd<O><<<n_rx, CFR_THREADS, smem, ctx->stream>>>(S, rx_offsets_dev, (const float2*)a_dev, tau_dev,
                                                                (float2*)H_dev); RT_COUNT(ctx);
        RT_CK_LAUNCH(ctx);
        return RT_OK;
    });
}

extern "C" __attribute__((visibility("default"))) rt_status rt_cfr_backward(rt_ctx* ctx, const int64_t* rx_offsets_dev, int32_t n_rx, const double* tau_dev,
                                     double f_center_hz, double delta_f_hz, int32_t n_sub, const void* grad_H_dev,
                                     void* grad_a_dev) {
    CfrShape S;
    rt_status s = check_cfr(ctx, rx_offsets_dev, n_rx, tau_dev, n_sub, f_center_hz, delta_f_hz, S);
    if (s != RT_OK) return s;
    if (!grad_H_dev || !grad_a_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null device pointer");
    if (tc_supported(ctx, n_sub)) {
        double* part;
        unsigned int* ctr;
        s = rt_cfr_fused_scratch(ctx, n_rx, &part, &ctr);
        if (s != RT_OK) return s;
        TcSplit sp;
        s = split_setup(ctx, n_sub, &sp);
        if (s != RT_OK) return s;
        return launch_tc<5>(ctx, S, rx_offsets_dev, n_rx, nullptr, tau_dev, nullptr, nullptr,
                            (const float2*)grad_H_dev, nullptr, (float2*)grad_a_dev, nullptr, part, ctr, sp);
    }
    const size_t smem = fwd_smem(S) + (size_t)S.N * 8;
    s = set_smem(ctx, k_cfr_bwd, smem);
    if (s != RT_OK) return s;
    k_cfr_bwd<<<n_rx, CFR_THREADS, smem, ctx->stream>>>(S, rx_offsets_dev, tau_dev, (const float2*)grad_H_dev,
                                                        (float2*)grad_a_dev); RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}



extern "C" __attribute__((visibility("default"))) rt_status rt_cfr_power_mse_fused(rt_ctx* ctx, const int64_t* rx_offsets_dev, int32_t n_rx,
                                            const void* a_dev, const double* tau_dev, double f_center_hz,
                                            double delta_f_hz, int32_t n_sub, const float* target_power_dev,
                                            const float* rx_weight_dev, float* loss_dev, void* grad_a_dev,
                                            void* H_dev) {
    CfrShape S;
    rt_status s = check_cfr(ctx, rx_offsets_dev, n_rx, tau_dev, n_sub, f_center_hz, delta_f_hz, S);
    if (s != RT_OK) return s;
    if (!a_dev || !target_power_dev || !rx_weight_dev || !loss_dev || !grad_a_dev)
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "null device pointer");
    double* part;
    unsigned int* done;
    s = rt_cfr_fused_scratch(ctx, n_rx, &part, &done);
    if (s != RT_OK) return s;
    if (tc_supported(ctx, n_sub)) {
        // receivers with many paths are deferred and split over CTAs (mode 3)
        TcSplit sp;
        s = split_setup(ctx, n_sub, &sp);
        if (s != RT_OK) return s;
        return launch_tc<3>(ctx, S, rx_offsets_dev, n_rx, (const float2*)a_dev, tau_dev, target_power_dev,
                            rx_weight_dev, nullptr, loss_dev, (float2*)grad_a_dev, (float2*)H_dev, part, done, sp);
    }
    const size_t smem = fwd_smem(S) + (size_t)S.N * 8;
    return dispatch_opt(ctx, S.N, [&](auto opt) -> rt_status {
        constexpr int O = decltype(opt)::value;
        rt_status e = set_smem(ctx, k_cfr_fused<O>, smem);
        if (e != RT_OK) return e;
        k_cfr_fused<O><<<n_rx, CFR_THREADS, smem, ctx->stream>>>(
            S, rx_offsets_dev, n_rx, (const float2*)a_dev, tau_dev, target_power_dev, rx_weight_dev, loss_dev,
            (float2*)grad_a_dev, (float2*)H_dev, part, done); RT_COUNT(ctx);
        RT_CK_LAUNCH(ctx);
        return RT_OK;
    });
}

// ---------------------------------------------------------------------------
// Allocation-free variant of rt_cfr_power_mse_fused.
//
// Some callers cannot allocate device memory when they run the loss: a serving
// or training loop that reserved its whole memory budget up front (cudaMalloc
// there can fail, or stall the device while the driver finds memory), or a host
// program whose own memory manager owns every device buffer and forbids other
// code from calling the CUDA allocator.  This entry point serves them: its only
// working memory is the fixed array below, which every GPU that loads the
// library holds from load until process exit.  The caller still passes all
// inputs and outputs.
//
// Limits and sharing: at most RT_NOALLOC_MAX_RX receivers per call (one double
// of loss partial each, plus a completion counter: 512 KiB + 256 B in total).
// All calls on a device share the array and it keeps the last call's contents;
// the counter is cleared before every launch and every partial is rewritten, so
// sequential calls are independent, but two calls that overlap on the GPU (for
// example on two streams) race on it.
#define RT_NOALLOC_MAX_RX 65536

static __device__ __align__(256) unsigned char g_noalloc_scratch[RT_NOALLOC_MAX_RX * sizeof(double) + 256];

// Device address of g_noalloc_scratch per device.  In host code the array's
// name only stands in for the symbol; its address on a device comes from
// cudaGetSymbolAddress, asked with that device current.  It is asked again on
// every call made outside a stream capture, so an address cached before a device
// reset (after which the array may live elsewhere) is never used; inside a
// capture the address of the last call outside one is used, and a first call
// inside a capture is refused.
static void* g_noalloc_addr[64];
static std::mutex g_noalloc_mu;

static rt_status noalloc_scratch_address(rt_ctx* ctx, unsigned char** base) {
    if (ctx->device < 0 || ctx->device >= 64) return rt_fail(ctx, RT_ERR_UNSUPPORTED, "device index >= 64");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    RT_CK(ctx, cudaStreamIsCapturing(ctx->stream, &cap));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (cap != cudaStreamCaptureStatusNone && !g_noalloc_addr[ctx->device])
        return rt_fail(ctx, RT_ERR_INVALID_ARG,
                       "the first allocation-free call on a device must come before any stream capture");
    if (cap == cudaStreamCaptureStatusNone) {
        int cur = -1;
        RT_CK(ctx, cudaGetDevice(&cur));
        if (cur != ctx->device) RT_CK(ctx, cudaSetDevice(ctx->device));
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (cur != ctx->device) cudaSetDevice(cur);
        if (e != cudaSuccess) return rt_cuda_fail(ctx, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[ctx->device] = p;
    }
    *base = static_cast<unsigned char*>(g_noalloc_addr[ctx->device]);
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_cfr_power_mse_fused_noalloc(
    rt_ctx* ctx, const int64_t* rx_offsets_dev, int32_t n_rx, const void* a_dev, const double* tau_dev,
    double f_center_hz, double delta_f_hz, int32_t n_sub, const float* target_power_dev, const float* rx_weight_dev,
    float* loss_dev, void* grad_a_dev, void* H_dev) {
    CfrShape S;
    rt_status s = check_cfr(ctx, rx_offsets_dev, n_rx, tau_dev, n_sub, f_center_hz, delta_f_hz, S);
    if (s != RT_OK) return s;
    if (n_rx > RT_NOALLOC_MAX_RX)
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_rx = %d exceeds the allocation-free limit of %d receivers", n_rx,
                       RT_NOALLOC_MAX_RX);
    if (!a_dev || !target_power_dev || !rx_weight_dev || !loss_dev || !grad_a_dev)
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "null device pointer");
    unsigned char* base = nullptr;
    s = noalloc_scratch_address(ctx, &base);
    if (s != RT_OK) return s;
    double* part = reinterpret_cast<double*>(base);
    unsigned int* done = reinterpret_cast<unsigned int*>(base + RT_NOALLOC_MAX_RX * sizeof(double));
    RT_CK(ctx, cudaMemsetAsync(done, 0, 2 * sizeof(unsigned int), ctx->stream));
    if (tc_supported(ctx, n_sub))
        return launch_tc<2>(ctx, S, rx_offsets_dev, n_rx, (const float2*)a_dev, tau_dev, target_power_dev,
                            rx_weight_dev, nullptr, loss_dev, (float2*)grad_a_dev, (float2*)H_dev, part, done);
    const size_t smem = fwd_smem(S) + (size_t)S.N * 8;
    return dispatch_opt(ctx, S.N, [&](auto opt) -> rt_status {
        constexpr int O = decltype(opt)::value;
        rt_status e = set_smem(ctx, k_cfr_fused<O>, smem);
        if (e != RT_OK) return e;
        k_cfr_fused<O><<<n_rx, CFR_THREADS, smem, ctx->stream>>>(
            S, rx_offsets_dev, n_rx, (const float2*)a_dev, tau_dev, target_power_dev, rx_weight_dev, loss_dev,
            (float2*)grad_a_dev, (float2*)H_dev, part, done);
        RT_COUNT(ctx);
        RT_CK_LAUNCH(ctx);
        return RT_OK;
    });
}

extern "C" __attribute__((visibility("default"))) rt_status rt_set_wait_limit(rt_ctx* ctx, int32_t polls) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (polls < 0 || polls > TC_WAIT_LIMIT)
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "polls = %d outside [0, %d]", polls, TC_WAIT_LIMIT);
    ctx->wait_limit = polls;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_set_cfr_tensor_cores(rt_ctx* ctx, int32_t enable) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (enable != 0 && enable != 1) return rt_fail(ctx, RT_ERR_INVALID_ARG, "enable must be 0 or 1");
    ctx->cfr_tensor_cores = enable;
    return RT_OK;
}
