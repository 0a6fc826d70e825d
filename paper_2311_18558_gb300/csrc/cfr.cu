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

#include <cmath>
#include <mutex>
#include <type_traits>

#include "rt_internal.cuh"

namespace {

constexpr int CFR_THREADS = 256;
constexpr int CH = 32;   // paths per shared-memory chunk

struct PathPhase {
    float p0;     // frac(f_0 tau) in cycles
    float uhi;    // multiple of 2^-12, |uhi| <= 1/2
    float ulo;
};

__device__ __forceinline__ PathPhase path_phase(double tau, double f0, double df) {
    PathPhase p;
    double x = f0 * tau;
    p.p0 = (float)(x - rint(x));
    double u = df * tau;
    double ur = u - rint(u);
    double hi = rint(ur * 4096.0) * (1.0 / 4096.0);
    p.uhi = (float)hi;
    p.ulo = (float)(ur - hi);
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

extern "C" __attribute__((visibility("default"))) rt_status rt_cfr(rt_ctx* ctx, const int64_t* rx_offsets_dev, int32_t n_rx, const void* a_dev,
                            const double* tau_dev, double f_center_hz, double delta_f_hz, int32_t n_sub, void* H_dev) {
    CfrShape S;
    rt_status s = check_cfr(ctx, rx_offsets_dev, n_rx, tau_dev, n_sub, f_center_hz, delta_f_hz, S);
    if (s != RT_OK) return s;
    if (!a_dev || !H_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null device pointer");
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
    const size_t smem = fwd_smem(S) + (size_t)S.N * 8;
    s = set_smem(ctx, k_cfr_bwd, smem);
    if (s != RT_OK) return s;
    k_cfr_bwd<<<n_rx, CFR_THREADS, smem, ctx->stream>>>(S, rx_offsets_dev, tau_dev, (const float2*)grad_H_dev,
                                                        (float2*)grad_a_dev); RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

// Loss partials and completion counter of the fused kernel (api.cu).
rt_status rt_cfr_fused_scratch(rt_ctx* ctx, int R, double** part, unsigned int** done);

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
// cudaGetSymbolAddress, asked once per device with that device current.
static void* g_noalloc_addr[64];
static std::mutex g_noalloc_mu;

static rt_status noalloc_scratch_address(rt_ctx* ctx, unsigned char** base) {
    if (ctx->device < 0 || ctx->device >= 64) return rt_fail(ctx, RT_ERR_UNSUPPORTED, "device index >= 64");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[ctx->device]) {
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
    RT_CK(ctx, cudaMemsetAsync(done, 0, sizeof(unsigned int), ctx->stream));
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
