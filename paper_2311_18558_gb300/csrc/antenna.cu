// Trainable antenna patterns (arXiv 2311.18558, Sec. III-B) on traced paths.
//
// A pattern is a mixture of M spherical Gaussians (von Mises-Fisher lobes):
//   G(r) = 4 pi eta sum_m w_m exp(lambda_m mu_m . r) / a_m,
//   a_m  = (2 pi / lambda_m) (exp(lambda_m) - exp(-lambda_m)),
// (the factor 4 pi makes the integral over the sphere 4 pi eta, as the
// normalisation of Sec. II-C asks), and the vertical polarization model
// C = [sqrt(G), 0] (zeta = 0) scales a path's coefficient by
// sqrt(G_T(k_1) G_R(-k_{q+1})), k_1 the departure and -k_{q+1} the arrival
// direction stored in the path records.  A lobe is evaluated as
//   exp(lambda c) / a = lambda exp(lambda (c - 1)) / (2 pi (1 - exp(-2 lambda))),
// which neither overflows for sharp lobes nor loses precision for flat ones.
// Packed pattern: 1 + 5M floats {eta, then per lobe w, lambda, mu_x, mu_y, mu_z}.
#include <cuda_runtime.h>

#include <algorithm>

#include "rt_internal.cuh"

namespace {

constexpr int ANT_MAX_LOBES = 8;
constexpr int ANT_THREADS = 256;
constexpr float FOUR_PI = 12.566370614359172f;

// exp(lambda c) / a(lambda)
__device__ __forceinline__ float lobe(float lam, float c) {
    lam = fmaxf(lam, 1e-20f);
    return lam * expf(lam * (c - 1.0f)) / (6.283185307179586f * -expm1f(-2.0f * lam));
}

// coth(lambda) - 1 / lambda (series below 1e-2, where the difference cancels)
__device__ __forceinline__ float coth_minus_inv(float lam) {
    if (lam < 1e-2f) return lam * (1.0f / 3.0f) - lam * lam * lam * (1.0f / 45.0f);
    return 1.0f / tanhf(lam) - 1.0f / lam;
}

__device__ __forceinline__ float gain_of(const float* pat, int M, float4 r) {
    float g = 0.0f;
    for (int m = 0; m < M; ++m) {
        const float* l = pat + 1 + 5 * m;
        g += l[0] * lobe(l[1], l[2] * r.x + l[3] * r.y + l[4] * r.z);
    }
    return FOUR_PI * pat[0] * g;
}

__global__ void __launch_bounds__(ANT_THREADS) k_antenna_apply(int64_t P, const float4* __restrict__ dir,
                                                               const float* __restrict__ tx, int mt,
                                                               const float* __restrict__ rx, int mr,
                                                               const float2* __restrict__ a_in, float2* __restrict__ a_out,
                                                               float* __restrict__ gt_out, float* __restrict__ gr_out) {
    __shared__ float s_tx[1 + 5 * ANT_MAX_LOBES], s_rx[1 + 5 * ANT_MAX_LOBES];
    if (tx)
        for (int k = threadIdx.x; k < 1 + 5 * mt; k += blockDim.x) s_tx[k] = tx[k];
    if (rx)
        for (int k = threadIdx.x; k < 1 + 5 * mr; k += blockDim.x) s_rx[k] = rx[k];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const float gt = tx ? gain_of(s_tx, mt, __ldg(dir + i)) : 1.0f;
        const float gr = rx ? gain_of(s_rx, mr, __ldg(dir + P + i)) : 1.0f;
        const float s = sqrtf(gt * gr);
        const float2 a = a_in[i];
        a_out[i] = make_float2(s * a.x, s * a.y);
        if (gt_out) gt_out[i] = gt;
        if (gr_out) gr_out[i] = gr;
    }
}

// dL/da_in = sqrt(G_T G_R) dL/da_out (a real scale)
__global__ void k_antenna_grad_a(int64_t P, const float* __restrict__ gt, const float* __restrict__ gr,
                                 const float2* __restrict__ g_out, float2* __restrict__ g_in) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const float s = sqrtf((gt ? gt[i] : 1.0f) * (gr ? gr[i] : 1.0f));
        const float2 g = g_out[i];
        g_in[i] = make_float2(s * g.x, s * g.y);
    }
}

// Gradient of one pattern (side 0: transmit, directions dir[0..P); side 1:
// receive, dir[P..2P)):  dL/dG = Re(conj(g) a_out) / (2 G) per path, then
//   dG/deta = G / eta, dG/dw_m = 4 pi eta L_m, dG/dlambda_m = 4 pi eta w_m L_m (c_m - coth lambda_m + 1/lambda_m),
//   dG/dmu_m = 4 pi eta w_m L_m lambda_m r,  L_m = exp(lambda_m c_m) / a_m, c_m = mu_m . r.
// Per-thread accumulators over the grid-stride paths, one block reduction,
// accumulated (+=) into grad (1 + 5M floats).
template <int M>
__global__ void __launch_bounds__(ANT_THREADS) k_antenna_grad_pattern(int64_t P, const float4* __restrict__ dir,
                                                                      const float* __restrict__ pat,
                                                                      const float* __restrict__ G,
                                                                      const float2* __restrict__ a_out,
                                                                      const float2* __restrict__ g_out,
                                                                      float* __restrict__ grad) {
    constexpr int NP = 1 + 5 * M;
    __shared__ float s_pat[NP], s_acc[NP];
    for (int k = threadIdx.x; k < NP; k += blockDim.x) {
        s_pat[k] = pat[k];
        s_acc[k] = 0.0f;
    }
    __syncthreads();
    float acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = 0.0f;
    const float eta = s_pat[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 g = g_out[i], a = a_out[i];
        const float Gi = G[i];
        if (!(Gi > 0.0f)) continue;
        const float dLdG = 0.5f * (g.x * a.x + g.y * a.y) / Gi;
        const float4 r = __ldg(dir + i);
        float sum = 0.0f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const float w = s_pat[1 + 5 * m], lam = s_pat[2 + 5 * m];
            const float c = s_pat[3 + 5 * m] * r.x + s_pat[4 + 5 * m] * r.y + s_pat[5 + 5 * m] * r.z;
            const float L = lobe(lam, c);
            const float base = FOUR_PI * eta * L * dLdG;
            sum += w * L;
            acc[1 + 5 * m] += base;
            acc[2 + 5 * m] += w * base * (c - coth_minus_inv(lam));
            const float bm = w * base * lam;
            acc[3 + 5 * m] += bm * r.x;
            acc[4 + 5 * m] += bm * r.y;
            acc[5 + 5 * m] += bm * r.z;
        }
        acc[0] += FOUR_PI * sum * dLdG;
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        float v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0.0f) atomicAdd(&s_acc[k], v);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NP; k += blockDim.x)
        if (s_acc[k] != 0.0f) atomicAdd(grad + k, s_acc[k]);
}

int ant_grid(const rt_ctx* ctx, int64_t P) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((P + ANT_THREADS - 1) / ANT_THREADS, (int64_t)ctx->num_sms * 8));
}

template <int M>
void launch_grad(rt_ctx* ctx, int64_t P, const float4* dir, const float* pat, const float* G, const float2* a_out,
                 const float2* g_out, float* grad) {
    k_antenna_grad_pattern<M><<<ant_grid(ctx, P), ANT_THREADS, 0, ctx->stream>>>(P, dir, pat, G, a_out, g_out, grad);
    RT_COUNT(ctx);
}

rt_status grad_dispatch(rt_ctx* ctx, int M, int64_t P, const float4* dir, const float* pat, const float* G,
                        const float2* a_out, const float2* g_out, float* grad) {
    switch (M) {
        case 1: launch_grad<1>(ctx, P, dir, pat, G, a_out, g_out, grad); break;
        case 2: launch_grad<2>(ctx, P, dir, pat, G, a_out, g_out, grad); break;
        case 3: launch_grad<3>(ctx, P, dir, pat, G, a_out, g_out, grad); break;
        case 4: launch_grad<4>(ctx, P, dir, pat, G, a_out, g_out, grad); break;
        case 5: launch_grad<5>(ctx, P, dir, pat, G, a_out, g_out, grad); break;
        case 6: launch_grad<6>(ctx, P, dir, pat, G, a_out, g_out, grad); break;
        case 7: launch_grad<7>(ctx, P, dir, pat, G, a_out, g_out, grad); break;
        case 8: launch_grad<8>(ctx, P, dir, pat, G, a_out, g_out, grad); break;
        default: return rt_fail(ctx, RT_ERR_INVALID_ARG, "a pattern has 1 to %d lobes", ANT_MAX_LOBES);
    }
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

rt_status check_pattern(rt_ctx* ctx, const float* pat, int M) {
    if (pat && (M < 1 || M > ANT_MAX_LOBES))
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "a pattern has 1 to %d lobes", ANT_MAX_LOBES);
    return RT_OK;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) rt_status rt_antenna_apply(
    rt_ctx* ctx, const rt_paths* paths, const float* tx_pattern_dev, int32_t tx_lobes, const float* rx_pattern_dev,
    int32_t rx_lobes, const void* a_dev, void* a_out_dev, float* gain_tx_dev, float* gain_rx_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!paths || !a_dev || !a_out_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    RT_REQUIRE_RESOLVED(ctx, paths);
    rt_status s = check_pattern(ctx, tx_pattern_dev, tx_lobes);
    if (s != RT_OK) return s;
    s = check_pattern(ctx, rx_pattern_dev, rx_lobes);
    if (s != RT_OK) return s;
    if (paths->P == 0) return RT_OK;
    k_antenna_apply<<<ant_grid(ctx, paths->P), ANT_THREADS, 0, ctx->stream>>>(
        paths->P, paths->d_dir, tx_pattern_dev, tx_lobes, rx_pattern_dev, rx_lobes, (const float2*)a_dev,
        (float2*)a_out_dev, gain_tx_dev, gain_rx_dev);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_antenna_apply_backward(
    rt_ctx* ctx, const rt_paths* paths, const float* tx_pattern_dev, int32_t tx_lobes, const float* rx_pattern_dev,
    int32_t rx_lobes, const void* a_out_dev, const float* gain_tx_dev, const float* gain_rx_dev,
    const void* grad_out_dev, void* grad_a_dev, float* grad_tx_dev, float* grad_rx_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!paths || !a_out_dev || !grad_out_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    RT_REQUIRE_RESOLVED(ctx, paths);
    if ((tx_pattern_dev && !gain_tx_dev) || (rx_pattern_dev && !gain_rx_dev))
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "the forward gains of every given pattern are required");
    rt_status s = check_pattern(ctx, tx_pattern_dev, tx_lobes);
    if (s != RT_OK) return s;
    s = check_pattern(ctx, rx_pattern_dev, rx_lobes);
    if (s != RT_OK) return s;
    const int64_t P = paths->P;
    if (P == 0) return RT_OK;
    const float2* go = (const float2*)grad_out_dev;
    const float2* ao = (const float2*)a_out_dev;
    if (grad_a_dev) {
        k_antenna_grad_a<<<ant_grid(ctx, P), ANT_THREADS, 0, ctx->stream>>>(
            P, tx_pattern_dev ? gain_tx_dev : nullptr, rx_pattern_dev ? gain_rx_dev : nullptr, go, (float2*)grad_a_dev);
        RT_COUNT(ctx);
        RT_CK_LAUNCH(ctx);
    }
    if (tx_pattern_dev && grad_tx_dev) {
        s = grad_dispatch(ctx, tx_lobes, P, paths->d_dir, tx_pattern_dev, gain_tx_dev, ao, go, grad_tx_dev);
        if (s != RT_OK) return s;
    }
    if (rx_pattern_dev && grad_rx_dev) {
        s = grad_dispatch(ctx, rx_lobes, P, paths->d_dir + P, rx_pattern_dev, gain_rx_dev, ao, go, grad_rx_dev);
        if (s != RT_OK) return s;
    }
    return RT_OK;
}
