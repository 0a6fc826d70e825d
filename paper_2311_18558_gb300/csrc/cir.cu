// The paper's calibration loss and metrics on the CFR (arXiv 2311.18558):
//   CIR by N-point IDFT (Sec. II-A):
//     h[l] = N^-1/2 sum_n H[n] exp(+j 2 pi n l / N),  n, l = -N/2 .. N/2-1,
//   total channel gain P = sum_l |h[l]|^2 (Eq. channel_gain), RMS delay spread
//   tau_RMS = sqrt(sum_l ((l - tau_bar) / W)^2 p_l / P), tau_bar = sum_l l p_l / P
//   (Eq. delay_spread, W = N df), the per-example loss
//   SMAPE(tau_RMS, tau^_RMS) + SMAPE(alpha P, P^) with SMAPE(x, y) = |x - y| / (x + y)
//   (Eq. smape, Eq. loss), the power scale alpha^ = sum P P^ / sum P^2 and its
//   moving average (Eq. alpha_hat, scaling_param), and ALE / RAE (Sec. IV-C).
//
// One CTA per receiver (persistent over receivers): the row's N-point transform
// runs in shared memory as a radix-2 Stockham FFT (self-sorting, ping-pong
// buffers).  The centred index ranges are handled by sign alternation:
// with n' = n + N/2, l' = l + N/2, exp(j 2 pi n l / N) =
// (-1)^(n' + l' + N/2) exp(j 2 pi n' l' / N).  Moments are accumulated in FP64
// in two passes (P and tau_bar first, then the central second moment), so the
// spread does not come from a difference of large sums.
// Readings: a CIR with P = 0 has tau_RMS = 0 and no gradient through its delay
// terms; SMAPE(0, 0) = 0; alpha scales the measured powers and carries no gradient.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "rt_internal.cuh"

rt_status rt_cfr_fused_scratch(rt_ctx* ctx, int R, double** part, unsigned int** done);

namespace {

constexpr int CIR_THREADS = 256;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place (ping-pong) radix-2 Stockham transform of a[0..N) with kernel
// exp(SIGN j 2 pi k m / N), unnormalised; returns the buffer holding the result.
template <int SIGN>
__device__ float2* stockham(float2* a, float2* b, int N) {
    const int half = N >> 1;
    for (int Ns = 1; Ns < N; Ns <<= 1) {
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            const int m = j & (Ns - 1);
            float s, c;
            sincospif((float)(SIGN * m) / (float)Ns, &s, &c);
            const float2 v0 = a[j];
            const float2 v1 = cmulf(a[j + half], make_float2(c, s));
            const int d = ((j - m) << 1) + m;
            b[d] = make_float2(v0.x + v1.x, v0.y + v1.y);
            b[d + Ns] = make_float2(v0.x - v1.x, v0.y - v1.y);
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
    }
    return a;
}

// Loads row r of H with the input sign (-1)^n', runs the inverse transform and
// applies the output sign (-1)^(l' + N/2) / sqrt(N): returns the buffer with h.
__device__ float2* cir_row(const float2* __restrict__ H, int64_t r, int N, float2* a, float2* b) {
    const float2* row = H + r * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const float2 v = row[k];
        a[k] = (k & 1) ? make_float2(-v.x, -v.y) : v;
    }
    __syncthreads();
    float2* h = stockham<+1>(a, b, N);
    const float sc = rsqrtf((float)N);
    const int flip = (N >> 1) & 1;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const float s = ((k + flip) & 1) ? -sc : sc;
        h[k] = make_float2(s * h[k].x, s * h[k].y);
    }
    __syncthreads();
    return h;
}

// Block sum of a double (all threads get the result); red holds blockDim/32 doubles.
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

struct CirStats {
    double P, tbar, trms;   // tbar in taps, trms in seconds
};

// P, tau_bar and tau_RMS of the CIR held in h (two passes over the buffer).
__device__ CirStats cir_stats(const float2* h, int N, double W, double* red) {
    double p0 = 0.0, p1 = 0.0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const double p = (double)h[k].x * h[k].x + (double)h[k].y * h[k].y;
        p0 += p;
        p1 += p * (double)(k - (N >> 1));
    }
    CirStats st;
    st.P = block_sum(p0, red);
    const double S1 = block_sum(p1, red);
    st.tbar = st.P > 0.0 ? S1 / st.P : 0.0;
    double p2 = 0.0;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const double p = (double)h[k].x * h[k].x + (double)h[k].y * h[k].y;
        const double d = (double)(k - (N >> 1)) - st.tbar;
        p2 += p * d * d;
    }
    const double S2 = block_sum(p2, red);
    st.trms = st.P > 0.0 ? sqrt(fmax(S2 / st.P, 0.0)) / W : 0.0;
    return st;
}

__device__ __forceinline__ double smape(double x, double y) {
    const double s = x + y;
    return s > 0.0 ? fabs(x - y) / s : 0.0;
}
__device__ __forceinline__ double smape_dy(double x, double y) {   // d SMAPE / dy
    const double s = x + y;
    if (!(s > 0.0)) return 0.0;
    const double sg = y > x ? 1.0 : (y < x ? -1.0 : 0.0);
    return 2.0 * x * sg / (s * s);
}

__global__ void __launch_bounds__(CIR_THREADS) k_cir(const float2* __restrict__ H, int R, int N, float2* __restrict__ h_out) {
    extern __shared__ float2 sbuf[];
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        float2* h = cir_row(H, r, N, sbuf, sbuf + N);
        for (int k = threadIdx.x; k < N; k += blockDim.x) h_out[(int64_t)r * N + k] = h[k];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(CIR_THREADS) k_cir_stats(const float2* __restrict__ H, int R, int N, double W,
                                                           float* __restrict__ P_out, float* __restrict__ t_out) {
    extern __shared__ float2 sbuf[];
    __shared__ double red[CIR_THREADS / 32];
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        float2* h = cir_row(H, r, N, sbuf, sbuf + N);
        const CirStats st = cir_stats(h, N, W, red);
        if (threadIdx.x == 0) {
            if (P_out) P_out[r] = (float)st.P;
            if (t_out) t_out[r] = (float)st.trms;
        }
        __syncthreads();
    }
}

// alpha^ = sum P P^ / sum P^2 (one block), then the moving average into
// state = {alpha, initialised}.
__global__ void k_power_scale(const float* __restrict__ Pm, const float* __restrict__ Pp, int n, float decay,
                              float* state) {
    __shared__ double red[CIR_THREADS / 32];
    double num = 0.0, den = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        num += (double)Pm[k] * Pp[k];
        den += (double)Pm[k] * Pm[k];
    }
    num = block_sum(num, red);
    den = block_sum(den, red);
    if (threadIdx.x == 0) {
        const double ah = den > 0.0 ? num / den : 1.0;
        const double prev = state[1] != 0.0f ? (double)state[0] : ah;   // alpha_0 = alpha^_1
        state[0] = (float)(decay * prev + (1.0 - decay) * ah);
        state[1] = 1.0f;
    }
}

// Loss of Eq. loss for every receiver (partials, summed by the last CTA in
// receiver order) and g_H = dL/dRe H + j dL/dIm H:
//   dL/dp_l = dL/dP^ + dL/dtau^ ((l - tau_bar)^2 / W^2 - tau^2) / (2 tau^ P^),
//   g_h = 2 dL/dp_l h_l,  g_H[n] = N^-1/2 sum_l g_h[l] exp(-j 2 pi n l / N).
__global__ void __launch_bounds__(CIR_THREADS) k_cir_loss(const float2* __restrict__ H, int R, int N, double W,
                                                          const float* __restrict__ Pm, const float* __restrict__ tm,
                                                          const float* __restrict__ alpha_state, float* __restrict__ loss,
                                                          float2* __restrict__ gH, float* __restrict__ P_out,
                                                          float* __restrict__ t_out, double* __restrict__ part,
                                                          unsigned int* __restrict__ ctr) {
    extern __shared__ float2 sbuf[];
    __shared__ double red[CIR_THREADS / 32];
    __shared__ bool s_last;
    const double alpha = alpha_state ? (double)alpha_state[0] : 1.0;
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        float2* h = cir_row(H, r, N, sbuf, sbuf + N);
        float2* other = h == sbuf ? sbuf + N : sbuf;
        const CirStats st = cir_stats(h, N, W, red);
        const double pm = alpha * (double)Pm[r], taum = (double)tm[r];
        if (threadIdx.x == 0) {
            part[r] = smape(taum, st.trms) + smape(pm, st.P);
            if (P_out) P_out[r] = (float)st.P;
            if (t_out) t_out[r] = (float)st.trms;
        }
        const double dP = smape_dy(pm, st.P) / R;
        const bool spread_ok = st.P > 0.0 && st.trms > 0.0;
        const double dT = spread_ok ? smape_dy(taum, st.trms) / R : 0.0;
        const double cT = spread_ok ? dT / (2.0 * st.trms * st.P) : 0.0;
        const double t2 = st.trms * st.trms;
        const float sc = rsqrtf((float)N);
        // adjoint of the centred IDFT: g_H[n'] = (-1)^n' (-1)^(N/2) N^-1/2
        // sum_l' (-1)^l' g_h[l'] exp(-j 2 pi n' l' / N); the input carries
        // g_h[l'] = 2 dL/dp_l h[l'] times (-1)^(l' + N/2) / sqrt(N)
        const int flip = (N >> 1) & 1;
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
            const double d = (double)(k - (N >> 1)) - st.tbar;
            const double g = 2.0 * (dP + cT * (d * d / (W * W) - t2));
            const float s = (float)g * (((k + flip) & 1) ? -sc : sc);
            other[k] = make_float2(s * h[k].x, s * h[k].y);
        }
        __syncthreads();
        float2* gt = stockham<-1>(other, h, N);
        float2* row = gH + (int64_t)r * N;
        for (int k = threadIdx.x; k < N; k += blockDim.x) {
            const float s = (k & 1) ? -1.0f : 1.0f;
            row[k] = make_float2(s * gt[k].x, s * gt[k].y);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ctr, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        double s = 0.0;
        for (int k = threadIdx.x; k < R; k += blockDim.x) s += ((volatile double*)part)[k];
        s = block_sum(s, red);
        if (threadIdx.x == 0) {
            *loss = (float)(s / R);
            ctr[0] = 0u;
        }
    }
}

__global__ void k_cir_metrics(const float* __restrict__ Pm, const float* __restrict__ tm, const float* __restrict__ Pp,
                              const float* __restrict__ tp, int n, const float* __restrict__ alpha_state,
                              float* __restrict__ ale, float* __restrict__ rae) {
    const double alpha = alpha_state ? (double)alpha_state[0] : 1.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (ale) ale[k] = (float)fabs(10.0 * log10(alpha * (double)Pm[k]) - 10.0 * log10((double)Pp[k]));
        if (rae) rae[k] = (float)(fabs((double)tm[k] - (double)tp[k]) / (double)tm[k]);
    }
}

bool pow2_ok(int n) { return n >= 2 && n <= 4096 && (n & (n - 1)) == 0; }

template <typename K>
rt_status cir_launch_attrs(rt_ctx* ctx, K kernel, size_t smem) {
    if (smem > 48 * 1024) RT_CK(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return RT_OK;
}

int cir_grid(const rt_ctx* ctx, int R) { return std::max(1, std::min(R, ctx->num_sms * 8)); }

}  // namespace

extern "C" __attribute__((visibility("default"))) rt_status rt_cir(rt_ctx* ctx, const void* H_dev, int32_t n_rx,
                                                                   int32_t n_sub, void* h_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!H_dev || !h_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null device pointer");
    if (n_rx < 1 || !pow2_ok(n_sub)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_rx >= 1 and n_sub a power of two in [2, 4096]");
    const size_t smem = (size_t)2 * n_sub * sizeof(float2);
    rt_status s = cir_launch_attrs(ctx, k_cir, smem);
    if (s != RT_OK) return s;
    k_cir<<<cir_grid(ctx, n_rx), CIR_THREADS, smem, ctx->stream>>>((const float2*)H_dev, n_rx, n_sub, (float2*)h_dev);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_cir_stats(rt_ctx* ctx, const void* H_dev, int32_t n_rx,
                                                                         int32_t n_sub, double delta_f_hz, float* P_dev,
                                                                         float* tau_rms_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!H_dev || (!P_dev && !tau_rms_dev)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null device pointer");
    if (n_rx < 1 || !pow2_ok(n_sub)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_rx >= 1 and n_sub a power of two in [2, 4096]");
    if (!(delta_f_hz > 0.0) || !std::isfinite(delta_f_hz)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "delta_f must be > 0");
    const size_t smem = (size_t)2 * n_sub * sizeof(float2);
    rt_status s = cir_launch_attrs(ctx, k_cir_stats, smem);
    if (s != RT_OK) return s;
    k_cir_stats<<<cir_grid(ctx, n_rx), CIR_THREADS, smem, ctx->stream>>>((const float2*)H_dev, n_rx, n_sub,
                                                                         n_sub * delta_f_hz, P_dev, tau_rms_dev);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_power_scale_ema(rt_ctx* ctx, const float* P_meas_dev,
                                                                               const float* P_pred_dev, int32_t n,
                                                                               float decay, float* state_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!P_meas_dev || !P_pred_dev || !state_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null device pointer");
    if (n < 1) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n must be >= 1");
    if (!(decay >= 0.0f && decay < 1.0f)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "decay must be in [0, 1)");
    k_power_scale<<<1, CIR_THREADS, 0, ctx->stream>>>(P_meas_dev, P_pred_dev, n, decay, state_dev);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_delay_spread_power_loss(
    rt_ctx* ctx, const void* H_dev, int32_t n_rx, int32_t n_sub, double delta_f_hz, const float* P_meas_dev,
    const float* tau_meas_dev, const float* alpha_state_dev, float* loss_dev, void* grad_H_dev, float* P_pred_dev,
    float* tau_pred_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!H_dev || !P_meas_dev || !tau_meas_dev || !loss_dev || !grad_H_dev)
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "null device pointer");
    if (n_rx < 1 || !pow2_ok(n_sub)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_rx >= 1 and n_sub a power of two in [2, 4096]");
    if (!(delta_f_hz > 0.0) || !std::isfinite(delta_f_hz)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "delta_f must be > 0");
    double* part;
    unsigned int* ctr;
    rt_status s = rt_cfr_fused_scratch(ctx, n_rx, &part, &ctr);
    if (s != RT_OK) return s;
    const size_t smem = (size_t)2 * n_sub * sizeof(float2);
    s = cir_launch_attrs(ctx, k_cir_loss, smem);
    if (s != RT_OK) return s;
    k_cir_loss<<<cir_grid(ctx, n_rx), CIR_THREADS, smem, ctx->stream>>>(
        (const float2*)H_dev, n_rx, n_sub, n_sub * delta_f_hz, P_meas_dev, tau_meas_dev, alpha_state_dev, loss_dev,
        (float2*)grad_H_dev, P_pred_dev, tau_pred_dev, part, ctr);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_cir_metrics(rt_ctx* ctx, const float* P_meas_dev,
                                                                           const float* tau_meas_dev,
                                                                           const float* P_pred_dev,
                                                                           const float* tau_pred_dev, int32_t n,
                                                                           const float* alpha_state_dev, float* ale_dev,
                                                                           float* rae_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!P_meas_dev || !tau_meas_dev || !P_pred_dev || !tau_pred_dev || (!ale_dev && !rae_dev))
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "null device pointer");
    if (n < 1) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n must be >= 1");
    k_cir_metrics<<<std::max(1, std::min((n + 255) / 256, ctx->num_sms * 4)), 256, 0, ctx->stream>>>(
        P_meas_dev, tau_meas_dev, P_pred_dev, tau_pred_dev, n, alpha_state_dev, ale_dev, rae_dev);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}
