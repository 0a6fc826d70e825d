// Neural materials (arXiv 2311.18558, Sec. III-D): an MLP maps the positional
// encoding of a point to (sigma, eps_r).  Here the point is each triangle's
// centroid, normalised to the unit cube by the scene's bounding box
// (p_bar = (c - b) / Delta_b, Delta_b its longest edge), encoded as
// [p_bar, sin(2^k pi p_bar), cos(2^k pi p_bar), k = 1..6] (39 features, Eq.
// pos_encoding), then 39 -> 128 -> 128 -> 128 -> 2 with ReLU, and
// sigma = exp(o_1), eps_r = 1 + exp(o_2) (Eq. trainable_materials_1/2).
//
// Precision: weights and every layer input are BF16; products are summed in
// FP32.  The contraction runs on the FP32 pipes (the tensor cores are used by
// the CFR only): each CTA keeps all weights in shared memory (76 KB) and walks
// tiles of 64 rows persistently; a thread owns a 4 x 8 block of a layer output.
//
// Backward: k_mlp_bwd_data recomputes nothing -- it reads the BF16 layer inputs
// saved by the forward pass, forms dL/do from dL/deps_r and dL/dsigma, and runs
// dZ_l = (dZ_{l+1} W_{l+1}^T) * relu'(z_l) down the layers, writing dZ_l (FP32);
// k_mlp_bwd_weights forms dW_l = A_l^T dZ_l and db_l with split-K and atomics.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "rt_internal.cuh"

namespace {

constexpr int IN = 39, INP = 40, WID = 128, OUT = 2;
constexpr int OFF_W1 = 0, OFF_W2 = INP * WID, OFF_W3 = OFF_W2 + WID * WID, OFF_W4 = OFF_W3 + WID * WID;
constexpr int NW = OFF_W4 + WID * OUT;                 // 38144 weights
constexpr int OFF_B1 = 0, OFF_B2 = WID, OFF_B3 = 2 * WID, OFF_B4 = 3 * WID;
constexpr int NB = 3 * WID + OUT;                      // 386 biases
constexpr int ACT = INP + 3 * WID;                     // saved layer inputs per row (424)
constexpr int TILE = 64;                               // rows per tile
constexpr int THREADS = 256;

struct MlpScene {
    const float4* tri_v;
    int n;
    float cx, cy, cz, inv_size;
};

__device__ __forceinline__ float bf(__nv_bfloat16 v) { return __bfloat162float(v); }

// Positional encoding feature f of row (point) p_bar, f < 40 (feature 39 = 0).
__device__ __forceinline__ float pe_feature(float3 pb, int f) {
    if (f < 3) return f == 0 ? pb.x : (f == 1 ? pb.y : pb.z);
    if (f >= IN) return 0.0f;
    int g = f - 3;                 // 6 features per frequency: sin x, y, z, cos x, y, z
    int k = g / 6 + 1, r = g % 6;
    float c = (r % 3) == 0 ? pb.x : ((r % 3) == 1 ? pb.y : pb.z);
    float s, co;
    sincospif((float)(1 << k) * c, &s, &co);   // sin/cos(2^k pi c)
    return r < 3 ? s : co;
}

// out[r][c] (FP32 registers, 4 rows x 8 cols per thread) = At^T W for K inputs,
// with At the transposed BF16 activations [K][TILE] and W BF16 [K][WID].
__device__ __forceinline__ void tile_gemm(const __nv_bfloat16* At, const __nv_bfloat16* W, int K, int r0, int c0,
                                          float (&acc)[4][8]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    for (int k = 0; k < K; ++k) {
        uint2 av = *reinterpret_cast<const uint2*>(At + k * TILE + r0);
        uint4 wv = *reinterpret_cast<const uint4*>(W + k * WID + c0);
        const __nv_bfloat16* a = reinterpret_cast<const __nv_bfloat16*>(&av);
        const __nv_bfloat16* w = reinterpret_cast<const __nv_bfloat16*>(&wv);
        float af[4], wf[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) af[i] = bf(a[i]);
#pragma unroll
        for (int j = 0; j < 8; ++j) wf[j] = bf(w[j]);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(af[i], wf[j], acc[i][j]);
    }
}

__global__ void __launch_bounds__(THREADS) k_mlp_fwd(MlpScene S, const __nv_bfloat16* __restrict__ w,
                                                     const float* __restrict__ b, float* __restrict__ eps,
                                                     float* __restrict__ sig, __nv_bfloat16* __restrict__ act) {
    extern __shared__ float4 smem4[];
    __nv_bfloat16* sW = reinterpret_cast<__nv_bfloat16*>(smem4);      // NW
    __nv_bfloat16* sA = sW + NW;                                      // [WID][TILE] transposed input
    __nv_bfloat16* sB = sA + WID * TILE;                              // [WID][TILE] transposed output
    for (int i = threadIdx.x; i < NW / 8; i += THREADS)
        reinterpret_cast<uint4*>(sW)[i] = __ldg(reinterpret_cast<const uint4*>(w) + i);
    const int tid = threadIdx.x;
    const int r0 = (tid / 16) * 4, c0 = (tid % 16) * 8;
    const int n_tiles = (S.n + TILE - 1) / TILE;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int row0 = tile * TILE;
        __syncthreads();
        // layer-1 input: encoding of the normalised centroids, rounded to BF16
        for (int e = tid; e < TILE * INP; e += THREADS) {
            int rr = e % TILE, f = e / TILE;
            int t = row0 + rr;
            float v = 0.0f;
            if (t < S.n) {
                float4 p0 = __ldg(S.tri_v + 3 * t), p1 = __ldg(S.tri_v + 3 * t + 1), p2 = __ldg(S.tri_v + 3 * t + 2);
                float3 pb = make_float3(((p0.x + p1.x + p2.x) * (1.0f / 3.0f) - S.cx) * S.inv_size,
                                        ((p0.y + p1.y + p2.y) * (1.0f / 3.0f) - S.cy) * S.inv_size,
                                        ((p0.z + p1.z + p2.z) * (1.0f / 3.0f) - S.cz) * S.inv_size);
                v = pe_feature(pb, f);
            }
            sA[f * TILE + rr] = __float2bfloat16_rn(v);
        }
        __syncthreads();
        __nv_bfloat16* in = sA;
        __nv_bfloat16* outb = sB;
        int K = INP;
        const int offw[3] = {OFF_W1, OFF_W2, OFF_W3};
        const int offb[3] = {OFF_B1, OFF_B2, OFF_B3};
        const int offa[3] = {0, INP, INP + WID};
        for (int l = 0; l < 3; ++l) {
            if (act) {   // save this layer's BF16 input for the backward pass
                for (int e = tid; e < TILE * K; e += THREADS) {
                    int rr = e / K, f = e % K;
                    if (row0 + rr < S.n) act[(int64_t)(row0 + rr) * ACT + offa[l] + f] = in[f * TILE + rr];
                }
            }
            float acc[4][8];
            tile_gemm(in, sW + offw[l], K, r0, c0, acc);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float bj = __ldg(b + offb[l] + c0 + j);
#pragma unroll
                for (int i = 0; i < 4; ++i) outb[(c0 + j) * TILE + r0 + i] = __float2bfloat16_rn(fmaxf(acc[i][j] + bj, 0.0f));
            }
            __syncthreads();
            __nv_bfloat16* t = in;
            in = outb;
            outb = t;
            K = WID;
        }
        if (act) {
            for (int e = tid; e < TILE * WID; e += THREADS) {
                int rr = e / WID, f = e % WID;
                if (row0 + rr < S.n) act[(int64_t)(row0 + rr) * ACT + INP + 2 * WID + f] = in[f * TILE + rr];
            }
        }
        // output layer (128 -> 2) and the material transforms
        if (tid < TILE * OUT) {
            int rr = tid / OUT, o = tid % OUT;
            float s = __ldg(b + OFF_B4 + o);
            for (int k = 0; k < WID; ++k) s = fmaf(bf(in[k * TILE + rr]), bf(sW[OFF_W4 + k * OUT + o]), s);
            int t = row0 + rr;
            if (t < S.n) {
                if (o == 0) sig[t] = expf(s);
                else eps[t] = 1.0f + expf(s);
            }
        }
    }
}

// Backward through the layers for tiles of 64 rows; writes dZ_l (FP32, row
// major [n][3][WID]) and accumulates dW4, db4.
__global__ void __launch_bounds__(THREADS) k_mlp_bwd_data(int n, const __nv_bfloat16* __restrict__ w,
                                                          const __nv_bfloat16* __restrict__ act,
                                                          const float* __restrict__ eps, const float* __restrict__ sig,
                                                          const float* __restrict__ geps,
                                                          const float* __restrict__ gsig, float* __restrict__ dz,
                                                          float* __restrict__ gw, float* __restrict__ gb) {
    extern __shared__ float4 smem4[];
    __nv_bfloat16* sWt = reinterpret_cast<__nv_bfloat16*>(smem4);   // W2^T, W3^T: [out][in]
    float* sG = reinterpret_cast<float*>(sWt + 2 * WID * WID);     // [WID][TILE] dZ (transposed)
    float* sH = sG + WID * TILE;                                    // [WID][TILE] next dZ
    float* sO = sH + WID * TILE;                                    // [TILE][OUT] dL/do
    __nv_bfloat16* sW4 = reinterpret_cast<__nv_bfloat16*>(sO + TILE * OUT);   // [WID][OUT]
    for (int i = threadIdx.x; i < WID * WID; i += THREADS) {
        int in_ = i / WID, o = i % WID;
        sWt[o * WID + in_] = w[OFF_W2 + i];
        sWt[WID * WID + o * WID + in_] = w[OFF_W3 + i];
    }
    for (int i = threadIdx.x; i < WID * OUT; i += THREADS) sW4[i] = w[OFF_W4 + i];
    const int tid = threadIdx.x;
    const int r0 = (tid / 16) * 4, c0 = (tid % 16) * 8;
    float gw4 = 0.0f, gb4 = 0.0f;
    const int n_tiles = (n + TILE - 1) / TILE;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int row0 = tile * TILE;
        __syncthreads();
        if (tid < TILE * OUT) {
            int rr = tid / OUT, o = tid % OUT, t = row0 + rr;
            float g = 0.0f;
            if (t < n) g = (o == 0) ? gsig[t] * sig[t] : geps[t] * (eps[t] - 1.0f);   // dL/do
            sO[rr * OUT + o] = g;
        }
        __syncthreads();
        // dW4[k][o] += sum_r a3[r][k] dO[r][o]; db4[o] += sum_r dO[r][o]  (thread (k, o))
        {
            int k = tid / OUT, o = tid % OUT;
            float s = 0.0f, sb = 0.0f;
            for (int rr = 0; rr < TILE; ++rr) {
                int t = row0 + rr;
                if (t >= n) break;
                float g = sO[rr * OUT + o];
                s = fmaf(bf(act[(int64_t)t * ACT + INP + 2 * WID + k]), g, s);
                sb += g;
            }
            gw4 += s;
            if (k == 0) gb4 += sb;
        }
        // dZ3[r][i] = (sum_o dO[r][o] W4[i][o]) * (a3[r][i] > 0)
        for (int e = tid; e < TILE * WID; e += THREADS) {
            int rr = e / WID, i = e % WID, t = row0 + rr;
            float v = 0.0f;
            if (t < n && bf(act[(int64_t)t * ACT + INP + 2 * WID + i]) > 0.0f)
                v = sO[rr * OUT] * bf(sW4[i * OUT]) + sO[rr * OUT + 1] * bf(sW4[i * OUT + 1]);
            sG[i * TILE + rr] = v;
            if (t < n) dz[(int64_t)t * 3 * WID + 2 * WID + i] = v;
        }
        __syncthreads();
        // dZ_{l-1} = (dZ_l W_l^T) * (a_{l-1} > 0) for l = 3, 2
        for (int l = 2; l >= 1; --l) {
            const __nv_bfloat16* Wt = sWt + (l - 1) * WID * WID;   // W_{l+1}^T [out][in]
            float acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
            for (int k = 0; k < WID; ++k) {
                float4 gv = *reinterpret_cast<const float4*>(sG + k * TILE + r0);
                uint4 wv = *reinterpret_cast<const uint4*>(Wt + k * WID + c0);
                const __nv_bfloat16* wb = reinterpret_cast<const __nv_bfloat16*>(&wv);
                float gf[4] = {gv.x, gv.y, gv.z, gv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(gf[i], bf(wb[j]), acc[i][j]);
            }
            const int aoff = INP + (l - 1) * WID;   // a_l is the input of layer l+1
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int t = row0 + r0 + i;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float v = 0.0f;
                    if (t < n && bf(act[(int64_t)t * ACT + aoff + c0 + j]) > 0.0f) v = acc[i][j];
                    sH[(c0 + j) * TILE + r0 + i] = v;
                    if (t < n) dz[(int64_t)t * 3 * WID + (l - 1) * WID + c0 + j] = v;
                }
            }
            __syncthreads();
            float* tmp = sG;
            sG = sH;
            sH = tmp;
        }
    }
    atomicAdd(gw + OFF_W4 + tid, gw4);   // tid = k * OUT + o covers the 256 weights of W4
    if (tid < OUT) atomicAdd(gb + OFF_B4 + tid, gb4);
}

// dW_l = A_l^T dZ_l, db_l = sum dZ_l: a CTA forms one 32 x 32 tile of one layer
// over one chunk of rows and adds it to the FP32 gradient with atomics.
__global__ void __launch_bounds__(THREADS) k_mlp_bwd_weights(int n, int chunk, const __nv_bfloat16* __restrict__ act,
                                                             const float* __restrict__ dz, float* __restrict__ gw,
                                                             float* __restrict__ gb) {
    __shared__ float sA[64][33];
    __shared__ float sZ[64][33];
    // tiles: layer 1: 2 x 4 (K = 40 padded to 64), layers 2, 3: 4 x 4
    int tix = blockIdx.x;
    int l, ti, tj;
    if (tix < 8) {
        l = 0;
        ti = tix / 4;
        tj = tix % 4;
    } else {
        l = 1 + (tix - 8) / 16;
        ti = ((tix - 8) % 16) / 4;
        tj = (tix - 8) % 4;
    }
    const int K = l == 0 ? INP : WID;
    const int aoff = l == 0 ? 0 : INP + (l - 1) * WID;
    const int woff = l == 0 ? OFF_W1 : (l == 1 ? OFF_W2 : OFF_W3);
    const int boff = l == 0 ? OFF_B1 : (l == 1 ? OFF_B2 : OFF_B3);
    const int rs = blockIdx.y * chunk, re = min(n, rs + chunk);
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 8 rows of 32 threads
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float accb = 0.0f;
    for (int base = rs; base < re; base += 64) {
        __syncthreads();
        for (int e = threadIdx.x; e < 64 * 32; e += THREADS) {
            int rr = e / 32, c = e % 32, t = base + rr;
            int i = ti * 32 + c, j = tj * 32 + c;
            sA[rr][c] = (t < re && i < K) ? bf(act[(int64_t)t * ACT + aoff + i]) : 0.0f;
            sZ[rr][c] = (t < re) ? dz[(int64_t)t * 3 * WID + l * WID + j] : 0.0f;
        }
        __syncthreads();
        for (int rr = 0; rr < 64; ++rr) {
            float z = sZ[rr][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fmaf(sA[rr][ty * 4 + q], z, acc[q]);
            if (ti == 0 && ty == 0) accb += z;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int i = ti * 32 + ty * 4 + q, j = tj * 32 + tx;
        if (i < K) atomicAdd(gw + woff + i * WID + j, acc[q]);
    }
    if (ti == 0 && ty == 0) atomicAdd(gb + boff + tj * 32 + tx, accb);
}

MlpScene make_scene(const rt_scene* sc) {
    MlpScene S;
    S.tri_v = sc->d_tri_v;
    S.n = sc->n_tris;
    S.cx = (float)(0.5 * (sc->lo[0] + sc->hi[0]));
    S.cy = (float)(0.5 * (sc->lo[1] + sc->hi[1]));
    S.cz = (float)(0.5 * (sc->lo[2] + sc->hi[2]));
    double size = std::max(sc->hi[0] - sc->lo[0], std::max(sc->hi[1] - sc->lo[1], sc->hi[2] - sc->lo[2]));
    S.inv_size = (float)(1.0 / size);
    return S;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) rt_status rt_mlp_forward(rt_ctx* ctx, const rt_scene* scene,
                                                                           const uint16_t* weights_bf16_dev,
                                                                           const float* bias_dev, float* eps_r_dev,
                                                                           float* sigma_dev, uint16_t* act_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!scene || !weights_bf16_dev || !bias_dev || !eps_r_dev || !sigma_dev)
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    if (((uintptr_t)weights_bf16_dev & 15) != 0) return rt_fail(ctx, RT_ERR_INVALID_ARG, "weights must be 16-byte aligned");
    const size_t smem = (size_t)NW * 2 + 2 * (size_t)WID * TILE * 2 + TILE * OUT * 4;
    RT_CK(ctx, cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int tiles = (scene->n_tris + TILE - 1) / TILE;
    const int grid = std::max(1, std::min(tiles, ctx->num_sms));
    k_mlp_fwd<<<grid, THREADS, smem, ctx->stream>>>(make_scene(scene), (const __nv_bfloat16*)weights_bf16_dev, bias_dev,
                                                    eps_r_dev, sigma_dev, (__nv_bfloat16*)act_dev);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_mlp_backward(
    rt_ctx* ctx, const rt_scene* scene, const uint16_t* weights_bf16_dev, const uint16_t* act_dev,
    const float* eps_r_dev, const float* sigma_dev, const float* grad_eps_r_dev, const float* grad_sigma_dev,
    float* dz_work_dev, float* grad_weights_dev, float* grad_bias_dev) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!scene || !weights_bf16_dev || !act_dev || !eps_r_dev || !sigma_dev || !grad_eps_r_dev || !grad_sigma_dev ||
        !dz_work_dev || !grad_weights_dev || !grad_bias_dev)
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    const int n = scene->n_tris;
    const size_t smem = 2 * (size_t)WID * WID * 2 + 2 * (size_t)WID * TILE * 4 + TILE * OUT * 4 + WID * OUT * 2;
    RT_CK(ctx, cudaFuncSetAttribute(k_mlp_bwd_data, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int tiles = (n + TILE - 1) / TILE;
    const int grid = std::max(1, std::min(tiles, ctx->num_sms));
    k_mlp_bwd_data<<<grid, THREADS, smem, ctx->stream>>>(n, (const __nv_bfloat16*)weights_bf16_dev,
                                                          (const __nv_bfloat16*)act_dev, eps_r_dev, sigma_dev,
                                                          grad_eps_r_dev, grad_sigma_dev, dz_work_dev, grad_weights_dev,
                                                          grad_bias_dev);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    const int splits = std::max(1, std::min(64, (n + 511) / 512));
    const int chunk = (n + splits - 1) / splits;
    k_mlp_bwd_weights<<<dim3(8 + 32, splits), THREADS, 0, ctx->stream>>>(n, chunk, (const __nv_bfloat16*)act_dev,
                                                                        dz_work_dev, grad_weights_dev, grad_bias_dev);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}
