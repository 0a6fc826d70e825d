// Per-path geometry records and the field computation of arXiv 2311.18558,
// Sec. II-B..D (Eq. cfr_cont, rel1, basis_transform, rel2, init,
// specular_reflection, fresnel-1/2), with its adjoint (Sec. III, Algorithm 1:
// gradients w.r.t. eps_r, sigma and the antenna gains, geometry held fixed).
//
// Record kernel (once per trace): FP64 directions k_j = (s_j - s_{j-1}) / d_j,
// delay tau = sum d_j / c, total length L, cos(theta_i) of every bounce and the
// real 2x2 basis changes D_1 .. D_{q+1}, stored FP32 in depth-slot-major SoA.
//
// Field kernels (every calibration step; HBM-bound streaming of the records):
//   v = D_1 C_T;  v <- D_{j+1} diag(r_perp,j, r_par,j) v  (j = 1..q);
//   a = lambda/(4 pi) sqrt(g_T g_R) / L * C_R^T v,
// with C_T = C_R = [1, 0] (vertical polarisation, zeta = 0, isotropic gain).
// The product of the spherical spreading factors of a chain of planar
// reflections is 1/L; the carrier phase exp(-j 2 pi f tau) is kept in tau.
#include <cuda_runtime.h>

#include "fresnel.cuh"
#include "vec3f.cuh"
#include "rt_internal.cuh"

namespace {

constexpr int MAT_PEC = 1 << 30;   // flag in the per-bounce material word of the records

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3(double x, double y, double z) { return D3{x, y, z}; }
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return d3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ double dotd(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// P paths (or *P_dev of them, at most P, when P_dev is given: the count of a trace
// that has not been read back); P is also the slot stride of tri, mc, Dm and dir.
__global__ void k_records(int64_t P, const int64_t* __restrict__ P_dev, int D, const double* __restrict__ pts,
                          const int32_t* __restrict__ depth, const int32_t* __restrict__ tri,
                          const double* __restrict__ tri_n64, const int32_t* __restrict__ tri_material,
                          const uint8_t* __restrict__ is_pec, double* tau, float* len, int2* mc, float4* Dm,
                          float4* dir) {
    if (P_dev) P = min(*P_dev, P);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const int q = depth[i];
        const double* pp = pts + (int64_t)i * (D + 2) * 3;
        D3 prev = d3(pp[0], pp[1], pp[2]);
        // lengths and delay in FP64; directions and every basis in FP32 (the records
        // are stored in FP32)
        F3 k[RT_MAX_DEPTH + 2];
        double L = 0.0;
        for (int j = 1; j <= q + 1; ++j) {
            D3 cur = d3(pp[3 * j], pp[3 * j + 1], pp[3 * j + 2]);
            D3 dv = sub(cur, prev);
            const double dj = sqrt(dotd(dv, dv));
            const float inv = 1.0f / (float)dj;
            k[j] = f3((float)dv.x * inv, (float)dv.y * inv, (float)dv.z * inv);
            L += dj;
            prev = cur;
        }
        tau[i] = L / RT_C0;
        len[i] = (float)L;
        F3 out_p, out_q;
        sph_basis_f(k[1], &out_p, &out_q);
        for (int j = 1; j <= q; ++j) {
            int t = tri[(int64_t)(j - 1) * P + i];
            F3 n = f3((float)tri_n64[4 * t], (float)tri_n64[4 * t + 1], (float)tri_n64[4 * t + 2]);
            if (fdot(k[j], n) > 0.0f) n = fscl(-1.0f, n);
            const float cos_i = -fdot(k[j], n);
            // at (numerically) normal incidence any transverse unit vector serves; the
            // previous outgoing p-vector is continued
            const F3 e_perp = perp_or_f(k[j], n, out_p);
            const F3 in_q = fcross(e_perp, k[j]);
            Dm[(int64_t)(j - 1) * P + i] =
                make_float4(fdot(e_perp, out_p), fdot(e_perp, out_q), fdot(in_q, out_p), fdot(in_q, out_q));
            const int mt = tri_material[t];
            mc[(int64_t)(j - 1) * P + i] = make_int2(mt | (is_pec[mt] ? MAT_PEC : 0), __float_as_int(cos_i));
            out_p = e_perp;
            out_q = fcross(e_perp, k[j + 1]);
        }
        F3 rp, rq;
        sph_basis_f(fscl(-1.0f, k[q + 1]), &rp, &rq);
        Dm[(int64_t)q * P + i] = make_float4(fdot(rp, out_p), fdot(rp, out_q), fdot(rq, out_p), fdot(rq, out_q));
        // departure and arrival directions, for direction-dependent antenna gains
        dir[i] = make_float4(k[1].x, k[1].y, k[1].z, 0.0f);
        dir[P + i] = make_float4(-k[q + 1].x, -k[q + 1].y, -k[q + 1].z, 0.0f);
    }
}

// complex FP32 helpers and fresnel<GRAD>: fresnel.cuh

struct FieldArgs {
    int64_t P;
    const int64_t* Pd;         // the count of paths of a trace that did not wait (at most P), or null
    int D;
    int n_mat;                 // entries of eps / sig (materials, or triangles when per_tri)
    const int32_t* depth;
    const int32_t* tri;
    const float* len;
    const int2* mc;
    const float4* Dm;
    const double* tau;
    const int32_t* tri_material;
    const uint8_t* is_pec;
    const float* eps;
    const float* sig;
    int per_tri;
    float inv_eps0w;   // 1 / (eps0 omega)
    float amp;         // lambda / (4 pi) sqrt(g_T g_R)
};

constexpr int ETA_SMEM = 64;  // per-material eta table in shared memory up to this many materials

// eta = eps_r - j sigma / (eps0 omega) of material (or triangle) m
__device__ __forceinline__ float2 eta_of(const FieldArgs& A, const float2* s_eta, int m) {
    if (s_eta) return s_eta[m];
    return make_float2(__ldg(A.eps + m), -__ldg(A.sig + m) * A.inv_eps0w);
}

// The records of one path, held in registers: depth q, total length L, the
// q + 1 basis changes D_1 .. D_{q+1}, the q material words (material | PEC flag,
// cos theta_i) and, for per-triangle materials, the q triangles.  Every load is
// issued before any arithmetic, so that all of a path's loads are in flight at
// once: the slot loads wait only for q.
template <bool PER_TRI>
struct PathRec {
    int q;
    float len;
    float4 D[RT_MAX_DEPTH + 1];
    int2 w[RT_MAX_DEPTH];
    int t[PER_TRI ? RT_MAX_DEPTH : 1];
};

template <bool PER_TRI>
__device__ __forceinline__ void rec_head(const FieldArgs& A, int64_t i, PathRec<PER_TRI>& r) {
    r.q = __ldg(A.depth + i);
    r.len = __ldg(A.len + i);
    r.D[0] = __ldg(A.Dm + i);
}

template <bool PER_TRI>
__device__ __forceinline__ void rec_slots(const FieldArgs& A, int64_t i, PathRec<PER_TRI>& r) {
#pragma unroll
    for (int j = 0; j < RT_MAX_DEPTH; ++j) {
        if (j < r.q) {
            const int64_t o = (int64_t)j * A.P + i;
            r.w[j] = __ldg(A.mc + o);
            if (PER_TRI) r.t[j] = __ldg(A.tri + o);
            r.D[j + 1] = __ldg(A.Dm + o + A.P);
        }
    }
}

// Fresnel coefficients of bounce j (and their derivatives w.r.t. eta if GRAD);
// returns the material (or triangle) index, -1 for a perfect conductor.
template <bool GRAD, bool PER_TRI>
__device__ __forceinline__ int bounce_coeffs(const FieldArgs& A, const float2* s_eta, const PathRec<PER_TRI>& r, int j,
                                             float2& rp, float2& rl, float2& drp, float2& drl) {
    if (r.w[j].x & MAT_PEC) {
        rp = make_float2(-1.0f, 0.0f);
        rl = make_float2(1.0f, 0.0f);
        return -1;
    }
    const int m = PER_TRI ? r.t[j] : r.w[j].x;
    fresnel<GRAD>(eta_of(A, s_eta, m), __int_as_float(r.w[j].y), rp, rl, drp, drl);
    return m;
}

// FWD_NP paths per thread, their records loaded together; the material gather of
// the step is a shared-memory table (or an L2-resident per-triangle array).
// Launched with one path per thread at 5 blocks of 256 per SM: with every record
// of a path in flight at once that keeps enough loads outstanding, while two
// paths per thread need ~106 registers and ran 40 % slower.
template <bool PER_TRI, int FWD_NP, int MINB>
__global__ void __launch_bounds__(256, MINB) k_fields_fwd(FieldArgs A, float2* __restrict__ a_out,
                                                       double* __restrict__ tau_out) {
    if (A.Pd) A.P = min(*A.Pd, A.P);   // slots of a trace that did not wait: its count (and stride)
    __shared__ float2 s_tab[ETA_SMEM];
    const bool smem_eta = !PER_TRI && A.n_mat <= ETA_SMEM;
    if (smem_eta) {
        for (int m = threadIdx.x; m < A.n_mat; m += blockDim.x)
            s_tab[m] = make_float2(A.eps[m], -A.sig[m] * A.inv_eps0w);
        __syncthreads();
    }
    const float2* s_eta = smem_eta ? s_tab : nullptr;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < A.P; i0 += FWD_NP * stride) {
        PathRec<PER_TRI> r[FWD_NP];
        int64_t idx[FWD_NP];
        double tau[FWD_NP];
#pragma unroll
        for (int k = 0; k < FWD_NP; ++k) {
            idx[k] = i0 + k * stride;
            r[k].q = -1;
            if (idx[k] < A.P) {
                rec_head(A, idx[k], r[k]);
                if (tau_out) tau[k] = __ldg(A.tau + idx[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < FWD_NP; ++k) rec_slots(A, idx[k], r[k]);
#pragma unroll
        for (int k = 0; k < FWD_NP; ++k) {
            if (r[k].q < 0) continue;
            // v = D_1 C_T with C_T = [1, 0]; v <- D_{j+1} diag(r_perp, r_par) v
            float2 v0 = make_float2(r[k].D[0].x, 0.0f), v1 = make_float2(r[k].D[0].z, 0.0f);
#pragma unroll
            for (int j = 0; j < RT_MAX_DEPTH; ++j) {
                if (j < r[k].q) {
                    float2 rp, rl, unused;
                    bounce_coeffs<false>(A, s_eta, r[k], j, rp, rl, unused, unused);
                    const float2 g0 = cmul(rp, v0), g1 = cmul(rl, v1);
                    const float4 e = r[k].D[j + 1];
                    v0 = cadd(cscale(e.x, g0), cscale(e.y, g1));
                    v1 = cadd(cscale(e.z, g0), cscale(e.w, g1));
                }
            }
            a_out[idx[k]] = cscale(A.amp / r[k].len, v0);
            if (tau_out) tau_out[idx[k]] = tau[k];
        }
    }
}

// Reduction of the per-material gradients: REGM > 0 keeps one shared-memory
// column per material and thread (few materials: no atomics on a handful of hot
// addresses), MAXM > 0 accumulates with shared-memory atomics, otherwise global
// atomics (per-triangle materials: scattered, little contention).  The records
// of a path are loaded once, into registers, and serve both walks.
template <int MAXM, int REGM, bool PER_TRI>
__global__ void __launch_bounds__(256, 3) k_fields_bwd(FieldArgs A, const float2* __restrict__ ga,
                                                       float* __restrict__ geps, float* __restrict__ gsig,
                                                       float* __restrict__ ggain, float inv_gtx, float inv_grx,
                                                       int n_mat) {
    if (A.Pd) A.P = min(*A.Pd, A.P);   // slots of a trace that did not wait: its count (and stride)
    __shared__ float s_eps[MAXM > 0 ? MAXM : 1], s_sig[MAXM > 0 ? MAXM : 1], s_gain[2];
    __shared__ float2 s_tab[ETA_SMEM];
    if (MAXM > 0)
        for (int m = threadIdx.x; m < n_mat; m += blockDim.x) s_eps[m] = s_sig[m] = 0.0f;
    if (threadIdx.x < 2) s_gain[threadIdx.x] = 0.0f;
    const bool smem_eta = !PER_TRI && A.n_mat <= ETA_SMEM;
    if (smem_eta)
        for (int m = threadIdx.x; m < A.n_mat; m += blockDim.x)
            s_tab[m] = make_float2(A.eps[m], -A.sig[m] * A.inv_eps0w);
    __syncthreads();
    const float2* s_eta = smem_eta ? s_tab : nullptr;
    // REGM materials: per-thread accumulator columns in shared memory
    // (s_col[m][tid]), summed over the block at the end
    __shared__ float s_col[REGM > 0 ? 2 * REGM * 256 : 1];
    if (REGM > 0)
        for (int k = threadIdx.x; k < 2 * REGM * 256; k += blockDim.x) s_col[k] = 0.0f;
    __shared__ float4 s_fr[RT_MAX_DEPTH][256];   // (r_perp, r_par) of each bounce, per thread
    __syncthreads();
    float gain_acc = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.P; i += (int64_t)gridDim.x * blockDim.x) {
        PathRec<PER_TRI> r;
        rec_head(A, i, r);
        const float2 g = __ldg(ga + i);
        rec_slots(A, i, r);
        const float scale = A.amp / r.len;
        float2 v0 = make_float2(r.D[0].x, 0.0f), v1 = make_float2(r.D[0].z, 0.0f);
        // forward walk: the Fresnel coefficients with their derivatives, once per
        // bounce; the reverse walk needs the coefficients (kept in shared memory) and
        // the derivatives times the field entering the bounce (p0, p1, in registers)
        float2 p0[RT_MAX_DEPTH], p1[RT_MAX_DEPTH];
        float4 last = r.D[0];   // D_{q+1}
#pragma unroll
        for (int j = 0; j < RT_MAX_DEPTH; ++j) {
            if (j < r.q) {
                float2 rp, rl, drp = make_float2(0.0f, 0.0f), drl = make_float2(0.0f, 0.0f);
                bounce_coeffs<true>(A, s_eta, r, j, rp, rl, drp, drl);
                p0[j] = cmul(drp, v0);
                p1[j] = cmul(drl, v1);
                s_fr[j][threadIdx.x] = make_float4(rp.x, rp.y, rl.x, rl.y);
                const float2 g0 = cmul(rp, v0), g1 = cmul(rl, v1);
                const float4 e = r.D[j + 1];
                v0 = cadd(cscale(e.x, g0), cscale(e.y, g1));
                v1 = cadd(cscale(e.z, g0), cscale(e.w, g1));
                last = e;
            }
        }
        const float2 a = cscale(scale, v0);
        // Re(conj(g) a) / (2 g_T) and / (2 g_R) share Re(conj(g) a)
        gain_acc += g.x * a.x + g.y * a.y;
        // reverse walk: l = scale * (row 0 of D_{q+1}) . Gamma_q D_q ... is the row
        // vector after bounce j; da/deta_j = l[0] in0_j dr_perp_j + l[1] in1_j dr_par_j.
        float2 l0 = make_float2(scale * last.x, 0.0f), l1 = make_float2(scale * last.y, 0.0f);
#pragma unroll
        for (int j = RT_MAX_DEPTH - 1; j >= 0; --j) {
            if (j < r.q) {
                const float4 c = s_fr[j][threadIdx.x];
                const float2 rp = make_float2(c.x, c.y), rl = make_float2(c.z, c.w);
                const int m = (r.w[j].x & MAT_PEC) ? -1 : (PER_TRI ? r.t[PER_TRI ? j : 0] : r.w[j].x);
                if (m >= 0) {
                    const float2 da = cadd(cmul(l0, p0[j]), cmul(l1, p1[j]));
                    // Re(conj(g) da) and Im(conj(g) da)
                    const float re = g.x * da.x + g.y * da.y;
                    const float im = g.x * da.y - g.y * da.x;
                    const float de = re, ds = im * A.inv_eps0w;   // da/dsigma = -j/(eps0 w) da/deta
                    if (REGM > 0) {
                        s_col[m * 256 + threadIdx.x] += de;
                        s_col[(REGM + m) * 256 + threadIdx.x] += ds;
                    } else if (MAXM > 0) {
                        atomicAdd(&s_eps[m], de);
                        atomicAdd(&s_sig[m], ds);
                    } else {
                        if (geps) atomicAdd(geps + m, de);
                        if (gsig) atomicAdd(gsig + m, ds);
                    }
                }
                const float2 h0 = cmul(l0, rp), h1 = cmul(l1, rl);
                const float4 e = r.D[j];
                l0 = cadd(cscale(e.x, h0), cscale(e.z, h1));
                l1 = cadd(cscale(e.y, h0), cscale(e.w, h1));
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) gain_acc += __shfl_down_sync(0xffffffffu, gain_acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_gain[0], gain_acc);
    if (REGM > 0) {
        __syncthreads();
        // one warp per (material, eps|sigma) column sum
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int col = warp; col < 2 * REGM; col += blockDim.x >> 5) {
            float v = 0.0f;
            for (int k = lane; k < 256; k += 32) v += s_col[col * 256 + k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            const int m = col % REGM;
            if (lane == 0 && m < n_mat) {
                if (col < REGM) atomicAdd(&s_eps[m], v);
                else atomicAdd(&s_sig[m], v);
            }
        }
    }
    __syncthreads();
    if (MAXM > 0) {
        for (int m = threadIdx.x; m < n_mat; m += blockDim.x) {
            if (geps && s_eps[m] != 0.0f) atomicAdd(geps + m, s_eps[m]);
            if (gsig && s_sig[m] != 0.0f) atomicAdd(gsig + m, s_sig[m]);
        }
    }
    if (threadIdx.x == 0 && ggain) {
        atomicAdd(ggain + 0, 0.5f * s_gain[0] * inv_gtx);
        atomicAdd(ggain + 1, 0.5f * s_gain[0] * inv_grx);
    }
}

FieldArgs make_args(const rt_paths* p, const float* eps, const float* sig, int per_tri, double freq, float gtx,
                    float grx) {
    FieldArgs A;
    A.P = p->P;
    A.Pd = p->d_count;
    A.D = p->D;
    A.depth = p->d_depth;
    A.tri = p->d_tri;

    A.n_mat = per_tri ? p->scene->n_tris : p->scene->n_materials;
    A.len = p->d_len;
    A.mc = p->d_mc;
    A.Dm = p->d_Dm;
    A.tau = p->d_tau;
    A.tri_material = p->scene->d_tri_material;
    A.is_pec = p->scene->d_is_pec;
    A.eps = eps;
    A.sig = sig;
    A.per_tri = per_tri;
    A.inv_eps0w = (float)(1.0 / (RT_EPS0 * 2.0 * RT_PI * freq));
    A.amp = (float)(RT_C0 / freq / (4.0 * RT_PI) * std::sqrt((double)gtx * (double)grx));
    return A;
}

int grid_for(const rt_ctx* ctx, int64_t n, int threads, int per_sm) {
    int64_t g = (n + threads - 1) / threads;
    int64_t cap = (int64_t)ctx->num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

rt_status rt_launch_paths_records(rt_ctx* ctx, rt_paths* p, const int64_t* P_dev) {
    cudaStream_t st = ctx->stream;
    const size_t Pa = p->P > 0 ? (size_t)p->P : 1;
    // one allocation for the five record arrays
    RtCarve c;
    const size_t o_tau = c.take(Pa * 8), o_len = c.take(Pa * 4), o_mc = c.take(Pa * p->D * 8),
                 o_Dm = c.take(Pa * (p->D + 1) * 16), o_dir = c.take(Pa * 2 * 16);
    char* b = nullptr;
    RT_CK(ctx, cudaMallocAsync((void**)&b, c.off, st));
    p->d_block_rec = b;
    p->d_tau = reinterpret_cast<double*>(b + o_tau);
    p->d_len = reinterpret_cast<float*>(b + o_len);
    p->d_mc = reinterpret_cast<int2*>(b + o_mc);
    p->d_Dm = reinterpret_cast<float4*>(b + o_Dm);
    p->d_dir = reinterpret_cast<float4*>(b + o_dir);
    if (p->P == 0) return RT_OK;
    k_records<<<grid_for(ctx, p->P, 32, 32), 32, 0, st>>>(p->P, P_dev, p->D, p->d_pts, p->d_depth, p->d_tri,
                                                           p->scene->d_tri_n64, p->scene->d_tri_material,
                                                           p->scene->d_is_pec, p->d_tau, p->d_len, p->d_mc,
                                                           p->d_Dm, p->d_dir); RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

rt_status rt_launch_fields_fwd(rt_ctx* ctx, const rt_paths* p, const float* eps, const float* sig, int per_tri,
                               double freq, float gtx, float grx, float2* a, double* tau) {
    if (p->P == 0) return RT_OK;
    FieldArgs A = make_args(p, eps, sig, per_tri, freq, gtx, grx);
    const int grid = grid_for(ctx, p->P, 256, 5);
    if (per_tri) k_fields_fwd<true, 1, 5><<<grid, 256, 0, ctx->stream>>>(A, a, tau);
    else k_fields_fwd<false, 1, 5><<<grid, 256, 0, ctx->stream>>>(A, a, tau);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

rt_status rt_launch_fields_bwd(rt_ctx* ctx, const rt_paths* p, const float* eps, const float* sig, int per_tri,
                               double freq, float gtx, float grx, const float2* ga, float* geps, float* gsig,
                               float* ggain) {
    if (p->P == 0) return RT_OK;
    FieldArgs A = make_args(p, eps, sig, per_tri, freq, gtx, grx);
    const int n_mat = per_tri ? p->scene->n_tris : p->scene->n_materials;
    const int grid = grid_for(ctx, p->P, 256, 3);
    if (!per_tri && n_mat <= 8)
        k_fields_bwd<8, 8, false><<<grid, 256, 0, ctx->stream>>>(A, ga, geps, gsig, ggain, 1.0f / gtx, 1.0f / grx,
                                                                 n_mat);
    else if (!per_tri && n_mat <= 64)
        k_fields_bwd<64, 0, false><<<grid, 256, 0, ctx->stream>>>(A, ga, geps, gsig, ggain, 1.0f / gtx, 1.0f / grx,
                                                                  n_mat);
    else if (!per_tri)
        k_fields_bwd<0, 0, false><<<grid, 256, 0, ctx->stream>>>(A, ga, geps, gsig, ggain, 1.0f / gtx, 1.0f / grx,
                                                                 n_mat);
    else
        k_fields_bwd<0, 0, true><<<grid, 256, 0, ctx->stream>>>(A, ga, geps, gsig, ggain, 1.0f / gtx, 1.0f / grx,
                                                                n_mat);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}
