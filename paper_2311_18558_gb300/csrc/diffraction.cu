// First-order diffraction (arXiv 2311.18558, Sec. II-D Eq. diffraction: F(E) =
// Q E A^d e^{-j k d}; Sec. II-F: candidate edges from the shoot-and-bouncing rays,
// points of diffraction by Keller's shortest-path principle; only paths
// Tx -> edge -> Rx).  The paper names its model without printing it: the uniform
// theory of diffraction (Kouyoumjian and Pathak, Proc. IEEE 1974) with Luebbers'
// coefficients for faces of finite conductivity (IEEE Trans. AP 1984), in an
// edge-fixed frame.  Written here from those publications.
//
// Wedges (built on the host once per scene, from the triangles' vertices): an
// edge is a pair of triangles sharing two vertex positions; it is a wedge when
// its exterior angle n pi, measured outside the solid from one face to the other
// with the winding normals taken as outward, has 1 < n <= 2 (n = 2: two
// coincident faces back to back, a screen).  Canonical frame: face 0 is the lower
// triangle id, t0 points from the edge into it, n0 is its normal, e = t0 x n0,
// the edge runs from E_s to E_s + l e.
//
// Tracing (rt_trace_diffraction):
//   1. candidate wedges: those with a face among the triangles the launch rays hit
//      first (the depth-1 candidates of a specular trace of the same transmitter);
//   2. k_dif_pairs, one thread per (candidate wedge, receiver), FP64 without
//      contraction: Keller's point x_Q = (x_T b + x_R a) / (a + b) on the edge line
//      (a, b the distances of Tx, Rx from it, x_T, x_R their abscissae); valid if
//      a, b > eps, 0 <= x_Q < l, both ends strictly in the exterior
//      (0 < phi', phi < n pi), both segments longer than eps and free of every
//      triangle but the two faces for t in (eps, len - eps) (exact any-hit);
//   3. per-receiver counts, a scan and an ordered expansion (by receiver, then by
//      wedge), then k_dif_records writes each path's records.
// Fields (rt_eval_fields_diffraction): per path
//   D_{s,h} = -e^{-j pi/4} / (2 n sqrt(2 pi k) sin beta_0) [T1 + T2 + R_0 T3 + R_n T4],
//   T_i = cot(eps_i / 2n) F(2 k L sin^2(eps_i / 2)), eps_i the reduced angles of
//   pi + (phi - phi'), pi - (phi - phi'), pi - (phi + phi'), pi + (phi + phi');
//   F(X) = 2 j sqrt(X) e^{jX} int_{sqrt X}^inf e^{-j t^2} dt (series below X = 2, the
//   Laplace continued fraction of the complementary error function above);
//   R_0 (R_n): Fresnel coefficients of the incidence (other) face at
//   cos theta = |sin beta_0 sin phi'| (|sin beta_0 sin(n pi - phi)|), r_perp for
//   the soft and r_par for the hard coefficient, -1 / +1 for a perfect conductor;
//   a = lambda / (4 pi) sqrt(g_T g_R) A^d / s' (D_s b_in b_out + D_h p_in p_out),
//   A^d = sqrt(s' / (s (s + s'))), L = s s' sin^2 beta_0 / (s + s'), with b_in, p_in
//   the projections of the transmit polarisation theta_hat(s') on the incident
//   edge-fixed basis (beta', phi') and b_out, p_out those of the diffracted basis
//   (beta, phi) on the receive polarisation theta_hat(-s).  The incidence face is
//   the face on the transmitter's side (phi' <= n pi / 2).  The delay is
//   tau = (s' + s) / c.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fresnel.cuh"
#include "rt_internal.cuh"
#include "segquery.cuh"

namespace {

constexpr int DIF_THREADS = 128;
constexpr int DIF_REC = 14;          // FP32 records per path (see k_dif_records)
constexpr double DIF_PI = 3.14159265358979323846;

int dif_grid(const rt_ctx* ctx, int64_t n, int threads, int per_sm) {
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)ctx->num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// ------------------------------------------------------------------ wedge table (host)
struct V3d {
    double x, y, z;
};
V3d vsub(V3d a, V3d b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3d vmul(double s, V3d a) { return {s * a.x, s * a.y, s * a.z}; }
double vdot(V3d a, V3d b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3d vcross(V3d a, V3d b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
V3d vunit(V3d a) { return vmul(1.0 / std::sqrt(vdot(a, a)), a); }
bool vsame(V3d a, V3d b) { return a.x == b.x && a.y == b.y && a.z == b.z; }

struct HalfEdge {
    float k[6];   // the two end vertices, lexicographically ordered
    int tri;
};

bool he_less(const HalfEdge& a, const HalfEdge& b) {
    for (int i = 0; i < 6; ++i)
        if (a.k[i] != b.k[i]) return a.k[i] < b.k[i];
    return a.tri < b.tri;
}

bool he_same_edge(const HalfEdge& a, const HalfEdge& b) {
    for (int i = 0; i < 6; ++i)
        if (a.k[i] != b.k[i]) return false;
    return true;
}

struct WedgeRec {
    int f0, fn;
    double g[14];   // start vertex, e, t0, n0, length, n
};

rt_status build_wedges(rt_ctx* ctx, rt_scene* sc) {
    const int T = sc->n_tris;
    std::vector<float4> tv((size_t)3 * T);
    RT_CK(ctx, cudaMemcpy(tv.data(), sc->d_tri_v, tv.size() * sizeof(float4), cudaMemcpyDeviceToHost));
    auto vert = [&](int t, int k) { return V3d{tv[3 * t + k].x, tv[3 * t + k].y, tv[3 * t + k].z}; };
    std::vector<HalfEdge> he;
    he.reserve((size_t)3 * T);
    for (int t = 0; t < T; ++t) {
        for (int k = 0; k < 3; ++k) {
            float4 p = tv[3 * t + k], q = tv[3 * t + (k + 1) % 3];
            const bool swap = (q.x < p.x) || (q.x == p.x && (q.y < p.y || (q.y == p.y && q.z < p.z)));
            if (swap) std::swap(p, q);
            he.push_back(HalfEdge{{p.x, p.y, p.z, q.x, q.y, q.z}, t});
        }
    }
    std::sort(he.begin(), he.end(), he_less);
    std::vector<WedgeRec> w;
    for (size_t i = 0; i < he.size();) {
        size_t j = i + 1;
        while (j < he.size() && he_same_edge(he[i], he[j])) ++j;
        if (j - i == 2 && he[i].tri != he[i + 1].tri) {
            const int f0 = he[i].tri, f1 = he[i + 1].tri;   // sorted: f0 < f1
            const V3d A{he[i].k[0], he[i].k[1], he[i].k[2]}, B{he[i].k[3], he[i].k[4], he[i].k[5]};
            const V3d er = vunit(vsub(B, A));
            auto into = [&](int t) {
                V3d c = vert(t, 0);
                for (int k = 0; k < 3; ++k)
                    if (!vsame(vert(t, k), A) && !vsame(vert(t, k), B)) c = vert(t, k);
                const V3d d = vsub(c, A);
                return vunit(vsub(d, vmul(vdot(d, er), er)));
            };
            auto normal = [&](int t) { return vunit(vcross(vsub(vert(t, 1), vert(t, 0)), vsub(vert(t, 2), vert(t, 0)))); };
            const V3d t0 = into(f0), t1 = into(f1), n0 = normal(f0), n1 = normal(f1);
            const V3d e = vdot(vcross(er, t0), n0) >= 0.0 ? er : vmul(-1.0, er);
            if (vdot(vmul(-1.0, vcross(e, t1)), n1) > 0.5) {
                double psi = std::atan2(vdot(t1, n0), vdot(t1, t0));
                if (psi < 0.0) psi += 2.0 * DIF_PI;
                if (psi < 1e-12) psi = 2.0 * DIF_PI;
                const double n = psi / DIF_PI;
                if (n > 1.0 + 1e-9) {
                    WedgeRec r;
                    r.f0 = f0;
                    r.fn = f1;
                    const V3d s = vdot(vsub(B, A), e) > 0.0 ? A : B;
                    const V3d v[4] = {s, e, t0, n0};
                    for (int k = 0; k < 4; ++k) {
                        r.g[3 * k] = v[k].x;
                        r.g[3 * k + 1] = v[k].y;
                        r.g[3 * k + 2] = v[k].z;
                    }
                    r.g[12] = std::sqrt(vdot(vsub(B, A), vsub(B, A)));
                    r.g[13] = n;
                    w.push_back(r);
                }
            }
        }
        i = j;
    }
    std::sort(w.begin(), w.end(), [](const WedgeRec& a, const WedgeRec& b) {
        return a.f0 != b.f0 ? a.f0 < b.f0 : a.fn < b.fn;
    });
    const int W = (int)w.size();
    std::vector<double> geo((size_t)14 * std::max(W, 1));
    std::vector<int2> faces(std::max(W, 1));
    std::vector<int32_t> tw((size_t)3 * std::max(T, 1), -1);
    sc->h_wedge_faces = new int32_t[2 * (size_t)std::max(W, 1)];
    sc->h_wedge_n = new double[std::max(W, 1)];
    for (int i = 0; i < W; ++i) {
        std::memcpy(&geo[(size_t)14 * i], w[i].g, sizeof(w[i].g));
        faces[i] = make_int2(w[i].f0, w[i].fn);
        sc->h_wedge_faces[2 * i] = w[i].f0;
        sc->h_wedge_faces[2 * i + 1] = w[i].fn;
        sc->h_wedge_n[i] = w[i].g[13];
        for (int f : {w[i].f0, w[i].fn})
            for (int k = 0; k < 3; ++k)
                if (tw[(size_t)3 * f + k] < 0) {
                    tw[(size_t)3 * f + k] = i;
                    break;
                }
    }
    RT_CK(ctx, cudaMalloc((void**)&sc->d_wedge, geo.size() * 8));
    RT_CK(ctx, cudaMalloc((void**)&sc->d_wedge_faces, faces.size() * sizeof(int2)));
    RT_CK(ctx, cudaMalloc((void**)&sc->d_tri_wedges, tw.size() * 4));
    RT_CK(ctx, cudaMemcpy(sc->d_wedge, geo.data(), geo.size() * 8, cudaMemcpyHostToDevice));
    RT_CK(ctx, cudaMemcpy(sc->d_wedge_faces, faces.data(), faces.size() * sizeof(int2), cudaMemcpyHostToDevice));
    RT_CK(ctx, cudaMemcpy(sc->d_tri_wedges, tw.data(), tw.size() * 4, cudaMemcpyHostToDevice));
    sc->n_wedges = W;
    return RT_OK;
}

rt_status ensure_wedges(rt_ctx* ctx, const rt_scene* scene) {
    rt_scene* sc = const_cast<rt_scene*>(scene);   // the wedge table is a cache of the scene
    if (sc->n_wedges >= 0) return RT_OK;
    return build_wedges(ctx, sc);
}

// ------------------------------------------------------------------ FP64 geometry (device, uncontracted)
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3sub(D3 a, D3 b) { return {dsub(a.x, b.x), dsub(a.y, b.y), dsub(a.z, b.z)}; }
__device__ __forceinline__ D3 d3add(D3 a, D3 b) { return {dadd(a.x, b.x), dadd(a.y, b.y), dadd(a.z, b.z)}; }
__device__ __forceinline__ D3 d3mul(double s, D3 a) { return {dmul(s, a.x), dmul(s, a.y), dmul(s, a.z)}; }
__device__ __forceinline__ double d3dot(D3 a, D3 b) { return dadd(dadd(dmul(a.x, b.x), dmul(a.y, b.y)), dmul(a.z, b.z)); }
__device__ __forceinline__ double d3norm(D3 a) { return sqrt(d3dot(a, a)); }
__device__ __forceinline__ D3 d3cross(D3 a, D3 b) {
    return {dsub(dmul(a.y, b.z), dmul(a.z, b.y)), dsub(dmul(a.z, b.x), dmul(a.x, b.z)),
            dsub(dmul(a.x, b.y), dmul(a.y, b.x))};
}

struct WedgeDev {
    D3 s, e, t0, n0;
    double len, n;
};

__device__ __forceinline__ WedgeDev load_wedge(const double* __restrict__ g, int w) {
    const double* p = g + (size_t)14 * w;
    WedgeDev r;
    r.s = {p[0], p[1], p[2]};
    r.e = {p[3], p[4], p[5]};
    r.t0 = {p[6], p[7], p[8]};
    r.n0 = {p[9], p[10], p[11]};
    r.len = p[12];
    r.n = p[13];
    return r;
}

// angle of direction d about the edge, from face 0 into the exterior, in [0, 2 pi)
__device__ __forceinline__ double wedge_angle(const WedgeDev& w, D3 d) {
    const D3 p = d3sub(d, d3mul(d3dot(d, w.e), w.e));
    double a = atan2(d3dot(p, w.n0), d3dot(p, w.t0));
    return a < 0.0 ? dadd(a, 2.0 * DIF_PI) : a;
}

struct Keller {
    D3 Q;
    double php, phi, sp, sd;
};

// Keller's point of the wedge for Tx T and Rx R, with the validity checks that
// need no scene query; false if the pair has no diffraction path.
__device__ __forceinline__ bool keller(const WedgeDev& w, D3 T, D3 R, double eps, Keller& k) {
    const D3 dT = d3sub(T, w.s), dR = d3sub(R, w.s);
    const double xT = d3dot(dT, w.e), xR = d3dot(dR, w.e);
    const double a = d3norm(d3sub(dT, d3mul(xT, w.e))), b = d3norm(d3sub(dR, d3mul(xR, w.e)));
    if (!(a > eps && b > eps)) return false;
    const double xQ = dadd(dmul(xT, b), dmul(xR, a)) / dadd(a, b);
    if (!(xQ >= 0.0 && xQ < w.len)) return false;
    k.Q = d3add(w.s, d3mul(xQ, w.e));
    k.php = wedge_angle(w, d3sub(T, k.Q));
    k.phi = wedge_angle(w, d3sub(R, k.Q));
    const double lim = w.n * DIF_PI;
    if (!(k.php > 0.0 && k.php < lim && k.phi > 0.0 && k.phi < lim)) return false;
    k.sp = d3norm(d3sub(k.Q, T));
    k.sd = d3norm(d3sub(R, k.Q));
    return k.sp > eps && k.sd > eps;
}

// Segment p0 -> p1 free of every triangle but f0, f1 for t in (eps, len - eps).
// One end is on the wedge's edge, which lies in the planes pl0, pl1 of both faces,
// so the segment meets those planes only at that end: their triangles are skipped.
__device__ __forceinline__ bool seg_clear(const BvhNode* nodes, const float4* tris, D3 p0, D3 p1, double eps, int f0,
                                          int f1, int pl0, int pl1, int32_t* status) {
    Ray64 r;
    r.o[0] = p0.x;
    r.o[1] = p0.y;
    r.o[2] = p0.z;
    const D3 d = d3sub(p1, p0);
    r.d[0] = d.x;
    r.d[1] = d.y;
    r.d[2] = d.z;
    const float3 o32 = make_float3((float)p0.x, (float)p0.y, (float)p0.z);
    const float3 d32 = make_float3((float)d.x, (float)d.y, (float)d.z);
    const float len2f = d32.x * d32.x + d32.y * d32.y + d32.z * d32.z;
    return !any_hit_seg(nodes, tris, r, o32, d32, len2f, eps, f0, status, f1, pl0, pl1);
}

// ------------------------------------------------------------------ tracing kernels
__global__ void k_dif_candidates(const uint64_t* __restrict__ cand, int64_t K, const int32_t* __restrict__ tri_wedges,
                                 uint8_t* __restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < K; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = cand[i];
        if (rt_key_depth(key) != 1) continue;
        const int t = rt_key_tri(key, 0);
        for (int k = 0; k < 3; ++k) {
            const int w = __ldg(tri_wedges + 3 * t + k);
            if (w >= 0) flag[w] = 1;
        }
    }
}

// Ordered compaction of flagged wedges by one block: list of candidate wedge ids.
__global__ void k_dif_compact(const uint8_t* __restrict__ flag, int W, int32_t* __restrict__ list, int32_t* count) {
    __shared__ int s_base;
    __shared__ int s_warp[32];
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int b0 = 0; b0 < W; b0 += blockDim.x) {
        const int i = b0 + threadIdx.x;
        const bool f = i < W && flag[i];
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        int off = s_base;
        for (int k = 0; k < warp; ++k) off += s_warp[k];
        if (f) list[off + __popc(m & ((1u << lane) - 1u))] = i;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int k = 0; k < nw; ++k) t += s_warp[k];
            s_base += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = s_base;
}

// FP32 copy of a candidate wedge for the prefilter of k_dif_pairs: edge start s,
// e, t0, n0, (sin n pi, cos n pi) (the other face's outward normal is
// sin(n pi) t0 - cos(n pi) n0), length, and the transmitter's abscissa xT and
// distance a from the edge line.
struct WedgeF {
    float4 a;   // s.x, s.y, s.z, len
    float4 b;   // e.x, e.y, e.z, xT
    float4 c;   // t0.x, t0.y, t0.z, a
    float4 d;   // n0.x, n0.y, n0.z, sin(n pi)
    float cn;   // cos(n pi)
};

__global__ void k_dif_prep(const double* __restrict__ wedge, const int32_t* __restrict__ cw, int Kw, D3 T,
                           float4* __restrict__ out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Kw; k += gridDim.x * blockDim.x) {
        const WedgeDev w = load_wedge(wedge, cw[k]);
        const D3 dT = d3sub(T, w.s);
        const double xT = d3dot(dT, w.e);
        const double a = d3norm(d3sub(dT, d3mul(xT, w.e)));
        double sn, cn;
        sincospi(w.n, &sn, &cn);
        float4* o = out + 5 * (size_t)k;
        o[0] = make_float4((float)w.s.x, (float)w.s.y, (float)w.s.z, (float)w.len);
        o[1] = make_float4((float)w.e.x, (float)w.e.y, (float)w.e.z, (float)xT);
        o[2] = make_float4((float)w.t0.x, (float)w.t0.y, (float)w.t0.z, (float)a);
        o[3] = make_float4((float)w.n0.x, (float)w.n0.y, (float)w.n0.z, (float)sn);
        o[4] = make_float4((float)cn, 0.0f, 0.0f, 0.0f);
    }
}

// FP32 prefilter of a (receiver, wedge) pair: false only where the FP64 tests of
// keller() certainly fail for the receiver, i.e. the receiver lies inside the
// wedge (behind both faces), closer to the edge line than eps, or Keller's
// abscissa lies outside [0, len), each by more than the margin m.  The FP32
// quantities carry errors of a few 1e-7 of the scene size (the records rounded
// from FP64 and a handful of FP32 operations), and m is 16 eps = 1.6e-5 of the
// scene diagonal.  The abscissa test is skipped when a + b is small, where the
// division would magnify those errors.
__device__ __forceinline__ bool dif_maybe(const float4* __restrict__ wf, float rx, float ry, float rz, float eps,
                                          float m) {
    const float4 A = __ldg(wf), B = __ldg(wf + 1), C = __ldg(wf + 2), Dd = __ldg(wf + 3);
    const float cn = __ldg(reinterpret_cast<const float*>(wf + 4));
    const float dx = rx - A.x, dy = ry - A.y, dz = rz - A.z;
    const float xR = dx * B.x + dy * B.y + dz * B.z;
    const float x0 = dx * C.x + dy * C.y + dz * C.z;
    const float y0 = dx * Dd.x + dy * Dd.y + dz * Dd.z;
    if (y0 < -m && x0 * Dd.w - y0 * cn < -m) return false;   // inside the wedge
    const float b = sqrtf(x0 * x0 + y0 * y0);
    if (b < eps - m) return false;
    const float a = C.w;
    if (a + b > 1000.0f * eps) {
        const float xQ = (B.w * b + xR * a) / (a + b);
        if (xQ < -m || xQ > A.w + m) return false;
    }
    return true;
}

struct DifArgs {
    const float4* wf;   // Kw x 5: WedgeF of the candidates
    const double* wedge;
    const int2* wfaces;
    const int32_t* cw;   // candidate wedge ids (ascending)
    int Kw;
    D3 tx;
    const double* rx;
    int R;
    double eps;
    const BvhNode* nodes;
    const float4* tris;
    const float4* tri_v;   // vertex records (plane ids in the second's .w)
    uint32_t* bits;
    int64_t words;
    int32_t* status;
};

// One thread per (receiver, candidate wedge); sets bit k of receiver r's row for
// every valid diffraction path.
__global__ void __launch_bounds__(DIF_THREADS) k_dif_pairs(DifArgs A) {
    const int64_t n = (int64_t)A.R * A.Kw;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / A.Kw), k = (int)(i - (int64_t)r * A.Kw);
        const D3 R{A.rx[3 * r], A.rx[3 * r + 1], A.rx[3 * r + 2]};
        if (!dif_maybe(A.wf + 5 * (size_t)k, (float)R.x, (float)R.y, (float)R.z, (float)A.eps, 16.0f * (float)A.eps))
            continue;
        const int wi = __ldg(A.cw + k);
        const WedgeDev w = load_wedge(A.wedge, wi);
        Keller kp;
        if (!keller(w, A.tx, R, A.eps, kp)) continue;
        const int2 f = __ldg(A.wfaces + wi);
        // the receiver's segment first: it rejects more pairs than the transmitter's
        // (measured on the street canyon: 25 % of the Keller-valid pairs see the
        // receiver, 64 % the transmitter), so fewer long segments are queried
        const int pl0 = __float_as_int(__ldg(A.tri_v + 3 * f.x + 1).w);
        const int pl1 = __float_as_int(__ldg(A.tri_v + 3 * f.y + 1).w);
        if (!seg_clear(A.nodes, A.tris, kp.Q, R, A.eps, f.x, f.y, pl0, pl1, A.status)) continue;
        if (!seg_clear(A.nodes, A.tris, A.tx, kp.Q, A.eps, f.x, f.y, pl0, pl1, A.status)) continue;
        atomicOr(A.bits + (int64_t)r * A.words + (k >> 5), 1u << (k & 31));
    }
}

__global__ void k_dif_row_count(const uint32_t* __restrict__ bits, int R, int64_t words, int64_t* counts) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < R;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int64_t c = 0;
        for (int64_t w = lane; w < words; w += 32) c += __popc(bits[r * words + w]);
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (lane == 0) counts[r] = c;
    }
}

// Exclusive scan of R counts by one block: offsets[0..R].
__global__ void k_dif_scan(const int64_t* __restrict__ counts, int R, int64_t* offsets) {
    __shared__ int64_t s[1024];
    __shared__ int64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < R; b0 += 1024) {
        const int i = b0 + threadIdx.x;
        s[threadIdx.x] = i < R ? counts[i] : 0;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int64_t v = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += v;
            __syncthreads();
        }
        if (i < R) offsets[i + 1] = s_carry + s[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) offsets[0] = 0;
}

// One warp per receiver: its set bits in order give (receiver, candidate) per path.
__global__ void k_dif_expand(const uint32_t* __restrict__ bits, int R, int64_t words, const int64_t* __restrict__ off,
                             int32_t* __restrict__ prx, int32_t* __restrict__ pk) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < R;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        int64_t base = off[r];
        for (int64_t w0 = 0; w0 < words; w0 += 32) {
            const int64_t w = w0 + lane;
            uint32_t b = w < words ? bits[r * words + w] : 0u;
            const int c = __popc(b);
            int pre = c;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, pre, o);
                if (lane >= o) pre += v;
            }
            const int total = __shfl_sync(0xffffffffu, pre, 31);
            int64_t pos = base + pre - c;
            while (b) {
                const int bit = __ffs(b) - 1;
                b &= b - 1;
                prx[pos] = (int32_t)r;
                pk[pos] = (int32_t)(w * 32 + bit);
                ++pos;
            }
            base += total;
        }
    }
}

__device__ __forceinline__ void theta_hat(double kx, double ky, double kz, double out[3]) {
    const double th = acos(fmin(1.0, fmax(-1.0, kz)));
    const double ph = (kx == 0.0 && ky == 0.0) ? 0.0 : atan2(ky, kx);
    out[0] = cos(th) * cos(ph);
    out[1] = cos(th) * sin(ph);
    out[2] = -sin(th);
}

// reduce y to eps in [-n pi, n pi] (y - 2 pi n N, N the nearest integer)
__device__ __forceinline__ double reduce_angle(double y, double n) {
    const double p = 2.0 * DIF_PI * n;
    return y - p * rint(y / p);
}

struct RecArgs {
    const double* wedge;
    const int2* wfaces;
    const int32_t* cw;
    D3 tx;
    const double* rx;
    int64_t P;
    const int32_t* prx;
    const int32_t* pk;
    float* rec;          // DIF_REC x P
    double* eps64;       // 4 x P: the reduced angles eps_1..eps_4 in FP64
    int2* faces;         // P: (incidence face, other face)
    double* tau;
    double* pts;         // P x 4 x 3: Tx, Q, Rx, 0
    float4* dir;         // 2 x P: departure direction s', arrival direction -s (as the specular records)
    int32_t* depth;
    int32_t* tri;        // 2 x P
};

// Records of every path: the geometry of the field kernels in FP32 (angles and
// reduced angles formed in FP64), the delay and the points in FP64.
//   rec[0] n, [1] sin beta_0, [2] L, [3] A^d / s', [4] b_in, [5] p_in, [6] b_out,
//   [7] p_out, [8] cos theta on the incidence face, [9] on the other face,
//   [10..13] eps of T1..T4.
__global__ void k_dif_records(RecArgs A) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.P; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = A.prx[i], wi = __ldg(A.cw + A.pk[i]);
        const WedgeDev w = load_wedge(A.wedge, wi);
        const D3 R{A.rx[3 * r], A.rx[3 * r + 1], A.rx[3 * r + 2]};
        Keller kp;
        keller(w, A.tx, R, 0.0, kp);   // valid: decided by k_dif_pairs
        const int2 f = __ldg(A.wfaces + wi);
        const double lim = w.n * DIF_PI;
        const bool swap = kp.php > 0.5 * lim;
        const double php = swap ? lim - kp.php : kp.php, phi = swap ? lim - kp.phi : kp.phi;
        const D3 s_in = d3mul(1.0 / kp.sp, d3sub(kp.Q, A.tx)), s_out = d3mul(1.0 / kp.sd, d3sub(R, kp.Q));
        const D3 ci = d3cross(w.e, s_in), co = d3cross(w.e, s_out);
        const double sinb = d3norm(ci);
        const D3 ph_in = d3mul(1.0 / sinb, ci), ph_out = d3mul(1.0 / d3norm(co), co);
        const D3 be_in = d3cross(s_in, ph_in), be_out = d3cross(s_out, ph_out);
        double ti[3], tr[3];
        theta_hat(s_in.x, s_in.y, s_in.z, ti);
        theta_hat(-s_out.x, -s_out.y, -s_out.z, tr);
        const D3 Ti{ti[0], ti[1], ti[2]}, Tr{tr[0], tr[1], tr[2]};
        const double L = kp.sd * kp.sp * sinb * sinb / (kp.sd + kp.sp);
        const double spread = sqrt(kp.sp / (kp.sd * (kp.sd + kp.sp))) / kp.sp;
        float* rec = A.rec;
        const int64_t P = A.P;
        rec[0 * P + i] = (float)w.n;
        rec[1 * P + i] = (float)sinb;
        rec[2 * P + i] = (float)L;
        rec[3 * P + i] = (float)spread;
        rec[4 * P + i] = (float)d3dot(Ti, be_in);
        rec[5 * P + i] = (float)d3dot(Ti, ph_in);
        rec[6 * P + i] = (float)d3dot(Tr, be_out);
        rec[7 * P + i] = (float)d3dot(Tr, ph_out);
        rec[8 * P + i] = (float)fabs(sinb * sin(php));
        rec[9 * P + i] = (float)fabs(sinb * sin(lim - phi));
        const double d = phi - php, s = phi + php;
        const double ep[4] = {reduce_angle(DIF_PI + d, w.n), reduce_angle(DIF_PI - d, w.n),
                              reduce_angle(DIF_PI - s, w.n), reduce_angle(DIF_PI + s, w.n)};
        for (int k = 0; k < 4; ++k) {
            rec[(10 + k) * P + i] = (float)ep[k];
            A.eps64[k * P + i] = ep[k];
        }
        const int fi = swap ? f.y : f.x, fo = swap ? f.x : f.y;
        A.faces[i] = make_int2(fi, fo);
        A.tri[i] = fi;
        A.tri[P + i] = fo;
        A.depth[i] = 1;
        A.dir[i] = make_float4((float)s_in.x, (float)s_in.y, (float)s_in.z, 0.0f);
        A.dir[P + i] = make_float4((float)-s_out.x, (float)-s_out.y, (float)-s_out.z, 0.0f);
        A.tau[i] = dadd(kp.sp, kp.sd) / RT_C0;
        double* pt = A.pts + (size_t)12 * i;
        const D3 pp[4] = {A.tx, kp.Q, R, D3{0.0, 0.0, 0.0}};
        for (int k = 0; k < 4; ++k) {
            pt[3 * k] = pp[k].x;
            pt[3 * k + 1] = pp[k].y;
            pt[3 * k + 2] = pp[k].z;
        }
    }
}

// ------------------------------------------------------------------ fields
// F(X) of Kouyoumjian-Pathak in FP32.  X < 2: F = 2 j u e^{jX} (sqrt(pi)/2 e^{-j pi/4}
// - u sum_k (-j X)^k / (k! (2k + 1))), u = sqrt(X) (16 terms); X >= 2: with
// z = e^{j pi/4} u, int_u^inf e^{-j t^2} dt = e^{-j pi/4} sqrt(pi)/2 erfc(z), and
// the Laplace continued fraction erfc(z) = e^{-z^2} / sqrt(pi) / (z + 1/2 / (z +
// 1 / (z + 3/2 / (z + ...)))) gives F = z / (z + 1/2 / (z + 1 / (z + ...))),
// evaluated bottom-up from depth ceil(4 + 90 / X) (its truncation error is below
// 2e-8 at every X >= 2, measured against a 30-digit evaluation).  Both stay within
// ~1e-6 of the exact value in FP32.
__device__ __forceinline__ float2 transition_fn(float X) {
    const float u = sqrtf(X);
    if (X < 2.0f) {
        float sr = 0.0f, si = 0.0f, tr = 1.0f, ti = 0.0f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float inv = 1.0f / (float)(2 * k + 1);
            sr += tr * inv;
            si += ti * inv;
            const float f = X / (float)(k + 1);
            const float nr = ti * f, ni = -tr * f;   // t *= -j X / (k + 1)
            tr = nr;
            ti = ni;
        }
        const float q = 0.62665706865775012f;   // sqrt(pi) / 2 * cos(pi / 4)
        const float Ir = q - u * sr, Ii = -q - u * si;
        float sx, cx;
        sincosf(X, &sx, &cx);
        const float er = cx * Ir - sx * Ii, ei = cx * Ii + sx * Ir;   // e^{jX} I
        return make_float2(-2.0f * u * ei, 2.0f * u * er);            // 2 j u (e^{jX} I)
    }
    const float zr = u * 0.70710678118654752f, zi = zr;
    float tr = zr, ti = zi;
    const int depth = (int)ceilf(4.0f + 90.0f / X);
    for (int k = depth; k >= 1; --k) {
        const float h = 0.5f * (float)k;
        const float inv = h / (tr * tr + ti * ti);
        const float nr = zr + tr * inv, ni = zi - ti * inv;   // t = z + h / t
        tr = nr;
        ti = ni;
    }
    const float inv = 1.0f / (tr * tr + ti * ti);
    return make_float2((zr * tr + zi * ti) * inv, (zi * tr - zr * ti) * inv);   // z / t
}

// T = cot(eps / 2n) F(2 k L sin^2(eps / 2)); at |eps| < 1e-10 the two leading terms
// of its expansion n [sqrt(2 pi k L) sgn(eps) - 2 k L eps e^{j pi/4}] e^{j pi/4}.
__device__ __forceinline__ float2 utd_term(float eps, float n, float kL) {
    const float c = 0.70710678118654752f;
    if (fabsf(eps) < 1e-10f) {
        const float a = sqrtf(2.0f * 3.14159265358979f * kL) * (eps < 0.0f ? -1.0f : 1.0f);
        const float b = 2.0f * kL * eps;   // times e^{j pi/4}
        // n [a - b e^{j pi/4}] e^{j pi/4} = n [a e^{j pi/4} - b j]
        return make_float2(n * a * c, n * (a * c - b));
    }
    const float s = sinf(0.5f * eps);
    const float2 F = transition_fn(2.0f * kL * s * s);
    float sn, cs;
    sincosf(eps / (2.0f * n), &sn, &cs);
    const float ct = cs / sn;
    return make_float2(F.x * ct, F.y * ct);
}

// FP64 versions for the paths whose bracket cancels (below): the series below
// X = 6 (40 terms), the continued fraction above from depth ceil(5 + 260 / X)
// (measured against a 30-digit evaluation: within 3e-14 for every X >= 6).
struct C64 {
    double x, y;
};
__device__ __forceinline__ C64 zmul(C64 a, C64 b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ C64 zadd(C64 a, C64 b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ C64 zdiv(C64 a, C64 b) {
    const double d = b.x * b.x + b.y * b.y;
    return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
__device__ __forceinline__ C64 zsqrt(C64 z) {   // principal root, as csqrt
    const double r = sqrt(z.x * z.x + z.y * z.y);
    if (z.x >= 0.0) {
        const double t = sqrt(0.5 * (r + z.x));
        return {t, t > 0.0 ? z.y / (2.0 * t) : 0.0};
    }
    const double t = sqrt(0.5 * (r - z.x));
    return {fabs(z.y) / (2.0 * t), copysign(t, z.y)};
}

__device__ C64 transition_fn64(double X) {
    const double u = sqrt(X);
    if (X < 6.0) {
        double sr = 0.0, si = 0.0, tr = 1.0, ti = 0.0;
        for (int k = 0; k < 40; ++k) {
            const double inv = 1.0 / (double)(2 * k + 1);
            sr += tr * inv;
            si += ti * inv;
            const double f = X / (double)(k + 1);
            const double nr = ti * f, ni = -tr * f;
            tr = nr;
            ti = ni;
        }
        const double q = 0.62665706865775012560;   // sqrt(pi) / 2 * cos(pi / 4)
        const double Ir = q - u * sr, Ii = -q - u * si;
        const double sx = sin(X), cx = cos(X);
        const double er = cx * Ir - sx * Ii, ei = cx * Ii + sx * Ir;
        return {-2.0 * u * ei, 2.0 * u * er};
    }
    const double zr = u * 0.70710678118654752440, zi = zr;
    double tr = zr, ti = zi;
    const int depth = (int)ceil(5.0 + 260.0 / X);
    for (int k = depth; k >= 1; --k) {
        const double inv = 0.5 * (double)k / (tr * tr + ti * ti);
        const double nr = zr + tr * inv, ni = zi - ti * inv;
        tr = nr;
        ti = ni;
    }
    return zdiv(C64{zr, zi}, C64{tr, ti});
}

__device__ C64 utd_term64(double eps, double n, double kL) {
    if (fabs(eps) < 1e-12) {
        const double a = sqrt(2.0 * DIF_PI * kL) * (eps < 0.0 ? -1.0 : 1.0), c = 0.70710678118654752440;
        return {n * a * c, n * (a * c - 2.0 * kL * eps)};
    }
    const double s = sin(0.5 * eps);
    const C64 F = transition_fn64(2.0 * kL * s * s);
    double sn, cs;
    sincos(eps / (2.0 * n), &sn, &cs);
    const double ct = cs / sn;
    return {F.x * ct, F.y * ct};
}

__device__ void fresnel64(C64 eta, double c, C64& rp, C64& rl) {
    const double s2 = fmax(0.0, 1.0 - c * c);
    const C64 s = zsqrt(C64{eta.x - s2, eta.y});
    rp = zdiv(C64{c - s.x, -s.y}, C64{c + s.x, s.y});
    const C64 ec{c * eta.x, c * eta.y};
    rl = zdiv(C64{ec.x - s.x, ec.y - s.y}, C64{ec.x + s.x, ec.y + s.y});
}

struct DifField {
    int64_t P;
    const float* rec;
    const double* eps64;
    const int2* faces;
    const int32_t* tri_material;
    const uint8_t* is_pec;
    const float* eps;
    const float* sig;
    int per_tri;
    float k, lam, w_eps0;   // wave number, wavelength, eps0 omega
    double k64, w_eps0_64;
    float gtx, grx;
};

struct DifPath {
    float2 pre, T3, T4, T12;
    float K, bb, pp;    // lambda / 4 pi sqrt(gT gR) A^d / s', b_in b_out, p_in p_out
    float c0, cn;
    int m0, mn;
    bool pec0, pecn;
};

__device__ __forceinline__ DifPath dif_path(const DifField& F, int64_t i) {
    const int64_t P = F.P;
    const float* r = F.rec;
    DifPath d;
    const float n = __ldg(r + i), sinb = __ldg(r + P + i), L = __ldg(r + 2 * P + i);
    const float kL = F.k * L;
    d.K = F.lam * 0.079577471545947668f * sqrtf(F.gtx * F.grx) * __ldg(r + 3 * P + i);   // lambda / (4 pi)
    d.bb = __ldg(r + 4 * P + i) * __ldg(r + 6 * P + i);
    d.pp = __ldg(r + 5 * P + i) * __ldg(r + 7 * P + i);
    d.c0 = __ldg(r + 8 * P + i);
    d.cn = __ldg(r + 9 * P + i);
    const float2 T1 = utd_term(__ldg(r + 10 * P + i), n, kL), T2 = utd_term(__ldg(r + 11 * P + i), n, kL);
    d.T3 = utd_term(__ldg(r + 12 * P + i), n, kL);
    d.T4 = utd_term(__ldg(r + 13 * P + i), n, kL);
    d.T12 = make_float2(T1.x + T2.x, T1.y + T2.y);
    // -e^{-j pi/4} / (2 n sqrt(2 pi k) sin beta_0)
    const float m = 1.0f / (2.0f * n * sqrtf(2.0f * 3.14159265358979f * F.k) * sinb);
    d.pre = make_float2(-0.70710678118654752f * m, 0.70710678118654752f * m);
    const int2 f = __ldg(F.faces + i);
    const int mt0 = __ldg(F.tri_material + f.x), mtn = __ldg(F.tri_material + f.y);
    d.pec0 = __ldg(F.is_pec + mt0) != 0;
    d.pecn = __ldg(F.is_pec + mtn) != 0;
    d.m0 = F.per_tri ? f.x : mt0;
    d.mn = F.per_tri ? f.y : mtn;
    return d;
}

__device__ __forceinline__ float2 eta_of(const DifField& F, int m) {
    return make_float2(__ldg(F.eps + m), -__ldg(F.sig + m) / F.w_eps0);
}

// v = b_in b_out [T1 + T2 + R_0s T3 + R_ns T4] + p_in p_out [T1 + T2 + R_0h T3 + R_nh T4]
// in FP32; `cancels` is set where |v| is below 1e-3 of the sum of the magnitudes
// of its terms (grazing incidence on, or grazing observation along, a face, where
// the field is nearly cancelled by its reflection): there the terms' FP32
// rounding (~1e-7 of each) would exceed 1e-4 of v, and the forward pass forms v
// again in FP64 (dif_bracket64).  About 0.5 % of the street canyon's paths.
__device__ __forceinline__ float2 dif_bracket(const DifPath& d, float2 R0s, float2 R0h, float2 Rns, float2 Rnh,
                                              bool& cancels) {
    const float2 bs = cadd(cadd(d.T12, cmul(R0s, d.T3)), cmul(Rns, d.T4));
    const float2 bh = cadd(cadd(d.T12, cmul(R0h, d.T3)), cmul(Rnh, d.T4));
    const float2 v = cadd(cscale(d.bb, bs), cscale(d.pp, bh));
    const float t3 = hypotf(d.T3.x, d.T3.y), t4 = hypotf(d.T4.x, d.T4.y), t12 = hypotf(d.T12.x, d.T12.y);
    const float mag = fabsf(d.bb) * (t12 + hypotf(R0s.x, R0s.y) * t3 + hypotf(Rns.x, Rns.y) * t4) +
                      fabsf(d.pp) * (t12 + hypotf(R0h.x, R0h.y) * t3 + hypotf(Rnh.x, Rnh.y) * t4);
    cancels = hypotf(v.x, v.y) < 1e-3f * mag;
    return v;
}

// v of dif_bracket in FP64 from the FP64 reduced angles and FP64 Fresnel coefficients.
__device__ float2 dif_bracket64(const DifField& F, const DifPath& d, int64_t i) {
    const int64_t P = F.P;
    const double n = __ldg(F.rec + i), kL = F.k64 * (double)__ldg(F.rec + 2 * P + i);
    C64 T[4];
    for (int k = 0; k < 4; ++k) T[k] = utd_term64(F.eps64[k * P + i], n, kL);
    C64 r0s{-1.0, 0.0}, r0h{1.0, 0.0}, rns{-1.0, 0.0}, rnh{1.0, 0.0};
    if (!d.pec0)
        fresnel64(C64{(double)__ldg(F.eps + d.m0), -(double)__ldg(F.sig + d.m0) / F.w_eps0_64}, (double)d.c0, r0s, r0h);
    if (!d.pecn)
        fresnel64(C64{(double)__ldg(F.eps + d.mn), -(double)__ldg(F.sig + d.mn) / F.w_eps0_64}, (double)d.cn, rns, rnh);
    const C64 u12 = zadd(T[0], T[1]);
    const C64 s = zadd(zadd(u12, zmul(r0s, T[2])), zmul(rns, T[3]));
    const C64 h = zadd(zadd(u12, zmul(r0h, T[2])), zmul(rnh, T[3]));
    return make_float2((float)(d.bb * s.x + d.pp * h.x), (float)(d.bb * s.y + d.pp * h.y));
}

// Forward in FP32; paths whose bracket cancels are appended to fb (fb[0] the
// count, reset before the launch, the list from fb + 4) for k_dif_fix.
__global__ void k_dif_fwd(DifField F, float2* __restrict__ a, double* __restrict__ tau_out,
                          const double* __restrict__ tau, int32_t* __restrict__ fb) {
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < F.P; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        bool cancels = false;
        if (i < F.P) {
            const DifPath d = dif_path(F, i);
            float2 R0s = make_float2(-1.0f, 0.0f), R0h = make_float2(1.0f, 0.0f), Rns = R0s, Rnh = R0h, u0, u1;
            if (!d.pec0) fresnel<false>(eta_of(F, d.m0), d.c0, R0s, R0h, u0, u1);
            if (!d.pecn) fresnel<false>(eta_of(F, d.mn), d.cn, Rns, Rnh, u0, u1);
            const float2 v = dif_bracket(d, R0s, R0h, Rns, Rnh, cancels);
            a[i] = cscale(d.K, cmul(d.pre, v));
            if (tau_out) tau_out[i] = tau[i];
        }
        // warp-aggregated append of the cancelling paths
        const unsigned m = __ballot_sync(0xffffffffu, cancels);
        if (m) {
            int base = 0;
            if (lane == 0) base = atomicAdd(fb, __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (cancels) fb[4 + base + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
        }
    }
}

// The listed paths again, with the bracket in FP64.  Item j goes to block
// j mod gridDim.x first, so that the few listed paths spread over all SMs (the
// FP64 pipe of one SM is the limit, not the lanes of a warp).
__global__ void k_dif_fix(DifField F, float2* __restrict__ a, const int32_t* __restrict__ fb) {
    const int n = *(volatile const int32_t*)fb;
    for (int j = threadIdx.x * gridDim.x + blockIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int64_t i = fb[4 + j];
        const DifPath d = dif_path(F, i);
        a[i] = cscale(d.K, cmul(d.pre, dif_bracket64(F, d, i)));
    }
}

// Adjoint: dL/deps_r = Re(conj(g) da/deta), dL/dsigma = Re(conj(g) da/deta (-j / (eps0 omega)))
// per face material, da/deta_0 = K pre T3 (b_in b_out dR_0s/deta + p_in p_out dR_0h/deta),
// likewise for face n with T4; dL/dg = Re(conj(g) a) / (2 g).  Gradients are
// accumulated (+=): per-block shared-memory sums for up to MAXM materials, else
// global atomics.
template <int MAXM>
__global__ void k_dif_bwd(DifField F, const float2* __restrict__ ga, float* __restrict__ geps, float* __restrict__ gsig,
                          float* __restrict__ ggain, int n_mat) {
    __shared__ float s_e[MAXM > 0 ? MAXM : 1], s_s[MAXM > 0 ? MAXM : 1], s_g[2];
    if (MAXM > 0)
        for (int m = threadIdx.x; m < n_mat; m += blockDim.x) s_e[m] = s_s[m] = 0.0f;
    if (threadIdx.x < 2) s_g[threadIdx.x] = 0.0f;
    __syncthreads();
    float gt = 0.0f, gr = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < F.P; i += (int64_t)gridDim.x * blockDim.x) {
        const DifPath d = dif_path(F, i);
        const float2 g = ga[i];
        float2 R0s = make_float2(-1.0f, 0.0f), R0h = make_float2(1.0f, 0.0f), Rns = R0s, Rnh = R0h;
        float2 d0s = make_float2(0.0f, 0.0f), d0h = d0s, dns = d0s, dnh = d0s;
        if (!d.pec0) fresnel<true>(eta_of(F, d.m0), d.c0, R0s, R0h, d0s, d0h);
        if (!d.pecn) fresnel<true>(eta_of(F, d.mn), d.cn, Rns, Rnh, dns, dnh);
        // a enters only the gain gradients, a sum over all paths: the FP32 bracket
        // suffices (the material terms below are products, free of cancellation)
        bool cancels;
        const float2 a = cscale(d.K, cmul(d.pre, dif_bracket(d, R0s, R0h, Rns, Rnh, cancels)));
        const float ra = g.x * a.x + g.y * a.y;   // Re(conj(g) a)
        gt += ra;
        gr += ra;
        const float2 kp = cscale(d.K, d.pre);
        for (int face = 0; face < 2; ++face) {
            if (face == 0 ? d.pec0 : d.pecn) continue;
            const float2 T = face == 0 ? d.T3 : d.T4;
            const float2 ds = face == 0 ? d0s : dns, dh = face == 0 ? d0h : dnh;
            const float2 da = cmul(cmul(kp, T), cadd(cscale(d.bb, ds), cscale(d.pp, dh)));   // da / deta
            const float ge = g.x * da.x + g.y * da.y;                                       // Re(conj(g) da)
            // da/dsigma = da/deta (-j / (eps0 omega)): Re(conj(g) (-j) da) / (eps0 omega)
            const float gs = (g.x * da.y - g.y * da.x) / F.w_eps0;
            const int m = face == 0 ? d.m0 : d.mn;
            if (MAXM > 0) {
                atomicAdd(s_e + m, ge);
                atomicAdd(s_s + m, gs);
            } else {
                atomicAdd(geps + m, ge);
                atomicAdd(gsig + m, gs);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        gt += __shfl_down_sync(0xffffffffu, gt, o);
        gr += __shfl_down_sync(0xffffffffu, gr, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(s_g, gt);
        atomicAdd(s_g + 1, gr);
    }
    __syncthreads();
    if (MAXM > 0)
        for (int m = threadIdx.x; m < n_mat; m += blockDim.x) {
            if (s_e[m] != 0.0f) atomicAdd(geps + m, s_e[m]);
            if (s_s[m] != 0.0f) atomicAdd(gsig + m, s_s[m]);
        }
    if (threadIdx.x == 0 && ggain) {
        atomicAdd(ggain, s_g[0] / (2.0f * F.gtx));
        atomicAdd(ggain + 1, s_g[1] / (2.0f * F.grx));
    }
}

}  // namespace

#define RT_EXPORT extern "C" __attribute__((visibility("default")))

RT_EXPORT rt_status rt_scene_wedges(rt_ctx* ctx, const rt_scene* scene, int32_t* n_wedges, int32_t* faces_host,
                                    double* n_host) {
    if (!ctx || !scene || !n_wedges) return RT_ERR_INVALID_ARG;
    rt_status s = ensure_wedges(ctx, scene);
    if (s != RT_OK) return s;
    *n_wedges = scene->n_wedges;
    if (faces_host) std::memcpy(faces_host, scene->h_wedge_faces, sizeof(int32_t) * 2 * (size_t)scene->n_wedges);
    if (n_host) std::memcpy(n_host, scene->h_wedge_n, sizeof(double) * (size_t)scene->n_wedges);
    return RT_OK;
}

RT_EXPORT rt_status rt_trace_diffraction(rt_ctx* ctx, const rt_scene* scene, const rt_paths* specular,
                                         const double tx[3], const double* rx_dev, int32_t n_rx, rt_paths** out) {
    if (!ctx || !scene || !specular || !tx || !out) return RT_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_rx < 1 || !rx_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_rx must be >= 1 with a receiver array");
    if (specular->kind != 0 || specular->scene != scene || !specular->d_cand)
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "specular must be a specular trace of this scene");
    RT_REQUIRE_RESOLVED(ctx, specular);
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(tx[c])) return rt_fail(ctx, RT_ERR_INVALID_ARG, "non-finite transmitter");
    rt_status s = ensure_wedges(ctx, scene);
    if (s != RT_OK) return s;
    cudaStream_t st = ctx->stream;
    const int W = scene->n_wedges;
    rt_paths* p = new rt_paths();
    p->scene = scene;
    p->stream = st;
    p->D = 2;
    p->R = n_rx;
    p->kind = 2;
    // temporaries of the call (freed on every exit)
    uint8_t* flag = nullptr;
    int32_t* list = nullptr;
    int32_t* count = nullptr;
    float4* wf = nullptr;
    uint32_t* bits = nullptr;
    int64_t* counts = nullptr;
    int32_t* pk = nullptr;
    auto release = [&]() {
        for (void* q : {(void*)flag, (void*)list, (void*)wf, (void*)bits, (void*)counts, (void*)pk})
            if (q) cudaFreeAsync(q, st);
    };
    auto fail = [&](rt_status e) {
        release();
        rt_paths_free(p);
        return e;
    };
#define DCK(call)                                                         \
    do {                                                                  \
        cudaError_t _e = (call);                                          \
        if (_e != cudaSuccess) return fail(rt_cuda_fail(ctx, _e, #call)); \
    } while (0)
    DCK(cudaMallocAsync((void**)&p->d_rx_offsets, (size_t)(n_rx + 1) * 8, st));
    // candidate wedges
    const size_t Wa = std::max(W, 1);
    DCK(cudaMallocAsync((void**)&flag, Wa, st));
    DCK(cudaMallocAsync((void**)&list, Wa * 4 + 64, st));
    count = list + Wa + 8;
    DCK(cudaMemsetAsync(flag, 0, Wa, st));
    if (W > 0 && specular->K > 0) {
        k_dif_candidates<<<dif_grid(ctx, specular->K, 256, 8), 256, 0, st>>>(specular->d_cand, specular->K,
                                                                            scene->d_tri_wedges, flag);
        RT_COUNT(ctx);
    }
    k_dif_compact<<<1, 1024, 0, st>>>(flag, W, list, count);
    RT_COUNT(ctx);
    DCK(cudaGetLastError());
    int64_t* hp = ctx->h_pinned;
    DCK(cudaMemcpyAsync(hp, count, 4, cudaMemcpyDeviceToHost, st));
    DCK(cudaStreamSynchronize(st));
    const int Kw = *(int32_t*)hp;   // p->K stays 0: a diffraction paths object has no candidate keys
    // valid (receiver, wedge) pairs
    const int64_t words = std::max<int64_t>(1, ((int64_t)Kw + 31) / 32);
    DCK(cudaMallocAsync((void**)&bits, (size_t)n_rx * words * 4, st));
    DCK(cudaMallocAsync((void**)&counts, (size_t)n_rx * 8, st));
    DCK(cudaMemsetAsync(bits, 0, (size_t)n_rx * words * 4, st));
    if (Kw > 0) {
        DCK(cudaMallocAsync((void**)&wf, (size_t)Kw * 5 * sizeof(float4), st));
        k_dif_prep<<<dif_grid(ctx, Kw, 128, 4), 128, 0, st>>>(scene->d_wedge, list, Kw, D3{tx[0], tx[1], tx[2]}, wf);
        RT_COUNT(ctx);
        DifArgs A{};
        A.wf = wf;
        A.wedge = scene->d_wedge;
        A.wfaces = scene->d_wedge_faces;
        A.cw = list;
        A.Kw = Kw;
        A.tx = D3{tx[0], tx[1], tx[2]};
        A.rx = rx_dev;
        A.R = n_rx;
        A.eps = scene->eps;
        A.nodes = scene->d_nodes;
        A.tris = scene->d_bvh_tris;
        A.tri_v = scene->d_tri_v;
        A.bits = bits;
        A.words = words;
        A.status = ctx->d_status;
        k_dif_pairs<<<dif_grid(ctx, (int64_t)n_rx * Kw, DIF_THREADS, 16), DIF_THREADS, 0, st>>>(A);
        RT_COUNT(ctx);
        DCK(cudaGetLastError());
    }
    k_dif_row_count<<<dif_grid(ctx, (int64_t)n_rx * 32, 256, 16), 256, 0, st>>>(bits, n_rx, words, counts);
    RT_COUNT(ctx);
    k_dif_scan<<<1, 1024, 0, st>>>(counts, n_rx, p->d_rx_offsets);
    RT_COUNT(ctx);
    DCK(cudaGetLastError());
    DCK(cudaMemcpyAsync(hp, p->d_rx_offsets + n_rx, 8, cudaMemcpyDeviceToHost, st));
    DCK(cudaStreamSynchronize(st));
    const int64_t P = hp[0];
    p->P = P;
    const size_t Pa = std::max<int64_t>(P, 1);
    {
        RtCarve c;
        const size_t o_pts = c.take(Pa * 4 * 3 * 8), o_depth = c.take(Pa * 4), o_rx = c.take(Pa * 4),
                     o_tri = c.take(Pa * 2 * 4);
        char* b = nullptr;
        DCK(cudaMallocAsync((void**)&b, c.off, st));
        p->d_block_geo = b;
        p->d_pts = reinterpret_cast<double*>(b + o_pts);
        p->d_depth = reinterpret_cast<int32_t*>(b + o_depth);
        p->d_rx = reinterpret_cast<int32_t*>(b + o_rx);
        p->d_tri = reinterpret_cast<int32_t*>(b + o_tri);
    }
    {
        RtCarve c;
        const size_t o_tau = c.take(Pa * 8), o_rec = c.take(Pa * DIF_REC * 4), o_f = c.take(Pa * sizeof(int2)),
                     o_dir = c.take(Pa * 2 * sizeof(float4)), o_e64 = c.take(Pa * 4 * 8),
                     o_fb = c.take((Pa + 4) * 4);
        char* b = nullptr;
        DCK(cudaMallocAsync((void**)&b, c.off, st));
        p->d_block_rec = b;
        p->d_tau = reinterpret_cast<double*>(b + o_tau);
        p->d_dir = reinterpret_cast<float4*>(b + o_dir);
        p->d_dif64 = reinterpret_cast<double*>(b + o_e64);
        p->d_dif_fb = reinterpret_cast<int32_t*>(b + o_fb);
        p->d_dif = reinterpret_cast<float*>(b + o_rec);
        p->d_dif_faces = reinterpret_cast<int2*>(b + o_f);
    }
    if (P > 0) {
        DCK(cudaMallocAsync((void**)&pk, Pa * 4, st));
        k_dif_expand<<<dif_grid(ctx, (int64_t)n_rx * 32, 256, 16), 256, 0, st>>>(bits, n_rx, words, p->d_rx_offsets,
                                                                                   p->d_rx, pk);
        RT_COUNT(ctx);
        RecArgs RA;
        RA.wedge = scene->d_wedge;
        RA.wfaces = scene->d_wedge_faces;
        RA.cw = list;
        RA.tx = D3{tx[0], tx[1], tx[2]};
        RA.rx = rx_dev;
        RA.P = P;
        RA.prx = p->d_rx;
        RA.pk = pk;
        RA.rec = p->d_dif;
        RA.eps64 = p->d_dif64;
        RA.faces = p->d_dif_faces;
        RA.tau = p->d_tau;
        RA.pts = p->d_pts;
        RA.dir = p->d_dir;
        RA.depth = p->d_depth;
        RA.tri = p->d_tri;
        k_dif_records<<<dif_grid(ctx, P, 128, 16), 128, 0, st>>>(RA);
        RT_COUNT(ctx);
        DCK(cudaGetLastError());
    }
    release();
#undef DCK
    *out = p;
    return RT_OK;
}

static rt_status dif_field_args(rt_ctx* ctx, const rt_paths* paths, const float* eps, const float* sig,
                                int32_t per_triangle, double freq_hz, float gtx, float grx, DifField& F) {
    if (!ctx || !paths) return RT_ERR_INVALID_ARG;
    if (paths->kind != 2) return rt_fail(ctx, RT_ERR_INVALID_ARG, "not a diffraction paths object");
    if (!eps || !sig) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null material array");
    if (per_triangle != 0 && per_triangle != 1) return rt_fail(ctx, RT_ERR_INVALID_ARG, "per_triangle must be 0 or 1");
    if (!(freq_hz > 0.0) || !std::isfinite(freq_hz)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "frequency must be > 0");
    if (!(gtx > 0.0f) || !(grx > 0.0f)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "antenna gains must be > 0");
    F.P = paths->P;
    F.rec = paths->d_dif;
    F.eps64 = paths->d_dif64;
    F.k64 = 2.0 * RT_PI * freq_hz / RT_C0;
    F.w_eps0_64 = RT_EPS0 * 2.0 * RT_PI * freq_hz;
    F.faces = paths->d_dif_faces;
    F.tri_material = paths->scene->d_tri_material;
    F.is_pec = paths->scene->d_is_pec;
    F.eps = eps;
    F.sig = sig;
    F.per_tri = per_triangle;
    F.k = (float)(2.0 * RT_PI * freq_hz / RT_C0);
    F.lam = (float)(RT_C0 / freq_hz);
    F.w_eps0 = (float)(RT_EPS0 * 2.0 * RT_PI * freq_hz);
    F.gtx = gtx;
    F.grx = grx;
    return RT_OK;
}

RT_EXPORT rt_status rt_eval_fields_diffraction(rt_ctx* ctx, const rt_paths* paths, const float* eps_r_dev,
                                               const float* sigma_dev, int32_t per_triangle, double freq_hz,
                                               float gain_tx, float gain_rx, void* a_dev, double* tau_dev) {
    DifField F;
    rt_status s = dif_field_args(ctx, paths, eps_r_dev, sigma_dev, per_triangle, freq_hz, gain_tx, gain_rx, F);
    if (s != RT_OK) return s;
    if (!a_dev && paths->P > 0) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null output");
    if (paths->P == 0) return RT_OK;
    RT_CK(ctx, cudaMemsetAsync(paths->d_dif_fb, 0, 4, ctx->stream));
    k_dif_fwd<<<dif_grid(ctx, paths->P, 256, 16), 256, 0, ctx->stream>>>(F, (float2*)a_dev, tau_dev, paths->d_tau,
                                                                         paths->d_dif_fb);
    RT_COUNT(ctx);
    k_dif_fix<<<ctx->num_sms, 64, 0, ctx->stream>>>(F, (float2*)a_dev, paths->d_dif_fb);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}

RT_EXPORT rt_status rt_eval_fields_diffraction_backward(rt_ctx* ctx, const rt_paths* paths, const float* eps_r_dev,
                                                        const float* sigma_dev, int32_t per_triangle, double freq_hz,
                                                        float gain_tx, float gain_rx, const void* grad_a_dev,
                                                        float* grad_eps_r_dev, float* grad_sigma_dev,
                                                        float* grad_gain_dev) {
    DifField F;
    rt_status s = dif_field_args(ctx, paths, eps_r_dev, sigma_dev, per_triangle, freq_hz, gain_tx, gain_rx, F);
    if (s != RT_OK) return s;
    if (!grad_eps_r_dev || !grad_sigma_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null gradient output");
    if (paths->P == 0) return RT_OK;
    if (!grad_a_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null dL/da");
    const int n_mat = per_triangle ? paths->scene->n_tris : paths->scene->n_materials;
    const int grid = dif_grid(ctx, paths->P, 256, 8);
    if (n_mat <= 256)
        k_dif_bwd<256><<<grid, 256, 0, ctx->stream>>>(F, (const float2*)grad_a_dev, grad_eps_r_dev, grad_sigma_dev,
                                                       grad_gain_dev, n_mat);
    else
        k_dif_bwd<0><<<grid, 256, 0, ctx->stream>>>(F, (const float2*)grad_a_dev, grad_eps_r_dev, grad_sigma_dev,
                                                     grad_gain_dev, n_mat);
    RT_COUNT(ctx);
    RT_CK_LAUNCH(ctx);
    return RT_OK;
}
