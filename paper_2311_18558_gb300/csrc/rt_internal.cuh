// Internal declarations of librt103 (GB300 / sm_103a).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "rt103.h"

// ---------------------------------------------------------------- constants
#define RT_C0 299792458.0              // speed of light [m/s] (CODATA)
#define RT_EPS0 8.8541878128e-12       // vacuum permittivity [F/m] (CODATA)
#define RT_PI 3.14159265358979323846
#define RT_MAX_DEPTH 4
#define RT_STACK 64                    // BVH traversal stack entries per thread
#define RT_MAX_VISITS (1 << 20)        // node-visit bound of one traversal

// ---------------------------------------------------------------- handles
#define RT_TRACE_WORDS 1024   // device trace words and pinned host words per context

struct rt_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int32_t* d_status = nullptr;       // sticky device status word (first error wins)
    // reusable scratch arena (grown on demand, freed with the context)
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // pinned host words for small readbacks (RT_TRACE_WORDS)
    int64_t* h_pinned = nullptr;
    // device words of one trace (RT_TRACE_WORDS): stage counters and capacity flags,
    // read back once at its end (batched traces: per-scene counts from word 64 on)
    unsigned long long* d_trace_words = nullptr;
    int64_t batch_paths_hint = 0;       // emitted paths of the last batched trace (0: none yet)
    struct rt_scene* batch_comb = nullptr;   // combined triangle tables of the last batch (one reference)
    std::vector<uint64_t> batch_key;    // serials of that batch's scenes
    // instrumentation
    int64_t launches = 0;              // kernels launched through this context
    int32_t profile = 0;               // bit 0: trace stage events, bit 1: traversal counters
    double stage_ms[8] = {0};
    unsigned long long* d_counters = nullptr;   // 8 device counters (bit 1)
    int64_t h_counters[8] = {0};                // host-side counts of the same slots
    cudaEvent_t ev[8] = {};                     // trace stage events (bit 0)
    // side stream for trace work that depends only on the inputs (the receivers'
    // tile order), forked from and joined back into the trace's stream
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int32_t* d_rx_order = nullptr;   // rx_order_cap entries
    int64_t rx_order_cap = 0;
    int32_t stage_pending = 0;                  // the last trace's events are recorded, not yet read
    // coherent processing order of the launch directions, per ray count (see trace.cu)
    int64_t sched_n = 0, sched_band = 0, sched_full = 0;
    int32_t* d_sched_order = nullptr;   // sched_band entries
    int32_t* d_sched_wrap = nullptr;    // sched_full entries
    float* d_sched_z = nullptr;         // sched_n entries: z of each launch direction
    // launch shapes of the tracing kernels (blocks per SM), set by the autotuner
    int tune_sbr_blocks_per_sm = 8;
    int tune_pairs_blocks_per_sm = 16;
    int tune_vis_blocks_per_sm = 8;
    int cfr_tensor_cores = 1;   // CFR on tcgen05 (3xTF32) where n_sub allows, else SIMT
    int32_t wait_limit = 0;     // polls of the CFR waits on other CTAs (0: the default 2^22)
    int32_t trace_async = 0;    // rt_trace_paths returns without waiting (paths counted on the device)
};

// Count one kernel launch of `ctx` (every launch site calls this).
#define RT_COUNT(ctx) (++(ctx)->launches)

// BVH2 node holding the boxes of both children (64 bytes).
//   a = (c0.lo.x, c0.lo.y, c0.lo.z, c0.hi.x)
//   b = (c0.hi.y, c0.hi.z, c1.lo.x, c1.lo.y)
//   c = (c1.lo.z, c1.hi.x, c1.hi.y, c1.hi.z)
//   d = (ref0, ref1, count0, count1): ref >= 0 -> inner node index ref;
//       ref < 0 -> leaf over the BVH-ordered triangles [first, first + count)
//       with ~ref = (first << 3) | (count - 1), count <= 8 (also in countN).
struct __align__(16) BvhNode {
    float4 a, b, c;
    int4 d;
};

struct rt_scene {
    rt_ctx* ctx = nullptr;
    int n_tris = 0, n_nodes = 0, n_materials = 0;
    int bvh_depth = 0;                 // most inner nodes on a root-to-leaf path (traversal stack bound)
    double diag = 0.0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};   // bounding box of the vertices [m]
    double eps = 0.0;                  // 1e-6 * diag: hit and segment guard [m]
    BvhNode* d_nodes = nullptr;
    float4* d_bvh_tris = nullptr;      // 3 float4 per triangle in BVH order: v0 (w = id bits), v1, v2
    float4* d_tri_v = nullptr;         // 3 float4 per triangle in original order: v0, v1, v2
    float4* d_tri_bary = nullptr;      // 3 float4 per triangle: plane (n, n.v0), g0 (h0), g1 (h1) (FP32)
    double* d_tri_n64 = nullptr;       // 4 doubles per triangle: unit normal (FP64), n.v0
    double* d_tri_bary64 = nullptr;    // 8 doubles per triangle: g0, h0, g1, h1 barycentric planes (FP64)
    int32_t* d_tri_material = nullptr;
    uint8_t* d_is_pec = nullptr;
    size_t hash_cap = 1u << 20;        // learned dedup table capacity
    size_t queue_cap = 1u << 20;       // learned visibility-queue capacity
    int64_t uniq_hint = 0;             // unique candidate keys of the last trace (0: none yet)
    int64_t paths_hint = 0;            // emitted paths of the last trace (0: none yet)
    uint8_t* h_is_pec = nullptr;       // host copy of the material PEC flags (batch checks)
    bool owns_tables_only = false;     // combined batch scene: no BVH, tables owned here
    int32_t refs = 0;                  // combined batch scene: paths objects and the context cache using it
    uint64_t serial = 0;               // unique per uploaded scene (keys the batch cache)
    // wedges for diffraction, built at the first rt_trace_diffraction / rt_scene_wedges
    int32_t n_wedges = -1;             // -1: not built yet
    double* d_wedge = nullptr;         // 14 doubles per wedge: start vertex, e, t0, n0 (3 each), length, n
    int2* d_wedge_faces = nullptr;     // per wedge (face 0, face n), face 0 < face n
    int32_t* d_tri_wedges = nullptr;   // 3 per triangle: wedges with the triangle as a face, -1 none
    int32_t* h_wedge_faces = nullptr;  // host copy of d_wedge_faces
    double* h_wedge_n = nullptr;       // host copy of n per wedge
};

struct rt_paths {
    const rt_scene* scene = nullptr;
    cudaStream_t stream = nullptr;     // stream the paths were made on (used to free them)
    int64_t P = 0, K = 0;
    int D = 0, R = 0;
    int64_t* d_rx_offsets = nullptr;   // R + 1
    // a trace that returned without waiting: P is the number of slots, the count
    // is d_count[0] (K in d_count[1], a capacity overflow flag in d_count[2]) until
    // rt_paths_resolve reads it
    int64_t* d_count = nullptr;
    int32_t* d_rx = nullptr;           // P
    int32_t* d_depth = nullptr;        // P
    int32_t* d_tri = nullptr;          // D x P (slot-major), -1 padded
    double* d_tau = nullptr;           // P
    float* d_len = nullptr;            // P
    int2* d_mc = nullptr;              // D x P per bounce j: .x material (bit 30 set for a PEC
                                       // material), .y the bits of cos(theta_i) as float
    float4* d_Dm = nullptr;            // (D + 1) x P basis changes D_1 .. D_{q+1} (row major 2x2)
    float4* d_dir = nullptr;           // 2 x P: departure direction k_1, arrival direction -k_{q+1} (unit, .w = 0)
    double* d_pts = nullptr;           // P x (D + 2) x 3
    uint64_t* d_cand = nullptr;        // K packed candidate keys
    rt_scene* owned_scene = nullptr;   // batch output: combined triangle tables, freed with the paths
    int32_t n_scenes = 1;              // batch output: number of traced scenes
    int64_t* h_scene_rx_off = nullptr; // batch output: receiver offset of each scene (n_scenes + 1)
    int64_t* h_scene_tri_off = nullptr;// batch output: triangle-id offset of each scene (n_scenes + 1)
    int32_t kind = 0;                  // 0: specular chains; 1: diffuse paths (last bounce diffuse);
                                       // 2: first-order diffraction paths
    int64_t n_rays = 0;                // diffuse paths: launch rays that sampled the surfaces
    const float2* d_chi = nullptr;     // diffuse paths: caller-owned per-path phases (chi_1, chi_2), or none
    float4* d_scat = nullptr;          // diffuse paths, P: (k_s.n, -k_i.k_s, k_r.k_s, 1/d_last) at the
                                       // diffuse point (n facing the incident wave)
    float* d_dif = nullptr;            // diffraction paths: DIF_REC x P records (in d_block_rec)
    double* d_dif64 = nullptr;         // diffraction paths: 4 x P reduced angles in FP64 (in d_block_rec)
    int32_t* d_dif_fb = nullptr;       // diffraction paths: count + list of paths re-evaluated in FP64
    int2* d_dif_faces = nullptr;       // diffraction paths: (incidence face, other face) per path
    // single allocations carved into several arrays (freed as a whole), or null
    void* d_block_geo = nullptr;       // d_rx, d_depth, d_tri, d_pts
    void* d_block_rec = nullptr;       // d_tau, d_len, d_mc, d_Dm, d_dir
};

// Offsets of arrays carved from one allocation, each on a 256-byte boundary.
struct RtCarve {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    }
};

// ---------------------------------------------------------------- error helpers
// Entry points that need the path count on the host refuse paths of a trace that
// returned without waiting (rt_paths_resolve first).
#define RT_REQUIRE_RESOLVED(ctx, p)                                                                     \
    do {                                                                                                \
        if ((p) && (p)->d_count)                                                                        \
            return rt_fail((ctx), RT_ERR_INVALID_ARG, "paths not resolved: call rt_paths_resolve first"); \
    } while (0)

rt_status rt_fail(rt_ctx* ctx, rt_status st, const char* fmt, ...);
rt_status rt_cuda_fail(rt_ctx* ctx, cudaError_t e, const char* what);
// Grow the context scratch arena to at least `bytes`; returns its base.
rt_status rt_scratch(rt_ctx* ctx, size_t bytes, void** base);
int32_t* rt_status_ptr(rt_ctx* ctx);
// Stage times of the last trace (profiling bit 0): waits for its last stage
// event and fills ctx->stage_ms; a no-op when nothing is pending.
rt_status rt_collect_stage_times(rt_ctx* ctx);

#define RT_CK(ctx, call)                                              \
    do {                                                              \
        cudaError_t _e = (call);                                      \
        if (_e != cudaSuccess) return rt_cuda_fail((ctx), _e, #call); \
    } while (0)

#define RT_CK_LAUNCH(ctx) RT_CK(ctx, cudaGetLastError())

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ void rt_set_status(int32_t* st, int32_t code) {
    if (st) atomicCAS(st, 0, code);
}

// Pack / unpack triangle sequences: id+1 in 16-bit fields, first bounce in the
// most significant field, 0 = no bounce.
__host__ __device__ __forceinline__ uint64_t rt_key_push(uint64_t key, int depth_before, int tri) {
    return key | ((uint64_t)(tri + 1) << (48 - 16 * depth_before));
}
__host__ __device__ __forceinline__ int rt_key_depth(uint64_t key) {
    int q = 0;
    for (int j = 0; j < 4; ++j) q += ((key >> (48 - 16 * j)) & 0xffffull) != 0;
    return q;
}
__host__ __device__ __forceinline__ int rt_key_tri(uint64_t key, int j) {
    return (int)((key >> (48 - 16 * j)) & 0xffffull) - 1;
}

// Kernel launchers (defined in the .cu files).
rt_status rt_launch_fields_fwd(rt_ctx* ctx, const rt_paths* p, const float* eps, const float* sig,
                               int per_tri, double freq, float gtx, float grx, float2* a, double* tau);
rt_status rt_launch_fields_bwd(rt_ctx* ctx, const rt_paths* p, const float* eps, const float* sig,
                               int per_tri, double freq, float gtx, float grx, const float2* ga,
                               float* geps, float* gsig, float* ggain);
// Geometry records (delay, length, cos(theta_i), basis changes) of every path
// from its points and triangles (d_pts, d_tri, d_depth must be filled).
// With P_dev, the paths are counted on the device (at most p->P, which then gives
// only the slots allocated): the records use that count as their stride.
rt_status rt_launch_paths_records(rt_ctx* ctx, rt_paths* p, const int64_t* P_dev = nullptr);
