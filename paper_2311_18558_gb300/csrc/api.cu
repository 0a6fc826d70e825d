// C ABI entry points of librt103: contexts, scenes (BVH build), path objects,
// field calls.  Tracing lives in trace.cu, CFR calls in cfr.cu.
#include <cuda_runtime.h>

#include <atomic>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "rt_internal.cuh"

// ---------------------------------------------------------------- errors / scratch

rt_status rt_fail(rt_ctx* ctx, rt_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

rt_status rt_cuda_fail(rt_ctx* ctx, cudaError_t e, const char* what) {
    rt_status st = (e == cudaErrorMemoryAllocation) ? RT_ERR_OOM : RT_ERR_CUDA;
    return rt_fail(ctx, st, "%s: %s", what, cudaGetErrorString(e));
}

rt_status rt_scratch(rt_ctx* ctx, size_t bytes, void** base) {
    if (bytes > ctx->scratch_bytes) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(ctx->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            return rt_fail(ctx, RT_ERR_CAPACITY,
                           "the scratch arena would grow inside a stream capture: run the call once before capturing");
        if (ctx->scratch) RT_CK(ctx, cudaFreeAsync(ctx->scratch, ctx->stream));
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
        size_t sz = bytes + bytes / 4 + (1 << 20);
        RT_CK(ctx, cudaMallocAsync(&ctx->scratch, sz, ctx->stream));
        ctx->scratch_bytes = sz;
    }
    *base = ctx->scratch;
    return RT_OK;
}

int32_t* rt_status_ptr(rt_ctx* ctx) { return ctx->d_status; }

// Loss partials of the fused CFR kernel: grow-only so that a call captured in a
// CUDA graph keeps valid pointers as long as n_rx does not grow.
struct LossScratch {
    double* part = nullptr;
    unsigned int* done = nullptr;
    int cap = 0;
    int* split_ints = nullptr;     // heavy-slot tables of the split fused CFR (6 per slot)
    int split_cap = 0;
    void* split_acc = nullptr;     // heavy-receiver grid rows
    size_t split_acc_bytes = 0;
    float* split_deconv = nullptr; // 4096 floats: per-column factors of the split receivers' transform
    int split_deconv_n = 0;        // n_sub the factors were made for (0: none yet)
};
static std::vector<std::pair<rt_ctx*, LossScratch>>& loss_table() {
    static std::vector<std::pair<rt_ctx*, LossScratch>> t;
    return t;
}

rt_status rt_cfr_fused_scratch(rt_ctx* ctx, int R, double** part, unsigned int** done) {
    LossScratch* ls = nullptr;
    for (auto& e : loss_table())
        if (e.first == ctx) ls = &e.second;
    if (!ls) {
        loss_table().push_back({ctx, LossScratch()});
        ls = &loss_table().back().second;
    }
    if (R > ls->cap) {
        if (ls->part) RT_CK(ctx, cudaFree(ls->part));
        if (ls->done) RT_CK(ctx, cudaFree(ls->done));
        ls->part = nullptr;
        ls->done = nullptr;
        int cap = std::max(R, 1024);
        RT_CK(ctx, cudaMalloc((void**)&ls->part, (size_t)cap * sizeof(double)));
        RT_CK(ctx, cudaMalloc((void**)&ls->done, 16 * sizeof(unsigned int)));
        RT_CK(ctx, cudaMemset(ls->done, 0, 16 * sizeof(unsigned int)));
        ls->cap = cap;
    }
    *part = ls->part;
    *done = ls->done;
    return RT_OK;
}

// Tables of the heavy-receiver split of the tensor-core fused CFR (grow-only,
// like the loss partials): 8 counters and 6 R ints (R heavy slots), zeroed when
// allocated, and acc_bytes for the slots' rows.
rt_status rt_cfr_split_scratch(rt_ctx* ctx, int R, size_t acc_bytes, int** ints, void** acc, float** deconv,
                               int** deconv_n) {
    LossScratch* ls = nullptr;
    for (auto& e : loss_table())
        if (e.first == ctx) ls = &e.second;
    if (!ls) {
        loss_table().push_back({ctx, LossScratch()});
        ls = &loss_table().back().second;
    }
    if (R > ls->split_cap) {
        if (ls->split_ints) RT_CK(ctx, cudaFree(ls->split_ints));
        ls->split_ints = nullptr;
        RT_CK(ctx, cudaMalloc((void**)&ls->split_ints, (6 * (size_t)R + 8) * sizeof(int)));
        RT_CK(ctx, cudaMemset(ls->split_ints, 0, (6 * (size_t)R + 8) * sizeof(int)));
        ls->split_cap = R;
    }
    if (acc_bytes > ls->split_acc_bytes) {
        if (ls->split_acc) RT_CK(ctx, cudaFree(ls->split_acc));
        ls->split_acc = nullptr;
        RT_CK(ctx, cudaMalloc(&ls->split_acc, acc_bytes));
        ls->split_acc_bytes = acc_bytes;
    }
    if (!ls->split_deconv) RT_CK(ctx, cudaMalloc((void**)&ls->split_deconv, 4096 * sizeof(float)));
    *ints = ls->split_ints;
    *acc = ls->split_acc;
    *deconv = ls->split_deconv;
    *deconv_n = &ls->split_deconv_n;
    return RT_OK;
}

static void loss_scratch_release(rt_ctx* ctx) {
    auto& t = loss_table();
    for (size_t i = 0; i < t.size(); ++i) {
        if (t[i].first == ctx) {
            if (t[i].second.part) cudaFree(t[i].second.part);
            if (t[i].second.done) cudaFree(t[i].second.done);
            if (t[i].second.split_ints) cudaFree(t[i].second.split_ints);
            if (t[i].second.split_acc) cudaFree(t[i].second.split_acc);
            if (t[i].second.split_deconv) cudaFree(t[i].second.split_deconv);
            t.erase(t.begin() + i);
            return;
        }
    }
}

// ---------------------------------------------------------------- context

extern "C" __attribute__((visibility("default"))) const char* rt_version(void) { return "rt103 1.0 (sm_103a)"; }

extern "C" __attribute__((visibility("default"))) rt_status rt_create(int device, void* cuda_stream, rt_ctx** out) {
    if (!out) return RT_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return RT_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return RT_ERR_CUDA;
    rt_ctx* ctx = new rt_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete ctx;
        return RT_ERR_CUDA;
    }
    if (prop.major < 10) {
        delete ctx;
        return RT_ERR_UNSUPPORTED;
    }
    ctx->num_sms = prop.multiProcessorCount;
    if (cudaMalloc((void**)&ctx->d_status, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->h_pinned, RT_TRACE_WORDS * 8) != cudaSuccess ||
        cudaMalloc((void**)&ctx->d_trace_words, RT_TRACE_WORDS * 8) != cudaSuccess) {
        delete ctx;
        return RT_ERR_OOM;
    }
    if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        delete ctx;
        return RT_ERR_CUDA;
    }
    *out = ctx;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_set_profiling(rt_ctx* ctx, int32_t flags) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (flags & ~3) return rt_fail(ctx, RT_ERR_INVALID_ARG, "profiling flags are bits 0 and 1");
    if ((flags & 1) && !ctx->ev[0])
        for (int k = 0; k < 8; ++k) RT_CK(ctx, cudaEventCreate(&ctx->ev[k]));
    if ((flags & 2) && !ctx->d_counters) RT_CK(ctx, cudaMalloc((void**)&ctx->d_counters, 8 * sizeof(unsigned long long)));
    if (ctx->d_counters) RT_CK(ctx, cudaMemsetAsync(ctx->d_counters, 0, 8 * sizeof(unsigned long long), ctx->stream));
    for (int k = 0; k < 8; ++k) {
        ctx->h_counters[k] = 0;
        ctx->stage_ms[k] = 0.0;
    }
    ctx->stage_pending = 0;
    ctx->profile = flags;
    return RT_OK;
}

rt_status rt_collect_stage_times(rt_ctx* ctx) {
    if (!ctx->stage_pending) return RT_OK;
    ctx->stage_pending = 0;
    RT_CK(ctx, cudaEventSynchronize(ctx->ev[5]));
    float ms = 0.f;
    // stages: SBR, dedup + sort (incl. candidate setup), image method, visibility, emission
    for (int k = 0; k < 5; ++k) {
        RT_CK(ctx, cudaEventElapsedTime(&ms, ctx->ev[k], ctx->ev[k + 1]));
        ctx->stage_ms[k] = ms;
    }
    RT_CK(ctx, cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[5]));
    ctx->stage_ms[5] = ms;
    RT_CK(ctx, cudaEventElapsedTime(&ms, ctx->ev[6], ctx->ev[7]));   // the SBR kernel alone
    ctx->stage_ms[6] = ms;
    RT_CK(ctx, cudaEventElapsedTime(&ms, ctx->ev[7], ctx->ev[1]));   // the FP64 re-trace
    ctx->stage_ms[7] = ms;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_profile_read(rt_ctx* ctx, int64_t* launches,
                                                                            double* stage_ms, int64_t* counters) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (launches) *launches = ctx->launches;
    if (stage_ms) {
        rt_status s = rt_collect_stage_times(ctx);
        if (s != RT_OK) return s;
        for (int k = 0; k < 8; ++k) stage_ms[k] = ctx->stage_ms[k];
    }
    if (counters) {
        unsigned long long d[8] = {0};
        if (ctx->d_counters) {
            RT_CK(ctx, cudaStreamSynchronize(ctx->stream));
            RT_CK(ctx, cudaMemcpy(d, ctx->d_counters, sizeof(d), cudaMemcpyDeviceToHost));
        }
        for (int k = 0; k < 8; ++k) counters[k] = (int64_t)d[k] + ctx->h_counters[k];
    }
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_destroy(rt_ctx* ctx) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    cudaStreamSynchronize(ctx->stream);
    for (int k = 0; k < 8; ++k)
        if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
    if (ctx->d_counters) cudaFree(ctx->d_counters);
    if (ctx->side) cudaStreamSynchronize(ctx->side);
    if (ctx->d_rx_order) cudaFree(ctx->d_rx_order);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->d_sched_order) cudaFree(ctx->d_sched_order);
    if (ctx->d_sched_wrap) cudaFree(ctx->d_sched_wrap);
    if (ctx->d_sched_z) cudaFree(ctx->d_sched_z);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->d_trace_words) cudaFree(ctx->d_trace_words);
    if (ctx->batch_comb && --ctx->batch_comb->refs == 0) rt_scene_free(ctx->batch_comb);
    loss_scratch_release(ctx);
    delete ctx;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_set_stream(rt_ctx* ctx, void* cuda_stream) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) const char* rt_last_error(const rt_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" __attribute__((visibility("default"))) rt_status rt_status_word(rt_ctx* ctx, int32_t* device_error) {
    if (!ctx || !device_error) return RT_ERR_INVALID_ARG;
    RT_CK(ctx, cudaStreamSynchronize(ctx->stream));
    RT_CK(ctx, cudaMemcpy(device_error, ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
    RT_CK(ctx, cudaMemset(ctx->d_status, 0, sizeof(int32_t)));
    return RT_OK;
}

// ---------------------------------------------------------------- BVH build (host)
// Binned-SAH BVH2 (16 bins per axis), at most 8 triangles per leaf, median
// split past depth 44 so the tree depth stays below the traversal stack.

namespace {

struct BTri {
    float lo[3], hi[3], c[3];
};
struct BNode {
    float lo[3], hi[3];
    int left = -1, right = -1, first = 0, count = 0;
};

constexpr int BINS = 16;
constexpr int LEAF_MAX = 8;

float area(const float* lo, const float* hi) {
    float e0 = std::max(0.0f, hi[0] - lo[0]), e1 = std::max(0.0f, hi[1] - lo[1]), e2 = std::max(0.0f, hi[2] - lo[2]);
    return 2.0f * (e0 * e1 + e1 * e2 + e2 * e0);
}

int build_rec(std::vector<BNode>& nodes, std::vector<int>& idx, const std::vector<BTri>& bt, int first, int count,
              int depth) {
    BNode nd;
    float clo[3], chi[3];
    for (int k = 0; k < 3; ++k) {
        nd.lo[k] = clo[k] = INFINITY;
        nd.hi[k] = chi[k] = -INFINITY;
    }
    for (int i = first; i < first + count; ++i) {
        const BTri& t = bt[idx[i]];
        for (int k = 0; k < 3; ++k) {
            nd.lo[k] = std::min(nd.lo[k], t.lo[k]);
            nd.hi[k] = std::max(nd.hi[k], t.hi[k]);
            clo[k] = std::min(clo[k], t.c[k]);
            chi[k] = std::max(chi[k], t.c[k]);
        }
    }
    nd.first = first;
    nd.count = count;
    int id = (int)nodes.size();
    nodes.push_back(nd);
    if (count <= 2) return id;

    int best_axis = -1, best_split = 0;
    float best_cost = INFINITY;
    if (depth <= 44) {
        for (int ax = 0; ax < 3; ++ax) {
            float ext = chi[ax] - clo[ax];
            if (!(ext > 0.0f)) continue;
            int cnt[BINS] = {0};
            float blo[BINS][3], bhi[BINS][3];
            for (int b = 0; b < BINS; ++b)
                for (int k = 0; k < 3; ++k) {
                    blo[b][k] = INFINITY;
                    bhi[b][k] = -INFINITY;
                }
            for (int i = first; i < first + count; ++i) {
                const BTri& t = bt[idx[i]];
                int b = std::min(BINS - 1, (int)((t.c[ax] - clo[ax]) / ext * BINS));
                cnt[b]++;
                for (int k = 0; k < 3; ++k) {
                    blo[b][k] = std::min(blo[b][k], t.lo[k]);
                    bhi[b][k] = std::max(bhi[b][k], t.hi[k]);
                }
            }
            float rlo[BINS][3], rhi[BINS][3];
            int rc[BINS];
            float alo[3] = {INFINITY, INFINITY, INFINITY}, ahi[3] = {-INFINITY, -INFINITY, -INFINITY};
            int ac = 0;
            for (int b = BINS - 1; b >= 1; --b) {
                for (int k = 0; k < 3; ++k) {
                    alo[k] = std::min(alo[k], blo[b][k]);
                    ahi[k] = std::max(ahi[k], bhi[b][k]);
                }
                ac += cnt[b];
                for (int k = 0; k < 3; ++k) {
                    rlo[b][k] = alo[k];
                    rhi[b][k] = ahi[k];
                }
                rc[b] = ac;
            }
            float llo[3] = {INFINITY, INFINITY, INFINITY}, lhi[3] = {-INFINITY, -INFINITY, -INFINITY};
            int lc = 0;
            for (int b = 0; b < BINS - 1; ++b) {
                for (int k = 0; k < 3; ++k) {
                    llo[k] = std::min(llo[k], blo[b][k]);
                    lhi[k] = std::max(lhi[k], bhi[b][k]);
                }
                lc += cnt[b];
                if (lc == 0 || rc[b + 1] == 0) continue;
                float cost = area(llo, lhi) * lc + area(rlo[b + 1], rhi[b + 1]) * rc[b + 1];
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = ax;
                    best_split = b + 1;
                }
            }
        }
    }
    float leaf_cost = area(nd.lo, nd.hi) * count;
    bool make_leaf = best_axis < 0 ? count <= LEAF_MAX : (best_cost + area(nd.lo, nd.hi) >= leaf_cost && count <= LEAF_MAX);
    if (make_leaf) return id;
    int mid;
    if (best_axis >= 0) {
        float ext = chi[best_axis] - clo[best_axis];
        auto it = std::partition(idx.begin() + first, idx.begin() + first + count, [&](int t) {
            int b = std::min(BINS - 1, (int)((bt[t].c[best_axis] - clo[best_axis]) / ext * BINS));
            return b < best_split;
        });
        mid = (int)(it - idx.begin());
    } else {
        mid = first;
    }
    if (mid <= first || mid >= first + count) {
        // median split along the widest centroid extent
        int ax = 0;
        for (int k = 1; k < 3; ++k)
            if (chi[k] - clo[k] > chi[ax] - clo[ax]) ax = k;
        mid = first + count / 2;
        std::nth_element(idx.begin() + first, idx.begin() + mid, idx.begin() + first + count, [&](int a, int b) {
            return bt[a].c[ax] < bt[b].c[ax] || (bt[a].c[ax] == bt[b].c[ax] && a < b);
        });
    }
    int l = build_rec(nodes, idx, bt, first, mid - first, depth + 1);
    int r = build_rec(nodes, idx, bt, mid, first + count - mid, depth + 1);
    nodes[id].left = l;
    nodes[id].right = r;
    return id;
}

__global__ void k_offsets_from_sorted(int64_t P, int R, const int32_t* __restrict__ rx, int64_t* offs) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= R; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = P;   // first i with rx[i] >= r
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (rx[mid] < r) lo = mid + 1;
            else hi = mid;
        }
        offs[r] = lo;
    }
}

}  // namespace

extern "C" __attribute__((visibility("default"))) rt_status rt_scene_upload(rt_ctx* ctx, const float* verts, int32_t n_verts, const int32_t* tris,
                                     int32_t n_tris, const int32_t* tri_material, int32_t n_materials,
                                     const uint8_t* is_pec, rt_scene** out) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!verts || !tris || !tri_material || !is_pec || !out) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    if (n_tris < 1 || n_tris > 65535) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_tris must be in [1, 65535]");
    if (n_verts < 3 || n_materials < 1) return rt_fail(ctx, RT_ERR_INVALID_ARG, "n_verts >= 3 and n_materials >= 1");
    *out = nullptr;
    for (int64_t i = 0; i < 3 * (int64_t)n_verts; ++i)
        if (!std::isfinite(verts[i])) return rt_fail(ctx, RT_ERR_NUMERIC, "non-finite vertex coordinate");
    std::vector<BTri> bt(n_tris);
    std::vector<float4> tv(3 * (size_t)n_tris), tb(3 * (size_t)n_tris);
    std::vector<double> tn(4 * (size_t)n_tris), tb64(8 * (size_t)n_tris);
    double glo[3] = {INFINITY, INFINITY, INFINITY}, ghi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int t = 0; t < n_tris; ++t) {
        double p[3][3];
        for (int v = 0; v < 3; ++v) {
            int vi = tris[3 * t + v];
            if (vi < 0 || vi >= n_verts) return rt_fail(ctx, RT_ERR_INVALID_ARG, "triangle %d: vertex index out of range", t);
            for (int k = 0; k < 3; ++k) p[v][k] = verts[3 * vi + k];
        }
        int m = tri_material[t];
        if (m < 0 || m >= n_materials) return rt_fail(ctx, RT_ERR_INVALID_ARG, "triangle %d: material out of range", t);
        double e1[3], e2[3], n[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = p[1][k] - p[0][k];
            e2[k] = p[2][k] - p[0][k];
        }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
        if (!(nn > 0.0)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "triangle %d is degenerate", t);
        double inv = 1.0 / std::sqrt(nn);
        double un[3] = {n[0] * inv, n[1] * inv, n[2] * inv};
        tn[4 * t + 0] = un[0];
        tn[4 * t + 1] = un[1];
        tn[4 * t + 2] = un[2];
        tn[4 * t + 3] = un[0] * p[0][0] + un[1] * p[0][1] + un[2] * p[0][2];
        for (int v = 0; v < 3; ++v) tv[3 * t + v] = make_float4((float)p[v][0], (float)p[v][1], (float)p[v][2], 0.0f);
        // barycentric planes: lambda_0 = g0.p + h0 with g0 = n x (v2 - v1) / |n|^2,
        // lambda_1 = g1.p + h1 with g1 = n x (v0 - v2) / |n|^2 (n unnormalised)
        auto bary = [&](int a, int b, float4& out, double* out64) {
            double d[3] = {p[b][0] - p[a][0], p[b][1] - p[a][1], p[b][2] - p[a][2]};
            double g[3] = {(n[1] * d[2] - n[2] * d[1]) / nn, (n[2] * d[0] - n[0] * d[2]) / nn,
                           (n[0] * d[1] - n[1] * d[0]) / nn};
            double h = -(g[0] * p[a][0] + g[1] * p[a][1] + g[2] * p[a][2]);
            out = make_float4((float)g[0], (float)g[1], (float)g[2], (float)h);
            out64[0] = g[0];
            out64[1] = g[1];
            out64[2] = g[2];
            out64[3] = h;
        };
        tb[3 * t] = make_float4((float)un[0], (float)un[1], (float)un[2], (float)tn[4 * t + 3]);
        bary(1, 2, tb[3 * t + 1], &tb64[8 * t]);
        bary(2, 0, tb[3 * t + 2], &tb64[8 * t + 4]);
        for (int k = 0; k < 3; ++k) {
            bt[t].lo[k] = (float)std::min({p[0][k], p[1][k], p[2][k]});
            bt[t].hi[k] = (float)std::max({p[0][k], p[1][k], p[2][k]});
            bt[t].c[k] = (float)((p[0][k] + p[1][k] + p[2][k]) / 3.0);
            glo[k] = std::min(glo[k], (double)bt[t].lo[k]);
            ghi[k] = std::max(ghi[k], (double)bt[t].hi[k]);
        }
    }
    for (int m = 0; m < n_materials; ++m)
        if (is_pec[m] > 1) return rt_fail(ctx, RT_ERR_INVALID_ARG, "material_is_pec must be 0 or 1");
    // plane ids: triangles whose FP64 plane records (unit normal, offset) are
    // bitwise equal share the id of the first of them.  A segment meets such a
    // plane once, so a triangle in the plane of a segment's end triangle can only
    // be met at that end (the visibility test skips it).  Stored in the .w of
    // the second vertex record (copied into the BVH triangle records).
    {
        struct Key {
            uint64_t b[4];
            bool operator==(const Key& o) const {
                return b[0] == o.b[0] && b[1] == o.b[1] && b[2] == o.b[2] && b[3] == o.b[3];
            }
        };
        struct KeyHash {
            size_t operator()(const Key& k) const {
                uint64_t h = 1469598103934665603ull;   // FNV-1a over the four words
                for (int i = 0; i < 4; ++i) h = (h ^ k.b[i]) * 1099511628211ull;
                return (size_t)h;
            }
        };
        std::unordered_map<Key, int32_t, KeyHash> first;
        first.reserve((size_t)n_tris * 2);
        for (int t = 0; t < n_tris; ++t) {
            Key k;
            double v[4];
            for (int i = 0; i < 4; ++i) v[i] = tn[4 * (size_t)t + i] + 0.0;   // -0.0 as +0.0
            std::memcpy(k.b, v, 32);
            const int32_t id = first.emplace(k, t).first->second;
            std::memcpy(&tv[3 * (size_t)t + 1].w, &id, 4);
        }
    }
    const double diag = std::sqrt((ghi[0] - glo[0]) * (ghi[0] - glo[0]) + (ghi[1] - glo[1]) * (ghi[1] - glo[1]) +
                                  (ghi[2] - glo[2]) * (ghi[2] - glo[2]));
    if (!(diag > 0.0)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "scene has zero extent");

    std::vector<BNode> nodes;
    std::vector<int> idx(n_tris);
    for (int t = 0; t < n_tris; ++t) idx[t] = t;
    build_rec(nodes, idx, bt, 0, n_tris, 0);

    // inner nodes in DFS order -> device layout with both child boxes
    const float pad = (float)(4e-6 * diag);
    std::vector<int> dev_index(nodes.size(), -1);
    std::vector<int> inner;
    {
        std::vector<int> st{0};
        while (!st.empty()) {
            int n = st.back();
            st.pop_back();
            if (nodes[n].left < 0) continue;
            dev_index[n] = (int)inner.size();
            inner.push_back(n);
            st.push_back(nodes[n].right);
            st.push_back(nodes[n].left);
        }
    }
    std::vector<BvhNode> dn;
    auto child = [&](int c, float* lo, float* hi, int& ref, int& cnt) {
        const BNode& b = nodes[c];
        for (int k = 0; k < 3; ++k) {
            lo[k] = b.lo[k] - pad;
            hi[k] = b.hi[k] + pad;
        }
        if (b.left < 0) {
            ref = b.first;
            cnt = b.count;
        } else {
            ref = dev_index[c];
            cnt = 0;
        }
    };
    if (inner.empty()) {
        // the whole scene is one leaf: root with that leaf and an empty child
        BvhNode r;
        float lo[3], hi[3];
        int ref, cnt;
        child(0, lo, hi, ref, cnt);
        r.a = make_float4(lo[0], lo[1], lo[2], hi[0]);
        r.b = make_float4(hi[1], hi[2], INFINITY, INFINITY);
        r.c = make_float4(INFINITY, -INFINITY, -INFINITY, -INFINITY);
        r.d = make_int4(cnt > 0 ? ~((ref << 3) | (cnt - 1)) : ref, ~0, cnt, 1);
        dn.push_back(r);
    } else {
        for (int n : inner) {
            float lo0[3], hi0[3], lo1[3], hi1[3];
            int r0, c0, r1, c1;
            child(nodes[n].left, lo0, hi0, r0, c0);
            child(nodes[n].right, lo1, hi1, r1, c1);
            BvhNode b;
            b.a = make_float4(lo0[0], lo0[1], lo0[2], hi0[0]);
            b.b = make_float4(hi0[1], hi0[2], lo1[0], lo1[1]);
            b.c = make_float4(lo1[2], hi1[0], hi1[1], hi1[2]);
            // child references as the traversal uses them: an inner child by its
            // node index (>= 0), a leaf as ~((first << 3) | (count - 1))
            b.d = make_int4(c0 > 0 ? ~((r0 << 3) | (c0 - 1)) : r0, c1 > 0 ? ~((r1 << 3) | (c1 - 1)) : r1, c0, c1);
            dn.push_back(b);
        }
    }
    std::vector<float4> btris(3 * (size_t)n_tris);
    for (int i = 0; i < n_tris; ++i) {
        int t = idx[i];
        btris[3 * i] = tv[3 * t];
        int id = t;
        float w;
        std::memcpy(&w, &id, 4);
        btris[3 * i].w = w;
        btris[3 * i + 1] = tv[3 * t + 1];
        btris[3 * i + 2] = tv[3 * t + 2];
    }

    rt_scene* sc = new rt_scene();
    static std::atomic<uint64_t> serials{0};
    sc->serial = ++serials;
    sc->ctx = ctx;
    sc->n_tris = n_tris;
    sc->n_nodes = (int)dn.size();
    {
        // most inner nodes on a root-to-leaf path: a traversal pushes at most one
        // child per inner node of its current path
        std::vector<std::pair<int, int>> st{{0, 1}};
        int depth = 1;
        while (!st.empty()) {
            const auto [n, dd] = st.back();
            st.pop_back();
            depth = std::max(depth, dd);
            for (int c : {dn[n].d.x, dn[n].d.y})
                if (c >= 0) st.push_back({c, dd + 1});
        }
        sc->bvh_depth = depth;
    }
    sc->n_materials = n_materials;
    sc->diag = diag;
    for (int k = 0; k < 3; ++k) {
        sc->lo[k] = glo[k];
        sc->hi[k] = ghi[k];
    }
    sc->eps = 1e-6 * diag;
    auto up = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(dst, bytes);
        if (e != cudaSuccess) return e;
        return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = up((void**)&sc->d_nodes, dn.data(), dn.size() * sizeof(BvhNode));
    if (e == cudaSuccess) e = up((void**)&sc->d_bvh_tris, btris.data(), btris.size() * sizeof(float4));
    if (e == cudaSuccess) e = up((void**)&sc->d_tri_v, tv.data(), tv.size() * sizeof(float4));
    if (e == cudaSuccess) e = up((void**)&sc->d_tri_bary, tb.data(), tb.size() * sizeof(float4));
    if (e == cudaSuccess) e = up((void**)&sc->d_tri_n64, tn.data(), tn.size() * sizeof(double));
    if (e == cudaSuccess) e = up((void**)&sc->d_tri_bary64, tb64.data(), tb64.size() * sizeof(double));
    if (e == cudaSuccess) e = up((void**)&sc->d_tri_material, tri_material, (size_t)n_tris * 4);
    if (e == cudaSuccess) e = up((void**)&sc->d_is_pec, is_pec, (size_t)n_materials);
    if (e != cudaSuccess) {
        rt_scene_free(sc);
        return rt_cuda_fail(ctx, e, "scene upload");
    }
    sc->h_is_pec = new uint8_t[n_materials];
    std::memcpy(sc->h_is_pec, is_pec, n_materials);
    *out = sc;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_scene_free(rt_scene* sc) {
    if (!sc) return RT_ERR_INVALID_ARG;
    cudaFree(sc->d_nodes);
    cudaFree(sc->d_bvh_tris);
    cudaFree(sc->d_tri_v);
    cudaFree(sc->d_tri_bary);
    cudaFree(sc->d_tri_n64);
    cudaFree(sc->d_tri_bary64);
    cudaFree(sc->d_tri_material);
    cudaFree(sc->d_is_pec);
    cudaFree(sc->d_wedge);
    cudaFree(sc->d_wedge_faces);
    cudaFree(sc->d_tri_wedges);
    delete[] sc->h_is_pec;
    delete[] sc->h_wedge_faces;
    delete[] sc->h_wedge_n;
    delete sc;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_scene_info(const rt_scene* sc, int32_t* n_tris, int32_t* n_nodes, double* diag) {
    if (!sc) return RT_ERR_INVALID_ARG;
    if (n_tris) *n_tris = sc->n_tris;
    if (n_nodes) *n_nodes = sc->n_nodes;
    if (diag) *diag = sc->diag;
    return RT_OK;
}

// ---------------------------------------------------------------- paths

extern "C" __attribute__((visibility("default"))) rt_status rt_paths_free(rt_paths* p) {
    if (!p) return RT_ERR_INVALID_ARG;
    cudaStream_t st = p->stream;
    if (p->d_block_geo) {
        cudaFreeAsync(p->d_block_geo, st);
        p->d_rx = nullptr;
        p->d_depth = nullptr;
        p->d_tri = nullptr;
        p->d_pts = nullptr;
    }
    if (p->d_block_rec) {
        cudaFreeAsync(p->d_block_rec, st);
        p->d_tau = nullptr;
        p->d_len = nullptr;
        p->d_mc = nullptr;
        p->d_Dm = nullptr;
        p->d_dir = nullptr;
    }
    void* ptrs[] = {p->d_rx_offsets, p->d_rx, p->d_depth, p->d_tri,  p->d_tau, p->d_len,
                    p->d_mc,         p->d_Dm, p->d_pts,   p->d_cand, p->d_dir, p->d_scat};
    for (void* q : ptrs)
        if (q) cudaFreeAsync(q, st);
    if (p->owned_scene && --p->owned_scene->refs == 0) {
        cudaStreamSynchronize(st);
        rt_scene_free(p->owned_scene);
    }
    delete[] p->h_scene_rx_off;
    delete[] p->h_scene_tri_off;
    delete p;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_paths_count(const rt_paths* p, int64_t* n_paths, int64_t* n_candidates) {
    if (!p) return RT_ERR_INVALID_ARG;
    if (n_paths) *n_paths = p->P;
    if (n_candidates) *n_candidates = p->K;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_paths_batch_info(const rt_paths* p, int32_t* n_scenes,
                                                                                int64_t* rx_off, int64_t* tri_off) {
    if (!p) return RT_ERR_INVALID_ARG;
    if (n_scenes) *n_scenes = p->n_scenes;
    for (int s = 0; s <= p->n_scenes; ++s) {
        if (rx_off) rx_off[s] = p->h_scene_rx_off ? p->h_scene_rx_off[s] : (s == 0 ? 0 : p->R);
        if (tri_off) tri_off[s] = p->h_scene_tri_off ? p->h_scene_tri_off[s] : (s == 0 ? 0 : p->scene->n_tris);
    }
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_paths_rx_offsets(const rt_paths* p, int64_t* offs) {
    if (!p || !offs) return RT_ERR_INVALID_ARG;
    rt_ctx* ctx = p->scene->ctx;
    RT_CK(ctx, cudaMemcpyAsync(offs, p->d_rx_offsets, (size_t)(p->R + 1) * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_paths_export(const rt_paths* p, int32_t* tri_seq, int32_t* depth, int32_t* rx, double* tau,
                                     double* points) {
    if (!p) return RT_ERR_INVALID_ARG;
    rt_ctx* ctx = p->scene->ctx;
    RT_REQUIRE_RESOLVED(ctx, p);
    cudaStream_t st = ctx->stream;
    if (p->P == 0) return RT_OK;
    if (tri_seq)
        for (int j = 0; j < p->D; ++j)
            RT_CK(ctx, cudaMemcpy2DAsync(tri_seq + j, (size_t)p->D * 4, p->d_tri + (size_t)j * p->P, 4, 4, p->P,
                                         cudaMemcpyDeviceToDevice, st));
    if (depth) RT_CK(ctx, cudaMemcpyAsync(depth, p->d_depth, p->P * 4, cudaMemcpyDeviceToDevice, st));
    if (rx) RT_CK(ctx, cudaMemcpyAsync(rx, p->d_rx, p->P * 4, cudaMemcpyDeviceToDevice, st));
    if (tau) RT_CK(ctx, cudaMemcpyAsync(tau, p->d_tau, p->P * 8, cudaMemcpyDeviceToDevice, st));
    if (points)
        RT_CK(ctx, cudaMemcpyAsync(points, p->d_pts, (size_t)p->P * (p->D + 2) * 3 * 8, cudaMemcpyDeviceToDevice, st));
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_paths_device_views(const rt_paths* p,
                                                                                  const int64_t** rx_offsets,
                                                                                  const double** tau) {
    if (!p) return RT_ERR_INVALID_ARG;
    if (rx_offsets) *rx_offsets = p->d_rx_offsets;
    if (tau) *tau = p->d_tau;
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_paths_candidates(const rt_paths* p, int32_t* seq) {
    if (!p || !seq) return RT_ERR_INVALID_ARG;
    rt_ctx* ctx = p->scene->ctx;
    RT_REQUIRE_RESOLVED(ctx, p);
    if (p->K == 0) return RT_OK;
    std::vector<uint64_t> keys(p->K);
    RT_CK(ctx, cudaMemcpyAsync(keys.data(), p->d_cand, p->K * 8, cudaMemcpyDeviceToHost, ctx->stream));
    RT_CK(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<int32_t> h((size_t)p->K * p->D);
    for (int64_t k = 0; k < p->K; ++k)
        for (int j = 0; j < p->D; ++j) h[(size_t)k * p->D + j] = rt_key_tri(keys[k], j);
    RT_CK(ctx, cudaMemcpyAsync(seq, h.data(), h.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    RT_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_paths_import(rt_ctx* ctx, const rt_scene* scene, int64_t n_paths, int32_t max_depth,
                                     int32_t n_rx, const int32_t* rx_dev, const int32_t* depth_dev,
                                     const int32_t* tri_seq_dev, const double* points_dev, rt_paths** out) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!scene || !out) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    if (n_paths < 0 || max_depth < 1 || max_depth > RT_MAX_DEPTH || n_rx < 1)
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "bad sizes");
    if (n_paths > 0 && (!rx_dev || !depth_dev || !tri_seq_dev || !points_dev))
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "null device pointer");
    *out = nullptr;
    cudaStream_t st = ctx->stream;
    rt_paths* p = new rt_paths();
    p->scene = scene;
    p->stream = st;
    p->P = n_paths;
    p->D = max_depth;
    p->R = n_rx;
    const size_t Pa = n_paths > 0 ? n_paths : 1;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** d, size_t b) {
        if (e == cudaSuccess) e = cudaMallocAsync(d, b, st);
    };
    A((void**)&p->d_rx_offsets, (size_t)(n_rx + 1) * 8);
    A((void**)&p->d_rx, Pa * 4);
    A((void**)&p->d_depth, Pa * 4);
    A((void**)&p->d_tri, Pa * max_depth * 4);
    A((void**)&p->d_pts, Pa * (max_depth + 2) * 3 * 8);
    if (e == cudaSuccess && n_paths > 0) {
        e = cudaMemcpyAsync(p->d_rx, rx_dev, n_paths * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_depth, depth_dev, n_paths * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_pts, points_dev, (size_t)n_paths * (max_depth + 2) * 3 * 8, cudaMemcpyDeviceToDevice, st);
        for (int j = 0; j < max_depth && e == cudaSuccess; ++j)
            e = cudaMemcpy2DAsync(p->d_tri + (size_t)j * n_paths, 4, tri_seq_dev + j, (size_t)max_depth * 4, 4, n_paths,
                                  cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess) {
        k_offsets_from_sorted<<<std::max(1, std::min(1024, (n_rx + 256) / 256)), 256, 0, st>>>(n_paths, n_rx, p->d_rx,
                                                                                                p->d_rx_offsets); RT_COUNT(ctx);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        rt_paths_free(p);
        return rt_cuda_fail(ctx, e, "paths import");
    }
    rt_status s = rt_launch_paths_records(ctx, p);
    if (s != RT_OK) {
        rt_paths_free(p);
        return s;
    }
    *out = p;
    return RT_OK;
}

// ---------------------------------------------------------------- fields

static rt_status check_fields(rt_ctx* ctx, const rt_paths* p, const float* eps, const float* sig, int per_tri,
                              double freq, float gtx, float grx) {
    if (!ctx) return RT_ERR_INVALID_ARG;
    if (!p || !eps || !sig) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null argument");
    if (p->kind != 0)
        return rt_fail(ctx, RT_ERR_INVALID_ARG,
                       "not a specular paths object (diffuse: rt_eval_fields_diffuse, diffraction: rt_eval_fields_diffraction)");
    if (per_tri != 0 && per_tri != 1) return rt_fail(ctx, RT_ERR_INVALID_ARG, "per_triangle must be 0 or 1");
    if (!(freq > 0.0) || !std::isfinite(freq)) return rt_fail(ctx, RT_ERR_INVALID_ARG, "freq_hz must be > 0");
    if (!(gtx > 0.0f) || !(grx > 0.0f) || !std::isfinite(gtx) || !std::isfinite(grx))
        return rt_fail(ctx, RT_ERR_INVALID_ARG, "antenna gains must be > 0");
    return RT_OK;
}

extern "C" __attribute__((visibility("default"))) rt_status rt_eval_fields(rt_ctx* ctx, const rt_paths* paths, const float* eps_r_dev, const float* sigma_dev,
                                    int32_t per_triangle, double freq_hz, float gain_tx, float gain_rx, void* a_dev,
                                    double* tau_dev) {
    rt_status s = check_fields(ctx, paths, eps_r_dev, sigma_dev, per_triangle, freq_hz, gain_tx, gain_rx);
    if (s != RT_OK) return s;
    if (!a_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null a_dev");
    return rt_launch_fields_fwd(ctx, paths, eps_r_dev, sigma_dev, per_triangle, freq_hz, gain_tx, gain_rx,
                                (float2*)a_dev, tau_dev);
}

extern "C" __attribute__((visibility("default"))) rt_status rt_eval_fields_backward(rt_ctx* ctx, const rt_paths* paths, const float* eps_r_dev,
                                             const float* sigma_dev, int32_t per_triangle, double freq_hz,
                                             float gain_tx, float gain_rx, const void* grad_a_dev,
                                             float* grad_eps_r_dev, float* grad_sigma_dev, float* grad_gain_dev) {
    rt_status s = check_fields(ctx, paths, eps_r_dev, sigma_dev, per_triangle, freq_hz, gain_tx, gain_rx);
    if (s != RT_OK) return s;
    if (!grad_a_dev) return rt_fail(ctx, RT_ERR_INVALID_ARG, "null grad_a_dev");
    return rt_launch_fields_bwd(ctx, paths, eps_r_dev, sigma_dev, per_triangle, freq_hz, gain_tx, gain_rx,
                                (const float2*)grad_a_dev, grad_eps_r_dev, grad_sigma_dev, grad_gain_dev);
}
