// api.cpp -- the C ABI of include/mcev.h: context, scene upload, per-frame
// setup and the host loop of Alg. 1 (rounds of batches over a device queue of
// undecided pixels, each round split into wavefront chunks).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mcev.h"
#include "bvh.h"
#include "kernels.h"
#include "quality.h"
#include "layout.h"
#include "tdist.h"

using namespace mcev;

// NVTX range for the lifetime of a scope (shows the library's calls, rounds
// and chunks on an Nsight timeline; a no-op when no tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// BVH node layout used unless mcev_params.bvh_width asks for the other
#ifndef MCEV_DEFAULT_BVH_WIDTH
#define MCEV_DEFAULT_BVH_WIDTH 2
#endif

namespace {

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct MeshInfo {
    int64_t first_tri, n_tri;   // in the uploaded triangle list
    int64_t tri_offset;         // first slot in the device triangle array
    int root;                   // BLAS root node (global index)
    float lo[3], hi[3];         // object-space bounds (root box)
};

struct Frame {
    DevFrame dev{};
    DevBuf buf;                 // TLAS nodes | instances | lights
    double time = 0.0;
    bool valid = false;
};

}  // namespace

struct mcev_ctx {
    int device = 0;
    int sms = 152;
    int32_t W = 0, H = 0;
    cudaStream_t stream = nullptr;
    mcev_alloc_fn alloc = nullptr;
    mcev_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    std::string err;
    mcev_params params{};
    int launches = 0;
    int32_t kcount[MCEV_K_CLASSES] = {0};
    double kms[MCEV_K_CLASSES] = {0};
    int64_t h2d = 0, d2h = 0;
    int64_t stats_pix = 0;                  // pixel visits of k_stats in the current call
    // profile mode: event pairs around launches, drained at round ends
    std::vector<cudaEvent_t> evpool;
    std::vector<int> evclass;
    size_t evused = 0;

    // host copy of the scene (needed per frame)
    bool have_scene = false;
    int32_t n_inst = 0, n_keys = 0, n_mats = 0;
    std::vector<float> vtx;                 // [tri][9] object space
    std::vector<int32_t> tri_mat;
    std::vector<MeshInfo> meshes;
    std::vector<int32_t> inst_mesh, inst_mat;
    std::vector<double> key_t, key_xf, cam_eye, cam_tgt, cam_up;
    double fov_deg = 45.0;
    std::vector<int32_t> mat_type;
    std::vector<float> mat_alb, mat_rough, mat_emit;
    std::vector<std::pair<int32_t, int64_t>> emitters;  // (instance, triangle)
    int32_t env_w = 0, env_h = 0;
    std::vector<float> env;
    bool env_ok = false;
    int sah_bins = 32, max_leaf = 4;
    int bvh_depth = 0;
    int bvh_width = MCEV_DEFAULT_BVH_WIDTH; // BLAS layout: 2 (two-wide nodes) or 8 (compressed wide)
    std::vector<float> tri_uv;              // [tri][6] texture coordinates (empty: no uvs)
    std::vector<char> inst_static;          // keyframes never change
    std::vector<float> static_vtx;          // world-space triangles of static instances
    bool has_static = false;
    int static_root = -1;
    float static_lo[3], static_hi[3];

    // device scene
    DevBuf d_quality;                       // event-quality scratch: two int32 volumes + accumulators
    DevBuf d_gemit;                         // FP64 emission-gradient accumulator of mcev_backward
    DevBuf d_nodes, d_wnodes, d_tris, d_tshade, d_uv, d_mats, d_env, d_marg, d_cond, d_tpdf;
    DevScene dsc{};
    Frame frames[2];

    // wavefront + per-pixel state
    DevBuf d_wave;
    Wave wave{};
    DevBuf d_counters;  // 16 int32: wave counters + error flag
    DevBuf d_pix;       // queues + cur + ref
    int32_t* queue[2] = {nullptr, nullptr};
    PixStats cur{}, ref{};
    bool ref_valid = false;
    double ref_time = 0.0;

    // batched renders run by this context: job table and union queues
    DevBuf d_jobs, d_bqueue;

    // device-resident round loop: its state and the stream graphs are captured on
    DevBuf d_round;
    cudaStream_t cap_stream = nullptr;

    // t critical values
    DevBuf d_tcrit;
    std::tuple<float, int, int, int, int> tcrit_key{-1.0f, -1, -1, -1, -1};

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

mcev_status fail(mcev_ctx* c, mcev_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MCEV_ERR_OOM : MCEV_ERR_CUDA,       \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define ST(call)                                   \
    do {                                           \
        mcev_status s_ = (call);                   \
        if (s_ != MCEV_OK) return s_;              \
    } while (0)

mcev_status dev_alloc(mcev_ctx* ctx, DevBuf& b, size_t bytes) {
    if (b.ptr && b.bytes >= bytes) return MCEV_OK;
    if (b.ptr) {
        if (ctx->alloc) ctx->free_fn(b.ptr, ctx->alloc_user);
        else cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
    }
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    if (ctx->alloc) {
        b.ptr = ctx->alloc(bytes, ctx->alloc_user);
        if (!b.ptr) return fail(ctx, MCEV_ERR_OOM, "allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&b.ptr, bytes);
        if (e != cudaSuccess) {
            b.ptr = nullptr;
            cudaGetLastError();
            return fail(ctx, MCEV_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        }
    }
    b.bytes = bytes;
    return MCEV_OK;
}

void dev_free(mcev_ctx* ctx, DevBuf& b) {
    if (!b.ptr) return;
    if (ctx->alloc) ctx->free_fn(b.ptr, ctx->alloc_user);
    else cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
}

mcev_status upload(mcev_ctx* ctx, DevBuf& b, const void* src, size_t bytes) {
    ST(dev_alloc(ctx, b, bytes));
    if (bytes) {
        CU(cudaMemcpyAsync(b.ptr, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        ctx->h2d += (int64_t)bytes;
    }
    return MCEV_OK;
}

// ---------------------------------------------------------------- per-kernel timing (profile mode)
mcev_status drain_events(mcev_ctx* ctx) {
    if (ctx->evused == 0) return MCEV_OK;
    CU(cudaEventSynchronize(ctx->evpool[ctx->evused - 1]));
    for (size_t i = 0; i + 1 < ctx->evused; i += 2) {
        float ms = 0.0f;
        CU(cudaEventElapsedTime(&ms, ctx->evpool[i], ctx->evpool[i + 1]));
        ctx->kms[ctx->evclass[i / 2]] += ms;
    }
    ctx->evused = 0;
    return MCEV_OK;
}

mcev_status ev_mark(mcev_ctx* ctx, int cls, bool start) {
    if (!ctx->params.profile) return MCEV_OK;
    if (start && ctx->evused + 2 > ctx->evpool.size()) {
        if (ctx->evpool.size() >= 8192) {
            ST(drain_events(ctx));
        } else {
            const size_t grow = ctx->evpool.size() ? ctx->evpool.size() : 256;
            for (size_t i = 0; i < grow; ++i) {
                cudaEvent_t e;
                CU(cudaEventCreate(&e));
                ctx->evpool.push_back(e);
            }
            ctx->evclass.resize(ctx->evpool.size() / 2);
        }
    }
    if (start) ctx->evclass[ctx->evused / 2] = cls;
    CU(cudaEventRecord(ctx->evpool[ctx->evused++], ctx->stream));
    return MCEV_OK;
}

const float* tri_uv_of(const mcev_ctx* ctx, int64_t prim) {
    static const float zeros[6] = {0, 0, 0, 0, 0, 0};
    return ctx->tri_uv.empty() ? zeros : &ctx->tri_uv[6 * (size_t)prim];
}

// ---------------------------------------------------------------- affine helpers (FP64)
void affine_inverse(const double* M, double* R) {
    const double a = M[0], b = M[1], c = M[2], d = M[4], e = M[5], f = M[6], g = M[8], h = M[9], i = M[10];
    const double A = e * i - f * h, B = -(d * i - f * g), Cc = d * h - e * g;
    const double det = a * A + b * B + c * Cc;
    const double id = 1.0 / det;
    const double inv[9] = {A * id, -(b * i - c * h) * id, (b * f - c * e) * id,
                           B * id, (a * i - c * g) * id,  -(a * f - c * d) * id,
                           Cc * id, -(a * h - b * g) * id, (a * e - b * d) * id};
    for (int r = 0; r < 3; ++r) {
        R[4 * r + 0] = inv[3 * r + 0];
        R[4 * r + 1] = inv[3 * r + 1];
        R[4 * r + 2] = inv[3 * r + 2];
        R[4 * r + 3] = -(inv[3 * r + 0] * M[3] + inv[3 * r + 1] * M[7] + inv[3 * r + 2] * M[11]);
    }
}

void xf_point(const double* M, const double* p, double* o) {
    for (int r = 0; r < 3; ++r) o[r] = M[4 * r] * p[0] + M[4 * r + 1] * p[1] + M[4 * r + 2] * p[2] + M[4 * r + 3];
}

void cross(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

double norm(const double* a) { return std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

uint32_t frame_key(double t) {
    uint64_t b;
    std::memcpy(&b, &t, sizeof b);
    return (uint32_t)(b ^ (b >> 32));
}

// ---------------------------------------------------------------- scene build
// One BVH per mesh that a moving instance uses (object space, shared by its
// instances) and one BVH over the world-space triangles of every instance
// whose keyframes never change (merged, so rays skip the instance level).
struct TriSrc {
    const float* v;  // 9 floats
    int32_t prim, mat, inst;
};

// texture coordinates of the uploaded triangle `prim` (6 floats; zeros without uvs)
const float* tri_uv_of(const mcev_ctx* ctx, int64_t prim);

mcev_status build_one(mcev_ctx* ctx, const std::vector<TriSrc>& src, std::vector<Node>& nodes,
                      std::vector<Node8>& wnodes, std::vector<float4>& tris, std::vector<float2>& uvs, int& root,
                      float lo_out[3], float hi_out[3], int& depth) {
    const int n = (int)src.size();
    std::vector<float> lo(3 * (size_t)n), hi(3 * (size_t)n), ce(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const float* v = src[i].v;
        for (int a = 0; a < 3; ++a) {
            lo[3 * i + a] = std::min(v[a], std::min(v[3 + a], v[6 + a]));
            hi[3 * i + a] = std::max(v[a], std::max(v[3 + a], v[6 + a]));
            ce[3 * i + a] = (float)(((double)v[a] + v[3 + a] + v[6 + a]) / 3.0);
        }
    }
    BuiltBvh b = build_bvh(lo.data(), hi.data(), ce.data(), n, ctx->sah_bins, ctx->max_leaf);
    const int64_t tri_off = (int64_t)tris.size() / 3;
    const std::vector<int>* leaf_order = &b.order;
    WideBvh wb;
    if (ctx->bvh_width == 8) {
        // the binary tree collapsed into compressed 8-wide nodes; the
        // triangles follow the wide leaves' order
        wb = collapse_wide(b, lo.data(), hi.data());
        if (!wb.ok) return fail(ctx, MCEV_ERR_STATE, "internal: wide BVH invariant violated");
        depth = std::max(depth, wb.depth);
        const uint32_t node_off = (uint32_t)wnodes.size();
        root = (int)node_off;
        for (Node8 nd : wb.nodes) {
            nd.child_base += node_off;
            nd.tri_base = (nd.tri_base & 0xE0000000u) | ((nd.tri_base & 0x1FFFFFFFu) + (uint32_t)tri_off);
            wnodes.push_back(nd);
        }
        leaf_order = &wb.tri_order;
    } else {
        depth = std::max(depth, b.depth);
        const int node_off = (int)nodes.size();
        root = node_off;
        for (Node nd : b.nodes) {
            if (nd.d.x >= 0) nd.d.x += node_off;
            else nd.d.x = ~(int)(tri_off + ~nd.d.x);
            if (nd.d.y >= 0) nd.d.y += node_off;
            else nd.d.y = ~(int)(tri_off + ~nd.d.y);
            nodes.push_back(nd);
        }
    }
    for (int k = 0; k < 3; ++k) {
        lo_out[k] = std::numeric_limits<float>::max();
        hi_out[k] = -std::numeric_limits<float>::max();
    }
    for (int i = 0; i < n; ++i) {
        const TriSrc& s = src[(*leaf_order)[i]];
        const float* v = s.v;
        float4 t0, t1, t2;
        t0.x = v[0]; t0.y = v[1]; t0.z = v[2];
        std::memcpy(&t0.w, &s.prim, 4);
        t1.x = v[3]; t1.y = v[4]; t1.z = v[5];
        std::memcpy(&t1.w, &s.mat, 4);
        t2.x = v[6]; t2.y = v[7]; t2.z = v[8];
        std::memcpy(&t2.w, &s.inst, 4);
        tris.push_back(t0);
        tris.push_back(t1);
        tris.push_back(t2);
        const float* tu = tri_uv_of(ctx, s.prim);
        for (int c = 0; c < 3; ++c) uvs.push_back(make_float2(tu[2 * c], tu[2 * c + 1]));
        for (int a = 0; a < 3; ++a) {
            lo_out[a] = std::min(lo_out[a], std::min(v[a], std::min(v[3 + a], v[6 + a])));
            hi_out[a] = std::max(hi_out[a], std::max(v[a], std::max(v[3 + a], v[6 + a])));
        }
    }
    return MCEV_OK;
}

mcev_status build_blas(mcev_ctx* ctx) {
    std::vector<Node> nodes;
    std::vector<Node8> wnodes;
    std::vector<float4> tris;
    std::vector<float2> uvs;
    tris.reserve(ctx->vtx.size() / 3);
    int depth = 0;
    const int ni = ctx->n_inst, nk = ctx->n_keys;
    ctx->inst_static.assign(ni, 1);
    for (int i = 0; i < ni; ++i)
        for (int k = 1; k < nk && ctx->inst_static[i]; ++k)
            if (std::memcmp(&ctx->key_xf[12 * ((size_t)k * ni + i)], &ctx->key_xf[12 * (size_t)i],
                            12 * sizeof(double)) != 0)
                ctx->inst_static[i] = 0;
    std::vector<char> mesh_dynamic(ctx->meshes.size(), 0);
    for (int i = 0; i < ni; ++i)
        if (!ctx->inst_static[i]) mesh_dynamic[ctx->inst_mesh[i]] = 1;
    for (size_t mi = 0; mi < ctx->meshes.size(); ++mi) {
        MeshInfo& m = ctx->meshes[mi];
        m.root = -1;
        if (!mesh_dynamic[mi]) continue;
        std::vector<TriSrc> src((size_t)m.n_tri);
        for (int64_t t = 0; t < m.n_tri; ++t) {
            const int64_t prim = m.first_tri + t;
            src[t] = TriSrc{&ctx->vtx[9 * (size_t)prim], (int32_t)prim, ctx->tri_mat[prim], -1};
        }
        ST(build_one(ctx, src, nodes, wnodes, tris, uvs, m.root, m.lo, m.hi, depth));
    }
    // merged static geometry in world space (keyframe 0 transform, FP64 -> FP32)
    ctx->static_vtx.clear();
    std::vector<TriSrc> ssrc;
    size_t n_static_tris = 0;
    for (int i = 0; i < ni; ++i)
        if (ctx->inst_static[i]) n_static_tris += (size_t)ctx->meshes[ctx->inst_mesh[i]].n_tri;
    // kernels address triangles as 3 * index in 32-bit arithmetic
    if (tris.size() / 3 + n_static_tris > ((size_t)1 << 29))
        return fail(ctx, MCEV_ERR_ARG, "more than 2^29 triangles once never-moving instances are baked");
    ctx->static_vtx.resize(9 * n_static_tris);
    ssrc.reserve(n_static_tris);
    size_t w = 0;
    for (int i = 0; i < ni; ++i) {
        if (!ctx->inst_static[i]) continue;
        const double* M = &ctx->key_xf[12 * (size_t)i];
        const MeshInfo& m = ctx->meshes[ctx->inst_mesh[i]];
        for (int64_t t = 0; t < m.n_tri; ++t) {
            const int64_t prim = m.first_tri + t;
            const float* v = &ctx->vtx[9 * (size_t)prim];
            float* o = &ctx->static_vtx[9 * w];
            for (int c = 0; c < 3; ++c) {
                const double p[3] = {v[3 * c], v[3 * c + 1], v[3 * c + 2]};
                double q[3];
                xf_point(M, p, q);
                o[3 * c] = (float)q[0];
                o[3 * c + 1] = (float)q[1];
                o[3 * c + 2] = (float)q[2];
            }
            const int32_t mat = ctx->inst_mat[i] >= 0 ? ctx->inst_mat[i] : ctx->tri_mat[prim];
            ssrc.push_back(TriSrc{o, (int32_t)prim, mat, i});
            ++w;
        }
    }
    ctx->static_root = -1;
    ctx->has_static = n_static_tris > 0;
    if (ctx->has_static)
        ST(build_one(ctx, ssrc, nodes, wnodes, tris, uvs, ctx->static_root, ctx->static_lo, ctx->static_hi, depth));
    if (nodes.empty()) {
        Node none;
        std::memset(&none, 0, sizeof none);
        nodes.push_back(none);
    }
    if (wnodes.empty()) {
        Node8 none;
        std::memset(&none, 0, sizeof none);
        wnodes.push_back(none);
    }
    if (tris.empty()) {
        tris.push_back(make_float4(0, 0, 0, 0));
        uvs.push_back(make_float2(0, 0));
    }
    // a traversal pushes at most one entry per inner-node level
    const int cap = ctx->bvh_width == 8 ? MCEV_WSTACK_HOST : MCEV_STACK_HOST;
    if (depth > cap) return fail(ctx, MCEV_ERR_ARG, "BVH depth %d exceeds the traversal stack (%d)", depth, cap);
    ctx->bvh_depth = depth;
    ST(upload(ctx, ctx->d_nodes, nodes.data(), nodes.size() * sizeof(Node)));
    ST(upload(ctx, ctx->d_wnodes, wnodes.data(), wnodes.size() * sizeof(Node8)));
    ctx->dsc.wnodes = (const uint4*)ctx->d_wnodes.ptr;
    ctx->dsc.wide = ctx->bvh_width == 8 ? 1 : 0;
    ST(upload(ctx, ctx->d_tris, tris.data(), tris.size() * sizeof(float4)));
    // shading records: the (object-space) edge cross product (v1 - v0) x (v2 - v0) of
    // each triangle's FP32 vertices, evaluated in FP64 and rounded, and its material
    std::vector<float4> tsh(tris.size() / 3);
    for (size_t t = 0; t < tsh.size(); ++t) {
        const float4 a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
        const double e1[3] = {(double)b.x - a.x, (double)b.y - a.y, (double)b.z - a.z};
        const double e2[3] = {(double)c.x - a.x, (double)c.y - a.y, (double)c.z - a.z};
        double cr[3];
        cross(e1, e2, cr);
        tsh[t] = make_float4((float)cr[0], (float)cr[1], (float)cr[2], b.w);
    }
    ST(upload(ctx, ctx->d_tshade, tsh.data(), tsh.size() * sizeof(float4)));
    ctx->dsc.tshade = (const float4*)ctx->d_tshade.ptr;
    ctx->dsc.nodes = (const Node*)ctx->d_nodes.ptr;
    ctx->dsc.tris = (const float4*)ctx->d_tris.ptr;
    if (!ctx->tri_uv.empty()) {
        ST(upload(ctx, ctx->d_uv, uvs.data(), uvs.size() * sizeof(float2)));
        ctx->dsc.tri_uv = (const float2*)ctx->d_uv.ptr;
    } else {
        ctx->dsc.tri_uv = nullptr;
    }
    for (auto& f : ctx->frames) f.valid = false;
    return MCEV_OK;
}

// Environment tables.  Row weights sum_j L_ij sin(pi (i + 1/2) / H), column
// weights L_ij; prefix sums in FP64 in index order, divided by the total and
// rounded to FP32, so the discrete texel choice is made on FP32 numbers.
mcev_status build_env(mcev_ctx* ctx) {
    const int W = ctx->env_w, H = ctx->env_h;
    std::vector<float> marg(H + 1), cond((size_t)H * (W + 1)), tpdf((size_t)W * H);
    std::vector<double> raw(W + 1), mraw(H + 1), rowsin(H);
    mraw[0] = 0.0;
    for (int i = 0; i < H; ++i) {
        const double sin_t = std::sin(M_PI * (i + 0.5) / H);
        rowsin[i] = sin_t;
        raw[0] = 0.0;
        for (int j = 0; j < W; ++j) raw[j + 1] = raw[j] + (double)ctx->env[(size_t)i * W + j];
        const double rowsum = raw[W];
        float* c = &cond[(size_t)i * (W + 1)];
        for (int j = 0; j < W; ++j) c[j] = rowsum > 0.0 ? (float)(raw[j] / rowsum) : (float)((double)j / W);
        c[W] = 1.0f;
        mraw[i + 1] = mraw[i] + rowsum * sin_t;
    }
    const double total = mraw[H];
    for (int i = 0; i < H; ++i) marg[i] = total > 0.0 ? (float)(mraw[i] / total) : (float)((double)i / H);
    marg[H] = 1.0f;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j)
            tpdf[(size_t)i * W + j] = total > 0.0 ? (float)((double)ctx->env[(size_t)i * W + j] * rowsin[i] / total *
                                                            (double)W * (double)H / (2.0 * M_PI * M_PI))
                                                  : 0.0f;
    ctx->env_ok = total > 0.0;
    ST(upload(ctx, ctx->d_env, ctx->env.data(), ctx->env.size() * sizeof(float)));
    ST(upload(ctx, ctx->d_marg, marg.data(), marg.size() * sizeof(float)));
    ST(upload(ctx, ctx->d_cond, cond.data(), cond.size() * sizeof(float)));
    ST(upload(ctx, ctx->d_tpdf, tpdf.data(), tpdf.size() * sizeof(float)));
    ctx->dsc.env = (const float*)ctx->d_env.ptr;
    ctx->dsc.env_marg = (const float*)ctx->d_marg.ptr;
    ctx->dsc.env_cond = (const float*)ctx->d_cond.ptr;
    ctx->dsc.env_tpdf = (const float*)ctx->d_tpdf.ptr;
    ctx->dsc.env_w = W;
    ctx->dsc.env_h = H;
    ctx->dsc.env_ok = ctx->env_ok ? 1 : 0;
    ctx->dsc.has_env = 1;
    return MCEV_OK;
}

// ---------------------------------------------------------------- per-frame state
mcev_status frame_setup(mcev_ctx* ctx, double t, int slot) {
    Frame& fr = ctx->frames[slot];
    if (fr.valid && fr.time == t) return MCEV_OK;
    const int ni = ctx->n_inst, nk = ctx->n_keys;
    int k = 0;
    double f = 0.0;
    if (nk > 1) {
        while (k + 1 < nk - 1 && ctx->key_t[k + 1] <= t) ++k;
        f = (t - ctx->key_t[k]) / (ctx->key_t[k + 1] - ctx->key_t[k]);
        f = std::min(1.0, std::max(0.0, f));
    }
    const int k1 = nk > 1 ? k + 1 : k;
    auto lerp = [f](double a, double b) { return (1.0 - f) * a + f * b; };
    std::vector<double> M((size_t)ni * 12), Mi((size_t)ni * 12);
    for (int i = 0; i < ni; ++i) {
        const double* A = &ctx->key_xf[12 * ((size_t)k * ni + i)];
        const double* B = &ctx->key_xf[12 * ((size_t)k1 * ni + i)];
        double* m = &M[12 * (size_t)i];
        for (int e = 0; e < 12; ++e) m[e] = lerp(A[e], B[e]);
        affine_inverse(m, &Mi[12 * (size_t)i]);
    }
    // instance records: every moving instance, then the merged static geometry
    std::vector<int> rec_inst;
    for (int i = 0; i < ni; ++i)
        if (!ctx->inst_static[i]) rec_inst.push_back(i);
    if (ctx->has_static) rec_inst.push_back(-1);
    const int nr = (int)rec_inst.size();
    std::vector<float> blo(3 * (size_t)nr), bhi(3 * (size_t)nr), bce(3 * (size_t)nr);
    std::vector<float4> inst((size_t)nr * 7);
    static const double ident[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    for (int r = 0; r < nr; ++r) {
        const int i = rec_inst[r];
        const double* m = i >= 0 ? &M[12 * (size_t)i] : ident;
        const double* mi = i >= 0 ? &Mi[12 * (size_t)i] : ident;
        const float* olo = i >= 0 ? ctx->meshes[ctx->inst_mesh[i]].lo : ctx->static_lo;
        const float* ohi = i >= 0 ? ctx->meshes[ctx->inst_mesh[i]].hi : ctx->static_hi;
        const bool empty = i >= 0 ? ctx->meshes[ctx->inst_mesh[i]].n_tri == 0 : false;
        float lo[3] = {std::numeric_limits<float>::max(), std::numeric_limits<float>::max(),
                       std::numeric_limits<float>::max()};
        float hi[3] = {-lo[0], -lo[1], -lo[2]};
        if (!empty) {
            for (int c = 0; c < 8; ++c) {
                const double q[3] = {(c & 1) ? ohi[0] : olo[0], (c & 2) ? ohi[1] : olo[1], (c & 4) ? ohi[2] : olo[2]};
                double wv[3];
                xf_point(m, q, wv);
                for (int a2 = 0; a2 < 3; ++a2) {
                    // round outwards so the FP32 box contains the FP64 corners
                    lo[a2] = std::min(lo[a2], std::nextafter((float)wv[a2], -INFINITY));
                    hi[a2] = std::max(hi[a2], std::nextafter((float)wv[a2], INFINITY));
                }
            }
        } else {
            for (int a2 = 0; a2 < 3; ++a2) lo[a2] = hi[a2] = 1e30f;
        }
        for (int a2 = 0; a2 < 3; ++a2) {
            blo[3 * r + a2] = lo[a2];
            bhi[3 * r + a2] = hi[a2];
            bce[3 * r + a2] = 0.5f * (lo[a2] + hi[a2]);
        }
        for (int row = 0; row < 3; ++row) {
            inst[7 * r + row] = make_float4((float)m[4 * row], (float)m[4 * row + 1], (float)m[4 * row + 2],
                                            (float)m[4 * row + 3]);
            inst[7 * r + 3 + row] = make_float4((float)mi[4 * row], (float)mi[4 * row + 1], (float)mi[4 * row + 2],
                                                (float)mi[4 * row + 3]);
        }
        int root = i >= 0 ? ctx->meshes[ctx->inst_mesh[i]].root : ctx->static_root;
        int ovr = i >= 0 ? ctx->inst_mat[i] : -1;
        int oid = i;
        float4 tail = make_float4(0, 0, 0, 0);
        std::memcpy(&tail.x, &root, 4);
        std::memcpy(&tail.y, &ovr, 4);
        std::memcpy(&tail.z, &oid, 4);
        inst[7 * r + 6] = tail;
    }
    // TLAS over the moving instances' records, one record per leaf; leaf
    // ref = ~record.  The merged static geometry (last record) stays out of
    // it: it spans the scene, and rays traverse it first.
    const int n_tlas = nr - (ctx->has_static ? 1 : 0);
    std::vector<Node> tlas;
    if (n_tlas > 1) {
        BuiltBvh b = build_bvh(blo.data(), bhi.data(), bce.data(), n_tlas, 16, 1);
        tlas = b.nodes;
        for (Node& nd : tlas) {
            if (nd.d.x < 0 && nd.d.z > 0) nd.d.x = ~b.order[~nd.d.x];
            if (nd.d.y < 0 && nd.d.w > 0) nd.d.y = ~b.order[~nd.d.y];
        }
        // the two-wide BLAS continue on the TLAS stack; wide BLAS have their own
        if (b.depth + (ctx->bvh_width == 8 ? 0 : ctx->bvh_depth) > MCEV_STACK_HOST)
            return fail(ctx, MCEV_ERR_ARG, "TLAS + BLAS depth exceeds the traversal stack (%d)", MCEV_STACK_HOST);
    }
    // emitters in world space
    std::vector<float4> lights(ctx->emitters.size() * 4);
    for (size_t l = 0; l < ctx->emitters.size(); ++l) {
        const int i = ctx->emitters[l].first;
        const int64_t prim = ctx->emitters[l].second;
        const double* m = &M[12 * (size_t)i];
        const float* v = &ctx->vtx[9 * (size_t)prim];
        double p[3][3];
        for (int c = 0; c < 3; ++c) {
            const double q[3] = {v[3 * c], v[3 * c + 1], v[3 * c + 2]};
            xf_point(m, q, p[c]);
        }
        double e1[3], e2[3], cr[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = p[1][a] - p[0][a];
            e2[a] = p[2][a] - p[0][a];
        }
        cross(e1, e2, cr);
        const double len = norm(cr);
        const int mat = ctx->inst_mat[i] >= 0 ? ctx->inst_mat[i] : ctx->tri_mat[prim];
        lights[4 * l + 0] = make_float4((float)p[0][0], (float)p[0][1], (float)p[0][2], ctx->mat_emit[mat]);
        lights[4 * l + 1] = make_float4((float)p[1][0], (float)p[1][1], (float)p[1][2], (float)(0.5 * len));
        float mat_bits;
        std::memcpy(&mat_bits, &mat, 4);
        lights[4 * l + 2] = make_float4((float)p[2][0], (float)p[2][1], (float)p[2][2], mat_bits);
        lights[4 * l + 3] = make_float4((float)(cr[0] / len), (float)(cr[1] / len), (float)(cr[2] / len), 0.0f);
    }
    const size_t nb_t = tlas.size() * sizeof(Node), nb_i = inst.size() * sizeof(float4),
                 nb_l = lights.size() * sizeof(float4);
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t total = al(nb_t) + al(nb_i) + al(nb_l);
    ST(dev_alloc(ctx, fr.buf, total));
    std::vector<char> host(total, 0);
    std::memcpy(host.data(), tlas.data(), nb_t);
    std::memcpy(host.data() + al(nb_t), inst.data(), nb_i);
    std::memcpy(host.data() + al(nb_t) + al(nb_i), lights.data(), nb_l);
    // the stream may still be reading the slot from an earlier frame
    CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaMemcpyAsync(fr.buf.ptr, host.data(), total, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->h2d += (int64_t)total;
    char* base = (char*)fr.buf.ptr;
    DevFrame& d = fr.dev;
    d.tlas = (const Node*)base;
    d.inst = (const float4*)(base + al(nb_t));
    d.lights = (const float4*)(base + al(nb_t) + al(nb_i));
    d.n_inst = nr;
    d.n_lights = (int32_t)ctx->emitters.size();
    d.n_tlas = n_tlas;
    d.static_rec = ctx->has_static ? n_tlas : -1;
    // camera (FP64 then rounded)
    double eye[3], tgt[3], up[3];
    for (int a = 0; a < 3; ++a) {
        eye[a] = lerp(ctx->cam_eye[3 * k + a], ctx->cam_eye[3 * k1 + a]);
        tgt[a] = lerp(ctx->cam_tgt[3 * k + a], ctx->cam_tgt[3 * k1 + a]);
        up[a] = lerp(ctx->cam_up[3 * k + a], ctx->cam_up[3 * k1 + a]);
    }
    double fwd[3] = {tgt[0] - eye[0], tgt[1] - eye[1], tgt[2] - eye[2]};
    const double fl = norm(fwd);
    for (double& x : fwd) x /= fl;
    double right[3], upv[3];
    cross(fwd, up, right);
    const double rl = norm(right);
    for (double& x : right) x /= rl;
    cross(right, fwd, upv);
    const double th = std::tan(0.5 * ctx->fov_deg * M_PI / 180.0);
    double sx, sy;
    if (ctx->W >= ctx->H) {
        sy = th;
        sx = th * (double)ctx->W / (double)ctx->H;
    } else {
        sx = th;
        sy = th * (double)ctx->H / (double)ctx->W;
    }
    for (int a = 0; a < 3; ++a) {
        d.eye[a] = (float)eye[a];
        d.fwd[a] = (float)fwd[a];
        d.right[a] = (float)(right[a] * sx);
        d.up[a] = (float)(upv[a] * sy);
    }
    d.key0 = (uint32_t)ctx->params.seed ^ frame_key(t);
    d.key1 = (uint32_t)(ctx->params.seed >> 32);
    const bool have_area = !ctx->emitters.empty();
    d.p_env = ctx->env_ok ? (have_area ? 0.5f : 1.0f) : 0.0f;
    d.p_area = have_area ? (ctx->env_ok ? 0.5f : 1.0f) : 0.0f;
    fr.time = t;
    fr.valid = true;
    // the other slot must not alias this time's state
    return MCEV_OK;
}

// ---------------------------------------------------------------- buffers
int64_t wave_cap(const mcev_ctx* ctx) {
    return ctx->params.wavefront > 0 ? ctx->params.wavefront : ((int64_t)1 << 25);
}

// Every chunk holds all the samples one call draws for a pixel in a round, so
// a per-pixel sample count above the wavefront capacity is refused.
mcev_status check_spp_fits(mcev_ctx* ctx, int64_t spp) {
    if (spp > wave_cap(ctx))
        return fail(ctx, MCEV_ERR_ARG, "%lld samples per pixel exceed the wavefront (%lld paths)", (long long)spp,
                    (long long)wave_cap(ctx));
    return MCEV_OK;
}

mcev_status ensure_wave(mcev_ctx* ctx) {
    const int64_t cap = wave_cap(ctx);
    if (ctx->d_wave.ptr && ctx->wave.cap == cap) return MCEV_OK;
    // path slots: L, sig, pflags, pix_k, Ltot, delta; per ray-queue slot (x2):
    // ray_o, ray_d, ray_s; hit; shadow: sh_o, sh_d, sh_c, sh_g, sh_m
    const size_t per = 4 + 4 + 4 + 8 + 4 + 4 + 2 * (16 + 16 + 16) + 16 + 16 + 16 + 4 + 4 + 4;
    ST(dev_alloc(ctx, ctx->d_wave, (size_t)cap * per + 64 * 256));
    char* p = (char*)ctx->d_wave.ptr;
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~size_t(255);
        return r;
    };
    Wave& w = ctx->wave;
    w.cap = cap;
    w.ray_o[0] = (float4*)take(16 * cap);
    w.ray_o[1] = (float4*)take(16 * cap);
    w.ray_d[0] = (float4*)take(16 * cap);
    w.ray_d[1] = (float4*)take(16 * cap);
    w.ray_s[0] = (float4*)take(16 * cap);
    w.ray_s[1] = (float4*)take(16 * cap);
    w.hit = (float4*)take(16 * cap);
    w.sh_o = (float4*)take(16 * cap);
    w.sh_d = (float4*)take(16 * cap);
    w.pix_k = (int2*)take(8 * cap);
    w.L = (float*)take(4 * cap);
    w.sig = (uint32_t*)take(4 * cap);
    w.pflags = (uint32_t*)take(4 * cap);
    w.sh_c = (float*)take(4 * cap);
    w.sh_g = (float*)take(4 * cap);
    w.sh_m = (int32_t*)take(4 * cap);
    w.Ltot = (float*)take(4 * cap);
    w.delta = (float*)take(4 * cap);
    if (!ctx->d_counters.ptr) {
        ST(dev_alloc(ctx, ctx->d_counters, 64 * sizeof(int32_t)));
        CU(cudaMemsetAsync(ctx->d_counters.ptr, 0, 64 * sizeof(int32_t), ctx->stream));
    }
    w.counters = (int32_t*)ctx->d_counters.ptr;
    return MCEV_OK;
}

mcev_status ensure_pixels(mcev_ctx* ctx) {
    if (ctx->d_pix.ptr) return MCEV_OK;
    const size_t n = (size_t)ctx->W * ctx->H;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    ST(dev_alloc(ctx, ctx->d_pix, 8 * al(4 * n)));
    char* p = (char*)ctx->d_pix.ptr;
    ctx->queue[0] = (int32_t*)p;
    ctx->queue[1] = (int32_t*)(p + al(4 * n));
    ctx->cur.n = (int32_t*)(p + 2 * al(4 * n));
    ctx->cur.mean = (float*)(p + 3 * al(4 * n));
    ctx->cur.m2 = (float*)(p + 4 * al(4 * n));
    ctx->ref.n = (int32_t*)(p + 5 * al(4 * n));
    ctx->ref.mean = (float*)(p + 6 * al(4 * n));
    ctx->ref.m2 = (float*)(p + 7 * al(4 * n));
    CU(cudaMemsetAsync(ctx->d_pix.ptr, 0, 8 * al(4 * n), ctx->stream));
    return MCEV_OK;
}

mcev_status ensure_tcrit(mcev_ctx* ctx, float alpha, int variant, int spp_min, int spp_batch, int spp_max) {
    auto key = std::make_tuple(alpha, variant, spp_min, spp_batch, spp_max);
    if (ctx->d_tcrit.ptr && key == ctx->tcrit_key) return MCEV_OK;
    std::vector<float> tab;
    for (int n = spp_min; n < spp_max; n += spp_batch) {
        const double p = variant == MCEV_TWO_TAILED ? 0.5 * (double)alpha : (double)alpha;
        tab.push_back((float)t_quantile_int(p, n - 1));
    }
    if (tab.empty()) tab.push_back(0.0f);
    ST(upload(ctx, ctx->d_tcrit, tab.data(), tab.size() * sizeof(float)));
    ctx->tcrit_key = key;
    return MCEV_OK;
}

DevParams dev_params(const mcev_ctx* ctx, bool want_sig) {
    DevParams P{};
    P.width = ctx->W;
    P.height = ctx->H;
    P.max_depth = ctx->params.max_depth;
    P.nee = ctx->params.nee;
    P.mis = ctx->params.mis;
    P.eps = ctx->params.eps;
    P.t_min = ctx->params.t_min;
    P.want_sig = want_sig ? 1 : 0;
    return P;
}

#define LAUNCH(cls, expr)                                                                             \
    do {                                                                                              \
        ST(ev_mark(ctx, cls, true));                                                                  \
        cudaError_t e_ = (expr);                                                                      \
        ++ctx->launches;                                                                              \
        ++ctx->kcount[cls];                                                                           \
        if (e_ != cudaSuccess)                                                                        \
            return fail(ctx, MCEV_ERR_CUDA, "launch %s failed: %s", #expr, cudaGetErrorString(e_));   \
        ST(ev_mark(ctx, cls, false));                                                                 \
    } while (0)

// 1: a bounce's shadow rays share one launch with the next bounce's closest hits
#ifndef MCEV_FUSE_SHADOW
#define MCEV_FUSE_SHADOW 1
#endif

// one chunk of n_paths = nj * spp_r paths through every bounce
// Batched render (several contexts' frame pairs in one set of rounds): the
// device job table, the union queues of (job << 24 | pixel) entries, and the
// largest depth / any NEE over the jobs (the per-path kernels use each job's
// own settings).
struct BatchRun {
    const Job* d_jobs = nullptr;
    int32_t* queue[2] = {nullptr, nullptr};
    int64_t q0 = 0;
    int32_t max_depth = 0;
    bool any_nee = false;
    bool wide = false;        // every job's BLAS use the wide layout
    bool any_tlas = false;    // some job's frame has two or more moving instances
};

// one chunk of n_paths = nj * spp_r paths through every bounce (with rc:
// the current chunk of the device-resident round loop, n_paths then being
// the wavefront capacity that sizes the launches)
mcev_status trace_chunk(mcev_ctx* ctx, const Frame& fr, const DevParams& P, const int32_t* queue, int64_t j0,
                        int32_t spp_r, int64_t k_base, int64_t n_paths, const BatchRun* B = nullptr,
                        const RoundCtl* rc = nullptr) {
    const Wave& w = ctx->wave;
    int32_t* err = ctx->wave.counters + 15;
    const Job* jobs = B ? B->d_jobs : nullptr;
    const int depth_max = B ? B->max_depth : P.max_depth;
    const bool nee = B ? B->any_nee : P.nee != 0;
    const bool wide = B ? B->wide : ctx->dsc.wide != 0;
    const bool tlas = B ? B->any_tlas : fr.dev.n_tlas >= 2;
    const int trav = (wide ? TRAV_WIDE : 0) | (tlas ? TRAV_TLAS : 0);
    NvtxRange range("mcev chunk");
    LAUNCH(MCEV_K_RAYGEN,
           launch_raygen(fr.dev, P, w, queue, j0, spp_r, k_base, n_paths, 0, ctx->sms, ctx->stream, jobs, rc));
    int cur = 0;
    LAUNCH(MCEV_K_EXTEND,
           launch_extend(ctx->dsc, fr.dev, P.t_min, w, cur, n_paths, err, ctx->sms, ctx->stream, jobs, trav));
    for (int depth = 0; depth <= depth_max; ++depth) {
        LAUNCH(MCEV_K_SHADE, launch_shade(ctx->dsc, fr.dev, P, w, cur, n_paths, ctx->sms, ctx->stream, jobs));
        if (depth < depth_max) {
#if MCEV_FUSE_SHADOW
            // this bounce's shadow rays and the next bounce's closest hits in one launch
            if (nee)
                LAUNCH(MCEV_K_EXTEND, launch_shadow_extend(ctx->dsc, fr.dev, P, w, cur, n_paths, err, ctx->sms,
                                                           ctx->stream, jobs, trav));
            else
                LAUNCH(MCEV_K_EXTEND, launch_extend(ctx->dsc, fr.dev, P.t_min, w, cur ^ 1, n_paths, err, ctx->sms,
                                                    ctx->stream, jobs, trav));
#else
            if (nee)
                LAUNCH(MCEV_K_SHADOW, launch_shadow(ctx->dsc, fr.dev, P, w, cur, n_paths, err, ctx->sms, ctx->stream,
                                                    jobs, trav));
            LAUNCH(MCEV_K_EXTEND, launch_extend(ctx->dsc, fr.dev, P.t_min, w, cur ^ 1, n_paths, err, ctx->sms,
                                                ctx->stream, jobs, trav));
#endif
        }
        cur ^= 1;
    }
    return MCEV_OK;
}

// Default wall-clock bound of the device-resident round loop.
constexpr int64_t kDefaultDeviceTimeoutUs = 300ll * 1000 * 1000;

// The rounds of run_rounds as one CUDA graph on the device (see kernels.cu,
// k_round_next): no host round trip until the frame is done.  The graph is
// captured on the context's capture stream and launched on its stream.
mcev_status run_rounds_device(mcev_ctx* ctx, const Frame& fr, StatsArgs A, int64_t* paths_out, int32_t* rounds_out,
                              const BatchRun* B) {
    NvtxRange range("mcev device round loop");
    const DevParams P = dev_params(ctx, false);
    int32_t* queue[2] = {ctx->queue[0], ctx->queue[1]};
    int64_t Q0 = (int64_t)ctx->W * ctx->H;
    if (B) {
        queue[0] = B->queue[0];
        queue[1] = B->queue[1];
        Q0 = B->q0;
    }
    const Job* jobs = B ? B->d_jobs : nullptr;
    ST(dev_alloc(ctx, ctx->d_round, sizeof(RoundCtl)));
    RoundCtl* rc = (RoundCtl*)ctx->d_round.ptr;
    if (!ctx->cap_stream) CU(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    RoundPlan plan{};
    plan.cap = ctx->wave.cap;
    plan.Q0 = Q0;
    plan.spp_min = A.spp_min;
    plan.spp_batch = A.spp_batch;
    plan.spp_max = A.spp_max;
    plan.window_max = ctx->params.batch_window > 0 ? ctx->params.batch_window : 16;
    const int64_t tus = ctx->params.device_timeout_us > 0 ? ctx->params.device_timeout_us : kDefaultDeviceTimeoutUs;
    plan.timeout_ns = (unsigned long long)tus * 1000ull;
    // chunks the schedule can need: rounds x chunks of the largest round
    const int64_t first = std::min(A.spp_min, A.spp_max);
    const int64_t rounds_max = 2 + (A.spp_max - first + A.spp_batch - 1) / std::max(1, A.spp_batch);
    const int64_t spp_r_max = std::max<int64_t>(first, std::min<int64_t>((int64_t)plan.window_max * A.spp_batch,
                                                                         A.spp_max));
    const int64_t chunks_max = (Q0 + std::max<int64_t>(1, plan.cap / spp_r_max) - 1) /
                               std::max<int64_t>(1, plan.cap / spp_r_max);
    plan.max_iters = (int32_t)std::min<int64_t>(rounds_max * (chunks_max + 1) + 4, 0x7fffffff);
    // one graph: init, then WHILE(chunk; round control)
    cudaGraph_t graph = nullptr, body = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = ctx->cap_stream;
    cudaStream_t saved = ctx->stream;
    const int32_t kc0[MCEV_K_CLASSES] = {ctx->kcount[0], ctx->kcount[1], ctx->kcount[2], ctx->kcount[3],
                                          ctx->kcount[4]};
    const int launches0 = ctx->launches;
    int body_launches = 0;
    int32_t body_kc[MCEV_K_CLASSES] = {0, 0, 0, 0, 0};
    auto build = [&]() -> mcev_status {
        CU(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle h;
        CU(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
        CU(cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        ctx->stream = cs;
        mcev_status st = MCEV_OK;
        cudaError_t e = launch_round_init(rc, ctx->wave, plan, queue[0], queue[1], B == nullptr, ctx->sms, cs);
        cudaGraphNode_t cond = nullptr;
        if (e == cudaSuccess) {
            cudaStreamCaptureStatus cst;
            cudaGraph_t g_out = nullptr;
            const cudaGraphNode_t* deps = nullptr;
            size_t ndeps = 0;
            e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g_out, &deps, nullptr, &ndeps);
            if (e == cudaSuccess) {
                cudaGraphNodeParams cp{};
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = h;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                e = cudaGraphAddNode(&cond, g_out, deps, nullptr, ndeps, &cp);
                if (e == cudaSuccess) {
                    body = cp.conditional.phGraph_out[0];
                    e = cudaStreamUpdateCaptureDependencies(cs, &cond, nullptr, 1, cudaStreamSetCaptureDependencies);
                }
            }
        }
        cudaGraph_t g2 = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g2);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            ctx->stream = saved;
            cudaGetLastError();
            return fail(ctx, MCEV_ERR_CUDA, "capturing the round loop failed: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        // the body: one chunk of every bounce, its statistics, the round control
        CU(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        const int l0 = ctx->launches;
        const int32_t k0[MCEV_K_CLASSES] = {ctx->kcount[0], ctx->kcount[1], ctx->kcount[2], ctx->kcount[3],
                                             ctx->kcount[4]};
        st = trace_chunk(ctx, fr, P, queue[0], 0, 1, 0, plan.cap, B, rc);
        if (st == MCEV_OK) {
            const cudaError_t el = launch_stats(ctx->wave, A, queue[0], 0, plan.cap, queue[1], ctx->sms, cs, jobs, rc);
            if (el != cudaSuccess) st = fail(ctx, MCEV_ERR_CUDA, "launch stats failed: %s", cudaGetErrorString(el));
            ++ctx->launches;
            ++ctx->kcount[MCEV_K_STATS];
        }
        if (st == MCEV_OK) {
            const cudaError_t el = launch_round_next(rc, ctx->wave, plan, h, cs);
            if (el != cudaSuccess) st = fail(ctx, MCEV_ERR_CUDA, "launch round control failed: %s", cudaGetErrorString(el));
            ++ctx->launches;
            ++ctx->kcount[MCEV_K_STATS];
        }
        body_launches = ctx->launches - l0;
        for (int i = 0; i < MCEV_K_CLASSES; ++i) body_kc[i] = ctx->kcount[i] - k0[i];
        cudaGraph_t b2 = nullptr;
        const cudaError_t e3 = cudaStreamEndCapture(cs, &b2);
        ctx->stream = saved;
        if (st != MCEV_OK) return st;
        if (e3 != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, MCEV_ERR_CUDA, "capturing the round body failed: %s", cudaGetErrorString(e3));
        }
        CU(cudaGraphInstantiate(&exec, graph, 0));
        return MCEV_OK;
    };
    mcev_status st = build();
    if (st == MCEV_OK) {
        const cudaError_t e = cudaGraphLaunch(exec, ctx->stream);
        if (e != cudaSuccess) st = fail(ctx, MCEV_ERR_CUDA, "cudaGraphLaunch failed: %s", cudaGetErrorString(e));
    }
    RoundCtl h_rc{};
    if (st == MCEV_OK) {
        const cudaError_t e1 = cudaMemcpyAsync(&h_rc, rc, sizeof h_rc, cudaMemcpyDeviceToHost, ctx->stream);
        const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamSynchronize(ctx->stream) : e1;
        if (e2 != cudaSuccess) st = fail(ctx, MCEV_ERR_CUDA, "round loop failed: %s", cudaGetErrorString(e2));
        ctx->d2h += (int64_t)sizeof h_rc;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    // launches that ran: the init kernel plus the body once per chunk
    ctx->launches = launches0 + 1 + body_launches * h_rc.iters;
    for (int i = 0; i < MCEV_K_CLASSES; ++i) ctx->kcount[i] = kc0[i] + body_kc[i] * h_rc.iters;
    ctx->kcount[MCEV_K_STATS] += 1;
    if (st != MCEV_OK) return st;
    ctx->stats_pix += h_rc.stats_pix;
    if (h_rc.status == RC_TIMEOUT)
        return fail(ctx, MCEV_ERR_TIMEOUT,
                    "the device-resident round loop stopped after %d chunks (bound: %d chunks, %lld us); the "
                    "frame is incomplete", h_rc.iters, plan.max_iters, (long long)tus);
    if (h_rc.status == RC_CAP)
        return fail(ctx, MCEV_ERR_STATE, "internal: %lld pixels undecided at the sample cap", (long long)h_rc.Q);
    if (paths_out) *paths_out = h_rc.paths;
    if (rounds_out) *rounds_out = h_rc.rounds;
    return MCEV_OK;
}

// Runs rounds of batches over the pixel queue until no pixel is undecided.
// mode REFERENCE: every pixel to spp_max samples, statistics -> ref.
// mode DETECT: Alg. 1 frame with the test variant in `A`.
// The rounds run on the device (one CUDA graph, run_rounds_device) unless
// per-launch timing is on or the caller asked for host-driven rounds.
mcev_status run_rounds(mcev_ctx* ctx, const Frame& fr, StatsArgs A, int64_t* paths_out, int32_t* rounds_out,
                       const BatchRun* B = nullptr) {
    if (!ctx->params.profile && !ctx->params.host_rounds) return run_rounds_device(ctx, fr, A, paths_out, rounds_out, B);
    NvtxRange range("mcev host rounds");
    const DevParams P = dev_params(ctx, false);
    int32_t* queue[2] = {ctx->queue[0], ctx->queue[1]};
    int64_t Q;
    if (B) {
        queue[0] = B->queue[0];
        queue[1] = B->queue[1];
        Q = B->q0;
    } else {
        Q = (int64_t)ctx->W * ctx->H;
        LAUNCH(MCEV_K_STATS, launch_iota(queue[0], Q, ctx->sms, ctx->stream));
    }
    const Job* jobs = B ? B->d_jobs : nullptr;
    int64_t n_done = 0, paths = 0;
    int rounds = 0, qi = 0;
    int32_t h_count = 0;
    const int64_t window_max = ctx->params.batch_window > 0 ? ctx->params.batch_window : 16;
    while (Q > 0) {
        // first round: spp_min samples; later rounds: a window of m batches
        // of spp_batch, as many as fill the wavefront (speculative samples of
        // pixels that decide inside the window are traced but not used)
        int32_t spp_r, sub;
        if (n_done == 0) {
            spp_r = sub = std::min(A.spp_min, A.spp_max);
        } else {
            sub = A.spp_batch;
            const int64_t left = (A.spp_max - n_done + sub - 1) / sub;
            int64_t m = std::max<int64_t>(1, ctx->wave.cap / std::max<int64_t>(1, Q * sub));
            m = std::min(std::min(m, left), window_max);
            spp_r = (int32_t)std::min<int64_t>(m * sub, A.spp_max - n_done);
        }
        NvtxRange round_range("mcev round");
        CU(cudaMemsetAsync(ctx->wave.counters + 3, 0, sizeof(int32_t), ctx->stream));
        A.spp_r = spp_r;
        A.sub = sub;
        A.k_base = n_done;
        const int64_t per_chunk = std::max<int64_t>(1, ctx->wave.cap / spp_r);
        for (int64_t j0 = 0; j0 < Q; j0 += per_chunk) {
            const int64_t nj = std::min(per_chunk, Q - j0);
            ST(trace_chunk(ctx, fr, P, queue[qi], j0, spp_r, n_done, nj * spp_r, B));
            LAUNCH(MCEV_K_STATS,
                   launch_stats(ctx->wave, A, queue[qi], j0, nj, queue[qi ^ 1], ctx->sms, ctx->stream, jobs, nullptr));
            ctx->stats_pix += nj;
        }
        paths += Q * spp_r;
        n_done += spp_r;
        ++rounds;
        CU(cudaMemcpyAsync(&h_count, ctx->wave.counters + 3, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        ctx->d2h += (int64_t)sizeof(int32_t);
        ST(drain_events(ctx));
        Q = h_count;
        qi ^= 1;
        if (n_done >= A.spp_max && Q != 0)
            return fail(ctx, MCEV_ERR_STATE, "internal: %lld pixels undecided at the sample cap", (long long)Q);
    }
    if (paths_out) *paths_out = paths;
    if (rounds_out) *rounds_out = rounds;
    return MCEV_OK;
}

void reset_call_counters(mcev_ctx* ctx) {
    ctx->launches = 0;
    for (int i = 0; i < MCEV_K_CLASSES; ++i) {
        ctx->kcount[i] = 0;
        ctx->kms[i] = 0.0;
    }
    ctx->h2d = ctx->d2h = 0;
    ctx->stats_pix = 0;
    ctx->evused = 0;
}

mcev_status fill_stats(mcev_ctx* ctx, mcev_stats* stats_out, int64_t paths, int64_t ref_paths, int32_t rounds) {
    int32_t c[64];
    CU(cudaMemcpyAsync(c, ctx->wave.counters, sizeof c, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->d2h += (int64_t)sizeof c;
    float ms = 0.0f;
    CU(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    uint64_t u[16];
    std::memcpy(u, c + 32, sizeof u);
    std::memset(stats_out, 0, sizeof *stats_out);
    stats_out->paths = paths;
    stats_out->samples_used = (int64_t)u[6];
    stats_out->ref_paths = ref_paths;
    stats_out->rounds = rounds;
    stats_out->kernel_launches = ctx->launches;
    stats_out->nonfinite = c[4];
    stats_out->events_pos = c[5];
    stats_out->events_neg = c[6];
    stats_out->pixels_at_cap = c[7];
    stats_out->gpu_ms = ms;
    stats_out->nodes_closest = (int64_t)u[0];
    stats_out->tris_closest = (int64_t)u[1];
    stats_out->nodes_shadow = (int64_t)u[2];
    stats_out->tris_shadow = (int64_t)u[3];
    stats_out->rays_closest = (int64_t)u[4];
    stats_out->rays_shadow = (int64_t)u[5];
    for (int i = 0; i < MCEV_K_CLASSES; ++i) {
        stats_out->kernel_count[i] = ctx->kcount[i];
        stats_out->kernel_ms[i] = ctx->kms[i];
    }
    stats_out->h2d_bytes = ctx->h2d;
    stats_out->stats_pixels = ctx->stats_pix;
    stats_out->d2h_bytes = ctx->d2h;
    stats_out->boxes_closest = (int64_t)u[7];
    stats_out->boxes_shadow = (int64_t)u[8];
    if (c[15]) return fail(ctx, MCEV_ERR_STATE, "traversal stack overflow");
    return MCEV_OK;
}

mcev_status check_ready(mcev_ctx* ctx) {
    if (!ctx) return MCEV_ERR_ARG;
    if (!ctx->have_scene) return fail(ctx, MCEV_ERR_STATE, "no scene uploaded");
    CU(cudaSetDevice(ctx->device));
    ST(ensure_wave(ctx));
    ST(ensure_pixels(ctx));
    return MCEV_OK;
}

mcev_status do_reference(mcev_ctx* ctx, double t0, int32_t spp, int64_t* paths) {
    NvtxRange range("mcev reference frame");
    ctx->ref_valid = false;   // overwritten from here on; valid again only when complete
    ST(frame_setup(ctx, t0, 0));
    StatsArgs A{};
    A.cur = ctx->cur;
    A.ref = ctx->ref;
    A.eps = ctx->params.eps;
    A.spp_min = spp;
    A.spp_batch = spp;
    A.spp_max = spp;
    A.mode = MODE_REFERENCE;
    A.tcrit = nullptr;
    ST(run_rounds(ctx, ctx->frames[0], A, paths, nullptr));
    ctx->ref_valid = true;
    ctx->ref_time = t0;
    return MCEV_OK;
}

}  // namespace

// =====================================================================================
extern "C" {

mcev_status mcev_create(mcev_ctx** out, int device, int32_t width, int32_t height) {
    if (!out) return MCEV_ERR_ARG;
    *out = nullptr;
    if (width <= 0 || height <= 0 || (int64_t)width * height > (int64_t)1 << 30) return MCEV_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return MCEV_ERR_CUDA;
    }
    mcev_ctx* ctx = new (std::nothrow) mcev_ctx();
    if (!ctx) return MCEV_ERR_OOM;
    ctx->device = device;
    ctx->W = width;
    ctx->H = height;
    if (cudaSetDevice(device) != cudaSuccess || cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return MCEV_ERR_CUDA;
    }
    mcev_params p{};
    p.eps = 1e-3f;
    p.t_min = 1e-4f;
    p.max_depth = 4;
    p.nee = 1;
    p.mis = 1;
    p.spp_min = 16;
    p.variant = MCEV_ONE_TAILED;
    p.se_mode = MCEV_SE_PAPER;
    p.seed = 20240815ull;
    p.wavefront = 0;
    ctx->params = p;
    *out = ctx;
    return MCEV_OK;
}

void mcev_destroy(mcev_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    DevBuf* bufs[] = {&ctx->d_nodes, &ctx->d_wnodes, &ctx->d_tris, &ctx->d_tshade, &ctx->d_uv, &ctx->d_mats, &ctx->d_env, &ctx->d_marg, &ctx->d_cond,
                      &ctx->d_tpdf, &ctx->frames[0].buf, &ctx->frames[1].buf, &ctx->d_wave, &ctx->d_counters,
                      &ctx->d_pix, &ctx->d_tcrit, &ctx->d_jobs, &ctx->d_bqueue, &ctx->d_quality, &ctx->d_gemit,
                      &ctx->d_round};
    for (DevBuf* b : bufs) dev_free(ctx, *b);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (cudaEvent_t e : ctx->evpool) cudaEventDestroy(e);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
}

const char* mcev_last_error(const mcev_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

mcev_status mcev_set_stream(mcev_ctx* ctx, void* stream) {
    if (!ctx) return MCEV_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return MCEV_OK;
}

mcev_status mcev_set_allocator(mcev_ctx* ctx, mcev_alloc_fn alloc, mcev_free_fn free_fn, void* user) {
    if (!ctx) return MCEV_ERR_ARG;
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(ctx, MCEV_ERR_ARG, "alloc and free must both be set");
    if (ctx->have_scene || ctx->d_wave.ptr || ctx->d_pix.ptr)
        return fail(ctx, MCEV_ERR_STATE, "set the allocator before uploading a scene");
    ctx->alloc = alloc;
    ctx->free_fn = free_fn;
    ctx->alloc_user = user;
    return MCEV_OK;
}

mcev_status mcev_scene_upload(mcev_ctx* ctx, const mcev_scene_desc* s) {
    NvtxRange range("mcev_scene_upload");
    if (!ctx) return MCEV_ERR_ARG;
    if (!s) return fail(ctx, MCEV_ERR_ARG, "null scene description");
    if (s->n_triangles < 0 || s->n_vertices < 0 || s->n_meshes < 0 || s->n_instances < 0 || s->n_keys < 1 ||
        s->n_materials < 1)
        return fail(ctx, MCEV_ERR_ARG, "negative count, no keyframe or no material");
    if (s->n_triangles > ((int64_t)1 << 30)) return fail(ctx, MCEV_ERR_ARG, "too many triangles");
    if ((s->n_triangles > 0 && (!s->vertices || !s->triangles || !s->tri_material)) ||
        (s->n_meshes > 0 && !s->mesh_ranges) || (s->n_instances > 0 && (!s->inst_mesh || !s->inst_material)) ||
        !s->key_times || (s->n_instances > 0 && !s->inst_xform) || !s->cam_eye || !s->cam_target || !s->cam_up ||
        !s->mat_type || !s->mat_albedo || !s->mat_rough || !s->mat_emit)
        return fail(ctx, MCEV_ERR_ARG, "null array in scene description");
    if (!(s->fov_deg > 0.0 && s->fov_deg < 180.0)) return fail(ctx, MCEV_ERR_ARG, "fov_deg out of (0, 180)");
    for (int k = 1; k < s->n_keys; ++k)
        if (!(s->key_times[k] > s->key_times[k - 1])) return fail(ctx, MCEV_ERR_ARG, "key times not increasing");
    for (int64_t t = 0; t < 3 * s->n_triangles; ++t)
        if (s->triangles[t] < 0 || s->triangles[t] >= s->n_vertices)
            return fail(ctx, MCEV_ERR_ARG, "triangle vertex index out of range");
    for (int64_t t = 0; t < s->n_triangles; ++t)
        if (s->tri_material[t] < 0 || s->tri_material[t] >= s->n_materials)
            return fail(ctx, MCEV_ERR_ARG, "triangle material out of range");
    for (int m = 0; m < s->n_meshes; ++m) {
        const int64_t f = s->mesh_ranges[2 * m], c = s->mesh_ranges[2 * m + 1];
        if (f < 0 || c < 0 || f + c > s->n_triangles) return fail(ctx, MCEV_ERR_ARG, "mesh range out of bounds");
    }
    for (int i = 0; i < s->n_instances; ++i) {
        if (s->inst_mesh[i] < 0 || s->inst_mesh[i] >= s->n_meshes)
            return fail(ctx, MCEV_ERR_ARG, "instance mesh out of range");
        if (s->inst_material[i] < -1 || s->inst_material[i] >= s->n_materials)
            return fail(ctx, MCEV_ERR_ARG, "instance material out of range");
    }
    for (int m = 0; m < s->n_materials; ++m) {
        if (s->mat_type[m] != MAT_DIFFUSE && s->mat_type[m] != MAT_GGX)
            return fail(ctx, MCEV_ERR_ARG, "unknown material type %d", s->mat_type[m]);
        if (s->mat_type[m] == MAT_GGX && !(s->mat_rough[m] > 0.0f))
            return fail(ctx, MCEV_ERR_ARG, "GGX material needs rough > 0");
        if (!(s->mat_albedo[m] >= 0.0f && s->mat_albedo[m] <= 1.0f) || !(s->mat_emit[m] >= 0.0f))
            return fail(ctx, MCEV_ERR_ARG, "albedo outside [0,1] or negative emission");
    }
    if (s->env && (s->env_w <= 0 || s->env_h <= 0)) return fail(ctx, MCEV_ERR_ARG, "bad environment size");
    if (s->mat_textured)
        for (int m = 0; m < s->n_materials; ++m)
            if (s->mat_textured[m] && s->mat_type[m] != MAT_DIFFUSE)
                return fail(ctx, MCEV_ERR_ARG, "only Lambertian materials can be textured");
    if (s->env)
        for (int64_t i = 0; i < (int64_t)s->env_w * s->env_h; ++i)
            if (!(s->env[i] >= 0.0f) || !std::isfinite(s->env[i]))
                return fail(ctx, MCEV_ERR_ARG, "environment texel negative or not finite");
    CU(cudaSetDevice(ctx->device));
    ctx->have_scene = false;
    ctx->ref_valid = false;
    ctx->vtx.resize(9 * (size_t)s->n_triangles);
    ctx->tri_mat.assign(s->tri_material, s->tri_material + s->n_triangles);
    ctx->tri_uv.clear();
    if (s->uvs) {
        ctx->tri_uv.resize(6 * (size_t)s->n_triangles);
        for (int64_t t = 0; t < s->n_triangles; ++t)
            for (int c = 0; c < 3; ++c)
                for (int a2 = 0; a2 < 2; ++a2)
                    ctx->tri_uv[6 * t + 2 * c + a2] = s->uvs[2 * (int64_t)s->triangles[3 * t + c] + a2];
    }
    for (int64_t t = 0; t < s->n_triangles; ++t)
        for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 3; ++a) ctx->vtx[9 * t + 3 * c + a] = s->vertices[3 * (int64_t)s->triangles[3 * t + c] + a];
    ctx->meshes.clear();
    for (int m = 0; m < s->n_meshes; ++m) {
        MeshInfo mi{};
        mi.first_tri = s->mesh_ranges[2 * m];
        mi.n_tri = s->mesh_ranges[2 * m + 1];
        ctx->meshes.push_back(mi);
    }
    ctx->n_inst = s->n_instances;
    ctx->inst_mesh.assign(s->inst_mesh, s->inst_mesh + s->n_instances);
    ctx->inst_mat.assign(s->inst_material, s->inst_material + s->n_instances);
    ctx->n_keys = s->n_keys;
    ctx->key_t.assign(s->key_times, s->key_times + s->n_keys);
    ctx->key_xf.assign(s->inst_xform, s->inst_xform + 12 * (size_t)s->n_keys * s->n_instances);
    ctx->cam_eye.assign(s->cam_eye, s->cam_eye + 3 * s->n_keys);
    ctx->cam_tgt.assign(s->cam_target, s->cam_target + 3 * s->n_keys);
    ctx->cam_up.assign(s->cam_up, s->cam_up + 3 * s->n_keys);
    ctx->fov_deg = s->fov_deg;
    ctx->n_mats = s->n_materials;
    ctx->mat_type.assign(s->mat_type, s->mat_type + s->n_materials);
    ctx->mat_alb.assign(s->mat_albedo, s->mat_albedo + s->n_materials);
    ctx->mat_rough.assign(s->mat_rough, s->mat_rough + s->n_materials);
    ctx->mat_emit.assign(s->mat_emit, s->mat_emit + s->n_materials);
    ctx->emitters.clear();
    for (int i = 0; i < s->n_instances; ++i) {
        const MeshInfo& m = ctx->meshes[ctx->inst_mesh[i]];
        for (int64_t t = 0; t < m.n_tri; ++t) {
            const int64_t prim = m.first_tri + t;
            const int mat = ctx->inst_mat[i] >= 0 ? ctx->inst_mat[i] : ctx->tri_mat[prim];
            if (ctx->mat_emit[mat] > 0.0f) ctx->emitters.emplace_back(i, prim);
        }
    }
    std::vector<float4> mats(s->n_materials);
    for (int m = 0; m < s->n_materials; ++m) {
        int ty = s->mat_type[m] | ((s->mat_textured && s->mat_textured[m]) ? MAT_TEXTURED : 0);
        float tf;
        std::memcpy(&tf, &ty, 4);
        mats[m] = make_float4(tf, s->mat_albedo[m], s->mat_rough[m], s->mat_emit[m]);
    }
    ST(upload(ctx, ctx->d_mats, mats.data(), mats.size() * sizeof(float4)));
    ctx->dsc.mats = (const float4*)ctx->d_mats.ptr;
    ctx->env_w = s->env ? s->env_w : 0;
    ctx->env_h = s->env ? s->env_h : 0;
    ctx->env.assign(s->env ? s->env : nullptr, s->env ? s->env + (size_t)s->env_w * s->env_h : nullptr);
    if (s->env) {
        ST(build_env(ctx));
    } else {
        ctx->env_ok = false;
        ctx->dsc.has_env = 0;
        ctx->dsc.env_ok = 0;
        ctx->dsc.env_w = ctx->dsc.env_h = 0;
    }
    ST(build_blas(ctx));
    ctx->have_scene = true;
    return MCEV_OK;
}

mcev_status mcev_build_bvh(mcev_ctx* ctx, int32_t sah_bins, int32_t max_leaf) {
    if (!ctx) return MCEV_ERR_ARG;
    if (sah_bins < 4 || sah_bins > 256 || max_leaf < 1 || max_leaf > 16)
        return fail(ctx, MCEV_ERR_ARG, "sah_bins in [4,256] and max_leaf in [1,16]");
    if (!ctx->have_scene) return fail(ctx, MCEV_ERR_STATE, "no scene uploaded");
    CU(cudaSetDevice(ctx->device));
    ctx->sah_bins = sah_bins;
    ctx->max_leaf = max_leaf;
    return build_blas(ctx);
}

mcev_status mcev_set_params(mcev_ctx* ctx, const mcev_params* p) {
    if (!ctx) return MCEV_ERR_ARG;
    if (!p) return fail(ctx, MCEV_ERR_ARG, "null params");
    if (!(p->eps > 0.0f) || !(p->t_min >= 0.0f) || p->max_depth < 0 || p->max_depth > 64 || p->spp_min < 2 ||
        p->variant < 0 || p->variant > 3 || p->se_mode < 0 || p->se_mode > 1 || p->wavefront < 0 ||
        p->batch_window < 0 || p->batch_window > 1024 ||
        (p->wavefront > 0 && p->wavefront < 1024) || p->wavefront > ((int64_t)1 << 30) ||
        (p->bvh_width != 0 && p->bvh_width != 2 && p->bvh_width != 8) || p->host_rounds < 0 ||
        p->host_rounds > 1 || p->device_timeout_us < 0)
        return fail(ctx, MCEV_ERR_ARG, "invalid render parameters");
    const bool reseed = p->seed != ctx->params.seed;
    const bool shape = p->eps != ctx->params.eps || p->t_min != ctx->params.t_min ||
                       p->max_depth != ctx->params.max_depth || p->nee != ctx->params.nee || p->mis != ctx->params.mis;
    const int width = p->bvh_width ? p->bvh_width : MCEV_DEFAULT_BVH_WIDTH;
    ctx->params = *p;
    if (reseed || shape) {
        ctx->ref_valid = false;
        for (auto& f : ctx->frames) f.valid = false;
    }
    if (width != ctx->bvh_width) {
        ctx->bvh_width = width;
        if (ctx->have_scene) {
            CU(cudaSetDevice(ctx->device));
            const mcev_status st = build_blas(ctx);
            if (st != MCEV_OK) {
                ctx->have_scene = false;   // half-built: the scene must be uploaded again
                return st;
            }
        }
    }
    return MCEV_OK;
}

mcev_status mcev_render_reference(mcev_ctx* ctx, double t0, int32_t spp) {
    ST(check_ready(ctx));
    if (spp < 2) return fail(ctx, MCEV_ERR_ARG, "spp must be >= 2");
    ST(check_spp_fits(ctx, spp));
    reset_call_counters(ctx);
    return do_reference(ctx, t0, spp, nullptr);
}

mcev_status mcev_render_events(mcev_ctx* ctx, double t0, double t1, float C, float alpha, int32_t spp_batch,
                               int32_t spp_max, int8_t* events_out, int32_t* spp_out, float* mean_out,
                               mcev_stats* stats_out) {
    NvtxRange range("mcev_render_events");
    ST(check_ready(ctx));
    if (!events_out) return fail(ctx, MCEV_ERR_ARG, "events_out is required");
    if (!(C >= 0.0f) || !(alpha > 0.0f && alpha < 1.0f) || spp_batch < 1 || spp_max < ctx->params.spp_min)
        return fail(ctx, MCEV_ERR_ARG, "need C >= 0, 0 < alpha < 1, spp_batch >= 1, spp_max >= spp_min");
    ST(check_spp_fits(ctx, spp_max));
    reset_call_counters(ctx);
    CU(cudaMemsetAsync(ctx->wave.counters + 4, 0, 60 * sizeof(int32_t), ctx->stream));
    CU(cudaEventRecord(ctx->ev0, ctx->stream));
    int64_t ref_paths = 0, paths = 0;
    int32_t rounds = 0;
    if (!ctx->ref_valid || ctx->ref_time != t0) ST(do_reference(ctx, t0, spp_max, &ref_paths));
    ST(frame_setup(ctx, t1, 1));
    ST(ensure_tcrit(ctx, alpha, ctx->params.variant, ctx->params.spp_min, spp_batch, spp_max));
    StatsArgs A{};
    A.cur = ctx->cur;
    A.ref = ctx->ref;
    A.tcrit = (const float*)ctx->d_tcrit.ptr;
    A.events = events_out;
    A.spp_out = spp_out;
    A.mean_out = mean_out;
    A.eps = ctx->params.eps;
    A.C = C;
    A.spp_min = ctx->params.spp_min;
    A.spp_batch = spp_batch;
    A.spp_max = spp_max;
    A.mode = MODE_DETECT;
    A.variant = ctx->params.variant;
    A.se_mode = ctx->params.se_mode;
    const mcev_status rs = run_rounds(ctx, ctx->frames[1], A, &paths, &rounds);
    if (rs != MCEV_OK) {
        ctx->ref_valid = false;   // some pixels may have updated their reference already
        return rs;
    }
    ctx->ref_valid = true;
    ctx->ref_time = t1;
    CU(cudaEventRecord(ctx->ev1, ctx->stream));
    ST(drain_events(ctx));
    if (stats_out) ST(fill_stats(ctx, stats_out, paths, ref_paths, rounds));
    return MCEV_OK;
}

mcev_status mcev_trace_samples(mcev_ctx* ctx, double t, const int32_t* pixels, int64_t n_pix, int64_t k0,
                               int32_t count, float* L_out, uint32_t* sig_out) {
    ST(check_ready(ctx));
    if (n_pix < 0 || k0 < 0 || count < 1 || k0 + count > ((int64_t)1 << 32))
        return fail(ctx, MCEV_ERR_ARG, "bad trace_samples sizes");
    if (n_pix == 0) return MCEV_OK;
    if (!pixels || !L_out) return fail(ctx, MCEV_ERR_ARG, "null pixels or L_out");
    ST(check_spp_fits(ctx, count));
    reset_call_counters(ctx);
    ST(frame_setup(ctx, t, 0));
    const DevParams P = dev_params(ctx, sig_out != nullptr);
    const int64_t per_chunk = std::max<int64_t>(1, ctx->wave.cap / count);
    for (int64_t j0 = 0; j0 < n_pix; j0 += per_chunk) {
        const int64_t nj = std::min(per_chunk, n_pix - j0);
        ST(trace_chunk(ctx, ctx->frames[0], P, pixels, j0, count, k0, nj * count, nullptr));
        LAUNCH(MCEV_K_STATS, launch_write_samples(ctx->wave, j0 * count, nj * count, L_out, sig_out, ctx->sms, ctx->stream));
    }
    return MCEV_OK;
}


mcev_status mcev_set_texture(mcev_ctx* ctx, const float* texture, int32_t width, int32_t height) {
    if (!ctx) return MCEV_ERR_ARG;
    if (texture && (width < 1 || height < 1)) return fail(ctx, MCEV_ERR_ARG, "bad texture size");
    ctx->dsc.tex = texture;
    ctx->dsc.tex_w = texture ? width : 0;
    ctx->dsc.tex_h = texture ? height : 0;
    return MCEV_OK;
}

mcev_status mcev_set_emission(mcev_ctx* ctx, const float* emission, int32_t n_materials) {
    if (!ctx) return MCEV_ERR_ARG;
    if (emission && n_materials != ctx->n_mats)
        return fail(ctx, MCEV_ERR_ARG, "emission has %d entries, the scene %d materials", n_materials, ctx->n_mats);
    ctx->dsc.emit = emission;
    return MCEV_OK;
}

mcev_status mcev_render_mean(mcev_ctx* ctx, double t, int32_t spp, float* mean_out) {
    NvtxRange range("mcev_render_mean");
    ST(check_ready(ctx));
    if (spp < 1 || !mean_out) return fail(ctx, MCEV_ERR_ARG, "need spp >= 1 and mean_out");
    ST(check_spp_fits(ctx, spp));
    reset_call_counters(ctx);
    ST(frame_setup(ctx, t, 0));
    StatsArgs A{};
    A.cur = ctx->cur;
    A.ref = ctx->ref;
    A.mean_out = mean_out;
    A.eps = ctx->params.eps;
    A.spp_min = A.spp_batch = A.spp_max = spp;
    A.mode = MODE_MEAN;
    return run_rounds(ctx, ctx->frames[0], A, nullptr, nullptr);
}

mcev_status mcev_backward(mcev_ctx* ctx, double t, int32_t spp, const float* grad_mean, float* grad_texture,
                          float* grad_emission) {
    NvtxRange range("mcev_backward");
    ST(check_ready(ctx));
    if (spp < 1 || !grad_mean) return fail(ctx, MCEV_ERR_ARG, "need spp >= 1 and grad_mean");
    ST(check_spp_fits(ctx, spp));
    if (grad_texture && !ctx->dsc.tex) return fail(ctx, MCEV_ERR_STATE, "no texture set");
    reset_call_counters(ctx);
    ST(frame_setup(ctx, t, 0));
    const int64_t npix = (int64_t)ctx->W * ctx->H;
    LAUNCH(MCEV_K_STATS, launch_iota(ctx->queue[0], npix, ctx->sms, ctx->stream));
    const DevParams P = dev_params(ctx, false);
    DevParams Padj = P;
    Padj.adjoint = 1;
    Padj.spp = spp;
    Padj.grad_mean = grad_mean;
    Padj.grad_tex = grad_texture;
    if (grad_emission) {
        ST(dev_alloc(ctx, ctx->d_gemit, sizeof(double) * std::max(1, ctx->n_mats)));
        CU(cudaMemsetAsync(ctx->d_gemit.ptr, 0, sizeof(double) * std::max(1, ctx->n_mats), ctx->stream));
        Padj.grad_emit = (double*)ctx->d_gemit.ptr;
    }
    const int64_t per_chunk = std::max<int64_t>(1, ctx->wave.cap / spp);
    for (int64_t j0 = 0; j0 < npix; j0 += per_chunk) {
        const int64_t nj = std::min(per_chunk, npix - j0);
        // pass 1: every path's radiance; pass 2: replay with the adjoint
        ST(trace_chunk(ctx, ctx->frames[0], P, ctx->queue[0], j0, spp, 0, nj * spp, nullptr));
        CU(cudaMemcpyAsync(ctx->wave.Ltot, ctx->wave.L, sizeof(float) * nj * spp, cudaMemcpyDeviceToDevice,
                           ctx->stream));
        ST(trace_chunk(ctx, ctx->frames[0], Padj, ctx->queue[0], j0, spp, 0, nj * spp, nullptr));
    }
    if (grad_emission && ctx->n_mats > 0)
        LAUNCH(MCEV_K_STATS, launch_add_f64(grad_emission, (const double*)ctx->d_gemit.ptr, ctx->n_mats, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ST(drain_events(ctx));
    return MCEV_OK;
}

mcev_status mcev_render_events_batch(mcev_ctx* runner, const mcev_job* jobs, int32_t n_jobs, float C, float alpha,
                                     int32_t spp_batch, int32_t spp_max, mcev_stats* stats_out) {
    NvtxRange range("mcev_render_events_batch");
    mcev_ctx* ctx = runner;
    if (!ctx) return MCEV_ERR_ARG;
    if (!jobs || n_jobs < 1 || n_jobs > 256) return fail(ctx, MCEV_ERR_ARG, "need 1..256 jobs");
    if (!(C >= 0.0f) || !(alpha > 0.0f && alpha < 1.0f) || spp_batch < 1)
        return fail(ctx, MCEV_ERR_ARG, "need C >= 0, 0 < alpha < 1, spp_batch >= 1");
    const mcev_ctx* j0c = jobs[0].ctx;
    if (!j0c) return fail(ctx, MCEV_ERR_ARG, "job 0 has no context");
    const int32_t spp_min = j0c->params.spp_min, variant = j0c->params.variant, se_mode = j0c->params.se_mode;
    if (spp_max < spp_min) return fail(ctx, MCEV_ERR_ARG, "spp_max < spp_min");
    ST(check_spp_fits(ctx, spp_max));
    for (int i = 0; i < n_jobs; ++i) {
        const mcev_ctx* c = jobs[i].ctx;
        if (!c || !c->have_scene) return fail(ctx, MCEV_ERR_STATE, "job %d: no context or no scene", i);
        if (c->device != ctx->device) return fail(ctx, MCEV_ERR_ARG, "job %d: context on another device", i);
        if ((int64_t)c->W * c->H > (1 << 24)) return fail(ctx, MCEV_ERR_ARG, "job %d: more than 2^24 pixels", i);
        if (!jobs[i].events_out) return fail(ctx, MCEV_ERR_ARG, "job %d: events_out is required", i);
        if (c->params.spp_min != spp_min || c->params.variant != variant || c->params.se_mode != se_mode)
            return fail(ctx, MCEV_ERR_ARG, "job %d: spp_min, variant and se_mode must match across jobs", i);
        if (c->bvh_width != j0c->bvh_width)
            return fail(ctx, MCEV_ERR_ARG, "job %d: every job's BVH must use the same node layout", i);
        for (int k = 0; k < i; ++k)
            if (jobs[k].ctx == c) return fail(ctx, MCEV_ERR_ARG, "jobs %d and %d share a context", k, i);
    }
    CU(cudaSetDevice(ctx->device));
    ST(ensure_wave(ctx));
    reset_call_counters(ctx);
    CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaMemsetAsync(ctx->wave.counters + 4, 0, 60 * sizeof(int32_t), ctx->stream));
    CU(cudaEventRecord(ctx->ev0, ctx->stream));
    for (int i = 0; i < n_jobs; ++i) {
        mcev_ctx* c = jobs[i].ctx;
        ST(ensure_pixels(c));
        CU(cudaStreamSynchronize(c->stream));
    }
    int64_t total = 0;
    for (int i = 0; i < n_jobs; ++i) total += (int64_t)jobs[i].ctx->W * jobs[i].ctx->H;
    ST(dev_alloc(ctx, ctx->d_bqueue, 2 * sizeof(int32_t) * (size_t)total));
    ST(dev_alloc(ctx, ctx->d_jobs, sizeof(Job) * (size_t)n_jobs));
    BatchRun B;
    B.wide = j0c->bvh_width == 8;
    B.d_jobs = (const Job*)ctx->d_jobs.ptr;
    B.queue[0] = (int32_t*)ctx->d_bqueue.ptr;
    B.queue[1] = B.queue[0] + total;
    // builds the job table of the listed jobs for frame slot `slot` and fills the queue
    auto prepare = [&](const std::vector<int>& list, int slot) -> mcev_status {
        std::vector<Job> tab(list.size());
        B.q0 = 0;
        B.max_depth = 0;
        B.any_nee = false;
        B.any_tlas = false;
        for (size_t q = 0; q < list.size(); ++q) {
            mcev_ctx* c = jobs[list[q]].ctx;
            Job& J = tab[q];
            std::memset(&J, 0, sizeof J);
            J.sc = c->dsc;
            J.fr = c->frames[slot].dev;
            J.P = dev_params(c, false);
            J.cur = c->cur;
            J.ref = c->ref;
            J.events = jobs[list[q]].events_out;
            J.spp_out = jobs[list[q]].spp_out;
            J.mean_out = jobs[list[q]].mean_out;
            B.max_depth = std::max(B.max_depth, c->params.max_depth);
            B.any_nee = B.any_nee || c->params.nee != 0;
            B.any_tlas = B.any_tlas || J.fr.n_tlas >= 2;
            const int64_t np = (int64_t)c->W * c->H;
            LAUNCH(MCEV_K_STATS, launch_fill_entries(B.queue[0] + B.q0, np, (int)q, ctx->sms, ctx->stream));
            B.q0 += np;
        }
        CU(cudaMemcpyAsync(ctx->d_jobs.ptr, tab.data(), sizeof(Job) * tab.size(), cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        ctx->h2d += (int64_t)(sizeof(Job) * tab.size());
        return MCEV_OK;
    };
    // first frame of Alg. 1 for the jobs whose reference is not at t0
    std::vector<int> need;
    for (int i = 0; i < n_jobs; ++i)
        if (!jobs[i].ctx->ref_valid || jobs[i].ctx->ref_time != jobs[i].t0) need.push_back(i);
    int64_t ref_paths = 0, paths = 0;
    int32_t rounds = 0;
    if (!need.empty()) {
        for (int i : need) ST(frame_setup(jobs[i].ctx, jobs[i].t0, 0));
        ST(prepare(need, 0));
        StatsArgs R{};
        R.spp_min = R.spp_batch = R.spp_max = spp_max;
        R.mode = MODE_REFERENCE;
        for (int i : need) jobs[i].ctx->ref_valid = false;
        ST(run_rounds(ctx, ctx->frames[0], R, &ref_paths, nullptr, &B));
        for (int i : need) {
            jobs[i].ctx->ref_valid = true;
            jobs[i].ctx->ref_time = jobs[i].t0;
        }
    }
    std::vector<int> all(n_jobs);
    for (int i = 0; i < n_jobs; ++i) {
        all[i] = i;
        ST(frame_setup(jobs[i].ctx, jobs[i].t1, 1));
    }
    ST(prepare(all, 1));
    ST(ensure_tcrit(ctx, alpha, variant, spp_min, spp_batch, spp_max));
    StatsArgs A{};
    A.tcrit = (const float*)ctx->d_tcrit.ptr;
    A.C = C;
    A.spp_min = spp_min;
    A.spp_batch = spp_batch;
    A.spp_max = spp_max;
    A.mode = MODE_DETECT;
    A.variant = variant;
    A.se_mode = se_mode;
    const mcev_status rs = run_rounds(ctx, ctx->frames[1], A, &paths, &rounds, &B);
    if (rs != MCEV_OK) {
        for (int i = 0; i < n_jobs; ++i) jobs[i].ctx->ref_valid = false;
        return rs;
    }
    for (int i = 0; i < n_jobs; ++i) {
        jobs[i].ctx->ref_valid = true;
        jobs[i].ctx->ref_time = jobs[i].t1;
    }
    CU(cudaEventRecord(ctx->ev1, ctx->stream));
    ST(drain_events(ctx));
    if (stats_out) ST(fill_stats(ctx, stats_out, paths, ref_paths, rounds));
    return MCEV_OK;
}

size_t mcev_state_bytes(const mcev_ctx* ctx) {
    if (!ctx) return 0;
    return 16 + 12 * (size_t)ctx->W * ctx->H;
}

mcev_status mcev_get_state(mcev_ctx* ctx, void* dev_buf, size_t bytes) {
    if (!ctx) return MCEV_ERR_ARG;
    if (!dev_buf || bytes != mcev_state_bytes(ctx)) return fail(ctx, MCEV_ERR_ARG, "state buffer size mismatch");
    CU(cudaSetDevice(ctx->device));
    ST(ensure_pixels(ctx));
    const size_t n = (size_t)ctx->W * ctx->H;
    char hdr[16] = {0};
    int32_t valid = ctx->ref_valid ? 1 : 0, npx = (int32_t)n;
    std::memcpy(hdr, &ctx->ref_time, 8);
    std::memcpy(hdr + 8, &valid, 4);
    std::memcpy(hdr + 12, &npx, 4);
    char* d = (char*)dev_buf;
    CU(cudaMemcpyAsync(d, hdr, 16, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemcpyAsync(d + 16, ctx->ref.n, 4 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(d + 16 + 4 * n, ctx->ref.mean, 4 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(d + 16 + 8 * n, ctx->ref.m2, 4 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return MCEV_OK;
}

mcev_status mcev_set_state(mcev_ctx* ctx, const void* dev_buf, size_t bytes) {
    if (!ctx) return MCEV_ERR_ARG;
    if (!dev_buf || bytes != mcev_state_bytes(ctx)) return fail(ctx, MCEV_ERR_ARG, "state buffer size mismatch");
    CU(cudaSetDevice(ctx->device));
    ST(ensure_pixels(ctx));
    const size_t n = (size_t)ctx->W * ctx->H;
    char hdr[16];
    const char* s = (const char*)dev_buf;
    CU(cudaMemcpyAsync(hdr, s, 16, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(ctx->ref.n, s + 16, 4 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->ref.mean, s + 16 + 4 * n, 4 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(ctx->ref.m2, s + 16 + 8 * n, 4 * n, cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    int32_t valid, npx;
    std::memcpy(&ctx->ref_time, hdr, 8);
    std::memcpy(&valid, hdr + 8, 4);
    std::memcpy(&npx, hdr + 12, 4);
    if (npx != (int32_t)n) {
        ctx->ref_valid = false;
        return fail(ctx, MCEV_ERR_ARG, "state blob is for %d pixels, context has %zu", npx, n);
    }
    ctx->ref_valid = valid != 0;
    return MCEV_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ event-video quality (Sec. 4.2)
mcev_status mcev_event_quality(mcev_ctx* ctx, const int8_t* a, const int8_t* b, int32_t width, int32_t height,
                               int32_t frames, int32_t tau2, int32_t* d2_a, int32_t* d2_b, mcev_quality* out) {
    if (!ctx) return MCEV_ERR_ARG;
    if (!a || !b || !out) return fail(ctx, MCEV_ERR_ARG, "need a, b and out");
    const int32_t mx = QUALITY_MAX_EXTENT;
    if (width < 1 || height < 1 || frames < 1 || width > mx || height > mx || frames > mx)
        return fail(ctx, MCEV_ERR_ARG, "extents must lie in 1..%d", mx);
    if (tau2 < 0) return fail(ctx, MCEV_ERR_ARG, "tau2 must be >= 0");
    CU(cudaSetDevice(ctx->device));
    const int64_t n = (int64_t)width * height * frames;
    const size_t vol = ((size_t)n * sizeof(int32_t) + 255) & ~size_t(255);
    const size_t stk = ((size_t)quality_stack_bytes(width, height, frames, ctx->sms) + 255) & ~size_t(255);
    ST(dev_alloc(ctx, ctx->d_quality, 2 * vol + stk + QACC_WORDS * sizeof(unsigned long long)));
    char* base = (char*)ctx->d_quality.ptr;
    QualityArgs A{};
    A.a = a;
    A.b = b;
    A.W = width;
    A.H = height;
    A.T = frames;
    A.tau2 = tau2;
    A.d2_a = d2_a;
    A.d2_b = d2_b;
    A.vol0 = (int32_t*)base;
    A.vol1 = (int32_t*)(base + vol);
    A.stack = base + 2 * vol;
    A.acc = (unsigned long long*)(base + 2 * vol + stk);
    int nl = 0;
    CU(cudaEventRecord(ctx->ev0, ctx->stream));
    CU(launch_quality(A, ctx->sms, ctx->stream, &nl));
    CU(cudaEventRecord(ctx->ev1, ctx->stream));
    std::vector<unsigned long long> acc(QACC_WORDS);
    CU(cudaMemcpyAsync(acc.data(), A.acc, QACC_WORDS * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->d2h += (int64_t)(QACC_WORDS * sizeof(unsigned long long));
    if (acc[QACC_BAD]) return fail(ctx, MCEV_ERR_ARG, "event values must be -1, 0 or +1");
    float ms = 0.0f;
    CU(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    mcev_quality q{};
    q.voxels = n;
    q.n_a = (int64_t)acc[QACC_NA];
    q.n_b = (int64_t)acc[QACC_NB];
    q.matched_a = (int64_t)acc[QACC_MATCH_A];
    q.matched_b = (int64_t)acc[QACC_MATCH_B];
    q.none_a = (int64_t)acc[QACC_NONE_A];
    q.none_b = (int64_t)acc[QACC_NONE_B];
    q.sq_diff = (int64_t)acc[QACC_SQ];
    double sa, sb;
    std::memcpy(&sa, &acc[QACC_SUM_A], sizeof sa);
    std::memcpy(&sb, &acc[QACC_SUM_B], sizeof sb);
    const double D = std::sqrt((double)(width - 1) * (width - 1) + (double)(height - 1) * (height - 1) +
                               (double)(frames - 1) * (frames - 1));
    q.diag = D;
    // distances of d^2 < QHIST come as counts per value
    for (int v = 1; v < QHIST; ++v) {
        sa += (double)acc[QACC_HIST_A + v] * std::sqrt((double)v);
        sb += (double)acc[QACC_HIST_B + v] * std::sqrt((double)v);
    }
    q.sum_dist_a = sa + (double)q.none_a * D;
    q.sum_dist_b = sb + (double)q.none_b * D;
    // frames mapped {-1, 0, 1} -> {0, 0.5, 1}: each unit of (a - b)^2 is 1/4
    const double mse = (double)q.sq_diff / (4.0 * (double)n);
    q.rmse = std::sqrt(mse);
    q.psnr = mse == 0.0 ? HUGE_VAL : -10.0 * std::log10(mse);
    q.precision = q.n_a ? (double)q.matched_a / (double)q.n_a : 1.0;
    q.recall = q.n_b ? (double)q.matched_b / (double)q.n_b : 1.0;
    q.f1 = q.precision + q.recall > 0.0 ? 2.0 * q.precision * q.recall / (q.precision + q.recall) : 0.0;
    const double ma = q.n_a ? q.sum_dist_a / (double)q.n_a : 0.0;
    const double mb = q.n_b ? q.sum_dist_b / (double)q.n_b : 0.0;
    q.pscd = D > 0.0 ? (ma + mb) / (2.0 * D) : 0.0;
    q.gpu_ms = ms;
    q.kernel_launches = nl;
    ctx->launches += nl;
    *out = q;
    return MCEV_OK;
}
