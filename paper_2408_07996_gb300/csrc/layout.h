// layout.h -- device data layout of the renderer (host and device view).
//
// Everything the kernels read is plain arrays in HBM:
//   BVH node (64 B, two child boxes in the parent so one node fetch tests
//   both children):
//     a = (L.lo.x, L.hi.x, L.lo.y, L.hi.y)   b = (R.lo.x, R.hi.x, R.lo.y, R.hi.y)
//     c = (L.lo.z, L.hi.z, R.lo.z, R.hi.z)   d = (L, R, Lcount, Rcount)
//   where a child >= 0 is an inner node and a child < 0 is a leaf holding
//   triangles [~child, ~child + count) of the triangle array (TLAS leaves
//   hold instance ids instead of triangles).
//   Triangle (48 B): v0.xyz|prim, v1.xyz|material, v2.xyz|instance, in BVH
//   leaf order; prim = index in the uploaded triangle list.  Triangles of a
//   mesh used by moving instances are in object space with instance = -1;
//   instances that never move are merged at upload into one world-space
//   BVH whose triangles carry their instance id and resolved material.
//   Instance record (112 B): M rows 0..2, Minv rows 0..2 (3x4 each, float4),
//   then (blas root node, material override, instance id or -1, 0).
//   Light (64 B): v0.xyz|Le, v1.xyz|area, v2.xyz|material, n.xyz|0 (world space).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#ifdef __CUDACC__
#define MCEV_HD __host__ __device__
#else
#define MCEV_HD
#endif

// Traversal stack per thread (TLAS + BLAS depth must fit): in shared memory
// (32 entries, thread-interleaved) when MCEV_SMEM_STACK, else in local memory.
#ifndef MCEV_SMEM_STACK
#define MCEV_SMEM_STACK 0
#endif
#if MCEV_SMEM_STACK
#define MCEV_STACK_HOST 32
#else
#define MCEV_STACK_HOST 96
#endif

// Wide-BVH traversal stack per thread: node groups (one per wide level).
#define MCEV_WSTACK_HOST 32

namespace mcev {

struct Node {
    float4 a, b, c;
    int4 d;
};

// Compressed 8-wide node (80 B, five 16-byte words): child boxes on a grid of
// step 2^(e_a - 127) per axis a anchored at (px, py, pz); child slot s spans
// [p + qlo[s] * step, p + qhi[s] * step] per axis (empty slots: qlo > qhi),
// every plane at least 1/16 step outside the child's exact box.
//   e_imask : e_x | e_y << 8 | e_z << 16 | imask << 24  (imask bit s: slot s
//             is an internal node)
//   child_base: first child node; internal children are stored contiguously
//             in slot order, so slot s's node is child_base + popc(imask below s)
//   tri_base : bits 0..28 first triangle of the leaf slots; bits 29..31 number
//             of non-empty slots - 1
//   trimask  : bit 3s + k set when slot s is a leaf of more than k triangles
//             (1..3 per leaf); the triangles of the leaf slots are contiguous
//             in slot order, so the one of bit b is tri_base + popc(trimask below b)
//   slots are assigned by direction: slot bit a set = child on the -a side of
//   the node centre, so a ray visits slot s in the order of s ^ ox, where ox
//   has bit a set when the ray's direction component a is >= 0.
struct Node8 {
    float px, py, pz;
    uint32_t e_imask;
    uint32_t child_base, tri_base;
    uint32_t trimask, pad;
    uint32_t qlo_x[2], qlo_y[2], qlo_z[2], qhi_x[2];
    uint32_t qhi_y[2], qhi_z[2];
};
static_assert(sizeof(Node8) == 80, "wide node is five 16-byte words");

enum { MAT_DIFFUSE = 0, MAT_GGX = 1 };
// material type word: low byte = BSDF, bit 8 = albedo from the texture
enum { MAT_TEXTURED = 0x100 };

struct DevScene {
    const Node* nodes;        // BLAS nodes of every mesh (two-wide layout)
    const uint4* wnodes;      // BLAS nodes of every mesh (compressed 8-wide layout: 5 uint4 per node)
    int32_t wide;             // 1: the BLAS roots index `wnodes`
    const float4* tris;       // 3 float4 per triangle, leaf order
    const float4* tshade;     // per triangle, leaf order: object-space (v1-v0)x(v2-v0), material (int bits)
    const float4* mats;       // (type, albedo, rough, emit)
    const float* env;         // [eh][ew] radiance
    const float* env_marg;    // [eh + 1] row CDF
    const float* env_cond;    // [eh][ew + 1] column CDFs
    const float* env_tpdf;    // [eh][ew]: texel pdf numerator, pdf = tpdf / sin(theta)
    int32_t env_w, env_h;
    int32_t env_ok;           // environment present with positive total radiance
    int32_t has_env;          // environment present (lookups on miss)
    const float2* tri_uv;     // 3 texture coordinates per triangle (leaf order), or null
    const float* tex;         // caller's RGB albedo texture [tex_h][tex_w][3], or null
    int32_t tex_w, tex_h;
    const float* emit;        // caller's emitted radiance per material (overrides the table), or null
};

struct DevFrame {
    const Node* tlas;         // TLAS nodes; leaves hold instance ids
    const float4* inst;       // 7 float4 per instance
    const float4* lights;     // 4 float4 per emissive triangle
    int32_t n_inst, n_lights;
    // records 0 .. n_tlas-1 (the moving instances) sit under the TLAS; with
    // n_tlas == 1 there is nothing to traverse.  The merged never-moving
    // geometry, if any, is record static_rec (= n_tlas) and is traversed on
    // its own, before the TLAS.
    int32_t n_tlas;
    int32_t static_rec;       // or -1
    float eye[3], fwd[3], right[3], up[3];  // right, up prescaled by tan(fov/2)*aspect
    uint32_t key0, key1;      // Philox key
    float p_env, p_area;      // NEE light-type selection probabilities
};

// Per-render settings, passed by value to the kernels.
struct DevParams {
    int32_t width, height;
    int32_t max_depth;
    int32_t nee, mis;
    float eps;
    float t_min;
    int32_t want_sig;         // maintain the decision signature
    // adjoint replay (mcev_backward): 1 in the second pass over a chunk
    int32_t adjoint;
    int32_t spp;              // samples per pixel of the replayed frame
    const float* grad_mean;   // d loss / d mean ln(L + eps), per pixel
    float* grad_tex;          // accumulated d loss / d texel RGB
    double* grad_emit;        // accumulated d loss / d emitted radiance, per material (FP64:
                              // millions of contributions land on a few materials)
};

// Wavefront buffers of one chunk (capacity = `cap` paths).
struct Wave {
    // per path slot p
    float* L;
    uint32_t* sig;
    uint32_t* pflags;         // pending flags of the last vertex (0xFFFFFFFF = none)
    int2* pix_k;              // (queue entry, sample index); written for batched renders only
    // ray queues (ping-pong) and hits, per queue slot
    float4* ray_o[2];         // xyz origin, w = path slot (int bits)
    float4* ray_d[2];         // xyz direction, w = depth (int bits)
    float4* ray_s[2];         // path state carried with the ray: throughput, pdf of the sampled
                              // direction, queue entry and sample index (int bits)
    float4* hit;              // t, instance, leaf-order triangle, 0   (inst < 0: miss)
    // shadow rays
    float4* sh_o;             // xyz origin, w = path slot
    float4* sh_d;             // xyz direction, w = t_max
    float* sh_c;              // unoccluded contribution
    float* sh_g;              // adjoint: contribution / emitted radiance of the sampled light
    int32_t* sh_m;            // adjoint: material of the sampled light (-1: environment)
    float* Ltot;              // adjoint: radiance of each path from the first pass
    float* delta;             // adjoint: d loss / d L of each path
    // Device counters, 64 int32 words; every slot the kernels use:
    //   [0], [1]  ray queue sizes (ping-pong queues 0 and 1)
    //   [2], [19] shadow-ray counts of the bounces traced from ray queue 0 / 1
    //   [3]       undecided pixels re-queued by the statistics kernel
    //   [4]       non-finite path values (counted as 0)
    //   [5], [6]  positive / negative events
    //   [7]       pixels decided at spp_max
    //   [8]       caller pixel id outside [0, n_total) (allocation-free step)
    //   [15]      traversal stack overflow
    //   from [32] on, uint64 words: [0] nodes and [1] triangles of closest-hit
    //   traversal, [2] nodes and [3] triangles of shadow rays, [4] closest-hit
    //   rays, [5] shadow rays, [6] samples that entered decisions, [7] and
    //   [8] ray/box tests of closest-hit and shadow traversal
    int32_t* counters;
    int64_t cap;
};

// Per-pixel statistics (SoA): count, mean and M2 of ln(L + eps).
struct PixStats {
    int32_t* n;
    float* mean;
    float* m2;
};

// One frame pair of a batched render: its context's scene, frame, render
// settings, per-pixel state and outputs.  Batched queue entries are
// (job << 24 | pixel).
struct Job {
    DevScene sc;
    DevFrame fr;
    DevParams P;
    PixStats cur, ref;
    int8_t* events;
    int32_t* spp_out;
    float* mean_out;
};

}  // namespace mcev
