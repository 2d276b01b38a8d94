// device.cuh -- device-side building blocks of the path tracer (FP32).
//
// Scene and sampling conventions (they define the samples the method
// averages, Sec. 3.1, and are restated independently by the test oracle):
//  * Philox4x32-10 (Salmon et al., SC 2011); counter (pixel, sample, vertex,
//    block), key (seed_lo ^ frame key, seed_hi); u = (x >> 8) * 2^-24.
//  * pinhole camera, box-filtered jitter, field of view on the shorter axis;
//  * watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013);
//  * Lambertian (cosine sampling) and GGX with Smith height-correlated
//    masking, Schlick Fresnel and visible-normal sampling (Heitz, JCGT 2018);
//  * lat-long environment, piecewise-constant importance sampling;
//  * uniform choice among emissive triangles, uniform area sampling.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace mcev {

#define MCEV_PI 3.14159265358979323846f
#define MCEV_STACK MCEV_STACK_HOST
// traversal kernels run 128-thread blocks; the shared stack interleaves threads
#define MCEV_TRAV_BLOCK 128
#if MCEV_SMEM_STACK
#define SIDX(i) ((i) * MCEV_TRAV_BLOCK)
#define MCEV_DECLARE_STACK(name)                               \
    __shared__ int name##_smem[MCEV_STACK * MCEV_TRAV_BLOCK];  \
    int* name = name##_smem + threadIdx.x
#else
#define SIDX(i) (i)
#define MCEV_DECLARE_STACK(name) int name[MCEV_STACK]
#endif

// ------------------------------------------------------------------ math
struct f3 {
    float x, y, z;
};
__device__ __forceinline__ f3 mk3(float x, float y, float z) { return f3{x, y, z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return mk3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return mk3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ f3 operator*(f3 a, float s) { return mk3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(f3 a, f3 b) { return fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)); }
__device__ __forceinline__ f3 cross3(f3 a, f3 b) {
    return mk3(fmaf(a.y, b.z, -(a.z * b.y)), fmaf(a.z, b.x, -(a.x * b.z)), fmaf(a.x, b.y, -(a.y * b.x)));
}
__device__ __forceinline__ f3 norm3(f3 a) { return a * (1.0f / sqrtf(dot3(a, a))); }
__device__ __forceinline__ f3 xyz(float4 v) { return mk3(v.x, v.y, v.z); }

// row-major 3x4 affine (rows r0, r1, r2)
__device__ __forceinline__ f3 xf_point(float4 r0, float4 r1, float4 r2, f3 p) {
    return mk3(fmaf(r0.z, p.z, fmaf(r0.y, p.y, fmaf(r0.x, p.x, r0.w))),
               fmaf(r1.z, p.z, fmaf(r1.y, p.y, fmaf(r1.x, p.x, r1.w))),
               fmaf(r2.z, p.z, fmaf(r2.y, p.y, fmaf(r2.x, p.x, r2.w))));
}
__device__ __forceinline__ f3 xf_vec(float4 r0, float4 r1, float4 r2, f3 p) {
    return mk3(dot3(xyz(r0), p), dot3(xyz(r1), p), dot3(xyz(r2), p));
}
// (A^-1)^T n from the rows of the inverse
__device__ __forceinline__ f3 xf_normal(float4 i0, float4 i1, float4 i2, f3 n) {
    return mk3(fmaf(i2.x, n.z, fmaf(i1.x, n.y, i0.x * n.x)), fmaf(i2.y, n.z, fmaf(i1.y, n.y, i0.y * n.x)),
               fmaf(i2.z, n.z, fmaf(i1.z, n.y, i0.z * n.x)));
}

// ------------------------------------------------------------------ Philox4x32-10
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }

// ------------------------------------------------------------------ ONB (Duff et al. 2017)
__device__ __forceinline__ void onb(f3 n, f3& t, f3& b) {
    const float sg = n.z >= 0.0f ? 1.0f : -1.0f;
    const float a = -1.0f / (sg + n.z);
    const float bb = n.x * n.y * a;
    t = mk3(1.0f + sg * n.x * n.x * a, sg * bb, -sg * n.x);
    b = mk3(bb, sg + n.y * n.y * a, -n.y);
}

// ------------------------------------------------------------------ BSDFs (local frame, n = +z)
__device__ __forceinline__ float ggx_lambda(float a, float z) {
    const float t2 = (1.0f - z * z) / (z * z);
    return 0.5f * (-1.0f + sqrtf(1.0f + a * a * t2));
}

// returns f(wo, wi); *pdf = pdf of sampling wi
__device__ __forceinline__ float bsdf_eval(int type, float albedo, float rough, f3 wo, f3 wi, float* pdf) {
    *pdf = 0.0f;
    if (!(wo.z > 0.0f) || !(wi.z > 0.0f)) return 0.0f;
    if (type == MAT_DIFFUSE) {
        *pdf = wi.z * (1.0f / MCEV_PI);
        return albedo * (1.0f / MCEV_PI);
    }
    const f3 h = norm3(wo + wi);
    const float a2 = rough * rough;
    const float k = h.z * h.z * (a2 - 1.0f) + 1.0f;
    const float D = a2 / (MCEV_PI * k * k);
    const float lo = ggx_lambda(rough, wo.z), li = ggx_lambda(rough, wi.z);
    const float G1 = 1.0f / (1.0f + lo);
    const float G2 = 1.0f / (1.0f + lo + li);
    const float c = dot3(wi, h);
    const float m = 1.0f - c;
    const float m2 = m * m;
    const float F = albedo + (1.0f - albedo) * (m2 * m2 * m);
    *pdf = G1 * D / (4.0f * wo.z);
    return F * D * G2 / (4.0f * wo.z * wi.z);
}

__device__ __forceinline__ f3 bsdf_sample(int type, float rough, f3 wo, float u1, float u2) {
    float s, c;
    sincosf(2.0f * MCEV_PI * u2, &s, &c);
    if (type == MAT_DIFFUSE) {
        const float r = sqrtf(u1);
        return mk3(r * c, r * s, sqrtf(fmaxf(0.0f, 1.0f - u1)));
    }
    const float a = rough;
    const f3 Vh = norm3(mk3(a * wo.x, a * wo.y, wo.z));
    const float lensq = Vh.x * Vh.x + Vh.y * Vh.y;
    const f3 T1 = lensq > 0.0f ? mk3(-Vh.y, Vh.x, 0.0f) * (1.0f / sqrtf(lensq)) : mk3(1.0f, 0.0f, 0.0f);
    const f3 T2 = cross3(Vh, T1);
    const float r = sqrtf(u1);
    const float t1 = r * c;
    float t2 = r * s;
    const float sh = 0.5f * (1.0f + Vh.z);
    t2 = (1.0f - sh) * sqrtf(1.0f - t1 * t1) + sh * t2;
    const f3 Nh = T1 * t1 + T2 * t2 + Vh * sqrtf(fmaxf(0.0f, 1.0f - t1 * t1 - t2 * t2));
    const f3 Ne = norm3(mk3(a * Nh.x, a * Nh.y, fmaxf(0.0f, Nh.z)));
    const float d = dot3(wo, Ne);
    return Ne * (2.0f * d) - wo;
}

// ------------------------------------------------------------------ environment
__device__ __forceinline__ void env_texel(const DevScene& sc, f3 d, int& row, int& col, float& sin_t) {
    const float cy = fminf(1.0f, fmaxf(-1.0f, d.y));
    const float theta = acosf(cy);
    float phi = atan2f(d.z, d.x);
    if (phi < 0.0f) phi += 2.0f * MCEV_PI;
    col = min((int)(phi / (2.0f * MCEV_PI) * (float)sc.env_w), sc.env_w - 1);
    row = min((int)(theta / MCEV_PI * (float)sc.env_h), sc.env_h - 1);
    sin_t = sinf(theta);
}

__device__ __forceinline__ float texel_pdf(const DevScene& sc, int row, int col, float sin_t) {
    if (!sc.env_ok || !(sin_t > 0.0f)) return 0.0f;
    return __ldg(sc.env_tpdf + (int64_t)row * sc.env_w + col) / sin_t;
}

// smallest k in [0, n) with u < cdf[k + 1]
__device__ __forceinline__ int cdf_pick(const float* cdf, int n, float u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (u < __ldg(cdf + mid + 1)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ f3 env_sample(const DevScene& sc, float u1, float u2, float& pdf, float& Le) {
    const int row = cdf_pick(sc.env_marg, sc.env_h, u1);
    const float m0 = __ldg(sc.env_marg + row), m1 = __ldg(sc.env_marg + row + 1);
    const float dv = (u1 - m0) / (m1 - m0);
    const float* c = sc.env_cond + (int64_t)row * (sc.env_w + 1);
    const int col = cdf_pick(c, sc.env_w, u2);
    const float c0 = __ldg(c + col), c1 = __ldg(c + col + 1);
    const float du = (u2 - c0) / (c1 - c0);
    const float theta = MCEV_PI * ((float)row + dv) / (float)sc.env_h;
    const float phi = 2.0f * MCEV_PI * ((float)col + du) / (float)sc.env_w;
    float st, ct, sp, cp;
    sincosf(theta, &st, &ct);
    sincosf(phi, &sp, &cp);
    Le = __ldg(sc.env + (int64_t)row * sc.env_w + col);
    pdf = texel_pdf(sc, row, col, st);
    return mk3(st * cp, ct, st * sp);
}

__device__ __forceinline__ float power_heuristic(float a, float b) {
    const float a2 = a * a, b2 = b * b;
    return a2 / (a2 + b2);
}

__device__ __forceinline__ uint32_t fnv(uint32_t h, uint32_t w) { return (h ^ w) * 16777619u; }

// ------------------------------------------------------------------ texture
// Barycentric coordinates (b1, b2) of point p in triangle (a, b, c) from the
// normal equations of p - a = b1 (b - a) + b2 (c - a).
__device__ __forceinline__ void barycentric(f3 p, f3 a, f3 b, f3 c, float& b1, float& b2) {
    const f3 e1 = b - a, e2 = c - a, vp = p - a;
    const float d00 = dot3(e1, e1), d01 = dot3(e1, e2), d11 = dot3(e2, e2);
    const float d20 = dot3(vp, e1), d21 = dot3(vp, e2);
    const float den = d00 * d11 - d01 * d01;
    b1 = (d11 * d20 - d01 * d21) / den;
    b2 = (d00 * d21 - d01 * d20) / den;
}

// nearest texel of texture coordinates (u, v), wrapped to [0, 1)
__device__ __forceinline__ int texel_of(const DevScene& sc, float u, float v) {
    u -= floorf(u);
    v -= floorf(v);
    // the clamps also catch u = 1 after rounding and NaN coordinates (degenerate triangles)
    const int ix = max(0, min((int)(u * (float)sc.tex_w), sc.tex_w - 1));
    const int iy = max(0, min((int)(v * (float)sc.tex_h), sc.tex_h - 1));
    return iy * sc.tex_w + ix;
}

// scalar albedo of an RGB texel: Rec. 709 luminance
#define MCEV_Y_R 0.2126f
#define MCEV_Y_G 0.7152f
#define MCEV_Y_B 0.0722f

// ------------------------------------------------------------------ intersection
// Watertight test: the ray is sheared so it becomes the +z axis; 2D edge
// functions U, V, W of the sheared vertices decide containment.
struct WRay {
    f3 o;
    f3 mx, my, mz;    // shear rows: x' = mx.A, y' = my.A, z' = mz.A for A = v - o
    f3 idir;          // 1/d with tiny components replaced, for slab tests
    f3 oidir;         // o * idir
};

__device__ __forceinline__ WRay make_wray(f3 o, f3 d) {
    WRay r;
    r.o = o;
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = 0;
    if (ay > ax && ay >= az) kz = 1;
    else if (az > ax && az > ay) kz = 2;
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const float dz = kz == 0 ? d.x : (kz == 1 ? d.y : d.z);
    if (dz < 0.0f) {
        const int t = kx;
        kx = ky;
        ky = t;
    }
    const float dkx = kx == 0 ? d.x : (kx == 1 ? d.y : d.z);
    const float dky = ky == 0 ? d.x : (ky == 1 ? d.y : d.z);
    const float Sx = dkx / dz, Sy = dky / dz, Sz = 1.0f / dz;
    r.mx = mk3(kx == 0 ? 1.0f : 0.0f, kx == 1 ? 1.0f : 0.0f, kx == 2 ? 1.0f : 0.0f);
    r.my = mk3(ky == 0 ? 1.0f : 0.0f, ky == 1 ? 1.0f : 0.0f, ky == 2 ? 1.0f : 0.0f);
    r.mz = mk3(kz == 0 ? Sz : 0.0f, kz == 1 ? Sz : 0.0f, kz == 2 ? Sz : 0.0f);
    if (kz == 0) { r.mx.x = -Sx; r.my.x = -Sy; }
    if (kz == 1) { r.mx.y = -Sx; r.my.y = -Sy; }
    if (kz == 2) { r.mx.z = -Sx; r.my.z = -Sy; }
    const float ooeps = 0x1p-80f;
    r.idir = mk3(1.0f / (fabsf(d.x) > ooeps ? d.x : copysignf(ooeps, d.x)),
                 1.0f / (fabsf(d.y) > ooeps ? d.y : copysignf(ooeps, d.y)),
                 1.0f / (fabsf(d.z) > ooeps ? d.z : copysignf(ooeps, d.z)));
    r.oidir = mk3(o.x * r.idir.x, o.y * r.idir.y, o.z * r.idir.z);
    return r;
}

// returns t in (tmin, tmax) or -1 (no hit); tmax inclusive when `incl`
__device__ __forceinline__ float tri_hit(const WRay& r, float4 p0, float4 p1, float4 p2, float tmin, float tmax) {
    const f3 A = xyz(p0) - r.o, B = xyz(p1) - r.o, C = xyz(p2) - r.o;
    const float Ax = dot3(r.mx, A), Ay = dot3(r.my, A);
    const float Bx = dot3(r.mx, B), By = dot3(r.my, B);
    const float Cx = dot3(r.mx, C), Cy = dot3(r.my, C);
    const float U = fmaf(Cx, By, -(Cy * Bx));
    const float V = fmaf(Ax, Cy, -(Ay * Cx));
    const float W = fmaf(Bx, Ay, -(By * Ax));
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return -1.0f;
    const float det = U + V + W;
    if (det == 0.0f) return -1.0f;
    const float T = fmaf(W, dot3(r.mz, C), fmaf(V, dot3(r.mz, B), U * dot3(r.mz, A)));
    const float t = T / det;
    return (t > tmin && t <= tmax) ? t : -1.0f;
}

// three-input minimum / maximum (single instructions on sm_100 and later)
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// slab test of both children of a node; returns hit mask (bit0 left, bit1 right)
__device__ __forceinline__ int node_hits(const WRay& r, const Node& n, float tmin, float tmax, float& tl, float& tr) {
    const float4 a = n.a, b = n.b, c = n.c;
    const float lx0 = fmaf(a.x, r.idir.x, -r.oidir.x), lx1 = fmaf(a.y, r.idir.x, -r.oidir.x);
    const float ly0 = fmaf(a.z, r.idir.y, -r.oidir.y), ly1 = fmaf(a.w, r.idir.y, -r.oidir.y);
    const float lz0 = fmaf(c.x, r.idir.z, -r.oidir.z), lz1 = fmaf(c.y, r.idir.z, -r.oidir.z);
    const float rx0 = fmaf(b.x, r.idir.x, -r.oidir.x), rx1 = fmaf(b.y, r.idir.x, -r.oidir.x);
    const float ry0 = fmaf(b.z, r.idir.y, -r.oidir.y), ry1 = fmaf(b.w, r.idir.y, -r.oidir.y);
    const float rz0 = fmaf(c.z, r.idir.z, -r.oidir.z), rz1 = fmaf(c.w, r.idir.z, -r.oidir.z);
    const float ln = max3f(fminf(lx0, lx1), fminf(ly0, ly1), fmaxf(fminf(lz0, lz1), tmin));
    const float lf = min3f(fmaxf(lx0, lx1), fmaxf(ly0, ly1), fminf(fmaxf(lz0, lz1), tmax));
    const float rn = max3f(fminf(rx0, rx1), fminf(ry0, ry1), fmaxf(fminf(rz0, rz1), tmin));
    const float rf = min3f(fmaxf(rx0, rx1), fmaxf(ry0, ry1), fminf(fmaxf(rz0, rz1), tmax));
    tl = ln;
    tr = rn;
    // (1 + 2^-20) slack keeps rounding in the slab arithmetic from culling a hit
    return (ln <= lf * 1.000001f + 1e-30f ? 1 : 0) | (rn <= rf * 1.000001f + 1e-30f ? 2 : 0);
}

__device__ __forceinline__ Node load_node(const Node* nodes, int i) {
    const float4* p = reinterpret_cast<const float4*>(nodes + i);
    Node n;
    n.a = __ldg(p);
    n.b = __ldg(p + 1);
    n.c = __ldg(p + 2);
    const float4 d = __ldg(p + 3);
    n.d = make_int4(__float_as_int(d.x), __float_as_int(d.y), __float_as_int(d.z), __float_as_int(d.w));
    return n;
}

struct Hit {
    float t;
    int inst;   // uploaded instance id (ties, signature)
    int tri;    // leaf-order triangle index
    int prim;   // uploaded triangle id (ties)
    int rec;    // instance record of the frame (transform)
};

__device__ __forceinline__ bool better_hit(float t, int inst, int prim, const Hit& h) {
    if (t < h.t) return true;
    if (t > h.t) return false;
    if (inst != h.inst) return inst < h.inst;
    return prim < h.prim;
}

// BLAS closest hit of an object-space ray; updates h
#define MCEV_NO_NODE (-0x7fffffff)
// any-hit traversal visits the nearer child first when MCEV_ANY_ORDERED
// (occluders are found sooner; ~1% faster shadow rays on the terrain frame)
#ifndef MCEV_ANY_ORDERED
#define MCEV_ANY_ORDERED 1
#endif

// ------------------------------------------------------------------ compressed 8-wide BLAS
// Traversal of the Node8 layout (layout.h).  A "node group" is a 64-bit word
// pair (child_base, bits): bits 24..31 mark the internal children of one node
// still to visit, indexed by visit key = slot ^ ox (ox: bit a set when the
// ray's direction component a is >= 0, so children on the -a side come first),
// bits 0..7 hold that node's imask, so slot s's node is
// child_base + popc(imask below s).
#define MCEV_WSTACK MCEV_WSTACK_HOST

// 1 + q * 2^-15 for the byte q of `w` at position b (a float whose mantissa
// holds q: 0x3F80_qq_00), built by one byte permute
__device__ __forceinline__ float qplane(uint32_t w, int b) {
    return __uint_as_float(__byte_perm(w, 0x3F800000u, 0x7604u | ((uint32_t)b << 4)));
}

// bit s of x moved to bit s ^ ox (x: 8 bits)
__device__ __forceinline__ uint32_t xor_permute8(uint32_t x, uint32_t ox) {
    x = (ox & 1u) ? (((x & 0x55u) << 1) | ((x >> 1) & 0x55u)) : x;
    x = (ox & 2u) ? (((x & 0x33u) << 2) | ((x >> 2) & 0x33u)) : x;
    x = (ox & 4u) ? (((x & 0x0Fu) << 4) | ((x >> 4) & 0x0Fu)) : x;
    return x;
}

// bit s of x (8 bits) copied to bits 3s, 3s+1, 3s+2
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
    x = (x | (x << 8)) & 0x00F00Fu;
    x = (x | (x << 4)) & 0x0C30C3u;
    x = (x | (x << 2)) & 0x249249u;
    return x * 7u;
}

// Tests the up to eight child boxes of wide node `idx` against the ray over
// [tmin, tmax].  Returns the 8-bit mask of hit slots and the node's child and
// triangle bases, imask and triangle mask.  A plane at q grid steps is
// p + q * 2^k; with f = 1 + q 2^-15 its ray parameter is f * A + B,
// A = 2^(k+15) / d, B = (p - o) / d - A: one FMA per plane, A exact, the
// other roundings far inside the 1/16-step margin the builder leaves around
// every child box.
__device__ __forceinline__ uint32_t wide_node_hits(const uint4* __restrict__ wn, uint32_t idx, const WRay& r,
                                                   uint32_t ox, float tmin, float tmax, uint32_t& child_base,
                                                   uint32_t& tri_base, uint32_t& imask, uint32_t& trimask,
                                                   int& nvalid) {
    const uint4* np = wn + 5 * (size_t)idx;
    const uint4 v0 = __ldg(np), v1 = __ldg(np + 1), v2 = __ldg(np + 2), v3 = __ldg(np + 3), v4 = __ldg(np + 4);
    const float Ax = __uint_as_float(((v0.w & 0xFFu) + 15u) << 23) * r.idir.x;
    const float Ay = __uint_as_float((((v0.w >> 8) & 0xFFu) + 15u) << 23) * r.idir.y;
    const float Az = __uint_as_float((((v0.w >> 16) & 0xFFu) + 15u) << 23) * r.idir.z;
    const float Bx = fmaf(__uint_as_float(v0.x) - r.o.x, r.idir.x, -Ax);
    const float By = fmaf(__uint_as_float(v0.y) - r.o.y, r.idir.y, -Ay);
    const float Bz = fmaf(__uint_as_float(v0.z) - r.o.z, r.idir.z, -Az);
    child_base = v1.x;
    tri_base = v1.y & 0x1FFFFFFFu;
    nvalid = (int)(v1.y >> 29) + 1;
    trimask = v1.z;
    imask = v0.w >> 24;
    // near and far plane words per axis: the low planes are near for d >= 0
    const bool sx = (ox & 1u) != 0, sy = (ox & 2u) != 0, sz = (ox & 4u) != 0;
    const uint32_t nx[2] = {sx ? v2.x : v3.z, sx ? v2.y : v3.w}, fx[2] = {sx ? v3.z : v2.x, sx ? v3.w : v2.y};
    const uint32_t ny[2] = {sy ? v2.z : v4.x, sy ? v2.w : v4.y}, fy[2] = {sy ? v4.x : v2.z, sy ? v4.y : v2.w};
    const uint32_t nz[2] = {sz ? v3.x : v4.z, sz ? v3.y : v4.w}, fz[2] = {sz ? v4.z : v3.x, sz ? v4.w : v3.y};
    uint32_t hit8 = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float tnx = fmaf(qplane(nx[h], b), Ax, Bx), tfx = fmaf(qplane(fx[h], b), Ax, Bx);
            const float tny = fmaf(qplane(ny[h], b), Ay, By), tfy = fmaf(qplane(fy[h], b), Ay, By);
            const float tnz = fmaf(qplane(nz[h], b), Az, Bz), tfz = fmaf(qplane(fz[h], b), Az, Bz);
            const float tn = max3f(tnx, tny, fmaxf(tnz, tmin));
            const float tf = min3f(tfx, tfy, fminf(tfz, tmax));
            if (tn <= tf) hit8 |= 1u << (4 * h + b);
        }
    }
    return hit8;
}

// Closest hit (kAny = false; updates h) or any hit in (tmin, tmax] (kAny =
// true; returns true at the first occluder) of an object-space ray in the
// wide BLAS rooted at `root`.  work: (node fetches, triangle tests, box tests).
template <bool kAny>
__device__ __forceinline__ bool blas_wide(const DevScene& sc, uint32_t root, int rec, int inst, const WRay& r,
                                          float tmin, float tmax, Hit& h, uint2* stack, int* err, int3& work) {
    const uint32_t ox = (r.idir.x >= 0.0f ? 1u : 0u) | (r.idir.y >= 0.0f ? 2u : 0u) | (r.idir.z >= 0.0f ? 4u : 0u);
    // the root as the only (internal, slot 0) child of a virtual parent
    uint2 g = make_uint2(root, (1u << (24 + ox)) | 1u);
    int sp = 0;
    // one loop iteration per node OR per triangle (as in the two-wide loop)
    uint32_t tb = 0, tbits = 0, tmask = 0;
    while (true) {
        if (tbits) {
            const uint32_t bit = (uint32_t)(__ffs(tbits) - 1);
            tbits &= tbits - 1;
            const uint32_t ti = tb + __popc(tmask & ((1u << bit) - 1u));
            const float4* tp = sc.tris + 3 * ti;
            const float4 p0 = __ldg(tp), p1 = __ldg(tp + 1), p2 = __ldg(tp + 2);
            work.y += 1;
            const float t = tri_hit(r, p0, p1, p2, tmin, kAny ? tmax : h.t);
            if (kAny) {
                if (t >= 0.0f) return true;
            } else {
                const int oi = inst >= 0 ? inst : __float_as_int(p2.w);
                if (t >= 0.0f && better_hit(t, oi, __float_as_int(p0.w), h)) {
                    h.t = t; h.inst = oi; h.tri = (int)ti; h.prim = __float_as_int(p0.w); h.rec = rec;
                }
            }
            continue;
        }
        if (!(g.y & 0xFF000000u)) {
            if (sp == 0) break;
            g = stack[--sp];
        }
        const uint32_t key = __ffs(g.y >> 24) - 1;
        g.y &= ~(1u << (24 + key));
        const uint32_t slot = key ^ ox;
        const uint32_t child = g.x + __popc(g.y & ((1u << slot) - 1u) & 0xFFu);
        if (g.y & 0xFF000000u) {
            if (sp < MCEV_WSTACK) stack[sp++] = g;
            else *err = 1;
        }
        uint32_t cb, im;
        int nv;
        const uint32_t hit8 = wide_node_hits(sc.wnodes, child, r, ox, tmin, kAny ? tmax : h.t, cb, tb, im, tmask, nv);
        work.x += 1;
        work.z += nv;
        g = make_uint2(cb, (xor_permute8(hit8 & im, ox) << 24) | im);
        tbits = spread3(hit8 & ~im) & tmask;
    }
    return false;
}

// Two-wide BLAS traversal, one loop iteration per node step OR per leaf
// triangle: a node step records its hit leaf children as a pending triangle
// range (sibling leaves are contiguous in the leaf order) instead of testing
// them at once, and the lane tests one pending triangle per iteration before
// its next node step.  Lanes testing triangles and lanes stepping through
// nodes then share warp iterations, instead of the warp running every lane's
// triangle loop while the others wait (measured: 75 % of warp-steps of the
// terrain frame carried such loops at 6 % lane activity).  Nodes and
// triangles are visited in the same order as a test-at-once traversal, so
// the closest hit is the same.
// rec: instance record; inst: its uploaded instance id, or -1 for the merged
// static geometry whose triangles carry their own instance id (v2.w).

__device__ __forceinline__ void blas_closest(const DevScene& sc, int root, int rec, int inst, const WRay& r,
                                                  float tmin, Hit& h, int* stack, int base, int* err, int3& work) {
    int sp = base, node = root;
    int pfirst = 0, pcount = 0;
    while (true) {
        if (pcount > 0) {
            const float4* tp = sc.tris + 3 * pfirst;
            const float4 p0 = __ldg(tp), p1 = __ldg(tp + 1), p2 = __ldg(tp + 2);
            const float t = tri_hit(r, p0, p1, p2, tmin, h.t);
            const int oi = inst >= 0 ? inst : __float_as_int(p2.w);
            if (t >= 0.0f && better_hit(t, oi, __float_as_int(p0.w), h)) {
                h.t = t; h.inst = oi; h.tri = pfirst; h.prim = __float_as_int(p0.w); h.rec = rec;
            }
            work.y += 1;
            ++pfirst;
            --pcount;
            continue;
        }
        if (node == MCEV_NO_NODE) {
            if (sp == base) break;
            node = stack[SIDX(--sp)];
        }
        const Node n = load_node(sc.nodes, node);
        work.x += 1;
        float tl, tr;
        const int m = node_hits(r, n, tmin, h.t, tl, tr);
        const bool lh = (m & 1) && n.d.x < 0, rh = (m & 2) && n.d.y < 0;
        pfirst = lh ? ~n.d.x : ~n.d.y;
        pcount = (lh ? n.d.z : 0) + (rh ? n.d.w : 0);
        const bool gl = (m & 1) && n.d.x >= 0 && tl <= h.t;
        const bool gr = (m & 2) && n.d.y >= 0 && tr <= h.t;
        int next = MCEV_NO_NODE;
        if (gl && gr) {
            const int nearc = tl <= tr ? n.d.x : n.d.y;
            const int farc = tl <= tr ? n.d.y : n.d.x;
            if (sp < MCEV_STACK) stack[SIDX(sp++)] = farc;
            else *err = 1;
            next = nearc;
        } else if (gl) {
            next = n.d.x;
        } else if (gr) {
            next = n.d.y;
        }
        node = next;
    }
}

__device__ __forceinline__ bool blas_any(const DevScene& sc, int root, const WRay& r, float tmin, float tmax,
                                              int* stack, int base, int* err, int3& work) {
    int sp = base, node = root;
    int pfirst = 0, pcount = 0;
    while (true) {
        if (pcount > 0) {
            const float4* tp = sc.tris + 3 * pfirst;
            work.y += 1;
            if (tri_hit(r, __ldg(tp), __ldg(tp + 1), __ldg(tp + 2), tmin, tmax) >= 0.0f) return true;
            ++pfirst;
            --pcount;
            continue;
        }
        if (node == MCEV_NO_NODE) {
            if (sp == base) return false;
            node = stack[SIDX(--sp)];
        }
        const Node n = load_node(sc.nodes, node);
        work.x += 1;
        float tl, tr;
        const int m = node_hits(r, n, tmin, tmax, tl, tr);
        const bool lh = (m & 1) && n.d.x < 0, rh = (m & 2) && n.d.y < 0;
        pfirst = lh ? ~n.d.x : ~n.d.y;
        pcount = (lh ? n.d.z : 0) + (rh ? n.d.w : 0);
        const bool gl = (m & 1) && n.d.x >= 0;
        const bool gr = (m & 2) && n.d.y >= 0;
        int next = MCEV_NO_NODE;
        if (gl && gr) {
#if MCEV_ANY_ORDERED
            const int nearc = tl <= tr ? n.d.x : n.d.y;
            const int farc = tl <= tr ? n.d.y : n.d.x;
#else
            const int nearc = n.d.x;
            const int farc = n.d.y;
#endif
            if (sp < MCEV_STACK) stack[SIDX(sp++)] = farc;
            else *err = 1;
            next = nearc;
        } else if (gl) {
            next = n.d.x;
        } else if (gr) {
            next = n.d.y;
        }
        node = next;
    }
}

// instance record: rows M0..M2, Minv0..Minv2, (root, override, instance id, 0)
__device__ __forceinline__ WRay object_ray(const DevFrame& fr, int rec, f3 o, f3 d, int& root, int& inst) {
    const float4* ip = fr.inst + 7 * rec;
    const float4 i0 = __ldg(ip + 3), i1 = __ldg(ip + 4), i2 = __ldg(ip + 5);
    const float4 tail = __ldg(ip + 6);
    root = __float_as_int(tail.x);
    inst = __float_as_int(tail.z);
    return make_wray(xf_point(i0, i1, i2, o), xf_vec(i0, i1, i2, d));
}

// BLAS traversal of either layout; `stack`/`base` are the two-wide stack,
// `wstack` the wide one.  work.z (box tests) is kept for the wide layout only:
// a two-wide node fetch always tests two boxes.
template <bool kWide>
__device__ __forceinline__ void blas_closest_any_layout(const DevScene& sc, int root, int rec, int inst, const WRay& r,
                                                        float tmin, Hit& h, int* stack, int base, uint2* wstack,
                                                        int* err, int3& work) {
    if (kWide) {
        blas_wide<false>(sc, (uint32_t)root, rec, inst, r, tmin, 0.0f, h, wstack, err, work);
    } else {
        blas_closest(sc, root, rec, inst, r, tmin, h, stack, base, err, work);
    }
}

template <bool kWide>
__device__ __forceinline__ bool blas_any_layout(const DevScene& sc, int root, const WRay& r, float tmin, float tmax,
                                                int* stack, int base, uint2* wstack, int* err, int3& work) {
    if (kWide) {
        Hit dummy;
        return blas_wide<true>(sc, (uint32_t)root, 0, 0, r, tmin, tmax, dummy, wstack, err, work);
    }
    return blas_any(sc, root, r, tmin, tmax, stack, base, err, work);
}

#define MCEV_DECLARE_WSTACK(name) uint2 name[kWide ? MCEV_WSTACK : 1]

// The slab-test part of make_wray (reciprocal direction and origin times it),
// enough for TLAS box tests; the same arithmetic as make_wray.
__device__ __forceinline__ void slab_ray(WRay& r, f3 o, f3 d) {
    const float ooeps = 0x1p-80f;
    r.idir = mk3(1.0f / (fabsf(d.x) > ooeps ? d.x : copysignf(ooeps, d.x)),
                 1.0f / (fabsf(d.y) > ooeps ? d.y : copysignf(ooeps, d.y)),
                 1.0f / (fabsf(d.z) > ooeps ? d.z : copysignf(ooeps, d.z)));
    r.oidir = mk3(o.x * r.idir.x, o.y * r.idir.y, o.z * r.idir.z);
}

// Two-level traversal of the moving instances (TLAS, then each hit
// instance's two-wide BLAS) as ONE loop: an iteration is a TLAS node step, a
// BLAS node step or one pending leaf triangle, whatever the lane is at, so
// lanes that entered different instances at different TLAS steps still
// advance together (with the BLAS loop nested in the TLAS loop, a warp ran
// the BLAS loop once for every group of lanes that reached a TLAS leaf
// together).  A TLAS step records its hit leaf children (one instance record
// each) as pending; they are entered before the next TLAS step, the TLAS node
// in hand waiting on the stack.  BLAS nodes are stacked above `base`, the
// TLAS stack height when the instance was entered.  kAny: any hit in
// (tmin, tmax]; else closest hit into h.  Returns whether an occluder was found
// (kAny).
template <bool kAny>
__device__ __forceinline__ bool two_level(const DevScene& sc, const DevFrame& fr, f3 o, f3 d, float tmin,
                                          float tmax, Hit& h, int* stack, int* err, int3& work) {
    WRay r;
    slab_ray(r, o, d);
    bool in_blas = false;
    int sp = 0, base = 0, node = 0;
    int pfirst = 0, pcount = 0;
    int pend0 = -1, pend1 = -1;
    int rec = -1, inst = -1;
    while (true) {
        if (pcount > 0) {
            const float4* tp = sc.tris + 3 * pfirst;
            const float4 p0 = __ldg(tp), p1 = __ldg(tp + 1), p2 = __ldg(tp + 2);
            work.y += 1;
            const float t = tri_hit(r, p0, p1, p2, tmin, kAny ? tmax : h.t);
            if (kAny) {
                if (t >= 0.0f) return true;
            } else {
                const int oi = inst >= 0 ? inst : __float_as_int(p2.w);
                if (t >= 0.0f && better_hit(t, oi, __float_as_int(p0.w), h)) {
                    h.t = t; h.inst = oi; h.tri = pfirst; h.prim = __float_as_int(p0.w); h.rec = rec;
                }
            }
            ++pfirst;
            --pcount;
            continue;
        }
        if (!in_blas && pend0 >= 0) {
            if (node != MCEV_NO_NODE) {
                if (sp < MCEV_STACK) stack[SIDX(sp++)] = node;
                else *err = 1;
            }
            rec = pend0;
            pend0 = pend1;
            pend1 = -1;
            r = object_ray(fr, rec, o, d, node, inst);
            in_blas = true;
            base = sp;
        }
        if (node == MCEV_NO_NODE) {
            if (in_blas && sp == base) {
                // instance done: back to the TLAS
                in_blas = false;
                slab_ray(r, o, d);
                if (pend0 >= 0) continue;
            }
            if (sp == 0) break;
            node = stack[SIDX(--sp)];
        }
        const Node n = load_node(in_blas ? sc.nodes : fr.tlas, node);
        work.x += 1;
        float tl, tr;
        const float tcut = kAny ? tmax : h.t;
        const int m = node_hits(r, n, tmin, tcut, tl, tr);
        const bool lh = (m & 1) && n.d.x < 0, rh = (m & 2) && n.d.y < 0;
        if (in_blas) {
            pfirst = lh ? ~n.d.x : ~n.d.y;
            pcount = (lh ? n.d.z : 0) + (rh ? n.d.w : 0);
        } else {
            pend0 = lh ? ~n.d.x : (rh ? ~n.d.y : -1);
            pend1 = (lh && rh) ? ~n.d.y : -1;
        }
        const bool gl = (m & 1) && n.d.x >= 0 && (kAny || tl <= h.t);
        const bool gr = (m & 2) && n.d.y >= 0 && (kAny || tr <= h.t);
        int next = MCEV_NO_NODE;
        if (gl && gr) {
            // nearer child first (any-hit: in BLAS only, as blas_any does)
            const bool lfirst = kAny ? (!(MCEV_ANY_ORDERED && in_blas) || tl <= tr) : tl <= tr;
            if (sp < MCEV_STACK) stack[SIDX(sp++)] = lfirst ? n.d.y : n.d.x;
            else *err = 1;
            next = lfirst ? n.d.x : n.d.y;
        } else if (gl) {
            next = n.d.x;
        } else if (gr) {
            next = n.d.y;
        }
        node = next;
    }
    return false;
}

// world-space closest hit over the two-level hierarchy (the TLAS is two-wide;
// BLAS in the scene's layout): the merged never-moving geometry first, then
// the TLAS of the moving instances, whose boxes the hit found so far culls.
// work: (node fetches, triangle tests, box tests of the wide layout)
template <bool kWide, bool kTlas>
__device__ __forceinline__ Hit closest_hit(const DevScene& sc, const DevFrame& fr, f3 o, f3 d, float tmin, int* err,
                                           int3& work) {
    Hit h;
    h.t = __int_as_float(0x7f800000);
    h.inst = -1;
    h.tri = -1;
    h.prim = -1;
    h.rec = -1;
    MCEV_DECLARE_STACK(stack);
    MCEV_DECLARE_WSTACK(wstack);
    if (fr.static_rec >= 0) {
        int root, oi;
        const WRay r = object_ray(fr, fr.static_rec, o, d, root, oi);
        blas_closest_any_layout<kWide>(sc, root, fr.static_rec, oi, r, tmin, h, stack, 0, wstack, err, work);
    }
    if (fr.n_tlas == 0) return h;
    if (!kTlas || fr.n_tlas == 1) {
        // (kTlas = false is launched only for frames with at most one moving instance)
        int root, oi;
        const WRay r = object_ray(fr, 0, o, d, root, oi);
        blas_closest_any_layout<kWide>(sc, root, 0, oi, r, tmin, h, stack, 0, wstack, err, work);
        return h;
    }
    if (!kWide) {
        two_level<false>(sc, fr, o, d, tmin, 0.0f, h, stack, err, work);
        return h;
    }
    // wide BLAS: the TLAS loop with each instance's traversal nested in it
    const WRay wr = make_wray(o, d);
    int sp = 0;
    int node = 0;
    while (true) {
        const Node n = load_node(fr.tlas, node);
        work.x += 1;
        if (kWide) work.z += 2;
        float tl, tr;
        const int m = node_hits(wr, n, tmin, h.t, tl, tr);
        for (int side = 0; side < 2; ++side) {
            const int child = side ? n.d.y : n.d.x;
            const int cnt = side ? n.d.w : n.d.z;
            if ((m & (1 << side)) && child < 0) {
                for (int i = 0; i < cnt; ++i) {
                    const int rec = ~child + i;
                    int root, oi;
                    const WRay r = object_ray(fr, rec, o, d, root, oi);
                    blas_closest_any_layout<kWide>(sc, root, rec, oi, r, tmin, h, stack, sp, wstack, err, work);
                }
            }
        }
        const bool gl = (m & 1) && n.d.x >= 0 && tl <= h.t;
        const bool gr = (m & 2) && n.d.y >= 0 && tr <= h.t;
        int next = -0x7fffffff;
        if (gl && gr) {
            const int nearc = tl <= tr ? n.d.x : n.d.y;
            const int farc = tl <= tr ? n.d.y : n.d.x;
            if (sp < MCEV_STACK) stack[SIDX(sp++)] = farc;
            else *err = 1;
            next = nearc;
        } else if (gl) {
            next = n.d.x;
        } else if (gr) {
            next = n.d.y;
        }
        if (next == -0x7fffffff) {
            if (sp == 0) break;
            next = stack[SIDX(--sp)];
        }
        node = next;
    }
    return h;
}

template <bool kWide, bool kTlas>
__device__ __forceinline__ bool occluded(const DevScene& sc, const DevFrame& fr, f3 o, f3 d, float tmin, float tmax,
                                         int* err, int3& work) {
    MCEV_DECLARE_STACK(stack);
    MCEV_DECLARE_WSTACK(wstack);
    if (fr.static_rec >= 0) {
        int root, oi;
        const WRay r = object_ray(fr, fr.static_rec, o, d, root, oi);
        if (blas_any_layout<kWide>(sc, root, r, tmin, tmax, stack, 0, wstack, err, work)) return true;
    }
    if (fr.n_tlas == 0) return false;
    if (!kTlas || fr.n_tlas == 1) {
        int root, oi;
        const WRay r = object_ray(fr, 0, o, d, root, oi);
        return blas_any_layout<kWide>(sc, root, r, tmin, tmax, stack, 0, wstack, err, work);
    }
    if (!kWide) {
        Hit dummy;
        return two_level<true>(sc, fr, o, d, tmin, tmax, dummy, stack, err, work);
    }
    const WRay wr = make_wray(o, d);
    int sp = 0;
    int node = 0;
    while (true) {
        const Node n = load_node(fr.tlas, node);
        work.x += 1;
        if (kWide) work.z += 2;
        float tl, tr;
        const int m = node_hits(wr, n, tmin, tmax, tl, tr);
        for (int side = 0; side < 2; ++side) {
            const int child = side ? n.d.y : n.d.x;
            const int cnt = side ? n.d.w : n.d.z;
            if ((m & (1 << side)) && child < 0) {
                for (int i = 0; i < cnt; ++i) {
                    const int rec = ~child + i;
                    int root, oi;
                    const WRay r = object_ray(fr, rec, o, d, root, oi);
                    if (blas_any_layout<kWide>(sc, root, r, tmin, tmax, stack, sp, wstack, err, work)) return true;
                }
            }
        }
        const bool gl = (m & 1) && n.d.x >= 0;
        const bool gr = (m & 2) && n.d.y >= 0;
        int next = -0x7fffffff;
        if (gl && gr) {
            if (sp < MCEV_STACK) stack[SIDX(sp++)] = n.d.y;
            else *err = 1;
            next = n.d.x;
        } else if (gl) {
            next = n.d.x;
        } else if (gr) {
            next = n.d.y;
        }
        if (next == -0x7fffffff) {
            if (sp == 0) return false;
            next = stack[SIDX(--sp)];
        }
        node = next;
    }
}

// ------------------------------------------------------------------ warp-aggregated append
__device__ __forceinline__ int warp_append(int* counter, bool pred) {
    const unsigned mask = __activemask();
    const unsigned ballot = __ballot_sync(mask, pred);
    if (!pred) return -1;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(ballot) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(ballot));
    base = __shfl_sync(ballot, base, leader);
    return base + __popc(ballot & ((1u << lane) - 1u));
}

}  // namespace mcev
