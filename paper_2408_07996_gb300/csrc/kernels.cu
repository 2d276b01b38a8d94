// kernels.cu -- wavefront path tracer and statistical event detector.
//
// One chunk of paths goes through
//   raygen -> [extend -> shade(+NEE) -> shadow] x (max_depth + 1) -> stats
// where extend/shade/shadow consume device-side ray queues (sizes in device
// counters, no host round trip) and `stats` fuses, per queued pixel, the
// log-luminance batch statistics (Sec. 3.1, Eq. 3-4), the Chan merge into the
// running statistics, the t-test of Eq. 7 (Sec. 3.2), the re-queue of
// undecided pixels (Sec. 3.3; one atomic per warp, since a warp owns a pixel)
// and the event rule with the reference update (Alg. 1, Eq. 1).  Rays and
// shadow rays are appended to their queues with warp-aggregated atomics.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/mcev.h"
#include "device.cuh"
#include "kernels.h"
#include "tdist.h"

namespace mcev {

// Minimum resident blocks per SM requested for the traversal kernels: 9
// blocks of 128 threads cap them at 56 registers (56% occupancy); traversal
// waits on node fetches, so more resident warps pay more than the few
// registers spilled (terrain frame traversal: 72 registers 1011 ms, 64
// registers 967 ms, 56 registers 943 ms, 48 registers 961 ms; whole terrain
// frames with the kernels that carry no TLAS code: 64 / 56 / 48 registers
// 1332 / 1289 / 1306 ms).  0 leaves the choice to the compiler.
#ifndef MCEV_TRAV_MINB
#define MCEV_TRAV_MINB 9
#endif
// The wide-node traversal keeps a whole node (five 16-byte words) and its
// eight child tests in flight: it gets its own cap.
#ifndef MCEV_WIDE_MINB
#define MCEV_WIDE_MINB 8
#endif
#define MCEV_TRAV_BOUNDS __launch_bounds__(MCEV_TRAV_BLOCK, kWide ? MCEV_WIDE_MINB : MCEV_TRAV_MINB)

static constexpr uint32_t NO_FLAGS = 0xFFFFFFFFu;

// shadow-ray count of the bounce whose ray queue is `cur` (double-buffered so
// a launch can trace one bounce's shadow rays while the next bounce's shade
// appends to the other slot)
__device__ __forceinline__ int sh_slot(int cur) { return cur ? 19 : 2; }
static constexpr uint32_t FNV_BASIS = 2166136261u;

// ------------------------------------------------------------------ raygen
// kBatch: queue entries are (job << 24 | pixel) and every path reads its
// job's frame and settings from the job table; otherwise entries are pixels
// of the single context whose frame and settings are kernel arguments.  A
// ray's `w` lane carries its bounce depth | job << 8.
template <bool kBatch>
__global__ void __launch_bounds__(256) k_raygen(DevFrame fr, DevParams P, Wave w, const int32_t* __restrict__ queue,
                                                int64_t j0, int32_t spp_r, int64_t k_base, int64_t n_paths, int cur,
                                                const Job* __restrict__ jobs, const RoundCtl* __restrict__ rc) {
    if (rc) {
        // sizes of the current chunk of the device-resident round loop
        queue = rc->queue[rc->qi];
        j0 = rc->j0;
        spp_r = rc->spp_r;
        k_base = rc->n_done;
        n_paths = rc->nj * (int64_t)rc->spp_r;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        w.counters[cur] = (int32_t)n_paths;
        w.counters[1 - cur] = 0;
        w.counters[2] = w.counters[19] = 0;
    }
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_paths; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = p / spp_r;
        const int32_t s = (int32_t)(p - j * spp_r);
        const int32_t entry = __ldg(queue + j0 + j);
        const int job = kBatch ? (int)((uint32_t)entry >> 24) : 0;
        const int32_t pix = kBatch ? (entry & 0xFFFFFF) : entry;
        const DevFrame& F = kBatch ? jobs[job].fr : fr;
        const DevParams& Q = kBatch ? jobs[job].P : P;
        const uint32_t k = (uint32_t)(k_base + s);
        const uint4 x = philox4x32_10(make_uint4((uint32_t)pix, k, 0u, 0u), F.key0, F.key1);
        const int px = pix % Q.width, py = pix / Q.width;
        const float fx = 2.0f * ((float)px + u01(x.x)) / (float)Q.width - 1.0f;
        const float fy = 1.0f - 2.0f * ((float)py + u01(x.y)) / (float)Q.height;
        const f3 d = norm3(mk3(F.fwd[0] + fx * F.right[0] + fy * F.up[0],
                               F.fwd[1] + fx * F.right[1] + fy * F.up[1],
                               F.fwd[2] + fx * F.right[2] + fy * F.up[2]));
        w.ray_o[cur][p] = make_float4(F.eye[0], F.eye[1], F.eye[2], __int_as_float((int)p));
        w.ray_d[cur][p] = make_float4(d.x, d.y, d.z, __int_as_float(job << 8));
        w.L[p] = 0.0f;
        if (kBatch) w.pix_k[p] = make_int2(entry, (int)k);   // the shadow kernel's job lookup
        w.ray_s[cur][p] = make_float4(1.0f, 0.0f, __int_as_float(entry), __int_as_float((int)k));
        if (Q.adjoint && Q.grad_mean) {
            // d loss / d L of this path: d loss / d mean * d mean / d ln(L + eps) * d ln(L + eps) / dL
            const float Lt = w.Ltot[p];
            w.delta[p] = isfinite(Lt) ? __ldg(Q.grad_mean + pix) / ((float)Q.spp * (Lt + Q.eps)) : 0.0f;
        }
        if (Q.want_sig) {
            w.sig[p] = FNV_BASIS;
            w.pflags[p] = NO_FLAGS;
        }
    }
}

// traversal work counters: 64-bit (nodes, tris) pairs after the int32
// counters, and the ray/box tests (two per node fetch of the two-wide BVH)
enum { WORK_CLOSEST = 0, WORK_SHADOW = 1 };
// Per-block accumulation of the traversal work counters: work_begin at the
// top of a ray loop (every thread of the block), add_work after it.  Each
// warp adds its sums in shared memory; the last warp of the block to finish
// adds the block's totals to the global counters (skipped when the block
// traced nothing), so a launch's global atomics on these three words scale
// with its busy blocks, not with its warps, and no warp waits for another.
struct WorkAcc {
    unsigned long long v[3];
    unsigned int done;
};

__device__ __forceinline__ WorkAcc& work_acc() {
    __shared__ WorkAcc acc;
    return acc;
}

__device__ __forceinline__ void work_begin() {
    WorkAcc& a = work_acc();
    if (threadIdx.x == 0) {
        a.v[0] = a.v[1] = a.v[2] = 0ull;
        a.done = 0u;
    }
    __syncthreads();
}

template <bool kWide>
__device__ __forceinline__ void add_work(const Wave& w, int which, int3 work) {
    WorkAcc& a = work_acc();
    // the whole warp, reconverged after its ray loop: one count per warp
    __syncwarp();
    const unsigned m = 0xffffffffu;
    const int nodes = __reduce_add_sync(m, work.x);
    const int tris = __reduce_add_sync(m, work.y);
    const int boxes = kWide ? __reduce_add_sync(m, work.z) : 2 * nodes;
    if ((threadIdx.x & 31) == 0) {
        if (nodes | tris) {
            atomicAdd(&a.v[0], (unsigned long long)nodes);
            atomicAdd(&a.v[1], (unsigned long long)tris);
            atomicAdd(&a.v[2], (unsigned long long)boxes);
        }
        __threadfence_block();
        if (atomicAdd(&a.done, 1u) == (blockDim.x >> 5) - 1u) {
            __threadfence_block();
            const unsigned long long n0 = atomicAdd(&a.v[0], 0ull), n1 = atomicAdd(&a.v[1], 0ull),
                                     n2 = atomicAdd(&a.v[2], 0ull);
            if (n0 | n1) {
                unsigned long long* c = reinterpret_cast<unsigned long long*>(w.counters + 32);
                atomicAdd(c + 2 * which, n0);
                atomicAdd(c + 2 * which + 1, n1);
                atomicAdd(c + 7 + which, n2);
            }
        }
    }
}

// ------------------------------------------------------------------ extend
// Closest hits of the rays of queue `cur`, indices first, first + stride, ...
// The first thread also clears the queue and shadow counters shade(cur) will
// append to.
template <bool kBatch, bool kWide, bool kTlas>
__device__ __forceinline__ void extend_rays(const DevScene& sc, const DevFrame& fr, float t_min, const Wave& w,
                                            int cur, int32_t* err, const Job* __restrict__ jobs, int64_t first,
                                            int64_t stride) {
    const int32_t n = *(volatile int32_t*)(w.counters + cur);
    if (first == 0) {
        w.counters[1 - cur] = 0;
        w.counters[sh_slot(cur)] = 0;
        atomicAdd(reinterpret_cast<unsigned long long*>(w.counters + 32) + 4, (unsigned long long)n);
    }
    int e = 0;
    int3 work = make_int3(0, 0, 0);
    work_begin();
    for (int64_t i = first; i < n; i += stride) {
        const float4 o = w.ray_o[cur][i];
        const float4 d = w.ray_d[cur][i];
        const int job = kBatch ? (__float_as_int(d.w) >> 8) : 0;
        const DevScene& S = kBatch ? jobs[job].sc : sc;
        const DevFrame& F = kBatch ? jobs[job].fr : fr;
        const float tmin = kBatch ? jobs[job].P.t_min : t_min;
        const Hit h = closest_hit<kWide, kTlas>(S, F, xyz(o), xyz(d), tmin, &e, work);
        w.hit[i] = make_float4(h.t, __int_as_float(h.inst), __int_as_float(h.tri), __int_as_float(h.rec));
    }
    if (e) atomicOr(err, 1);
    add_work<kWide>(w, WORK_CLOSEST, work);
}

template <bool kBatch, bool kWide, bool kTlas>
__global__ void MCEV_TRAV_BOUNDS k_extend(DevScene sc, DevFrame fr, float t_min, Wave w, int cur, int32_t* err,
                                          const Job* __restrict__ jobs) {
    extend_rays<kBatch, kWide, kTlas>(sc, fr, t_min, w, cur, err, jobs, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                               (int64_t)gridDim.x * blockDim.x);
}

// ------------------------------------------------------------------ shade + NEE + BSDF sampling
// shade is latency bound on per-path gathers: 64 registers (8 blocks/SM)
// measured 15% faster than the unconstrained 80-register build
#ifndef MCEV_SHADE_MINB
#define MCEV_SHADE_MINB 8
#endif
#if MCEV_SHADE_MINB > 0
#define MCEV_SHADE_BOUNDS __launch_bounds__(128, MCEV_SHADE_MINB)
#else
#define MCEV_SHADE_BOUNDS __launch_bounds__(128)
#endif
template <bool kBatch>
__global__ void MCEV_SHADE_BOUNDS k_shade(DevScene sc, DevFrame fr, DevParams P, Wave w, int cur,
                                          const Job* __restrict__ jobs) {
    const int32_t n = *(volatile int32_t*)(w.counters + cur);
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 ro = w.ray_o[cur][i];
        const float4 rd = w.ray_d[cur][i];
        const int p = __float_as_int(ro.w);
        const int depth = __float_as_int(rd.w) & 0xFF;
        const int job = kBatch ? (__float_as_int(rd.w) >> 8) : 0;
        const DevScene& S = kBatch ? jobs[job].sc : sc;
        const DevFrame& F = kBatch ? jobs[job].fr : fr;
        const DevParams& Q = kBatch ? jobs[job].P : P;
        const float4 hv = w.hit[i];
        const int inst = __float_as_int(hv.y);
        const float4 rs = w.ray_s[cur][i];
        float beta = rs.x;
        // radiance this vertex adds to the path (emission on a hit, the
        // environment on a miss); the path's total is updated only when
        // something is added
        float Ladd = 0.0f;
        const float pdf_prev = rs.y;
        float pdf_next = 0.0f;
        uint32_t sig = 0, pflags = NO_FLAGS;
        if (Q.want_sig) {
            sig = w.sig[p];
            const uint32_t pf = w.pflags[p];
            if (pf != NO_FLAGS) sig = fnv(sig, pf);
        }
        const f3 d = xyz(rd);
        bool cont = false, shadow = false;
        f3 P0 = mk3(0, 0, 0), wi_next = mk3(0, 0, 0), sh_dir = mk3(0, 0, 0);
        float sh_tmax = 0.0f, sh_c = 0.0f, sh_g = 0.0f;
        int sh_m = -1;
        if (inst < 0) {
            // miss: environment radiance (Sec. 3.1 samples the light reaching the pixel)
            if (Q.want_sig) sig = fnv(sig, 0xFFFFFFFFu);
            if (S.has_env) {
                int row, col;
                float st;
                env_texel(S, d, row, col, st);
                if (Q.want_sig) sig = fnv(sig, (uint32_t)(row * S.env_w + col));
                const float Le = __ldg(S.env + (int64_t)row * S.env_w + col);
                float wgt = 1.0f;
                if (depth > 0 && Q.nee) wgt = Q.mis ? power_heuristic(pdf_prev, F.p_env * texel_pdf(S, row, col, st)) : 0.0f;
                Ladd = beta * wgt * Le;
            } else if (Q.want_sig) {
                sig = fnv(sig, 0xFFFFFFFEu);
            }
        } else {
            const int tri = __float_as_int(hv.z);
            // the shading record (edge cross product, material) serves most
            // hits; the vertices are read only for textured albedo, emitter
            // MIS weights and the decision signature
            const float4 tsh = __ldg(S.tshade + tri);
            const float4* tp = S.tris + 3 * tri;
            const float4* ip = F.inst + 7 * __float_as_int(hv.w);
            const float4 i0 = __ldg(ip + 3), i1 = __ldg(ip + 4), i2 = __ldg(ip + 5);
            const int ovr = __float_as_int(__ldg(ip + 6).y);
            if (Q.want_sig) {
                sig = fnv(sig, (uint32_t)inst);
                sig = fnv(sig, (uint32_t)__float_as_int(__ldg(tp).w));
            }
            const float t = hv.x;
            P0 = xyz(ro) + d * t;
            const f3 ng = norm3(xf_normal(i0, i1, i2, xyz(tsh)));
            const f3 wo = d * -1.0f;
            const int mat = ovr >= 0 ? ovr : __float_as_int(tsh.w);
            const float4 mv = __ldg(S.mats + mat);
            const int tword = __float_as_int(mv.x);
            const int type = tword & 0xFF;
            float alb = mv.y;
            const float rough = mv.z;
            // the override applies to the scene's emitters only (NEE samples that fixed set)
            const float emit = (S.emit && mv.w > 0.0f) ? __ldg(S.emit + mat) : mv.w;
            int texel = -1;
            if ((tword & MAT_TEXTURED) && S.tex && S.tri_uv) {
                // albedo = luminance of the nearest texel at the hit's texture coordinates
                const float4 q0 = __ldg(tp), q1 = __ldg(tp + 1), q2 = __ldg(tp + 2);
                float b1, b2;
                barycentric(xf_point(i0, i1, i2, P0), xyz(q0), xyz(q1), xyz(q2), b1, b2);
                const float b0 = 1.0f - b1 - b2;
                const float2 t0 = __ldg(S.tri_uv + 3 * tri), t1 = __ldg(S.tri_uv + 3 * tri + 1),
                             t2 = __ldg(S.tri_uv + 3 * tri + 2);
                texel = texel_of(S, b0 * t0.x + b1 * t1.x + b2 * t2.x, b0 * t0.y + b1 * t1.y + b2 * t2.y);
                const float* rgb = S.tex + 3 * (int64_t)texel;
                alb = MCEV_Y_R * __ldg(rgb) + MCEV_Y_G * __ldg(rgb + 1) + MCEV_Y_B * __ldg(rgb + 2);
                if (Q.want_sig) sig = fnv(sig, (uint32_t)texel);
            }
            const float dlt = Q.adjoint ? w.delta[p] : 0.0f;
            uint32_t flags = 0;
            const float cos_o = dot3(ng, wo);
            if (emit > 0.0f && cos_o > 0.0f) {
                flags |= 1u;
                float wgt = 1.0f;
                if (depth > 0 && Q.nee) {
                    if (!Q.mis) {
                        wgt = 0.0f;
                    } else {
                        const float4 q0 = __ldg(tp), q1 = __ldg(tp + 1), q2 = __ldg(tp + 2);
                        const float4 m0 = __ldg(ip), m1 = __ldg(ip + 1), m2 = __ldg(ip + 2);
                        const f3 e1 = xyz(q1) - xyz(q0), e2 = xyz(q2) - xyz(q0);
                        const f3 we1 = xf_vec(m0, m1, m2, e1), we2 = xf_vec(m0, m1, m2, e2);
                        const f3 wc = cross3(we1, we2);
                        const float area = 0.5f * sqrtf(dot3(wc, wc));
                        const float pl = F.p_area / ((float)F.n_lights * area) * t * t / cos_o;
                        wgt = power_heuristic(pdf_prev, pl);
                    }
                }
                Ladd = beta * wgt * emit;
                if (Q.adjoint && Q.grad_emit) atomicAdd(Q.grad_emit + mat, (double)(dlt * beta * wgt));
            }
            if (depth < Q.max_depth && alb > 0.0f) {
                // adjoint: every contribution after this vertex carries one factor of its albedo
                if (Q.adjoint && texel >= 0 && Q.grad_tex && dlt != 0.0f) {
                    const float g = dlt * (w.Ltot[p] - (w.L[p] + Ladd)) / alb;
                    float* gt = Q.grad_tex + 3 * (int64_t)texel;
                    atomicAdd(gt, g * MCEV_Y_R);
                    atomicAdd(gt + 1, g * MCEV_Y_G);
                    atomicAdd(gt + 2, g * MCEV_Y_B);
                }
                const f3 nn = cos_o < 0.0f ? ng * -1.0f : ng;
                f3 tb, bt;
                onb(nn, tb, bt);
                const f3 wol = mk3(dot3(wo, tb), dot3(wo, bt), dot3(wo, nn));
                const uint32_t ent = (uint32_t)__float_as_int(rs.z);
                const uint2 pk = make_uint2(kBatch ? (ent & 0xFFFFFFu) : ent, (uint32_t)__float_as_int(rs.w));
                // next-event estimation
                if (Q.nee && (S.env_ok || F.n_lights > 0)) {
                    const uint4 x = philox4x32_10(make_uint4(pk.x, pk.y, (uint32_t)(depth + 1), 0u), F.key0, F.key1);
                    const bool use_env = S.env_ok && (F.n_lights == 0 || u01(x.x) < 0.5f);
                    f3 wi = mk3(0, 0, 0);
                    float pl = 0.0f, Le = 0.0f, tmax = __int_as_float(0x7f800000);
                    int lmat = -1;
                    if (use_env) {
                        float pdf;
                        wi = env_sample(S, u01(x.z), u01(x.w), pdf, Le);
                        pl = F.p_env * pdf;
                    } else {
                        const uint64_t mm = (uint64_t)(x.y >> 8);
                        const int li = (int)((mm * (uint64_t)F.n_lights) >> 24);
                        const float4* lp = F.lights + 4 * li;
                        const float4 a0 = __ldg(lp), a1 = __ldg(lp + 1), a2 = __ldg(lp + 2), an = __ldg(lp + 3);
                        const float su = sqrtf(u01(x.z));
                        const float b0 = 1.0f - su, b1 = u01(x.w) * su, b2 = 1.0f - b0 - b1;
                        const f3 Ql = xyz(a0) * b0 + xyz(a1) * b1 + xyz(a2) * b2;
                        const f3 dv = Ql - P0;
                        const float dist = sqrtf(dot3(dv, dv));
                        wi = dv * (1.0f / dist);
                        const float cl = -dot3(xyz(an), wi);
                        if (cl > 0.0f) {
                            pl = F.p_area / ((float)F.n_lights * a1.w) * dist * dist / cl;
                            lmat = __float_as_int(a2.w);
                            Le = S.emit ? __ldg(S.emit + lmat) : a0.w;
                        }
                        tmax = dist - Q.t_min;
                    }
                    if (pl > 0.0f && Le > 0.0f) {
                        const f3 wil = mk3(dot3(wi, tb), dot3(wi, bt), dot3(wi, nn));
                        float pb;
                        const float f = bsdf_eval(type, alb, rough, wol, wil, &pb);
                        if (f > 0.0f && wil.z > 0.0f) {
                            flags |= 2u;
                            const float wgt = Q.mis ? power_heuristic(pl, pb) : 1.0f;
                            sh_c = beta * f * wil.z * Le * wgt / pl;
                            sh_g = beta * f * wil.z * wgt / pl;
                            sh_m = lmat;
                            sh_dir = wi;
                            sh_tmax = tmax;
                            shadow = true;
                        }
                    }
                }
                // BSDF sampling of the continuation
                const uint4 y = philox4x32_10(make_uint4(pk.x, pk.y, (uint32_t)(depth + 1), 1u), F.key0, F.key1);
                const f3 wil = bsdf_sample(type, rough, wol, u01(y.x), u01(y.y));
                float pb;
                const float f = bsdf_eval(type, alb, rough, wol, wil, &pb);
                if (f > 0.0f && pb > 0.0f && wil.z > 0.0f) {
                    flags |= 8u;
                    beta *= f * wil.z / pb;
                    pdf_next = pb;
                    wi_next = norm3(tb * wil.x + bt * wil.y + nn * wil.z);
                    cont = true;
                }
            }
            pflags = flags;
        }
        if (Ladd != 0.0f) w.L[p] += Ladd;
        if (Q.want_sig) {
            w.sig[p] = sig;
            w.pflags[p] = pflags;
        }
        const int si = warp_append(w.counters + sh_slot(cur), shadow);
        if (shadow) {
            w.sh_o[si] = make_float4(P0.x, P0.y, P0.z, __int_as_float(p));
            w.sh_d[si] = make_float4(sh_dir.x, sh_dir.y, sh_dir.z, sh_tmax);
            w.sh_c[si] = sh_c;
            if (Q.adjoint) {
                w.sh_g[si] = sh_g;
                w.sh_m[si] = sh_m;
            }
        }
        const int ni = warp_append(w.counters + (1 - cur), cont);
        if (cont) {
            w.ray_o[1 - cur][ni] = make_float4(P0.x, P0.y, P0.z, __int_as_float(p));
            w.ray_d[1 - cur][ni] = make_float4(wi_next.x, wi_next.y, wi_next.z, __int_as_float((depth + 1) | (job << 8)));
            w.ray_s[1 - cur][ni] = make_float4(beta, pdf_next, rs.z, rs.w);
        }
    }
}

// ------------------------------------------------------------------ shadow rays
// the light sample of shadow ray i reaches path p: add its contribution
__device__ __forceinline__ void shadow_unoccluded(const Wave& w, const DevParams& Q, int i, int p) {
    w.L[p] += w.sh_c[i];
    if (Q.want_sig) w.pflags[p] |= 4u;
    if (Q.adjoint && Q.grad_emit && w.sh_m[i] >= 0) atomicAdd(Q.grad_emit + w.sh_m[i], (double)(w.delta[p] * w.sh_g[i]));
}

// Shadow rays appended by shade(cur), indices first, first + stride, ...
template <bool kBatch, bool kWide, bool kTlas>
__device__ __forceinline__ void shadow_rays(const DevScene& sc, const DevFrame& fr, const DevParams& P,
                                            const Wave& w, int cur, int32_t* err, const Job* __restrict__ jobs,
                                            int64_t first, int64_t stride) {
    const int32_t n = *(volatile int32_t*)(w.counters + sh_slot(cur));
    if (first == 0) atomicAdd(reinterpret_cast<unsigned long long*>(w.counters + 32) + 5, (unsigned long long)n);
    int e = 0;
    int3 work = make_int3(0, 0, 0);
    work_begin();
    for (int64_t i = first; i < n; i += stride) {
        const float4 o = w.sh_o[i];
        const float4 d = w.sh_d[i];
        const int p = __float_as_int(o.w);
        const int job = kBatch ? (int)((uint32_t)w.pix_k[p].x >> 24) : 0;
        const DevScene& S = kBatch ? jobs[job].sc : sc;
        const DevFrame& F = kBatch ? jobs[job].fr : fr;
        const DevParams& Q = kBatch ? jobs[job].P : P;
        if (!occluded<kWide, kTlas>(S, F, xyz(o), xyz(d), Q.t_min, d.w, &e, work)) shadow_unoccluded(w, Q, (int)i, p);
    }
    if (e) atomicOr(err, 1);
    add_work<kWide>(w, WORK_SHADOW, work);
}

template <bool kBatch, bool kWide, bool kTlas>
__global__ void MCEV_TRAV_BOUNDS k_shadow(DevScene sc, DevFrame fr, DevParams P, Wave w, int cur, int32_t* err,
                                          const Job* __restrict__ jobs) {
    shadow_rays<kBatch, kWide, kTlas>(sc, fr, P, w, cur, err, jobs, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                               (int64_t)gridDim.x * blockDim.x);
}

// One launch for the shadow rays of bounce d (appended by shade with queue
// `cur`) and the closest hits of bounce d + 1 (queue 1 - cur): the first
// `g_ext` blocks extend, the rest trace shadow rays.  Two independent traversal
// workloads in one grid keep the SMs busy while the other's longest rays finish.
template <bool kBatch, bool kWide, bool kTlas>
__global__ void MCEV_TRAV_BOUNDS k_shadow_extend(DevScene sc, DevFrame fr, DevParams P, Wave w, int cur,
                                                 int32_t g_ext, int32_t* err, const Job* __restrict__ jobs) {
    if ((int32_t)blockIdx.x < g_ext)
        extend_rays<kBatch, kWide, kTlas>(sc, fr, P.t_min, w, 1 - cur, err, jobs,
                                   blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)g_ext * blockDim.x);
    else
        shadow_rays<kBatch, kWide, kTlas>(sc, fr, P, w, cur, err, jobs,
                                   (blockIdx.x - g_ext) * (int64_t)blockDim.x + threadIdx.x,
                                   (int64_t)(gridDim.x - g_ext) * blockDim.x);
}

// ------------------------------------------------------------------ per-pixel statistics + test + requeue + events
struct Moments {
    float n, mean, m2;
};
__device__ __forceinline__ Moments chan(Moments a, Moments b) {
    const float n = a.n + b.n;
    if (n == 0.0f) return a;
    const float dl = b.mean - a.mean;
    Moments r;
    r.n = n;
    r.mean = a.mean + dl * (b.n / n);
    r.m2 = a.m2 + b.m2 + dl * dl * (a.n * b.n / n);
    return r;
}

// kChecked: caller-supplied pixel ids and counts are range-checked (the
// allocation-free entry point); the renderer's own queues use <false>.
// log of a path value: the fast hardware logarithm by default (its error,
// ~1e-7 absolute near 1, is far below the statistics' own noise)
#ifndef MCEV_FAST_LOG
#define MCEV_FAST_LOG 1
#endif
#if MCEV_FAST_LOG
#define MCEV_LOG(x) __logf(x)
#else
#define MCEV_LOG(x) logf(x)
#endif

template <bool kChecked, bool kBatch>
__global__ void __launch_bounds__(256) k_stats(Wave w, StatsArgs A0, const int32_t* __restrict__ queue, int64_t j0,
                                               int64_t n_pix, int32_t* __restrict__ next_queue,
                                               const Job* __restrict__ jobs, const RoundCtl* __restrict__ rc) {
    if (rc) {
        // sizes of the current chunk of the device-resident round loop
        queue = rc->queue[rc->qi];
        next_queue = rc->queue[rc->qi ^ 1];
        j0 = rc->j0;
        n_pix = rc->nj;
        A0.spp_r = rc->spp_r;
        A0.sub = rc->sub;
        A0.k_base = rc->n_done;
    }
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = warp0; j < n_pix; j += nwarps) {
        const int32_t entry = __ldg(queue + j0 + j);
        const int32_t pix = kBatch ? (entry & 0xFFFFFF) : entry;
        // per-pixel state and outputs of the pixel's job
        StatsArgs A = A0;
        if (kBatch) {
            const Job& J = jobs[(uint32_t)entry >> 24];
            A.cur = J.cur;
            A.ref = J.ref;
            A.events = J.events;
            A.spp_out = J.spp_out;
            A.mean_out = J.mean_out;
            A.eps = J.P.eps;
        }
        if (kChecked && (pix < 0 || (int64_t)pix >= A.n_total)) {
            if (lane == 0) atomicOr(w.counters + 8, 1);
            continue;
        }
        // The round traced spp_r samples of this pixel: one batch, or a window
        // of several spp_batch-sized batches.  Each batch is merged and tested
        // in order exactly as Alg. 1 would; once the pixel is decided, the
        // rest of the window is left unused.  Every lane computes the same
        // statistics (butterfly merges in a fixed order), so the decisions
        // are warp-uniform.
        Moments c{0.0f, 0.0f, 0.0f};
        if (A.k_base > 0) c = Moments{(float)A.cur.n[pix], A.cur.mean[pix], A.cur.m2[pix]};
        const bool detect = A.mode == MODE_DETECT;
        const float ma = detect ? A.ref.mean[pix] : 0.0f;
        const int32_t na = detect ? A.ref.n[pix] : 0;
        const float va = (detect && na > 1) ? A.ref.m2[pix] / (float)(na - 1) : 0.0f;
        int bad = 0;
        bool decided = false;
        int32_t n = (int32_t)c.n;
        const float* Lp = w.L + j * A.spp_r;
        for (int s0 = 0; s0 < A.spp_r && !decided; s0 += A.sub) {
            const int s1 = min(s0 + A.sub, A.spp_r);
            // moments of this batch from sums shifted by one warp-uniform value
            // (the running mean, or the batch's first sample for a pixel's
            // first batch), so lanes merge by plain addition: the butterfly
            // below adds a + b on one lane and b + a on its partner, which
            // are the same bits, so every lane ends with identical sums
            float sh;
            if (c.n > 0.0f) {
                sh = c.mean;
            } else {
                const float L0 = Lp[s0];
                sh = MCEV_LOG((isfinite(L0) ? L0 : 0.0f) + A.eps);
            }
            float s1d = 0.0f, s2d = 0.0f;
            int cnt = 0;
            for (int s = s0 + lane; s < s1; s += 32) {
                float Lv = Lp[s];
                if (!isfinite(Lv)) {
                    Lv = 0.0f;
                    ++bad;
                }
                const float d = MCEV_LOG(Lv + A.eps) - sh;
                s1d += d;
                s2d = fmaf(d, d, s2d);
                ++cnt;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                s1d += __shfl_xor_sync(0xffffffffu, s1d, off);
                s2d += __shfl_xor_sync(0xffffffffu, s2d, off);
                cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
            }
            Moments m{0.0f, 0.0f, 0.0f};
            if (cnt > 0) {
                const float fn = (float)cnt;
                const float md = s1d / fn;
                m = Moments{fn, sh + md, fmaxf(s2d - s1d * md, 0.0f)};
            }
            c = (A.k_base == 0 && s0 == 0) ? m : chan(c, m);
            n = (int32_t)c.n;
            if (!detect) continue;
            decided = n >= A.spp_max;
            if (!decided && A.variant != VAR_UNIFORM) {
                const float gap = fabsf(c.mean - ma);
                if (A.variant == VAR_MEAN_ONLY) {
                    decided = gap < A.C;
                } else {
                    const float vb = c.m2 / (float)(n - 1);
                    const float se2 = A.se_mode == SE_WELCH ? va / (float)na + vb / (float)n : (va + vb) / (float)n;
                    if (se2 == 0.0f) {
                        decided = gap < A.C;
                    } else if (kChecked && n < A.spp_min) {
                        decided = false;
                    } else {
                        const float t = (gap - A.C) / sqrtf(se2);
                        int r = (n - A.spp_min) / A.spp_batch;
                        if (kChecked) r = min(r, (A.spp_max - A.spp_min + A.spp_batch - 1) / A.spp_batch - 1);
                        const float tc = __ldg(A.tcrit + r);
                        decided = A.variant == VAR_TWO_TAILED ? (t < tc || t > -tc) : (t < tc);
                    }
                }
            }
        }
        bad = __reduce_add_sync(0xffffffffu, bad);
        if (lane != 0) continue;
        if (bad) atomicAdd(w.counters + 4, bad);
        A.cur.n[pix] = n;
        A.cur.mean[pix] = c.mean;
        A.cur.m2[pix] = c.m2;
        if (!detect) {
            if (n >= A.spp_max && A.mode == MODE_MEAN) {
                A.mean_out[pix] = c.mean;
                if (A.spp_out) A.spp_out[pix] = n;
            } else if (n >= A.spp_max) {
                A.ref.n[pix] = n;
                A.ref.mean[pix] = c.mean;
                A.ref.m2[pix] = c.m2;
            } else {
                next_queue[atomicAdd(w.counters + 3, 1)] = entry;
            }
            continue;
        }
        if (!decided) {
            next_queue[atomicAdd(w.counters + 3, 1)] = entry;
            continue;
        }
        const float delta = c.mean - ma;
        int8_t ev = 0;
        if (fabsf(delta) > A.C) {
            ev = delta > 0.0f ? 1 : -1;
            A.ref.n[pix] = n;
            A.ref.mean[pix] = c.mean;
            A.ref.m2[pix] = c.m2;
            atomicAdd(w.counters + (ev > 0 ? 5 : 6), 1);
        }
        if (n >= A.spp_max) atomicAdd(w.counters + 7, 1);
        atomicAdd(reinterpret_cast<unsigned long long*>(w.counters + 32) + 6, (unsigned long long)n);
        A.events[pix] = ev;
        if (A.spp_out) A.spp_out[pix] = n;
        if (A.mean_out) A.mean_out[pix] = c.mean;
    }
}

// ------------------------------------------------------------------ tracePaths output
__global__ void k_write_samples(Wave w, int64_t out0, int64_t n_paths, float* __restrict__ L_out,
                                uint32_t* __restrict__ sig_out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_paths; p += (int64_t)gridDim.x * blockDim.x) {
        L_out[out0 + p] = w.L[p];
        if (sig_out) {
            uint32_t s = w.sig[p];
            const uint32_t pf = w.pflags[p];
            if (pf != NO_FLAGS) s = fnv(s, pf);
            sig_out[out0 + p] = s;
        }
    }
}

__global__ void k_iota(int32_t* q, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        q[i] = (int32_t)i;
}

// ------------------------------------------------------------------ launchers
// Traversal grids: up to 72 blocks of 128 threads per SM (8 waves of the 9
// resident blocks), each thread striding over the ray queue.  Per-ray
// traversal cost is heavy-tailed, and smaller per-block shares let the block
// scheduler even out the SMs' ends (terrain frame: 16 / 36 / 72 / 144 blocks
// per SM 1286 / 1245 / 1239 / 1261 ms; one ray per thread with no cap
// 1992 ms, the empty blocks of late, small rounds costing more).
#ifndef MCEV_TRAV_BLOCKS_PER_SM
#define MCEV_TRAV_BLOCKS_PER_SM 72
#endif

static int grid_for(int64_t work, int block, int sms, int per_sm) {
    int64_t g = (work + block - 1) / block;
    const int64_t cap = (int64_t)sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

cudaError_t launch_raygen(const DevFrame& fr, const DevParams& P, const Wave& w, const int32_t* queue, int64_t j0,
                          int32_t spp_r, int64_t k_base, int64_t n_paths, int cur, int sms, cudaStream_t st,
                          const Job* jobs, const RoundCtl* rc) {
    // with rc, n_paths is the wavefront capacity (the chunk's size is on the device)
    if (jobs)
        k_raygen<true><<<grid_for(n_paths, 256, sms, 16), 256, 0, st>>>(fr, P, w, queue, j0, spp_r, k_base, n_paths,
                                                                          cur, jobs, rc);
    else
        k_raygen<false><<<grid_for(n_paths, 256, sms, 16), 256, 0, st>>>(fr, P, w, queue, j0, spp_r, k_base, n_paths,
                                                                           cur, nullptr, rc);
    return cudaGetLastError();
}

// traversal launches: kBatch x kWide instantiations picked at run time
// traversal kernels by (batched jobs, BLAS layout, moving instances under a TLAS)
#define MCEV_TRAV_LAUNCH3(kernel, kb, grid, jobs_, ...)                                                   \
    do {                                                                                                  \
        if (trav & TRAV_WIDE) {                                                                           \
            if (trav & TRAV_TLAS) kernel<kb, true, true><<<grid, MCEV_TRAV_BLOCK, 0, st>>>(__VA_ARGS__, jobs_); \
            else kernel<kb, true, false><<<grid, MCEV_TRAV_BLOCK, 0, st>>>(__VA_ARGS__, jobs_);          \
        } else {                                                                                          \
            if (trav & TRAV_TLAS) kernel<kb, false, true><<<grid, MCEV_TRAV_BLOCK, 0, st>>>(__VA_ARGS__, jobs_); \
            else kernel<kb, false, false><<<grid, MCEV_TRAV_BLOCK, 0, st>>>(__VA_ARGS__, jobs_);         \
        }                                                                                                 \
    } while (0)
#define MCEV_TRAV_DISPATCH(kernel, grid, ...)                                                             \
    do {                                                                                                  \
        if (jobs) MCEV_TRAV_LAUNCH3(kernel, true, grid, jobs, __VA_ARGS__);                               \
        else MCEV_TRAV_LAUNCH3(kernel, false, grid, nullptr, __VA_ARGS__);                                \
    } while (0)

cudaError_t launch_extend(const DevScene& sc, const DevFrame& fr, float t_min, const Wave& w, int cur, int64_t max_n,
                          int32_t* err, int sms, cudaStream_t st, const Job* jobs, int trav) {
    MCEV_TRAV_DISPATCH(k_extend, grid_for(max_n, MCEV_TRAV_BLOCK, sms, MCEV_TRAV_BLOCKS_PER_SM), sc, fr, t_min, w, cur,
                       err);
    return cudaGetLastError();
}

cudaError_t launch_shade(const DevScene& sc, const DevFrame& fr, const DevParams& P, const Wave& w, int cur,
                         int64_t max_n, int sms, cudaStream_t st, const Job* jobs) {
    if (jobs)
        k_shade<true><<<grid_for(max_n, 128, sms, 16), 128, 0, st>>>(sc, fr, P, w, cur, jobs);
    else
        k_shade<false><<<grid_for(max_n, 128, sms, 16), 128, 0, st>>>(sc, fr, P, w, cur, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_shadow(const DevScene& sc, const DevFrame& fr, const DevParams& P, const Wave& w, int cur,
                          int64_t max_n, int32_t* err, int sms, cudaStream_t st, const Job* jobs, int trav) {
    MCEV_TRAV_DISPATCH(k_shadow, grid_for(max_n, MCEV_TRAV_BLOCK, sms, MCEV_TRAV_BLOCKS_PER_SM), sc, fr, P, w, cur,
                       err);
    return cudaGetLastError();
}

cudaError_t launch_shadow_extend(const DevScene& sc, const DevFrame& fr, const DevParams& P, const Wave& w, int cur,
                                 int64_t max_n, int32_t* err, int sms, cudaStream_t st, const Job* jobs, int trav) {
    const int g = grid_for(max_n, MCEV_TRAV_BLOCK, sms, MCEV_TRAV_BLOCKS_PER_SM);
    MCEV_TRAV_DISPATCH(k_shadow_extend, 2 * g, sc, fr, P, w, cur, g, err);
    return cudaGetLastError();
}

cudaError_t launch_stats(const Wave& w, const StatsArgs& A, const int32_t* queue, int64_t j0, int64_t n_pix,
                         int32_t* next_queue, int sms, cudaStream_t st, const Job* jobs, const RoundCtl* rc) {
    // with rc, n_pix is an upper bound of the chunk's pixels (the size is on the device)
    if (jobs)
        k_stats<false, true><<<grid_for(n_pix * 32, 256, sms, 8), 256, 0, st>>>(w, A, queue, j0, n_pix, next_queue,
                                                                                 jobs, rc);
    else
        k_stats<false, false><<<grid_for(n_pix * 32, 256, sms, 8), 256, 0, st>>>(w, A, queue, j0, n_pix, next_queue,
                                                                                  nullptr, rc);
    return cudaGetLastError();
}

static cudaError_t launch_stats_checked(const Wave& w, const StatsArgs& A, const int32_t* queue, int64_t n_pix,
                                        int32_t* next_queue, int sms, cudaStream_t st) {
    k_stats<true, false><<<grid_for(n_pix * 32, 256, sms, 8), 256, 0, st>>>(w, A, queue, 0, n_pix, next_queue,
                                                                             nullptr, nullptr);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ device-resident round loop
// The rounds of Alg. 1's sampling schedule (Sec. 3.3) without the host: a
// CUDA graph runs k_round_init, then a conditional WHILE node whose body is
// one wavefront chunk (raygen, bounces, statistics) followed by
// k_round_next, which moves to the next chunk of the round or, at the end
// of a round, reads the number of re-queued pixels and sizes the next round
// (first round spp_min samples, then windows of spp_batch batches that fill
// the wavefront), and clears the condition when no pixel is left.  The loop
// is bounded: after plan.max_iters chunks, or plan.timeout_ns of wall clock
// (%globaltimer), it stops with RC_TIMEOUT, which the host reports as
// MCEV_ERR_TIMEOUT.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void round_first_chunk(RoundCtl* rc, const RoundPlan& plan) {
    rc->per_chunk = max((int64_t)1, plan.cap / rc->spp_r);
    rc->j0 = 0;
    rc->nj = min(rc->per_chunk, rc->Q);
}

__global__ void k_round_init(RoundCtl* rc, Wave w, RoundPlan plan, int32_t* q0, int32_t* q1, int iota) {
    if (iota)
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < plan.Q0; i += (int64_t)gridDim.x * blockDim.x)
            q0[i] = (int32_t)i;
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    rc->queue[0] = q0;
    rc->queue[1] = q1;
    rc->Q = plan.Q0;
    rc->n_done = 0;
    rc->paths = 0;
    rc->stats_pix = 0;
    rc->qi = 0;
    rc->rounds = 0;
    rc->iters = 0;
    rc->status = RC_OK;
    rc->spp_r = rc->sub = min(plan.spp_min, plan.spp_max);
    round_first_chunk(rc, plan);
    w.counters[3] = 0;
    rc->t_start = global_ns();
}

__global__ void k_round_next(RoundCtl* rc, Wave w, RoundPlan plan, cudaGraphConditionalHandle h) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    rc->iters += 1;
    rc->stats_pix += rc->nj;
    unsigned int go = 1;
    if (rc->iters >= plan.max_iters || global_ns() - rc->t_start > plan.timeout_ns) {
        rc->status = RC_TIMEOUT;
        go = 0;
    } else if (rc->j0 + rc->per_chunk < rc->Q) {
        rc->j0 += rc->per_chunk;
        rc->nj = min(rc->per_chunk, rc->Q - rc->j0);
    } else {
        // the round is done: its undecided pixels form the next round
        rc->paths += rc->Q * (int64_t)rc->spp_r;
        rc->n_done += rc->spp_r;
        rc->rounds += 1;
        const int32_t q = *(volatile int32_t*)(w.counters + 3);
        w.counters[3] = 0;
        rc->qi ^= 1;
        rc->Q = q;
        if (q == 0) {
            go = 0;
        } else if (rc->n_done >= plan.spp_max) {
            rc->status = RC_CAP;
            go = 0;
        } else {
            const int64_t sub = plan.spp_batch;
            const int64_t left = (plan.spp_max - rc->n_done + sub - 1) / sub;
            int64_t m = max((int64_t)1, plan.cap / max((int64_t)1, (int64_t)q * sub));
            m = min(min(m, left), (int64_t)plan.window_max);
            rc->sub = (int32_t)sub;
            rc->spp_r = (int32_t)min(m * sub, (int64_t)plan.spp_max - rc->n_done);
            round_first_chunk(rc, plan);
        }
    }
    cudaGraphSetConditional(h, go);
}

cudaError_t launch_round_init(RoundCtl* rc, const Wave& w, const RoundPlan& plan, int32_t* q0, int32_t* q1,
                              bool iota, int sms, cudaStream_t st) {
    k_round_init<<<iota ? grid_for(plan.Q0, 256, sms, 8) : 1, 256, 0, st>>>(rc, w, plan, q0, q1, iota ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_round_next(RoundCtl* rc, const Wave& w, const RoundPlan& plan, cudaGraphConditionalHandle h,
                              cudaStream_t st) {
    k_round_next<<<1, 32, 0, st>>>(rc, w, plan, h);
    return cudaGetLastError();
}

// out[i] += (float)acc[i]
__global__ void k_add_f64(float* __restrict__ out, const double* __restrict__ acc, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] += (float)acc[i];
}

cudaError_t launch_add_f64(float* out, const double* acc, int n, cudaStream_t st) {
    k_add_f64<<<(n + 255) / 256, 256, 0, st>>>(out, acc, n);
    return cudaGetLastError();
}

// queue entries (job << 24 | pixel) of one job
__global__ void k_fill_entries(int32_t* q, int64_t n, int job) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        q[i] = (int32_t)(((uint32_t)job << 24) | (uint32_t)i);
}

cudaError_t launch_fill_entries(int32_t* q, int64_t n, int job, int sms, cudaStream_t st) {
    k_fill_entries<<<grid_for(n, 256, sms, 8), 256, 0, st>>>(q, n, job);
    return cudaGetLastError();
}

cudaError_t launch_write_samples(const Wave& w, int64_t out0, int64_t n_paths, float* L_out, uint32_t* sig_out,
                                 int sms, cudaStream_t st) {
    k_write_samples<<<grid_for(n_paths, 256, sms, 8), 256, 0, st>>>(w, out0, n_paths, L_out, sig_out);
    return cudaGetLastError();
}

cudaError_t launch_iota(int32_t* q, int64_t n, int sms, cudaStream_t st) {
    k_iota<<<grid_for(n, 256, sms, 8), 256, 0, st>>>(q, n);
    return cudaGetLastError();
}

}  // namespace mcev

// ------------------------------------------------------------------ allocation-free detector step
// Scratch of mcev_detect_batch_static: int32 counters [0, 256) in the layout
// of Wave::counters (layout.h lists every slot; k_stats uses [3]-[8] and the
// uint64 word [32 + 6]) followed by the critical-t table.  It lives in the
// library image so the call never allocates; host code reaches it only
// through the address cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_detect_scratch[MCEV_DETECT_STATIC_SCRATCH_BYTES];

namespace {

struct StaticDevice {
    void* scratch = nullptr;
    int sms = 0;
    bool ready = false;
};
constexpr int kMaxDevices = 64;
StaticDevice g_static_dev[kMaxDevices];
std::mutex g_static_mu;

mcev_status static_fail(const mcev_detect_args* a, mcev_status s, const char* msg) {
    if (a && a->err_msg && a->err_len > 0) {
        size_t i = 0;
        for (; msg[i] && i + 1 < a->err_len; ++i) a->err_msg[i] = msg[i];
        a->err_msg[i] = 0;
    }
    return s;
}

}  // namespace

extern "C" mcev_status mcev_detect_batch_static(const mcev_detect_args* a, int64_t* n_undecided) {
    using namespace mcev;
    if (!a || !n_undecided) return MCEV_ERR_ARG;
    if (!a->L || !a->pixels || !a->cur_n || !a->cur_mean || !a->cur_m2 || !a->ref_n || !a->ref_mean ||
        !a->ref_m2 || !a->events || !a->undecided)
        return static_fail(a, MCEV_ERR_ARG, "mcev_detect_batch_static: a required pointer is NULL");
    if (a->n_pix < 0 || a->n_total < 1 || a->spp_r < 1 || a->k_base < 0 || a->reserved0 != 0 || a->spp_min < 2 ||
        a->spp_batch < 1 || a->spp_max < a->spp_min || a->k_base + a->spp_r > a->spp_max ||
        (a->k_base == 0 && a->spp_r != a->spp_min) || !(a->eps > 0.0f) || !(a->C >= 0.0f) ||
        !(a->alpha > 0.0f && a->alpha < 1.0f) || a->variant < 0 || a->variant > 3 || a->se_mode < 0 ||
        a->se_mode > 1 || (int64_t)a->n_pix * a->spp_r > ((int64_t)1 << 40))
        return static_fail(a, MCEV_ERR_ARG, "mcev_detect_batch_static: inconsistent sizes or settings");
    // Later calls must start on the test schedule spp_min + r * spp_batch and
    // cover whole batches (only the last batch of the frame may be shorter, as
    // it ends at spp_max), so that the kernel tests at every schedule point the
    // window crosses and each test reads the critical value of its own count.
    if (a->k_base > 0 && (a->k_base < a->spp_min || (a->k_base - a->spp_min) % a->spp_batch != 0 ||
                          (a->spp_r % a->spp_batch != 0 && a->k_base + a->spp_r != a->spp_max)))
        return static_fail(a, MCEV_ERR_ARG,
                           "mcev_detect_batch_static: call off the test schedule: k_base must be spp_min + r * "
                           "spp_batch and spp_r a multiple of spp_batch (or end at spp_max)");
    const int64_t n_tests = (a->spp_max - a->spp_min + a->spp_batch - 1) / a->spp_batch;
    if (n_tests > MCEV_DETECT_STATIC_MAX_TESTS)
        return static_fail(a, MCEV_ERR_ARG,
                           "mcev_detect_batch_static: the schedule needs more than 4096 t-tests; the fixed "
                           "scratch holds 4096 critical values (raise spp_batch or lower spp_max)");
    *n_undecided = 0;
    if (a->n_pix == 0) return MCEV_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return static_fail(a, MCEV_ERR_CUDA, "mcev_detect_batch_static: no usable current CUDA device");
    }
    StaticDevice sd;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        StaticDevice& s = g_static_dev[dev];
        if (!s.ready) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_detect_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return static_fail(a, MCEV_ERR_CUDA, "mcev_detect_batch_static: cudaGetSymbolAddress failed");
            }
            int sms = 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                return static_fail(a, MCEV_ERR_CUDA, "mcev_detect_batch_static: device query failed");
            }
            s.scratch = p;
            s.sms = sms;
            s.ready = true;
        }
        sd = s;
    }
    cudaStream_t st = (cudaStream_t)a->stream;
    int32_t* counters = (int32_t*)sd.scratch;
    float* tcrit = (float*)((unsigned char*)sd.scratch + 256);
    float tab[MCEV_DETECT_STATIC_MAX_TESTS];
    int nt = 0;
    if (a->variant == VAR_ONE_TAILED || a->variant == VAR_TWO_TAILED) {
        const double p = a->variant == VAR_TWO_TAILED ? 0.5 * (double)a->alpha : (double)a->alpha;
        for (int n = a->spp_min; n < a->spp_max; n += a->spp_batch) tab[nt++] = (float)t_quantile_int(p, n - 1);
    }
    if (cudaMemsetAsync(counters, 0, 256, st) != cudaSuccess ||
        (nt > 0 && cudaMemcpyAsync(tcrit, tab, sizeof(float) * nt, cudaMemcpyHostToDevice, st) != cudaSuccess)) {
        cudaGetLastError();
        return static_fail(a, MCEV_ERR_CUDA, "mcev_detect_batch_static: scratch initialisation failed");
    }
    Wave w{};
    w.L = const_cast<float*>(a->L);
    w.counters = counters;
    StatsArgs A{};
    A.cur = PixStats{a->cur_n, a->cur_mean, a->cur_m2};
    A.ref = PixStats{a->ref_n, a->ref_mean, a->ref_m2};
    A.tcrit = tcrit;
    A.events = a->events;
    A.spp_out = a->spp_out;
    A.mean_out = a->mean_out;
    A.eps = a->eps;
    A.C = a->C;
    A.spp_r = a->spp_r;
    // the first call is the first batch (spp_min samples, one test at its
    // end); a later call's samples are merged and tested one spp_batch at a time
    A.sub = a->k_base == 0 ? a->spp_r : a->spp_batch;
    A.k_base = a->k_base;
    A.spp_min = a->spp_min;
    A.spp_batch = a->spp_batch;
    A.spp_max = a->spp_max;
    A.mode = MODE_DETECT;
    A.variant = a->variant;
    A.se_mode = a->se_mode;
    A.n_total = a->n_total;
    if (launch_stats_checked(w, A, a->pixels, a->n_pix, a->undecided, sd.sms, st) != cudaSuccess)
        return static_fail(a, MCEV_ERR_CUDA, "mcev_detect_batch_static: kernel launch failed");
    int32_t c[16];
    if (cudaMemcpyAsync(c, counters, sizeof c, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return static_fail(a, MCEV_ERR_CUDA, "mcev_detect_batch_static: kernel or copy failed");
    }
    *n_undecided = c[3];
    if (c[8])
        return static_fail(a, MCEV_ERR_ARG,
                           "mcev_detect_batch_static: a pixel id was outside [0, n_total); those pixels were skipped");
    return MCEV_OK;
}
