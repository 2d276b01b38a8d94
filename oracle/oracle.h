/*
 * oracle.h -- plain FP64 CPU restatement of the event renderer of
 * "Monte Carlo Path Tracing and Statistical Event Detection for Event Camera
 * Simulation" (arXiv 2408.07996).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  It
 * shares no code, header, table or helper with the CUDA path, and it is
 * written for a reader checking it against the paper, not for speed.
 *
 * What it computes (paper sections in brackets):
 *   - tracePaths(q, s, N) [Sec. 3, Alg. 1]: N unidirectional path-traced
 *     radiance samples of pixel q at time s (next-event estimation and
 *     power-heuristic MIS, as in pbrt-v4's PathIntegrator [Sec. 3.3]);
 *   - per-path log luminance y = ln(L + eps) [Sec. 3.1, Eq. 3] and its sample
 *     mean and unbiased variance [Eq. 3-4, calcMeanVar of Alg. 1];
 *   - the t-value [Eq. 7] and the one-tailed Student t-test [Sec. 3.2]
 *     with the sampling schedule of Sec. 3.3 (first test at spp_min, then
 *     every spp_batch samples, cap spp_max);
 *   - event emission and reference update [Alg. 1, Eq. 1].
 */
#ifndef MCEV_ORACLE_H
#define MCEV_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------- Philox4x32-10 (Salmon et al., SC'11) ---------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* u = (x >> 8) * 2^-24, exact in FP32 and FP64 */
double orc_u01(uint32_t x);

/* ---------------- Student t distribution ---------------- */
double orc_betainc(double a, double b, double x); /* regularized I_x(a, b) */
double orc_t_cdf(double t, double nu);            /* P(T <= t), nu degrees of freedom */
double orc_t_ppf(double p, double nu);            /* inverse of orc_t_cdf by bisection */

/* ---------------- scene ---------------- */
typedef struct orc_scene orc_scene;

orc_scene* orc_scene_create(
    int64_t n_vertices, const float* vertices,
    int64_t n_triangles, const int32_t* triangles, const int32_t* tri_material,
    int32_t n_meshes, const int32_t* mesh_ranges,
    int32_t n_instances, const int32_t* inst_mesh, const int32_t* inst_material,
    int32_t n_keys, const double* key_times, const double* inst_xform,
    const double* cam_eye, const double* cam_target, const double* cam_up, double fov_deg,
    int32_t n_materials, const int32_t* mat_type, const float* mat_albedo,
    const float* mat_rough, const float* mat_emit,
    int32_t env_w, int32_t env_h, const float* env);
void orc_scene_free(orc_scene* s);

/* Texturing: per-vertex texture coordinates [n_vertices][2], per-material
 * flag (1 = Lambertian albedo from the texture) and an RGB texture
 * [tex_h][tex_w][3]; a textured hit takes the Rec. 709 luminance of the
 * nearest texel at its barycentrically interpolated, wrapped coordinates. */
void orc_scene_set_texture(orc_scene* s, const float* uvs, const int32_t* triangles, const int32_t* mat_textured,
                           int32_t tex_w, int32_t tex_h, const float* texture);
/* Emitted radiance per material replacing the scene's table for the
 * materials the table makes emissive (the emitter set stays fixed). */
void orc_scene_set_emission(orc_scene* s, const float* emission);

/* render settings shared by every oracle entry point */
typedef struct {
    int32_t width, height;
    int32_t max_depth;   /* scattering vertices with NEE + BSDF sampling */
    int32_t nee, mis;    /* next-event estimation on/off; MIS on/off */
    double  eps;         /* y = ln(L + eps) */
    double  t_min;       /* ray epsilon in scene units */
    uint64_t seed;
} orc_params;

/* Closest hit of one world-space ray (tests: BVH vs brute force). */
int orc_closest_hit(const orc_scene* s, double time, const double o[3], const double d[3],
                    double t_min, double t_max, int use_bvh,
                    double* t_out, int32_t* inst_out, int32_t* prim_out);

/* Camera ray through film position (fx_pix, fy_pix) in pixel units (pixel
 * (px, py) with jitter (u0, u1) is at (px + u0, py + u1)). */
void orc_camera_ray(const orc_scene* s, const orc_params* p, double time, double fx_pix,
                    double fy_pix, double o[3], double d[3]);

/* Path-traced radiance of samples k0..k0+count-1 of each listed pixel at
 * `time` (tracePaths).  out_L/out_sig are [n_pix][count]; out_sig is a
 * 32-bit FNV-1a hash of every discrete decision along the path (hit ids,
 * environment texel, emission/NEE/visibility/sampling flags).  Returns the
 * number of non-finite path values that were replaced by 0. */
int64_t orc_trace_samples(const orc_scene* s, const orc_params* p, double time,
                          const int32_t* pixels, int64_t n_pix, int64_t k0, int64_t count,
                          double* out_L, uint32_t* out_sig);

/* Environment sampling / pdf (tests of the importance sampler). */
int orc_env_sample(const orc_scene* s, double u1, double u2, double dir[3], double* pdf, double* Le);
double orc_env_pdf(const orc_scene* s, const double dir[3]);
double orc_env_radiance(const orc_scene* s, const double dir[3]);

/* BSDF (tests): type 0 Lambertian, 1 GGX.  Vectors in a local frame with
 * the normal along +z.  Returns f; writes the pdf of sampling wi. */
double orc_bsdf_eval(int type, double albedo, double rough, const double wo[3],
                     const double wi[3], double* pdf);
void   orc_bsdf_sample(int type, double rough, const double wo[3], double u1, double u2,
                       double wi[3]);

/* ---------------- Algorithm 1 ---------------- */
enum { ORC_ONE_TAILED = 0, ORC_TWO_TAILED = 1, ORC_MEAN_ONLY = 2, ORC_UNIFORM = 3 };
enum { ORC_SE_PAPER = 0, ORC_SE_WELCH = 1 };

typedef struct {
    double C, alpha;
    int32_t spp_min, spp_batch, spp_max;
    int32_t variant, se_mode;
} orc_detect;

/* sample mean and unbiased variance of y[0..n), two passes (Eq. 3-4) */
void orc_mean_var(const double* y, int64_t n, double* mean, double* var);

/* samples k0..k0+count-1 of one pixel as y = ln(L + eps) */
typedef void (*orc_draw_fn)(void* ctx, int64_t k0, int64_t count, double* y);

/* One pixel's frame of Alg. 1 drawing its samples in order from `draw`. */
void orc_detect_pixel_cb(const orc_detect* d, orc_draw_fn draw, void* ctx,
                         int64_t* ref_n, double* ref_mean, double* ref_var,
                         int8_t* event, int32_t* n_used, double* mean, double* var,
                         double* margin_t, double* margin_c);

/* One pixel's frame of Alg. 1 on caller-supplied log-luminance samples
 * y[0..spp_max) (the samples the pixel would draw in order).  ref_* is the
 * reference state (count, mean, unbiased variance); it is updated in place
 * when an event fires.  Outputs: event in {-1,0,+1}, samples used, mean and
 * variance at stop, and the distances of the decisions from their
 * thresholds: min over tests |t - t_crit| and | |mu_b-mu_a| - C |. */
void orc_detect_pixel(const orc_detect* d, const double* y,
                      int64_t* ref_n, double* ref_mean, double* ref_var,
                      int8_t* event, int32_t* n_used, double* mean, double* var,
                      double* margin_t, double* margin_c);

/* Full Alg. 1 frame on path-traced samples for the listed pixels.  When
 * `make_ref` is set the reference state is first computed at t0 with
 * spp_max samples (the first frame of Alg. 1).  All per-pixel arrays are
 * [n_pix].  Returns the number of non-finite path values replaced by 0. */
int64_t orc_render_events(const orc_scene* s, const orc_params* p, const orc_detect* d,
                          double t0, double t1, const int32_t* pixels, int64_t n_pix,
                          int make_ref, int64_t* ref_n, double* ref_mean, double* ref_var,
                          int8_t* events, int32_t* n_used, double* mean, double* var,
                          double* margin_t, double* margin_c);

/* First frame of Alg. 1 for the listed pixels: count, mean and unbiased
 * variance of `spp` log-luminance samples at `time`. */
int64_t orc_reference(const orc_scene* s, const orc_params* p, int32_t spp, double time,
                      const int32_t* pixels, int64_t n_pix,
                      int64_t* ref_n, double* ref_mean, double* ref_var);

#ifdef __cplusplus
}
#endif
#endif
