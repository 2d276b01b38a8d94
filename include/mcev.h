/*
 * mcev.h -- C ABI of the GB300 event-camera renderer.
 *
 * The library renders events the way "Monte Carlo Path Tracing and
 * Statistical Event Detection for Event Camera Simulation" (arXiv 2408.07996)
 * describes: per pixel it path-traces log luminance samples at two times,
 * keeps their running mean and variance, runs a one-tailed Student t-test of
 * whether the log-brightness gap is below the event threshold (Sec. 3.2,
 * Eq. 7), re-queues only the undecided pixels for another batch of paths
 * (Sec. 3.3) and emits an event with its polarity where the gap exceeds the
 * threshold (Alg. 1, Eq. 1).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an mcev_status and never aborts or throws.  On an
 *    error the message is available from mcev_last_error(ctx).
 *  - "device" pointers are CUDA device pointers on the context's device;
 *    "host" pointers are ordinary host memory.  Caller-owned buffers stay
 *    owned by the caller; the library copies what it needs.
 *  - All GPU work runs on the context's stream (mcev_set_stream; default:
 *    the legacy default stream).  Calls are stream-ordered; a call that
 *    returns host results synchronises the stream first.
 *  - Pixels are indexed p = y * width + x, with y = 0 the top image row.
 *  - Not thread-safe per context: one host thread drives a context at a time.
 */
#ifndef MCEV_H
#define MCEV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcev_ctx mcev_ctx;

typedef enum {
    MCEV_OK = 0,
    MCEV_ERR_ARG = -1,      /* invalid argument (null, out of range, wrong size) */
    MCEV_ERR_CUDA = -2,     /* a CUDA runtime call failed; see mcev_last_error */
    MCEV_ERR_OOM = -3,      /* device or host allocation failed */
    MCEV_ERR_TIMEOUT = -4,  /* the device-resident round loop hit its bound (mcev_params.device_timeout_us,
                               or more chunks than the sampling schedule can need); the frame is incomplete */
    MCEV_ERR_STATE = -5,    /* call out of order (e.g. render before scene upload) */
    MCEV_ERR_NUMERIC = -6   /* reserved for numeric failures surfaced as errors */
} mcev_status;

/* Detector variants (Sec. 3.2 and its discussion; Sec. 4 baseline). */
enum {
    MCEV_ONE_TAILED = 0,    /* the paper's method: stop iff F_{n-1}(t) < alpha */
    MCEV_TWO_TAILED = 1,    /* ablation: stop iff either tail is below alpha/2 */
    MCEV_MEAN_ONLY = 2,     /* ablation: stop iff |mu_b - mu_a| < C */
    MCEV_UNIFORM = 3        /* baseline: every pixel to spp_max, same event rule */
};
/* Standard error of Eq. 7: the paper's sqrt((s_a^2 + s_b^2) / n_b), or Welch's
 * sqrt(s_a^2 / n_a + s_b^2 / n_b). */
enum { MCEV_SE_PAPER = 0, MCEV_SE_WELCH = 1 };

/* Scene description; every pointer is HOST memory and is copied.
 * Triangles index a shared vertex pool; a mesh is a contiguous triangle
 * range; an instance places a mesh with a row-major 3x4 object-to-world
 * affine matrix per keyframe (linearly interpolated between keyframes,
 * clamped outside).  Materials: type 0 Lambertian (albedo), 1 GGX
 * reflector (albedo = Schlick normal-incidence reflectance, rough = GGX
 * alpha).  emit > 0 makes a triangle a one-sided emitter on the side of its
 * winding normal (v1-v0)x(v2-v0); such triangles are also sampled by NEE.
 * env: [env_h][env_w] latitude-longitude scalar radiance, row 0 at +y,
 * azimuth measured from +x towards +z; NULL for a black background. */
typedef struct {
    int64_t n_vertices;
    const float* vertices;       /* [n_vertices][3] */
    int64_t n_triangles;
    const int32_t* triangles;    /* [n_triangles][3] vertex indices */
    const int32_t* tri_material; /* [n_triangles] */
    int32_t n_meshes;
    const int32_t* mesh_ranges;  /* [n_meshes][2] = (first triangle, count) */
    int32_t n_instances;
    const int32_t* inst_mesh;     /* [n_instances] */
    const int32_t* inst_material; /* [n_instances] override material id, or -1 */
    int32_t n_keys;
    const double* key_times;      /* [n_keys], strictly increasing */
    const double* inst_xform;     /* [n_keys][n_instances][12] */
    const double* cam_eye;        /* [n_keys][3] */
    const double* cam_target;     /* [n_keys][3] */
    const double* cam_up;         /* [n_keys][3] */
    double fov_deg;               /* full field of view across the shorter image axis */
    int32_t n_materials;
    const int32_t* mat_type;      /* [n_materials] */
    const float* mat_albedo;      /* [n_materials] */
    const float* mat_rough;       /* [n_materials] */
    const float* mat_emit;        /* [n_materials] */
    int32_t env_w, env_h;
    const float* env;             /* [env_h][env_w] or NULL */
    const float* uvs;             /* [n_vertices][2] texture coordinates, or NULL */
    const int32_t* mat_textured;  /* [n_materials]: 1 = Lambertian albedo read from the texture set by
                                     mcev_set_texture (luminance of the nearest texel), or NULL */
} mcev_scene_desc;

/* Render settings (mcev_set_params). */
typedef struct {
    float eps;          /* dark level: each path contributes y = ln(L + eps) (Sec. 3.1) */
    float t_min;        /* ray epsilon in scene units (self-intersection offset) */
    int32_t max_depth;  /* scattering vertices with NEE + BSDF sampling (pbrt-v4 maxdepth) */
    int32_t nee;        /* 1: next-event estimation at every vertex */
    int32_t mis;        /* 1: power-heuristic MIS between NEE and BSDF sampling */
    int32_t spp_min;    /* samples before the first t-test (Sec. 3.3: 256); >= 2 */
    int32_t variant;    /* MCEV_ONE_TAILED ... MCEV_UNIFORM */
    int32_t se_mode;    /* MCEV_SE_PAPER or MCEV_SE_WELCH */
    uint64_t seed;      /* Philox key seed */
    int64_t wavefront;  /* max paths in flight per chunk (1024..2^30); 0 = library default (2^25).
                           A chunk holds all of a pixel's samples of one round, so calls
                           whose per-pixel sample count (spp_max, count, spp) exceeds it
                           fail with MCEV_ERR_ARG */
    int32_t profile;    /* 1: time every kernel launch with CUDA events (mcev_stats.kernel_ms) */
    int32_t batch_window; /* after the first batch, a round may trace up to this many batches of
                             spp_batch per undecided pixel at once (as many as fill the wavefront),
                             merging and testing them in order; samples after a pixel's decision
                             are unused.  1 = one batch per round; 0 = library default (16). */
    int32_t bvh_width;  /* node layout of the per-mesh BVHs: 2 (two children per node) or 8
                           (compressed 8-wide nodes with 8-bit child boxes); 0 = library default.
                           Changing it rebuilds the BVHs of an uploaded scene.  Results are the
                           same up to rare FP32 box-culling decisions near a ray's origin. */
    int32_t host_rounds;/* 0 (default): the rounds of a frame run on the device as one CUDA graph
                           (a conditional loop: trace a chunk, merge and test, size the next chunk
                           or round), with no host round trip until the frame is done; 1: the
                           host drives the rounds, reading the number of undecided pixels back
                           after each.  profile = 1 implies host-driven rounds (per-launch timing).
                           Both give identical results. */
    int32_t device_timeout_us; /* wall-clock bound of the device-resident loop in microseconds
                           (0 = library default, 300 s); past it the loop stops after its current
                           chunk and the call returns MCEV_ERR_TIMEOUT */
} mcev_params;

/* kernel classes reported in mcev_stats.  MCEV_K_EXTEND counts the traversal
 * launches: closest hits, and the shadow rays a bounce traces in the same
 * launch as the next bounce's closest hits (MCEV_K_SHADOW then stays 0). */
enum { MCEV_K_RAYGEN = 0, MCEV_K_EXTEND = 1, MCEV_K_SHADE = 2, MCEV_K_SHADOW = 3, MCEV_K_STATS = 4,
       MCEV_K_CLASSES = 5 };

/* Per-call counters (mcev_render_events, optional). */
typedef struct {
    int64_t paths;          /* path samples traced for the t1 frame */
    int64_t samples_used;   /* samples that entered the decisions (sum of per-pixel counts) */
    int64_t ref_paths;      /* path samples traced for a t0 reference frame (0 if reused) */
    int32_t rounds;         /* batch rounds at t1 */
    int32_t kernel_launches;/* kernels launched by this call */
    int64_t events_pos, events_neg;
    int64_t pixels_at_cap;  /* pixels that used spp_max samples */
    int64_t nonfinite;      /* path values that were not finite and counted as 0 */
    double gpu_ms;          /* device time of the call (CUDA events) */
    /* traversal work: BVH nodes fetched and ray/triangle tests, for
     * closest-hit and for shadow (any-hit) rays (ray/box tests below) */
    int64_t nodes_closest, tris_closest, nodes_shadow, tris_shadow;
    int64_t rays_closest, rays_shadow;
    /* per kernel class (MCEV_K_*): launches, and summed device time in ms
     * when mcev_params.profile = 1 (else 0) */
    int32_t kernel_count[MCEV_K_CLASSES];
    int32_t reserved;
    double kernel_ms[MCEV_K_CLASSES];
    int64_t h2d_bytes, d2h_bytes;   /* host<->device copies made by the call */
    int64_t stats_pixels;   /* pixel visits of the statistics kernel (sum over its launches) */
    int64_t boxes_closest, boxes_shadow;  /* ray/box slab tests of the traversals (a two-wide node
                                             fetch tests 2 boxes, a wide node one per child) */
} mcev_stats;

/* Creates a context on CUDA device `device` for width x height images.
 * *out receives the context (NULL on failure).  Errors: ARG, CUDA, OOM.
 * No paper passage: infrastructure. */
mcev_status mcev_create(mcev_ctx** out, int device, int32_t width, int32_t height);

/* Frees every resource of the context (NULL is a no-op).
 * No paper passage: infrastructure. */
void mcev_destroy(mcev_ctx* ctx);

/* Last error message of the context ("" when none); valid until the next call.
 * No paper passage: infrastructure. */
const char* mcev_last_error(const mcev_ctx* ctx);

/* Uses `stream` (a cudaStream_t, e.g. torch's current stream) for all later
 * GPU work of this context; NULL selects the legacy default stream.
 * No paper passage: infrastructure. */
mcev_status mcev_set_stream(mcev_ctx* ctx, void* stream);

/* Routes the context's device allocations through alloc/free (e.g. a
 * framework's caching allocator).  alloc returns NULL on failure, which
 * the library reports as MCEV_ERR_OOM.  Must be called before
 * mcev_scene_upload; NULL restores cudaMalloc/cudaFree.
 * No paper passage: infrastructure. */
typedef void* (*mcev_alloc_fn)(size_t bytes, void* user);
typedef void (*mcev_free_fn)(void* ptr, void* user);
mcev_status mcev_set_allocator(mcev_ctx* ctx, mcev_alloc_fn alloc, mcev_free_fn free_fn, void* user);

/* Copies the scene to the device (see mcev_scene_desc) and builds one
 * bounding volume hierarchy per mesh with default settings.  Invalidates
 * the reference state.  Errors: ARG (bad index, size or key order), OOM, CUDA.
 * Paper: the scenes of Sec. 4 (diffuse and glossy surfaces, area lights, an
 * environment map, camera and object motion over time) that the path tracer
 * of Sec. 3.1 / 3.3 renders. */
mcev_status mcev_scene_upload(mcev_ctx* ctx, const mcev_scene_desc* desc);

/* Rebuilds the per-mesh BVHs with a binned surface-area heuristic of
 * `sah_bins` bins (4..256) and leaves of at most `max_leaf` (1..16)
 * triangles.  Errors: ARG, STATE (no scene), OOM, CUDA.
 * No paper passage: the acceleration structure is the renderer's (the
 * paper relies on pbrt-v4's, Sec. 3.3). */
mcev_status mcev_build_bvh(mcev_ctx* ctx, int32_t sah_bins, int32_t max_leaf);

/* Sets render settings (see mcev_params); a new bvh_width rebuilds the BVHs of
 * the uploaded scene.  Errors: ARG (the settings are unchanged), and OOM or
 * CUDA from that rebuild (the scene must then be uploaded again).
 * Paper: eps is the dark level of the log samples (Sec. 3.1), spp_min the
 * first test point (Sec. 3.3), variant and se_mode the test of Sec. 3.2 and
 * its ablations (Table 2); the rest is infrastructure. */
mcev_status mcev_set_params(mcev_ctx* ctx, const mcev_params* params);

/* First frame of Alg. 1: renders every pixel at time t0 with spp samples and
 * stores (count, mean, M2) of ln(L + eps) as the reference state.  Errors:
 * ARG, STATE, OOM, CUDA, TIMEOUT.
 * Paper: Alg. 1 (the reference frame rendered at the full sample count). */
mcev_status mcev_render_reference(mcev_ctx* ctx, double t0, int32_t spp);

/* One frame of Alg. 1 for the pair (t0, t1).  If the reference state is not
 * valid or was last set for a time other than t0, the reference is first
 * rendered at t0 with spp_max samples.  Then every pixel is sampled at t1
 * in a first batch of params.spp_min samples and further batches of
 * spp_batch, the t-test (Eq. 7 with the chosen variant and standard error)
 * deciding after each batch whether the pixel stops, up to spp_max.  A
 * decided pixel with |mean_t1 - mean_ref| > C gets event sign(gap) and its
 * statistics become the new reference (Alg. 1); the reference time becomes t1.
 *   events_out : device int8 [H*W], required: -1, 0, +1 per pixel
 *   spp_out    : device int32 [H*W] or NULL: samples used per pixel
 *   mean_out   : device float [H*W] or NULL: mean ln(L + eps) at t1
 *   stats_out  : host or NULL; filled when non-NULL
 * The call returns when the frame is done.  By default the rounds run on the
 * device (one CUDA graph per call whose loop sizes every round from the
 * number of pixels the previous one re-queued) and the stream is
 * synchronised once at the end; with host_rounds = 1 (or profile = 1) every
 * round reads that number back to the host instead.  If the device loop hits
 * its bound the call returns MCEV_ERR_TIMEOUT: the outputs are incomplete and
 * the reference state is invalidated (the next call renders it again), and
 * the context stays usable.
 * Sample k of pixel p at time t uses the same random numbers in every mode,
 * so adaptive samples are a prefix of the uniform ones.
 * Errors: ARG (C < 0, alpha outside (0,1), spp_batch < 1, spp_max < spp_min,
 * spp_max above the wavefront), STATE, OOM, CUDA, TIMEOUT.
 * Paper: Alg. 1 (one frame of its loop), Sec. 3.1 (log-luminance samples),
 * Sec. 3.2 and Eq. 7 (the t-test), Sec. 3.3 (batches and the cap), Eq. 1
 * (the event rule). */
mcev_status mcev_render_events(mcev_ctx* ctx, double t0, double t1, float C, float alpha,
                               int32_t spp_batch, int32_t spp_max, int8_t* events_out,
                               int32_t* spp_out, float* mean_out, mcev_stats* stats_out);

/* ------------------------------------------------------------------------
 * Differentiable rendering (path-replay adjoint).  The texture and the
 * emission values are caller-owned DEVICE buffers that the library reads at
 * render time (keep them alive and unchanged while a call runs); setting
 * them does not copy.  Gradients cover textured Lambertian albedo and
 * emitted radiance; geometry and visibility are held fixed.
 * ------------------------------------------------------------------------ */

/* RGB albedo texture [height][width][3] (device float) used by textured
 * materials; NULL restores the materials' table albedo.  Errors: ARG.
 * No paper passage: the differentiable-rendering extension. */
mcev_status mcev_set_texture(mcev_ctx* ctx, const float* texture, int32_t width, int32_t height);

/* Emitted radiance per material (device float [n_materials]) overriding the
 * scene's table for the materials that the table makes emissive (value > 0);
 * entries of the other materials are ignored, since the set of emitters that
 * next-event estimation samples is fixed by the scene.  An override <= 0
 * turns that emitter dark.  NULL restores the table.
 * Errors: ARG (n != material count).
 * No paper passage: the differentiable-rendering extension. */
mcev_status mcev_set_emission(mcev_ctx* ctx, const float* emission, int32_t n_materials);

/* Per-pixel mean of ln(L + eps) over samples 0..spp-1 at time t (every
 * pixel the same count; the reference state is not touched).
 *   mean_out: device float [H*W].  Errors: ARG, STATE, OOM, CUDA, TIMEOUT.
 * Paper: the sample mean of log luminance of Sec. 3.1 at a fixed count; its
 * use for gradients is the differentiable-rendering extension. */
mcev_status mcev_render_mean(mcev_ctx* ctx, double t, int32_t spp, float* mean_out);

/* Adjoint of mcev_render_mean (path-replay backpropagation): given
 * grad_mean = d loss / d mean (device float [H*W]), ADDS d loss / d texel
 * RGB to grad_texture (device float [th][tw][3], may be NULL) and
 * d loss / d emitted radiance to grad_emission (device float [n_materials],
 * may be NULL), replaying the same samples with the same random numbers.
 * Errors: ARG, STATE, OOM, CUDA.
 * No paper passage: the differentiable-rendering extension. */
mcev_status mcev_backward(mcev_ctx* ctx, double t, int32_t spp, const float* grad_mean, float* grad_texture,
                          float* grad_emission);

/* One frame pair of a batched render. */
typedef struct {
    mcev_ctx* ctx;          /* scene, camera, image size, settings and reference state of this job */
    double t0, t1;          /* the frame pair, as in mcev_render_events */
    int8_t* events_out;     /* device int8 [H*W] of ctx, required */
    int32_t* spp_out;       /* device int32 [H*W] or NULL */
    float* mean_out;        /* device float [H*W] or NULL */
} mcev_job;

/* Batched Alg. 1 frames: every job's frame pair is rendered exactly as
 * mcev_render_events would render it on its own context (same samples, same
 * decisions, same outputs and reference update), but all jobs' pixels share
 * one queue of undecided pixels, one set of rounds and the same wavefront
 * chunks, so many small frames (different scenes and image sizes) keep the
 * GPU as busy as one large frame.  References missing at t0 are rendered
 * first, also batched.  The runner context (which may also be one of the
 * jobs' contexts) supplies the stream, allocator, wavefront buffers and the
 * reported counters.  All jobs must share spp_min, variant and se_mode (the
 * schedule) and the BVH node layout (bvh_width); every other setting is per job.  Jobs must use distinct
 * contexts on the runner's device, of at most 2^24 pixels each; n_jobs is
 * 1..256.  Errors: ARG, STATE, OOM, CUDA, TIMEOUT.
 * Paper: Alg. 1 per job; sharing rounds across jobs is infrastructure. */
mcev_status mcev_render_events_batch(mcev_ctx* runner, const mcev_job* jobs, int32_t n_jobs, float C, float alpha,
                                     int32_t spp_batch, int32_t spp_max, mcev_stats* stats_out);

/* tracePaths(q, s, N) of Alg. 1: path-traced radiance of samples
 * k0 .. k0+count-1 of each listed pixel at time t.
 *   pixels : device int32 [n_pix], values in [0, H*W) (may be NULL when n_pix = 0)
 *   L_out  : device float [n_pix][count]
 *   sig_out: device uint32 [n_pix][count] or NULL: FNV-1a hash of every
 *            discrete decision along the path (hit instance/triangle ids,
 *            environment texel, emission, NEE, visibility and sampling flags)
 * Errors: ARG, STATE, OOM, CUDA.
 * Paper: tracePaths of Alg. 1; the samples of Sec. 3.1. */
mcev_status mcev_trace_samples(mcev_ctx* ctx, double t, const int32_t* pixels, int64_t n_pix,
                               int64_t k0, int32_t count, float* L_out, uint32_t* sig_out);

/* Size in bytes of the reference-state blob: a 16-byte header (double
 * reference time, int32 valid flag, int32 pixel count) followed by int32
 * n[H*W], float mean[H*W], float M2[H*W].
 * Paper: the reference statistics Alg. 1 carries from frame to frame; the
 * blob format is infrastructure. */
size_t mcev_state_bytes(const mcev_ctx* ctx);

/* Copies the reference state (checkpoint) into a device buffer of
 * mcev_state_bytes() bytes; mcev_set_state restores it (resume).  The state
 * plus the reference time is all Alg. 1 carries between frames.
 * Errors: ARG (NULL or wrong size), CUDA.
 * Paper: Alg. 1 (the reference it keeps); checkpoint and resume are
 * infrastructure. */
mcev_status mcev_get_state(mcev_ctx* ctx, void* dev_buf, size_t bytes);
mcev_status mcev_set_state(mcev_ctx* ctx, const void* dev_buf, size_t bytes);

/* ------------------------------------------------------------------------
 * Allocation-free detector step.  The paper has no counterpart: this is an
 * interface of this library for callers that cannot allocate device memory
 * themselves or let a library do it - for example a renderer embedded in a
 * host application whose memory pool owns the whole GPU, or a real-time loop
 * that must not pay for the device synchronisation cudaMalloc/cudaFree imply.
 * Such a caller brings its own path radiance samples and its own per-pixel
 * state buffers and runs the same fused statistics / t-test / re-queue /
 * event kernel that mcev_render_events uses, one batch per call.
 *
 * Memory: the kernel's scratch (the re-queue counter, event counters and the
 * table of critical t values) is a fixed 16,640-byte array in the library's
 * device image (MCEV_DETECT_STATIC_SCRATCH_BYTES).  Every GPU that loads the
 * library holds it until the process exits.  The call makes no cudaMalloc,
 * cudaFree, allocator-hook or framework allocation.
 *
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call on
 * each device before any stream capture begins.
 *
 * Sharing: every call on a device uses the same array.  Each call clears
 * the counters and rewrites the table before its kernel runs, so nothing
 * carries over between calls, but calls whose GPU work overlaps (different
 * streams, or several host threads) race on the array and must be
 * serialised by the caller.  The call synchronises `stream` to return the
 * number of undecided pixels.
 * ------------------------------------------------------------------------ */
#define MCEV_DETECT_STATIC_MAX_TESTS 4096
#define MCEV_DETECT_STATIC_SCRATCH_BYTES (256 + 4 * MCEV_DETECT_STATIC_MAX_TESTS)

typedef struct {
    const float* L;          /* device [n_pix][spp_r]: radiance of this batch's paths, pixel-major */
    const int32_t* pixels;   /* device [n_pix]: pixel ids indexing the per-pixel arrays below */
    int64_t n_pix;
    int64_t n_total;         /* length of every per-pixel array; ids outside [0, n_total) are skipped
                                and reported as MCEV_ERR_ARG */
    int32_t spp_r;           /* samples per pixel in this batch (>= 1) */
    int32_t reserved0;       /* must be 0 */
    int64_t k_base;          /* samples every listed pixel already has this frame (0: first batch) */
    int32_t* cur_n;          /* device per-pixel running statistics of the frame (in/out) */
    float* cur_mean;
    float* cur_m2;
    int32_t* ref_n;          /* device per-pixel reference statistics (in/out; replaced on an event) */
    float* ref_mean;
    float* ref_m2;
    int8_t* events;          /* device per-pixel event map, written for pixels decided by this call */
    int32_t* spp_out;        /* device per-pixel sample counts of decided pixels, or NULL */
    float* mean_out;         /* device per-pixel mean ln(L + eps) of decided pixels, or NULL */
    int32_t* undecided;      /* device [n_pix] out: pixels that need another batch (any order) */
    float eps, C, alpha;
    int32_t spp_min, spp_batch, spp_max;
    int32_t variant, se_mode;/* as in mcev_params */
    void* stream;            /* cudaStream_t; NULL = legacy default stream */
    char* err_msg;           /* host, optional: receives a message when the call fails */
    size_t err_len;
} mcev_detect_args;

/* Runs the detector on one window of samples without allocating: merges
 * each listed pixel's spp_r samples y = ln(L + eps) into its running
 * statistics one batch at a time, tests it at every sample count
 * spp_min + r * spp_batch below spp_max that the window reaches, and either
 * lists it in `undecided` or writes its event, sample count and mean
 * (updating the reference on an event); samples after a pixel's decision are
 * ignored.  The schedule is enforced: the first call of a frame has
 * k_base = 0 and spp_r = spp_min; every later call starts on the schedule
 * (k_base = spp_min + r * spp_batch) and covers whole batches (spp_r a
 * multiple of spp_batch, or ending exactly at spp_max).  Pixel ids outside
 * [0, n_total) are skipped, the other pixels are still processed, and the
 * call then returns MCEV_ERR_ARG.  *n_undecided (host) receives the number
 * of pixels listed.
 * Errors: MCEV_ERR_ARG for null or inconsistent arguments, calls off the
 * schedule, out-of-range pixel ids, and schedules needing more than
 * MCEV_DETECT_STATIC_MAX_TESTS tests (the table would not fit the fixed
 * scratch); MCEV_ERR_CUDA for failed CUDA calls. */
mcev_status mcev_detect_batch_static(const mcev_detect_args* args, int64_t* n_undecided);

/* ------------------------------------------------------------------------
 * Quality metrics of event videos (Sec. 4.2)
 *
 * The paper scores an event video against the uniform-sampling baseline by
 * the RMSE and PSNR of its event frames (negative / no / positive event
 * stored as 0 / 0.5 / 1) and by an F1 score and a chamfer distance ("PSCD")
 * of signed point clouds, one point (x, y, t) with its polarity per event,
 * where only points of equal polarity are compared.  The thresholds behind
 * the last two are not given; these are this library's definitions:
 *   - coordinates are lattice units (pixel column, pixel row, frame index);
 *   - d(a, B) = Euclidean distance from a to the nearest point of B with a's
 *     polarity, or the lattice diagonal D = sqrt((W-1)^2+(H-1)^2+(T-1)^2)
 *     when B has no point of that polarity;
 *   - a point is matched when d^2 <= tau2; precision = matched a / |A|,
 *     recall = matched b / |B| (1 for an empty cloud), F1 = 2PR/(P+R);
 *   - PSCD = (mean_a d(a, B) + mean_b d(b, A)) / (2 D);
 *   - MSE over all W*H*T mapped values, RMSE = sqrt(MSE),
 *     PSNR = -10 log10(MSE) (HUGE_VAL for identical videos).
 * The distances are exact (integer distance transform on the GPU).
 * ------------------------------------------------------------------------ */
typedef struct mcev_quality {
    int64_t voxels;       /* W * H * T */
    int64_t n_a, n_b;     /* events in a, in b */
    int64_t matched_a;    /* events of a with d^2 <= tau2 */
    int64_t matched_b;
    int64_t none_a;       /* events of a whose polarity b lacks (d = D) */
    int64_t none_b;
    int64_t sq_diff;      /* sum over voxels of (a - b)^2 on the raw values */
    double sum_dist_a;    /* sum over a's events of d(a, B), lattice units */
    double sum_dist_b;
    double diag;          /* D */
    double rmse, psnr, precision, recall, f1, pscd;
    float gpu_ms;         /* device time of the call */
    int32_t kernel_launches;
} mcev_quality;

/* Metrics of event video `a` against `b`: device int8 arrays
 * [frames][height][width] of {-1, 0, +1} (caller-owned, read only).
 * tau2: squared match radius in lattice units (3: the 26 neighbours).
 * d2_a / d2_b: optional device int32 [frames*height*width] receiving, at each
 * event voxel of a (of b), the squared distance d^2 to the other video's
 * nearest same-polarity event, -2 where it has none, and -1 at voxels
 * without an event; NULL to skip.  Results go to *out (host).  The context
 * needs no scene; scratch (8 bytes per voxel, plus up to 2 GiB of envelope
 * stacks) is allocated through it.
 * Errors: ARG (NULL inputs, an extent outside 1..16384, tau2 < 0, a value
 * outside {-1, 0, 1}), OOM, CUDA.
 * Paper: the quality metrics of Sec. 4.2 (RMSE, PSNR, F1, PSCD). */
mcev_status mcev_event_quality(mcev_ctx* ctx, const int8_t* a, const int8_t* b, int32_t width, int32_t height,
                               int32_t frames, int32_t tau2, int32_t* d2_a, int32_t* d2_b, mcev_quality* out);

#ifdef __cplusplus
}
#endif
#endif
