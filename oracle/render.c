/* FP64 path tracer: the tracePaths(q, s, N) of Alg. 1 (Sec. 3, Sec. 3.3).
 * Test infrastructure only; plain and slow on purpose.
 *
 * Light transport follows pbrt-v4's PathIntegrator, which the paper modifies
 * (Sec. 3.3): unidirectional path tracing, next-event estimation at every
 * scattering vertex, power-heuristic multiple importance sampling, no Russian
 * roulette.  The scene conventions (one-sided emitters, two-sided scattering,
 * keyframed rigid instances, latitude-longitude environment) and every random
 * number's Philox counter are fixed in the project design notes; this file
 * restates them without sharing code with the GPU path.
 *
 * Per path, with beta the path throughput and depth the index of the ray
 * segment (0 = camera ray):
 *   miss           : L += beta * w * Le_env(d)
 *   emissive hit   : L += beta * w * Le             (front side only)
 *   depth==max_depth or black surface: stop
 *   NEE            : L += beta * f * |cos| * Le * w / pdf_light   if visible
 *   BSDF sample    : beta *= f * |cos| / pdf_bsdf
 * w = 1 for camera rays or without NEE, 0 for BSDF hits with NEE but no MIS,
 * else the power heuristic pdf_a^2 / (pdf_a^2 + pdf_b^2). */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define PI 3.14159265358979323846

typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double len(v3 a) { return sqrt(dot(a, a)); }
static v3 nrm(v3 a) { return scl(a, 1.0 / len(a)); }
static double comp(v3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

/* ------------------------------------------------------------------ */
/* scene storage                                                       */
/* ------------------------------------------------------------------ */

typedef struct {
    double lo[3], hi[3];
    int32_t left, right;   /* children (inner node) */
    int32_t first, count;  /* range in the mesh's triangle order (leaf: count > 0) */
} onode;

typedef struct {
    int64_t first_tri, n_tri;
    onode* nodes;
    int64_t n_nodes;
    int64_t* order;        /* global triangle ids in leaf order */
} omesh;

struct orc_scene {
    int64_t nt;
    double* tv;            /* [nt][9] object-space vertices v0,v1,v2 per triangle */
    int32_t* tri_mat;
    int32_t nm;
    omesh* meshes;
    int32_t ni;
    int32_t* inst_mesh;
    int32_t* inst_mat;
    int32_t nk;
    double* key_t;
    double* key_xf;        /* [nk][ni][12] */
    double* cam_eye;
    double* cam_tgt;
    double* cam_up;
    double fov_deg;
    int32_t nmat;
    int32_t* mtype;
    double *malb, *mrough, *memit;
    double* memit0;        /* the table's emission: fixes which materials emit */
    /* environment */
    int32_t ew, eh;
    double* env;           /* [eh][ew] */
    double* marg;          /* [eh+1] row CDF, values rounded to FP32 */
    double* cond;          /* [eh][ew+1] column CDFs, values rounded to FP32 */
    double env_total;      /* sum_ij L_ij sin(theta_i) */
    /* texturing */
    double* tri_uv;        /* [nt][6] or NULL */
    int32_t* mat_tex;      /* [nmat] or NULL */
    int32_t tw, th;
    double* tex;           /* [th][tw][3] */
    /* emissive (instance, triangle) pairs in instance-then-triangle order */
    int64_t n_lights;
    int32_t* light_inst;
    int64_t* light_prim;
};

/* ---------------- median-split BVH per mesh (plain, for speed only) ---------------- */

typedef struct {
    const double* tv;
    double* cen;           /* centroid per local triangle [3] */
    int64_t* idx;          /* local triangle ids being partitioned */
    onode* nodes;
    int64_t n_nodes, cap;
} bvh_build;

static void tri_bounds(const double* v, double lo[3], double hi[3]) {
    for (int a = 0; a < 3; ++a) {
        lo[a] = fmin(v[a], fmin(v[3 + a], v[6 + a]));
        hi[a] = fmax(v[a], fmax(v[3 + a], v[6 + a]));
    }
}

static void select_kth(bvh_build* b, int64_t lo, int64_t hi, int64_t k, int axis) {
    /* quickselect: after return idx[lo..k) <= idx[k] <= idx[k..hi) by centroid */
    while (hi - lo > 1) {
        double pivot = b->cen[3 * b->idx[(lo + hi) / 2] + axis];
        int64_t i = lo, j = hi - 1;
        while (i <= j) {
            while (b->cen[3 * b->idx[i] + axis] < pivot) ++i;
            while (b->cen[3 * b->idx[j] + axis] > pivot) --j;
            if (i <= j) {
                int64_t t = b->idx[i]; b->idx[i] = b->idx[j]; b->idx[j] = t;
                ++i; --j;
            }
        }
        if (k <= j) hi = j + 1;
        else if (k >= i) lo = i;
        else return;
    }
}

static int32_t build_node(bvh_build* b, int64_t first_global, int64_t lo, int64_t hi) {
    if (b->n_nodes == b->cap) {
        b->cap *= 2;
        b->nodes = (onode*)realloc(b->nodes, sizeof(onode) * b->cap);
    }
    int32_t me = (int32_t)b->n_nodes++;
    onode nd;
    double clo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, chi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int a = 0; a < 3; ++a) { nd.lo[a] = DBL_MAX; nd.hi[a] = -DBL_MAX; }
    for (int64_t i = lo; i < hi; ++i) {
        double tlo[3], thi[3];
        tri_bounds(b->tv + 9 * (first_global + b->idx[i]), tlo, thi);
        for (int a = 0; a < 3; ++a) {
            nd.lo[a] = fmin(nd.lo[a], tlo[a]);
            nd.hi[a] = fmax(nd.hi[a], thi[a]);
            double c = b->cen[3 * b->idx[i] + a];
            clo[a] = fmin(clo[a], c);
            chi[a] = fmax(chi[a], c);
        }
    }
    /* pad so that rounding in the slab test can never cull a real hit */
    for (int a = 0; a < 3; ++a) {
        double pad = 1e-9 * (fabs(nd.lo[a]) + fabs(nd.hi[a]) + 1e-300) + 1e-12;
        nd.lo[a] -= pad;
        nd.hi[a] += pad;
    }
    if (hi - lo <= 4) {
        nd.left = nd.right = -1;
        nd.first = (int32_t)lo;
        nd.count = (int32_t)(hi - lo);
        b->nodes[me] = nd;
        return me;
    }
    int axis = 0;
    double ext = -1.0;
    for (int a = 0; a < 3; ++a)
        if (chi[a] - clo[a] > ext) { ext = chi[a] - clo[a]; axis = a; }
    int64_t mid = (lo + hi) / 2;
    select_kth(b, lo, hi, mid, axis);
    nd.first = 0;
    nd.count = 0;
    b->nodes[me] = nd;
    int32_t l = build_node(b, first_global, lo, mid);
    int32_t r = build_node(b, first_global, mid, hi);
    b->nodes[me].left = l;
    b->nodes[me].right = r;
    return me;
}

static void build_mesh_bvh(orc_scene* s, omesh* m) {
    m->n_nodes = 0;
    m->nodes = NULL;
    m->order = NULL;
    if (m->n_tri == 0) return;
    bvh_build b;
    b.tv = s->tv;
    b.cen = (double*)malloc(sizeof(double) * 3 * m->n_tri);
    b.idx = (int64_t*)malloc(sizeof(int64_t) * m->n_tri);
    for (int64_t i = 0; i < m->n_tri; ++i) {
        const double* v = s->tv + 9 * (m->first_tri + i);
        for (int a = 0; a < 3; ++a) b.cen[3 * i + a] = (v[a] + v[3 + a] + v[6 + a]) / 3.0;
        b.idx[i] = i;
    }
    b.cap = 1024;
    b.n_nodes = 0;
    b.nodes = (onode*)malloc(sizeof(onode) * b.cap);
    build_node(&b, m->first_tri, 0, m->n_tri);
    m->nodes = b.nodes;
    m->n_nodes = b.n_nodes;
    m->order = (int64_t*)malloc(sizeof(int64_t) * m->n_tri);
    for (int64_t i = 0; i < m->n_tri; ++i) m->order[i] = m->first_tri + b.idx[i];
    free(b.cen);
    free(b.idx);
}

/* ---------------- environment CDFs ---------------- */
/* Row weights are sum_j L_ij * sin(pi (i + 1/2) / H); each row's column
 * weights are L_ij.  Prefix sums run in FP64 in index order, are divided by
 * the total, and are then rounded to FP32 so that the discrete choice of a
 * texel is made on the same FP32 numbers as on the GPU. */
static void build_env(orc_scene* s) {
    int W = s->ew, H = s->eh;
    s->marg = (double*)malloc(sizeof(double) * (H + 1));
    s->cond = (double*)malloc(sizeof(double) * H * (W + 1));
    double* raw = (double*)malloc(sizeof(double) * (W + 1));
    double* mraw = (double*)malloc(sizeof(double) * (H + 1));
    mraw[0] = 0.0;
    for (int i = 0; i < H; ++i) {
        double sin_t = sin(PI * (i + 0.5) / H);
        raw[0] = 0.0;
        for (int j = 0; j < W; ++j) raw[j + 1] = raw[j] + s->env[(int64_t)i * W + j];
        double rowsum = raw[W];
        double* c = s->cond + (int64_t)i * (W + 1);
        for (int j = 0; j < W; ++j)
            c[j] = rowsum > 0.0 ? (double)(float)(raw[j] / rowsum) : (double)(float)((double)j / W);
        c[W] = 1.0;
        mraw[i + 1] = mraw[i] + rowsum * sin_t;
    }
    s->env_total = mraw[H];
    for (int i = 0; i < H; ++i)
        s->marg[i] = s->env_total > 0.0 ? (double)(float)(mraw[i] / s->env_total)
                                        : (double)(float)((double)i / H);
    s->marg[H] = 1.0;
    free(raw);
    free(mraw);
}

orc_scene* orc_scene_create(
    int64_t n_vertices, const float* vertices,
    int64_t n_triangles, const int32_t* triangles, const int32_t* tri_material,
    int32_t n_meshes, const int32_t* mesh_ranges,
    int32_t n_instances, const int32_t* inst_mesh, const int32_t* inst_material,
    int32_t n_keys, const double* key_times, const double* inst_xform,
    const double* cam_eye, const double* cam_target, const double* cam_up, double fov_deg,
    int32_t n_materials, const int32_t* mat_type, const float* mat_albedo,
    const float* mat_rough, const float* mat_emit,
    int32_t env_w, int32_t env_h, const float* env) {
    (void)n_vertices;
    orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
    s->nt = n_triangles;
    s->tv = (double*)malloc(sizeof(double) * 9 * (n_triangles > 0 ? n_triangles : 1));
    s->tri_mat = (int32_t*)malloc(sizeof(int32_t) * (n_triangles > 0 ? n_triangles : 1));
    for (int64_t t = 0; t < n_triangles; ++t) {
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a)
                s->tv[9 * t + 3 * k + a] = (double)vertices[3 * (int64_t)triangles[3 * t + k] + a];
        s->tri_mat[t] = tri_material[t];
    }
    s->nm = n_meshes;
    s->meshes = (omesh*)calloc(n_meshes > 0 ? n_meshes : 1, sizeof(omesh));
    for (int m = 0; m < n_meshes; ++m) {
        s->meshes[m].first_tri = mesh_ranges[2 * m];
        s->meshes[m].n_tri = mesh_ranges[2 * m + 1];
        build_mesh_bvh(s, &s->meshes[m]);
    }
    s->ni = n_instances;
    s->inst_mesh = (int32_t*)malloc(sizeof(int32_t) * (n_instances + 1));
    s->inst_mat = (int32_t*)malloc(sizeof(int32_t) * (n_instances + 1));
    memcpy(s->inst_mesh, inst_mesh, sizeof(int32_t) * n_instances);
    memcpy(s->inst_mat, inst_material, sizeof(int32_t) * n_instances);
    s->nk = n_keys;
    s->key_t = (double*)malloc(sizeof(double) * n_keys);
    memcpy(s->key_t, key_times, sizeof(double) * n_keys);
    s->key_xf = (double*)malloc(sizeof(double) * 12 * ((int64_t)n_keys * n_instances + 1));
    memcpy(s->key_xf, inst_xform, sizeof(double) * 12 * (int64_t)n_keys * n_instances);
    s->cam_eye = (double*)malloc(sizeof(double) * 3 * n_keys);
    s->cam_tgt = (double*)malloc(sizeof(double) * 3 * n_keys);
    s->cam_up = (double*)malloc(sizeof(double) * 3 * n_keys);
    memcpy(s->cam_eye, cam_eye, sizeof(double) * 3 * n_keys);
    memcpy(s->cam_tgt, cam_target, sizeof(double) * 3 * n_keys);
    memcpy(s->cam_up, cam_up, sizeof(double) * 3 * n_keys);
    s->fov_deg = fov_deg;
    s->nmat = n_materials;
    s->mtype = (int32_t*)malloc(sizeof(int32_t) * n_materials);
    s->malb = (double*)malloc(sizeof(double) * n_materials);
    s->mrough = (double*)malloc(sizeof(double) * n_materials);
    s->memit = (double*)malloc(sizeof(double) * n_materials);
    s->memit0 = (double*)malloc(sizeof(double) * n_materials);
    for (int i = 0; i < n_materials; ++i) {
        s->memit0[i] = mat_emit[i];
        s->mtype[i] = mat_type[i];
        s->malb[i] = mat_albedo[i];
        s->mrough[i] = mat_rough[i];
        s->memit[i] = mat_emit[i];
    }
    /* emissive triangles never change over time: list them once */
    s->n_lights = 0;
    s->light_inst = NULL;
    s->light_prim = NULL;
    int64_t cap = 0;
    for (int i = 0; i < n_instances; ++i) {
        const omesh* m = &s->meshes[inst_mesh[i]];
        for (int64_t tt = 0; tt < m->n_tri; ++tt) {
            int64_t prim = m->first_tri + tt;
            int32_t mat = inst_material[i] >= 0 ? inst_material[i] : tri_material[prim];
            if (!(mat_emit[mat] > 0.0f)) continue;
            if (s->n_lights == cap) {
                cap = cap ? 2 * cap : 16;
                s->light_inst = (int32_t*)realloc(s->light_inst, sizeof(int32_t) * cap);
                s->light_prim = (int64_t*)realloc(s->light_prim, sizeof(int64_t) * cap);
            }
            s->light_inst[s->n_lights] = i;
            s->light_prim[s->n_lights] = prim;
            ++s->n_lights;
        }
    }
    s->ew = env ? env_w : 0;
    s->eh = env ? env_h : 0;
    if (env) {
        s->env = (double*)malloc(sizeof(double) * (int64_t)env_w * env_h);
        for (int64_t i = 0; i < (int64_t)env_w * env_h; ++i) s->env[i] = env[i];
        build_env(s);
    }
    return s;
}

void orc_scene_free(orc_scene* s) {
    if (!s) return;
    for (int m = 0; m < s->nm; ++m) {
        free(s->meshes[m].nodes);
        free(s->meshes[m].order);
    }
    free(s->meshes); free(s->tv); free(s->tri_mat); free(s->inst_mesh); free(s->inst_mat);
    free(s->key_t); free(s->key_xf); free(s->cam_eye); free(s->cam_tgt); free(s->cam_up);
    free(s->mtype); free(s->malb); free(s->mrough); free(s->memit); free(s->memit0);
    free(s->env); free(s->marg); free(s->cond);
    free(s->light_inst); free(s->light_prim);
    free(s->tri_uv); free(s->mat_tex); free(s->tex);
    free(s);
}

void orc_scene_set_texture(orc_scene* s, const float* uvs, const int32_t* triangles, const int32_t* mat_textured,
                           int32_t tex_w, int32_t tex_h, const float* texture) {
    free(s->tri_uv); free(s->mat_tex); free(s->tex);
    s->tri_uv = (double*)malloc(sizeof(double) * 6 * (s->nt > 0 ? s->nt : 1));
    for (int64_t t = 0; t < s->nt; ++t)
        for (int c = 0; c < 3; ++c)
            for (int a = 0; a < 2; ++a)
                s->tri_uv[6 * t + 2 * c + a] = uvs[2 * (int64_t)triangles[3 * t + c] + a];
    s->mat_tex = (int32_t*)malloc(sizeof(int32_t) * s->nmat);
    for (int m = 0; m < s->nmat; ++m) s->mat_tex[m] = mat_textured[m];
    s->tw = tex_w;
    s->th = tex_h;
    s->tex = (double*)malloc(sizeof(double) * 3 * (int64_t)tex_w * tex_h);
    for (int64_t i = 0; i < 3 * (int64_t)tex_w * tex_h; ++i) s->tex[i] = texture[i];
}

void orc_scene_set_emission(orc_scene* s, const float* emission) {
    for (int m = 0; m < s->nmat; ++m)
        if (s->memit0[m] > 0.0) s->memit[m] = emission[m];
}

/* ------------------------------------------------------------------ */
/* frame state at one time                                              */
/* ------------------------------------------------------------------ */

typedef struct {
    double M[12], Minv[12];
    double lo[3], hi[3];   /* world AABB */
} oinst;

typedef struct {
    v3 v0, v1, v2, n;
    double area, Le;
    int32_t inst;
    int64_t prim;
} olight;

typedef struct {
    double time;
    uint32_t key[2];
    oinst* inst;
    v3 eye, fwd, right, up;
    double sx, sy;
    int32_t n_lights;
    olight* lights;
} oframe;

/* keyframe bracket: largest k with key_t[k] <= t, clamped to [0, nk-2] */
static void key_bracket(const orc_scene* s, double t, int* k, double* f) {
    if (s->nk == 1) { *k = 0; *f = 0.0; return; }
    int kk = 0;
    while (kk + 1 < s->nk - 1 && s->key_t[kk + 1] <= t) ++kk;
    double fr = (t - s->key_t[kk]) / (s->key_t[kk + 1] - s->key_t[kk]);
    if (fr < 0.0) fr = 0.0;
    if (fr > 1.0) fr = 1.0;
    *k = kk;
    *f = fr;
}

static double lerp(double a, double b, double f) { return (1.0 - f) * a + f * b; }

static void affine_inverse(const double* M, double* R) {
    /* inverse of [A | b] is [A^-1 | -A^-1 b], A^-1 by cofactors */
    double a = M[0], b = M[1], c = M[2], d = M[4], e = M[5], f = M[6], g = M[8], h = M[9], i = M[10];
    double A = e * i - f * h, B = -(d * i - f * g), Cc = d * h - e * g;
    double det = a * A + b * B + c * Cc;
    double id = 1.0 / det;
    double inv[9] = {A * id, -(b * i - c * h) * id, (b * f - c * e) * id,
                     B * id, (a * i - c * g) * id, -(a * f - c * d) * id,
                     Cc * id, -(a * h - b * g) * id, (a * e - b * d) * id};
    for (int r = 0; r < 3; ++r) {
        R[4 * r + 0] = inv[3 * r + 0];
        R[4 * r + 1] = inv[3 * r + 1];
        R[4 * r + 2] = inv[3 * r + 2];
        R[4 * r + 3] = -(inv[3 * r + 0] * M[3] + inv[3 * r + 1] * M[7] + inv[3 * r + 2] * M[11]);
    }
}

static v3 xf_point(const double* M, v3 p) {
    return mk(M[0] * p.x + M[1] * p.y + M[2] * p.z + M[3],
              M[4] * p.x + M[5] * p.y + M[6] * p.z + M[7],
              M[8] * p.x + M[9] * p.y + M[10] * p.z + M[11]);
}
static v3 xf_vec(const double* M, v3 p) {
    return mk(M[0] * p.x + M[1] * p.y + M[2] * p.z,
              M[4] * p.x + M[5] * p.y + M[6] * p.z,
              M[8] * p.x + M[9] * p.y + M[10] * p.z);
}
/* normal transform: (A^-1)^T n */
static v3 xf_normal(const double* Minv, v3 n) {
    return mk(Minv[0] * n.x + Minv[4] * n.y + Minv[8] * n.z,
              Minv[1] * n.x + Minv[5] * n.y + Minv[9] * n.z,
              Minv[2] * n.x + Minv[6] * n.y + Minv[10] * n.z);
}

static int material_of(const orc_scene* s, int32_t inst, int64_t prim) {
    int32_t o = s->inst_mat[inst];
    return o >= 0 ? o : s->tri_mat[prim];
}

static uint32_t frame_key(double t) {
    uint64_t b;
    memcpy(&b, &t, sizeof b);
    return (uint32_t)(b ^ (b >> 32));
}

static void frame_setup(const orc_scene* s, const orc_params* p, double t, oframe* fr) {
    fr->time = t;
    fr->key[0] = (uint32_t)p->seed ^ frame_key(t);
    fr->key[1] = (uint32_t)(p->seed >> 32);
    int k;
    double f;
    key_bracket(s, t, &k, &f);
    fr->inst = (oinst*)calloc(s->ni > 0 ? s->ni : 1, sizeof(oinst));
    for (int i = 0; i < s->ni; ++i) {
        oinst* in = &fr->inst[i];
        const double* A = s->key_xf + 12 * ((int64_t)k * s->ni + i);
        const double* B = s->key_xf + 12 * ((int64_t)(s->nk > 1 ? k + 1 : k) * s->ni + i);
        for (int e = 0; e < 12; ++e) in->M[e] = lerp(A[e], B[e], f);
        affine_inverse(in->M, in->Minv);
        const omesh* m = &s->meshes[s->inst_mesh[i]];
        for (int a = 0; a < 3; ++a) { in->lo[a] = DBL_MAX; in->hi[a] = -DBL_MAX; }
        if (m->n_nodes > 0) {
            const onode* r = &m->nodes[0];
            for (int c = 0; c < 8; ++c) {
                v3 q = mk((c & 1) ? r->hi[0] : r->lo[0], (c & 2) ? r->hi[1] : r->lo[1],
                          (c & 4) ? r->hi[2] : r->lo[2]);
                v3 w = xf_point(in->M, q);
                for (int a = 0; a < 3; ++a) {
                    in->lo[a] = fmin(in->lo[a], comp(w, a));
                    in->hi[a] = fmax(in->hi[a], comp(w, a));
                }
            }
            for (int a = 0; a < 3; ++a) {
                double pad = 1e-9 * (fabs(in->lo[a]) + fabs(in->hi[a])) + 1e-12;
                in->lo[a] -= pad;
                in->hi[a] += pad;
            }
        }
    }
    /* world-space emitters */
    fr->n_lights = (int32_t)s->n_lights;
    fr->lights = (olight*)calloc(s->n_lights > 0 ? s->n_lights : 1, sizeof(olight));
    for (int64_t l = 0; l < s->n_lights; ++l) {
        int32_t i = s->light_inst[l];
        int64_t prim = s->light_prim[l];
        const double* M = fr->inst[i].M;
        const double* v = s->tv + 9 * prim;
        olight* L = &fr->lights[l];
        L->v0 = xf_point(M, mk(v[0], v[1], v[2]));
        L->v1 = xf_point(M, mk(v[3], v[4], v[5]));
        L->v2 = xf_point(M, mk(v[6], v[7], v[8]));
        v3 c = cross(sub(L->v1, L->v0), sub(L->v2, L->v0));
        L->area = 0.5 * len(c);
        L->n = nrm(c);
        L->Le = s->memit[material_of(s, i, prim)];
        L->inst = i;
        L->prim = prim;
    }
    /* camera */
    v3 e0 = mk(s->cam_eye[3 * k], s->cam_eye[3 * k + 1], s->cam_eye[3 * k + 2]);
    v3 t0 = mk(s->cam_tgt[3 * k], s->cam_tgt[3 * k + 1], s->cam_tgt[3 * k + 2]);
    v3 u0 = mk(s->cam_up[3 * k], s->cam_up[3 * k + 1], s->cam_up[3 * k + 2]);
    int k1 = s->nk > 1 ? k + 1 : k;
    v3 e1 = mk(s->cam_eye[3 * k1], s->cam_eye[3 * k1 + 1], s->cam_eye[3 * k1 + 2]);
    v3 t1 = mk(s->cam_tgt[3 * k1], s->cam_tgt[3 * k1 + 1], s->cam_tgt[3 * k1 + 2]);
    v3 u1 = mk(s->cam_up[3 * k1], s->cam_up[3 * k1 + 1], s->cam_up[3 * k1 + 2]);
    v3 eye = mk(lerp(e0.x, e1.x, f), lerp(e0.y, e1.y, f), lerp(e0.z, e1.z, f));
    v3 tgt = mk(lerp(t0.x, t1.x, f), lerp(t0.y, t1.y, f), lerp(t0.z, t1.z, f));
    v3 up = mk(lerp(u0.x, u1.x, f), lerp(u0.y, u1.y, f), lerp(u0.z, u1.z, f));
    fr->eye = eye;
    fr->fwd = nrm(sub(tgt, eye));
    fr->right = nrm(cross(fr->fwd, up));
    fr->up = cross(fr->right, fr->fwd);
    double th = tan(0.5 * s->fov_deg * PI / 180.0);
    if (p->width >= p->height) {
        fr->sy = th;
        fr->sx = th * (double)p->width / (double)p->height;
    } else {
        fr->sx = th;
        fr->sy = th * (double)p->height / (double)p->width;
    }
}

static void frame_free(oframe* fr) {
    free(fr->inst);
    free(fr->lights);
}

/* ------------------------------------------------------------------ */
/* intersection                                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    v3 o, d;
    int kx, ky, kz;
    double Sx, Sy, Sz;
} oray;

/* watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013):
 * shear/scale into a frame where the ray is the +z axis, then the 2D edge
 * functions U, V, W decide containment exactly at shared edges. */
static void ray_prepare(oray* r) {
    double ax = fabs(r->d.x), ay = fabs(r->d.y), az = fabs(r->d.z);
    int kz = 0;
    if (ay > ax && ay >= az) kz = 1;
    else if (az > ax && az > ay) kz = 2;
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (comp(r->d, kz) < 0.0) { int t = kx; kx = ky; ky = t; }
    r->kx = kx; r->ky = ky; r->kz = kz;
    r->Sx = comp(r->d, kx) / comp(r->d, kz);
    r->Sy = comp(r->d, ky) / comp(r->d, kz);
    r->Sz = 1.0 / comp(r->d, kz);
}

static int tri_hit(const oray* r, const double* v, double tmin, double tmax, double* tout) {
    v3 A = sub(mk(v[0], v[1], v[2]), r->o);
    v3 B = sub(mk(v[3], v[4], v[5]), r->o);
    v3 C = sub(mk(v[6], v[7], v[8]), r->o);
    double Ax = comp(A, r->kx) - r->Sx * comp(A, r->kz);
    double Ay = comp(A, r->ky) - r->Sy * comp(A, r->kz);
    double Bx = comp(B, r->kx) - r->Sx * comp(B, r->kz);
    double By = comp(B, r->ky) - r->Sy * comp(B, r->kz);
    double Cx = comp(C, r->kx) - r->Sx * comp(C, r->kz);
    double Cy = comp(C, r->ky) - r->Sy * comp(C, r->kz);
    double U = Cx * By - Cy * Bx;
    double V = Ax * Cy - Ay * Cx;
    double W = Bx * Ay - By * Ax;
    if ((U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0)) return 0;
    double det = U + V + W;
    if (det == 0.0) return 0;
    double Az = r->Sz * comp(A, r->kz);
    double Bz = r->Sz * comp(B, r->kz);
    double Cz = r->Sz * comp(C, r->kz);
    double T = U * Az + V * Bz + W * Cz;
    double t = T / det;
    if (!(t > tmin && t < tmax)) return 0;
    *tout = t;
    return 1;
}

static int box_hit(const double lo[3], const double hi[3], v3 o, v3 d, double tmin, double tmax) {
    double t0 = tmin, t1 = tmax;
    for (int a = 0; a < 3; ++a) {
        double oa = comp(o, a), da = comp(d, a);
        if (da == 0.0) {
            if (oa < lo[a] || oa > hi[a]) return 0;
            continue;
        }
        double ta = (lo[a] - oa) / da, tb = (hi[a] - oa) / da;
        if (ta > tb) { double t = ta; ta = tb; tb = t; }
        tb *= 1.0 + 1e-12;
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    return 1;
}

typedef struct {
    double t;
    int32_t inst;
    int64_t prim;
} ohit;

/* closest hit; ties in t go to the smaller (instance, triangle) pair */
static int better(double t, int32_t inst, int64_t prim, const ohit* h) {
    if (t < h->t) return 1;
    if (t > h->t) return 0;
    if (inst != h->inst) return inst < h->inst;
    return prim < h->prim;
}

static void mesh_closest(const orc_scene* s, const omesh* m, const oray* r, int32_t inst,
                         double tmin, int use_bvh, ohit* h) {
    if (m->n_tri == 0) return;
    if (!use_bvh) {
        for (int64_t i = 0; i < m->n_tri; ++i) {
            int64_t prim = m->first_tri + i;
            double t;
            if (tri_hit(r, s->tv + 9 * prim, tmin, INFINITY, &t) && t <= h->t
                && better(t, inst, prim, h)) {
                h->t = t; h->inst = inst; h->prim = prim;
            }
        }
        return;
    }
    int32_t stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const onode* nd = &m->nodes[stack[--sp]];
        if (!box_hit(nd->lo, nd->hi, r->o, r->d, tmin, h->t)) continue;
        if (nd->count > 0) {
            for (int32_t i = 0; i < nd->count; ++i) {
                int64_t prim = m->order[nd->first + i];
                double t;
                if (tri_hit(r, s->tv + 9 * prim, tmin, INFINITY, &t) && t <= h->t
                    && better(t, inst, prim, h)) {
                    h->t = t; h->inst = inst; h->prim = prim;
                }
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
}

static int mesh_any(const orc_scene* s, const omesh* m, const oray* r, double tmin, double tmax) {
    if (m->n_tri == 0) return 0;
    int32_t stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const onode* nd = &m->nodes[stack[--sp]];
        if (!box_hit(nd->lo, nd->hi, r->o, r->d, tmin, tmax)) continue;
        if (nd->count > 0) {
            for (int32_t i = 0; i < nd->count; ++i) {
                double t;
                if (tri_hit(r, s->tv + 9 * m->order[nd->first + i], tmin, tmax, &t)) return 1;
            }
        } else {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
        }
    }
    return 0;
}

static void object_ray(const oinst* in, v3 o, v3 d, oray* r) {
    r->o = xf_point(in->Minv, o);
    r->d = xf_vec(in->Minv, d);
    ray_prepare(r);
}

static int scene_closest(const orc_scene* s, const oframe* fr, v3 o, v3 d, double tmin, double tmax,
                         int use_bvh, ohit* h) {
    h->t = tmax;
    h->inst = -1;
    h->prim = -1;
    for (int32_t i = 0; i < s->ni; ++i) {
        const oinst* in = &fr->inst[i];
        if (use_bvh && !box_hit(in->lo, in->hi, o, d, tmin, h->t)) continue;
        oray r;
        object_ray(in, o, d, &r);
        mesh_closest(s, &s->meshes[s->inst_mesh[i]], &r, i, tmin, use_bvh, h);
    }
    return h->inst >= 0;
}

static int scene_occluded(const orc_scene* s, const oframe* fr, v3 o, v3 d, double tmin, double tmax) {
    for (int32_t i = 0; i < s->ni; ++i) {
        const oinst* in = &fr->inst[i];
        if (!box_hit(in->lo, in->hi, o, d, tmin, tmax)) continue;
        oray r;
        object_ray(in, o, d, &r);
        if (mesh_any(s, &s->meshes[s->inst_mesh[i]], &r, tmin, tmax)) return 1;
    }
    return 0;
}

int orc_closest_hit(const orc_scene* s, double time, const double o[3], const double d[3],
                    double t_min, double t_max, int use_bvh,
                    double* t_out, int32_t* inst_out, int32_t* prim_out) {
    orc_params p;
    memset(&p, 0, sizeof p);
    p.width = p.height = 1;
    oframe fr;
    frame_setup(s, &p, time, &fr);
    ohit h;
    int hit = scene_closest(s, &fr, mk(o[0], o[1], o[2]), mk(d[0], d[1], d[2]), t_min, t_max, use_bvh, &h);
    *t_out = h.t;
    *inst_out = h.inst;
    *prim_out = (int32_t)h.prim;
    frame_free(&fr);
    return hit;
}

/* world-space unit geometric normal (winding orientation) of a hit */
static v3 hit_normal(const orc_scene* s, const oframe* fr, const ohit* h) {
    const double* v = s->tv + 9 * h->prim;
    v3 e1 = mk(v[3] - v[0], v[4] - v[1], v[5] - v[2]);
    v3 e2 = mk(v[6] - v[0], v[7] - v[1], v[8] - v[2]);
    return nrm(xf_normal(fr->inst[h->inst].Minv, cross(e1, e2)));
}

static double hit_world_area(const orc_scene* s, const oframe* fr, const ohit* h) {
    const double* v = s->tv + 9 * h->prim;
    const double* M = fr->inst[h->inst].M;
    v3 a = xf_point(M, mk(v[0], v[1], v[2]));
    v3 b = xf_point(M, mk(v[3], v[4], v[5]));
    v3 c = xf_point(M, mk(v[6], v[7], v[8]));
    return 0.5 * len(cross(sub(b, a), sub(c, a)));
}

/* ------------------------------------------------------------------ */
/* environment                                                         */
/* ------------------------------------------------------------------ */

static void env_texel(const orc_scene* s, v3 d, int* row, int* col, double* sin_t) {
    double cy = d.y < -1.0 ? -1.0 : (d.y > 1.0 ? 1.0 : d.y);
    double theta = acos(cy);
    double phi = atan2(d.z, d.x);
    if (phi < 0.0) phi += 2.0 * PI;
    int c = (int)(phi / (2.0 * PI) * s->ew);
    int r = (int)(theta / PI * s->eh);
    if (c > s->ew - 1) c = s->ew - 1;
    if (r > s->eh - 1) r = s->eh - 1;
    *row = r;
    *col = c;
    *sin_t = sin(theta);
}

static double texel_pdf(const orc_scene* s, int row, int col, double sin_t) {
    if (!(s->env_total > 0.0) || !(sin_t > 0.0)) return 0.0;
    double w = s->env[(int64_t)row * s->ew + col] * sin(PI * (row + 0.5) / s->eh);
    return w / s->env_total * (double)s->ew * (double)s->eh / (2.0 * PI * PI * sin_t);
}

double orc_env_radiance(const orc_scene* s, const double dir[3]) {
    if (!s->env) return 0.0;
    int r, c;
    double st;
    env_texel(s, mk(dir[0], dir[1], dir[2]), &r, &c, &st);
    return s->env[(int64_t)r * s->ew + c];
}

double orc_env_pdf(const orc_scene* s, const double dir[3]) {
    if (!s->env) return 0.0;
    int r, c;
    double st;
    env_texel(s, mk(dir[0], dir[1], dir[2]), &r, &c, &st);
    return texel_pdf(s, r, c, st);
}

/* smallest k in [0, n) with u < cdf[k+1] */
static int cdf_pick(const double* cdf, int n, double u) {
    for (int k = 0; k < n; ++k)
        if (u < cdf[k + 1]) return k;
    return n - 1;
}

int orc_env_sample(const orc_scene* s, double u1, double u2, double dir[3], double* pdf, double* Le) {
    if (!s->env || !(s->env_total > 0.0)) return 0;
    int row = cdf_pick(s->marg, s->eh, u1);
    double dv = (u1 - s->marg[row]) / (s->marg[row + 1] - s->marg[row]);
    const double* c = s->cond + (int64_t)row * (s->ew + 1);
    int col = cdf_pick(c, s->ew, u2);
    double du = (u2 - c[col]) / (c[col + 1] - c[col]);
    double theta = PI * (row + dv) / s->eh;
    double phi = 2.0 * PI * (col + du) / s->ew;
    double st = sin(theta);
    dir[0] = st * cos(phi);
    dir[1] = cos(theta);
    dir[2] = st * sin(phi);
    *Le = s->env[(int64_t)row * s->ew + col];
    *pdf = texel_pdf(s, row, col, st);
    return 1;
}

/* ------------------------------------------------------------------ */
/* BSDFs in a local frame (normal = +z)                                */
/* ------------------------------------------------------------------ */

static double ggx_D(double a, double cz) {
    double a2 = a * a;
    double k = cz * cz * (a2 - 1.0) + 1.0;
    return a2 / (PI * k * k);
}
static double ggx_lambda(double a, double z) {
    double t2 = (1.0 - z * z) / (z * z);
    return 0.5 * (-1.0 + sqrt(1.0 + a * a * t2));
}

double orc_bsdf_eval(int type, double albedo, double rough, const double wo[3], const double wi[3],
                     double* pdf) {
    *pdf = 0.0;
    if (!(wo[2] > 0.0) || !(wi[2] > 0.0)) return 0.0;
    if (type == 0) {
        *pdf = wi[2] / PI;
        return albedo / PI;
    }
    v3 h = nrm(mk(wo[0] + wi[0], wo[1] + wi[1], wo[2] + wi[2]));
    double D = ggx_D(rough, h.z);
    double lo = ggx_lambda(rough, wo[2]), li = ggx_lambda(rough, wi[2]);
    double G1 = 1.0 / (1.0 + lo);
    double G2 = 1.0 / (1.0 + lo + li);
    double c = wi[0] * h.x + wi[1] * h.y + wi[2] * h.z;
    double m = 1.0 - c;
    double F = albedo + (1.0 - albedo) * m * m * m * m * m;
    *pdf = G1 * D / (4.0 * wo[2]);
    return F * D * G2 / (4.0 * wo[2] * wi[2]);
}

/* Lambertian: cosine-weighted hemisphere, r = sqrt(u1), phi = 2 pi u2.
 * GGX: visible-normal sampling (Heitz, JCGT 2018), then mirror wo about it. */
void orc_bsdf_sample(int type, double rough, const double wo[3], double u1, double u2, double wi[3]) {
    if (type == 0) {
        double r = sqrt(u1), phi = 2.0 * PI * u2;
        wi[0] = r * cos(phi);
        wi[1] = r * sin(phi);
        wi[2] = sqrt(fmax(0.0, 1.0 - u1));
        return;
    }
    double a = rough;
    v3 Vh = nrm(mk(a * wo[0], a * wo[1], wo[2]));
    double lensq = Vh.x * Vh.x + Vh.y * Vh.y;
    v3 T1 = lensq > 0.0 ? scl(mk(-Vh.y, Vh.x, 0.0), 1.0 / sqrt(lensq)) : mk(1.0, 0.0, 0.0);
    v3 T2 = cross(Vh, T1);
    double r = sqrt(u1), phi = 2.0 * PI * u2;
    double t1 = r * cos(phi), t2 = r * sin(phi);
    double sh = 0.5 * (1.0 + Vh.z);
    t2 = (1.0 - sh) * sqrt(1.0 - t1 * t1) + sh * t2;
    v3 Nh = add(add(scl(T1, t1), scl(T2, t2)), scl(Vh, sqrt(fmax(0.0, 1.0 - t1 * t1 - t2 * t2))));
    v3 Ne = nrm(mk(a * Nh.x, a * Nh.y, fmax(0.0, Nh.z)));
    double c = wo[0] * Ne.x + wo[1] * Ne.y + wo[2] * Ne.z;
    wi[0] = 2.0 * c * Ne.x - wo[0];
    wi[1] = 2.0 * c * Ne.y - wo[1];
    wi[2] = 2.0 * c * Ne.z - wo[2];
}

/* orthonormal basis around n (Duff et al., JCGT 2017), sign(+0) = +1 */
static void onb(v3 n, v3* t, v3* b) {
    double sg = n.z >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + n.z);
    double bb = n.x * n.y * a;
    *t = mk(1.0 + sg * n.x * n.x * a, sg * bb, -sg * n.x);
    *b = mk(bb, sg + n.y * n.y * a, -n.y);
}

static double power_heuristic(double a, double b) {
    double a2 = a * a, b2 = b * b;
    return a2 / (a2 + b2);
}

static uint32_t fnv(uint32_t h, uint32_t w) { return (h ^ w) * 16777619u; }

/* ------------------------------------------------------------------ */
/* one path                                                            */
/* ------------------------------------------------------------------ */

static void rng4(const oframe* fr, uint32_t pix, uint32_t k, uint32_t bounce, uint32_t blk, uint32_t x[4]) {
    uint32_t c[4] = {pix, k, bounce, blk};
    orc_philox4x32_10(c, fr->key, x);
}

static double trace_path(const orc_scene* s, const orc_params* p, const oframe* fr,
                         int32_t pix, int64_t k, uint32_t* sig_out) {
    uint32_t sig = 2166136261u;
    int px = pix % p->width, py = pix / p->width;
    uint32_t x[4];
    rng4(fr, (uint32_t)pix, (uint32_t)k, 0u, 0u, x);
    double fx = 2.0 * ((double)px + orc_u01(x[0])) / (double)p->width - 1.0;
    double fy = 1.0 - 2.0 * ((double)py + orc_u01(x[1])) / (double)p->height;
    v3 o = fr->eye;
    v3 d = nrm(add(fr->fwd, add(scl(fr->right, fx * fr->sx), scl(fr->up, fy * fr->sy))));
    int env_ok = s->env != NULL && s->env_total > 0.0;
    int have_area = fr->n_lights > 0;
    double p_env = env_ok ? (have_area ? 0.5 : 1.0) : 0.0;
    double p_area = have_area ? (env_ok ? 0.5 : 1.0) : 0.0;
    double L = 0.0, beta = 1.0, pdf_prev = 0.0;
    for (int depth = 0;; ++depth) {
        ohit h;
        if (!scene_closest(s, fr, o, d, p->t_min, INFINITY, 1, &h)) {
            sig = fnv(sig, 0xFFFFFFFFu);
            if (s->env) {
                int row, col;
                double st;
                env_texel(s, d, &row, &col, &st);
                sig = fnv(sig, (uint32_t)(row * s->ew + col));
                double Le = s->env[(int64_t)row * s->ew + col];
                double w = 1.0;
                if (depth > 0 && p->nee) {
                    if (!p->mis) w = 0.0;
                    else w = power_heuristic(pdf_prev, p_env * texel_pdf(s, row, col, st));
                }
                L += beta * w * Le;
            } else {
                sig = fnv(sig, 0xFFFFFFFEu);
            }
            break;
        }
        sig = fnv(sig, (uint32_t)h.inst);
        sig = fnv(sig, (uint32_t)h.prim);
        v3 P = add(o, scl(d, h.t));
        v3 ng = hit_normal(s, fr, &h);
        v3 wo = scl(d, -1.0);
        int mat = material_of(s, h.inst, h.prim);
        double alb = s->malb[mat];
        if (s->tex && s->mat_tex && s->mat_tex[mat]) {
            /* barycentric coordinates of the hit in the object-space triangle */
            const double* v = s->tv + 9 * h.prim;
            v3 a = mk(v[0], v[1], v[2]), b = mk(v[3], v[4], v[5]), c = mk(v[6], v[7], v[8]);
            v3 po = xf_point(fr->inst[h.inst].Minv, P);
            v3 e1 = sub(b, a), e2 = sub(c, a), vp = sub(po, a);
            double d00 = dot(e1, e1), d01 = dot(e1, e2), d11 = dot(e2, e2), d20 = dot(vp, e1), d21 = dot(vp, e2);
            double den = d00 * d11 - d01 * d01;
            double b1 = (d11 * d20 - d01 * d21) / den, b2 = (d00 * d21 - d01 * d20) / den, b0 = 1.0 - b1 - b2;
            const double* uv = s->tri_uv + 6 * h.prim;
            double u = b0 * uv[0] + b1 * uv[2] + b2 * uv[4];
            double vv = b0 * uv[1] + b1 * uv[3] + b2 * uv[5];
            if (!isfinite(u)) u = 0.0; /* degenerate triangle */
            if (!isfinite(vv)) vv = 0.0;
            u -= floor(u);
            vv -= floor(vv);
            int ix = (int)(u * s->tw), iy = (int)(vv * s->th);
            if (ix > s->tw - 1) ix = s->tw - 1;
            if (iy > s->th - 1) iy = s->th - 1;
            int64_t texel = (int64_t)iy * s->tw + ix;
            const double* rgb = s->tex + 3 * texel;
            alb = 0.2126 * rgb[0] + 0.7152 * rgb[1] + 0.0722 * rgb[2];
            sig = fnv(sig, (uint32_t)texel);
        }
        uint32_t flags = 0;
        double cos_o = dot(ng, wo);
        if (s->memit[mat] > 0.0 && cos_o > 0.0) {
            flags |= 1u;
            double w = 1.0;
            if (depth > 0 && p->nee) {
                if (!p->mis) w = 0.0;
                else {
                    double area = hit_world_area(s, fr, &h);
                    double pl = p_area / ((double)fr->n_lights * area) * h.t * h.t / cos_o;
                    w = power_heuristic(pdf_prev, pl);
                }
            }
            L += beta * w * s->memit[mat];
        }
        if (depth == p->max_depth || !(alb > 0.0)) {
            sig = fnv(sig, flags);
            break;
        }
        v3 n = cos_o < 0.0 ? scl(ng, -1.0) : ng;
        v3 tb, bt;
        onb(n, &tb, &bt);
        double wol[3] = {dot(wo, tb), dot(wo, bt), dot(wo, n)};
        int type = s->mtype[mat];
        double rough = s->mrough[mat];
        /* next-event estimation */
        if (p->nee && (env_ok || have_area)) {
            rng4(fr, (uint32_t)pix, (uint32_t)k, (uint32_t)(depth + 1), 0u, x);
            int use_env = env_ok && (!have_area || orc_u01(x[0]) < 0.5);
            v3 wi = mk(0, 0, 0);
            double pl = 0.0, Le = 0.0, tmax = INFINITY;
            if (use_env) {
                double dir[3], pdf;
                orc_env_sample(s, orc_u01(x[2]), orc_u01(x[3]), dir, &pdf, &Le);
                wi = mk(dir[0], dir[1], dir[2]);
                pl = p_env * pdf;
            } else {
                uint64_t m = (uint64_t)(x[1] >> 8);
                int64_t li = (int64_t)((m * (uint64_t)fr->n_lights) >> 24);
                const olight* lt = &fr->lights[li];
                double su = sqrt(orc_u01(x[2]));
                double b0 = 1.0 - su, b1 = orc_u01(x[3]) * su, b2 = 1.0 - b0 - b1;
                v3 Q = add(add(scl(lt->v0, b0), scl(lt->v1, b1)), scl(lt->v2, b2));
                v3 dv = sub(Q, P);
                double dist = len(dv);
                wi = scl(dv, 1.0 / dist);
                double cl = -dot(lt->n, wi);
                if (cl > 0.0) {
                    pl = p_area / ((double)fr->n_lights * lt->area) * dist * dist / cl;
                    Le = lt->Le;
                }
                tmax = dist - p->t_min;
            }
            if (pl > 0.0 && Le > 0.0) {
                double wil[3] = {dot(wi, tb), dot(wi, bt), dot(wi, n)};
                double pb;
                double f = orc_bsdf_eval(type, alb, rough, wol, wil, &pb);
                double ci = wil[2];
                if (f > 0.0 && ci > 0.0) {
                    flags |= 2u;
                    double w = p->mis ? power_heuristic(pl, pb) : 1.0;
                    double contrib = beta * f * ci * Le * w / pl;
                    if (!scene_occluded(s, fr, P, wi, p->t_min, tmax)) {
                        flags |= 4u;
                        L += contrib;
                    }
                }
            }
        }
        /* BSDF sampling */
        rng4(fr, (uint32_t)pix, (uint32_t)k, (uint32_t)(depth + 1), 1u, x);
        double wil[3];
        orc_bsdf_sample(type, rough, wol, orc_u01(x[0]), orc_u01(x[1]), wil);
        double pb;
        double f = orc_bsdf_eval(type, alb, rough, wol, wil, &pb);
        if (!(f > 0.0 && pb > 0.0 && wil[2] > 0.0)) {
            sig = fnv(sig, flags);
            break;
        }
        flags |= 8u;
        sig = fnv(sig, flags);
        beta *= f * wil[2] / pb;
        pdf_prev = pb;
        v3 wi = add(add(scl(tb, wil[0]), scl(bt, wil[1])), scl(n, wil[2]));
        o = P;
        d = nrm(wi);
    }
    *sig_out = sig;
    return L;
}

int64_t orc_trace_samples(const orc_scene* s, const orc_params* p, double time,
                          const int32_t* pixels, int64_t n_pix, int64_t k0, int64_t count,
                          double* out_L, uint32_t* out_sig) {
    oframe fr;
    frame_setup(s, p, time, &fr);
    int64_t bad = 0;
    for (int64_t i = 0; i < n_pix; ++i)
        for (int64_t k = 0; k < count; ++k) {
            uint32_t sg;
            double L = trace_path(s, p, &fr, pixels[i], k0 + k, &sg);
            if (!isfinite(L)) { L = 0.0; ++bad; }
            out_L[i * count + k] = L;
            if (out_sig) out_sig[i * count + k] = sg;
        }
    frame_free(&fr);
    return bad;
}

/* ------------------------------------------------------------------ */
/* Alg. 1 over path-traced samples                                      */
/* ------------------------------------------------------------------ */

typedef struct {
    const orc_scene* s;
    const orc_params* p;
    const oframe* fr;
    int32_t pixel;
    int64_t bad;
} path_src;

static void draw_paths(void* ctx, int64_t k0, int64_t count, double* y) {
    path_src* ps = (path_src*)ctx;
    for (int64_t k = 0; k < count; ++k) {
        uint32_t sg;
        double L = trace_path(ps->s, ps->p, ps->fr, ps->pixel, k0 + k, &sg);
        if (!isfinite(L)) { L = 0.0; ++ps->bad; }
        y[k] = log(L + ps->p->eps);
    }
}

int64_t orc_render_events(const orc_scene* s, const orc_params* p, const orc_detect* d,
                          double t0, double t1, const int32_t* pixels, int64_t n_pix,
                          int make_ref, int64_t* ref_n, double* ref_mean, double* ref_var,
                          int8_t* events, int32_t* n_used, double* mean, double* var,
                          double* margin_t, double* margin_c) {
    oframe f0, f1;
    if (make_ref) frame_setup(s, p, t0, &f0);
    frame_setup(s, p, t1, &f1);
    double* y = (double*)malloc(sizeof(double) * (d->spp_max > 0 ? d->spp_max : 1));
    int64_t bad = 0;
    for (int64_t i = 0; i < n_pix; ++i) {
        if (make_ref) {
            /* first frame of Alg. 1: spp_max samples at t0 */
            path_src src0 = {s, p, &f0, pixels[i], 0};
            draw_paths(&src0, 0, d->spp_max, y);
            bad += src0.bad;
            ref_n[i] = d->spp_max;
            orc_mean_var(y, d->spp_max, &ref_mean[i], &ref_var[i]);
        }
        path_src src = {s, p, &f1, pixels[i], 0};
        orc_detect_pixel_cb(d, draw_paths, &src, &ref_n[i], &ref_mean[i], &ref_var[i],
                            &events[i], &n_used[i], &mean[i], &var[i], &margin_t[i], &margin_c[i]);
        bad += src.bad;
    }
    free(y);
    if (make_ref) frame_free(&f0);
    frame_free(&f1);
    return bad;
}

int64_t orc_reference(const orc_scene* s, const orc_params* p, int32_t spp, double time,
                      const int32_t* pixels, int64_t n_pix,
                      int64_t* ref_n, double* ref_mean, double* ref_var) {
    oframe fr;
    frame_setup(s, p, time, &fr);
    double* y = (double*)malloc(sizeof(double) * (spp > 0 ? spp : 1));
    int64_t bad = 0;
    for (int64_t i = 0; i < n_pix; ++i) {
        path_src src = {s, p, &fr, pixels[i], 0};
        draw_paths(&src, 0, spp, y);
        bad += src.bad;
        ref_n[i] = spp;
        orc_mean_var(y, spp, &ref_mean[i], &ref_var[i]);
    }
    free(y);
    frame_free(&fr);
    return bad;
}

void orc_camera_ray(const orc_scene* s, const orc_params* p, double time, double fx_pix,
                    double fy_pix, double o[3], double d[3]) {
    oframe fr;
    frame_setup(s, p, time, &fr);
    double fx = 2.0 * fx_pix / (double)p->width - 1.0;
    double fy = 1.0 - 2.0 * fy_pix / (double)p->height;
    v3 dd = nrm(add(fr.fwd, add(scl(fr.right, fx * fr.sx), scl(fr.up, fy * fr.sy))));
    o[0] = fr.eye.x; o[1] = fr.eye.y; o[2] = fr.eye.z;
    d[0] = dd.x; d[1] = dd.y; d[2] = dd.z;
    frame_free(&fr);
}
