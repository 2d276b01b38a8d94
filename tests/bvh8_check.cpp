// Host check of the compressed 8-wide BVH builder (bvh.cpp + bvh8.cpp).
//
// For a triangle set it builds the binary SAH BVH, collapses it and checks:
//  1. the builder's own invariants (WideBvh::ok);
//  2. every triangle's box lies inside the dequantized box of its leaf slot
//     and of every ancestor slot, with at least 1/32 grid step to spare;
//  3. a closest-hit search that follows the node format's rules (visit keys
//     slot ^ octant, internal child rank by popc of imask, triangle index by
//     popc of the triangle mask, a stack of node groups) with exact box tests
//     in double precision finds the same nearest triangle as brute force, for
//     random rays.
// Usage: bvh8_check <scene kind 0..2> <n> <seed>.  Prints "OK" or the failure.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "bvh.h"

using namespace mcev;

static uint64_t rng_state;
static double urand() {
    rng_state = rng_state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(rng_state >> 11) * 0x1p-53;
}

struct Tri {
    double v[3][3];
};

static bool fail(const char* what, long a = 0, long b = 0) {
    std::printf("FAIL %s %ld %ld\n", what, a, b);
    return false;
}

// ray / triangle (Moller-Trumbore in double); returns t or -1
static double tri_t(const Tri& T, const double o[3], const double d[3]) {
    double e1[3], e2[3], p[3], q[3], s[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = T.v[1][a] - T.v[0][a];
        e2[a] = T.v[2][a] - T.v[0][a];
        s[a] = o[a] - T.v[0][a];
    }
    p[0] = d[1] * e2[2] - d[2] * e2[1];
    p[1] = d[2] * e2[0] - d[0] * e2[2];
    p[2] = d[0] * e2[1] - d[1] * e2[0];
    const double det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
    if (std::fabs(det) < 1e-300) return -1;
    const double u = (s[0] * p[0] + s[1] * p[1] + s[2] * p[2]) / det;
    q[0] = s[1] * e1[2] - s[2] * e1[1];
    q[1] = s[2] * e1[0] - s[0] * e1[2];
    q[2] = s[0] * e1[1] - s[1] * e1[0];
    const double v = (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]) / det;
    const double t = (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]) / det;
    if (u < 0 || v < 0 || u + v > 1 || t <= 1e-9) return -1;
    return t;
}

static uint8_t byte_of(const uint32_t w[2], int s) { return (uint8_t)(w[s >> 2] >> (8 * (s & 3))); }

struct DBox {
    double lo[3], hi[3];
};

static DBox slot_box(const Node8& n, int s) {
    DBox b;
    const double p[3] = {n.px, n.py, n.pz};
    const uint32_t* lo[3] = {n.qlo_x, n.qlo_y, n.qlo_z};
    const uint32_t* hi[3] = {n.qhi_x, n.qhi_y, n.qhi_z};
    for (int a = 0; a < 3; ++a) {
        const double step = std::ldexp(1.0, (int)((n.e_imask >> (8 * a)) & 0xFF) - 127);
        b.lo[a] = p[a] + step * byte_of(lo[a], s);
        b.hi[a] = p[a] + step * byte_of(hi[a], s);
    }
    return b;
}

static double min_step(const Node8& n) {
    double m = 1e300;
    for (int a = 0; a < 3; ++a) m = std::fmin(m, std::ldexp(1.0, (int)((n.e_imask >> (8 * a)) & 0xFF) - 127));
    return m;
}

static bool box_hit(const DBox& b, const double o[3], const double d[3], double tmax) {
    double tn = 0.0, tf = tmax;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < b.lo[a] || o[a] > b.hi[a]) return false;
            continue;
        }
        double t0 = (b.lo[a] - o[a]) / d[a], t1 = (b.hi[a] - o[a]) / d[a];
        if (t0 > t1) std::swap(t0, t1);
        tn = std::fmax(tn, t0);
        tf = std::fmin(tf, t1);
    }
    return tn <= tf;
}

int main(int argc, char** argv) {
    const int kind = argc > 1 ? std::atoi(argv[1]) : 0;
    const int n = argc > 2 ? std::atoi(argv[2]) : 1000;
    rng_state = argc > 3 ? std::strtoull(argv[3], nullptr, 10) : 1;
    std::vector<Tri> tris(n);
    for (int i = 0; i < n; ++i) {
        Tri& T = tris[i];
        if (kind == 0) {          // soup of small triangles in a box far from the origin
            double c[3] = {100 + 10 * urand(), -50 + 10 * urand(), 30 * urand()};
            for (int k = 0; k < 3; ++k)
                for (int a = 0; a < 3; ++a) T.v[k][a] = c[a] + 0.2 * (urand() - 0.5);
        } else if (kind == 1) {   // height field (a terrain): grid cells split in two
            const int g = (int)std::sqrt((double)n / 2) + 1;
            const int cell = i / 2, cx = cell % g, cy = cell / g;
            auto h = [](int x, int y) { return 0.3 * std::sin(0.7 * x) * std::cos(0.4 * y); };
            const double x0 = cx, y0 = cy;
            const double P[4][3] = {{x0, h(cx, cy), y0}, {x0 + 1, h(cx + 1, cy), y0},
                                    {x0, h(cx, cy + 1), y0 + 1}, {x0 + 1, h(cx + 1, cy + 1), y0 + 1}};
            const int idx[2][3] = {{0, 1, 2}, {1, 3, 2}};
            for (int k = 0; k < 3; ++k)
                for (int a = 0; a < 3; ++a) T.v[k][a] = P[idx[i & 1][k]][a];
        } else {                  // axis-aligned quads (zero thickness boxes), Cornell-like
            const int axis = i % 3;
            const double off = (double)(i / 3 % 7);
            const double u0 = urand() * 5, v0 = urand() * 5;
            const double Q[3][2] = {{u0, v0}, {u0 + 1, v0}, {u0, v0 + 1}};
            for (int k = 0; k < 3; ++k) {
                T.v[k][axis] = off;
                T.v[k][(axis + 1) % 3] = Q[k][0];
                T.v[k][(axis + 2) % 3] = Q[k][1];
            }
        }
    }
    std::vector<float> lo(3 * n), hi(3 * n), ce(3 * n);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            // FP32 copies of the vertices, as the library keeps them
            float v0 = (float)tris[i].v[0][a], v1 = (float)tris[i].v[1][a], v2 = (float)tris[i].v[2][a];
            tris[i].v[0][a] = v0;
            tris[i].v[1][a] = v1;
            tris[i].v[2][a] = v2;
            lo[3 * i + a] = std::fmin(v0, std::fmin(v1, v2));
            hi[3 * i + a] = std::fmax(v0, std::fmax(v1, v2));
            ce[3 * i + a] = (float)(((double)v0 + v1 + v2) / 3.0);
        }
    const BuiltBvh b = build_bvh(lo.data(), hi.data(), ce.data(), n, 32, 4);
    const WideBvh w = collapse_wide(b, lo.data(), hi.data());
    if (!w.ok) return fail("builder invariants"), 1;
    // 2. containment through every ancestor
    struct Item {
        uint32_t node;
        std::vector<DBox> anc;
    };
    std::vector<Item> st;
    st.push_back({0, {}});
    std::vector<int> seen(n, 0);
    while (!st.empty()) {
        Item it = st.back();
        st.pop_back();
        const Node8& nd = w.nodes[it.node];
        const uint32_t imask = nd.e_imask >> 24;
        const double margin = min_step(nd) / 32.0;
        for (int s = 0; s < 8; ++s) {
            const uint32_t t3 = (nd.trimask >> (3 * s)) & 7u;
            if (!(imask >> s & 1) && !t3) continue;
            const DBox sb = slot_box(nd, s);
            std::vector<DBox> anc = it.anc;
            anc.push_back(sb);
            if (imask >> s & 1) {
                const uint32_t child = nd.child_base + __builtin_popcount(imask & ((1u << s) - 1u));
                st.push_back({child, anc});
            } else {
                const uint32_t off = __builtin_popcount(nd.trimask & ((1u << (3 * s)) - 1u));
                const uint32_t cnt = __builtin_popcount(t3);
                for (uint32_t k = 0; k < cnt; ++k) {
                    const int prim = w.tri_order[(nd.tri_base & 0x1FFFFFFFu) + off + k];
                    ++seen[prim];
                    for (size_t q = 0; q < anc.size(); ++q)
                        for (int a = 0; a < 3; ++a) {
                            const double mg = q + 1 == anc.size() ? margin : 0.0;
                            if (lo[3 * prim + a] < anc[q].lo[a] + mg || hi[3 * prim + a] > anc[q].hi[a] - mg)
                                return fail("containment", prim, (long)q), 1;
                        }
                }
            }
        }
    }
    for (int i = 0; i < n; ++i)
        if (seen[i] != 1) return fail("triangle referenced", i, seen[i]), 1;
    // 3. closest hits through the node format's traversal rules
    double blo[3] = {1e300, 1e300, 1e300}, bhi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < 3 * n; ++i) {
        blo[i % 3] = std::fmin(blo[i % 3], lo[i]);
        bhi[i % 3] = std::fmax(bhi[i % 3], hi[i]);
    }
    int hits = 0;
    for (int r = 0; r < 2000; ++r) {
        double o[3], d[3], tgt[3], len = 0;
        for (int a = 0; a < 3; ++a) {
            const double ext = bhi[a] - blo[a] + 1.0;
            o[a] = blo[a] - 0.5 + ext * urand();
            tgt[a] = blo[a] - 0.5 + ext * urand();
            d[a] = tgt[a] - o[a];
            len += d[a] * d[a];
        }
        if (r % 4 == 0) d[r % 3] = 0.0;   // axis-parallel components
        double best = 1e300;
        int best_p = -1;
        for (int i = 0; i < n; ++i) {
            const double t = tri_t(tris[i], o, d);
            if (t >= 0 && t < best) {
                best = t;
                best_p = i;
            }
        }
        const uint32_t ox = (d[0] >= 0 ? 1u : 0u) | (d[1] >= 0 ? 2u : 0u) | (d[2] >= 0 ? 4u : 0u);
        uint32_t gx = 0, gy = (1u << (24 + ox)) | 1u;
        std::vector<std::pair<uint32_t, uint32_t>> stack;
        double h = 1e300;
        int hp = -1;
        uint32_t tm = 0;
        while (true) {
            uint32_t tb = 0, tbits = 0;
            if (gy & 0xFF000000u) {
                const uint32_t key = __builtin_ctz(gy >> 24);
                gy &= ~(1u << (24 + key));
                const uint32_t slot = key ^ ox;
                const uint32_t child = gx + __builtin_popcount(gy & ((1u << slot) - 1u) & 0xFFu);
                if (gy & 0xFF000000u) stack.push_back({gx, gy});
                const Node8& nd = w.nodes[child];
                const uint32_t imask = nd.e_imask >> 24;
                uint32_t keys = 0;
                tbits = 0;
                for (int s = 0; s < 8; ++s) {
                    const uint32_t t3 = (nd.trimask >> (3 * s)) & 7u;
                    if ((!(imask >> s & 1) && !t3) || !box_hit(slot_box(nd, s), o, d, h)) continue;
                    if (imask >> s & 1) keys |= 1u << (s ^ ox);
                    else tbits |= t3 << (3 * s);
                }
                gx = nd.child_base;
                gy = (keys << 24) | imask;
                tb = nd.tri_base & 0x1FFFFFFFu;
                tm = nd.trimask;
            }
            while (tbits) {
                const uint32_t bit = __builtin_ctz(tbits);
                const uint32_t ti = tb + __builtin_popcount(tm & ((1u << bit) - 1u));
                tbits &= tbits - 1;
                const int prim = w.tri_order[ti];
                const double t = tri_t(tris[prim], o, d);
                if (t >= 0 && t < h) {
                    h = t;
                    hp = prim;
                }
            }
            if (!(gy & 0xFF000000u)) {
                if (stack.empty()) break;
                gx = stack.back().first;
                gy = stack.back().second;
                stack.pop_back();
            }
        }
        if (hp != best_p && !(hp >= 0 && best_p >= 0 && std::fabs(h - best) <= 1e-12 * best))
            return fail("closest hit", r, hp), 1;
        hits += best_p >= 0;
    }
    std::printf("OK nodes %zu depth %d hits %d\n", w.nodes.size(), w.depth, hits);
    return 0;
}
