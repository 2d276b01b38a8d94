// bvh8.cpp -- compressed 8-wide BVH built by collapsing the binned-SAH binary
// tree, after Ylitie, Karras and Laine, "Efficient incoherent ray traversal on
// GPUs through compressed wide BVHs" (HPG 2017): child boxes quantised to 8
// bits per plane on a power-of-two grid anchored at the node's lower corner,
// internal children stored contiguously, leaf triangles contiguous from a base
// index, children placed in slots by direction so that a ray visits them
// nearest-first by octant alone.  Children are marked by an internal-child mask
// and a 3-bit-per-slot triangle mask (layout.h) rather than per-child bytes.
//
// Collapse rule: a wide node starts from the two children of a binary node
// and repeatedly opens the candidate of largest surface area (an inner binary
// node, or a leaf of more than three triangles, split in half along its
// longest axis) until it has eight children or nothing can be opened.  A
// child is then either a leaf of one to three triangles or another wide node.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

#include "bvh.h"

namespace mcev {

namespace {

struct CBox {
    float lo[3], hi[3];
    void reset() {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::numeric_limits<float>::max();
            hi[a] = -std::numeric_limits<float>::max();
        }
    }
    void grow(const CBox& b) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], b.lo[a]);
            hi[a] = std::max(hi[a], b.hi[a]);
        }
    }
    double area() const {
        if (lo[0] > hi[0]) return 0.0;
        const double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1], dz = (double)hi[2] - lo[2];
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

// A subtree of the binary BVH: an inner node (node >= 0) or a run of
// primitives [first, first + count) of the leaf order.
struct Cand {
    CBox box;
    int node;
    int first, count;
};

struct Collapser {
    const BuiltBvh& b;
    std::vector<int> order;       // leaf order of the binary tree (runs re-sorted when split)
    const float* plo;
    const float* phi;
    std::vector<Node8> out;
    std::vector<int> tri_order;   // positions in `order`
    int depth = 0;
    bool ok = true;

    Collapser(const BuiltBvh& b_, const float* lo, const float* hi) : b(b_), order(b_.order), plo(lo), phi(hi) {}

    CBox prims_box(int first, int count) const {
        CBox r;
        r.reset();
        for (int i = first; i < first + count; ++i) {
            const int p = order[i];
            for (int a = 0; a < 3; ++a) {
                r.lo[a] = std::min(r.lo[a], plo[3 * p + a]);
                r.hi[a] = std::max(r.hi[a], phi[3 * p + a]);
            }
        }
        return r;
    }

    // children of binary node n as candidates (empty leaves dropped)
    void children_of(int n, std::vector<Cand>& c) const {
        const Node& nd = b.nodes[n];
        for (int side = 0; side < 2; ++side) {
            const float4 xy = side ? nd.b : nd.a;
            Cand k;
            k.box.lo[0] = xy.x;
            k.box.hi[0] = xy.y;
            k.box.lo[1] = xy.z;
            k.box.hi[1] = xy.w;
            k.box.lo[2] = side ? nd.c.z : nd.c.x;
            k.box.hi[2] = side ? nd.c.w : nd.c.y;
            const int ref = side ? nd.d.y : nd.d.x;
            const int cnt = side ? nd.d.w : nd.d.z;
            if (ref >= 0) {
                k.node = ref;
                k.first = k.count = 0;
            } else {
                if (cnt == 0) continue;
                k.node = -1;
                k.first = ~ref;
                k.count = cnt;
            }
            c.push_back(k);
        }
    }

    bool openable(const Cand& c) const { return c.node >= 0 || c.count > 3; }

    // splits a leaf run in half along the longest axis of its centroids
    void split_leaf(const Cand& c, Cand& l, Cand& r) {
        CBox cb;
        cb.reset();
        for (int i = c.first; i < c.first + c.count; ++i) {
            const int p = order[i];
            for (int a = 0; a < 3; ++a) {
                const float m = 0.5f * (plo[3 * p + a] + phi[3 * p + a]);
                cb.lo[a] = std::min(cb.lo[a], m);
                cb.hi[a] = std::max(cb.hi[a], m);
            }
        }
        int axis = 0;
        for (int a = 1; a < 3; ++a)
            if (cb.hi[a] - cb.lo[a] > cb.hi[axis] - cb.lo[axis]) axis = a;
        std::stable_sort(order.begin() + c.first, order.begin() + c.first + c.count, [&](int x, int y) {
            return plo[3 * x + axis] + phi[3 * x + axis] < plo[3 * y + axis] + phi[3 * y + axis];
        });
        const int h = (c.count + 1) / 2;
        l.node = r.node = -1;
        l.first = c.first;
        l.count = h;
        r.first = c.first + h;
        r.count = c.count - h;
        l.box = prims_box(l.first, l.count);
        r.box = prims_box(r.first, r.count);
    }

    // Fills wide node `idx` from its candidate children and recurses.
    void emit(int idx, std::vector<Cand> cands, int level) {
        depth = std::max(depth, level);
        while (cands.size() < 8) {
            int best = -1;
            double best_area = -1.0;
            for (size_t i = 0; i < cands.size(); ++i)
                if (openable(cands[i]) && cands[i].box.area() > best_area) {
                    best_area = cands[i].box.area();
                    best = (int)i;
                }
            if (best < 0) break;
            const Cand c = cands[best];
            cands.erase(cands.begin() + best);
            if (c.node >= 0) {
                children_of(c.node, cands);
            } else {
                Cand l, r;
                split_leaf(c, l, r);
                cands.push_back(l);
                cands.push_back(r);
            }
        }
        const int n = (int)cands.size();
        CBox nb;
        nb.reset();
        for (const Cand& c : cands) nb.grow(c.box);
        // slots by direction: slot bit a set = child towards -a of the node centre
        int slot_of[8];
        bool used_slot[8] = {false, false, false, false, false, false, false, false};
        bool placed[8] = {false, false, false, false, false, false, false, false};
        double cost[8][8];
        for (int i = 0; i < n; ++i) {
            double dc[3];
            for (int a = 0; a < 3; ++a)
                dc[a] = 0.5 * ((double)cands[i].box.lo[a] + cands[i].box.hi[a]) -
                        0.5 * ((double)nb.lo[a] + nb.hi[a]);
            for (int s = 0; s < 8; ++s)
                cost[i][s] = ((s & 1) ? -dc[0] : dc[0]) + ((s & 2) ? -dc[1] : dc[1]) + ((s & 4) ? -dc[2] : dc[2]);
        }
        for (int round = 0; round < n; ++round) {
            int bi = -1, bs = -1;
            double bc = -std::numeric_limits<double>::max();
            for (int i = 0; i < n; ++i) {
                if (placed[i]) continue;
                for (int s = 0; s < 8; ++s)
                    if (!used_slot[s] && cost[i][s] > bc) {
                        bc = cost[i][s];
                        bi = i;
                        bs = s;
                    }
            }
            placed[bi] = true;
            used_slot[bs] = true;
            slot_of[bi] = bs;
        }
        int cand_in_slot[8];
        for (int s = 0; s < 8; ++s) cand_in_slot[s] = -1;
        for (int i = 0; i < n; ++i) cand_in_slot[slot_of[i]] = i;

        Node8 nd;
        std::memset(&nd, 0, sizeof nd);
        // per-axis grid: step s = 2^k >= extent / 253 (and not below 2^-20 of
        // the coordinates, so the anchor differs from the corner in FP32),
        // anchored half a step below the node's lower corner
        double step[3];
        float anchor[3];
        for (int a = 0; a < 3; ++a) {
            const double lo = nb.lo[a], hi = nb.hi[a];
            const double mag = std::max(std::fabs(lo), std::fabs(hi));
            const double raw = std::max(std::max((hi - lo) / 253.0, mag * 0x1p-20), 0x1p-100);
            int k;
            std::frexp(raw, &k);              // raw = f * 2^k, f in [0.5, 1): 2^k >= raw
            if (std::ldexp(1.0, k - 1) >= raw) --k;
            step[a] = std::ldexp(1.0, k);
            float p = (float)(lo - 0.5 * step[a]);
            if ((double)p > lo - 0.5 * step[a]) p = std::nextafter(p, -std::numeric_limits<float>::infinity());
            anchor[a] = p;
            const int e = k + 127;
            if (e < 1 || e > 254 - 15) ok = false;   // 2^(k+15) must stay a normal float
            nd.e_imask |= (uint32_t)(std::min(std::max(e, 0), 255)) << (8 * a);
        }
        nd.px = anchor[0];
        nd.py = anchor[1];
        nd.pz = anchor[2];
        uint8_t qlo[3][8], qhi[3][8];
        uint32_t trimask = 0;
        for (int s = 0; s < 8; ++s) {
            for (int a = 0; a < 3; ++a) {
                qlo[a][s] = 255;
                qhi[a][s] = 0;
            }
        }
        int n_inner = 0, n_tris = 0, imask = 0;
        const int child_base = (int)out.size();
        for (int s = 0; s < 8; ++s)
            if (cand_in_slot[s] >= 0 && openable(cands[cand_in_slot[s]])) {
                imask |= 1 << s;
                ++n_inner;
            }
        out.resize(out.size() + n_inner);
        const int tri_base = (int)tri_order.size();
        for (int s = 0; s < 8; ++s) {
            const int ci = cand_in_slot[s];
            if (ci < 0) continue;
            const Cand& c = cands[ci];
            for (int a = 0; a < 3; ++a) {
                // planes at least 1/16 step outside the child's box (FP32
                // evaluation of a plane is accurate to far less than that)
                const double fl = std::floor(((double)c.box.lo[a] - anchor[a]) / step[a] - 1.0 / 16.0);
                const double fh = std::ceil(((double)c.box.hi[a] - anchor[a]) / step[a] + 1.0 / 16.0);
                if (fl < 0.0 || fh > 255.0) ok = false;
                qlo[a][s] = (uint8_t)std::min(std::max(fl, 0.0), 255.0);
                qhi[a][s] = (uint8_t)std::min(std::max(fh, 0.0), 255.0);
            }
            if (!(imask & (1 << s))) {
                if (c.count < 1 || c.count > 3) ok = false;
                trimask |= (uint32_t)((1 << c.count) - 1) << (3 * s);
                for (int i = 0; i < c.count; ++i) tri_order.push_back(c.first + i);
                n_tris += c.count;
            }
        }
        nd.e_imask |= (uint32_t)imask << 24;
        nd.child_base = (uint32_t)child_base;
        if (tri_order.size() >= ((size_t)1 << 29) || n < 1) ok = false;
        nd.tri_base = (uint32_t)tri_base | ((uint32_t)(n - 1) << 29);
        nd.trimask = trimask;
        for (int s = 0; s < 8; ++s) {
            reinterpret_cast<uint8_t*>(nd.qlo_x)[s] = qlo[0][s];
            reinterpret_cast<uint8_t*>(nd.qlo_y)[s] = qlo[1][s];
            reinterpret_cast<uint8_t*>(nd.qlo_z)[s] = qlo[2][s];
            reinterpret_cast<uint8_t*>(nd.qhi_x)[s] = qhi[0][s];
            reinterpret_cast<uint8_t*>(nd.qhi_y)[s] = qhi[1][s];
            reinterpret_cast<uint8_t*>(nd.qhi_z)[s] = qhi[2][s];
        }
        out[idx] = nd;
        // children in slot order, each filled before its own subtree
        int k = 0;
        for (int s = 0; s < 8; ++s) {
            if (!(imask & (1 << s))) continue;
            const Cand& c = cands[cand_in_slot[s]];
            std::vector<Cand> sub;
            if (c.node >= 0) {
                children_of(c.node, sub);
            } else {
                Cand l, r;
                split_leaf(c, l, r);
                sub.push_back(l);
                sub.push_back(r);
            }
            emit(child_base + k, sub, level + 1);
            ++k;
        }
    }
};

}  // namespace

WideBvh collapse_wide(const BuiltBvh& b, const float* prim_lo, const float* prim_hi) {
    WideBvh w;
    Collapser c(b, prim_lo, prim_hi);
    c.out.reserve(b.nodes.size() / 3 + 1);
    c.out.resize(1);
    std::vector<Cand> root;
    if (!b.nodes.empty()) c.children_of(0, root);
    if (root.empty()) {
        // no triangles: a root with no children (every slot empty)
        Node8 nd;
        std::memset(&nd, 0, sizeof nd);
        for (int s = 0; s < 8; ++s) {
            reinterpret_cast<uint8_t*>(nd.qlo_x)[s] = reinterpret_cast<uint8_t*>(nd.qlo_y)[s] =
                reinterpret_cast<uint8_t*>(nd.qlo_z)[s] = 255;
        }
        nd.e_imask = 127u | (127u << 8) | (127u << 16);
        c.out[0] = nd;
        w.nodes = c.out;
        w.depth = 1;
        w.ok = true;
        return w;
    }
    c.emit(0, root, 1);
    w.nodes = std::move(c.out);
    w.depth = c.depth;
    w.ok = c.ok;
    w.tri_order.reserve(c.tri_order.size());
    for (int i : c.tri_order) w.tri_order.push_back(c.order[i]);
    // every primitive exactly once
    std::vector<char> seen(b.order.size(), 0);
    for (int p : w.tri_order) {
        if (p < 0 || (size_t)p >= seen.size() || seen[p]) w.ok = false;
        else seen[p] = 1;
    }
    if (w.tri_order.size() != b.order.size()) w.ok = false;
    // every index a traversal can form stays inside the arrays, and children
    // come after their parent (the node graph is a tree, so traversal ends)
    for (size_t i = 0; i < w.nodes.size(); ++i) {
        const Node8& nd = w.nodes[i];
        const uint32_t imask = nd.e_imask >> 24;
        if (imask && (nd.child_base <= i || (size_t)nd.child_base + __builtin_popcount(imask) > w.nodes.size()))
            w.ok = false;
        if (nd.trimask >> 24) w.ok = false;
        for (int s = 0; s < 8; ++s) {
            const uint32_t t3 = (nd.trimask >> (3 * s)) & 7u;
            if (((imask >> s) & 1u) && t3) w.ok = false;
            if (t3 != 0 && t3 != 1 && t3 != 3 && t3 != 7) w.ok = false;
        }
        if ((size_t)(nd.tri_base & 0x1FFFFFFFu) + __builtin_popcount(nd.trimask) > w.tri_order.size()) w.ok = false;
    }
    return w;
}

}  // namespace mcev
