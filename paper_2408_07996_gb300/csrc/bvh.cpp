// bvh.cpp -- binned surface-area-heuristic BVH builder (Wald, "On fast
// construction of SAH-based bounding volume hierarchies", RT 2007), emitting
// the two-children-per-node layout of layout.h.
#include "bvh.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

namespace mcev {

namespace {

struct Box {
    float lo[3], hi[3];
    void reset() {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::numeric_limits<float>::max();
            hi[a] = -std::numeric_limits<float>::max();
        }
    }
    void grow(const Box& b) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], b.lo[a]);
            hi[a] = std::max(hi[a], b.hi[a]);
        }
    }
    double area() const {
        if (lo[0] > hi[0]) return 0.0;
        const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

struct TmpNode {
    Box box;
    int left = -1, right = -1;  // children in tmp array (inner)
    int first = 0, count = 0;   // leaf range in `order`
};

struct Builder {
    const float* lo;
    const float* hi;
    std::vector<float> cen;
    std::vector<int> order;
    std::vector<TmpNode> nodes;
    int bins, max_leaf;

    Box prim_box(int i) const {
        Box b;
        for (int a = 0; a < 3; ++a) {
            b.lo[a] = lo[3 * i + a];
            b.hi[a] = hi[3 * i + a];
        }
        return b;
    }

    int make_leaf(int first, int count, const Box& b) {
        TmpNode n;
        n.box = b;
        n.first = first;
        n.count = count;
        nodes.push_back(n);
        return (int)nodes.size() - 1;
    }

    int build(int first, int count, int depth) {
        Box b, cb;
        b.reset();
        cb.reset();
        for (int i = first; i < first + count; ++i) {
            const int p = order[i];
            b.grow(prim_box(p));
            for (int a = 0; a < 3; ++a) {
                cb.lo[a] = std::min(cb.lo[a], cen[3 * p + a]);
                cb.hi[a] = std::max(cb.hi[a], cen[3 * p + a]);
            }
        }
        if (count <= 1) return make_leaf(first, count, b);
        int axis = 0;
        float ext = cb.hi[0] - cb.lo[0];
        for (int a = 1; a < 3; ++a)
            if (cb.hi[a] - cb.lo[a] > ext) {
                ext = cb.hi[a] - cb.lo[a];
                axis = a;
            }
        int mid = -1;
        const bool force_median = depth >= 48 || !(ext > 0.0f);
        if (!force_median) {
            // binned SAH over all three axes
            double best = std::numeric_limits<double>::max();
            int best_axis = -1, best_bin = -1;
            std::vector<Box> bb(bins);
            std::vector<int> bc(bins);
            std::vector<double> rarea(bins);
            std::vector<int> rcount(bins);
            for (int a = 0; a < 3; ++a) {
                const float clo = cb.lo[a], chi = cb.hi[a];
                if (!(chi > clo)) continue;
                const double scale = (double)bins / ((double)chi - (double)clo);
                for (int k = 0; k < bins; ++k) {
                    bb[k].reset();
                    bc[k] = 0;
                }
                for (int i = first; i < first + count; ++i) {
                    const int p = order[i];
                    int k = (int)(((double)cen[3 * p + a] - clo) * scale);
                    k = std::min(std::max(k, 0), bins - 1);
                    bb[k].grow(prim_box(p));
                    ++bc[k];
                }
                Box acc;
                acc.reset();
                int cnt = 0;
                for (int k = bins - 1; k > 0; --k) {
                    acc.grow(bb[k]);
                    cnt += bc[k];
                    rarea[k] = acc.area();
                    rcount[k] = cnt;
                }
                acc.reset();
                cnt = 0;
                for (int k = 0; k < bins - 1; ++k) {
                    acc.grow(bb[k]);
                    cnt += bc[k];
                    if (cnt == 0 || rcount[k + 1] == 0) continue;
                    const double c = acc.area() * cnt + rarea[k + 1] * rcount[k + 1];
                    if (c < best) {
                        best = c;
                        best_axis = a;
                        best_bin = k;
                    }
                }
            }
            const double parent = b.area();
            // SAH: traversal cost 1, intersection cost 1 per triangle
            const double split_cost = 1.0 + (parent > 0.0 ? best / parent : (double)count);
            if (count <= max_leaf && (best_axis < 0 || split_cost >= (double)count))
                return make_leaf(first, count, b);
            if (best_axis >= 0) {
                const float clo = cb.lo[best_axis], chi = cb.hi[best_axis];
                const double scale = (double)bins / ((double)chi - (double)clo);
                int* beg = order.data() + first;
                int* end = beg + count;
                int* m = std::partition(beg, end, [&](int p) {
                    int k = (int)(((double)cen[3 * p + best_axis] - clo) * scale);
                    k = std::min(std::max(k, 0), bins - 1);
                    return k <= best_bin;
                });
                mid = (int)(m - order.data());
                if (mid == first || mid == first + count) mid = -1;
            }
        }
        if (mid < 0) {
            if (count <= max_leaf) return make_leaf(first, count, b);
            mid = first + count / 2;
            std::nth_element(order.begin() + first, order.begin() + mid, order.begin() + first + count,
                             [&](int x, int y) { return cen[3 * x + axis] < cen[3 * y + axis]; });
        }
        TmpNode n;
        n.box = b;
        nodes.push_back(n);
        const int me = (int)nodes.size() - 1;
        const int l = build(first, mid - first, depth + 1);
        const int r = build(mid, first + count - mid, depth + 1);
        nodes[me].left = l;
        nodes[me].right = r;
        return me;
    }
};

void put_child(Node& n, int side, const TmpNode& c, int ref) {
    if (side == 0) {
        n.a.x = c.box.lo[0]; n.a.y = c.box.hi[0]; n.a.z = c.box.lo[1]; n.a.w = c.box.hi[1];
        n.c.x = c.box.lo[2]; n.c.y = c.box.hi[2];
        n.d.x = ref;
        n.d.z = c.left < 0 ? c.count : 0;
    } else {
        n.b.x = c.box.lo[0]; n.b.y = c.box.hi[0]; n.b.z = c.box.lo[1]; n.b.w = c.box.hi[1];
        n.c.z = c.box.lo[2]; n.c.w = c.box.hi[2];
        n.d.y = ref;
        n.d.w = c.left < 0 ? c.count : 0;
    }
}

}  // namespace

BuiltBvh build_bvh(const float* prim_lo, const float* prim_hi, const float* centroid, int n, int bins,
                   int max_leaf) {
    BuiltBvh out;
    out.depth = 0;
    Builder B;
    B.lo = prim_lo;
    B.hi = prim_hi;
    B.cen.assign(centroid, centroid + 3 * (size_t)n);
    B.order.resize(n);
    for (int i = 0; i < n; ++i) B.order[i] = i;
    B.bins = bins;
    B.max_leaf = max_leaf;
    B.nodes.reserve(n > 0 ? 2 * n : 1);
    if (n > 0) B.build(0, n, 0);
    out.order = B.order;
    // flatten: every emitted Node is an inner node of the temporary tree; its
    // children are either emitted Nodes (index >= 0) or leaves (~first).
    std::vector<int> emit_index(B.nodes.size(), -1);
    Node empty;
    std::memset(&empty, 0, sizeof empty);
    auto leaf_ref = [](const TmpNode& c) { return ~c.first; };
    if (n == 0 || B.nodes[0].left < 0) {
        // single leaf (or nothing): root with the leaf on the left, an empty
        // leaf on the right
        Node root = empty;
        TmpNode leaf;
        if (n > 0) leaf = B.nodes[0];
        else {
            leaf.box.reset();
            leaf.first = 0;
            leaf.count = 0;
        }
        put_child(root, 0, leaf, leaf_ref(leaf));
        TmpNode none;
        none.box.reset();
        none.first = 0;
        none.count = 0;
        put_child(root, 1, none, ~0);
        out.nodes.push_back(root);
        out.depth = 1;
        return out;
    }
    // depth-first emission, left child right after its parent
    struct Item {
        int tmp, depth;
    };
    std::vector<Item> stack;
    stack.push_back({0, 1});
    std::vector<int> order_of_emit;
    while (!stack.empty()) {
        const Item it = stack.back();
        stack.pop_back();
        emit_index[it.tmp] = (int)order_of_emit.size();
        order_of_emit.push_back(it.tmp);
        out.depth = std::max(out.depth, it.depth);
        const TmpNode& t = B.nodes[it.tmp];
        if (B.nodes[t.right].left >= 0) stack.push_back({t.right, it.depth + 1});
        if (B.nodes[t.left].left >= 0) stack.push_back({t.left, it.depth + 1});
    }
    out.nodes.resize(order_of_emit.size(), empty);
    for (size_t k = 0; k < order_of_emit.size(); ++k) {
        const TmpNode& t = B.nodes[order_of_emit[k]];
        const TmpNode& L = B.nodes[t.left];
        const TmpNode& R = B.nodes[t.right];
        put_child(out.nodes[k], 0, L, L.left >= 0 ? emit_index[t.left] : leaf_ref(L));
        put_child(out.nodes[k], 1, R, R.left >= 0 ? emit_index[t.right] : leaf_ref(R));
    }
    return out;
}

}  // namespace mcev
