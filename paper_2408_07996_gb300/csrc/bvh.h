// bvh.h -- host BVH builder.
#pragma once
#include <vector>

#include "layout.h"

namespace mcev {

struct BuiltBvh {
    std::vector<Node> nodes;  // node 0 is the root; leaf refs are ~(first index into `order`)
    std::vector<int> order;   // primitive ids in leaf order
    int depth;                // deepest inner node level (stack bound for traversal)
};

// prim_lo/prim_hi/centroid: [n][3].  bins: SAH bins; max_leaf: leaf size cap.
BuiltBvh build_bvh(const float* prim_lo, const float* prim_hi, const float* centroid, int n, int bins, int max_leaf);

struct WideBvh {
    std::vector<Node8> nodes;  // node 0 is the root; child_base / tri_base are local
    std::vector<int> tri_order;// primitive ids in the order the leaves reference them
    int depth;                 // levels of wide nodes (stack bound for traversal)
    bool ok;                   // every invariant held (primitives once, planes in range)
};

// Collapses a binary BVH over primitives with boxes prim_lo/prim_hi [n][3]
// into the compressed 8-wide layout of layout.h.
WideBvh collapse_wide(const BuiltBvh& b, const float* prim_lo, const float* prim_hi);

}  // namespace mcev
