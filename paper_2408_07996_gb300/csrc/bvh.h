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

}  // namespace mcev
