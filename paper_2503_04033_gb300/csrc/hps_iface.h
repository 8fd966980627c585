// Internal: the nested-dissection plan of the interface system of a uniform
// box grid (host side, no CUDA).  Shared by the host plan query
// (hps_iface_plan.cpp) and the GPU factorisation and solve (hps_iface.cu).
#pragma once

#include <vector>

namespace hps {

// An interface face of the grid: the plane `plane` (0 < plane < nb[axis])
// normal to `axis`, at cell (c1, c2) of the other two axes in increasing axis
// order.  Its q^2 nodes are ordered as on both boxes that share it (lower
// free axis fastest), so a face-block position maps node for node.
struct IfFace {
    int axis, plane, c1, c2;
    bool operator<(const IfFace& o) const
    {
        if (axis != o.axis) return axis < o.axis;
        if (plane != o.plane) return plane < o.plane;
        if (c2 != o.c2) return c2 < o.c2;
        return c1 < o.c1;
    }
    bool operator==(const IfFace& o) const
    {
        return axis == o.axis && plane == o.plane && c1 == o.c1 && c2 == o.c2;
    }
};

// One node of the merge tree.  Leaves (ids 0 .. nbox-1, the box index) keep
// their local face slots (x-, x+, y-, y+[, z-, z+]), Dirichlet ones marked
// absent; a merge node's boundary is the list `faces` (interface faces only),
// whose slot i covers positions i s .. (i+1) s - 1 of the node's vectors
// (s = q^2 nodes per face in 3-D, q per edge in 2-D).
// For a merge node with children a and b split at plane `split` of `axis`:
//   a1: slots of a's faces not on the separator (in a's order)
//   a3: slots of a's faces on the separator, in separator order
//   b2, b3: the same for b.
// The node's boundary is [a's faces at a1, then b's faces at b2].
struct IfNode {
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int child[2] = {-1, -1};
    int height = 0, axis = -1, split = 0;
    std::vector<IfFace> faces;          // merge nodes: boundary faces in slot order
    std::vector<char> leaf_iface;       // leaves: which local faces are interface faces
    std::vector<int> a1, a3, b2, b3;
};

struct IfPlan {
    int p = 0, q = 0, nb[3] = {0, 0, 0}, nbox = 0;
    int nfaces = 6;                       // faces of a leaf: 6 (3-D boxes) or 4 (2-D boxes, nb[2] = 1)
    std::vector<IfNode> nodes;            // leaves first (box order), then merges by height, root last
    std::vector<std::vector<int>> levels; // merge-node ids of height 1, 2, ...
};

// Builds the plan: the box range is halved recursively along its longest axis
// (in boxes; ties to the lower axis).  nfaces = 6 for a grid of 3-D boxes,
// 4 for a grid of 2-D boxes (edges x-, x+, y-, y+; nb[2] must be 1), where a
// "face" is an edge of q nodes.  Returns false for invalid sizes.
bool build_iface_plan(int p, const int nb[3], IfPlan* out, int nfaces = 6);

}  // namespace hps
