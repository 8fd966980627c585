// Nested-dissection plan of the interface system (host only).
//
// The interface system of Sec. 3.1 couples the face nodes shared by
// neighbouring leaf boxes through the blocks of their DtN maps.  The original
// HPS method (described in Sec. 3 as the alternative to the sparse
// factorisation) eliminates it hierarchically: boxes are merged in pairs,
// the nodes of the face between the two halves are eliminated, and the
// merged box carries a DtN map on its own boundary, level after level.
// This file fixes that tree for a uniform grid of nb[0] x nb[1] x nb[2]
// boxes: which boxes each merge joins, which faces it eliminates, and how
// the boundary slots of the children map onto it.
#include <algorithm>
#include <utility>

#include "../../include/hps.h"
#include "hps_iface.h"

namespace hps {

namespace {

struct Builder {
    const int* nb;
    int nfaces = 6;
    std::vector<IfNode> tmp;   // merges in creation order
    bool failed = false;

    static IfFace leaf_face(const int c[3], int f)
    {
        const int axis = f / 2;
        IfFace F;
        F.axis = axis;
        F.plane = c[axis] + (f % 2);
        F.c1 = axis == 0 ? c[1] : c[0];
        F.c2 = axis == 2 ? c[1] : c[2];
        return F;
    }

    // Boundary faces of node `id` (leaf: box index; merge: -(k+1)) with slots.
    void faces_of(int id, std::vector<std::pair<IfFace, int>>* out) const
    {
        out->clear();
        if (id >= 0) {
            const int c[3] = {id % nb[0], (id / nb[0]) % nb[1], id / (nb[0] * nb[1])};
            for (int f = 0; f < nfaces; ++f) {
                const IfFace F = leaf_face(c, f);
                if (F.plane > 0 && F.plane < nb[F.axis]) out->push_back({F, f});
            }
        } else {
            const IfNode& N = tmp[-id - 1];
            for (int s = 0; s < (int)N.faces.size(); ++s) out->push_back({N.faces[s], s});
        }
    }

    int height_of(int id) const { return id >= 0 ? 0 : tmp[-id - 1].height; }

    int make(const int lo[3], const int hi[3])
    {
        int len[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
        if (len[0] == 1 && len[1] == 1 && len[2] == 1) return lo[0] + nb[0] * (lo[1] + nb[1] * lo[2]);
        int a = 0;
        for (int k = 1; k < 3; ++k)
            if (len[k] > len[a]) a = k;
        const int s = lo[a] + len[a] / 2;
        int mid_hi[3] = {hi[0], hi[1], hi[2]}, mid_lo[3] = {lo[0], lo[1], lo[2]};
        mid_hi[a] = s;
        mid_lo[a] = s;
        const int ca = make(lo, mid_hi);
        if (failed) return 0;
        const int cb = make(mid_lo, hi);
        if (failed) return 0;
        IfNode N;
        for (int k = 0; k < 3; ++k) { N.lo[k] = lo[k]; N.hi[k] = hi[k]; }
        N.child[0] = ca;
        N.child[1] = cb;
        N.axis = a;
        N.split = s;
        N.height = 1 + std::max(height_of(ca), height_of(cb));
        std::vector<std::pair<IfFace, int>> fa, fb, sa, sb;
        faces_of(ca, &fa);
        faces_of(cb, &fb);
        for (auto& e : fa) {
            if (e.first.axis == a && e.first.plane == s) sa.push_back(e);
            else { N.a1.push_back(e.second); N.faces.push_back(e.first); }
        }
        for (auto& e : fb) {
            if (e.first.axis == a && e.first.plane == s) sb.push_back(e);
            else { N.b2.push_back(e.second); N.faces.push_back(e.first); }
        }
        auto by_face = [](const std::pair<IfFace, int>& x, const std::pair<IfFace, int>& y) { return x.first < y.first; };
        std::sort(sa.begin(), sa.end(), by_face);
        std::sort(sb.begin(), sb.end(), by_face);
        if (sa.size() != sb.size()) { failed = true; return 0; }   // cannot happen on a uniform grid
        for (size_t i = 0; i < sa.size(); ++i) {
            if (!(sa[i].first == sb[i].first)) { failed = true; return 0; }
            N.a3.push_back(sa[i].second);
            N.b3.push_back(sb[i].second);
        }
        tmp.push_back(std::move(N));
        return -(int)tmp.size();
    }
};

}  // namespace

bool build_iface_plan(int p, const int nb[3], IfPlan* out, int nfaces)
{
    if (p < 3 || p > 24 || !nb || nb[0] < 1 || nb[1] < 1 || nb[2] < 1) return false;
    if (nfaces != 6 && !(nfaces == 4 && nb[2] == 1)) return false;
    if ((long long)nb[0] * nb[1] * nb[2] > (1 << 20)) return false;
    IfPlan P;
    P.p = p;
    P.q = p - 2;
    for (int k = 0; k < 3; ++k) P.nb[k] = nb[k];
    P.nbox = nb[0] * nb[1] * nb[2];
    P.nfaces = nfaces;
    Builder B;
    B.nb = nb;
    B.nfaces = nfaces;
    const int lo[3] = {0, 0, 0};
    B.make(lo, nb);
    if (B.failed) return false;
    // leaves
    P.nodes.resize(P.nbox);
    for (int box = 0; box < P.nbox; ++box) {
        IfNode& L = P.nodes[box];
        const int c[3] = {box % nb[0], (box / nb[0]) % nb[1], box / (nb[0] * nb[1])};
        for (int k = 0; k < 3; ++k) { L.lo[k] = c[k]; L.hi[k] = c[k] + 1; }
        L.leaf_iface.resize(nfaces);
        for (int f = 0; f < nfaces; ++f) {
            const IfFace F = Builder::leaf_face(c, f);
            L.leaf_iface[f] = (F.plane > 0 && F.plane < nb[F.axis]) ? 1 : 0;
        }
    }
    // merges ordered by height (then creation order), root last
    const int nm = (int)B.tmp.size();
    std::vector<int> order(nm);
    for (int i = 0; i < nm; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return B.tmp[x].height < B.tmp[y].height; });
    std::vector<int> newid(nm);
    for (int r = 0; r < nm; ++r) newid[order[r]] = P.nbox + r;
    auto remap = [&](int id) { return id >= 0 ? id : newid[-id - 1]; };
    int hmax = 0;
    for (int r = 0; r < nm; ++r) {
        IfNode N = B.tmp[order[r]];
        N.child[0] = remap(N.child[0]);
        N.child[1] = remap(N.child[1]);
        hmax = std::max(hmax, N.height);
        P.nodes.push_back(std::move(N));
    }
    P.levels.assign(hmax, {});
    for (int r = 0; r < nm; ++r) P.levels[P.nodes[P.nbox + r].height - 1].push_back(P.nbox + r);
    *out = std::move(P);
    return true;
}

}  // namespace hps

namespace {

hps_status plan_arrays(const hps::IfPlan& P, int* n_merge, int* n_list, int* nodes, int* lists);

}  // namespace

// The merge tree as plain arrays (host, no GPU): see hps.h.
extern "C" hps_status hps_interface_plan(int p, const int nb[3], int* n_merge, int* n_list, int* nodes, int* lists)
{
    hps::IfPlan P;
    if (!hps::build_iface_plan(p, nb, &P)) return HPS_EINVAL;
    return plan_arrays(P, n_merge, n_list, nodes, lists);
}

extern "C" hps_status hps_interface2d_plan(int p, const int nb[2], int* n_merge, int* n_list, int* nodes, int* lists)
{
    if (!nb) return HPS_EINVAL;
    const int nb3[3] = {nb[0], nb[1], 1};
    hps::IfPlan P;
    if (!hps::build_iface_plan(p, nb3, &P, 4)) return HPS_EINVAL;
    return plan_arrays(P, n_merge, n_list, nodes, lists);
}

namespace {

hps_status plan_arrays(const hps::IfPlan& P, int* n_merge, int* n_list, int* nodes, int* lists)
{
    const int nm = (int)P.nodes.size() - P.nbox;
    int nl = 0;
    for (int r = 0; r < nm; ++r) {
        const hps::IfNode& N = P.nodes[P.nbox + r];
        nl += (int)(N.a1.size() + N.a3.size() + N.b2.size() + N.b3.size());
    }
    if (n_merge) *n_merge = nm;
    if (n_list) *n_list = nl;
    if (!nodes && !lists) return HPS_OK;
    if (!nodes || !lists) return HPS_EINVAL;
    int off = 0;
    for (int r = 0; r < nm; ++r) {
        const hps::IfNode& N = P.nodes[P.nbox + r];
        int* row = nodes + 8 * r;
        row[0] = N.child[0];
        row[1] = N.child[1];
        row[2] = N.height;
        row[3] = N.axis;
        row[4] = (int)N.a1.size();
        row[5] = (int)N.a3.size();
        row[6] = (int)N.b2.size();
        row[7] = off;
        for (int v : N.a1) lists[off++] = v;
        for (int v : N.a3) lists[off++] = v;
        for (int v : N.b2) lists[off++] = v;
        for (int v : N.b3) lists[off++] = v;
    }
    return HPS_OK;
}

}  // namespace
