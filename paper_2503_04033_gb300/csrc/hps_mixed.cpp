// Host side of the two-level solve on box grids of mixed orders p (adaptive
// p; Sec. 6 names adaptivity in the local order as a setting the scheme can
// serve).  Every box keeps its own collocation (Sec. 2.1) and DtN map, which
// hps_leaf_groups builds on the GPU per order.  A face shared by boxes of
// different orders carries its unknowns on the face grid of the higher
// order; a box sees them through polynomial interpolation to its own face
// nodes (P), and its fluxes reach the face grids through the interpolation
// the other way (Q).  The interface system is sum_tau Q_tau T_tau P_tau
// (Sec. 3.1's assembly with the interpolation inserted), its right-hand side
// -sum_tau Q_tau h_tau minus the Dirichlet coupling; the box traces of a
// solution are P_tau applied to it.  Numbering and layout: see hps.h.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/hps.h"

namespace hps {
void cheb_nodes(int p, double* t);
}

namespace {

constexpr int kMixedMaxP = 24;

struct MixedGrid {
    int nx = 0, ny = 0, nz = 0;
    int64_t Fx = 0, Fy = 0, Fz = 0, Dx = 0, Dy = 0, Dz = 0, nfi = 0, nfd = 0;
    std::vector<int> face_p;         // per face (interface faces, then Dirichlet faces)
    std::vector<int64_t> face_off;   // first unknown of each face, and the total
    int64_t n_iface = 0, n_dir = 0;
};

// Face f (x-, x+, y-, y+, z-, z+) of box (bx, by, bz): its index among all
// faces (interface faces first, then the Dirichlet faces).
int64_t face_index(const MixedGrid& g, int bx, int by, int bz, int f, bool* iface)
{
    const int axis = f / 2, side = f % 2;
    const int c[3] = {bx, by, bz};
    const int nax[3] = {g.nx, g.ny, g.nz};
    const int plane = c[axis] + side;
    if (plane == 0 || plane == nax[axis]) {
        const int s = plane == 0 ? 0 : 1;
        *iface = false;
        int64_t id;
        if (axis == 0) id = s + 2 * (int64_t)(by + (int64_t)g.ny * bz);
        else if (axis == 1) id = g.Dx + s + 2 * (int64_t)(bx + (int64_t)g.nx * bz);
        else id = g.Dx + g.Dy + s + 2 * (int64_t)(bx + (int64_t)g.nx * by);
        return g.nfi + id;
    }
    *iface = true;
    if (axis == 0) return (plane - 1) + (int64_t)(g.nx - 1) * (by + (int64_t)g.ny * bz);
    if (axis == 1) return g.Fx + bx + (int64_t)g.nx * ((plane - 1) + (int64_t)(g.ny - 1) * bz);
    return g.Fx + g.Fy + bx + (int64_t)g.nx * (by + (int64_t)g.ny * (plane - 1));
}

void box_coords(const MixedGrid& g, int64_t box, int* bx, int* by, int* bz)
{
    *bx = (int)(box % g.nx);
    *by = (int)((box / g.nx) % g.ny);
    *bz = (int)(box / ((int64_t)g.nx * g.ny));
}

hps_status make_grid(const int nb[3], const int* p_box, MixedGrid& g)
{
    if (!nb || !p_box || nb[0] < 1 || nb[1] < 1 || nb[2] < 1) return HPS_EINVAL;
    g.nx = nb[0]; g.ny = nb[1]; g.nz = nb[2];
    const int64_t nbox = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t b = 0; b < nbox; ++b)
        if (p_box[b] < 3 || p_box[b] > kMixedMaxP) return HPS_EINVAL;
    g.Fx = (int64_t)(g.nx - 1) * g.ny * g.nz;
    g.Fy = (int64_t)g.nx * (g.ny - 1) * g.nz;
    g.Fz = (int64_t)g.nx * g.ny * (g.nz - 1);
    g.Dx = 2 * (int64_t)g.ny * g.nz;
    g.Dy = 2 * (int64_t)g.nx * g.nz;
    g.Dz = 2 * (int64_t)g.nx * g.ny;
    g.nfi = g.Fx + g.Fy + g.Fz;
    g.nfd = g.Dx + g.Dy + g.Dz;
    g.face_p.assign((size_t)(g.nfi + g.nfd), 0);
    for (int64_t b = 0; b < nbox; ++b) {
        int bx, by, bz;
        box_coords(g, b, &bx, &by, &bz);
        for (int f = 0; f < 6; ++f) {
            bool it;
            const int64_t id = face_index(g, bx, by, bz, f, &it);
            if (p_box[b] > g.face_p[id]) g.face_p[id] = p_box[b];
        }
    }
    g.face_off.assign(g.face_p.size() + 1, 0);
    for (size_t i = 0; i < g.face_p.size(); ++i) {
        const int64_t q = g.face_p[i] - 2;
        g.face_off[i + 1] = g.face_off[i] + q * q;
    }
    g.n_iface = g.face_off[(size_t)g.nfi];
    g.n_dir = g.face_off.back() - g.n_iface;
    return HPS_OK;
}

// 1-D Lagrange matrix L [q_dst][q_src] from the q_src interior
// Chebyshev-Lobatto points of order p_src to those of order p_dst.
std::vector<double> lagrange(int p_src, int p_dst)
{
    std::vector<double> ts(p_src), td(p_dst);
    hps::cheb_nodes(p_src, ts.data());
    hps::cheb_nodes(p_dst, td.data());
    const int qs = p_src - 2, qd = p_dst - 2;
    std::vector<double> L((size_t)qd * qs, 1.0);
    for (int i = 0; i < qd; ++i)
        for (int j = 0; j < qs; ++j) {
            double v = 1.0;
            for (int k = 0; k < qs; ++k)
                if (k != j) v *= (td[i + 1] - ts[k + 1]) / (ts[j + 1] - ts[k + 1]);
            L[(size_t)i * qs + j] = v;
        }
    return L;
}

// The face operator of one face of a box: values on the q_dst^2 face nodes
// (face-local, lower free axis fastest) from the q_src^2 ones, as a dense
// [q_dst^2][q_src^2] block (the tensor product of the 1-D Lagrange matrix),
// or empty when the orders agree (identity).
struct FaceOp {
    int qs = 0, qd = 0;
    std::vector<double> A;
};

FaceOp face_op(int p_src, int p_dst)
{
    FaceOp op;
    op.qs = p_src - 2;
    op.qd = p_dst - 2;
    if (p_src == p_dst) return op;
    const std::vector<double> L = lagrange(p_src, p_dst);
    const int qs = op.qs, qd = op.qd, ns = qs * qs, nd = qd * qd;
    op.A.assign((size_t)nd * ns, 0.0);
    for (int bd = 0; bd < qd; ++bd)
        for (int ad = 0; ad < qd; ++ad)
            for (int bs = 0; bs < qs; ++bs)
                for (int as = 0; as < qs; ++as)
                    op.A[(size_t)(ad + qd * bd) * ns + (as + qs * bs)] = L[(size_t)bd * qs + bs] * L[(size_t)ad * qs + as];
    return op;
}

// Per box: for each local face, the face index, its first unknown, its
// order, and the two interpolation operators (P: face grid -> box face
// nodes, Q: box face nodes -> face grid).
struct BoxFaces {
    int64_t fid[6], off[6];
    int pf[6];
    bool iface[6];
    FaceOp P[6], Q[6];
};

void box_faces(const MixedGrid& g, const int* p_box, int64_t box, BoxFaces& bf)
{
    int bx, by, bz;
    box_coords(g, box, &bx, &by, &bz);
    const int p = p_box[box];
    for (int f = 0; f < 6; ++f) {
        bf.fid[f] = face_index(g, bx, by, bz, f, &bf.iface[f]);
        bf.off[f] = g.face_off[(size_t)bf.fid[f]];
        bf.pf[f] = g.face_p[(size_t)bf.fid[f]];
        bf.P[f] = face_op(bf.pf[f], p);
        bf.Q[f] = face_op(p, bf.pf[f]);
    }
}

// y = op x (op identity when empty), lengths qd^2 and qs^2.
void apply(const FaceOp& op, const double* x, double* y)
{
    const int ns = op.qs * op.qs, nd = op.qd * op.qd;
    if (op.A.empty()) {
        std::memcpy(y, x, sizeof(double) * ns);
        return;
    }
    for (int i = 0; i < nd; ++i) {
        double acc = 0.0;
        for (int j = 0; j < ns; ++j) acc += op.A[(size_t)i * ns + j] * x[j];
        y[i] = acc;
    }
}

}  // namespace

extern "C" {

hps_status hps_mixed_layout(const int nb[3], const int* p_box, int64_t* n_iface, int64_t* n_dir, int* face_p,
                            int64_t* face_off)
{
    MixedGrid g;
    hps_status rc = make_grid(nb, p_box, g);
    if (rc != HPS_OK) return rc;
    if (n_iface) *n_iface = g.n_iface;
    if (n_dir) *n_dir = g.n_dir;
    if (face_p) std::memcpy(face_p, g.face_p.data(), sizeof(int) * g.face_p.size());
    if (face_off) std::memcpy(face_off, g.face_off.data(), sizeof(int64_t) * g.face_off.size());
    return HPS_OK;
}

hps_status hps_mixed_face_coords(const int nb[3], const int* p_box, const double lo[3], const double L[3], double* xyz)
{
    if (!lo || !L || !xyz) return HPS_EINVAL;
    MixedGrid g;
    hps_status rc = make_grid(nb, p_box, g);
    if (rc != HPS_OK) return rc;
    const double h[3] = {L[0] / g.nx, L[1] / g.ny, L[2] / g.nz};
    const int64_t nbox = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t b = 0; b < nbox; ++b) {
        int c[3];
        box_coords(g, b, &c[0], &c[1], &c[2]);
        BoxFaces bf;
        box_faces(g, p_box, b, bf);
        for (int f = 0; f < 6; ++f) {
            const int pf = bf.pf[f], q = pf - 2, axis = f / 2;
            const int u = axis == 0 ? 1 : 0, v = axis == 2 ? 1 : 2;   // the free axes, lower first
            std::vector<double> t(pf);
            hps::cheb_nodes(pf, t.data());
            for (int bb = 0; bb < q; ++bb)
                for (int aa = 0; aa < q; ++aa) {
                    double* x = xyz + 3 * (bf.off[f] + aa + (int64_t)q * bb);
                    x[axis] = lo[axis] + h[axis] * (c[axis] + (f % 2));
                    x[u] = lo[u] + h[u] * (c[u] + 0.5 * (t[aa + 1] + 1.0));
                    x[v] = lo[v] + h[v] * (c[v] + 0.5 * (t[bb + 1] + 1.0));
                }
        }
    }
    return HPS_OK;
}

hps_status hps_mixed_assemble(const int nb[3], const int* p_box, const double* const* T, int64_t* nnz, int64_t* rows,
                              int64_t* cols, double* vals, int64_t* nnz_d, int64_t* rows_d, int64_t* cols_d,
                              double* vals_d)
{
    MixedGrid g;
    hps_status rc = make_grid(nb, p_box, g);
    if (rc != HPS_OK) return rc;
    const int64_t nbox = (int64_t)g.nx * g.ny * g.nz;
    const bool fill = rows && cols && vals;
    if (fill && !T) return HPS_EINVAL;
    int64_t k = 0, kd = 0;
    for (int64_t b = 0; b < nbox; ++b) {
        BoxFaces bf;
        box_faces(g, p_box, b, bf);
        const int p = p_box[b], q = p - 2, qq = q * q, m = 6 * qq;
        // the box's block of the system: rows on the face grids of its
        // interface faces, columns on the face grids of all its faces
        for (int fr = 0; fr < 6; ++fr) {
            if (!bf.iface[fr]) continue;
            const int nr = (bf.pf[fr] - 2) * (bf.pf[fr] - 2);
            for (int fc = 0; fc < 6; ++fc) {
                const int nc = (bf.pf[fc] - 2) * (bf.pf[fc] - 2);
                const bool dir = !bf.iface[fc];
                if (!fill || (dir && !(rows_d && cols_d && vals_d))) {
                    (dir ? kd : k) += (int64_t)nr * nc;
                    continue;
                }
                if (!T[b]) return HPS_EINVAL;
                // block = Q_fr T[fr, fc] P_fc
                std::vector<double> Tb((size_t)qq * qq), tmp((size_t)qq * nc), blk((size_t)nr * nc);
                for (int i = 0; i < qq; ++i)
                    for (int j = 0; j < qq; ++j) Tb[(size_t)i * qq + j] = T[b][(size_t)(fr * qq + i) * m + fc * qq + j];
                // tmp = T_blk P_fc (column j: T_blk times column j of P_fc),
                // then blk = Q_fr tmp; identity operators are skipped
                if (bf.P[fc].A.empty()) {
                    tmp = Tb;
                } else {
                    std::vector<double> e(nc), pc(qq);
                    for (int j = 0; j < nc; ++j) {
                        std::fill(e.begin(), e.end(), 0.0);
                        e[j] = 1.0;
                        apply(bf.P[fc], e.data(), pc.data());
                        for (int i = 0; i < qq; ++i) {
                            double acc = 0.0;
                            for (int l = 0; l < qq; ++l) acc += Tb[(size_t)i * qq + l] * pc[l];
                            tmp[(size_t)i * nc + j] = acc;
                        }
                    }
                }
                if (bf.Q[fr].A.empty()) {
                    blk = tmp;
                } else {
                    std::vector<double> colv(qq), out(nr);
                    for (int j = 0; j < nc; ++j) {
                        for (int i = 0; i < qq; ++i) colv[i] = tmp[(size_t)i * nc + j];
                        apply(bf.Q[fr], colv.data(), out.data());
                        for (int i = 0; i < nr; ++i) blk[(size_t)i * nc + j] = out[i];
                    }
                }
                for (int i = 0; i < nr; ++i)
                    for (int j = 0; j < nc; ++j) {
                        const int64_t r = bf.off[fr] + i;
                        const int64_t c = bf.off[fc] + j;
                        if (dir) {
                            rows_d[kd] = r; cols_d[kd] = c - g.n_iface; vals_d[kd] = blk[(size_t)i * nc + j]; ++kd;
                        } else {
                            rows[k] = r; cols[k] = c; vals[k] = blk[(size_t)i * nc + j]; ++k;
                        }
                    }
            }
        }
    }
    if (nnz) *nnz = k;
    if (nnz_d) *nnz_d = kd;
    return HPS_OK;
}

hps_status hps_mixed_reduce(const int nb[3], const int* p_box, const double* const* hflux, double* r)
{
    if (!hflux || !r) return HPS_EINVAL;
    MixedGrid g;
    hps_status rc = make_grid(nb, p_box, g);
    if (rc != HPS_OK) return rc;
    std::memset(r, 0, sizeof(double) * (size_t)(g.n_iface + g.n_dir));
    const int64_t nbox = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t b = 0; b < nbox; ++b) {
        if (!hflux[b]) return HPS_EINVAL;
        BoxFaces bf;
        box_faces(g, p_box, b, bf);
        const int q = p_box[b] - 2, qq = q * q;
        for (int f = 0; f < 6; ++f) {
            const int nf = (bf.pf[f] - 2) * (bf.pf[f] - 2);
            std::vector<double> out(nf);
            apply(bf.Q[f], hflux[b] + (size_t)f * qq, out.data());
            for (int i = 0; i < nf; ++i) r[bf.off[f] + i] += out[i];
        }
    }
    return HPS_OK;
}

hps_status hps_mixed_traces(const int nb[3], const int* p_box, const double* u, double* const* ub)
{
    if (!u || !ub) return HPS_EINVAL;
    MixedGrid g;
    hps_status rc = make_grid(nb, p_box, g);
    if (rc != HPS_OK) return rc;
    const int64_t nbox = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t b = 0; b < nbox; ++b) {
        if (!ub[b]) return HPS_EINVAL;
        BoxFaces bf;
        box_faces(g, p_box, b, bf);
        const int q = p_box[b] - 2, qq = q * q;
        for (int f = 0; f < 6; ++f) apply(bf.P[f], u + bf.off[f], ub[b] + (size_t)f * qq);
    }
    return HPS_OK;
}

}  // extern "C"
