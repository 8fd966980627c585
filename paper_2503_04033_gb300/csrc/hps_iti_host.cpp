// Host assembly of the two-level system on ItI maps (the ItI variant of HPS,
// Sec. 6).  Unknowns: every box's incoming impedance data on its m face
// nodes, in box order (index box m + r, r the box's face-node order).  On a
// face shared by boxes tau and sigma the incoming data of one side is minus
// the outgoing data of the other (u and the flux continuous, the normals
// opposite): f_tau + R_sigma f_sigma = -hout_sigma at the matching node (the
// same within-face index on the opposite local face).  On a Dirichlet face
// u = g gives (R_tau - I) f_tau = -hout_tau - 2 i eta g.  Complex values are
// interleaved (real, imaginary) doubles.  Numbering of boxes: see hps.h.
#include <cstdint>
#include <cstring>

#include "../../include/hps.h"

namespace {

constexpr int kItiHostMaxP = 16;

struct Box3 {
    int nx, ny, nz;
};

// Neighbour of box (bx, by, bz) across local face f, or -1 on the boundary.
int64_t neighbour(const Box3& g, int bx, int by, int bz, int f)
{
    int c[3] = {bx, by, bz};
    const int n[3] = {g.nx, g.ny, g.nz};
    const int axis = f / 2;
    c[axis] += (f % 2) ? 1 : -1;
    if (c[axis] < 0 || c[axis] >= n[axis]) return -1;
    return c[0] + (int64_t)g.nx * (c[1] + (int64_t)g.ny * c[2]);
}

bool make(int p, const int nb[3], Box3& g, int& m)
{
    if (p < 4 || p > kItiHostMaxP || !nb || nb[0] < 1 || nb[1] < 1 || nb[2] < 1) return false;
    g.nx = nb[0]; g.ny = nb[1]; g.nz = nb[2];
    m = 6 * (p - 2) * (p - 2);
    return true;
}

}  // namespace

extern "C" {

hps_status hps_iti_assemble(int p, const int nb[3], const double* R, int64_t* nnz, int64_t* rows, int64_t* cols,
                            double* vals)
{
    Box3 g;
    int m;
    if (!make(p, nb, g, m)) return HPS_EINVAL;
    const int qq = m / 6;
    const int64_t nbox = (int64_t)g.nx * g.ny * g.nz;
    const bool fill = rows && cols && vals;
    if (fill && !R) return HPS_EINVAL;
    int64_t k = 0;
    for (int64_t box = 0; box < nbox; ++box) {
        const int bx = (int)(box % g.nx), by = (int)((box / g.nx) % g.ny), bz = (int)(box / ((int64_t)g.nx * g.ny));
        for (int r = 0; r < m; ++r) {
            const int f = r / qq, s = r - f * qq;
            const int64_t sg = neighbour(g, bx, by, bz, f);
            const int64_t row = box * m + r;
            if (sg >= 0) {   // f_tau[r] + sum_l R_sigma[r'][l] f_sigma[l]
                const int rp = (f ^ 1) * qq + s;
                if (fill) {
                    rows[k] = row; cols[k] = row; vals[2 * k] = 1.0; vals[2 * k + 1] = 0.0;
                }
                ++k;
                for (int l = 0; l < m; ++l, ++k)
                    if (fill) {
                        rows[k] = row;
                        cols[k] = sg * m + l;
                        const double* e = R + 2 * ((sg * m + rp) * (int64_t)m + l);
                        vals[2 * k] = e[0];
                        vals[2 * k + 1] = e[1];
                    }
            } else {         // sum_l (R_tau[r][l] - delta_rl) f_tau[l]
                for (int l = 0; l < m; ++l, ++k)
                    if (fill) {
                        rows[k] = row;
                        cols[k] = box * m + l;
                        const double* e = R + 2 * ((box * m + r) * (int64_t)m + l);
                        vals[2 * k] = e[0] - (l == r ? 1.0 : 0.0);
                        vals[2 * k + 1] = e[1];
                    }
            }
        }
    }
    if (nnz) *nnz = k;
    return HPS_OK;
}

hps_status hps_iti_rhs(int p, const int nb[3], double eta, const double* hout, const double* g_face, double* rhs)
{
    Box3 g;
    int m;
    if (!make(p, nb, g, m) || !rhs || !(eta != 0.0)) return HPS_EINVAL;
    const int qq = m / 6;
    const int64_t nbox = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t box = 0; box < nbox; ++box) {
        const int bx = (int)(box % g.nx), by = (int)((box / g.nx) % g.ny), bz = (int)(box / ((int64_t)g.nx * g.ny));
        for (int r = 0; r < m; ++r) {
            const int f = r / qq, s = r - f * qq;
            const int64_t sg = neighbour(g, bx, by, bz, f);
            double* o = rhs + 2 * (box * m + r);
            if (sg >= 0) {
                const int rp = (f ^ 1) * qq + s;
                o[0] = hout ? -hout[2 * (sg * m + rp)] : 0.0;
                o[1] = hout ? -hout[2 * (sg * m + rp) + 1] : 0.0;
            } else {
                const double gv = g_face ? g_face[box * m + r] : 0.0;
                o[0] = hout ? -hout[2 * (box * m + r)] : 0.0;
                o[1] = (hout ? -hout[2 * (box * m + r) + 1] : 0.0) - 2.0 * eta * gv;
            }
        }
    }
    return HPS_OK;
}

}  // extern "C"
