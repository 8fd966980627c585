// Host assembly of the interface system from the leaf DtN blocks (Sec. 3.1:
// "row and column index arrays that align each T^tau to the subsets of u_b
// that reside on the box boundary"; Algorithm 1 adds each T^tau to its slot
// of the global sparse T).  Numbering convention: see hps.h.
#include <cstdint>
#include <cstring>

#include "../../include/hps.h"

namespace {

struct Grid {
    int nx, ny, nz, q;
    int64_t Fx, Fy, Fz, Dx, Dy, Dz;
};

// Face f (x-, x+, y-, y+, z-, z+) of box (bx, by, bz): interface or Dirichlet
// face, and its id.
void face_of(const Grid& g, int bx, int by, int bz, int f, bool* iface, int64_t* id)
{
    const int axis = f / 2, side = f % 2;
    const int c[3] = {bx, by, bz};
    const int nax[3] = {g.nx, g.ny, g.nz};
    const int plane = c[axis] + side;
    if (plane == 0 || plane == nax[axis]) {
        const int s = plane == 0 ? 0 : 1;
        *iface = false;
        if (axis == 0) *id = s + 2 * (int64_t)(by + (int64_t)g.ny * bz);
        else if (axis == 1) *id = g.Dx + s + 2 * (int64_t)(bx + (int64_t)g.nx * bz);
        else *id = g.Dx + g.Dy + s + 2 * (int64_t)(bx + (int64_t)g.nx * by);
        return;
    }
    *iface = true;
    if (axis == 0) *id = (plane - 1) + (int64_t)(g.nx - 1) * (by + (int64_t)g.ny * bz);
    else if (axis == 1) *id = g.Fx + bx + (int64_t)g.nx * ((plane - 1) + (int64_t)(g.ny - 1) * bz);
    else *id = g.Fx + g.Fy + bx + (int64_t)g.nx * (by + (int64_t)g.ny * (plane - 1));
}

}  // namespace

extern "C" hps_status hps_assemble_interface_blocks(int p, const int nb[3], const double* T_host, int64_t* nnz,
                                                    int64_t* rows, int64_t* cols, double* vals, int64_t* nnz_d,
                                                    int64_t* rows_d, int64_t* cols_d, double* vals_d,
                                                    int64_t* n_iface, int64_t* n_dir)
{
    if (p < 3 || p > 24 || !nb || nb[0] < 1 || nb[1] < 1 || nb[2] < 1) return HPS_EINVAL;
    Grid g;
    g.nx = nb[0]; g.ny = nb[1]; g.nz = nb[2]; g.q = p - 2;
    g.Fx = (int64_t)(g.nx - 1) * g.ny * g.nz;
    g.Fy = (int64_t)g.nx * (g.ny - 1) * g.nz;
    g.Fz = (int64_t)g.nx * g.ny * (g.nz - 1);
    g.Dx = 2 * (int64_t)g.ny * g.nz;
    g.Dy = 2 * (int64_t)g.nx * g.nz;
    g.Dz = 2 * (int64_t)g.nx * g.ny;
    const int64_t qq = (int64_t)g.q * g.q, m = 6 * qq;
    const int64_t nbox = (int64_t)g.nx * g.ny * g.nz;
    // Count: per box, (#interface face nodes)^2 and (#iface)(#dirichlet) entries.
    int64_t cnt = 0, cnt_d = 0;
    for (int64_t box = 0; box < nbox; ++box) {
        const int bx = (int)(box % g.nx), by = (int)((box / g.nx) % g.ny), bz = (int)(box / ((int64_t)g.nx * g.ny));
        int ni = 0;
        for (int f = 0; f < 6; ++f) {
            bool it; int64_t id;
            face_of(g, bx, by, bz, f, &it, &id);
            ni += it ? 1 : 0;
        }
        cnt += (int64_t)ni * qq * ni * qq;
        cnt_d += (int64_t)ni * qq * (6 - ni) * qq;
    }
    if (n_iface) *n_iface = (g.Fx + g.Fy + g.Fz) * qq;
    if (n_dir) *n_dir = (g.Dx + g.Dy + g.Dz) * qq;
    if (nnz) *nnz = cnt;
    if (nnz_d) *nnz_d = cnt_d;
    const bool want = rows && cols && vals;
    const bool want_d = rows_d && cols_d && vals_d;
    if (!want && !want_d) return HPS_OK;
    if (!T_host) return HPS_EINVAL;
    int64_t e = 0, ed = 0;
    bool isi[6];
    int64_t fid[6];
    for (int64_t box = 0; box < nbox; ++box) {
        const int bx = (int)(box % g.nx), by = (int)((box / g.nx) % g.ny), bz = (int)(box / ((int64_t)g.nx * g.ny));
        for (int f = 0; f < 6; ++f) face_of(g, bx, by, bz, f, &isi[f], &fid[f]);
        const double* Tb = T_host + box * m * m;
        for (int64_t r = 0; r < m; ++r) {
            const int fr = (int)(r / qq);
            if (!isi[fr]) continue;
            const int64_t grow = fid[fr] * qq + r % qq;
            for (int64_t c = 0; c < m; ++c) {
                const int fc = (int)(c / qq);
                const int64_t gcol = fid[fc] * qq + c % qq;
                if (isi[fc]) {
                    if (want) { rows[e] = grow; cols[e] = gcol; vals[e] = Tb[r * m + c]; }
                    ++e;
                } else {
                    if (want_d) { rows_d[ed] = grow; cols_d[ed] = gcol; vals_d[ed] = Tb[r * m + c]; }
                    ++ed;
                }
            }
        }
    }
    return HPS_OK;
}
