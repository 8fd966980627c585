"""Two-level solve on a box grid of mixed orders p (adaptive p), FP64.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).

The paper's closing section (Sec. 6) names adaptivity in the local order p
as a setting the two-level scheme can in principle serve.  Reading used
here (the paper gives no formulation): each box keeps its own collocation
of order p_tau (Sec. 2.1) and its own DtN map; a face shared by boxes of
different orders carries its unknowns on the face grid of the higher order
(the interior Chebyshev-Lobatto points of that order in each free
direction), the lower-order box sees them through polynomial interpolation
to its own face nodes, and its fluxes are interpolated back to the face
grid before the flux balance.  With P_tau (face unknowns to the box's face
nodes) and Q_tau (the box's face nodes to the face grids), box tau adds
Q_tau (T_tau P_tau u + h_tau) to the balance of every face unknown it
touches (Sec. 3.1's assembly with the interpolation operators inserted).
Faces on the domain boundary carry the Dirichlet data on the box's own face
nodes.  With a single order P_tau = Q_tau = I and this is the uniform
two-level solve.

Numbering: faces as in ``InterfaceGrid`` (interface faces of each normal axis
in turn, then the Dirichlet faces), each face's unknowns contiguous in
face-local order (lower free axis fastest), faces one after another.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import leaf_dtn, leaf_particular, node_coords, nodes, sizes
from .global_solve import InterfaceGrid, face_node_grid_indices


def lagrange_1d(src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """L [len(dst), len(src)]: values at dst of the polynomial through the
    points src (the Lagrange basis written out as products)."""
    L = np.ones((len(dst), len(src)))
    for j, xj in enumerate(src):
        for k, xk in enumerate(src):
            if k != j:
                L[:, j] *= (dst - xk) / (xj - xk)
    return L


def face_points(p: int) -> np.ndarray:
    """The q = p - 2 interior Chebyshev-Lobatto points of order p on [-1, 1]."""
    return nodes(p)[1:-1]


def face_interp(p_src: int, p_dst: int) -> np.ndarray:
    """[q_dst^2, q_src^2]: face-local values (lower free axis fastest) of the
    tensor polynomial through the order-p_src face nodes at the order-p_dst
    face nodes."""
    L = lagrange_1d(face_points(p_src), face_points(p_dst))
    return np.kron(L, L)


class MixedGrid:
    """Uniform boxes of an nx x ny x nz grid with per-box orders p_box."""

    def __init__(self, p_box, nb, lo=(0.0, 0.0, 0.0), L=(1.0, 1.0, 1.0)):
        self.p_box = np.asarray(p_box, dtype=np.int64)
        self.nb = tuple(int(v) for v in nb)
        self.g = InterfaceGrid(4, nb, lo, L)          # face ids and box geometry only
        self.h = self.g.h
        assert len(self.p_box) == self.g.nbox
        nf = self.g.n_iface_faces + self.g.n_dir_faces
        self.face_p = np.zeros(nf, dtype=np.int64)
        for box in range(self.g.nbox):
            for f in range(6):
                it, fid = self.g.face_id(box, f)
                gid = fid if it else self.g.n_iface_faces + fid
                self.face_p[gid] = max(self.face_p[gid], self.p_box[box])
        qq = (self.face_p - 2) ** 2
        self.face_off = np.concatenate([[0], np.cumsum(qq)])
        self.n_iface = int(self.face_off[self.g.n_iface_faces])
        self.n_dir = int(self.face_off[-1] - self.n_iface)

    @property
    def nbox(self) -> int:
        return self.g.nbox

    def box_lo(self, box: int) -> np.ndarray:
        return self.g.box_lo(box)

    def box_faces(self, box: int):
        """Per local face f: (is_interface, global face index, face order)."""
        out = []
        for f in range(6):
            it, fid = self.g.face_id(box, f)
            gid = fid if it else self.g.n_iface_faces + fid
            out.append((it, gid, int(self.face_p[gid])))
        return out

    def box_maps(self, box: int):
        """(P [m, n_all], Q [n_all, m]) of a box as sparse matrices over all
        face unknowns (interface first, then Dirichlet, n_all = n_iface +
        n_dir): P takes them to the box's face nodes, Q takes values on the
        box's face nodes to the face grids."""
        p = int(self.p_box[box])
        q = p - 2
        qq = q * q
        n_all = self.n_iface + self.n_dir
        P = sp.lil_matrix((6 * qq, n_all))
        Q = sp.lil_matrix((n_all, 6 * qq))
        for f, (_, gid, pf) in enumerate(self.box_faces(box)):
            o = int(self.face_off[gid])
            qf = (pf - 2) ** 2
            Pf = face_interp(pf, p) if pf != p else np.eye(qq)
            Qf = face_interp(p, pf) if pf != p else np.eye(qq)
            P[f * qq:(f + 1) * qq, o:o + qf] = Pf
            Q[o:o + qf, f * qq:(f + 1) * qq] = Qf
        return P.tocsr(), Q.tocsr()

    def face_node_coords(self) -> np.ndarray:
        """Coordinates [n_iface + n_dir, 3] of every face unknown."""
        out = np.empty((self.n_iface + self.n_dir, 3))
        for box in range(self.nbox):
            lo = self.box_lo(box)
            for f, (_, gid, pf) in enumerate(self.box_faces(box)):
                xyz = node_coords(int(pf), lo, self.h)
                q = pf - 2
                fi = face_node_grid_indices(int(pf))[f * q * q:(f + 1) * q * q]
                o = int(self.face_off[gid])
                out[o:o + q * q] = xyz[fi]
        return out


def mixed_solve(grid: MixedGrid, kappa: float, b_fn, f_fn, g_fn):
    """The two-level solve on a mixed-order grid with the oracle's leaf
    routines and a host sparse LU.  Returns the face unknowns, the per-box
    interior solutions (list, box order) and the assembled system."""
    ni, nd = grid.n_iface, grid.n_dir
    g_all = g_fn(grid.face_node_coords())
    g_dir = g_all[ni:]
    A = sp.csr_matrix((ni + nd, ni + nd))
    rhs = np.zeros(ni + nd)
    keep = []
    for box in range(grid.nbox):
        p = int(grid.p_box[box])
        x = node_coords(p, grid.box_lo(box), grid.h)
        b, f = b_fn(x), f_fn(x)
        T, S, info = leaf_dtn(p, grid.h, kappa, b)
        assert info == 0, f"box {box}: singular A_ii"
        v, hf, info = leaf_particular(p, grid.h, kappa, b, f[None, :])
        assert info == 0
        P, Q = grid.box_maps(box)
        A = A + Q @ sp.csr_matrix(T) @ P
        rhs -= Q @ hf[0]
        keep.append((S, v[0], P))
    A = A.tocsc()
    Aii, Aid = A[:ni, :ni], A[:ni, ni:]
    u_if = spla.splu(Aii).solve(rhs[:ni] - Aid @ g_dir) if ni else np.zeros(0)
    u_all = np.concatenate([u_if, g_dir])
    u_int = [v + S @ (P @ u_all) for (S, v, P) in keep]
    return {"u_iface": u_if, "g_dir": g_dir, "u_int": u_int, "A": A, "rhs": rhs}
