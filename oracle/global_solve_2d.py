"""Global two-level solve on a uniform 2-D grid of boxes, for end-to-end checks.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).

The 2-D form of ``oracle.global_solve``: ``InterfaceGrid2D`` numbers the
interface and Dirichlet edge nodes of an nx x ny grid of boxes (edges of each
normal axis in turn, box-row order, q nodes per edge in the order of their
free index); ``hps_solve_2d`` runs the two stages with the oracle's 2-D leaf
routines and a host sparse LU of the interface system (Sec. 3.1 assembly);
``dense_global_solve_2d`` assembles the full collocation system (interior
rows, flux-sum rows on shared edges, identity rows on Dirichlet nodes) and
solves it densely, the brute-force check.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import leaf_dtn_2d, leaf_matrix_2d, leaf_particular_2d, node_coords_2d, sizes_2d


class InterfaceGrid2D:
    """Box (bx, by) has index bx + nx by and spans [lo + (bx, by) h, lo + (bx+1, by+1) h]."""

    def __init__(self, p: int, nb, lo=(0.0, 0.0), L=(1.0, 1.0)):
        self.p = p
        self.q = p - 2
        self.nb = tuple(int(v) for v in nb)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.h = np.asarray(L, dtype=np.float64) / np.asarray(self.nb, dtype=np.float64)
        nx, ny = self.nb
        self.Fx, self.Fy = (nx - 1) * ny, nx * (ny - 1)
        self.Dx, self.Dy = 2 * ny, 2 * nx
        self.n_iface = (self.Fx + self.Fy) * self.q
        self.n_dir = (self.Dx + self.Dy) * self.q

    @property
    def nbox(self) -> int:
        return self.nb[0] * self.nb[1]

    def box_coords(self, box: int):
        return box % self.nb[0], box // self.nb[0]

    def box_lo(self, box: int) -> np.ndarray:
        return self.lo + np.asarray(self.box_coords(box), dtype=np.float64) * self.h

    def edge_id(self, box: int, f: int):
        """(is_interface, edge id) of local edge f (x-, x+, y-, y+)."""
        nx, ny = self.nb
        c = self.box_coords(box)
        axis, side = f // 2, f % 2
        plane = c[axis] + side
        if plane == 0 or plane == self.nb[axis]:
            s = 0 if plane == 0 else 1
            if axis == 0:
                return False, s + 2 * c[1]
            return False, self.Dx + s + 2 * c[0]
        if axis == 0:
            return True, (plane - 1) + (nx - 1) * c[1]
        return True, self.Fx + c[0] + nx * (plane - 1)

    def local_to_global(self, box: int):
        """For the m edge nodes of a box: (is_interface[m], global id[m])."""
        q = self.q
        isi = np.empty(4 * q, dtype=bool)
        gid = np.empty(4 * q, dtype=np.int64)
        for f in range(4):
            it, eid = self.edge_id(box, f)
            isi[f * q:(f + 1) * q] = it
            gid[f * q:(f + 1) * q] = eid * q + np.arange(q)
        return isi, gid

    def kept_coords(self, box: int):
        """(interior coordinates [n, 2], edge-node coordinates [m, 2]) of a box."""
        p, q = self.p, self.q
        xy = node_coords_2d(p, self.box_lo(box), self.h)
        ii = np.array([(i + 1) + p * (j + 1) for j in range(q) for i in range(q)])
        e = p - 1
        fi = []
        for f in range(4):
            side = 0 if f % 2 == 0 else e
            for a in range(1, q + 1):
                fi.append(side + p * a if f // 2 == 0 else a + p * side)
        return xy[ii], xy[np.asarray(fi)]

    def dirichlet_coords(self) -> np.ndarray:
        out = np.empty((self.n_dir, 2))
        for box in range(self.nbox):
            _, xe = self.kept_coords(box)
            isi, gid = self.local_to_global(box)
            out[gid[~isi]] = xe[~isi]
        return out


def hps_solve_2d(grid: InterfaceGrid2D, kappa: float, b_boxes, f_boxes, g_dir):
    """Two-level solve with per-box b and f [p^2] (grid order) and Dirichlet
    values g_dir [n_dir]: per-box T, S, v, h; the interface system
    T u_b = -sum h - T_ID g; host sparse LU; u_i = v + S u_b."""
    p, (n, m) = grid.p, sizes_2d(grid.p)
    rows, cols, vals = [], [], []
    rhs = np.zeros(grid.n_iface)
    keep = []
    for box in range(grid.nbox):
        T, S, info = leaf_dtn_2d(p, grid.h, kappa, b_boxes[box])
        assert info == 0
        v, hf, info = leaf_particular_2d(p, grid.h, kappa, b_boxes[box], f_boxes[box][None, :])
        assert info == 0
        isi, gid = grid.local_to_global(box)
        ri, rd = np.nonzero(isi)[0], np.nonzero(~isi)[0]
        rr, cc = np.meshgrid(gid[ri], gid[ri], indexing="ij")
        rows.append(rr.reshape(-1)); cols.append(cc.reshape(-1)); vals.append(T[np.ix_(ri, ri)].reshape(-1))
        np.add.at(rhs, gid[ri], -hf[0, ri])
        if len(rd):
            np.add.at(rhs, gid[ri], -T[np.ix_(ri, rd)] @ g_dir[gid[rd]])
        keep.append((S, v[0], isi, gid))
    Tg = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(grid.n_iface, grid.n_iface)).tocsc()
    u_iface = spla.splu(Tg).solve(rhs) if grid.n_iface else np.zeros(0)
    u_int = np.empty((grid.nbox, n))
    for box, (S, v, isi, gid) in enumerate(keep):
        ub = np.empty(m)
        ub[isi] = u_iface[gid[isi]]
        ub[~isi] = g_dir[gid[~isi]]
        u_int[box] = v + S @ ub
    return {"u_iface": u_iface, "u_int": u_int}


def dense_global_solve_2d(grid: InterfaceGrid2D, kappa: float, b_boxes, f_boxes, g_dir):
    """Brute force: unknowns are every box's interior nodes, then interface
    nodes, then Dirichlet nodes; rows are each box's interior rows of A^tau,
    on each shared edge node the sum of both boxes' outward normal
    derivatives = 0, and u = g on Dirichlet nodes."""
    p, (n, m) = grid.p, sizes_2d(grid.p)
    nbox = grid.nbox
    off_i, off_d = nbox * n, nbox * n + grid.n_iface
    Ntot = off_d + grid.n_dir
    G = np.zeros((Ntot, Ntot))
    rhs = np.zeros(Ntot)
    q = p - 2
    ii = np.array([(i + 1) + p * (j + 1) for j in range(q) for i in range(q)])
    for box in range(nbox):
        A = leaf_matrix_2d(p, grid.h, kappa, b_boxes[box])
        isi, gid = grid.local_to_global(box)
        glob = np.concatenate([box * n + np.arange(n), np.where(isi, off_i + gid, off_d + gid)])
        G[np.ix_(glob[:n], glob)] += A[:n, :]
        rhs[glob[:n]] += f_boxes[box][ii]
        fr = np.nonzero(isi)[0]
        G[np.ix_(off_i + gid[fr], glob)] += A[n + fr, :]
    d = np.arange(grid.n_dir)
    G[off_d + d, :] = 0.0
    G[off_d + d, off_d + d] = 1.0
    rhs[off_d + d] = g_dir
    u = np.linalg.solve(G, rhs)
    return {"u_int": u[:off_i].reshape(nbox, n), "u_iface": u[off_i:off_d]}
