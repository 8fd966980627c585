"""Global two-level solve on a uniform box grid, for end-to-end checks.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).

* ``InterfaceGrid`` numbers the interface and Dirichlet face nodes of an
  nx x ny x nz grid of leaf boxes.  The numbering is the library's documented
  convention, written out here independently (faces of each normal axis in
  turn, box-column order, q^2 nodes per face in face-local order).
* ``hps_solve`` runs the paper's two stages (Algorithms 1 and 2) with the
  oracle's leaf routines: per-box T, S, v, h; assembly of the sparse interface
  system T u_b = -sum h - T_ID g (Sec. 3.1, "row and column index arrays");
  a plain host sparse LU (the stand-in for MUMPS, Sec. 3.2); reconstruction
  u_i = v + S u_b.
* ``dense_global_solve`` is the brute-force check: it assembles the full
  collocation system of Eq. 3/Eq. 4 (interior PDE rows, flux-sum rows on the
  shared faces, identity rows for Dirichlet nodes) with no static condensation
  and solves it densely.  The two are algebraically the same discrete system.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import leaf_dtn, leaf_matrix, leaf_particular, node_coords, sizes


class InterfaceGrid:
    """Face-node numbering for a uniform grid of leaf boxes.

    Box (bx, by, bz) has index bx + nx (by + ny bz) and spans
    [lo + (bx, by, bz) * h, lo + (bx+1, by+1, bz+1) * h].
    """

    def __init__(self, p: int, nb, lo=(0.0, 0.0, 0.0), L=(1.0, 1.0, 1.0)):
        self.p = p
        self.q = p - 2
        self.nb = tuple(int(v) for v in nb)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.h = np.asarray(L, dtype=np.float64) / np.asarray(self.nb, dtype=np.float64)
        nx, ny, nz = self.nb
        self.Fx, self.Fy, self.Fz = (nx - 1) * ny * nz, nx * (ny - 1) * nz, nx * ny * (nz - 1)
        self.Dx, self.Dy, self.Dz = 2 * ny * nz, 2 * nx * nz, 2 * nx * ny
        self.n_iface_faces = self.Fx + self.Fy + self.Fz
        self.n_dir_faces = self.Dx + self.Dy + self.Dz
        self.n_iface = self.n_iface_faces * self.q * self.q
        self.n_dir = self.n_dir_faces * self.q * self.q

    @property
    def nbox(self) -> int:
        nx, ny, nz = self.nb
        return nx * ny * nz

    def box_coords(self, box: int):
        nx, ny, _ = self.nb
        return box % nx, (box // nx) % ny, box // (nx * ny)

    def box_lo(self, box: int) -> np.ndarray:
        return self.lo + np.asarray(self.box_coords(box), dtype=np.float64) * self.h

    def face_id(self, box: int, f: int):
        """(is_interface, face id) of local face f (x-, x+, y-, y+, z-, z+)."""
        nx, ny, nz = self.nb
        c = self.box_coords(box)
        axis, side = f // 2, f % 2
        plane = c[axis] + side
        nax = self.nb[axis]
        if plane == 0 or plane == nax:
            s = 0 if plane == 0 else 1
            if axis == 0:
                return False, s + 2 * (c[1] + ny * c[2])
            if axis == 1:
                return False, self.Dx + s + 2 * (c[0] + nx * c[2])
            return False, self.Dx + self.Dy + s + 2 * (c[0] + nx * c[1])
        if axis == 0:
            return True, (plane - 1) + (nx - 1) * (c[1] + ny * c[2])
        if axis == 1:
            return True, self.Fx + c[0] + nx * ((plane - 1) + (ny - 1) * c[2])
        return True, self.Fx + self.Fy + c[0] + nx * (c[1] + ny * (plane - 1))

    def local_to_global(self, box: int):
        """For the m face nodes of a box: (is_interface[m], global id[m])."""
        qq = self.q * self.q
        isi = np.empty(6 * qq, dtype=bool)
        gid = np.empty(6 * qq, dtype=np.int64)
        for f in range(6):
            it, fid = self.face_id(box, f)
            isi[f * qq:(f + 1) * qq] = it
            gid[f * qq:(f + 1) * qq] = fid * qq + np.arange(qq)
        return isi, gid

    def dirichlet_coords(self) -> np.ndarray:
        """Coordinates [n_dir, 3] of the Dirichlet face nodes."""
        out = np.empty((self.n_dir, 3))
        p, qq = self.p, self.q * self.q
        for box in range(self.nbox):
            xyz = node_coords(p, self.box_lo(box), self.h)
            isi, gid = self.local_to_global(box)
            fx = face_node_grid_indices(p)
            for r in range(6 * qq):
                if not isi[r]:
                    out[gid[r]] = xyz[fx[r]]
        return out


def face_node_grid_indices(p: int) -> np.ndarray:
    """Grid index (i + p j + p^2 k) of each of the m face nodes, in kept order."""
    q = p - 2
    e = p - 1
    out = []
    for f in range(6):
        axis, side = f // 2, (0 if f % 2 == 0 else e)
        for bb in range(1, q + 1):
            for aa in range(1, q + 1):
                if axis == 0:
                    i, j, k = side, aa, bb
                elif axis == 1:
                    i, j, k = aa, side, bb
                else:
                    i, j, k = aa, bb, side
                out.append(i + p * j + p * p * k)
    return np.asarray(out, dtype=np.int64)


def interior_grid_indices(p: int) -> np.ndarray:
    """Grid index of each of the n interior nodes, in interior order."""
    q = p - 2
    r = np.arange(1, q + 1)
    k, j, i = np.meshgrid(r, r, r, indexing="ij")
    return (i + p * j + p * p * k).reshape(-1).astype(np.int64)


def hps_solve(grid: InterfaceGrid, kappa: float, b_fn, f_fn, g_fn):
    """Two-level HPS solve with the oracle's leaf routines.

    b_fn, f_fn, g_fn map an [N,3] coordinate array to values.  Returns a dict
    with the interface solution, per-box interior solutions and coordinates.
    """
    p = grid.p
    xyz = [node_coords(p, grid.box_lo(box), grid.h) for box in range(grid.nbox)]
    g_dir = g_fn(grid.dirichlet_coords()) if grid.n_dir else np.zeros(0)
    return hps_solve_boxes(grid, kappa, [b_fn(x) for x in xyz], [f_fn(x) for x in xyz], g_dir)


def hps_solve_boxes(grid: InterfaceGrid, kappa: float, b_boxes, f_boxes, g_dir, beta_boxes=None):
    """hps_solve with b and f given per box as nodal arrays [p^3] (grid order)
    and the Dirichlet values g_dir [n_dir]; beta_boxes (per box [3, p^3], or
    None) adds the first-order term div(beta u) to the operator."""
    p, (n, m) = grid.p, sizes(grid.p)
    nbox = grid.nbox
    rows, cols, vals = [], [], []
    rhs = np.zeros(grid.n_iface)
    S_all, v_all, maps = [], [], []
    for box in range(nbox):
        b = b_boxes[box]
        f = f_boxes[box]
        beta = beta_boxes[box] if beta_boxes is not None else None
        T, S, info = leaf_dtn(p, grid.h, kappa, b, beta=beta)
        assert info == 0, f"box {box}: singular A_ii"
        v, hf, info = leaf_particular(p, grid.h, kappa, b, f[None, :], beta=beta)
        assert info == 0
        isi, gid = grid.local_to_global(box)
        ri = np.nonzero(isi)[0]
        rd = np.nonzero(~isi)[0]
        Tii = T[np.ix_(ri, ri)]
        rr, cc = np.meshgrid(gid[ri], gid[ri], indexing="ij")
        rows.append(rr.reshape(-1)); cols.append(cc.reshape(-1)); vals.append(Tii.reshape(-1))
        np.add.at(rhs, gid[ri], -hf[0, ri])
        if len(rd):
            np.add.at(rhs, gid[ri], -T[np.ix_(ri, rd)] @ g_dir[gid[rd]])
        S_all.append(S); v_all.append(v[0]); maps.append((isi, gid))
    Tg = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(grid.n_iface, grid.n_iface)).tocsc()
    u_iface = spla.splu(Tg).solve(rhs) if grid.n_iface else np.zeros(0)
    u_int = np.empty((nbox, n))
    for box in range(nbox):
        isi, gid = maps[box]
        ub = np.empty(m)
        ub[isi] = u_iface[gid[isi]]
        ub[~isi] = g_dir[gid[~isi]]
        u_int[box] = v_all[box] + S_all[box] @ ub
    return {"u_iface": u_iface, "u_int": u_int, "g_dir": g_dir, "T_global": Tg, "rhs": rhs}


def iface_coords(grid: InterfaceGrid) -> np.ndarray:
    out = np.empty((grid.n_iface, 3))
    p, qq = grid.p, grid.q * grid.q
    fx = face_node_grid_indices(p)
    for box in range(grid.nbox):
        xyz = node_coords(p, grid.box_lo(box), grid.h)
        isi, gid = grid.local_to_global(box)
        for r in range(6 * qq):
            if isi[r]:
                out[gid[r]] = xyz[fx[r]]
    return out


def interior_coords(grid: InterfaceGrid) -> np.ndarray:
    p = grid.p
    ii = interior_grid_indices(p)
    return np.stack([node_coords(p, grid.box_lo(b), grid.h)[ii] for b in range(grid.nbox)])


def dense_global_solve(grid: InterfaceGrid, kappa: float, b_fn, f_fn, g_fn, f_boxes=None, beta_boxes=None):
    """Brute force: the full collocation system, assembled and solved densely.

    Unknowns: every box's interior nodes, then interface nodes, then Dirichlet
    nodes.  Rows: each box's interior rows of A^tau (Eq. 3); on each shared
    face node the sum of both boxes' outward normal derivatives (Eq. 4) = 0;
    u = g on Dirichlet nodes.  f_boxes (per-box nodal arrays) replaces f_fn
    when given; beta_boxes adds div(beta u) as in hps_solve_boxes.
    """
    p, (n, m) = grid.p, sizes(grid.p)
    nbox = grid.nbox
    off_i, off_d = nbox * n, nbox * n + grid.n_iface
    Ntot = off_d + grid.n_dir
    G = np.zeros((Ntot, Ntot))
    rhs = np.zeros(Ntot)
    ii = interior_grid_indices(p)
    for box in range(nbox):
        xyz = node_coords(p, grid.box_lo(box), grid.h)
        A = leaf_matrix(p, grid.h, kappa, b_fn(xyz), beta_boxes[box] if beta_boxes is not None else None)
        isi, gid = grid.local_to_global(box)
        glob = np.concatenate([box * n + np.arange(n), np.where(isi, off_i + gid, off_d + gid)])
        G[np.ix_(glob[:n], glob)] += A[:n, :]
        rhs[glob[:n]] += (f_boxes[box] if f_boxes is not None else f_fn(xyz))[ii]
        fr = np.nonzero(isi)[0]
        G[np.ix_(off_i + gid[fr], glob)] += A[n + fr, :]
    if grid.n_dir:
        d = np.arange(grid.n_dir)
        G[off_d + d, :] = 0.0
        G[off_d + d, off_d + d] = 1.0
        rhs[off_d + d] = g_fn(grid.dirichlet_coords())
    u = np.linalg.solve(G, rhs)
    return {"u_int": u[:off_i].reshape(nbox, n), "u_iface": u[off_i:off_d], "u_dir": u[off_d:]}


def full_fields(grid: InterfaceGrid, u_int, u_iface, g_dir):
    """Per-box nodal arrays [nbox, p^3]: interior values from u_int, face values
    from the interface solution or the Dirichlet data; edges and corners 0
    (no kept-node row reads them)."""
    p = grid.p
    ii, fi = interior_grid_indices(p), face_node_grid_indices(p)
    out = np.zeros((grid.nbox, p ** 3))
    for box in range(grid.nbox):
        isi, gid = grid.local_to_global(box)
        out[box, ii] = u_int[box]
        out[box, fi] = np.where(isi, u_iface[np.where(isi, gid, 0)] if grid.n_iface else 0.0,
                                g_dir[np.where(~isi, gid, 0)] if grid.n_dir else 0.0)
    return out


def crank_nicolson_heat(grid: InterfaceGrid, kappa_d: float, dt: float, nsteps: int, u0_fn, vel_fn=None):
    """u_t = kappa_d Lap u - div(vel u) on the grid's domain (vel_fn None: the
    heat equation), u = 0 on its boundary, by the Crank-Nicolson steps of
    Sec. 4.4 with the HPS solve of every step.

    With c = 2 / (dt kappa_d) and L = c - Lap + div(beta .), beta = vel / kappa_d,
    a step is L u^{n+1} = 2 c u^n - L u^n, and L is the leaf operator
    -Lap + div(beta u) - kappa^2 b u with kappa^2 = c and b = -1, whose interior
    rows apply_interior evaluates for the right-hand side.  Returns the
    interior and interface values after nsteps (and the full fields).
    """
    from . import apply_interior
    p = grid.p
    c = 2.0 / (dt * kappa_d)
    kappa = float(np.sqrt(c))
    b = -np.ones(p ** 3)
    xyz = [node_coords(p, grid.box_lo(box), grid.h) for box in range(grid.nbox)]
    beta = [vel_fn(x).T / kappa_d for x in xyz] if vel_fn is not None else [None] * grid.nbox
    u = np.stack([u0_fn(x) for x in xyz])
    g_dir = np.zeros(grid.n_dir)
    res = None
    for _ in range(nsteps):
        f = [2.0 * c * u[box] - apply_interior(p, grid.h, kappa, b, u[box], beta[box]) for box in range(grid.nbox)]
        res = hps_solve_boxes(grid, kappa, [b] * grid.nbox, f, g_dir,
                              beta if vel_fn is not None else None)
        u = full_fields(grid, res["u_int"], res["u_iface"], g_dir)
    return {"u_int": res["u_int"], "u_iface": res["u_iface"], "u_full": u, "kappa": kappa, "c": c,
            "beta": beta}
