"""FP64 oracle of the leaf impedance-to-impedance (ItI) map.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).

The paper's closing section (Sec. 6) names HPS built on
impedance-to-impedance maps (Gillman, Barnett and Martinsson's formulation)
as a variant the two-level scheme adapts to; such maps do not fail where
kappa^2 is a Dirichlet eigenvalue of a box, as DtN maps do.  On the leaf
collocation of Sec. 2.1 (the
kept nodes: interior and face nodes, Eq. 2's rows) the ItI map R takes
impedance data f = du/dn + i eta u on the face nodes to g = du/dn - i eta u
for the solution u of the homogeneous equation in the box:

    [ A_ii   A_ib            ] [u_i]   [0]
    [ A_bi   A_bb + i eta I  ] [u_b] = [f],     g = f - 2 i eta u_b.

Unlike the DtN map it never inverts A_ii on its own, so it exists where
kappa^2 is a Dirichlet eigenvalue of the box's interior block.  Where T
exists, the block elimination of u_i gives (T + i eta I) u_b = f, so
R = (T - i eta I)(T + i eta I)^{-1}: that identity is the first pin.
"""
from __future__ import annotations

import numpy as np

from . import leaf_matrix, sizes


def leaf_iti(p: int, h, kappa: float, b: np.ndarray, eta: float) -> np.ndarray:
    """R [m, m] (complex) of one box: the kept-node collocation matrix with
    i eta added on the face rows' own unknowns, solved for the m unit
    impedance data vectors (numpy's complex LU solve as the step)."""
    n, m = sizes(p)
    A = leaf_matrix(p, h, kappa, b).astype(np.complex128)
    A[n:, n:] += 1j * eta * np.eye(m)
    rhs = np.zeros((n + m, m), dtype=np.complex128)
    rhs[n:, :] = np.eye(m)
    ub = np.linalg.solve(A, rhs)[n:, :]
    return np.eye(m) - 2j * eta * ub


def iti_from_dtn(T: np.ndarray, eta: float) -> np.ndarray:
    """(T - i eta I)(T + i eta I)^{-1}: the ItI map of a box whose DtN map is T."""
    m = T.shape[0]
    E = 1j * eta * np.eye(m)
    return np.linalg.solve((T + E).T, (T - E).T).T


def leaf_iti_ops(p: int, h, kappa: float, b: np.ndarray, eta: float, f=None):
    """(R [m, m], S [n, m], v [nrhs, n] or None, hout [nrhs, m] or None),
    complex, of one box: R and the interior solution operator S for unit
    incoming impedance data; for loads f [nrhs, p^3] (interior values used,
    zero incoming impedance) the interior solution v and the outgoing
    impedance hout = -2 i eta u_b of that solution."""
    from .global_solve import interior_grid_indices
    n, m = sizes(p)
    A = leaf_matrix(p, h, kappa, b).astype(np.complex128)
    A[n:, n:] += 1j * eta * np.eye(m)
    nr = 0 if f is None else np.atleast_2d(f).shape[0]
    rhs = np.zeros((n + m, m + nr), dtype=np.complex128)
    rhs[n:, :m] = np.eye(m)
    if nr:
        rhs[:n, m:] = np.atleast_2d(f)[:, interior_grid_indices(p)].T
    X = np.linalg.solve(A, rhs)
    R = np.eye(m) - 2j * eta * X[n:, :m]
    S = X[:n, :m]
    if not nr:
        return R, S, None, None
    return R, S, X[:n, m:].T, (-2j * eta * X[n:, m:]).T


def iti_solve(grid, kappa: float, eta: float, b_fn, f_fn, g_fn):
    """Two-level solve on ItI maps (uniform grid of InterfaceGrid): the
    unknowns are every box's incoming impedance data on its m face nodes.
    On a face shared by boxes tau and sigma the incoming data of one side is
    minus the outgoing data of the other (continuity of u and of the flux
    with opposite normals): f_tau + R_sigma f_sigma + hout_sigma = 0 at the
    matching node; on a Dirichlet face u = g gives R_tau f_tau + hout_tau -
    f_tau = -2 i eta g.  Then u_b = (f - g_out) / (2 i eta) and
    u_i = S f + v.  Returns the per-box interior solutions (complex) and the
    per-box face values."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from . import node_coords
    from .global_solve import face_node_grid_indices
    p = grid.p
    n, m = sizes(p)
    nbox = grid.nbox
    ops, gvals = [], []
    for box in range(nbox):
        x = node_coords(p, grid.box_lo(box), grid.h)
        ops.append(leaf_iti_ops(p, grid.h, kappa, b_fn(x), eta, f_fn(x)[None, :]))
        gvals.append(g_fn(x[face_node_grid_indices(p)]))
    # partner of (box, face node): the same face id's node on the other box
    owner = {}
    for box in range(nbox):
        isi, gid = grid.local_to_global(box)
        for r in range(m):
            if isi[r]:
                owner.setdefault(int(gid[r]), []).append((box, r))
    N = nbox * m
    rows, cols, vals = [], [], []
    rhs = np.zeros(N, dtype=np.complex128)
    for box in range(nbox):
        R, S, v, ho = ops[box]
        isi, gid = grid.local_to_global(box)
        for r in range(m):
            row = box * m + r
            if isi[r]:
                (b0, r0), (b1, r1) = owner[int(gid[r])]
                sb, sr = (b1, r1) if (b0, r0) == (box, r) else (b0, r0)
                Rs, _, _, hos = ops[sb]
                rows += [row] * (m + 1)
                cols += [row] + list(sb * m + np.arange(m))
                vals += [1.0] + list(Rs[sr, :])
                rhs[row] = -hos[0, sr]
            else:
                rows += [row] * m
                cols += list(box * m + np.arange(m))
                rr = np.array(R[r, :])
                rr[r] -= 1.0
                vals += list(rr)
                rhs[row] = -ho[0, r] - 2j * eta * gvals[box][r]
    A = sp.coo_matrix((np.asarray(vals, dtype=np.complex128), (rows, cols)), shape=(N, N)).tocsc()
    fin = spla.splu(A).solve(rhs)
    u_int, u_b = [], []
    for box in range(nbox):
        R, S, v, ho = ops[box]
        fb = fin[box * m:(box + 1) * m]
        g_out = R @ fb + ho[0]
        u_b.append((fb - g_out) / (2j * eta))
        u_int.append(S @ fb + v[0])
    return {"u_int": u_int, "u_b": u_b, "f_in": fin, "A": A, "rhs": rhs}
