"""Leaf reduction for operators with cross terms, on Legendre face grids.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).

Remark 1 of Sec. 2.1: edge and corner nodes of a box can be dropped only when
the operator has no cross terms d_a d_b u (a != b).  With cross terms, each
face's data lives on a (p-1) x (p-1) tensor grid of Gauss-Legendre nodes
instead of the p x p Chebyshev grid, and the global system again has no
nodes on edges or corners.  Sec. 4.3 needs exactly this: the parameter map of
a curved domain gives variable coefficients with a cross term.

The operator, with a symmetric coefficient tensor C(x), first-order
coefficients d(x) and the wavenumber term as in Eq. 1:

    A u = - sum_{a,b} C_ab d_a d_b u + sum_a d_a(x) d_a u - kappa^2 b(x) u.

Per box (everything dense, written from the definitions; p <= 10 here):

* nodes: the p^3 Chebyshev-Lobatto tensor grid (the oracle's own ``nodes``
  and ``diff``), interior I (q^3 nodes) and boundary E (every other node:
  faces, edges, corners);
* Legendre face grids: per face (x-, x+, y-, y+, z-, z+) the (p-1)^2 tensor
  points of the (p-1)-point Gauss-Legendre rule in the face's two free
  coordinates, lower axis fastest;
* P (p^3 x 6(p-1)^2): Dirichlet data on the Legendre grids to values at the
  boundary Chebyshev nodes; a node on one face takes that face's polynomial
  interpolant (degree p-2 per coordinate) evaluated there, a node shared by
  several faces (edges, corners) the average over them (the reading of
  Remark 1 this build takes: the paper leaves it to the cited works);
* S = -A_II^{-1} A_IE P_E (interior values from face data), v = A_II^{-1} f_I;
* N: the outward normal derivative at each face's p x p Chebyshev nodes,
  from the full-grid values; Q: each face's p x p values to its Legendre
  grid by the degree-(p-1) interpolant;
* T = Q N [S; P_E] (the DtN map, 6(p-1)^2 square), h = Q N [v; 0].

The global system over a box grid is Eq. 4's flux balance at every Legendre
node of a shared face, with the Legendre nodes of the domain boundary as
Dirichlet data (``LegendreGrid``, ``hps_solve_cross``).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import diff, nodes
from .global_solve import InterfaceGrid


def sizes_cross(p: int):
    """(n interior nodes, m Legendre face nodes) of a box."""
    return (p - 2) ** 3, 6 * (p - 1) ** 2


def legendre_nodes(N: int) -> np.ndarray:
    """The N Gauss-Legendre nodes on [-1, 1], ascending: the roots of P_N,
    found by Newton's method on the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, started from cos(pi (i + 3/4) /
    (N + 1/2))."""
    x = np.cos(np.pi * (np.arange(N) + 0.75) / (N + 0.5))
    for _ in range(100):
        p0, p1 = np.ones_like(x), x.copy()
        for k in range(1, N):
            p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        # P_N = p1, P_{N-1} = p0; P_N' = N (x P_N - P_{N-1}) / (x^2 - 1)
        dp = N * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.abs(dx).max() < 1e-16:
            break
    return np.sort(x)


def lagrange_matrix(src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """L[i, j] = l_j(dst_i) for the Lagrange basis l_j of the nodes src (the
    product formula written out): L @ values at src = the interpolant at dst."""
    L = np.ones((len(dst), len(src)))
    for j in range(len(src)):
        for m in range(len(src)):
            if m != j:
                L[:, j] *= (dst - src[m]) / (src[j] - src[m])
    return L


def interp_matrices(p: int):
    """(G, Q): G (p x (p-1)) takes values at the p-1 Legendre nodes to the p
    Chebyshev nodes (the end points included), Q ((p-1) x p) the reverse."""
    t, g = nodes(p), legendre_nodes(p - 1)
    return lagrange_matrix(g, t), lagrange_matrix(t, g)


def full_index(p: int, i: int, j: int, k: int) -> int:
    return i + p * j + p * p * k


def interior_set(p: int) -> np.ndarray:
    q = p - 2
    r = np.arange(1, q + 1)
    k, j, i = np.meshgrid(r, r, r, indexing="ij")
    return (i + p * j + p * p * k).reshape(-1)


def boundary_set(p: int) -> np.ndarray:
    inner = np.zeros(p ** 3, dtype=bool)
    inner[interior_set(p)] = True
    return np.nonzero(~inner)[0]


def _face_axes(f: int):
    """(normal axis, end index side, free axes (u, v) with u < v)."""
    a = f // 2
    free = [x for x in range(3) if x != a]
    return a, f % 2, free[0], free[1]


def cross_operator(p: int, h, kappa: float, C: np.ndarray, d, b: np.ndarray) -> np.ndarray:
    """The p^3 x p^3 collocation matrix of A on the box's full grid.
    C [6, p^3]: C11, C22, C33, C12, C13, C23 at the nodes; d [3, p^3] or None;
    b [p^3].  Node (i, j, k) has index i + p j + p^2 k."""
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (3,))
    Dh = diff(p)
    I = np.eye(p)
    Ds = []
    for a in range(3):
        Da = (2.0 / h[a]) * Dh
        mats = [I, I, I]
        mats[a] = Da
        Ds.append(np.kron(mats[2], np.kron(mats[1], mats[0])))   # axis 0 fastest
    comp = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (0, 2): 4, (1, 2): 5}
    A = np.zeros((p ** 3, p ** 3))
    for a in range(3):
        for bb in range(3):
            c = C[comp[(min(a, bb), max(a, bb))]]
            A -= c[:, None] * (Ds[a] @ Ds[bb])
    if d is not None:
        for a in range(3):
            A += np.asarray(d[a])[:, None] * Ds[a]
    A -= kappa ** 2 * np.diag(np.asarray(b, dtype=np.float64))
    return A


def dirichlet_interp(p: int) -> np.ndarray:
    """P [p^3, 6 (p-1)^2]: Legendre face data to the boundary Chebyshev nodes
    (rows of interior nodes are zero); shared nodes average their faces."""
    G, _ = interp_matrices(p)
    e, pl = p - 1, p - 1
    ml = pl * pl
    P = np.zeros((p ** 3, 6 * ml))
    count = np.zeros(p ** 3)
    for f in range(6):
        a, side, u, v = _face_axes(f)
        for iv in range(p):
            for iu in range(p):
                idx = [0, 0, 0]
                idx[a] = 0 if side == 0 else e
                idx[u], idx[v] = iu, iv
                count[full_index(p, *idx)] += 1
    for f in range(6):
        a, side, u, v = _face_axes(f)
        for iv in range(p):
            for iu in range(p):
                idx = [0, 0, 0]
                idx[a] = 0 if side == 0 else e
                idx[u], idx[v] = iu, iv
                r = full_index(p, *idx)
                w = 1.0 / count[r]
                for t in range(pl):
                    for s in range(pl):
                        P[r, f * ml + s + pl * t] += w * G[iu, s] * G[iv, t]
    return P


def normal_derivative(p: int, h) -> np.ndarray:
    """N [6 p^2, p^3]: outward normal derivative at each face's p x p
    Chebyshev nodes (face node (iu, iv) at row f p^2 + iu + p iv)."""
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (3,))
    Dh = diff(p)
    e = p - 1
    N = np.zeros((6 * p * p, p ** 3))
    for f in range(6):
        a, side, u, v = _face_axes(f)
        Da = (2.0 / h[a]) * Dh
        end = 0 if side == 0 else e
        sgn = -1.0 if side == 0 else 1.0
        for iv in range(p):
            for iu in range(p):
                row = f * p * p + iu + p * iv
                for l in range(p):
                    idx = [0, 0, 0]
                    idx[a] = l
                    idx[u], idx[v] = iu, iv
                    N[row, full_index(p, *idx)] += sgn * Da[end, l]
    return N


def face_projection(p: int) -> np.ndarray:
    """Q_f [6 (p-1)^2, 6 p^2]: each face's p x p Chebyshev values to its
    Legendre grid (Q on both face coordinates)."""
    _, Q = interp_matrices(p)
    pl = p - 1
    Qf = np.zeros((6 * pl * pl, 6 * p * p))
    QQ = np.kron(Q, Q)   # rows s + pl t (s fastest), cols iu + p iv
    for f in range(6):
        Qf[f * pl * pl:(f + 1) * pl * pl, f * p * p:(f + 1) * p * p] = QQ
    return Qf


def leaf_cross(p: int, h, kappa: float, C: np.ndarray, d, b: np.ndarray, f=None):
    """(T [m, m], S [n, m], v [nrhs, n] or None, hflux [nrhs, m] or None) of
    one box, m = 6 (p-1)^2: S = -A_II^{-1} A_IE P_E, T = Q N [S; P_E],
    v = A_II^{-1} f_I, h = Q N [v; 0].  f [nrhs, p^3] (or [p^3]) or None."""
    A = cross_operator(p, h, kappa, C, d, b)
    Iset, Eset = interior_set(p), boundary_set(p)
    P = dirichlet_interp(p)
    Aii = A[np.ix_(Iset, Iset)]
    Aie = A[np.ix_(Iset, Eset)]
    S = -np.linalg.solve(Aii, Aie @ P[Eset])
    U = P.copy()
    U[Iset] = S
    NQ = face_projection(p) @ normal_derivative(p, h)
    T = NQ @ U
    if f is None:
        return T, S, None, None
    F = np.atleast_2d(np.asarray(f, dtype=np.float64))
    v = np.linalg.solve(Aii, F[:, Iset].T).T
    V = np.zeros((F.shape[0], p ** 3))
    V[:, Iset] = v
    return T, S, v, (NQ @ V.T).T


def legendre_face_coords(p: int, lo, h) -> np.ndarray:
    """Physical coordinates [6 (p-1)^2, 3] of a box's Legendre face nodes."""
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (3,))
    lo = np.asarray(lo, dtype=np.float64)
    g = legendre_nodes(p - 1)
    pl = p - 1
    out = np.empty((6 * pl * pl, 3))
    for f in range(6):
        a, side, u, v = _face_axes(f)
        for t in range(pl):
            for s in range(pl):
                x = np.empty(3)
                x[a] = lo[a] + (h[a] if side else 0.0)
                x[u] = lo[u] + h[u] * (g[s] + 1.0) / 2.0
                x[v] = lo[v] + h[v] * (g[t] + 1.0) / 2.0
                out[f * pl * pl + s + pl * t] = x
    return out


class LegendreGrid(InterfaceGrid):
    """The interface numbering of ``InterfaceGrid`` with (p-1)^2 Legendre
    nodes per face instead of (p-2)^2 Chebyshev ones."""

    def __init__(self, p: int, nb, lo=(0.0, 0.0, 0.0), L=(1.0, 1.0, 1.0)):
        super().__init__(p, nb, lo, L)
        self.q = p - 1
        self.n_iface = self.n_iface_faces * self.q * self.q
        self.n_dir = self.n_dir_faces * self.q * self.q

    def dirichlet_coords(self) -> np.ndarray:
        out = np.empty((self.n_dir, 3))
        for box in range(self.nbox):
            xyz = legendre_face_coords(self.p, self.box_lo(box), self.h)
            isi, gid = self.local_to_global(box)
            out[gid[~isi]] = xyz[~isi]
        return out


def hps_solve_cross(grid: LegendreGrid, kappa: float, C_fn, d_fn, b_fn, f_fn, g_fn):
    """Two-level solve with the cross-term leaf maps: per box T, S, v, h; the
    interface system sum_tau (T u_b + h) = 0 at every shared Legendre node
    with the domain boundary's Legendre nodes as Dirichlet data g; a host
    sparse LU; u_i = v + S u_b.  C_fn(x) [6, N], d_fn(x) [3, N] or None,
    b_fn(x), f_fn(x), g_fn(x) on node coordinates x [N, 3].  Returns the
    interface values and the interior values [nbox, n]."""
    from . import node_coords
    p = grid.p
    n, m = sizes_cross(p)
    g = g_fn(grid.dirichlet_coords())
    rows, cols, vals = [], [], []
    rhs = np.zeros(grid.n_iface)
    leaves = []
    for box in range(grid.nbox):
        xyz = node_coords(p, grid.box_lo(box), grid.h)
        T, S, v, hf = leaf_cross(p, grid.h, kappa, C_fn(xyz), None if d_fn is None else d_fn(xyz), b_fn(xyz),
                                 f_fn(xyz)[None, :])
        isi, gid = grid.local_to_global(box)
        leaves.append((S, v[0], isi, gid))
        ii = np.nonzero(isi)[0]
        dd = np.nonzero(~isi)[0]
        r, c = np.meshgrid(gid[ii], gid[ii], indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(T[np.ix_(ii, ii)].ravel())
        np.add.at(rhs, gid[ii], -(hf[0][ii] + T[np.ix_(ii, dd)] @ g[gid[dd]]))
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(grid.n_iface, grid.n_iface)).tocsc()
    u_if = spla.splu(K).solve(rhs)
    u_int = np.empty((grid.nbox, n))
    for box, (S, v, isi, gid) in enumerate(leaves):
        ub = np.empty(m)
        ub[isi] = u_if[gid[isi]]
        ub[~isi] = g[gid[~isi]]
        u_int[box] = v + S @ ub
    return u_if, u_int
