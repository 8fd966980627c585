"""Pins of the 2-D oracle (the method on a p x p grid per box; four edges of
p - 2 nodes, corners dropped).  As for 3-D: polynomial reproduction, the
kappa = 0 invariants of the DtN map, LAPACK's solve, the particular-solution
identities, the brute-force global collocation solve and spectral
convergence on a manufactured solution."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import global_solve_2d as g2

NORMALS = np.array([[-1, 0], [1, 0], [0, -1], [0, 1]], dtype=np.float64)


def kept_2d(p):
    """(interior grid indices [n], edge grid indices [m], edge id of each edge node [m])."""
    q, e = p - 2, p - 1
    ii = np.array([(i + 1) + p * (j + 1) for j in range(q) for i in range(q)])
    fi, fid = [], []
    for f in range(4):
        side = 0 if f % 2 == 0 else e
        for a in range(1, q + 1):
            fi.append(side + p * a if f // 2 == 0 else a + p * side)
            fid.append(f)
    return ii, np.asarray(fi), np.asarray(fid)


class Poly2:
    """u = sum c s_x^a s_y^b in box-local coordinates s = (x - ctr) / (h / 2)."""

    def __init__(self, terms, ctr, h):
        self.terms = terms
        self.ctr = np.asarray(ctr, dtype=np.float64)
        self.sc = 2.0 / np.asarray(h, dtype=np.float64)

    @staticmethod
    def _d(s, a, d):
        if a < d:
            return np.zeros_like(s)
        coef = 1.0
        for t in range(d):
            coef *= a - t
        return coef * s ** (a - d)

    def value(self, xy):
        s = (xy - self.ctr) * self.sc
        return sum(c * self._d(s[:, 0], a, 0) * self._d(s[:, 1], b, 0) for c, a, b in self.terms)

    def grad(self, xy):
        s = (xy - self.ctr) * self.sc
        g = np.zeros_like(xy)
        for c, a, b in self.terms:
            g[:, 0] += c * self._d(s[:, 0], a, 1) * self.sc[0] * self._d(s[:, 1], b, 0)
            g[:, 1] += c * self._d(s[:, 0], a, 0) * self._d(s[:, 1], b, 1) * self.sc[1]
        return g

    def laplacian(self, xy):
        s = (xy - self.ctr) * self.sc
        return sum(c * (self._d(s[:, 0], a, 2) * self.sc[0] ** 2 * self._d(s[:, 1], b, 0)
                        + self._d(s[:, 0], a, 0) * self._d(s[:, 1], b, 2) * self.sc[1] ** 2)
                   for c, a, b in self.terms)


def _box(p, lo=(0.3, -0.2), h=(0.4, 0.25)):
    return p, np.asarray(lo), np.asarray(h), oracle.node_coords_2d(p, lo, h)


def test_sizes_and_kept_index():
    for p in (3, 6, 11):
        q = p - 2
        assert oracle.sizes_2d(p) == (q * q, 4 * q)
        idx = [oracle.kept_index_2d(p, i, j) for j in range(p) for i in range(p)]
        assert sorted(v for v in idx if v >= 0) == list(range(q * q + 4 * q))
        assert sum(v < 0 for v in idx) == 4            # the corners


@pytest.mark.parametrize("kappa", [0.0, 4.0])
def test_operator_exact_on_polynomials(kappa):
    p, lo, h, xy = _box(9)
    rng = np.random.default_rng(3)
    b = rng.uniform(0.5, 1.5, p * p)
    A = oracle.leaf_matrix_2d(p, h, kappa, b)
    ii, fi, fid = kept_2d(p)
    for _ in range(3):
        u = Poly2([(rng.standard_normal(), *rng.integers(0, p, 2)) for _ in range(5)], lo + h / 2, h)
        uk = np.concatenate([u.value(xy[ii]), u.value(xy[fi])])
        r = A @ uk
        want_i = -u.laplacian(xy[ii]) - kappa ** 2 * b[ii] * u.value(xy[ii])
        want_b = (u.grad(xy[fi]) * NORMALS[fid]).sum(axis=1)
        scale = max(np.abs(want_i).max(), 1.0)
        assert np.abs(r[:len(ii)] - want_i).max() < 1e-10 * scale
        assert np.abs(r[len(ii):] - want_b).max() < 1e-11 * max(np.abs(want_b).max(), 1.0)


def test_kappa0_invariants_and_harmonic_polynomials():
    p, lo, h, xy = _box(10)
    T, S, info = oracle.leaf_dtn_2d(p, h, 0.0, np.ones(p * p))
    assert info == 0
    ii, fi, fid = kept_2d(p)
    assert np.abs(T.sum(axis=1)).max() < 1e-10 * np.abs(T).max()
    assert np.abs(S.sum(axis=1) - 1.0).max() < 1e-12
    harmonic = [
        (lambda x, y: 2 * x - 3 * y + 1, lambda x, y: (2 + 0 * x, -3 + 0 * x)),
        (lambda x, y: x * y, lambda x, y: (y, x)),
        (lambda x, y: x * x - y * y, lambda x, y: (2 * x, -2 * y)),
        (lambda x, y: x ** 3 - 3 * x * y * y, lambda x, y: (3 * x * x - 3 * y * y, -6 * x * y)),
        (lambda x, y: x ** 4 - 6 * x * x * y * y + y ** 4, lambda x, y: (4 * x ** 3 - 12 * x * y * y,
                                                                         4 * y ** 3 - 12 * x * x * y)),
    ]
    for u, g in harmonic:
        ub = u(xy[fi, 0], xy[fi, 1])
        gx, gy = g(xy[fi, 0], xy[fi, 1])
        dn = gx * NORMALS[fid, 0] + gy * NORMALS[fid, 1]
        assert np.abs(T @ ub - dn).max() < 1e-9 * max(np.abs(dn).max(), 1.0)
        ui = u(xy[ii, 0], xy[ii, 1])
        assert np.abs(S @ ub - ui).max() < 1e-11 * max(np.abs(ui).max(), 1.0)


def test_S_equals_lapack_solve():
    p, lo, h, xy = _box(8)
    b = 1.0 + 0.3 * np.sin(3 * xy[:, 0] + xy[:, 1])
    A = oracle.leaf_matrix_2d(p, h, 6.0, b)
    n, m = oracle.sizes_2d(p)
    T, S, info = oracle.leaf_dtn_2d(p, h, 6.0, b)
    S_ref = -np.linalg.solve(A[:n, :n], A[:n, n:])
    assert np.abs(S - S_ref).max() < 1e-12 * np.abs(S_ref).max()
    T_ref = A[n:, n:] + A[n:, :n] @ S_ref
    assert np.abs(T - T_ref).max() < 1e-12 * np.abs(T_ref).max()
    # the planted mistake T = A_bi S (no A_bb) breaks the kappa = 0 invariant
    A0 = oracle.leaf_matrix_2d(p, h, 0.0, b)
    S0 = -np.linalg.solve(A0[:n, :n], A0[:n, n:])
    assert np.abs((A0[n:, :n] @ S0).sum(axis=1)).max() > 1.0


def test_particular_identities():
    p, lo, h, xy = _box(9)
    kappa = 3.0
    b = 1.0 + 0.2 * np.cos(xy[:, 0] - 2 * xy[:, 1])
    rng = np.random.default_rng(7)
    u = Poly2([(rng.standard_normal(), *rng.integers(0, p, 2)) for _ in range(6)], lo + h / 2, h)
    f = -u.laplacian(xy) - kappa ** 2 * b * u.value(xy)
    T, S, _ = oracle.leaf_dtn_2d(p, h, kappa, b)
    v, hf, info = oracle.leaf_particular_2d(p, h, kappa, b, f[None, :])
    assert info == 0
    ii, fi, fid = kept_2d(p)
    ub = u.value(xy[fi])
    ui = u.value(xy[ii])
    assert np.abs(v[0] + S @ ub - ui).max() < 1e-10 * np.abs(ui).max()
    dn = (u.grad(xy[fi]) * NORMALS[fid]).sum(axis=1)
    assert np.abs(T @ ub + hf[0] - dn).max() < 1e-9 * np.abs(dn).max()


@pytest.mark.parametrize("nb,kappa", [((2, 2), 0.0), ((3, 2), 5.0)])
def test_two_level_equals_dense_bruteforce(nb, kappa):
    p = 7
    grid = g2.InterfaceGrid2D(p, nb, lo=(0.1, -0.3), L=(1.0, 0.8))
    rng = np.random.default_rng(2)
    xy = [oracle.node_coords_2d(p, grid.box_lo(bx), grid.h) for bx in range(grid.nbox)]
    b = [1.0 + 0.3 * np.sin(2 * x[:, 0] + x[:, 1]) for x in xy]
    f = [np.cos(x[:, 0] - x[:, 1]) for x in xy]
    g = rng.standard_normal(grid.n_dir)
    r = g2.hps_solve_2d(grid, kappa, b, f, g)
    d = g2.dense_global_solve_2d(grid, kappa, b, f, g)
    scale = np.abs(d["u_int"]).max()
    assert np.abs(r["u_int"] - d["u_int"]).max() < 1e-11 * scale
    assert np.abs(r["u_iface"] - d["u_iface"]).max() < 1e-11 * scale


def test_manufactured_spectral_convergence():
    """u = sin(pi x) sin(2 pi y) on the unit square, b = 1: f = (5 pi^2 - kappa^2) u,
    g = 0; the error decays spectrally in p."""
    kappa = 7.0
    errs = []
    for p in (6, 9, 12, 15):
        grid = g2.InterfaceGrid2D(p, (2, 2))
        xy = [oracle.node_coords_2d(p, grid.box_lo(bx), grid.h) for bx in range(grid.nbox)]
        uex = lambda x: np.sin(math.pi * x[:, 0]) * np.sin(2 * math.pi * x[:, 1])
        f = [(5 * math.pi ** 2 - kappa ** 2) * uex(x) for x in xy]
        r = g2.hps_solve_2d(grid, kappa, [np.ones(p * p)] * grid.nbox, f, np.zeros(grid.n_dir))
        ui = np.stack([uex(grid.kept_coords(bx)[0]) for bx in range(grid.nbox)])
        errs.append(np.abs(r["u_int"] - ui).max())
    assert all(b < a / 10 for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-9, errs


def test_square_symmetries_of_T():
    """For constant b on a square box the DtN map commutes with the symmetries
    of the square: the reflection x -> -x swaps edges x- and x+ and keeps the
    node order on them while reversing it on the y-edges; the transpose
    (x, y) -> (y, x) swaps the x-edges with the y-edges."""
    p = 9
    q = p - 2
    T, _, info = oracle.leaf_dtn_2d(p, (0.5, 0.5), 3.0, np.ones(p * p), want_S=False)
    assert info == 0
    rev = np.arange(q)[::-1]
    a = np.arange(q)
    # x -> -x
    P1 = np.concatenate([1 * q + a, 0 * q + a, 2 * q + rev, 3 * q + rev])
    # (x, y) -> (y, x)
    P2 = np.concatenate([2 * q + a, 3 * q + a, 0 * q + a, 1 * q + a])
    for P in (P1, P2):
        assert np.abs(T[np.ix_(P, P)] - T).max() < 1e-11 * np.abs(T).max()
    # a non-square box breaks the transpose symmetry
    T2, _, _ = oracle.leaf_dtn_2d(p, (0.5, 0.3), 3.0, np.ones(p * p), want_S=False)
    assert np.abs(T2[np.ix_(P2, P2)] - T2).max() > 1e-3 * np.abs(T2).max()
