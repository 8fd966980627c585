"""Pins for the mixed-order (adaptive p) two-level solve of the oracle
(oracle/adaptive.py): the interpolation matrices, the reduction to the
uniform solve, exact reproduction of a harmonic polynomial on a grid of two
orders, and spectral convergence to a plane wave."""
from __future__ import annotations

import numpy as np

import oracle
from oracle import adaptive as ad
from oracle.global_solve import InterfaceGrid, hps_solve, interior_grid_indices


def _checker(pc, pf, nb=(2, 2, 2)):
    nx, ny, _ = nb
    return [pc if (i % nx + (i // nx) % ny + i // (nx * ny)) % 2 == 0 else pf for i in range(int(np.prod(nb)))]


def _interior_error(grid, r, u):
    err = 0.0
    for box in range(grid.nbox):
        p = int(grid.p_box[box])
        x = oracle.node_coords(p, grid.box_lo(box), grid.h)
        err = max(err, float(np.abs(r["u_int"][box] - u(x[interior_grid_indices(p)])).max()))
    return err


def test_face_interpolation_is_exact_on_polynomials():
    """face_interp reproduces tensor polynomials of degree below the source
    order's face point count, both ways between orders 6 and 9."""
    rng = np.random.default_rng(0)
    for ps, pd in ((6, 9), (9, 6)):
        ts, td = ad.face_points(ps), ad.face_points(pd)
        deg = ps - 3
        c = rng.standard_normal((deg + 1, deg + 1))
        poly = lambda a, b: sum(c[i, j] * a ** i * b ** j for i in range(deg + 1) for j in range(deg + 1))
        A, B = np.meshgrid(ts, ts, indexing="xy")       # lower free axis fastest
        Ad, Bd = np.meshgrid(td, td, indexing="xy")
        got = ad.face_interp(ps, pd) @ poly(A, B).reshape(-1)
        assert np.abs(got - poly(Ad, Bd).reshape(-1)).max() < 1e-12


def test_one_order_reduces_to_the_uniform_solve():
    p = 6
    b_fn = lambda x: 1 + 0.3 * np.sin(x[:, 0] + 2 * x[:, 1])
    f_fn = lambda x: np.cos(x[:, 2])
    g_fn = lambda x: x[:, 0] * x[:, 1] + np.sin(x[:, 2])
    ru = hps_solve(InterfaceGrid(p, (2, 2, 2)), 5.0, b_fn, f_fn, g_fn)
    rm = ad.mixed_solve(ad.MixedGrid([p] * 8, (2, 2, 2)), 5.0, b_fn, f_fn, g_fn)
    assert np.abs(ru["u_iface"] - rm["u_iface"]).max() < 1e-13
    assert max(np.abs(a - b).max() for a, b in zip(ru["u_int"], rm["u_int"])) < 1e-13


def test_mixed_orders_reproduce_a_harmonic_cubic():
    """Orders 6 and 8 in a checkerboard: a harmonic polynomial of degree 3
    (below every box's face point count) is reproduced to rounding, on the
    interface unknowns and in every interior."""
    grid = ad.MixedGrid(_checker(6, 8), (2, 2, 2))
    u = lambda x: (x[:, 0] ** 3 - 3 * x[:, 0] * x[:, 1] ** 2 + x[:, 2] ** 2 - 0.5 * (x[:, 0] ** 2 + x[:, 1] ** 2)
                   + x[:, 0] * x[:, 2])
    r = ad.mixed_solve(grid, 0.0, lambda x: np.ones(len(x)), lambda x: np.zeros(len(x)), u)
    assert _interior_error(grid, r, u) < 1e-12
    assert np.abs(r["u_iface"] - u(grid.face_node_coords()[:grid.n_iface])).max() < 1e-12


def test_mixed_orders_converge_spectrally():
    """A plane wave (kappa = 8) on checkerboards of orders (p, p + 2): the
    interior error falls by more than 30x per step in p."""
    k = 8.0
    d = np.array([1.0, 2.0, -0.5])
    d /= np.linalg.norm(d)
    pw = lambda x: np.cos(k * (x @ d) + 0.3)
    errs = []
    for pc in (6, 8, 10):
        grid = ad.MixedGrid(_checker(pc, pc + 2), (2, 2, 2))
        r = ad.mixed_solve(grid, k, lambda x: np.ones(len(x)), lambda x: np.zeros(len(x)), pw)
        errs.append(_interior_error(grid, r, pw))
    assert all(e2 < e1 / 30 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5, errs
