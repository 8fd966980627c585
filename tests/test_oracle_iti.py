"""Pins for the FP64 oracle of the leaf impedance-to-impedance map
(oracle/iti.py): the block-elimination identity with the pinned DtN map, the
impedance data of an exact Helmholtz solution, the behaviour at a Dirichlet
resonance of the box, and the large-eta limit."""
from __future__ import annotations

import numpy as np

import oracle
from oracle import iti
from oracle.global_solve import face_node_grid_indices


def _plane_wave_data(p, h, kappa, eta, phase=0.3):
    """(f, g) = (u_n + i eta u, u_n - i eta u) at the face nodes of the box
    [0, h] for u = cos(kappa d.x + phase), a solution of -Lap u - kappa^2 u = 0."""
    x = oracle.node_coords(p, np.zeros(3), h)
    d = np.array([1.0, 2.0, -0.5])
    d /= np.linalg.norm(d)
    ph = kappa * (x @ d) + phase
    u = np.cos(ph)
    grad = -np.sin(ph)[:, None] * kappa * d[None, :]
    fi = face_node_grid_indices(p)
    q = p - 2
    nrm = np.zeros((6 * q * q, 3))
    for f in range(6):
        nrm[f * q * q:(f + 1) * q * q, f >> 1] = 1.0 if f & 1 else -1.0
    un = (grad[fi] * nrm).sum(axis=1)
    return un + 1j * eta * u[fi], un - 1j * eta * u[fi]


def test_iti_is_the_dtn_cayley_transform():
    """Away from resonances R = (T - i eta I)(T + i eta I)^{-1}, with T from
    the oracle's own LU (variable b, anisotropic box)."""
    p, h, kappa = 6, np.array([0.3, 0.25, 0.35]), 7.0
    x = oracle.node_coords(p, np.array([0.1, 0.2, 0.0]), h)
    b = 1 + 0.3 * np.sin(3 * x[:, 0]) * np.cos(2 * x[:, 1])
    T, _, info = oracle.leaf_dtn(p, h, kappa, b, want_S=False)
    assert info == 0
    for eta in (kappa, 2.5):
        R = iti.leaf_iti(p, h, kappa, b, eta)
        assert np.abs(R - iti.iti_from_dtn(T, eta)).max() <= 1e-12 * np.abs(R).max()


def test_iti_maps_impedance_data_of_an_exact_solution():
    """R (u_n + i eta u) = u_n - i eta u for a plane wave, to the
    discretisation error, which decays spectrally in p."""
    h = np.array([0.2, 0.2, 0.2])
    errs = []
    for p in (6, 8, 10, 12):
        f, g = _plane_wave_data(p, h, 10.0, 10.0)
        R = iti.leaf_iti(p, h, 10.0, np.ones(p ** 3), 10.0)
        errs.append(np.abs(R @ f - g).max() / np.abs(g).max())
    assert all(e2 < 1e-2 * e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-10, errs


def test_iti_exists_at_a_dirichlet_resonance():
    """With kappa^2 the smallest eigenvalue of the box's interior block
    (b = 1, p = 10), A_ii is singular to rounding and the DtN map blows up;
    the ItI map stays of moderate norm and maps the plane wave's impedance
    data as accurately as it does three per cent off the resonance (the
    discretisation error at kappa h = 5.4)."""
    p, h = 10, np.array([0.2, 0.2, 0.2])
    n, m = oracle.sizes(p)
    Aii = oracle.leaf_matrix(p, h, 0.0, np.ones(p ** 3))[:n, :n]
    ev = np.linalg.eigvals(Aii)
    lam = np.sort(ev[np.abs(ev.imag) < 1e-8].real)[0]
    assert abs(lam - 3 * (np.pi / 0.2) ** 2) < 1e-3 * lam     # near the continuous 3 (pi / h)^2
    kappa = float(np.sqrt(lam))
    T, _, _ = oracle.leaf_dtn(p, h, kappa, np.ones(p ** 3), want_S=False)
    assert np.abs(T).max() > 1e10
    err = []
    for k in (kappa, 1.03 * kappa):
        R = iti.leaf_iti(p, h, k, np.ones(p ** 3), k)
        assert np.linalg.norm(R, 2) < 10.0
        f, g = _plane_wave_data(p, h, k, k)
        err.append(np.abs(R @ f - g).max() / np.abs(g).max())
    assert err[0] < 1e-4 and err[0] < 2 * err[1], err


def test_iti_large_eta_limit():
    """For eta much larger than the DtN map's entries, impedance data are
    dominated by i eta u and R tends to -I."""
    p, h, kappa = 6, np.array([0.25, 0.25, 0.25]), 5.0
    R = iti.leaf_iti(p, h, kappa, np.ones(p ** 3), 1e9)
    assert np.abs(R + np.eye(R.shape[0])).max() < 1e-5


def _resonant_setup(p=8):
    """2 x 2 x 2 boxes of side 1/2 with kappa^2 the smallest eigenvalue of the
    interior block of a b = 1 box; only the corner box at the origin has
    b = 1 (the others 1.25), so the whole domain is not resonant."""
    from oracle.global_solve import InterfaceGrid
    grid = InterfaceGrid(p, (2, 2, 2))
    n, m = oracle.sizes(p)
    Aii = oracle.leaf_matrix(p, grid.h, 0.0, np.ones(p ** 3))[:n, :n]
    ev = np.linalg.eigvals(Aii)
    kappa = float(np.sqrt(np.sort(ev[np.abs(ev.imag) < 1e-8].real)[0]))
    b_fn = lambda x: np.where((x[:, 0] < 0.5 - 1e-12) & (x[:, 1] < 0.5 - 1e-12) & (x[:, 2] < 0.5 - 1e-12), 1.0, 1.25)
    return grid, kappa, b_fn


def test_iti_global_solve_equals_the_dtn_solve():
    """Away from resonances the two-level solve on ItI maps gives the DtN
    solve's discrete solution (variable b, a load, Dirichlet data)."""
    from oracle.global_solve import InterfaceGrid, hps_solve
    grid = InterfaceGrid(6, (2, 2, 2))
    b_fn = lambda x: 1 + 0.3 * np.sin(x[:, 0] + 2 * x[:, 1])
    f_fn = lambda x: np.cos(x[:, 2])
    g_fn = lambda x: x[:, 0] * x[:, 1] + np.sin(x[:, 2])
    rd = hps_solve(grid, 5.0, b_fn, f_fn, g_fn)
    for eta in (5.0, 2.0):
        ri = iti.iti_solve(grid, 5.0, eta, b_fn, f_fn, g_fn)
        scale = max(np.abs(u).max() for u in rd["u_int"])
        assert max(np.abs(a - b).max() for a, b in zip(ri["u_int"], rd["u_int"])) < 1e-11 * scale


def test_iti_global_solve_survives_a_resonant_box():
    """With one box at a Dirichlet resonance the DtN solve is wrong by
    several per cent (its A_ii is singular to rounding), while the ItI solve
    equals the dense collocation solve of the whole system, which never
    inverts a box's interior block."""
    from oracle.global_solve import dense_global_solve, hps_solve
    grid, kappa, b_fn = _resonant_setup()
    zero = lambda x: np.zeros(len(x))
    g_fn = lambda x: np.cos(3 * x[:, 0] + x[:, 1]) + x[:, 2]
    ref = np.asarray(dense_global_solve(grid, kappa, b_fn, zero, g_fn)["u_int"])
    scale = np.abs(ref).max()
    ri = np.array(iti.iti_solve(grid, kappa, kappa, b_fn, zero, g_fn)["u_int"])
    assert np.abs(ri - ref).max() < 1e-12 * scale
    rd = np.array(hps_solve(grid, kappa, b_fn, zero, g_fn)["u_int"])
    assert np.abs(rd - ref).max() > 1e-3 * scale
