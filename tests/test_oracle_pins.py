"""Pins for the FP64 CPU oracle: closed forms, exact invariants, a library
special case and a brute-force global solve.  None of these calls the CUDA
library; each would fail on a plausible mistake in the oracle (a dropped term,
a wrong sign or index, a transposed operand), and the mutation tests at the
end check that for the mistakes the paper's own text invites."""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import hps_inputs as hi
import oracle
from oracle import global_solve as gs
from tests._geom import FACE_NORMALS, HARMONIC, TensorPoly, kept_grid_indices

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ 1-D (Sec. 2.1)

def test_nodes_are_chebyshev_lobatto():
    for p in range(3, 22):
        t = oracle.nodes(p)
        N = p - 1
        assert t[0] == -1.0 and t[-1] == 1.0
        assert np.all(np.diff(t) > 0)
        np.testing.assert_array_equal(t, -t[::-1])          # exact symmetry
        # interior nodes are the extrema of T_N: T_N'(t) = N U_{N-1}(t) = 0
        th = np.arccos(np.clip(t[1:-1], -1, 1))
        assert np.abs(np.sin(N * th)).max() < 1e-12


def test_diff_golden_small():
    g = json.load(open(os.path.join(GOLDEN, "cheb_small.json")))
    for key, p in (("N1", 2), ("N2", 3)):
        np.testing.assert_allclose(oracle.nodes(p), g[key]["nodes"], atol=1e-15)
        np.testing.assert_allclose(oracle.diff(p), np.array(g[key]["D"]), atol=1e-14)


def test_diff_closed_form_entries():
    for p in range(3, 22):
        N, t, D = p - 1, oracle.nodes(p), oracle.diff(p)
        c = (2 * N * N + 1) / 6.0
        assert abs(D[0, 0] + c) < 1e-12 * c and abs(D[N, N] - c) < 1e-12 * c
        j = np.arange(1, N)
        np.testing.assert_allclose(np.diag(D)[1:-1], -t[j] / (2 * (1 - t[j] ** 2)), rtol=1e-11, atol=1e-12)
        i, jj = 2 % p, (p - 1)
        if i != jj:
            ci, cj = (2.0 if i in (0, N) else 1.0), (2.0 if jj in (0, N) else 1.0)
            assert abs(D[i, jj] - ci / cj * (-1) ** (i + jj) / (t[i] - t[jj])) < 1e-12 * abs(D[i, jj])


@pytest.mark.parametrize("p", [3, 4, 6, 8, 12, 16, 20])
def test_diff_exact_on_polynomials(p):
    t, D = oracle.nodes(p), oracle.diff(p)
    for k in range(p):
        exact = k * t ** (k - 1) if k else np.zeros(p)
        assert np.abs(D @ t ** k - exact).max() < 1e-13 * p * p * max(1, k)


# ------------------------------------------------------------------ index sets (Remark 1)

@pytest.mark.parametrize("p", [3, 4, 5, 8, 12])
def test_index_sets(p):
    n, m = oracle.sizes(p)
    q = p - 2
    assert (n, m) == (q ** 3, 6 * q * q)
    seen = set()
    dropped = 0
    for k in range(p):
        for j in range(p):
            for i in range(p):
                idx = oracle.kept_index(p, i, j, k)
                if idx < 0:
                    dropped += 1
                else:
                    seen.add(idx)
    assert dropped == 12 * q + 8
    assert seen == set(range(n + m))


# ------------------------------------------------------------------ operator rows (Eq. 2, Eq. 4)

@pytest.mark.parametrize("p,h,kappa", [(6, (0.5, 0.5, 0.5), 0.0), (8, (0.125, 0.25, 0.2), 20.0), (9, (1.0, 0.3, 0.7), 7.0)])
def test_operator_exact_on_polynomials(p, h, kappa):
    rng = np.random.default_rng(p)
    lo = np.array([0.1, -0.3, 0.4])
    xyz = oracle.node_coords(p, lo, h)
    b = 0.5 + rng.random(p ** 3)
    A = oracle.leaf_matrix(p, h, kappa, b)
    interior, face, fid = kept_grid_indices(p)
    kept = np.concatenate([interior, face])
    for _ in range(3):
        u = TensorPoly.random(rng, p, lo + 0.5 * np.asarray(h), h)
        uk = u.value(xyz[kept])
        Au = A @ uk
        exp_i = -u.laplacian(xyz[interior]) - kappa ** 2 * b[interior] * u.value(xyz[interior])
        exp_b = (u.grad(xyz[face]) * FACE_NORMALS[fid]).sum(axis=1)
        scale = np.abs(A).max() * np.abs(uk).max()
        assert np.abs(Au[: len(interior)] - exp_i).max() < 1e-12 * scale
        assert np.abs(Au[len(interior):] - exp_b).max() < 1e-12 * scale


def test_boundary_blocks_shared_across_boxes():
    """Sec. 3.1: A_bi and A_bb do not depend on the operator's coefficients;
    A_ib does not either (kappa^2 b sits on the A_ii diagonal only)."""
    p, h = 7, (0.25, 0.25, 0.25)
    rng = np.random.default_rng(3)
    B1 = oracle.split_blocks(p, oracle.leaf_matrix(p, h, 0.0, np.ones(p ** 3)))
    B2 = oracle.split_blocks(p, oracle.leaf_matrix(p, h, 30.0, 0.5 + rng.random(p ** 3)))
    for a, c in zip(B1[1:], B2[1:]):
        np.testing.assert_array_equal(a, c)
    assert not np.array_equal(B1[0], B2[0])


# ------------------------------------------------------------------ LU (Algorithm 1)

def test_lu_reproduces_matrix_and_matches_lapack():
    p, h = 8, (0.125,) * 3
    b = hi.fourier_b_field().b(oracle.node_coords(p, (0.25, 0.5, 0.0), h))
    Aii, Aib, _, _ = oracle.split_blocks(p, oracle.leaf_matrix(p, h, 40.0, b))
    LU, piv, info = oracle.lu(Aii)
    assert info == 0
    n = Aii.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    PA = Aii.copy()
    for k in range(n):
        PA[[k, piv[k]]] = PA[[piv[k], k]]
    assert np.abs(L @ U - PA).max() < 1e-13 * np.abs(Aii).max()
    assert np.abs(L).max() <= 1.0 + 1e-15                    # partial pivoting bound
    S_lapack = np.linalg.solve(Aii, -Aib)
    T, S, info = oracle.leaf_dtn(p, h, 40.0, b)
    assert np.abs(S - S_lapack).max() < 1e-12 * np.abs(S_lapack).max()


def test_lu_flags_singular_matrix():
    A = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [0.0, 0.0, 1.0]])
    _, _, info = oracle.lu(A)
    assert info == 2


# ------------------------------------------------------------------ S and T (Sec. 2.2, Eq. 8)

@pytest.mark.parametrize("p", [5, 8, 10])
def test_dtn_exact_invariants_kappa0(p):
    h = np.array([0.5, 0.25, 0.4])
    lo = np.array([0.3, -0.1, 0.2])
    T, S, info = oracle.leaf_dtn(p, h, 0.0, np.full(p ** 3, 1.3))
    assert info == 0
    xyz = oracle.node_coords(p, lo, h)
    interior, face, fid = kept_grid_indices(p)
    Ts = np.abs(T).max()
    assert np.abs(T @ np.ones(T.shape[1])).max() < 1e-12 * Ts            # T 1 = 0
    assert np.abs(S @ np.ones(S.shape[1]) - 1).max() < 1e-12              # S 1 = 1
    for name, fn, gr in HARMONIC:
        if name in ("x3-3xy2", "y2z-z3/3") and p < 4:
            continue
        xb, xi = xyz[face], xyz[interior]
        phi = fn(*xb.T)
        dn = (np.stack(gr(*xb.T), axis=1) * FACE_NORMALS[fid]).sum(axis=1)
        scale = Ts * np.abs(phi).max() + 1.0
        assert np.abs(T @ phi - dn).max() < 1e-11 * scale, name
        assert np.abs(S @ phi - fn(*xi.T)).max() < 1e-11 * (np.abs(phi).max() + 1), name


@pytest.mark.parametrize("p,kappa", [(6, 20.0), (9, 12.0)])
def test_polynomial_reproduction_any_b(p, kappa):
    """For u of degree <= p-1 per variable and ANY b: the local problem with
    f = -Lap u - kappa^2 b u and u_b = u on the faces has the exact solution u,
    so v + S u_b = u_i and T u_b + A_bi v = du/dn."""
    rng = np.random.default_rng(11)
    h = np.array([0.125, 0.125, 0.125])
    lo = np.array([0.5, 0.25, 0.0])
    xyz = oracle.node_coords(p, lo, h)
    b = hi.fourier_b_field().b(xyz)
    interior, face, fid = kept_grid_indices(p)
    T, S, info = oracle.leaf_dtn(p, h, kappa, b)
    assert info == 0
    for _ in range(2):
        u = TensorPoly.random(rng, p, lo + h / 2, h)
        f = -u.laplacian(xyz) - kappa ** 2 * b * u.value(xyz)
        v, hf, info = oracle.leaf_particular(p, h, kappa, b, f)
        ub = u.value(xyz[face])
        ui = u.value(xyz[interior])
        scale = np.abs(ui).max()
        assert np.abs(v[0] + S @ ub - ui).max() < 1e-10 * scale
        dn = (u.grad(xyz[face]) * FACE_NORMALS[fid]).sum(axis=1)
        assert np.abs(T @ ub + hf[0] - dn).max() < 1e-10 * np.abs(T).max() * scale
        ur, info = oracle.leaf_reconstruct(p, h, kappa, b, v, ub)
        assert np.abs(ur[0] - ui).max() < 1e-10 * scale


def test_residuals_and_batch_invariance():
    p, h = 8, (0.125,) * 3
    field = hi.fourier_b_field()
    b0 = field.b(oracle.node_coords(p, (0.0, 0.0, 0.0), h))
    b1 = field.b(oracle.node_coords(p, (0.5, 0.375, 0.75), h))
    Aii, Aib, _, _ = oracle.split_blocks(p, oracle.leaf_matrix(p, h, 40.0, b1))
    T, S, info = oracle.leaf_dtn(p, h, 40.0, b1)
    assert np.abs(Aii @ S + Aib).max() < 1e-13 * np.abs(Aii).max() * np.abs(S).max() * Aii.shape[0] ** 0.5
    Tb, Sb, st = oracle.batch_dtn(p, h, 40.0, np.stack([b0, b1, b1, b0]), want_S=True, nthreads=2)
    assert (st == 0).all()
    np.testing.assert_array_equal(Tb[1], Tb[2])
    np.testing.assert_array_equal(Tb[0], Tb[3])
    np.testing.assert_array_equal(Tb[1], T)
    np.testing.assert_array_equal(Sb[1], S)


def _sym_perm(p, fmap):
    """Permutation of the kept face nodes induced by a grid symmetry."""
    interior, face, _ = kept_grid_indices(p)
    n = len(interior)
    perm = []
    for g in face:
        i, j, k = g % p, (g // p) % p, g // (p * p)
        i2, j2, k2 = fmap(i, j, k)
        perm.append(oracle.kept_index(p, i2, j2, k2) - n)
    return np.asarray(perm)


@pytest.mark.parametrize("sym", ["reflect_x", "swap_xy", "rotate_xyz"])
def test_cube_symmetry_constant_b(sym):
    p = 7
    e = p - 1
    T, _, _ = oracle.leaf_dtn(p, (0.25,) * 3, 9.0, np.full(p ** 3, 0.8))
    fmap = {"reflect_x": lambda i, j, k: (e - i, j, k),
            "swap_xy": lambda i, j, k: (j, i, k),
            "rotate_xyz": lambda i, j, k: (k, i, j)}[sym]
    P = _sym_perm(p, fmap)
    assert sorted(P) == list(range(T.shape[0]))
    assert np.abs(T[np.ix_(P, P)] - T).max() < 1e-11 * np.abs(T).max()


# ------------------------------------------------------------------ global (Sec. 3.2, Sec. 4.1)

def _manufactured_fns(kappa):
    return (lambda x: np.ones(len(x)), lambda x: hi.manufactured(x, kappa)[1],
            lambda x: hi.manufactured(x, kappa)[2])


@pytest.mark.parametrize("kappa", [0.0, 10.0])
def test_e2e_equals_dense_bruteforce(kappa):
    grid = gs.InterfaceGrid(8, (2, 2, 2))
    b_fn, f_fn, g_fn = _manufactured_fns(kappa)
    r = gs.hps_solve(grid, kappa, b_fn, f_fn, g_fn)
    d = gs.dense_global_solve(grid, kappa, b_fn, f_fn, g_fn)
    assert grid.n_iface == 432
    scale = np.abs(d["u_int"]).max()
    assert np.abs(r["u_int"] - d["u_int"]).max() < 1e-11 * scale
    assert np.abs(r["u_iface"] - d["u_iface"]).max() < 1e-11 * scale


def test_e2e_variable_b_equals_dense_bruteforce():
    grid = gs.InterfaceGrid(6, (2, 1, 2), L=(1.0, 0.5, 1.0))
    kappa = 8.0
    r = gs.hps_solve(grid, kappa, hi.gaussian_dip_b, lambda x: np.ones(len(x)), lambda x: 0 * x[:, 0])
    d = gs.dense_global_solve(grid, kappa, hi.gaussian_dip_b, lambda x: np.ones(len(x)), lambda x: 0 * x[:, 0])
    scale = np.abs(d["u_int"]).max()
    assert np.abs(r["u_int"] - d["u_int"]).max() < 1e-11 * scale


def test_manufactured_spectral_convergence():
    kappa = 10.0
    errs = []
    for p in (6, 8, 10, 12):
        grid = gs.InterfaceGrid(p, (2, 2, 2))
        r = gs.hps_solve(grid, kappa, *_manufactured_fns(kappa))
        ui = hi.manufactured(gs.interior_coords(grid), kappa)[0]
        ub = hi.manufactured(gs.iface_coords(grid), kappa)[0]
        num = np.sqrt(((r["u_int"] - ui) ** 2).sum() + ((r["u_iface"] - ub) ** 2).sum())
        errs.append(num / np.sqrt((ui ** 2).sum() + (ub ** 2).sum()))
    errs = np.array(errs)
    assert np.all(errs[1:] < errs[:-1] / 30), errs        # spectral decay in p
    assert errs[-1] < 2e-10, errs


def _green_error(p, nb, kappa):
    """Relative l2 error over the interior and interface nodes of the two-level
    solve of Lap u + kappa^2 u = 0 on the Sec. 4.1 box with the Green's
    function's boundary values."""
    grid = gs.InterfaceGrid(p, nb, lo=hi.GREEN_LO, L=hi.GREEN_L)
    g = lambda x: hi.green(x, kappa)
    r = gs.hps_solve(grid, kappa, lambda x: np.ones(len(x)), lambda x: np.zeros(len(x)), g)
    ue = np.concatenate([g(gs.interior_coords(grid)).reshape(-1), g(gs.iface_coords(grid))])
    uc = np.concatenate([r["u_int"].reshape(-1), r["u_iface"]])
    return np.linalg.norm(uc - ue) / np.linalg.norm(ue)


def test_green_function_accuracy_of_sec_4_1():
    """Sec. 4.1: with the Green's function as exact solution on
    [-1.1, 0.1] x [1, 2] x [1.2, 2.2], the Poisson error decays spectrally in
    p and under h-refinement and reaches the paper's floor (about 1e-13);
    the Helmholtz error at kappa = 16 also decays in p."""
    e = [_green_error(p, (2, 2, 2), 0.0) for p in (6, 8, 10, 12)]
    assert all(b < a / 20 for a, b in zip(e, e[1:])), e
    assert e[-1] < 1e-12, e
    assert _green_error(8, (3, 3, 3), 0.0) < e[1] / 4          # h-refinement at fixed p
    eh = [_green_error(p, (2, 2, 2), 16.0) for p in (8, 10, 12)]
    assert all(b < a / 10 for a, b in zip(eh, eh[1:])), eh


# ------------------------------------------------------------------ time stepping (Sec. 4.4)

@pytest.mark.parametrize("kappa", [0.0, 3.0])
def test_apply_interior_exact_on_polynomials(kappa):
    """A u at the interior nodes for a polynomial field of degree < p in each
    variable: the collocation Laplacian is exact there, so A u = -Lap u - kappa^2 b u
    to rounding (an independent closed form; a wrong sign, axis or scale of a
    line term fails it)."""
    p, h, lo = 8, np.array([0.5, 0.4, 0.3]), np.array([0.1, 0.2, 0.3])
    xyz = oracle.node_coords(p, lo, h)
    x, y, z = xyz.T
    u = x ** 2 * y + z ** 3 + x * y * z - 2.0 * y ** 4
    lap = 2.0 * y + 6.0 * z - 24.0 * y ** 2
    b = np.cos(x) + 2.0
    out = oracle.apply_interior(p, h, kappa, b, u)
    ii = gs.interior_grid_indices(p)
    exp = -lap - kappa ** 2 * b * u
    assert np.abs(out[ii] - exp[ii]).max() < 1e-11 * np.abs(exp[ii]).max()
    mask = np.ones(p ** 3, dtype=bool)
    mask[ii] = False
    assert np.all(out[mask] == 0.0)


@pytest.mark.parametrize("p", [6, 9])
def test_first_order_term_exact_on_polynomials(p):
    """div(beta u) for polynomial beta and u (each product of degree < p in every
    variable) is exact under collocation: the interior rows of A with beta
    reproduce -Lap u + div(beta u) - kappa^2 b u to rounding."""
    h, lo, kappa = np.array([0.4, 0.5, 0.3]), np.array([0.2, -0.1, 0.3]), 2.0
    xyz = oracle.node_coords(p, lo, h)
    x, y, z = xyz.T
    u = x * y + z ** 2
    beta = np.stack([y, x * z, 1.0 + x])
    b = 1.0 + 0.5 * np.sin(x + y)
    div = y ** 2 + x * z * x + (1.0 + x) * 2.0 * z        # d/dx(y u) + d/dy(x z u) + d/dz((1 + x) u)
    exp = -2.0 + div - kappa ** 2 * b * u
    ii = gs.interior_grid_indices(p)
    out = oracle.apply_interior(p, h, kappa, b, u, beta)
    assert np.abs(out[ii] - exp[ii]).max() < 1e-11 * np.abs(exp[ii]).max()
    # the same matrix with the sign of the first-order term flipped misses by its size
    bad = oracle.apply_interior(p, h, kappa, b, u, -beta)
    assert np.abs(bad[ii] - exp[ii]).max() > 0.1 * np.abs(div[ii]).max()


def test_convection_diffusion_step_equals_dense_bruteforce():
    """One Crank-Nicolson step of u_t = kappa_d Lap u - div(vel u) through the
    two-level HPS solve equals the dense solve of the same global system."""
    grid = gs.InterfaceGrid(6, (2, 1, 2), L=(1.0, 0.5, 1.0))
    u0 = lambda X: np.sin(np.pi * X[:, 0]) * np.sin(2 * np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
    vel = lambda X: np.stack([-np.cos(X[:, 0]) * np.sin(X[:, 1]) * X[:, 2],
                              np.sin(X[:, 0]) * np.cos(X[:, 1]) * X[:, 2], 0 * X[:, 0]], axis=1)
    r = gs.crank_nicolson_heat(grid, 0.05, 0.05, 1, u0, vel)
    p, b = grid.p, -np.ones(grid.p ** 3)
    xyz = [oracle.node_coords(p, grid.box_lo(bx), grid.h) for bx in range(grid.nbox)]
    f = [2 * r["c"] * u0(x) - oracle.apply_interior(p, grid.h, r["kappa"], b, u0(x), r["beta"][bx])
         for bx, x in enumerate(xyz)]
    d = gs.dense_global_solve(grid, r["kappa"], lambda X: -np.ones(len(X)), None, lambda X: 0 * X[:, 0],
                              f_boxes=f, beta_boxes=r["beta"])
    scale = np.abs(d["u_int"]).max()
    assert np.abs(r["u_int"] - d["u_int"]).max() < 1e-11 * scale
    assert np.abs(r["u_iface"] - d["u_iface"]).max() < 1e-11 * scale


def test_crank_nicolson_step_equals_dense_bruteforce():
    """One Crank-Nicolson step through the two-level HPS solve equals the dense
    solve of the same global collocation system with the same right-hand
    side."""
    grid = gs.InterfaceGrid(6, (2, 1, 2), L=(1.0, 0.5, 1.0))
    u0 = lambda X: np.sin(np.pi * X[:, 0]) * np.sin(2 * np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
    r = gs.crank_nicolson_heat(grid, 0.1, 0.05, 1, u0)
    p, b = grid.p, -np.ones(grid.p ** 3)
    xyz = [oracle.node_coords(p, grid.box_lo(bx), grid.h) for bx in range(grid.nbox)]
    f = [2 * r["c"] * u0(x) - oracle.apply_interior(p, grid.h, r["kappa"], b, u0(x)) for x in xyz]
    d = gs.dense_global_solve(grid, r["kappa"], lambda X: -np.ones(len(X)), None, lambda X: 0 * X[:, 0],
                              f_boxes=f)
    scale = np.abs(d["u_int"]).max()
    assert np.abs(r["u_int"] - d["u_int"]).max() < 1e-11 * scale
    assert np.abs(r["u_iface"] - d["u_iface"]).max() < 1e-11 * scale


def test_crank_nicolson_second_order_in_time():
    """u_t = kappa_d Lap u on the unit cube with u = 0 on its boundary: from
    u0 = sin(pi x) sin(pi y) sin(pi z) the exact solution decays as
    exp(-3 pi^2 kappa_d t).  At p = 10 the spatial error is far below the time
    error, so halving dt divides the error by four (second order)."""
    grid = gs.InterfaceGrid(10, (2, 2, 2))
    u0 = lambda X: np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
    kd, T = 0.05, 0.5
    ex = np.exp(-3 * np.pi ** 2 * kd * T) * u0(gs.interior_coords(grid).reshape(-1, 3)).reshape(grid.nbox, -1)
    err = [np.abs(gs.crank_nicolson_heat(grid, kd, T / s, s, u0)["u_int"] - ex).max() for s in (5, 10)]
    assert 3.8 < err[0] / err[1] < 4.2, err
    assert err[1] < 2e-4, err


# ------------------------------------------------------------------ planted mistakes

def test_pins_catch_planted_mistakes():
    """Mistakes planted in oracle outputs fail the pins above.  The first is
    the reading that Algorithm 1's third bullet suggests (T = A_bi S, no A_bb);
    Eq. 8 gives A_bb + A_bi S, and T 1 = 0 at kappa = 0 decides it."""
    p, h = 6, np.array([0.5, 0.5, 0.5])
    A = oracle.leaf_matrix(p, h, 0.0, np.ones(p ** 3))
    Aii, Aib, Abi, Abb = oracle.split_blocks(p, A)
    T, S, _ = oracle.leaf_dtn(p, h, 0.0, np.ones(p ** 3))
    one = np.ones(T.shape[1])
    tol = 1e-12 * np.abs(T).max()
    assert np.abs(T @ one).max() < tol
    assert np.abs((Abi @ S) @ one).max() > 1e3 * tol                 # dropped A_bb
    assert np.abs((Abb - Abi @ S) @ one).max() > 1e3 * tol           # wrong sign of S
    xyz = oracle.node_coords(p, (0, 0, 0), h)
    interior, face, fid = kept_grid_indices(p)
    phi = xyz[face][:, 0]                                           # linear trace x
    dn = FACE_NORMALS[fid][:, 0]
    assert np.abs(T @ phi - dn).max() < 1e-10
    assert np.abs(-T @ phi - dn).max() > 0.5                         # inward normal
    assert np.abs(T.T @ phi - dn).max() > 1e-6                       # transposed T
