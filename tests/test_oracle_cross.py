"""Pins of the cross-term oracle (oracle/cross.py) to what the mathematics fixes.

Remark 1 (Sec. 2.1): with cross terms d_a d_b u the face data lives on
(p-1) x (p-1) Gauss-Legendre grids; Sec. 4.3's curved domain is the case that
needs it.  Each pin would fail for a plausible mistake in the oracle: the
Legendre nodes against LAPACK-backed numpy, the interpolations and the
operator exact on polynomials of their degree, the DtN map exact on
polynomial solutions (a wrong sign, factor or index in a cross term, the
normal derivative or an interpolation breaks it), the two-level solve equal
to a dense solve of the same discrete system and converging spectrally to an
exact plane wave on the curved domain.
"""
from __future__ import annotations

import numpy as np
import pytest

import hps_inputs as hi
import oracle
from oracle import cross as cx


def _poly3(rng, deg):
    """A random tensor polynomial of degree <= deg per variable, with its
    value, gradient and Hessian functions (monomials written out)."""
    c = rng.standard_normal((deg + 1, deg + 1, deg + 1)) / (1 + np.arange(deg + 1))[:, None, None]

    def val(x, dx=(0, 0, 0)):
        out = np.zeros(len(x))
        for i in range(deg + 1):
            for j in range(deg + 1):
                for k in range(deg + 1):
                    e = (i, j, k)
                    coef = c[i, j, k]
                    term = np.full(len(x), coef)
                    for a in range(3):
                        ea, da = e[a], dx[a]
                        if da > ea:
                            term = 0.0 * term
                            break
                        fac = 1.0
                        for t in range(da):
                            fac *= ea - t
                        term = term * fac * x[:, a] ** (ea - da)
                    out += term
        return out
    return val


def _const_C(c12=0.3, c13=-0.2, c23=0.15, diag=(1.0, 1.4, 0.8)):
    return np.array([diag[0], diag[1], diag[2], c12, c13, c23])


def _var_C(x):
    """A smooth symmetric positive-definite coefficient field with all cross terms."""
    C = np.stack([1.0 + 0.2 * np.sin(x[:, 0]), 1.3 + 0.1 * x[:, 1], 0.9 + 0.05 * x[:, 2] ** 2,
                  0.25 * np.cos(x[:, 2]), -0.15 + 0.05 * x[:, 0], 0.1 * np.sin(x[:, 1])])
    return C


def test_legendre_nodes_match_numpy_leggauss():
    for N in range(1, 15):
        ref, _ = np.polynomial.legendre.leggauss(N)
        assert np.abs(cx.legendre_nodes(N) - np.sort(ref)).max() < 1e-14


@pytest.mark.parametrize("p", [4, 6, 9])
def test_interpolation_matrices_exact_on_polynomials(p):
    G, Q = cx.interp_matrices(p)
    t, g = oracle.nodes(p), cx.legendre_nodes(p - 1)
    for deg in range(p - 1):            # G: from p-1 Legendre nodes, exact to degree p-2
        assert np.abs(G @ g ** deg - t ** deg).max() < 1e-12
    for deg in range(p):                # Q: from p Chebyshev nodes, exact to degree p-1
        assert np.abs(Q @ t ** deg - g ** deg).max() < 1e-12
    assert np.abs(G[:, :].sum(axis=1) - 1).max() < 1e-13 and np.abs(Q.sum(axis=1) - 1).max() < 1e-13


@pytest.mark.parametrize("p", [5, 7])
def test_operator_exact_on_tensor_polynomials(p):
    """A u at every node equals -sum C_ab u_ab + d . grad u - kappa^2 b u for a
    polynomial of degree p-1 per variable, with variable C (all cross terms),
    d and b, on an anisotropic box."""
    rng = np.random.default_rng(p)
    lo, h, kappa = np.array([0.3, -0.2, 1.1]), np.array([0.4, 0.25, 0.3]), 3.0
    x = oracle.node_coords(p, lo, h)
    u = _poly3(rng, p - 1)
    C = _var_C(x)
    d = np.stack([np.cos(x[:, 1]), 0.3 * x[:, 0], -0.2 * np.ones(len(x))])
    b = 1.0 + 0.3 * x[:, 2]
    A = cx.cross_operator(p, h, kappa, C, d, b)
    pairs = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (0, 2): 4, (1, 2): 5}
    exact = -kappa ** 2 * b * u(x)
    for (a, c), ci in pairs.items():
        dd = [0, 0, 0]
        dd[a] += 1
        dd[c] += 1
        exact -= (1.0 if a == c else 2.0) * C[ci] * u(x, tuple(dd))
    for a in range(3):
        dd = [0, 0, 0]
        dd[a] = 1
        exact += d[a] * u(x, tuple(dd))
    got = A @ u(x)
    assert np.abs(got - exact).max() < 1e-9 * np.abs(exact).max()


def _harmonic_quadratics(C):
    """Quadratics u = x^T Q x + l^T x with sum_ab C_ab Q_ab = 0 (so that
    -sum C_ab u_ab = 0): returns (Q, l) pairs."""
    Cm = np.array([[C[0], C[3], C[4]], [C[3], C[1], C[5]], [C[4], C[5], C[2]]])
    out = [(np.zeros((3, 3)), np.array([0.7, -0.4, 1.1]))]          # linear
    out.append((np.array([[0, 1, 0], [1, 0, 0], [0, 0, -2 * Cm[0, 1] / Cm[2, 2]]]) * 0.5, np.zeros(3)))   # x y - c12/c33 z^2
    out.append((np.diag([Cm[1, 1], -Cm[0, 0], 0.0]), np.array([0.0, 0.3, 0.0])))                        # c22 x^2 - c11 y^2
    out.append((np.array([[0, 0, 0], [0, 0, 1], [0, 1, 0]]) * 0.5 - np.diag([Cm[1, 2] / Cm[0, 0], 0, 0]), np.zeros(3)))
    return out


@pytest.mark.parametrize("p", [5, 6, 8])
def test_dtn_exact_on_operator_harmonic_quadratics(p):
    """kappa = 0, constant C with cross terms: for linear and C-harmonic
    quadratic u (degree 2 <= p - 2, exact on the Legendre face grids), S g = u
    at the interior nodes and T g = du/dn at the Legendre nodes; T 1 = 0."""
    lo, h = np.array([0.2, -0.5, 0.4]), np.array([0.5, 0.35, 0.45])
    x = oracle.node_coords(p, lo, h)
    xf = cx.legendre_face_coords(p, lo, h)
    Cc = _const_C()
    C = np.repeat(Cc[:, None], p ** 3, axis=1)
    T, S, _, _ = cx.leaf_cross(p, h, 0.0, C, None, np.ones(p ** 3))
    Iset = cx.interior_set(p)
    normals = np.zeros((len(xf), 3))
    pl = (p - 1) ** 2
    for f in range(6):
        normals[f * pl:(f + 1) * pl, f // 2] = -1.0 if f % 2 == 0 else 1.0
    assert np.abs(T.sum(axis=1)).max() < 1e-10 * np.abs(T).max()
    for Qm, l in _harmonic_quadratics(Cc):
        u = lambda y: np.einsum("ni,ij,nj->n", y, Qm, y) + y @ l
        grad = lambda y: 2 * y @ Qm + l
        g = u(xf)
        assert np.abs(S @ g - u(x)[Iset]).max() < 1e-10 * max(1.0, np.abs(u(x)).max())
        dn = (grad(xf) * normals).sum(axis=1)
        assert np.abs(T @ g - dn).max() < 1e-9 * max(1.0, np.abs(dn).max())


@pytest.mark.parametrize("p", [6, 8])
def test_polynomial_reproduction_any_coefficients(p):
    """Variable C, d, b and kappa != 0: for a polynomial u of degree p - 2 per
    variable with f = A u, v + S g = u at the interior nodes and T g + h =
    du/dn at the Legendre nodes (collocation and every interpolation exact)."""
    rng = np.random.default_rng(10 + p)
    lo, h, kappa = np.array([1.1, -1.0, -1.2]), np.array([0.5, 0.5, 0.7]), 4.0
    x = oracle.node_coords(p, lo, h)
    xf = cx.legendre_face_coords(p, lo, h)
    u = _poly3(rng, p - 2)
    C, d = _var_C(x), np.stack([0.2 * x[:, 1], np.sin(x[:, 0]), 0.1 * np.ones(len(x))])
    b = 1.0 + 0.2 * np.cos(x[:, 0])
    A = cx.cross_operator(p, h, kappa, C, d, b)
    f = A @ u(x)
    T, S, v, hf = cx.leaf_cross(p, h, kappa, C, d, b, f[None, :])
    Iset = cx.interior_set(p)
    g = u(xf)
    scale = np.abs(u(x)).max()
    assert np.abs(v[0] + S @ g - u(x)[Iset]).max() < 1e-9 * scale
    pl = (p - 1) ** 2
    dn = np.empty(len(xf))
    for fc in range(6):
        a = fc // 2
        dd = [0, 0, 0]
        dd[a] = 1
        dn[fc * pl:(fc + 1) * pl] = (-1.0 if fc % 2 == 0 else 1.0) * u(xf[fc * pl:(fc + 1) * pl], tuple(dd))
    assert np.abs(T @ g + hf[0] - dn).max() < 1e-8 * np.abs(dn).max()


def test_planted_missing_cross_factor_fails():
    """A cross term counted once instead of twice (C_ab d_a d_b for a < b
    only) breaks the polynomial reproduction: the pin above detects it."""
    p = 6
    rng = np.random.default_rng(3)
    lo, h = np.zeros(3), np.array([0.5] * 3)
    x = oracle.node_coords(p, lo, h)
    u = _poly3(rng, p - 2)
    C = _var_C(x)
    A = cx.cross_operator(p, h, 0.0, C, None, np.ones(p ** 3))
    C_half = C.copy()
    C_half[3:] *= 0.5
    A_bad = cx.cross_operator(p, h, 0.0, C_half, None, np.ones(p ** 3))
    f = A_bad @ u(x)        # a load from the wrong operator
    T, S, v, hf = cx.leaf_cross(p, h, 0.0, C, None, np.ones(p ** 3), f[None, :])
    g = u(cx.legendre_face_coords(p, lo, h))
    assert np.abs(v[0] + S @ g - u(x)[cx.interior_set(p)]).max() > 1e-4 * np.abs(u(x)).max()
    assert np.abs(A @ u(x) - f).max() > 1e-3 * np.abs(f).max()


@pytest.mark.slow
def test_curved_domain_plane_wave_converges_spectrally():
    """Sec. 4.3: the Helmholtz equation on the sinusoidal domain pulled back to
    the reference box [1.1, 2.1] x [-1, 0] x [-1.2, 0.2]; the exact solution is
    a plane wave sin(k . y) of the physical coordinates with kappa = |k| (so
    f = 0).  On 4 x 2 x 2 boxes the two-level solve's error falls by more than
    10 per two orders (3.9e-3, 1.4e-4, 5.2e-6 at p = 5, 7, 9) and by more than
    5 when the boxes along x1 double (psi oscillates along x1)."""
    kappa = float(np.linalg.norm(hi.CURVED_K))
    uref = hi.curved_plane_wave
    def err(p, nb):
        grid = cx.LegendreGrid(p, nb, lo=hi.CURVED_LO, L=hi.CURVED_L)
        _, u_int = cx.hps_solve_cross(grid, kappa, lambda x: hi.curved_coefficients(x)[0],
                                      lambda x: hi.curved_coefficients(x)[1], lambda x: np.ones(len(x)),
                                      lambda x: np.zeros(len(x)), uref)
        exact = np.stack([uref(oracle.node_coords(p, grid.box_lo(bx), grid.h))[cx.interior_set(p)]
                          for bx in range(grid.nbox)])
        return np.abs(u_int - exact).max() / np.abs(exact).max()

    errs = [err(p, (4, 2, 2)) for p in (5, 7, 9)]
    assert errs[1] < 0.1 * errs[0] and errs[2] < 0.1 * errs[1] and errs[2] < 1e-4, errs
    assert err(7, (2, 2, 2)) > 5.0 * errs[1]          # h-refinement: 2 -> 4 boxes along x1


def test_two_level_solve_equals_dense_global_solve():
    """2 x 1 x 1 boxes, variable C with cross terms: static condensation then
    the interface system (the two-level solve) equals one dense solve of the
    whole discrete system (interior collocation rows of both boxes with their
    face data, flux balance rows at the shared Legendre nodes)."""
    p, kappa = 6, 2.5
    grid = cx.LegendreGrid(p, (2, 1, 1), lo=(0.0, 0.0, 0.0), L=(1.0, 0.6, 0.7))
    Cf = _var_C
    df = lambda x: np.stack([0.1 * x[:, 2], -0.2 * x[:, 0], 0.3 * np.ones(len(x))])
    bf = lambda x: 1.0 + 0.1 * x[:, 1]
    ff = lambda x: np.cos(x[:, 0] + 2 * x[:, 1]) + x[:, 2]
    gf = lambda x: np.sin(x[:, 0]) * np.exp(x[:, 1]) + x[:, 2] ** 2
    u_if, u_int = cx.hps_solve_cross(grid, kappa, Cf, df, bf, ff, gf)
    n, m = cx.sizes_cross(p)
    Iset, Eset = cx.interior_set(p), cx.boundary_set(p)
    P = cx.dirichlet_interp(p)
    NQ = cx.face_projection(p) @ cx.normal_derivative(p, grid.h)
    g = gf(grid.dirichlet_coords())
    nI, nF = grid.nbox * n, grid.n_iface
    K = np.zeros((nI + nF, nI + nF))
    rhs = np.zeros(nI + nF)
    for bx in range(grid.nbox):
        x = oracle.node_coords(p, grid.box_lo(bx), grid.h)
        A = cx.cross_operator(p, grid.h, kappa, Cf(x), df(x), bf(x))
        isi, gid = grid.local_to_global(bx)
        r0 = bx * n
        K[r0:r0 + n, r0:r0 + n] = A[np.ix_(Iset, Iset)]
        AieP = A[np.ix_(Iset, Eset)] @ P[Eset]        # n x m: interior rows against the box's face data
        K[r0:r0 + n, nI + gid[isi]] += AieP[:, isi]
        rhs[r0:r0 + n] = ff(x)[Iset] - AieP[:, ~isi] @ g[gid[~isi]]
        NI = NQ[:, Iset]                               # flux rows of this box at its face nodes
        NE = NQ @ P                                    # flux from its face data
        rows = nI + gid[isi]
        K[np.ix_(rows, np.arange(r0, r0 + n))] += NI[isi]
        K[np.ix_(rows, nI + gid[isi])] += NE[np.ix_(isi, isi)]
        rhs[rows] -= NE[np.ix_(isi, ~isi)] @ g[gid[~isi]]
    sol = np.linalg.solve(K, rhs)
    assert np.abs(sol[nI:] - u_if).max() < 1e-10 * np.abs(u_if).max()
    assert np.abs(sol[:nI].reshape(grid.nbox, n) - u_int).max() < 1e-10 * np.abs(u_int).max()
