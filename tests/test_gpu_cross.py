"""Cross-term leaves on Legendre face grids (Remark 1 of Sec. 2.1, Sec. 4.3)
on the GPU through the C ABI, against the FP64 oracle (oracle/cross.py).

FP64 path: T, S, v, h and the reconstruction within 1e-11 of the oracle
(relative Frobenius per box and element-wise against the largest entry);
the curved-domain problem solved with the GPU's leaf maps and a host sparse
LU equals the oracle's two-level solve and reaches the plane wave.
"""
from __future__ import annotations

import numpy as np
import pytest

import hps_inputs as hi
import oracle
import paper_2503_04033_gb300 as H
from oracle import cross as cx
from tests._cases import max_rel, rel_fro

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _fields(node_fn, p, lows, h, curved):
    C, d, b = [], [], []
    for lo in lows:
        x = node_fn(p, lo, h)
        if curved:
            Cx, dx = hi.curved_coefficients(x)
            bx = np.ones(len(x))
        else:
            Cx, dx, bx = hi.cross_field(x)
        C.append(Cx)
        d.append(dx)
        b.append(bx)
    return np.stack(C), np.stack(d), np.stack(b)


def gpu_cross(p, h, kappa, lows, curved, nrhs=0, loads=None, want_S=True):
    import torch
    n, m = H.hps_leaf_cross_sizes(p)
    nbox = len(lows)
    C, d, b = _fields(H.hps_leaf_nodes, p, lows, h, curved)
    T = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
    S = torch.empty(nbox, n, m, dtype=torch.float64, device="cuda") if want_S else None
    st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
    f = v = hf = None
    if nrhs:
        f = _dev(np.stack([hi.load_values(loads, H.hps_leaf_nodes(p, lo, h)) for lo in lows]))
        v = torch.empty(nbox, nrhs, n, dtype=torch.float64, device="cuda")
        hf = torch.empty(nbox, nrhs, m, dtype=torch.float64, device="cuda")
    H.hps_leaf_cross_solve(p, h, kappa, nbox, _dev(C), _dev(d), _dev(b), nrhs, f, T, S, v, hf, st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all(), st
    out = (T.cpu().numpy(), S.cpu().numpy() if want_S else None)
    if nrhs:
        out += (v.cpu().numpy(), hf.cpu().numpy())
    return out


def _close(got, ref, tol, what):
    assert rel_fro(got, ref).max() < tol, (what, rel_fro(got, ref).max())
    assert max_rel(got, ref) < tol, (what, max_rel(got, ref))


@pytest.mark.parametrize("p", [4, 5, 6, 8, 10])
@pytest.mark.parametrize("curved", [False, True], ids=["cross-field", "curved-map"])
def test_cross_leaf_parity(p, curved):
    """T, S, v and h of three boxes (anisotropic sides) with every cross term
    (or the curved domain's map) against the oracle's dense definitions."""
    h = np.array([0.3, 0.25, 0.35])
    rng = np.random.default_rng(p)
    lows = np.asarray(hi.CURVED_LO) + rng.integers(0, 3, size=(3, 3)) * h
    kappa, nrhs = 6.0, 3
    loads = hi.fourier_b_per_box(nrhs, 40 + p)
    T, S, v, hf = gpu_cross(p, h, kappa, lows, curved, nrhs, loads)
    C, d, b = _fields(oracle.node_coords, p, lows, h, curved)
    for bx, lo in enumerate(lows):
        x = oracle.node_coords(p, lo, h)
        To, So, vo, ho = cx.leaf_cross(p, h, kappa, C[bx], d[bx], b[bx], hi.load_values(loads, x))
        _close(T[bx:bx + 1], To[None], TOL, ("T", bx))
        _close(S[bx:bx + 1], So[None], TOL, ("S", bx))
        _close(v[bx:bx + 1], vo[None], TOL, ("v", bx))
        _close(hf[bx:bx + 1], ho[None], TOL, ("h", bx))


def test_cross_nodes_and_reconstruct():
    """The library's Legendre face nodes equal the oracle's; u_i = v + S u_b on
    the device equals the oracle's product."""
    import torch
    p, h = 7, np.array([0.2, 0.3, 0.25])
    lows = np.array([[0.1, 0.2, 0.3], [0.5, -0.4, 0.0]])
    for lo in lows:
        assert np.abs(H.hps_leaf_cross_nodes(p, lo, h) - cx.legendre_face_coords(p, lo, h)).max() < 1e-15
    T, S, v, hf = gpu_cross(p, h, 3.0, lows, False, 2, hi.fourier_b_per_box(2, 9))
    n, m = H.hps_leaf_cross_sizes(p)
    ub = hi.random_boundary_data(len(lows), 2, m)
    ui = torch.empty(len(lows), 2, n, dtype=torch.float64, device="cuda")
    H.hps_leaf_cross_reconstruct(p, len(lows), 2, _dev(S), _dev(v), _dev(ub), ui)
    torch.cuda.synchronize()
    ref = v + np.einsum("bnm,brm->brn", S, ub)
    _close(ui.cpu().numpy(), ref, 1e-13, "u_i")


def test_curved_domain_solve_with_gpu_leaves():
    """Sec. 4.3's curved domain on 4 x 2 x 2 boxes at p = 8: the GPU's leaf maps
    assembled into the interface system on the host (the oracle's numbering
    and sparse LU) and the GPU's reconstruction give the oracle's two-level
    solution to 1e-10, and the plane wave to the discretisation error."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import torch
    p = 8
    kappa = float(np.linalg.norm(hi.CURVED_K))
    grid = cx.LegendreGrid(p, (4, 2, 2), lo=hi.CURVED_LO, L=hi.CURVED_L)
    lows = np.stack([grid.box_lo(bx) for bx in range(grid.nbox)])
    n, m = H.hps_leaf_cross_sizes(p)
    T, S = gpu_cross(p, grid.h, kappa, lows, True)
    g = hi.curved_plane_wave(grid.dirichlet_coords())
    rows, cols, vals = [], [], []
    rhs = np.zeros(grid.n_iface)
    for bx in range(grid.nbox):
        isi, gid = grid.local_to_global(bx)
        ii, dd = np.nonzero(isi)[0], np.nonzero(~isi)[0]
        r, c = np.meshgrid(gid[ii], gid[ii], indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(T[bx][np.ix_(ii, ii)].ravel())
        np.add.at(rhs, gid[ii], -(T[bx][np.ix_(ii, dd)] @ g[gid[dd]]))
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(grid.n_iface, grid.n_iface)).tocsc()
    u_if = spla.splu(K).solve(rhs)
    ub = np.empty((grid.nbox, 1, m))
    for bx in range(grid.nbox):
        isi, gid = grid.local_to_global(bx)
        ub[bx, 0, isi] = u_if[gid[isi]]
        ub[bx, 0, ~isi] = g[gid[~isi]]
    ui = torch.empty(grid.nbox, 1, n, dtype=torch.float64, device="cuda")
    H.hps_leaf_cross_reconstruct(p, grid.nbox, 1, _dev(S), None, _dev(ub), ui)
    torch.cuda.synchronize()
    ui = ui.cpu().numpy()[:, 0, :]
    _, u_ref = cx.hps_solve_cross(grid, kappa, lambda x: hi.curved_coefficients(x)[0],
                                  lambda x: hi.curved_coefficients(x)[1], lambda x: np.ones(len(x)),
                                  lambda x: np.zeros(len(x)), hi.curved_plane_wave)
    scale = np.abs(u_ref).max()
    assert np.abs(ui - u_ref).max() < 1e-10 * scale
    exact = np.stack([hi.curved_plane_wave(H.hps_leaf_nodes(p, lo, grid.h))[cx.interior_set(p)] for lo in lows])
    assert np.abs(ui - exact).max() < 1e-3 * np.abs(exact).max()


def test_cross_argument_errors():
    import torch
    b = torch.ones(1, 27, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HpsError) as e:
        H.hps_leaf_cross_solve(3, 1.0, 0.0, 1, b, None, b, 0, None, b, None)
    assert e.value.status == H.HPS_EINVAL
    with pytest.raises(H.HpsError):
        H.hps_leaf_cross_sizes(17)
