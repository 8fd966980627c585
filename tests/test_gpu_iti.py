"""Leaf impedance-to-impedance maps on the GPU through the C ABI, against the
FP64 oracle (oracle/iti.py): element-wise parity on boxes with variable b
and anisotropic sides, including a box at a Dirichlet resonance (where the
DtN map does not exist), and the argument checks."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2503_04033_gb300 as H
from oracle import iti
from tests._cases import max_rel

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _gpu_iti(p, h, kappa, eta, bs):
    import torch
    n, m = H.hps_leaf_sizes(p)
    kind = H.LeafKind(p, h, kappa)
    b = torch.from_numpy(np.ascontiguousarray(np.stack(bs))).cuda()
    R = torch.empty(len(bs), m, m, dtype=torch.complex128, device="cuda")
    st = torch.full((len(bs),), -1, dtype=torch.int32, device="cuda")
    H.hps_leaf_iti(kind, eta, len(bs), b, R, st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all(), st
    return R.cpu().numpy()


@pytest.mark.parametrize("p", [4, 5, 6, 8])
def test_iti_parity(p):
    """Three boxes of a variable field (anisotropic sides), two values of
    eta: every entry within 1e-11 of the oracle's largest."""
    h = np.array([0.3, 0.25, 0.35])
    rng = np.random.default_rng(p)
    lows = rng.uniform(-1, 1, size=(3, 3))
    kappa = 9.0
    bs = []
    for lo in lows:
        x = oracle.node_coords(p, lo, h)
        bs.append(1 + 0.4 * np.sin(2 * x[:, 0] + x[:, 2]) * np.cos(3 * x[:, 1]))
    for eta in (kappa, -3.5):
        R = _gpu_iti(p, h, kappa, eta, bs)
        for bx in range(3):
            Ro = iti.leaf_iti(p, h, kappa, bs[bx], eta)
            assert max_rel(R[bx:bx + 1], Ro[None]) < TOL, (p, eta, bx, max_rel(R[bx:bx + 1], Ro[None]))


def test_iti_at_a_dirichlet_resonance():
    """kappa^2 the smallest eigenvalue of the box's interior block (b = 1,
    p = 8): the GPU map equals the oracle's and stays of moderate norm."""
    p, h = 8, np.array([0.2, 0.2, 0.2])
    n, m = oracle.sizes(p)
    Aii = oracle.leaf_matrix(p, h, 0.0, np.ones(p ** 3))[:n, :n]
    ev = np.linalg.eigvals(Aii)
    kappa = float(np.sqrt(np.sort(ev[np.abs(ev.imag) < 1e-8].real)[0]))
    R = _gpu_iti(p, h, kappa, kappa, [np.ones(p ** 3)])
    Ro = iti.leaf_iti(p, h, kappa, np.ones(p ** 3), kappa)
    assert max_rel(R, Ro[None]) < 1e-10
    assert np.linalg.norm(R[0], 2) < 10.0


def test_iti_argument_errors():
    import torch
    b = torch.ones(1, 64, dtype=torch.float64, device="cuda")
    R = torch.empty(1, 24, 24, dtype=torch.complex128, device="cuda")
    for kind, eta in ((H.LeafKind(3, 0.5, 1.0), 1.0), (H.LeafKind(4, 0.5, 1.0), 0.0),
                      (H.LeafKind(4, -0.5, 1.0), 1.0), (H.LeafKind(17, 0.5, 1.0), 1.0)):
        with pytest.raises(H.HpsError) as e:
            H.hps_leaf_iti(kind, eta, 1, b, R)
        assert e.value.status == H.HPS_EINVAL


@pytest.mark.parametrize("p", [5, 6])
def test_iti_operators_with_loads_parity(p):
    """S, v and hout of hps_leaf_iti_solve (two loads) against the oracle's
    leaf_iti_ops, every entry within 1e-11 of the largest."""
    import torch
    h = np.array([0.3, 0.25, 0.35])
    kappa, eta, nrhs = 8.0, 5.0, 2
    rng = np.random.default_rng(30 + p)
    lows = rng.uniform(-1, 1, size=(2, 3))
    n, m = H.hps_leaf_sizes(p)
    bs, fs = [], []
    for lo in lows:
        x = oracle.node_coords(p, lo, h)
        bs.append(1 + 0.3 * np.cos(x[:, 0] - x[:, 1]))
        fs.append(np.stack([np.sin(x[:, 2] + c) for c in range(nrhs)]))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    c128 = lambda *s: torch.empty(*s, dtype=torch.complex128, device="cuda")
    R, S, v, ho = c128(2, m, m), c128(2, n, m), c128(2, nrhs, n), c128(2, nrhs, m)
    st = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    H.hps_leaf_iti_solve(H.LeafKind(p, h, kappa), eta, 2, dev(np.stack(bs)), nrhs, dev(np.stack(fs)), R, S, v, ho, st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    for bx in range(2):
        Ro, So, vo, hoo = iti.leaf_iti_ops(p, h, kappa, bs[bx], eta, fs[bx])
        for got, want in ((R, Ro), (S, So), (v, vo), (ho, hoo)):
            assert max_rel(got[bx:bx + 1].cpu().numpy(), want[None]) < TOL


def test_iti_two_level_solve_at_a_resonant_box():
    """2 x 2 x 2 boxes at p = 8 with the corner box at a Dirichlet resonance
    (b = 1 there, 1.25 elsewhere), a load and Dirichlet data: the GPU's ItI
    leaves, the library's host assembly, a host sparse LU and the GPU
    reconstruction give the oracle's ItI solve and the dense collocation
    solve of the whole system (which the DtN route misses by per cents)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import torch
    from oracle.global_solve import InterfaceGrid, dense_global_solve, face_node_grid_indices
    p = 8
    grid = InterfaceGrid(p, (2, 2, 2))
    n, m = H.hps_leaf_sizes(p)
    Aii = oracle.leaf_matrix(p, grid.h, 0.0, np.ones(p ** 3))[:n, :n]
    ev = np.linalg.eigvals(Aii)
    kappa = float(np.sqrt(np.sort(ev[np.abs(ev.imag) < 1e-8].real)[0]))
    eta = kappa
    b_fn = lambda x: np.where((x[:, 0] < 0.5 - 1e-12) & (x[:, 1] < 0.5 - 1e-12) & (x[:, 2] < 0.5 - 1e-12), 1.0, 1.25)
    f_fn = lambda x: np.cos(2 * x[:, 2])
    g_fn = lambda x: np.cos(3 * x[:, 0] + x[:, 1]) + x[:, 2]
    xs = [H.hps_leaf_nodes(p, grid.box_lo(bx), grid.h) for bx in range(8)]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    c128 = lambda *s: torch.empty(*s, dtype=torch.complex128, device="cuda")
    R, S, v, ho = c128(8, m, m), c128(8, n, m), c128(8, 1, n), c128(8, 1, m)
    st = torch.full((8,), -1, dtype=torch.int32, device="cuda")
    H.hps_leaf_iti_solve(H.LeafKind(p, grid.h, kappa), eta, 8, dev(np.stack([b_fn(x) for x in xs])), 1,
                         dev(np.stack([f_fn(x)[None, :] for x in xs])), R, S, v, ho, st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    r, c, vals = H.hps_iti_assemble(p, (2, 2, 2), R.cpu().numpy())
    A = sp.coo_matrix((vals, (r, c)), shape=(8 * m, 8 * m)).tocsc()
    fi = face_node_grid_indices(p)
    rhs = H.hps_iti_rhs(p, (2, 2, 2), eta, ho.cpu().numpy()[:, 0, :], np.stack([g_fn(x[fi]) for x in xs]))
    fin = spla.splu(A).solve(rhs)
    ui, ub = c128(8, 1, n), c128(8, 1, m)
    H.hps_leaf_iti_reconstruct(p, eta, 8, 1, R, S, v, ho, dev(fin.reshape(8, 1, m)), ui, ub)
    torch.cuda.synchronize()
    ui = ui.cpu().numpy()[:, 0, :]
    ro = np.array(iti.iti_solve(grid, kappa, eta, b_fn, f_fn, g_fn)["u_int"])
    ref = np.asarray(dense_global_solve(grid, kappa, b_fn, f_fn, g_fn)["u_int"])
    scale = np.abs(ref).max()
    assert np.abs(ui - ro).max() < 1e-10 * scale
    assert np.abs(ui - ref).max() < 1e-10 * scale
    # the face values: the trace of the solution on every box's face nodes
    ro_b = np.array(iti.iti_solve(grid, kappa, eta, b_fn, f_fn, g_fn)["u_b"])
    assert np.abs(ub.cpu().numpy()[:, 0, :] - ro_b).max() < 1e-10 * scale
