"""The 2-D leaf reduction on the GPU against the 2-D oracle: T, S, v, h per
box, and a two-level solve whose leaf work runs on the device (interface
system by the host sparse LU, as in the oracle)."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import paper_2503_04033_gb300 as H
from oracle import global_solve_2d as g2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = H.hps_create(0, 0)
    yield c
    H.hps_destroy(c)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _b_field(x):
    return 1.0 + 0.4 * np.sin(3 * x[:, 0] - x[:, 1])


def _loads(x, nrhs):
    return np.stack([np.cos((r + 1) * x[:, 0]) * np.exp(-r * x[:, 1]) for r in range(nrhs)])


@pytest.mark.parametrize("p,kappa,nrhs", [(5, 0.0, 0), (9, 7.0, 2), (16, 12.0, 1), (13, 3.0, 3)])
def test_leaf2d_parity(p, kappa, nrhs):
    import torch
    h = (0.3, 0.2)
    lows = [(0.1 * k, -0.05 * k) for k in range(6)]
    nbox = len(lows)
    n, m = H.hps_leaf2d_sizes(p)
    xg = [H.hps_leaf_nodes(p, (lo[0], lo[1], 0.0), (h[0], h[1], 1.0)) for lo in lows]   # 3-D nodes, z = 0 plane
    xg = [x[:p * p, :2] for x in xg]
    b = np.stack([_b_field(x) for x in xg])
    f = np.stack([_loads(x, nrhs) for x in xg]) if nrhs else None
    T = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
    S = torch.empty(nbox, n, m, dtype=torch.float64, device="cuda")
    v = torch.empty(nbox, nrhs, n, dtype=torch.float64, device="cuda") if nrhs else None
    hf = torch.empty(nbox, nrhs, m, dtype=torch.float64, device="cuda") if nrhs else None
    st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
    H.hps_leaf2d_solve(p, h, kappa, nbox, _dev(b), nrhs, _dev(f) if nrhs else None, T, S, v, hf, st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    for bx in range(nbox):
        xo = oracle.node_coords_2d(p, lows[bx], h)
        bo = _b_field(xo)
        To, So, info = oracle.leaf_dtn_2d(p, h, kappa, bo)
        assert info == 0
        Tg = T[bx].cpu().numpy()
        assert np.linalg.norm(Tg - To) < 1e-11 * np.linalg.norm(To)
        assert np.linalg.norm(S[bx].cpu().numpy() - So) < 1e-11 * np.linalg.norm(So)
        if nrhs:
            vo, ho, _ = oracle.leaf_particular_2d(p, h, kappa, bo, _loads(xo, nrhs))
            assert np.linalg.norm(v[bx].cpu().numpy() - vo) < 1e-11 * np.linalg.norm(vo)
            assert np.linalg.norm(hf[bx].cpu().numpy() - ho) < 1e-11 * np.linalg.norm(ho)


def test_leaf2d_two_level_solve():
    """Leaf maps, particular solutions and reconstruction on the device;
    the interface system assembled and solved on the host; equals the
    oracle's two-level solve (and so the dense collocation solve)."""
    import torch
    p, kappa = 9, 6.0
    grid = g2.InterfaceGrid2D(p, (3, 2), lo=(0.1, -0.3), L=(1.2, 0.8))
    nbox = grid.nbox
    n, m = H.hps_leaf2d_sizes(p)
    rng = np.random.default_rng(9)
    xo = [oracle.node_coords_2d(p, grid.box_lo(bx), grid.h) for bx in range(nbox)]
    bo = [_b_field(x) for x in xo]
    fo = [_loads(x, 1)[0] for x in xo]
    g_dir = rng.standard_normal(grid.n_dir)
    ref = g2.hps_solve_2d(grid, kappa, bo, fo, g_dir)
    xg = [H.hps_leaf_nodes(p, (*grid.box_lo(bx), 0.0), (*grid.h, 1.0))[:p * p, :2] for bx in range(nbox)]
    T = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
    S = torch.empty(nbox, n, m, dtype=torch.float64, device="cuda")
    v = torch.empty(nbox, 1, n, dtype=torch.float64, device="cuda")
    hf = torch.empty(nbox, 1, m, dtype=torch.float64, device="cuda")
    H.hps_leaf2d_solve(p, grid.h, kappa, nbox, _dev(np.stack([_b_field(x) for x in xg])), 1,
                       _dev(np.stack([_loads(x, 1) for x in xg])), T, S, v, hf)
    torch.cuda.synchronize()
    Tn, hn = T.cpu().numpy(), hf.cpu().numpy()[:, 0, :]
    rows, cols, vals = [], [], []
    rhs = np.zeros(grid.n_iface)
    maps = [grid.local_to_global(bx) for bx in range(nbox)]
    for bx, (isi, gid) in enumerate(maps):
        ri, rd = np.nonzero(isi)[0], np.nonzero(~isi)[0]
        rr, cc = np.meshgrid(gid[ri], gid[ri], indexing="ij")
        rows.append(rr.reshape(-1)); cols.append(cc.reshape(-1)); vals.append(Tn[bx][np.ix_(ri, ri)].reshape(-1))
        np.add.at(rhs, gid[ri], -hn[bx, ri] - Tn[bx][np.ix_(ri, rd)] @ g_dir[gid[rd]])
    Tg = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(grid.n_iface, grid.n_iface)).tocsc()
    u_if = spla.splu(Tg).solve(rhs)
    ub = np.empty((nbox, 1, m))
    for bx, (isi, gid) in enumerate(maps):
        ub[bx, 0, isi] = u_if[gid[isi]]
        ub[bx, 0, ~isi] = g_dir[gid[~isi]]
    ui = torch.empty(nbox, 1, n, dtype=torch.float64, device="cuda")
    H.hps_leaf2d_reconstruct(p, nbox, 1, S, v, _dev(ub), ui)
    torch.cuda.synchronize()
    scale = np.abs(ref["u_int"]).max()
    assert np.abs(u_if - ref["u_iface"]).max() < 1e-11 * scale
    assert np.abs(ui.cpu().numpy()[:, 0, :] - ref["u_int"]).max() < 1e-11 * scale


def test_leaf2d_argument_errors():
    import torch
    b = torch.ones(2, 25, dtype=torch.float64, device="cuda")
    T = torch.empty(2, 12, 12, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HpsError):
        H.hps_leaf2d_solve(2, (0.5, 0.5), 1.0, 2, b, 0, None, T)
    with pytest.raises(H.HpsError):
        H.hps_leaf2d_solve(5, (0.0, 0.5), 1.0, 2, b, 0, None, T)
    with pytest.raises(H.HpsError):
        H.hps_leaf2d_solve(5, (0.5, 0.5), 1.0, 2, b, 1, None, T)   # loads without f, v, h
    with pytest.raises(H.HpsError):
        H.hps_leaf2d_reconstruct(5, 2, 1, None, None, T, T)


@pytest.mark.parametrize("iprec", [H.HPS_FP64, H.HPS_FP32_IR], ids=["fp64", "fp32ir"])
@pytest.mark.parametrize("nb", [(3, 2), (4, 4), (1, 3)])
def test_leaf2d_all_gpu_two_level_solve(ctx, nb, iprec):
    """The whole 2-D Dirichlet problem on the device: leaf maps, the interface
    factorisation and solve (nested dissection over the box grid), the
    reconstruction; equals the oracle's two-level solve."""
    import torch
    p, kappa = 8, 5.0
    grid = g2.InterfaceGrid2D(p, nb, lo=(0.1, -0.3), L=(1.2, 0.8))
    nbox = grid.nbox
    n, m = H.hps_leaf2d_sizes(p)
    rng = np.random.default_rng(12)
    xo = [oracle.node_coords_2d(p, grid.box_lo(bx), grid.h) for bx in range(nbox)]
    g_dir = rng.standard_normal(grid.n_dir)
    ref = g2.hps_solve_2d(grid, kappa, [_b_field(x) for x in xo], [_loads(x, 1)[0] for x in xo], g_dir)
    xg = [H.hps_leaf_nodes(p, (*grid.box_lo(bx), 0.0), (*grid.h, 1.0))[:p * p, :2] for bx in range(nbox)]
    T = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
    S = torch.empty(nbox, n, m, dtype=torch.float64, device="cuda")
    v = torch.empty(nbox, 1, n, dtype=torch.float64, device="cuda")
    hf = torch.empty(nbox, 1, m, dtype=torch.float64, device="cuda")
    H.hps_leaf2d_solve(p, grid.h, kappa, nbox, _dev(np.stack([_b_field(x) for x in xg])), 1,
                       _dev(np.stack([_loads(x, 1) for x in xg])), T, S, v, hf)
    g = np.zeros((nbox, 1, m))
    for bx in range(nbox):
        isi, gid = grid.local_to_global(bx)
        g[bx, 0, ~isi] = g_dir[gid[~isi]]
    ub = torch.empty(nbox, 1, m, dtype=torch.float64, device="cuda")
    ui = torch.empty(nbox, 1, n, dtype=torch.float64, device="cuda")
    F = H.hps_interface2d_factor(ctx, p, nb, T, 1, iprec)
    try:
        H.hps_interface_solve(F, 1, hf, _dev(g), ub)
        H.hps_leaf2d_reconstruct(p, nbox, 1, S, v, ub, ui)
        torch.cuda.synchronize()
    finally:
        H.hps_interface_destroy(F)
    scale = np.abs(ref["u_int"]).max()
    ubn = ub.cpu().numpy()[:, 0, :]
    for bx in range(nbox):
        isi, gid = grid.local_to_global(bx)
        assert np.abs(ubn[bx, isi] - ref["u_iface"][gid[isi]]).max() < 1e-11 * scale
    assert np.abs(ui.cpu().numpy()[:, 0, :] - ref["u_int"]).max() < 1e-11 * scale

