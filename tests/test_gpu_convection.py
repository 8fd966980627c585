"""The first-order term div(beta u) (the convection of Sec. 4.4's example):
DtN maps, particular solutions, reconstructions, stored factorisations and
the operator application with a velocity-like field beta, against the FP64
oracle's kept-node collocation with the same term; and the library's
Crank-Nicolson convection-diffusion loop against the oracle's.
"""
from __future__ import annotations

import numpy as np
import pytest

import hps_inputs as hi
import oracle
import paper_2503_04033_gb300 as H
from oracle import global_solve as gs
from tests._cases import box_b, max_rel, rel_fro

pytestmark = pytest.mark.gpu

PRECS = [
    pytest.param(H.HPS_FP64, 0, 1e-11, id="fp64"),
    pytest.param(H.HPS_FP32_IR, 1, 1e-10, id="fp32ir-fp16"),
    pytest.param(H.HPS_FP32_IR, 0, 1e-10, id="fp32ir-tf32"),
    pytest.param(H.HPS_BF16_IR, 1, 1e-10, id="bf16ir"),
]


@pytest.fixture(scope="module")
def ctx():
    c = H.hps_create(0, 0)
    yield c
    H.hps_destroy(c)


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def velocity(X):
    """The circular field of Sec. 4.4's example, [N, 3]."""
    return np.stack([-np.cos(X[:, 0]) * np.sin(X[:, 1]) * X[:, 2],
                     np.sin(X[:, 0]) * np.cos(X[:, 1]) * X[:, 2], 0.0 * X[:, 0]], axis=1)


def beta_boxes(p, lows, h, scale):
    """[nbox, 3, p^3]: scale * velocity + a constant drift at every node."""
    out = []
    for lo in lows:
        X = H.hps_leaf_nodes(p, lo, h)
        out.append((scale * velocity(X) + np.array([0.7, -0.4, 0.3]) * scale).T)
    return np.stack(out)


@pytest.mark.parametrize("prec,fp16,tol", PRECS)
@pytest.mark.parametrize("p", [8, 9])
def test_dtn_particular_reconstruct_with_first_order_term(ctx, prec, fp16, tol, p):
    import torch
    H.hps_set_option(ctx, H.HPS_OPT_FP16_OPERANDS, fp16)
    H.hps_set_option(ctx, H.HPS_OPT_TENSOR_CORES, 1)
    h, kappa, nbox = np.array([0.2, 0.25, 0.15]), 9.0, 3
    lows = np.random.default_rng(p).integers(0, 4, size=(nbox, 3)) * h
    field = hi.fourier_b_field().b
    bt = beta_boxes(p, lows, h, 6.0)
    kind = H.LeafKind(p, h, kappa, _dev(bt))
    n, m = H.hps_leaf_sizes(p)
    b = _dev(box_b(H.hps_leaf_nodes, p, lows, h, field))
    T = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
    S = torch.empty(nbox, n, m, dtype=torch.float64, device="cuda")
    st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
    H.hps_leaf_build_dtn(ctx, kind, nbox, b, T, S, prec, st)
    loads = hi.fourier_b_per_box(2, 31)
    fg = np.stack([hi.load_values(loads, H.hps_leaf_nodes(p, lo, h)) for lo in lows])
    v = torch.empty(nbox, 2, n, dtype=torch.float64, device="cuda")
    hf = torch.empty(nbox, 2, m, dtype=torch.float64, device="cuda")
    st2 = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
    H.hps_leaf_particular(ctx, kind, nbox, 2, b, _dev(fg), v, hf, prec, st2)
    ub = hi.random_boundary_data(nbox, 2, m)
    v0 = np.random.default_rng(9).standard_normal((nbox, 2, n))
    ui = torch.empty(nbox, 2, n, dtype=torch.float64, device="cuda")
    st3 = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
    H.hps_leaf_reconstruct(ctx, kind, nbox, 2, b, None, _dev(v0), _dev(ub), ui, prec, st3)
    torch.cuda.synchronize()
    H.hps_set_option(ctx, H.HPS_OPT_FP16_OPERANDS, 1)
    for s_ in (st, st2, st3):
        assert (s_.cpu().numpy() == 0).all()
    for bx in range(nbox):
        xyz = oracle.node_coords(p, lows[bx], h)
        To, So, info = oracle.leaf_dtn(p, h, kappa, field(xyz), beta=bt[bx])
        assert info == 0
        assert rel_fro(T[bx:bx + 1].cpu().numpy(), To[None]).max() < tol
        assert max_rel(T[bx:bx + 1].cpu().numpy(), To[None]) < tol
        assert rel_fro(S[bx:bx + 1].cpu().numpy(), So[None]).max() < tol
        assert max_rel(S[bx:bx + 1].cpu().numpy(), So[None]) < tol
        vo, ho, _ = oracle.leaf_particular(p, h, kappa, field(xyz), hi.load_values(loads, xyz), beta=bt[bx])
        assert rel_fro(v[bx:bx + 1].cpu().numpy(), vo[None]).max() < tol
        assert max_rel(v[bx:bx + 1].cpu().numpy(), vo[None]) < tol
        assert rel_fro(hf[bx:bx + 1].cpu().numpy(), ho[None]).max() < tol
        assert max_rel(hf[bx:bx + 1].cpu().numpy(), ho[None]) < tol
        uo, _ = oracle.leaf_reconstruct(p, h, kappa, field(xyz), v0[bx], ub[bx], beta=bt[bx])
        assert rel_fro(ui[bx:bx + 1].cpu().numpy(), uo[None]).max() < tol
        assert max_rel(ui[bx:bx + 1].cpu().numpy(), uo[None]) < tol


@pytest.mark.parametrize("prec,tol", [(H.HPS_FP64, 1e-11), (H.HPS_FP32_IR, 1e-10)], ids=["fp64", "fp32ir"])
def test_factored_and_apply_with_first_order_term(ctx, prec, tol):
    import torch
    p, h, kappa, nbox = 9, np.array([0.125] * 3), 12.0, 2
    lows = np.random.default_rng(3).integers(0, 4, size=(nbox, 3)) * h
    field = hi.gaussian_dip_b
    bt = beta_boxes(p, lows, h, 4.0)
    kind = H.LeafKind(p, h, kappa, _dev(bt))
    n, m = H.hps_leaf_sizes(p)
    bv = box_b(H.hps_leaf_nodes, p, lows, h, field)
    b = _dev(bv)
    F = H.hps_leaf_factor(ctx, kind, nbox, b, 3, prec)
    try:
        loads = hi.fourier_b_per_box(3, 5)
        fg = np.stack([hi.load_values(loads, H.hps_leaf_nodes(p, lo, h)) for lo in lows])
        v = torch.empty(nbox, 3, n, dtype=torch.float64, device="cuda")
        hf = torch.empty(nbox, 3, m, dtype=torch.float64, device="cuda")
        st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
        H.hps_leaf_solve_factored(F, 3, _dev(fg), v, hf, st)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        for bx in range(nbox):
            vo, ho, _ = oracle.leaf_particular(p, h, kappa, bv[bx], fg[bx], beta=bt[bx])
            assert rel_fro(v[bx:bx + 1].cpu().numpy(), vo[None]).max() < tol
            assert max_rel(v[bx:bx + 1].cpu().numpy(), vo[None]) < tol
            assert rel_fro(hf[bx:bx + 1].cpu().numpy(), ho[None]).max() < tol
            assert max_rel(hf[bx:bx + 1].cpu().numpy(), ho[None]) < tol
    finally:
        H.hps_leaf_factors_destroy(F)
    u = np.random.default_rng(8).standard_normal((nbox, 2, p ** 3))
    out = torch.empty(nbox, 2, p ** 3, dtype=torch.float64, device="cuda")
    H.hps_leaf_apply(ctx, kind, nbox, 2, b, _dev(u), out)
    got = out.cpu().numpy()
    for bx in range(nbox):
        for c in range(2):
            ref = oracle.apply_interior(p, h, kappa, bv[bx], u[bx, c], bt[bx])
            assert np.abs(got[bx, c] - ref).max() < 1e-12 * np.abs(ref).max()


def test_convection_diffusion_crank_nicolson_matches_oracle(ctx):
    """The paper's convection-diffusion example (circular velocity field,
    kappa_d small against the convection) on the unit cube, 2 x 2 x 2 boxes:
    the library's loop (stored factors, hps_leaf_apply, host interface LU)
    against the oracle's, 6 steps."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import torch
    grid = gs.InterfaceGrid(8, (2, 2, 2))
    kd, dt, nsteps = 0.02, 0.05, 6
    u0 = lambda X: np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])
    p, nbox = grid.p, grid.nbox
    n, m = H.hps_leaf_sizes(p)
    c = 2.0 / (dt * kd)
    xyz = [H.hps_leaf_nodes(p, grid.box_lo(bx), grid.h) for bx in range(nbox)]
    bt = np.stack([velocity(X).T / kd for X in xyz])
    kind = H.LeafKind(p, grid.h, float(np.sqrt(c)), _dev(bt))
    b = torch.full((nbox, p ** 3), -1.0, dtype=torch.float64, device="cuda")
    T = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
    H.hps_leaf_build_dtn(ctx, kind, nbox, b, T, None, H.HPS_FP32_IR)
    torch.cuda.synchronize()
    rows, cols, vals, _, _, _, ni, _ = H.hps_assemble_interface_blocks(p, grid.nb, T.cpu().numpy())
    lu = spla.splu(sp.coo_matrix((vals, (rows, cols)), shape=(ni, ni)).tocsc())
    F = H.hps_leaf_factor(ctx, kind, nbox, b, 1, H.HPS_FP32_IR)
    try:
        ii, fi = gs.interior_grid_indices(p), gs.face_node_grid_indices(p)
        maps = [grid.local_to_global(bx) for bx in range(nbox)]
        u = _dev(np.stack([u0(X) for X in xyz])[:, None, :])
        Au = torch.empty_like(u)
        v = torch.empty(nbox, 1, n, dtype=torch.float64, device="cuda")
        hf = torch.empty(nbox, 1, m, dtype=torch.float64, device="cuda")
        ui = torch.empty(nbox, 1, n, dtype=torch.float64, device="cuda")
        u_if = np.zeros(ni)
        for _ in range(nsteps):
            H.hps_leaf_apply(ctx, kind, nbox, 1, b, u, Au)
            H.hps_leaf_solve_factored(F, 1, (2.0 * c * u - Au).contiguous(), v, hf)
            hf_np = hf.cpu().numpy()[:, 0, :]
            rhs = np.zeros(ni)
            for bx in range(nbox):
                isi, gid = maps[bx]
                np.add.at(rhs, gid[isi], -hf_np[bx, isi])
            u_if = lu.solve(rhs)
            ub = np.zeros((nbox, m))
            for bx in range(nbox):
                isi, gid = maps[bx]
                ub[bx, isi] = u_if[gid[isi]]
            H.hps_leaf_reconstruct_factored(F, 1, v, _dev(ub[:, None, :]), ui)
            un = np.zeros((nbox, p ** 3))
            un[:, ii] = ui.cpu().numpy()[:, 0, :]
            un[:, fi] = ub
            u = _dev(un[:, None, :])
        ref = gs.crank_nicolson_heat(grid, kd, dt, nsteps, u0, velocity)
        scale = np.abs(ref["u_int"]).max()
        assert np.abs(ui.cpu().numpy()[:, 0, :] - ref["u_int"]).max() < 1e-9 * scale
        assert np.abs(u_if - ref["u_iface"]).max() < 1e-9 * scale
    finally:
        H.hps_leaf_factors_destroy(F)
