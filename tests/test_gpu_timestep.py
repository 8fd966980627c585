"""Crank-Nicolson time stepping of the heat equation with the library
(Sec. 4.4): the DtN maps and the interior factorisations are built once;
each step is one operator application (hps_leaf_apply) for the right-hand
side, one particular solve and one reconstruction with the stored factors;
the interface system is a host sparse LU factored once (the stand-in for the
paper's MUMPS).  Against the oracle's own time loop and the exact solution.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2503_04033_gb300 as H
from oracle import global_solve as gs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = H.hps_create(0, 0)
    yield c
    H.hps_destroy(c)


def _u0(X):
    return np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1]) * np.sin(np.pi * X[:, 2])


def library_crank_nicolson(ctx, grid, kappa_d, dt, nsteps, prec, u0, iface="host"):
    """The time loop on the library's calls; returns (u_int [nbox, n], u_iface).
    iface: "host" solves the interface system with a host sparse LU of the
    assembled blocks, "gpu" with the library's interface factorisation."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import torch
    p, nbox = grid.p, grid.nbox
    n, m = H.hps_leaf_sizes(p)
    c = 2.0 / (dt * kappa_d)
    kind = H.LeafKind(p, grid.h, float(np.sqrt(c)))      # (c - Lap) = -Lap - kappa^2 b with b = -1
    b = torch.full((nbox, p ** 3), -1.0, dtype=torch.float64, device="cuda")
    T = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
    H.hps_leaf_build_dtn(ctx, kind, nbox, b, T, None, prec)
    torch.cuda.synchronize()
    rows, cols, vals, _, _, _, ni, _ = H.hps_assemble_interface_blocks(p, grid.nb, T.cpu().numpy())
    lu = spla.splu(sp.coo_matrix((vals, (rows, cols)), shape=(ni, ni)).tocsc())
    F = H.hps_leaf_factor(ctx, kind, nbox, b, 1, prec)
    FI = H.hps_interface_factor(ctx, p, grid.nb, T, 1) if iface == "gpu" else None
    try:
        ii, fi = gs.interior_grid_indices(p), gs.face_node_grid_indices(p)
        maps = [grid.local_to_global(bx) for bx in range(nbox)]
        u_np = np.stack([u0(H.hps_leaf_nodes(p, grid.box_lo(bx), grid.h)) for bx in range(nbox)])
        u = torch.from_numpy(u_np[:, None, :].copy()).cuda()
        Au = torch.empty_like(u)
        v = torch.empty(nbox, 1, n, dtype=torch.float64, device="cuda")
        hf = torch.empty(nbox, 1, m, dtype=torch.float64, device="cuda")
        ui = torch.empty(nbox, 1, n, dtype=torch.float64, device="cuda")
        st = torch.zeros(nbox, dtype=torch.int32, device="cuda")
        u_if = np.zeros(ni)
        for _ in range(nsteps):
            H.hps_leaf_apply(ctx, kind, nbox, 1, b, u, Au)
            f = (2.0 * c * u - Au).contiguous()
            H.hps_leaf_solve_factored(F, 1, f, v, hf, st)
            if FI is not None:
                ub_d = torch.empty(nbox, 1, m, dtype=torch.float64, device="cuda")
                H.hps_interface_solve(FI, 1, hf, None, ub_d)
                ub = ub_d.cpu().numpy()[:, 0, :]
                u_if = np.zeros(ni)
                for bx in range(nbox):
                    isi, gid = maps[bx]
                    u_if[gid[isi]] = ub[bx, isi]
            else:
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
            H.hps_leaf_reconstruct_factored(F, 1, v, torch.from_numpy(ub[:, None, :].copy()).cuda(), ui, st)
            torch.cuda.synchronize()
            assert (st.cpu().numpy() == 0).all()
            u_np = np.zeros((nbox, p ** 3))
            u_np[:, ii] = ui.cpu().numpy()[:, 0, :]
            u_np[:, fi] = ub
            u = torch.from_numpy(u_np[:, None, :].copy()).cuda()
        return ui.cpu().numpy()[:, 0, :], u_if
    finally:
        H.hps_leaf_factors_destroy(F)
        if FI is not None:
            H.hps_interface_destroy(FI)


def test_apply_matches_oracle(ctx):
    """hps_leaf_apply against the oracle's interior rows on random fields."""
    import torch
    p, h, kappa, nbox, nf = 9, np.array([0.2, 0.25, 0.15]), 7.0, 3, 2
    rng = np.random.default_rng(4)
    b = rng.uniform(0.5, 1.5, (nbox, p ** 3))
    u = rng.standard_normal((nbox, nf, p ** 3))
    out = torch.empty(nbox, nf, p ** 3, dtype=torch.float64, device="cuda")
    H.hps_leaf_apply(ctx, H.LeafKind(p, h, kappa), nbox, nf, torch.from_numpy(b).cuda(),
                     torch.from_numpy(u).cuda(), out)
    got = out.cpu().numpy()
    for bx in range(nbox):
        for c in range(nf):
            ref = oracle.apply_interior(p, h, kappa, b[bx], u[bx, c])
            assert np.abs(got[bx, c] - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("iface", ["host", "gpu"])
@pytest.mark.parametrize("prec,tol", [(H.HPS_FP64, 1e-11), (H.HPS_FP32_IR, 1e-9)], ids=["fp64", "fp32ir"])
def test_crank_nicolson_heat_matches_oracle_and_exact(ctx, prec, tol, iface):
    grid = gs.InterfaceGrid(10, (2, 2, 2))
    kd, dt, nsteps = 0.05, 0.05, 10
    ui, u_if = library_crank_nicolson(ctx, grid, kd, dt, nsteps, prec, _u0, iface)
    ref = gs.crank_nicolson_heat(grid, kd, dt, nsteps, _u0)
    scale = np.abs(ref["u_int"]).max()
    assert np.abs(ui - ref["u_int"]).max() < tol * scale
    assert np.abs(u_if - ref["u_iface"]).max() < tol * scale
    exact = np.exp(-3 * np.pi ** 2 * kd * dt * nsteps) * _u0(gs.interior_coords(grid).reshape(-1, 3))
    assert np.abs(ui.reshape(-1) - exact).max() < 2e-4
