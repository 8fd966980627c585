"""The two-level solve on a grid of mixed orders (adaptive p) with the GPU's
leaves: one hps_leaf_groups call builds T, S, v and h for both orders, the
library's host routines assemble the interface system with the face
interpolation, a host sparse LU solves it (the paper's arrangement, MUMPS
there), and hps_leaf_reconstruct gives the interiors.  Against the oracle's
mixed-order solve (oracle/adaptive.py) and the exact plane wave."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
import paper_2503_04033_gb300 as H
from oracle import adaptive as ad
from oracle.global_solve import interior_grid_indices

pytestmark = pytest.mark.gpu

K = 8.0
D = np.array([1.0, 2.0, -0.5]) / np.linalg.norm([1.0, 2.0, -0.5])


def _pw(x):
    return np.cos(K * (x @ D) + 0.3)


def _b(x):
    return 1.0 + 0.0 * x[:, 0]


def _f(x):
    return 0.0 * x[:, 0]


def _gpu_mixed(nb, pb, prec):
    import torch
    grid = ad.MixedGrid(pb, nb)                       # geometry only (box corners, h)
    h = grid.h
    nbox = len(pb)
    ctx = H.hps_create(0, 0)
    try:
        groups, idx = [], {}
        for p in sorted(set(pb)):
            boxes = [i for i in range(nbox) if pb[i] == p]
            idx[p] = boxes
            n, m = H.hps_leaf_sizes(p)
            b = np.stack([_b(H.hps_leaf_nodes(p, grid.box_lo(i), h)) for i in boxes])
            f = np.stack([_f(H.hps_leaf_nodes(p, grid.box_lo(i), h)) for i in boxes])[:, None, :]
            groups.append({"p": p, "h": h, "kappa": [K] * len(boxes),
                           "b": torch.from_numpy(b).cuda(), "f": torch.from_numpy(np.ascontiguousarray(f)).cuda(),
                           "T": torch.empty(len(boxes), m, m, dtype=torch.float64, device="cuda"),
                           "S": torch.empty(len(boxes), n, m, dtype=torch.float64, device="cuda"),
                           "v": torch.empty(len(boxes), 1, n, dtype=torch.float64, device="cuda"),
                           "hflux": torch.empty(len(boxes), 1, m, dtype=torch.float64, device="cuda"),
                           "box_status": torch.full((len(boxes),), -1, dtype=torch.int32, device="cuda")})
        H.hps_leaf_groups(ctx, groups, prec)
        torch.cuda.synchronize()
        T_box, h_box = [None] * nbox, [None] * nbox
        for g in groups:
            assert (g["box_status"].cpu().numpy() == 0).all()
            for j, i in enumerate(idx[g["p"]]):
                T_box[i] = g["T"][j].cpu().numpy()
                h_box[i] = g["hflux"][j, 0].cpu().numpy()
        ni, nd, _, _ = H.hps_mixed_layout(nb, pb)
        xyz = H.hps_mixed_face_coords(nb, pb, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
        g_dir = _pw(xyz[ni:])
        r, c, v, rd, cd, vd = H.hps_mixed_assemble(nb, pb, T_box)
        A = sp.coo_matrix((v, (r, c)), shape=(ni, ni)).tocsc()
        Ad = sp.coo_matrix((vd, (rd, cd)), shape=(ni, nd)).tocsr()
        rhs = -H.hps_mixed_reduce(nb, pb, h_box)[:ni] - Ad @ g_dir
        u_if = spla.splu(A).solve(rhs)
        ub = H.hps_mixed_traces(nb, pb, np.concatenate([u_if, g_dir]))
        u_int = [None] * nbox
        for g in groups:
            p, boxes = g["p"], idx[g["p"]]
            n, m = H.hps_leaf_sizes(p)
            ubd = torch.from_numpy(np.stack([ub[i] for i in boxes])[:, None, :].copy()).cuda()
            ui = torch.empty(len(boxes), 1, n, dtype=torch.float64, device="cuda")
            H.hps_leaf_reconstruct(ctx, H.LeafKind(p, h, K), len(boxes), 1, g["b"], g["S"], g["v"], ubd, ui, prec)
            torch.cuda.synchronize()
            for j, i in enumerate(boxes):
                u_int[i] = ui[j, 0].cpu().numpy()
        return grid, u_if, u_int
    finally:
        H.hps_destroy(ctx)


@pytest.mark.parametrize("prec,tol", [(H.HPS_FP64, 1e-11), (H.HPS_FP32_IR, 1e-9)], ids=["fp64", "fp32ir"])
def test_mixed_orders_solve_with_gpu_leaves(prec, tol):
    """2 x 2 x 2 boxes, orders 6 and 8 in a checkerboard, kappa = 8: the
    interface solution and every interior equal the oracle's mixed-order
    solve, and the plane wave to the discretisation error."""
    nb = (2, 2, 2)
    pb = [6 if (i % 2 + (i // 2) % 2 + i // 4) % 2 == 0 else 8 for i in range(8)]
    grid, u_if, u_int = _gpu_mixed(nb, pb, prec)
    ro = ad.mixed_solve(ad.MixedGrid(pb, nb), K, _b, _f, _pw)
    scale = np.abs(ro["u_iface"]).max()
    assert np.abs(u_if - ro["u_iface"]).max() < tol * scale
    err = 0.0
    for box in range(8):
        assert np.abs(u_int[box] - ro["u_int"][box]).max() < tol * scale
        p = pb[box]
        x = oracle.node_coords(p, grid.box_lo(box), grid.h)
        err = max(err, float(np.abs(u_int[box] - _pw(x[interior_grid_indices(p)])).max()))
    assert err < 2e-2, err


def test_mixed_orders_three_orders_in_a_row():
    """4 x 1 x 1 boxes of orders 6, 8, 10, 8 (FP64): the oracle's solution."""
    nb = (4, 1, 1)
    pb = [6, 8, 10, 8]
    _, u_if, u_int = _gpu_mixed(nb, pb, H.HPS_FP64)
    ro = ad.mixed_solve(ad.MixedGrid(pb, nb), K, _b, _f, _pw)
    scale = np.abs(ro["u_iface"]).max()
    assert np.abs(u_if - ro["u_iface"]).max() < 1e-11 * scale
    for box in range(4):
        assert np.abs(u_int[box] - ro["u_int"][box]).max() < 1e-11 * scale
