"""Stored factorisations (hps_leaf_factor): A_ii of each box factored once,
then several load batches solved with the same factors (the build stage
applied once, as for the paper's time stepping, Sec. 4.4).  Every solve is
checked against the FP64 oracle's particular solutions and reconstructions.
"""
from __future__ import annotations

import numpy as np
import pytest

import hps_inputs as hi
import oracle
import paper_2503_04033_gb300 as H
from tests._cases import box_b, max_rel, rel_fro

pytestmark = pytest.mark.gpu

PRECS = [
    pytest.param(H.HPS_FP64, 1, 1e-11, id="fp64"),
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


@pytest.mark.parametrize("prec,fp16,tol", PRECS)
@pytest.mark.parametrize("p", [9, 12])
def test_factor_once_solve_many(ctx, prec, fp16, tol, p):
    """One factorisation, three load batches of different widths (up to
    nrhs_max), then a reconstruction: all within tol of the oracle."""
    import torch
    H.hps_set_option(ctx, H.HPS_OPT_FP16_OPERANDS, fp16)
    h, kappa, nbox = np.array([0.125, 0.15, 0.1]), 20.0, 3
    rng = np.random.default_rng(p)
    lows = rng.integers(0, 4, size=(nbox, 3)) * h
    field = hi.fourier_b_field().b
    n, m = H.hps_leaf_sizes(p)
    kind = H.LeafKind(p, h, kappa)
    fst = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
    F = H.hps_leaf_factor(ctx, kind, nbox, _dev(box_b(H.hps_leaf_nodes, p, lows, h, field)), 6, prec, fst)
    try:
        torch.cuda.synchronize()
        assert (fst.cpu().numpy() == 0).all()
        bvals = [field(oracle.node_coords(p, lows[bx], h)) for bx in range(nbox)]
        for nrhs, seed in ((4, 77), (2, 78), (6, 79)):
            loads = hi.fourier_b_per_box(nrhs, seed)
            fg = np.stack([hi.load_values(loads, H.hps_leaf_nodes(p, lo, h)) for lo in lows])
            v = torch.empty(nbox, nrhs, n, dtype=torch.float64, device="cuda")
            hf = torch.empty(nbox, nrhs, m, dtype=torch.float64, device="cuda")
            st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
            H.hps_leaf_solve_factored(F, nrhs, _dev(fg), v, hf, st)
            torch.cuda.synchronize()
            assert (st.cpu().numpy() == 0).all()
            for bx in range(nbox):
                xyz = oracle.node_coords(p, lows[bx], h)
                vo, ho, info = oracle.leaf_particular(p, h, kappa, bvals[bx], hi.load_values(loads, xyz))
                assert info == 0
                assert rel_fro(v[bx:bx + 1].cpu().numpy(), vo[None]).max() < tol
                assert max_rel(v[bx:bx + 1].cpu().numpy(), vo[None]) < tol
                assert rel_fro(hf[bx:bx + 1].cpu().numpy(), ho[None]).max() < tol
                assert max_rel(hf[bx:bx + 1].cpu().numpy(), ho[None]) < tol
        nr = 2
        ub_np = hi.random_boundary_data(nbox, nr, m)
        v_np = np.random.default_rng(5).standard_normal((nbox, nr, n))
        ui = torch.empty(nbox, nr, n, dtype=torch.float64, device="cuda")
        st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
        H.hps_leaf_reconstruct_factored(F, nr, _dev(v_np), _dev(ub_np), ui, st)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        for bx in range(nbox):
            uo, info = oracle.leaf_reconstruct(p, h, kappa, bvals[bx], v_np[bx], ub_np[bx])
            assert info == 0
            assert rel_fro(ui[bx:bx + 1].cpu().numpy(), uo[None]).max() < tol
            assert max_rel(ui[bx:bx + 1].cpu().numpy(), uo[None]) < tol
    finally:
        H.hps_leaf_factors_destroy(F)
        H.hps_set_option(ctx, H.HPS_OPT_FP16_OPERANDS, 1)


def test_factored_matches_one_shot_particular(ctx):
    """The stored-factor solve and hps_leaf_particular run the same kernels on
    the same factors: results within FP64 refinement noise of each other."""
    import torch
    p, h, kappa, nbox, nrhs = 12, np.array([0.125] * 3), 30.0, 4, 3
    lows = np.random.default_rng(2).integers(0, 4, size=(nbox, 3)) * h
    b = _dev(box_b(H.hps_leaf_nodes, p, lows, h, hi.fourier_b_field().b))
    loads = hi.fourier_b_per_box(nrhs, 11)
    f = _dev(np.stack([hi.load_values(loads, H.hps_leaf_nodes(p, lo, h)) for lo in lows]))
    n, m = H.hps_leaf_sizes(p)
    kind = H.LeafKind(p, h, kappa)
    v1 = torch.empty(nbox, nrhs, n, dtype=torch.float64, device="cuda")
    h1 = torch.empty(nbox, nrhs, m, dtype=torch.float64, device="cuda")
    H.hps_leaf_particular(ctx, kind, nbox, nrhs, b, f, v1, h1, H.HPS_FP32_IR)
    F = H.hps_leaf_factor(ctx, kind, nbox, b, nrhs, H.HPS_FP32_IR)
    try:
        v2, h2 = torch.empty_like(v1), torch.empty_like(h1)
        H.hps_leaf_solve_factored(F, nrhs, f, v2, h2)
        torch.cuda.synchronize()
        assert rel_fro(v1.cpu().numpy(), v2.cpu().numpy()).max() < 1e-11
        assert max_rel(v1.cpu().numpy(), v2.cpu().numpy()) < 1e-11
        assert rel_fro(h1.cpu().numpy(), h2.cpu().numpy()).max() < 1e-11
        assert max_rel(h1.cpu().numpy(), h2.cpu().numpy()) < 1e-11
    finally:
        H.hps_leaf_factors_destroy(F)


def test_factored_singular_box_and_arguments(ctx):
    """A box whose A_ii is exactly singular (host-side test hook) is flagged
    at factorisation and keeps its status in every later solve; the others
    solve normally.  nrhs beyond nrhs_max is an argument error."""
    import torch
    p, h, kappa, nbox = 8, np.array([0.125] * 3), 10.0, 3
    lows = np.zeros((nbox, 3))
    b = _dev(box_b(H.hps_leaf_nodes, p, lows, h, hi.gaussian_dip_b))
    kind = H.LeafKind(p, h, kappa)
    n, m = H.hps_leaf_sizes(p)
    fst = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
    H.hps_set_option(ctx, H.HPS_OPT_TEST_SINGULAR_BOX, 1)
    try:
        F = H.hps_leaf_factor(ctx, kind, nbox, b, 2, H.HPS_FP32_IR, fst)
    finally:
        H.hps_set_option(ctx, H.HPS_OPT_TEST_SINGULAR_BOX, -1)
    try:
        torch.cuda.synchronize()
        assert fst.cpu().numpy().tolist() == [0, H.HPS_ESINGULAR, 0]
        loads = hi.fourier_b_per_box(1, 3)
        f = _dev(np.stack([hi.load_values(loads, H.hps_leaf_nodes(p, lo, h)) for lo in lows]))
        v = torch.empty(nbox, 1, n, dtype=torch.float64, device="cuda")
        hf = torch.empty(nbox, 1, m, dtype=torch.float64, device="cuda")
        st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
        H.hps_leaf_solve_factored(F, 1, f, v, hf, st)
        torch.cuda.synchronize()
        s = st.cpu().numpy()
        assert s[1] == H.HPS_ESINGULAR and s[0] == 0 and s[2] == 0
        with pytest.raises(H.HpsError):
            H.hps_leaf_solve_factored(F, 3, f, v, hf, st)
    finally:
        H.hps_leaf_factors_destroy(F)


def test_factored_solves_replay_as_graphs(ctx):
    """With HPS_OPT_GRAPHS a stored-factor solve is captured once and replayed:
    new load values in the same arrays give the results of an uncaptured
    solve, bit for bit."""
    import torch
    p, h, kappa, nbox, nrhs = 9, np.array([0.125] * 3), 15.0, 3, 2
    lows = np.random.default_rng(6).integers(0, 4, size=(nbox, 3)) * h
    b = _dev(box_b(H.hps_leaf_nodes, p, lows, h, hi.fourier_b_field().b))
    kind = H.LeafKind(p, h, kappa)
    n, m = H.hps_leaf_sizes(p)
    F = H.hps_leaf_factor(ctx, kind, nbox, b, nrhs, H.HPS_FP32_IR)
    f = torch.empty(nbox, nrhs, p ** 3, dtype=torch.float64, device="cuda")
    v = torch.empty(nbox, nrhs, n, dtype=torch.float64, device="cuda")
    hf = torch.empty(nbox, nrhs, m, dtype=torch.float64, device="cuda")
    try:
        results = {}
        for graphs in (0, 1):
            H.hps_set_option(ctx, H.HPS_OPT_GRAPHS, graphs)
            out = []
            for seed in (40, 41, 42):    # same arrays, new values: the graph is replayed
                loads = hi.fourier_b_per_box(nrhs, seed)
                f.copy_(_dev(np.stack([hi.load_values(loads, H.hps_leaf_nodes(p, lo, h)) for lo in lows])))
                H.hps_leaf_solve_factored(F, nrhs, f, v, hf)
                torch.cuda.synchronize()
                out.append((v.cpu().numpy().copy(), hf.cpu().numpy().copy()))
            results[graphs] = out
        for (v0, h0), (v1, h1) in zip(results[0], results[1]):
            assert np.array_equal(v0, v1) and np.array_equal(h0, h1)
    finally:
        H.hps_set_option(ctx, H.HPS_OPT_GRAPHS, 0)
        H.hps_leaf_factors_destroy(F)

