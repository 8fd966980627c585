"""Parity of the CUDA leaf reduction against the FP64 oracle, through the C ABI.

Tolerances (relative Frobenius error per box, against the oracle):
  FP64 path            1e-11 on T, S, v, h, u_i
  FP32 + refinement    1e-10 on T, S, v, h, u_i
Both bounds sit well above the forward error of either side (cond(A_ii) is
~1e3-1e4 on these workloads, times FP64 rounding) and far below what an
indexing or sign mistake would give.
"""
from __future__ import annotations

import numpy as np
import pytest

import hps_inputs as hi
import oracle
import paper_2503_04033_gb300 as H
from tests._cases import box_b, config_grid, max_rel, rel_fro

pytestmark = pytest.mark.gpu

PRECS = [
    pytest.param(H.HPS_FP64, 0, 1e-11, id="fp64"),
    pytest.param(H.HPS_FP32_IR, 0, 1e-10, id="fp32ir-cudacore"),
    pytest.param(H.HPS_FP32_IR, 1, 1e-10, id="fp32ir-tcgen05"),
    pytest.param(H.HPS_BF16_IR, 1, 1e-10, id="bf16ir-tcgen05"),
    pytest.param(H.HPS_FP32_IR, 2, 1e-10, id="fp32ir-tcgen05-fp16"),
]


def set_tc(ctx, tc):
    """tc: 0 CUDA cores, 1 tcgen05 (the default operand format), 2 tcgen05
    with the scaled 2 x FP16 operands."""
    H.hps_set_option(ctx, H.HPS_OPT_TENSOR_CORES, 1 if tc else 0)
    H.hps_set_option(ctx, H.HPS_OPT_FP16_OPERANDS, 1 if tc == 2 else 0)


@pytest.fixture(scope="module")
def ctx():
    c = H.hps_create(0, 0)
    yield c
    H.hps_destroy(c)


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def gpu_dtn(ctx, p, h, kappa, b_np, prec, tc, want_S=True, block=0):
    import torch
    set_tc(ctx, tc)
    H.hps_set_option(ctx, H.HPS_OPT_BLOCK, block)
    n, m = H.hps_leaf_sizes(p)
    nbox = b_np.shape[0]
    b = _dev(b_np)
    T = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
    S = torch.empty(nbox, n, m, dtype=torch.float64, device="cuda") if want_S else None
    st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
    H.hps_leaf_build_dtn(ctx, H.LeafKind(p, h, kappa), nbox, b, T, S, prec, st)
    torch.cuda.synchronize()
    return T.cpu().numpy(), (S.cpu().numpy() if want_S else None), st.cpu().numpy()


def _lows(nbox, h, seed=0):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 4, size=(nbox, 3)) * np.asarray(h)


@pytest.mark.parametrize("prec,tc,tol", PRECS)
@pytest.mark.parametrize("p,nbox", [(3, 2), (5, 3), (8, 4), (9, 3), (10, 2)])
def test_dtn_parity_small(ctx, p, nbox, prec, tc, tol):
    h = np.array([0.125, 0.2, 0.15])
    kappa = 12.0
    lows = _lows(nbox, h, p)
    field = hi.fourier_b_field().b
    b_gpu = box_b(H.hps_leaf_nodes, p, lows, h, field)
    b_or = box_b(oracle.node_coords, p, lows, h, field)
    T, S, st = gpu_dtn(ctx, p, h, kappa, b_gpu, prec, tc)
    To, So, sto = oracle.batch_dtn(p, h, kappa, b_or, want_S=True)
    assert (sto == 0).all() and (st == 0).all(), st
    assert rel_fro(T, To).max() < tol, rel_fro(T, To)
    assert max_rel(T, To) < tol
    assert rel_fro(S, So).max() < tol, rel_fro(S, So)
    assert max_rel(S, So) < tol


@pytest.mark.parametrize("tc", [1, 2], ids=["tf32", "fp16"])
@pytest.mark.parametrize("p,nbox,block", [(8, 3, 0), (9, 3, 32), (12, 2, 64), (16, 2, 0)])
def test_tcgen05_epilogue_forms_agree(ctx, p, nbox, block, tc):
    """The TMA epilogue (aligned outputs; n = 343 at p = 9 leaves the
    right-hand-side block unaligned, so both forms run in one call) and the
    cp.async epilogue compute src - acc identically: bit-equal T and S in both
    forms, and they match the oracle."""
    h = np.array([0.125, 0.2, 0.15])
    kappa = 15.0
    lows = _lows(nbox, h, 7 + p)
    field = hi.fourier_b_field().b
    b_gpu = box_b(H.hps_leaf_nodes, p, lows, h, field)
    try:
        H.hps_set_option(ctx, H.HPS_OPT_TC_EPILOGUE, 1)
        T1, S1, st1 = gpu_dtn(ctx, p, h, kappa, b_gpu, H.HPS_FP32_IR, tc, block=block)
    finally:
        H.hps_set_option(ctx, H.HPS_OPT_TC_EPILOGUE, 0)
    T0, S0, st0 = gpu_dtn(ctx, p, h, kappa, b_gpu, H.HPS_FP32_IR, tc, block=block)
    assert (st0 == 0).all() and (st1 == 0).all(), (st0, st1)
    assert np.array_equal(T0, T1) and np.array_equal(S0, S1)
    if p <= 12:
        To, _, _ = oracle.batch_dtn(p, h, kappa, box_b(oracle.node_coords, p, lows, h, field), want_S=False)
        assert rel_fro(T0, To).max() < 1e-10
        assert max_rel(T0, To) < 1e-10


@pytest.mark.parametrize("tc", [1, 2], ids=["tf32", "fp16"])
@pytest.mark.parametrize("p,nbox,block", [(8, 3, 32), (9, 2, 32), (12, 2, 64), (13, 2, 64), (16, 2, 0)])
def test_tcgen05_lu_units_match_single_steps(ctx, p, nbox, block, tc):
    """Joining LU steps into units of up to 4 (the default), 2 and 8
    (look-ahead factorisation, unit-deep products) against one step at a
    time: all within 1e-10 of the oracle and of each other.  The block sizes
    give 7, 11, 16, 21 and 22 steps, so the units end ragged (4 + 2 + 1, 8 +
    2 + 1, a single step after whole units, a last step narrower than the
    block)."""
    h = np.array([0.125, 0.2, 0.15])
    kappa = 18.0
    lows = _lows(nbox, h, 11 + p)
    field = hi.fourier_b_field().b
    b_gpu = box_b(H.hps_leaf_nodes, p, lows, h, field)
    res = {}
    units = (1, 2, 8) if block in (32, 64) else (1, 2)   # 8 steps of 32 or 64 columns: K = 256 or 512
    try:
        for unit in units:
            H.hps_set_option(ctx, H.HPS_OPT_LU_UNIT, unit)
            res[unit] = gpu_dtn(ctx, p, h, kappa, b_gpu, H.HPS_FP32_IR, tc, block=block)
    finally:
        H.hps_set_option(ctx, H.HPS_OPT_LU_UNIT, 4)
    res[4] = gpu_dtn(ctx, p, h, kappa, b_gpu, H.HPS_FP32_IR, tc, block=block)
    T0, S0, st0 = res[4]
    for unit in units:
        T1, S1, st1 = res[unit]
        assert (st0 == 0).all() and (st1 == 0).all(), (unit, st0, st1)
        assert rel_fro(T0, T1).max() < 1e-10 and rel_fro(S0, S1).max() < 1e-10, unit
        assert max_rel(T0, T1) < 1e-10 and max_rel(S0, S1) < 1e-10, unit
    if p <= 13:
        To, So, _ = oracle.batch_dtn(p, h, kappa, box_b(oracle.node_coords, p, lows, h, field), want_S=True)
        assert rel_fro(T0, To).max() < 1e-10 and rel_fro(S0, So).max() < 1e-10
        assert max_rel(T0, To) < 1e-10 and max_rel(S0, So) < 1e-10


@pytest.mark.parametrize("tc", [1, 2], ids=["tf32", "fp16"])
@pytest.mark.parametrize("hs,kappa", [(1e-3, 1.2e3), (4.0, 0.3)], ids=["tiny", "huge"])
def test_tcgen05_extreme_box_sizes(ctx, tc, hs, kappa):
    """Boxes of side 1e-3 and 4 put the entries of A_ii near 1e11 and 0.1
    (D^2 scales as 1/h^2): far outside FP16's range before its power-of-two
    operand scaling, and the refinement's stopping rule sees the same
    relative sizes.  Both tensor-core formats match the oracle to 1e-10."""
    p, nbox = 9, 2
    h = np.array([hs, 1.25 * hs, 0.8 * hs])
    lows = _lows(nbox, h, 3)
    field = hi.gaussian_dip_b
    T, S, st = gpu_dtn(ctx, p, h, kappa, box_b(H.hps_leaf_nodes, p, lows, h, field), H.HPS_FP32_IR, tc)
    To, So, _ = oracle.batch_dtn(p, h, kappa, box_b(oracle.node_coords, p, lows, h, field), want_S=True)
    assert (st == 0).all(), st
    assert rel_fro(T, To).max() < 1e-10 and rel_fro(S, So).max() < 1e-10
    assert max_rel(T, To) < 1e-10 and max_rel(S, So) < 1e-10


@pytest.mark.parametrize("prec", [H.HPS_FP32_IR, H.HPS_BF16_IR], ids=["fp32ir", "bf16ir"])
@pytest.mark.parametrize("p,nbox", [(9, 3), (12, 2), (16, 2)])
def test_residual_precision_modes(ctx, prec, p, nbox):
    """Every residual precision mode of the refinement (0: all FP64; 1:
    double-float first residual, held for one FP64 correction; 2:
    double-float first, FP64 later; 3, the default: double-float first and
    later for well-conditioned boxes, FP64 for the others) gives T and S
    within 1e-10 of each other (and of the oracle at p <= 12).  In mode 1
    every box takes at least two corrections and at most one more than with
    FP64 residuals.  p = 9 has an odd line length (q = 7)."""
    h = np.array([0.125, 0.2, 0.15])
    kappa = 18.0
    lows = _lows(nbox, h, 5 + p)
    field = hi.fourier_b_field().b
    b_np = box_b(H.hps_leaf_nodes, p, lows, h, field)
    res = {}
    try:
        for df in (0, 1, 2, 3):
            H.hps_set_option(ctx, H.HPS_OPT_RESIDUAL_DF, df)
            T, S, st = gpu_dtn(ctx, p, h, kappa, b_np, prec, 1)
            assert (st == 0).all(), (df, st)
            its, _ = H.hps_last_refinement(ctx, nbox)
            res[df] = (T, S, its.copy())
    finally:
        H.hps_set_option(ctx, H.HPS_OPT_RESIDUAL_DF, 3)
    T0, S0, i0 = res[0]
    for df in (1, 2, 3):
        T1, S1, i1 = res[df]
        assert rel_fro(T0, T1).max() < 1e-10 and rel_fro(S0, S1).max() < 1e-10, df
        assert max_rel(T0, T1) < 1e-10 and max_rel(S0, S1) < 1e-10, df
    assert (res[1][2] >= 2).all() and (res[1][2] <= i0 + 1).all(), (i0, res[1][2])
    if p <= 12:
        To, So, _ = oracle.batch_dtn(p, h, kappa, box_b(oracle.node_coords, p, lows, h, field), want_S=True)
        for df in (0, 3):
            T1, S1, _ = res[df]
            assert rel_fro(T1, To).max() < 1e-10 and rel_fro(S1, So).max() < 1e-10, df
            assert max_rel(T1, To) < 1e-10 and max_rel(S1, So) < 1e-10, df


@pytest.mark.parametrize("prec,tc,tol", PRECS)
@pytest.mark.parametrize("block", [32, 64])
def test_dtn_parity_block_sizes(ctx, prec, tc, tol, block):
    """Several LU blocks with a ragged last block (n = 343 at p = 9)."""
    p, h, kappa = 9, np.array([0.25, 0.25, 0.25]), 7.0
    lows = _lows(2, h, 3)
    field = hi.gaussian_dip_b
    T, S, st = gpu_dtn(ctx, p, h, kappa, box_b(H.hps_leaf_nodes, p, lows, h, field), prec, tc, block=block)
    To, So, _ = oracle.batch_dtn(p, h, kappa, box_b(oracle.node_coords, p, lows, h, field), want_S=True)
    assert (st == 0).all()
    assert rel_fro(T, To).max() < tol and rel_fro(S, So).max() < tol
    assert max_rel(T, To) < tol and max_rel(S, So) < tol


@pytest.mark.parametrize("prec,tc,tol", PRECS)
@pytest.mark.parametrize("kappa", [0.0, 10.0])
def test_dtn_manufactured_grid(ctx, prec, tc, tol, kappa):
    p, h, _, lows, field = config_grid("manufactured")
    T, S, st = gpu_dtn(ctx, p, h, kappa, box_b(H.hps_leaf_nodes, p, lows, h, field), prec, tc)
    To, So, _ = oracle.batch_dtn(p, h, kappa, box_b(oracle.node_coords, p, lows, h, field), want_S=True)
    assert (st == 0).all()
    assert rel_fro(T, To).max() < tol and rel_fro(S, So).max() < tol
    assert max_rel(T, To) < tol and max_rel(S, So) < tol
    if kappa == 0.0:
        assert np.abs(T.sum(axis=2)).max() < 1e-9 * np.abs(T).max()      # T 1 = 0


@pytest.mark.parametrize("prec,tc,tol", [PRECS[0], PRECS[2]])
def test_dtn_dip_512_boxes_sampled(ctx, prec, tc, tol):
    """Full 8x8x8 grid at p = 12 on the GPU; sampled boxes against the oracle."""
    p, h, kappa, lows, field = config_grid("dip")
    T, S, st = gpu_dtn(ctx, p, h, kappa, box_b(H.hps_leaf_nodes, p, lows, h, field), prec, tc)
    assert (st == 0).all()
    for box in (0, 273, 511):
        To, So, info = oracle.leaf_dtn(p, h, kappa, field(oracle.node_coords(p, lows[box], h)))
        assert info == 0
        assert rel_fro(T[box:box + 1], To[None]).max() < tol
        assert max_rel(T[box:box + 1], To[None]) < tol
        assert rel_fro(S[box:box + 1], So[None]).max() < tol
        assert max_rel(S[box:box + 1], So[None]) < tol


@pytest.mark.parametrize("prec,tc", [(H.HPS_FP32_IR, 1), (H.HPS_BF16_IR, 1), (H.HPS_FP32_IR, 2)],
                         ids=["fp32ir", "bf16ir", "fp32ir-fp16"])
def test_dtn_fourier16_512_boxes_sampled(ctx, prec, tc):
    """The p = 16 mixed-precision workload at full size (512 boxes, kappa = 40),
    tensor-core LU (3 x TF32, 3 x BF16 or scaled 2 x FP16) + FP64 refinement; two boxes and the
    most-refined box against the oracle, and 32 evenly spaced boxes plus the
    8 most-refined ones against the plain FP64 GPU path."""
    import torch
    p, h, kappa, lows, field = config_grid("fourier16")
    b_gpu = box_b(H.hps_leaf_nodes, p, lows, h, field)
    T, _, st = gpu_dtn(ctx, p, h, kappa, b_gpu, prec, tc, want_S=False)
    assert (st == 0).all(), np.unique(st, return_counts=True)
    it, rel = H.hps_last_refinement(ctx, len(lows))
    assert (it >= 1).all() and (it <= 8).all(), (it.min(), it.max())
    hardest = np.argsort(-(it * 100.0 + rel / max(rel.max(), 1e-300)))[:8]
    for box in (5, 300, int(hardest[0])):
        To, _, info = oracle.leaf_dtn(p, h, kappa, field(oracle.node_coords(p, lows[box], h)), want_S=False)
        assert info == 0
        assert rel_fro(T[box:box + 1], To[None]).max() < 1e-10
        assert max_rel(T[box:box + 1], To[None]) < 1e-10
    sel = np.unique(np.concatenate([np.arange(0, 512, 16), hardest]))
    T64, _, st64 = gpu_dtn(ctx, p, h, kappa, b_gpu[sel], H.HPS_FP64, 0, want_S=False)
    assert (st64 == 0).all()
    assert rel_fro(T[sel], T64).max() < 1e-10
    assert max_rel(T[sel], T64) < 1e-10
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec,tc,tol", PRECS)
def test_particular_parity(ctx, prec, tc, tol):
    import torch
    set_tc(ctx, tc)
    p, h, kappa, nbox, nrhs = 9, np.array([0.125] * 3), 20.0, 3, 4
    lows = _lows(nbox, h, 9)
    field = hi.fourier_b_field().b
    loads = hi.fourier_b_per_box(nrhs, 77)
    fg = np.stack([hi.load_values(loads, H.hps_leaf_nodes(p, lo, h)) for lo in lows])
    n, m = H.hps_leaf_sizes(p)
    v = torch.empty(nbox, nrhs, n, dtype=torch.float64, device="cuda")
    hf = torch.empty(nbox, nrhs, m, dtype=torch.float64, device="cuda")
    st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
    H.hps_leaf_particular(ctx, H.LeafKind(p, h, kappa), nbox, nrhs, _dev(box_b(H.hps_leaf_nodes, p, lows, h, field)),
                          _dev(fg), v, hf, prec, st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    for bx in range(nbox):
        xyz = oracle.node_coords(p, lows[bx], h)
        vo, ho, info = oracle.leaf_particular(p, h, kappa, field(xyz), hi.load_values(loads, xyz))
        assert info == 0
        assert rel_fro(v[bx:bx + 1].cpu().numpy(), vo[None]).max() < tol
        assert max_rel(v[bx:bx + 1].cpu().numpy(), vo[None]) < tol
        assert rel_fro(hf[bx:bx + 1].cpu().numpy(), ho[None]).max() < tol
        assert max_rel(hf[bx:bx + 1].cpu().numpy(), ho[None]) < tol


@pytest.mark.parametrize("prec,tc,tol", PRECS)
@pytest.mark.parametrize("stored", [True, False])
def test_reconstruct_parity(ctx, prec, tc, tol, stored):
    import torch
    p, h, kappa, nbox, nrhs = 8, np.array([0.125] * 3), 15.0, 3, 2
    lows = _lows(nbox, h, 4)
    field = hi.gaussian_dip_b
    n, m = H.hps_leaf_sizes(p)
    b = _dev(box_b(H.hps_leaf_nodes, p, lows, h, field))
    ub_np = hi.random_boundary_data(nbox, nrhs, m)
    v_np = np.random.default_rng(5).standard_normal((nbox, nrhs, n))
    S = None
    if stored:
        _, S_np, st = gpu_dtn(ctx, p, h, kappa, box_b(H.hps_leaf_nodes, p, lows, h, field), prec, tc)
        S = _dev(S_np)
    set_tc(ctx, tc)
    ui = torch.empty(nbox, nrhs, n, dtype=torch.float64, device="cuda")
    st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
    H.hps_leaf_reconstruct(ctx, H.LeafKind(p, h, kappa), nbox, nrhs, b, S, _dev(v_np), _dev(ub_np), ui, prec, st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    for bx in range(nbox):
        uo, info = oracle.leaf_reconstruct(p, h, kappa, field(oracle.node_coords(p, lows[bx], h)), v_np[bx], ub_np[bx])
        assert rel_fro(ui[bx:bx + 1].cpu().numpy(), uo[None]).max() < tol
        assert max_rel(ui[bx:bx + 1].cpu().numpy(), uo[None]) < tol


@pytest.mark.parametrize("prec", [H.HPS_FP64, H.HPS_FP32_IR])
def test_status_singular_and_nonfinite(ctx, prec):
    """Host-side fault injection: the test hook zeroes row 0 of box 1's A_ii,
    which partial pivoting must meet as an exactly zero pivot; a NaN in box 2's
    b is reported as invalid input.  Box 0 is untouched."""
    p, h, kappa = 6, np.array([0.25] * 3), 5.0
    b = np.ones((3, p ** 3))
    b[2, 1 + p + p * p] = np.nan            # interior node (1,1,1)
    H.hps_set_option(ctx, H.HPS_OPT_TEST_SINGULAR_BOX, 1)
    try:
        _, _, st = gpu_dtn(ctx, p, h, kappa, b, prec, 1)
    finally:
        H.hps_set_option(ctx, H.HPS_OPT_TEST_SINGULAR_BOX, -1)
    assert st[0] == 0 and st[1] == H.HPS_ESINGULAR and st[2] == H.HPS_EINVAL, st


def test_argument_errors(ctx):
    import torch
    T = torch.empty(1, 6, 6, dtype=torch.float64, device="cuda")
    b = torch.ones(1, 27, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HpsError) as e:
        H.hps_leaf_build_dtn(ctx, H.LeafKind(2, 1.0, 0.0), 1, b, T)
    assert e.value.status == H.HPS_EINVAL
    with pytest.raises(H.HpsError):
        H.hps_leaf_build_dtn(ctx, H.LeafKind(3, 1.0, 0.0), 1, b, T, prec=7)
    H.hps_leaf_build_dtn(ctx, H.LeafKind(3, 1.0, 0.0), 0, b, T)            # nbox = 0: no-op


def test_chunked_workspace_matches(ctx):
    """A workspace that holds 3 boxes processes 8 boxes in chunks, bit-identically."""
    p, h, kappa = 8, np.array([0.125] * 3), 25.0
    lows = _lows(8, h, 8)
    b = box_b(H.hps_leaf_nodes, p, lows, h, hi.fourier_b_field().b)
    T_all, _, _ = gpu_dtn(ctx, p, h, kappa, b, H.HPS_FP32_IR, 1, want_S=False)
    small = H.hps_create(0, 3 * H.hps_workspace_per_box(p, H.HPS_FP32_IR) + 4096)
    try:
        T_ch, _, st = gpu_dtn(small, p, h, kappa, b, H.HPS_FP32_IR, 1, want_S=False)
    finally:
        H.hps_destroy(small)
    assert (st == 0).all()
    np.testing.assert_array_equal(T_all, T_ch)


@pytest.mark.parametrize("prec", [H.HPS_FP64, H.HPS_FP32_IR], ids=["fp64", "fp32ir"])
def test_dtn_into_pinned_host_memory(ctx, prec):
    """T written by the call straight into pinned host memory (the kernels
    store across the host link) equals T written to device memory, bit for
    bit, and matches the oracle."""
    import torch
    p, h, kappa = 12, np.array([0.125] * 3), 30.0
    lows = _lows(5, h, 12)
    b = box_b(H.hps_leaf_nodes, p, lows, h, hi.fourier_b_field().b)
    T_dev, _, _ = gpu_dtn(ctx, p, h, kappa, b, prec, 2 if prec != H.HPS_FP64 else 0, want_S=False)
    n, m = H.hps_leaf_sizes(p)
    T_host = torch.full((len(lows), m, m), float("nan"), dtype=torch.float64).pin_memory()
    st = torch.full((len(lows),), -1, dtype=torch.int32, device="cuda")
    bt = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    H.hps_leaf_build_dtn(ctx, H.LeafKind(p, h, kappa), len(lows), bt, T_host, None, prec, st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    np.testing.assert_array_equal(T_host.numpy(), T_dev)
    To, _, info = oracle.leaf_dtn(p, h, kappa, b[0], want_S=False)
    assert info == 0 and max_rel(T_host.numpy()[:1], To[None]) < 1e-10


def test_end_to_end_manufactured(ctx):
    """Config of the manufactured solution: the GPU's T, v, h feed the library's
    interface assembly and a host sparse LU; the GPU reconstructs u_i.  Matches
    the oracle's own two-level solve to 1e-11 and the exact solution to the
    discretisation error."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import torch
    from oracle import global_solve as gs
    kappa = 10.0
    p, h, _, lows, field = config_grid("manufactured")
    nbox = len(lows)
    n, m = H.hps_leaf_sizes(p)
    kind = H.LeafKind(p, h, kappa)
    set_tc(ctx, 1)
    b = _dev(box_b(H.hps_leaf_nodes, p, lows, h, field))
    f = _dev(np.stack([hi.manufactured(H.hps_leaf_nodes(p, lo, h), kappa)[1] for lo in lows])[:, None, :])
    T = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
    v = torch.empty(nbox, 1, n, dtype=torch.float64, device="cuda")
    hf = torch.empty(nbox, 1, m, dtype=torch.float64, device="cuda")
    H.hps_leaf_build_dtn(ctx, kind, nbox, b, T, None, H.HPS_FP64)
    H.hps_leaf_particular(ctx, kind, nbox, 1, b, f, v, hf, H.HPS_FP64)
    torch.cuda.synchronize()
    rows, cols, vals, rd, cd, vd, ni, nd = H.hps_assemble_interface_blocks(p, (2, 2, 2), T.cpu().numpy())
    Tg = sp.coo_matrix((vals, (rows, cols)), shape=(ni, ni)).tocsc()
    grid = gs.InterfaceGrid(p, (2, 2, 2))
    g = hi.manufactured(grid.dirichlet_coords(), kappa)[2]
    rhs = -sp.coo_matrix((vd, (rd, cd)), shape=(ni, nd)) @ g
    hf_np = hf.cpu().numpy()[:, 0, :]
    ub = np.empty((nbox, m))
    for bx in range(nbox):
        isi, gid = grid.local_to_global(bx)
        np.add.at(rhs, gid[isi], -hf_np[bx, isi])
    u_if = spla.splu(Tg).solve(rhs)
    for bx in range(nbox):
        isi, gid = grid.local_to_global(bx)
        ub[bx, isi] = u_if[gid[isi]]
        ub[bx, ~isi] = g[gid[~isi]]
    ui = torch.empty(nbox, 1, n, dtype=torch.float64, device="cuda")
    H.hps_leaf_reconstruct(ctx, kind, nbox, 1, b, None, v, _dev(ub[:, None, :]), ui, H.HPS_FP32_IR)
    torch.cuda.synchronize()
    ref = gs.hps_solve(grid, kappa, lambda x: np.ones(len(x)), lambda x: hi.manufactured(x, kappa)[1],
                       lambda x: hi.manufactured(x, kappa)[2])
    scale = np.abs(ref["u_int"]).max()
    assert np.abs(u_if - ref["u_iface"]).max() < 1e-11 * scale
    assert np.abs(ui.cpu().numpy()[:, 0, :] - ref["u_int"]).max() < 1e-10 * scale
    exact = hi.manufactured(gs.interior_coords(grid), kappa)[0]
    assert np.abs(ui.cpu().numpy()[:, 0, :] - exact).max() < 1e-4


@pytest.mark.parametrize("seed", [1, 20250304])
def test_integer_pipe_conversions_match_hardware(seed):
    """The refinement kernels convert FP64 <-> FP32 on the integer pipe; over
    16 M values (all exponents, float range limits, rounding ties) both
    directions agree bit for bit with the hardware conversions."""
    assert H.hps_selftest_conversions(0, 1 << 24, seed) == (0, 0)


@pytest.mark.parametrize("p", [21, 24])
def test_largest_orders_mixed_vs_fp64(ctx, p):
    """The largest supported orders (n = 6859 and 10648 interior nodes: the
    panel's inner block shrinks to a few columns, the tables and operator
    copies are at their largest), one box: both mixed precisions against the
    plain FP64 GPU path (the CPU oracle would take minutes at this size), the
    FP32 path in both of its operand formats."""
    import torch
    h = np.array([0.125] * 3)
    lows = np.array([[0.25, 0.5, 0.125]])
    b = box_b(H.hps_leaf_nodes, p, lows, h, hi.fourier_b_field().b)
    T64, _, st64 = gpu_dtn(ctx, p, h, 30.0, b, H.HPS_FP64, 0, want_S=False)
    assert (st64 == 0).all()
    for prec, tc in ((H.HPS_FP32_IR, 1), (H.HPS_FP32_IR, 2), (H.HPS_BF16_IR, 1)):
        T, _, st = gpu_dtn(ctx, p, h, 30.0, b, prec, tc, want_S=False)
        assert (st == 0).all(), st
        assert rel_fro(T, T64).max() < 1e-10, rel_fro(T, T64)
        assert max_rel(T, T64) < 1e-10
    torch.cuda.empty_cache()



def test_every_order_fp32ir_matches_fp64_path(ctx):
    """Every order p = 3..24 (one to 84 LU steps, last steps from 1 to 128
    columns wide, every unit layout): the tensor-core FP32 + refinement T of
    two boxes equals the FP64 path's T to 1e-11 of its largest entry."""
    import torch
    set_tc(ctx, 2)
    H.hps_set_option(ctx, H.HPS_OPT_BLOCK, 0)
    h = np.array([0.125] * 3)
    for p in range(3, 25):
        n, m = H.hps_leaf_sizes(p)
        b = np.stack([1 + 0.3 * np.sin(2 * oracle.node_coords(p, np.array([0.1 * i, 0.0, 0.2]), h)[:, 0])
                      for i in range(2)])
        bt = _dev(b)
        out = {}
        for prec in (H.HPS_FP64, H.HPS_FP32_IR):
            T = torch.empty(2, m, m, dtype=torch.float64, device="cuda")
            st = torch.full((2,), -1, dtype=torch.int32, device="cuda")
            H.hps_leaf_build_dtn(ctx, H.LeafKind(p, h, 12.0), 2, bt, T, None, prec, st)
            torch.cuda.synchronize()
            assert (st.cpu().numpy() == 0).all(), (p, prec)
            out[prec] = T.cpu().numpy()
        assert max_rel(out[H.HPS_FP32_IR], out[H.HPS_FP64]) < 1e-11, p
