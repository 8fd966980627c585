"""The no-allocation FP64 DtN build against the regular entry point.

hps_leaf_build_dtn_noalloc exists for callers that cannot allocate device
memory (their GPU memory belongs to another allocator, or cudaMalloc's implicit
synchronisation is too costly in their loop); it keeps all scratch in one
static device array of the library.  Both entry points build the operator
tables with the same helper and run the same kernels per box, so T must come
out identical, bit for bit.  This file is collected last on purpose, so that a
failure here stops a -x run only after every other test has run.
"""
from __future__ import annotations

import numpy as np
import pytest

import hps_inputs as hi
import paper_2503_04033_gb300 as H
from tests._cases import box_b

pytestmark = pytest.mark.gpu


def _regular(ctx, p, h, kappa, b):
    import torch
    n, m = H.hps_leaf_sizes(p)
    nbox = b.shape[0]
    T = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
    st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
    H.hps_leaf_build_dtn(ctx, H.LeafKind(p, h, kappa), nbox, b, T, None, H.HPS_FP64, st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    return T.cpu().numpy()


def _noalloc(p, h, kappa, b, with_status=True):
    import torch
    n, m = H.hps_leaf_sizes(p)
    nbox = b.shape[0]
    T = torch.full((nbox, m, m), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda") if with_status else None
    H.hps_leaf_build_dtn_noalloc(H.LeafKind(p, h, kappa), nbox, b, T, st)
    torch.cuda.synchronize()
    if with_status:
        assert (st.cpu().numpy() == 0).all()
    return T.cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice():
    """Two calls in a row with a different order p and box size (the scratch
    keeps the first call's tables and status words), the second without a
    status array (its status words then live in the scratch as well)."""
    import torch
    ctx = H.hps_create(0, 0)
    try:
        cases = [(8, (5, 4, 2), 17.0, hi.fourier_b_field().b, True),   # 40 boxes: several scratch chunks
                 (10, (3, 2, 2), 11.0, hi.gaussian_dip_b, False)]
        for call, (p, grid, kappa, field, with_status) in enumerate(cases):
            lows, h = hi.box_grid_lo(grid)
            b = torch.from_numpy(box_b(H.hps_leaf_nodes, p, lows, h, field)).cuda()
            T_ref = _regular(ctx, p, h, kappa, b)
            T = _noalloc(p, h, kappa, b, with_status)
            assert np.isfinite(T).all(), call
            assert np.array_equal(T, T_ref), (call, np.abs(T - T_ref).max())
    finally:
        H.hps_destroy(ctx)


def test_noalloc_largest_order_and_rejection():
    """p = 14 (about 60 MiB of workspace for one box) fits the 64 MiB scratch;
    p = 15 returns HPS_ENOMEM with nothing enqueued."""
    import torch
    ctx = H.hps_create(0, 0)
    try:
        lows, h = hi.box_grid_lo((2, 1, 1))
        b = torch.from_numpy(box_b(H.hps_leaf_nodes, 14, lows, h, hi.gaussian_dip_b)).cuda()
        assert np.array_equal(_noalloc(14, h, 9.0, b), _regular(ctx, 14, h, 9.0, b))
    finally:
        H.hps_destroy(ctx)
    p = 15
    b = torch.ones(1, p ** 3, dtype=torch.float64, device="cuda")
    n, m = H.hps_leaf_sizes(p)
    T = torch.empty(1, m, m, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HpsError) as e:
        H.hps_leaf_build_dtn_noalloc(H.LeafKind(p, 0.125, 40.0), 1, b, T)
    assert e.value.status == H.HPS_ENOMEM
