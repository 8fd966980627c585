"""The no-allocation FP64 DtN build against the regular entry point.

hps_leaf_build_dtn_noalloc exists for callers that cannot allocate device
memory (their GPU memory belongs to another allocator, or cudaMalloc's implicit
synchronisation is too costly in their loop); it keeps all scratch in one
static device array of the library.  This file is collected last on purpose,
so that a failure here stops a -x run only after every other test has run.
"""
from __future__ import annotations

import numpy as np
import pytest

import hps_inputs as hi
import paper_2503_04033_gb300 as H
from tests._cases import box_b, rel_fro

pytestmark = pytest.mark.gpu


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    p, kappa = 8, 17.0
    lows, h = hi.box_grid_lo((5, 4, 2))            # 40 boxes: more than one scratch chunk at p = 8
    n, m = H.hps_leaf_sizes(p)
    ctx = H.hps_create(0, 0)
    try:
        for call, field in enumerate((hi.fourier_b_field().b, hi.gaussian_dip_b)):
            b = torch.from_numpy(box_b(H.hps_leaf_nodes, p, lows, h, field)).cuda()
            nbox = b.shape[0]
            T_ref = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
            st_ref = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
            H.hps_leaf_build_dtn(ctx, H.LeafKind(p, h, kappa), nbox, b, T_ref, None, H.HPS_FP64, st_ref)
            T = torch.full((nbox, m, m), float("nan"), dtype=torch.float64, device="cuda")
            st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
            H.hps_leaf_build_dtn_noalloc(H.LeafKind(p, h, kappa), nbox, b, T, st)
            torch.cuda.synchronize()
            assert (st.cpu().numpy() == 0).all() and (st_ref.cpu().numpy() == 0).all(), call
            err = rel_fro(T.cpu().numpy(), T_ref.cpu().numpy())
            assert err.max() < 1e-11, (call, err.max())
    finally:
        H.hps_destroy(ctx)


def test_noalloc_rejects_boxes_larger_than_its_scratch():
    import torch
    p = 16
    b = torch.ones(1, p ** 3, dtype=torch.float64, device="cuda")
    n, m = H.hps_leaf_sizes(p)
    T = torch.empty(1, m, m, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HpsError) as e:
        H.hps_leaf_build_dtn_noalloc(H.LeafKind(p, 0.125, 40.0), 1, b, T)
    assert e.value.status == H.HPS_ENOMEM
