"""Failure detection of the tensor-core products without a GPU fault.

Every mbarrier wait of the tcgen05 update kernel is bounded.  The test hook
HPS_OPT_TEST_TC_TIMEOUT makes one product launch issue no operand loads, so
its first wait has nothing that will ever complete it; the wait gives up
after 2 ms, the launch drains what it has in flight (the epilogue's source
loads, any MMAs), frees its tensor memory and returns, and every box of the
call reports HPS_ETIMEOUT.  A normal call on the same context right after
must succeed and match the oracle: the context stays usable.
"""
from __future__ import annotations

import numpy as np
import pytest

import hps_inputs as hi
import oracle
import paper_2503_04033_gb300 as H
from tests._cases import box_b, max_rel, rel_fro

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp16", [1, 0], ids=["fp16", "tf32"])
def test_stalled_product_reports_timeout_then_recovers(fp16):
    import torch
    p, kappa = 9, 14.0
    lows, h = hi.box_grid_lo((2, 2, 1))
    field = hi.fourier_b_field().b
    n, m = H.hps_leaf_sizes(p)
    nbox = len(lows)
    b = torch.from_numpy(box_b(H.hps_leaf_nodes, p, lows, h, field)).cuda()
    ctx = H.hps_create(0, 0)
    try:
        H.hps_set_option(ctx, H.HPS_OPT_TENSOR_CORES, 1)
        H.hps_set_option(ctx, H.HPS_OPT_FP16_OPERANDS, fp16)
        T = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
        st = torch.full((nbox,), -1, dtype=torch.int32, device="cuda")
        H.hps_set_option(ctx, H.HPS_OPT_TEST_TC_TIMEOUT, 1)
        H.hps_leaf_build_dtn(ctx, H.LeafKind(p, h, kappa), nbox, b, T, None, H.HPS_FP32_IR, st)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == H.HPS_ETIMEOUT).all(), st
        # the hook fires once: the next call runs normally on the same context
        st.fill_(-1)
        H.hps_leaf_build_dtn(ctx, H.LeafKind(p, h, kappa), nbox, b, T, None, H.HPS_FP32_IR, st)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all(), st
    finally:
        H.hps_destroy(ctx)
    To, _, sto = oracle.batch_dtn(p, h, kappa, box_b(oracle.node_coords, p, lows, h, field))
    assert (sto == 0).all()
    Tg = T.cpu().numpy()
    assert rel_fro(Tg, To).max() < 1e-10 and max_rel(Tg, To) < 1e-10
