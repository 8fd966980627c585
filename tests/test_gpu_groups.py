"""Mixed batches (hps_leaf_groups): orders p in one call, a wavenumber per box,
DtN maps and particular solutions from one factorisation, CUDA-graph replay
and block autotuning, all against the FP64 oracle."""
from __future__ import annotations

import os

import numpy as np
import pytest

import hps_inputs as hi
import oracle
import paper_2503_04033_gb300 as H
from tests._cases import max_rel, rel_fro

pytestmark = pytest.mark.gpu

TOL = {H.HPS_FP64: 1e-11, H.HPS_FP32_IR: 1e-10, H.HPS_BF16_IR: 1e-10}


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def make_group(p, lows, h, kappas, field, loads, with_T=True, with_S=False):
    import torch
    n, m = H.hps_leaf_sizes(p)
    nbox = len(lows)
    b = np.stack([field(H.hps_leaf_nodes(p, lo, h)) for lo in lows])
    g = {"p": p, "h": h, "kappa": np.asarray(kappas, dtype=np.float64), "b": _dev(b),
         "box_status": torch.full((nbox,), -1, dtype=torch.int32, device="cuda")}
    if with_T:
        g["T"] = torch.empty(nbox, m, m, dtype=torch.float64, device="cuda")
    if with_S:
        g["S"] = torch.empty(nbox, n, m, dtype=torch.float64, device="cuda")
    if loads:
        f = np.stack([hi.load_values(loads, H.hps_leaf_nodes(p, lo, h)) for lo in lows])
        g["f"] = _dev(f)
        g["v"] = torch.empty(nbox, len(loads), n, dtype=torch.float64, device="cuda")
        g["hflux"] = torch.empty(nbox, len(loads), m, dtype=torch.float64, device="cuda")
    return g


def check_group(g, lows, field, loads, tol, boxes=None):
    p, h = g["p"], np.broadcast_to(np.asarray(g["h"], dtype=np.float64), (3,))
    assert (g["box_status"].cpu().numpy() == 0).all(), g["box_status"]
    for bx in (range(len(lows)) if boxes is None else boxes):
        xyz = oracle.node_coords(p, lows[bx], h)
        kap = float(g["kappa"][bx])
        pairs = []
        if "T" in g:
            To, So, info = oracle.leaf_dtn(p, h, kap, field(xyz), want_S="S" in g)
            assert info == 0
            pairs.append((g["T"][bx:bx + 1].cpu().numpy(), To[None]))
            if "S" in g:
                pairs.append((g["S"][bx:bx + 1].cpu().numpy(), So[None]))
        if loads:
            vo, ho, info = oracle.leaf_particular(p, h, kap, field(xyz), hi.load_values(loads, xyz))
            assert info == 0
            pairs += [(g["v"][bx:bx + 1].cpu().numpy(), vo[None]), (g["hflux"][bx:bx + 1].cpu().numpy(), ho[None])]
        for got, ref in pairs:
            assert rel_fro(got, ref).max() < tol, (p, bx, rel_fro(got, ref).max())
            assert max_rel(got, ref) < tol, (p, bx, max_rel(got, ref))


@pytest.fixture(scope="module")
def ctx():
    c = H.hps_create(0, 0)
    yield c
    H.hps_destroy(c)


@pytest.mark.parametrize("prec", [H.HPS_FP64, H.HPS_FP32_IR, H.HPS_BF16_IR])
def test_groups_mixed_p_kappa_loads(ctx, prec):
    import torch
    H.hps_set_option(ctx, H.HPS_OPT_TENSOR_CORES, 1)
    rng = np.random.default_rng(3)
    h = np.array([0.125] * 3)
    field = hi.fourier_b_field().b
    loads = hi.fourier_b_per_box(3, 11)
    spec = [(5, 3, True, True, loads), (8, 4, True, False, loads), (6, 2, False, False, loads), (9, 2, True, True, [])]
    groups, lows_all = [], []
    for p, nb, wT, wS, ld in spec:
        lows = rng.integers(0, 8, size=(nb, 3)) * h
        kap = rng.choice([10.0, 20.0, 40.0], size=nb)
        groups.append(make_group(p, lows, h, kap, field, ld, with_T=wT, with_S=wS))
        lows_all.append((lows, ld))
    H.hps_leaf_groups(ctx, groups, prec)
    torch.cuda.synchronize()
    for g, (lows, ld) in zip(groups, lows_all):
        check_group(g, lows, field, ld, TOL[prec])


def test_groups_graph_replay_matches_direct(ctx):
    """With graphs on, the first call captures and the second replays; new
    values of b and kappa in the same buffers are picked up."""
    import torch
    h = np.array([0.25] * 3)
    lows = np.array([[0, 0, 0], [0.25, 0.5, 0], [0.5, 0.25, 0.75]])
    field1, field2 = hi.fourier_b_field().b, hi.gaussian_dip_b
    loads = hi.fourier_b_per_box(2, 5)
    g = make_group(8, lows, h, [12.0, 15.0, 18.0], field1, loads)
    H.hps_set_option(ctx, H.HPS_OPT_GRAPHS, 1)
    try:
        H.hps_leaf_groups(ctx, [g], H.HPS_FP32_IR)
        torch.cuda.synchronize()
        check_group(g, lows, field1, loads, 1e-10)
        g["b"].copy_(_dev(np.stack([field2(H.hps_leaf_nodes(8, lo, h)) for lo in lows])))
        g["kappa"] = np.array([9.0, 21.0, 30.0])
        g["T"].fill_(float("nan"))
        H.hps_leaf_groups(ctx, [g], H.HPS_FP32_IR)        # replay of the cached graph
        torch.cuda.synchronize()
        check_group(g, lows, field2, loads, 1e-10)
    finally:
        H.hps_set_option(ctx, H.HPS_OPT_GRAPHS, 0)


def test_autotune_writes_cache_and_matches(tmp_path, monkeypatch):
    import torch
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("HPS_TUNE_CACHE", str(cache))
    c = H.hps_create(0, 0)
    try:
        H.hps_set_option(c, H.HPS_OPT_AUTOTUNE, 1)
        h = np.array([0.125] * 3)
        lows = np.array([[0, 0, 0], [0.5, 0.5, 0.5]])
        field = hi.gaussian_dip_b
        g = make_group(10, lows, h, [20.0, 25.0], field, [])
        H.hps_leaf_groups(c, [g], H.HPS_FP32_IR)
        torch.cuda.synchronize()
        check_group(g, lows, field, [], 1e-10)
    finally:
        H.hps_destroy(c)
    rows = [list(map(int, ln.split())) for ln in cache.read_text().splitlines()]
    assert any(r[0] == 10 and r[1] == H.HPS_FP32_IR and r[3] in (64, 128) for r in rows), rows


def test_uneven_batch_p8_to_p20_sampled(ctx):
    """The uneven workload's shape: orders 8, 12, 16, 20 in one call, kappa per
    box from {10, 20, 40, 60}, 32 loads per box at every order (DtN map and
    particular solutions from one factorisation); sampled boxes vs the
    oracle, including a p = 20 box's T, v and h."""
    import torch
    d = hi.uneven_batch(nbox=24, nloads=32)
    groups, meta = [], []
    for p in (8, 12, 16, 20):
        sel = np.nonzero(d["p"] == p)[0][:3]
        if len(sel) == 0:
            continue
        loads = d["loads"]
        groups.append(make_group(p, d["lo"][sel], d["h"], d["kappa"][sel], d["b_field"].b, loads))
        meta.append((d["lo"][sel], loads, [0] if p == 20 else None))
    H.hps_set_option(ctx, H.HPS_OPT_TENSOR_CORES, 1)
    H.hps_leaf_groups(ctx, groups, H.HPS_FP32_IR)
    torch.cuda.synchronize()
    for g, (lows, loads, boxes) in zip(groups, meta):
        check_group(g, lows, d["b_field"].b, loads, 1e-10, boxes=boxes)


@pytest.mark.parametrize("graphs", [0, 1], ids=["direct", "graph"])
def test_groups_concurrent_equals_sequential(ctx, graphs):
    """Four orders run concurrently (one stream and workspace slice each,
    the default) give bit-identical maps and loads to the same batch run one
    group after another, also when the call is captured into a graph."""
    import torch
    rng = np.random.default_rng(21)
    h = np.array([0.125] * 3)
    field = hi.fourier_b_field().b
    loads = hi.fourier_b_per_box(2, 13)
    spec = [(6, 3), (8, 5), (10, 2), (12, 2)]
    groups = []
    for p, nb in spec:
        lows = rng.integers(0, 8, size=(nb, 3)) * h
        groups.append(make_group(p, lows, h, rng.choice([10.0, 30.0], size=nb), field, loads))
    outs = []
    H.hps_set_option(ctx, H.HPS_OPT_GRAPHS, graphs)
    try:
        for conc in (0, 1, 1):
            H.hps_set_option(ctx, H.HPS_OPT_GROUPS_CONCURRENT, conc)
            for g in groups:
                g["T"].fill_(float("nan"))
            H.hps_leaf_groups(ctx, groups, H.HPS_FP32_IR)
            torch.cuda.synchronize()
            outs.append([(g["T"].cpu().numpy(), g["v"].cpu().numpy(), g["hflux"].cpu().numpy()) for g in groups])
            for g in groups:
                assert (g["box_status"].cpu().numpy() == 0).all()
    finally:
        H.hps_set_option(ctx, H.HPS_OPT_GROUPS_CONCURRENT, 1)
        H.hps_set_option(ctx, H.HPS_OPT_GRAPHS, 0)
    for run in outs[1:]:
        for a, b in zip(outs[0], run):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
