"""CPU-side checks of the C ABI library: it loads, exports every function that
include/hps.h declares, and its host-only routines (sizes, nodes, interface
assembly) agree with the oracle.  No kernel runs here."""
from __future__ import annotations

import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import global_solve as gs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H():
    import paper_2503_04033_gb300 as H
    if not os.path.exists(H.library_path()):
        from paper_2503_04033_gb300 import build
        build.build()
    H.load_library()
    return H


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hps.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hps_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_function(H):
    names = declared_functions()
    assert len(names) >= 14, names
    lib = H.load_library()
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(H.EXPORTED_SYMBOLS)


def test_sizes_and_nodes(H):
    for p in (3, 8, 16, 20, 24):
        q = p - 2
        assert H.hps_leaf_sizes(p) == (q ** 3, 6 * q * q)
    for bad in (2, 25, -1):
        with pytest.raises(H.HpsError):
            H.hps_leaf_sizes(bad)
    lo, h = (0.25, -0.5, 1.0), (0.125, 0.25, 0.5)
    np.testing.assert_allclose(H.hps_leaf_nodes(11, lo, h), oracle.node_coords(11, lo, h), rtol=0, atol=1e-15)
    assert H.hps_workspace_per_box(16, H.HPS_FP32_IR) > H.hps_workspace_per_box(8, H.HPS_FP32_IR) > 0


def test_create_without_device_fails_cleanly(H):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(H.HpsError) as e:
        H.hps_create(0, 0)
    assert e.value.status in (H.HPS_ECUDA, H.HPS_EINVAL)


@pytest.mark.parametrize("nb", [(2, 2, 2), (3, 1, 2), (1, 1, 1)])
def test_interface_assembly_matches_oracle(H, nb):
    p = 5
    grid = gs.InterfaceGrid(p, nb, L=(1.0, 0.7, 1.3))
    rng = np.random.default_rng(1)
    n, m = oracle.sizes(p)
    T = rng.standard_normal((grid.nbox, m, m))
    nnz, nnz_d, ni, nd = H.hps_assemble_interface_blocks(p, nb)
    assert (ni, nd) == (grid.n_iface, grid.n_dir)
    rows, cols, vals, rd, cd, vd, ni2, nd2 = H.hps_assemble_interface_blocks(p, nb, T)
    assert len(vals) == nnz and len(vd) == nnz_d and (ni2, nd2) == (ni, nd)
    # oracle's assembly, written independently in oracle.global_solve
    Ti = np.zeros((ni, ni))
    Td = np.zeros((ni, nd))
    for box in range(grid.nbox):
        isi, gid = grid.local_to_global(box)
        ri, rd_ = np.nonzero(isi)[0], np.nonzero(~isi)[0]
        Ti[np.ix_(gid[ri], gid[ri])] += T[box][np.ix_(ri, ri)]
        Td[np.ix_(gid[ri], gid[rd_])] += T[box][np.ix_(ri, rd_)]
    if ni:
        A = sp.coo_matrix((vals, (rows, cols)), shape=(ni, ni)).toarray()
        np.testing.assert_allclose(A, Ti, rtol=0, atol=1e-14)
    if ni and nd:
        Ad = sp.coo_matrix((vd, (rd, cd)), shape=(ni, nd)).toarray()
        np.testing.assert_allclose(Ad, Td, rtol=0, atol=1e-14)


def test_assembly_rejects_bad_arguments(H):
    with pytest.raises(H.HpsError):
        H.hps_assemble_interface_blocks(2, (2, 2, 2))
    with pytest.raises(H.HpsError):
        H.hps_assemble_interface_blocks(8, (0, 2, 2))


def test_binding_refuses_short_arrays_before_any_launch():
    """The leaf bindings check tensor sizes against nbox and p on the host:
    a b with fewer than nbox p^3 entries is refused before the library is
    called (no device access happens)."""
    import pytest
    import torch
    import paper_2503_04033_gb300 as H
    kind = H.LeafKind(8, 0.125, 10.0)
    n, m = H.hps_leaf_sizes(8)
    b = torch.zeros(3 * 8 ** 3, dtype=torch.float64)
    T = torch.zeros(4 * m * m, dtype=torch.float64)
    with pytest.raises(ValueError, match="b:"):
        H.hps_leaf_build_dtn(None, kind, 4, b, T)
    with pytest.raises(ValueError, match="ub:"):
        H.hps_leaf_reconstruct(None, kind, 4, 1, torch.zeros(4 * 8 ** 3, dtype=torch.float64), None, None,
                               torch.zeros(4 * m - 1, dtype=torch.float64), torch.zeros(4 * n, dtype=torch.float64))
