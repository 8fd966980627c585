"""The library's host assembly of the two-level system on ItI maps against
the oracle's (oracle/iti.py): matrix and right-hand side from the same leaf
operators.  Host code only: runs without a GPU."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import paper_2503_04033_gb300 as H
from oracle import iti
from oracle.global_solve import InterfaceGrid, face_node_grid_indices


@pytest.mark.parametrize("nb", [(2, 2, 2), (3, 1, 2)])
def test_iti_assembly_matches_the_oracle(nb):
    p, kappa, eta = 5, 6.0, 4.0
    grid = InterfaceGrid(p, nb)
    b_fn = lambda x: 1 + 0.3 * np.sin(x[:, 0] + 2 * x[:, 1])
    f_fn = lambda x: np.cos(x[:, 2])
    g_fn = lambda x: x[:, 0] * x[:, 1] + np.sin(x[:, 2])
    ro = iti.iti_solve(grid, kappa, eta, b_fn, f_fn, g_fn)
    Rs, hs, gs = [], [], []
    for box in range(grid.nbox):
        x = oracle.node_coords(p, grid.box_lo(box), grid.h)
        R, S, v, ho = iti.leaf_iti_ops(p, grid.h, kappa, b_fn(x), eta, f_fn(x)[None, :])
        Rs.append(R)
        hs.append(ho[0])
        gs.append(g_fn(x[face_node_grid_indices(p)]))
    r, c, v = H.hps_iti_assemble(p, nb, np.stack(Rs))
    N = grid.nbox * Rs[0].shape[0]
    A = sp.coo_matrix((v, (r, c)), shape=(N, N)).toarray()
    Ao = ro["A"].toarray()
    assert np.abs(A - Ao).max() < 1e-13 * np.abs(Ao).max()
    rhs = H.hps_iti_rhs(p, nb, eta, np.stack(hs), np.stack(gs))
    assert np.abs(rhs - ro["rhs"]).max() < 1e-13 * np.abs(ro["rhs"]).max()


def test_iti_host_argument_errors():
    with pytest.raises(H.HpsError):
        H.hps_iti_rhs(3, (2, 2, 2), 1.0)
    with pytest.raises(H.HpsError):
        H.hps_iti_rhs(5, (2, 2, 2), 0.0)
