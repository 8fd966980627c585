"""The library's host routines of the mixed-order (adaptive p) interface
system against the oracle (oracle/adaptive.py): layout, face coordinates,
the assembled matrix blocks, the reduced fluxes and the box traces.  Host
code only: runs without a GPU."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import paper_2503_04033_gb300 as H
from oracle import adaptive as ad


def _grid(nb, kind):
    n = int(np.prod(nb))
    rng = np.random.default_rng(n + kind)
    if kind == 0:
        return [6 if (i % nb[0] + (i // nb[0]) % nb[1] + i // (nb[0] * nb[1])) % 2 == 0 else 8 for i in range(n)]
    return list(rng.choice([5, 6, 7, 9], size=n))


@pytest.mark.parametrize("nb,kind", [((2, 2, 2), 0), ((3, 2, 1), 1), ((2, 1, 2), 1)])
def test_mixed_host_routines_match_the_oracle(nb, kind):
    pb = _grid(nb, kind)
    og = ad.MixedGrid(pb, nb, lo=(0.1, -0.2, 0.0), L=(1.0, 0.8, 1.2))
    ni, nd, fp, fo = H.hps_mixed_layout(nb, pb)
    assert (ni, nd) == (og.n_iface, og.n_dir)
    assert np.array_equal(fp, og.face_p) and np.array_equal(fo, og.face_off)
    xyz = H.hps_mixed_face_coords(nb, pb, (0.1, -0.2, 0.0), (1.0, 0.8, 1.2))
    assert np.abs(xyz - og.face_node_coords()).max() < 1e-14
    rng = np.random.default_rng(3)
    Ts = [rng.standard_normal((6 * (p - 2) ** 2,) * 2) for p in pb]
    hs = [rng.standard_normal(6 * (p - 2) ** 2) for p in pb]
    A = sp.csr_matrix((ni + nd, ni + nd))
    red = np.zeros(ni + nd)
    maps = []
    for box in range(og.nbox):
        P, Q = og.box_maps(box)
        A = A + Q @ sp.csr_matrix(Ts[box]) @ P
        red += Q @ hs[box]
        maps.append(P)
    r, c, v, rd, cd, vd = H.hps_mixed_assemble(nb, pb, Ts)
    Ai = sp.coo_matrix((v, (r, c)), shape=(ni, ni)).toarray()
    Ad = sp.coo_matrix((vd, (rd, cd)), shape=(ni, nd)).toarray()
    ref = A.toarray()
    scale = np.abs(ref).max()
    assert np.abs(Ai - ref[:ni, :ni]).max() < 1e-12 * scale
    assert np.abs(Ad - ref[:ni, ni:]).max() < 1e-12 * scale
    assert np.abs(H.hps_mixed_reduce(nb, pb, hs) - red).max() < 1e-12 * np.abs(red).max()
    u = rng.standard_normal(ni + nd)
    for box, ub in enumerate(H.hps_mixed_traces(nb, pb, u)):
        assert np.abs(ub - maps[box] @ u).max() < 1e-12 * np.abs(u).max()


def test_mixed_host_argument_errors():
    with pytest.raises(H.HpsError):
        H.hps_mixed_layout((2, 2, 2), [6] * 7 + [2])
    with pytest.raises(H.HpsError):
        H.hps_mixed_layout((2, 0, 2), [])
    with pytest.raises(ValueError):
        H.hps_mixed_layout((2, 2, 2), [6] * 7)
