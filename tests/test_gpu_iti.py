"""Leaf impedance-to-impedance maps on the GPU through the C ABI, against the
FP64 oracle (oracle/iti.py): element-wise parity on boxes with variable b
and anisotropic sides, including a box at a Dirichlet resonance (where the
DtN map does not exist), and the argument checks."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2503_04033_gb300 as H
from oracle import iti
from tests._cases import max_rel

pytestmark = pytest.mark.gpu

TOL = 1e-11


def _gpu_iti(p, h, kappa, eta, bs):
    import torch
    n, m = H.hps_leaf_sizes(p)
    kind = H.LeafKind(p, h, kappa)
    b = torch.from_numpy(np.ascontiguousarray(np.stack(bs))).cuda()
    R = torch.empty(len(bs), m, m, dtype=torch.complex128, device="cuda")
    st = torch.full((len(bs),), -1, dtype=torch.int32, device="cuda")
    H.hps_leaf_iti(kind, eta, len(bs), b, R, st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all(), st
    return R.cpu().numpy()


@pytest.mark.parametrize("p", [4, 5, 6, 8])
def test_iti_parity(p):
    """Three boxes of a variable field (anisotropic sides), two values of
    eta: every entry within 1e-11 of the oracle's largest."""
    h = np.array([0.3, 0.25, 0.35])
    rng = np.random.default_rng(p)
    lows = rng.uniform(-1, 1, size=(3, 3))
    kappa = 9.0
    bs = []
    for lo in lows:
        x = oracle.node_coords(p, lo, h)
        bs.append(1 + 0.4 * np.sin(2 * x[:, 0] + x[:, 2]) * np.cos(3 * x[:, 1]))
    for eta in (kappa, -3.5):
        R = _gpu_iti(p, h, kappa, eta, bs)
        for bx in range(3):
            Ro = iti.leaf_iti(p, h, kappa, bs[bx], eta)
            assert max_rel(R[bx:bx + 1], Ro[None]) < TOL, (p, eta, bx, max_rel(R[bx:bx + 1], Ro[None]))


def test_iti_at_a_dirichlet_resonance():
    """kappa^2 the smallest eigenvalue of the box's interior block (b = 1,
    p = 8): the GPU map equals the oracle's and stays of moderate norm."""
    p, h = 8, np.array([0.2, 0.2, 0.2])
    n, m = oracle.sizes(p)
    Aii = oracle.leaf_matrix(p, h, 0.0, np.ones(p ** 3))[:n, :n]
    ev = np.linalg.eigvals(Aii)
    kappa = float(np.sqrt(np.sort(ev[np.abs(ev.imag) < 1e-8].real)[0]))
    R = _gpu_iti(p, h, kappa, kappa, [np.ones(p ** 3)])
    Ro = iti.leaf_iti(p, h, kappa, np.ones(p ** 3), kappa)
    assert max_rel(R, Ro[None]) < 1e-10
    assert np.linalg.norm(R[0], 2) < 10.0


def test_iti_argument_errors():
    import torch
    b = torch.ones(1, 64, dtype=torch.float64, device="cuda")
    R = torch.empty(1, 24, 24, dtype=torch.complex128, device="cuda")
    for kind, eta in ((H.LeafKind(3, 0.5, 1.0), 1.0), (H.LeafKind(4, 0.5, 1.0), 0.0),
                      (H.LeafKind(4, -0.5, 1.0), 1.0), (H.LeafKind(17, 0.5, 1.0), 1.0)):
        with pytest.raises(H.HpsError) as e:
            H.hps_leaf_iti(kind, eta, 1, b, R)
        assert e.value.status == H.HPS_EINVAL
