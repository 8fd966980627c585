"""FP64 oracle of the leaf impedance-to-impedance (ItI) map.

TEST INFRASTRUCTURE ONLY (part of the oracle; see ``oracle/__init__.py``).

The paper's closing section (Sec. 6) names HPS built on
impedance-to-impedance maps (Gillman, Barnett and Martinsson's formulation)
as a variant the two-level scheme adapts to; such maps do not fail where
kappa^2 is a Dirichlet eigenvalue of a box, as DtN maps do.  On the leaf
collocation of Sec. 2.1 (the
kept nodes: interior and face nodes, Eq. 2's rows) the ItI map R takes
impedance data f = du/dn + i eta u on the face nodes to g = du/dn - i eta u
for the solution u of the homogeneous equation in the box:

    [ A_ii   A_ib            ] [u_i]   [0]
    [ A_bi   A_bb + i eta I  ] [u_b] = [f],     g = f - 2 i eta u_b.

Unlike the DtN map it never inverts A_ii on its own, so it exists where
kappa^2 is a Dirichlet eigenvalue of the box's interior block.  Where T
exists, the block elimination of u_i gives (T + i eta I) u_b = f, so
R = (T - i eta I)(T + i eta I)^{-1}: that identity is the first pin.
"""
from __future__ import annotations

import numpy as np

from . import leaf_matrix, sizes


def leaf_iti(p: int, h, kappa: float, b: np.ndarray, eta: float) -> np.ndarray:
    """R [m, m] (complex) of one box: the kept-node collocation matrix with
    i eta added on the face rows' own unknowns, solved for the m unit
    impedance data vectors (numpy's complex LU solve as the step)."""
    n, m = sizes(p)
    A = leaf_matrix(p, h, kappa, b).astype(np.complex128)
    A[n:, n:] += 1j * eta * np.eye(m)
    rhs = np.zeros((n + m, m), dtype=np.complex128)
    rhs[n:, :] = np.eye(m)
    ub = np.linalg.solve(A, rhs)[n:, :]
    return np.eye(m) - 2j * eta * ub


def iti_from_dtn(T: np.ndarray, eta: float) -> np.ndarray:
    """(T - i eta I)(T + i eta I)^{-1}: the ItI map of a box whose DtN map is T."""
    m = T.shape[0]
    E = 1j * eta * np.eye(m)
    return np.linalg.solve((T + E).T, (T - E).T).T
