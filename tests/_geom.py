"""Closed-form test fields for the leaf reduction (no method arithmetic).

Polynomials of degree <= p-1 in each variable are reproduced exactly by the
Chebyshev collocation, so their Laplacian and normal derivatives give exact
expected values for S, T, v and h at any b.
"""
from __future__ import annotations

import numpy as np

FACE_NORMALS = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]], dtype=np.float64)


def kept_grid_indices(p: int):
    """(interior grid indices [n], face grid indices [m], face id of each face node [m])."""
    q = p - 2
    r = np.arange(1, q + 1)
    k, j, i = np.meshgrid(r, r, r, indexing="ij")
    interior = (i + p * j + p * p * k).reshape(-1)
    e = p - 1
    face, fid = [], []
    for f in range(6):
        axis, side = f // 2, (0 if f % 2 == 0 else e)
        for bb in range(1, q + 1):
            for aa in range(1, q + 1):
                g = [aa, bb]
                ijk = g[:axis] + [side] + g[axis:]
                face.append(ijk[0] + p * ijk[1] + p * p * ijk[2])
                fid.append(f)
    return interior.astype(np.int64), np.asarray(face, dtype=np.int64), np.asarray(fid)


class TensorPoly:
    """u = sum_t c_t sx^a_t sy^b_t sz^c_t in box-local coordinates s = (x - ctr)/(h/2)."""

    def __init__(self, terms, ctr, h):
        self.terms = [(float(c), int(a), int(b), int(d)) for c, a, b, d in terms]
        self.ctr = np.asarray(ctr, dtype=np.float64)
        self.sc = 2.0 / np.asarray(h, dtype=np.float64)

    @staticmethod
    def random(rng, p, ctr, h, nterms=6):
        terms = [(rng.standard_normal(), *rng.integers(0, p, size=3)) for _ in range(nterms)]
        return TensorPoly(terms, ctr, h)

    def _s(self, xyz):
        return (xyz - self.ctr) * self.sc

    @staticmethod
    def _pw(s, a, d):
        """d-th derivative of s^a."""
        if a < d:
            return np.zeros_like(s)
        coef = 1.0
        for t in range(d):
            coef *= a - t
        return coef * s ** (a - d)

    def value(self, xyz):
        s = self._s(xyz)
        return sum(c * self._pw(s[:, 0], a, 0) * self._pw(s[:, 1], b, 0) * self._pw(s[:, 2], d, 0)
                   for c, a, b, d in self.terms)

    def grad(self, xyz):
        s = self._s(xyz)
        g = np.zeros_like(xyz)
        for c, a, b, d in self.terms:
            X, Y, Z = (self._pw(s[:, 0], a, 0), self._pw(s[:, 1], b, 0), self._pw(s[:, 2], d, 0))
            g[:, 0] += c * self._pw(s[:, 0], a, 1) * self.sc[0] * Y * Z
            g[:, 1] += c * X * self._pw(s[:, 1], b, 1) * self.sc[1] * Z
            g[:, 2] += c * X * Y * self._pw(s[:, 2], d, 1) * self.sc[2]
        return g

    def laplacian(self, xyz):
        s = self._s(xyz)
        out = np.zeros(len(xyz))
        for c, a, b, d in self.terms:
            X, Y, Z = (self._pw(s[:, 0], a, 0), self._pw(s[:, 1], b, 0), self._pw(s[:, 2], d, 0))
            out += c * (self._pw(s[:, 0], a, 2) * self.sc[0] ** 2 * Y * Z
                        + X * self._pw(s[:, 1], b, 2) * self.sc[1] ** 2 * Z
                        + X * Y * self._pw(s[:, 2], d, 2) * self.sc[2] ** 2)
        return out


HARMONIC = [
    ("x", lambda x, y, z: x, lambda x, y, z: (np.ones_like(x), 0 * x, 0 * x)),
    ("xy", lambda x, y, z: x * y, lambda x, y, z: (y, x, 0 * x)),
    ("x2-y2", lambda x, y, z: x * x - y * y, lambda x, y, z: (2 * x, -2 * y, 0 * x)),
    ("xyz", lambda x, y, z: x * y * z, lambda x, y, z: (y * z, x * z, x * y)),
    ("x3-3xy2", lambda x, y, z: x ** 3 - 3 * x * y * y, lambda x, y, z: (3 * x * x - 3 * y * y, -6 * x * y, 0 * x)),
    ("y2z-z3/3", lambda x, y, z: y * y * z - z ** 3 / 3, lambda x, y, z: (0 * x, 2 * y * z, y * y - z * z)),
    ("x2+y2-2z2", lambda x, y, z: x * x + y * y - 2 * z * z, lambda x, y, z: (2 * x, 2 * y, -4 * z)),
]
