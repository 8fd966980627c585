"""Seeded synthetic inputs shared by the oracle and the CUDA library's tests.

This module holds none of the method's arithmetic: it draws random fields and
evaluates them at coordinates the caller supplies (each side computes its own
node coordinates).  Every law is seeded through numpy's PCG64, so both sides
receive bit-identical coefficient tables.

Workloads (shaped like the paper's Sec. 4 experiments, which use analytic
data; no dataset is involved):

* ``manufactured``: u = sin(pi x) sin(2 pi y) sin(pi z) on the unit cube with
  b = 1, so f = (6 pi^2 - kappa^2) u and g = 0 on the boundary.
* ``gaussian_dip_b``: b = 1 - 0.5 exp(-|x - c|^2 / 0.04), c = (0.5, 0.5, 0.5).
* ``green``: the accuracy study of Sec. 4.1 on the box GREEN_LO + [0, GREEN_L]
  = [-1.1, 0.1] x [1, 2] x [1.2, 2.2]: u = cos(kappa |x|) / (4 pi |x|), the
  free-space Green's function of Lap u + kappa^2 u (kappa = 0: Poisson), used
  as the exact solution and its boundary values as g (b = 1, f = 0).
* ``curved``: the curved domain of Sec. 4.3, {(x1, x2 / psi(x1), x3)} with
  psi(z) = 1 - sin(6 z) / 4 over the reference box CURVED_LO + [0, CURVED_L]
  = [1.1, 2.1] x [-1, 0] x [-1.2, 0.2]: the coefficients of the Helmholtz
  operator pulled back to the reference box (``curved_coefficients``), the
  map to physical coordinates (``curved_to_physical``) and a plane wave
  sin(k . y) of the physical coordinates as an exact solution with
  kappa = |k| (``curved_plane_wave``).
* ``cross_field``: a smooth symmetric positive-definite coefficient tensor
  with every cross term, plus first-order coefficients, for parity tests of
  the cross-term leaves.
* ``FourierField``: 1 + 0.5 sum_{q=1}^{16} a_q cos(2 pi k_q . x + phi_q), with
  k_q uniform over the nonzero integer vectors of length <= 4,
  a_q ~ N(0, 1/16), phi_q ~ U[0, 2 pi); clipped to [0.5, 1.5] for b, and
  unclipped (mean 0) for body loads.
"""
from __future__ import annotations

import math

import numpy as np

SEED_MIXED = 20250304      # p = 16 mixed-precision workload
SEED_UNEVEN = 20250305     # uneven batch (mixed p, kappa, 32 loads)
SEED_TRAIN = 1             # learned-surrogate training boxes
SEED_HELDOUT = 2           # learned-surrogate held-out boxes


def box_grid_lo(nb, L=(1.0, 1.0, 1.0), lo=(0.0, 0.0, 0.0)):
    """Lower corners [nbox, 3] and box size h[3] of a uniform nx x ny x nz grid,
    box index bx + nx (by + ny bz)."""
    nx, ny, nz = (int(v) for v in nb)
    h = np.asarray(L, dtype=np.float64) / np.array([nx, ny, nz], dtype=np.float64)
    bz, by, bx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = np.stack([bx.reshape(-1), by.reshape(-1), bz.reshape(-1)], axis=1).astype(np.float64)
    return np.asarray(lo, dtype=np.float64) + idx * h, h


def manufactured(xyz: np.ndarray, kappa: float):
    """(u, f, g) of the manufactured solution at coordinates [..., 3]."""
    x, y, z = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    u = np.sin(math.pi * x) * np.sin(2 * math.pi * y) * np.sin(math.pi * z)
    f = (6 * math.pi ** 2 - kappa ** 2) * u
    return u, f, u


GREEN_LO = (-1.1, 1.0, 1.2)
GREEN_L = (1.2, 1.0, 1.0)


def green(xyz: np.ndarray, kappa: float) -> np.ndarray:
    """cos(kappa |x|) / (4 pi |x|) at coordinates [..., 3] (the origin lies
    outside the Sec. 4.1 domain)."""
    r = np.sqrt((xyz ** 2).sum(axis=-1))
    return np.cos(kappa * r) / (4.0 * math.pi * r)


def gaussian_dip_b(xyz: np.ndarray) -> np.ndarray:
    r2 = ((xyz - 0.5) ** 2).sum(axis=-1)
    return 1.0 - 0.5 * np.exp(-r2 / 0.04)


def _integer_wavevectors(kmax: float) -> np.ndarray:
    r = int(math.floor(kmax))
    g = np.arange(-r, r + 1)
    kx, ky, kz = np.meshgrid(g, g, g, indexing="ij")
    k = np.stack([kx.reshape(-1), ky.reshape(-1), kz.reshape(-1)], axis=1)
    n2 = (k ** 2).sum(axis=1)
    return k[(n2 > 0) & (n2 <= kmax * kmax)]


class FourierField:
    """One draw of the smooth random field law (see module docstring)."""

    def __init__(self, rng: np.random.Generator, n_modes: int = 16, kmax: float = 4.0):
        ks = _integer_wavevectors(kmax)
        self.k = ks[rng.integers(0, len(ks), size=n_modes)].astype(np.float64)
        self.a = rng.normal(0.0, 0.25, size=n_modes)
        self.phi = rng.uniform(0.0, 2 * math.pi, size=n_modes)

    def sum(self, xyz: np.ndarray) -> np.ndarray:
        ph = 2 * math.pi * (xyz @ self.k.T) + self.phi
        return (np.cos(ph) * self.a).sum(axis=-1)

    def b(self, xyz: np.ndarray) -> np.ndarray:
        return np.clip(1.0 + 0.5 * self.sum(xyz), 0.5, 1.5)


def fourier_b_field(seed: int = SEED_MIXED) -> FourierField:
    """The single global b field of the p = 16 workload (one draw, seed fixed)."""
    return FourierField(np.random.default_rng(seed))


def fourier_b_per_box(nbox: int, seed: int) -> list:
    """Independent b fields, one per box (the learned-surrogate data sets)."""
    rng = np.random.default_rng(seed)
    return [FourierField(rng) for _ in range(nbox)]


def uneven_batch(nbox: int = 1024, seed: int = SEED_UNEVEN, nloads: int = 32,
                 ps=(8, 12, 16, 20), kappas=(10.0, 20.0, 40.0, 60.0)):
    """Draws for the uneven batch: per box p, kappa, a b field and `nloads`
    load fields.  Boxes have h = 1/8 and sit at seeded cells of the unit cube."""
    rng = np.random.default_rng(seed)
    p = rng.choice(np.asarray(ps), size=nbox)
    kappa = rng.choice(np.asarray(kappas, dtype=np.float64), size=nbox)
    cell = rng.integers(0, 8, size=(nbox, 3)).astype(np.float64)
    bfield = FourierField(rng)
    loads = [FourierField(rng) for _ in range(nloads)]
    return {"p": p, "kappa": kappa, "lo": cell / 8.0, "h": np.full(3, 1.0 / 8.0),
            "b_field": bfield, "loads": loads}


def load_values(loads, xyz: np.ndarray) -> np.ndarray:
    """[nloads, N] values of the load fields at coordinates [N, 3]."""
    return np.stack([L.sum(xyz) for L in loads])


def random_boundary_data(nbox: int, nrhs: int, m: int, seed: int = 7) -> np.ndarray:
    """Seeded boundary traces u_b [nbox, nrhs, m] for reconstruction tests."""
    return np.random.default_rng(seed).standard_normal((nbox, nrhs, m))


# ------------------------------------------------------------ operators with cross terms

CURVED_LO = (1.1, -1.0, -1.2)
CURVED_L = (1.0, 1.0, 1.4)
CURVED_K = (1.0, 2.0, -0.5)


def curved_psi(z):
    """psi(z) = 1 - sin(6 z) / 4 and its first two derivatives."""
    return 1.0 - 0.25 * np.sin(6.0 * z), -1.5 * np.cos(6.0 * z), 9.0 * np.sin(6.0 * z)


def curved_to_physical(x: np.ndarray) -> np.ndarray:
    """Reference point (x1, x2, x3) -> physical point (x1, x2 / psi(x1), x3)."""
    ps, _, _ = curved_psi(x[:, 0])
    return np.stack([x[:, 0], x[:, 1] / ps, x[:, 2]], axis=1)


def curved_coefficients(x: np.ndarray):
    """(C [6, N], d [3, N]) of -Lap u - kappa^2 u on the curved domain in the
    reference coordinates, in the form -sum C_ab u_ab + sum d_a u_a: the
    parameter map of Sec. 4.3, -u_11 - ((psi' x2 / psi)^2 + psi^2) u_22 - u_33
    - 2 (psi' x2 / psi) u_12 - (psi'' x2 / psi) u_2 (its "psi(x_i)" read as
    psi(x1)).  C = (C11, C22, C33, C12, C13, C23)."""
    x1, x2 = x[:, 0], x[:, 1]
    ps, dps, ddps = curved_psi(x1)
    r = dps * x2 / ps
    one, zero = np.ones(len(x)), np.zeros(len(x))
    return np.stack([one, r * r + ps * ps, one, r, zero, zero]), np.stack([zero, -ddps * x2 / ps, zero])


def curved_plane_wave(x: np.ndarray, k=CURVED_K) -> np.ndarray:
    """sin(k . y) at the physical points y of reference points x: a solution
    of -Lap u - |k|^2 u = 0."""
    return np.sin(curved_to_physical(x) @ np.asarray(k, dtype=np.float64))


def cross_field(x: np.ndarray):
    """(C [6, N], d [3, N], b [N]): a smooth SPD coefficient tensor with all
    three cross terms, smooth first-order coefficients and b."""
    C = np.stack([1.0 + 0.2 * np.sin(x[:, 0]), 1.3 + 0.1 * x[:, 1], 0.9 + 0.05 * x[:, 2] ** 2,
                  0.25 * np.cos(x[:, 2]), -0.15 + 0.05 * x[:, 0], 0.1 * np.sin(x[:, 1])])
    d = np.stack([0.2 * x[:, 1], np.sin(x[:, 0]), 0.1 * np.ones(len(x))])
    b = 1.0 + 0.2 * np.cos(x[:, 0])
    return C, d, b
