"""Seeded workloads for the parity tests, built from ``hps_inputs``.

Each side computes node coordinates with its own routine (the oracle's
``node_coords`` or the library's ``hps_leaf_nodes``) and evaluates the same
seeded field there, so the two sides never exchange arrays.
"""
from __future__ import annotations

import numpy as np

import hps_inputs as hi


def box_b(node_fn, p, lows, h, field):
    """b [nbox, p^3] of a field evaluated at each box's nodes."""
    return np.stack([field(node_fn(p, lo, h)) for lo in lows])


def config_grid(name):
    """(p, h[3], kappa, lows [nbox,3], field) of a named workload."""
    if name == "manufactured":          # 2x2x2, p = 8, b = 1
        lows, h = hi.box_grid_lo((2, 2, 2))
        return 8, h, 10.0, lows, lambda x: np.ones(len(x))
    if name == "dip":                   # 8x8x8, p = 12, kappa = 20
        lows, h = hi.box_grid_lo((8, 8, 8))
        return 12, h, 20.0, lows, hi.gaussian_dip_b
    if name == "fourier16":             # 8x8x8, p = 16, kappa = 40
        lows, h = hi.box_grid_lo((8, 8, 8))
        return 16, h, 40.0, lows, hi.fourier_b_field().b
    raise KeyError(name)


def rel_fro(a, b):
    """Per-box relative Frobenius error ||a - b|| / ||b|| over the last two axes."""
    a = np.asarray(a)
    b = np.asarray(b)
    ax = tuple(range(1, a.ndim))
    return np.sqrt(((a - b) ** 2).sum(axis=ax)) / np.sqrt((b ** 2).sum(axis=ax))


def max_rel(a, b):
    """Largest per-box element-wise error relative to the box's largest entry,
    max |a - b| / max |b| over the last axes: it catches a single wrong entry
    that the Frobenius norm would average away."""
    a = np.asarray(a)
    b = np.asarray(b)
    ax = tuple(range(1, a.ndim))
    return float((np.abs(a - b).max(axis=ax) / np.abs(b).max(axis=ax)).max())
