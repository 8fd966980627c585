"""Pins for the FP64 oracle of the learned correction's network: BF16
rounding against hand-computed values, and the backward pass against
central finite differences."""
from __future__ import annotations

import numpy as np

from oracle import mlp


def test_bf16_round_to_nearest_even():
    ulp = 2.0 ** -7                                 # BF16 spacing at 1 (7 stored mantissa bits)
    vals = np.array([1.0, 1 + ulp / 2, 1 + 3 * ulp / 4, 1 + ulp + ulp / 2, -2.5, 3.140625])
    want = np.array([1.0, 1.0, 1 + ulp, 1 + 2 * ulp, -2.5, 3.140625])
    np.testing.assert_array_equal(mlp.bf16_round(vals), want)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    dims = [7, 6, 5, 2 * 4 * 2]
    m, r, B = 4, 2, 3
    n = sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(3))
    theta = rng.standard_normal(n) * 0.5
    b = 1 + 0.3 * rng.standard_normal((B, dims[0]))
    dT = rng.standard_normal((B, m, m))
    L, g = mlp.loss_and_grad(theta, dims, m, r, b, dT, 0.7, bf16=False)
    eps = 1e-6
    for i in rng.choice(n, size=40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (mlp.loss_and_grad(tp, dims, m, r, b, dT, 0.7, bf16=False)[0]
              - mlp.loss_and_grad(tm, dims, m, r, b, dT, 0.7, bf16=False)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])
