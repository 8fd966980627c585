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


def test_rounded_operands_stay_within_the_bf16_bound():
    """The variant with BF16 product operands (what the tensor cores compute)
    departs from the unrounded oracle by about the BF16 unit roundoff 2^-9,
    and does depart (the roundings are applied)."""
    rng = np.random.default_rng(3)
    dims = [12, 10, 9, 2 * 6 * 3]
    m, r, B = 6, 3, 4
    n = sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(3))
    theta = rng.standard_normal(n) * 0.4
    b = 1 + 0.3 * rng.standard_normal((B, dims[0]))
    dT = rng.standard_normal((B, m, m))
    L0, g0 = mlp.loss_and_grad(theta, dims, m, r, b, dT, 0.9)
    L1, g1 = mlp.loss_and_grad(theta, dims, m, r, b, dT, 0.9, act_bf16=True)
    u = 2.0 ** -9
    assert 0 < abs(L1 - L0) <= 8 * u * L0
    rel = np.linalg.norm(g1 - g0) / np.linalg.norm(g0)
    assert u / 16 < rel <= 16 * u, rel
    y0 = mlp.forward(theta, dims, m, r, b)
    y1 = mlp.forward(theta, dims, m, r, b, act_bf16=True)
    assert 0 < np.abs(y1 - y0).max() <= 8 * u * np.abs(y0).max()


def test_forward_is_the_loss_paths_forward():
    """forward() gives the y whose factors the loss uses: with dT = 0 and a
    huge scale the loss is mean((U V^T)^2) of forward()'s U, V."""
    rng = np.random.default_rng(4)
    dims = [5, 4, 3, 2 * 3 * 2]
    m, r, B = 3, 2, 2
    n = sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(3))
    theta = rng.standard_normal(n) * 0.5
    b = 1 + 0.3 * rng.standard_normal((B, dims[0]))
    for act in (False, True):
        y = mlp.forward(theta, dims, m, r, b, act_bf16=act)
        q = mlp.bf16_round if act else (lambda v: v)
        U = q(y[:, :m * r]).reshape(B, m, r)
        V = q(y[:, m * r:]).reshape(B, m, r)
        L, _ = mlp.loss_and_grad(theta, dims, m, r, b, np.zeros((B, m, m)), 1.0, act_bf16=act)
        assert abs(L - ((U @ V.transpose(0, 2, 1)) ** 2).mean()) <= 1e-14 * L
