"""Pins for the cost-model oracle (oracle/mlp.py): BF16 rounding against known values, and
the analytic gradient of the plain FP64 network against central finite differences."""
import numpy as np

from oracle import mlp


def test_bf16_rounding_known_values():
    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1.0 + 2.0 ** -9) == 1.0                     # below half an ulp (2^-8)
    assert mlp.bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7     # above half: rounds up
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0                     # tie: to even
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6     # tie: to even (up)
    assert mlp.bf16(-2.5) == -2.5 and mlp.bf16(0.0) == 0.0


def test_parameter_count():
    assert mlp.NPARAM == 1313


def test_gradient_matches_finite_differences():
    g = np.random.default_rng(0)
    p = g.normal(0, 0.3, mlp.NPARAM)
    x = g.normal(0, 1, (40, 6))
    t = g.normal(0, 1, 40)
    loss, grad = mlp.loss_and_grad(p, x, t, bf16_storage=False)
    idx = g.choice(mlp.NPARAM, 60, replace=False)
    h = 1e-6
    for k in idx:
        dp = np.zeros_like(p)
        dp[k] = h
        lp, _ = mlp.loss_and_grad(p + dp, x, t, bf16_storage=False)
        lm, _ = mlp.loss_and_grad(p - dp, x, t, bf16_storage=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, grad[k])
