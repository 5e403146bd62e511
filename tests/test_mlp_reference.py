"""Pins of the FP64 reference network used to check the library's training kernels:
central finite differences of the loss, and the SiLU derivative."""
import numpy as np
import pytest

from oracle import mlp_ref as R


def test_silu_derivative_matches_finite_differences():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    fd = (R.silu(z + h) - R.silu(z - h)) / (2 * h)
    assert np.allclose(R.dsilu(z), fd, rtol=1e-8, atol=1e-10)


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(4)
    theta = R.init_params(1) * 0.5
    theta += 0.01 * rng.standard_normal(theta.size)    # non-zero biases too
    X = rng.standard_normal((6, 16))
    Y = rng.standard_normal((6, 10))
    M = (rng.uniform(size=(6, 10)) > 0.3).astype(float)
    L, g = R.loss_and_grad(theta, X, Y, M)
    idx = rng.choice(theta.size, 60, replace=False)
    # include a few biases of every layer
    offs = np.cumsum([0] + [w[0] * w[1] + b[0] for w, b in R.param_shapes()])
    for l, (w, b) in enumerate(R.param_shapes()):
        idx = np.append(idx, offs[l] + w[0] * w[1] + rng.integers(b[0]))
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (R.loss_and_grad(tp, X, Y, M)[0] - R.loss_and_grad(tm, X, Y, M)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9), k


def test_parameter_count():
    assert R.n_params() == 16 * 128 + 128 + 3 * (128 * 128 + 128) + 128 * 10 + 10
