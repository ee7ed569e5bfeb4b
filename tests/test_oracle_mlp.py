"""Pins of the FP64 surrogate-MLP oracle: GELU derivatives, forward-mode input tangents and the
hand-written gradient of the Sobolev loss, each against central finite differences."""
import numpy as np
import pytest

from oracle import mlp

SIZES = [7, 12, 12, 2]


def test_gelu_derivatives_fd():
    x = np.linspace(-4, 4, 41)
    h = 1e-5
    np.testing.assert_allclose(mlp.gelu_d1(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-9)
    np.testing.assert_allclose(mlp.gelu_d2(x), (mlp.gelu_d1(x + h) - mlp.gelu_d1(x - h)) / (2 * h), atol=1e-9)
    assert mlp.gelu(0.0) == 0.0 and mlp.gelu_d1(0.0) == pytest.approx(0.5)
    assert mlp.gelu(30.0) == pytest.approx(30.0) and mlp.gelu(-30.0) == pytest.approx(0.0, abs=1e-12)


def test_forward_tangents_match_fd():
    params = mlp.init_params(SIZES, 3)
    x = np.random.default_rng(4).uniform(-1, 1, size=(5, 7))
    y, dy, _ = mlp.forward(params, x)
    h = 1e-6
    for k in range(7):
        xp, xm = x.copy(), x.copy()
        xp[:, k] += h
        xm[:, k] -= h
        fd = (mlp.forward(params, xp)[0] - mlp.forward(params, xm)[0]) / (2 * h)
        np.testing.assert_allclose(dy[:, :, k], fd, rtol=1e-6, atol=1e-9)


def test_sobolev_gradient_matches_fd():
    params = mlp.init_params(SIZES, 5)
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, size=(6, 7))
    t = rng.standard_normal((6, 2))
    dt = rng.standard_normal((6, 2, 7))
    lam = 0.3
    L, grads = mlp.loss_and_grad(params, x, t, dt, lam)
    assert L == pytest.approx(mlp.sobolev_loss(*mlp.forward(params, x)[:2], t, dt, lam), rel=1e-14)
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for (i, j) in [(0, 0), (1, 3), (W.shape[0] - 1, W.shape[1] - 1)]:
            Wp = [(w.copy(), bb.copy()) for (w, bb) in params]
            Wm = [(w.copy(), bb.copy()) for (w, bb) in params]
            Wp[l][0][i, j] += h
            Wm[l][0][i, j] -= h
            fd = (mlp.loss_and_grad(Wp, x, t, dt, lam)[0] - mlp.loss_and_grad(Wm, x, t, dt, lam)[0]) / (2 * h)
            assert grads[l][0][i, j] == pytest.approx(fd, rel=1e-6, abs=1e-9), (l, i, j)
        for i in [0, b.size - 1]:
            Wp = [(w.copy(), bb.copy()) for (w, bb) in params]
            Wm = [(w.copy(), bb.copy()) for (w, bb) in params]
            Wp[l][1][i] += h
            Wm[l][1][i] -= h
            fd = (mlp.loss_and_grad(Wp, x, t, dt, lam)[0] - mlp.loss_and_grad(Wm, x, t, dt, lam)[0]) / (2 * h)
            assert grads[l][1][i] == pytest.approx(fd, rel=1e-6, abs=1e-9), (l, i)
