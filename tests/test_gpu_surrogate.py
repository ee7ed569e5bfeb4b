"""Surrogate MLP kernels (BF16 tensor-core GEMMs, FP32 accumulation) against the FP64 numpy oracle.

Tolerances follow from BF16 operands (8 significant bits; relative rounding 2^-9 per operand, a
few 1e-3 after accumulation over 256 terms and three layers): forward values and input tangents
within 3e-2 of their scale, the Sobolev loss within 3e-2 relative, and the gradient vector within
5e-2 relative in norm with a cosine similarity above 0.998.
"""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu

SIZES = [7, 256, 256, 256, 2]


def flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for (W, b) in params]).astype(np.float32)


def unflat(v, sizes):
    out, o = [], 0
    for l in range(len(sizes) - 1):
        n_in, n_out = sizes[l], sizes[l + 1]
        W = v[o:o + n_in * n_out].reshape(n_out, n_in)
        o += n_in * n_out
        b = v[o:o + n_out]
        o += n_out
        out.append((W.astype(np.float64), b.astype(np.float64)))
    return out


@pytest.fixture(scope="module")
def lib():
    from paper_2511_21839_gb300 import adpic, build

    build.build()
    return adpic


def make(lib, seed=1, B=64):
    params = mlp.init_params(SIZES, seed)
    for l, (W, b) in enumerate(params):
        b += np.random.default_rng(seed + 10 + l).standard_normal(b.shape) * 0.1
    m = lib.ad_pic_mlp_create(7, 256, 3, 2, 512)
    n = lib.ad_pic_mlp_num_params(m)
    v = flat(params)
    assert n == v.size
    lib.ad_pic_mlp_set_params(m, v)
    # the oracle sees exactly the FP32 parameters the device holds
    return m, unflat(v, SIZES), n


def test_forward_values_and_tangents(lib):
    m, params, n = make(lib)
    x = np.random.default_rng(2).uniform(-1, 1, size=(64, 7))
    y, dy = lib.ad_pic_mlp_forward(m, x, 2)
    yr, dyr, _ = mlp.forward(params, x.astype(np.float32).astype(np.float64))
    assert np.abs(y - yr).max() < 3e-2 * np.abs(yr).max()
    assert np.abs(dy - dyr).max() < 3e-2 * np.abs(dyr).max()
    lib.ad_pic_mlp_destroy(m)


def test_loss_and_gradient(lib):
    m, params, n = make(lib, seed=3)
    rng = np.random.default_rng(4)
    B = 96
    x = rng.uniform(-1, 1, size=(B, 7))
    t = rng.standard_normal((B, 2))
    dt = rng.standard_normal((B, 2, 7)) * 0.5
    lam = 0.5
    loss, g = lib.ad_pic_mlp_loss_grad(m, x, t, dt, lam, n)
    xr = x.astype(np.float32).astype(np.float64)
    tr = t.astype(np.float32).astype(np.float64)
    dtr = dt.astype(np.float32).astype(np.float64)
    Lr, gr = mlp.loss_and_grad(params, xr, tr, dtr, lam)
    gref = flat([(dW, db) for (dW, db) in gr]).astype(np.float64)
    assert loss == pytest.approx(Lr, rel=3e-2)
    cos = float(np.dot(g, gref) / (np.linalg.norm(g) * np.linalg.norm(gref)))
    rel = float(np.linalg.norm(g - gref) / np.linalg.norm(gref))
    print(f"loss {loss:.6g} vs {Lr:.6g}; gradient cosine {cos:.6f}, relative error {rel:.3e}")
    assert cos > 0.998 and rel < 5e-2
    lib.ad_pic_mlp_destroy(m)


def test_adam_fits_a_smooth_map_with_derivatives(lib):
    """A known smooth map and its exact Jacobian: the Sobolev fit drives both errors down."""
    m, params, n = make(lib, seed=5)
    rng = np.random.default_rng(6)
    A = rng.standard_normal((2, 7)) * 0.4

    def target(x):
        z = x @ A.T
        return np.sin(z) + 0.3 * z ** 2, (np.cos(z) + 0.6 * z)[:, :, None] * A[None, :, :]

    losses = []
    for step in range(400):
        x = rng.uniform(-1, 1, size=(256, 7))
        t, dt = target(x)
        losses.append(lib.ad_pic_mlp_adam_step(m, x, t, dt, 1.0, 1e-3))
    assert np.mean(losses[-20:]) < 0.05 * np.mean(losses[:5])
    x = rng.uniform(-1, 1, size=(128, 7))
    t, dt = target(x)
    y, dy = lib.ad_pic_mlp_forward(m, x, 2)
    assert np.sqrt(np.mean((y - t) ** 2)) < 0.1 * np.sqrt(np.mean(t ** 2))
    assert np.sqrt(np.mean((dy - dt) ** 2)) < 0.2 * np.sqrt(np.mean(dt ** 2))
    lib.ad_pic_mlp_destroy(m)
