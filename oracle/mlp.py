"""Plain FP64 numpy oracle of the surrogate MLP (test infrastructure only).

The network maps the 7 normalised lattice parameters to the 2 normalised
final emittances: L dense layers with GELU (x Phi(x)) between them and a
linear output layer. Besides the values it propagates, in forward mode, the
input tangents (the 7 derivatives of every activation with respect to the
inputs), so the Sobolev loss

    L = 1/B sum_b [ sum_o (y_bo - t_bo)^2 + lam sum_o sum_k (dy_bok - dt_bok)^2 ]

can fit the values and the exact dual-PIC derivatives together. The gradient
of L with respect to every weight and bias is written out by hand (reverse
mode through the primal and tangent paths; the tangent path depends on the
primal pre-activations through GELU'(h), which brings in GELU''(h)).
"""
import math

import numpy as np


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_d1(x):
    """d/dx [x Phi(x)] = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * _phi(x)


def gelu_d2(x):
    """d^2/dx^2 [x Phi(x)] = phi(x) (2 - x^2)."""
    return _phi(x) * (2.0 - x * x)


def _phi(x):
    return np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def _erf(x):
    from scipy.special import erf
    return erf(x)


def init_params(sizes, seed):
    """He-style initialisation: W_l [n_out][n_in] ~ N(0, 2/n_in) (1/n_in for the last layer), b = 0."""
    rng = np.random.default_rng(seed)
    params = []
    for l in range(len(sizes) - 1):
        n_in, n_out = sizes[l], sizes[l + 1]
        scale = math.sqrt((1.0 if l == len(sizes) - 2 else 2.0) / n_in)
        params.append((rng.standard_normal((n_out, n_in)) * scale, np.zeros(n_out)))
    return params


def forward(params, x):
    """x [B][n_in] -> y [B][n_out], dy [B][n_out][n_in] and the cache for backward."""
    B, n_in = x.shape
    a = x.astype(np.float64)
    ta = np.broadcast_to(np.eye(n_in), (B, n_in, n_in)).transpose(0, 2, 1).copy()   # [B][k][feature]
    cache = []
    for l, (W, b) in enumerate(params):
        h = a @ W.T + b                      # primal pre-activation
        th = ta @ W.T                        # tangents [B][k][out]
        last = l == len(params) - 1
        cache.append((a, ta, h, th))
        if last:
            a, ta = h, th
        else:
            a = gelu(h)
            ta = gelu_d1(h)[:, None, :] * th
    y = a
    dy = ta.transpose(0, 2, 1)               # [B][out][k]
    return y, dy, cache


def sobolev_loss(y, dy, t, dt, lam):
    B = y.shape[0]
    return (np.sum((y - t) ** 2) + lam * np.sum((dy - dt) ** 2)) / B


def loss_and_grad(params, x, t, dt, lam):
    """Sobolev loss and its gradient [(dW, db) per layer], by hand-written reverse mode."""
    y, dy, cache = forward(params, x)
    B = x.shape[0]
    L = sobolev_loss(y, dy, t, dt, lam)
    g = 2.0 * (y - t) / B                          # dL/dy        [B][out]
    gt = (2.0 * lam * (dy - dt) / B).transpose(0, 2, 1)   # dL/d(tangent of y) [B][k][out]
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        a, ta, h, th = cache[l]
        last = l == len(params) - 1
        if last:
            gh, gth = g, gt
        else:
            d1 = gelu_d1(h)
            d2 = gelu_d2(h)
            # a = gelu(h), ta = gelu'(h) th  =>  dL/dh = g gelu'(h) + sum_k gt_k th_k gelu''(h)
            gh = g * d1 + np.sum(gt * th, axis=1) * d2
            gth = gt * d1[:, None, :]
        dW = gh.T @ a + np.einsum("bko,bki->oi", gth, ta)
        db = gh.sum(axis=0)
        grads[l] = (dW, db)
        g = gh @ W
        gt = gth @ W
    return L, grads
