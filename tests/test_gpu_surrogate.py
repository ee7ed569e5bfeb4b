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


def blocks(v, sizes):
    """(name, slice) of every weight and bias block of the flat parameter vector."""
    out, o = [], 0
    for l in range(len(sizes) - 1):
        n = sizes[l] * sizes[l + 1]
        out.append((f"W{l}", slice(o, o + n)))
        o += n
        out.append((f"b{l}", slice(o, o + sizes[l + 1])))
        o += sizes[l + 1]
    return out


def test_gradient_element_wise(lib):
    """Every element of the gradient against the FP64 oracle, relative to the largest element of its
    weight or bias block. BF16 operands carry 8 significant bits; the gradient of a weight is a sum
    over the 96 x 8 rows of products of BF16 activations and BF16 output gradients, each relatively
    off by up to 2^-8, and the errors of the layers above add in: 2e-2 of the block's largest element."""
    m, params, n = make(lib, seed=13)
    rng = np.random.default_rng(14)
    B = 96
    x = rng.uniform(-1, 1, size=(B, 7))
    t = rng.standard_normal((B, 2))
    dt = rng.standard_normal((B, 2, 7)) * 0.5
    _, g = lib.ad_pic_mlp_loss_grad(m, x, t, dt, 0.5, n)
    f32 = lambda a: a.astype(np.float32).astype(np.float64)
    _, gr = mlp.loss_and_grad(params, f32(x), f32(t), f32(dt), 0.5)
    gref = flat([(dW, db) for (dW, db) in gr]).astype(np.float64)
    worst = 0.0
    for name, sl in blocks(gref, SIZES):
        err = np.abs(g[sl] - gref[sl]).max() / np.abs(gref[sl]).max()
        print(f"  {name}: max element error {err:.2e} of the block's largest")
        worst = max(worst, err)
        assert err < 2e-2, name
    lib.ad_pic_mlp_destroy(m)


def test_adam_update_matches_a_numpy_step(lib):
    """One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, first step) on the device gradient: the new
    FP32 parameters element-wise against numpy's update of the same parameters with that gradient."""
    m, params, n = make(lib, seed=15)
    rng = np.random.default_rng(16)
    B = 64
    x = rng.uniform(-1, 1, size=(B, 7))
    t = rng.standard_normal((B, 2))
    dt = rng.standard_normal((B, 2, 7)) * 0.5
    p0 = lib.ad_pic_mlp_get_params(m, n).astype(np.float64)
    _, g = lib.ad_pic_mlp_loss_grad(m, x, t, dt, 0.5, n)
    lr = 1e-3
    lib.ad_pic_mlp_adam_step(m, x, t, dt, 0.5, lr)
    p1 = lib.ad_pic_mlp_get_params(m, n).astype(np.float64)
    g = g.astype(np.float64)
    mm = 0.1 * g
    vv = 0.001 * g * g
    ref = p0 - lr * (mm / 0.1) / (np.sqrt(vv / 0.001) + 1e-8)
    np.testing.assert_allclose(p1, ref, rtol=2e-6, atol=2e-9)
    lib.ad_pic_mlp_destroy(m)


def test_device_resident_training_matches_the_host_loop_and_is_faster(lib):
    """The same training problem through ad_pic_mlp_train (dataset on the device, one graph replay
    per step) and through one host call per step: both fit the map, and the device path's step rate
    and tensor throughput are reported (GEMM flops counted: 3 passes of 2 R K N per layer)."""
    rng = np.random.default_rng(17)
    A = rng.standard_normal((2, 7)) * 0.4

    def target(x):
        z = x @ A.T
        return np.sin(z) + 0.3 * z ** 2, (np.cos(z) + 0.6 * z)[:, :, None] * A[None, :, :]

    X = rng.uniform(-1, 1, size=(4096, 7))
    T, dT = target(X)
    steps, B = 300, 512
    m, _, n = make(lib, seed=18)
    lib.ad_pic_mlp_set_dataset(m, X, T, dT)
    lib.ad_pic_mlp_train(m, 5, B, 1.0, 1e-3, 1e-3)            # capture + warm-up
    loss, ms = lib.ad_pic_mlp_train(m, steps, B, 1.0, 1e-3, 1e-4)
    R = B * 8
    flops = 3 * 2 * R * (7 * 256 + 256 * 256 * 2 + 256 * 2)
    print(f"device-resident training: {ms / steps:.3f} ms per step, {flops * steps / (ms * 1e-3) / 1e12:.2f} "
          f"TFLOP/s of GEMM work, final loss {loss:.3e}")
    Xv = rng.uniform(-1, 1, size=(256, 7))
    Tv, dTv = target(Xv)
    y, dy = lib.ad_pic_mlp_forward(m, Xv, 2)
    assert np.sqrt(np.mean((y - Tv) ** 2)) < 0.1 * np.sqrt(np.mean(Tv ** 2))
    assert np.sqrt(np.mean((dy - dTv) ** 2)) < 0.2 * np.sqrt(np.mean(dTv ** 2))
    lib.ad_pic_mlp_destroy(m)
    import time
    m2, _, _ = make(lib, seed=18)
    t0 = time.perf_counter()
    for s_ in range(30):
        idx = rng.choice(4096, size=B, replace=False)
        lib.ad_pic_mlp_adam_step(m2, X[idx], T[idx], dT[idx], 1.0, 1e-3)
    host_ms = 1e3 * (time.perf_counter() - t0) / 30
    print(f"host loop: {host_ms:.3f} ms per step")
    assert ms / steps < host_ms
    lib.ad_pic_mlp_destroy(m2)


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


# ---------------------------------------------------------------- the surrogate workflow

@pytest.fixture(scope="module")
def workflow(lib):
    """4,096 single-period dual-PIC runs of the 10,000-particle, 32^3, P = 7 FODO problem at
    lattice parameters drawn uniformly within +-20 % (seed 5) on the batched runtime; 90 % train
    the network with the Sobolev loss, 10 % are held out."""
    from paper_2511_21839_gb300 import surrogate as S

    prob = S.Problem()
    X, Y, dY = S.generate_dataset(prob, 4096, seed=5)
    ntr = int(0.9 * len(X))
    sur = S.Surrogate()
    sur.fit(X[:ntr], Y[:ntr], dY[:ntr], steps=3000, lam=1.0)
    yield S, prob, (X, Y, dY, ntr), sur
    sur.close()
    prob.close()


def test_dataset_matches_single_runs(workflow):
    """Batched dataset runs reproduce the single-instance dual PIC at the same parameters."""
    S, prob, (X, Y, dY, ntr), sur = workflow
    for i in (0, 1, 4095):
        y, dy = prob.evaluate(X[i])
        assert np.abs(y - Y[i]).max() < 1e-7
        assert np.abs(dy - dY[i]).max() < 1e-4 * np.abs(dY[i]).max()


def test_surrogate_generalises_and_sobolev_loss_helps_derivatives(workflow):
    """Held-out relative rms errors of values and derivatives; training on values alone (lam = 0)
    leaves the derivatives markedly worse."""
    S, prob, (X, Y, dY, ntr), sur = workflow
    ev, ed = sur.errors(X[ntr:], Y[ntr:], dY[ntr:])
    plain = S.Surrogate()
    plain.fit(X[:ntr], Y[:ntr], dY[:ntr], steps=3000, lam=0.0)
    pv, pd = plain.errors(X[ntr:], Y[ntr:], dY[ntr:])
    plain.close()
    print(f"held-out: Sobolev value {ev:.3f} derivative {ed:.3f}; values only: value {pv:.3f} derivative {pd:.3f}")
    assert ev < 0.1 and ed < 0.06
    assert ed < 0.6 * pd


def test_warm_start_needs_fewer_dual_pic_runs(workflow):
    """Target emittances of hidden lattices: the surrogate-warm-started search reaches every target
    (judged by a fresh dual-PIC run) with fewer dual-PIC evaluations in total than BFGS on dual-PIC
    gradients alone, and the surrogate's own optimum, before any correction, is already verified
    close by the PIC. The plain BFGS baseline may stall on the piecewise-smooth CIC response; its
    runs are counted as spent."""
    S, prob, (X, Y, dY, ntr), sur = workflow
    scale = sur.y_scale
    rng = np.random.default_rng(9)
    ftol = 1e-4                                   # residual 1 % of the spread of each emittance
    cold = warm = stalled = 0
    for k in range(8):
        target = prob.evaluate(rng.uniform(-0.8, 0.8, size=7))[0]
        x0 = np.zeros(7)
        f0 = S.objective(*prob.evaluate(x0), target, scale)[0]
        xs, _, _ = S.bfgs(lambda x: S.objective(*(a[0] for a in sur.predict(x)), target, scale), x0,
                          -np.ones(7), np.ones(7), max_iter=200)
        fs = S.objective(*prob.evaluate(xs), target, scale)[0]
        xc, fc, nc = S.search_cold(prob, target, x0, ftol, max_evals=80, scale=scale)
        xw, fw, nw = S.search_warm(prob, sur, target, x0, ftol, max_evals=80, scale=scale)
        print(f"target {k}: f(x0) {f0:.2e}, f(surrogate optimum) {fs:.2e}; cold {nc} runs -> {fc:.1e}, "
              f"warm {nw} runs -> {fw:.1e}")
        assert fs < 0.05 * f0
        # the final point is judged by a fresh dual-PIC run
        assert S.objective(*prob.evaluate(xw), target, scale)[0] < ftol
        cold += nc
        warm += nw
        stalled += fc >= ftol
    print(f"dual-PIC runs over 8 targets: cold {cold} ({stalled} stalled above the target), warm {warm}")
    assert warm < 0.7 * cold
