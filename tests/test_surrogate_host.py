"""Host logic of the surrogate-warm-started design search (no GPU).

The optimiser is pinned on problems with known minima (a convex quadratic, where BFGS with a
sufficiently accurate line search terminates in at most n + few steps, and the Rosenbrock valley).
The warm-started search is run on a synthetic problem with exact derivatives standing in for the
dual PIC, with surrogates of known quality: a perfect one, a biased one, and a useless one (the
search must still reach the target through the dual-PIC fallback, never trusting the surrogate).
"""
import numpy as np
import pytest

from paper_2511_21839_gb300 import surrogate as S


def test_bfgs_quadratic():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((7, 7))
    H = A @ A.T + 0.5 * np.eye(7)
    xs = rng.uniform(-0.5, 0.5, 7)

    def fg(x):
        d = x - xs
        return float(0.5 * d @ H @ d), H @ d

    x, f, calls = S.bfgs(fg, np.zeros(7), -np.ones(7), np.ones(7), max_iter=200, ftol=1e-20)
    assert np.abs(x - xs).max() < 1e-7
    assert f < 1e-14


def test_bfgs_rosenbrock_and_box():
    def fg(x):
        a, b = x
        f = (1 - a) ** 2 + 100 * (b - a * a) ** 2
        return f, np.array([-2 * (1 - a) - 400 * a * (b - a * a), 200 * (b - a * a)])

    x, f, _ = S.bfgs(fg, np.array([-1.2, 1.0]), -2 * np.ones(2), 2 * np.ones(2), max_iter=500, ftol=1e-16)
    assert np.abs(x - 1).max() < 1e-5
    # the box is respected: the minimum of (x - 3)^2 inside [-1, 1] is at the bound
    x, f, _ = S.bfgs(lambda x: (float(np.sum((x - 3) ** 2)), 2 * (x - 3)), np.zeros(3), -np.ones(3), np.ones(3))
    assert np.allclose(x, 1.0)


def test_objective_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    J = rng.standard_normal((2, 7))
    t = np.array([0.3, -0.2])
    scale = np.array([0.5, 2.0])

    def yf(x):
        return np.tanh(J @ x), (1 - np.tanh(J @ x) ** 2)[:, None] * J

    x = rng.uniform(-1, 1, 7)
    f, g = S.objective(*yf(x), t, scale)
    for k in range(7):
        e = np.zeros(7)
        e[k] = 1e-6
        fd = (S.objective(*yf(x + e), t, scale)[0] - S.objective(*yf(x - e), t, scale)[0]) / 2e-6
        assert fd == pytest.approx(g[k], rel=1e-6, abs=1e-9)


class FakeProblem:
    """Two smooth outputs of seven parameters with exact Jacobians (a stand-in for the dual PIC)."""

    def __init__(self, seed=2):
        rng = np.random.default_rng(seed)
        self.J = rng.standard_normal((2, 7)) * 0.3
        self.Q = rng.standard_normal((2, 7, 7)) * 0.05
        self.evaluations = 0

    def exact(self, x):
        Qs = self.Q + self.Q.transpose(0, 2, 1)
        y = self.J @ x + 0.5 * np.einsum("i,oij,j->o", x, Qs, x) + 0.1 * np.sin(2 * x[:2])
        dy = self.J + np.einsum("oij,j->oi", Qs, x)
        dy[0, 0] += 0.2 * np.cos(2 * x[0])
        dy[1, 1] += 0.2 * np.cos(2 * x[1])
        return y, dy

    def evaluate(self, x):
        self.evaluations += 1
        return self.exact(np.asarray(x, dtype=np.float64))


class FakeSurrogate:
    def __init__(self, fn):
        self.fn = fn

    def predict(self, X):
        X = np.atleast_2d(X)
        ys, dys = zip(*(self.fn(x) for x in X))
        return np.array(ys), np.array(dys)


def targets(prob, count=5, seed=3):
    rng = np.random.default_rng(seed)
    return [prob.exact(rng.uniform(-0.7, 0.7, 7))[0] for _ in range(count)]


def test_warm_start_with_exact_surrogate_needs_few_evaluations():
    prob = FakeProblem()
    sur = FakeSurrogate(prob.exact)
    for t in targets(prob):
        x, f, n = S.search_warm(prob, sur, t, np.zeros(7), ftol=1e-12)
        assert f < 1e-12
        assert n <= 3


def test_warm_start_beats_cold_with_a_biased_surrogate():
    prob = FakeProblem()
    rng = np.random.default_rng(4)
    B = rng.standard_normal((2, 7)) * 0.05

    def biased(x):
        y, dy = prob.exact(x)
        return y + 0.03 * np.cos(B @ x * 10), dy - 0.3 * (np.sin(B @ x * 10))[:, None] * B

    sur = FakeSurrogate(biased)
    cold = warm = 0
    for t in targets(prob):
        _, fc, nc = S.search_cold(prob, t, np.zeros(7), ftol=1e-12, max_evals=200)
        _, fw, nw = S.search_warm(prob, sur, t, np.zeros(7), ftol=1e-12, max_evals=200)
        assert fc < 1e-12 and fw < 1e-12
        cold += nc
        warm += nw
    assert warm < cold


def test_useless_surrogate_falls_back_to_the_dual_pic():
    prob = FakeProblem()
    sur = FakeSurrogate(lambda x: (np.array([5.0, -5.0]) + x[:2], np.eye(2, 7)))
    for t in targets(prob, 3):
        x, f, n = S.search_warm(prob, sur, t, np.zeros(7), ftol=1e-12, max_evals=200)
        y, _ = prob.exact(x)
        assert f < 1e-12 and np.abs(y - t).max() < 1e-6
