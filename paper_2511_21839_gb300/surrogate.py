"""Learned surrogate of the dual PIC and the design search it warm-starts.

The dual PIC gives the final emittances and their exact derivatives with
respect to the seven lattice parameters in one run (Sec. 4). A batch of such
runs at perturbed lattices is the training set of a small MLP fitted with a
Sobolev loss on values and derivatives (csrc/mlp.cu). The surrogate then
warm-starts the variable-metric (BFGS) search for lattice parameters that
give target emittances (Sec. 3 uses BFGS with AD gradients for matching).
Each outer step minimises, by BFGS, the objective of the surrogate shifted
to agree with the dual PIC in value and gradient at the current point (the
exact derivatives make this first-order correction possible), inside a trust
region; the proposed point is then checked by a full dual-PIC run and kept
only if it improves the objective. When the proposals stop improving, BFGS
continues on dual-PIC gradients alone, so the PIC stays both the arbiter of the
surrogate's error and the fallback.

Coordinates: x = (p / p_nominal - 1) / rel in [-1, 1]^7; outputs
y = eps / eps_nominal; dy/dx = (d eps / d p) rel p_nominal / eps_nominal.
"""
import math

import numpy as np

from . import adpic
from . import inputs as I

REL = 0.2


def to_params(x, p_nom, rel=REL):
    return np.asarray(p_nom) * (1.0 + rel * np.asarray(x))


def to_x(p, p_nom, rel=REL):
    return (np.asarray(p) / np.asarray(p_nom) - 1.0) / rel


class Problem:
    """One configuration of the dual PIC (the single-period FODO run by default) at any lattice."""

    def __init__(self, n_particles=10_000, grid=32, seed=1, precision=adpic.AD_PIC_FP32_MIXED, kicks=20):
        self.N = n_particles
        self.grid = (grid, grid, grid)
        self.precision = precision
        self.kicks = kicks
        self.beam = I.workload("fodo_10k_32").beam
        self.normals = I.normals(seed, n_particles)
        self.p_nom = np.array(I.Lattice().params(), dtype=np.float64)
        self.sim = None
        self._last = None
        self.evaluations = 0
        self.eps_nom = self._eps(self.p_nom)[0]
        self.evaluations = 0

    def _eps(self, p):
        if self.sim is None:
            self.sim = adpic.ADPIC(self.grid, self.N, 7, self.precision)
        self.sim.set_beam(self.beam, self.normals)
        self.sim.set_lattice(I.Lattice.from_params(p))
        self.sim.run(self.kicks)
        self.evaluations += 1
        return self.sim.moments()

    def evaluate(self, x):
        """Normalised emittances y [2] and dy/dx [2][7] at normalised parameters x (one dual-PIC run;
        a repeat of the last point is answered from memory and not counted)."""
        x = np.asarray(x, dtype=np.float64)
        if self._last is not None and np.array_equal(self._last[0], x):
            return self._last[1].copy(), self._last[2].copy()
        p = to_params(x, self.p_nom)
        v, d = self._eps(p)
        y = v / self.eps_nom
        dy = d * (REL * self.p_nom)[None, :] / self.eps_nom[:, None]
        self._last = (x.copy(), y.copy(), dy.copy())
        return y, dy

    def close(self):
        if self.sim is not None:
            self.sim.close()
            self.sim = None


def generate_dataset(problem, n_runs, seed=5, chunk=512):
    """n_runs dual-PIC runs at parameters x ~ U(-1, 1)^7 (p within +-20 %), on the batched runtime."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, size=(n_runs, 7))
    Y = np.zeros((n_runs, 2))
    dY = np.zeros((n_runs, 2, 7))
    for c0 in range(0, n_runs, chunk):
        c1 = min(n_runs, c0 + chunk)
        b = adpic.Batch([problem.grid] * (c1 - c0), [problem.N] * (c1 - c0), precision=adpic.AD_PIC_FP32_MIXED)
        for i in range(c1 - c0):
            b.set_beam(i, problem.beam, problem.normals)
            b.set_lattice(i, I.Lattice.from_params(to_params(X[c0 + i], problem.p_nom)))
        b.run(problem.kicks)
        for i in range(c1 - c0):
            v, d = b.moments(i)
            Y[c0 + i] = v / problem.eps_nom
            dY[c0 + i] = d * (REL * problem.p_nom)[None, :] / problem.eps_nom[:, None]
        b.close()
    return X, Y, dY


class Surrogate:
    """MLP n_in -> width (x hidden, GELU) -> n_out trained with the Sobolev loss on (X, Y, dY); the
    FODO problem's network is 7 -> 256 -> 256 -> 256 -> 2.

    The network fits (y - y_shift) / y_scale per output; derivatives are scaled alike."""

    def __init__(self, width=256, hidden=3, max_batch=512, seed=0, n_in=7, n_out=2):
        self.n_in, self.n_out = n_in, n_out
        self.m = adpic.ad_pic_mlp_create(n_in, width, hidden, n_out, max_batch)
        self.n_params = adpic.ad_pic_mlp_num_params(self.m)
        self.max_batch = max_batch
        self.sizes = [n_in] + [width] * hidden + [n_out]
        rng = np.random.default_rng(seed)
        parts = []
        for l in range(len(self.sizes) - 1):
            n_in, n_out = self.sizes[l], self.sizes[l + 1]
            scale = math.sqrt((1.0 if l == len(self.sizes) - 2 else 2.0) / n_in)
            parts += [rng.standard_normal(n_in * n_out) * scale, np.zeros(n_out)]
        adpic.ad_pic_mlp_set_params(self.m, np.concatenate(parts))
        self.y_shift = np.zeros(n_out)
        self.y_scale = np.ones(n_out)

    def fit(self, X, Y, dY, steps=3000, lam=1.0, lr=2e-3, lr_final=2e-5, seed=0, device=True, epochs_in_order=8):
        """Adam on mini-batches of max_batch samples, learning rate decayed geometrically from lr to
        lr_final. device=True: the training set goes to the device once, as `epochs_in_order`
        shuffled passes one after the other, and every step is a graph replay on the device
        (ad_pic_mlp_train); returns (final loss, ms of the steps). device=False: one host call per
        step with a fresh random mini-batch (ad_pic_mlp_adam_step); returns the loss of every step."""
        self.y_shift = Y.mean(axis=0)
        self.y_scale = Y.std(axis=0) + 1e-12
        T = (Y - self.y_shift) / self.y_scale
        dT = dY / self.y_scale[None, :, None]
        rng = np.random.default_rng(seed)
        n = X.shape[0]
        B = min(self.max_batch, n)
        if device:
            order = np.concatenate([rng.permutation(n) for _ in range(epochs_in_order)])
            adpic.ad_pic_mlp_set_dataset(self.m, X[order], T[order], dT[order])
            return adpic.ad_pic_mlp_train(self.m, steps, B, lam, lr, lr_final)
        decay = (lr_final / lr) ** (1.0 / max(steps - 1, 1))
        hist = np.zeros(steps)
        for s in range(steps):
            idx = rng.choice(n, size=B, replace=False)
            hist[s] = adpic.ad_pic_mlp_adam_step(self.m, X[idx], T[idx], dT[idx], lam, lr * decay ** s)
        return hist

    def predict(self, X):
        """Surrogate values [B][n_out] and derivatives [B][n_out][n_in] in the problem's normalised units."""
        X = np.atleast_2d(X)
        ys, dys = [], []
        for c0 in range(0, X.shape[0], self.max_batch):
            y, dy = adpic.ad_pic_mlp_forward(self.m, X[c0:c0 + self.max_batch], self.n_out)
            ys.append(y.astype(np.float64) * self.y_scale + self.y_shift)
            dys.append(dy.astype(np.float64) * self.y_scale[None, :, None])
        return np.concatenate(ys), np.concatenate(dys)

    def errors(self, X, Y, dY):
        """Relative rms errors of values (against the spread of Y) and of derivatives."""
        y, dy = self.predict(X)
        return (float(np.sqrt(np.mean((y - Y) ** 2)) / np.sqrt(np.mean((Y - Y.mean(0)) ** 2))),
                float(np.sqrt(np.mean((dy - dY) ** 2)) / np.sqrt(np.mean(dY ** 2))))

    def close(self):
        if self.m:
            adpic.ad_pic_mlp_destroy(self.m)
            self.m = None


def objective(y, dy, target, scale=1.0):
    """f = sum_o ((y_o - target_o) / scale_o)^2 and its gradient in x."""
    s = np.broadcast_to(np.asarray(scale, dtype=np.float64), np.shape(target))
    r = (np.asarray(y) - target) / s
    return float(np.sum(r * r)), 2.0 * (r / s) @ dy


def bfgs(fg, x0, lo, hi, max_iter=50, ftol=0.0, gtol=1e-14, max_evals=None, first_step=0.1):
    """Projected BFGS inside the box [lo, hi]: inverse-Hessian update of the variable-metric method,
    initial inverse Hessian rescaled by s.y / y.y after the first step, backtracking Armijo line
    search along the projected step; a failed line search restarts from the steepest-descent step
    once before giving up. fg(x) -> (f, g). Returns (x, f, calls to fg)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    x = np.clip(np.asarray(x0, dtype=np.float64), lo, hi)
    f, g = fg(x)
    calls = 1
    n = x.size
    Hinv = None
    for _ in range(max_iter):
        if f <= ftol or np.linalg.norm(g) <= gtol:
            break
        if Hinv is None:
            d = -g * (first_step / max(np.abs(g).max(), 1e-300))
        else:
            d = -Hinv @ g
            if d @ g >= 0:
                Hinv = None
                d = -g * (first_step / max(np.abs(g).max(), 1e-300))
        t = 1.0
        accepted = False
        while max_evals is None or calls < max_evals:
            xn = np.clip(x + t * d, lo, hi)
            s = xn - x
            if not np.any(s):
                break
            fn, gn = fg(xn)
            calls += 1
            if fn <= f + 1e-4 * (g @ s):
                accepted = True
                break
            t *= 0.5
            if t < 1e-6:
                break
        if not accepted:
            if Hinv is None:
                break
            Hinv = None             # restart once from the scaled steepest-descent step
            continue
        yv = gn - g
        sy = s @ yv
        if sy > 1e-300:
            if Hinv is None:
                Hinv = np.eye(n) * (sy / (yv @ yv))
            rho = 1.0 / sy
            V = np.eye(n) - rho * np.outer(s, yv)
            Hinv = V @ Hinv @ V.T + rho * np.outer(s, s)
        x, f, g = xn, fn, gn
    return x, f, calls


def search_cold(problem, target, x0, ftol, max_evals=60, scale=1.0):
    """BFGS on dual-PIC values and gradients alone. Returns (x, f, dual-PIC evaluations)."""
    problem.evaluations = 0

    def fg(x):
        return objective(*problem.evaluate(x), target, scale)

    n = np.size(x0)
    x, f, _ = bfgs(fg, x0, -np.ones(n), np.ones(n), max_iter=max_evals, ftol=ftol, max_evals=max_evals)
    return x, f, problem.evaluations


def search_warm(problem, surrogate, target, x0, ftol, max_evals=60, radius=0.5, scale=1.0):
    """Surrogate-warm-started search (see the module docstring). Returns (x, f, dual-PIC evaluations)."""
    problem.evaluations = 0
    x = np.clip(np.asarray(x0, dtype=np.float64), -1.0, 1.0)
    y, dy = problem.evaluate(x)
    f = objective(y, dy, target, scale)[0]
    while f > ftol and problem.evaluations < max_evals and radius > 1e-4:
        ys, dys = surrogate.predict(x)
        c0, c1, xc = y - ys[0], dy - dys[0], x.copy()

        def fg_s(z):
            yz, dyz = surrogate.predict(z)
            return objective(yz[0] + c0 + c1 @ (z - xc), dyz[0] + c1, target, scale)

        lo, hi = np.maximum(-1.0, x - radius), np.minimum(1.0, x + radius)
        z, _, _ = bfgs(fg_s, x, lo, hi, max_iter=200, ftol=ftol * 1e-4)
        yz, dyz = problem.evaluate(z)                 # the full dual PIC checks every proposal
        fz = objective(yz, dyz, target, scale)[0]
        if fz < f:
            x, y, dy, f = z, yz, dyz, fz
            radius = min(1.0, 2.0 * radius)
        else:
            radius *= 0.25
    if f > ftol and problem.evaluations < max_evals:
        used = problem.evaluations

        def fg(xp):
            return objective(*problem.evaluate(xp), target, scale)

        n = x.size
        x, f, _ = bfgs(fg, x, -np.ones(n), np.ones(n), max_iter=max_evals, ftol=ftol,
                       max_evals=max_evals - used)
    return x, f, problem.evaluations
