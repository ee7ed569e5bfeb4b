"""Gradient-based re-matching of the matching section with space charge (Sec. 4).

The four matching quadrupoles between two periodic FODO lattices (the Sec. 3 matching problem) are
re-optimised for an intense beam: every objective evaluation is one dual PIC run of the bunch through
the matching section on the GPU (ad_pic_set_beamline, ad_pic_run), the beam's Twiss functions at the
entrance of the second lattice come from the dual beam moments (beta = <u^2>_c / eps, alpha =
-<u p>_c / eps, centred, with their exact derivatives w.r.t. the four strengths), and Eq. 6 and its
gradient drive the same variable-metric BFGS as the zero-current problem. The zero-current optics
solution (optics.TwissMatch, single-particle dual tracking on the GPU) is the warm start. Host logic
only: every number comes from the library.
"""
import math

import numpy as np

from . import adpic
from . import inputs as I
from . import optics
from .surrogate import Surrogate, bfgs, search_warm

DRIFT, QUAD = 0.3, 0.1
KICKS_DRIFT, KICKS_QUAD = 3, 2


def bunch_charge_for_current(current_A, sigma_z=1e-3, kinetic_eV=1.0e9):
    """Charge of a Gaussian bunch whose peak current Q beta0 c / (sqrt(2 pi) sigma_z) is current_A."""
    _, beta, _ = I.relativistic(kinetic_eV)
    return current_A * math.sqrt(2.0 * math.pi) * sigma_z / (beta * 299792458.0)


def beam_twiss(mom, n_deriv):
    """Dual (beta_x, alpha_x, beta_y, alpha_y) [4][n_deriv + 1] of a moment record [3][5][C]: centred
    second moments a = <u^2>_c, b = <u p>_c, c = <p^2>_c, eps = sqrt(a c - b^2), beta = a / eps,
    alpha = -b / eps (Eqs. 2-4 applied to the Sec. 4 moment definitions)."""
    out = np.zeros((4, n_deriv + 1))
    for pl in range(2):
        m = mom[pl][:, :n_deriv + 1]

        def mul(x, y):
            r = np.empty_like(x)
            r[0] = x[0] * y[0]
            r[1:] = x[0] * y[1:] + y[0] * x[1:]
            return r

        a = m[2] - mul(m[0], m[0])
        b = m[3] - mul(m[0], m[1])
        c = m[4] - mul(m[1], m[1])
        e2 = mul(a, c) - mul(b, b)
        eps = np.empty_like(e2)
        eps[0] = math.sqrt(e2[0])
        eps[1:] = e2[1:] / (2 * eps[0])

        def div(x, y):
            r = np.empty_like(x)
            r[0] = x[0] / y[0]
            r[1:] = (x[1:] * y[0] - y[1:] * x[0]) / (y[0] * y[0])
            return r

        out[2 * pl] = div(a, eps)
        out[2 * pl + 1] = -div(b, eps)
    return out


class PicMatch:
    """Re-matching of the four quadrupoles for a bunch of `current_A` peak current: a Gaussian bunch
    matched (at zero current) to the first lattice's periodic Twiss functions enters the matching
    section; Eq. 6 compares its Twiss functions at the exit with the second lattice's periodic ones."""

    def __init__(self, current_A=100.0, n_particles=16384, grid=32, precision=adpic.AD_PIC_FP64,
                 k_first=optics.FODO_K, k_second=16.0, seed=7):
        self.zero = optics.TwissMatch(k_first, k_second)
        self.k_second = k_second
        t1 = optics.periodic_twiss(optics.fodo_cell(k_first, slots=None))[:, 0]
        self.target = self.zero.target
        self.N = int(n_particles)
        self.grid = (grid, grid, grid)
        self.P = 7                                   # slots 0..3: the four strengths; 4..6 unused
        sigma_z = 1e-3
        base = I.default_beam(7)
        self.beam = I.Beam(kinetic_eV=base.kinetic_eV, mass_eV=base.mass_eV, charge_e=base.charge_e,
                           bunch_charge_C=bunch_charge_for_current(current_A, sigma_z), eps_n=base.eps_n,
                           alpha=(t1[1], t1[3], 0.0), beta=(t1[0], t1[2], base.beta[2]),
                           twiss_slot=(-1,) * 6)
        self.normals = I.normals(seed, self.N)
        self.sim = adpic.ADPIC(self.grid, self.N, self.P, precision)
        self.evaluations = 0

    def section(self, ks):
        line = optics.matching_section(ks, DRIFT, QUAD)
        kicks = [KICKS_QUAD if t == 1 else KICKS_DRIFT for (t, _, _, _, _) in line]
        return line, kicks

    def run(self, ks, extra=None):
        """Dual PIC run of the bunch through the matching section (and `extra` (line, kicks) after it);
        returns the moment history (one record per pass end)."""
        line, kicks = self.section(ks)
        if extra is not None:
            line, kicks = line + extra[0], kicks + extra[1]
        self.sim.set_beamline(line, kicks)
        self.sim.set_beam(self.beam, self.normals)
        self.sim.run(sum(kicks))
        return self.sim.history()

    def twiss(self, ks):
        self.evaluations += 1
        return beam_twiss(self.run(ks)[-1], 4)

    def objective(self, ks):
        t = self.twiss(ks)
        bxt, _, byt, _ = self.target
        w = np.array([1.0 / bxt ** 2, 1.0, 1.0 / byt ** 2, 1.0])
        r = t[:, 0] - self.target
        return float(np.sum(w * r * r)), 2.0 * (w * r) @ t[:, 1:]

    def bfgs(self, k0, ftol=1e-10, max_iter=60):
        self.evaluations = 0
        x, f, _ = bfgs(self.objective, np.asarray(k0, dtype=np.float64), -60 * np.ones(4), 60 * np.ones(4),
                       max_iter=max_iter, ftol=ftol, first_step=1.0)
        return x, f, self.evaluations

    def envelope_beat(self, ks, periods=8):
        """Relative spread (std / mean) of the rms beam sizes at the ends of `periods` cells of the
        second lattice after the section: a mismatched beam's envelope beats."""
        cell = optics.fodo_cell(self.k_second, slots=None)
        kicks = [KICKS_QUAD if t == 1 else 4 for (t, _, _, _, _) in cell]
        sizes = []
        line, lk = self.section(ks)
        self.sim.set_beamline(line + cell * periods, lk + kicks * periods)
        self.sim.set_beam(self.beam, self.normals)
        n_sec, n_cell = sum(lk), sum(kicks)
        self.sim.run(n_sec)
        for _ in range(periods):
            self.sim.run(n_cell)
            m = self.sim.moments_full()
            sizes.append([math.sqrt(m[pl][2][0] - m[pl][0][0] ** 2) for pl in range(2)])
        s = np.array(sizes)
        return s.std(axis=0) / s.mean(axis=0)

    def close(self):
        self.sim.close()


class MatchProblem:
    """The re-matching in normalised strengths x in [-1, 1]^4 around `center`, k = center (1 + rel x),
    in the form the surrogate machinery takes: evaluate(x) runs the dual PIC through the section and
    returns the exit Twiss functions (beta_x, alpha_x, beta_y, alpha_y) over `scale` (the weights of
    Eq. 6: the target betas, 1 for the alphas) and their exact derivatives in x."""

    def __init__(self, pm, center, rel=0.2):
        self.pm = pm
        self.center = np.asarray(center, dtype=np.float64)
        self.rel = rel
        bxt, _, byt, _ = pm.target
        self.scale = np.array([bxt, 1.0, byt, 1.0])
        self.target = np.asarray(pm.target) / self.scale
        self.evaluations = 0

    def strengths(self, x):
        return self.center * (1.0 + self.rel * np.asarray(x))

    def evaluate(self, x):
        self.evaluations += 1
        t = self.pm.twiss(self.strengths(x))
        y = t[:, 0] / self.scale
        dy = t[:, 1:5] * (self.center * self.rel)[None, :] / self.scale[:, None]
        return y, dy

    def dataset(self, n, seed=11):
        """n dual-PIC runs at x ~ U(-1, 1)^4: inputs, values and derivatives."""
        X = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, 4))
        Y = np.zeros((n, 4))
        dY = np.zeros((n, 4, 4))
        for i in range(n):
            Y[i], dY[i] = self.evaluate(X[i])
        self.evaluations = 0
        return X, Y, dY


def surrogate_rematch(pm, center, n_train=256, rel=0.2, ftol=1e-9, max_evals=60, width=128, steps=3000):
    """The re-matching warm-started by a learned surrogate: a 4 -> width^3 -> 4 MLP is fitted with
    the Sobolev loss to n_train dual-PIC runs around `center` (values and exact derivatives), then the
    trust-region search of surrogate.search_warm proposes strengths from BFGS on the surrogate
    (corrected to the last dual-PIC value and gradient), and a full dual-PIC run checks every proposal;
    BFGS on dual-PIC gradients finishes. Returns (strengths, Eq. 6 value, dual-PIC evaluations of the
    search, training-set runs, held-out surrogate errors)."""
    prob = MatchProblem(pm, center, rel)
    X, Y, dY = prob.dataset(n_train + n_train // 8)
    Xt, Yt, dYt = X[:n_train], Y[:n_train], dY[:n_train]
    sur = Surrogate(width=width, hidden=3, max_batch=min(512, n_train), seed=1, n_in=4, n_out=4)
    sur.fit(Xt, Yt, dYt, steps=steps, lam=1.0, lr=2e-3, lr_final=2e-5)
    errs = sur.errors(X[n_train:], Y[n_train:], dY[n_train:])
    x, f, evals = search_warm(prob, sur, prob.target, np.zeros(4), ftol, max_evals=max_evals, radius=0.5)
    sur.close()
    return prob.strengths(x), f, evals, len(X), errs

