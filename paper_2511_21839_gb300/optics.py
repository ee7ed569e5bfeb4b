"""Single-particle dual optics workflows of Sec. 3 on the GPU library.

Beamlines are lists of (type, L, k, slot_L, slot_k) tuples (type 0 drift, 1 thick quadrupole of
normalised strength k in 1/m^2); every number the workflows need comes from the C ABI calls
ad_pic_twiss_batch and ad_pic_track_batch (dual FP64 on the GPU). What is here is host logic only:
building beamlines, the matching objective of Eq. 6 from the Twiss functions and their derivatives,
and the two optimisers the paper compares (variable-metric BFGS on the exact gradient against the
derivative-free Nelder-Mead simplex).
"""
import numpy as np

from . import adpic
from .surrogate import bfgs

# The FODO cell of the Sec. 3 examples: quadrupole strengths +-22 1/m^2 (the paper's values), 0.1 m
# quadrupoles, drifts 0.25 / 0.5 / 0.25 m (the paper gives no lengths; these give a stable cell
# with 77 degrees of phase advance)
FODO_LENGTHS = (0.25, 0.1, 0.5, 0.1, 0.25)
FODO_K = 22.0
LATTICE_SLOTS = (0, 1, 2, 3, 4, 5, 6)     # L_D1, L_Q1, k_Q1, L_D2, L_Q2, k_Q2, L_D3 (the paper's order)


def fodo_cell(k=FODO_K, lengths=FODO_LENGTHS, slots=LATTICE_SLOTS):
    """Drift, focusing quad, drift, defocusing quad, drift; slots=None holds every parameter constant."""
    s = slots if slots is not None else (-1,) * 7
    L = lengths
    return [(0, L[0], 0.0, s[0], -1), (1, L[1], k, s[1], s[2]), (0, L[2], 0.0, s[3], -1),
            (1, L[3], -k, s[4], s[5]), (0, L[4], 0.0, s[6], -1)]


def matching_section(ks, drift=0.3, quad=0.1):
    """Four quadrupoles between five drifts; the strengths are the derivative slots 0..3."""
    bl = []
    for i, k in enumerate(ks):
        bl += [(0, drift, 0.0, -1, -1), (1, quad, float(k), -1, i)]
    return bl + [(0, drift, 0.0, -1, -1)]


def periodic_twiss(cell, n_deriv=0):
    """Periodic (beta_x, alpha_x, beta_y, alpha_y) of a cell with derivatives: [4][n_deriv + 1]."""
    return adpic.ad_pic_twiss_batch([cell], n_deriv, n_cell=len(cell))[0]


def relative_twiss_sensitivities(cell, n_deriv=7):
    """x dT / (T dx) of the periodic Twiss functions T w.r.t. the cell's parameters x (Sec. 3)."""
    t = periodic_twiss(cell, n_deriv)
    x = np.zeros(n_deriv)
    for typ, L, k, sL, sk in cell:
        if sL >= 0:
            x[sL] = L
        if typ == 1 and sk >= 0:
            x[sk] = k
    return t[:, 1:] * x[None, :] / t[:, :1]


class TwissMatch:
    """The Sec. 3 matching problem: the periodic Twiss functions of one FODO lattice, transported
    through four matching quadrupoles, must equal the periodic Twiss functions of a second FODO
    lattice at its entrance. objective(k) is Eq. 6 and its exact gradient; every evaluation is one
    dual GPU evaluation of the cell plus the section (counted in self.evaluations)."""

    def __init__(self, k_first=FODO_K, k_second=16.0):
        self.first = fodo_cell(k_first, slots=None)
        self.target = periodic_twiss(fodo_cell(k_second, slots=None))[:, 0]
        self.evaluations = 0

    def twiss(self, ks):
        self.evaluations += 1
        return adpic.ad_pic_twiss_batch([self.first + matching_section(ks)], 4, n_cell=len(self.first))[0]

    def objective(self, ks):
        t = self.twiss(ks)
        bxt, axt, byt, ayt = self.target
        w = np.array([1.0 / bxt ** 2, 1.0, 1.0 / byt ** 2, 1.0])
        r = t[:, 0] - self.target
        return float(np.sum(w * r * r)), 2.0 * (w * r) @ t[:, 1:]

    def bfgs(self, k0, ftol=1e-14, max_iter=200):
        self.evaluations = 0
        x, f, _ = bfgs(self.objective, np.asarray(k0, dtype=np.float64), -60 * np.ones(4), 60 * np.ones(4),
                       max_iter=max_iter, ftol=ftol, first_step=1.0)
        return x, f, self.evaluations

    def nelder_mead(self, k0, ftol=1e-14, max_evals=3000):
        """Derivative-free simplex search (scipy's Nelder-Mead); returns (x, f, evaluations to reach ftol
        or the number made if it never does)."""
        from scipy.optimize import minimize

        self.evaluations = 0
        best = []

        def f(k):
            v = self.objective(k)[0]
            best.append(v)
            return v

        r = minimize(f, np.asarray(k0, dtype=np.float64), method="Nelder-Mead",
                     options=dict(xatol=1e-12, fatol=1e-18, maxfev=max_evals))
        b = np.minimum.accumulate(best)
        reached = np.nonzero(b <= ftol)[0]
        return r.x, float(r.fun), int(reached[0] + 1) if reached.size else len(best)
