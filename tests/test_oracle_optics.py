"""Pins of the oracle's single-particle dual optics (Sec. 3) against the mathematics.

Element maps against the matrix exponential of the linear equations of motion x'' = -k x (scipy's
expm, an independent route to the thick-lens matrix of Eq. "quadtr"), their parameter derivatives
against the exact Frechet derivative of the exponential; Twiss transport (Eq. 5) against the
congruence B(s) = M B(0) M^T of the Twiss matrix and the invariant beta gamma - alpha^2 = 1; the
periodic Twiss functions as the fixed point of one cell; tracking against powers of the cell matrix
and the closed form cos(n mu) I + sin(n mu) J. Derivatives of composite quantities against central
finite differences of the oracle's value part.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm, expm_frechet

import oracle

# the Sec. 3 FODO cell at k = +-22 1/m^2 (lengths: a reading, the paper gives only the strengths)
FODO = [(0, 0.25, 0.0, 0, -1), (1, 0.1, 22.0, 1, 2), (0, 0.5, 0.0, 3, -1), (1, 0.1, -22.0, 4, 5), (0, 0.25, 0.0, 6, -1)]
P = 7


def generator(k):
    return np.array([[0.0, 1.0], [-k, 0.0]])


def expm_matrix(beamline, plane):
    M = np.eye(2)
    for t, L, k, _, _ in beamline:
        kk = (k if plane == 0 else -k) if t == 1 else 0.0
        M = expm(generator(kk) * L) @ M
    return M


def params(beamline):
    """Values of the derivative slots (L and k of each element) as a flat dict slot -> value."""
    out = {}
    for t, L, k, sL, sk in beamline:
        if sL >= 0:
            out[sL] = L
        if t == 1 and sk >= 0:
            out[sk] = k
    return out


def with_param(beamline, slot, value):
    res = []
    for t, L, k, sL, sk in beamline:
        if sL == slot:
            L = value
        if t == 1 and sk == slot:
            k = value
        res.append((t, L, k, sL, sk))
    return res


def central_fd(fn, beamline, slot, rel=1e-6):
    v = params(beamline)[slot]
    h = rel * abs(v)
    return (fn(with_param(beamline, slot, v + h)) - fn(with_param(beamline, slot, v - h))) / (2 * h)


@pytest.mark.parametrize("k", [22.0, -22.0, 0.0, 3.7])
def test_element_matrix_and_derivatives_match_the_exponential(k):
    L = 0.13
    el = [(1 if k != 0 else 0, L, k, 0, 1 if k != 0 else -1)]
    m = oracle.beamline_matrix(el, 2)
    for plane in (0, 1):
        kk = k if plane == 0 else -k
        A = generator(kk)
        ref = expm(A * L)
        np.testing.assert_allclose(m[plane, :, 0].reshape(2, 2), ref, rtol=1e-13, atol=1e-15)
        # d/dL exp(A L) = A exp(A L); d/dk exp(A L) = Frechet derivative in the direction dA/dk L
        np.testing.assert_allclose(m[plane, :, 1].reshape(2, 2), A @ ref, rtol=1e-12, atol=1e-14)
        if k != 0:
            dA = np.array([[0.0, 0.0], [-1.0 if plane == 0 else 1.0, 0.0]]) * L
            _, dref = expm_frechet(A * L, dA)
            np.testing.assert_allclose(m[plane, :, 2].reshape(2, 2), dref, rtol=1e-11, atol=1e-14)


def test_beamline_matrix_is_the_product_and_symplectic():
    m = oracle.beamline_matrix(FODO, P)
    for plane in (0, 1):
        M = m[plane, :, 0].reshape(2, 2)
        np.testing.assert_allclose(M, expm_matrix(FODO, plane), rtol=1e-12, atol=1e-14)
        # det M = 1 for every parameter: its dual derivative vanishes
        m11, m12, m21, m22 = m[plane]
        ddet = m11[1:] * m22[0] + m11[0] * m22[1:] - m12[1:] * m21[0] - m12[0] * m21[1:]
        assert abs(m11[0] * m22[0] - m12[0] * m21[0] - 1.0) < 1e-13
        assert np.abs(ddet).max() < 1e-12
        for slot in range(P):
            fd = central_fd(lambda bl: expm_matrix(bl, plane).ravel(), FODO, slot)
            np.testing.assert_allclose(m[plane, :, slot + 1], fd, rtol=2e-7, atol=1e-9)


def twiss_matrix(beta, alpha):
    return np.array([[beta, -alpha], [-alpha, (1 + alpha * alpha) / beta]])


def test_twiss_transport_eq5_is_the_congruence_and_keeps_the_invariant():
    t0 = np.array([1.7, 0.4, 0.6, -0.9])
    out = oracle.twiss(FODO, P, t0)
    for plane in (0, 1):
        M = expm_matrix(FODO, plane)
        B1 = M @ twiss_matrix(t0[2 * plane], t0[2 * plane + 1]) @ M.T
        assert out[2 * plane, 0] == pytest.approx(B1[0, 0], rel=1e-12)
        assert out[2 * plane + 1, 0] == pytest.approx(-B1[0, 1], rel=1e-12, abs=1e-13)
        beta, alpha = out[2 * plane], out[2 * plane + 1]
        # beta gamma - alpha^2 = 1 with gamma = (1 + alpha^2) / beta holds identically; its dual
        # derivative is zero only if beta and alpha derivatives are consistent with B1 = M B0 M^T
        for slot in range(P):
            def f(bl):
                Mp = expm_matrix(bl, plane)
                B = Mp @ twiss_matrix(t0[2 * plane], t0[2 * plane + 1]) @ Mp.T
                return np.array([B[0, 0], -B[0, 1]])
            fd = central_fd(f, FODO, slot)
            np.testing.assert_allclose([beta[slot + 1], alpha[slot + 1]], fd, rtol=2e-7, atol=1e-8)


def test_drift_twiss_closed_form():
    b0, a0, s = 2.3, -0.7, 1.9
    g0 = (1 + a0 * a0) / b0
    out = oracle.twiss([(0, s, 0.0, 0, -1)], 1, np.array([b0, a0, b0, a0]))
    assert out[0, 0] == pytest.approx(b0 - 2 * a0 * s + g0 * s * s, rel=1e-14)
    assert out[1, 0] == pytest.approx(a0 - g0 * s, rel=1e-14)
    assert out[0, 1] == pytest.approx(-2 * a0 + 2 * g0 * s, rel=1e-13)       # d beta / d s
    assert out[1, 1] == pytest.approx(-g0, rel=1e-13)                        # d alpha / d s


def test_periodic_twiss_is_the_fixed_point_of_the_cell():
    per = oracle.periodic_twiss(FODO, P)
    once = oracle.twiss(FODO, P, per[:, 0])
    np.testing.assert_allclose(once[:, 0], per[:, 0], rtol=1e-12, atol=1e-13)
    for plane in (0, 1):
        M = expm_matrix(FODO, plane)
        mu = math.acos(0.5 * np.trace(M))
        s = math.copysign(math.sin(mu), M[0, 1])
        assert per[2 * plane, 0] == pytest.approx(M[0, 1] / s, rel=1e-13)
    for slot in range(P):
        fd = central_fd(lambda bl: oracle.periodic_twiss(bl, 0)[:, 0], FODO, slot)
        np.testing.assert_allclose(per[:, slot + 1], fd, rtol=2e-6, atol=1e-7)
    with pytest.raises(ValueError):
        oracle.periodic_twiss([(0, 0.5, 0, -1, -1), (1, 0.1, 22.0, -1, -1), (0, 1.0, 0, -1, -1),
                               (1, 0.1, -22.0, -1, -1), (0, 0.5, 0, -1, -1)], 0)


def test_tracking_is_the_power_of_the_cell_matrix():
    rng = np.random.default_rng(5)
    x0 = rng.normal(size=(5, 4)) * 1e-3
    n = 37
    out = oracle.track(FODO, P, x0, n)
    per = oracle.periodic_twiss(FODO, 0)
    for plane in (0, 1):
        M = expm_matrix(FODO, plane)
        Mn = np.linalg.matrix_power(M, n)
        # closed form through the Twiss parameters: M^n = cos(n mu) I + sin(n mu) J
        mu = math.acos(0.5 * np.trace(M))
        beta, alpha = per[2 * plane, 0], per[2 * plane + 1, 0]
        J = np.array([[alpha, beta], [-(1 + alpha * alpha) / beta, -alpha]])
        sgn = math.copysign(1.0, M[0, 1])
        np.testing.assert_allclose(Mn, math.cos(n * mu) * np.eye(2) + sgn * math.sin(n * mu) * J, atol=1e-11)
        ref = x0[:, 2 * plane:2 * plane + 2] @ Mn.T
        np.testing.assert_allclose(out[:, 2 * plane:2 * plane + 2, 0], ref, rtol=1e-11, atol=1e-15)
    for slot in range(P):
        fd = central_fd(lambda bl: oracle.track(bl, 0, x0, n)[:, :, 0], FODO, slot)
        scale = np.abs(fd).max()
        assert np.abs(out[:, :, slot + 1] - fd).max() < 1e-6 * scale
