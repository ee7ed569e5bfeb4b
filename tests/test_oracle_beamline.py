"""Pins of the oracle's PIC on a general beamline (the matching-section runs of Sec. 4).

The FODO period written as a beamline (strengths k = g / B rho given directly) reproduces the FODO
form: the same values bit for bit, and derivatives w.r.t. k that are B rho times those w.r.t. g. At
zero current one pass through a beamline is its linear map: the matrix exponentials of the elements
(scipy's expm) for the values and the exact Frechet derivative for the strength derivatives.
"""
import numpy as np
import pytest
from scipy.linalg import expm, expm_frechet

import oracle
from paper_2511_21839_gb300 import inputs as I


def fodo_line(brho, lat):
    """(type, L, k, slot_L, slot_k) of the FODO period with k = g / B rho, the paper's slot order."""
    kf, kd = lat.g[0] / brho, lat.g[1] / brho
    return [(0, lat.L[0], 0.0, 0, -1), (1, lat.L[1], kf, 1, 2), (0, lat.L[2], 0.0, 3, -1),
            (1, lat.L[3], kd, 4, 5), (0, lat.L[4], 0.0, 6, -1)]


def test_fodo_as_beamline_reproduces_the_fodo_form():
    w = I.workload("fodo_10k_32")
    N = 2000
    kw = I.orc_kwargs(w, n_particles=N, grid=(16, 16, 16))
    o = oracle.Oracle(**kw)
    brho = o.constants()["brho"]
    ol = oracle.Oracle(line=fodo_line(brho, w.lattice), line_kicks=w.lattice.kicks, **kw)
    nrm = I.normals(21, N)
    s1, s2 = o.beam_init(nrm), ol.beam_init(nrm)
    h1, _ = o.run(s1, 20)
    h2, _ = ol.run(s2, 20)
    assert np.array_equal(s1[:, :, 0], s2[:, :, 0]) and np.array_equal(h1[..., 0], h2[..., 0])
    e1, e2 = o.emittance(h1[-1]), ol.emittance(h2[-1])
    for slot in (2, 5):                                  # strengths: d/dk = B rho d/dg
        np.testing.assert_allclose(e2[:2, slot + 1], brho * e1[:2, slot + 1], rtol=1e-9)
    for slot in (0, 1, 3, 4, 6):                         # lengths: the same derivative
        np.testing.assert_allclose(e2[:2, slot + 1], e1[:2, slot + 1], rtol=1e-9)


def test_zero_current_pass_is_the_beamline_map():
    line = [(0, 0.3, 0.0, -1, -1), (1, 0.1, 21.0, -1, 0), (0, 0.3, 0.0, -1, -1), (1, 0.1, -19.5, -1, 1),
            (0, 0.3, 0.0, -1, -1), (1, 0.1, 18.0, -1, 2), (0, 0.3, 0.0, -1, -1), (1, 0.1, -20.5, -1, 3),
            (0, 0.3, 0.0, 4, -1)]
    kicks = [2, 3, 4, 1, 2, 2, 3, 2, 5]
    w = I.workload("fodo_10k_32")
    N = 500
    kw = I.orc_kwargs(w, n_particles=N, grid=(16, 16, 16))
    kw["bunch_charge_C"] = 0.0
    o = oracle.Oracle(line=line, line_kicks=kicks, **kw)
    st = o.beam_init(I.normals(22, N))
    x0 = st[:, :, 0].copy()
    o.run(st, sum(kicks))
    for plane in (0, 1):
        M = np.eye(2)
        dM = [np.zeros((2, 2)) for _ in range(5)]        # derivatives w.r.t. slots 0..4
        for t, L, k, sL, sk in line:
            kk = (k if plane == 0 else -k) if t == 1 else 0.0
            A = np.array([[0.0, 1.0], [-kk, 0.0]])
            E = expm(A * L)
            for s in range(5):                           # product rule through the beamline
                dE = np.zeros((2, 2))
                if t == 1 and sk == s:
                    _, dE = expm_frechet(A * L, np.array([[0.0, 0.0], [-1.0 if plane == 0 else 1.0, 0.0]]) * L)
                if sL == s:
                    dE = A @ E
                dM[s] = dE @ M + E @ dM[s]
            M = E @ M
        u0 = x0[2 * plane:2 * plane + 2]
        got = st[2 * plane:2 * plane + 2]
        np.testing.assert_allclose(got[:, :, 0], M @ u0, rtol=1e-12, atol=1e-16)
        for s in range(5):
            ref = dM[s] @ u0
            assert np.abs(got[:, :, s + 1] - ref).max() < 1e-11 * np.abs(ref).max()
