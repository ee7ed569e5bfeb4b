"""Single-particle dual optics on the GPU (Sec. 3) against the oracle: Twiss functions and their
derivatives of many beamlines at once, element-by-element dual tracking for several derivative
counts, and the 4-quadrupole matching with BFGS on the exact gradient against Nelder-Mead.

All FP64. Bounds: Twiss functions 1e-12 relative per value, derivatives 1e-11 of each row's largest
(the two sides evaluate the same dual arithmetic in different orders); tracking after tens of
periods 1e-11 of each channel's largest.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2511_21839_gb300 import adpic, build

    build.build()
    return adpic


def perturbed_cells(n, seed=1):
    from paper_2511_21839_gb300 import optics

    rng = np.random.default_rng(seed)
    cells = []
    for _ in range(n):
        L = np.array(optics.FODO_LENGTHS) * (1 + rng.uniform(-0.1, 0.1, 5))
        k = optics.FODO_K * (1 + rng.uniform(-0.1, 0.1))
        cells.append(optics.fodo_cell(k, tuple(L)))
    return cells


def close_rows(gpu, ref, rtol_v, rtol_d):
    np.testing.assert_allclose(gpu[..., 0], ref[..., 0], rtol=rtol_v, atol=0)
    scale = np.abs(ref[..., 1:]).max(axis=-1, keepdims=True)
    err = np.abs(gpu[..., 1:] - ref[..., 1:]) / np.where(scale > 0, scale, 1.0)
    assert err.max() < rtol_d, err.max()
    return err.max()


def test_periodic_twiss_batch_vs_oracle(lib):
    cells = perturbed_cells(300)
    out = lib.ad_pic_twiss_batch(cells, 7, n_cell=5)
    for i in (0, 1, 17, 123, 299):
        close_rows(out[i], oracle.periodic_twiss(cells[i], 7), 1e-12, 1e-11)


def test_twiss_transport_batch_vs_oracle(lib):
    from paper_2511_21839_gb300 import optics

    rng = np.random.default_rng(2)
    lines = [optics.matching_section(rng.uniform(10, 30, 4) * np.array([1, -1, 1, -1])) for _ in range(64)]
    t0 = np.column_stack([rng.uniform(0.5, 3, 64), rng.uniform(-2, 2, 64), rng.uniform(0.5, 3, 64),
                          rng.uniform(-2, 2, 64)])
    out = lib.ad_pic_twiss_batch(lines, 4, twiss0=t0)
    for i in range(0, 64, 9):
        close_rows(out[i], oracle.twiss(lines[i], 4, t0[i]), 1e-12, 1e-11)


def test_unstable_cell_is_reported(lib):
    from paper_2511_21839_gb300 import optics

    bad = optics.fodo_cell(22.0, (0.5, 0.1, 1.0, 0.1, 0.5))
    with pytest.raises(lib.AdPicError) as e:
        lib.ad_pic_twiss_batch([bad], 7, n_cell=5)
    assert e.value.status == -10


@pytest.mark.parametrize("P", [0, 1, 7, 9, 13, 31])
def test_tracking_vs_oracle(lib, P):
    from paper_2511_21839_gb300 import optics

    cell = optics.fodo_cell()
    cell = [(t, L, k, sL if sL < P else -1, sk if sk < P else -1) for (t, L, k, sL, sk) in cell]
    if P > 7:                                        # more slots: a second copy of the cell with its own slots
        extra = [(t, L, k, sL + 7 if sL >= 0 and sL + 7 < P else -1, sk + 7 if sk >= 0 and sk + 7 < P else -1)
                 for (t, L, k, sL, sk) in optics.fodo_cell()]
        cell = cell + extra
    rng = np.random.default_rng(3)
    x0 = rng.normal(size=(37, 4)) * 1e-3            # a ragged batch (not a multiple of the block)
    n_rep = 40
    out, ms = lib.ad_pic_track_batch(x0, cell, P, n_rep)
    ref = oracle.track(cell, P, x0, n_rep)
    scale = np.abs(ref).max(axis=0, keepdims=True)
    err = np.abs(out - ref) / np.where(scale > 0, scale, 1.0)
    print(f"P={P}: max error {err.max():.2e}, kernel {ms:.3f} ms")
    assert err.max() < 1e-11


def test_matching_bfgs_needs_fewer_evaluations_than_nelder_mead(lib):
    """Sec. 3: the four matching quadrupoles found by BFGS on the exact dual gradient of Eq. 6, and
    by the derivative-free simplex; BFGS reaches the target in far fewer objective evaluations."""
    from paper_2511_21839_gb300 import optics

    m = optics.TwissMatch()
    k0 = [20.0, -20.0, 20.0, -20.0]
    xb, fb, nb = m.bfgs(k0, ftol=1e-12)
    xn, fn, nn = m.nelder_mead(k0, ftol=1e-12)
    print(f"BFGS: f = {fb:.2e} after {nb} evaluations; Nelder-Mead: f <= 1e-12 after {nn}")
    assert fb <= 1e-12
    assert nb * 4 < nn
    # the matched section delivers the second lattice's periodic Twiss functions
    t = m.twiss(xb)[:, 0]
    np.testing.assert_allclose(t, m.target, rtol=2e-6, atol=2e-6)
    # and the oracle agrees on the matched lattice
    ref = oracle.twiss(optics.matching_section(xb), 4, oracle.periodic_twiss(m.first, 0)[:, 0])
    np.testing.assert_allclose(t, ref[:, 0], rtol=1e-12)


def test_relative_sensitivities_match_the_oracle(lib):
    """x dT / (T dx) of the periodic Twiss functions w.r.t. the seven cell parameters (Sec. 3 figure)."""
    from paper_2511_21839_gb300 import optics

    cell = optics.fodo_cell()
    rel = optics.relative_twiss_sensitivities(cell)
    ref = oracle.periodic_twiss(cell, 7)
    x = np.array([0.25, 0.1, 22.0, 0.5, 0.1, -22.0, 0.25])
    np.testing.assert_allclose(rel, ref[:, 1:] * x / ref[:, :1], rtol=1e-10, atol=1e-12)
