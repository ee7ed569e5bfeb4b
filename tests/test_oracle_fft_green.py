"""Pins of the oracle's FFT, integrated Green's function and Hockney convolution."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2511_21839_gb300 import inputs as I

EPS0 = 8.8541878128e-12


@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 256])
def test_fft_matches_dft_definition(n):
    rng = np.random.default_rng(n)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    j = np.arange(n)
    W = np.exp(-2j * np.pi * np.outer(j, j) / n)       # X_k = sum_j x_j exp(-2 pi i j k / n)
    np.testing.assert_allclose(oracle.fft1d(z, -1), W @ z, rtol=0, atol=1e-12 * max(1, n))
    np.testing.assert_allclose(oracle.fft1d(z, +1), np.conj(W) @ z, rtol=0, atol=1e-12 * max(1, n))


def _box_quad(x, y, z, hx, hy, hz):
    f = lambda zz, yy, xx: 1.0 / math.sqrt(xx * xx + yy * yy + zz * zz)
    v, _ = integrate.tplquad(f, x - hx / 2, x + hx / 2, y - hy / 2, y + hy / 2, z - hz / 2, z + hz / 2,
                             epsabs=1e-14, epsrel=1e-12)
    return v / (4 * math.pi * EPS0 * hx * hy * hz)


def _self_cell(hx, hy, hz):
    """Cell average of 1/(4 pi eps0 r) over the box centred at the origin: split the box into six
    pyramids with apex at the origin; a pyramid over a face at distance d contributes
    (d/2) * integral over the face of dA/|s|."""
    total = 0.0
    for d, (a, b) in ((hx / 2, (hy, hz)), (hy / 2, (hx, hz)), (hz / 2, (hx, hy))):
        v, _ = integrate.dblquad(lambda v_, u_: 1.0 / math.sqrt(d * d + u_ * u_ + v_ * v_),
                                 -a / 2, a / 2, -b / 2, b / 2, epsabs=1e-15, epsrel=1e-13)
        total += 2 * (d / 2) * v
    return total / (4 * math.pi * EPS0 * hx * hy * hz)


def test_igf_self_cell_pyramids():
    for h in [(1.0, 1.0, 1.0), (1e-4, 1.3e-4, 2.7e-4), (2.0, 0.5, 1.0)]:
        np.testing.assert_allclose(oracle.igf(0, 0, 0, *h), _self_cell(*h), rtol=1e-12)


@pytest.mark.parametrize("off", [(1, 0, 0), (1, 1, 0), (2, 1, 3), (0, 0, 1)])
def test_igf_off_cells_quadrature(off):
    h = (1.0, 1.3, 2.1)
    x, y, z = (o * hh for o, hh in zip(off, h))
    np.testing.assert_allclose(oracle.igf(x, y, z, *h), _box_quad(x, y, z, *h), rtol=1e-10)


def test_igf_far_field_is_point_charge():
    # for a cube the second-order correction vanishes (1/r is harmonic): error ~ (h/r)^4
    for r in [10.0, 20.0, 40.0]:
        g = oracle.igf(r, 0.3 * r, 0.2 * r, 1, 1, 1) * 4 * math.pi * EPS0
        dist = r * math.sqrt(1 + 0.09 + 0.04)
        assert abs(g * dist - 1) < 0.5 * (1.0 / dist) ** 4


def _small(n=8, P=1, N=1):
    w = I.workload("fodo_10k_32")
    return oracle.Oracle(**I.orc_kwargs(w, n_particles=N, grid=(n, n, n), n_deriv=P))


@pytest.mark.parametrize("shape", [(8, 8, 8), (8, 16, 8)])
def test_hockney_matches_direct_sum(shape):
    w = I.workload("fodo_10k_32")
    o = oracle.Oracle(**I.orc_kwargs(w, n_particles=1, grid=shape, n_deriv=1))
    rng = np.random.default_rng(5)
    rho = rng.standard_normal(o.grid_shape()) * 1e-12
    geom = np.array([-1e-3, -1e-3, -1e-3, 1e-4, 1.5e-4, 0.7e-4])
    phi_fft = o.solve(geom, rho)
    phi_dir = o.solve_direct(geom, rho)
    np.testing.assert_allclose(phi_fft, phi_dir, rtol=0, atol=1e-13 * np.abs(phi_dir).max())


def test_green_even_extension():
    o = _small(8)
    geom = np.array([0, 0, 0, 1e-4, 2e-4, 3e-4])
    G = o.green(geom)
    g0 = o.constants()["gamma0"]
    # index i and 2n - i hold the same offset magnitude
    np.testing.assert_array_equal(G[:, :, 1:8], G[:, :, 15:8:-1])
    np.testing.assert_array_equal(G[1:8], G[15:8:-1])
    assert G[0, 0, 1] == pytest.approx(oracle.igf(1e-4, 0, 0, 1e-4, 2e-4, 3e-4 * g0), rel=1e-15)
