"""Pins of the oracle's kinetic energy as a dual input (Sec. 4: beam parameters as AD variables).

With the energy E in a derivative slot, gamma0, beta0 gamma0, B rho and the kick constants become
dual, and so does the rest-frame z spacing gamma0 hz of the integrated Green's function and of the
field. The pins check each piece against something other than the oracle's own dual arithmetic:
closed-form derivatives of the relativistic constants, central differences of the Green's function
in its cell size, the FFT convolution against the direct sum, and the derivative of a whole run
against central differences of value-only runs at frozen geometry.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2511_21839_gb300 import inputs as I

QE = 1.602176634e-19
CL = 299792458.0


def make(n=16, N=1000, P=7, beam=None, lattice=None):
    w = I.workload("fodo_10k_32")
    kw = I.orc_kwargs(w, n_particles=N, grid=(n, n, n) if isinstance(n, int) else n, n_deriv=P,
                      lattice=lattice, beam=beam)
    return oracle.Oracle(**kw)


def energy_beam(slot=0, **kw):
    w = I.workload("fodo_10k_32")
    return I.Beam(**{**w.beam.__dict__, "energy_slot": slot, **kw})


@pytest.mark.parametrize("off", [(0, 0, 0), (1, 0, 0), (0, 0, 1), (1, 2, 1), (3, 1, 4), (0, 5, 2), (7, 6, 9)])
def test_igf_cell_size_derivative_matches_central_fd(off):
    """dG/dhz with the node offset k hz moving with hz, against a central difference of orc_igf
    (Richardson-extrapolated, so the truncation error is O(h^4))."""
    hx, hy, hz = 1.0e-3, 1.3e-3, 2.1e-3
    i, j, k = off
    g, dg = oracle.igf_dhz(i * hx, j * hy, float(k), hx, hy, hz)
    # the two corner forms (k hz +- hz/2 and (k +- 1/2) hz) round differently, and the 8-corner
    # difference cancels about log10(r^3 / (hx hy hz)) digits
    assert g == pytest.approx(oracle.igf(i * hx, j * hy, k * hz, hx, hy, hz), rel=1e-10)

    def cd(h):
        return (oracle.igf(i * hx, j * hy, k * (hz + h), hx, hy, hz + h) -
                oracle.igf(i * hx, j * hy, k * (hz - h), hx, hy, hz - h)) / (2 * h)

    h = 1e-3 * hz
    fd = (4 * cd(h / 2) - cd(h)) / 3
    assert dg == pytest.approx(fd, rel=1e-7, abs=1e-9 * abs(g) / hz)


def test_dual_constants_match_closed_forms_and_fd():
    """d gamma0/dE = 1/(m c^2), d(beta0 gamma0)/dE = 1/(beta0 m c^2), d(B rho)/dE = (m c / q)/(beta0 m c^2)
    in closed form; the kick constants against central differences of orc_constants in E."""
    b = energy_beam(0)
    o = make(N=10, P=1, beam=b)
    d = o.dual_constants()
    c = o.constants()
    m = b.mass_eV
    g0, b0 = c["gamma0"], c["beta0"]
    assert d[0, 0] == g0 and d[1, 0] == pytest.approx(b0 * g0, rel=1e-15)
    assert d[0, 1] == pytest.approx(1.0 / m, rel=1e-14)
    assert d[1, 1] == pytest.approx(1.0 / (b0 * m), rel=1e-12)
    mass_kg = m * QE / CL ** 2
    assert d[2, 1] == pytest.approx(mass_kg * CL / (b.charge_e * QE) / (b0 * m), rel=1e-12)
    assert d[5, 1] == pytest.approx(2 * g0 / m, rel=1e-14)          # d gamma0^2 / dE
    E = b.kinetic_eV
    for idx, key in ((3, "kappa_perp"), (4, "kappa_z")):
        vals = []
        for s in (1, -1):
            bb = I.Beam(**{**b.__dict__, "kinetic_eV": E + s * 1e3, "energy_slot": -1})
            vals.append(make(N=10, P=0, beam=bb).constants()[key])
        fd = (vals[0] - vals[1]) / 2e3
        assert d[idx, 1] == pytest.approx(fd, rel=1e-7), key


def test_energy_slot_leaves_values_and_other_derivatives():
    """Adding the energy as slot 7 of P = 8 changes neither the value part nor the seven lattice
    derivatives of a P = 7 run (up to the rounding of the dual quotient in E_z)."""
    lat = I.Lattice()
    o7 = make(N=1500, P=7, lattice=lat)
    o8 = make(N=1500, P=8, lattice=lat, beam=energy_beam(7))
    nrm = I.normals(41, 1500)
    s7, s8 = o7.beam_init(nrm), o8.beam_init(nrm)
    np.testing.assert_array_equal(s8[:, :, :8], s7)
    h7, _ = o7.run(s7, 20)
    h8, _ = o8.run(s8, 20)
    e7, e8 = o7.emittance(h7[-1]), o8.emittance(h8[-1])
    np.testing.assert_allclose(e8[:, :8], e7, rtol=1e-10, atol=1e-10 * np.abs(e7).max())
    assert np.abs(e8[:2, 8]).min() > 0


def test_fft_solve_matches_direct_sum_with_energy():
    """The Hockney FFT solve with the dual Green's term (phi_E += dG/dE * rho_0) against the
    brute-force direct sum on an 8^3 grid."""
    o = make(n=8, N=10, P=3, beam=energy_beam(1))
    rng = np.random.default_rng(5)
    rho = rng.standard_normal(o.grid_shape())
    geom = np.array([-1e-3, -1e-3, -1e-3, 2.5e-4, 3e-4, 2e-4])
    phi = o.solve(geom, rho)
    phid = o.solve_direct(geom, rho)
    np.testing.assert_allclose(phi, phid, rtol=1e-9, atol=1e-12 * np.abs(phid).max())
    # the energy channel differs from a plain convolution by (dG/dE) * rho_0 alone (a numpy FFT
    # convolution of the doubled-grid dG/dE with the zero-padded rho_0)
    o0 = make(n=8, N=10, P=3)
    phi0 = o0.solve(geom, rho)
    np.testing.assert_allclose(phi[[0, 1, 3]], phi0[[0, 1, 3]], rtol=1e-12, atol=1e-14 * np.abs(phi0).max())
    GE = o.green_denergy(geom)
    pad = np.zeros_like(GE)
    pad[:8, :8, :8] = rho[0]
    term = np.fft.irfftn(np.fft.rfftn(GE) * np.fft.rfftn(pad), s=GE.shape)[:8, :8, :8]
    assert np.abs(term).max() > 0
    np.testing.assert_allclose(phi[2] - phi0[2], term, rtol=0, atol=1e-4 * np.abs(term).max())


def test_energy_derivative_matches_central_fd_frozen_geometry():
    """d eps / dE of a whole period (energy in slot 0, lattice in slots 1-6) against central
    differences of value-only runs at frozen geometry; the best step of a sweep, as for the other
    parameters (the CIC response is only piecewise smooth)."""
    b = energy_beam(0)
    lat = I.Lattice(deriv_slot=(-1, 1, 2, 3, 4, 5, 6))
    o = make(n=16, N=3000, P=7, beam=b, lattice=lat)
    nrm = I.normals(42, o.N)
    st = o.beam_init(nrm)
    hist, geom = o.run(st, 20, geom_mode=1)
    d = o.emittance(hist[-1])[:3, 1]          # x, y and z: E_z reaches only the z plane
    E = b.kinetic_eV
    errs = []
    for hrel in (1e-4, 1e-5, 1e-6, 1e-7):
        h = hrel * E
        vals = []
        for ee in (E + h, E - h):
            bb = I.Beam(**{**b.__dict__, "kinetic_eV": ee, "energy_slot": -1})
            ov = make(n=16, N=o.N, P=0, beam=bb)
            sv = ov.beam_init(nrm)
            hv, _ = ov.run(sv, 20, geom=geom.copy(), geom_mode=2)
            vals.append(ov.emittance(hv[-1])[:3, 0])
        errs.append(np.abs((vals[0] - vals[1]) / (2 * h) - d))
    best = np.min(errs, axis=0)
    assert np.all(best < 1e-5 * np.abs(d)), (best, d)


def test_energy_derivative_of_the_longitudinal_drift_term():
    """At zero current the z map alone carries the energy through 1/gamma0^2: after one period
    dz/dE of a particle with delta != 0 equals L_period delta d(1/gamma0^2)/dE."""
    b = energy_beam(0, bunch_charge_C=0.0)
    lat = I.Lattice(deriv_slot=(-1,) * 7)
    o = make(n=16, N=400, P=1, beam=b, lattice=lat)
    st = o.beam_init(I.normals(43, o.N))
    z0, dl0, dz0 = st[4, :, 0].copy(), st[5, :, 0].copy(), st[4, :, 1].copy()
    o.run(st, 20)
    g0 = o.constants()["gamma0"]
    Lp = sum(lat.L)
    dinv = -2.0 / g0 ** 3 / b.mass_eV
    ddl0 = st[5, :, 1]                       # delta is not kicked at zero current
    np.testing.assert_allclose(st[5, :, 0], dl0, rtol=0, atol=0)
    pred = dz0 + Lp * (dl0 * dinv + ddl0 / g0 ** 2)
    np.testing.assert_allclose(st[4, :, 1], pred, rtol=1e-10, atol=1e-12 * np.abs(pred).max())
    assert math.isfinite(z0.sum())
