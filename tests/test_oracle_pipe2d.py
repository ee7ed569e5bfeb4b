"""Pins of the oracle's 2D conducting-pipe PIC (Sec. 4: bilinear deposit, sine-transform Poisson
solve with phi = 0 on the walls, central-difference field, the kick of H2 = K phi / 2).

- A single sine mode of the density is solved exactly: phi = rho / gamma_lm^2 (Eq. for phi^lm).
- A line charge against the exact Green's function of the grounded rectangle written as a single
  series in x with sinh factors in y (an independent route to the same boundary-value problem).
- A uniform round beam far from the walls: the kick is K x tau / r^2 inside (the classic perveance
  kick of the envelope equation), which fixes the normalisation of phi and the factor 2 pi K.
- Charge conservation, zero-current emittance conservation, and central finite differences of whole
  runs against the dual derivatives (lattice parameters and the beam current).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2511_21839_gb300 import inputs as I


def cfg(P=0, n=32, N=1, I_A=100.0, a=0.02, b=0.02, lat=None, current_slot=-1, beta=(1.0, 1.0)):
    lat = lat or I.Lattice()
    return dict(P=P, nx=n, ny=n, N=N, a=a, b=b, kinetic_eV=1e9, mass_eV=I.PROTON_MASS_EV, charge_e=1.0,
                current_A=I_A, eps_n=[1e-6, 1e-6], alpha=[0.0, 0.0], beta=list(beta), L=list(lat.L),
                g=list(lat.g), kicks=list(lat.kicks),
                lat_slot=[s if 0 <= s < P else -1 for s in lat.deriv_slot], current_slot=current_slot)


@pytest.mark.parametrize("l,m", [(1, 1), (3, 2), (7, 11)])
def test_single_sine_mode_is_solved_exactly(l, m):
    o = oracle.Oracle2D(**cfg(n=32, a=0.03, b=0.02))
    i = np.arange(33)
    mode = np.sin(np.pi * m * i / 32)[:, None] * np.sin(np.pi * l * i / 32)[None, :]   # [y][x]
    phi = o.solve(mode[None])
    g2 = (l * np.pi / 0.03) ** 2 + (m * np.pi / 0.02) ** 2
    np.testing.assert_allclose(phi[0], mode / g2, atol=1e-12 * np.abs(mode / g2).max())


def rect_green(x, y, x0, y0, a, b, terms=400):
    """Potential of a unit line charge (lap phi = -delta) at (x0, y0) in the grounded a x b rectangle:
    phi = sum_l (2 / a) sin(al x0) sin(al x) sinh(al y<) sinh(al (b - y>)) / (al sinh(al b))."""
    s = 0.0
    ylo, yhi = min(y, y0), max(y, y0)
    for l in range(1, terms + 1):
        al = l * math.pi / a
        # sinh(al ylo) sinh(al (b - yhi)) / sinh(al b), written with exponentials that do not overflow
        g = (math.exp(al * (ylo - yhi)) - math.exp(-al * (ylo + yhi)) - math.exp(al * (ylo + yhi - 2 * b))
             + math.exp(-al * (2 * b - yhi + ylo))) / (2.0 * (1.0 - math.exp(-2 * al * b)))
        s += 2.0 / a * math.sin(al * x0) * math.sin(al * x) * g / al
    return s


def test_line_charge_matches_the_rectangle_green_function():
    n, a, b = 64, 0.03, 0.02
    o = oracle.Oracle2D(**cfg(n=n, a=a, b=b))
    hx, hy = a / n, b / n
    i0, j0 = 24, 40                                  # a node: the bilinear weight is 1 there
    rho = np.zeros((1, n + 1, n + 1))
    rho[0, j0, i0] = 1.0 / (hx * hy)
    phi = o.solve(rho)[0]
    errs = []
    for (i, j) in [(8, 8), (40, 12), (56, 56), (24, 52), (10, 40)]:
        ref = rect_green(i * hx, j * hy, i0 * hx, j0 * hy, a, b)
        errs.append(abs(phi[j, i] - ref) / abs(ref))
    assert max(errs) < 0.02, errs


def quiet_disk(r, h):
    xs = np.arange(-r, r + h, h) + 0.37 * h
    X, Y = np.meshgrid(xs, xs + 0.21 * h - 0.37 * h)
    m = X ** 2 + Y ** 2 < r * r
    return X[m], Y[m]


def test_uniform_beam_kick_is_the_perveance_kick():
    r = 2e-3
    X, Y = quiet_disk(r, r / 60)
    N = X.size
    o = oracle.Oracle2D(**cfg(n=128, N=N, a=0.04, b=0.04, I_A=100.0))
    st = np.zeros((4, N, 1))
    st[0, :, 0], st[2, :, 0] = X, Y
    E = o.field(o.solve(o.deposit(st)))
    before = st.copy()
    o.kick(st, E, 0)                                  # a D1 kick: tau = 0.5 / 4
    tau = 0.5 / 4
    K = o.constants()["K"]
    inner = X ** 2 + Y ** 2 < (0.6 * r) ** 2
    for d, c in ((0, X), (1, Y)):
        dp = st[2 * d + 1, :, 0] - before[2 * d + 1, :, 0]
        slope = np.sum(dp[inner] * c[inner]) / np.sum(c[inner] ** 2)
        assert slope == pytest.approx(K * tau / r ** 2, rel=0.03), d


def test_deposit_conserves_the_normalised_charge():
    P, N = 7, 3000
    o = oracle.Oracle2D(**cfg(P=P, n=32, N=N))
    st = o.beam_init(I.normals(3, N)[:4])
    rho = o.deposit(st)
    h = 0.02 / 32
    assert rho[0].sum() * h * h == pytest.approx(1.0, rel=1e-13)
    assert np.abs(rho[1:].sum(axis=(1, 2))).max() * h * h < 1e-12


def test_zero_current_conserves_emittance():
    P, N = 7, 2000
    o = oracle.Oracle2D(**cfg(P=P, n=32, N=N, I_A=0.0, beta=(1.8, 1.8)))
    st = o.beam_init(I.normals(4, N)[:4])
    e0 = o.emittance(o.moments(st))
    h = o.run(st, 20)
    e1 = o.emittance(h[-1])
    np.testing.assert_allclose(e1[:, 0], e0[:, 0], rtol=1e-12)
    assert np.abs(e1[:, 1:]).max() < 1e-12 * e0[:, 0].max()


def test_whole_run_derivatives_match_central_fd():
    """Lattice slots 1..6 and the beam current in slot 0 (fixed pipe grid: no frozen geometry needed);
    the best step of a sweep, as the CIC response is piecewise smooth."""
    P, N = 7, 2000
    lat = I.Lattice(deriv_slot=(-1, 1, 2, 3, 4, 5, 6))
    base = cfg(P=P, n=32, N=N, I_A=100.0, beta=(1.8, 1.8), lat=lat, current_slot=0)
    nrm = I.normals(5, N)[:4]
    o = oracle.Oracle2D(**base)
    st = o.beam_init(nrm)
    d = o.emittance(o.run(st, 20)[-1])

    def value(**over):
        kw = dict(base, P=0, current_slot=-1)
        kw["lat_slot"] = [-1] * 7
        kw.update(over)
        ov = oracle.Oracle2D(**kw)
        sv = ov.beam_init(nrm)
        return ov.emittance(ov.run(sv, 20)[-1])[:, 0]

    params = [("current_A", None, 100.0)] + [("lat", j, v) for j, v in enumerate(lat.params())][1:]
    slots = [0] + list(range(1, 7))
    scale = np.abs(d[:, 1:]).max(axis=1)
    for (kind, j, v), s in zip(params, slots):
        best = None
        for hrel in (1e-3, 1e-4, 1e-5, 1e-6):
            h = hrel * abs(v)
            if kind == "current_A":
                fp, fm = value(current_A=v + h), value(current_A=v - h)
            else:
                pp, pm = np.array(lat.params(), dtype=float), np.array(lat.params(), dtype=float)
                pp[j] += h
                pm[j] -= h
                lp, lm = I.Lattice.from_params(pp), I.Lattice.from_params(pm)
                fp = value(L=list(lp.L), g=list(lp.g))
                fm = value(L=list(lm.L), g=list(lm.g))
            err = np.abs((fp - fm) / (2 * h) - d[:, s + 1])
            best = err if best is None else np.minimum(best, err)
        assert np.all(best < 1e-4 * scale), (kind, j, best / scale)
