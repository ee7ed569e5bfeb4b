"""Pins of the oracle's PIC stages and whole-run properties against the paper and the mathematics."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2511_21839_gb300 import inputs as I

EPS0 = 8.8541878128e-12
QE = 1.602176634e-19
CL = 299792458.0


def make(n=16, N=1000, P=7, q=None, lattice=None, beam=None, wname="fodo_10k_32"):
    w = I.workload(wname)
    kw = I.orc_kwargs(w, n_particles=N, grid=(n, n, n) if isinstance(n, int) else n, n_deriv=P,
                      lattice=lattice, beam=beam)
    if q is not None:
        kw["bunch_charge_C"] = q
    return oracle.Oracle(**kw)


def beam_state(o, seed=1):
    return o.beam_init(I.normals(seed, o.N))


# ---------------------------------------------------------------- constants

def test_reference_particle_constants():
    o = make()
    c = o.constants()
    mp = I.PROTON_MASS_EV
    E = 1e9 + mp
    pc = math.sqrt(E * E - mp * mp)                       # eV
    assert c["gamma0"] == pytest.approx(E / mp, rel=1e-15)
    assert c["beta0"] == pytest.approx(pc / E, rel=1e-14)
    assert c["brho"] == pytest.approx(pc / CL, rel=1e-14)  # T m for unit charge
    assert c["p0"] == pytest.approx(pc * QE / CL, rel=1e-14)


# ---------------------------------------------------------------- beam init

def test_beam_init_moments_and_twiss_seeds():
    w = I.workload("fodo_10k_32")
    beam = I.default_beam(13)
    o = make(N=2000, P=13, beam=beam)
    nrm = I.normals(3, o.N)
    st = o.beam_init(nrm)
    scale = np.abs(st).max(axis=1)
    assert np.all(np.abs(st.mean(axis=1)) <= 1e-14 * scale)
    g, b, _ = I.relativistic()
    eps = 1e-6 / (g * b)
    bx = beam.beta[0]
    u1 = nrm[0] - nrm[0].mean()
    # x = sqrt(eps beta) u1 - mean, exactly
    np.testing.assert_allclose(st[0, :, 0], math.sqrt(eps * bx) * nrm[0] - np.mean(math.sqrt(eps * bx) * nrm[0]),
                               rtol=0, atol=1e-17)
    # derivative channels by complex step of the same closed form
    h = 1e-40

    def xp(alpha, beta, e):
        x = np.sqrt(e * beta) * nrm[0]
        p = np.sqrt(e / beta) * (nrm[1] - alpha * nrm[0])
        return x - x.mean(), p - p.mean()

    base = [0.0, bx, eps]
    for j, slot in enumerate(beam.twiss_slot[:3]):
        arg = [complex(v) for v in base]
        arg[j] += 1j * h * (1.0 if j != 2 else eps)
        x, p = xp(*arg)
        scale = 1.0 if j != 2 else eps
        np.testing.assert_allclose(st[0, :, slot + 1] * scale, x.imag / h, rtol=1e-12, atol=1e-22)
        np.testing.assert_allclose(st[1, :, slot + 1] * scale, p.imag / h, rtol=1e-12, atol=1e-22)
    assert np.all(st[2:4, :, 1:4] == 0)     # lattice slots start at zero


# ---------------------------------------------------------------- geometry + deposit

def test_geometry_margins():
    o = make(n=(16, 32, 8), N=3000)
    st = beam_state(o)
    geom = o.geometry(st)
    for d, n in enumerate((16, 32, 8)):
        u = (st[2 * d, :, 0] - geom[d]) / geom[3 + d]
        assert u.min() == pytest.approx(1.5, abs=1e-9)
        assert u.max() == pytest.approx(n - 2.5, abs=1e-9)


def test_deposit_single_particle_weights():
    o = make(n=8, N=1, P=2)
    st = np.zeros(o.state_shape())
    pos = (0.37e-3, -0.21e-3, 0.05e-3)
    for d in range(3):
        st[2 * d, 0, 0] = pos[d]
    st[0, 0, 1] = 1.0           # dx/dp1
    st[4, 0, 2] = -2.0          # dz/dp2
    geom = np.array([-1e-3, -1.1e-3, -0.9e-3, 0.3e-3, 0.35e-3, 0.25e-3])
    rho = o.deposit(st, geom)
    qm = o.constants()["q_macro"]
    u = [(pos[d] - geom[d]) / geom[3 + d] for d in range(3)]
    i = [int(math.floor(v)) for v in u]
    f = [v - k for v, k in zip(u, i)]
    exp = np.zeros((3, 8, 8, 8))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                wx = (1 - f[0], f[0])[a]
                wy = (1 - f[1], f[1])[b]
                wz = (1 - f[2], f[2])[c]
                node = (i[2] + c, i[1] + b, i[0] + a)
                exp[0][node] = qm * wx * wy * wz
                exp[1][node] = qm * (1 if a else -1) / geom[3] * wy * wz
                exp[2][node] = qm * -2.0 * (1 if c else -1) / geom[5] * wx * wy
    np.testing.assert_allclose(rho, exp, rtol=1e-13, atol=1e-30)


def test_deposit_charge_conservation_and_fd():
    o = make(n=16, N=4000, P=7)
    st = beam_state(o)
    st[:, :, 1:] = np.random.default_rng(2).standard_normal(st[:, :, 1:].shape) * 1e-5
    geom = o.geometry(st)
    rho = o.deposit(st, geom)
    qm = o.constants()["q_macro"]
    assert rho[0].sum() == pytest.approx(o.N * qm, rel=1e-14)
    np.testing.assert_allclose(rho[1:].sum(axis=(1, 2, 3)), 0, atol=1e-14 * o.N * qm)
    # channel k = derivative of the value deposit along the particles' derivative directions,
    # exact (CIC is linear inside a cell) for displacements that cross no cell edge
    o0 = make(n=16, N=4000, P=0)
    k = 3
    t = 1e-6
    sp = st[:, :, :1].copy(); sp[..., 0] += t * st[:, :, k]
    sm = st[:, :, :1].copy(); sm[..., 0] -= t * st[:, :, k]
    fd = (o0.deposit(np.ascontiguousarray(sp), geom)[0] - o0.deposit(np.ascontiguousarray(sm), geom)[0]) / (2 * t)
    np.testing.assert_allclose(rho[k], fd, rtol=0, atol=1e-7 * np.abs(rho[k]).max())


# ---------------------------------------------------------------- field + gather

def test_field_exact_for_quadratic_potential():
    o = make(n=(8, 16, 8), N=1, P=1)
    geom = np.array([-1e-3, -2e-3, -3e-3, 1e-4, 2e-4, 3e-4])
    g0 = o.constants()["gamma0"]
    nz, ny, nx = 8, 16, 8
    X = geom[0] + geom[3] * np.arange(nx)
    Y = geom[1] + geom[4] * np.arange(ny)
    Z = (geom[2] + geom[5] * np.arange(nz)) * g0       # rest-frame z
    Zg, Yg, Xg = np.meshgrid(Z, Y, X, indexing="ij")
    phi = np.stack([3 * Xg ** 2 - Yg * Zg + 2 * Xg, 5 * Zg ** 2 + Xg * Yg])
    E = o.field(geom, phi)
    exp = np.stack([np.stack([-(6 * Xg + 2), Zg, Yg]), np.stack([-Yg, -Xg, -10 * Zg])])
    exp = exp.transpose(1, 0, 2, 3, 4)      # [3][C]
    inner = (slice(None), slice(None), slice(1, -1), slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(E[inner], exp[inner], rtol=1e-9, atol=1e-9 * np.abs(exp).max())
    assert np.all(E[:, :, 0] == 0) and np.all(E[:, :, :, :, -1] == 0)


def test_gather_exact_for_linear_field():
    o = make(n=16, N=500, P=4)
    st = beam_state(o)
    st[:, :, 1:] = np.random.default_rng(4).standard_normal(st[:, :, 1:].shape) * 1e-4
    geom = o.geometry(st)
    X = geom[0] + geom[3] * np.arange(16)
    Zg, Yg, Xg = np.meshgrid(geom[2] + geom[5] * np.arange(16), geom[1] + geom[4] * np.arange(16), X, indexing="ij")
    A = np.array([[1.0, 2e3, -1e3, 5e2], [-2.0, 3e2, 4e3, -1e3], [0.5, -7e2, 1e2, 2e3]])
    E = np.zeros((3, o.C, 16, 16, 16))
    for d in range(3):
        E[d, 0] = A[d, 0] + A[d, 1] * Xg + A[d, 2] * Yg + A[d, 3] * Zg
        E[d, 2] = 7.0 * A[d, 1] * Xg       # a derivative channel that is itself a field
    Ep = o.gather(st, geom, E)
    x, y, z = st[0], st[2], st[4]
    for d in range(3):
        v = A[d, 0] + A[d, 1] * x[:, 0] + A[d, 2] * y[:, 0] + A[d, 3] * z[:, 0]
        np.testing.assert_allclose(Ep[d, :, 0], v, rtol=1e-12, atol=1e-12 * np.abs(v).max())
        for k in range(1, o.C):
            dk = A[d, 1] * x[:, k] + A[d, 2] * y[:, k] + A[d, 3] * z[:, k]
            if k == 2:
                dk = dk + 7.0 * A[d, 1] * x[:, 0]
            np.testing.assert_allclose(Ep[d, :, k], dk, rtol=1e-10, atol=1e-10 * np.abs(dk).max())


# ---------------------------------------------------------------- maps (zero current)

def _lens(k, L):
    if k == 0:
        return np.array([[1, L], [0, 1]], dtype=complex)
    w = np.sqrt(complex(k))
    return np.array([[np.cos(w * L), np.sin(w * L) / w], [-w * np.sin(w * L), np.cos(w * L)]])


def _fodo(p, brho, plane):
    s = 1 if plane == 0 else -1
    ks = (0, s * p[2] / brho, 0, s * p[5] / brho, 0)
    Ls = (p[0], p[1], p[3], p[4], p[6])
    M = np.eye(2, dtype=complex)
    for k, L in zip(ks, Ls):
        M = _lens(k, L) @ M
    return M


def test_half_maps_match_thick_lens_and_complex_step():
    o = make(P=7)
    brho = o.constants()["brho"]
    p = np.array(I.Lattice().params(), dtype=complex)
    kick = 4                       # first QF kick: element QF, tau = L_QF / 2
    m = o.half_map(kick)
    h = 1e-30
    for plane in range(2):
        s = 1 if plane == 0 else -1

        def half(pp):
            return _lens(s * pp[2] / brho, pp[1] / 2 / 2)
        M = half(p)
        np.testing.assert_allclose(m[plane, :, 0], M.real.ravel(), rtol=1e-14)
        for k in range(7):
            pp = p.copy(); pp[k] += 1j * h
            np.testing.assert_allclose(m[plane, :, k + 1], (half(pp).imag / h).ravel(), rtol=1e-12, atol=1e-16)


@pytest.fixture(scope="module")
def zero_current_run():
    o = make(n=16, N=3000, P=7, q=0.0)
    st0 = beam_state(o, 7)
    st = st0.copy()
    hist, _ = o.run(st, 20)
    return o, st0, st, hist


def test_zero_current_matches_fodo_matrix_and_derivatives(zero_current_run):
    o, st0, st, _ = zero_current_run
    brho = o.constants()["brho"]
    g0 = o.constants()["gamma0"]
    p = np.array(I.Lattice().params(), dtype=complex)
    h = 1e-30
    for plane in range(2):
        M = _fodo(p, brho, plane).real
        u0, p0 = st0[2 * plane, :, 0], st0[2 * plane + 1, :, 0]
        np.testing.assert_allclose(st[2 * plane, :, 0], M[0, 0] * u0 + M[0, 1] * p0, rtol=1e-12, atol=1e-18)
        np.testing.assert_allclose(st[2 * plane + 1, :, 0], M[1, 0] * u0 + M[1, 1] * p0, rtol=1e-12, atol=1e-18)
        for k in range(7):
            pp = p.copy(); pp[k] += 1j * h
            dM = _fodo(pp, brho, plane).imag / h
            np.testing.assert_allclose(st[2 * plane, :, k + 1], dM[0, 0] * u0 + dM[0, 1] * p0, rtol=1e-10,
                                       atol=1e-16)
    # longitudinal: z += L_total delta / gamma0^2, d z / d L_e = delta / gamma0^2
    Ltot = sum(I.LENGTHS)
    np.testing.assert_allclose(st[4, :, 0], st0[4, :, 0] + Ltot * st0[5, :, 0] / g0 ** 2, rtol=1e-12, atol=1e-18)
    for slot in (0, 1, 3, 4, 6):
        np.testing.assert_allclose(st[4, :, slot + 1], st0[5, :, 0] / g0 ** 2, rtol=1e-12, atol=1e-20)


def test_zero_current_emittance_conserved(zero_current_run):
    o, st0, st, hist = zero_current_run
    e0 = o.emittance(o.moments(st0))
    e1 = o.emittance(hist[-1])
    np.testing.assert_allclose(e1[:, 0], e0[:, 0], rtol=1e-12)
    assert np.all(np.abs(e1[:2, 1:]) < 1e-11 * e0[:2, :1])


def test_zero_current_twiss_transport_eq5(zero_current_run):
    o, st0, st, hist = zero_current_run
    brho = o.constants()["brho"]
    for plane in range(2):
        M = _fodo(np.array(I.Lattice().params(), dtype=complex), brho, plane).real
        (m11, m12), (m21, m22) = M
        T = np.array([[m11 ** 2, -2 * m11 * m12, m12 ** 2],
                      [-m11 * m21, m11 * m22 + m12 * m21, -m12 * m22],
                      [m21 ** 2, -2 * m21 * m22, m22 ** 2]])

        def twiss(s):
            u, p = s[2 * plane, :, 0], s[2 * plane + 1, :, 0]
            a, b, c = np.var(u), np.mean((u - u.mean()) * (p - p.mean())), np.var(p)
            e = math.sqrt(a * c - b * b)
            return np.array([a / e, -b / e, c / e])
        np.testing.assert_allclose(twiss(st), T @ twiss(st0), rtol=1e-10)


# ---------------------------------------------------------------- P2: values independent of derivatives

def test_value_part_equals_value_only_run():
    o7 = make(n=16, N=2000, P=7)
    o0 = make(n=16, N=2000, P=0)
    nrm = I.normals(9, 2000)
    s7 = o7.beam_init(nrm)
    s0 = o0.beam_init(nrm)
    h7, g7 = o7.run(s7, 6)
    h0, g0 = o0.run(s0, 6)
    np.testing.assert_array_equal(s7[:, :, 0], s0[:, :, 0])
    np.testing.assert_array_equal(h7[..., 0], h0[..., 0])


# ---------------------------------------------------------------- P6: physics of the field

def _quiet_ellipsoid(a, b, c, d):
    """Points of a cubic lattice of spacing d inside the ellipsoid (x/a)^2+(y/b)^2+(z/c)^2 < 1."""
    xs = np.arange(-a, a + d, d) + 0.5 * d * 0.37
    ys = np.arange(-b, b + d, d) + 0.5 * d * 0.23
    zs = np.arange(-c, c + d, d) + 0.5 * d * 0.11
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    m = (X / a) ** 2 + (Y / b) ** 2 + (Z / c) ** 2 < 1
    return X[m], Y[m], Z[m]


def _ellipsoid_factor(a, b, c, axis):
    """(abc/2) int_0^inf ds / ((a_axis^2 + s) sqrt((a^2+s)(b^2+s)(c^2+s))), scale-free; with
    s = t / (1 - t) the range becomes [0, 1)."""
    m = max(a, b, c)
    a, b, c = a / m, b / m, c / m
    ax = (a, b, c)

    def f(t):
        s = t / (1.0 - t)
        return 1.0 / ((ax[axis] ** 2 + s) * math.sqrt((a * a + s) * (b * b + s) * (c * c + s))) / (1.0 - t) ** 2
    v, _ = integrate.quad(f, 0, 1, epsabs=0, epsrel=1e-13, limit=200)
    return a * b * c / 2 * v


@pytest.mark.parametrize("axes", [(1e-3, 1e-3, 1e-3), (1e-3, 1.5e-3, 2.5e-3)])
def test_uniform_ellipsoid_linear_field(axes):
    """Interior field of a uniformly charged ellipsoid (rest frame) is linear with the
    depolarisation factors; a sphere gives rho r / (3 eps0)."""
    o_probe = make(n=32, N=1, P=0)
    g0 = o_probe.constants()["gamma0"]
    a, b, c = axes
    X, Y, Zr = _quiet_ellipsoid(a, b, c, 0.04e-3)
    N = X.size
    Q = 1e-10
    o = make(n=32, N=N, P=0, q=Q)
    st = np.zeros((6, N, 1))
    st[0, :, 0], st[2, :, 0], st[4, :, 0] = X, Y, Zr / g0     # lab z = rest z / gamma0
    geom = o.geometry(st)
    rho_rest = Q / (4.0 / 3.0 * math.pi * a * b * c)
    Ep = o.gather(st, geom, o.field(geom, o.solve(geom, o.deposit(st, geom))))
    inner = (X / a) ** 2 + (Y / b) ** 2 + (Zr / c) ** 2 < 0.5 ** 2
    for d, coordv in enumerate((X, Y, Zr)):
        exact = rho_rest / EPS0 * _ellipsoid_factor(a, b, c, d) * coordv
        err = np.abs(Ep[d, inner, 0] - exact[inner]).max() / np.abs(exact[inner]).max()
        assert err < 0.03, (d, err)
        if a == b == c:
            np.testing.assert_allclose(_ellipsoid_factor(a, b, c, d), 1.0 / 3.0, rtol=1e-10)


def test_kick_matches_paper_perveance_for_long_beam():
    """Long uniform beam: the transverse kick per unit length approaches K x / a^2 with the
    2D perveance K = q I / (2 pi eps0 p0 v0^2 gamma0^2) of Sec. 4 (H2 = K phi / 2)."""
    a, clab = 1e-3, 30e-3
    o_probe = make(n=32, N=1, P=0)
    c = o_probe.constants()
    g0, b0 = c["gamma0"], c["beta0"]
    crest = clab * g0
    X, Y, Zr = _quiet_ellipsoid(a, a, crest, 0.05e-3 * np.array(1.0))
    # thin out along z to keep the sample small while staying uniform
    keep = np.ones(X.size, dtype=bool)
    N = int(keep.sum())
    Q = 1e-10
    o = make(n=(32, 32, 64), N=N, P=0, q=Q)
    st = np.zeros((6, N, 1))
    st[0, :, 0], st[2, :, 0], st[4, :, 0] = X[keep], Y[keep], Zr[keep] / g0
    geom = o.geometry(st)
    E = o.field(geom, o.solve(geom, o.deposit(st, geom)))
    before = st.copy()
    kick = 0                    # a D1 kick: tau = 0.5 / 4
    o.kick(st, geom, E, kick)
    tau = 0.5 / 4
    dpx = st[1, :, 0] - before[1, :, 0]
    x = before[0, :, 0]
    zc = np.abs(before[4, :, 0]) < 0.1 * clab
    inner = zc & (X ** 2 + Y ** 2 < (0.5 * a) ** 2)
    lam0 = 3 * Q / (4 * clab)                       # centre line density (lab) of a uniform ellipsoid
    v0 = b0 * CL
    I_peak = lam0 * v0
    p0 = c["p0"]
    K = QE * I_peak / (2 * math.pi * EPS0 * p0 * v0 ** 2 * g0 ** 2)
    # finite length: exact ellipsoid factor over its infinite-cylinder limit (1/2)
    corr = _ellipsoid_factor(a, a, crest, 0) / 0.5
    pred = K * x[inner] * tau / a ** 2 * corr * (1 - (0.0) ** 2)
    slope = np.sum(dpx[inner] * x[inner]) / np.sum(x[inner] ** 2)
    pred_slope = K * tau / a ** 2 * corr
    assert slope == pytest.approx(pred_slope, rel=0.03)


def test_kick_constants_closed_form():
    """Kick coefficients from the Lorentz force alone, recomputed here from CODATA: over a path
    tau (time tau / v0) the longitudinal field, which a boost along z leaves unchanged, changes
    p_z by q E_z tau / v0, so delta = dp / p0 changes by q E_z,rest tau / (p0 v0); the transverse
    electric and magnetic forces of the co-moving bunch combine to q E_perp,lab / gamma0^2 =
    q E_perp,rest / gamma0, so p_x / p0 changes by q E_perp,rest tau / (gamma0 p0 v0) (Sec. 4, map
    M2, the Coulomb and vector potentials combined)."""
    o = make()
    c = o.constants()
    mp = I.PROTON_MASS_EV
    E = 1e9 + mp
    pc = math.sqrt(E * E - mp * mp)
    p0 = pc * QE / CL                                     # kg m / s
    v0 = pc / E * CL
    g0 = E / mp
    assert c["kappa_z"] == pytest.approx(QE / (p0 * v0), rel=1e-13)
    assert c["kappa_perp"] == pytest.approx(QE / (g0 * p0 * v0), rel=1e-13)
    assert c["kappa_perp"] / c["kappa_z"] == pytest.approx(1.0 / g0, rel=1e-14)


def test_longitudinal_kick_inside_uniform_sphere():
    """The energy kick of Sec. 4's map M2 inside a uniformly charged sphere (rest frame): the
    rest-frame field E_z = rho z_rest / (3 eps0) is exact inside, so delta changes by
    q tau rho z_rest / (3 eps0 p0 v0), with p0 and v0 of the reference particle. An extra factor
    1/gamma0 (as in the transverse kick) or 1/beta0 in the longitudinal coefficient fails this by
    50 % or 14 %."""
    o_probe = make(n=32, N=1, P=0)
    c0 = o_probe.constants()
    g0 = c0["gamma0"]
    a = 1e-3
    X, Y, Zr = _quiet_ellipsoid(a, a, a, 0.04e-3)
    N = X.size
    Q = 1e-10
    o = make(n=32, N=N, P=0, q=Q)
    st = np.zeros((6, N, 1))
    st[0, :, 0], st[2, :, 0], st[4, :, 0] = X, Y, Zr / g0     # lab z = rest z / gamma0
    geom = o.geometry(st)
    E = o.field(geom, o.solve(geom, o.deposit(st, geom)))
    before = st.copy()
    o.kick(st, geom, E, 0)                                   # a D1 kick: tau = 0.5 m / 4
    tau = 0.5 / 4
    ddelta = st[5, :, 0] - before[5, :, 0]
    assert np.array_equal(st[4], before[4]) and np.array_equal(st[0], before[0])
    inner = X ** 2 + Y ** 2 + Zr ** 2 < (0.5 * a) ** 2
    mp = I.PROTON_MASS_EV
    Etot = 1e9 + mp
    pc = math.sqrt(Etot * Etot - mp * mp)
    p0 = pc * QE / CL
    v0 = pc / Etot * CL
    rho_rest = Q / (4.0 / 3.0 * math.pi * a ** 3)
    pred_slope = QE * tau * rho_rest / (3 * EPS0 * p0 * v0)   # d(delta) / d(z_rest)
    slope = np.sum(ddelta[inner] * Zr[inner]) / np.sum(Zr[inner] ** 2)
    assert slope == pytest.approx(pred_slope, rel=0.03)
    # and the transverse kick of the same sphere, for the ratio of the two coefficients
    dpx = st[1, :, 0] - before[1, :, 0]
    slope_x = np.sum(dpx[inner] * X[inner]) / np.sum(X[inner] ** 2)
    assert slope_x / slope == pytest.approx(1.0 / g0, rel=0.03)


# ---------------------------------------------------------------- P8: emittance of a constructed ensemble

def test_emittance_constructed_ensemble():
    o = make(N=4, P=2)
    a, b = 2e-3, 3e-4
    st = np.zeros((6, 4, 3))
    st[0, :, 0] = [a, -a, 0, 0]
    st[0, :, 1] = [1, -1, 0, 0]            # dx/da
    st[1, :, 0] = [0, 0, b, -b]
    st[1, :, 2] = [0, 0, 1, -1]            # dpx/db
    st[2, :, 0] = [1e-3, 2e-3, 4e-3, 5e-3]  # y plane: a shifted, correlated set
    st[3, :, 0] = [1e-4, 3e-4, 2e-4, 6e-4]
    e = o.emittance(o.moments(st))
    np.testing.assert_allclose(e[0], [a * b / 2, b / 2, a / 2], rtol=1e-14)
    y, py = st[2, :, 0], st[3, :, 0]
    cov = np.cov(np.vstack([y, py]), bias=True)
    assert e[1, 0] == pytest.approx(math.sqrt(np.linalg.det(cov)), rel=1e-12)


# ---------------------------------------------------------------- P7: derivatives vs central FD

@pytest.fixture(scope="module")
def fd_case():
    o = make(n=16, N=3000, P=7)
    nrm = I.normals(21, o.N)
    st = o.beam_init(nrm)
    hist, geom = o.run(st, 20, geom_mode=1)
    eps = o.emittance(hist[-1])[:2]
    return o, nrm, geom, eps


def _eps_value_only(params, nrm, geom, beam=None, n=16):
    lat = I.Lattice.from_params(params)
    o = make(n=n, N=nrm.shape[1], P=0, lattice=lat, beam=beam)
    st = o.beam_init(nrm)
    hist, _ = o.run(st, 20, geom=geom.copy(), geom_mode=2)
    return o.emittance(hist[-1])[:2, 0]


def test_derivatives_match_central_fd_frozen_geometry(fd_case):
    o, nrm, geom, eps = fd_case
    base = np.array(I.Lattice().params())
    best = np.zeros((2, 7))
    for k in range(7):
        errs = []
        for hrel in (1e-4, 1e-5, 1e-6, 1e-7):
            h = hrel * abs(base[k])
            pp, pm = base.copy(), base.copy()
            pp[k] += h
            pm[k] -= h
            fd = (_eps_value_only(pp, nrm, geom) - _eps_value_only(pm, nrm, geom)) / (2 * h)
            errs.append(np.abs(fd - eps[:, k + 1]))
        best[:, k] = np.min(errs, axis=0)
    # The value of a CIC PIC run is only piecewise smooth in the parameters (a particle crossing a
    # cell edge is a kink), so central FD converges to the dual derivative only in a window of h
    # between the kink (large h) and rounding (small h) errors; the best h of the sweep is taken.
    scale = np.abs(eps[:, 1:]).max(axis=1, keepdims=True)
    assert (best / scale).max() < 1e-5, best / scale
    denom = np.maximum(np.abs(eps[:, 1:]), 1e-3 * scale)
    assert (best / denom).max() < 1e-3, best / denom


def test_twiss_derivatives_match_central_fd():
    beam = I.default_beam(13)
    o = make(n=16, N=2000, P=13, beam=beam)
    nrm = I.normals(22, o.N)
    st = o.beam_init(nrm)
    hist, geom = o.run(st, 20, geom_mode=1)
    eps = o.emittance(hist[-1])[:2]
    g, b, _ = I.relativistic()
    epsg = 1e-6 / (g * b)
    names = [("alpha", 0, 1.0), ("beta", 0, beam.beta[0]), ("eps", 0, epsg),
             ("alpha", 1, 1.0), ("beta", 1, beam.beta[1]), ("eps", 1, epsg)]
    for j, (kind, pl, scale) in enumerate(names):
        h = 1e-6 * scale
        vals = []
        for sgn in (1, -1):
            bb = I.default_beam(0)
            alpha, beta, epsn = list(bb.alpha), list(bb.beta), list(bb.eps_n)
            if kind == "alpha":
                alpha[pl] += sgn * h
            elif kind == "beta":
                beta[pl] += sgn * h
            else:
                epsn[pl] = (epsg + sgn * h) * g * b
            bb.alpha, bb.beta, bb.eps_n = tuple(alpha), tuple(beta), tuple(epsn)
            vals.append(_eps_value_only(I.Lattice().params(), nrm, geom, beam=bb))
        fd = (vals[0] - vals[1]) / (2 * h)
        ad = eps[:, 8 + j]
        scale = np.abs(eps[:, 8:]).max(axis=1)
        assert np.all(np.abs(fd - ad) / scale < 1e-5), (kind, pl, fd, ad)


# ---------------------------------------------------------------- P9: second-order splitting

def test_split_integrator_second_order():
    base = I.Lattice()
    finals = []
    for mult in (1, 2, 4, 8):
        lat = I.Lattice(kicks=tuple(k * mult for k in base.kicks))
        o = make(n=16, N=1500, P=0, lattice=lat, q=20 * I.default_beam().bunch_charge_C)
        st = o.beam_init(I.normals(31, o.N))
        o.run(st, 20 * mult)
        finals.append(st[:, :, 0].copy())
    e = [np.sqrt(np.mean((finals[i] - finals[-1]) ** 2)) for i in range(3)]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    # second order with the finest run as reference: e_i ~ tau_i^2 - tau_8^2, so the ratios
    # are (1 - 1/64) / (1/4 - 1/64) = 4.2 and (1/4 - 1/64) / (1/16 - 1/64) = 5
    assert abs(r1 - 4.2) < 0.8 and abs(r2 - 5.0) < 1.2, (e, r1, r2)


# ---------------------------------------------------------------- the bunch charge as an AD variable

def test_charge_channel_of_the_deposit_is_rho_over_q():
    """With the bunch charge Q in slot 0 the deposit is linear in Q: channel 1 of rho equals
    rho_0 / Q at every node (Sec. 4: the beam current as a dual input)."""
    w = I.workload("fodo_10k_32")
    b = I.Beam(**{**w.beam.__dict__, "charge_slot": 0})
    lat = I.Lattice(deriv_slot=(-1, 1, 2, 3, 4, 5, 6))
    o = make(n=16, N=2000, P=7, beam=b, lattice=lat)
    st = o.beam_init(I.normals(23, o.N))
    geom = o.geometry(st)
    rho = o.deposit(st, geom)
    q = b.bunch_charge_C
    np.testing.assert_allclose(rho[1], rho[0] / q, rtol=1e-13, atol=1e-12 * np.abs(rho[0] / q).max())


def test_charge_derivative_matches_central_fd_frozen_geometry():
    """d eps / dQ of a whole period against central differences of value-only runs at frozen
    geometry (best step of a sweep, as for the lattice parameters)."""
    w = I.workload("fodo_10k_32")
    b = I.Beam(**{**w.beam.__dict__, "charge_slot": 0})
    lat = I.Lattice(deriv_slot=(-1, 1, 2, 3, 4, 5, 6))
    o = make(n=16, N=3000, P=7, beam=b, lattice=lat)
    nrm = I.normals(24, o.N)
    st = o.beam_init(nrm)
    hist, geom = o.run(st, 20, geom_mode=1)
    d = o.emittance(hist[-1])[:2, 1]
    q = b.bunch_charge_C
    errs = []
    for hrel in (1e-3, 1e-4, 1e-5, 1e-6):
        h = hrel * q
        vals = []
        for qq in (q + h, q - h):
            bb = I.Beam(**{**w.beam.__dict__, "bunch_charge_C": qq})
            ov = make(n=16, N=o.N, P=0, beam=bb)
            sv = ov.beam_init(nrm)
            hv, _ = ov.run(sv, 20, geom=geom.copy(), geom_mode=2)
            vals.append(ov.emittance(hv[-1])[:2, 0])
        errs.append(np.abs((vals[0] - vals[1]) / (2 * h) - d))
    best = np.min(errs, axis=0)
    assert np.all(best < 1e-5 * np.abs(d)), (best, d)
