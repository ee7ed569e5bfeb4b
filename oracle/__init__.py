"""ctypes wrapper of the plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by the cpu_baseline / reference leg of bench.py. The product path never
imports this package. It shares no code with the CUDA library.
"""
import ctypes as ct
import os

import numpy as np

from . import build as _build

MAXC = 32


class OrcElement(ct.Structure):
    _fields_ = [("type", ct.c_int32), ("slot_L", ct.c_int32), ("slot_k", ct.c_int32), ("pad", ct.c_int32),
                ("L", ct.c_double), ("k", ct.c_double)]


class OrcConfig(ct.Structure):
    _fields_ = [
        ("P", ct.c_int32), ("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32),
        ("N", ct.c_int64),
        ("kinetic_eV", ct.c_double), ("mass_eV", ct.c_double), ("charge_e", ct.c_double),
        ("bunch_charge_C", ct.c_double),
        ("eps_n", ct.c_double * 3), ("alpha", ct.c_double * 3), ("beta", ct.c_double * 3),
        ("twiss_slot", ct.c_int32 * 6),
        ("L", ct.c_double * 5), ("g", ct.c_double * 2),
        ("kicks", ct.c_int32 * 5), ("lat_slot", ct.c_int32 * 7),
        ("n_line", ct.c_int32), ("pad_line", ct.c_int32),
        ("line", ct.POINTER(OrcElement)), ("line_kicks", ct.POINTER(ct.c_int32)),
        ("charge_slot", ct.c_int32), ("energy_slot", ct.c_int32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ct.CDLL(path)
        dp = ct.POINTER(ct.c_double)
        cp = ct.POINTER(OrcConfig)
        sig = {
            "orc_constants": (None, [cp, dp]),
            "orc_dual_op": (None, [ct.c_int, ct.c_int, dp, dp, dp]),
            "orc_testfn": (None, [dp, dp]),
            "orc_fft1d": (ct.c_int, [dp, dp, ct.c_int, ct.c_int]),
            "orc_igf": (ct.c_double, [ct.c_double] * 6),
            "orc_igf_dhz": (None, [ct.c_double] * 6 + [dp]),
            "orc_dual_constants": (None, [cp, dp]),
            "orc_green_denergy": (None, [cp, dp, dp]),
            "orc_beam_init": (ct.c_int, [cp, dp, dp]),
            "orc_half_map": (None, [cp, ct.c_int64, dp]),
            "orc_apply_half_map": (None, [cp, dp, ct.c_int64]),
            "orc_geometry": (ct.c_int, [cp, dp, dp]),
            "orc_deposit": (ct.c_int, [cp, dp, dp, dp]),
            "orc_green": (None, [cp, dp, dp]),
            "orc_solve": (ct.c_int, [cp, dp, dp, dp]),
            "orc_solve_direct": (ct.c_int, [cp, dp, dp, dp]),
            "orc_field": (None, [cp, dp, dp, dp]),
            "orc_gather": (ct.c_int, [cp, dp, dp, dp, dp]),
            "orc_kick": (ct.c_int, [cp, dp, dp, dp, ct.c_int64]),
            "orc_moments": (None, [cp, dp, dp]),
            "orc_emittance": (None, [cp, dp, dp]),
            "orc_run": (ct.c_int, [cp, dp, ct.c_int64, ct.c_int, dp, dp, ct.c_int]),
            "orc_beamline_matrix": (None, [ct.c_int, ct.POINTER(OrcElement), ct.c_int, dp]),
            "orc_twiss": (None, [ct.c_int, ct.POINTER(OrcElement), ct.c_int, dp, dp]),
            "orc_periodic_twiss": (ct.c_int, [ct.c_int, ct.POINTER(OrcElement), ct.c_int, dp]),
            "orc_track": (None, [ct.c_int, ct.POINTER(OrcElement), ct.c_int, ct.c_int64, ct.c_int64, dp, dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _check(st, what):
    if st < 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")
    return st


class Oracle:
    """FP64 oracle bound to one configuration (a plain dict of the fields of OrcConfig)."""

    def __init__(self, line=None, line_kicks=None, **kw):
        """kw: the fields of OrcConfig; line: a beamline [(type, L, k, slot_L, slot_k)] with
        line_kicks kicks per element, in place of the FODO period."""
        c = OrcConfig()
        c.charge_slot = -1
        c.energy_slot = -1
        if line is not None:
            self._line = elements(line)
            self._line_kicks = (ct.c_int32 * len(line))(*[int(v) for v in line_kicks])
            c.n_line = len(line)
            c.line = ct.cast(self._line, ct.POINTER(OrcElement))
            c.line_kicks = ct.cast(self._line_kicks, ct.POINTER(ct.c_int32))
        for k, v in kw.items():
            f = getattr(c, k)
            if isinstance(f, ct.Array):
                for i, x in enumerate(v):
                    f[i] = x
            else:
                setattr(c, k, v)
        self.cfg = c
        self.C = c.P + 1
        self.N = c.N
        self.n = (c.nx, c.ny, c.nz)
        self._L = lib()

    @property
    def ref(self):
        return ct.byref(self.cfg)

    def constants(self):
        out = np.zeros(8)
        self._L.orc_constants(self.ref, _p(out))
        keys = ["gamma0", "beta0", "p0", "brho", "kappa_perp", "kappa_z", "q_macro", "q"]
        return dict(zip(keys, out.tolist()))

    def dual_constants(self):
        """gamma0, beta0 gamma0, B rho, kappa_perp, kappa_z, gamma0^2 as duals [6][C]."""
        out = np.zeros((6, self.C))
        self._L.orc_dual_constants(self.ref, _p(out))
        return out

    def green_denergy(self, geom):
        geom = np.ascontiguousarray(geom, dtype=np.float64)
        nx, ny, nz = self.n
        out = np.zeros((2 * nz, 2 * ny, 2 * nx))
        self._L.orc_green_denergy(self.ref, _p(geom), _p(out))
        return out

    def state_shape(self):
        return (6, self.N, self.C)

    def grid_shape(self):
        nx, ny, nz = self.n
        return (self.C, nz, ny, nx)

    def beam_init(self, normals):
        normals = np.ascontiguousarray(normals, dtype=np.float64)
        assert normals.shape == (6, self.N)
        st = np.zeros(self.state_shape())
        _check(self._L.orc_beam_init(self.ref, _p(normals), _p(st)), "beam_init")
        return st

    def half_map(self, kick):
        m = np.zeros((3, 4, self.C))
        self._L.orc_half_map(self.ref, kick, _p(m))
        return m

    def apply_half_map(self, state, kick):
        self._L.orc_apply_half_map(self.ref, _p(state), kick)

    def geometry(self, state):
        g = np.zeros(6)
        _check(self._L.orc_geometry(self.ref, _p(state), _p(g)), "geometry")
        return g

    def deposit(self, state, geom):
        rho = np.zeros(self.grid_shape())
        _check(self._L.orc_deposit(self.ref, _p(state), _p(np.ascontiguousarray(geom)), _p(rho)), "deposit")
        return rho

    def green(self, geom):
        nx, ny, nz = self.n
        G = np.zeros((2 * nz, 2 * ny, 2 * nx))
        self._L.orc_green(self.ref, _p(np.ascontiguousarray(geom)), _p(G))
        return G

    def solve(self, geom, rho):
        phi = np.zeros(self.grid_shape())
        _check(self._L.orc_solve(self.ref, _p(np.ascontiguousarray(geom)), _p(np.ascontiguousarray(rho)), _p(phi)),
               "solve")
        return phi

    def solve_direct(self, geom, rho):
        phi = np.zeros(self.grid_shape())
        _check(self._L.orc_solve_direct(self.ref, _p(np.ascontiguousarray(geom)), _p(np.ascontiguousarray(rho)),
                                        _p(phi)), "solve_direct")
        return phi

    def field(self, geom, phi):
        E = np.zeros((3,) + self.grid_shape())
        self._L.orc_field(self.ref, _p(np.ascontiguousarray(geom)), _p(np.ascontiguousarray(phi)), _p(E))
        return E

    def gather(self, state, geom, E):
        Ep = np.zeros((3, self.N, self.C))
        _check(self._L.orc_gather(self.ref, _p(state), _p(np.ascontiguousarray(geom)),
                                  _p(np.ascontiguousarray(E)), _p(Ep)), "gather")
        return Ep

    def kick(self, state, geom, E, kick):
        _check(self._L.orc_kick(self.ref, _p(state), _p(np.ascontiguousarray(geom)),
                                _p(np.ascontiguousarray(E)), kick), "kick")

    def moments(self, state):
        m = np.zeros((3, 5, self.C))
        self._L.orc_moments(self.ref, _p(state), _p(m))
        return m

    def emittance(self, mom):
        e = np.zeros((3, self.C))
        self._L.orc_emittance(self.ref, _p(np.ascontiguousarray(mom)), _p(e))
        return e

    def run(self, state, n_kicks, kick0=0, geom=None, geom_mode=0):
        """Advance `state` in place; returns (moment records [R][3][5][C], geometry [n_kicks][6])."""
        kpp = sum(self._line_kicks) if self.cfg.n_line > 0 else sum(self.cfg.kicks)
        nrec = n_kicks // max(kpp, 1) + 2
        hist = np.zeros((nrec, 3, 5, self.C))
        if geom is None:
            geom = np.zeros((max(n_kicks, 1), 6))
        r = _check(self._L.orc_run(self.ref, _p(state), kick0, n_kicks, _p(hist), _p(geom), geom_mode), "run")
        return hist[:r], geom[:n_kicks]


def dual_op(op, f, g=None):
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.zeros_like(f) if g is None else np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros_like(f)
    ops = {"add": 0, "sub": 1, "mul": 2, "div": 3, "sqrt": 4, "sin": 5, "cos": 6, "sinh": 7, "cosh": 8, "exp": 9}
    lib().orc_dual_op(ops[op], f.size, _p(f), _p(g), _p(out))
    return out


def testfn(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(6)
    lib().orc_testfn(_p(x), _p(out))
    return out


def fft1d(z, sign=-1):
    re = np.ascontiguousarray(z.real, dtype=np.float64).copy()
    im = np.ascontiguousarray(z.imag, dtype=np.float64).copy()
    _check(lib().orc_fft1d(_p(re), _p(im), re.size, sign), "fft1d")
    return re + 1j * im


def igf(x, y, z, hx, hy, hz):
    return lib().orc_igf(x, y, z, hx, hy, hz)


def igf_dhz(x, y, kz, hx, hy, hz):
    """(G, dG/dhz) at the node offset (x, y, kz hz), the z offset moving with hz."""
    out = np.zeros(2)
    lib().orc_igf_dhz(x, y, kz, hx, hy, hz, _p(out))
    return out[0], out[1]


def threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


# ---------------------------------------------------------------- single-particle dual optics (Sec. 3)

def elements(beamline):
    """ctypes array of OrcElement from (type, L, k, slot_L, slot_k) tuples."""
    arr = (OrcElement * len(beamline))()
    for i, (t, L, k, sL, sk) in enumerate(beamline):
        arr[i] = OrcElement(int(t), int(sL), int(sk), 0, float(L), float(k))
    return arr


def beamline_matrix(beamline, P):
    m = np.zeros((2, 4, P + 1))
    lib().orc_beamline_matrix(P, elements(beamline), len(beamline), _p(m))
    return m


def twiss(beamline, P, twiss0):
    out = np.zeros((4, P + 1))
    lib().orc_twiss(P, elements(beamline), len(beamline), _p(np.ascontiguousarray(twiss0, dtype=np.float64)),
                    _p(out))
    return out


def periodic_twiss(beamline, P):
    out = np.zeros((4, P + 1))
    st = lib().orc_periodic_twiss(P, elements(beamline), len(beamline), _p(out))
    if st != 0:
        raise ValueError("unstable cell")
    return out


def track(beamline, P, x0, n_repeat):
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    out = np.zeros((x0.shape[0], 4, P + 1))
    lib().orc_track(P, elements(beamline), len(beamline), int(n_repeat), x0.shape[0], _p(x0), _p(out))
    return out


# ---------------------------------------------------------------- 2D PIC in a conducting pipe (Sec. 4)

class Orc2DConfig(ct.Structure):
    _fields_ = [("P", ct.c_int32), ("nx", ct.c_int32), ("ny", ct.c_int32), ("current_slot", ct.c_int32),
                ("N", ct.c_int64), ("a", ct.c_double), ("b", ct.c_double),
                ("kinetic_eV", ct.c_double), ("mass_eV", ct.c_double), ("charge_e", ct.c_double),
                ("current_A", ct.c_double), ("eps_n", ct.c_double * 2), ("alpha", ct.c_double * 2),
                ("beta", ct.c_double * 2), ("L", ct.c_double * 5), ("g", ct.c_double * 2),
                ("kicks", ct.c_int32 * 5), ("lat_slot", ct.c_int32 * 7)]


_lib2d = None


def lib2d():
    global _lib2d
    if _lib2d is None:
        L = lib()
        dp = ct.POINTER(ct.c_double)
        cp = ct.POINTER(Orc2DConfig)
        sig = {
            "orc2d_constants": (None, [cp, dp]),
            "orc2d_beam_init": (ct.c_int, [cp, dp, dp]),
            "orc2d_deposit": (ct.c_int, [cp, dp, dp]),
            "orc2d_solve": (None, [cp, dp, dp]),
            "orc2d_field": (None, [cp, dp, dp]),
            "orc2d_kick": (ct.c_int, [cp, dp, dp, ct.c_int64]),
            "orc2d_moments": (None, [cp, dp, dp]),
            "orc2d_run": (ct.c_int, [cp, dp, ct.c_int64, ct.c_int, dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib2d = L
    return _lib2d


class Oracle2D:
    """FP64 oracle of the 2D conducting-pipe PIC bound to one configuration (fields of Orc2DConfig)."""

    def __init__(self, **kw):
        c = Orc2DConfig()
        c.current_slot = -1
        for k, v in kw.items():
            f = getattr(c, k)
            if isinstance(f, ct.Array):
                for i, x in enumerate(v):
                    f[i] = x
            else:
                setattr(c, k, v)
        self.cfg = c
        self.C = c.P + 1
        self.N = c.N
        self._L = lib2d()

    @property
    def ref(self):
        return ct.byref(self.cfg)

    def constants(self):
        out = np.zeros(5)
        self._L.orc2d_constants(self.ref, _p(out))
        return dict(zip(["gamma0", "beta0", "p0", "brho", "K"], out.tolist()))

    def grid_shape(self):
        return (self.C, self.cfg.ny + 1, self.cfg.nx + 1)

    def beam_init(self, normals):
        normals = np.ascontiguousarray(normals, dtype=np.float64)
        st = np.zeros((4, self.N, self.C))
        _check(self._L.orc2d_beam_init(self.ref, _p(normals), _p(st)), "2d beam_init")
        return st

    def deposit(self, state):
        n = np.zeros(self.grid_shape())
        _check(self._L.orc2d_deposit(self.ref, _p(np.ascontiguousarray(state)), _p(n)), "2d deposit")
        return n

    def solve(self, n):
        phi = np.zeros(self.grid_shape())
        self._L.orc2d_solve(self.ref, _p(np.ascontiguousarray(n)), _p(phi))
        return phi

    def field(self, phi):
        E = np.zeros((2,) + self.grid_shape())
        self._L.orc2d_field(self.ref, _p(np.ascontiguousarray(phi)), _p(E))
        return E

    def kick(self, state, E, kick):
        _check(self._L.orc2d_kick(self.ref, _p(state), _p(np.ascontiguousarray(E)), kick), "2d kick")

    def moments(self, state):
        m = np.zeros((2, 5, self.C))
        self._L.orc2d_moments(self.ref, _p(np.ascontiguousarray(state)), _p(m))
        return m

    def run(self, state, n_kicks, kick0=0):
        kpp = sum(self.cfg.kicks)
        hist = np.zeros((n_kicks // max(kpp, 1) + 2, 2, 5, self.C))
        r = _check(self._L.orc2d_run(self.ref, _p(state), kick0, n_kicks, _p(hist)), "2d run")
        return hist[:r]

    def emittance(self, mom):
        """Dual rms emittances [2][C] from moments [2][5][C] (the 3D oracle's formula, planes x, y)."""
        m3 = np.zeros((3, 5, self.C))
        m3[:2] = mom
        m3[2, 2, 0] = m3[2, 4, 0] = 1.0
        o = Oracle(P=self.cfg.P, nx=8, ny=8, nz=8, N=1)
        return o.emittance(m3)[:2]
