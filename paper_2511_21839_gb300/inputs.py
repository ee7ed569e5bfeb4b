"""Seeded synthetic inputs and workload recipes.

This module holds no step of the PIC method: it only fixes the numbers a run
starts from (lattice, beam and grid parameters, the bunch charge, and the
standard-normal draws of the initial distribution). Both the CUDA library and
the CPU oracle receive the same values from here; nothing here calls either.

Workloads (the FODO example of Sec. 1 / Sec. 4, here in 3D):
  single period     FODO D 0.5 m / QF 0.1 m at +10 T/m / D 1.0 m / QD 0.1 m at -10 T/m / D 0.5 m,
                    1 GeV protons, 10,000 macroparticles, 32^3, 20 kicks, P = 7
  1M-particle run   same lattice and beam, 1,048,576 macroparticles, 64^3, 10 periods, P = 7
  large run         16,777,216 macroparticles, 128^3, 20 periods, P = 13 (7 lattice + 6 Twiss)
  batched scan      256 instances, +-10 % lattice perturbations, log-uniform particle counts
  surrogate data    4,096 single-period runs with +-20 % lattice perturbations
"""
from dataclasses import dataclass, field
import math

import numpy as np

# CODATA 2018 (kept here only to derive the bunch charge of the recipe)
_C = 299792458.0
_QE = 1.602176634e-19
_EPS0 = 8.8541878128e-12
PROTON_MASS_EV = 938.27208816e6
PROTON_RADIUS_M = _QE ** 2 / (4.0 * math.pi * _EPS0 * PROTON_MASS_EV * _QE)

KICKS = (4, 2, 8, 2, 4)                      # D1, QF, D2, QD, D3
LENGTHS = (0.5, 0.1, 1.0, 0.1, 0.5)          # m
GRADIENTS = (10.0, -10.0)                    # T/m
LATTICE_PARAM_NAMES = ("L_D1", "L_QF", "g_QF", "L_D2", "L_QD", "g_QD", "L_D3")
TWISS_PARAM_NAMES = ("alpha_x", "beta_x", "eps_x", "alpha_y", "beta_y", "eps_y")


@dataclass
class Lattice:
    L: tuple = LENGTHS
    g: tuple = GRADIENTS
    kicks: tuple = KICKS
    deriv_slot: tuple = (0, 1, 2, 3, 4, 5, 6)

    def params(self):
        """The seven lattice parameters in slot order (L_D1, L_QF, g_QF, L_D2, L_QD, g_QD, L_D3)."""
        return (self.L[0], self.L[1], self.g[0], self.L[2], self.L[3], self.g[1], self.L[4])

    @staticmethod
    def from_params(p, kicks=KICKS, deriv_slot=(0, 1, 2, 3, 4, 5, 6)):
        return Lattice(L=(p[0], p[1], p[3], p[4], p[6]), g=(p[2], p[5]), kicks=tuple(kicks),
                       deriv_slot=tuple(deriv_slot))


@dataclass
class Beam:
    kinetic_eV: float = 1.0e9
    mass_eV: float = PROTON_MASS_EV
    charge_e: float = 1.0
    bunch_charge_C: float = 0.0
    eps_n: tuple = (1e-6, 1e-6, 1e-6)
    alpha: tuple = (0.0, 0.0, 0.0)
    beta: tuple = (0.0, 0.0, 0.0)
    twiss_slot: tuple = (-1, -1, -1, -1, -1, -1)
    charge_slot: int = -1          # derivative slot of the bunch charge (-1: constant)
    energy_slot: int = -1          # derivative slot of the kinetic energy (-1: constant)


@dataclass
class Workload:
    name: str
    n_particles: int
    grid: tuple
    n_deriv: int
    periods: int
    seed: int
    lattice: Lattice = field(default_factory=Lattice)
    beam: Beam = field(default_factory=Beam)

    @property
    def kicks_per_period(self):
        return sum(self.lattice.kicks)

    @property
    def n_kicks(self):
        return self.periods * self.kicks_per_period


def relativistic(kinetic_eV=1.0e9, mass_eV=PROTON_MASS_EV):
    gamma = 1.0 + kinetic_eV / mass_eV
    beta = math.sqrt(1.0 - 1.0 / gamma ** 2)
    brho = gamma * beta * mass_eV / _C
    return gamma, beta, brho


def _thick_lens(k, length):
    """Textbook 2x2 matrix of a quadrupole of strength k (1/m^2) or drift (k = 0)."""
    if k > 0:
        w = math.sqrt(k)
        return np.array([[math.cos(w * length), math.sin(w * length) / w],
                         [-w * math.sin(w * length), math.cos(w * length)]])
    if k < 0:
        w = math.sqrt(-k)
        return np.array([[math.cosh(w * length), math.sinh(w * length) / w],
                         [w * math.sinh(w * length), math.cosh(w * length)]])
    return np.array([[1.0, length], [0.0, 1.0]])


def fodo_phase_advance(lat: Lattice, kinetic_eV=1.0e9, mass_eV=PROTON_MASS_EV):
    """Zero-current phase advance per period (rad) in x, from the trace of the cell matrix."""
    _, _, brho = relativistic(kinetic_eV, mass_eV)
    ks = (0.0, lat.g[0] / brho, 0.0, lat.g[1] / brho, 0.0)
    M = np.eye(2)
    for k, L in zip(ks, lat.L):
        M = _thick_lens(k, L) @ M
    return math.acos(0.5 * np.trace(M)), M


def bunch_charge_for_depression(ratio=0.7, sigma_z=1e-3, eps_n=1e-6, lat: Lattice = None,
                                kinetic_eV=1.0e9, mass_eV=PROTON_MASS_EV):
    """Bunch charge giving the tune depression `ratio` in the smooth, matched-KV approximation.

    The 3D bunch is replaced by a coasting beam of its centre line density
    N/(sqrt(2 pi) sigma_z); its generalised perveance is
    K = 2 N r_p / (sqrt(2 pi) sigma_z beta0^2 gamma0^3), and the KV envelope
    in smooth focusing k0 = mu0 / L_cell gives nu/nu0 = sqrt(1+u^2) - u with
    u = K / (2 (4 eps_rms) k0).
    """
    lat = lat or Lattice()
    gamma, beta, _ = relativistic(kinetic_eV, mass_eV)
    eps = eps_n / (beta * gamma)
    mu0, _ = fodo_phase_advance(lat, kinetic_eV, mass_eV)
    k0 = mu0 / sum(lat.L)
    u = (1.0 - ratio ** 2) / (2.0 * ratio)
    K = 2.0 * u * 4.0 * eps * k0
    r_p = PROTON_RADIUS_M * PROTON_MASS_EV / mass_eV
    n_real = K * math.sqrt(2.0 * math.pi) * sigma_z * beta ** 2 * gamma ** 3 / (2.0 * r_p)
    return n_real * _QE


def default_beam(n_deriv=7, sigma=(1e-3, 1e-3, 1e-3), eps_n=(1e-6, 1e-6, 1e-6), kinetic_eV=1.0e9,
                 tune_depression=0.7, lat: Lattice = None):
    gamma, beta, _ = relativistic(kinetic_eV)
    eps = [e / (beta * gamma) for e in eps_n]
    betas = tuple(s * s / e for s, e in zip(sigma, eps))
    q = bunch_charge_for_depression(tune_depression, sigma[2], eps_n[0], lat, kinetic_eV)
    slots = (7, 8, 9, 10, 11, 12) if n_deriv == 13 else (-1,) * 6
    return Beam(kinetic_eV=kinetic_eV, bunch_charge_C=q, eps_n=tuple(eps_n), alpha=(0.0, 0.0, 0.0),
                beta=betas, twiss_slot=slots)


def workload(name: str) -> Workload:
    if name == "fodo_10k_32":
        return Workload(name, 10_000, (32, 32, 32), 7, 1, 1, Lattice(), default_beam(7))
    if name == "fodo_1m_64":
        return Workload(name, 1_048_576, (64, 64, 64), 7, 10, 2, Lattice(), default_beam(7))
    if name == "fodo_16m_128":
        return Workload(name, 16_777_216, (128, 128, 128), 13, 20, 4, Lattice(), default_beam(13))
    raise KeyError(name)


def normals(seed: int, n: int) -> np.ndarray:
    """Standard-normal draws [6][n] (x: u1,u2; y: u3,u4; z: u5,u6) of the initial distribution."""
    return np.random.default_rng(seed).standard_normal((6, n))


def perturbed_params(seed: int, count: int, rel: float, base=None) -> np.ndarray:
    """count x 7 lattice parameter sets, each scaled by (1 + U(-rel, rel))."""
    base = np.asarray(base if base is not None else Lattice().params(), dtype=np.float64)
    rng = np.random.default_rng(seed)
    return base[None, :] * (1.0 + rng.uniform(-rel, rel, size=(count, base.size)))


def batched_scan(seed: int = 3, count: int = 256, periods: int = 5):
    """Instances of the batched sensitivity scan: (params [count][7], n_particles [count], grid n [count])."""
    rng = np.random.default_rng(seed)
    base = np.asarray(Lattice().params())
    params = base[None, :] * (1.0 + rng.uniform(-0.1, 0.1, size=(count, 7)))
    npart = np.rint(np.exp(rng.uniform(math.log(16384), math.log(262144), size=count))).astype(np.int64)
    grid = np.where(rng.uniform(size=count) < 0.5, 32, 64).astype(np.int32)
    return params, npart, grid, periods


def orc_kwargs(w: Workload, n_particles=None, grid=None, n_deriv=None, lattice=None, beam=None):
    """The oracle's configuration fields for a workload (plain values only)."""
    lat = lattice or w.lattice
    b = beam or w.beam
    g = grid or w.grid
    P = w.n_deriv if n_deriv is None else n_deriv
    return dict(P=P, nx=g[0], ny=g[1], nz=g[2], N=w.n_particles if n_particles is None else n_particles,
                kinetic_eV=b.kinetic_eV, mass_eV=b.mass_eV, charge_e=b.charge_e, bunch_charge_C=b.bunch_charge_C,
                eps_n=b.eps_n, alpha=b.alpha, beta=b.beta,
                twiss_slot=[s if (0 <= s < P) else -1 for s in b.twiss_slot],
                L=lat.L, g=lat.g, kicks=lat.kicks,
                lat_slot=[s if (0 <= s < P) else -1 for s in lat.deriv_slot],
                charge_slot=b.charge_slot if 0 <= b.charge_slot < P else -1,
                energy_slot=b.energy_slot if 0 <= b.energy_slot < P else -1)
