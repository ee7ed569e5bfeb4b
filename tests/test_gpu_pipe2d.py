"""The 2D conducting-pipe dual PIC (Sec. 4's own solver) on the GPU against the oracle.

A 100 A coasting proton beam (1 GeV, 1 mm rms) in a 20 mm x 20 mm pipe on 128 x 128 cells, the beam
current as AD variable (slot 0) and six lattice parameters (slots 1-6), one FODO period of 20 kicks.
Bounds as in tests/parity_metrics.py: FP64 emittances 1e-10 and derivatives der_tol(0, N); FP32
emittances 1e-5 and derivatives der_tol(1, N); final particle values element-wise.
"""
import numpy as np
import pytest

import oracle
from paper_2511_21839_gb300 import inputs as I
from parity_metrics import der_tol, report

pytestmark = pytest.mark.gpu

N, CELLS, W, CURRENT = 10_000, (128, 128), (0.02, 0.02), 100.0
LAT = I.Lattice(deriv_slot=(-1, 1, 2, 3, 4, 5, 6))


@pytest.fixture(scope="module")
def adpic():
    from paper_2511_21839_gb300 import adpic as A
    from paper_2511_21839_gb300 import build

    build.build()
    return A


def oracle2d(beam, n=N):
    return oracle.Oracle2D(P=7, nx=CELLS[0], ny=CELLS[1], N=n, a=W[0], b=W[1], kinetic_eV=beam.kinetic_eV,
                           mass_eV=beam.mass_eV, charge_e=beam.charge_e, current_A=CURRENT,
                           eps_n=list(beam.eps_n[:2]), alpha=list(beam.alpha[:2]), beta=list(beam.beta[:2]),
                           L=list(LAT.L), g=list(LAT.g), kicks=list(LAT.kicks), lat_slot=list(LAT.deriv_slot),
                           current_slot=0)


@pytest.fixture(scope="module")
def reference():
    beam = I.default_beam(7)
    o = oracle2d(beam)
    nrm = I.normals(51, N)[:4]
    st0 = o.beam_init(nrm)
    st = st0.copy()
    hist = o.run(st, 20)
    return beam, nrm, st0, st, hist, o


@pytest.mark.parametrize("prec", [0, 1])
def test_pipe2d_run_vs_oracle(adpic, reference, prec):
    beam, nrm, st0, st, hist, o = reference
    sim = adpic.Pipe2D(CELLS, W, N, 7, prec)
    sim.set_beam(beam, CURRENT, 0, nrm)
    sim.set_lattice(LAT)
    init = sim.get_particles()
    np.testing.assert_allclose(init[:, :, 0], st0[:, :, 0], rtol=0, atol=1e-18 if prec == 0 else 1e-9)
    sim.run(20)
    vals, der = sim.moments()
    ref = o.emittance(hist[-1])
    ev, ed = report(f"pipe2d prec={prec}", vals, der, ref)
    assert ev < (1e-10 if prec == 0 else 1e-5) and ed < der_tol(prec, N)
    assert np.abs(ref[:, 1]).min() > 0                        # the current derivative is not trivial
    fin = sim.get_particles()
    scale = np.abs(st[:, :, 0]).max(axis=1, keepdims=True)
    err = np.abs(fin[:, :, 0] - st[:, :, 0]) / scale
    assert err.max() < (1e-9 if prec == 0 else 2e-4), err.max()
    sim.close()


def test_pipe2d_particle_at_the_wall_is_reported(adpic):
    beam = I.default_beam(7)
    sim = adpic.Pipe2D(CELLS, W, 100, 7, 0)
    sim.set_beam(beam, CURRENT, -1, I.normals(52, 100)[:4])
    sim.set_lattice(LAT)
    st = sim.get_particles()
    st[0, 3, 0] = 0.0099                                  # 0.1 mm from the wall at x = +10 mm
    sim.set_particles(st)
    with pytest.raises(adpic.AdPicError) as e:
        sim.run(1)
    assert e.value.status == -6
    sim.close()
