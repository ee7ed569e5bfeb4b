"""The kinetic energy as a dual input on the GPU (Sec. 4: beam parameters as AD variables) against
the FP64 oracle.

The energy is slot 0 and the six lattice parameters slots 1-6 (P = 7). The energy reaches every
stage: the beam's geometric emittance, the quadrupole strengths through B rho, the z drift through
1/gamma0^2, the kick constants, the rest-frame spacing gamma0 hz of the Green's function (one more
convolution per kick, dG/dE with rho_0) and E_z. Bounds as in test_gpu_parity.py.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_2511_21839_gb300 import inputs as I
from parity_metrics import der_tol, grid_tol, report

pytestmark = pytest.mark.gpu

TOL = {0: dict(eps=1e-10, grid=1e-11), 1: dict(eps=1e-5, grid=2e-5)}
LAT = I.Lattice(deriv_slot=(-1, 1, 2, 3, 4, 5, 6))


@pytest.fixture(scope="module")
def adpic():
    from paper_2511_21839_gb300 import adpic as A
    from paper_2511_21839_gb300 import build

    build.build()
    A.lib()
    return A


def energy_beam(**kw):
    w = I.workload("fodo_10k_32")
    return I.Beam(**{**w.beam.__dict__, "energy_slot": 0, **kw})


def chan_err(gpu, ref):
    g = gpu.reshape(gpu.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    scale = np.abs(r).max(axis=1, keepdims=True)
    return (np.abs(g - r) / np.where(scale > 0, scale, 1.0)).max(axis=1)


ENERGY_STAGE_CASES = [
    ((16, 32, 16), 7),
    ((16, 32, 16), 13),     # 16-channel records: the energy term's copy and add stride over 16
    ((64, 64, 64), 7),      # the benched grid (slab convolution)
    ((128, 128, 128), 7),   # the five-pass convolution carries the energy term too
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("grid,P", ENERGY_STAGE_CASES, ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_energy_stage_parity(adpic, prec, grid, P):
    """Potential, field and kick of one kick element-wise against the oracle on the same state: the
    energy channel of phi carries (dG/dE) * rho_0, that of E_z the dual rest-frame spacing."""
    N = 4099
    b = energy_beam()
    w = I.workload("fodo_10k_32")
    o = oracle.Oracle(**I.orc_kwargs(w, n_particles=N, grid=grid, n_deriv=P, beam=b, lattice=LAT))
    sim = adpic.ADPIC(grid, N, P, prec)
    sim.set_beam(b)
    sim.set_lattice(LAT)
    st = o.beam_init(I.normals(61, N))
    o.apply_half_map(st, 0)
    if prec == 1:
        st = st.astype(np.float32).astype(np.float64)
    sim.set_particles(st)
    tol = grid_tol(prec, grid)
    geom = sim.stage(0)
    rho_ref = o.deposit(st, geom)
    phi = sim.stage(2)
    phi_ref = o.solve(geom, rho_ref)
    e = chan_err(phi, phi_ref)
    print(f"  phi per channel {np.array2string(e, precision=1)}")
    assert e.max() < tol
    # the energy term is a visible part of its channel
    o0 = oracle.Oracle(**I.orc_kwargs(w, n_particles=N, grid=grid, n_deriv=P,
                                      beam=I.Beam(**{**b.__dict__, "energy_slot": -1}), lattice=LAT))
    plain = o0.solve(geom, rho_ref)
    assert np.abs(phi_ref[1] - plain[1]).max() > 10 * tol * np.abs(phi_ref[1]).max()
    E = sim.stage(3)
    E_ref = o.field(geom, phi_ref)
    e = chan_err(E.reshape(3 * (P + 1), -1), E_ref.reshape(3 * (P + 1), -1))
    print(f"  E per channel max {e.max():.2e}")
    assert e.max() < 5 * tol
    sim.stage(4, kick=5)
    after = sim.get_particles()
    ref = st.copy()
    o.kick(ref, geom, E_ref, 5)
    for c in (1, 3, 5):
        dref = np.abs(ref[c] - st[c]).max(axis=0, keepdims=True)
        bound = tol * 10 * dref + (2.4e-7 * np.abs(ref[c]) if prec == 1 else 0.0)
        assert np.all(np.abs(after[c] - ref[c]) <= bound + 1e-300), c
    sim.close()


RUN_N, RUN_GRID = 10_000, (32, 32, 32)


@pytest.fixture(scope="module")
def energy_reference():
    b = energy_beam()
    w = I.workload("fodo_10k_32")
    o = oracle.Oracle(**I.orc_kwargs(w, n_particles=RUN_N, grid=RUN_GRID, beam=b, lattice=LAT))
    nrm = I.normals(62, RUN_N)
    st = o.beam_init(nrm)
    hist, _ = o.run(st, 20)
    return o, b, nrm, hist


@pytest.mark.parametrize("prec", [0, 1])
def test_energy_run_vs_oracle(adpic, energy_reference, prec):
    """One FODO period of 10,000 particles on 32^3: the dual emittances of all three planes (E_z
    reaches the z plane only) against the oracle, per component."""
    N, grid = RUN_N, RUN_GRID
    o, b, nrm, hist = energy_reference
    sim = adpic.ADPIC(grid, N, 7, prec)
    sim.set_beam(b, nrm)
    sim.set_lattice(LAT)
    sim.run(20)
    h = sim.history()
    e_gpu = o.emittance(h[-1])
    ref = o.emittance(hist[-1])
    ev, ed = report(f"energy slot prec={prec}", e_gpu[:, 0], e_gpu[:, 1:], ref)
    assert ev < TOL[prec]["eps"] and ed < der_tol(prec, N)
    assert np.all(np.abs(ref[:, 1]) > 0)
    sim.close()


def test_energy_checkpoint_resume(adpic):
    """run(40) equals run(20), save, load into a fresh handle, run(20), with the energy slot."""
    N, grid = 3000, (16, 16, 16)
    b = energy_beam()
    nrm = I.normals(63, N)
    a = adpic.ADPIC(grid, N, 7, 0)
    a.set_beam(b, nrm)
    a.set_lattice(LAT)
    a.run(40)
    ref = a.history()[-1]
    a.close()
    s1 = adpic.ADPIC(grid, N, 7, 0)
    s1.set_beam(b, nrm)
    s1.set_lattice(LAT)
    s1.run(20)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        s1.save(path)
        s1.close()
        s2 = adpic.ADPIC(grid, N, 7, 0)
        s2.load(path)
        s2.run(20)
    got = s2.history()[-1]
    s2.close()
    scale = np.abs(ref).max(axis=(1, 2), keepdims=True)
    assert (np.abs(got - ref) / scale).max() < 1e-11


def test_energy_slot_is_validated(adpic):
    """The energy slot must differ from the charge slot; the batched runtime and the 2D pipe do not
    take it (AD_PIC_ERR_UNSUPPORTED)."""
    b = energy_beam(charge_slot=0)
    sim = adpic.ADPIC((16, 16, 16), 100, 7, 0)
    with pytest.raises(adpic.AdPicError) as e:
        sim.set_beam(b)
    assert e.value.status == -1                          # AD_PIC_ERR_INVALID_ARG
    sim.close()
    bt = adpic.Batch([(32, 32, 32)], [100])
    with pytest.raises(adpic.AdPicError) as e:
        bt.set_beam(0, energy_beam(), I.normals(64, 100))
    assert e.value.status == -8                          # AD_PIC_ERR_UNSUPPORTED
    bt.close()
    p2 = adpic.Pipe2D((32, 32), (0.02, 0.02), 100, 7, 0)
    with pytest.raises(adpic.AdPicError) as e:
        p2.set_beam(energy_beam(), 1.0, -1, I.normals(65, 100)[:4])
    assert e.value.status == -8                          # AD_PIC_ERR_UNSUPPORTED
    p2.close()
