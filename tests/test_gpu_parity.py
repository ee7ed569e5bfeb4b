"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (stated per result):
  FP64 path   emittances 1e-10 relative; each emittance derivative 1e-10 relative (runs on fewer
              than 10,000 particles: 2e-9, the algorithm's own floor there); potential and field
              stages 1e-11 of the channel's max on small grids, growing with the Green's function's
              cancellation on large ones (parity_metrics.grid_tol)
  FP32 path   emittances 1e-5 relative; each emittance derivative 1e-4 relative at the 1M-particle
              configuration, max(1e-4, 3e-2 / sqrt(N)) on N particles (parity_metrics.der_tol);
              grid stages 2e-5 of the channel's max
A derivative's relative error has the denominator max(|d_k|, 1e-3 max_j |d_j|) per emittance
(tests/parity_metrics.py). Both sides sum the beam moments with compensated (error-free) sums:
the emittance derivatives cancel strongly (the emittance barely changes while the second moments
do), and plain FP64 sums left the oracle itself 8e-10 apart between thread counts; with the
compensated sums two oracle runs with different summation orders agree to 1.4e-11.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2511_21839_gb300 import inputs as I
from parity_metrics import der_tol, grid_tol, rel_der_components, rel_eps, report

pytestmark = pytest.mark.gpu

TOL = {0: dict(eps=1e-10, der=1e-10, grid=1e-11, state=1e-9), 1: dict(eps=1e-5, der=1e-4, grid=2e-5, state=2e-4)}


@pytest.fixture(scope="module")
def adpic():
    from paper_2511_21839_gb300 import build
    from paper_2511_21839_gb300 import adpic as A

    build.build()
    A.lib()
    return A


def chan_close(gpu, ref, tol, axis_chan):
    """Element-wise comparison relative to the max of each channel."""
    g = np.moveaxis(gpu, axis_chan, 0).reshape(gpu.shape[axis_chan], -1)
    r = np.moveaxis(ref, axis_chan, 0).reshape(ref.shape[axis_chan], -1)
    scale = np.abs(r).max(axis=1, keepdims=True)
    scale = np.where(scale > 0, scale, 1.0)
    err = (np.abs(g - r) / scale).max()
    print(f"  element-wise error {err:.2e} (bound {tol:.1e})")
    assert err < tol, err
    return err


def make_pair(adpic, N, grid, P, prec, wname="fodo_10k_32", beam=None, q=None):
    w = I.workload(wname)
    b = beam or (w.beam if P == 7 else I.default_beam(13))
    if q is not None:
        b = I.Beam(**{**b.__dict__, "bunch_charge_C": q})
    kw = I.orc_kwargs(w, n_particles=N, grid=grid, n_deriv=P, beam=b)
    o = oracle.Oracle(**kw)
    sim = adpic.ADPIC(grid, N, P, prec)
    sim.set_beam(b)
    sim.set_lattice(w.lattice)
    return o, sim, w, b


# ---------------------------------------------------------------- stages

STAGE_CASES = [
    ((16, 32, 16), 7, 5003),      # small anisotropic grid
    ((16, 32, 16), 13, 5003),
    ((16, 8, 8), 7, 1501),        # the smallest dimensions: 16 y columns per slab, fewer than a chunk
    ((64, 64, 64), 7, 4099),      # the benched grid: slab convolution (x pass, one CTA per (y, z) slab)
    ((128, 128, 128), 13, 3001),  # the large instance's grid: five-pass convolution, 129-point DCTs
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("grid,P,N", STAGE_CASES, ids=lambda v: "x".join(map(str, v)) if isinstance(v, tuple) else str(v))
def test_stage_parity(adpic, prec, grid, P, N):
    """Every stage of one kick element-wise against the oracle on the same state: geometry, deposit,
    potential, field (each channel relative to its max) and the kick of each momentum channel."""
    o, sim, w, b = make_pair(adpic, N, grid, P, prec)
    st = o.beam_init(I.normals(41, N))
    o.apply_half_map(st, 0)
    if prec == 1:
        st32 = st.astype(np.float32).astype(np.float64)   # the FP32 state the GPU holds
        st = st32
    sim.set_particles(st)
    tol = grid_tol(prec, grid)
    geom = sim.stage(0)
    gref = o.geometry(st)
    np.testing.assert_allclose(geom, gref, rtol=1e-12 if prec == 0 else 1e-6)
    rho = sim.stage(1)
    rho_ref = o.deposit(st, geom)
    chan_close(rho, rho_ref, TOL[prec]["grid"], 0)
    assert abs(rho[0].sum() - o.constants()["q_macro"] * N) < 1e-6 * o.constants()["q_macro"] * N
    phi = sim.stage(2)
    phi_ref = o.solve(geom, rho_ref)
    chan_close(phi, phi_ref, tol, 0)
    E = sim.stage(3)
    E_ref = o.field(geom, phi_ref)
    chan_close(E.reshape(3 * o.C, -1), E_ref.reshape(3 * o.C, -1), tol * 5, 0)
    sim.stage(4, kick=5)
    after = sim.get_particles()
    ref = st.copy()
    o.kick(ref, geom, E_ref, 5)
    # the kick changes only the momenta: compare the change relative to its own scale; in FP32 the
    # updated momentum is also rounded to the state's precision, a bound of one ulp of |p|
    for c in (1, 3, 5):
        dref = np.abs(ref[c] - st[c]).max(axis=0, keepdims=True)
        bound = tol * 10 * dref + (2.4e-7 * np.abs(ref[c]) if prec == 1 else 0.0)
        assert np.all(np.abs(after[c] - ref[c]) <= bound + 1e-300), c
    for c in (0, 2, 4):
        assert np.array_equal(after[c], st[c])
    sim.close()


# ---------------------------------------------------------------- whole runs

@pytest.fixture(scope="module")
def config1_ref():
    w = I.workload("fodo_10k_32")
    o = oracle.Oracle(**I.orc_kwargs(w))
    nrm = I.normals(w.seed, w.n_particles)
    st0 = o.beam_init(nrm)
    st = st0.copy()
    hist, _ = o.run(st, w.n_kicks)
    return w, nrm, st0, st, hist, o


@pytest.mark.parametrize("prec", [0, 1])
def test_config1_single_period(adpic, config1_ref, prec):
    """10,000 particles, 32^3, one FODO period of 20 kicks, P = 7, GPU init from the same normals."""
    w, nrm, st0, st, hist, o = config1_ref
    sim = adpic.ADPIC(w.grid, w.n_particles, 7, prec)
    sim.set_beam(w.beam, nrm)
    sim.set_lattice(w.lattice)
    init = sim.get_particles()
    chan_close(init.reshape(6, -1, 8), st0, 1e-14 if prec == 0 else 1e-7, 2)
    sim.run(w.n_kicks)
    vals, der = sim.moments()
    ref = o.emittance(hist[-1])[:2]
    ev, ed = report(f"config1 prec={prec}", vals, der, ref)
    assert ev < TOL[prec]["eps"] and ed < der_tol(prec, w.n_particles)
    gh = sim.history()
    assert gh.shape[0] == 2
    # record 0 = moments of the initial state: second moments element-wise, means (zero up to
    # rounding after the mean removal) against the rms size of their plane
    m0 = o.moments(st0)
    chan_close(gh[0][:, 2:].reshape(9, -1), m0[:, 2:].reshape(9, -1), 1e-12 if prec == 0 else 1e-5, 0)
    rms = np.sqrt(m0[:, 2:3, :1] + m0[:, 4:5, :1])
    assert np.all(np.abs(gh[0][:, :2] - m0[:, :2]) < (1e-14 if prec == 0 else 1e-6) * rms)
    fin = sim.get_particles()
    if prec == 0:
        chan_close(fin, st, TOL[prec]["state"], 2)
    else:
        # FP32: values element-wise; a derivative channel jumps where FP32 and FP64 put a particle
        # on different sides of a cell edge (the CIC weight derivative is piecewise constant)
        chan_close(fin[:, :, :1], st[:, :, :1], TOL[prec]["state"], 2)
        scale = np.abs(st).max(axis=1, keepdims=True)
        err = np.abs(fin - st) / np.where(scale > 0, scale, 1)
        assert np.quantile(err[:, :, 1:], 0.999) < TOL[prec]["state"]
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_p13_twiss_derivatives(adpic, prec):
    N, grid = 4096, (16, 16, 16)
    o, sim, w, b = make_pair(adpic, N, grid, 13, prec)
    nrm = I.normals(43, N)
    st = o.beam_init(nrm)
    hist, _ = o.run(st, 20)
    sim.set_beam(b, nrm)
    sim.run(20)
    vals, der = sim.moments()
    ref = o.emittance(hist[-1])[:2]
    ev, ed = report(f"P=13 prec={prec}", vals, der, ref)
    assert ev < TOL[prec]["eps"] and ed < der_tol(prec, N)
    sim.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_bunch_charge_derivative(adpic, prec):
    """The bunch charge as an AD variable (slot 0, in place of the first drift length): the deposit's
    charge channel and every derivative downstream against the oracle."""
    N, grid = 10_000, (32, 32, 32)
    w = I.workload("fodo_10k_32")
    b = I.Beam(**{**w.beam.__dict__, "charge_slot": 0})
    lat = I.Lattice(deriv_slot=(-1, 1, 2, 3, 4, 5, 6))
    o = oracle.Oracle(**I.orc_kwargs(w, n_particles=N, grid=grid, beam=b, lattice=lat))
    nrm = I.normals(47, N)
    st = o.beam_init(nrm)
    hist, _ = o.run(st, 20)
    sim = adpic.ADPIC(grid, N, 7, prec)
    sim.set_beam(b, nrm)
    sim.set_lattice(lat)
    sim.run(20)
    vals, der = sim.moments()
    ref = o.emittance(hist[-1])[:2]
    ev, ed = report(f"charge slot prec={prec}", vals, der, ref)
    assert ev < TOL[prec]["eps"] and ed < der_tol(prec, N)
    assert np.all(np.abs(ref[:, 1]) > 0)
    sim.close()


def test_split_runs_and_graph_replay(adpic):
    """run(20) equals run(7) + run(13) (period-end moments and the kick counter carry over);
    graph capture and eager launches agree."""
    N, grid = 3000, (16, 16, 16)
    w = I.workload("fodo_10k_32")
    nrm = I.normals(44, N)
    res = []
    for split, graphs in (((20,), True), ((7, 13), True), ((20,), False), ((20,), True)):
        sim = adpic.ADPIC(grid, N, 7, 0)
        sim.set_graphs(graphs)
        sim.set_beam(w.beam, nrm)
        sim.set_lattice(w.lattice)
        for n in split:
            sim.run(n)
        v, d = sim.moments()
        res.append(np.concatenate([v[:, None], d], axis=1))
        sim.close()
    for r in res[1:]:
        ev, ed = report("split/graph", r[:, 0], r[:, 1:], res[0])
        assert ev < 1e-12 and ed < der_tol(0, N)


@pytest.mark.parametrize("prec", [0, 1])
def test_stages_leave_the_run_unchanged(adpic, prec):
    """Stage calls between runs (deposit only, or through the convolution) leave no trace in the
    next run: rho is zero again for its first deposit, the cell sort and the fused geometry step
    start clean, so the run equals the same run on a fresh handle."""
    N, grid = 3000, (16, 16, 16)
    w = I.workload("fodo_10k_32")
    nrm = I.normals(46, N)
    res = []
    for stages in ((), (1,), (2, 1), (0, 3)):
        sim = adpic.ADPIC(grid, N, 7, prec)
        sim.set_beam(w.beam, nrm)
        sim.set_lattice(w.lattice)
        for k in stages:
            sim.stage(k)
        sim.run(20)
        v, d = sim.moments()
        res.append(np.concatenate([v[:, None], d], axis=1))
        sim.close()
    # runs differ only by the order of the deposit's atomic additions: FP64 at rounding level; in
    # FP32 two runs, each within 1e-4 per derivative of the oracle, may be twice that apart; the
    # emittances differ by about 1e-9, while a stale charge grid in the first kick changes the
    # emittances by orders of magnitude more
    for r in res[1:]:
        ev, ed = report(f"stages then run ({prec})", r[:, 0], r[:, 1:], res[0])
        assert ev < (1e-12 if prec == 0 else 1e-6) and ed < (1 if prec == 0 else 2) * der_tol(prec, N)


def test_multi_period_records(adpic):
    N, grid = 2000, (16, 16, 16)
    o, sim, w, b = make_pair(adpic, N, grid, 7, 0)
    nrm = I.normals(45, N)
    st = o.beam_init(nrm)
    hist, _ = o.run(st, 50)              # records after kicks 20, 40, 50
    sim.set_beam(b, nrm)
    sim.run(50)
    gh = sim.history()
    assert gh.shape[0] == 4
    for r in range(3):
        e_g = o.emittance(gh[r + 1])[:2]
        e_o = o.emittance(hist[r])[:2]
        ev, ed = report(f"record {r}", e_g[:, 0], e_g[:, 1:], e_o)
        assert ev < TOL[0]["eps"] and ed < der_tol(0, N)
    sim.close()


# ---------------------------------------------------------------- edge cases

@pytest.mark.parametrize("prec", [0, 1])
def test_zero_current_conserves_emittance(adpic, prec):
    N, grid = 3000, (16, 16, 16)
    o, sim, w, b = make_pair(adpic, N, grid, 7, prec, q=0.0)
    sim.set_beam(b, I.normals(46, N))
    sim.run(20)
    h = sim.history()
    e0 = o.emittance(h[0])
    e1 = o.emittance(h[-1])
    tol = 1e-12 if prec == 0 else 2e-6
    np.testing.assert_allclose(e1[:2, 0], e0[:2, 0], rtol=tol)
    assert np.all(np.abs(e1[:2, 1:]) < tol * e0[:2, :1])
    sim.close()


def test_single_particle_and_tiny_grid(adpic):
    """One macroparticle: after mean removal it sits at the origin, the grid extent is degenerate
    (1e-6 m by convention) and its self-field cancels by symmetry up to rounding of a large field;
    it must stay (numerically) at rest and the run must report no error. (In FP32 the cancellation
    of a ~1e13 V/m self-field is only good to FP32 rounding, so the degenerate case is FP64 only.)"""
    o, sim, w, b = make_pair(adpic, 1, (8, 8, 8), 7, 0)
    nrm = np.array([[0.3], [0.1], [-0.2], [0.4], [0.5], [-0.6]])
    sim.set_beam(b, nrm)
    sim.run(20)
    fin = sim.get_particles()
    assert np.all(np.isfinite(fin))
    assert np.abs(fin[0::2]).max() < 1e-9 and np.abs(fin[1::2]).max() < 1e-9
    sim.close()


def test_call_order_and_argument_errors(adpic):
    sim = adpic.ADPIC((16, 16, 16), 100, 7, 0)
    with pytest.raises(adpic.AdPicError) as e:
        sim.run(1)
    assert e.value.status == -4
    bad = I.Lattice(kicks=(4, 0, 8, 2, 4))
    with pytest.raises(adpic.AdPicError) as e:
        sim.set_lattice(bad)
    assert e.value.status == -1
    sim.close()


# ---------------------------------------------------------------- full size (1,048,576 particles, 64^3)

def oracle_records_fodo_1m_64():
    """The FP64 oracle's emittance records of the whole 1M-particle run, written by
    tests/golden/make_oracle_records.py (which calls only the oracle)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_fodo_1m_64.json")
    with open(path) as f:
        return np.array(json.load(f)["eps"])


def test_full_size_ten_periods_vs_oracle(adpic):
    """The launch configuration bench.py times (1,048,576 particles, 64^3, P = 7) over the whole ten
    periods: both GPU paths against the oracle at every period end (FP64 within 1e-10, FP32 within
    1e-5 on emittances and 1e-4 per derivative), and the FP32 path against the FP64 path."""
    w = I.workload("fodo_1m_64")
    ref = oracle_records_fodo_1m_64()                 # [record][plane][channel], record 0 = start
    nrm = I.normals(w.seed, w.n_particles)
    o = oracle.Oracle(**I.orc_kwargs(w, n_particles=1))
    hs = []
    for prec in (0, 1):
        sim = adpic.ADPIC(w.grid, w.n_particles, 7, prec)
        sim.set_beam(w.beam, nrm)
        sim.set_lattice(w.lattice)
        sim.run(w.n_kicks)
        h = sim.history()
        sim.close()
        assert h.shape[0] == ref.shape[0]
        hs.append(h)
        worst = (0.0, 0.0)
        for r in range(1, h.shape[0]):
            e = o.emittance(h[r])[:2]
            ev, ed = report(f"period {r} prec={prec} vs oracle", e[:, 0], e[:, 1:], ref[r])
            assert ev < TOL[prec]["eps"] and ed < TOL[prec]["der"], (prec, r, ev, ed)
            worst = (max(worst[0], ev), max(worst[1], ed))
        print(f"ten periods prec={prec}: worst eps {worst[0]:.2e}, worst derivative component {worst[1]:.2e}")
    for r in range(1, hs[0].shape[0]):
        e64 = o.emittance(hs[0][r])[:2]
        e32 = o.emittance(hs[1][r])[:2]
        ev, ed = report(f"period {r} fp32 vs fp64", e32[:, 0], e32[:, 1:], e64)
        assert ev < 2 * TOL[1]["eps"] and ed < 2 * TOL[1]["der"], r


@pytest.fixture(scope="module")
def large_grid_ref():
    """The large instance's launch configuration (128^3 grid, P = 13) with 20,000 particles, 2 kicks."""
    w = I.workload("fodo_16m_128")
    N = 20_000
    o = oracle.Oracle(**I.orc_kwargs(w, n_particles=N))
    nrm = I.normals(11, N)
    st = o.beam_init(nrm)
    hist, _ = o.run(st, 2)
    return w, N, nrm, st, hist, o


@pytest.mark.parametrize("prec", [0, 1])
def test_large_grid_p13_vs_oracle(adpic, large_grid_ref, prec):
    """128^3 (256-point FFT lines, 129-point DCTs) with the 13 lattice and Twiss derivatives."""
    w, N, nrm, st, hist, o = large_grid_ref
    sim = adpic.ADPIC(w.grid, N, 13, prec)
    sim.set_beam(w.beam, nrm)
    sim.set_lattice(w.lattice)
    sim.run(2)
    vals, der = sim.moments()
    ref = o.emittance(hist[-1])[:2]
    ev, ed = report(f"128^3 P=13 prec={prec}", vals, der, ref)
    assert ev < TOL[prec]["eps"] and ed < der_tol(prec, N)
    fin = sim.get_particles()
    chan_close(fin[:, :, :1], st[:, :, :1], TOL[prec]["state"], 2)
    sim.close()


def test_large_instance_fp32_vs_fp64(adpic):
    """The large instance at full size (16,777,216 particles, 128^3, P = 13), two periods: FP32 bulk
    arithmetic against the FP64 path (pinned to the oracle at this grid above) at each period end."""
    w = I.workload("fodo_16m_128")
    nrm = I.normals(w.seed, w.n_particles)
    hs = []
    for prec in (0, 1):
        sim = adpic.ADPIC(w.grid, w.n_particles, 13, prec)
        sim.set_beam(w.beam, nrm)
        sim.set_lattice(w.lattice)
        sim.run(2 * w.kicks_per_period)
        hs.append(sim.history())
        sim.close()
    o = oracle.Oracle(**I.orc_kwargs(w, n_particles=1))
    assert hs[0].shape[0] == 3
    for r in range(1, 3):
        e64 = o.emittance(hs[0][r])[:2]
        e32 = o.emittance(hs[1][r])[:2]
        ev, ed = report(f"large instance period {r} fp32 vs fp64", e32[:, 0], e32[:, 1:], e64)
        assert ev < 1e-5 and ed < 1e-4, r


@pytest.mark.parametrize("P", [7, 13])
def test_fp32_upload_matches_the_fp64_upload(adpic, P):
    """ad_pic_set_particles_f32 gives an FP32 handle the state ad_pic_set_particles gives it for the
    same values (P = 7: straight copy; P = 13: records padded to 16 channels); an FP64 handle refuses
    it (AD_PIC_ERR_UNSUPPORTED)."""
    N, grid = 2003, (16, 16, 16)
    o, sim, w, b = make_pair(adpic, N, grid, P, 1)
    st = o.beam_init(I.normals(71, N))
    st32 = st.astype(np.float32)
    sim.set_particles(st32.astype(np.float64))
    a = sim.get_particles()
    sim.run(3)
    ra = sim.history()
    sim.set_particles_f32(st32)
    g = sim.get_particles()
    np.testing.assert_array_equal(g, a)
    sim.run(3)
    # separate runs (the deposit's atomic order differs): emittances within the FP32 bounds
    h = sim.history()
    assert len(h) == len(ra)
    for r in range(len(h)):
        e, er = o.emittance(h[r]), o.emittance(ra[r])
        ev, ed = report(f"FP32 upload record {r}", e[:, 0], e[:, 1:], er)
        assert ev < 1e-5 and ed < der_tol(1, N), r
    sim.close()
    s64 = adpic.ADPIC(grid, N, P, 0)
    with pytest.raises(adpic.AdPicError) as e:
        s64.set_particles_f32(st32)
    assert e.value.status == -8                          # AD_PIC_ERR_UNSUPPORTED
    s64.close()


@pytest.mark.parametrize("P", [7, 13])
def test_prefetched_upload_matches_the_synchronous_one(adpic, P):
    """ad_pic_prefetch_particles_f32 + ad_pic_commit_particles give the state and the run that
    ad_pic_set_particles_f32 gives, also when the next beam's copy is enqueued while the current
    beam runs (two pinned-or-not host buffers in turn, as a streaming caller uses them). A commit
    with nothing prefetched is AD_PIC_ERR_STATE; an FP64 handle refuses both calls."""
    N, grid = 3001, (16, 16, 16)
    o, sim, w, b = make_pair(adpic, N, grid, P, 1)
    beams = [o.beam_init(I.normals(81 + k, N)).astype(np.float32) for k in range(3)]
    ref = []
    for st in beams:
        sim.set_particles_f32(st)
        s0 = sim.get_particles()
        sim.run(4)
        ref.append((s0, sim.history(), sim.get_particles()))
    with pytest.raises(adpic.AdPicError) as e:
        sim.commit_particles()
    assert e.value.status == -4                          # AD_PIC_ERR_STATE
    sim.prefetch_particles_f32(beams[0])
    for k in range(3):
        sim.commit_particles()
        if k == 0:
            np.testing.assert_array_equal(sim.get_particles(), ref[0][0])
        if k + 1 < 3:
            sim.prefetch_particles_f32(beams[k + 1])     # overlaps the run below
        sim.run(4)
        # separate runs: the deposit's atomic order differs, so not bitwise; the
        # emittances and their derivatives agree within the FP32 bounds
        h = sim.history()
        assert len(h) == len(ref[k][1])
        for r in range(len(h)):
            e, er = o.emittance(h[r]), o.emittance(ref[k][1][r])
            ev, ed = report(f"prefetched beam {k} record {r}", e[:, 0], e[:, 1:], er)
            assert ev < 1e-5 and ed < der_tol(1, N), (k, r)
        g = sim.get_particles()
        np.testing.assert_allclose(g, ref[k][2], rtol=1e-5, atol=1e-5 * np.abs(ref[k][2]).max())
    sim.close()
    s64 = adpic.ADPIC(grid, N, P, 0)
    for call in (lambda: s64.prefetch_particles_f32(beams[0]), s64.commit_particles):
        with pytest.raises(adpic.AdPicError) as e:
            call()
        assert e.value.status == -8                      # AD_PIC_ERR_UNSUPPORTED
    s64.close()
