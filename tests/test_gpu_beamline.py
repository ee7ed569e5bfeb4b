"""The dual PIC on a general beamline (ad_pic_set_beamline) against the oracle, and the space-charge
re-matching of the matching section with BFGS on dual-PIC gradients (Sec. 4).

Bounds as in tests/parity_metrics.py: FP64 emittances 1e-10 and derivatives der_tol(0, N); FP32
emittances 1e-5 and derivatives der_tol(1, N).
"""
import numpy as np
import pytest

import oracle
from paper_2511_21839_gb300 import inputs as I
from parity_metrics import der_tol, report

pytestmark = pytest.mark.gpu

LINE = [(0, 0.3, 0.0, 4, -1), (1, 0.1, 21.0, -1, 0), (0, 0.3, 0.0, -1, -1), (1, 0.1, -19.5, -1, 1),
        (0, 0.3, 0.0, 5, -1), (1, 0.1, 18.0, 6, 2), (0, 0.3, 0.0, -1, -1), (1, 0.1, -20.5, -1, 3),
        (0, 0.3, 0.0, -1, -1)]
KICKS = [3, 2, 3, 2, 3, 2, 3, 2, 3]


@pytest.fixture(scope="module")
def adpic():
    from paper_2511_21839_gb300 import adpic as A
    from paper_2511_21839_gb300 import build

    build.build()
    return A


@pytest.mark.parametrize("prec", [0, 1])
def test_beamline_run_vs_oracle(adpic, prec):
    """Two passes through a strongly focusing matching section with a 100 A bunch (at the FODO's
    0.12 nC the emittance derivatives w.r.t. the strengths are a few 1e-5 of the emittance per unit k,
    so small that their errors are those of the emittance itself)."""
    from paper_2511_21839_gb300 import design

    N, grid = 10_000, (32, 32, 32)
    w = I.workload("fodo_10k_32")
    beam = I.Beam(**{**w.beam.__dict__, "bunch_charge_C": design.bunch_charge_for_current(100.0)})
    kw = I.orc_kwargs(w, n_particles=N, grid=grid, beam=beam)
    o = oracle.Oracle(line=LINE, line_kicks=KICKS, **kw)
    nrm = I.normals(31, N)
    st = o.beam_init(nrm)
    hist, _ = o.run(st, 2 * sum(KICKS))                 # two passes: records at both pass ends
    sim = adpic.ADPIC(grid, N, 7, prec)
    sim.set_beam(beam, nrm)
    sim.set_beamline(LINE, KICKS)
    sim.run(2 * sum(KICKS))
    h = sim.history()
    assert h.shape[0] == 3
    for r in (1, 2):
        e = o.emittance(h[r])[:2]
        ref = o.emittance(hist[r - 1])[:2]
        ev, ed = report(f"beamline pass {r} prec={prec}", e[:, 0], e[:, 1:], ref)
        assert ev < (1e-10 if prec == 0 else 1e-5) and ed < der_tol(prec, N)
    sim.close()


def test_beamline_checkpoint_carries_the_line(adpic, tmp_path):
    N, grid = 3000, (16, 16, 16)
    w = I.workload("fodo_10k_32")
    nrm = I.normals(32, N)

    def make():
        s = adpic.ADPIC(grid, N, 7, 0)
        s.set_beam(w.beam, nrm)
        s.set_beamline(LINE, KICKS)
        return s

    a = make()
    a.run(2 * sum(KICKS))
    va, _ = a.moments()
    a.close()
    b = make()
    b.run(sum(KICKS))
    path = str(tmp_path / "line.bin")
    b.save(path)
    b.close()
    c = adpic.ADPIC(grid, N, 7, 0)
    c.load(path)
    c.run(sum(KICKS))
    vc, _ = c.moments()
    c.close()
    np.testing.assert_allclose(vc, va, rtol=1e-12)


def test_space_charge_rematching_with_bfgs(adpic):
    """Sec. 4: at 100 A the zero-current matching solution no longer delivers the second lattice's
    Twiss functions; BFGS on dual-PIC gradients, warm-started from the zero-current solution, brings
    Eq. 6 down by orders of magnitude. The rms envelope through eight cells of the second lattice is
    printed for both settings (the target is the second lattice's zero-current periodic solution,
    which a space-charge-depressed beam does not keep exactly)."""
    from paper_2511_21839_gb300 import design

    pm = design.PicMatch(current_A=100.0, n_particles=16384, grid=32)
    k_zero, f_zero_optics, n_opt = pm.zero.bfgs([20.0, -20.0, 20.0, -20.0], ftol=1e-14)
    f_start, _ = pm.objective(k_zero)
    k_sc, f_sc, evals = pm.bfgs(k_zero, ftol=1e-9)
    print(f"zero-current match: optics f = {f_zero_optics:.1e} ({n_opt} evaluations); with 100 A space charge "
          f"f = {f_start:.3e}; after {evals} dual-PIC evaluations f = {f_sc:.3e}; strengths {k_zero} -> {k_sc}")
    assert f_start > 1e-4                      # space charge spoils the zero-current match
    assert f_sc < 1e-3 * f_start
    beat0 = pm.envelope_beat(k_zero)
    beat1 = pm.envelope_beat(k_sc)
    print(f"envelope beat over 8 cells (x, y): zero-current match {beat0}, space-charge match {beat1}")
    assert np.all(np.isfinite(beat0)) and np.all(np.isfinite(beat1))
    # every evaluation is verified by the oracle at the optimum: one more run of the oracle's PIC
    line, kicks = pm.section(k_sc)
    w = I.workload("fodo_10k_32")
    o = oracle.Oracle(line=line, line_kicks=kicks,
                      **I.orc_kwargs(w, n_particles=pm.N, grid=pm.grid, n_deriv=7, beam=pm.beam))
    st = o.beam_init(pm.normals)
    hist, _ = o.run(st, sum(kicks))
    t_gpu = pm.twiss(k_sc)
    t_orc = design.beam_twiss(hist[-1], 4)
    np.testing.assert_allclose(t_gpu[:, 0], t_orc[:, 0], rtol=1e-10)
    pm.close()


def test_rematching_from_cold_optics_and_surrogate_starts(adpic):
    """The Eq. 6 re-matching at 100 A from three starts, dual-PIC evaluations counted until f <= 1e-9
    (reported):
    cold BFGS from the generic guess (+-20 m^-2), BFGS warm-started from the zero-current optics
    solution, and the surrogate warm start (Sec. 4 and the learned-surrogate search: a 4 -> 128^3 -> 4
    MLP fitted with the Sobolev loss to dual-PIC runs within +-20 % of the zero-current solution, every
    proposal checked by a full dual-PIC run)."""
    from paper_2511_21839_gb300 import design

    pm = design.PicMatch(current_A=100.0, n_particles=16384, grid=32)
    k_zero, _, _ = pm.zero.bfgs([20.0, -20.0, 20.0, -20.0], ftol=1e-14)
    ftol = 1e-9
    k_c, f_c, n_cold = pm.bfgs([20.0, -20.0, 20.0, -20.0], ftol=ftol)
    k_o, f_o, n_opt = pm.bfgs(k_zero, ftol=ftol)
    k_s, f_s, n_sur, n_train, errs = design.surrogate_rematch(pm, k_zero, ftol=ftol)
    print(f"dual-PIC evaluations to f <= {ftol:.0e}: cold {n_cold} (f {f_c:.1e}), optics warm start {n_opt} "
          f"(f {f_o:.1e}), surrogate warm start {n_sur} (f {f_s:.1e}; surrogate trained on {n_train} runs, "
          f"held-out value/derivative errors {errs[0]:.3f}/{errs[1]:.3f})")
    print(f"strengths: cold {k_c}, optics start {k_o}, surrogate start {k_s}")
    # all three reach the target and the same matching solution; the counts are reported, not ranked:
    # with exact dual-PIC gradients this 4-parameter problem takes BFGS 15-30 evaluations from any of
    # the starts (the surrogate pays off on the 7-parameter emittance search, test_gpu_surrogate.py)
    assert max(f_c, f_o, f_s) <= ftol
    np.testing.assert_allclose(k_c, k_o, rtol=1e-3)
    np.testing.assert_allclose(k_s, k_o, rtol=1e-3)
    assert errs[0] < 0.05 and errs[1] < 0.1
    pm.close()
