"""Failure detection without a GPU fault: every failure here is made on the host or by a bounded
wait that runs out, and every case checks the status the host reads and that the handle stays usable
(or at least destroyable).

- A push whose tile waits may not poll at all gives up: ad_pic_run returns AD_PIC_ERR_TIMEOUT,
  the particles must be set again, and the next run (default limit) equals a fresh handle's run.
- The default limit's duration is measured: a wait that runs out all of its polls.
- A non-finite coordinate gives AD_PIC_ERR_NONFINITE; coordinates whose span overflows FP32 in the
  cell computation give AD_PIC_ERR_OUT_OF_GRID (the index clamp keeps every access in bounds).
- Host-side injection (ADPIC_FAULT) of a failed allocation and a failed launch.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2511_21839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N, GRID = 3000, (16, 16, 16)


@pytest.fixture(scope="module")
def adpic():
    from paper_2511_21839_gb300 import adpic as A
    from paper_2511_21839_gb300 import build

    build.build()
    return A


def fresh(adpic, prec, nrm):
    w = I.workload("fodo_10k_32")
    sim = adpic.ADPIC(GRID, N, 7, prec)
    sim.set_beam(w.beam, nrm)
    sim.set_lattice(w.lattice)
    return sim


@pytest.mark.parametrize("prec", [0, 1])
def test_push_wait_runs_out(adpic, prec):
    nrm = I.normals(71, N)
    ref = fresh(adpic, prec, nrm)
    ref.run(20)
    v_ref, d_ref = ref.moments()
    ref.close()

    sim = fresh(adpic, prec, nrm)
    start = sim.get_particles()
    sim.set_wait_limit(0)
    with pytest.raises(adpic.AdPicError) as e:
        sim.run(3)
    assert e.value.status == -7                        # AD_PIC_ERR_TIMEOUT
    with pytest.raises(adpic.AdPicError) as e:          # the state is not valid any more
        sim.get_particles()
    assert e.value.status == -4
    with pytest.raises(adpic.AdPicError) as e:
        sim.run(1)
    assert e.value.status == -4
    # set the state again, default limit: the error word starts clear and the run equals a fresh one
    sim.set_wait_limit(-1)
    sim.set_particles(start)
    sim.run(20)
    v, d = sim.moments()
    sim.close()
    np.testing.assert_allclose(v, v_ref, rtol=1e-12 if prec == 0 else 1e-6)
    scale = np.abs(d_ref).max(axis=1, keepdims=True)
    assert np.abs(d - d_ref).max() < (1e-10 if prec == 0 else 2e-4) * scale.max()


def test_default_wait_limit_is_bounded(adpic):
    """The push gives up after 2^18 failed polls; a wait that runs out all of them ends within a
    second on the device (each failed poll suspends the thread for a system-dependent time)."""
    ms_small, failed = adpic.ad_pic_wait_probe(1 << 12)
    assert failed == 1 << 12
    projected = ms_small * (1 << 6)
    print(f"2^12 failed polls: {ms_small:.3f} ms (2^18 projected {projected:.1f} ms)")
    assert projected < 5000.0
    ms, failed = adpic.ad_pic_wait_probe(1 << 18)
    print(f"2^18 failed polls: {ms:.1f} ms ({1e3 * ms / (1 << 18):.2f} us per poll)")
    assert failed == 1 << 18
    assert ms < 1000.0


@pytest.mark.parametrize("prec", [0, 1])
def test_nonfinite_coordinate_is_reported(adpic, prec):
    nrm = I.normals(72, N)
    sim = fresh(adpic, prec, nrm)
    st = sim.get_particles()
    bad = st.copy()
    bad[2, 17, 0] = np.nan                              # one particle's y
    sim.set_particles(bad)
    with pytest.raises(adpic.AdPicError) as e:
        sim.run(2)
    assert e.value.status == -5                         # AD_PIC_ERR_NONFINITE
    # the handle stays usable: a finite state runs clean
    sim.set_particles(st)
    sim.run(2)
    assert np.all(np.isfinite(sim.moments()[0]))
    sim.close()


def test_out_of_grid_is_reported(adpic):
    """Two particles at +-3e38 m: the grid geometry (FP64) is finite, but (x - origin) / h overflows
    FP32 for the far particle, so its cell falls outside the stencil range; the index is clamped
    and the run reports AD_PIC_ERR_OUT_OF_GRID."""
    nrm = I.normals(73, N)
    sim = fresh(adpic, 1, nrm)
    st = sim.get_particles()
    bad = st.copy()
    bad[0, 5, 0] = 3e38
    bad[0, 6, 0] = -3e38
    sim.set_particles(bad)
    with pytest.raises(adpic.AdPicError) as e:
        sim.stage(1)                                    # the deposit of the current state
    assert e.value.status in (-6, -5)
    with pytest.raises(adpic.AdPicError) as e:
        sim.run(1)
    assert e.value.status in (-6, -5)
    sim.set_particles(st)
    sim.run(1)
    sim.close()


@pytest.mark.parametrize("after", [0, 5])
def test_injected_allocation_failure(adpic, after, monkeypatch):
    monkeypatch.setenv("ADPIC_FAULT", f"alloc:{after}")
    with pytest.raises(adpic.AdPicError) as e:
        adpic.ADPIC(GRID, N, 7, 0)
    assert e.value.status == -2                         # AD_PIC_ERR_OOM, nothing leaked to the caller
    monkeypatch.delenv("ADPIC_FAULT")
    sim = adpic.ADPIC(GRID, N, 7, 0)                    # and the next handle is fine
    sim.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_injected_launch_failure(adpic, graphs, monkeypatch):
    nrm = I.normals(74, N)
    ref = fresh(adpic, 0, nrm)
    ref.run(20)
    v_ref, _ = ref.moments()
    ref.close()
    sim = fresh(adpic, 0, nrm)
    sim.set_graphs(graphs)
    monkeypatch.setenv("ADPIC_FAULT", "launch")
    with pytest.raises(adpic.AdPicError) as e:
        sim.run(20)
    assert e.value.status == -3                         # AD_PIC_ERR_CUDA; nothing advanced
    monkeypatch.delenv("ADPIC_FAULT")
    sim.run(20)
    v, _ = sim.moments()
    sim.close()
    np.testing.assert_allclose(v, v_ref, rtol=1e-12)
