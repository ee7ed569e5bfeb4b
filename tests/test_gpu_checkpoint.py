"""Checkpoint and resume through the C ABI: run 2k kicks = run k, save, load into a fresh handle,
run k. The two runs differ only in the order of the deposit's floating-point atomic additions (the
same as two uninterrupted runs), so FP64 agrees to rounding level (emittances 1e-12, each derivative
within the FP64 floor at this size, particle values 1e-9 of their channel's max) and FP32 within the
FP32 path's own spread (emittances 1e-6, twice the FP32 derivative bound). A checkpoint in the middle
of a period adds one moment record (every run records after its last kick); the records at period
ends are the same."""
import os

import numpy as np
import pytest

from paper_2511_21839_gb300 import inputs as I
from parity_metrics import der_tol, rel_der_components, rel_eps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adpic():
    from paper_2511_21839_gb300 import adpic as A
    from paper_2511_21839_gb300 import build

    build.build()
    return A


@pytest.mark.parametrize("prec,P,k", [(0, 7, 30), (1, 7, 30), (0, 13, 10), (1, 13, 10)])
def test_resume_equals_uninterrupted_run(adpic, tmp_path, prec, P, k):
    N, grid = 4001, (16, 16, 16)
    w = I.workload("fodo_10k_32")
    beam = w.beam if P == 7 else I.default_beam(13)
    nrm = I.normals(81, N)

    def make():
        sim = adpic.ADPIC(grid, N, P, prec)
        sim.set_beam(beam, nrm)
        sim.set_lattice(w.lattice)
        return sim

    whole = make()
    whole.run(2 * k)
    v1, d1 = whole.moments()
    h1 = whole.history()
    s1 = whole.get_particles()
    whole.close()

    first = make()
    first.run(k)
    path = str(tmp_path / "ckpt.bin")
    first.save(path)
    first.close()
    second = adpic.ADPIC(grid, N, P, prec)              # a fresh handle: everything comes from the file
    second.load(path)
    second.run(k)
    v2, d2 = second.moments()
    h2 = second.history()
    s2 = second.get_particles()
    second.close()

    kpp = sum(w.lattice.kicks)
    if k % kpp:                                          # the extra record of the first run's last kick
        h2 = np.delete(h2, 1 + k // kpp, axis=0)
    assert h2.shape == h1.shape                          # the history continues across the checkpoint
    ev = rel_eps(v2, v1).max()
    ed = rel_der_components(d2, d1).max()
    print(f"resume prec={prec} P={P}: eps {ev:.2e}, derivative per component {ed:.2e}")
    assert ev < (1e-12 if prec == 0 else 1e-6) and ed < (1 if prec == 0 else 2) * der_tol(prec, N)
    np.testing.assert_allclose(h2[:, :, 2:], h1[:, :, 2:], rtol=1e-9 if prec == 0 else 1e-4,
                               atol=1e-9 * np.abs(h1[:, :, 2:]).max())
    scale = np.abs(s1).max(axis=1, keepdims=True)
    err = np.abs(s2 - s1) / np.where(scale > 0, scale, 1)
    assert err[:, :, 0].max() < (1e-9 if prec == 0 else 2e-4)


def test_load_rejects_another_configuration(adpic, tmp_path):
    w = I.workload("fodo_10k_32")
    sim = adpic.ADPIC((16, 16, 16), 1000, 7, 0)
    sim.set_beam(w.beam, I.normals(82, 1000))
    sim.set_lattice(w.lattice)
    path = str(tmp_path / "a.bin")
    sim.save(path)
    sim.close()
    other = adpic.ADPIC((16, 16, 16), 1001, 7, 0)
    with pytest.raises(adpic.AdPicError) as e:
        other.load(path)
    assert e.value.status == -1
    with pytest.raises(adpic.AdPicError) as e:
        other.load(str(tmp_path / "missing.bin"))
    assert e.value.status == -9
    with open(path, "r+b") as f:                         # a truncated file
        f.truncate(200)
    same = adpic.ADPIC((16, 16, 16), 1000, 7, 0)
    with pytest.raises(adpic.AdPicError) as e:
        same.load(path)
    assert e.value.status == -9
    with pytest.raises(adpic.AdPicError) as e:           # no particles after a failed load
        same.run(1)
    assert e.value.status == -4
    other.close()
    same.close()
