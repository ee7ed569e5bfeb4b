"""The allocation-free moment entry point against the regular one.

ad_pic_moments_device exists for callers that cannot let the library
allocate device memory (code inside another framework's memory budget, or
latency-critical loops that must not take the synchronisation cudaMalloc and
cudaFree can bring). It reduces a caller-owned device state with its
partial sums in a static device array. This file is collected last so that a
failure here stops a -x run only after every other test has run.
"""
import numpy as np
import pytest

import oracle
from paper_2511_21839_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def term_scale(state):
    """Mean |term| of every summed quantity [3][5][C]: u_k, p_k and the dual products of Eq. 2."""
    out = np.zeros((3, 5, state.shape[2]))
    for pl in range(3):
        u, p = state[2 * pl], state[2 * pl + 1]
        u0, p0 = u[:, :1], p[:, :1]
        out[pl, 0] = np.abs(u).mean(axis=0)
        out[pl, 1] = np.abs(p).mean(axis=0)
        out[pl, 2] = np.abs(2 * u0 * u).mean(axis=0)
        out[pl, 3] = (np.abs(u0 * p) + np.abs(p0 * u)).mean(axis=0)
        out[pl, 4] = np.abs(2 * p0 * p).mean(axis=0)
    return np.where(out > 0, out, 1.0)


@pytest.mark.parametrize("prec,P", [(0, 7), (1, 7), (0, 13), (1, 13)])
def test_no_alloc_moments_match_regular_entry_point(prec, P):
    torch = pytest.importorskip("torch")
    from paper_2511_21839_gb300 import adpic, build

    build.build()
    N, grid = 100_003, (16, 16, 16)
    w = I.workload("fodo_10k_32")
    beam = w.beam if P == 7 else I.default_beam(13)
    o = oracle.Oracle(**I.orc_kwargs(w, n_particles=N, grid=grid, n_deriv=P, beam=beam))
    state = o.beam_init(I.normals(61, N))
    o.apply_half_map(state, 0)

    # regular entry point: upload, zero-kick run records the moments of the state
    sim = adpic.ADPIC(grid, N, P, prec)
    sim.set_beam(beam)
    sim.set_lattice(w.lattice)
    sim.set_particles(state)
    sim.run(0)
    ref = sim.moments_full()
    sim.close()

    C, CP = P + 1, (8 if P == 7 else 16)
    dtype = torch.float64 if prec == 0 else torch.float32
    dev = torch.zeros((6, N, CP), dtype=dtype, device="cuda")
    dev[:, :, :C] = torch.from_numpy(state).to(dtype=dtype, device="cuda")
    stream = torch.cuda.current_stream()
    tol = 1e-12 if prec == 0 else 1e-6
    for call in range(2):
        out = torch.full((15 * CP,), float("nan"), dtype=torch.float64, device="cuda")
        adpic.ad_pic_moments_device(dev.data_ptr(), N, P, prec, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        full = out.cpu().numpy().reshape(3, 5, CP)
        assert np.all(full[:, :, C:] == 0), call          # padding channels carry nothing
        got = full[:, :, :C]
        assert np.all(np.isfinite(got)), call
        # two summation orders of the same terms differ by rounding relative to the mean absolute
        # term, not to the sum (a mean removed beam has means that are zero up to rounding)
        err = np.abs(got - ref) / term_scale(state)
        assert err.max() < tol, f"call {call}: max scaled error {err.max():.3e}"


def test_no_alloc_small_call_after_large_and_layout_change():
    """Calls share the partial-sum array and keep what the last call left there. After a call that
    fills all of its blocks, a call on 37 particles leaves almost every block without particles: those
    blocks must write zero partials, so the result equals the oracle's moments of the small state.
    Then a 13-derivative FP32 call follows a 7-derivative FP64 one (another channel layout of the
    same array)."""
    torch = pytest.importorskip("torch")
    from paper_2511_21839_gb300 import adpic, build

    build.build()
    w = I.workload("fodo_10k_32")
    stream = torch.cuda.current_stream()

    def call(state, P, prec):
        N, C = state.shape[1], P + 1
        CP = 8 if P == 7 else 16
        dtype = torch.float64 if prec == 0 else torch.float32
        dev = torch.zeros((6, N, CP), dtype=dtype, device="cuda")
        dev[:, :, :C] = torch.from_numpy(state).to(dtype=dtype, device="cuda")
        out = torch.full((15 * CP,), float("nan"), dtype=torch.float64, device="cuda")
        adpic.ad_pic_moments_device(dev.data_ptr(), N, P, prec, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        full = out.cpu().numpy().reshape(3, 5, CP)
        assert np.all(full[:, :, C:] == 0)
        return full[:, :, :C]

    def beam(P, N, seed):
        b = w.beam if P == 7 else I.default_beam(13)
        o = oracle.Oracle(**I.orc_kwargs(w, n_particles=N, grid=(16, 16, 16), n_deriv=P, beam=b))
        st = o.beam_init(I.normals(seed, N))
        o.apply_half_map(st, 0)
        return o, st

    o_big, big = beam(7, 100_003, 62)
    call(big, 7, 0)                                          # every block gets particles
    o_small, small = beam(7, 37, 63)
    got = call(small, 7, 0)
    ref = o_small.moments(small)
    err = np.abs(got - ref) / term_scale(small)
    assert err.max() < 1e-12, err.max()
    o13, st13 = beam(13, 5_001, 64)
    got = call(st13.astype(np.float32).astype(np.float64), 13, 1)
    ref = o13.moments(st13.astype(np.float32).astype(np.float64))
    err = np.abs(got - ref) / term_scale(st13)
    assert err.max() < 1e-9, err.max()


def test_no_alloc_rejects_unsupported_sizes():
    pytest.importorskip("torch")
    from paper_2511_21839_gb300 import adpic, build

    build.build()
    with pytest.raises(adpic.AdPicError) as e:
        adpic.ad_pic_moments_device(1, 10, 20, 0, 1)
    assert e.value.status == -1
