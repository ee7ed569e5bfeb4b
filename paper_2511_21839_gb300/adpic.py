"""Thin ctypes binding of the C ABI in include/ad_pic.h (argument marshalling only).

Every entry point keeps its C name. The library must be built (see build.py);
importing this module on a machine where libadpic.so is missing raises at
load time: there is no CPU fallback.
"""
import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libadpic.so")

AD_PIC_FP64 = 0
AD_PIC_FP32_MIXED = 1

STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA runtime error", -4: "call out of order",
          -5: "non-finite particle coordinate", -6: "particle outside the grid stencil",
          -7: "bounded device wait timed out", -8: "unsupported",
          -9: "checkpoint file could not be read or written", -10: "cell has no periodic Twiss solution"}


class ad_pic_grid(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int)]


class ad_pic_lattice(ct.Structure):
    _fields_ = [("L", ct.c_double * 5), ("g", ct.c_double * 2), ("kicks", ct.c_int * 5), ("deriv_slot", ct.c_int * 7)]


class ad_pic_beam(ct.Structure):
    _fields_ = [("kinetic_eV", ct.c_double), ("mass_eV", ct.c_double), ("charge_e", ct.c_double),
                ("bunch_charge_C", ct.c_double), ("eps_n", ct.c_double * 3), ("alpha", ct.c_double * 3),
                ("beta", ct.c_double * 3), ("twiss_deriv_slot", ct.c_int * 6), ("charge_deriv_slot", ct.c_int),
                ("energy_deriv_slot", ct.c_int)]


AD_PIC_DRIFT = 0
AD_PIC_QUAD = 1


class ad_pic_element(ct.Structure):
    _fields_ = [("type", ct.c_int), ("slot_L", ct.c_int), ("slot_k", ct.c_int), ("pad", ct.c_int),
                ("L", ct.c_double), ("k", ct.c_double)]


class AdPicError(RuntimeError):
    def __init__(self, fn, status):
        super().__init__(f"{fn} failed: {STATUS.get(status, status)} ({status})")
        self.status = status


_lib = None


def lib():
    """Load libadpic.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first (paper_2511_21839_gb300/build.py)")
        L = ct.CDLL(LIB_PATH)
        vp = ct.c_void_p
        dp = ct.POINTER(ct.c_double)
        sig = {
            "ad_pic_create": (ct.c_int, [ct.POINTER(ad_pic_grid), ct.c_int64, ct.c_int, ct.c_int, ct.POINTER(vp)]),
            "ad_pic_set_beam": (ct.c_int, [vp, ct.POINTER(ad_pic_beam), dp]),
            "ad_pic_set_particles": (ct.c_int, [vp, dp]),
            "ad_pic_set_particles_f32": (ct.c_int, [vp, ct.POINTER(ct.c_float)]),
            "ad_pic_prefetch_particles_f32": (ct.c_int, [vp, ct.POINTER(ct.c_float)]),
            "ad_pic_commit_particles": (ct.c_int, [vp]),
            "ad_pic_get_particles": (ct.c_int, [vp, dp]),
            "ad_pic_set_lattice": (ct.c_int, [vp, ct.POINTER(ad_pic_lattice)]),
            "ad_pic_run": (ct.c_int, [vp, ct.c_int]),
            "ad_pic_moments": (ct.c_int, [vp, dp, dp]),
            "ad_pic_moments_full": (ct.c_int, [vp, dp]),
            "ad_pic_history": (ct.c_int, [vp, dp, ct.c_int, ct.POINTER(ct.c_int)]),
            "ad_pic_set_stream": (ct.c_int, [vp, vp]),
            "ad_pic_set_graphs": (ct.c_int, [vp, ct.c_int]),
            "ad_pic_set_timing": (ct.c_int, [vp, ct.c_uint]),
            "ad_pic_timing": (ct.c_int, [vp, dp, ct.POINTER(ct.c_int64), ct.c_int]),
            "ad_pic_kernel_name": (ct.c_char_p, [ct.c_int]),
            "ad_pic_kernel_classes": (ct.c_int, []),
            "ad_pic_stage": (ct.c_int, [vp, ct.c_int, ct.c_int64, dp]),
            "ad_pic_constants": (ct.c_int, [vp, dp]),
            "ad_pic_launches": (ct.c_int, [vp, ct.POINTER(ct.c_int64)]),
            "ad_pic_moments_device": (ct.c_int, [vp, ct.c_int64, ct.c_int, ct.c_int, vp, vp]),
            "ad_pic_fma_peak": (ct.c_int, [ct.c_int, dp]),
            "ad_pic_twiss_batch": (ct.c_int, [ct.c_int, ct.c_int, ct.POINTER(ad_pic_element), ct.c_int, ct.c_int,
                                              dp, dp]),
            "ad_pic_track_batch": (ct.c_int, [ct.c_int64, dp, ct.c_int, ct.POINTER(ad_pic_element), ct.c_int,
                                              ct.c_int64, dp, dp]),
            "ad_pic_set_beamline": (ct.c_int, [vp, ct.c_int, ct.POINTER(ad_pic_element), ct.POINTER(ct.c_int)]),
            "ad_pic2d_create": (ct.c_int, [ct.c_int, ct.c_int, ct.c_double, ct.c_double, ct.c_int64, ct.c_int,
                                           ct.c_int, ct.POINTER(vp)]),
            "ad_pic2d_set_beam": (ct.c_int, [vp, ct.POINTER(ad_pic_beam), ct.c_double, ct.c_int, dp]),
            "ad_pic2d_set_particles": (ct.c_int, [vp, dp]),
            "ad_pic2d_get_particles": (ct.c_int, [vp, dp]),
            "ad_pic2d_set_lattice": (ct.c_int, [vp, ct.POINTER(ad_pic_lattice)]),
            "ad_pic2d_run": (ct.c_int, [vp, ct.c_int]),
            "ad_pic2d_moments": (ct.c_int, [vp, dp, dp]),
            "ad_pic2d_moments_full": (ct.c_int, [vp, dp]),
            "ad_pic2d_history": (ct.c_int, [vp, dp, ct.c_int, ct.POINTER(ct.c_int)]),
            "ad_pic2d_destroy": (None, [vp]),
            "ad_pic_save": (ct.c_int, [vp, ct.c_char_p]),
            "ad_pic_load": (ct.c_int, [vp, ct.c_char_p]),
            "ad_pic_set_wait_limit": (ct.c_int, [vp, ct.c_int]),
            "ad_pic_wait_probe": (ct.c_int, [ct.c_int, dp, ct.POINTER(ct.c_int)]),
            "ad_pic_batch_create": (ct.c_int, [ct.c_int, ct.POINTER(ad_pic_grid), ct.POINTER(ct.c_int64), ct.c_int,
                                               ct.c_int, ct.POINTER(vp)]),
            "ad_pic_batch_set_beam": (ct.c_int, [vp, ct.c_int, ct.POINTER(ad_pic_beam), dp]),
            "ad_pic_batch_set_particles": (ct.c_int, [vp, ct.c_int, dp]),
            "ad_pic_batch_set_lattice": (ct.c_int, [vp, ct.c_int, ct.POINTER(ad_pic_lattice)]),
            "ad_pic_batch_moments": (ct.c_int, [vp, ct.c_int, dp, dp]),
            "ad_pic_batch_history": (ct.c_int, [vp, ct.c_int, dp, ct.c_int, ct.POINTER(ct.c_int)]),
            "ad_pic_batch_get_particles": (ct.c_int, [vp, ct.c_int, dp]),
            "ad_pic_batch_run": (ct.c_int, [vp, ct.c_int]),
            "ad_pic_batch_set_mode": (ct.c_int, [vp, ct.c_int]),
            "ad_pic_batch_tuning": (ct.c_int, [vp, ct.POINTER(ct.c_int), dp]),
            "ad_pic_batch_set_stream": (ct.c_int, [vp, vp]),
            "ad_pic_batch_set_tiles": (ct.c_int, [vp, ct.POINTER(ct.c_int)]),
            "ad_pic_batch_tiles": (ct.c_int, [vp, ct.POINTER(ct.c_int), dp]),
            "ad_pic_batch_destroy": (None, [vp]),
            "ad_pic_mlp_create": (ct.c_int, [ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.POINTER(vp)]),
            "ad_pic_mlp_num_params": (ct.c_int, [vp, ct.POINTER(ct.c_int64)]),
            "ad_pic_mlp_set_params": (ct.c_int, [vp, ct.POINTER(ct.c_float)]),
            "ad_pic_mlp_get_params": (ct.c_int, [vp, ct.POINTER(ct.c_float)]),
            "ad_pic_mlp_forward": (ct.c_int, [vp, ct.POINTER(ct.c_float), ct.c_int, ct.POINTER(ct.c_float),
                                              ct.POINTER(ct.c_float)]),
            "ad_pic_mlp_loss_grad": (ct.c_int, [vp, ct.POINTER(ct.c_float), ct.POINTER(ct.c_float),
                                                ct.POINTER(ct.c_float), ct.c_int, ct.c_float, dp,
                                                ct.POINTER(ct.c_float)]),
            "ad_pic_mlp_adam_step": (ct.c_int, [vp, ct.POINTER(ct.c_float), ct.POINTER(ct.c_float),
                                                ct.POINTER(ct.c_float), ct.c_int, ct.c_float, ct.c_float, dp]),
            "ad_pic_mlp_destroy": (None, [vp]),
            "ad_pic_mlp_set_dataset": (ct.c_int, [vp, ct.POINTER(ct.c_float), ct.POINTER(ct.c_float),
                                                  ct.POINTER(ct.c_float), ct.c_int]),
            "ad_pic_mlp_train": (ct.c_int, [vp, ct.c_int, ct.c_int, ct.c_float, ct.c_float, ct.c_float, dp, dp]),
            "ad_pic_destroy": (None, [vp]),
            "ad_pic_strerror": (ct.c_char_p, [ct.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _ck(fn, st):
    if st != 0:
        raise AdPicError(fn, st)


# ------------------------------------------------------------------ C names

def ad_pic_create(grid, n_particles, n_deriv, precision):
    h = ct.c_void_p()
    g = ad_pic_grid(*grid)
    _ck("ad_pic_create", lib().ad_pic_create(ct.byref(g), int(n_particles), int(n_deriv), int(precision), ct.byref(h)))
    return h


def ad_pic_set_beam(h, beam: ad_pic_beam, normals=None):
    nrm = None if normals is None else np.ascontiguousarray(normals, dtype=np.float64)
    _ck("ad_pic_set_beam", lib().ad_pic_set_beam(h, ct.byref(beam), None if nrm is None else _p(nrm)))


def ad_pic_set_particles(h, state):
    s = np.ascontiguousarray(state, dtype=np.float64)
    _ck("ad_pic_set_particles", lib().ad_pic_set_particles(h, _p(s)))


def ad_pic_set_particles_f32(h, state):
    s = np.ascontiguousarray(state, dtype=np.float32)
    _ck("ad_pic_set_particles_f32", lib().ad_pic_set_particles_f32(h, s.ctypes.data_as(ct.POINTER(ct.c_float))))


def ad_pic_prefetch_particles_f32(h, state):
    """Enqueue the asynchronous upload; returns the array whose memory is being
    copied, which the caller keeps alive and unchanged until the copy is done."""
    s = np.ascontiguousarray(state, dtype=np.float32)
    _ck("ad_pic_prefetch_particles_f32",
        lib().ad_pic_prefetch_particles_f32(h, s.ctypes.data_as(ct.POINTER(ct.c_float))))
    return s


def ad_pic_commit_particles(h):
    _ck("ad_pic_commit_particles", lib().ad_pic_commit_particles(h))


def ad_pic_get_particles(h, out):
    _ck("ad_pic_get_particles", lib().ad_pic_get_particles(h, _p(out)))
    return out


def ad_pic_set_lattice(h, lat: ad_pic_lattice):
    _ck("ad_pic_set_lattice", lib().ad_pic_set_lattice(h, ct.byref(lat)))


def ad_pic_run(h, n_steps):
    st = lib().ad_pic_run(h, int(n_steps))
    _ck("ad_pic_run", st)


def ad_pic_moments(h, P):
    v = np.zeros(2)
    d = np.zeros(2 * P)
    _ck("ad_pic_moments", lib().ad_pic_moments(h, _p(v), _p(d)))
    return v, d.reshape(2, P)


def ad_pic_moments_full(h, C):
    m = np.zeros((3, 5, C))
    _ck("ad_pic_moments_full", lib().ad_pic_moments_full(h, _p(m)))
    return m


def ad_pic_history(h, C):
    n = ct.c_int()
    _ck("ad_pic_history", lib().ad_pic_history(h, None, 0, ct.byref(n)))
    out = np.zeros((n.value, 3, 5, C))
    if n.value:
        _ck("ad_pic_history", lib().ad_pic_history(h, _p(out), n.value, ct.byref(n)))
    return out


def ad_pic_set_stream(h, stream_ptr):
    _ck("ad_pic_set_stream", lib().ad_pic_set_stream(h, ct.c_void_p(stream_ptr) if stream_ptr else None))


def ad_pic_set_graphs(h, enable):
    _ck("ad_pic_set_graphs", lib().ad_pic_set_graphs(h, int(bool(enable))))


def ad_pic_set_timing(h, mask):
    _ck("ad_pic_set_timing", lib().ad_pic_set_timing(h, int(mask)))


def ad_pic_timing(h):
    n = lib().ad_pic_kernel_classes()
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    _ck("ad_pic_timing", lib().ad_pic_timing(h, _p(ms), cnt.ctypes.data_as(ct.POINTER(ct.c_int64)), n))
    return {lib().ad_pic_kernel_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(n)}


def ad_pic_kernel_classes():
    return int(lib().ad_pic_kernel_classes())


def ad_pic_kernel_name(cls):
    return lib().ad_pic_kernel_name(int(cls)).decode()


def ad_pic_stage(h, stage, kick, out=None):
    _ck("ad_pic_stage", lib().ad_pic_stage(h, int(stage), int(kick), None if out is None else _p(out)))
    return out


def ad_pic_moments_device(state_ptr, n_particles, n_deriv, precision, mom_ptr, stream_ptr=None):
    """Allocation-free dual moments of a device state (device pointers as integers); enqueues only."""
    _ck("ad_pic_moments_device", lib().ad_pic_moments_device(ct.c_void_p(state_ptr), int(n_particles), int(n_deriv),
                                                             int(precision), ct.c_void_p(mom_ptr),
                                                             ct.c_void_p(stream_ptr) if stream_ptr else None))


def ad_pic_fma_peak(precision):
    t = ct.c_double()
    _ck("ad_pic_fma_peak", lib().ad_pic_fma_peak(int(precision), ct.byref(t)))
    return t.value


def make_elements(beamlines):
    """ad_pic_element array from a list of beamlines, each a list of (type, L, k, slot_L, slot_k)."""
    flat = [e for bl in beamlines for e in bl]
    arr = (ad_pic_element * len(flat))()
    for i, (t, L, k, sL, sk) in enumerate(flat):
        arr[i] = ad_pic_element(int(t), int(sL), int(sk), 0, float(L), float(k))
    return arr


def ad_pic_twiss_batch(beamlines, n_deriv, n_cell=0, twiss0=None):
    """Twiss functions at the end of each beamline (all of equal length): [n_inst][4][n_deriv+1]."""
    n_inst, n_elem = len(beamlines), len(beamlines[0])
    out = np.zeros((n_inst, 4, n_deriv + 1))
    t0 = None if twiss0 is None else np.ascontiguousarray(twiss0, dtype=np.float64).reshape(n_inst, 4)
    _ck("ad_pic_twiss_batch", lib().ad_pic_twiss_batch(n_inst, n_elem, make_elements(beamlines), int(n_deriv),
                                                       int(n_cell), None if t0 is None else _p(t0), _p(out)))
    return out


def ad_pic_track_batch(x0, beamline, n_deriv, n_repeat):
    """Dual tracking of particles x0 [n][4]: (out [n][4][n_deriv+1], kernel ms)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    out = np.zeros((x0.shape[0], 4, n_deriv + 1))
    ms = ct.c_double()
    _ck("ad_pic_track_batch", lib().ad_pic_track_batch(x0.shape[0], _p(x0), len(beamline), make_elements([beamline]),
                                                       int(n_deriv), int(n_repeat), _p(out), ct.byref(ms)))
    return out, ms.value


def ad_pic_set_beamline(h, beamline, kicks):
    k = (ct.c_int * len(kicks))(*[int(v) for v in kicks])
    _ck("ad_pic_set_beamline", lib().ad_pic_set_beamline(h, len(beamline), make_elements([beamline]), k))


def ad_pic_save(h, path):
    _ck("ad_pic_save", lib().ad_pic_save(h, os.fsencode(path)))


def ad_pic_load(h, path):
    _ck("ad_pic_load", lib().ad_pic_load(h, os.fsencode(path)))


def ad_pic_set_wait_limit(h, polls):
    _ck("ad_pic_set_wait_limit", lib().ad_pic_set_wait_limit(h, int(polls)))


def ad_pic_wait_probe(polls):
    ms = ct.c_double()
    failed = ct.c_int()
    _ck("ad_pic_wait_probe", lib().ad_pic_wait_probe(int(polls), ct.byref(ms), ct.byref(failed)))
    return ms.value, failed.value


def ad_pic_launches(h):
    n = ct.c_int64()
    _ck("ad_pic_launches", lib().ad_pic_launches(h, ct.byref(n)))
    return n.value


def ad_pic_constants(h):
    out = np.zeros(8)
    _ck("ad_pic_constants", lib().ad_pic_constants(h, _p(out)))
    keys = ["gamma0", "beta0", "p0", "brho", "kappa_perp", "kappa_z", "q_macro", "q"]
    return dict(zip(keys, out.tolist()))


def ad_pic_destroy(h):
    if h:
        lib().ad_pic_destroy(h)


def ad_pic_strerror(status):
    return lib().ad_pic_strerror(int(status)).decode()


def ad_pic_batch_create(grids, n_particles, n_deriv, precision):
    n = len(grids)
    g = (ad_pic_grid * n)(*[ad_pic_grid(*gr) for gr in grids])
    npart = (ct.c_int64 * n)(*[int(v) for v in n_particles])
    b = ct.c_void_p()
    _ck("ad_pic_batch_create", lib().ad_pic_batch_create(n, g, npart, int(n_deriv), int(precision), ct.byref(b)))
    return b


def ad_pic_batch_set_beam(b, inst, beam: ad_pic_beam, normals=None):
    nrm = None if normals is None else np.ascontiguousarray(normals, dtype=np.float64)
    _ck("ad_pic_batch_set_beam", lib().ad_pic_batch_set_beam(b, int(inst), ct.byref(beam),
                                                             None if nrm is None else _p(nrm)))


def ad_pic_batch_set_particles(b, inst, state):
    s = np.ascontiguousarray(state, dtype=np.float64)
    _ck("ad_pic_batch_set_particles", lib().ad_pic_batch_set_particles(b, int(inst), _p(s)))


def ad_pic_batch_set_lattice(b, inst, lat: ad_pic_lattice):
    _ck("ad_pic_batch_set_lattice", lib().ad_pic_batch_set_lattice(b, int(inst), ct.byref(lat)))


def ad_pic_batch_run(b, n_steps):
    _ck("ad_pic_batch_run", lib().ad_pic_batch_run(b, int(n_steps)))


def ad_pic_batch_moments(b, inst, P):
    v = np.zeros(2)
    d = np.zeros(2 * P)
    _ck("ad_pic_batch_moments", lib().ad_pic_batch_moments(b, int(inst), _p(v), _p(d)))
    return v, d.reshape(2, P)


def ad_pic_batch_history(b, inst, C):
    n = ct.c_int()
    _ck("ad_pic_batch_history", lib().ad_pic_batch_history(b, int(inst), None, 0, ct.byref(n)))
    out = np.zeros((n.value, 3, 5, C))
    if n.value:
        _ck("ad_pic_batch_history", lib().ad_pic_batch_history(b, int(inst), _p(out), n.value, ct.byref(n)))
    return out


def ad_pic_batch_get_particles(b, inst, out):
    _ck("ad_pic_batch_get_particles", lib().ad_pic_batch_get_particles(b, int(inst), _p(out)))
    return out


def ad_pic_batch_set_mode(b, mode):
    _ck("ad_pic_batch_set_mode", lib().ad_pic_batch_set_mode(b, int(mode)))


def ad_pic_batch_tuning(b):
    m = ct.c_int()
    ms = np.zeros(3)
    _ck("ad_pic_batch_tuning", lib().ad_pic_batch_tuning(b, ct.byref(m), _p(ms)))
    return m.value, ms


def ad_pic_batch_set_tiles(b, tiles=None):
    t = None if tiles is None else (ct.c_int * 4)(*[int(v) for v in tiles])
    _ck("ad_pic_batch_set_tiles", lib().ad_pic_batch_set_tiles(b, t))


def ad_pic_batch_tiles(b):
    t = (ct.c_int * 4)()
    ms = ct.c_double()
    _ck("ad_pic_batch_tiles", lib().ad_pic_batch_tiles(b, t, ct.byref(ms)))
    return list(t), ms.value


def ad_pic_batch_set_stream(b, stream_ptr):
    _ck("ad_pic_batch_set_stream", lib().ad_pic_batch_set_stream(b, ct.c_void_p(stream_ptr) if stream_ptr else None))


def ad_pic_batch_destroy(b):
    if b:
        lib().ad_pic_batch_destroy(b)


def _pf(a):
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ct.POINTER(ct.c_float))


def ad_pic_mlp_create(n_in, width, hidden, n_out, max_batch):
    m = ct.c_void_p()
    _ck("ad_pic_mlp_create", lib().ad_pic_mlp_create(int(n_in), int(width), int(hidden), int(n_out), int(max_batch),
                                                     ct.byref(m)))
    return m


def ad_pic_mlp_num_params(m):
    n = ct.c_int64()
    _ck("ad_pic_mlp_num_params", lib().ad_pic_mlp_num_params(m, ct.byref(n)))
    return n.value


def ad_pic_mlp_set_params(m, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _ck("ad_pic_mlp_set_params", lib().ad_pic_mlp_set_params(m, _pf(p)))


def ad_pic_mlp_get_params(m, n):
    p = np.zeros(n, dtype=np.float32)
    _ck("ad_pic_mlp_get_params", lib().ad_pic_mlp_get_params(m, _pf(p)))
    return p


def ad_pic_mlp_forward(m, x, n_out, want_dy=True):
    x = np.ascontiguousarray(x, dtype=np.float32)
    B, n_in = x.shape
    y = np.zeros((B, n_out), dtype=np.float32)
    dy = np.zeros((B, n_out, n_in), dtype=np.float32) if want_dy else None
    _ck("ad_pic_mlp_forward", lib().ad_pic_mlp_forward(m, _pf(x), B, _pf(y), _pf(dy) if want_dy else None))
    return y, dy


def ad_pic_mlp_loss_grad(m, x, t, dt, lam, n_params):
    x, t, dt = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, t, dt))
    loss = ct.c_double()
    g = np.zeros(n_params, dtype=np.float32)
    _ck("ad_pic_mlp_loss_grad", lib().ad_pic_mlp_loss_grad(m, _pf(x), _pf(t), _pf(dt), x.shape[0], float(lam),
                                                           ct.byref(loss), _pf(g)))
    return loss.value, g


def ad_pic_mlp_adam_step(m, x, t, dt, lam, lr):
    x, t, dt = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, t, dt))
    loss = ct.c_double()
    _ck("ad_pic_mlp_adam_step", lib().ad_pic_mlp_adam_step(m, _pf(x), _pf(t), _pf(dt), x.shape[0], float(lam),
                                                           float(lr), ct.byref(loss)))
    return loss.value


def ad_pic_mlp_set_dataset(m, x, t, dt):
    x, t, dt = (np.ascontiguousarray(a, dtype=np.float32) for a in (x, t, dt))
    _ck("ad_pic_mlp_set_dataset", lib().ad_pic_mlp_set_dataset(m, _pf(x), _pf(t), _pf(dt), x.shape[0]))


def ad_pic_mlp_train(m, steps, B, lam, lr0, lr1):
    """Device-resident Adam steps; returns (last loss, CUDA-event ms of the steps)."""
    loss = ct.c_double()
    ms = ct.c_double()
    _ck("ad_pic_mlp_train", lib().ad_pic_mlp_train(m, int(steps), int(B), float(lam), float(lr0), float(lr1),
                                                   ct.byref(loss), ct.byref(ms)))
    return loss.value, ms.value


def ad_pic_mlp_destroy(m):
    if m:
        lib().ad_pic_mlp_destroy(m)


# ------------------------------------------------------------------ convenience wrapper

def make_beam(b) -> ad_pic_beam:
    """ad_pic_beam from any object with the fields of inputs.Beam."""
    return ad_pic_beam(b.kinetic_eV, b.mass_eV, b.charge_e, b.bunch_charge_C, (ct.c_double * 3)(*b.eps_n),
                       (ct.c_double * 3)(*b.alpha), (ct.c_double * 3)(*b.beta), (ct.c_int * 6)(*b.twiss_slot),
                       int(getattr(b, "charge_slot", -1)), int(getattr(b, "energy_slot", -1)))


def make_lattice(lat) -> ad_pic_lattice:
    """ad_pic_lattice from any object with the fields of inputs.Lattice."""
    return ad_pic_lattice((ct.c_double * 5)(*lat.L), (ct.c_double * 2)(*lat.g), (ct.c_int * 5)(*lat.kicks),
                          (ct.c_int * 7)(*lat.deriv_slot))


class ADPIC:
    """One simulation handle (owns the device memory of one dual PIC instance)."""

    def __init__(self, grid, n_particles, n_deriv=7, precision=AD_PIC_FP64):
        self.grid = tuple(grid)
        self.N = int(n_particles)
        self.P = int(n_deriv)
        self.C = self.P + 1
        self.precision = precision
        self.h = ad_pic_create(self.grid, self.N, self.P, precision)

    def close(self):
        if self.h:
            ad_pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_beam(self, beam, normals=None):
        ad_pic_set_beam(self.h, make_beam(beam), normals)

    def set_lattice(self, lat):
        ad_pic_set_lattice(self.h, make_lattice(lat))

    def set_particles(self, state):
        ad_pic_set_particles(self.h, state)

    def set_particles_f32(self, state):
        ad_pic_set_particles_f32(self.h, state)

    def prefetch_particles_f32(self, state):
        # the source arrays of the copies that may still be in flight stay referenced
        src = ad_pic_prefetch_particles_f32(self.h, state)
        self._prefetch_src = (getattr(self, "_prefetch_src", (None, None))[-1], src)

    def commit_particles(self):
        ad_pic_commit_particles(self.h)

    def get_particles(self):
        return ad_pic_get_particles(self.h, np.zeros((6, self.N, self.C)))

    def run(self, n_steps):
        ad_pic_run(self.h, n_steps)

    def moments(self):
        return ad_pic_moments(self.h, self.P)

    def moments_full(self):
        return ad_pic_moments_full(self.h, self.C)

    def history(self):
        return ad_pic_history(self.h, self.C)

    def stage(self, stage, kick=0):
        nx, ny, nz = self.grid
        shapes = {0: (6,), 1: (self.C, nz, ny, nx), 2: (self.C, nz, ny, nx), 3: (3, self.C, nz, ny, nx)}
        out = np.zeros(shapes[stage]) if stage in shapes else None
        return ad_pic_stage(self.h, stage, kick, out)

    def constants(self):
        return ad_pic_constants(self.h)

    def launches(self):
        return ad_pic_launches(self.h)

    def set_stream(self, ptr):
        ad_pic_set_stream(self.h, ptr)

    def set_graphs(self, on):
        ad_pic_set_graphs(self.h, on)

    def set_timing(self, mask):
        ad_pic_set_timing(self.h, mask)

    def timing(self):
        return ad_pic_timing(self.h)

    def save(self, path):
        ad_pic_save(self.h, path)

    def load(self, path):
        ad_pic_load(self.h, path)

    def set_wait_limit(self, polls):
        ad_pic_set_wait_limit(self.h, polls)

    def set_beamline(self, beamline, kicks):
        ad_pic_set_beamline(self.h, beamline, kicks)


def ad_pic2d_create(nx, ny, a, b, n_particles, n_deriv, precision):
    h = ct.c_void_p()
    _ck("ad_pic2d_create", lib().ad_pic2d_create(int(nx), int(ny), float(a), float(b), int(n_particles),
                                                 int(n_deriv), int(precision), ct.byref(h)))
    return h


def ad_pic2d_set_beam(h, beam, current_A, current_slot=-1, normals=None):
    nrm = None if normals is None else np.ascontiguousarray(normals, dtype=np.float64)
    _ck("ad_pic2d_set_beam", lib().ad_pic2d_set_beam(h, ct.byref(beam), float(current_A), int(current_slot),
                                                     None if nrm is None else _p(nrm)))


def ad_pic2d_set_particles(h, state):
    s = np.ascontiguousarray(state, dtype=np.float64)
    _ck("ad_pic2d_set_particles", lib().ad_pic2d_set_particles(h, _p(s)))


def ad_pic2d_get_particles(h, out):
    _ck("ad_pic2d_get_particles", lib().ad_pic2d_get_particles(h, _p(out)))
    return out


def ad_pic2d_set_lattice(h, lat):
    _ck("ad_pic2d_set_lattice", lib().ad_pic2d_set_lattice(h, ct.byref(lat)))


def ad_pic2d_run(h, n_steps):
    _ck("ad_pic2d_run", lib().ad_pic2d_run(h, int(n_steps)))


def ad_pic2d_moments(h, P):
    v = np.zeros(2)
    d = np.zeros(2 * P)
    _ck("ad_pic2d_moments", lib().ad_pic2d_moments(h, _p(v), _p(d)))
    return v, d.reshape(2, P)


def ad_pic2d_moments_full(h, C):
    m = np.zeros((2, 5, C))
    _ck("ad_pic2d_moments_full", lib().ad_pic2d_moments_full(h, _p(m)))
    return m


def ad_pic2d_history(h, C):
    n = ct.c_int()
    _ck("ad_pic2d_history", lib().ad_pic2d_history(h, None, 0, ct.byref(n)))
    out = np.zeros((n.value, 2, 5, C))
    if n.value:
        _ck("ad_pic2d_history", lib().ad_pic2d_history(h, _p(out), n.value, ct.byref(n)))
    return out


def ad_pic2d_destroy(h):
    if h:
        lib().ad_pic2d_destroy(h)


class Pipe2D:
    """One 2D conducting-pipe dual PIC instance (Sec. 4's solver)."""

    def __init__(self, cells, widths, n_particles, n_deriv=7, precision=AD_PIC_FP64):
        self.N, self.P, self.C = int(n_particles), int(n_deriv), int(n_deriv) + 1
        self.h = ad_pic2d_create(cells[0], cells[1], widths[0], widths[1], self.N, self.P, precision)

    def set_beam(self, beam, current_A, current_slot=-1, normals=None):
        ad_pic2d_set_beam(self.h, make_beam(beam), current_A, current_slot, normals)

    def set_lattice(self, lat):
        ad_pic2d_set_lattice(self.h, make_lattice(lat))

    def set_particles(self, state):
        ad_pic2d_set_particles(self.h, state)

    def get_particles(self):
        return ad_pic2d_get_particles(self.h, np.zeros((4, self.N, self.C)))

    def run(self, n):
        ad_pic2d_run(self.h, n)

    def moments(self):
        return ad_pic2d_moments(self.h, self.P)

    def history(self):
        return ad_pic2d_history(self.h, self.C)

    def close(self):
        if self.h:
            ad_pic2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many instances advanced together (the batched scan)."""

    def __init__(self, grids, n_particles, precision=AD_PIC_FP32_MIXED, n_deriv=7):
        self.n = len(grids)
        self.P = n_deriv
        self.C = n_deriv + 1
        self.N = [int(v) for v in n_particles]
        self.b = ad_pic_batch_create([tuple(g) for g in grids], self.N, n_deriv, precision)

    def close(self):
        if self.b:
            ad_pic_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_beam(self, i, beam, normals=None):
        ad_pic_batch_set_beam(self.b, i, make_beam(beam), normals)

    def set_lattice(self, i, lat):
        ad_pic_batch_set_lattice(self.b, i, make_lattice(lat))

    def run(self, n_steps):
        ad_pic_batch_run(self.b, n_steps)

    def moments(self, i):
        return ad_pic_batch_moments(self.b, i, self.P)

    def history(self, i):
        return ad_pic_batch_history(self.b, i, self.C)

    def get_particles(self, i):
        return ad_pic_batch_get_particles(self.b, i, np.zeros((6, self.N[i], self.C)))

    def set_mode(self, mode):
        ad_pic_batch_set_mode(self.b, mode)

    def tuning(self):
        return ad_pic_batch_tuning(self.b)

    def set_tiles(self, tiles=None):
        ad_pic_batch_set_tiles(self.b, tiles)

    def tiles(self):
        return ad_pic_batch_tiles(self.b)
