"""Benchmark of the dual-number 3D space-charge PIC step on GB300.

Workload: the 1M-particle FODO run - 1,048,576 macroparticles, 64^3 grid,
P = 7 lattice derivatives, 1 GeV protons. One step = one FODO period: 20
space-charge kicks (each: geometry, CIC deposit of 8 dual channels, Green's
function, Hockney FFT convolution, FD field, gather + kick + maps) and the
period-end FP64 dual moment reduction. Metric: dual particle-steps/s =
particles x kicks / time, whole job.

  python bench.py [--gpus N --steps K --warmup W]    CUDA path (FP32 bulk + FP64 reductions); beside it
                                                      the plain FP64 path, the accuracy of both against
                                                      the oracle on the timed run, the large instance
                                                      (16.8M particles, 128^3, P = 13) and the batched
                                                      scan (256 instances)
  python bench.py --impl reference [...]              the FP64 CPU oracle on the host cores
  python bench.py --workload fodo_16m_128 [...]       the large instance as the headline
  python bench.py --workload batch [...]              the batched scan as the headline
Multi-GPU (torchrun): independent replicas, one instance per rank (weak scaling).
"""
import argparse
import ctypes as ct
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dual particle-steps/s (1M p, 64³, P=7), FP32/batched vs plain FP64 at fixed error"
UNIT = "dual particle-steps/s"
METRICS = {"fodo_1m_64": METRIC,
           "fodo_16m_128": "dual particle-steps/s (16.8M p, 128³, P=13), FP32 dual arithmetic with FP64 reductions"}
CPU_KICKS = {"fodo_1m_64": 8, "fodo_16m_128": 1}
PRECISION_NOTE = ("FP32 particles/deposit/FFT/field/push; FP64 geometry and Green's-function integrals; "
                  "moment sums compensated (each FP32 product formed exactly as a float pair, lane sums "
                  "in float pairs, warp/block/grid sums in FP64 pairs)")


def workload_config(w, extra=None):
    cfg = {"workload": f"{w.name}: FODO period (D 0.5 / QF 0.1 m +10 T/m / D 1.0 / QD 0.1 m -10 T/m / D 0.5), "
                       f"1 GeV protons, {w.n_particles} macroparticles, {w.grid[0]}x{w.grid[1]}x{w.grid[2]} grid, "
                       f"P={w.n_deriv}, step = one period of {w.kicks_per_period} kicks + FP64 moments",
           "particles": w.n_particles, "grid": list(w.grid), "n_deriv": w.n_deriv,
           "kicks_per_step": w.kicks_per_period,
           "l2": f"inputs larger than L2: the dual particle state is "
                 f"{w.n_particles * 6 * (w.n_deriv + 1) * 4 / 1e6:.0f} MB (FP32) / "
                 f"{w.n_particles * 6 * (w.n_deriv + 1) * 8 / 1e6:.0f} MB (FP64)",
           "parallelism": "replicas (one independent instance per GPU, no collective)",
           "precision": PRECISION_NOTE}
    if extra:
        cfg.update(extra)
    return cfg


def rank_seed(w, rank):
    """Seed of a rank's replica: every rank advances its own, independent instance."""
    return w.seed + 1000 * rank


def max_over_ranks(x, dist, device):
    """The slowest rank's value (the job ends when its last rank does)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws, particles, kicks, ms):
    """Whole-job dual particle-steps/s: all ranks' particle-steps over the slowest rank's time."""
    return ws * particles * kicks / (ms / 1000.0)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def kick_bytes(N, grid, C, w):
    """Algorithmic bytes of one kick (the method must move each once): the dual particle state read
    and written, rho written and read, the field written and read, and the two-pass slab FFT model
    of the convolution (fwd-xy write, z-pass read and write, inv-xy read of the pruned (2n)^2 x n
    intermediate, ceil(C/2) packed channel pairs)."""
    n3 = grid[0] * grid[1] * grid[2]
    particles = N * 2 * 6 * C * w
    rho = C * n3 * w * 2
    field = 3 * C * n3 * w * 2
    fft = math.ceil(C / 2) * 4 * (4 * n3) * 2 * w
    return {"particles": particles, "rho": rho, "field": field, "fft_model": fft,
            "total": particles + rho + field + fft}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- CPU oracle (baseline / reference arm)

def oracle_rate(w, kicks):
    """Time the FP64 oracle on the host cores on `kicks` kicks of the workload; particle-steps/s."""
    import oracle
    from paper_2511_21839_gb300 import inputs as I

    o = oracle.Oracle(**I.orc_kwargs(w))
    st = o.beam_init(I.normals(w.seed, w.n_particles))
    t0 = time.perf_counter()
    o.run(st, kicks)
    dt = time.perf_counter() - t0
    return w.n_particles * kicks / dt, dt


def host_cores():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2511_21839_gb300 import inputs as I

    w = I.workload(args.workload if args.workload != "batch" else "fodo_1m_64")
    kicks_per_sample = 1
    for _ in range(args.warmup):
        oracle_rate(w, kicks_per_sample)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_rate(w, kicks_per_sample)
        times.append(dt)
    ms_kick = 1000.0 * sum(times) / len(times)
    value = w.n_particles * kicks_per_sample / (ms_kick / 1000.0)
    sample = (f"each step times {kicks_per_sample} kick of the {w.name} workload ({w.n_particles} particles, "
              f"{w.grid[0]}^3, P={w.n_deriv}) in the FP64 oracle, OpenMP over particles; ms_per_step is the "
              f"projected time of a full period of {w.kicks_per_period} kicks at that rate")
    line = {"impl": "reference", "metric": METRICS[w.name], "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_kick * w.kicks_per_period,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """SM clock and throttle reasons sampled every few ms through NVML (read only; nvidia-smi as a
    fallback) while a measurement runs."""

    REASONS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20,
               "sw_power_cap": 0x4}

    def __init__(self, index, period_s=0.005):
        self.index = index
        self.period = period_s
        self.samples = []
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None
        self._nvml = None
        self._dev = None
        self._proc = None
        self._path = None

    def _init_nvml(self):
        try:
            nv = ct.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return False
            dev = ct.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(ct.c_uint(self.index), ct.byref(dev)) != 0:
                return False
            mx = ct.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(dev, ct.c_int(1), ct.byref(mx)) == 0:   # NVML_CLOCK_SM
                self.max_mhz = float(mx.value)
            self._reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
            self._nvml, self._dev = nv, dev
            return True
        except (OSError, AttributeError):
            return False

    def _loop(self):
        nv, dev = self._nvml, self._dev
        clk = ct.c_uint()
        rs = ct.c_ulonglong()
        while not self._stop.is_set():
            ok = nv.nvmlDeviceGetClockInfo(dev, ct.c_int(1), ct.byref(clk)) == 0
            okr = self._reasons_fn(dev, ct.byref(rs)) == 0
            if ok:
                self.samples.append((float(clk.value), int(rs.value) if okr else 0))
            time.sleep(self.period)

    def start(self):
        if self._init_nvml():
            self._thread = threading.Thread(target=self._loop, daemon=True)
            self._thread.start()
            return
        fd, self._path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self._proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                           "--format=csv,noheader,nounits", "-lms", "50"],
                                          stdout=open(self._path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self._proc = None

    def stop(self):
        if self._thread is not None:
            self._stop.set()
            self._thread.join()
            if not self.samples:
                return None
            reasons = sorted({n for _, r in self.samples for n, bit in self.REASONS.items() if r & bit})
            return {"sm_mhz": statistics.median([c for c, _ in self.samples]), "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(self.samples), "source": "nvml"}
        if self._proc is None:
            return None
        self._proc.terminate()
        try:
            self._proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self._proc.kill()
        rows = [[p.strip() for p in line.split(",")] for line in open(self._path)]
        rows = [r for r in rows if len(r) >= 9]
        os.unlink(self._path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "source": "nvidia-smi"}


# ---------------------------------------------------------------- helpers of the native arm

def profile_value(name, key, src_hash):
    """A number `key: value` from the committed ncu summary profiles/<name>, if that summary was
    taken on the current kernel sources (`kernel_src_sha256: H`), else None."""
    import re

    try:
        text = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None
    h = re.search(r"kernel_src_sha256:\s*([0-9a-f]{64})", text)
    b = re.search(rf"{key}:\s*([0-9.eE+]+)", text)
    if not h or not b or h.group(1) != src_hash:
        return None
    return float(b.group(1))


def kernel_src_hash():
    """SHA-256 over the sources that make up the particle kernels (push, deposit, moments)."""
    h = hashlib.sha256()
    for f in ("particles.cu", "particles_dev.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2511_21839_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def rel_errors(e, ref):
    """(max emittance error, max per-component derivative error) of emittance records e vs ref
    ([plane][channel]); the derivative denominator is max(|d_k|, 1e-3 max_j |d_j|) per emittance."""
    ev = np.abs(e[:, 0] - ref[:, 0]) / np.abs(ref[:, 0])
    den = np.maximum(np.abs(ref[:, 1:]), 1e-3 * np.abs(ref[:, 1:]).max(axis=1, keepdims=True))
    ed = np.abs(e[:, 1:] - ref[:, 1:]) / np.where(den > 0, den, 1.0)
    return float(ev.max()), float(ed.max())


def emittances(mom):
    """Dual rms emittances [plane x, y][channel] of a moment record [3][5][C] (centred, Sec. 4):
    plain host arithmetic on the library's FP64 moments, for the accuracy report only."""
    out = []
    for pl in range(2):
        m = mom[pl]
        a = m[2].copy(); a[0] -= m[0][0] ** 2; a[1:] -= 2 * m[0][0] * m[0][1:]
        b = m[3].copy(); b[0] -= m[0][0] * m[1][0]; b[1:] -= m[0][0] * m[1][1:] + m[1][0] * m[0][1:]
        c = m[4].copy(); c[0] -= m[1][0] ** 2; c[1:] -= 2 * m[1][0] * m[1][1:]
        e0 = math.sqrt(a[0] * c[0] - b[0] * b[0])
        d = (a[1:] * c[0] + a[0] * c[1:] - 2 * b[0] * b[1:]) / (2 * e0)
        out.append(np.r_[e0, d])
    return np.array(out)


def oracle_records(name):
    """The oracle's emittance records of a workload, if stored (tests/golden, written by the oracle)."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{name}.json")
    try:
        return np.array(json.load(open(path))["eps"])
    except (OSError, ValueError, KeyError):
        return None


def accuracy(hist32, hist64, ref):
    """FP32 vs FP64 and both vs the oracle at every period end both runs reached."""
    n = min(hist32.shape[0], hist64.shape[0])
    out = {"periods_compared": n - 1}
    w32 = (0.0, 0.0)
    for r in range(1, n):
        ev, ed = rel_errors(emittances(hist32[r]), emittances(hist64[r]))
        w32 = (max(w32[0], ev), max(w32[1], ed))
    out["fp32_vs_fp64"] = {"eps_rel": w32[0], "deriv_rel_per_component": w32[1]}
    if ref is not None:
        for name, h in (("fp32_vs_oracle", hist32), ("fp64_vs_oracle", hist64)):
            m = min(h.shape[0], ref.shape[0])
            worst = (0.0, 0.0)
            for r in range(1, m):
                ev, ed = rel_errors(emittances(h[r]), ref[r])
                worst = (max(worst[0], ev), max(worst[1], ed))
            out[name] = {"eps_rel": worst[0], "deriv_rel_per_component": worst[1], "periods": m - 1}
    out["bounds"] = {"fp64": {"eps_rel": 1e-10, "deriv_rel_per_component": 1e-10},
                     "fp32": {"eps_rel": 1e-5, "deriv_rel_per_component": 1e-4}}
    ok = w32[0] < 2e-5 and w32[1] < 2e-4
    if "fp32_vs_oracle" in out:
        ok = ok and out["fp32_vs_oracle"]["eps_rel"] < 1e-5 and out["fp32_vs_oracle"]["deriv_rel_per_component"] < 1e-4
        ok = ok and out["fp64_vs_oracle"]["eps_rel"] < 1e-10 and \
            out["fp64_vs_oracle"]["deriv_rel_per_component"] < 1e-10
    out["within_bounds"] = bool(ok)
    return out


def ensure_periods(sim, kicks, n_records):
    while sim.history().shape[0] < n_records:
        sim.run(kicks)


def timed_runs(sim, steps, kicks, torch, sampler=None):
    """Event-timed `steps` runs of one period on the library's stream (torch's current stream)."""
    l0 = sim.launches()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        sim.run(kicks)
    e1.record()
    torch.cuda.synchronize()
    ck = sampler.stop() if sampler else None
    return e0.elapsed_time(e1) / steps, sim.launches() - l0, ck


def class_times(sim, kicks, periods):
    """Per kernel class: ms per launch, launches per period (CUDA events around every launch)."""
    sim.set_timing(0xFF)
    sim.run(kicks)                                  # captures the graph with the events
    sim.set_timing(0xFF)
    for _ in range(periods):
        sim.run(kicks)
    t = sim.timing()
    sim.set_timing(0)
    return {k: {"ms_per_launch": v[0] / max(v[1], 1), "launches_per_step": v[1] / periods}
            for k, v in t.items() if v[1] > 0}


def e2e_measure(args, sim, w, kicks, ws, barrier):
    """End to end through the public API with host buffers: every step uploads the dual state from
    pinned host memory, runs the period and reads the emittances back. The FP32-mixed handle takes
    its state in FP32 (the device state it holds either way), and the next step's upload
    (ad_pic_prefetch_particles_f32) runs while the current step runs; the synchronous upload
    (ad_pic_set_particles_f32) is timed too. The FP64 handle uploads FP64, synchronously."""
    import torch

    from paper_2511_21839_gb300 import adpic

    f32 = sim.precision == adpic.AD_PIC_FP32_MIXED
    # two pinned host buffers used in turn, as a caller streaming beams would
    states = [torch.empty((6, w.n_particles, w.n_deriv + 1), dtype=torch.float32 if f32 else torch.float64,
                          pin_memory=True) for _ in range(2)]
    for st in states:
        st.numpy()[...] = sim.get_particles()
    upload = sim.set_particles_f32 if f32 else sim.set_particles

    def synchronous(steps):
        for k in range(steps):
            upload(states[k % 2].numpy())
            sim.run(kicks)
            sim.moments()

    def pipelined(steps):
        # every step's upload is inside the timed region; step k + 1's copy
        # runs on the handle's copy stream while step k runs
        sim.prefetch_particles_f32(states[0].numpy())
        for k in range(steps):
            sim.commit_particles()
            if k + 1 < steps:
                sim.prefetch_particles_f32(states[(k + 1) % 2].numpy())
            sim.run(kicks)
            sim.moments()

    def timed(fn):
        fn(2)
        barrier()
        t0 = time.perf_counter()
        fn(args.steps)
        barrier()
        return 1000.0 * (time.perf_counter() - t0) / args.steps

    sync_ms = timed(synchronous)
    e2e_ms = timed(pipelined) if f32 else sync_ms
    h2d = states[0].numel() * states[0].element_size()
    d2h = 8 * (2 + 2 * w.n_deriv) + 15 * 8 * (w.n_deriv + 1) + 4
    rate = lambda ms: ws * w.n_particles * kicks / (ms / 1000.0)
    return rate(e2e_ms), e2e_ms, h2d, d2h, {"value": rate(sync_ms), "ms_per_step": sync_ms}


def large_instance(args, stream, adpic, I, torch, peaks):
    """Compact run of the large instance (16,777,216 particles, 128^3, P = 13): FP32-mixed rate,
    per-kernel rates, the plain FP64 rate and FP32 vs FP64 accuracy at the common period ends."""
    w = I.workload("fodo_16m_128")
    kicks = w.kicks_per_period
    nrm = I.normals(w.seed, w.n_particles)
    out = {"workload": f"{w.name}: {w.n_particles} particles, 128^3, P=13, step = one period of {kicks} kicks"}

    def make(prec):
        sim = adpic.ADPIC(w.grid, w.n_particles, w.n_deriv, prec)
        sim.set_stream(stream.cuda_stream)
        sim.set_beam(w.beam, nrm)
        sim.set_lattice(w.lattice)
        return sim

    sim = make(adpic.AD_PIC_FP32_MIXED)
    sim.run(kicks)                                  # warm-up (and the graph)
    ms, _, _ = timed_runs(sim, args.large_steps, kicks, torch)
    out["value"] = w.n_particles * kicks / (ms / 1000.0)
    out["ms_per_step"] = ms
    out["steps"] = args.large_steps
    ct_ = class_times(sim, kicks, 1)
    kb = kick_bytes(w.n_particles, w.grid, w.n_deriv + 1, 4)
    hbm = peaks.get("hbm_gbs", 6800.0)
    n3 = w.grid[0] * w.grid[1] * w.grid[2]
    C = w.n_deriv + 1
    per = {}
    alg = {"push": w.n_particles * 2 * 6 * C * 4 + 3 * C * n3 * 4,
           "deposit": w.n_particles * 3 * C * 4 + C * n3 * 4}
    for k, v in ct_.items():
        e = {"ms_per_launch": v["ms_per_launch"], "launches_per_step": v["launches_per_step"]}
        if k in alg:
            gbs = alg[k] / (v["ms_per_launch"] / 1000.0) / 1e9
            e.update({"algorithmic_bytes_per_launch": alg[k], "achieved_gbs": gbs, "frac_of_measured_hbm": gbs / hbm})
        per[k] = e
    out["per_kernel_class"] = per
    out["roofline_step"] = {"bytes_per_kick": kb["total"], "achieved_gbs": kb["total"] * kicks / (ms / 1000.0) / 1e9,
                            "frac_of_measured_hbm": kb["total"] * kicks / (ms / 1000.0) / 1e9 / hbm}
    h32 = sim.history()
    sim.close()
    if not args.no_fp64:
        sim64 = make(adpic.AD_PIC_FP64)
        ms64, _, _ = timed_runs(sim64, 1, kicks, torch)
        h64 = sim64.history()
        sim64.close()
        out["fp64_plain"] = {"value": w.n_particles * kicks / (ms64 / 1000.0), "ms_per_step": ms64,
                             "fp32_speedup": ms64 / ms}
        out["accuracy"] = accuracy(h32, h64, None)
    return out


def batch_scan(args, adpic, I, torch):
    """The batched sensitivity scan (256 instances, +-10 % lattices, 16k-262k particles, 32^3/64^3,
    P = 7, 5 periods) on the batched runtime; step = the whole scan from the initial beams."""
    params, npart, grid, periods = I.batched_scan(3, args.batch_instances)
    w = I.workload("fodo_10k_32")
    grids = [(int(g), int(g), int(g)) for g in grid]
    b = adpic.Batch(grids, [int(v) for v in npart])
    nrms = [I.normals(10_000 + i, int(npart[i])) for i in range(len(grids))]

    def reset():
        for i in range(len(grids)):
            b.set_beam(i, w.beam, nrms[i])
            b.set_lattice(i, I.Lattice.from_params(params[i]))

    reset()
    kicks = w.kicks_per_period * periods
    b.run(0)
    t0 = time.perf_counter()
    b.run(kicks)                                   # the tuner times the modes on this first run
    torch.cuda.synchronize()
    first = time.perf_counter() - t0
    times = []
    for _ in range(args.batch_steps):
        reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run(kicks)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    mode, ms = b.tuning()
    b.close()
    total = int(np.sum(npart)) * kicks
    step = min(times)
    return {"workload": f"batched scan: {len(grids)} instances, {int(np.sum(npart))} particles, "
                        f"{int(np.sum(np.array(grid) == 32))} on 32^3 and {int(np.sum(np.array(grid) == 64))} on "
                        f"64^3, {kicks} kicks; step = the whole scan, best of {args.batch_steps}",
            "value": total / step, "ms_per_step": 1000 * step,
            "mode": {1: "persistent, 1 block/SM", 2: "persistent, 2 blocks/SM", 3: "phased launches"}[mode],
            "tuner_ms_per_kick": [float(x) for x in ms], "first_run_s_incl_tuning": first}


def nvml_index(dev):
    """NVML index of CUDA device `dev` (CUDA_VISIBLE_DEVICES maps it when set to plain indices)."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = [p.strip() for p in vis.split(",") if p.strip()]
    if parts and all(p.isdigit() for p in parts) and dev < len(parts):
        return int(parts[dev])
    return dev


def track_flops(P):
    """Algorithmic FP64 flops of one particle through one element (both planes): per plane the
    values (m11 x + m12 p, m21 x + m22 p: 2 multiplies and 2 fused multiply-adds) and, per derivative
    channel and coordinate, 3 fused multiply-adds and a multiply (d(M z) = M dz + (dM) z)."""
    return 2 * (6 + 14 * P)


def tracking(adpic, P, n_part, turns, periods, fma64=None):
    """Dual tracking of n_part particles through `turns` x `periods` FODO cells of Sec. 3 (5 elements
    each), element by element; rate in particle-element-steps/s and the FP64 ALU roofline."""
    from paper_2511_21839_gb300 import optics

    cell = optics.fodo_cell()
    cell = [(t, L, k, sL if sL < P else -1, sk if sk < P else -1) for (t, L, k, sL, sk) in cell]
    rng = np.random.default_rng(11)
    x0 = rng.normal(size=(n_part, 4)) * 1e-3
    adpic.ad_pic_track_batch(x0[:64], cell, P, 2)            # warm-up (module load)
    _, ms = adpic.ad_pic_track_batch(x0, cell, P, turns * periods)
    steps = n_part * turns * periods * len(cell)
    rate = steps / (ms / 1000.0)
    out = {"n_deriv": P, "particles": n_part, "turns": turns, "periods": periods, "kernel_ms": ms,
           "particle_element_steps_per_s": rate, "fp64_tflops": rate * track_flops(P) / 1e12}
    if fma64:
        out["frac_of_measured_fp64_fma"] = out["fp64_tflops"] / fma64
    return out


def run_track(args):
    """The Sec. 3 tracking benchmark: one particle through 1000 turns x 100 FODO periods for several
    numbers of control variables (the paper's figure), and batched throughput at the same counts."""
    from paper_2511_21839_gb300 import adpic, build

    build.build()
    fma64 = adpic.ad_pic_fma_peak(adpic.AD_PIC_FP64)
    rows = []
    for P in (1, 3, 7, 13, 31):
        single = tracking(adpic, P, 1, 1000, 100)
        batch = tracking(adpic, P, args.track_particles, 10, 100, fma64)
        rows.append({"n_deriv": P, "single_particle_ms": single["kernel_ms"], "batched": batch})
    b7 = next(r for r in rows if r["n_deriv"] == 7)["batched"]
    line = {"metric": "particle-element-steps/s, dual tracking through FODO cells (Sec. 3), P=7",
            "value": b7["particle_element_steps_per_s"], "unit": "particle-element-steps/s", "n_gpus": 1,
            "steps": 1, "warmup": 1, "ms_per_step": b7["kernel_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.track_particles} particles x 10 turns x 100 FODO cells (5 elements) per "
                                   "step; single particle: 1000 turns x 100 cells", "fp64_fma_peak_tflops": fma64},
            "sweep": rows}
    print(json.dumps(line))
    return 0


def pipe2d(adpic, I, torch, n_part, cells, periods=1):
    """The 2D conducting-pipe dual PIC (Sec. 4's solver): n_part particles, cells x cells on a 40 mm
    pipe (the cell of the 128-cell, 20 mm parity case; the 1 mm beam's 5-sigma tails of a million
    particles stay clear of the walls), 100 A, one FODO period per step, FP32-mixed and FP64; dual
    particle-steps/s (wall clock around a synchronised run)."""
    beam = I.default_beam(7)
    lat = I.Lattice(deriv_slot=(-1, 1, 2, 3, 4, 5, 6))
    nrm = I.normals(53, n_part)[:4]
    out = {"workload": f"2D pipe 40 x 40 mm, {cells}x{cells} cells, {n_part} particles, 100 A (current in slot 0), "
                       f"P=7, step = one period of 20 kicks"}
    for name, prec in (("fp32", adpic.AD_PIC_FP32_MIXED), ("fp64", adpic.AD_PIC_FP64)):
        sim = adpic.Pipe2D((cells, cells), (0.04, 0.04), n_part, 7, prec)
        sim.set_beam(beam, 100.0, 0, nrm)
        sim.set_lattice(lat)
        sim.run(20)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.run(20 * periods)
        torch.cuda.synchronize()
        ms = 1000.0 * (time.perf_counter() - t0) / periods
        sim.close()
        out[name] = {"value": n_part * 20 / (ms / 1000.0), "ms_per_step": ms}
    return out


def energy_slot_cost(adpic, I, torch, w, nrm, stream, periods=3):
    """The kinetic energy as a dual input (slot 0, lattice in slots 1-6) on the headline workload:
    period time against the same run without it (the energy adds one Green's spectrum on the side
    stream and one single-pair convolution per kick). CUDA events on the library's stream."""
    import dataclasses

    lat = I.Lattice(deriv_slot=(-1, 1, 2, 3, 4, 5, 6))
    out = {"workload": f"{w.name} with the energy in slot 0 and the lattice in slots 1-6, FP32-mixed"}
    for name, slot in (("without", -1), ("with", 0)):
        b = dataclasses.replace(w.beam, energy_slot=slot)
        sim = adpic.ADPIC(w.grid, w.n_particles, w.n_deriv, adpic.AD_PIC_FP32_MIXED)
        sim.set_stream(stream.cuda_stream)
        sim.set_beam(b, nrm)
        sim.set_lattice(lat)
        sim.run(w.kicks_per_period)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(periods):
            sim.run(w.kicks_per_period)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / periods
        sim.close()
        out[name] = {"ms_per_step": ms, "value": w.n_particles * w.kicks_per_period / (ms / 1000.0)}
    out["cost"] = out["with"]["ms_per_step"] / out["without"]["ms_per_step"]
    return out


def surrogate_training(adpic, peaks, steps=200, B=512):
    """The surrogate's device-resident training (7 -> 256 x 3 -> 2, GELU, B samples x 8 rows of
    primal and input tangents per step, Sobolev loss, Adam): ms per step by CUDA events inside the
    library around the graph replays, and the GEMM work of a step (3 passes of 2 R K N per layer)
    against the measured bf16 peak."""
    import numpy as np

    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, size=(4096, 7))
    A = rng.standard_normal((2, 7)) * 0.4
    z = X @ A.T
    T, dT = np.sin(z), np.cos(z)[:, :, None] * A[None, :, :]
    m = adpic.ad_pic_mlp_create(7, 256, 3, 2, B)
    n = adpic.ad_pic_mlp_num_params(m)
    adpic.ad_pic_mlp_set_params(m, (rng.standard_normal(n) * 0.05).astype(np.float32))
    adpic.ad_pic_mlp_set_dataset(m, X, T, dT)
    adpic.ad_pic_mlp_train(m, 5, B, 1.0, 1e-3, 1e-3)       # graph capture and warm-up
    _, ms = adpic.ad_pic_mlp_train(m, steps, B, 1.0, 1e-3, 1e-4)
    adpic.ad_pic_mlp_destroy(m)
    R = B * 8
    flops = 3 * 2 * R * (7 * 256 + 256 * 256 * 2 + 256 * 2)
    tf = flops * steps / (ms * 1e-3) / 1e12
    peak = peaks.get("bf16_tflops")
    return {"workload": f"MLP 7-256-256-256-2, batch {B} samples x 8 rows (primal + 7 tangents), Sobolev loss, "
                        f"Adam; {steps} steps", "ms_per_step": ms / steps, "gemm_flops_per_step": flops,
            "gemm_tflops": tf, "bf16_peak_tflops": peak, "frac_of_measured_bf16": tf / peak if peak else None,
            "ms_per_step_at_peak": flops / (peak * 1e12) * 1e3 if peak else None}


def cufft_comparison(torch, n=64, C=8, reps=20):
    """For comparison only (not a product path): the same zero-padded Hockney convolution as one kick's
    x / (y, z) / inverse-x kernels, done by cuFFT through torch.fft: the C channels of an n^3 density in a
    (2n)^3 zero-padded FP32 buffer, batched R2C, times a real (2n, 2n, n+1) spectrum, C2R. Timed with
    CUDA events on the current stream; the zero padding and the extraction of the n^3 result are not
    timed (the library's kernels do them inside their passes)."""
    M = 2 * n
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.zeros((C, M, M, M), device="cuda", dtype=torch.float32)
    x[:, :n, :n, :n] = torch.randn((C, n, n, n), device="cuda", generator=g)
    G = torch.rand((M, M, M // 2 + 1), device="cuda", generator=g)

    def conv():
        X = torch.fft.rfftn(x, dim=(1, 2, 3))
        X *= G
        return torch.fft.irfftn(X, s=(M, M, M), dim=(1, 2, 3))

    for _ in range(3):
        conv()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        conv()
    e1.record()
    torch.cuda.synchronize()
    return {"what": f"cuFFT (torch.fft) R2C + spectrum product + C2R of {C} channels on the {M}^3 zero-padded "
                    f"grid, comparison only", "ms_per_convolution": e0.elapsed_time(e1) / reps}


def run_native(args):
    import torch

    from paper_2511_21839_gb300 import adpic, build
    from paper_2511_21839_gb300 import inputs as I

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
    build.build()
    dev = torch.cuda.current_device()
    w = I.workload(args.workload)
    kicks = w.kicks_per_period
    nrm = I.normals(rank_seed(w, rank), w.n_particles)
    stream = torch.cuda.Stream()        # one non-default stream shared by the library and the events
    torch.cuda.set_stream(stream)
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def make(prec):
        sim = adpic.ADPIC(w.grid, w.n_particles, w.n_deriv, prec)
        sim.set_stream(stream.cuda_stream)
        sim.set_beam(w.beam, nrm)
        sim.set_lattice(w.lattice)
        return sim

    if args.fp64_only:
        # the plain FP64 path alone (the run an FP64 instruction-count capture profiles): one
        # untimed period, then --steps periods
        sim64 = make(adpic.AD_PIC_FP64)
        sim64.run(kicks)
        barrier()
        ms64, _, _ = timed_runs(sim64, args.steps, kicks, torch)
        sim64.close()
        if rank == 0:
            print(json.dumps({"fp64_only": True, "workload": w.name, "ms_per_period": ms64,
                              "periods": args.steps, "kicks_per_period": kicks}))
        return 0

    # ---- FP32 bulk / compensated FP64 reductions (headline)
    sim = make(adpic.AD_PIC_FP32_MIXED)
    for _ in range(args.warmup):
        sim.run(kicks)
    sim.set_timing(0)
    sim.run(kicks)                      # captures the timed graph outside the timed region
    barrier()
    ms_step, launches, ck = timed_runs(sim, args.steps, kicks, torch, ClockSampler(nvml_index(dev)))
    # the push's average launch duration, from a second timed pass with CUDA events around every
    # push launch in the graph (on the launching stream); event nodes inside the graph cost the
    # step a little, so the headline pass above has none
    sim.set_timing(1 << 0)
    sim.run(kicks)
    sim.set_timing(1 << 0)
    for _ in range(max(2, args.steps // 2)):
        sim.run(kicks)
    barrier()
    tpush = sim.timing()["push"]
    push_ms = tpush[0] / max(tpush[1], 1)
    sim.set_timing(0)
    kernels = class_times(sim, kicks, 2) if rank == 0 else None
    ensure_periods(sim, kicks, w.periods + 1)
    hist32 = sim.history()
    ms_step = max_over_ranks(ms_step, dist, "cuda")
    value = job_rate(ws, w.n_particles, kicks, ms_step)

    if args.no_e2e:
        e2e = None
    else:
        ev_, e2e_ms, h2d, d2h, sync = e2e_measure(args, sim, w, kicks, ws, barrier)
        e2e = {"value": ev_, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": e2e_ms,
               "upload": ("ad_pic_prefetch_particles_f32 of the next step's beam overlapping this step's run, "
                          "ad_pic_commit_particles at the step's start" if sim.precision == adpic.AD_PIC_FP32_MIXED else
                          "ad_pic_set_particles (synchronous)"),
               "synchronous_upload": sync}
    sim.close()

    # ---- plain FP64 path on the same workload and beam, and the accuracy of both on these runs
    fp64 = None
    acc = None
    C = w.n_deriv + 1
    if not args.no_fp64:
        sim64 = make(adpic.AD_PIC_FP64)
        for _ in range(min(args.warmup, 3)):
            sim64.run(kicks)
        sim64.run(kicks)
        ms64, _, _ = timed_runs(sim64, max(2, args.steps // 4), kicks, torch)
        ensure_periods(sim64, kicks, w.periods + 1)
        hist64 = sim64.history()
        sim64.close()
        v64 = w.n_particles * kicks / (ms64 / 1000.0)
        fp64 = {"value": ws * v64, "ms_per_step": ms64, "dtype": "f64", "fp32_speedup": ms64 / ms_step}
        flops = profile_value(f"flops_{w.name}.md", "fp64_flops_per_particle_step", kernel_src_hash())
        fma64 = adpic.ad_pic_fma_peak(adpic.AD_PIC_FP64)
        fma32 = adpic.ad_pic_fma_peak(adpic.AD_PIC_FP32_MIXED)
        fp64["fma_peaks_tflops"] = {"fp64": fma64, "fp32": fma32, "source": "measured (ad_pic_fma_peak)"}
        if flops:
            ach = flops * w.n_particles * kicks / (ms64 / 1000.0) / 1e12
            fp64["roofline"] = {"bound": "alu", "achieved": ach, "peak": fma64, "unit": "TFLOP/s",
                                "frac": ach / fma64, "flops_per_particle_step": flops,
                                "flops_source": f"profiles/flops_{w.name}.md (ncu FP64 instruction counts)"}
        acc = accuracy(hist32, hist64, oracle_records(w.name) if rank_seed(w, rank) == w.seed else None)
        acc["records"] = "period ends of the FP32 run (the timed one) and of the FP64 run, same initial beam"

    # ---- roofline of the dominant kernel (gather + kick + push): algorithmic bytes per launch
    # = particles x (read + write of 6 coordinates x C channels x 4 B) + one read of the
    #   rest-frame field grid (3 x C x n^3 x 4 B)
    nodes = w.grid[0] * w.grid[1] * w.grid[2]
    alg_bytes = w.n_particles * 2 * 6 * C * 4 + 3 * C * nodes * 4
    achieved = alg_bytes / (push_ms / 1000.0) / 1e9
    traffic = profile_value(f"push_{w.name}.md", "dram_bytes_per_launch", kernel_src_hash())
    roof = {"bound": "hbm", "kernel": "push_tma_kernel (CIC gather + kick + dual maps)", "achieved": achieved,
            "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": push_ms,
            "traffic": None if traffic is None else int(traffic)}
    kb = kick_bytes(w.n_particles, w.grid, C, 4)
    step_bytes = kicks * kb["total"]
    step_gbs = step_bytes / (ms_step / 1000.0) / 1e9
    roof_step = {"bound": "hbm", "what": "whole step (20 kicks): algorithmic bytes of every kick (particles, rho, "
                                         "field, FFT model) over the event-timed step", "achieved": step_gbs,
                 "peak": hbm, "unit": "GB/s", "frac": step_gbs / hbm, "bytes_per_kick": kb}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        kicks_cpu = args.cpu_kicks or CPU_KICKS[w.name]
        rate, dt = oracle_rate(w, kicks_cpu)
        cpu = {"value": rate, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": f"{kicks_cpu} kicks of the {w.name} workload on the host cores ({dt:.1f} s)"}

    large = batch = track = pipe = surr = energy = None
    if rank == 0 and w.name == "fodo_1m_64" and not args.no_energy:
        energy = energy_slot_cost(adpic, I, torch, w, nrm, stream)
    if rank == 0 and w.name == "fodo_1m_64" and not args.no_pipe2d:
        pipe = pipe2d(adpic, I, torch, 1_048_576, 256)
    if rank == 0 and w.name == "fodo_1m_64" and not args.no_surrogate:
        surr = surrogate_training(adpic, peaks)
    if rank == 0 and kernels is not None and "fft" in kernels:
        try:
            cf = cufft_comparison(torch, w.grid[0], C)
            cf["ours_ms_per_convolution"] = kernels["fft"]["ms_per_launch"]
            kernels["fft_vs_cufft"] = cf
        except RuntimeError as e:          # torch built without cuFFT: the comparison is skipped
            kernels["fft_vs_cufft"] = {"unavailable": str(e).splitlines()[0]}
    if rank == 0 and w.name == "fodo_1m_64" and not args.no_track:
        fma64 = fp64["fma_peaks_tflops"]["fp64"] if fp64 else adpic.ad_pic_fma_peak(adpic.AD_PIC_FP64)
        track = tracking(adpic, 7, args.track_particles, 10, 100, fma64)
    if rank == 0 and w.name == "fodo_1m_64" and not args.no_large:
        large = large_instance(args, stream, adpic, I, torch, peaks)
    if rank == 0 and w.name == "fodo_1m_64" and not args.no_batch:
        batch = batch_scan(args, adpic, I, torch)

    if rank == 0:
        line = {"metric": METRICS[w.name], "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(w),
                "roofline": roof, "roofline_step": roof_step, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": ck, "fp64_plain": fp64, "accuracy": acc,
                "kernels": kernels, "large_instance": large, "batched_scan": batch,
                "single_particle_tracking": track, "pipe2d": pipe, "surrogate_training": surr,
                "energy_slot": energy}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batch_headline(args):
    import torch

    from paper_2511_21839_gb300 import adpic, build
    from paper_2511_21839_gb300 import inputs as I

    ws, rank, _ = dist_env()
    build.build()
    r = batch_scan(args, adpic, I, torch)
    line = {"metric": "dual particle-steps/s, batched sensitivity scan (256 instances, 16k-262k particles, "
                      "32^3/64^3, P=7, 5 periods)", "value": r["value"], "unit": UNIT, "n_gpus": ws,
            "steps": args.batch_steps, "warmup": 1, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": r["workload"], "mode": r["mode"], "tuner_ms_per_kick": r["tuner_ms_per_kick"],
                       "first_run_s_incl_tuning": r["first_run_s_incl_tuning"]}}
    if rank == 0:
        print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-kicks", type=int, default=0, help="oracle kicks of the CPU baseline (0: per workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the large-instance sub-result")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-scan sub-result")
    ap.add_argument("--large-steps", type=int, default=3)
    ap.add_argument("--batch-steps", type=int, default=2)
    ap.add_argument("--no-track", action="store_true", help="skip the single-particle tracking sub-result")
    ap.add_argument("--no-pipe2d", action="store_true", help="skip the 2D conducting-pipe sub-result")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate training sub-result")
    ap.add_argument("--no-energy", action="store_true", help="skip the energy-slot sub-result")
    ap.add_argument("--fp64-only", action="store_true",
                    help="run only the plain FP64 path (one untimed period, then --steps periods)")
    ap.add_argument("--track-particles", type=int, default=65536)
    ap.add_argument("--workload", choices=["fodo_1m_64", "fodo_16m_128", "batch", "track"], default="fodo_1m_64")
    ap.add_argument("--batch-instances", type=int, default=256)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch_headline(args)
    if args.workload == "track":
        return run_track(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
