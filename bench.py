"""Benchmark of the dual-number 3D space-charge PIC step on GB300.

Workload: the 1M-particle FODO run - 1,048,576 macroparticles, 64^3 grid,
P = 7 lattice derivatives, 1 GeV protons. One step = one FODO period: 20
space-charge kicks (each: geometry, CIC deposit of 8 dual channels, Green's
function, Hockney FFT convolution, FD field, gather + kick + maps) and the
period-end FP64 dual moment reduction. Metric: dual particle-steps/s =
particles x kicks / time, whole job.

  python bench.py [--gpus N --steps K --warmup W]         CUDA path (FP32 bulk + FP64 reductions;
                                                           the plain FP64 path is measured beside it)
  python bench.py --impl reference [...]                   the FP64 CPU oracle on the host cores
  python bench.py --workload fodo_16m_128 [...]            the large instance: 16,777,216 particles,
                                                           128^3, P = 13 (7 lattice + 6 Twiss derivatives)
  python bench.py --workload batch [...]                   the batched scan of 256 instances
Multi-GPU (torchrun): independent replicas, one instance per rank (weak scaling).
"""
import argparse
import hashlib
import json

import numpy as np
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dual particle-steps/s (1M p, 64³, P=7), FP32/batched vs plain FP64 at fixed error"
UNIT = "dual particle-steps/s"
WORKLOAD = "fodo_1m_64"
METRICS = {"fodo_1m_64": METRIC,
           "fodo_16m_128": "dual particle-steps/s (16.8M p, 128³, P=13), FP32 dual arithmetic with FP64 reductions"}
CPU_KICKS = {"fodo_1m_64": 8, "fodo_16m_128": 1}


def workload_config(w, extra=None):
    cfg = {"workload": f"{w.name}: FODO period (D 0.5 / QF 0.1 m +10 T/m / D 1.0 / QD 0.1 m -10 T/m / D 0.5), "
                       f"1 GeV protons, {w.n_particles} macroparticles, {w.grid[0]}x{w.grid[1]}x{w.grid[2]} grid, "
                       f"P={w.n_deriv}, step = one period of {w.kicks_per_period} kicks + FP64 moments",
           "particles": w.n_particles, "grid": list(w.grid), "n_deriv": w.n_deriv,
           "kicks_per_step": w.kicks_per_period,
           "l2": f"inputs larger than L2: the dual particle state is "
                 f"{w.n_particles * 6 * (w.n_deriv + 1) * 4 / 1e6:.0f} MB (FP32) / "
                 f"{w.n_particles * 6 * (w.n_deriv + 1) * 8 / 1e6:.0f} MB (FP64)",
           "parallelism": "replicas (one independent instance per GPU, no collective)"}
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


# ---------------------------------------------------------------- CPU oracle (baseline / reference arm)

def oracle_rate(w, kicks, threads=None):
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

    w = I.workload(args.workload)
    kicks_per_step = 1
    for _ in range(args.warmup):
        oracle_rate(w, kicks_per_step)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_rate(w, kicks_per_step)
        times.append(dt)
    ms = 1000.0 * sum(times) / len(times)
    value = w.n_particles * kicks_per_step / (ms / 1000.0)
    sample = (f"each step: {kicks_per_step} kick of the {w.name} workload ({w.n_particles} particles, "
              f"{w.grid[0]}^3, P={w.n_deriv}), FP64 oracle, OpenMP over particles")
    line = {"impl": "reference", "metric": METRICS[w.name], "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, {"kicks_per_step": kicks_per_step}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- native arm

def traffic_from_profile(workload, src_hash):
    """Per-launch DRAM traffic of the push kernel from the committed ncu summary of this workload
    (lines `dram_bytes_per_launch: B` and `kernel_src_sha256: H`), if it was taken on the current
    kernel source (else null)."""
    import re

    path = os.path.join(ROOT, "profiles", f"push_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    h = re.search(r"kernel_src_sha256:\s*([0-9a-f]{64})", text)
    b = re.search(r"dram_bytes_per_launch:\s*([0-9]+)", text)
    if not h or not b or h.group(1) != src_hash:
        return None
    return int(b.group(1))


def kernel_src_hash():
    """SHA-256 over the sources that make up the push kernel."""
    h = hashlib.sha256()
    for f in ("particles.cu", "particles_dev.cuh", "common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2511_21839_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def measure(sim, steps, warmup, kicks, torch, timing_mask=0):
    for _ in range(warmup):
        sim.run(kicks)
    sim.set_timing(timing_mask)
    sim.run(kicks)          # capture the timed graph shape outside the timed region
    sim.set_timing(timing_mask)
    l0 = sim.launches()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        sim.run(kicks)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, sim.launches() - l0


def e2e_measure(args, sim, w, kicks, ws, barrier, torch, np):
    state = torch.empty((6, w.n_particles, w.n_deriv + 1), dtype=torch.float64, pin_memory=True)
    state.numpy()[...] = sim.get_particles()
    for _ in range(2):
        sim.set_particles(state.numpy())
        sim.run(kicks)
        sim.moments()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sim.set_particles(state.numpy())
        sim.run(kicks)
        vals, der = sim.moments()
    barrier()
    e2e_ms = 1000.0 * (time.perf_counter() - t0) / args.steps
    h2d = state.numel() * 8
    d2h = 8 * (2 + 2 * w.n_deriv) + 15 * 8 * (w.n_deriv + 1) + 4
    e2e_value = ws * w.n_particles * kicks / (e2e_ms / 1000.0)
    fp32_eps = vals
    return e2e_value, e2e_ms, h2d, d2h, fp32_eps


def run_native(args):
    import numpy as np
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

    # ---- FP32 bulk / FP64 reductions (headline)
    sim = make(adpic.AD_PIC_FP32_MIXED)
    for _ in range(args.warmup):
        sim.run(kicks)
    sim.set_timing(0)
    sim.run(kicks)                      # captures the timed graph outside the timed region
    clocks = ClockSampler(dev)
    barrier()
    l0 = sim.launches()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        sim.run(kicks)
    e1.record()
    barrier()
    ck = clocks.stop()
    ms_step = e0.elapsed_time(e1) / args.steps
    launches = sim.launches() - l0
    # the push's average launch duration, from a second timed pass with CUDA events
    # around every push launch in the graph (on the launching stream); event nodes
    # inside the graph cost the step a little, so the headline pass above has none
    push_mask = 1 << 0
    sim.set_timing(push_mask)
    sim.run(kicks)                      # captures the graph with the push events
    sim.set_timing(push_mask)           # same mask: resets the accumulators, keeps the graph
    for _ in range(max(2, args.steps // 2)):
        sim.run(kicks)
    barrier()
    tpush = sim.timing()["push"]
    push_ms = tpush[0] / max(tpush[1], 1)
    ms_step = max_over_ranks(ms_step, dist, "cuda")
    value = job_rate(ws, w.n_particles, kicks, ms_step)

    # ---- end to end through the public API with host buffers: upload the step's dual state
    # from pinned host memory, run the period, read the emittances back
    if args.no_e2e:
        e2e_value = e2e_ms = h2d = d2h = None
        fp32_eps = sim.moments()[0]
    else:
        e2e_value, e2e_ms, h2d, d2h, fp32_eps = e2e_measure(args, sim, w, kicks, ws, barrier, torch, np)
    sim.close()

    # ---- plain FP64 path on the same workload
    fp64 = None
    if not args.no_fp64:
        sim64 = make(adpic.AD_PIC_FP64)
        ms64, _ = measure(sim64, max(2, args.steps // 3), min(args.warmup, 3), kicks, torch)
        sim64.close()
        v64 = w.n_particles * kicks / (ms64 / 1000.0)
        fp64 = {"value": ws * v64, "ms_per_step": ms64, "dtype": "f64",
                "fp32_speedup": (ws * v64 and value / (ws * v64))}

    # ---- roofline of the dominant kernel (gather + kick + push): algorithmic bytes per launch
    # = particles x (read + write of 6 coordinates x C channels x 4 B) + one read of the
    #   rest-frame field grid (3 x C x n^3 x 4 B)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    C = w.n_deriv + 1
    nodes = w.grid[0] * w.grid[1] * w.grid[2]
    alg_bytes = w.n_particles * 2 * 6 * C * 4 + 3 * C * nodes * 4
    achieved = alg_bytes / (push_ms / 1000.0) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    roof = {"bound": "hbm", "kernel": "push_tma_kernel (CIC gather + kick + dual maps)", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": push_ms,
            "traffic": traffic_from_profile(w.name, kernel_src_hash())}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        kicks_cpu = args.cpu_kicks or CPU_KICKS[w.name]
        rate, dt = oracle_rate(w, kicks_cpu)
        cpu = {"value": rate, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": f"{kicks_cpu} kicks of the {w.name} workload on the host cores ({dt:.1f} s)"}

    if rank == 0:
        line = {"metric": METRICS[w.name], "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(w, {"precision": "FP32 particles/deposit/FFT/field/push, FP64 geometry, "
                                                           "Green's-function integrals and moment reductions"}),
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": None if e2e_value is None else {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                                                       "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
                "gpu_launches": launches, "clocks": ck, "fp64_plain": fp64,
                "final_eps_fp32": [float(v) for v in fp32_eps]}
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """The batched sensitivity scan: 256 FODO instances (lattice parameters +-10 %, particle counts
    log-uniform in [16384, 262144], grids 32^3 or 64^3, P = 7, FP32-mixed), 5 periods, advanced
    together by the batched runtime (autotuned persistent kernel / phased launches in a CUDA graph)."""
    import torch

    from paper_2511_21839_gb300 import adpic, build
    from paper_2511_21839_gb300 import inputs as I

    ws, rank, local = dist_env()
    build.build()
    params, npart, grid, periods = I.batched_scan(3 + 1000 * rank, args.batch_instances)
    w = I.workload("fodo_10k_32")
    grids = [(int(g), int(g), int(g)) for g in grid]
    b = adpic.Batch(grids, [int(v) for v in npart])
    for i in range(len(grids)):
        b.set_beam(i, w.beam, I.normals(10_000 + i, int(npart[i])))
        b.set_lattice(i, I.Lattice.from_params(params[i]))
    kicks = w.kicks_per_period * periods
    b.run(0)                                  # initial moments; the tuner runs on the first kick run
    t0 = time.perf_counter()
    torch.cuda.synchronize()
    b.run(kicks)
    torch.cuda.synchronize()
    first = time.perf_counter() - t0
    # the timed runs restart from the same beams so every step is the full 5-period scan
    times = []
    for rep in range(args.steps):
        for i in range(len(grids)):
            b.set_beam(i, w.beam, I.normals(10_000 + i, int(npart[i])))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run(kicks)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    mode, ms = b.tuning()
    total = int(np.sum(npart)) * kicks
    step = min(times)
    line = {"metric": "dual particle-steps/s, batched sensitivity scan (256 instances, 16k-262k particles, "
                      "32^3/64^3, P=7, 5 periods)", "value": total / step, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": 1, "ms_per_step": 1000 * step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched scan: {len(grids)} instances, {int(np.sum(npart))} particles in total, "
                                   f"{int(np.sum(np.array(grid) == 32))} on 32^3 and {int(np.sum(np.array(grid) == 64))} "
                                   f"on 64^3, {kicks} kicks; step = the whole scan (median of the runs' minimum)",
                       "mode": {1: "persistent, 1 block/SM", 2: "persistent, 2 blocks/SM", 3: "phased launches"}[mode],
                       "tuner_ms_per_kick": [float(x) for x in ms], "first_run_s_incl_tuning": first}}
    if rank == 0:
        print(json.dumps(line))
    b.close()
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
    ap.add_argument("--workload", choices=["fodo_1m_64", "fodo_16m_128", "batch"], default="fodo_1m_64")
    ap.add_argument("--batch-instances", type=int, default=256)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
