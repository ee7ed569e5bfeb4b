"""Host logic of the multi-GPU replica runs, on CPU with two gloo ranks.

bench.py under torchrun gives every rank its own instance (seeded per rank, no
collective on the data path), takes the slowest rank's step time and reports the
whole job's rate. The same helpers are exercised here with the gloo backend.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    from paper_2511_21839_gb300 import inputs as I

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w = I.workload("fodo_1m_64")
    local_ms = 5.0 + 2.5 * rank                          # the slower rank sets the step time
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.job_rate(ws, w.n_particles, w.kicks_per_period, ms)
    seed = bench.rank_seed(w, rank)
    first = float(I.normals(seed, 4)[0, 0])
    out.put((rank, ms, rate, seed, first))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_replicas_take_the_slowest_rank_and_sum_the_work():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=90) for _ in range(2))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    (r0, ms0, rate0, s0, f0), (r1, ms1, rate1, s1, f1) = res
    assert ms0 == ms1 == 7.5                               # max over ranks
    sys.path.insert(0, ROOT)
    from paper_2511_21839_gb300 import inputs as I

    w = I.workload("fodo_1m_64")
    assert rate0 == rate1 == pytest.approx(2 * w.n_particles * w.kicks_per_period / 7.5e-3)
    assert s0 != s1 and f0 != f1                           # independent replicas


def test_push_traffic_record_is_read_only_for_its_source():
    """bench.py reports a figure from a committed ncu record only while the kernel sources hash to
    the value stored with it."""
    import re

    sys.path.insert(0, ROOT)
    import bench

    text = open(os.path.join(ROOT, "profiles", "push_fodo_1m_64.md")).read()
    stored = re.search(r"kernel_src_sha256:\s*([0-9a-f]{64})", text).group(1)
    b = int(re.search(r"dram_bytes_per_launch:\s*([0-9]+)", text).group(1))
    assert bench.profile_value("push_fodo_1m_64.md", "dram_bytes_per_launch", stored) == b
    assert bench.profile_value("push_fodo_1m_64.md", "dram_bytes_per_launch", "0" * 64) is None
    assert bench.profile_value("push_no_such_workload.md", "dram_bytes_per_launch", stored) is None
    assert re.fullmatch(r"[0-9a-f]{64}", bench.kernel_src_hash())


def test_bench_accuracy_helpers_match_the_oracle_records():
    """The bench's host emittance helper reproduces the oracle's emittances from its stored moment
    records, and the kick's algorithmic bytes match the figures of the roofline model."""
    import json

    sys.path.insert(0, ROOT)
    import bench

    doc = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_fodo_1m_64.json")))
    for mom, eps in zip(doc["moments"][1:], doc["eps"][1:]):
        ev, ed = bench.rel_errors(bench.emittances(np.array(mom)), np.array(eps))
        assert ev < 1e-14 and ed < 1e-12
    kb = bench.kick_bytes(1_048_576, (64, 64, 64), 8, 4)
    assert kb["particles"] == 402_653_184
    assert kb["rho"] + kb["field"] == 67_108_864
    assert kb["fft_model"] == 134_217_728
