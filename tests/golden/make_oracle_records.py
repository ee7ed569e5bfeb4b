"""Write the FP64 oracle's moment records of the 1M-particle FODO run (1,048,576 particles, 64^3,
P = 7, ten periods of 20 kicks) to oracle_fodo_1m_64.json, for the GPU parity tests.

Calls only oracle/ (and the input recipe); nothing here comes from the CUDA path. The oracle's
moments use compensated sums, so the stored values do not depend on the thread count beyond the
rounding of the particle trajectories.

    python tests/golden/make_oracle_records.py [--periods 10]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2511_21839_gb300 import inputs as I  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--periods", type=int, default=10)
    ap.add_argument("--out", default=os.path.join(HERE, "oracle_fodo_1m_64.json"))
    args = ap.parse_args()
    w = I.workload("fodo_1m_64")
    o = oracle.Oracle(**I.orc_kwargs(w))
    st = o.beam_init(I.normals(w.seed, w.n_particles))
    recs = [o.moments(st)]
    t0 = time.time()
    for p in range(args.periods):
        hist, _ = o.run(st, w.kicks_per_period, kick0=p * w.kicks_per_period)
        recs.append(hist[-1])
        print(f"period {p + 1}: {time.time() - t0:.0f} s", flush=True)
    eps = [o.emittance(r)[:2].tolist() for r in recs]
    doc = {"workload": "fodo_1m_64: 1,048,576 particles, 64^3 grid, P = 7, FODO period of 20 kicks, seed 2",
           "written_by": "tests/golden/make_oracle_records.py (FP64 oracle only)",
           "threads": oracle.threads(),
           "records": "record 0 = initial state, record r = end of period r",
           "layout": "eps[record][plane x, y][channel: value, d/d(L_D1, L_QF, g_QF, L_D2, L_QD, g_QD, L_D3)]",
           "moments_layout": "moments[record][plane x, y, z][<u>, <p>, <u^2>, <u p>, <p^2>][channel]",
           "eps": eps,
           "moments": [np.asarray(r).tolist() for r in recs]}
    with open(args.out, "w") as f:
        json.dump(doc, f, indent=0)
    print("wrote", args.out)


if __name__ == "__main__":
    main()
