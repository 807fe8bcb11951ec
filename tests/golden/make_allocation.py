"""Write tests/golden/mlmc_allocation_graphene.json: the fixed per-level sample
counts M_l of the graphene MLMC workload at TOL = 1e-3, from an oracle pilot.

Calls only oracle/ (and the synthetic workload parameters): for every level a
pilot of seeded level samples (eq. (2.6) differences, Sec. 3.3 coupling) gives
V_l = max over the energy grid of the sample variance; the work per sample is
the flop model W_l = sum over the level's eigen-solves of n^3 (Sec. 4.4, cost
per solve ~ N^6); eq. (2.7) then gives M_l.  Also records the oracle's own
seconds per level sample (one core each), used as context.

Run: python tests/golden/make_allocation.py [--procs P]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

PILOT = [400, 120, 24, 6]
SEED_OFFSET = 7_000_000   # pilot sample indices start here (disjoint from the bench's)


def _one(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import mlmc
    from synthetic import model_params, workload
    level, sample = args
    w = workload("graphene_mlmc")
    prm = model_params(w)
    t0 = time.perf_counter()
    Y = mlmc.level_sample(prm, w["levels"], level, sample, w["seed"])["Y"]
    return level, Y.tolist(), time.perf_counter() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count())
    a = ap.parse_args()
    import numpy as np
    from oracle import mlmc
    from synthetic import workload
    w = workload("graphene_mlmc")
    jobs = [(l, SEED_OFFSET + s) for l in range(4) for s in range(PILOT[l])]
    jobs.sort(key=lambda j: -j[0])
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.procs) as pool:
        res = pool.map(_one, jobs, chunksize=1)
    Ys = {l: [] for l in range(4)}
    secs = {l: [] for l in range(4)}
    for l, y, t in res:
        Ys[l].append(y)
        secs[l].append(t)
    V, W = [], []
    for l, (N, K) in enumerate(w["levels"]):
        Y = np.array(Ys[l])
        V.append(float(np.max(Y.var(axis=0, ddof=1))))
        nf = 2 * N * N
        work = K * K * nf ** 3
        if l > 0:
            Kc = w["levels"][l - 1][1]
            work += 4 * Kc * Kc * (nf // 4) ** 3
        W.append(float(work))
    Mi, M = mlmc.optimal_samples(V, W, w["tol"], w["theta"], w["c_alpha"])
    out = {
        "workload": "graphene_mlmc", "tol": w["tol"], "theta": w["theta"], "c_alpha": w["c_alpha"],
        "levels": w["levels"], "pilot_samples": PILOT, "pilot_first_sample": SEED_OFFSET,
        "V": V, "W_flop_model": W, "M": [int(x) for x in Mi], "M_real": [float(x) for x in M],
        "oracle_seconds_per_sample": [float(np.mean(secs[l])) for l in range(4)],
        "generator": "tests/golden/make_allocation.py (oracle only)",
    }
    with open(os.path.join(HERE, "mlmc_allocation_graphene.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
