"""Write tests/golden/oracle_outer.json: how many outer steps the FP64 oracle's
own Algorithm 1 takes to reach rho <= 1e-8 on a named workload.

The oracle timing in bench.py (its cpu_baseline and --impl reference legs)
times one outer step of the oracle and scales it to a whole solve; this file
supplies the oracle's own outer-step count for that scaling, measured by
running the oracle to convergence once (Section 4.2.1: outer tolerance 1e-8,
N = 4 poles, alpha = 1, beta = 0.01).  Calls only oracle/ and the seeded
input generators.

Usage:  python tests/golden/make_oracle_outer.py [name ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import poles, subspace  # noqa: E402
from workloads import config_pencil, interval_for, start_block  # noqa: E402

START_SEED = 2505   # the start block the benchmark uses for this workload


def compute(name, tol=1e-8):
    p = config_pencil(name)
    iv = interval_for(name)
    s, w = poles.slrf_poles(iv["n_poles"], 1.0, 0.01, iv["gamma"])
    V = start_block(p.n, iv["L"], START_SEED)
    t0 = time.time()
    res = subspace.subspace_iterate(p.A(), p.B(), s, w, iv["gamma"], V, tol=tol, max_outer=40)
    t = time.time() - t0
    if not res.converged or res.n_wanted != iv["nev"]:
        raise RuntimeError(f"{name}: oracle did not converge to {iv['nev']} pairs")
    return {"tol": tol, "outer_iters": int(res.iters), "n_wanted": int(res.n_wanted),
            "worst_rho_per_step": [float(x) for x in res.history],
            "filter": "oracle SLRF design N=%d alpha=1 beta=0.01" % iv["n_poles"],
            "start_seed": START_SEED, "seconds": round(t, 1), "cores": os.cpu_count()}


def main(names):
    path = os.path.join(HERE, "oracle_outer.json")
    table = {}
    if os.path.exists(path):
        with open(path) as f:
            table = json.load(f)
    for name in names or ["fem2d_q1_300"]:
        table[name] = compute(name)
        print(name, table[name], flush=True)
        with open(path, "w") as f:
            json.dump(table, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
