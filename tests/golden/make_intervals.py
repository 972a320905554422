"""Write tests/golden/intervals.json: the wanted interval and reference spectrum
of each named workload, computed by the FP64 oracle only.

For each workload the interval is (0, gamma] with gamma midway between the
oracle's lambda_NEV and lambda_{NEV+1}, so that exactly NEV eigenvalues lie in
it (the paper asks for all eigenvalues in (0, gamma], Section 1, and places no
eigenvalue on gamma).  The count is confirmed by Sylvester inertia of
A - gamma B.  The 1D spectrum is the closed form.

Usage:  python tests/golden/make_intervals.py [name ...]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import inertia  # noqa: E402
from workloads import CONFIGS, config_pencil  # noqa: E402


def compute(name):
    c = CONFIGS[name]
    p = config_pencil(name)
    nev = c["nev"]
    t0 = time.time()
    if c["kind"] == "1d":
        lam = inertia.lambda_1d(p.n)[: c["L"] + 5]
        source = "closed form (6/h^2)(1-cos k pi h)/(2+cos k pi h)"
    else:
        lam, _ = inertia.lowest_eigs(p.A(), p.B(), nev + 10)
        source = "scipy eigsh shift-invert about 0 (ARPACK), tol 1e-14"
    gamma = 0.5 * (lam[nev - 1] + lam[nev])
    if c["kind"] == "1d":
        count = inertia.count_below_1d(p.n, gamma)
        count_how = "Sturm recurrence on A - gamma B"
    else:
        count = inertia.count_below_sparse(p.A(), p.B(), gamma)
        count_how = "negative pivots of symmetric sparse LU of A - gamma B"
    if count != nev:
        raise RuntimeError(f"{name}: inertia count {count} != {nev}")
    return {
        "n": int(p.n), "nnz": int(p.nnz), "nev": nev, "L": c["L"], "n_poles": c["n_poles"],
        "gamma": float(gamma),
        "lambda_nev": float(lam[nev - 1]), "lambda_nev_plus_1": float(lam[nev]),
        "relative_gap": float((lam[nev] - lam[nev - 1]) / lam[nev]),
        "lambda": [float(v) for v in lam],
        "source": source, "inertia_count": int(count), "count_method": count_how,
        "seconds": round(time.time() - t0, 1),
    }


def main(names):
    path = os.path.join(HERE, "intervals.json")
    table = {}
    if os.path.exists(path):
        with open(path) as f:
            table = json.load(f)
    for name in names or list(CONFIGS):
        table[name] = compute(name)
        print(name, table[name]["gamma"], table[name]["seconds"], "s", flush=True)
        with open(path, "w") as f:
            json.dump(table, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:])
