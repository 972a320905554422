"""Benchmark: converged eigenpairs per second of the rational-filter eigensolver.

One step = one complete Algorithm 1 solve (filter by batched COCG over all
poles x columns, Cholesky-QR2, Rayleigh-Ritz, residuals, until every Ritz pair
in (0, gamma] has rho <= 1e-8) of the 2D Q1 workload: 300 x 300 bilinear
elements, lognormal coefficient, n = 89 401, 100 eigenvalues in (0, gamma],
subspace L = 150, N = 4 SLRF poles (alpha = 1, beta = 0.01), mixed precision
(FP32 Krylov on the FP64 residual, FP64 projection).  Inputs are synthetic and
seeded; the start block and the pencil are resident on the device before the
timed region.

The same line carries, as sub-records (skipped with --no-extra), the 3D
elasticity workload (40^3 nodes x 3 dof, n = 187 200, 200 eigenpairs, with
the shifted product's roofline against a measured FP32 FMA peak), the batch
of 64 independent pencils, and a served request stream (the first requests
of the seeded 1000-request Poisson stream, p50/p99 latency).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run; ranks are independent replicas
(the solve does not shard: weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "fem2d_q1_300"
METRIC = "eigenpairs/s at resid 1e-8 (2D Q1 n=89401, 100 eigenpairs, mixed FP32/FP64)"
UNIT = "eigenpairs/s"
TOL = 1e-8
MAX_OUTER = 40
# kernel classes that can carry the roofline: the source file their kernels
# live in (digest checked against the ncu summary) and that summary
ROOFLINE_SOURCES = {"shifted_spmm": "krylov.cu", "mg_fine": "mg.cu"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def source_digest(kclass: str) -> str:
    path = os.path.join(ROOT, "paper_2503_21618_gb300", "csrc", ROOFLINE_SOURCES[kclass])
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def ncu_traffic_per_launch(kclass: str):
    """DRAM bytes per launch of the roofline kernel class from the committed
    ncu summary, or None if absent or taken on a different kernel source."""
    summary = os.path.join(ROOT, "profiles", f"{kclass}_fem2d_q1_300.md")
    if not os.path.exists(summary):
        return None, "no ncu summary"
    text = open(summary).read()
    m = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    d = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    if not m:
        return None, "summary has no traffic line"
    if not d or d.group(1) != source_digest(kclass):
        return None, "kernel changed since the ncu capture"
    return float(m.group(1)), "ncu"


def aggregate(seconds: float, units: float, device="cpu"):
    """Whole-job throughput of replicas: units summed over ranks, divided by
    the slowest rank's time (max over ranks).  Returns (value, t_max, units)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item()), float(u.item())


# ---------------------------------------------------------------------------
# oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_outer_step_seconds(p, iv, L, n_poles):
    """Time one outer step of the oracle's Algorithm 1 (exact sparse LU per pole)."""
    import numpy as np
    from oracle import filter as ofilt
    from oracle import poles, rr
    from workloads import start_block
    s, w = poles.slrf_poles(n_poles, 1.0, 0.01, iv["gamma"])
    V = start_block(p.n, L, 2505)
    A, B = p.A(), p.B()
    t0 = time.perf_counter()
    U = ofilt.filter_apply(A, B, s, w, V)
    theta, X = rr.rayleigh_ritz(A, B, U)
    rr.residuals(A, B, X, theta)
    t = time.perf_counter() - t0
    del np
    return t


def oracle_outer_count(name: str) -> int:
    """Outer steps the FP64 oracle's own Algorithm 1 takes to rho <= 1e-8 on
    this workload (written by tests/golden/make_oracle_outer.py, which runs
    the oracle to convergence once)."""
    with open(os.path.join(ROOT, "tests", "golden", "oracle_outer.json")) as f:
        return int(json.load(f)[name]["outer_iters"])


def cpu_baseline(p, iv):
    t = oracle_outer_step_seconds(p, iv, iv["L"], iv["n_poles"])
    outer = oracle_outer_count(WORKLOAD)
    return {"value": iv["nev"] / (t * outer), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"one outer step of the FP64 oracle Algorithm 1 (SuperLU per pole, dense eigh) on "
                       f"{WORKLOAD}: {t:.2f} s, times the oracle's own {outer} outer steps to rho <= 1e-8 "
                       f"(measured by running the oracle to convergence); SuperLU single-threaded, BLAS on up to "
                       f"{os.cpu_count()} threads")}


def run_reference(args, rank, world):
    """The oracle arm: each step is ONE outer step of the FP64 oracle's
    Algorithm 1 (a bounded sample of the solve); the metric extrapolates a
    whole solve as that step time times the oracle's own outer-step count."""
    if rank != 0:
        return
    from workloads import config_pencil, interval_for
    p = config_pencil(WORKLOAD)
    iv = interval_for(WORKLOAD)
    outer = oracle_outer_count(WORKLOAD)
    for _ in range(args.warmup):
        oracle_outer_step_seconds(p, iv, iv["L"], iv["n_poles"])
    t0 = time.perf_counter()
    times = [oracle_outer_step_seconds(p, iv, iv["L"], iv["n_poles"]) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    t_step = statistics.mean(times)
    value = iv["nev"] / (t_step * outer)
    sample = (f"each step is one outer step of the FP64 oracle Algorithm 1 (SuperLU per pole, dense eigh) on "
              f"{WORKLOAD}; value = {iv['nev']} eigenpairs / (mean step time x {outer}, the oracle's own outer-step "
              f"count to rho <= 1e-8)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3 / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": p.n, "nnz": p.nnz, "L": iv["L"], "nev": iv["nev"],
                       "n_poles": iv["n_poles"], "step": "one oracle outer step",
                       "oracle_outer_steps_per_solve": outer},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# many problems: batched pencils and a served request stream
# ---------------------------------------------------------------------------
def serve_stream(pkg, count, n_lo=10000, n_hi=500000, nev_lo=20, nev_hi=200, rate=1.0, workers=2):
    """Submit a seeded Poisson-arrival stream of 2D/3D eigen-solve requests to
    the library's server; return latency percentiles and throughput."""
    import numpy as np
    from workloads import serving_stream
    stream = serving_stream(count, n_lo=n_lo, n_hi=n_hi, nev_lo=nev_lo, nev_hi=nev_hi, rate_per_s=rate)
    filters = [pkg.design_poles("slrf", 4, pr["gamma"], 1.0, 0.01) for _, pr in stream]
    srv = pkg.api.Server(n_workers=workers)
    t0 = time.perf_counter()
    tickets = []
    for (t_arr, pr), f in zip(stream, filters):
        delay = t_arr - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(pr["pencil"], f, pr["gamma"], pr["V0"], tol=TOL, max_outer=MAX_OUTER))
    lat, conv, statuses, sizes, detail = [], 0, [], [], []
    for t, (t_arr, pr) in zip(tickets, stream):
        th, X, r, nc, st, rep, lt = srv.poll(t, wait=True)
        lat.append(lt)
        conv += nc if st == pkg.OK else 0
        statuses.append(int(st))
        sizes.append(int(pr["pencil"].n))
        if len(detail) < 64:
            detail.append({"kind": pr["kind"], "n": int(pr["pencil"].n), "nev": int(pr["nev_target"]),
                           "arrival_s": round(float(t_arr), 3), "status": int(st), "latency_ms": round(float(lt), 1),
                           "solve_ms": round(float(rep.ms_total), 1), "outer": int(rep.outer_iters)})
    wall = time.perf_counter() - t0
    srv.close()
    return {"requests": count, "workers": workers, "arrival_rate_per_s": rate,
            "n_range": [min(sizes), max(sizes)], "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "eigenpairs_per_s": conv / wall, "wall_s": wall,
            "converged_eigenpairs": conv, "ok": sum(1 for x in statuses if x == 0), "detail": detail}


def run_serve(args, pkg, rank, world):
    if rank != 0:
        return
    res = serve_stream(pkg, args.requests, rate=0.5, workers=4)
    print(json.dumps({"metric": "served eigenpairs/s and latency (2D/3D FE requests, Poisson arrivals)",
                      "value": res["eigenpairs_per_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
                      "data": "synthetic", "dtype": "f32/f64", "config": {"workload": "serve"}, "serving": res}),
          flush=True)


def run_filters(args, pkg, rank, world):
    """The paper's filter comparison (Section 3.2, Tables 4 and 5) on the 2D
    workload: the same solve with SLRF and circle-quadrature pole sets."""
    if rank != 0:
        return
    import torch
    from workloads import config_pencil, interval_for, start_block
    p = config_pencil(WORKLOAD)
    iv = interval_for(WORKLOAD)
    g = iv["gamma"]
    V0 = torch.from_numpy(start_block(p.n, iv["L"], 2505)).cuda()
    cases = [("SLRF a=1 b=0.01", pkg.design_poles("slrf", 4, g, 1.0, 0.01)),
             ("SLRF a=0.5 b=0.01", pkg.design_poles("slrf", 4, g, 0.5, 0.01)),
             ("SLRF a=2 b=0.01", pkg.design_poles("slrf", 4, g, 2.0, 0.01)),
             ("SLRF a=1 b=1", pkg.design_poles("slrf", 4, g, 1.0, 1.0)),
             ("midpoint", pkg.design_poles("midpoint", 4, g)),
             ("Gauss-Legendre", pkg.design_poles("gauss_legendre", 4, g)),
             ("Gauss-Chebyshev", pkg.design_poles("gauss_chebyshev", 4, g))]
    # one fixed preconditioner for every pole set (the paper's Table 4 uses one
    # ILU setting): Jacobi, so that the iteration counts show the pole placement
    h = pkg.Handle(p, pkg.default_opts(precond=pkg.PRECOND_JACOBI))
    rows = []
    for name, f in cases:
        h.subspace_iterate(f, g, V0, tol=TOL, max_outer=MAX_OUTER)   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        th, X, r, nc, st, rep = h.subspace_iterate(f, g, V0, tol=TOL, max_outer=MAX_OUTER)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        sep = abs(sum((-2.0 * (w / (g - s) ** 2)).real for s, w in zip(f.sigma, f.w)))
        rows.append({"filter": name, "status": int(st), "converged": int(nc), "seconds": round(t, 3),
                     "eigenpairs_per_s": round((nc if st == pkg.OK else 0) / t, 2), "outer_iters": rep.outer_iters,
                     "spmv_total": int(rep.spmv), "spmv_per_outer": round(rep.spmv / max(1, rep.outer_iters), 1),
                     "iters_per_pole": [round(x, 1) for x in list(rep.iters_per_pole)[:4]],
                     "min_imag_pole_over_gamma": round(float(min(f.sigma.imag)) / g, 4),
                     "separation_factor_gamma": round(sep * g, 3)})
    h.close()
    print(json.dumps({"metric": "filter comparison (2D Q1 n=89401, 100 eigenpairs, N=4 poles)",
                      "unit": UNIT, "data": "synthetic", "config": {"workload": WORKLOAD, "precond": "jacobi"},
                      "rows": rows}), flush=True)


def run_batch(args, pkg, rank, world):
    import torch
    from workloads import batch_workload
    probs = batch_workload(args.problems)
    filters = [pkg.design_poles("slrf", 4, pr["gamma"], 1.0, 0.01) for pr in probs]
    V0s = [torch.from_numpy(pr["V0"]).cuda() for pr in probs]
    streams = [torch.cuda.Stream() for _ in probs]
    handles = [pkg.Handle(pr["pencil"], stream=st) for pr, st in zip(probs, streams)]
    gam = [pr["gamma"] for pr in probs]
    pkg.api.batch_iterate(handles, filters, gam, V0s, tol=TOL, max_outer=MAX_OUTER)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = pkg.api.batch_iterate(handles, filters, gam, V0s, tol=TOL, max_outer=MAX_OUTER)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    # every eigenpair that passed both gates counts, also from problems that
    # stopped short of all wanted pairs (stagnation, iteration cap)
    conv = sum(r[3] for r in res)
    t0 = time.perf_counter()
    for h, f, g, v in zip(handles, filters, gam, V0s):
        h.subspace_iterate(f, g, v, tol=TOL, max_outer=MAX_OUTER)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    if rank == 0:
        print(json.dumps({"metric": "batched eigenpairs/s (64 FE pencils, n log-uniform in [1k, 50k])",
                          "value": conv / t_batch, "unit": UNIT, "n_gpus": world, "higher_is_better": True,
                          "data": "synthetic", "dtype": "f32/f64",
                          "config": {"workload": "batch", "problems": len(probs),
                                     "kinds": {k: sum(1 for p in probs if p["kind"] == k) for k in ("1d", "2d", "3d")}},
                          "seconds_batched": t_batch, "seconds_one_by_one": t_seq,
                          "eigenpairs_per_s_one_by_one": conv / t_seq, "converged_eigenpairs": conv,
                          "ok": sum(1 for r in res if r[4] == pkg.OK),
                          "not_ok": [{"kind": pr["kind"], "n": int(pr["pencil"].n), "nev": int(pr["nev_target"]),
                                      "status": int(r[4]), "n_conv": int(r[3]), "n_wanted": int(r[5].n_wanted),
                                      "outer": int(r[5].outer_iters), "max_resid": float(r[5].max_resid),
                                      "iters_per_pole": [round(x, 1) for x in r[5].iters_per_pole[:4]]}
                                     for pr, r in zip(probs, res) if r[4] != pkg.OK]}), flush=True)
    for h in handles:
        h.close()


# ---------------------------------------------------------------------------
# sub-records of the default line: the 3D elasticity and batched configs
# ---------------------------------------------------------------------------
def class_mask(pkg, names):
    m = 0
    for i in range(pkg.api.NKERNEL_CLASSES):
        if pkg.api.class_name(i) in names:
            m |= 1 << i
    return m


def spmm_formats(pkg, p, f, V0, hbm_peak):
    """The 2D workload's shifted product in its CSR row-group form against
    SELL-C-sigma (two chunk/sorting-window shapes): one filter application per
    form with every shifted-product launch timed by CUDA events; algorithmic
    bytes as in the roofline (pattern + FP32 pairs once, P read and Q written
    for the active columns)."""
    import torch
    out = {}
    for name, kw in (("csr_rowgroup", dict(spmm_kernel=1)),
                     ("sell_c32_sigma256", dict(spmm_kernel=4, sell_c=32, sell_sigma=256)),
                     ("sell_c8_sigma1", dict(spmm_kernel=4, sell_c=8, sell_sigma=1))):
        h = pkg.Handle(p, pkg.default_opts(profile=1, profile_mask=class_mask(pkg, {"shifted_spmm"}), **kw))
        h.filter_apply(f, V0)                       # warm-up
        torch.cuda.synchronize()
        _, st, rep = h.filter_apply(f, V0)
        k = rep.as_dict()["kernels"].get("shifted_spmm", {"launches": 0, "ms": 0.0, "bytes": 0.0})
        h.close()
        gbs = k["bytes"] / (k["ms"] / 1e3) / 1e9 if k["ms"] else None
        out[name] = {"spmm_kernel": int(rep.spmm_kernel), "launches": k["launches"],
                     "avg_launch_us": k["ms"] / k["launches"] * 1e3 if k["launches"] else None,
                     "achieved_gbs": gbs, "frac": gbs / hbm_peak if gbs and hbm_peak else None}
    return out


def bench_3d(pkg, fp32_peak):
    """One timed solve of the 3D elasticity workload (40^3 nodes x 3 dof,
    n = 187 200, 200 eigenpairs, L = 300, N = 4, mixed precision), after a
    one-outer-step warm-up; the shifted product's FP32 throughput against the
    measured FP32 FMA peak (its arithmetic intensity, ~37 flop per HBM byte,
    is above the HBM ridge)."""
    import numpy as np
    import torch
    from workloads import config_pencil, interval_for, start_block
    name = "fem3d_elastic_40"
    p = config_pencil(name)
    iv = interval_for(name)
    f = pkg.design_poles("slrf", iv["n_poles"], iv["gamma"], 1.0, 0.01)
    t0 = time.perf_counter()
    h = pkg.Handle(p, pkg.default_opts(profile=1, profile_mask=class_mask(pkg, {"shifted_spmm"})))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    V0 = torch.from_numpy(start_block(p.n, iv["L"], 2506)).cuda()
    h.subspace_iterate(f, iv["gamma"], V0, tol=TOL, max_outer=1)          # warm-up: workspace, modules
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    theta, X, resid, nc, st, rep = h.subspace_iterate(f, iv["gamma"], V0, tol=TOL, max_outer=MAX_OUTER)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    lam = np.array(iv["lambda"][: iv["nev"]])
    th = theta.cpu().numpy()[: iv["nev"]]
    k = rep.as_dict()["kernels"].get("shifted_spmm", {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0})
    h.close()
    ach = k["flops"] / (k["ms"] / 1e3) if k["ms"] else None
    return {"workload": name, "n": p.n, "nnz": p.nnz, "L": iv["L"], "nev": iv["nev"], "n_poles": iv["n_poles"],
            "precision": "mixed", "precond": "jacobi (AUTO on 3-dof node-block pencils)",
            "spmm_kernel": int(rep.spmm_kernel),
            "value": (int(nc) if st == pkg.OK else 0) / t, "unit": UNIT, "seconds": t, "status": int(st),
            "converged": int(nc), "outer_iters": rep.outer_iters, "max_resid": rep.max_resid,
            "max_rel_eig_err_vs_oracle": float(np.max(np.abs(th - lam) / lam)) if int(nc) == iv["nev"] else None,
            "iters_per_pole": [round(x, 1) for x in list(rep.iters_per_pole)[: iv["n_poles"]]],
            "setup_s": t_setup, "warmup": "one outer step", "steps": 1,
            "roofline": {"kernel": "shifted_spmm", "bound": "alu", "achieved": ach / 1e12 if ach else None,
                         "peak": fp32_peak / 1e12 if fp32_peak else None, "unit": "TFLOP/s",
                         "frac": (ach / fp32_peak) if ach and fp32_peak else None,
                         "peak_source": "measured FP32 FMA (slrf_fma_peak)",
                         "achieved_gbs": (k["bytes"] / (k["ms"] / 1e3) / 1e9) if k["ms"] else None,
                         "launches": k["launches"],
                         "avg_launch_us": (k["ms"] / k["launches"] * 1e3) if k["launches"] else None}}


def status_counts(pkg, statuses):
    names = {getattr(pkg.api, k): k for k in ("OK", "NOT_CONVERGED", "STAGNATION", "BREAKDOWN", "SUBSPACE_TOO_SMALL",
                                               "CHOLQR_FAIL", "ETIMEOUT", "ENOMEM", "EBUDGET")}
    out = {}
    for st in statuses:
        key = names.get(int(st), str(int(st)))
        out[key] = out.get(key, 0) + 1
    return out


def bench_batch(pkg, count=64):
    """The batched config: 64 independent FE pencils (n log-uniform in
    [1k, 50k], kinds 1D/2D/3D), each on its own handle and stream, solved
    together by slrf_batch_iterate; one timed batch after a one-outer-step
    warm-up of every handle."""
    import torch
    from workloads import batch_workload
    probs = batch_workload(count)
    filters = [pkg.design_poles("slrf", 4, pr["gamma"], 1.0, 0.01) for pr in probs]
    V0s = [torch.from_numpy(pr["V0"]).cuda() for pr in probs]
    streams = [torch.cuda.Stream() for _ in probs]
    t0 = time.perf_counter()
    handles = [pkg.Handle(pr["pencil"], stream=st) for pr, st in zip(probs, streams)]
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    gam = [pr["gamma"] for pr in probs]
    pkg.api.batch_iterate(handles, filters, gam, V0s, tol=TOL, max_outer=1)     # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = pkg.api.batch_iterate(handles, filters, gam, V0s, tol=TOL, max_outer=MAX_OUTER)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    for h in handles:
        h.close()
    conv = sum(r[3] for r in res)
    return {"workload": "batch", "problems": len(probs),
            "kinds": {k: sum(1 for p in probs if p["kind"] == k) for k in ("1d", "2d", "3d")},
            "n_range": [min(int(p["pencil"].n) for p in probs), max(int(p["pencil"].n) for p in probs)],
            "value": conv / t, "unit": UNIT, "seconds": t, "converged_eigenpairs": int(conv),
            "ok": sum(1 for r in res if r[4] == pkg.OK), "statuses": status_counts(pkg, [r[4] for r in res]),
            "setup_s": t_setup, "warmup": "one outer step per problem", "steps": 1,
            "counting": "every eigenpair that passed both gates, also from problems that stopped short"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 GPU baseline solve")
    ap.add_argument("--workload", default="fem2d_q1_300", choices=["fem2d_q1_300", "batch", "serve", "filters"])
    ap.add_argument("--requests", type=int, default=16, help="serve: number of requests")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the 3D elasticity, batched and served sub-records of the default line")
    ap.add_argument("--problems", type=int, default=64, help="batch: number of pencils")
    args = ap.parse_args()
    rank, world, local = dist_env()

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() and args.impl == "ours" else "gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            dist.destroy_process_group()
        return

    import numpy as np
    torch.cuda.set_device(local)
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import paper_2503_21618_gb300 as pkg
    from workloads import config_pencil, interval_for, start_block

    if args.workload == "batch":
        run_batch(args, pkg, rank, world)
        return
    if args.workload == "serve":
        run_serve(args, pkg, rank, world)
        return
    if args.workload == "filters":
        run_filters(args, pkg, rank, world)
        return

    p = config_pencil(WORKLOAD)
    iv = interval_for(WORKLOAD)
    L, nev, N = iv["L"], iv["nev"], iv["n_poles"]
    f = pkg.design_poles("slrf", N, iv["gamma"], 1.0, 0.01)
    # the timed steps record CUDA events around the launches of the roofline
    # classes only; the share of every class comes from one more, fully
    # profiled step after the timed region
    rmask = 0
    for i in range(pkg.api.NKERNEL_CLASSES):
        if pkg.api.class_name(i) in ROOFLINE_SOURCES:
            rmask |= 1 << i
    opts = pkg.default_opts(profile=1, profile_mask=rmask)
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    h = pkg.Handle(p, opts)     # pencil upload, row groups, multigrid hierarchy (host)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    V0 = torch.from_numpy(start_block(p.n, L, 2505)).cuda()
    theta = torch.empty(L, dtype=torch.float64, device="cuda")
    X = torch.empty_like(V0)
    resid = torch.empty(L, dtype=torch.float64, device="cuda")

    def step():
        return h.subspace_iterate(f, iv["gamma"], V0, tol=TOL, max_outer=MAX_OUTER, theta=theta, X=X, resid=resid)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    reps, conv, outer = [], [], []
    for _ in range(args.steps):
        *_, nconv, st, rep = step()
        reps.append(rep.as_dict())
        conv.append(int(nconv) if st == pkg.OK else 0)
        outer.append(rep.outer_iters)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    value, t_max, _ = aggregate(t, float(sum(conv)), "cuda")

    # roofline of the dominant kernel from the live per-launch events
    tot = {}
    for r in reps:
        for k, v in r["kernels"].items():
            a = tot.setdefault(k, {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0})
            for key in a:
                a[key] += v[key]
    # the roofline kernel: the class with the largest device time
    rclass = max((c for c in ROOFLINE_SOURCES if c in tot), key=lambda c: tot[c]["ms"])
    k = tot[rclass]
    peaks, peak_src = measured_peaks()
    achieved = (k["bytes"] / k["launches"]) / (k["ms"] / k["launches"] / 1e3) / 1e9 if k["launches"] else None
    traffic, traffic_src = ncu_traffic_per_launch(rclass)
    launches = sum(r["kernel_launches"] for r in reps)
    h.set_opts(profile=1, profile_mask=0)
    *_, rep_all = step()
    h.set_opts(profile=1, profile_mask=rmask)
    ka = rep_all.as_dict()["kernels"]
    kshare = {kk: round(v["ms"] / max(1e-9, sum(x["ms"] for x in ka.values())), 4) for kk, v in ka.items()}

    # end to end: the public host-buffer call, inputs copied from pinned host memory every step
    e2e = None
    if rank == 0 or world > 1:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        V0h = pin(start_block(p.n, L, 2505))
        hp = type(p)(n=p.n, row_ptr=pin(p.row_ptr), col_idx=pin(p.col_idx), a_val=pin(p.a_val), b_val=pin(p.b_val))
        h2d = p.row_ptr.nbytes + p.col_idx.nbytes + p.a_val.nbytes + p.b_val.nbytes + V0h.nbytes
        d2h = p.n * L * 8 + 2 * L * 8
        # results land in pinned host arrays (allocated once, like the inputs)
        th_o, X_o, r_o = pin(np.zeros(L)), pin(np.zeros((p.n, L))), pin(np.zeros(L))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_conv = 0
        for _ in range(args.steps):
            he = pkg.Handle(hp, pkg.default_opts())
            th_h, X_h, r_h, nc, st, _ = he.subspace_iterate_host(f, iv["gamma"], V0h, tol=TOL, max_outer=MAX_OUTER,
                                                                 theta=th_o, X=X_o, resid=r_o)
            he.close()
            e_conv += int(nc) if st == pkg.OK else 0
        te = time.perf_counter() - t0
        e2e_value, _, _ = aggregate(te, float(e_conv), "cuda")
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "includes": "handle creation from host CSR, V0 upload, solve, X/theta/resid download "
                           "(pinned host buffers)"}

    plain = None
    if not args.no_plain and rank == 0:
        hp64 = pkg.Handle(p, pkg.default_opts(precision=pkg.PREC_FP64, inner_tol=1e-13, inner_maxit=1000))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        *_, nc, st, rep = hp64.subspace_iterate(f, iv["gamma"], V0, tol=TOL, max_outer=MAX_OUTER)
        torch.cuda.synchronize()
        tp = time.perf_counter() - t0
        plain = {"value": (int(nc) if st == pkg.OK else 0) / tp, "unit": UNIT, "seconds": tp,
                 "status": int(st), "outer_iters": rep.outer_iters, "max_resid": rep.max_resid}
        hp64.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": p.n, "nnz": p.nnz, "L": L, "nev": nev, "n_poles": N,
                       "filter": "SLRF alpha=1 beta=0.01 (library designer)", "precision": "mixed",
                       "inner_tol": opts.inner_tol, "tol": TOL, "parallelism": f"replicas x{world}",
                       "precond": "multigrid (smoothed aggregation)" if "mg_fine" in tot else "jacobi",
                       "spmm_kernel": {1: "row groups", 2: "staged (bulk copies to shared memory)",
                                       3: "node blocks", 4: "SELL-C-sigma"}.get(
                           reps[0]["spmm_kernel"], str(reps[0]["spmm_kernel"])) if reps else None,
                       "l2": "inputs larger than L2 (Krylov state 1.29 GB per solve)"},
            "converged_per_step": conv, "outer_iters": outer,
            "gpu_launches": int(launches),
            "clocks": clk,
            "roofline": {"kernel": rclass, "bound": "hbm", "achieved": achieved,
                         "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                         "frac": (achieved / peaks["hbm_gbs"]) if achieved else None,
                         "peak_source": f"{peak_src} hbm_gbs", "traffic": traffic,
                         "traffic_source": traffic_src,
                         "launches": k["launches"], "avg_launch_us": (k["ms"] / k["launches"] * 1e3)
                         if k["launches"] else None},
            "kernel_time_share": kshare,
            "time_split": {"setup_ms": t_setup * 1e3,
                           "krylov_ms_per_step": sum(r["ms_krylov"] for r in reps) / len(reps),
                           "rr_ms_per_step": sum(r["ms_rr"] for r in reps) / len(reps),
                           "setup": "handle creation: pencil upload, row groups and the other SpMM forms; the multigrid hierarchy is built on a host thread that the first solve waits for after its first projection"},
            "e2e": e2e,
        }
        if plain is not None:
            line["plain_fp64"] = plain
        if "shifted_spmm" in tot and tot["shifted_spmm"]["launches"]:
            ks = tot["shifted_spmm"]
            ach_s = ks["bytes"] / (ks["ms"] / 1e3) / 1e9
            line["spmm_roofline"] = {"kernel": "shifted_spmm", "bound": "hbm", "achieved": ach_s,
                                     "peak": peaks.get("hbm_gbs"), "unit": "GB/s", "frac": ach_s / peaks["hbm_gbs"],
                                     "peak_source": f"{peak_src} hbm_gbs", "launches": ks["launches"],
                                     "avg_launch_us": ks["ms"] / ks["launches"] * 1e3}
        if not args.no_extra:
            line["spmm_formats"] = spmm_formats(pkg, p, f, V0, peaks.get("hbm_gbs"))
            line["configs"] = {}
            fp32_peak = pkg.api.fma_peak(pkg.PREC_MIXED)
            line["fp32_fma_peak_tflops"] = fp32_peak / 1e12
            line["configs"]["fem3d_elastic_40"] = bench_3d(pkg, fp32_peak)
            line["configs"]["batch64"] = bench_batch(pkg)
            sv = serve_stream(pkg, count=args.requests, rate=0.5, workers=4)
            sv["cut"] = (f"the first {args.requests} requests of the seeded 1000-request stream (same n, NEV and "
                         f"arrival-time distribution), cut to fit the run")
            line["configs"]["serve"] = sv
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(p, iv)
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
