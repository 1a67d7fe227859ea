"""Lid-driven cubic cavity (Sec. 4): centreline profiles at Re = 100, 400, 1000 and the
stability-threshold sweep, FPC-LBM against the Maxwellian central-moment (MCM) collision.

Setup (Sec. 4): closed box L^3 with half-way bounce-back on every face; the wall y = L - 1/2 moves
along x at U0 = Ma cs (momentum-corrected bounce-back), every other wall rests; fluid initially
at rest with rho = 1.  Re = U0 L / nu, nu = cs^2 (tau - 1/2), unit rates for the moments of
order >= 3 (drift = 0, the paper's experimental choice).

accuracy:  Ma = 0.1, run each Re until the centreline profiles u_x(y) (on x = z = L/2) and
           u_y(x) (on y = z = L/2) change by less than --tol U0 over one convective time L/U0,
           or --max-tc convective times.  With --levels L1 L2 ... the profiles of successive
           resolutions are compared at the coarse cell centres (self-convergence; no benchmark
           data is used).
stability: Ma = 0.2, for each L and collision the smallest tau (resolution --dtau) whose run
           stays finite for --steps steps, then Re_max = U0 L / nu(tau).  The paper scans tau
           upwards in steps of dtau; here the threshold is bracketed by bisection and then
           confirmed the paper's way: the --verify next increments above it must be stable too
           (otherwise the scan continues above the failure).

Usage: python -m paper_2410_09739_gb300.cavity_study accuracy [--levels 75 150] ...
       python -m paper_2410_09739_gb300.cavity_study stability [--sizes 48 64 80 96] ...
Prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2410_09739_gb300 import fpclbm as F  # noqa: E402

CS = 1.0 / math.sqrt(3.0)
MODELS = {"fpc": F.FPCLBM_DIFF_FP, "mcm": F.FPCLBM_DIFF_EQUILIBRIUM}


def tau_of(Re, U0, L):
    return 0.5 + 3.0 * U0 * L / Re


def cavity(L, tau, U0, model, precision="fp32", stream=0):
    lat = F.Lattice(L, L, L, precision, F.FPCLBM_BC_BOX, stream)
    lat.set_params(tau, 0.0, MODELS[model])
    lat.set_wall_velocity(U0)
    one = np.ones((L, L, L))
    lat.init_fields(one, 0 * one, 0 * one, 0 * one)
    return lat


def centrelines(lat, L):
    """u_x(y) on x = z = L/2 and u_y(x) on y = z = L/2 (mean of the two middle cells if L is even)."""
    rho, ux, uy, uz = (a.reshape(L, L, L) for a in lat.moments())  # [z, y, x]
    m = [L // 2] if L % 2 else [L // 2 - 1, L // 2]
    ux_y = np.mean([ux[z, :, x] for z in m for x in m], axis=0)
    uy_x = np.mean([uy[z, y, :] for z in m for y in m], axis=0)
    return ux_y, uy_x


def run_accuracy(args):
    U0 = args.ma * CS
    out = []
    for Re in args.re:
        per_level = {}
        for L in args.levels:
            for model in args.models:
                tau = tau_of(Re, U0, L)
                tc = int(round(L / U0))
                t0 = time.perf_counter()
                with cavity(L, tau, U0, model, args.precision) as lat:
                    prev = None
                    n_tc, change = 0, float("inf")
                    while n_tc < args.max_tc:
                        lat.step(tc)
                        n_tc += 1
                        cur = np.concatenate(centrelines(lat, L)) / U0
                        if prev is not None:
                            change = float(np.max(np.abs(cur - prev)))
                            if change < args.tol:
                                break
                        prev = cur
                    ux_y, uy_x = centrelines(lat, L)
                wall = time.perf_counter() - t0
                steps = n_tc * tc
                print(json.dumps({"Re": Re, "L": L, "model": model, "convective_times": n_tc, "change": change,
                                  "seconds": wall}), file=sys.stderr, flush=True)
                per_level[(L, model)] = (ux_y / U0, uy_x / U0)
                out.append({
                    "Re": Re, "L": L, "model": model, "tau": tau, "steps": steps, "convective_times": n_tc,
                    "last_change": change, "converged": change < args.tol,
                    "min_ux_over_U0": float(np.min(ux_y / U0)),
                    "y_of_min_ux_over_L": float((np.argmin(ux_y) + 0.5) / L),
                    "max_uy_over_U0": float(np.max(uy_x / U0)), "min_uy_over_U0": float(np.min(uy_x / U0)),
                    "ux_y_over_U0": [round(float(v), 6) for v in ux_y / U0],
                    "uy_x_over_U0": [round(float(v), 6) for v in uy_x / U0],
                    "mlups": L**3 * steps / wall / 1e6, "seconds": wall,
                })
        # self-convergence: successive levels at the coarse cell centres (fine cells 2i, 2i+1)
        for model in args.models:
            for Lc, Lf in zip(args.levels[:-1], args.levels[1:]):
                if Lf != 2 * Lc:
                    continue
                c, f = per_level[(Lc, model)], per_level[(Lf, model)]
                d = max(float(np.max(np.abs(c[k] - 0.5 * (f[k][0::2] + f[k][1::2])))) for k in (0, 1))
                out.append({"Re": Re, "model": model, "levels": [Lc, Lf], "max_centreline_diff_over_U0": d})
    return {"study": "lid-driven cavity accuracy", "Ma": args.ma, "U0": U0, "precision": args.precision,
            "results": out}


class Prober:
    """Runs one cavity to --steps steps (or until it diverges) per tau and remembers the answers."""

    def __init__(self, L, model, U0, args, stream):
        self.L, self.model, self.U0, self.args, self.stream = L, model, U0, args, stream
        self.seen = {}
        self.runs = 0
        self.steps_total = 0
        self.seconds = 0.0

    def stable(self, tau):
        key = round(tau, 9)
        if key in self.seen:
            return self.seen[key]
        t0 = time.perf_counter()
        ok, done = True, 0
        with cavity(self.L, tau, self.U0, self.model, self.args.precision, self.stream) as lat:
            while done < self.args.steps:
                n = min(self.args.chunk, self.args.steps - done)
                try:
                    lat.step(n)
                except F.FpclbmError as e:
                    if e.code != F.FPCLBM_ERR_DIVERGED:
                        raise
                    ok = False
                    done += n
                    break
                done += n
        self.seconds += time.perf_counter() - t0
        self.runs += 1
        self.steps_total += done
        self.seen[key] = ok
        return ok


def threshold(p: Prober, args):
    """Smallest tau on the grid 1/2 + k dtau that stays stable, with the next --verify grid points."""
    dt = args.dtau
    tau = lambda k: 0.5 + k * dt  # noqa: E731
    lo, hi = 1, int(round((args.tau_hi - 0.5) / dt))
    if p.stable(tau(lo)):
        return tau(lo), "stable at the smallest tau tried"
    while not p.stable(tau(hi)):
        lo, hi = hi, 2 * hi
        if tau(hi) > 1.0:
            return None, "no stable tau below 1"
    while hi - lo > 1:  # invariant: tau(lo) unstable, tau(hi) stable
        mid = (lo + hi) // 2
        if p.stable(tau(mid)):
            hi = mid
        else:
            lo = mid
    # confirm: the next `verify` grid points must be stable too, else continue above the failure
    cand, k = hi, 1
    while k <= args.verify:
        if p.stable(tau(cand + k)):
            k += 1
        else:
            cand = cand + k + 1
            while not p.stable(tau(cand)):
                cand += 1
            k = 1
    return tau(cand), "ok"


def run_stability(args):
    """Every (L, collision) threshold search runs in its own host thread on its own CUDA stream, so
    the small boxes' launches overlap instead of leaving the GPU idle between them."""
    import torch

    U0 = args.ma * CS
    jobs = [(L, model) for L in args.sizes for model in args.models]
    probers, answers, threads = {}, {}, []
    for job in jobs:
        stream = torch.cuda.Stream()
        p = Prober(job[0], job[1], U0, args, stream.cuda_stream)
        probers[job] = (p, stream)

        def work(job=job, p=p):
            try:
                answers[job] = threshold(p, args)
            except Exception as e:  # report, do not hang the other searches
                answers[job] = (None, "error: %s" % e)
            print(json.dumps({"L": job[0], "model": job[1], "tau_min": answers[job][0], "note": answers[job][1],
                              "runs": p.runs, "seconds": p.seconds}), file=sys.stderr, flush=True)

        th = threading.Thread(target=work)
        th.start()
        threads.append(th)
    for th in threads:
        th.join()
    results = []
    for job in jobs:
        L, model = job
        p, _ = probers[job]
        tau, note = answers[job]
        nu = (tau - 0.5) / 3.0 if tau else None
        results.append({"L": L, "model": model, "tau_min": tau, "Re_max": U0 * L / nu if tau else None,
                        "note": note, "runs": p.runs, "steps_run": p.steps_total, "seconds": p.seconds,
                        "largest_unstable_taus": sorted(t for t, ok in p.seen.items() if not ok)[-3:],
                        "smallest_stable_taus": sorted(t for t, ok in p.seen.items() if ok)[:3]})
    return {"study": "lid-driven cavity stability threshold", "Ma": args.ma, "U0": U0, "steps": args.steps,
            "dtau": args.dtau, "verify": args.verify, "precision": args.precision, "results": results}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    a = sub.add_parser("accuracy")
    a.add_argument("--re", type=float, nargs="+", default=[100.0, 400.0, 1000.0])
    a.add_argument("--levels", type=int, nargs="+", default=[75, 150])
    a.add_argument("--models", nargs="+", default=["fpc"], choices=sorted(MODELS))
    a.add_argument("--ma", type=float, default=0.1)
    a.add_argument("--tol", type=float, default=1e-4, help="steady when profiles change < tol U0 per L/U0")
    a.add_argument("--max-tc", type=int, default=150, help="maximum convective times L/U0")
    a.add_argument("--precision", default="fp32")
    s = sub.add_parser("stability")
    s.add_argument("--sizes", type=int, nargs="+", default=[48, 64, 80, 96])
    s.add_argument("--models", nargs="+", default=["fpc", "mcm"], choices=sorted(MODELS))
    s.add_argument("--ma", type=float, default=0.2)
    s.add_argument("--steps", type=int, default=500000)
    s.add_argument("--chunk", type=int, default=5000)
    s.add_argument("--dtau", type=float, default=5e-5)
    s.add_argument("--tau-hi", type=float, default=0.52)
    s.add_argument("--verify", type=int, default=10)
    s.add_argument("--precision", default="fp32")
    return ap.parse_args(argv)


def main(argv=None):
    args = parse(argv)
    t0 = time.perf_counter()
    res = run_accuracy(args) if args.cmd == "accuracy" else run_stability(args)
    res["wall_seconds"] = time.perf_counter() - t0
    print(json.dumps(res))


if __name__ == "__main__":
    main()
