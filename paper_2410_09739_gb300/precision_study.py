"""Storage-precision errors of the GPU path against its own FP64 run, per workload.

Each workload runs the same number of steps from the same initial fields with FP64, FP32, FP16 and
BF16 population storage (the arithmetic is FP64 for the first and FP32 for the others).  Reported
per storage type: max and RMS over cells of |u - u_fp64| / U (all three components; U is the
workload's velocity scale) and the relative mass difference.  The FP64 path itself is at oracle
parity (per-step relative difference below 1e-12), so these are errors of the reduced precision.

Workloads (the performance configurations of the paper's test cases, Sec. 4):
  tgv      Taylor-Green vortex, Re = 1600, 256^3 periodic, U = u0 = 0.05
  tgv512   the same on 512^3 (viscosity from Re at that size)
  channel  walls in y, body force, Re_tau = 180, 384 x 192 x 192, U = bulk velocity 16 u*
  cavity   lid-driven cubic cavity, Re = 1000, Ma = 0.1, 150^3, U = lid velocity
  shear2d  D2Q9 doubly periodic shear layers, Re = 30000, Ma = 0.2, 4096^2, U = layer velocity

Usage: python -m paper_2410_09739_gb300.precision_study [--steps 1000] [--workloads tgv tgv512 channel ...]
Prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2410_09739_gb300 import fpclbm as F  # noqa: E402
import workloads as W  # noqa: E402

CS = 1.0 / math.sqrt(3.0)
PRECISIONS = ("fp64", "fp32", "fp16", "bf16")


def workload(name):
    """(make(prec) -> lattice with fields set, velocity scale U, description)."""
    if name in ("tgv", "tgv512"):
        n, u0 = (256 if name == "tgv" else 512), 0.05
        tau = 3 * W.tgv_viscosity(n, u0, 1600.0) + 0.5
        flds = W.tgv(n, u0)

        def make(prec):
            lat = F.Lattice(n, n, n, prec)
            lat.set_params(tau)
            lat.init_fields(*flds)
            return lat
        return make, u0, "TGV Re=1600 %d^3, u0=0.05, tau=%.6f" % (n, tau)
    if name == "channel":
        nx, ny, nz, us = 384, 192, 192, 0.005
        H = ny / 2
        tau = 3 * (us * H / 180.0) + 0.5
        flds = W.channel_fields(nx, ny, nz, us, seed=7)

        def make(prec):
            lat = F.Lattice(nx, ny, nz, prec, F.FPCLBM_BC_WALLS_Y)
            lat.set_params(tau)
            lat.set_force(us * us / H, 0.0, 0.0)
            lat.init_fields(*flds)
            return lat
        return make, 16 * us, "channel Re_tau=180 384x192x192, tau=%.6f, bulk 16u*" % tau
    if name == "cavity":
        n, U = 150, 0.1 * CS
        tau = 0.5 + 3 * U * n / 1000.0
        one = np.ones((n, n, n))

        def make(prec):
            lat = F.Lattice(n, n, n, prec, F.FPCLBM_BC_BOX)
            lat.set_params(tau)
            lat.set_wall_velocity(U)
            lat.init_fields(one, 0 * one, 0 * one, 0 * one)
            return lat
        return make, U, "lid-driven cavity 150^3, Re=1000, Ma=0.1, tau=%.6f" % tau
    if name == "shear2d":
        n, U = 4096, 0.2 * CS
        tau = 0.5 + 3 * U * n / 30000.0
        flds = W.shear_layers(n, U)

        def make(prec):
            lat = F.Lattice2D(n, n, prec)
            lat.set_params(tau)
            lat.init_fields(*flds)
            return lat
        return make, U, "D2Q9 shear layers 4096^2, Re=30000, Ma=0.2, tau=%.6f" % tau
    raise ValueError("unknown workload %r" % name)


def device_moments(lat, torch):
    """rho, u of every cell as device tensors (fpclbm_moments / fpclbm2d_moments on the device)."""
    nf = 3 if isinstance(lat, F.Lattice2D) else 4
    outs = [torch.empty(lat.ncells, dtype=torch.float64, device="cuda") for _ in range(nf)]
    (F.fpclbm2d_moments if nf == 3 else F.fpclbm_moments)(lat.h, *outs, on_device=1)
    return outs


def run(name, steps):
    import torch
    make, U, desc = workload(name)
    ref = None
    out = {"workload": name, "description": desc, "steps": steps, "U": U}
    for prec in PRECISIONS:
        t0 = time.perf_counter()
        with make(prec) as lat:
            lat.step(steps)
            m = device_moments(lat, torch)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        rho, vel = m[0], m[1:]
        if ref is None:  # the FP64 run, kept on the device
            ref = (float(torch.sum(rho)), vel)
            out["fp64_seconds"] = secs
            continue
        d = [v - r for v, r in zip(vel, ref[1])]
        finite = all(bool(torch.isfinite(x).all()) for x in d)
        mx = max(float(torch.max(torch.abs(x))) for x in d) / U if finite else float("inf")
        rms = math.sqrt(sum(float(torch.mean(x * x)) for x in d) / len(d)) / U if finite else float("inf")
        out[prec] = {"max_du_over_U": mx, "rms_du_over_U": rms,
                     "mass_rel": float(abs(float(torch.sum(rho)) - ref[0]) / ref[0]), "seconds": secs}
        print("%s %s: max %.3e rms %.3e" % (name, prec, mx, rms), file=sys.stderr, flush=True)
        del rho, vel, d, m
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--workloads", nargs="+", default=["tgv", "tgv512", "channel", "cavity", "shear2d"])
    args = ap.parse_args(argv)
    t0 = time.perf_counter()
    res = [run(w, args.steps) for w in args.workloads]
    print(json.dumps({"study": "storage precision vs FP64", "results": res, "wall_seconds": time.perf_counter() - t0}))


if __name__ == "__main__":
    main()
