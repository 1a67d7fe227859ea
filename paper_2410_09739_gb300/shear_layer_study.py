"""Doubly periodic shear layers (Sec. 4, 2D numerical-performance study) with the D2Q9 FPC-LBM
and the MCM-LBM (FPCLBM_DIFF_EQUILIBRIUM) on the GPU.

Setup (Sec. 4): periodic L x L box, coordinates scaled by L, u_x = U tanh(4 (y - 1/4) / w) for
y <= 1/2 and U tanh(4 (3/4 - y) / w) above, u_y = delta sin(2 pi (x + 1/4)), w = delta = 0.05,
Re = U L / nu = 30000, Ma = U / cs, run to t = 1 (T = L / U steps).  Cases: Ma 0.05 ... 0.6 at
L = 64, 128, 256 with the bulk rate omega_3 = 1, and Ma 0.05, 0.2, 0.3 with omega_3 = 0.35
(large bulk viscosity); higher-order rates 1.

The paper judges the cases by eye from vorticity plots (one rolled-up vortex per layer, or
spurious secondary vortices).  This study reports numbers instead: whether the run stayed finite,
the number of vortex blobs of each sign (connected regions, periodic, where the vorticity averaged
onto 64 x 64 cells exceeds half of its peak magnitude: 1 and 1 for a clean roll-up of the two
layers, more when secondary vortices form), and the L2 distance of the vorticity field, sampled at t = 1 onto the 64 x 64
grid, from the finest FPC run of the same Mach number and bulk rate.

Usage: python -m paper_2410_09739_gb300.shear_layer_study [--sizes 64 128 256] [--precision fp64]
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

import workloads as W  # noqa: E402
from paper_2410_09739_gb300 import fpclbm as F  # noqa: E402

CS = 1.0 / math.sqrt(3.0)
MODELS = {"fpc": F.FPCLBM_DIFF_FP, "mcm": F.FPCLBM_DIFF_EQUILIBRIUM}


def vorticity(ux, uy, L, U):
    """dv/dx - du/dy by periodic central differences, in units of U / L."""
    dvdx = (np.roll(uy, -1, axis=1) - np.roll(uy, 1, axis=1)) / 2
    dudy = (np.roll(ux, -1, axis=0) - np.roll(ux, 1, axis=0)) / 2
    return (dvdx - dudy) * L / U


def blobs(mask):
    """Connected regions (4-neighbour, periodic in both directions) of a boolean field."""
    ny, nx = mask.shape
    lab = np.zeros(mask.shape, dtype=np.int64)
    n = 0
    for j0, i0 in zip(*np.nonzero(mask)):
        if lab[j0, i0]:
            continue
        n += 1
        lab[j0, i0] = n
        stack = [(j0, i0)]
        while stack:
            j, i = stack.pop()
            for dj, di in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                jj, ii = (j + dj) % ny, (i + di) % nx
                if mask[jj, ii] and not lab[jj, ii]:
                    lab[jj, ii] = n
                    stack.append((jj, ii))
    return n


def cores(om, frac=0.5):
    """Vortex blobs of each sign: connected regions where +om (-om) exceeds frac of the peak |om|."""
    thr = frac * np.max(np.abs(om))
    return [blobs(om > thr), blobs(-om > thr)]


def sample64(om, L):
    """Average the vorticity onto 64 x 64 cells (L a multiple of 64)."""
    r = L // 64
    return om.reshape(64, r, 64, r).mean(axis=(1, 3))


def run_case(L, ma, model, bulk, precision, re=30000.0):
    U = ma * CS
    nu = U * L / re
    tau = 3 * nu + 0.5
    T = int(round(L / U))
    t0 = time.perf_counter()
    status = "ok"
    with F.Lattice2D(L, L, precision) as lat:
        lat.set_params(tau, bulk, 0.0, MODELS[model])
        lat.init_fields(*W.shear_layers(L, U))
        try:
            lat.step(T)
            rho, ux, uy = lat.moments()
        except F.FpclbmError as e:
            if e.code != F.FPCLBM_ERR_DIVERGED:
                raise
            status = "diverged"
    secs = time.perf_counter() - t0
    res = {"L": L, "Ma": ma, "model": model, "omega_3": bulk, "tau": tau, "steps": T, "status": status,
           "seconds": secs}
    om = None
    if status == "ok":
        om = vorticity(ux, uy, L, U)
        if not np.all(np.isfinite(om)):
            res["status"] = "non-finite"
            return res, None
        pos, neg = cores(sample64(om, L) if L % 64 == 0 else om)
        res.update({"cores_pos": pos, "cores_neg": neg, "max_abs_vorticity": float(np.max(np.abs(om))),
                    "rho_min": float(rho.min()), "rho_max": float(rho.max())})
    return res, om


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", type=int, nargs="+", default=[64, 128, 256])
    ap.add_argument("--machs", type=float, nargs="+", default=[0.05, 0.2, 0.3, 0.4, 0.5, 0.6])
    ap.add_argument("--bulk-machs", type=float, nargs="+", default=[0.05, 0.2, 0.3])
    ap.add_argument("--precision", default="fp64")
    args = ap.parse_args(argv)
    t0 = time.perf_counter()
    cases = [(ma, 1.0) for ma in args.machs] + [(ma, 0.35) for ma in args.bulk_machs]
    results = []
    for ma, bulk in cases:
        fields = {}
        for L in args.sizes:
            for model in MODELS:
                res, om = run_case(L, ma, model, bulk, args.precision)
                if om is not None and L % 64 == 0:
                    fields[(L, model)] = sample64(om, L)
                results.append(res)
                print(json.dumps(res), file=sys.stderr, flush=True)
        ref = fields.get((max(args.sizes), "fpc"))
        if ref is not None:
            for r in results[-2 * len(args.sizes):]:
                f = fields.get((r["L"], r["model"]))
                if f is not None:
                    r["vorticity_l2_vs_finest_fpc"] = float(np.linalg.norm(f - ref) / np.linalg.norm(ref))
    print(json.dumps({"study": "doubly periodic shear layers, D2Q9 FPC vs MCM", "Re": 30000, "t": 1.0,
                      "precision": args.precision, "results": results,
                      "wall_seconds": time.perf_counter() - t0}))


if __name__ == "__main__":
    main()
