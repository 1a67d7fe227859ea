"""Turbulent half-channel LES (Sec. 4): FPC-LBM with the Smagorinsky model and van Driest damping
on a half channel closed by a specular symmetry plane, driven by F_x = u*^2 / H.

Domain 2 pi H x H x pi H (x, y wall-normal, z), wall at y = -1/2, symmetry plane at y = H - 1/2,
Re* = u* H / nu.  Initial state: the lower half of a laminar channel of height 2H with bulk
velocity 16 u* plus seeded +-10 % perturbations and (--vortices A) large-scale streaks and
streamwise vortices of amplitude A u* (spanwise wavenumber 4, streamwise 2; the wall-normal
shapes vanish at the wall and respect the symmetry plane), which let the flow transition within
a few friction times instead of relaminarising.  After --spinup friction times T* = H / u*,
statistics over --collect T* (every --every steps; averages over x, z and time):
mean U(y), rms fluctuations, Reynolds shear stress -<u'v'>, all in wall units with the nominal u*.

The paper compares with DNS data that are not reproduced here; the mean profile is set beside the
textbook law of the wall instead: u+ = y+ in the viscous sublayer (y+ < 5) and
u+ = ln(y+) / 0.41 + 5.2 in the log layer (30 < y+ < 0.3 Re*), and the total shear stress is
checked against its exact linear profile u*^2 (1 - y/H) (momentum balance of the statistically
steady channel: viscous + resolved Reynolds + subgrid stress).

--full runs the full channel of the channel configuration instead: walls at y = -1/2 and
2H - 1/2, domain --domain nx ny nz (default 4H x 2H x 2H, i.e. 384 x 192 x 192 at H = 96), the
laminar profile with noise and streaks/vortices spanning the whole height; statistics fold the two
halves (u, w even and v odd about the centre plane) and the momentum-balance residual
max |nu dU/dy - <u'v'> - u*^2 (1 - y/H)| / u*^2 over the half height is reported.

Usage: python -m paper_2410_09739_gb300.channel_les_study [--H 64] [--re-tau 180] [--full] ...
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


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--H", type=int, default=64, help="half-channel height in cells")
    p.add_argument("--re-tau", type=float, default=180.0)
    p.add_argument("--u-star", type=float, default=0.006)
    p.add_argument("--cs", type=float, default=0.1, help="Smagorinsky constant")
    p.add_argument("--a-plus", type=float, default=26.0, help="van Driest constant")
    p.add_argument("--spinup", type=float, default=40.0, help="friction times before statistics")
    p.add_argument("--collect", type=float, default=20.0, help="friction times of statistics")
    p.add_argument("--every", type=int, default=200, help="steps between samples")
    p.add_argument("--precision", default="fp32")
    p.add_argument("--model", default="smagorinsky", choices=["smagorinsky", "none"])
    p.add_argument("--vortices", type=float, default=4.0, help="streak/vortex amplitude in units of u*")
    p.add_argument("--full", action="store_true", help="full channel with two walls (channel configuration)")
    p.add_argument("--domain", type=int, nargs=3, default=None, help="nx ny nz (full channel)")
    p.add_argument("--seed", type=int, default=7)
    return p.parse_args(argv)


def perturbation(nx, ny, nz, H, amp, full=False):
    """Large-scale streaks and streamwise vortices (spanwise wavenumber 4, streamwise 2).
    Half channel (wall at y = 0, symmetry plane at y = H): u' ~ sin(pi y / 2H) cos(k_z z),
    v' ~ sin(pi y / H) sin(k_z z) cos(k_x x), w' ~ cos(pi y / H) cos(k_z z) sin(k_x x) -- zero u',
    v' at the wall, zero v' and du'/dy at the symmetry plane.  full (walls at y = 0 and y = H):
    every component ~ sin(pi y / H), so v' crosses the centre plane and breaks the mirror symmetry
    of the laminar state."""
    x = 2 * math.pi * np.arange(nx) / nx
    z = 2 * math.pi * np.arange(nz) / nz
    y = (np.arange(ny) + 0.5) / H
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    if full:
        shape = np.sin(math.pi * Y)
        return (amp * shape * np.cos(4 * Z), 0.5 * amp * shape * np.sin(4 * Z) * np.cos(2 * X),
                0.5 * amp * shape * np.cos(4 * Z) * np.sin(2 * X))
    du = amp * np.sin(0.5 * math.pi * Y) * np.cos(4 * Z)
    dv = 0.5 * amp * np.sin(math.pi * Y) * np.sin(4 * Z) * np.cos(2 * X)
    dw = 0.5 * amp * np.cos(math.pi * Y) * (1 - np.exp(-8 * Y)) * np.cos(4 * Z) * np.sin(2 * X)
    return du, dv, dw


def run(args):
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    H = args.H
    if args.full:
        nx, ny, nz = args.domain if args.domain else (4 * H, 2 * H, 2 * H)
        assert ny == 2 * H, "full channel: ny = 2H"
    else:
        nx, ny, nz = int(round(2 * math.pi * H)), H, int(round(math.pi * H))
    us = args.u_star
    nu = us * H / args.re_tau
    tau = 3.0 * nu + 0.5
    Fx = us * us / H
    Tstar = H / us
    lat = F.Lattice(nx, ny, nz, args.precision, F.FPCLBM_BC_WALLS_Y if args.full else F.FPCLBM_BC_HALF_CHANNEL,
                    stream=stream)
    if args.model == "smagorinsky":
        lat.set_params(tau, 0.0, F.FPCLBM_DIFF_FP_SMAGORINSKY)
        lat.set_smagorinsky(args.cs, us, args.a_plus)
    else:
        lat.set_params(tau)
    lat.set_force(Fx, 0.0, 0.0)
    rho, ux, uy, uz = (np.ascontiguousarray(a[:, :H, :]) for a in W.channel_fields(nx, 2 * H, nz, us,
                                                                                      seed=args.seed))
    if args.full:  # the whole laminar channel, then perturbations spanning both halves
        rho, ux, uy, uz = W.channel_fields(nx, 2 * H, nz, us, seed=args.seed)
        if args.vortices > 0:
            du, dv, dw = perturbation(nx, 2 * H, nz, 2 * H, args.vortices * us, full=True)
            ux, uy, uz = ux + du, uy + dv, uz + dw
    elif args.vortices > 0:
        du, dv, dw = perturbation(nx, H, nz, H, args.vortices * us)
        ux, uy, uz = ux + du, uy + dv, uz + dw
    lat.init_fields(*(np.ascontiguousarray(a) for a in (rho, ux, uy, uz)))

    t0 = time.perf_counter()
    n_spin = int(round(args.spinup * Tstar))
    done = 0
    while done < n_spin:
        k = min(8192, n_spin - done)
        lat.step(k)
        done += k
    spin_s = time.perf_counter() - t0

    n = nx * ny * nz
    buf = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(4)]
    acc = {k: torch.zeros(ny, dtype=torch.float64, device="cuda") for k in ("u", "v", "w", "uu", "vv", "ww", "uv")}
    n_coll = int(round(args.collect * Tstar))
    samples = 0
    t0 = time.perf_counter()
    done = 0
    while done < n_coll:
        lat.step(args.every)
        done += args.every
        F.fpclbm_moments(lat.h, *buf, on_device=1)
        u, v, w = (b.view(nz, ny, nx) for b in buf[1:])
        acc["u"] += u.mean(dim=(0, 2))
        acc["v"] += v.mean(dim=(0, 2))
        acc["w"] += w.mean(dim=(0, 2))
        acc["uu"] += (u * u).mean(dim=(0, 2))
        acc["vv"] += (v * v).mean(dim=(0, 2))
        acc["ww"] += (w * w).mean(dim=(0, 2))
        acc["uv"] += (u * v).mean(dim=(0, 2))
        samples += 1
    torch.cuda.synchronize()
    coll_s = time.perf_counter() - t0
    m = {k: (a / samples).cpu().numpy() for k, a in acc.items()}
    lat.close()
    if args.full:  # fold the upper half onto the lower one
        for k in m:
            sgn = -1.0 if k in ("v", "uv") else 1.0
            m[k] = 0.5 * (m[k][:H] + sgn * m[k][::-1][:H])

    U, V, Wm = m["u"], m["v"], m["w"]
    urms = np.sqrt(np.maximum(m["uu"] - U * U, 0))
    vrms = np.sqrt(np.maximum(m["vv"] - V * V, 0))
    wrms = np.sqrt(np.maximum(m["ww"] - Wm * Wm, 0))
    uv = m["uv"] - U * V
    y = np.arange(H) + 0.5  # distance of the row centre from the wall
    yplus = y * us / nu
    uplus = U / us
    law = np.where(yplus < 5, yplus, np.where(yplus > 30, np.log(np.maximum(yplus, 1e-30)) / 0.41 + 5.2, np.nan))
    visc = (yplus < 5)
    logr = (yplus > 30) & (yplus < 0.3 * args.re_tau)
    # momentum balance: nu dU/dy - <u'v'> (+ subgrid) = u*^2 (1 - y/H); resolved part reported
    dUdy = np.gradient(U, y)
    resolved = nu * dUdy - uv
    exact = us * us * (1 - y / H)
    steps = n_spin + n_coll
    return {
        "study": ("full channel, FPC-LBM" if args.full else "half channel, FPC-LBM") +
                 (" + Smagorinsky/van Driest LES" if args.model == "smagorinsky" else ""),
        "config": {"domain": [nx, ny, nz], "H": H, "re_tau": args.re_tau, "u_star": us, "nu": nu, "tau": tau,
                   "Fx": Fx, "Cs": args.cs if args.model == "smagorinsky" else 0.0, "A_plus": args.a_plus,
                   "friction_time_steps": Tstar, "spinup_T": args.spinup, "collect_T": args.collect,
                   "samples": samples, "precision": args.precision, "model": args.model,
                   "vortices_over_u_star": args.vortices},
        "bulk_velocity_over_u_star": float(np.mean(U) / us),
        "centreline_u_plus": float(uplus[-1]),
        "viscous_sublayer_max_abs_dev_u_plus": float(np.nanmax(np.abs(uplus[visc] - law[visc]))) if visc.any() else None,
        "log_layer_max_abs_dev_u_plus": float(np.nanmax(np.abs(uplus[logr] - law[logr]))) if logr.any() else None,
        "log_layer_rows": int(logr.sum()),
        "resolved_stress_over_total_at_y_H_0p5": float(np.interp(0.5 * H, y, resolved / np.maximum(exact, 1e-30))),
        "momentum_balance_max_residual_over_u_star2": float(np.max(np.abs(resolved - exact)) / us**2),
        "y_plus": [round(float(v), 3) for v in yplus],
        "u_plus": [round(float(v), 4) for v in uplus],
        "urms_plus": [round(float(v), 4) for v in urms / us],
        "vrms_plus": [round(float(v), 4) for v in vrms / us],
        "wrms_plus": [round(float(v), 4) for v in wrms / us],
        "uv_plus": [round(float(v), 4) for v in -uv / us**2],
        "seconds": {"spinup": spin_s, "collect": coll_s},
        "mlups": n * steps / (spin_s + coll_s) / 1e6,
    }


def main(argv=None):
    print(json.dumps(run(parse(argv))))


if __name__ == "__main__":
    main()
