"""Learned-closure study: coarse-grid FPC-LBM with the learned shear-rate correction
against the plain coarse run and the box-filtered fine run of the same channel.

Steps (all simulation, filtering and training on the GPU through the C ABI):
  1. fine channel (walls in y, body force F = u*^2 / H, Re_tau = u* H / nu), spin-up;
  2. during a collection window: every `snap` friction times, filter the fine
     state onto r^3 blocks (fpclbm_closure_sample: features + eddy-viscosity
     labels) and accumulate the fine mean velocity profile U(y);
  3. train the closure network on the collected samples (fpclbm_closure_train);
  4. coarse runs (acoustic scaling: dx, dt x r, nu / r, F x r), started from the
     filtered fine velocity at the start of the window, over the same physical
     time: plain FPC-LBM, FPC-LBM + learned closure, and FPC-LBM + the paper's
     Smagorinsky/van Driest subgrid model (Sec. 4) as the non-learned baseline,
     accumulating U(y);
  5. L2-relative profile error of each coarse run against the filtered fine
     profile, and the wall-clock speed-up of the coarse run over the fine run
     for equal physical time on the same GPU.

With --windows K the fine run continues through K successive collection windows after one
spin-up, each with its own training and coarse runs: K independent estimates of the errors and
their spread from one spin-up.

With --flow tgv the same pipeline runs on decaying turbulence instead: the Taylor-Green vortex in a
periodic box, fine n^3 against (n/r)^3, comparing the coarse runs' kinetic energy with the filtered
fine kinetic energy over time (decay() below).

Usage: python -m paper_2410_09739_gb300.closure_study [--fine 384 192 192] [--r 4] [--windows 2] ...
       python -m paper_2410_09739_gb300.closure_study --flow tgv --fine 256 256 256 --r 2
Prints one JSON object (progress on stderr).
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
    p.add_argument("--fine", type=int, nargs=3, default=(384, 192, 192), help="fine nx ny nz (ny = 2H)")
    p.add_argument("--r", type=int, default=4, help="coarsening factor")
    p.add_argument("--re-tau", type=float, default=395.0)
    p.add_argument("--u-star", type=float, default=0.005)
    p.add_argument("--spinup", type=float, default=20.0, help="fine spin-up in friction times H/u*")
    p.add_argument("--collect", type=float, default=10.0, help="collection window in friction times")
    p.add_argument("--snap", type=float, default=0.5, help="friction times between training snapshots")
    p.add_argument("--epochs", type=int, default=30)
    p.add_argument("--batch", type=int, default=1024)
    p.add_argument("--lr", type=float, default=2e-3)
    p.add_argument("--precision", default="bf16")
    p.add_argument("--seed", type=int, default=7)
    p.add_argument("--cs", type=float, default=0.1, help="Smagorinsky constant of the non-learned baseline")
    p.add_argument("--out", default=None, help="also write the JSON result to this file (after every window)")
    p.add_argument("--flow", default="channel", choices=["channel", "tgv"],
                   help="channel (walls, body force, mean profile) or tgv (decaying Taylor-Green vortex in a "
                        "periodic box, kinetic-energy history)")
    p.add_argument("--re", type=float, default=1600.0, help="tgv: Reynolds number u0 L / nu, L = n / (2 pi)")
    p.add_argument("--t-end", type=float, default=15.0, help="tgv: convective times L / u0")
    p.add_argument("--dt", type=float, default=0.5, help="tgv: convective times between snapshots")
    p.add_argument("--windows", type=int, default=1,
                   help="successive collection windows of the same fine run, each with its own training and "
                        "coarse runs (run-to-run spread)")
    p.add_argument("--vortices", type=float, default=0.0,
                   help="amplitude (units of u*) of large-scale streaks and streamwise vortices added to the "
                        "fine run's initial state to trigger transition (0: laminar profile and noise only)")
    return p.parse_args(argv)


class Profile:
    """Running mean of U(y) = <u_x> over x, z and time (device tensors, host result)."""

    def __init__(self, torch, shape):
        self.torch = torch
        self.shape = shape
        self.sum = None
        self.n = 0
        n = shape[0] * shape[1] * shape[2]
        self.buf = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(4)]

    def add(self, lat):
        F.fpclbm_moments(lat.h, *self.buf, on_device=1)
        ux = self.buf[1].view(*self.shape)  # [nz, ny, nx]
        p = ux.mean(dim=(0, 2))
        self.sum = p if self.sum is None else self.sum + p
        self.n += 1

    def mean(self):
        return (self.sum / self.n).cpu().numpy()


def log(msg):
    print("[closure_study %7.1f s] %s" % (time.perf_counter() - _T0, msg), file=sys.stderr, flush=True)


_T0 = time.perf_counter()


def window(fine, args, geo, seed):
    """One collection window of the fine run (continuing it), training, and the coarse runs over the
    same physical time.  Returns the window's record."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    (nxf, nyf, nzf), (nxc, nyc, nzc), r = geo["fine"], geo["coarse"], geo["r"]
    tau_c, Fc, Tf, Tc, us = geo["tau_c"], geo["F_c"], geo["T_f"], geo["T_c"], geo["u_star"]
    out = {"seed": seed}
    # collection window: every `snap` friction times filter the fine state onto r^3 blocks (features,
    # labels) and accumulate the fine mean profile
    nc = nxc * nyc * nzc
    n_snap = max(1, int(round(args.collect / args.snap)))
    X = torch.empty((n_snap * nc, 9), dtype=torch.float32, device="cuda")
    T = torch.empty(n_snap * nc, dtype=torch.float32, device="cuda")
    snap_steps = int(round(args.snap * Tf))
    prof_f = Profile(torch, (nzf, nyf, nxf))
    X0 = None
    fine_steps, fine_s = 0, 0.0
    for s in range(n_snap):
        F.fpclbm_closure_sample(fine.h, r, tau_c, X[s * nc:(s + 1) * nc], T[s * nc:(s + 1) * nc], on_device=1)
        if s == 0:
            X0 = X[:nc].clone()
        prof_f.add(fine)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fine.step(snap_steps)
        fine_s += time.perf_counter() - t0
        fine_steps += snap_steps
    prof_f.add(fine)
    U_fine = prof_f.mean().reshape(nyc, r).mean(axis=1)  # filtered onto coarse rows
    log("window %d: %d fine steps collected in %.1f s" % (seed, fine_steps, fine_s))

    # training on the window's samples
    t0 = time.perf_counter()
    w, losses = F.fpclbm_closure_train(X, T, n_snap * nc, args.epochs, args.batch, args.lr, seed=seed,
                                       stream=stream)
    train_s = time.perf_counter() - t0
    labels = T.cpu().numpy()
    out["training"] = {"samples": n_snap * nc, "epochs": args.epochs, "loss_first": float(losses[0]),
                       "loss_last": float(losses[-1]), "seconds": train_s,
                       "label_mean": float(labels.mean()), "label_min": float(labels.min())}
    del X, T

    # coarse runs from the filtered velocity at the start of the window
    u0 = X0[:, 6:9].double().cpu().numpy()
    fields = (np.ones(nc), np.ascontiguousarray(u0[:, 0]), np.ascontiguousarray(u0[:, 1]),
              np.ascontiguousarray(u0[:, 2]))
    coarse_res = {}
    for name in ("plain", "learned", "smagorinsky"):
        lat = F.Lattice(nxc, nyc, nzc, args.precision, F.FPCLBM_BC_WALLS_Y, stream=stream)
        if name == "learned":
            lat.set_closure(w)
            lat.set_params(tau_c, 0.0, F.FPCLBM_DIFF_FP_LEARNED)
        elif name == "smagorinsky":  # the paper's own subgrid model (Sec. 4) as the non-learned baseline
            lat.set_params(tau_c, 0.0, F.FPCLBM_DIFF_FP_SMAGORINSKY)
            lat.set_smagorinsky(args.cs, us, 26.0)  # acoustic scaling: u* is the same in coarse lattice units
        else:
            lat.set_params(tau_c)
        lat.set_force(Fc, 0.0, 0.0)
        lat.init_fields(*fields)
        prof = Profile(torch, (nzc, nyc, nxc))
        per = max(1, int(round(args.snap * Tc)))
        status, secs, steps = "ok", 0.0, 0
        try:
            for s in range(n_snap):
                prof.add(lat)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                lat.step(per)
                secs += time.perf_counter() - t0
                steps += per
            prof.add(lat)
            U = prof.mean()
            err = float(np.linalg.norm(U - U_fine) / np.linalg.norm(U_fine))
        except F.FpclbmError as e:
            status, U, err = "diverged after %d steps (%s)" % (steps, e), None, None
        coarse_res[name] = {"status": status, "profile_l2_rel_error": err, "steps": steps, "seconds": secs,
                            "U": None if U is None else [float(v) for v in U]}
        lat.close()
    out["U_fine_filtered"] = [float(v) for v in U_fine]
    out["coarse"] = coarse_res
    # speed-up for equal physical time (per friction time)
    fine_per_T = fine_s / (fine_steps / Tf)
    for name, res in coarse_res.items():
        if res["steps"]:
            res["speedup_vs_fine"] = fine_per_T / (res["seconds"] / (res["steps"] / Tc))
    out["fine"] = {"collect_seconds": fine_s, "collect_steps": fine_steps, "seconds_per_friction_time": fine_per_T}
    log("window %d: errors %s" % (seed, {k: v["profile_l2_rel_error"] for k, v in coarse_res.items()}))
    return out


def run(args):
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    nxf, nyf, nzf = args.fine
    r = args.r
    Hf = nyf / 2.0
    us = args.u_star
    nu_f = us * Hf / args.re_tau
    tau_f = 3.0 * nu_f + 0.5
    Ff = us * us / Hf
    Tf = Hf / us  # fine steps per friction time
    nxc, nyc, nzc = nxf // r, nyf // r, nzf // r
    nu_c = nu_f / r
    tau_c = 3.0 * nu_c + 0.5
    Fc = Ff * r
    Tc = Tf / r
    geo = {"fine": (nxf, nyf, nzf), "coarse": (nxc, nyc, nzc), "r": r, "tau_c": tau_c, "F_c": Fc, "T_f": Tf,
           "T_c": Tc, "u_star": us}
    out = {"config": {"fine": [nxf, nyf, nzf], "coarse": [nxc, nyc, nzc], "r": r, "re_tau": args.re_tau,
                      "u_star": us, "tau_fine": tau_f, "tau_coarse": tau_c, "F_fine": Ff, "F_coarse": Fc,
                      "friction_time_fine_steps": Tf, "precision": args.precision,
                      "spinup_T": args.spinup, "collect_T": args.collect, "snap_T": args.snap,
                      "windows": args.windows, "vortices_over_u_star": args.vortices, "seed": args.seed,
                      "epochs": args.epochs, "batch": args.batch, "lr": args.lr, "cs": args.cs}}

    # fine spin-up
    fine = F.Lattice(nxf, nyf, nzf, args.precision, F.FPCLBM_BC_WALLS_Y, stream=stream)
    fine.set_params(tau_f)
    fine.set_force(Ff, 0.0, 0.0)
    rho0, ux0, uy0, uz0 = W.channel_fields(nxf, nyf, nzf, us, seed=args.seed)
    if args.vortices > 0:
        from paper_2410_09739_gb300.channel_les_study import perturbation
        du, dv, dw = perturbation(nxf, nyf, nzf, nyf, args.vortices * us, full=True)
        ux0, uy0, uz0 = ux0 + du, uy0 + dv, uz0 + dw
    fine.init_fields(rho0, ux0, uy0, uz0)
    del rho0, ux0, uy0, uz0
    n_spin = int(round(args.spinup * Tf))
    t0 = time.perf_counter()
    done = 0
    while done < n_spin:
        k = min(4096, n_spin - done)
        fine.step(k)
        done += k
        if done % (8 * 4096) == 0 or done == n_spin:
            log("spin-up %d / %d fine steps" % (done, n_spin))
    out["spinup_seconds"] = time.perf_counter() - t0

    # successive windows of the same fine run: one training and one set of coarse runs each
    wins = []
    for k in range(args.windows):
        wins.append(window(fine, args, geo, args.seed + k))
        if args.out:  # partial result after every window
            with open(args.out, "w") as fh:
                json.dump(dict(out, windows=wins, partial=k + 1 < args.windows), fh)
    fine.close()
    out["windows"] = wins
    # the first window under the keys of a single-window study
    out["U_fine_filtered"], out["coarse"], out["training"] = wins[0]["U_fine_filtered"], wins[0]["coarse"], \
        wins[0]["training"]
    out["fine"] = wins[0]["fine"]
    summ = {}
    for name in ("plain", "learned", "smagorinsky"):
        errs = [w["coarse"][name]["profile_l2_rel_error"] for w in wins]
        errs = [e for e in errs if e is not None]
        sp = [w["coarse"][name].get("speedup_vs_fine") for w in wins]
        sp = [v for v in sp if v]
        summ[name] = {"errors": errs, "mean_error": float(np.mean(errs)) if errs else None,
                      "spread": float(np.max(errs) - np.min(errs)) if errs else None,
                      "mean_speedup_vs_fine": float(np.mean(sp)) if sp else None}
    out["summary"] = summ
    return out


def decay(args):
    """Decaying turbulence: the Taylor-Green vortex at Reynolds number args.re in a periodic box,
    fine n^3 and coarse (n/r)^3 (acoustic scaling: the same Re on both grids).  The fine run is
    box-filtered every args.dt convective times (features, labels, filtered kinetic energy), the
    network is trained on all snapshots, and coarse runs from the filtered initial field (plain,
    learned, Smagorinsky without wall damping) record their kinetic energy at the same times.
    Error of a coarse run: RMS over the snapshots of KE_coarse / KE_filtered - 1."""
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    nf, r, u0 = args.fine[0], args.r, 0.05
    n = nf // r
    nu_f = W.tgv_viscosity(nf, u0, args.re)
    tau_f, tau_c = 3.0 * nu_f + 0.5, 3.0 * nu_f / r + 0.5
    Tc = (n / (2.0 * math.pi)) / u0  # coarse steps per convective time
    per_c = max(1, int(round(args.dt * Tc)))
    n_snap = int(round(args.t_end / args.dt)) + 1
    nc = n ** 3
    out = {"config": {"flow": "tgv", "fine": nf, "coarse": n, "r": r, "re": args.re, "u0": u0, "tau_fine": tau_f,
                      "tau_coarse": tau_c, "t_end": args.t_end, "dt": args.dt, "coarse_steps_per_snapshot": per_c,
                      "precision": args.precision, "epochs": args.epochs, "batch": args.batch, "lr": args.lr,
                      "seed": args.seed, "cs": args.cs}}
    fine = F.Lattice(nf, nf, nf, args.precision, stream=stream)
    fine.set_params(tau_f)
    fine.init_fields(*W.tgv(nf, u0))
    X = torch.empty((n_snap * nc, 9), dtype=torch.float32, device="cuda")
    T = torch.empty(n_snap * nc, dtype=torch.float32, device="cuda")
    ke_f = []
    t0 = time.perf_counter()
    for k in range(n_snap):
        F.fpclbm_closure_sample(fine.h, r, tau_c, X[k * nc:(k + 1) * nc], T[k * nc:(k + 1) * nc], on_device=1)
        u = X[k * nc:(k + 1) * nc, 6:9].double()
        ke_f.append(0.5 * float((u * u).sum(dim=1).mean()))
        if k < n_snap - 1:
            fine.step(r * per_c)
    fine.close()
    fine_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    w, losses = F.fpclbm_closure_train(X, T, n_snap * nc, args.epochs, args.batch, args.lr, seed=args.seed,
                                       stream=stream)
    labels = T.cpu().numpy()
    out["training"] = {"samples": n_snap * nc, "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
                       "seconds": time.perf_counter() - t0, "label_mean": float(labels.mean()),
                       "label_min": float(labels.min())}
    u0c = X[:nc, 6:9].double().cpu().numpy()
    del X, T
    fields = (np.ones(nc), np.ascontiguousarray(u0c[:, 0]), np.ascontiguousarray(u0c[:, 1]),
              np.ascontiguousarray(u0c[:, 2]))
    buf = [torch.empty(nc, dtype=torch.float64, device="cuda") for _ in range(4)]
    kef = np.array(ke_f)
    runs = {}
    for name in ("plain", "learned", "smagorinsky"):
        lat = F.Lattice(n, n, n, args.precision, stream=stream)
        if name == "learned":
            lat.set_closure(w)
            lat.set_params(tau_c, 0.0, F.FPCLBM_DIFF_FP_LEARNED)
        elif name == "smagorinsky":  # no walls: no van Driest damping
            lat.set_params(tau_c, 0.0, F.FPCLBM_DIFF_FP_SMAGORINSKY)
            lat.set_smagorinsky(args.cs, 0.0, 0.0)
        else:
            lat.set_params(tau_c)
        lat.init_fields(*fields)
        ke, status, secs = [], "ok", 0.0
        try:
            for k in range(n_snap):
                F.fpclbm_moments(lat.h, *buf, on_device=1)
                ke.append(0.5 * float((buf[1] ** 2 + buf[2] ** 2 + buf[3] ** 2).mean()))
                if k < n_snap - 1:
                    torch.cuda.synchronize()
                    t1 = time.perf_counter()
                    lat.step(per_c)
                    secs += time.perf_counter() - t1
        except F.FpclbmError as e:
            status = "diverged at snapshot %d (%s)" % (len(ke), e)
        lat.close()
        kc = np.array(ke)
        err = float(np.sqrt(np.mean((kc / kef[:len(kc)] - 1.0) ** 2))) if status == "ok" else None
        runs[name] = {"status": status, "ke_rel_rms_error": err, "seconds": secs,
                      "ke_over_ke0": [float(v / ke_f[0]) for v in ke]}
    out["ke_fine_over_ke0"] = [float(v / ke_f[0]) for v in ke_f]
    out["coarse"] = runs
    out["fine_seconds"] = fine_s
    out["errors"] = {k: v["ke_rel_rms_error"] for k, v in runs.items()}
    return out


def main(argv=None):
    args = parse(argv)
    res = decay(args) if args.flow == "tgv" else run(args)
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
