"""Benchmark of the D3Q27 FPC-LBM fused stream-and-collide step on GB300.

Workload (the metric's configuration): 3D Taylor-Green vortex at Re = 1600 on
a periodic 256^3 lattice, u0 = 0.05, viscosity from Re, FP32 arithmetic with
FP32 deviation storage (--precision selects fp16/bf16 storage or fp64).  One
bench "step" = --inner LBM time steps (one fpclbm_step call).

Reported:
  value     MLUPS = cells * LBM steps / device time / 1e6, inputs resident in
            HBM (1.8 GB of populations >> 129 MB L2, so no L2 flush needed)
  e2e       same metric through the C ABI with host buffers: every bench step
            copies rho, u from pinned host memory (init_fields), runs --inner
            steps and reads rho, u back (moments)
  roofline  step kernel: algorithmic bytes 54 * b per cell update over the
            measured average launch duration, against MEASURED_PEAKS.json
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the workload

--impl reference times the FP64 CPU oracle (the only reference there is) on a
bounded sample of the same workload and prints the same JSON line.
Multi-GPU (torchrun): every rank runs its own box (replicas, weak scaling);
there is no data exchange.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "D3Q27 FPC-LBM MLUPS & % HBM roofline; closure speedup at stated error"
BYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}
# the GB300's nominal HBM3e bandwidth (~8 TB/s), beside the measured copy bandwidth of MEASURED_PEAKS.json
NOMINAL_HBM_GBS = 8000.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--size", type=int, default=256, help="TGV box side")
    p.add_argument("--precision", default="fp32", choices=list(BYTES))
    p.add_argument("--inner", type=int, default=64, help="LBM steps per bench step")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--drift", type=float, default=0.0,
                   help="omega_FP of the headline line: rates k * drift for orders k >= 3 (0: unit rates)")
    p.add_argument("--no-variants", action="store_true",
                   help="skip the secondary entries (fp16/bf16 storage, general rates)")
    p.add_argument("--workload", default="tgv", choices=["tgv", "channel", "cavity", "ensemble", "shear2d", "closure"])
    return p.parse_args()


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    # the reference arm (CPU oracle) runs on rank 0 alone; other ranks exit without work
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


STEP_KERNEL_SOURCES = ("common.cuh", "collide.cuh", "pair.cuh", "closure.cuh", "cell.cuh", "step_kernel.cuh", "stage.cuh",
                       "step_fp32.cu",
                       "step_fp32_odd.cu", "step_fp16.cu", "step_fp16_odd.cu", "step_bf16.cu", "step_bf16_odd.cu",
                       "step_fp64.cu", "step_kernels.cu", "internal.h")


def kernel_source_hash():
    """Hash of the sources that define the single-box step kernel."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2410_09739_gb300", "csrc")
    for name in STEP_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_entry(precision):
    """The committed ncu record of the step kernel for this storage type, if it was taken on the
    current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    return rec.get("entries", {}).get(precision)


def ncu_traffic(precision, n):
    """dram bytes per launch of the step kernel (n^3 TGV) from the committed ncu record, or None."""
    ent = ncu_entry(precision)
    return float(ent["bytes_per_cell"]) * n ** 3 if ent and "bytes_per_cell" in ent else None


# FP32 lane operations per second of the FMA pipes: 152 SMs x 128 lanes x 2.07 GHz (maximum SM clock)
ALU_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12


def alu_roofline(precision, mlups):
    """The ALU roofline of a 16-bit storage entry: fp32 lane operations per cell (ncu instruction
    classes of the same kernel source; a packed operation counts two) against the FMA pipes' peak."""
    ent = ncu_entry(precision)
    if not ent or "fp32_lane_ops_per_cell" not in ent:
        return None
    ops = float(ent["fp32_lane_ops_per_cell"])
    ach = mlups * 1e6 * ops / 1e12
    return {"bound": "alu", "lane_ops_per_cell": ops, "achieved": ach, "peak": ALU_PEAK_TOPS,
            "unit": "T lane-op/s", "frac": ach / ALU_PEAK_TOPS,
            "peak_source": "152 SMs x 128 FP32 lanes x 2.07 GHz"}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for ln in fh:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def cpu_oracle_sample(n, tau, u0, target_s=12.0, target_1_s=6.0):
    """Time the FP64 oracle on a bounded sample of the workload: z-slabs of the TGV fields, one
    plane per host thread (the oracle's parallel loop runs over z-planes), stepped for ~target_s
    seconds on all threads, then one plane for ~target_1_s seconds on one thread (the per-core
    figure).  The slab is periodic in z: the same arithmetic per cell as the full box."""
    import oracle as O
    rho, ux, uy, uz = W.tgv(n, u0)
    om = O.rates(tau)
    cores = O.threads()

    def timed(planes, budget):
        sl = [np.ascontiguousarray(a[:planes]) for a in (rho, ux, uy, uz)]
        f = O.init_equilibrium(*sl)
        done, t0 = 0, time.perf_counter()
        while True:
            f = O.step(f, omega=om)
            done += 1
            el = time.perf_counter() - t0
            if el >= budget:
                return sl[0].size * done / el / 1e6, done, el

    planes = max(1, min(cores, n))
    v, done, el = timed(planes, target_s)
    O.set_threads(1)
    try:
        v1, done1, el1 = timed(1, target_1_s)
    finally:
        O.set_threads(cores)
    return {"value": v, "unit": "MLUPS", "cores": min(cores, planes), "kind": "oracle",
            "single_thread_value": v1, "cpu": cpu_model(),
            "sample": "%d x %d x %d slab of the %d^3 TGV fields, %d FP64 oracle steps in %.1f s on %d threads; "
                      "%d x %d x 1, %d steps in %.1f s on 1 thread" % (n, n, planes, n, done, el, min(cores, planes),
                                                                    n, n, done1, el1)}


def cpu_oracle_sample_2d(L, tau, U, target_s=15.0):
    """The D2Q9 FP64 oracle on a 256 x 256 sample of the shear-layer workload (~target_s seconds)."""
    from oracle import oracle2d as O2
    import oracle as O
    n = min(L, 256)
    f = O2.init_equilibrium(*W.shear_layers(n, U))
    om = O2.rates(tau)
    done, t0 = 0, time.perf_counter()
    while True:
        f = O2.step(f, omega=om)
        done += 1
        el = time.perf_counter() - t0
        if el >= target_s:
            break
    return {"value": n * n * done / el / 1e6, "unit": "MLUPS", "cores": O.threads(), "kind": "oracle",
            "sample": "%d x %d shear layers (D2Q9), %d FP64 oracle steps, %.1f s" % (n, n, done, el)}


def tgv_workload(n, tau):
    """The TGV workload's name in the config of both arms."""
    return "TGV Re=1600 %d^3 periodic, u0=0.05, tau=%.6f" % (n, tau)


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload != "tgv":
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm (the FP64 CPU oracle) is timed "
                          "on the TGV workload only; run it without --workload"}), flush=True)
        return
    n, u0 = args.size, 0.05
    tau = 3 * W.tgv_viscosity(n, u0, 1600.0) + 0.5
    import oracle as O
    rho, ux, uy, uz = W.tgv(n, u0)
    planes = max(1, min(O.threads(), n))  # one z-plane per host thread (the oracle's parallel loop)
    sl = [np.ascontiguousarray(a[:planes]) for a in (rho, ux, uy, uz)]
    f = O.init_equilibrium(*sl)
    om = O.rates(tau)
    cells = sl[0].size
    for _ in range(args.warmup):
        f = O.step(f, omega=om)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = O.step(f, omega=om)
    el = time.perf_counter() - t0
    v = cells * args.steps / el / 1e6
    sample = "%d x %d x %d slab of the %d^3 TGV fields (periodic in z), one FP64 oracle step per bench step, %s" % (
        n, n, planes, n, cpu_model())
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": tgv_workload(n, tau), "precision": "fp64", "sample": sample,
                   "l2": "inputs larger than L2 not applicable (CPU)"},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": planes, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def kernel_name(F, workload, launch):
    """The step kernel that ran, from the launch the autotuner chose (fpclbm_get_launch)."""
    if workload == "shear2d":
        return "fpc::k_step2d (D2Q9, AA even/odd)"
    ens = workload == "ensemble"
    v = launch["variant"]
    if v == 3:
        return ("fpc::k_step_stage (AA even/odd; whole slot rows through %d shared-memory stages by bulk "
                "asynchronous copies, two cells per thread, blocks of %d; collision mode %d: %s)"
                % (launch["minb"], launch["block"], launch["mode"], F.LAUNCH_MODES.get(launch["mode"], "?")))
    if v == 2:
        base = "fpc::k_ens_pair" if ens else "fpc::k_step_pair"
        shape = "two cells per thread, blocks of 128"
    elif v == 1:
        base, shape = "fpc::k_step_pipe", "cp.async-pipelined, blocks of %d" % launch["block"]
    else:
        base = "fpc::k_ens_step" if ens else "fpc::k_step"
        shape = "one cell per thread, blocks of %d" % launch["block"]
    return "%s (AA even/odd; %s, register-cap class %d; collision mode %d: %s)" % (
        base, shape, launch["minb"], launch["mode"], F.LAUNCH_MODES.get(launch["mode"], "?"))


def time_ours(lat, F, torch, args, n, steps, warmup, inner):
    """Device-resident timing: CUDA events on the library's stream around `steps` fpclbm_step calls."""
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        lat.step(inner)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        lat.step(inner)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def closure_weights(seed):
    """Seeded random closure weights (4865, layer shapes 9-64-64-1, scaled by 1/sqrt(fan-in)) as
    bf16 bit patterns (round to nearest even)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, 1 / 3.0, 64 * 9), np.zeros(64), rng.normal(0, 1 / 8.0, 64 * 64), np.zeros(64),
             rng.normal(0, 1 / 8.0 * 0.01, 64), np.zeros(1)]
    a = np.concatenate(parts).astype(np.float32).view(np.uint32).astype(np.uint64)
    return ((a + ((a >> 16) & 1) + 0x7FFF) >> 16).astype(np.uint16)


def setup(args, F, prec, stream, drift=0.0, learned=True, workload=None):
    """Build the lattice of a workload (default: the chosen one); returns (lat, flat fields,
    cells, config dict).  drift > 0 selects the rates k * drift of orders k >= 3 (TGV only);
    learned=False runs the closure workload's coarse channel without the closure."""
    workload = workload or args.workload
    if workload == "tgv":
        n, u0 = args.size, 0.05
        tau = 3 * W.tgv_viscosity(n, u0, 1600.0) + 0.5
        lat = F.Lattice(n, n, n, prec, F.FPCLBM_BC_PERIODIC, stream=stream)
        lat.set_params(tau, drift)
        flds = W.tgv(n, u0)
        cfg = {"workload": tgv_workload(n, tau)}
        if drift > 0:
            cfg["drift"] = drift
    elif workload == "channel":
        nx, ny, nz, u_star = 384, 192, 192, 0.005
        H = ny / 2
        tau = 3 * (u_star * H / 180.0) + 0.5
        lat = F.Lattice(nx, ny, nz, prec, F.FPCLBM_BC_WALLS_Y, stream=stream)
        lat.set_params(tau)
        lat.set_force(u_star ** 2 / H, 0.0, 0.0)
        flds = W.channel_fields(nx, ny, nz, u_star, seed=7)
        cfg = {"workload": "channel Re_tau=180 384x192x192, y walls, body force, tau=%.6f" % tau}
    elif workload == "cavity":
        n, U0 = 150, 0.1 / 3 ** 0.5
        tau = 0.5 + 3 * U0 * n / 1000.0
        lat = F.Lattice(n, n, n, prec, F.FPCLBM_BC_BOX, stream=stream)
        lat.set_params(tau)
        lat.set_wall_velocity(U0)
        one = np.ones((n, n, n))
        flds = (one, 0 * one, 0 * one, 0 * one)
        cfg = {"workload": "lid-driven cubic cavity 150^3, Re=1000, Ma=0.1, walls on all faces, tau=%.6f" % tau}
    elif workload == "closure":
        # the learned closure's coarse channel: 192 x 96 x 96, Re_tau = 395 (H = 48, u* = 0.005), BF16
        # storage by default; the headline leg runs the learned mode with seeded random bf16 weights
        # (the inference cost does not depend on their values), the secondary leg plain FPC-LBM
        nx, ny, nz, u_star = 192, 96, 96, 0.005
        H = ny / 2
        tau = 3 * (u_star * H / 395.0) + 0.5
        lat = F.Lattice(nx, ny, nz, prec, F.FPCLBM_BC_WALLS_Y, stream=stream)
        if learned:
            lat.set_closure(closure_weights(seed=11))
            lat.set_params(tau, 0.0, F.FPCLBM_DIFF_FP_LEARNED)
        else:
            lat.set_params(tau)
        lat.set_force(u_star ** 2 / H, 0.0, 0.0)
        flds = W.channel_fields(nx, ny, nz, u_star, seed=7)
        cfg = {"workload": "learned-closure coarse channel Re_tau=395 192x96x96, y walls, body force, tau=%.6f, "
                           "%s" % (tau, "FP + learned closure (MLP 9-64-64-1, random bf16 weights)" if learned
                                   else "plain FP")}
    elif workload == "shear2d":
        n, U = 4096, 0.2 / 3 ** 0.5
        tau = 0.5 + 3 * U * n / 30000.0
        lat = F.Lattice2D(n, n, prec, stream=stream)
        lat.set_params(tau)
        flds = W.shear_layers(n, U)
        cfg = {"workload": "D2Q9 doubly periodic shear layers 4096^2, Re=30000, Ma=0.2, tau=%.6f" % tau}
    else:
        sides, taus = W.ensemble_config(256, seed=2410)
        dims = [(s_, s_, s_) for s_ in sides]
        lat = F.Lattice.ensemble(dims, taus, "fp32", stream=stream)
        lat.set_params(1.0)
        flds = W.ensemble_fields(sides, seed=2410)
        cfg = {"workload": "ensemble of 256 periodic boxes, sides in {32,48,64,96}, tau in [0.505,0.6], "
                           "solenoidal u_rms=0.04", "cells": int(sum(s_ ** 3 for s_ in sides))}
    flat = [np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1) for a in flds]
    if len(flat[0]) != lat.ncells:
        flat = [np.concatenate([np.asarray(f[q]).reshape(-1) for f in flds]) for q in range(4)]
    lat.init_fields(*flat)
    return lat, flat, lat.ncells, cfg


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from paper_2410_09739_gb300 import fpclbm as F
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream().cuda_stream
    prec0 = args.precision if args.workload != "ensemble" else "fp32"
    if args.workload == "closure" and args.precision == "fp32" and "--precision" not in sys.argv:
        prec0 = "bf16"  # the closure study's storage
    two_d = args.workload == "shear2d"
    qb = 18 if two_d else 54  # algorithmic bytes per cell update in units of the storage size
    results = {}
    # legs: the headline line first, then the secondary entries: 16-bit deviation storage of the
    # same workload and, for the TGV, the general-rate kernel with omega_k = k * drift for k >= 3,
    # the Re_tau = 180 channel (BF16 storage), the 256-box ensemble and the lid-driven cavity
    legs = [("headline", prec0, args.drift, True, args.workload)]
    if args.workload == "closure":
        legs.append(("plain_coarse", prec0, 0.0, False, "closure"))
    elif not args.no_variants and args.workload != "ensemble":
        legs += [(p, p, args.drift, True, args.workload) for p in ("fp16", "bf16") if p != prec0]
        if args.workload == "tgv" and args.drift == 0.0:
            legs.append(("fp32_general_rates", "fp32", 0.3, True, "tgv"))
            legs += [("channel_bf16", "bf16", 0.0, True, "channel"), ("ensemble_fp32", "fp32", 0.0, True, "ensemble"),
                     ("cavity_fp32", "fp32", 0.0, True, "cavity")]
    cfg = None
    for key, prec, drift, learned, wl in legs:
        lat, flat, ncell, c = setup(args, F, prec, stream, drift, learned, wl)
        if cfg is None:
            cfg = c
        barrier(world)
        clocks = Clocks(local) if rank == 0 else None
        if clocks:
            clocks.start()
        el = time_ours(lat, F, torch, args, ncell, args.steps, args.warmup, args.inner)
        ck = clocks.stop() if clocks else None
        el = max_over_ranks(el, world)
        results[key] = {"seconds": el, "clocks": ck, "launch": lat.launch() if not two_d else None,
                        "prec": prec, "drift": drift, "cells": ncell, "workload": wl,
                        "description": c["workload"]}
        if key == "headline":
            # e2e: host buffers through the C ABI, copies inside the timed region
            nf = 3 if two_d else 4
            hb = [torch.empty(ncell, dtype=torch.float64).pin_memory().numpy() for _ in range(2 * nf)]
            for a, src in zip(hb[:nf], flat):
                a[:] = src
            init, mom = ((F.fpclbm2d_init_fields, F.fpclbm2d_moments) if two_d else
                         (F.fpclbm_init_fields, F.fpclbm_moments))
            for _ in range(2):
                init(lat.h, *hb[:nf], on_device=0)
                lat.step(args.inner)
                mom(lat.h, *hb[nf:], on_device=0)
            barrier(world)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                init(lat.h, *hb[:nf], on_device=0)
                lat.step(args.inner)
                mom(lat.h, *hb[nf:], on_device=0)
            results[key]["e2e_s"] = max_over_ranks(time.perf_counter() - t0, world)
        lat.close()
    if rank != 0:
        return
    prec = prec0
    ncell = results["headline"]["cells"]
    el = results["headline"]["seconds"]
    value = ncell * args.inner * args.steps * world / el / 1e6
    launches = args.inner * args.steps
    per_launch = el / launches
    alg_bytes = qb * BYTES[prec] * ncell
    peak, peak_kind = peaks()
    achieved = alg_bytes / per_launch / 1e9
    cfg.update({"precision": prec, "storage": prec, "lbm_steps_per_bench_step": args.inner,
                "l2": "inputs larger than L2 (%.2f GB populations)" % (27 * BYTES[prec] * ncell / 1e9),
                "parallelism": "replicas" if world > 1 else "1 GPU"})
    kname = kernel_name(F, args.workload, results["headline"]["launch"])
    out = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec != "fp64" else "f64", "data": "synthetic",
        "config": cfg,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_nominal": NOMINAL_HBM_GBS,
                     "frac_nominal": achieved / NOMINAL_HBM_GBS,
                     "traffic": ncu_traffic(prec, args.size) if args.workload == "tgv" else None,
                     "peak_source": peak_kind, "kernel": kname, "algorithmic_bytes_per_launch": alg_bytes},
        "e2e": {"value": ncell * args.inner * args.steps * world / results["headline"]["e2e_s"] / 1e6,
                "unit": "MLUPS",
                "h2d_bytes_per_step": (3 if two_d else 4) * 8 * ncell,
                "d2h_bytes_per_step": (3 if two_d else 4) * 8 * ncell},
        "gpu_launches": launches,
        "clocks": results["headline"]["clocks"],
    }
    if args.drift > 0:
        cfg["drift"] = args.drift
    if len(results) > 1:
        out["variants"] = {}
        for key, r in results.items():
            if key == "headline":
                continue
            ach = qb * BYTES[r["prec"]] * r["cells"] / (r["seconds"] / launches) / 1e9
            out["variants"][key] = {
                "storage": r["prec"], "drift": r["drift"], "MLUPS": r["cells"] * launches * world / r["seconds"] / 1e6,
                "ms_per_step": r["seconds"] / args.steps * 1e3, "achieved_gbs": ach, "frac": ach / peak,
                "frac_nominal": ach / NOMINAL_HBM_GBS, "clocks": r["clocks"],
                "kernel": kernel_name(F, r["workload"], r["launch"])}
            if r["workload"] != args.workload:
                out["variants"][key]["workload"] = r["description"]
            elif args.workload == "tgv" and args.size == 256 and r["prec"] in ("fp16", "bf16") and r["drift"] == 0:
                alu = alu_roofline(r["prec"], out["variants"][key]["MLUPS"])
                if alu:
                    out["variants"][key]["alu_roofline"] = alu
    if world == 1 and not args.no_cpu_baseline:
        if two_d:
            U = 0.2 / 3 ** 0.5
            out["cpu_baseline"] = cpu_oracle_sample_2d(4096, 0.5 + 3 * U * 256 / 30000.0, U)
        else:
            n, u0 = args.size, 0.05
            out["cpu_baseline"] = cpu_oracle_sample(n, 3 * W.tgv_viscosity(n, u0, 1600.0) + 0.5, u0)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
