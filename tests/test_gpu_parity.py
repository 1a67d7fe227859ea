"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (written per test, derived from the arithmetic):
  * FP64 path: max |f_gpu - f_oracle| <= 1e-12 * max |f| per step (the stated
    bound); both sides are fp64, so the gap is rounding order only.
  * FP32 path: every operation rounds at 2^-24 relative to values that are
    deviations from the rest state (|g| <~ 0.1 here); a bound of 1e-6
    absolute per step on f covers ~100 such roundings with margin.
  * 16-bit storage: the oracle starts from the GPU's own rounded populations
    (read back exactly), so one step differs by the final rounding of the
    deviation, <= 2^-11 |g~| (fp16) or 2^-8 |g~| (bf16), plus the fp32 term.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle_local import LocalOracle
from paper_2410_09739_gb300 import fpclbm as F

pytestmark = pytest.mark.gpu

W_REST = O.equilibrium(1.0, [0, 0, 0])


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def near_eq_populations(nx, ny, nz, seed, u_amp=0.05, noise=0.02):
    """Equilibrium of random fields plus a random non-equilibrium part (host, oracle side)."""
    rho, ux, uy, uz = W.random_fields(nx, ny, nz, seed, u_amp=u_amp)
    f = O.init_equilibrium(rho, ux, uy, uz)
    rng = np.random.default_rng(seed + 1000)
    return f * (1.0 + noise * rng.uniform(-1, 1, f.shape))


def random_rates(seed):
    rng = np.random.default_rng(seed)
    om = rng.uniform(0.4, 1.8, 27)
    om[:4] = rng.uniform(-1, 3, 4)  # no effect on the result
    return om


def make(nx, ny, nz, prec, bc=0, F_=(0, 0, 0), omega=None, tau=None, drift=0.0, mode=0):
    lat = F.Lattice(nx, ny, nz, prec, bc)
    if omega is not None:
        lat.set_params(1.0, 0.0, mode)
        lat.set_rates(omega)
    else:
        lat.set_params(tau if tau is not None else 0.8, drift, mode)
    lat.set_force(*F_)
    return lat


SHAPES = [(1, 1, 1), (2, 2, 2), (3, 3, 3), (4, 4, 4), (5, 4, 3), (17, 9, 5), (33, 7, 6)]


@pytest.mark.parametrize("shape", SHAPES)
def test_init_matches_oracle_equilibrium(shape):
    nx, ny, nz = shape
    rho, ux, uy, uz = W.random_fields(nx, ny, nz, seed=5, u_amp=0.1)
    with make(nx, ny, nz, "fp64") as lat:
        lat.init_fields(rho, ux, uy, uz)
        got = lat.get_populations()
    assert rel(got, O.init_equilibrium(rho, ux, uy, uz)) < 1e-14


@pytest.mark.parametrize("prec,unit,slack", [("fp32", 2.0 ** -24, 1e-14), ("fp16", 2.0 ** -11, 1e-7),
                                             ("bf16", 2.0 ** -8, 1e-7)])
@pytest.mark.parametrize("shape", [(5, 4, 3), (33, 7, 6)])
def test_init_reduced_precision_is_rounded_equilibrium(shape, prec, unit, slack):
    """Each stored deviation is the oracle's equilibrium deviation rounded once to the storage type:
    |g_stored - g| <= unit |g| (round to nearest), plus a slack for the oracle's own fp64 LU
    rounding (fp32) or for the fp32 arithmetic of the 16-bit init and fp16 subnormals (16-bit)."""
    nx, ny, nz = shape
    rho, ux, uy, uz = W.random_fields(nx, ny, nz, seed=15, u_amp=0.1)
    with make(nx, ny, nz, prec) as lat:
        lat.init_fields(rho, ux, uy, uz)
        got = lat.get_populations()
    g = O.init_equilibrium(rho, ux, uy, uz) - W_REST[:, None, None, None]
    err = np.abs((got - W_REST[:, None, None, None]) - g)
    assert np.all(err <= unit * np.abs(g) + slack), float(np.max(err - unit * np.abs(g)))


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("bc", [0, 1])
def test_moments_reduced_precision_are_fp64_sums(prec, bc):
    """The moments of fp32 / 16-bit storage sum the stored deviations in fp32 with compensation: the
    result must equal the oracle's fp64 density and half-force velocity (Step 7) of the same stored
    populations up to rounding (a plain fp32 sum would be off by ~1e-9; the compensated sums and the
    fp64 ones agree to ~1e-16, so 1e-12 leaves a wide margin).  Odd step count: the moments read the
    AA odd layout."""
    nx, ny, nz = 17, 9, 5
    Fv = (1e-4, -5e-5, 2e-5)
    rho, ux, uy, uz = W.random_fields(nx, ny, nz, seed=16, u_amp=0.08)
    with make(nx, ny, nz, prec, bc, Fv, tau=0.7) as lat:
        lat.init_fields(rho, ux, uy, uz)
        lat.step(3)
        got = lat.moments()
        f = lat.get_populations()
    ref = O.moments(f, Fv)
    for x, y in zip(got, ref):
        assert np.max(np.abs(x.reshape(y.shape) - y)) <= 1e-12


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("mode", [0, 1])
def test_one_step_fp64_random_populations(shape, bc, force, mode):
    nx, ny, nz = shape
    seed = nx * 1000 + ny * 100 + nz * 10 + bc * 7 + force * 3 + mode
    f0 = W.random_populations(nx * ny * nz, seed).reshape(27, nz, ny, nx)
    Fv = (2e-3, -1e-3, 1.5e-3) if force else (0, 0, 0)
    om = random_rates(seed)
    with make(nx, ny, nz, "fp64", bc, Fv, omega=om, mode=mode) as lat:
        lat.set_populations(f0)
        lat.step(1)
        got = lat.get_populations()
    ref = O.step(f0, bc=bc, F=Fv, omega=om, mode=mode)
    assert rel(got, ref) <= 1e-12


@pytest.mark.parametrize("shape", [(3, 3, 3), (17, 9, 5)])
@pytest.mark.parametrize("bc", [0, 1, 2, 3])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("force", [False, True])
def test_one_step_fp64_unit_high_rates(shape, bc, mode, force):
    """Rates of orders 3-6 exactly 1 (the paper's default) select the unit-rate kernels, which set
    those moments to their attractors plus half their sources; random populations far from
    equilibrium, random shear and bulk rates, every boundary kind (closed box with a moving lid),
    with and without a body force."""
    nx, ny, nz = shape
    seed = 500 + nx + bc * 7 + mode + 11 * force
    f0 = W.random_populations(nx * ny * nz, seed).reshape(27, nz, ny, nx)
    om = random_rates(seed)
    om[10:] = 1.0
    uw = 0.03 if bc == 2 else 0.0
    Fv = (2e-3, -1e-3, 1.5e-3) if force else (0, 0, 0)
    with make(nx, ny, nz, "fp64", bc, Fv, omega=om, mode=mode) as lat:
        if bc == 2:
            lat.set_wall_velocity(uw)
        lat.set_populations(f0)
        lat.step(1)
        got = lat.get_populations()
    ref = O.step(f0, bc=bc, F=Fv, omega=om, mode=mode, uw=(uw, 0.0, 0.0))
    assert rel(got, ref) <= 1e-12


@pytest.mark.parametrize("nsteps", [2, 3, 10, 33, 70])
@pytest.mark.parametrize("bc", [0, 1])
def test_multi_step_fp64(nsteps, bc):
    """Covers both AA parities, the odd-count readback and the captured graph (>= 32 steps)."""
    nx, ny, nz = 17, 9, 5
    f0 = near_eq_populations(nx, ny, nz, seed=nsteps)
    Fv = (1e-4, 2e-5, -3e-5)
    om = O.rates(0.7, 0.3)
    with make(nx, ny, nz, "fp64", bc, Fv, tau=0.7, drift=0.3) as lat:
        lat.set_populations(f0)
        lat.step(nsteps)
        got = lat.get_populations()
        assert lat.step_count() == nsteps
    ref = O.run(f0, nsteps, bc=bc, F=Fv, omega=om)
    assert rel(got, ref) <= 1e-12 * nsteps


def test_split_step_calls_equal_one_call():
    nx, ny, nz = 9, 6, 5
    f0 = near_eq_populations(nx, ny, nz, seed=3)
    with make(nx, ny, nz, "fp64", 1, (1e-4, 0, 0), tau=0.6) as a, make(nx, ny, nz, "fp64", 1, (1e-4, 0, 0),
                                                                        tau=0.6) as b:
        a.set_populations(f0)
        b.set_populations(f0)
        a.step(77)
        for n in (1, 2, 33, 5, 36):
            b.step(n)
        assert np.array_equal(a.get_populations(), b.get_populations())


def test_tgv_32_fp64_200_steps_matches_oracle():
    """Config: 3D Taylor-Green vortex, FP64, periodic 32^3, rho = 1, u0 = 0.05, tau = 0.6, 200 steps."""
    n, u0, tau, steps = 32, 0.05, 0.6, 200
    rho, ux, uy, uz = W.tgv(n, u0)
    with make(n, n, n, "fp64", tau=tau) as lat:
        lat.init_fields(rho, ux, uy, uz)
        lat.step(steps)
        got = lat.get_populations()
        r, a, b, c = lat.moments()
    ref = O.run(O.init_equilibrium(rho, ux, uy, uz), steps, omega=O.rates(tau))
    assert rel(got, ref) <= 1e-10
    # kinetic energy against the low-Re decay exp(-6 nu k^2 t), reported: an equilibrium start
    # has no viscous stress (initial transient) and Re ~ 7.6 adds nonlinear transfer, so the
    # curve is only approximate (the oracle itself sits 5-13% off it at 16^3); the viscosity is
    # pinned by the fitted decay rates in test_oracle_pins.py
    nu = (tau - 0.5) / 3.0
    k = 2 * math.pi / n
    r0, a0, b0, c0 = (np.asarray(v) for v in (rho, ux, uy, uz))
    ke0 = np.sum(r0 * (a0 ** 2 + b0 ** 2 + c0 ** 2))
    ke = np.sum(r * (a * a + b * b + c * c))
    dev = ke / ke0 / math.exp(-6 * nu * k * k * steps) - 1
    print("TGV 32^3 KE(200)/analytic - 1 = %+.4f" % dev)
    assert abs(dev) < 0.15


@pytest.mark.parametrize("prec,unit", [("fp32", 0.0), ("fp16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("force", [True, False])  # without force: the unit-rate kernels
def test_one_step_reduced_precision(prec, unit, bc, force):
    nx, ny, nz = 17, 9, 5
    f0 = near_eq_populations(nx, ny, nz, seed=11)
    Fv = (1e-4, 0, 5e-5) if force else (0, 0, 0)
    om = O.rates(0.6)
    with make(nx, ny, nz, prec, bc, Fv, tau=0.6) as lat:
        lat.set_populations(f0)
        fq = lat.get_populations()  # the stored (rounded) state, exactly
        lat.step(1)
        got = lat.get_populations()
    ref = O.step(fq, bc=bc, F=Fv, omega=om)
    w = W_REST[:, None, None, None]
    bound = unit * np.abs(ref - w) + 1e-6
    assert np.all(np.abs(got - ref) <= bound)


def test_moments_and_diagnostics_fp64():
    nx, ny, nz = 17, 9, 5
    f0 = near_eq_populations(nx, ny, nz, seed=21)
    Fv = (1e-4, -5e-5, 0)
    with make(nx, ny, nz, "fp64", 1, Fv, tau=0.9) as lat:
        lat.set_populations(f0)
        lat.step(5)
        r, a, b, c = lat.moments()
        d = lat.diagnostics()
    ref = O.run(f0, 5, bc=1, F=Fv, omega=O.rates(0.9))
    R, A, B, C = O.moments(ref, Fv)
    for x, y in ((r, R), (a, A), (b, B), (c, C)):
        assert np.max(np.abs(x - y)) < 1e-13
    expect = [R.sum(), (R * A).sum(), (R * B).sum(), (R * C).sum(), 0.5 * (R * (A * A + B * B + C * C)).sum()]
    assert np.allclose(d, expect, rtol=1e-13, atol=1e-16)


def test_moments_on_device_match_host():
    torch = pytest.importorskip("torch")
    nx, ny, nz = 17, 9, 5
    rho, ux, uy, uz = W.random_fields(nx, ny, nz, seed=8)
    with make(nx, ny, nz, "fp32", tau=0.7) as lat:
        lat.init_fields(rho, ux, uy, uz)
        lat.step(3)
        host = lat.moments()
        dev = [torch.empty(nx * ny * nz, dtype=torch.float64, device="cuda") for _ in range(4)]
        F.fpclbm_moments(lat.h, *dev, on_device=1)
        torch.cuda.synchronize()
        for h_, d_ in zip(host, dev):
            assert np.array_equal(h_.reshape(-1), d_.cpu().numpy())
        # device-side init from torch tensors gives the same state as host init
        t = [torch.tensor(np.ascontiguousarray(v).reshape(-1), device="cuda") for v in (rho, ux, uy, uz)]
        F.fpclbm_init_fields(lat.h, *t, on_device=1)
        a = lat.get_populations()
        lat.init_fields(rho, ux, uy, uz)
        assert np.array_equal(a, lat.get_populations())


def test_divergence_is_reported():
    nx, ny, nz = 8, 8, 8
    f0 = near_eq_populations(nx, ny, nz, seed=2)
    f0[:, 3, 4, 5] = np.nan
    with make(nx, ny, nz, "fp32", tau=0.7) as lat:
        lat.set_populations(f0)
        with pytest.raises(F.FpclbmError) as e:
            lat.step(4)
        assert e.value.code == F.FPCLBM_ERR_DIVERGED
    f0 = near_eq_populations(nx, ny, nz, seed=2)
    f0[:, 1, 1, 1] = -0.1  # negative density
    with make(nx, ny, nz, "fp32", tau=0.7) as lat:
        lat.set_populations(f0)
        with pytest.raises(F.FpclbmError) as e:
            lat.step(1)
        assert e.value.code == F.FPCLBM_ERR_DIVERGED


def test_parameter_and_state_errors():
    with F.Lattice(4, 4, 4, "fp32") as lat:
        with pytest.raises(F.FpclbmError) as e:
            lat.step(1)
        assert e.value.code == F.FPCLBM_ERR_STATE
        with pytest.raises(F.FpclbmError) as e:
            lat.set_params(0.45)  # omega = 2.22
        assert e.value.code == F.FPCLBM_ERR_PARAM
        with pytest.raises(F.FpclbmError) as e:
            lat.set_params(0.8, 0.7)  # order 3 rate 2.1
        assert e.value.code == F.FPCLBM_ERR_PARAM
        om = np.ones(27)
        om[20] = 2.0
        with pytest.raises(F.FpclbmError) as e:
            lat.set_rates(om)
        assert e.value.code == F.FPCLBM_ERR_PARAM
        with pytest.raises(F.FpclbmError) as e:
            lat.set_params(0.8, 0.0, F.FPCLBM_DIFF_FP_LEARNED)  # no closure installed
        assert e.value.code == F.FPCLBM_ERR_STATE
        with pytest.raises(F.FpclbmError):
            lat.set_force(float("nan"), 0, 0)


def test_pinned_host_fields_equal_pageable():
    """Page-locked host buffers are read and written in place by the kernels (no staging copy);
    the results equal those of ordinary host memory bit for bit, for the 3D and the D2Q9 handle."""
    torch = pytest.importorskip("torch")
    nx, ny, nz = 19, 11, 7
    flds = [np.ascontiguousarray(a).reshape(-1) for a in W.random_fields(nx, ny, nz, seed=12)]
    pinned = [torch.from_numpy(a.copy()).pin_memory() for a in flds]
    outs = {}
    for kind, src in (("pageable", flds), ("pinned", [t.numpy() for t in pinned])):
        with make(nx, ny, nz, "fp32", tau=0.7) as lat:
            F.fpclbm_init_fields(lat.h, *src, on_device=0)
            lat.step(3)
            if kind == "pinned":
                dst = [torch.empty(nx * ny * nz, dtype=torch.float64).pin_memory() for _ in range(4)]
                F.fpclbm_moments(lat.h, *[t.numpy() for t in dst], on_device=0)
                outs[kind] = [t.numpy().copy() for t in dst]
            else:
                dst = [np.empty(nx * ny * nz) for _ in range(4)]
                F.fpclbm_moments(lat.h, *dst, on_device=0)
                outs[kind] = dst
    for a, b in zip(outs["pageable"], outs["pinned"]):
        assert np.array_equal(a, b)
    L = 24
    f2d = [np.ascontiguousarray(a).reshape(-1) for a in W.shear_layers(L, 0.05)]
    p2d = [torch.from_numpy(a.copy()).pin_memory() for a in f2d]
    res = []
    for src, pin in ((f2d, False), ([t.numpy() for t in p2d], True)):
        with F.Lattice2D(L, L, "fp32") as lat:
            lat.set_params(0.6)
            F.fpclbm2d_init_fields(lat.h, *src, on_device=0)
            lat.step(3)
            if pin:
                dst = [torch.empty(L * L, dtype=torch.float64).pin_memory() for _ in range(3)]
                F.fpclbm2d_moments(lat.h, *[t.numpy() for t in dst], on_device=0)
                res.append([t.numpy().copy() for t in dst])
            else:
                dst = [np.empty(L * L) for _ in range(3)]
                F.fpclbm2d_moments(lat.h, *dst, on_device=0)
                res.append(dst)
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_launch_query_names_the_collision_mode():
    with make(8, 8, 8, "fp32", tau=0.7) as lat:
        lat.init_fields(*W.random_fields(8, 8, 8, seed=4))
        with pytest.raises(F.FpclbmError):  # nothing chosen before the first step
            lat.launch()
        lat.step(2)
        got = lat.launch()
        assert got["mode"] == 4  # default rates, no force: FP with unit rates of orders 3-6
        if got["variant"] == 3:  # row-staged: block 160 or 288, minb holds the stage count
            assert got["block"] in (160, 288) and 2 <= got["minb"] <= 6
        else:
            assert got["variant"] in (0, 1, 2) and got["block"] in (128, 256) and 1 <= got["minb"] <= 4
        lat.set_force(1e-5, 0, 0)  # a force keeps the unit-rate kernels (half the sources)
        lat.step(2)
        assert lat.launch()["mode"] == 4
        lat.set_force(0, 0, 0)
        om = O.rates(0.7)
        om[12] = 1.1  # one third-order rate off 1: general kernels again
        lat.set_rates(om)
        lat.step(2)
        assert lat.launch()["mode"] == 0


def test_graph_replay_equals_single_launches_bitwise():
    n = 48
    rho, ux, uy, uz = W.tgv(n, 0.05)
    with make(n, n, n, "fp32", tau=0.55) as a, make(n, n, n, "fp32", tau=0.55) as b:
        a.init_fields(rho, ux, uy, uz)
        b.init_fields(rho, ux, uy, uz)
        a.step(64)
        for _ in range(64):
            b.step(1)
        for x, y in zip(a.moments(), b.moments()):
            assert np.array_equal(x, y)


def _sample_cells(nx, ny, nz, rng, k=12):
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (0, ny - 1, nz // 2), (nx - 1, 0, 1), (nx // 2, ny // 2, nz // 2)]
    pts += [tuple(int(v) for v in (rng.integers(nx), rng.integers(ny), rng.integers(nz))) for _ in range(k)]
    return pts


def _check_sampled(lat, shape_xyz, bc, Fv, om, unit, seed, steps=(1, 2)):
    """Full-size run in the bench's launch configuration, checked at sampled cells against the oracle's
    light-cone recursion started from the GPU's own stored initial populations."""
    nx, ny, nz = shape_xyz
    rng = np.random.default_rng(seed)
    cells = _sample_cells(nx, ny, nz, rng)
    # initial populations of every cell of the light cones (radius 2), read from the device
    need = sorted({((x + dx) % nx, (y + dy) % ny, (z + dz) % nz) for x, y, z in cells
                   for dx in range(-2, 3) for dy in range(-2, 3) for dz in range(-2, 3)})
    flat = [x + nx * (y + ny * z) for x, y, z in need]
    f0 = lat.populations_at(flat)
    table = {c: f0[:, i] for i, c in enumerate(need)}
    loc = LocalOracle((nz, ny, nx), lambda x, y, z: table[(x, y, z)], bc=bc, F=Fv, omega=om)
    gmax = float(np.max(np.abs(f0 - W_REST[:, None])))  # largest stored deviation in the cones
    flat_s = [x + nx * (y + ny * z) for x, y, z in cells]
    t = 0
    for target in steps:
        lat.step(target - t)
        t = target
        got = lat.populations_at(flat_s)
        for i, (x, y, z) in enumerate(cells):
            ref = loc.pre(x, y, z, t)
            # each step rounds the stored deviation once (<= unit |g|) and carries the earlier
            # roundings through a collision of gain <~ 2: (2t - 1) unit (|g~| + max |g|)
            bound = unit * (2 * t - 1) * (np.abs(ref - W_REST) + gmax) + 1e-6
            assert np.all(np.abs(got[:, i] - ref) <= bound), (t, (x, y, z), np.max(np.abs(got[:, i] - ref)))


def test_full_size_tgv_256_fp32_sampled():
    """Config: TGV Re = 1600 at 256^3, FP32, sampled cells after one even and one odd step."""
    n, u0 = 256, 0.05
    nu = W.tgv_viscosity(n, u0, 1600.0)
    tau = 3 * nu + 0.5
    rho, ux, uy, uz = W.tgv(n, u0)
    with make(n, n, n, "fp32", tau=tau) as lat:
        lat.init_fields(rho, ux, uy, uz)
        _check_sampled(lat, (n, n, n), 0, (0, 0, 0), O.rates(tau), 0.0, seed=1)


@pytest.mark.parametrize("prec,unit", [("fp32", 0.0), ("fp16", 2.0 ** -11)])
def test_full_size_tgv_512_sampled(prec, unit):
    """Config: TGV Re = 1600 at 512^3 (14.5 GB FP32, 7.2 GB FP16 on the device), sampled cells after
    one even and one odd step, in the launch configuration the autotuner picks for that size."""
    n, u0 = 512, 0.05
    tau = 3 * W.tgv_viscosity(n, u0, 1600.0) + 0.5
    rho, ux, uy, uz = W.tgv(n, u0)
    with make(n, n, n, prec, tau=tau) as lat:
        lat.init_fields(rho, ux, uy, uz)
        del rho, ux, uy, uz
        _check_sampled(lat, (n, n, n), 0, (0, 0, 0), O.rates(tau), unit, seed=3)


def test_full_size_channel_bf16_sampled():
    """Config: channel 384 x 192 x 192, walls in y, body force, BF16 storage; sampled cells."""
    nx, ny, nz = 384, 192, 192
    u_star = 0.005
    H = ny / 2
    nu = u_star * H / 180.0
    tau = 3 * nu + 0.5
    Fx = u_star ** 2 / H
    rho, ux, uy, uz = W.channel_fields(nx, ny, nz, u_star, seed=7)
    with make(nx, ny, nz, "bf16", 1, (Fx, 0, 0), tau=tau) as lat:
        lat.init_fields(rho, ux, uy, uz)
        _check_sampled(lat, (nx, ny, nz), 1, (Fx, 0, 0), O.rates(tau), 2.0 ** -8, seed=2)


def test_velocity_error_after_1000_steps():
    """Stated bound: FP32 path within 1e-5 (relative to u0) in velocity after 1000 steps of the
    256^3 Re = 1600 TGV, against the FP64 GPU path (itself at oracle parity).  The 16-bit storage
    variants have no stated bound; their errors are measured and printed (max and RMS of |du|/u0)
    and checked against about twice the values the storage-precision study measured on this
    workload (FP16 max 1.17e-2 / RMS 1.53e-3, BF16 9.49e-2 / 2.24e-2), so a regression of 2x fails."""
    torch = pytest.importorskip("torch")
    n, u0, steps = 256, 0.05, 1000
    nu = W.tgv_viscosity(n, u0, 1600.0)
    tau = 3 * nu + 0.5
    rho, ux, uy, uz = W.tgv(n, u0)
    outs = {}
    for prec in ("fp64", "fp32", "fp16", "bf16"):
        with make(n, n, n, prec, tau=tau) as lat:
            lat.init_fields(rho, ux, uy, uz)
            lat.step(steps)
            dev = [torch.empty(n ** 3, dtype=torch.float64, device="cuda") for _ in range(4)]
            F.fpclbm_moments(lat.h, *dev, on_device=1)
            outs[prec] = dev
    errs = {}
    for prec in ("fp32", "fp16", "bf16"):
        d = [outs[prec][q] - outs["fp64"][q] for q in (1, 2, 3)]
        mx = max(float(x.abs().max()) for x in d) / u0
        rms = float(torch.sqrt(sum((x * x).mean() for x in d) / 3)) / u0
        errs[prec] = (mx, rms)
        print("%s storage, max |du|/u0 after %d steps: %.3e (rms %.3e)" % (prec, steps, mx, rms))
    assert errs["fp32"][0] <= 1e-5
    assert errs["fp16"][0] <= 2.4e-2 and errs["fp16"][1] <= 3.1e-3
    assert errs["bf16"][0] <= 1.9e-1 and errs["bf16"][1] <= 4.5e-2
