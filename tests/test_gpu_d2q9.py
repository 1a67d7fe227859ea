"""The D2Q9 FPC-LBM on the GPU (fpclbm2d_*), through the C ABI, against the FP64 2D oracle.

Tolerances as in 3D: FP64 within 1e-12 relative per step, FP32 within 1e-6 absolute per step,
16-bit storage within the final rounding of the deviations (one step from the GPU's own state).
"""
import math

import numpy as np
import pytest

from oracle import oracle2d as O2
from paper_2410_09739_gb300 import fpclbm as F

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def near_eq(nx, ny, seed, u_amp=0.08, noise=0.05):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.03 * rng.uniform(-1, 1, (ny, nx))
    ux, uy = (u_amp * rng.uniform(-1, 1, (ny, nx)) for _ in range(2))
    f = O2.init_equilibrium(rho, ux, uy)
    return f * (1 + noise * rng.uniform(-1, 1, f.shape))


SHAPES = [(1, 1), (2, 3), (5, 4), (33, 7), (64, 9)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mode", [F.FPCLBM_DIFF_FP, F.FPCLBM_DIFF_EQUILIBRIUM])
@pytest.mark.parametrize("force", [False, True])
def test_fp64_matches_oracle(shape, mode, force):
    nx, ny = shape
    f0 = near_eq(nx, ny, nx * 10 + ny + mode + 3 * force)
    Fv = (2e-4, -3e-4) if force else (0.0, 0.0)
    rng = np.random.default_rng(nx + ny)
    om = rng.uniform(0.6, 1.6, 9)  # moderate rates: the rough random state stays stable for 48 steps
    om[5] = om[4]  # isotropic shear viscosity
    with F.Lattice2D(nx, ny, "fp64") as lat:
        lat.set_params(1.0, 0.0, 0.0, mode)
        lat.set_rates(om)
        lat.set_force(*Fv)
        lat.set_populations(f0)
        ref = f0
        for n in (1, 2, 5, 40):  # 1, 3, 8, 48 steps: both parities and the captured graph
            lat.step(n)
            ref = O2.run(ref, n, F=Fv, omega=om, mode=mode)
            assert rel(lat.get_populations(), ref) <= 1e-12 * (n + 1), n


def test_init_and_moments_match_oracle():
    nx, ny = 17, 11
    rng = np.random.default_rng(2)
    rho = 1 + 0.05 * rng.uniform(-1, 1, (ny, nx))
    ux, uy = (0.1 * rng.uniform(-1, 1, (ny, nx)) for _ in range(2))
    with F.Lattice2D(nx, ny, "fp64") as lat:
        lat.init_fields(rho, ux, uy)
        assert rel(lat.get_populations(), O2.init_equilibrium(rho, ux, uy)) <= 1e-14
        lat.set_force(1e-3, 2e-3)
        lat.step(3)
        r, u, v = lat.moments()
        fg = lat.get_populations()
    r2, u2, v2 = O2.moments(fg, (1e-3, 2e-3))
    assert max(np.max(np.abs(r - r2)), np.max(np.abs(u - u2)), np.max(np.abs(v - v2))) <= 1e-14


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_lower_precision(prec):
    nx, ny = 48, 40
    f0 = near_eq(nx, ny, 5)
    om = O2.rates(0.6, 0.35)
    with F.Lattice2D(nx, ny, prec) as lat:
        lat.set_params(0.6, 0.35)
        lat.set_force(1e-4, 0.0)
        lat.set_populations(f0)
        fq = lat.get_populations()
        n = 10 if prec == "fp32" else 1
        lat.step(n)
        got = lat.get_populations()
    ref = O2.run(fq, n, F=(1e-4, 0.0), omega=om)
    g_max = np.max(np.abs(ref - O2.equilibrium(1.0, (0, 0))[:, None, None]))
    tol = {"fp32": 1e-6 * n, "fp16": 2.0 ** -11 * g_max + 1e-6, "bf16": 2.0 ** -8 * g_max + 1e-6}[prec]
    assert np.max(np.abs(got - ref)) <= tol


def test_shear_wave_viscosity_fp32():
    """nu = cs^2 (1/omega_2d - 1/2) from the decay of u_x = U sin(ky) on the GPU (FP32)."""
    n, tau = 64, 0.7
    k = 2 * math.pi / n
    y = np.arange(n)
    ux = 1e-3 * np.sin(k * y)[:, None] * np.ones((1, 4))
    with F.Lattice2D(4, n, "fp32") as lat:
        lat.set_params(tau)
        lat.init_fields(np.ones((n, 4)), ux, np.zeros((n, 4)))
        amps, ts = [], []
        for i in range(10):
            lat.step(64)
            u = lat.moments()[1]
            amps.append(2 / n * u[:, 0] @ np.sin(k * y))
            ts.append(64 * (i + 1))
    rate = -np.polyfit(ts, np.log(amps), 1)[0]
    assert abs(rate / ((tau - 0.5) / 3 * k * k) - 1) < 0.01


def test_errors():
    with pytest.raises(F.FpclbmError) as e:
        F.Lattice2D(0, 4, "fp32")
    assert e.value.code == F.FPCLBM_ERR_ARG
    with F.Lattice2D(4, 4, "fp32") as lat:
        with pytest.raises(F.FpclbmError) as e:
            lat.step(1)
        assert e.value.code == F.FPCLBM_ERR_STATE
        with pytest.raises(F.FpclbmError) as e:
            lat.set_params(0.4)  # omega = 2.5
        assert e.value.code == F.FPCLBM_ERR_PARAM
        with pytest.raises(F.FpclbmError):
            lat.set_params(0.6, 0.0, 0.0, F.FPCLBM_DIFF_FP_LEARNED)
        one = np.ones((4, 4))
        lat.init_fields(one, 0 * one, 0 * one)
        f = lat.get_populations()
        f[0, 1, 1] = -5.0
        lat.set_populations(f)
        with pytest.raises(F.FpclbmError) as e:
            lat.step(1)
        assert e.value.code == F.FPCLBM_ERR_DIVERGED


@pytest.mark.parametrize("shape", [(1, 1), (2, 3), (5, 4), (33, 7), (64, 9)])
@pytest.mark.parametrize("mode", [F.FPCLBM_DIFF_FP, F.FPCLBM_DIFF_EQUILIBRIUM])
@pytest.mark.parametrize("lid", [0.0, 0.06])
def test_fp64_closed_box_matches_oracle(shape, mode, lid):
    """2D lid-driven cavity walls (bounce-back on all four sides, moving wall y = ny - 1/2)."""
    nx, ny = shape
    f0 = near_eq(nx, ny, 500 + nx + ny + mode)
    rng = np.random.default_rng(nx * ny)
    om = rng.uniform(0.6, 1.6, 9)
    om[5] = om[4]
    Fv = (1e-4, -2e-4)
    with F.Lattice2D(nx, ny, "fp64") as lat:
        lat.set_params(1.0, 0.0, 0.0, mode)
        lat.set_rates(om)
        lat.set_force(*Fv)
        lat.set_boundary(F.FPCLBM_BC_BOX, lid)
        lat.set_populations(f0)
        ref = f0
        for n in (1, 2, 5, 40):
            lat.step(n)
            ref = O2.run(ref, n, F=Fv, omega=om, mode=mode, bc=O2.BC_BOX, uw=lid)
            assert rel(lat.get_populations(), ref) <= 1e-12 * (n + 1), n
            r, u, v = lat.moments()
            r2, u2, v2 = O2.moments(ref, Fv)
            assert np.max(np.abs(u - u2)) <= 1e-12


def test_closed_box_fp32_and_errors():
    n = 48
    one = np.ones((n, n))
    with F.Lattice2D(n, n, "fp32") as lat:
        with pytest.raises(F.FpclbmError):
            lat.set_boundary(F.FPCLBM_BC_PERIODIC, 0.1)  # a lid needs the closed box
        with pytest.raises(F.FpclbmError):
            lat.set_boundary(F.FPCLBM_BC_WALLS_Y)
        lat.set_boundary(F.FPCLBM_BC_BOX, 0.08)
        lat.set_params(0.56)
        lat.init_fields(one, 0 * one, 0 * one)
        f0 = lat.get_populations()
        lat.step(7)
        got = lat.get_populations()
        with pytest.raises(F.FpclbmError) as e:
            lat.set_boundary(F.FPCLBM_BC_PERIODIC)  # odd step count
        assert e.value.code == F.FPCLBM_ERR_STATE
    ref = O2.run(f0, 7, omega=O2.rates(0.56), bc=O2.BC_BOX, uw=0.08)
    assert np.max(np.abs(got - ref)) <= 7e-6
    assert abs(got.sum() - f0.sum()) <= 1e-4 * f0.sum()
