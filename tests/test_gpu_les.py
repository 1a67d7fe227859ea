"""Half channel (specular symmetry plane) and the Smagorinsky mode on the GPU, through the C ABI,
against the FP64 oracle (Sec. 4, turbulent channel LES).

Tolerances: FP64 path within 1e-12 relative per step (rounding order only: the kernel takes the
closed-form root of the Smagorinsky relation, the oracle bisects the relation itself); FP32 path
within 1e-6 absolute per step.  Odd and even step counts exercise both AA parities (the symmetry
plane acts on the odd step's loads and stores only).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2410_09739_gb300 import fpclbm as F

pytestmark = pytest.mark.gpu

E = O.velocity_set()
MIR = [int(np.where((E == E[a] * np.array([1, -1, 1])).all(axis=1))[0][0]) for a in range(27)]


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def near_eq(nx, ny, nz, seed, u_amp=0.05, noise=0.02):
    rho, ux, uy, uz = W.random_fields(nx, ny, nz, seed, u_amp=u_amp)
    f = O.init_equilibrium(rho, ux, uy, uz)
    rng = np.random.default_rng(seed + 1000)
    return f * (1.0 + noise * rng.uniform(-1, 1, f.shape))


SHAPES = [(1, 1, 1), (2, 3, 2), (5, 4, 3), (17, 9, 5), (33, 7, 6)]
LES = (0.17, 0.01, 26.0)


# the half channel with and without the Smagorinsky mode, and the Smagorinsky mode on the other
# boundary kinds (plain periodic and channel runs are covered by the parity tests)
CASES = [(shape, bc, les, force)
         for force in (False, True) for les in (False, True)
         for bc in (F.FPCLBM_BC_HALF_CHANNEL, F.FPCLBM_BC_WALLS_Y, F.FPCLBM_BC_PERIODIC)
         for shape in SHAPES if bc == F.FPCLBM_BC_HALF_CHANNEL or les]


@pytest.mark.parametrize("shape,bc,les,force", CASES)
def test_fp64_half_channel_and_les_match_oracle(shape, bc, les, force):
    nx, ny, nz = shape
    seed = nx * 100 + ny * 10 + nz + 7 * bc + 3 * force + les
    f0 = near_eq(nx, ny, nz, seed, noise=0.05)
    Fv = (2e-4, 0.0, 1.5e-4) if force else (0, 0, 0)
    tau = 0.53
    om = O.rates(tau)
    with F.Lattice(nx, ny, nz, "fp64", bc) as lat:
        lat.set_params(tau, 0.0, F.FPCLBM_DIFF_FP_SMAGORINSKY if les else F.FPCLBM_DIFF_FP)
        if les:
            lat.set_smagorinsky(*LES)
        lat.set_force(*Fv)
        lat.set_populations(f0)
        ref = f0
        for n in (1, 2, 5):  # 1, 3, 8 steps
            lat.step(n)
            ref = O.run(ref, n, bc=bc, F=Fv, omega=om, les=LES if les else None)
            got = lat.get_populations()
            assert rel(got, ref) <= 1e-12 * 8, n


def test_smagorinsky_changes_the_step():
    f0 = near_eq(9, 8, 7, 5, noise=0.05)
    outs = []
    for les in (None, LES):
        with F.Lattice(9, 8, 7, "fp64", F.FPCLBM_BC_HALF_CHANNEL) as lat:
            lat.set_params(0.52, 0.0, F.FPCLBM_DIFF_FP_SMAGORINSKY if les else F.FPCLBM_DIFF_FP)
            if les:
                lat.set_smagorinsky(*les)
            lat.set_populations(f0)
            lat.step(3)
            outs.append(lat.get_populations())
    assert np.max(np.abs(outs[0] - outs[1])) > 1e-6


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_lower_precision_les_half_channel(prec):
    nx, ny, nz = 16, 12, 10
    f0 = near_eq(nx, ny, nz, 91, noise=0.03)
    Fv = (1e-4, 0.0, 0.0)
    with F.Lattice(nx, ny, nz, prec, F.FPCLBM_BC_HALF_CHANNEL) as lat:
        lat.set_params(0.52, 0.0, F.FPCLBM_DIFF_FP_SMAGORINSKY)
        lat.set_smagorinsky(*LES)
        lat.set_force(*Fv)
        lat.set_populations(f0)
        fq = lat.get_populations()
        n = 6 if prec == "fp32" else 1
        lat.step(n)
        got = lat.get_populations()
    ref = O.run(fq, n, bc=O.BC_HALF_CHANNEL, F=Fv, omega=O.rates(0.52), les=LES)
    tol = 1e-6 * n if prec == "fp32" else 2.0 ** -8 * 0.1 + 1e-6
    assert np.max(np.abs(got - ref)) <= tol


def test_half_channel_equals_mirrored_full_channel_fp64():
    nx, ny, nz = 12, 6, 5
    f_half = near_eq(nx, ny, nz, 13)
    full0 = np.empty((27, nz, 2 * ny, nx))
    full0[:, :, :ny] = f_half
    for a in range(27):
        full0[a, :, ny:] = f_half[MIR[a], :, ::-1]
    outs = []
    for bc, f0, h in ((F.FPCLBM_BC_HALF_CHANNEL, f_half, ny), (F.FPCLBM_BC_WALLS_Y, full0, 2 * ny)):
        with F.Lattice(nx, h, nz, "fp64", bc) as lat:
            lat.set_params(0.55, 0.0, F.FPCLBM_DIFF_FP_SMAGORINSKY)
            lat.set_smagorinsky(*LES)
            lat.set_force(2e-4, 0.0, 0.0)
            lat.set_populations(f0)
            lat.step(41)
            outs.append(lat.get_populations())
    assert np.max(np.abs(outs[0] - outs[1][:, :, :ny])) <= 1e-13


def test_mode_and_boundary_combinations_are_checked():
    one = np.ones((4, 4, 4))
    with F.Lattice(4, 4, 4, "fp32", F.FPCLBM_BC_BOX) as lat:
        lat.set_params(0.6, 0.0, F.FPCLBM_DIFF_FP_SMAGORINSKY)
        lat.init_fields(one, 0 * one, 0 * one, 0 * one)
        with pytest.raises(F.FpclbmError) as e:
            lat.step(1)
        assert e.value.code == F.FPCLBM_ERR_ARG
    with F.Lattice(4, 4, 4, "fp32", F.FPCLBM_BC_HALF_CHANNEL) as lat:
        with pytest.raises(F.FpclbmError):
            lat.set_smagorinsky(-0.1)
        with pytest.raises(F.FpclbmError):
            lat.set_wall_velocity(0.1)
    with F.Lattice.ensemble([(8, 8, 8)], [0.7]) as ens:
        with pytest.raises(F.FpclbmError):
            ens.set_smagorinsky(0.17)
        with pytest.raises(F.FpclbmError):
            ens.set_params(0.7, 0.0, F.FPCLBM_DIFF_FP_SMAGORINSKY)
