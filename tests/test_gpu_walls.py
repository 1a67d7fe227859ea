"""Closed-box walls and the moving wall y = ny - 1/2 on the GPU, through the C ABI, against the
FP64 oracle (Sec. 4, cubic cavity).

Tolerances as in the periodic parity tests: the FP64 path within 1e-12 relative per step (rounding
order only), the FP32 path within 1e-6 absolute per step.  Odd and even step counts exercise both
AA parities (bounce-back is realised on the load side in one and on the store side in the other).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2410_09739_gb300 import fpclbm as F

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def near_eq(nx, ny, nz, seed, u_amp=0.05, noise=0.02):
    rho, ux, uy, uz = W.random_fields(nx, ny, nz, seed, u_amp=u_amp)
    f = O.init_equilibrium(rho, ux, uy, uz)
    rng = np.random.default_rng(seed + 1000)
    return f * (1.0 + noise * rng.uniform(-1, 1, f.shape))


SHAPES = [(1, 1, 1), (2, 3, 2), (5, 4, 3), (17, 9, 5), (33, 7, 6)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bc,lid", [(F.FPCLBM_BC_BOX, (0.0, 0.0)), (F.FPCLBM_BC_BOX, (0.06, -0.04)),
                                    (F.FPCLBM_BC_WALLS_Y, (0.05, 0.02))])
@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("mode", [0, 1])
def test_fp64_walls_match_oracle(shape, bc, lid, force, mode):
    nx, ny, nz = shape
    seed = nx * 100 + ny * 10 + nz + 7 * bc + 3 * force + mode
    f0 = near_eq(nx, ny, nz, seed)
    Fv = (2e-4, -1e-4, 1.5e-4) if force else (0, 0, 0)
    om = O.rates(0.7, 0.3 if mode == 0 else 0.0)
    uw = (lid[0], 0.0, lid[1])
    with F.Lattice(nx, ny, nz, "fp64", bc) as lat:
        lat.set_params(0.7, 0.3 if mode == 0 else 0.0, mode)
        lat.set_force(*Fv)
        lat.set_wall_velocity(*lid)
        lat.set_populations(f0)
        ref = f0
        for n in (1, 2, 5):  # 1, 3, 8 steps: odd, odd, even
            lat.step(n)
            ref = O.run(ref, n, bc=bc, F=Fv, omega=om, mode=mode, uw=uw)
            got = lat.get_populations()
            assert rel(got, ref) <= 1e-12 * 8, n


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_lower_precision_cavity_steps(prec):
    """FP32: within 1e-6 per step of the oracle over 6 steps.  BF16 storage: the same from the
    GPU's own rounded state, one step, within the bf16 rounding of the deviations."""
    nx, ny, nz = 12, 10, 9
    f0 = near_eq(nx, ny, nz, 77)
    om = O.rates(0.6)
    with F.Lattice(nx, ny, nz, prec, F.FPCLBM_BC_BOX) as lat:
        lat.set_params(0.6)
        lat.set_wall_velocity(0.08, 0.0)
        lat.set_populations(f0)
        fq = lat.get_populations()
        n = 6 if prec == "fp32" else 1
        lat.step(n)
        got = lat.get_populations()
    ref = O.run(fq, n, bc=O.BC_BOX, omega=om, uw=(0.08, 0, 0))
    tol = 1e-6 * n if prec == "fp32" else 2.0 ** -8 * 0.1 + 1e-6
    assert np.max(np.abs(got - ref)) <= tol


def test_couette_steady_profile():
    """Plane Couette flow through the channel kernel with a moving upper wall: the FP64 GPU run
    reaches u_x = U (y + 1/2) / ny up to the scheme's O(U^3) defect (exact at tau = 1)."""
    ny, U = 16, 0.01
    z = np.zeros((4, ny, 8))
    with F.Lattice(8, ny, 4, "fp64", F.FPCLBM_BC_WALLS_Y) as lat:
        lat.set_params(1.0)
        lat.set_wall_velocity(U)
        lat.init_fields(z + 1, z, z, z)
        lat.step(4000)
        rho, ux, uy, uz = (a.reshape(4, ny, 8) for a in lat.moments())
    exact = U * (np.arange(ny) + 0.5) / ny
    assert np.max(np.abs(ux - exact[None, :, None])) <= 1e-12
    assert np.max(np.abs(uy)) <= 1e-14 and np.max(np.abs(uz)) <= 1e-14


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cavity_conserves_mass_and_mirror_symmetry(prec):
    n = 24
    one = np.ones((n, n, n))
    with F.Lattice(n, n, n, prec, F.FPCLBM_BC_BOX) as lat:
        lat.set_params(0.56)
        lat.set_wall_velocity(0.1)
        lat.init_fields(one, 0 * one, 0 * one, 0 * one)
        m0 = lat.diagnostics()[0]
        lat.step(301)
        m1 = lat.diagnostics()[0]
        rho, ux, uy, uz = (a.reshape(n, n, n) for a in lat.moments())
    assert abs(m1 - m0) <= (1e-12 if prec == "fp64" else 1e-6) * m0
    assert np.max(np.abs(ux)) > 0.01
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.max(np.abs(ux - ux[::-1])) <= tol and np.max(np.abs(uz + uz[::-1])) <= tol


def test_wall_velocity_argument_errors():
    with F.Lattice(4, 4, 4, "fp32") as lat:
        with pytest.raises(F.FpclbmError) as e:
            lat.set_wall_velocity(0.1)
        assert e.value.code == F.FPCLBM_ERR_ARG
    with F.Lattice(4, 4, 4, "fp32", F.FPCLBM_BC_BOX) as lat:
        with pytest.raises(F.FpclbmError):
            lat.set_wall_velocity(float("nan"))
    with F.Lattice.ensemble([(8, 8, 8)], [0.7]) as ens:
        with pytest.raises(F.FpclbmError):
            ens.set_wall_velocity(0.1)
