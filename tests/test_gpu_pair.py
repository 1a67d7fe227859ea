"""The paired step variant (two cells per thread on the packed fp32 pipe, launch variant 2) against
the FP64 oracle and against the one-cell-per-thread variant.

Forced with FPCLBM_LAUNCH = "128:2:2" (block 128, register cap of 4 blocks, variant 2).  Odd cell
counts leave the last thread with one cell.  Tolerances as for the fp32 path: 1e-6 absolute per
step against the oracle; the two variants differ only by fma contraction choices, so they agree
within the same bound.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2410_09739_gb300 import fpclbm as F

pytestmark = pytest.mark.gpu


def near_eq(nx, ny, nz, seed, u_amp=0.05, noise=0.02):
    rho, ux, uy, uz = W.random_fields(nx, ny, nz, seed, u_amp=u_amp)
    f = O.init_equilibrium(rho, ux, uy, uz)
    rng = np.random.default_rng(seed + 1000)
    return f * (1.0 + noise * rng.uniform(-1, 1, f.shape))


def run(monkeypatch, variant, shape, prec, bc, force, mode, f0, n, drift=None):
    """drift None: 0.3 in the FP mode (general kernels), 0 in the MCM mode (without force: the
    unit-rate kernels)."""
    monkeypatch.setenv("FPCLBM_LAUNCH", "128:2:%d" % variant)
    nx, ny, nz = shape
    if drift is None:
        drift = 0.3 if mode == 0 else 0.0
    with F.Lattice(nx, ny, nz, prec, bc) as lat:
        lat.set_params(0.7, drift, mode)
        lat.set_force(*((2e-4, -1e-4, 1e-4) if force else (0, 0, 0)))
        lat.set_populations(f0)
        fq = lat.get_populations()
        lat.step(n)
        return fq, lat.get_populations()


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 3, 3), (5, 4, 3), (17, 9, 5), (33, 7, 6)])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("mode", [0, 1])
def test_pair_fp32_matches_oracle(monkeypatch, shape, bc, force, mode):
    nx, ny, nz = shape
    f0 = near_eq(nx, ny, nz, nx + 10 * ny + 100 * nz + bc + 2 * force + 4 * mode)
    Fv = (2e-4, -1e-4, 1e-4) if force else (0, 0, 0)
    for n in (1, 2, 5):
        fq, got = run(monkeypatch, 2, shape, "fp32", bc, force, mode, f0, n)
        ref = O.run(fq, n, bc=bc, F=Fv, omega=O.rates(0.7, 0.3 if mode == 0 else 0.0), mode=mode)
        assert np.max(np.abs(got - ref)) <= 1e-6 * n, n


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("shape", [(40, 33, 17), (64, 32, 31)])
def test_pair_equals_single_variant(monkeypatch, prec, shape):
    """40 steps (the captured-graph path) of both variants from the same state."""
    nx, ny, nz = shape
    f0 = near_eq(nx, ny, nz, 77)
    _, a = run(monkeypatch, 0, shape, prec, 1, True, 0, f0, 40)
    _, b = run(monkeypatch, 2, shape, prec, 1, True, 0, f0, 40)
    ulp = {"fp32": 1e-6, "fp16": 2.0 ** -11 * 0.05, "bf16": 2.0 ** -8 * 0.05}[prec]
    # 16-bit storage: a one-ulp difference in a stored deviation occurs where the two contraction
    # choices straddle a rounding boundary, and such flips propagate for the remaining steps
    d = np.abs(a - b)
    assert np.max(d) <= 40 * 1e-7 + 8 * ulp
    assert np.mean(d) <= 40 * 1e-8 + 0.25 * ulp



@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 3, 3), (17, 9, 5), (33, 7, 6)])
@pytest.mark.parametrize("bc", [0, 1])
def test_pair_unit_rates_fp32_matches_oracle(monkeypatch, shape, bc):
    """FP mode with the default rates and no force: the unit-rate paired kernels (the even step on
    neighbouring cells with vector accesses, the odd step through the interior fast path)."""
    nx, ny, nz = shape
    f0 = near_eq(nx, ny, nz, 300 + nx + bc)
    for n in (1, 2, 5):
        fq, got = run(monkeypatch, 2, shape, "fp32", bc, False, 0, f0, n, drift=0.0)
        ref = O.run(fq, n, bc=bc, omega=O.rates(0.7), mode=0)
        assert np.max(np.abs(got - ref)) <= 1e-6 * n, n


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("shape", [(41, 33, 17), (64, 32, 31)])
def test_pair_unit_rates_equals_single_variant(monkeypatch, prec, shape):
    """40 steps of the unit-rate kernels, paired against one cell per thread (41 x 33 x 17 has an
    odd cell count: the even step's last thread holds one cell)."""
    nx, ny, nz = shape
    f0 = near_eq(nx, ny, nz, 78)
    _, a = run(monkeypatch, 0, shape, prec, 1, False, 0, f0, 40, drift=0.0)
    _, b = run(monkeypatch, 2, shape, prec, 1, False, 0, f0, 40, drift=0.0)
    ulp = {"fp32": 1e-6, "fp16": 2.0 ** -11 * 0.05, "bf16": 2.0 ** -8 * 0.05}[prec]
    d = np.abs(a - b)
    assert np.max(d) <= 40 * 1e-7 + 8 * ulp
    assert np.mean(d) <= 40 * 1e-8 + 0.25 * ulp


@pytest.mark.parametrize("shape", [(6, 5, 4), (7, 6, 5), (16, 9, 6)])
@pytest.mark.parametrize("bc,lid", [(1, 0.05), (2, 0.05), (2, 0.0), (3, 0.0)])
@pytest.mark.parametrize("drift", [0.0, 0.3])
def test_pair_walls_and_lid_match_oracle(monkeypatch, shape, bc, lid, drift):
    """The paired kernel on a channel with a moving top wall, the closed box (lid moving or at rest)
    and the half channel, against the oracle: the moving-wall correction is applied per lane, and
    even nx takes the neighbouring-cell odd step where x is periodic (channel)."""
    monkeypatch.setenv("FPCLBM_LAUNCH", "128:2:2")
    nx, ny, nz = shape
    f0 = near_eq(nx, ny, nz, 900 + nx + 10 * bc + int(100 * lid))
    with F.Lattice(nx, ny, nz, "fp32", bc) as lat:
        lat.set_params(0.7, drift)
        if lid:
            lat.set_wall_velocity(lid)
        lat.set_populations(f0)
        fq = lat.get_populations()
        lat.step(5)
        got = lat.get_populations()
        assert lat.launch()["variant"] == 2
    ref = O.run(fq, 5, bc=bc, omega=O.rates(0.7, drift), uw=(lid, 0.0, 0.0))
    assert np.max(np.abs(got - ref)) <= 5e-6
