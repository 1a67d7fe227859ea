"""Batched ensemble of independent periodic boxes (one persistent launch per time step)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2410_09739_gb300 import fpclbm as F

pytestmark = pytest.mark.gpu

DIMS = [(5, 4, 3), (8, 8, 8), (17, 9, 5), (1, 1, 1), (33, 7, 6)]
TAUS = [0.55, 0.8, 0.62, 1.1, 0.505]


def fields(seed):
    out = []
    for k, (nx, ny, nz) in enumerate(DIMS):
        out.append(W.random_fields(nx, ny, nz, seed + k, u_amp=0.05))
    return out


def concat(fs):
    return [np.concatenate([f[q].reshape(-1) for f in fs]) for q in range(4)]


@pytest.mark.parametrize("launch", ["", "128:4:2", "128:3:2"])
@pytest.mark.parametrize("nsteps", [1, 2, 7, 40])
def test_each_box_matches_oracle_and_single_box(monkeypatch, nsteps, launch):
    """launch: the default configuration, or the paired kernel (two cells of a tile per thread) with
    either register cap, forced through FPCLBM_LAUNCH.  The boxes' last tiles are ragged, so some
    threads hold one cell."""
    monkeypatch.setenv("FPCLBM_LAUNCH", launch)
    fs = fields(10 * nsteps)
    with F.Lattice.ensemble(DIMS, TAUS, "fp32") as ens:
        ens.set_params(1.0)
        ens.init_fields(*concat(fs))
        ens.step(nsteps)
        got = ens.get_populations()
        assert ens.step_count() == nsteps
    c0 = 0
    for (nx, ny, nz), tau, fld in zip(DIMS, TAUS, fs):
        n = nx * ny * nz
        mine = got[:, c0:c0 + n].reshape(27, nz, ny, nx)
        c0 += n
        ref = O.run(O.init_equilibrium(*fld), nsteps, omega=O.rates(tau))
        # fp32 arithmetic and storage: <= 1e-6 absolute per step (see test_gpu_parity.py)
        assert np.max(np.abs(mine - ref)) <= 1e-6 * nsteps
        with F.Lattice(nx, ny, nz, "fp32") as one:
            one.set_params(tau)
            one.init_fields(*fld)
            one.step(nsteps)
            assert np.array_equal(one.get_populations(), mine)


@pytest.mark.parametrize("launch", ["", "128:4:2"])
def test_generic_rates_and_force_match_oracle_and_single_box(monkeypatch, launch):
    """Rates of orders >= 3 other than 1 (drift 0.2) and a body force: the general collision kernels
    (the default rates without force take the unit-rate kernels)."""
    monkeypatch.setenv("FPCLBM_LAUNCH", launch)
    fs = fields(77)
    Fv = (2e-5, -1e-5, 1.5e-5)
    nsteps = 5
    with F.Lattice.ensemble(DIMS, TAUS, "fp32") as ens:
        ens.set_params(1.0, 0.2)
        ens.set_force(*Fv)
        ens.init_fields(*concat(fs))
        ens.step(nsteps)
        got = ens.get_populations()
    c0 = 0
    for (nx, ny, nz), tau, fld in zip(DIMS, TAUS, fs):
        n = nx * ny * nz
        mine = got[:, c0:c0 + n].reshape(27, nz, ny, nx)
        c0 += n
        ref = O.run(O.init_equilibrium(*fld), nsteps, F=Fv, omega=O.rates(tau, 0.2))
        assert np.max(np.abs(mine - ref)) <= 1e-6 * nsteps
        with F.Lattice(nx, ny, nz, "fp32") as one:
            one.set_params(tau, 0.2)
            one.set_force(*Fv)
            one.init_fields(*fld)
            one.step(nsteps)
            assert np.array_equal(one.get_populations(), mine)


def test_ensemble_mcm_mode_and_diagnostics():
    fs = fields(3)
    with F.Lattice.ensemble(DIMS, TAUS, "fp32") as ens:
        ens.set_params(1.0, 0.0, F.FPCLBM_DIFF_EQUILIBRIUM)
        ens.init_fields(*concat(fs))
        ens.step(3)
        got = ens.get_populations()
        d = ens.diagnostics()
        r, a, b, c = ens.moments()
    c0 = 0
    for (nx, ny, nz), tau, fld in zip(DIMS, TAUS, fs):
        n = nx * ny * nz
        ref = O.run(O.init_equilibrium(*fld), 3, omega=O.rates(tau), mode=O.EQ_MODE_MCM)
        assert np.max(np.abs(got[:, c0:c0 + n].reshape(27, nz, ny, nx) - ref)) <= 3e-6
        c0 += n
    expect = [r.sum(), (r * a).sum(), (r * b).sum(), (r * c).sum(), 0.5 * (r * (a * a + b * b + c * c)).sum()]
    assert np.allclose(d, expect, rtol=1e-12, atol=1e-14)


def test_ensemble_argument_errors():
    with pytest.raises(F.FpclbmError) as e:
        F.Lattice.ensemble([(4, 4, 4)], [0.45], "fp32")
    assert e.value.code == F.FPCLBM_ERR_PARAM
    with pytest.raises(F.FpclbmError) as e:
        F.Lattice.ensemble([(4, 4, 4)], [0.8], "fp64")
    assert e.value.code == F.FPCLBM_ERR_ARG
    with pytest.raises(F.FpclbmError) as e:
        F.Lattice.ensemble([(4, 0, 4)], [0.8], "fp32")
    assert e.value.code == F.FPCLBM_ERR_ARG
    with F.Lattice.ensemble([(4, 4, 4)], [0.8], "fp32") as ens:
        with pytest.raises(F.FpclbmError):
            ens.set_rates(np.ones(27))


def test_ensemble_config_shapes_run():
    """Config: 256 periodic boxes with sides from {32, 48, 64, 96}, tau in [0.505, 0.6], solenoidal
    fields with u_rms = 0.04 (a 16-box slice here; the full ensemble runs in bench.py)."""
    sides, taus = W.ensemble_config(16, seed=5)
    dims = [(s, s, s) for s in sides]
    flds = [W.solenoidal_field(s, seed=100 + i) for i, s in enumerate(sides)]
    with F.Lattice.ensemble(dims, taus, "fp32") as ens:
        ens.set_params(1.0)
        ens.init_fields(*concat(flds))
        d0 = ens.diagnostics()
        ens.step(100)
        d1 = ens.diagnostics()
    assert abs(d1[0] - d0[0]) / d0[0] < 1e-6        # mass
    assert np.all(np.abs(d1[1:4]) < 1e-6 * d0[0])   # zero mean momentum stays zero
    assert 0 < d1[4] < d0[4]                          # kinetic energy decays
