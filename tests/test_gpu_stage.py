"""The row-staged step variant (launch variant 3: whole slot rows moved through shared memory by
bulk asynchronous copies, two neighbouring cells per thread) against the paired variant and the
FP64 oracle.

The staged kernel pairs the same cells (x, x + 1) as the paired kernel's neighbouring-cell steps,
runs the same collision code (every f2 operation an explicit round-to-nearest intrinsic, so no
contraction choice differs) and the same conversions to and from the storage type: its stored
state must equal the paired kernel's bit for bit, step after step, in every storage type.  Against
the oracle it meets the fp32 path's bound of 1e-6 absolute per step.

Forced with FPCLBM_LAUNCH = "128:2:3[:stages]"; the variant needs rows of a multiple of 16 bytes
(nx a multiple of 8 for 16-bit storage, of 4 for fp32) and falls back to the paired kernel
otherwise.
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


FORCE = (2e-4, -1e-4, 1e-4)


def run(monkeypatch, launch, shape, prec, bc, force, mode, drift, f0, n):
    """Populations after n steps from f0 with a forced launch; also the launch the library took."""
    monkeypatch.setenv("FPCLBM_LAUNCH", launch)
    nx, ny, nz = shape
    with F.Lattice(nx, ny, nz, prec, bc) as lat:
        lat.set_params(0.7, drift, mode)
        lat.set_force(*(FORCE if force else (0, 0, 0)))
        lat.set_populations(f0)
        fq = lat.get_populations()
        lat.step(n)
        return fq, lat.get_populations(), lat.launch()


# (mode, drift): general FP rates, FP unit rates, MCM general rates, MCM unit rates
MODES = [(0, 0.3), (0, 0.0), (1, 0.3), (1, 0.0)]


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp32"])
@pytest.mark.parametrize("shape", [(8, 3, 2), (16, 5, 3), (24, 7, 6), (40, 9, 5)])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("mode,drift", MODES)
def test_stage_equals_paired_bitwise(monkeypatch, prec, shape, bc, force, mode, drift):
    nx, ny, nz = shape
    f0 = near_eq(nx, ny, nz, 7 * nx + ny + 3 * nz + bc + 2 * force + 4 * mode)
    for n in (1, 2, 5):
        _, a, la = run(monkeypatch, "128:2:2", shape, prec, bc, force, mode, drift, f0, n)
        _, b, lb = run(monkeypatch, "128:2:3", shape, prec, bc, force, mode, drift, f0, n)
        assert la["variant"] == 2 and lb["variant"] == 3
        assert np.array_equal(a, b), (n, float(np.max(np.abs(a - b))))


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("stages", [3, 4, 6])
@pytest.mark.parametrize("shape,bc", [((64, 32, 31), 1), ((48, 20, 16), 0)])
def test_stage_equals_paired_many_steps(monkeypatch, prec, stages, shape, bc):
    """40 steps (the captured-graph path, both parities many times) with force in a channel, and
    ring depths 3, 4 and 6: more rows than CTAs, so every CTA cycles its stages."""
    nx, ny, nz = shape
    f0 = near_eq(nx, ny, nz, 91 + stages)
    _, a, _ = run(monkeypatch, "128:2:2", shape, prec, bc, True, 0, 0.0, f0, 40)
    _, b, lb = run(monkeypatch, "128:2:3:%d" % stages, shape, prec, bc, True, 0, 0.0, f0, 40)
    assert lb["variant"] == 3
    assert np.array_equal(a, b), float(np.max(np.abs(a - b)))


@pytest.mark.parametrize("shape", [(8, 1, 1), (4, 4, 4), (16, 9, 5), (32, 7, 6)])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("mode,drift", MODES)
def test_stage_fp32_matches_oracle(monkeypatch, shape, bc, force, mode, drift):
    nx, ny, nz = shape
    f0 = near_eq(nx, ny, nz, 500 + nx + 10 * ny + bc + 2 * force + 4 * mode)
    Fv = FORCE if force else (0, 0, 0)
    for n in (1, 2, 5):
        fq, got, lau = run(monkeypatch, "128:2:3", shape, "fp32", bc, force, mode, drift, f0, n)
        assert lau["variant"] == 3
        ref = O.run(fq, n, bc=bc, F=Fv, omega=O.rates(0.7, drift), mode=mode)
        assert np.max(np.abs(got - ref)) <= 1e-6 * n, n


@pytest.mark.parametrize("prec", ["bf16", "fp16", "fp32"])
@pytest.mark.parametrize("shape", [(264, 3, 2), (384, 4, 3), (392, 2, 3)])
@pytest.mark.parametrize("bc", [0, 1])
def test_stage_wide_rows_equal_paired_bitwise(monkeypatch, prec, shape, bc):
    """Rows of 257-384 cells take tiles of 384 (six consumer warps), longer rows tiles of 512 (eight
    consumer warps); unit rates with force (the channel's collision) and general rates, two steps."""
    nx, ny, nz = shape
    f0 = near_eq(nx, ny, nz, nx + 7 * bc)
    for mode, drift in ((0, 0.0), (0, 0.3)):
        _, a, la = run(monkeypatch, "128:2:2", shape, prec, bc, True, mode, drift, f0, 2)
        _, b, lb = run(monkeypatch, "128:2:3", shape, prec, bc, True, mode, drift, f0, 2)
        assert la["variant"] == 2 and lb["variant"] == 3
        assert lb["block"] == (224 if nx <= 384 else 288)
        assert np.array_equal(a, b), float(np.max(np.abs(a - b)))


@pytest.mark.parametrize("prec,shape", [("bf16", (12, 4, 4)), ("fp16", (20, 3, 3)), ("fp32", (6, 4, 4))])
def test_stage_falls_back_when_rows_are_not_16_byte_multiples(monkeypatch, prec, shape):
    nx, ny, nz = shape
    f0 = near_eq(nx, ny, nz, 3)
    _, a, la = run(monkeypatch, "128:2:3", shape, prec, 1, True, 0, 0.0, f0, 3)
    _, b, _ = run(monkeypatch, "128:2:2", shape, prec, 1, True, 0, 0.0, f0, 3)
    assert la["variant"] == 2
    assert np.array_equal(a, b)


def test_stage_full_size_bf16_tgv_256_matches_paired(monkeypatch):
    """The 256^3 BF16 TGV of the bench, 6 steps, staged against paired on sampled cells (every
    cell of the rows at the box's faces and edges, plus random cells)."""
    n = 256
    tau = 3 * W.tgv_viscosity(n, 0.05, 1600.0) + 0.5
    rho, ux, uy, uz = W.tgv(n, 0.05)
    rng = np.random.default_rng(5)
    rows = [(y, z) for y in (0, 1, n - 1) for z in (0, n // 2, n - 1)]
    cells = np.concatenate([np.arange(n) + n * (y + n * z) for y, z in rows] +
                           [rng.integers(0, n ** 3, 4096)]).astype(np.int64)
    out = []
    for launch in ("128:2:2", "128:2:3"):
        monkeypatch.setenv("FPCLBM_LAUNCH", launch)
        with F.Lattice(n, n, n, "bf16", F.FPCLBM_BC_PERIODIC) as lat:
            lat.set_params(tau)
            lat.init_fields(rho, ux, uy, uz)
            lat.step(6)
            assert lat.launch()["variant"] == int(launch[-1])
            out.append(lat.populations_at(cells))
    assert np.array_equal(out[0], out[1])
