"""fpclbm_diagnostics_noalloc: the diagnostics for callers that cannot allocate device memory.

Such callers (code inside an application that owns all device memory through
its own pool, or a loop that must not pay for allocation) pass device pointers
to their populations and to a 5-double result; the library keeps its partial
sums in a fixed device array instead of allocating.  This file is collected
last so that a run stopping at the first failure has run every other test
first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import workloads as W
from paper_2410_09739_gb300 import fpclbm as F

pytestmark = pytest.mark.gpu


def _device_pops(lat, torch):
    return torch.from_numpy(np.ascontiguousarray(lat.get_populations().reshape(-1))).cuda()


def test_noalloc_diagnostics_match_handle_diagnostics_twice():
    torch = pytest.importorskip("torch")
    nx, ny, nz = 40, 24, 18  # 17280 cells: several blocks and a ragged tail
    Fv = (2e-5, -1e-5, 5e-6)
    rho, ux, uy, uz = W.channel_fields(nx, ny, nz, 0.01, seed=4)
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with F.Lattice(nx, ny, nz, "fp32", F.FPCLBM_BC_WALLS_Y) as lat:
        lat.set_params(0.6)
        lat.set_force(*Fv)
        lat.init_fields(rho, ux, uy, uz)
        for nsteps in (3, 4):  # two calls in a row, the second on a different state (odd parity)
            lat.step(nsteps)
            expect = lat.diagnostics()
            f = _device_pops(lat, torch)
            F.fpclbm_diagnostics_noalloc(f, nx * ny * nz, *Fv, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            # both sides sum the same fp64 values in different orders
            assert np.allclose(got, expect, rtol=1e-12, atol=1e-15), (got, expect)


def test_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    f = torch.zeros(27, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    for n in (0, -5, 2 ** 31):
        with pytest.raises(F.FpclbmError) as e:
            F.fpclbm_diagnostics_noalloc(f, n, 0, 0, 0, out)
        assert e.value.code == F.FPCLBM_ERR_ARG
        assert "ncells" in F.fpclbm_last_error(None)


def test_noalloc_rejects_too_short_buffers_before_any_launch():
    torch = pytest.importorskip("torch")
    f = torch.zeros(27 * 8, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        F.fpclbm_diagnostics_noalloc(f, 9, 0, 0, 0, out)
    with pytest.raises(ValueError):
        F.fpclbm_diagnostics_noalloc(f, 8, 0, 0, 0, out[:4])
