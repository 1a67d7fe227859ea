"""The light-cone helper behind the full-size sampled parity tests (tests/oracle_local.py) against
full oracle runs: at every cell of small periodic and channel lattices, after one and two steps,
it must give the oracle's populations (both evaluate the same collision; only the bookkeeping of
which neighbour feeds which population differs)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle_local import LocalOracle


@pytest.mark.parametrize("bc,force", [(0, False), (1, True), (1, False)])
def test_local_recursion_equals_full_oracle_run(bc, force):
    nx, ny, nz = 5, 4, 3
    rho, ux, uy, uz = W.random_fields(nx, ny, nz, 21 + bc, u_amp=0.05)
    rng = np.random.default_rng(3)
    f0 = O.init_equilibrium(rho, ux, uy, uz) * (1 + 0.02 * rng.uniform(-1, 1, (27, nz, ny, nx)))
    Fv = (1e-4, 0.0, -5e-5) if force else (0.0, 0.0, 0.0)
    om = O.rates(0.7, 0.2)
    loc = LocalOracle((nz, ny, nx), lambda x, y, z: f0[:, z, y, x], bc=bc, F=Fv, omega=om)
    for t in (1, 2):
        full = O.run(f0, t, bc=bc, F=Fv, omega=om)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    assert np.max(np.abs(loc.pre(x, y, z, t) - full[:, z, y, x])) <= 1e-15, (t, x, y, z)
