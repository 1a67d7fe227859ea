"""Oracle populations at a few sampled cells of a large lattice (test helper).

f_a(x, t) = [collide(f(x - e_a, t-1))]_a with half-way bounce-back on y walls
(f_a(x, t) = [collide(f(x, t-1))]_abar when x - e_a lies in a wall).  The
recursion touches only the light cone of the sampled cell (5^3 cells for
t = 2), so the FP64 oracle can check single cells of full-size runs.
"""
from __future__ import annotations

import numpy as np

import oracle as O


class LocalOracle:
    def __init__(self, shape_zyx, f0_at, bc=0, F=(0.0, 0.0, 0.0), omega=None, mode=0):
        """f0_at(x, y, z) -> initial populations (27,) of that cell."""
        self.nz, self.ny, self.nx = shape_zyx
        self.f0_at = f0_at
        self.bc = bc
        self.F = np.asarray(F, float)
        self.omega = np.ones(27) if omega is None else np.asarray(omega, float)
        self.mode = mode
        self.e = O.velocity_set()
        self.opp = [int(np.where((self.e == -self.e[a]).all(axis=1))[0][0]) for a in range(27)]
        self._pre = {}
        self._post = {}

    def pre(self, x, y, z, t):
        """Populations entering the collision at (x, y, z) at time t."""
        key = (x, y, z, t)
        if key in self._pre:
            return self._pre[key]
        if t == 0:
            f = np.asarray(self.f0_at(x, y, z), float)
        else:
            f = np.empty(27)
            for a in range(27):
                ex, ey, ez = self.e[a]
                sy = y - ey
                if self.bc == 1 and (sy < 0 or sy >= self.ny):
                    f[a] = self.post(x, y, z, t - 1)[self.opp[a]]
                else:
                    f[a] = self.post((x - ex) % self.nx, sy % self.ny, (z - ez) % self.nz, t - 1)[a]
        self._pre[key] = f
        return f

    def post(self, x, y, z, t):
        key = (x, y, z, t)
        if key not in self._post:
            self._post[key] = O.collide(self.pre(x, y, z, t), self.F, self.omega, self.mode)
        return self._post[key]
