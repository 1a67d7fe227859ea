"""Exact discrete dispersion of a small shear wave under the FPC-LBM step (test helper for the
oracle pins of the 3D and 2D lattices)."""
import math

import numpy as np

CS2 = 1.0 / 3.0


def shear_wave_discrete_rate(n, tau, r3):
    """Exact per-step decay rate of a small shear wave u_x = U sin(k y), k = 2 pi / n, under the
    linearised scheme (von Neumann analysis of collide-and-stream).

    With the flow in x and variation in y only, sum the populations over e_z (D3Q27; D2Q9 has no e_z)
    and weight them by e_x.
    The three moments j = m_100, P = m_110, Q = m_120 of that x-odd part evolve on their own:
    collision keeps j (no force), relaxes P (the central kappa_110, attractor 0) at the shear rate
    omega = 1/tau and relaxes Q (raw m_120 = kappa_120 + c_s^2 j to first order in u, third-order
    attractor 0) at the third-order rate r3; streaming moves the e_y = +-1 parts by one cell, a factor
    exp(-+ i k) on a Fourier mode.  The wave decays with the largest eigenvalue lambda of the 3x3
    step matrix: rate = -ln |lambda|.  For r3 = 1, rate = nu k^2 (1 + (1 - tau)^2 k^2 / 3 + O(k^4)),
    nu = c_s^2 (tau - 1/2)."""
    k = 2 * math.pi / n
    c, s = math.cos(k), math.sin(k)
    collide = np.array([[1, 0, 0], [0, 1 - 1 / tau, 0], [r3 * CS2, 0, 1 - r3]], dtype=complex)
    stream = np.array([[1, -1j * s, -(1 - c)], [0, c, -1j * s], [0, -1j * s, c]], dtype=complex)
    lam = np.linalg.eigvals(stream @ collide)
    return -math.log(float(np.max(np.abs(lam))))
