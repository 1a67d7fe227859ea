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


def sound_wave_step_matrix_2d(n, omega, mcm=False):
    """Linearised D2Q9 step of a plane sound wave along x (rho and u_x vary with x only, u_y = 0),
    for the Fourier mode exp(i k x), k = 2 pi / n (von Neumann analysis of collide-and-stream).

    Sum the populations over e_y with the weights 1 and e_y^2: the six moments m_00 = rho,
    m_10 = j, m_20, m_02, m_12, m_22 of those two sums evolve on their own.  State: their deviations
    (r, j, p, q, s, w) from the rest values (1, 0, c_s^2, c_s^2, 0, c_s^4).  Collision, to first
    order around rest (u = j): the central kappa_20, kappa_02 differ from c_s^2 rho by
    a = p - c_s^2 r, b = q - c_s^2 r; the bulk part a + b relaxes at omega_3 and the deviatoric part
    a - b at omega_4 (2D Step 3 grouping), both toward 0; kappa_12 = m_12 - c_s^2 j relaxes at
    omega_7 toward 0 and goes back to raw with + c_s^2 j; kappa_22 - c_s^4 rho = w - c_s^4 r relaxes
    at omega_8 toward the linearised attractor: c_s^2 (a~ + b~) for the FP diffusion tensor
    D' = kappa~_ij / rho (kappa^Mv_22 = kappa~_20 kappa~_02 / rho), 0 for the Maxwellian (MCM)
    one.  Streaming moves the e_x = +-1 populations of both sums by one cell (factor exp(-+ i k)).
    Returns the complex 6x6 matrix of one step; its eigenvalue pair of largest modulus is the
    sound mode."""
    k = 2 * math.pi / n
    w3, w4, w7, w8 = (float(omega[i]) for i in (3, 4, 7, 8))

    def collide(x):
        r, j, p, q, s, w = x
        a, b = p - CS2 * r, q - CS2 * r
        bulk, dev = (1 - w3) * (a + b), (1 - w4) * (a - b)
        at, bt = (bulk + dev) / 2, (bulk - dev) / 2
        w0 = w - CS2 * CS2 * r
        att = 0.0 if mcm else CS2 * bulk
        return np.array([r, j, CS2 * r + at, CS2 * r + bt, (1 - w7) * (s - CS2 * j) + CS2 * j,
                         CS2 * CS2 * r + w0 + w8 * (att - w0)], dtype=complex)

    def stream(x):
        r, j, p, q, s, w = x
        ph = {e: np.exp(-1j * k * e) for e in (-1, 0, 1)}
        a = {0: ph[0] * (r - p), 1: ph[1] * (p + j) / 2, -1: ph[-1] * (p - j) / 2}
        b = {0: ph[0] * (q - w), 1: ph[1] * (w + s) / 2, -1: ph[-1] * (w - s) / 2}
        return np.array([a[0] + a[1] + a[-1], a[1] - a[-1], a[1] + a[-1],
                         b[0] + b[1] + b[-1], b[1] - b[-1], b[1] + b[-1]])

    eye = np.eye(6)
    C = np.stack([collide(eye[i]) for i in range(6)], axis=1)
    S = np.stack([stream(eye[i]) for i in range(6)], axis=1)
    return S @ C


def prony_pair(xs):
    """(p, q) of the recurrence x(t+2) = p x(t+1) - q x(t) that a complex-conjugate eigenvalue
    pair lambda, lambda* gives (p = 2 Re lambda, q = |lambda|^2), least squares over a series."""
    xs = np.asarray(xs)
    A = np.stack([np.concatenate([xs[1:-1].real, xs[1:-1].imag]),
                  -np.concatenate([xs[:-2].real, xs[:-2].imag])], axis=1)
    b = np.concatenate([xs[2:].real, xs[2:].imag])
    (p, q), *_ = np.linalg.lstsq(A, b, rcond=None)
    return float(p), float(q)


def sound_wave_step_matrix_3d(n, omega, mcm=False):
    """Linearised D3Q27 step of a plane sound wave along x (rho and u_x vary with x only), for the
    Fourier mode exp(i k x), k = 2 pi / n (von Neumann analysis of collide-and-stream).

    Sum the populations over (e_y, e_z) with the weights 1, e_y^2 (equal to the e_z^2 sum by
    symmetry) and e_y^2 e_z^2: the nine moments m_000 = rho, m_100 = j, m_200; m_020, m_120, m_220;
    m_022, m_122, m_222 of those three sums evolve on their own.  State: their deviations
    (r, j, p, q, s, w, v, t, z) from the rest values (1, 0, c_s^2, c_s^2, 0, c_s^4, c_s^4, 0, c_s^6).
    Collision, to first order around rest (u = j), in the chain order of Step 3:
      * kappa_200 and kappa_020 = kappa_002 differ from c_s^2 rho by a = p - c_s^2 r, b = q - c_s^2 r;
        the bulk part a + 2b relaxes at omega_7 and the deviatoric part a - b at omega_8 = omega_9,
        both toward 0, giving a~, b~;
      * kappa_120 = m_120 - c_s^2 j relaxes at omega_10 toward 0 (raw again: + c_s^2 j);
      * kappa_220 - c_s^4 rho = w - c_s^4 r and kappa_022 - c_s^4 rho = v - c_s^4 r relax at omega_17
        toward kappa~_200 kappa~_020 / rho and kappa~_020 kappa~_002 / rho, linearised
        c_s^2 (a~ + b~) and 2 c_s^2 b~ (FP diffusion tensor, post-collision second moments);
      * kappa_122 = m_122 - c_s^4 j relaxes at omega_23 toward
        (2 / 5 rho)(kappa~_020 kappa~_102 + kappa~_002 kappa~_120), linearised (4/5) c_s^2 kappa~_120;
      * kappa_222 - c_s^6 rho relaxes at omega_26 toward
        (1 / 3 rho)(kappa~_200 kappa~_022 + kappa~_020 kappa~_202 + kappa~_002 kappa~_220), linearised
        (c_s^4 (a~ + 2 b~) + c_s^2 (e~ + 2 d~)) / 3 with d~, e~ the post-collision deviations of
        kappa_220 and kappa_022;
    every attractor above second order is 0 (its Maxwellian value, relative to rest) for MCM.
    Streaming moves the e_x = +-1 populations of the three sums by one cell (factor exp(-+ i k)).
    The last three moments are driven by the first six without feeding back, so the sound mode
    (the eigenvalue pair of largest modulus) does not depend on the fifth- and sixth-order
    attractors; one step of the full matrix does.  All rates of one order must be equal (as
    set_params makes them): the plane wave does not see the grouping inside an order above the
    second.  Returns the complex 9x9 matrix of one step."""
    k = 2 * math.pi / n
    wb, ws, r3, r4, r5, r6 = (float(omega[i]) for i in (7, 8, 10, 17, 23, 26))
    c2, c4, c6 = CS2, CS2 ** 2, CS2 ** 3

    def collide(x):
        r, j, p, q, s, w, v, t, z = x
        a, b = p - c2 * r, q - c2 * r
        bulk, dev = (1 - wb) * (a + 2 * b), (1 - ws) * (a - b)
        at, bt = (bulk + 2 * dev) / 3, (bulk - dev) / 3
        k120 = (1 - r3) * (s - c2 * j)
        d, e = w - c4 * r, v - c4 * r
        dt = d + r4 * ((0.0 if mcm else c2 * (at + bt)) - d)
        et = e + r4 * ((0.0 if mcm else 2 * c2 * bt) - e)
        k122 = t - c4 * j
        k122 = k122 + r5 * ((0.0 if mcm else 0.8 * c2 * k120) - k122)
        g = z - c6 * r
        g = g + r6 * ((0.0 if mcm else (c4 * (at + 2 * bt) + c2 * (et + 2 * dt)) / 3) - g)
        return np.array([r, j, c2 * r + at, c2 * r + bt, k120 + c2 * j, c4 * r + dt, c4 * r + et,
                         k122 + c4 * j, c6 * r + g], dtype=complex)

    def stream(x):
        ph = {e: np.exp(-1j * k * e) for e in (-1, 0, 1)}
        out = []
        for m0, m1, m2 in ((x[0], x[1], x[2]), (x[3], x[4], x[5]), (x[6], x[7], x[8])):
            a = {0: ph[0] * (m0 - m2), 1: ph[1] * (m2 + m1) / 2, -1: ph[-1] * (m2 - m1) / 2}
            out += [a[0] + a[1] + a[-1], a[1] - a[-1], a[1] + a[-1]]
        return np.array(out)

    eye = np.eye(9)
    C = np.stack([collide(eye[i]) for i in range(9)], axis=1)
    S = np.stack([stream(eye[i]) for i in range(9)], axis=1)
    return S @ C


# (e_x, e_y, e_z) exponents of the nine moments of sound_wave_step_matrix_3d, in its state order
SOUND_WAVE_MOMENTS_3D = [(a, b, c) for (b, c) in ((0, 0), (2, 0), (2, 2)) for a in (0, 1, 2)]


def crossing_shear_wave_step_matrix(kx, kz, omega, mcm=False):
    """Linearised D3Q27 step of a small flow u_y(x, z) (no variation along y, rho = 1), for the
    Fourier mode exp(i (kx x + kz z)); the crossing shear waves u_y = U cos(k x) cos(k z) of the
    hyperviscosity study (Sec. 4) are four such modes with the same matrix up to mirror symmetry.

    Weight the populations by e_y and sum over e_y: the nine raw moments m_a1c (a, c in 0..2) of
    that y-odd part evolve on their own.  Collision, to first order around rest (u_y = m_010), with
    central kappa_a1c = m_a1c - u_y m_a0c and the rest values m_000 = 1, m_200 = m_002 = c_s^2,
    m_202 = c_s^4:
      * kappa_110, kappa_011 relax at the shear rate omega_4 = omega_6 toward 0;
      * kappa_210, kappa_012, kappa_111 relax at the third-order rate toward 0;
      * kappa_211, kappa_112 relax at the fourth-order rate toward kappa~_200 kappa~_011 / rho and
        kappa~_002 kappa~_110 / rho, linearised c_s^2 kappa~_011 and c_s^2 kappa~_110 (FP diffusion
        tensor, post-collision second moments), 0 for the Maxwellian (MCM) attractors;
      * kappa_212 relaxes at the fifth-order rate toward
        (2 / 5 rho)(kappa~_200 kappa~_012 + kappa~_002 kappa~_210), linearised
        (2/5) c_s^2 (kappa~_012 + kappa~_210), 0 for MCM;
    and back with m_a1c = kappa~_a1c + u_y m_a0c.  Streaming moves the (e_x, e_z) populations of the
    y-odd part by (e_x, e_z): a factor exp(-i (kx e_x + kz e_z)).  The fourth-order attractors are
    where FP and MCM differ for this flow: with the Maxwellian ones the wave loses amplitude far
    faster than exp(-nu (kx^2 + kz^2) t), the hyperviscosity the paper reports for MCM.  Returns
    the complex 9x9 matrix of one step on the state m_a1c flattened as [a][c]."""
    c2, c4 = CS2, CS2 * CS2
    w, r3, r4, r5 = (float(omega[i]) for i in (4, 10, 17, 23))

    def collide(m):
        m = m.reshape(3, 3)
        u = m[0, 0]
        t110, t011 = (1 - w) * m[1, 0], (1 - w) * m[0, 1]
        t210, t012, t111 = (1 - r3) * (m[2, 0] - c2 * u), (1 - r3) * (m[0, 2] - c2 * u), (1 - r3) * m[1, 1]
        t211 = m[2, 1] + r4 * ((0.0 if mcm else c2 * t011) - m[2, 1])
        t112 = m[1, 2] + r4 * ((0.0 if mcm else c2 * t110) - m[1, 2])
        k212 = m[2, 2] - c4 * u
        t212 = k212 + r5 * ((0.0 if mcm else 0.4 * c2 * (t012 + t210)) - k212)
        return np.array([[u, t011, t012 + c2 * u], [t110, t111, t112], [t210 + c2 * u, t211, t212 + c4 * u]],
                        dtype=complex).reshape(-1)

    es = (0, 1, -1)
    to_values = np.array([[1, 0, -1], [0, 0.5, 0.5], [0, -0.5, 0.5]])  # e = 0, +1, -1 from (m0, m1, m2)
    to_moments = np.array([[1, 1, 1], [0, 1, -1], [0, 1, 1]])         # (m0, m1, m2) from e = 0, +1, -1
    shift = np.array([[np.exp(-1j * (kx * ex + kz * ez)) for ez in es] for ex in es])

    def stream(m):
        h = to_values @ m.reshape(3, 3) @ to_values.T
        return (to_moments @ (h * shift) @ to_moments.T).reshape(-1)

    eye = np.eye(9)
    C = np.stack([collide(eye[i]) for i in range(9)], axis=1)
    S = np.stack([stream(eye[i].astype(complex)) for i in range(9)], axis=1)
    return S @ C
