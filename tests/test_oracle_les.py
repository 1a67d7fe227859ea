"""Pins of the oracle's half channel (specular symmetry plane) and of the Smagorinsky model with
van Driest damping (Sec. 4, turbulent channel LES).

* The half channel must reproduce, to rounding, the lower half of a full channel of twice the
  height started from a mirror-symmetric state: specular reflection at the mid plane is exactly
  what the mirror image supplies there.
* The Smagorinsky relaxation time is pinned by a known-answer construction: populations whose
  non-equilibrium second moments are those of a chosen strain rate S at the relaxation time
  tau* = tau0 + (C_s D)^2 |S| / cs^2 must give back tau*.
"""
import numpy as np
import pytest

import oracle as O

E = O.velocity_set()
MIR = [int(np.where((E == E[a] * np.array([1, -1, 1])).all(axis=1))[0][0]) for a in range(27)]
MNP = [tuple(v) for v in O.moment_exponents()]
CS2 = 1.0 / 3.0


def near_eq(nx, ny, nz, seed, amp=0.05, noise=0.02):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.02 * rng.uniform(-1, 1, (nz, ny, nx))
    u = [amp * rng.uniform(-1, 1, (nz, ny, nx)) for _ in range(3)]
    f = O.init_equilibrium(rho, *u)
    return f * (1 + noise * rng.uniform(-1, 1, f.shape))


def mirrored_full(f_half):
    _, nz, ny, nx = f_half.shape
    full = np.empty((27, nz, 2 * ny, nx))
    full[:, :, :ny] = f_half
    for a in range(27):
        full[a, :, ny:] = f_half[MIR[a], :, ::-1]
    return full


@pytest.mark.parametrize("mode,drift", [(O.EQ_MODE_FP, 0.3), (O.EQ_MODE_MCM, 0.0), (O.EQ_MODE_FP, 0.0)])
@pytest.mark.parametrize("les", [None, (0.17, 0.01, 26.0)])
def test_half_channel_is_the_lower_half_of_a_mirrored_channel(mode, drift, les):
    nx, ny, nz = 4, 3, 5
    f_half = near_eq(nx, ny, nz, seed=11)
    Fv = (3e-4, 0.0, -2e-4)
    om = O.rates(0.62, drift)
    half = O.run(f_half, 5, bc=O.BC_HALF_CHANNEL, F=Fv, omega=om, mode=mode, les=les)
    full = O.run(mirrored_full(f_half), 5, bc=O.BC_WALLS_Y, F=Fv, omega=om, mode=mode, les=les)
    assert np.max(np.abs(half - full[:, :, :ny])) <= 1e-14
    # and the upper half stays the mirror image
    assert np.max(np.abs(mirrored_full(half) - full)) <= 1e-14


def test_half_channel_specular_link_closed_form():
    """From a uniform equilibrium, a population leaving the top row along (ex, +1, ez) arrives
    along (ex, -1, ez) in the top row at x + ex, z + ez (periodic); the wall rows bounce back."""
    nx, ny, nz = 3, 2, 4
    u = (0.03, 0.0, -0.02)  # no normal velocity: the uniform state is compatible with both boundaries
    one = np.ones((nz, ny, nx))
    feq = O.equilibrium(1.0, u)
    got = O.step(O.init_equilibrium(one, u[0] * one, u[1] * one, u[2] * one), bc=O.BC_HALF_CHANNEL,
                 omega=O.rates(0.7))
    exp = np.broadcast_to(feq[:, None, None, None], got.shape).copy()
    opp = [int(np.where((E == -E[a]).all(axis=1))[0][0]) for a in range(27)]
    for a in range(27):
        if E[a, 1] == -1:
            exp[opp[a], :, 0, :] = feq[a]          # bounce-back at y = -1/2
        if E[a, 1] == 1:
            exp[MIR[a], :, ny - 1, :] = feq[a]     # specular at y = ny - 1/2 (uniform: shift invisible)
    assert np.max(np.abs(got - exp)) <= 1e-15
    # the shift itself: a marked population in one top cell moves to (x + ex, z + ez)
    f0 = O.init_equilibrium(one, 0 * one, 0 * one, 0 * one)
    a = int(np.where((E == [1, 1, 1]).all(axis=1))[0][0])
    out = O.step(f0, bc=O.BC_HALF_CHANNEL, omega=np.ones(27) * 1.0)
    rest = out.copy()
    f1 = f0.copy()
    f1[:, 2, ny - 1, 1] = O.equilibrium(1.0, (0.02, 0.0, 0.01))  # perturb one top cell at x=1, z=2
    out1 = O.step(f1, bc=O.BC_HALF_CHANNEL, omega=np.ones(27))
    diff = np.abs(out1 - rest)[MIR[a], :, ny - 1, :]
    assert diff[3 % nz, 2] > 1e-6  # arrived at x = 1 + 1, z = 2 + 1
    assert np.sum(diff > 1e-12) == 1


def central_state(rho, u, Pi):
    """Populations with central moments rho, 0, cs^2 rho delta + Pi (second order), Maxwellian above."""
    M = O.maxwell_moments(rho)
    kap = np.array([M[m, n, p] for (m, n, p) in MNP])
    for (i, j), v in np.ndenumerate(Pi):
        e = [0, 0, 0]
        e[i] += 1
        e[j] += 1
        k = MNP.index(tuple(e))
        if i <= j:
            kap[k] += v
    return np.linalg.solve(O.central_matrix(u), kap)


def random_strain(seed, scale=1e-3):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(3, 3)) * scale
    S = 0.5 * (A + A.T)
    return S - np.trace(S) / 3 * np.eye(3)


@pytest.mark.parametrize("seed", range(5))
def test_smagorinsky_tau_known_answer(seed):
    rng = np.random.default_rng(100 + seed)
    rho, u = 1 + 0.05 * rng.uniform(-1, 1), 0.05 * rng.uniform(-1, 1, 3)
    tau0, c2 = rng.uniform(0.501, 0.8), rng.uniform(0.0, 0.05)
    S = random_strain(seed)
    tau_star = tau0 + c2 * np.sqrt(2 * np.sum(S * S)) / CS2
    Pi = -2 * rho * CS2 * tau_star * S
    f = central_state(rho, u, Pi)
    assert O.smagorinsky_tau(f, (0, 0, 0), tau0, c2) == pytest.approx(tau_star, rel=1e-13)
    # an isotropic part of the non-equilibrium moments belongs to the bulk rate: no effect
    f_iso = central_state(rho, u, Pi + 3e-4 * np.eye(3))
    assert O.smagorinsky_tau(f_iso, (0, 0, 0), tau0, c2) == pytest.approx(tau_star, rel=1e-13)
    # and the closed-form root of tau^2 - tau0 tau - c2 |Pi| / (2 rho cs^4) = 0
    Pn = np.sqrt(2 * np.sum(Pi * Pi))
    assert tau_star == pytest.approx(0.5 * (tau0 + np.sqrt(tau0**2 + 2 * c2 * Pn / (rho * CS2 * CS2))), rel=1e-13)
    assert O.smagorinsky_tau(f, (0, 0, 0), tau0, 0.0) == tau0


def test_les_without_model_constant_is_the_plain_step():
    f = near_eq(5, 4, 3, seed=3)
    om = O.rates(0.56)
    a = O.step(f, bc=O.BC_WALLS_Y, F=(1e-4, 0, 0), omega=om)
    b = O.step(f, bc=O.BC_WALLS_Y, F=(1e-4, 0, 0), omega=om, les=(0.0, 0.01, 26.0))
    assert np.max(np.abs(a - b)) <= 1e-15


def test_van_driest_damping_per_row():
    """Uniform sheared state in a channel: each interior population arrives from row y - e_y, so it
    carries the relaxation time of that row, tau*(y) from (C_s D(y))^2 with
    D = 1 - exp(-y+ / A+), y+ = (distance of the row centre to the nearest wall) u* / nu."""
    nx, ny, nz = 2, 8, 2
    tau0, Cs, ustar, Aplus = 0.52, 0.17, 0.02, 26.0
    nu = CS2 * (tau0 - 0.5)
    S = random_strain(7, scale=5e-3)
    rho, u = 1.0, np.array([0.02, 0.0, 0.01])

    def tau_row(y):
        yw = min(y + 0.5, ny - 0.5 - y)
        c2 = (Cs * (1 - np.exp(-yw * ustar / nu / Aplus))) ** 2
        # self-consistent state for this row's tau is not needed: tau*(y) is the root for the given Pi
        Pn = np.sqrt(2 * np.sum(Pi * Pi))
        return 0.5 * (tau0 + np.sqrt(tau0**2 + 2 * c2 * Pn / (rho * CS2 * CS2)))

    Pi = -2 * rho * CS2 * tau0 * S
    fc = central_state(rho, u, Pi)
    f = np.broadcast_to(fc[:, None, None, None], (27, nz, ny, nx)).copy()
    om = O.rates(tau0)
    got = O.step(f, bc=O.BC_WALLS_Y, omega=om, les=(Cs, ustar, Aplus))
    for y in range(1, ny - 1):
        for a in range(27):
            ys = y - E[a, 1]
            o = om.copy()
            o[[4, 5, 6, 8, 9]] = 1.0 / tau_row(ys)
            want = O.collide(fc, (0, 0, 0), o)[a]
            assert abs(got[a, 0, y, 0] - want) <= 1e-15, (y, a)
