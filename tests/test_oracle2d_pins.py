"""Pins of the D2Q9 FP64 oracle (Sec. 2 and the appendix on the 2D algorithm) against what the
paper and the mathematics fix: the printed Step 1 raw moments, rest weights, conservation,
equilibrium invariance, the printed fourth-order attractor and source list, the MCM special case
(a single-rate relaxation to the equilibrium), and the transport coefficients of
Eq. (transportcoeff2DFPCLBM) from decaying shear and sound waves."""
import math
import os

import numpy as np
import pytest

from dispersion import prony_pair, shear_wave_discrete_rate, sound_wave_step_matrix_2d
from oracle import oracle2d as O2

HERE = os.path.dirname(os.path.abspath(__file__))
CS2 = 1.0 / 3.0
E = O2.velocity_set()
MN = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (2, 1), (1, 2), (2, 2)]


def rand_f(seed, spread=0.5):
    rng = np.random.default_rng(seed)
    w = O2.equilibrium(1.0, (0, 0))
    return w * (1 + spread * rng.uniform(-1, 1, 9))


def fields(f, F=(0, 0)):
    rho = f.sum()
    return rho, (f @ E + 0.5 * np.asarray(F)) / rho


def central(f, u):
    return O2.central_matrix(u) @ f


def test_step1_raw_moments_match_printed_rows():
    P = O2.central_matrix((0.0, 0.0))
    rows = {}
    for line in open(os.path.join(HERE, "golden", "appendix_2d_step1_raw_moments.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, *c = line.split()
        rows[(int(name[0]), int(name[1]))] = np.array([float(v) for v in c])
    assert len(rows) == 9
    for i, mn in enumerate(MN):
        assert np.array_equal(P[i], rows[mn]), mn


def test_rest_weights():
    w = O2.equilibrium(1.0, (0.0, 0.0))
    assert np.allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=0, atol=4e-16)  # LU round-off (1 ulp of 4/9)


@pytest.mark.parametrize("mode", [0, 1])
def test_collision_conserves_mass_and_adds_force(mode):
    rng = np.random.default_rng(3)
    for s in range(5):
        f = rand_f(s)
        F = rng.uniform(-3e-3, 3e-3, 2)
        om = rng.uniform(0.3, 1.9, 9)
        ft = O2.collide(f, F, om, mode)
        assert abs(ft.sum() - f.sum()) < 1e-15
        assert np.allclose(ft @ E, f @ E + F, rtol=0, atol=1e-15)


@pytest.mark.parametrize("mode", [0, 1])
def test_equilibrium_is_invariant(mode):
    rng = np.random.default_rng(4)
    for _ in range(5):
        rho, u = 1 + 0.1 * rng.uniform(-1, 1), 0.1 * rng.uniform(-1, 1, 2)
        feq = O2.equilibrium(rho, u)
        ft = O2.collide(feq, (0, 0), rng.uniform(0.2, 1.9, 9), mode)
        assert np.max(np.abs(ft - feq)) < 1e-15


def test_fourth_order_attractor_is_the_printed_form():
    """Boxed kappa_22^Mv = (k~20 k~02 + 2 k~11^2) / rho (Sec. 2) from the generic formula with
    D' = k~_ij / rho and the post-collision second moments as lower moments."""
    rng = np.random.default_rng(8)
    for _ in range(5):
        rho = 1 + 0.1 * rng.uniform(-1, 1)
        k20, k02, k11 = CS2 * rho + 0.01 * rng.normal(), CS2 * rho + 0.01 * rng.normal(), 0.01 * rng.normal()
        Pi = np.zeros((3, 3))
        Pi[0, 0], Pi[2, 0], Pi[0, 2], Pi[1, 1] = rho, k20, k02, k11
        D = (k20 / rho, k02 / rho, k11 / rho)
        got = O2.attractor_generic(2, 2, Pi, D)
        assert got == pytest.approx((k20 * k02 + 2 * k11 * k11) / rho, rel=1e-14)
        assert O2.attractor_generic(2, 1, Pi, D) == 0.0 and O2.attractor_generic(1, 2, Pi, D) == 0.0


def test_chain_uses_post_collision_second_moments():
    """With omega_8 = 1 the post-collision k~22 equals its attractor built from the relaxed
    second moments (not the pre-collision ones)."""
    f = rand_f(11, spread=0.8)
    om = np.ones(9)
    om[3], om[4], om[5] = 0.7, 1.3, 1.6
    ft = O2.collide(f, (0, 0), om, 0)
    rho, u = fields(f)
    kt = central(ft, u)
    k20, k02, k11 = kt[3], kt[4], kt[5]
    assert kt[8] == pytest.approx((k20 * k02 + 2 * k11 * k11) / rho, rel=1e-13)
    k = central(f, u)
    assert abs(kt[8] - (k[3] * k[4] + 2 * k[5] ** 2) / rho) > 1e-6


def test_sources_with_zero_rates_match_printed_list():
    """Eq. (sourceCM2D): with every rate 0, C(u)(f~ - f) = sigma: sigma_10 = Fx, sigma_01 = Fy,
    second order 0, sigma_21 = 2 Fx/rho k11 + Fy/rho k20, sigma_12 = Fx/rho k02 + 2 Fy/rho k11
    (Eq. forcing:2D; the printed sigma_12 carries the factor 1 on its Fy term, reading G19),
    sigma_22 = 2 (Fx/rho k12 + Fy/rho k21)."""
    f = rand_f(5, spread=0.8)
    F = np.array([3e-3, -2e-3])
    rho, u = fields(f, F)
    ft = O2.collide(f, F, np.zeros(9), 0)
    sig = O2.central_matrix(u) @ (ft - f)
    k = central(f, u)
    fx, fy = F / rho
    tol = 1e-14
    assert abs(sig[1] - F[0]) < tol and abs(sig[2] - F[1]) < tol
    assert max(abs(sig[3]), abs(sig[4]), abs(sig[5])) < tol
    assert abs(sig[6] - (2 * fx * k[5] + fy * k[3])) < tol
    assert abs(sig[7] - (fx * k[4] + 2 * fy * k[5])) < tol
    assert abs(sig[8] - 2 * (fx * k[7] + fy * k[6])) < tol
    assert abs(sig[6]) > 1e-5


def test_mcm_with_equal_rates_is_single_relaxation():
    """Relaxing every central moment at one rate omega toward the Maxwellian moments is linear:
    f~ = f + omega (f^eq(rho, u) - f) (no force)."""
    for s in range(4):
        f = rand_f(20 + s, spread=0.6)
        rho, u = fields(f)
        w = 0.4 + 0.3 * s
        ft = O2.collide(f, (0, 0), np.full(9, w), 1)
        assert np.max(np.abs(ft - (f + w * (O2.equilibrium(rho, u) - f)))) < 1e-15


def test_fp_differs_from_mcm_off_equilibrium():
    f = rand_f(30, spread=0.8)
    om = O2.rates(0.6)
    assert np.max(np.abs(O2.collide(f, (0, 0), om, 0) - O2.collide(f, (0, 0), om, 1))) > 1e-5


def _decay_rate(vals, ts):
    return -np.polyfit(ts, np.log(vals), 1)[0]


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_shear_wave_viscosity(tau):
    """u_x = U sin(k y) decays at nu k^2, nu = cs^2 (1/omega_2d - 1/2)."""
    n = 32
    k = 2 * math.pi / n
    y = np.arange(n)
    ux = 1e-4 * np.sin(k * y)[:, None] * np.ones((1, 2))
    f = O2.init_equilibrium(np.ones((n, 2)), ux, np.zeros((n, 2)))
    om = O2.rates(tau)
    amps, ts, t = [], [], 0
    for _ in range(12):
        f = O2.run(f, 10, omega=om)
        t += 10
        _, u, _ = O2.moments(f)
        amps.append(2 / n * u[:, 0] @ np.sin(k * y))
        ts.append(t)
    nu = CS2 * (tau - 0.5)
    assert abs(_decay_rate(amps, ts) / (nu * k * k) - 1) < 0.01


@pytest.mark.parametrize("tau,bulk,drift", [(0.6, 0.0, 0.0), (1.0, 0.0, 0.0), (0.6, 0.0, 0.3), (0.7, 1.5, 0.2)])
def test_shear_wave_decay_matches_discrete_dispersion(tau, bulk, drift):
    """The 2D shear wave decays exactly as the scheme's discrete dispersion relation says (the same
    3x3 map of j, m_11, m_12 as in 3D: shear rates omega_4 = omega_5 = 1/tau, third-order rates
    omega_6 = omega_7 = 1 or 3 drift), whatever the bulk rate."""
    om = O2.rates(tau, bulk, drift)
    for n in (16, 32):
        k = 2 * math.pi / n
        y = np.arange(n)
        ux = 1e-4 * np.sin(k * y)[:, None] * np.ones((1, 2))
        f = O2.init_equilibrium(np.ones((n, 2)), ux, np.zeros((n, 2)))
        chunk = 20 * (n // 16) ** 2
        amps, ts = [], []
        for i in range(16):
            f = O2.run(f, chunk, omega=om)
            if i >= 3:  # past the decay of the non-hydrodynamic modes
                _, u, _ = O2.moments(f)
                amps.append(2 / n * u[:, 0] @ np.sin(k * y))
                ts.append(chunk * (i + 1))
        rate = _decay_rate(np.abs(amps), ts)
        exact = shear_wave_discrete_rate(n, tau, float(om[6]))
        assert abs(rate / exact - 1) < 5e-8, (n, rate, exact)


@pytest.mark.parametrize("tau,bulk,drift,mode", [(0.8, 0.0, 0.0, 0), (0.8, 0.5, 0.0, 0), (0.8, 1.6, 0.0, 0),
                                              (0.6, 0.5, 0.3, 0), (0.8, 0.5, 0.0, 1)])
def test_sound_wave_matches_discrete_dispersion(tau, bulk, drift, mode):
    """A plane sound wave rho = 1 + eps cos(k x) evolves with the acoustic eigenvalue pair of the
    scheme's linearised step (dispersion.sound_wave_step_matrix_2d): sound speed, shear and bulk
    rates (Eq. transportcoeff2DFPCLBM), third- and fourth-order rates and the fourth-order
    attractor (Eq. Mvcmattractor2D with the diffusion tensor of Sec. 2) all enter.  Measured by a
    Prony fit of the density's Fourier coefficient once the non-hydrodynamic modes have died out.
    With a bulk rate other than 1 the FP and MCM attractors give different eigenvalues, and the
    fit must pick the one of the mode that ran."""
    om = O2.rates(tau, bulk, drift)
    for n in (16, 32):
        k = 2 * math.pi / n
        x = np.arange(n)
        rho = (1 + 1e-5 * np.cos(k * x))[None, :] * np.ones((2, 1))
        f = O2.init_equilibrium(rho, np.zeros((2, n)), np.zeros((2, n)))
        xs = []
        for t in range(400):
            f = O2.step(f, omega=om, mode=mode)
            if t >= 60:
                r, _, _ = O2.moments(f)
                xs.append(np.mean((r[0] - 1) * np.exp(-1j * k * x)))
        p, q = prony_pair(xs)
        lam = np.linalg.eigvals(sound_wave_step_matrix_2d(n, om, mcm=(mode == 1)))
        lam = lam[np.argmax(np.abs(lam))]
        assert abs(p - 2 * lam.real) < 1e-8 and abs(q - abs(lam) ** 2) < 1e-8, (n, p, q, lam)
        other = np.linalg.eigvals(sound_wave_step_matrix_2d(n, om, mcm=(mode != 1)))
        other = other[np.argmax(np.abs(other))]
        if bulk not in (0.0, 1.0) and n == 16:
            assert abs(q - abs(other) ** 2) > 1e-6


@pytest.mark.parametrize("bulk", [0.5, 1.0, 1.6])
def test_sound_wave_bulk_viscosity(bulk):
    """A standing acoustic wave loses energy at k^2 (nu + zeta), zeta = cs^2 (1/omega_2s - 1/2)
    (Eq. transportcoeff2DFPCLBM; the 2D longitudinal viscosity is nu + zeta)."""
    n, tau = 32, 0.8
    k = 2 * math.pi / n
    x = np.arange(n)
    rho = (1 + 1e-5 * np.sin(k * x))[None, :] * np.ones((2, 1))
    f = O2.init_equilibrium(rho, np.zeros((2, n)), np.zeros((2, n)))
    om = O2.rates(tau, bulk)
    s, c = np.sin(k * x), np.cos(k * x)
    en, ts, t = [], [], 0
    for i in range(60):
        f = O2.run(f, 5, omega=om)
        t += 5
        r, u, _ = O2.moments(f)
        dr, v = r[0] - 1.0, u[0]
        rs, rc = 2 / n * dr @ s, 2 / n * dr @ c
        vs, vc = 2 / n * v @ s, 2 / n * v @ c
        if i >= 4:
            en.append(CS2 * (rs * rs + rc * rc) + (vs * vs + vc * vc))
            ts.append(t)
    nu, zeta = CS2 * (tau - 0.5), CS2 * (1 / bulk - 0.5)
    assert abs(_decay_rate(en, ts) / (k * k * (nu + zeta)) - 1) < 0.02


def test_streaming_moves_each_population_along_its_link():
    nx, ny = 5, 4
    f = np.zeros((9, ny, nx))
    f[:, 1, 2] = O2.equilibrium(1.0, (0, 0))
    rest = np.broadcast_to(O2.equilibrium(1.0, (0, 0))[:, None, None], f.shape).copy()
    rest[:, 1, 2] = 0
    f = f + rest
    out = O2.step(f, omega=np.ones(9))
    for a in range(9):
        assert out[a, (1 + E[a, 1]) % ny, (2 + E[a, 0]) % nx] == pytest.approx(f[a, 1, 2], abs=1e-16)


@pytest.mark.parametrize("uw", [0.0, 0.07])
def test_box_one_step_from_uniform_flow(uw):
    """Closed box with a moving lid (2D cavity, Sec. 4): from a uniform equilibrium only the links
    leaving the box change, f_opp(a)(x) = feq_a - 2 w_a rho e_ax uw / cs^2 (correction only through
    the row y = ny, corners included)."""
    nx, ny = 5, 4
    u = (0.03, -0.02)
    one = np.ones((ny, nx))
    feq = O2.equilibrium(1.0, u)
    w = O2.equilibrium(1.0, (0, 0))
    got = O2.step(O2.init_equilibrium(one, u[0] * one, u[1] * one), omega=O2.rates(0.8), bc=O2.BC_BOX, uw=uw)
    exp = np.broadcast_to(feq[:, None, None], got.shape).copy()
    opp = [int(np.where((E == -E[a]).all(axis=1))[0][0]) for a in range(9)]
    for y in range(ny):
        for x in range(nx):
            for a in range(9):
                xd, yd = x + E[a, 0], y + E[a, 1]
                if xd < 0 or xd >= nx or yd < 0 or yd >= ny:
                    v = feq[a]
                    if yd == ny:
                        v -= 2 * w[a] * E[a, 0] * uw / CS2
                    exp[opp[a], y, x] = v
    assert np.max(np.abs(got - exp)) <= 1e-15


def test_cavity_conserves_mass_and_rejects_bad_boundaries():
    n = 6
    one = np.ones((n, n))
    f0 = O2.init_equilibrium(one, 0 * one, 0 * one)
    f = O2.run(f0, 50, omega=O2.rates(0.6), bc=O2.BC_BOX, uw=0.1)
    assert abs(f.sum() - f0.sum()) <= 1e-12 * f0.sum()
    _, ux, _ = O2.moments(f)
    assert ux[-1].mean() > 0.01  # the lid drags the top row
    with pytest.raises(ValueError):
        O2.step(f0, bc=O2.BC_PERIODIC, uw=0.1)
    with pytest.raises(ValueError):
        O2.step(f0, bc=1)
