"""Pins of the oracle's wall boundaries: half-way bounce-back on the y walls and on all six faces
of a closed box, and the moving-wall momentum correction of the wall y = ny - 1/2 (Sec. 4, cubic
cavity).  Each pin is a closed form or a symmetry that a dropped term, a wrong sign, a wrong
factor or a transposed axis in the oracle's streaming would break.
"""
import numpy as np
import pytest

import oracle as O

E = O.velocity_set()
OPP = [int(np.where((E == -E[a]).all(axis=1))[0][0]) for a in range(27)]
W = O.equilibrium(1.0, (0.0, 0.0, 0.0))


def uniform(nx, ny, nz, u):
    one = np.ones((nz, ny, nx))
    return O.init_equilibrium(one, u[0] * one, u[1] * one, u[2] * one)


@pytest.mark.parametrize("lid", [(0.0, 0.0, 0.0), (0.04, 0.0, -0.03)])
def test_box_one_step_from_uniform_flow(lid):
    """A uniform equilibrium is a fixed point of collision (invariance pinned elsewhere) and of
    periodic streaming, so after one step in a closed box only the reflected links differ:
    f_opp(a)(x) = feq_a - 2 w_a rho (e_a . uw) / cs^2 (correction only through the layer y = ny),
    for every link a whose destination x + e_a is outside the box on any axis."""
    nx, ny, nz = 4, 3, 5
    u = np.array([0.03, -0.02, 0.01])
    feq = O.equilibrium(1.0, u)
    f0 = uniform(nx, ny, nz, u)
    got = O.step(f0, bc=O.BC_BOX, omega=O.rates(0.8), uw=lid)
    exp = np.empty_like(f0)
    for a in range(27):
        exp[a] = feq[a]
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for a in range(27):
                    d = np.array([x, y, z]) + E[a]
                    if (d < 0).any() or (d >= (nx, ny, nz)).any():
                        v = feq[a]
                        if d[1] == ny:
                            v -= 2 * W[a] * 1.0 * (E[a] @ np.asarray(lid)) * 3.0
                        exp[OPP[a], z, y, x] = v
    assert np.max(np.abs(got - exp)) <= 1e-15


def test_walls_y_one_step_is_periodic_in_x_and_z():
    """bc = 1: the same closed form with walls only at y = -1/2, ny - 1/2 (x and z periodic)."""
    nx, ny, nz = 3, 4, 2
    u = np.array([0.02, 0.01, -0.03])
    feq = O.equilibrium(1.0, u)
    got = O.step(uniform(nx, ny, nz, u), bc=O.BC_WALLS_Y, omega=O.rates(0.7), uw=(0.05, 0, 0))
    exp = np.broadcast_to(feq[:, None, None, None], got.shape).copy()
    for a in range(27):
        if E[a, 1] == 1:
            exp[OPP[a], :, ny - 1, :] = feq[a] - 6 * W[a] * E[a, 0] * 0.05
        if E[a, 1] == -1:
            exp[OPP[a], :, 0, :] = feq[a]
    assert np.max(np.abs(got - exp)) <= 1e-15


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_couette_profile(tau):
    """Plane Couette flow (wall y = -1/2 at rest, wall y = ny - 1/2 moving at U along x): the
    steady profile is u_x = U (y + 1/2) / ny.  With unit higher-order rates the scheme reaches it
    up to an O(U^3) compressibility defect, exactly (round-off) at tau = 1."""
    ny = 8
    errs = []
    for U in (0.01, 0.002):
        f = O.run(uniform(1, ny, 1, (0, 0, 0)), 6000 if tau < 1 else 2500, bc=O.BC_WALLS_Y,
                  omega=O.rates(tau), uw=(U, 0, 0))
        rho, ux, uy, uz = O.moments(f)
        exact = U * (np.arange(ny) + 0.5) / ny
        errs.append(np.max(np.abs(ux[0, :, 0] - exact)))
        assert np.max(np.abs(uy)) <= 1e-13 and np.max(np.abs(uz)) <= 1e-13
        if tau == 1.0:
            assert errs[-1] <= 1e-14
    if tau != 1.0:
        # the defect is cubic in U: the linear (wall-correction) term is exact
        assert errs[0] / 0.01**3 == pytest.approx(errs[1] / 0.002**3, rel=1e-3)
        assert errs[1] / 0.002 <= 1e-6


def test_couette_along_z_is_the_transpose():
    """The lid velocity enters as e_a . uw: a lid along z gives the x <-> z mirror of a lid along x."""
    ny = 6
    fx = O.run(uniform(1, ny, 1, (0, 0, 0)), 200, bc=O.BC_WALLS_Y, omega=O.rates(0.9), uw=(0.03, 0, 0))
    fz = O.run(uniform(1, ny, 1, (0, 0, 0)), 200, bc=O.BC_WALLS_Y, omega=O.rates(0.9), uw=(0, 0, 0.03))
    _, ux, uy, uz = O.moments(fx)
    _, vx, vy, vz = O.moments(fz)
    assert np.max(np.abs(ux - vz)) <= 1e-15 and np.max(np.abs(uz - vx)) <= 1e-15
    assert np.max(np.abs(uy - vy)) <= 1e-15


def test_cavity_mass_and_symmetries():
    """Lid-driven closed box: mass is conserved exactly (the nine lid corrections of a top cell
    sum to zero), the flow is mirror-symmetric in z about the mid plane, and a lid along z gives
    the x <-> z transpose of a lid along x (same code path for the x and z walls)."""
    n = 5
    f0 = uniform(n, n, n, (0, 0, 0))
    om = O.rates(0.65)
    fx = O.run(f0, 40, bc=O.BC_BOX, omega=om, uw=(0.05, 0, 0))
    fz = O.run(f0, 40, bc=O.BC_BOX, omega=om, uw=(0, 0, 0.05))
    assert abs(fx.sum() - f0.sum()) <= 1e-12 * f0.sum()
    rho, ux, uy, uz = O.moments(fx)
    assert np.max(np.abs(ux)) > 1e-3  # the lid drove a flow
    assert np.max(np.abs(rho - rho[::-1])) <= 1e-14
    assert np.max(np.abs(ux - ux[::-1])) <= 1e-14 and np.max(np.abs(uz + uz[::-1])) <= 1e-14
    r2, vx, vy, vz = O.moments(fz)
    T = (2, 1, 0)  # [z, y, x] -> [x, y, z]
    assert np.max(np.abs(np.transpose(rho, T) - r2)) <= 1e-14
    assert np.max(np.abs(np.transpose(ux, T) - vz)) <= 1e-14
    assert np.max(np.abs(np.transpose(uz, T) - vx)) <= 1e-14
    assert np.max(np.abs(np.transpose(uy, T) - vy)) <= 1e-14


def test_closed_box_at_rest_stays_at_rest():
    f0 = uniform(3, 4, 5, (0, 0, 0))
    f = O.run(f0, 5, bc=O.BC_BOX, omega=O.rates(0.55))
    assert np.max(np.abs(f - f0)) <= 2e-15  # LU round-off of the collision


def test_bad_boundary_arguments_are_rejected():
    f0 = uniform(2, 2, 2, (0, 0, 0))
    with pytest.raises(ValueError):
        O.step(f0, bc=O.BC_WALLS_Y, uw=(0, 0.01, 0))  # normal wall velocity
    with pytest.raises(ValueError):
        O.step(f0, bc=O.BC_PERIODIC, uw=(0.01, 0, 0))  # no wall to move
    with pytest.raises(ValueError):
        O.step(f0, bc=4)
    with pytest.raises(ValueError):
        O.step(f0, bc=O.BC_HALF_CHANNEL, uw=(0.01, 0, 0))  # a symmetry plane does not move
