"""Pins of the FP64 closure oracle (oracle/closure.py) against closed forms and finite differences."""
import numpy as np
import pytest

from oracle import closure as C

CS2 = 1.0 / 3.0


def data(seed, B=64):
    rng = np.random.default_rng(seed)
    X = np.concatenate([rng.normal(scale=1e-3, size=(B, 6)), rng.normal(scale=0.05, size=(B, 3))], axis=1)
    t = rng.normal(scale=0.05, size=B)
    return X * 40.0, t  # O(0.1) inputs, as after input scaling


def test_parameter_count_and_layout():
    assert C.N_PARAMS == 4865
    th = np.arange(C.N_PARAMS, dtype=float)
    p = C.unpack(th)
    assert p["W1"].shape == (64, 9) and p["W1"][0, 0] == 0 and p["W1"][1, 0] == 9
    assert p["b1"][0] == 576 and p["W2"][0, 0] == 640 and p["b2"][0] == 4736
    assert p["W3"][0, 0] == 4800 and p["b3"][0] == 4864
    assert np.array_equal(C.pack(p), th)


def test_forward_closed_forms():
    th = np.zeros(C.N_PARAMS)
    p = C.unpack(th)
    p["b3"][0] = 0.25
    X, _ = data(0)
    y, _ = C.forward(C.pack(p), X)
    assert np.all(y == 0.25)
    # one path: W1[0,0] = a, W2[0,0] = b, W3[0,0] = c: y = c tanh(b tanh(a x0))
    p["W1"][0, 0], p["W2"][0, 0], p["W3"][0, 0], p["b3"][0] = 0.7, -1.3, 2.0, 0.0
    y, _ = C.forward(C.pack(p), X)
    assert np.allclose(y, 2.0 * np.tanh(-1.3 * np.tanh(0.7 * X[:, 0])), rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_backward_matches_finite_differences(seed):
    th = C.init_params(seed)
    X, t = data(seed + 10)
    L, g = C.loss_and_grad(th, X, t)
    assert abs(L - C.loss(th, X, t)) < 1e-15
    rng = np.random.default_rng(seed)
    idx = list(rng.choice(C.N_PARAMS, 60, replace=False)) + [0, 575, 576, 4735, 4800, 4864]
    fd = C.fd_grad(th, X, t, idx)
    assert np.max(np.abs(fd - g[idx])) <= 1e-7 * max(1e-3, np.max(np.abs(g[idx])))


def test_adam_first_step_is_sign_step():
    g = np.array([3.0, -0.5, 1e-3])
    th, m, v = C.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(th, -0.01 * np.sign(g), rtol=0, atol=1e-15)


def test_delta_omega_label():
    tau = 0.6
    nu = CS2 * (tau - 0.5)
    assert C.delta_omega_label(nu, 0.0) == 0.0
    nut = 0.05
    assert abs(C.delta_omega_label(nu, nut) - (1.0 / (tau + nut / CS2) - 1.0 / tau)) < 1e-15
    assert C.delta_omega_label(nu, nut) < 0


def test_box_filter_constant_and_linear():
    a = np.full((8, 8, 8), 3.5)
    assert np.all(C.box_filter(a, 4) == 3.5)
    z, y, x = np.meshgrid(np.arange(8.), np.arange(8.), np.arange(8.), indexing="ij")
    f = 2 * x - y + 0.5 * z
    fb = C.box_filter(f, 4)
    zc = yc = xc = np.array([1.5, 5.5])
    Zc, Yc, Xc = np.meshgrid(zc, yc, xc, indexing="ij")
    assert np.allclose(fb, 2 * Xc - Yc + 0.5 * Zc, atol=1e-14)


def test_eddy_viscosity_recovers_a_planted_nu_t():
    """A filtered field whose SGS stress is exactly -2 nu0 S (plus an isotropic part) gives nu_t = nu0;
    the opposite sign (backscatter) is clipped to 0."""
    n = 8
    z, y, x = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), np.arange(n, dtype=float),
                          indexing="ij")
    k = 2 * np.pi / n
    ux = 0.01 * np.sin(k * y)
    uy = 0.02 * np.sin(k * z)
    uz = 0.015 * np.sin(k * x)
    u = [ux, uy, uz]
    ax = {0: 2, 1: 1, 2: 0}
    d = lambda f, j: 0.5 * (np.roll(f, -1, axis=ax[j]) - np.roll(f, 1, axis=ax[j]))  # noqa: E731
    S = [[0.5 * (d(u[i], j) + d(u[j], i)) for j in range(3)] for i in range(3)]
    for nu0, expect in ((0.004, 0.004), (-0.004, 0.0)):
        uu = {}
        for i in range(3):
            for j in range(i, 3):
                uu[(i, j)] = u[i] * u[j] - 2 * nu0 * S[i][j] + (0.3 if i == j else 0.0)
        nut = C.eddy_viscosity(u, uu, walls_y=False)
        mask = sum(S[i][j] ** 2 for i in range(3) for j in range(3)) > 1e-14
        assert np.allclose(nut[mask], expect, rtol=1e-10, atol=1e-15)


def test_wall_derivative_is_exact_for_quadratics_vanishing_at_the_walls():
    """Filtered velocity between no-slip walls at y = -1/2 and cy - 1/2: the derivative at every
    row, the first and last included, is exact for (y + 1/2)(cy - 1/2 - y) and for profiles
    linear near one wall; a first-order one-sided difference at the end rows is not."""
    cy = 6
    y = np.arange(cy, dtype=float)
    for prof, dprof in (((y + 0.5) * (cy - 0.5 - y), (cy - 0.5 - y) - (y + 0.5)),):
        g = np.broadcast_to(prof[None, :, None], (2, cy, 3)).copy()
        d = C.wall_ddy(g)
        assert np.allclose(d, np.broadcast_to(dprof[None, :, None], g.shape), rtol=0, atol=1e-13)
        one_sided = g[:, 1, :] - g[:, 0, :]
        assert np.max(np.abs(one_sided - dprof[0])) > 0.1
    lin = np.broadcast_to((y + 0.5)[None, :, None], (2, cy, 3))  # vanishes at y = -1/2
    assert np.allclose(C.wall_ddy(lin)[:, :-1, :], 1.0, rtol=0, atol=1e-13)
