"""FP64 CPU oracle of the learned closure (test infrastructure only).

The paper has no learned closure; its channel flow uses a Smagorinsky LES
(Sec. 4).  The closure here is a small per-cell network that corrects the
shear relaxation rate of the coarse-grid FPC-LBM:

  inputs  x = (kappa_200 - cs2 rho, kappa_020 - cs2 rho, kappa_002 - cs2 rho,
               kappa_110, kappa_101, kappa_011, u_x, u_y, u_z)
          (the six non-equilibrium second-order central moments, whose
          attractors are cs2 rho on the diagonal and 0 off it, Sec. 3, plus u)
  network h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3
          (9 -> 64 -> 64 -> 1, weights row-major out x in)
  output  delta omega added to the shear rates omega_4,5,6,8,9

The training target (label) of a coarse cell is the change of the shear rate
that an eddy viscosity nu_t adds to the molecular one, using the lattice
relation nu = cs2 (1/omega - 1/2) of Eq. (transportcoeff3DFPCLBM):
  delta omega = 1 / ((nu + nu_t)/cs2 + 1/2) - 1 / (nu/cs2 + 1/2),
with nu_t from the box-filtered fine-grid fields by the least-squares
eddy-viscosity fit nu_t = max(0, -tau^d_ij S_ij / (2 S_kl S_kl)),
tau_ij = avg(u_i u_j) - avg(u_i) avg(u_j), S_ij the strain rate of the
filtered velocity from central differences.

Everything is plain numpy in float64: forward pass, mean-squared-error loss,
backward pass by the chain rule, and a central finite-difference gradient for
the pins.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 9, 64
SHAPES = (("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (1, N_H)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 4865


def unpack(theta: np.ndarray) -> dict:
    """Flat parameter vector (the order of fpclbm_set_closure) -> named arrays."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[k:k + n].reshape(shp)
        k += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def init_params(seed: int) -> np.ndarray:
    """Uniform(+-1/sqrt(fan_in)) weights, zero biases (a plain default)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            lim = 1.0 / np.sqrt(shp[1])
            p[name] = rng.uniform(-lim, lim, shp)
        else:
            p[name] = np.zeros(shp)
    return pack(p)


def forward(theta, X):
    """X [B, 9] -> (y [B], cache)."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(a2)
    y = (h2 @ p["W3"].T + p["b3"])[:, 0]
    return y, (X, h1, h2, p)


def loss(theta, X, t) -> float:
    """Mean squared error 1/B sum (y - t)^2."""
    y, _ = forward(theta, X)
    d = y - np.asarray(t, dtype=np.float64)
    return float(np.mean(d * d))


def loss_and_grad(theta, X, t):
    """Loss and its gradient (flat, same order as theta) by the chain rule."""
    y, (X, h1, h2, p) = forward(theta, X)
    B = X.shape[0]
    d = y - np.asarray(t, dtype=np.float64)
    L = float(np.mean(d * d))
    gy = (2.0 / B) * d                      # dL/dy            [B]
    gW3 = gy[None, :] @ h2                  # [1, 64]
    gb3 = np.array([gy.sum()])
    gh2 = gy[:, None] * p["W3"]             # [B, 64]
    ga2 = gh2 * (1.0 - h2 * h2)
    gW2 = ga2.T @ h1
    gb2 = ga2.sum(axis=0)
    gh1 = ga2 @ p["W2"]
    ga1 = gh1 * (1.0 - h1 * h1)
    gW1 = ga1.T @ X
    gb1 = ga1.sum(axis=0)
    g = pack({"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3})
    return L, g


def fd_grad(theta, X, t, idx, h=1e-6) -> np.ndarray:
    """Central finite differences of the loss for the parameter indices idx."""
    theta = np.asarray(theta, dtype=np.float64)
    out = np.zeros(len(idx))
    for k, i in enumerate(idx):
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        out[k] = (loss(tp, X, t) - loss(tm, X, t)) / (2 * h)
    return out


def adam_step(theta, g, m, v, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) in float64; returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def delta_omega_label(nu: float, nu_t, cs2: float = 1.0 / 3.0):
    """Shear-rate change that adds nu_t to nu: 1/((nu+nu_t)/cs2 + 1/2) - 1/(nu/cs2 + 1/2)."""
    nu_t = np.asarray(nu_t, dtype=np.float64)
    return 1.0 / ((nu + nu_t) / cs2 + 0.5) - 1.0 / (nu / cs2 + 0.5)


def box_filter(field, r: int):
    """Average over non-overlapping r^3 blocks of a [nz, ny, nx] array."""
    a = np.asarray(field, dtype=np.float64)
    nz, ny, nx = a.shape
    return a.reshape(nz // r, r, ny // r, r, nx // r, r).mean(axis=(1, 3, 5))


def wall_ddy(g):
    """d/dy of a filtered field [nz, cy, nx] between no-slip walls at y = -1/2 and cy - 1/2 (coarse
    units): central differences inside; at the first and last row the derivative of the quadratic
    through the wall value 0 and the two nearest rows (y = -1/2, 0, 1: g_0 + g_1 / 3, mirrored at
    the top), exact for quadratics that vanish at the walls."""
    a = np.asarray(g, dtype=np.float64)
    d = 0.5 * (np.roll(a, -1, axis=1) - np.roll(a, 1, axis=1))
    d[:, 0, :] = a[:, 0, :] + a[:, 1, :] / 3.0
    d[:, -1, :] = -(a[:, -1, :] + a[:, -2, :] / 3.0)
    return d


def sample(rho, ux, uy, uz, r: int, tau_c: float, walls_y: bool, cs2: float = 1.0 / 3.0):
    """Features [nc, 9] and labels [nc] of r^3 box-filtered fine fields (x fastest).

    features: -2 rho cs2 tau_c S_ij (ij = xx, yy, zz, xy, xz, yz) of the filtered velocity (the
    coarse non-equilibrium second moments of Appendix C Eq. noneqmmoments3D with 1/omega -> tau),
    then the filtered velocity; label: delta_omega_label(cs2 (tau_c - 1/2), nu_t)."""
    f = [np.asarray(a, dtype=np.float64) for a in (rho, ux, uy, uz)]
    rb = box_filter(f[0], r)
    ub = [box_filter(c, r) for c in f[1:]]
    uu = {(i, j): box_filter(f[1 + i] * f[1 + j], r) for i in range(3) for j in range(i, 3)}
    nut = eddy_viscosity(ub, uu, walls_y=walls_y)
    axes = {0: 2, 1: 1, 2: 0}

    def ddx(g, d):
        if d == 1 and walls_y:
            return wall_ddy(g)
        return 0.5 * (np.roll(g, -1, axis=axes[d]) - np.roll(g, 1, axis=axes[d]))

    grad = [[ddx(ub[i], j) for j in range(3)] for i in range(3)]
    S = [[0.5 * (grad[i][j] + grad[j][i]) for j in range(3)] for i in range(3)]
    pre = -2.0 * rb * cs2 * tau_c
    X = np.stack([pre * S[0][0], pre * S[1][1], pre * S[2][2], pre * S[0][1], pre * S[0][2], pre * S[1][2],
                  ub[0], ub[1], ub[2]], axis=-1).reshape(-1, 9)
    T = delta_omega_label(cs2 * (tau_c - 0.5), nut, cs2).reshape(-1)
    return X, T


def eddy_viscosity(ubar, uu_bar, walls_y: bool = True):
    """nu_t = max(0, -tau^d_ij S_ij / (2 S_kl S_kl)) on the filtered grid.

    ubar: (ux, uy, uz) filtered velocities [nz, ny, nx] (filter spacing = 1 coarse cell)
    uu_bar: dict (i, j) -> filtered u_i u_j for i <= j
    Central differences, periodic in x and z; at the y ends with walls_y the wall-aware derivative
    of wall_ddy (the no-slip wall value 0 at y = -1/2 and cy - 1/2).
    """
    u = [np.asarray(c, dtype=np.float64) for c in ubar]
    axes = {0: 2, 1: 1, 2: 0}   # velocity direction -> array axis (x -> 2, y -> 1, z -> 0)

    def ddx(f, d):
        ax = axes[d]
        if d == 1 and walls_y:
            return wall_ddy(f)
        return 0.5 * (np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax))

    grad = [[ddx(u[i], j) for j in range(3)] for i in range(3)]   # grad[i][j] = d u_i / d x_j
    S = [[0.5 * (grad[i][j] + grad[j][i]) for j in range(3)] for i in range(3)]
    tau = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            a, b = min(i, j), max(i, j)
            tau[i][j] = uu_bar[(a, b)] - u[i] * u[j]
    tr = (tau[0][0] + tau[1][1] + tau[2][2]) / 3.0
    num = 0.0
    den = 0.0
    for i in range(3):
        for j in range(3):
            td = tau[i][j] - (tr if i == j else 0.0)
            num = num + td * S[i][j]
            den = den + S[i][j] * S[i][j]
    with np.errstate(divide="ignore", invalid="ignore"):
        nut = np.where(den > 0, -num / (2.0 * den), 0.0)
    return np.maximum(nut, 0.0)
