"""Seeded synthetic inputs shared by the tests, the smoke check and bench.py.

This module holds NO arithmetic of the method: it only draws initial density
and velocity fields (and raw positive population vectors for one-step brute
force checks) with the shapes, sizes and value distributions of the paper's
workloads.  Both the FP64 CPU oracle and the CUDA path receive the same arrays
and each turns them into populations with its own code.

Fields are float64 arrays shaped [nz, ny, nx] (x fastest, cell centres at
integer coordinates).
"""
from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0  # lattice speed of sound squared (equation of state p = cs^2 rho)


def _grid(nx: int, ny: int, nz: int):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def tgv(n: int, u0: float, rho0: float = 1.0):
    """3D Taylor-Green vortex on a periodic n^3 box.

    u = u0 sin(kx) cos(ky) cos(kz), v = -u0 cos(kx) sin(ky) cos(kz), w = 0,
    k = 2 pi / n; the density carries the vortex's pressure field divided by
    cs^2: rho = rho0 + rho0 u0^2/16 (cos 2kx + cos 2ky)(cos 2kz + 2) / cs^2.
    """
    x, y, z = _grid(n, n, n)
    k = 2.0 * math.pi / n
    ux = u0 * np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
    uy = -u0 * np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    uz = np.zeros_like(ux)
    rho = rho0 + rho0 * u0 * u0 / 16.0 * (np.cos(2 * k * x) + np.cos(2 * k * y)) * (np.cos(2 * k * z) + 2.0) / CS2
    return rho, ux, uy, uz


def tgv_viscosity(n: int, u0: float, re: float) -> float:
    """Kinematic viscosity of a TGV at Reynolds number re = u0 L / nu, L = n / 2 pi."""
    return u0 * (n / (2.0 * math.pi)) / re


def shear_wave(ny: int, amp: float, nx: int = 1, nz: int = 1):
    """u_x = amp sin(2 pi y / ny), rho = 1 (transverse shear wave along y)."""
    x, y, z = _grid(nx, ny, nz)
    ux = amp * np.sin(2.0 * math.pi * y / ny)
    return np.ones_like(ux), ux, np.zeros_like(ux), np.zeros_like(ux)


def density_wave(ny: int, eps: float, nx: int = 1, nz: int = 1):
    """rho = 1 + eps sin(2 pi y / ny), u = 0 (longitudinal acoustic wave)."""
    x, y, z = _grid(nx, ny, nz)
    rho = 1.0 + eps * np.sin(2.0 * math.pi * y / ny)
    zero = np.zeros_like(rho)
    return rho, zero, zero.copy(), zero.copy()


def crossing_shear_waves(n: int, amp: float):
    """Orthogonal crossing shear waves: u_y = amp cos(k x) cos(k z), k = 2 pi / n."""
    x, y, z = _grid(n, n, n)
    k = 2.0 * math.pi / n
    uy = amp * np.cos(k * x) * np.cos(k * z)
    zero = np.zeros_like(uy)
    return np.ones_like(uy), zero, uy, zero.copy()


def poiseuille_profile(ny: int, force: float, nu: float, rho0: float = 1.0) -> np.ndarray:
    """Steady plane Poiseuille u_x(y) between walls at y = -1/2 and ny - 1/2."""
    y = np.arange(ny, dtype=np.float64)
    return force / (2.0 * rho0 * nu) * (y + 0.5) * (ny - 0.5 - y)


def random_fields(nx: int, ny: int, nz: int, seed: int, u_amp: float = 0.05, rho_amp: float = 0.02):
    """Cell-wise uniform random fields: rho in 1 +- rho_amp, each u component in +-u_amp."""
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    rho = 1.0 + rho_amp * rng.uniform(-1.0, 1.0, shape)
    ux, uy, uz = (u_amp * rng.uniform(-1.0, 1.0, shape) for _ in range(3))
    return rho, ux, uy, uz


def random_populations(n_cells: int, seed: int, spread: float = 0.5) -> np.ndarray:
    """Positive raw populations [27, n_cells]: (1/27)(1 + spread * U[0, 1)).

    Far from any equilibrium on purpose, so that every moment of the collision
    carries a non-trivial value in a one-step brute-force comparison.
    """
    rng = np.random.default_rng(seed)
    return (1.0 + spread * rng.random((27, n_cells))) / 27.0


def channel_fields(nx: int, ny: int, nz: int, u_star: float, seed: int, bulk_factor: float = 16.0,
                   perturb: float = 0.10):
    """Channel initial condition: walls at y = -1/2 and ny - 1/2, laminar parabola with bulk
    velocity bulk_factor * u_star, plus uniform random perturbations of +-perturb times the
    centreline velocity on every component (seeded)."""
    y = np.arange(ny, dtype=np.float64)
    h = float(ny)
    eta = (y + 0.5) / h
    ub = bulk_factor * u_star
    prof = 6.0 * ub * eta * (1.0 - eta)  # mean of the parabola = ub
    ucl = 1.5 * ub
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    ux = np.broadcast_to(prof[None, :, None], shape).copy()
    amp = perturb * ucl
    ux += amp * rng.uniform(-1.0, 1.0, shape)
    uy = amp * rng.uniform(-1.0, 1.0, shape)
    uz = amp * rng.uniform(-1.0, 1.0, shape)
    return np.ones(shape), ux, uy, uz


def solenoidal_field(n: int, seed: int, k_peak: float = 4.0, u_rms: float = 0.04):
    """Random divergence-free velocity on a periodic n^3 box with energy spectrum
    E(k) ~ k^4 exp(-2 (k / k_peak)^2), random phases, rescaled so that
    sqrt(<u.u>/3) = u_rms.  Returns (rho, ux, uy, uz) with rho = 1."""
    rng = np.random.default_rng(seed)
    kf = np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(kf, kf, kf, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    kk_safe = np.where(kk == 0, 1.0, kk)
    spec = kk_safe ** 4 * np.exp(-2.0 * (kk_safe / k_peak) ** 2)
    amp = np.sqrt(spec / (4.0 * math.pi * kk_safe ** 2))
    amp[kk == 0] = 0.0
    comps = []
    for _ in range(3):
        phase = rng.uniform(0.0, 2.0 * math.pi, kk.shape)
        mag = rng.normal(size=kk.shape)
        comps.append(amp * mag * np.exp(1j * phase))
    vx, vy, vz = comps
    # project out the component along k (solenoidal), then take the real part of the
    # inverse transform, which keeps the field divergence-free (Hermitian symmetrisation)
    dot = (vx * kx + vy * ky + vz * kz) / (kk_safe ** 2)
    vx = vx - dot * kx
    vy = vy - dot * ky
    vz = vz - dot * kz
    ux = np.real(np.fft.ifftn(vx))
    uy = np.real(np.fft.ifftn(vy))
    uz = np.real(np.fft.ifftn(vz))
    rms = math.sqrt(float(np.mean(ux * ux + uy * uy + uz * uz)) / 3.0)
    s = u_rms / rms
    return np.ones((n, n, n)), ux * s, uy * s, uz * s


ENSEMBLE_SIDES = (32, 48, 64, 96)


def ensemble_config(n_boxes: int = 256, seed: int = 2410, tau_lo: float = 0.505, tau_hi: float = 0.6):
    """Box sides drawn uniformly from {32, 48, 64, 96} and tau ~ U[tau_lo, tau_hi] (seeded)."""
    rng = np.random.default_rng(seed)
    sides = rng.choice(np.array(ENSEMBLE_SIDES), size=n_boxes)
    taus = rng.uniform(tau_lo, tau_hi, size=n_boxes)
    return [int(s) for s in sides], [float(t) for t in taus]


def ensemble_fields(sides, seed: int = 2410):
    """Initial fields of an ensemble: one seeded solenoidal field per distinct side, and for every
    box a random periodic shift and axis permutation of it (both keep the field divergence-free
    and its spectrum), so that boxes differ without one FFT per box."""
    rng = np.random.default_rng(seed)
    base = {s: solenoidal_field(s, seed + s) for s in sorted(set(sides))}
    out = []
    for s in sides:
        rho, ux, uy, uz = base[s]
        perm = rng.permutation(3)                # new axis order (z, y, x) <- old
        shift = tuple(int(v) for v in rng.integers(0, s, 3))
        comps = [uz, uy, ux]                      # component along array axis 0, 1, 2
        moved = [np.roll(np.transpose(comps[perm[i]], perm), shift, axis=(0, 1, 2)) for i in range(3)]
        out.append((np.ones((s, s, s)), moved[2], moved[1], moved[0]))
    return out


def shear_layers(L: int, U: float, w: float = 0.05, delta: float = 0.05):
    """Doubly periodic shear layers on an L x L grid (coordinates scaled by L, cell centres):
    u_x = U tanh(4 (y - 1/4) / w) for y <= 1/2, U tanh(4 (3/4 - y) / w) above, and
    u_y = U delta sin(2 pi (x + 1/4)).  Returns (rho, ux, uy) shaped [y, x] with rho = 1."""
    c = (np.arange(L) + 0.5) / L
    x, y = np.meshgrid(c, c)
    ux = np.where(y <= 0.5, U * np.tanh(4 * (y - 0.25) / w), U * np.tanh(4 * (0.75 - y) / w))
    uy = U * delta * np.sin(2 * np.pi * (x + 0.25))
    return np.ones((L, L)), ux, uy
