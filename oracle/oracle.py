"""ctypes binding of the FP64 CPU oracle (``fpc_oracle.c``).

TEST INFRASTRUCTURE.  Every function here is a thin marshalling layer over the
C oracle, which states the FPC-LBM of arXiv 2410.09739 literally (explicit
27x27 central-moment matrix, LU solves, generic attractor formula).  See the
header of ``fpc_oracle.c`` for the passages each step follows.

Population arrays are ``float64[27, nz, ny, nx]`` holding full populations.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "lib", "velocity_set", "moment_exponents", "central_matrix", "grouping_matrix",
    "attractor_generic", "maxwell_moments", "collide", "equilibrium", "init_equilibrium",
    "step", "run", "moments", "rates", "threads", "set_threads", "EQ_MODE_FP", "EQ_MODE_MCM",
    "BC_PERIODIC", "BC_WALLS_Y", "BC_BOX", "BC_HALF_CHANNEL", "smagorinsky_tau",
]

EQ_MODE_FP = 0   # diffusion tensor of Eq. (diffusion-tensor-parameter-3D)
EQ_MODE_MCM = 1  # Maxwellian central moments at every order

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_central_matrix.argtypes = [_D, _D]
        L.orc_grouping_matrix.argtypes = [_D]
        L.orc_attractor_generic.argtypes = [ctypes.c_int] * 3 + [_D, _D]
        L.orc_attractor_generic.restype = ctypes.c_double
        L.orc_maxwell_moments.argtypes = [ctypes.c_double, _D]
        L.orc_collide.argtypes = [_D, _D, _D, ctypes.c_int, _D]
        L.orc_collide.restype = ctypes.c_int
        L.orc_equilibrium.argtypes = [ctypes.c_double, _D, _D]
        L.orc_equilibrium.restype = ctypes.c_int
        L.orc_init_equilibrium.argtypes = [ctypes.c_int] * 3 + [_D] * 5
        L.orc_init_equilibrium.restype = ctypes.c_int
        L.orc_step_les.argtypes = [ctypes.c_int] * 4 + [_D, _D, _D, _D, ctypes.c_int, _D, _D]
        L.orc_step_les.restype = ctypes.c_int
        L.orc_run_les.argtypes = [ctypes.c_int] * 4 + [_D, _D, _D, _D, ctypes.c_int, ctypes.c_long, _D, _D]
        L.orc_run_les.restype = ctypes.c_int
        L.orc_smagorinsky_tau.argtypes = [_D, _D, ctypes.c_double, ctypes.c_double]
        L.orc_smagorinsky_tau.restype = ctypes.c_double
        L.orc_moments.argtypes = [ctypes.c_int] * 3 + [_D, _D, _D, _D, _D, _D]
        L.orc_rates.argtypes = [ctypes.c_double, ctypes.c_double, _D]
        L.orc_velocity_set.argtypes = [_I, _I, _I]
        L.orc_moment_exponents.argtypes = [_I]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _arr(x, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.shape, n)
    return a


def velocity_set() -> np.ndarray:
    """e_alpha as int array [27, 3] (Sec. 3 D3Q27 list)."""
    ex, ey, ez = (np.zeros(27, np.int32) for _ in range(3))
    lib().orc_velocity_set(*(v.ctypes.data_as(_I) for v in (ex, ey, ez)))
    return np.stack([ex, ey, ez], axis=1)


def moment_exponents() -> np.ndarray:
    """(m, n, p) of the central-moment vector m^c, int array [27, 3]."""
    out = np.zeros(81, np.int32)
    lib().orc_moment_exponents(out.ctypes.data_as(_I))
    return out.reshape(27, 3)


def central_matrix(u) -> np.ndarray:
    """C(u)[i, a] = prod (e_a - u)^(m_i, n_i, p_i); C(0) is the projection P."""
    C = np.zeros((27, 27))
    lib().orc_central_matrix(_p(_arr(u, 3)), _p(C))
    return C


def grouping_matrix() -> np.ndarray:
    G = np.zeros((27, 27))
    lib().orc_grouping_matrix(_p(G))
    return G


def attractor_generic(m: int, n: int, p: int, Pi, D) -> float:
    """Eq. (Mvcmattractor3D); Pi is [3,3,3] indexed [m,n,p], D is 3x3."""
    return lib().orc_attractor_generic(m, n, p, _p(_arr(Pi, 27)), _p(_arr(D, 9)))


def maxwell_moments(rho: float) -> np.ndarray:
    M = np.zeros(27)
    lib().orc_maxwell_moments(rho, _p(M))
    return M.reshape(3, 3, 3)


def collide(f, F=(0.0, 0.0, 0.0), omega=None, mode: int = EQ_MODE_FP) -> np.ndarray:
    """Post-collision populations of one cell (Appendix D Steps 7, 1-5)."""
    if omega is None:
        omega = np.ones(27)
    out = np.zeros(27)
    rc = lib().orc_collide(_p(_arr(f, 27)), _p(_arr(F, 3)), _p(_arr(omega, 27)), int(mode), _p(out))
    if rc != 0:
        raise FloatingPointError("singular central-moment matrix")
    return out


def equilibrium(rho: float, u) -> np.ndarray:
    out = np.zeros(27)
    if lib().orc_equilibrium(float(rho), _p(_arr(u, 3)), _p(out)) != 0:
        raise FloatingPointError("singular central-moment matrix")
    return out


def init_equilibrium(rho, ux, uy, uz) -> np.ndarray:
    """Equilibrium populations [27, nz, ny, nx] of fields shaped [nz, ny, nx]."""
    rho, ux, uy, uz = (_arr(a) for a in (rho, ux, uy, uz))
    nz, ny, nx = rho.shape
    f = np.zeros((27, nz, ny, nx))
    if lib().orc_init_equilibrium(nx, ny, nz, _p(rho), _p(ux), _p(uy), _p(uz), _p(f)) != 0:
        raise FloatingPointError("singular central-moment matrix")
    return f


BC_PERIODIC, BC_WALLS_Y, BC_BOX, BC_HALF_CHANNEL = 0, 1, 2, 3


def _check(rc: int):
    if rc == -2:
        raise ValueError("bad boundary condition or wall velocity (bc in 0..3, tangential lid, no lid when periodic "
                         "or half channel)")
    if rc != 0:
        raise FloatingPointError("singular central-moment matrix")


def _les(les):
    return None if les is None else _p(_arr(les, 3))


def step(f, bc: int = 0, F=(0.0, 0.0, 0.0), omega=None, mode: int = EQ_MODE_FP, uw=(0.0, 0.0, 0.0),
         les=None) -> np.ndarray:
    """One time step (collide + stream); returns the new populations.  bc: 0 periodic, 1 walls at
    y = -1/2, ny - 1/2, 2 closed box, 3 half channel (wall at y = -1/2, symmetry plane at ny - 1/2);
    uw: velocity of the wall at y = ny - 1/2; les: (C_s, u*, A+) for the Smagorinsky model with
    van Driest damping, or None."""
    f = _arr(f)
    _, nz, ny, nx = f.shape
    out = np.zeros_like(f)
    if omega is None:
        omega = np.ones(27)
    _check(lib().orc_step_les(nx, ny, nz, int(bc), _p(f), _p(out), _p(_arr(F, 3)), _p(_arr(omega, 27)), int(mode),
                              _p(_arr(uw, 3)), _les(les)))
    return out


def run(f, nsteps: int, bc: int = 0, F=(0.0, 0.0, 0.0), omega=None, mode: int = EQ_MODE_FP,
        uw=(0.0, 0.0, 0.0), les=None) -> np.ndarray:
    """``nsteps`` time steps; returns the new populations (input untouched)."""
    f = _arr(f).copy()
    _, nz, ny, nx = f.shape
    work = np.zeros_like(f)
    if omega is None:
        omega = np.ones(27)
    _check(lib().orc_run_les(nx, ny, nz, int(bc), _p(f), _p(work), _p(_arr(F, 3)), _p(_arr(omega, 27)),
                             int(mode), int(nsteps), _p(_arr(uw, 3)), _les(les)))
    return f


def smagorinsky_tau(f, F=(0.0, 0.0, 0.0), tau0: float = 0.6, c2: float = 0.0) -> float:
    """Effective shear relaxation time of one cell under the Smagorinsky model, c2 = (C_s Delta D)^2."""
    return float(lib().orc_smagorinsky_tau(_p(_arr(f, 27)), _p(_arr(F, 3)), float(tau0), float(c2)))


def moments(f, F=(0.0, 0.0, 0.0)):
    """(rho, ux, uy, uz) per cell (Appendix D Step 7), each [nz, ny, nx]."""
    f = _arr(f)
    _, nz, ny, nx = f.shape
    outs = [np.zeros((nz, ny, nx)) for _ in range(4)]
    lib().orc_moments(nx, ny, nz, _p(f), _p(_arr(F, 3)), *(_p(o) for o in outs))
    return tuple(outs)


def rates(tau: float, drift: float = 0.0) -> np.ndarray:
    """omega_0..omega_26 for a shear relaxation time tau and drift omega_FP."""
    out = np.zeros(27)
    lib().orc_rates(float(tau), float(drift), _p(out))
    return out


def threads() -> int:
    """Threads the OpenMP runtime will use for the oracle's parallel loops."""
    L = lib()
    L.orc_max_threads.restype = ctypes.c_int
    return int(L.orc_max_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (CPU-baseline timing)."""
    lib().orc_set_threads(ctypes.c_int(int(n)))
