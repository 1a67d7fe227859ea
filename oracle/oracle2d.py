"""ctypes binding of the FP64 CPU oracle of the D2Q9 FPC-LBM (``fpc2d_oracle.c``).

TEST INFRASTRUCTURE.  Thin marshalling over the C oracle (explicit 9x9 central-moment matrix, LU
solves, generic attractor formula Eq. (Mvcmattractor2D)).  Population arrays are
``float64[9, ny, nx]`` holding full populations, velocity order of Sec. 2.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .oracle import lib as _lib3

__all__ = ["velocity_set", "central_matrix", "grouping_matrix", "attractor_generic", "collide", "equilibrium",
           "init_equilibrium", "step", "run", "moments", "rates", "BC_PERIODIC", "BC_BOX"]

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_ready = False


def lib():
    global _ready
    L = _lib3()
    if not _ready:
        L.orc2_central_matrix.argtypes = [_D, _D]
        L.orc2_grouping_matrix.argtypes = [_D]
        L.orc2_attractor_generic.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        L.orc2_attractor_generic.restype = ctypes.c_double
        L.orc2_collide.argtypes = [_D, _D, _D, ctypes.c_int, _D]
        L.orc2_collide.restype = ctypes.c_int
        L.orc2_equilibrium.argtypes = [ctypes.c_double, _D, _D]
        L.orc2_equilibrium.restype = ctypes.c_int
        L.orc2_init_equilibrium.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        L.orc2_init_equilibrium.restype = ctypes.c_int
        L.orc2_step_bc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, ctypes.c_int,
                                   ctypes.c_double]
        L.orc2_step_bc.restype = ctypes.c_int
        L.orc2_run_bc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, ctypes.c_int, ctypes.c_long,
                                  ctypes.c_double]
        L.orc2_run_bc.restype = ctypes.c_int
        L.orc2_moments.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D]
        L.orc2_rates.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
        L.orc2_velocity_set.argtypes = [_I, _I]
        _ready = True
    return L


def _p(a):
    return a.ctypes.data_as(_D)


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


def _ok(rc):
    if rc == -2:
        raise ValueError("bc must be 0 (periodic) or 2 (closed box); a lid needs the box")
    if rc != 0:
        raise FloatingPointError("singular central-moment matrix")


BC_PERIODIC, BC_BOX = 0, 2


def velocity_set() -> np.ndarray:
    ex, ey = (np.zeros(9, dtype=np.int32) for _ in range(2))
    lib().orc2_velocity_set(ex.ctypes.data_as(_I), ey.ctypes.data_as(_I))
    return np.stack([ex, ey], axis=1)


def central_matrix(u) -> np.ndarray:
    C = np.zeros((9, 9))
    lib().orc2_central_matrix(_p(_arr(u, 2)), _p(C))
    return C


def grouping_matrix() -> np.ndarray:
    G = np.zeros((9, 9))
    lib().orc2_grouping_matrix(_p(G))
    return G


def attractor_generic(m: int, n: int, Pi, D) -> float:
    """Eq. (Mvcmattractor2D); Pi is [3, 3] indexed [m, n], D = (Dxx, Dyy, Dxy)."""
    return lib().orc2_attractor_generic(m, n, _p(_arr(Pi, 9)), _p(_arr(D, 3)))


def collide(f, F=(0.0, 0.0), omega=None, mode: int = 0) -> np.ndarray:
    out = np.zeros(9)
    om = np.ones(9) if omega is None else omega
    _ok(lib().orc2_collide(_p(_arr(f, 9)), _p(_arr(F, 2)), _p(_arr(om, 9)), int(mode), _p(out)))
    return out


def equilibrium(rho: float, u) -> np.ndarray:
    out = np.zeros(9)
    _ok(lib().orc2_equilibrium(float(rho), _p(_arr(u, 2)), _p(out)))
    return out


def init_equilibrium(rho, ux, uy) -> np.ndarray:
    rho, ux, uy = (_arr(a) for a in (rho, ux, uy))
    ny, nx = rho.shape
    f = np.zeros((9, ny, nx))
    _ok(lib().orc2_init_equilibrium(nx, ny, _p(rho), _p(ux), _p(uy), _p(f)))
    return f


def step(f, F=(0.0, 0.0), omega=None, mode: int = 0, bc: int = 0, uw: float = 0.0) -> np.ndarray:
    """One step; bc 0 periodic, 2 closed box whose wall y = ny - 1/2 moves along x at uw."""
    f = _arr(f)
    _, ny, nx = f.shape
    out = np.zeros_like(f)
    om = np.ones(9) if omega is None else omega
    _ok(lib().orc2_step_bc(nx, ny, int(bc), _p(f), _p(out), _p(_arr(F, 2)), _p(_arr(om, 9)), int(mode), float(uw)))
    return out


def run(f, nsteps: int, F=(0.0, 0.0), omega=None, mode: int = 0, bc: int = 0, uw: float = 0.0) -> np.ndarray:
    f = _arr(f).copy()
    _, ny, nx = f.shape
    work = np.zeros_like(f)
    om = np.ones(9) if omega is None else omega
    _ok(lib().orc2_run_bc(nx, ny, int(bc), _p(f), _p(work), _p(_arr(F, 2)), _p(_arr(om, 9)), int(mode),
                          int(nsteps), float(uw)))
    return f


def moments(f, F=(0.0, 0.0)):
    f = _arr(f)
    _, ny, nx = f.shape
    outs = [np.zeros((ny, nx)) for _ in range(3)]
    lib().orc2_moments(nx, ny, _p(f), _p(_arr(F, 2)), *(_p(o) for o in outs))
    return tuple(outs)


def rates(tau: float, bulk: float = 0.0, drift: float = 0.0) -> np.ndarray:
    out = np.zeros(9)
    lib().orc2_rates(float(tau), float(bulk), float(drift), _p(out))
    return out
