"""Thin ctypes binding of libfpclbm.so (include/fpclbm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The module-level functions carry the C names; ``Lattice`` is a
small convenience wrapper over them.  There is no CPU fallback: if the shared
library is missing or fails to load, every call raises.

Arrays passed to the library are float64.  Host arrays may be numpy arrays or
CPU torch tensors; device arrays (``on_device=1``) must be CUDA torch tensors
on the handle's device.  Field arrays are shaped [nz, ny, nx] (x fastest) or
flat; population arrays are [27, N] in the paper's alpha order.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfpclbm.so")

FPCLBM_OK = 0
FPCLBM_ERR_ARG = -1
FPCLBM_ERR_ALLOC = -2
FPCLBM_ERR_CUDA = -3
FPCLBM_ERR_PARAM = -4
FPCLBM_ERR_STATE = -5
FPCLBM_ERR_DIVERGED = -6
FPCLBM_ERR_TIMEOUT = -7

FPCLBM_FP64 = 0
FPCLBM_FP32 = 1
FPCLBM_FP32_STORE_FP16 = 2
FPCLBM_FP32_STORE_BF16 = 3

FPCLBM_BC_PERIODIC = 0
FPCLBM_BC_WALLS_Y = 1
FPCLBM_BC_BOX = 2
FPCLBM_BC_HALF_CHANNEL = 3

FPCLBM_DIFF_FP = 0
FPCLBM_DIFF_EQUILIBRIUM = 1
FPCLBM_DIFF_FP_LEARNED = 2
FPCLBM_DIFF_FP_SMAGORINSKY = 3

PRECISIONS = {"fp64": FPCLBM_FP64, "fp32": FPCLBM_FP32, "fp16": FPCLBM_FP32_STORE_FP16,
              "bf16": FPCLBM_FP32_STORE_BF16}

EXPORTED = ("fpclbm_create", "fpclbm_create_ensemble", "fpclbm_init_fields", "fpclbm_set_params",
            "fpclbm_set_rates", "fpclbm_set_force", "fpclbm_set_wall_velocity", "fpclbm_set_smagorinsky", "fpclbm_step", "fpclbm_moments", "fpclbm_diagnostics",
            "fpclbm_get_populations", "fpclbm_get_populations_at", "fpclbm_set_populations", "fpclbm_get_step_count", "fpclbm_get_launch", "fpclbm_set_closure",
            "fpclbm_state_bytes", "fpclbm_get_state", "fpclbm_set_state", "fpclbm_test_alloc_hook",
            "fpclbm_destroy", "fpclbm_last_error", "fpclbm_diagnostics_noalloc", "fpclbm_closure_sample",
            "fpclbm_closure_train", "fpclbm_closure_grad", "fpclbm_closure_pack",
            "fpclbm2d_create", "fpclbm2d_init_fields", "fpclbm2d_set_params", "fpclbm2d_set_rates",
            "fpclbm2d_set_force", "fpclbm2d_set_boundary", "fpclbm2d_step", "fpclbm2d_moments", "fpclbm2d_get_populations",
            "fpclbm2d_set_populations", "fpclbm2d_destroy", "fpclbm2d_last_error")


class FpclbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("fpclbm error %d: %s" % (code, msg))
        self.code = code


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def load(path: str = LIB_PATH):
    """Load libfpclbm.so (no fallback: raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError("libfpclbm.so not built: %s (run __graft_entry__.build())" % path)
    L = ctypes.CDLL(path)
    L.fpclbm_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, _P]
    L.fpclbm_create_ensemble.argtypes = [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int), _D,
                                         ctypes.c_int, _P]
    L.fpclbm_init_fields.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int]
    L.fpclbm_set_params.argtypes = [_P, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    L.fpclbm_set_rates.argtypes = [_P, _D]
    L.fpclbm_set_force.argtypes = [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.fpclbm_set_wall_velocity.argtypes = [_P, ctypes.c_double, ctypes.c_double]
    L.fpclbm_set_smagorinsky.argtypes = [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.fpclbm_step.argtypes = [_P, ctypes.c_longlong]
    L.fpclbm_moments.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int]
    L.fpclbm_diagnostics.argtypes = [_P, _D]
    L.fpclbm_get_populations.argtypes = [_P, _P]
    L.fpclbm_get_populations_at.argtypes = [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int, _P]
    L.fpclbm_set_populations.argtypes = [_P, _P]
    L.fpclbm_get_step_count.argtypes = [_P, ctypes.POINTER(ctypes.c_longlong)]
    L.fpclbm_get_launch.argtypes = [_P, ctypes.POINTER(ctypes.c_int)]
    L.fpclbm_state_bytes.argtypes = [_P, ctypes.POINTER(ctypes.c_ulonglong)]
    L.fpclbm_get_state.argtypes = [_P, _P, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_longlong)]
    L.fpclbm_set_state.argtypes = [_P, _P, ctypes.c_ulonglong, ctypes.c_longlong]
    L.fpclbm_test_alloc_hook.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]
    L.fpclbm_set_closure.argtypes = [_P, ctypes.POINTER(ctypes.c_ushort), ctypes.c_int]
    L.fpclbm_diagnostics_noalloc.argtypes = [_P, ctypes.c_longlong, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, _P, _P]
    L.fpclbm_closure_sample.argtypes = [_P, ctypes.c_int, ctypes.c_double, _P, _P, ctypes.c_int]
    L.fpclbm_closure_train.argtypes = [_P, _P, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_ushort), _D, _P]
    L.fpclbm_closure_grad.argtypes = [_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_ushort), _P, _D, _P]
    L.fpclbm_closure_pack.argtypes = [ctypes.POINTER(ctypes.c_ushort), ctypes.c_int, ctypes.POINTER(ctypes.c_uint),
                                      ctypes.c_int]
    L.fpclbm_destroy.argtypes = [_P]
    L.fpclbm_last_error.argtypes = [_P]
    L.fpclbm_last_error.restype = ctypes.c_char_p
    L.fpclbm2d_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]
    L.fpclbm2d_init_fields.argtypes = [_P, _P, _P, _P, ctypes.c_int]
    L.fpclbm2d_set_params.argtypes = [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    L.fpclbm2d_set_rates.argtypes = [_P, _D]
    L.fpclbm2d_set_force.argtypes = [_P, ctypes.c_double, ctypes.c_double]
    L.fpclbm2d_set_boundary.argtypes = [_P, ctypes.c_int, ctypes.c_double]
    L.fpclbm2d_step.argtypes = [_P, ctypes.c_longlong]
    L.fpclbm2d_moments.argtypes = [_P, _P, _P, _P, ctypes.c_int]
    L.fpclbm2d_get_populations.argtypes = [_P, _P]
    L.fpclbm2d_set_populations.argtypes = [_P, _P]
    L.fpclbm2d_destroy.argtypes = [_P]
    L.fpclbm2d_last_error.argtypes = [_P]
    L.fpclbm2d_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if not name.endswith("last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(h, rc: int):
    if rc != FPCLBM_OK:
        msg = load().fpclbm_last_error(h)
        raise FpclbmError(rc, msg.decode() if msg else "")
    return rc


def _ptr(a, on_device: bool):
    """Raw data pointer of a float64 array (numpy, or torch CPU/CUDA tensor)."""
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise TypeError("tensor must be contiguous float64")
            if a.is_cuda != bool(on_device):
                raise TypeError("tensor device does not match on_device=%d" % on_device)
            return ctypes.c_void_p(a.data_ptr())
    except ImportError:  # pragma: no cover
        pass
    if on_device:
        raise TypeError("on_device=1 needs a CUDA torch tensor")
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("host arrays must be C-contiguous float64 numpy arrays")
    return ctypes.c_void_p(a.ctypes.data)


# --- functions with the C names ---------------------------------------------------------

def fpclbm_create(nx: int, ny: int, nz: int, precision: int, bc: int = FPCLBM_BC_PERIODIC, stream: int = 0):
    h = _P()
    rc = load().fpclbm_create(ctypes.byref(h), nx, ny, nz, precision, bc, _P(stream) if stream else None)
    _check(None, rc)
    return h


def fpclbm_create_ensemble(dims, tau, precision: int = FPCLBM_FP32, stream: int = 0):
    dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1))
    tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64).reshape(-1))
    h = _P()
    rc = load().fpclbm_create_ensemble(ctypes.byref(h), len(tau), dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                       tau.ctypes.data_as(_D), precision, _P(stream) if stream else None)
    _check(None, rc)
    return h


def fpclbm_init_fields(h, rho, ux, uy, uz, on_device: int = 0):
    return _check(h, load().fpclbm_init_fields(h, *(_ptr(a, on_device) for a in (rho, ux, uy, uz)), on_device))


def fpclbm_set_params(h, tau: float, drift: float = 0.0, diffusion: int = FPCLBM_DIFF_FP):
    return _check(h, load().fpclbm_set_params(h, float(tau), float(drift), int(diffusion)))


def fpclbm_set_rates(h, omega):
    om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64)).reshape(-1)
    if om.size != 27:
        raise ValueError("omega needs 27 rates, got %d" % om.size)
    return _check(h, load().fpclbm_set_rates(h, om.ctypes.data_as(_D)))


def fpclbm_set_force(h, Fx: float, Fy: float, Fz: float):
    return _check(h, load().fpclbm_set_force(h, float(Fx), float(Fy), float(Fz)))


def fpclbm_set_wall_velocity(h, ux: float, uz: float):
    return _check(h, load().fpclbm_set_wall_velocity(h, float(ux), float(uz)))


def fpclbm_set_smagorinsky(h, cs: float, u_star: float, a_plus: float):
    return _check(h, load().fpclbm_set_smagorinsky(h, float(cs), float(u_star), float(a_plus)))


def fpclbm_step(h, n: int):
    return _check(h, load().fpclbm_step(h, int(n)))


def fpclbm_moments(h, rho, ux, uy, uz, on_device: int = 0):
    return _check(h, load().fpclbm_moments(h, *(_ptr(a, on_device) for a in (rho, ux, uy, uz)), on_device))


def fpclbm_diagnostics(h) -> np.ndarray:
    out = np.zeros(5)
    _check(h, load().fpclbm_diagnostics(h, out.ctypes.data_as(_D)))
    return out


def fpclbm_get_populations(h, f):
    return _check(h, load().fpclbm_get_populations(h, _ptr(f, 0)))


def fpclbm_get_populations_at(h, cells) -> np.ndarray:
    """Populations [27, n] of the listed flat cell indices."""
    c = np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1))
    out = np.empty((27, c.size))
    _check(h, load().fpclbm_get_populations_at(h, c.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), c.size,
                                               _ptr(out, 0)))
    return out


def fpclbm_set_populations(h, f):
    return _check(h, load().fpclbm_set_populations(h, _ptr(f, 0)))


def fpclbm_get_step_count(h) -> int:
    v = ctypes.c_longlong()
    _check(h, load().fpclbm_get_step_count(h, ctypes.byref(v)))
    return v.value


def fpclbm_state_bytes(h) -> int:
    v = ctypes.c_ulonglong()
    _check(h, load().fpclbm_state_bytes(h, ctypes.byref(v)))
    return v.value


def fpclbm_get_state(h):
    """(raw state as a uint8 numpy array, step count): the stored deviations in the storage type."""
    raw = np.empty(fpclbm_state_bytes(h), dtype=np.uint8)
    steps = ctypes.c_longlong()
    _check(h, load().fpclbm_get_state(h, raw.ctypes.data_as(_P), raw.size, ctypes.byref(steps)))
    return raw, steps.value


def fpclbm_set_state(h, raw, steps: int):
    raw = np.ascontiguousarray(raw)
    if raw.dtype != np.uint8:
        raise TypeError("raw state must be a uint8 array (as returned by fpclbm_get_state)")
    return _check(h, load().fpclbm_set_state(h, raw.ctypes.data_as(_P), raw.size, int(steps)))


def fpclbm_test_alloc_hook(fail_after: int = -2) -> int:
    """Arm (fail_after >= 0) or disarm (-1) the injected allocation failure; returns the number of
    live allocations of the library."""
    live = ctypes.c_longlong()
    load().fpclbm_test_alloc_hook(int(fail_after), ctypes.byref(live))
    return live.value


LAUNCH_MODES = {0: "FP", 1: "MCM", 2: "FP + learned closure", 3: "FP + Smagorinsky",
                4: "FP, unit rates of orders 3-6", 5: "MCM, unit rates of orders 3-6",
                6: "FP + learned closure, unit rates of orders 3-6"}


def fpclbm_get_launch(h) -> dict:
    """The step kernel's launch: threads per block, register-cap class, variant, collision mode."""
    v = (ctypes.c_int * 4)()
    _check(h, load().fpclbm_get_launch(h, v))
    return {"block": v[0], "minb": v[1], "variant": v[2], "mode": v[3]}


def fpclbm_set_closure(h, bf16_bits):
    w = np.ascontiguousarray(np.asarray(bf16_bits, dtype=np.uint16))
    return _check(h, load().fpclbm_set_closure(h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_ushort)), w.size))


CLOSURE_PACK_WORDS = 3012


def fpclbm_closure_pack(bf16_bits) -> np.ndarray:
    """The closure's 4865 bf16 weights in the device layout of the fused inference (uint32 words;
    host code, no GPU needed)."""
    w = np.ascontiguousarray(np.asarray(bf16_bits, dtype=np.uint16))
    out = np.zeros(CLOSURE_PACK_WORDS, dtype=np.uint32)
    rc = load().fpclbm_closure_pack(w.ctypes.data_as(ctypes.POINTER(ctypes.c_ushort)), w.size,
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)), out.size)
    if rc != FPCLBM_OK:
        raise FpclbmError(rc, "fpclbm_closure_pack: %d weights" % w.size)
    return out


def noalloc_args_check(f_numel: int, f_device: int, out_numel: int, out_device: int, current_device: int,
                       ncells: int):
    """Host-side checks of fpclbm_diagnostics_noalloc's buffers, made before any CUDA call: the C
    entry point sees only raw pointers, so a cell count beyond the populations' length would make
    its kernel read past the end of f.  Raises ValueError on a mismatch."""
    ncells = int(ncells)
    # counts outside [1, 2^31 - 1] are left to the library, which rejects them with FPCLBM_ERR_ARG
    if 1 <= ncells <= 2 ** 31 - 1 and f_numel < 27 * ncells:
        raise ValueError("f_dev holds %d values, fewer than 27 * ncells = %d" % (f_numel, 27 * ncells))
    if out_numel < 5:
        raise ValueError("out_dev holds %d values, needs 5" % out_numel)
    if not (f_device == out_device == current_device):
        raise ValueError("f_dev (cuda:%s) and out_dev (cuda:%s) must be on the current device cuda:%s"
                         % (f_device, out_device, current_device))


def fpclbm_diagnostics_noalloc(f_dev, ncells: int, Fx: float, Fy: float, Fz: float, out_dev, stream: int = 0):
    """Diagnostics of full populations already on the device, without any allocation by the
    library: f_dev is a CUDA float64 tensor of at least 27 * ncells values (alpha-major), out_dev
    a CUDA float64 tensor of at least 5, both on the current device.  Runs on `stream` (a
    cudaStream_t handle, 0 = default) and does not synchronise."""
    import torch
    for name, t in (("f_dev", f_dev), ("out_dev", out_dev)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("%s must be a CUDA torch tensor" % name)
    noalloc_args_check(f_dev.numel(), f_dev.device.index, out_dev.numel(), out_dev.device.index,
                       torch.cuda.current_device(), ncells)
    rc = load().fpclbm_diagnostics_noalloc(_ptr(f_dev, 1), int(ncells), float(Fx), float(Fy), float(Fz),
                                           _ptr(out_dev, 1), _P(stream) if stream else None)
    return _check(None, rc)


def _fptr(a, on_device: bool):
    """Pointer of a float32 array (numpy host array, or torch tensor on the matching device)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float32 or not a.is_contiguous() or a.is_cuda != bool(on_device):
                raise TypeError("need a contiguous float32 tensor on the %s" % ("GPU" if on_device else "host"))
            return ctypes.c_void_p(a.data_ptr())
    except ImportError:  # pragma: no cover
        pass
    if on_device:
        raise TypeError("on_device=1 needs a CUDA torch tensor")
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]):
        raise TypeError("host arrays must be C-contiguous float32 numpy arrays")
    return ctypes.c_void_p(a.ctypes.data)


def fpclbm_closure_sample(h, r: int, tau_coarse: float, X, T, on_device: int = 0):
    """Features X [nc, 9] and labels T [nc] (float32) of the r^3-filtered fine box."""
    return _check(h, load().fpclbm_closure_sample(h, int(r), float(tau_coarse), _fptr(X, on_device),
                                                  _fptr(T, on_device), int(on_device)))


def fpclbm_closure_train(X_dev, T_dev, n: int, epochs: int, batch: int, lr: float, seed: int = 0, stream: int = 0):
    """Train on device tensors; returns (bf16 weight bits [4865] uint16, loss per epoch)."""
    w = np.zeros(4865, dtype=np.uint16)
    losses = np.zeros(int(epochs))
    rc = load().fpclbm_closure_train(_fptr(X_dev, 1), _fptr(T_dev, 1), int(n), int(epochs), int(batch), float(lr),
                                     int(seed), w.ctypes.data_as(ctypes.POINTER(ctypes.c_ushort)),
                                     losses.ctypes.data_as(_D), _P(stream) if stream else None)
    _check(None, rc)
    return w, losses


def fpclbm_closure_grad(X_dev, T_dev, n: int, bf16_bits, stream: int = 0):
    """(loss, grad [4865] float32) of the network with the given bf16 weights on device samples."""
    w = np.ascontiguousarray(np.asarray(bf16_bits, dtype=np.uint16))
    g = np.zeros(4865, dtype=np.float32)
    loss = ctypes.c_double()
    rc = load().fpclbm_closure_grad(_fptr(X_dev, 1), _fptr(T_dev, 1), int(n),
                                    w.ctypes.data_as(ctypes.POINTER(ctypes.c_ushort)), _fptr(g, 0),
                                    ctypes.byref(loss), _P(stream) if stream else None)
    _check(None, rc)
    return loss.value, g


def fpclbm_destroy(h):
    return load().fpclbm_destroy(h)


def fpclbm_last_error(h) -> str:
    m = load().fpclbm_last_error(h)
    return m.decode() if m else ""


# --- convenience wrapper ------------------------------------------------------------------

class Lattice:
    """One box (or ensemble) handle; methods map 1:1 onto the C calls."""

    def __init__(self, nx: int, ny: int, nz: int, precision="fp32", bc: int = FPCLBM_BC_PERIODIC, stream: int = 0):
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.shape = (nz, ny, nx)
        self.ncells = nx * ny * nz
        self.h = fpclbm_create(nx, ny, nz, self.precision, bc, stream)

    @classmethod
    def ensemble(cls, dims, tau, precision="fp32", stream: int = 0):
        self = cls.__new__(cls)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        d = np.asarray(dims, dtype=np.int64).reshape(-1, 3)
        self.shape = None
        self.ncells = int(np.sum(np.prod(d, axis=1)))
        self.h = fpclbm_create_ensemble(d, tau, self.precision, stream)
        return self

    def close(self):
        if getattr(self, "h", None) is not None:
            fpclbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _f64(a):
        return np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)

    @classmethod
    def _sized(cls, a, n, what):
        """float64, flat and exactly n values: the library reads n values behind the pointer."""
        a = cls._f64(a)
        if a.size != n:
            raise ValueError("%s: expected %d values, got %d" % (what, n, a.size))
        return a

    def init_fields(self, rho, ux, uy, uz):
        arrs = [self._sized(a, self.ncells, q) for a, q in zip((rho, ux, uy, uz), ("rho", "ux", "uy", "uz"))]
        return fpclbm_init_fields(self.h, *arrs, on_device=0)

    def set_params(self, tau, drift=0.0, diffusion=FPCLBM_DIFF_FP):
        return fpclbm_set_params(self.h, tau, drift, diffusion)

    def set_rates(self, omega):
        return fpclbm_set_rates(self.h, omega)

    def set_force(self, Fx, Fy=0.0, Fz=0.0):
        return fpclbm_set_force(self.h, Fx, Fy, Fz)

    def set_wall_velocity(self, ux, uz=0.0):
        return fpclbm_set_wall_velocity(self.h, ux, uz)

    def set_smagorinsky(self, cs, u_star=0.0, a_plus=26.0):
        return fpclbm_set_smagorinsky(self.h, cs, u_star, a_plus)

    def step(self, n: int = 1):
        return fpclbm_step(self.h, n)

    def moments(self):
        outs = [np.empty(self.ncells) for _ in range(4)]
        fpclbm_moments(self.h, *outs, on_device=0)
        if self.shape is not None:
            outs = [o.reshape(self.shape) for o in outs]
        return tuple(outs)

    def diagnostics(self):
        return fpclbm_diagnostics(self.h)

    def get_populations(self):
        f = np.empty((27, self.ncells))
        fpclbm_get_populations(self.h, f)
        return f.reshape((27,) + self.shape) if self.shape is not None else f

    def set_populations(self, f):
        return fpclbm_set_populations(self.h, self._sized(f, 27 * self.ncells, "populations"))

    def populations_at(self, cells):
        return fpclbm_get_populations_at(self.h, cells)

    def step_count(self) -> int:
        return fpclbm_get_step_count(self.h)

    def launch(self) -> dict:
        return fpclbm_get_launch(self.h)

    def get_state(self):
        return fpclbm_get_state(self.h)

    def set_state(self, raw, steps: int):
        return fpclbm_set_state(self.h, raw, steps)

    def set_closure(self, bf16_bits):
        return fpclbm_set_closure(self.h, bf16_bits)


# --- the 2D (D2Q9) handle -----------------------------------------------------------------

def _check2(h, rc: int):
    if rc != FPCLBM_OK:
        msg = load().fpclbm2d_last_error(h)
        raise FpclbmError(rc, msg.decode() if msg else "")
    return rc


def fpclbm2d_create(nx: int, ny: int, precision: int, stream: int = 0):
    h = _P()
    _check2(None, load().fpclbm2d_create(ctypes.byref(h), nx, ny, precision, _P(stream) if stream else None))
    return h


def fpclbm2d_init_fields(h, rho, ux, uy, on_device: int = 0):
    return _check2(h, load().fpclbm2d_init_fields(h, *(_ptr(a, on_device) for a in (rho, ux, uy)), int(on_device)))


def fpclbm2d_set_params(h, tau: float, bulk_rate: float = 0.0, drift: float = 0.0, diffusion: int = FPCLBM_DIFF_FP):
    return _check2(h, load().fpclbm2d_set_params(h, float(tau), float(bulk_rate), float(drift), int(diffusion)))


def fpclbm2d_set_rates(h, omega):
    om = np.ascontiguousarray(np.asarray(omega, dtype=np.float64)).reshape(-1)
    if om.size != 9:
        raise ValueError("omega needs 9 rates, got %d" % om.size)
    return _check2(h, load().fpclbm2d_set_rates(h, om.ctypes.data_as(_D)))


def fpclbm2d_set_force(h, Fx: float, Fy: float):
    return _check2(h, load().fpclbm2d_set_force(h, float(Fx), float(Fy)))


def fpclbm2d_set_boundary(h, bc: int, lid_ux: float = 0.0):
    return _check2(h, load().fpclbm2d_set_boundary(h, int(bc), float(lid_ux)))


def fpclbm2d_step(h, n: int):
    return _check2(h, load().fpclbm2d_step(h, int(n)))


def fpclbm2d_moments(h, rho, ux, uy, on_device: int = 0):
    return _check2(h, load().fpclbm2d_moments(h, *(_ptr(a, on_device) for a in (rho, ux, uy)), int(on_device)))


def fpclbm2d_get_populations(h, f):
    return _check2(h, load().fpclbm2d_get_populations(h, _ptr(f, 0)))


def fpclbm2d_set_populations(h, f):
    return _check2(h, load().fpclbm2d_set_populations(h, _ptr(f, 0)))


def fpclbm2d_destroy(h):
    return load().fpclbm2d_destroy(h)


def fpclbm2d_last_error(h) -> str:
    m = load().fpclbm2d_last_error(h)
    return m.decode() if m else ""


class Lattice2D:
    """One periodic D2Q9 box; methods map 1:1 onto the fpclbm2d_* calls.  Arrays are [ny, nx]."""

    def __init__(self, nx: int, ny: int, precision="fp32", stream: int = 0):
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.shape = (ny, nx)
        self.ncells = nx * ny
        self.h = fpclbm2d_create(nx, ny, self.precision, stream)

    def close(self):
        if getattr(self, "h", None) is not None:
            fpclbm2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _f64(a):
        return np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)

    @classmethod
    def _sized(cls, a, n, what):
        """float64, flat and exactly n values: the library reads n values behind the pointer."""
        a = cls._f64(a)
        if a.size != n:
            raise ValueError("%s: expected %d values, got %d" % (what, n, a.size))
        return a

    def init_fields(self, rho, ux, uy):
        return fpclbm2d_init_fields(self.h, *(self._sized(a, self.ncells, q) for a, q in
                                              zip((rho, ux, uy), ("rho", "ux", "uy"))))

    def set_params(self, tau, bulk_rate=0.0, drift=0.0, diffusion=FPCLBM_DIFF_FP):
        return fpclbm2d_set_params(self.h, tau, bulk_rate, drift, diffusion)

    def set_rates(self, omega):
        return fpclbm2d_set_rates(self.h, omega)

    def set_force(self, Fx, Fy=0.0):
        return fpclbm2d_set_force(self.h, Fx, Fy)

    def set_boundary(self, bc, lid_ux=0.0):
        return fpclbm2d_set_boundary(self.h, bc, lid_ux)

    def step(self, n: int = 1):
        return fpclbm2d_step(self.h, n)

    def moments(self):
        outs = [np.empty(self.ncells) for _ in range(3)]
        fpclbm2d_moments(self.h, *outs)
        return tuple(o.reshape(self.shape) for o in outs)

    def get_populations(self):
        f = np.empty((9, self.ncells))
        fpclbm2d_get_populations(self.h, f)
        return f.reshape((9,) + self.shape)

    def set_populations(self, f):
        return fpclbm2d_set_populations(self.h, self._sized(f, 9 * self.ncells, "populations"))
