"""The C ABI library builds, loads and exports every symbol the header declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fpclbm.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"FPCLBM_API\s+[\w\s\*]+?\b(fpclbm(?:2d)?_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2410_09739_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for core in ("fpclbm_create", "fpclbm_init_fields", "fpclbm_set_params", "fpclbm_step", "fpclbm_moments",
                 "fpclbm_destroy"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2410_09739_gb300 import fpclbm as F
    assert sorted(F.EXPORTED) == declared_symbols()
    for name in declared_symbols():
        assert callable(getattr(F, name)), name


def test_null_handle_calls_fail_cleanly(lib):
    lib.fpclbm_destroy.argtypes = [ctypes.c_void_p]
    assert lib.fpclbm_destroy(None) == 0
    lib.fpclbm_step.argtypes = [ctypes.c_void_p, ctypes.c_longlong]
    assert lib.fpclbm_step(None, 1) == -1
    lib.fpclbm_last_error.restype = ctypes.c_char_p
    lib.fpclbm_last_error.argtypes = [ctypes.c_void_p]
    assert isinstance(lib.fpclbm_last_error(None), bytes)


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    h = ctypes.c_void_p()
    lib.fpclbm_create.argtypes = [ctypes.POINTER(ctypes.c_void_p)] + [ctypes.c_int] * 5 + [ctypes.c_void_p]
    assert lib.fpclbm_create(ctypes.byref(h), 0, 4, 4, 1, 0, None) == -1
    assert lib.fpclbm_create(ctypes.byref(h), 4, 4, 4, 9, 0, None) == -1
    assert lib.fpclbm_create(ctypes.byref(h), 4, 4, 4, 1, 7, None) == -1
    assert lib.fpclbm_create(ctypes.byref(h), 1024, 1024, 1024, 1, 0, None) == -1
    assert h.value is None
    assert b"dimensions" in lib.fpclbm_last_error(None) or True


def test_missing_library_raises(tmp_path):
    from paper_2410_09739_gb300 import fpclbm as F
    saved = F._lib
    try:
        F._lib = None
        with pytest.raises(FileNotFoundError):
            F.load(str(tmp_path / "nope.so"))
    finally:
        F._lib = saved


def test_wrappers_reject_wrongly_sized_arrays_before_calling_the_library():
    """The C ABI cannot see the length of a host buffer; the Python wrappers check it, so a wrong
    size raises instead of letting the library read past the end of the array."""
    import numpy as np
    from paper_2410_09739_gb300 import fpclbm as F
    lat = F.Lattice.__new__(F.Lattice)  # no device handle: every check must fire before the call
    lat.ncells, lat.shape, lat.h = 4 * 3 * 2, (2, 3, 4), None
    good = np.ones((2, 3, 4))
    with pytest.raises(ValueError, match="uy"):
        lat.init_fields(good, good, np.ones(5), good)
    with pytest.raises(ValueError, match="populations"):
        lat.set_populations(np.ones((27, 23)))
    lat2 = F.Lattice2D.__new__(F.Lattice2D)
    lat2.ncells, lat2.shape, lat2.h = 12, (3, 4), None
    with pytest.raises(ValueError, match="rho"):
        lat2.init_fields(np.ones(11), np.ones(12), np.ones(12))
    with pytest.raises(ValueError, match="populations"):
        lat2.set_populations(np.ones((9, 13)))
    with pytest.raises(ValueError, match="27 rates"):
        F.fpclbm_set_rates(None, np.ones(26))
    with pytest.raises(ValueError, match="9 rates"):
        F.fpclbm2d_set_rates(None, np.ones(10))


def test_other_entry_points_reject_bad_arguments_before_touching_the_device(lib):
    """Argument checks of the ensemble, D2Q9 and no-allocation entry points run on the host before
    any CUDA call, so they can be exercised without a GPU."""
    P = ctypes.c_void_p
    h = P()
    lib.fpclbm_create_ensemble.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_int, P]
    dims = (ctypes.c_int * 6)(8, 8, 8, 4, 0, 4)
    tau = (ctypes.c_double * 2)(0.6, 0.6)
    assert lib.fpclbm_create_ensemble(ctypes.byref(h), 0, dims, tau, 1, None) == -1       # no boxes
    assert lib.fpclbm_create_ensemble(ctypes.byref(h), 1, dims, tau, 0, None) == -1       # FP32 only
    assert lib.fpclbm_create_ensemble(ctypes.byref(h), 2, dims, tau, 1, None) == -1       # a side of 0
    bad_tau = (ctypes.c_double * 1)(0.4)                                                   # 1/tau = 2.5
    assert lib.fpclbm_create_ensemble(ctypes.byref(h), 1, dims, bad_tau, 1, None) == -4
    assert h.value is None
    lib.fpclbm2d_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
    assert lib.fpclbm2d_create(ctypes.byref(h), 0, 8, 1, None) == -1
    assert lib.fpclbm2d_create(ctypes.byref(h), 8, 8, 7, None) == -1
    assert lib.fpclbm2d_create(ctypes.byref(h), 65536, 65536, 1, None) == -1
    assert h.value is None
    lib.fpclbm_diagnostics_noalloc.argtypes = [P, ctypes.c_longlong, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, P, P]
    dummy = P(256)  # never dereferenced: every call below fails its checks first
    assert lib.fpclbm_diagnostics_noalloc(None, 8, 0.0, 0.0, 0.0, dummy, None) == -1
    assert lib.fpclbm_diagnostics_noalloc(dummy, 0, 0.0, 0.0, 0.0, dummy, None) == -1
    assert lib.fpclbm_diagnostics_noalloc(dummy, 2 ** 31, 0.0, 0.0, 0.0, dummy, None) == -1
    assert lib.fpclbm_diagnostics_noalloc(dummy, 8, float("inf"), 0.0, 0.0, dummy, None) == -1
    lib.fpclbm_last_error.restype = ctypes.c_char_p
    lib.fpclbm_last_error.argtypes = [P]
    assert b"finite" in lib.fpclbm_last_error(None)


def test_noalloc_wrapper_checks_buffers_before_calling_the_library():
    """fpclbm_diagnostics_noalloc's C entry point sees raw device pointers only; the wrapper checks
    the populations' length against 27 * ncells, the result's length and the devices first."""
    from paper_2410_09739_gb300 import fpclbm as F
    ok = dict(f_numel=27 * 10, f_device=0, out_numel=5, out_device=0, current_device=0, ncells=10)
    F.noalloc_args_check(**ok)
    for bad in (dict(f_numel=27 * 10 - 1), dict(ncells=11), dict(out_numel=4), dict(f_device=1),
                dict(out_device=1), dict(current_device=1)):
        with pytest.raises(ValueError):
            F.noalloc_args_check(**{**ok, **bad})
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):  # host tensors are not device pointers
        F.fpclbm_diagnostics_noalloc(torch.zeros(27, dtype=torch.float64), 1, 0, 0, 0,
                                     torch.zeros(5, dtype=torch.float64))
