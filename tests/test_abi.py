"""Host-only checks of the C ABI: the library loads, exports every symbol the
header declares, and rejects invalid arguments before touching the GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tc():
    import __graft_entry__ as g
    g.build()
    from paper_1908_00587_gb300 import tc as mod
    return mod


def _declared():
    src = open(os.path.join(ROOT, "include", "tc.h")).read()
    return sorted(set(re.findall(r"^\s*(?:tc_status|const char \*)\s*(tc_\w+)\s*\(", src, re.M)))


def test_header_symbols_exported(tc):
    import ctypes
    lib = ctypes.CDLL(tc.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) <= set(tc.EXPORTED)


@pytest.mark.parametrize("args", [
    (8, 32, 32, 0.5, 1.0, 100.0, 0.0, 0.0, 1.0),      # Nr < 9
    (16, 31, 32, 0.5, 1.0, 100.0, 0.0, 0.0, 1.0),     # Ntheta odd
    (16, 32, 14, 0.5, 1.0, 100.0, 0.0, 0.0, 1.0),     # Nz has factor 7
    (16, 2, 32, 0.5, 1.0, 100.0, 0.0, 0.0, 1.0),      # Ntheta < 4
    (16, 32, 32, 1.0, 1.0, 100.0, 0.0, 0.0, 1.0),     # eta = 1
    (16, 32, 32, 0.0, 1.0, 100.0, 0.0, 0.0, 1.0),     # eta = 0
    (16, 32, 32, 0.5, 0.0, 100.0, 0.0, 0.0, 1.0),     # Lz = 0
    (16, 32, 32, 0.5, 1.0, 100.0, 0.0, 1e3, 0.0),     # Pr = 0 with Ra != 0
    (16, 32, 32, 0.5, 1.0, float("nan"), 0.0, 0.0, 1.0),
    (2048, 32, 32, 0.5, 1.0, 100.0, 0.0, 0.0, 1.0),   # Nr too large
])
def test_create_rejects_bad_arguments(tc, args):
    with pytest.raises(tc.TCError) as e:
        tc.tc_create(*args)
    assert e.value.name == "TC_ERR_ARG"


def test_null_handles(tc):
    import ctypes
    lib = ctypes.CDLL(tc.LIB_PATH)
    lib.tc_destroy.argtypes = [ctypes.c_void_p]
    assert lib.tc_destroy(None) == 0
    lib.tc_set_option.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_double]
    assert lib.tc_set_option(None, b"cfl", 0.3) == 1
    lib.tc_step.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
    assert lib.tc_step(None, 1, 1e-3, None) == 1
    lib.tc_diagnostics.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.tc_diagnostics(None, None) == 1
    lib.tc_get_clock.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.tc_get_clock(None, None, None) == 1
    lib.tc_set_clock.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
    assert lib.tc_set_clock(None, 0.0, 1e-4) == 1


def test_status_strings(tc):
    for s in range(9):
        assert tc.tc_status_string(s)
    assert "unknown" in tc.tc_status_string(42)


def test_fp64_rate_rejects_bad_arguments(tc):
    """The measurement aid validates its arguments before touching the device."""
    import ctypes
    lib = ctypes.CDLL(tc.LIB_PATH)
    lib.tc_measure_fp64_rate.argtypes = [ctypes.c_double, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_double)]
    out = ctypes.c_double(0.0)
    assert lib.tc_measure_fp64_rate(0.0, None, ctypes.byref(out)) == 1
    assert lib.tc_measure_fp64_rate(-5.0, None, ctypes.byref(out)) == 1
    assert lib.tc_measure_fp64_rate(2e4, None, ctypes.byref(out)) == 1
    assert lib.tc_measure_fp64_rate(100.0, None, None) == 1


def test_binding_rejects_short_or_host_buffers(tc):
    """The binding checks dtype, size and device placement of state buffers
    before any library call, so a short or host buffer never reaches a kernel
    (these raise before touching the GPU)."""
    import numpy as np
    nf, Nr, M1, NK = 3, 16, 4, 7    # Ntheta = Nz = 12: M = K = 3
    good = np.zeros((nf, Nr, M1, NK), dtype=np.complex128)
    with pytest.raises(ValueError):            # host arrays are not device pointers
        tc.tc_nonlinear_noalloc(Nr, 12, 12, 0.5, 1.0, 0.0, 1.0, good, good)
    with pytest.raises((ValueError, TypeError)):
        tc._sized(good[:, :8], good.size, "short", False)
    with pytest.raises(ValueError):
        tc._sized(good.real.copy(), good.size, "float64", False)
    p, where = tc._sized(good, good.size, "ok", False)
    assert where == 0 and p == good.ctypes.data
