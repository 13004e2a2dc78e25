"""The allocation-free nonlinear entry point against the context-based one.

tc_nonlinear_noalloc serves callers that cannot call cudaMalloc (a host
application whose pool owns the device memory, or a latency-critical loop
where an allocation could synchronise the device).  It keeps all its scratch
in one static device array, so this test checks, through the C ABI, that two
calls in a row reproduce what tc_nonlinear computes with its own allocated
buffers: the second call must not depend on what the first left behind.
This file is collected last so that a run stopping at the first failure has
run every other test already.
"""
import numpy as np
import pytest

from inputs import Workload, random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1908_00587_gb300 import tc as mod
    return mod


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


CASES = [
    Workload("na1", Nr=24, Ntheta=32, Nz=36, eta=0.71, Lz=2.0, Re_i=300.0, Re_o=-50.0,
             Ra=2e3, Pr=0.7),
    Workload("na2", Nr=17, Ntheta=30, Nz=20, eta=0.5, Lz=1.3, Re_i=90.0),
]


def test_noalloc_matches_context_entry_point_twice(tc):
    for call, wl in enumerate(CASES + CASES[:1]):   # different sizes, then back
        nf = 4 if wl.Ra else 3
        M, K = (wl.Ntheta - 1) // 3, (wl.Nz - 1) // 3
        X = random_state(700 + call, nf, wl.Nr, M, K)
        run = tc.Run.from_workload(wl)
        ref = _dev(np.zeros_like(X))
        rate_ref = tc.tc_nonlinear(run.ctx, _dev(X), ref)
        run.close()
        for rep in range(2):                           # two calls in a row
            out = _dev(np.full_like(X, np.nan))
            rate = tc.tc_nonlinear_noalloc(wl.Nr, wl.Ntheta, wl.Nz, wl.eta, wl.Lz, wl.Ra,
                                           wl.Pr, _dev(X), out)
            got, want = out.cpu().numpy(), ref.cpu().numpy()
            assert np.all(np.isfinite(got)), (call, rep)
            assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), (call, rep)
            assert abs(rate - rate_ref) <= 1e-13 * rate_ref, (call, rep)


def test_noalloc_rejects_sizes_beyond_its_scratch(tc):
    """Sizes are rejected by the library before it touches either buffer, so
    the raw C entry point is called with a small placeholder buffer (the
    Python wrapper would refuse it first, for its size)."""
    import ctypes
    x = _dev(np.zeros(8, dtype=np.complex128))
    p = ctypes.c_void_p(x.data_ptr())
    rate = ctypes.c_double(0.0)

    def status(*sizes):
        return tc.STATUS[tc._lib.tc_nonlinear_noalloc(*sizes, p, p, None, ctypes.byref(rate))]

    assert status(300, 32, 32, 0.5, 1.0, 0.0, 1.0) == "TC_ERR_UNSUPPORTED"
    # fits the size limits, not the 32 MiB
    assert status(128, 128, 128, 0.5, 1.0, 1e3, 0.7) == "TC_ERR_UNSUPPORTED"
    assert status(16, 31, 32, 0.5, 1.0, 0.0, 1.0) == "TC_ERR_ARG"
