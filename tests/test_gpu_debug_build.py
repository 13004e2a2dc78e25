"""The debug build (libtc_debug.so, -DTC_DEBUG) on small oracle-parity cases.

compute-sanitizer is not available here, so the debug build's own index
checks stand in for it (the paper's QA runs short tests with runtime checks
and out-of-bounds detection, Sec. 2.5): every checked access of the step,
stage and adjoint kernels must stay in range (no check bit set) while the
results still match the oracle.  It runs in a child process because the
binding loads one library per process (TC_LIB=debug)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
from inputs import Workload, psi_coefficients, temperature_coefficients, random_state
from oracle import Model
from paper_1908_00587_gb300 import tc
assert tc.LIB_PATH.endswith("libtc_debug.so")
tc.tc_debug_flags(clear=True)
worst = 0.0
for (Nr, Nt, Nz, Ra) in [(16, 12, 24, 300.0), (21, 30, 20, 0.0), (12, 64, 36, 500.0)]:
    wl = Workload("dbg", Nr=Nr, Ntheta=Nt, Nz=Nz, eta=0.6, Lz=2.0, Re_i=80.0, Re_o=-20.0,
                  Ra=Ra, Pr=0.9, amp=1e-2, mp=2, kp=2, amp_T=1e-2 if Ra else 0.0, seed=11,
                  dt=2e-3)
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    tco = temperature_coefficients(wl.seed, wl.mp, wl.kp) if Ra else None
    run = tc.Run.from_workload(wl)
    run.init_perturbation(psi, wl.amp, tco, wl.amp_T)
    run.step(3, wl.dt)
    got = run.get_state()
    mdl = Model(wl, "fft")
    X, _ = mdl.run(mdl.initial_state(psi, tco), 3, wl.dt)
    w = (mdl.g.w * mdl.g.r)[:, None, None] * mdl.sp.cm[None, :, None]
    for f in range(got.shape[0]):
        e = float(np.sqrt(np.sum(w * np.abs(got[f] - X[f]) ** 2) / np.sum(w * np.abs(X[f]) ** 2)))
        worst = max(worst, e)
    # the adjoint kernels (sweeps transposed) and the mixed form's kernels
    Xd = torch.from_numpy(got).cuda()
    lam = torch.from_numpy(random_state(5, run.nf, Nr, run.M, run.K)).cuda()
    if Ra == 0.0:
        tc.tc_adjoint_step(run.ctx, Xd, wl.dt, lam)
        tc.tc_set_option(run.ctx, "precision", 1)
        run.step(2, wl.dt)
    run.close()
flags = tc.tc_debug_flags()
print(f"debug build: worst rel L2 vs oracle {worst:.3e}, check bits {flags:#x}")
assert flags == 0, hex(flags)
assert worst <= 1e-10, worst
print("DEBUG_BUILD_OK")
"""


@pytest.mark.gpu
def test_debug_build_runs_clean_and_matches_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    env = dict(os.environ, TC_LIB="debug", PYTHONPATH=ROOT)
    res = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=600)
    print(res.stdout[-2000:], res.stderr[-2000:])
    assert res.returncode == 0 and "DEBUG_BUILD_OK" in res.stdout


def test_debug_entry_point_is_unsupported_in_the_normal_build():
    """In libtc.so the checks compile away and tc_debug_flags says so (no
    device call is made, so this runs without a GPU)."""
    import __graft_entry__ as g
    g.build()
    from paper_1908_00587_gb300 import tc
    if tc.LIB_PATH.endswith("libtc_debug.so"):
        pytest.skip("the debug build is loaded in this process")
    with pytest.raises(tc.TCError) as e:
        tc.tc_debug_flags()
    assert e.value.name == "TC_ERR_UNSUPPORTED"


def test_debug_library_exports_the_same_symbols():
    import ctypes
    import __graft_entry__ as g
    g.build()
    from paper_1908_00587_gb300 import build, tc
    lib = ctypes.CDLL(build.LIB_DEBUG)
    for name in tc.EXPORTED:
        assert hasattr(lib, name), name
