"""GPU restart with a change of resolution against the oracle's regrid.

The interpolation itself differs from the oracle only by rounding (barycentric
weights on the GPU side, the Lagrange product form in the oracle): 1e-12 of
the largest coefficient.  A coarse run restarted on a finer grid and stepped
on matches the same sequence in the oracle to relative L2 1e-10.
"""
import math

import numpy as np
import pytest

from inputs import Workload, psi_coefficients, random_state, temperature_coefficients
from oracle import Model
from oracle.regrid import regrid

pytestmark = pytest.mark.gpu

COARSE = Workload("rg_c", Nr=16, Ntheta=24, Nz=24, eta=0.6, Lz=2.4, Re_i=90.0, Re_o=-20.0,
                  amp=3e-2, mp=3, kp=3, seed=41, dt=1e-3)
FINE = COARSE.scaled(name="rg_f", Nr=27, Ntheta=36, Nz=40)


@pytest.fixture(scope="module")
def tc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1908_00587_gb300 import tc as mod
    return mod


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel_l2(mdl, a, b):
    w = (mdl.g.w * mdl.g.r)[:, None, None] * mdl.sp.cm[None, :, None]
    return max(float(np.sqrt(np.sum(w * np.abs(a[f] - b[f]) ** 2) / np.sum(w * np.abs(b[f]) ** 2)))
               for f in range(a.shape[0]))


@pytest.mark.parametrize("src,dst,where", [(COARSE, FINE, 0), (FINE, COARSE, 1),
                                           (COARSE, COARSE, 0)])
def test_regrid_matches_oracle(tc, src, dst, where):
    ms, md = Model(src), Model(dst)
    X = random_state(42, ms.nf, src.Nr, ms.M, ms.K)
    ref = regrid(X, src.eta, md)
    run = tc.Run.from_workload(dst)
    run.set_state_regrid(X if where == 0 else dev(X), src.eta, src.Lz)
    got = run.get_state()
    run.close()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_regrid_adds_conductive_temperature(tc):
    heated = FINE.scaled(Ra=1200.0, Pr=0.7)
    ms, md = Model(COARSE), Model(heated)
    X = random_state(43, 3, COARSE.Nr, ms.M, ms.K)
    ref = regrid(X, COARSE.eta, md)
    run = tc.Run.from_workload(heated)
    base = run.get_state()            # the library's own discrete basic state
    run.set_state_regrid(X, COARSE.eta, COARSE.Lz)
    got = run.get_state()
    run.close()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    np.testing.assert_array_equal(got[3], base[3])


def test_restart_on_finer_grid_matches_oracle(tc):
    psi = psi_coefficients(COARSE.seed, COARSE.mp, COARSE.kp)
    run_c = tc.Run.from_workload(COARSE)
    run_c.init_perturbation(psi, COARSE.amp)
    run_c.step(15, COARSE.dt)
    Xc = run_c.get_state()
    run_c.close()
    run_f = tc.Run.from_workload(FINE)
    run_f.set_state_regrid(Xc, COARSE.eta, COARSE.Lz)
    run_f.step(15, FINE.dt)
    got = run_f.get_state()
    run_f.close()
    mc, mf = Model(COARSE, "fft"), Model(FINE, "fft")
    X = mc.initial_state(psi)
    for _ in range(15):
        X, _, _, _ = mc.step(X, COARSE.dt)
    assert rel_l2(mc, Xc, X) <= 1e-10
    X = regrid(X, COARSE.eta, mf)
    for _ in range(15):
        X, _, _, _ = mf.step(X, FINE.dt)
    assert rel_l2(mf, got, X) <= 1e-10


def test_regrid_rejects_other_geometry(tc):
    st = {v: k for k, v in tc.STATUS.items()}
    run = tc.Run.from_workload(FINE)
    ms = Model(COARSE)
    X = random_state(44, ms.nf, COARSE.Nr, ms.M, ms.K)
    for eta, Lz in ((0.5, COARSE.Lz), (COARSE.eta, 2.0)):
        assert tc._lib.tc_set_state_regrid(run.ctx, X.ctypes.data, COARSE.Nr, ms.M, ms.K, 3,
                                           eta, Lz, 0) == st["TC_ERR_ARG"]
    run.close()
