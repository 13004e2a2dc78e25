"""Error paths of a running context, made on the host or by the numerics, never
by a GPU fault: a step whose state turns non-finite, and a memory budget that
refuses allocations made after tc_create.  The context stays usable after each."""
import numpy as np
import pytest

from inputs import Workload, psi_coefficients

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


WL = Workload("err", Nr=16, Ntheta=16, Nz=16, eta=0.6, Lz=1.7, Re_i=1e4, Re_o=0.0,
              amp=1e-1, mp=2, kp=2, seed=9, dt=1e-5)


def test_step_that_blows_up_reports_nonfinite(tc):
    """A fixed step of dt = 1 at Re_i = 1e4 puts the explicit nonlinear term
    at a CFL number of ~1e5: the perturbation grows without bound and
    overflows within a few steps.  tc_step must return TC_ERR_NONFINITE (the
    exponent check of the corrector's output), and the context must take a
    valid state and step normally afterwards."""
    run = tc.Run.from_workload(WL)
    base = run.get_state()
    run.init_perturbation(psi_coefficients(WL.seed, WL.mp, WL.kp), WL.amp)
    with pytest.raises(tc.TCError) as e:
        for _ in range(20):
            run.step(10, 1.0)
    assert e.value.name == "TC_ERR_NONFINITE"
    assert not np.all(np.isfinite(run.get_state()))
    run.set_state(base)
    run.step(3, WL.dt)
    X = run.get_state()
    assert np.all(np.isfinite(X))
    assert np.abs(X - base).max() <= 1e-12 * np.abs(base).max()   # basic state kept
    run.close()


def test_memory_budget_refuses_later_allocations(tc):
    """With the budget at what tc_create allocated, every later allocation
    returns TC_ERR_OOM and changes nothing; lifting the budget lets the same
    calls through, and the results equal those of a run that never hit it."""
    import torch
    psi = psi_coefficients(WL.seed, WL.mp, WL.kp)
    run = tc.Run.from_workload(WL)
    run.init_perturbation(psi, WL.amp)
    X0 = run.get_state()
    held = tc.tc_get_info(run.ctx).device_bytes
    tc.tc_set_option(run.ctx, "memory_budget", held)

    def oom(fn):
        with pytest.raises(tc.TCError) as e:
            fn()
        assert e.value.name == "TC_ERR_OOM"

    oom(lambda: tc.tc_set_option(run.ctx, "precision", 1))          # FP32 state copy
    Xd = torch.from_numpy(X0).cuda()
    lam = torch.zeros_like(Xd)
    oom(lambda: tc.tc_adjoint_step(run.ctx, Xd, WL.dt, lam))         # adjoint buffers
    oom(lambda: run.step(5000, WL.dt))                                # longer step history
    oom(lambda: tc.tc_set_option(run.ctx, "flux_constraint", 1))     # flux response
    oom(lambda: run.set_state_regrid(X0, WL.eta, WL.Lz))             # regrid scratch
    assert tc.tc_get_info(run.ctx).device_bytes == held
    np.testing.assert_array_equal(run.get_state(), X0)               # nothing changed
    run.step(4, WL.dt)                                                # still steps
    X_budget = run.get_state()
    tc.tc_set_option(run.ctx, "memory_budget", 0)                    # lifted
    tc.tc_adjoint_step(run.ctx, Xd, WL.dt, lam)
    assert tc.tc_get_info(run.ctx).device_bytes > held
    run.close()
    ref = tc.Run.from_workload(WL)
    ref.init_perturbation(psi, WL.amp)
    ref.step(4, WL.dt)
    np.testing.assert_array_equal(ref.get_state(), X_budget)
    ref.close()
