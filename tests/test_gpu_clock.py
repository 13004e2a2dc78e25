"""The run's clock (simulated time and the dynamic step's memory).

tc_set_state forgets the step history, so the next dynamic step is the CFL
step dt* itself; tc_set_clock puts a saved history back.  A run restarted
from host memory before every step, state and clock, must follow the run
stepped on the device: the same steps and the state to round-off (the
restart takes the Laplacian by its stencil where the device run reuses the
last stage's equation, and symmetrises the m = 0 column).  The step rule
(Sec. 2.1, dynamic time-step control): dt* when dt* < dt_prev or dt* > 1.1
dt_prev, else dt_prev."""
import numpy as np
import pytest

from inputs import WORKLOADS, psi_coefficients, temperature_coefficients

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


WL = WORKLOADS["tc_fp64T_nr64_n128"].scaled(Nr=24, Ntheta=32, Nz=48, mp=4, kp=4)


def _run(tc, steps_before=0):
    run = tc.Run.from_workload(WL)
    tco = temperature_coefficients(WL.seed, WL.mp, WL.kp)
    run.init_perturbation(psi_coefficients(WL.seed, WL.mp, WL.kp), WL.amp, tco, WL.amp_T)
    if steps_before:
        run.step(steps_before, 0.0)
    return run


def _rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_clock_follows_steps_and_resets(tc):
    run = _run(tc)
    assert run.get_clock() == (0.0, 0.0)
    used = run.step(3, 0.0)
    t, dtp = run.get_clock()
    assert dtp == used[-1]
    assert t == (used[0] + used[1]) + used[2]
    run.set_clock(1.25, 3e-4)
    assert run.get_clock() == (1.25, 3e-4)
    run.set_state(run.get_state())
    assert run.get_clock() == (0.0, 0.0)
    for bad in [(float("nan"), 1e-4), (0.0, -1e-4), (0.0, float("inf"))]:
        with pytest.raises(tc.TCError) as e:
            run.set_clock(*bad)
        assert e.value.name == "TC_ERR_ARG"
    run.close()


def test_step_rule_against_the_clock(tc):
    """With the state fixed, the first dynamic step is decided by dt* (from the
    CFL rate that tc_nonlinear reports for the same state) and dt_prev."""
    import torch
    run = _run(tc, steps_before=2)
    # tc_set_state symmetrises the m = 0 column; take the state it keeps, so
    # that the rate below is the rate of the state each step starts from
    run.set_state(run.get_state())
    X = run.get_state()
    Xd = torch.from_numpy(X).cuda()
    Nd = torch.empty_like(Xd)
    rate = tc.tc_nonlinear(run.ctx, Xd, Nd)
    dt_star = min(WL.dt_max, WL.cfl / rate)
    assert dt_star < WL.dt_max   # the CFL bound is the active one here
    for dtp, expect in [(0.0, dt_star),                 # no history
                        (dt_star / 1.05, dt_star / 1.05),   # dt* within (dt_prev, 1.1 dt_prev]: kept
                        (dt_star / 2.0, dt_star),       # dt* above 1.1 dt_prev
                        (dt_star * 1.5, dt_star)]:      # dt* below dt_prev
        run.set_state(X)
        run.set_clock(0.0, dtp)
        used = run.step(1, 0.0)
        assert used[0] == expect, (dtp, used[0], expect)
    run.close()


def test_host_restart_with_clock_follows_device_run(tc):
    n = 8
    A = _run(tc, steps_before=3)
    X0 = A.get_state()
    t0, dtp0 = A.get_clock()
    dA = A.step(n, 0.0)
    XA = A.get_state()
    tA, _ = A.get_clock()
    A.close()

    B = _run(tc)
    X = X0.copy()
    t, dtp = t0, dtp0
    dB = []
    for _ in range(n):
        B.set_state(X)
        B.set_clock(t, dtp)
        dtp = float(B.step(1, 0.0)[0])
        t += dtp
        dB.append(dtp)
        B.get_state(X)
    assert B.get_clock()[0] == t
    B.close()
    np.testing.assert_allclose(dB, dA, rtol=1e-12, atol=0.0)
    assert abs(t - tA) <= 1e-12 * tA
    assert _rel_l2(X, XA) <= 1e-10


def test_long_call_matches_split_calls(tc):
    """tc_step reads the step history through a pinned buffer of 1024 steps
    and through pageable memory for longer calls: one call of 1100 dynamic
    steps and calls of 1000 and 100 give the same steps, clock and state,
    bit for bit (a tiny grid, so that the steps are quick)."""
    wl = WORKLOADS["tc_fp64_nr32_n32"].scaled(Nr=12, Ntheta=8, Nz=12, mp=2, kp=2)
    res = []
    for split in ((1100,), (1000, 100)):
        run = tc.Run.from_workload(wl)
        run.init_perturbation(psi_coefficients(wl.seed, wl.mp, wl.kp), wl.amp)
        used = np.concatenate([run.step(n, 0.0) for n in split])
        res.append((used, run.get_clock(), run.get_state()))
        run.close()
    assert len(res[0][0]) == 1100
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1][1] == res[1][1][1]
    assert abs(res[0][1][0] - res[1][1][0]) <= 1e-12 * res[0][1][0]
    assert np.array_equal(res[0][2], res[1][2])
