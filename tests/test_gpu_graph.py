"""tc_step replays one captured step as a CUDA graph; the results, the step
history and the launch count must be exactly those of launching the kernels
one by one (option "graph" = 0), and option changes must re-capture."""
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


def _run(tc, wl, graph, plan):
    run = tc.Run.from_workload(wl)
    run.set_option("graph", graph)
    tco = temperature_coefficients(wl.seed, wl.mp, wl.kp) if wl.Ra else None
    run.init_perturbation(psi_coefficients(wl.seed, wl.mp, wl.kp), wl.amp, tco, wl.amp_T)
    l0 = tc.tc_get_info(run.ctx).launches
    dts = []
    for n, dt, opts in plan:
        for k, v in opts.items():
            run.set_option(k, v)
        dts.append(run.step(n, dt))
    launches = tc.tc_get_info(run.ctx).launches - l0
    X = run.get_state()
    d = run.diagnostics()
    run.close()
    return X, np.concatenate(dts), launches, d


def test_graph_replay_matches_direct_launches(tc):
    wl = WORKLOADS["tc_fp64T_nr64_n128"].scaled(Nr=20, Ntheta=24, Nz=36, mp=4, kp=4)
    plan = [(7, 0.0, {}),                       # dynamic dt, 7 steps in one call
            (3, 0.0, {"cfl": 0.2}),             # option change: re-capture
            (4, 2e-4, {}),                      # fixed dt: re-capture
            (2, 2e-4, {"n_corr": 2}),
            (1, 0.0, {"n_corr": 1})]
    Xg, dg, lg, diag_g = _run(tc, wl, 1, plan)
    Xd, dd, ld, diag_d = _run(tc, wl, 0, plan)
    np.testing.assert_array_equal(Xg, Xd)
    np.testing.assert_array_equal(dg, dd)
    assert lg == ld
    assert diag_g["corr_diff"] == diag_d["corr_diff"]
    assert len(dg) == 17 and np.all(dg > 0)
