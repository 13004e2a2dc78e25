"""Ensemble form: independent runs of uneven size replayed as one CUDA graph
(mode 0, default) or in one persistent launch (mode 1).

Each member must give exactly what the same run gives on its own (the launch
mode only changes when and where each CTA tile runs; the autotuned tiles only
change which CTA computes a transform), and small FP64 members are pinned to
the oracle.  Per-member fixed step: dt = min(1e-3, 0.25 / CFL rate of u0).
"""
import numpy as np
import pytest

from inputs import ensemble_members, psi_coefficients
from oracle import Model

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


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _init(tc, ctx, wl):
    tc.tc_init_perturbation(ctx, psi_coefficients(wl.seed, wl.mp, wl.kp), wl.amp)
    info = tc.tc_get_info(ctx)
    shape = (info.nfields, info.Nr, info.M + 1, 2 * info.K + 1)
    X = np.empty(shape, dtype=np.complex128)
    tc.tc_get_state(ctx, X)
    out = dev(np.zeros_like(X))
    rate = tc.tc_nonlinear(ctx, dev(X), out)
    return min(1e-3, 0.25 / rate), shape


@pytest.mark.parametrize("mode", [1, 0], ids=["persistent", "graph"])
def test_ensemble_members_match_single_runs_bitwise(tc, mode):
    members = [w.scaled(precision=i % 2) for i, w in enumerate(ensemble_members(6))]
    ens = tc.tc_ensemble_create(members, autotune_tiles=True)
    tc.tc_ensemble_set_mode(ens, mode)
    assert tc.tc_ensemble_get_mode(ens) == mode
    dts, shapes, tensor = [], [], []
    for i, wl in enumerate(members):
        dt, shape = _init(tc, tc.tc_ensemble_member(ens, i), wl)
        dts.append(dt)
        shapes.append(shape)
        info = tc.tc_get_info(tc.tc_ensemble_member(ens, i))
        assert info.tile_mb >= 1 and info.tile_lb >= 1
        tensor.append((info.tensor_theta, info.tensor_z))
    tc.tc_ensemble_step(ens, 7, dts)
    tc.tc_ensemble_step(ens, 5, dts)       # the same plan (graph) again
    if mode == 1:
        assert tc.tc_ensemble_kernels_per_step(ens) == 1
    else:
        assert tc.tc_ensemble_kernels_per_step(ens) > 18 * len(members) - 1
    got = []
    for i in range(len(members)):
        X = np.empty(shapes[i], dtype=np.complex128)
        tc.tc_get_state(tc.tc_ensemble_member(ens, i), X)
        got.append(X)
    tc.tc_ensemble_destroy(ens)
    for i, wl in enumerate(members):
        run = tc.Run.from_workload(wl)       # default tiles, plain launches
        # the transform paths the tuner chose for this member's size class
        # (tiles change nothing; the tensor-core paths change round-off)
        tc.tc_set_option(run.ctx, "tensor_theta", tensor[i][0])
        tc.tc_set_option(run.ctx, "tensor_z", tensor[i][1])
        dt, _ = _init(tc, run.ctx, wl)
        assert dt == dts[i]
        run.step(12, dt)
        ref = run.get_state()
        run.close()
        if mode == 0:
            assert np.array_equal(got[i], ref), i
        else:
            # one compiled kernel for every stage: the compiler may fuse
            # multiplies and adds differently from the per-stage kernels, so
            # the persistent mode agrees to round-off, not bit for bit
            rel = np.abs(got[i] - ref).max() / np.abs(ref).max()
            print(f"persistent member {i}: max rel difference to the run alone {rel:.2e}")
            assert rel <= 1e-13, (i, rel)


def test_ensemble_members_match_oracle(tc):
    members = [w.scaled(Nr=24, Ntheta=32, Nz=32) for w in ensemble_members(2)]
    ens = tc.tc_ensemble_create(members, autotune_tiles=True)
    dts = [_init(tc, tc.tc_ensemble_member(ens, i), wl)[0] for i, wl in enumerate(members)]
    tc.tc_ensemble_step(ens, 20, dts)
    for i, wl in enumerate(members):
        mdl = Model(wl, "fft")
        X = mdl.initial_state(psi_coefficients(wl.seed, wl.mp, wl.kp))
        X, _ = mdl.run(X, 20, dts[i])
        got = np.empty(X.shape, dtype=np.complex128)
        tc.tc_get_state(tc.tc_ensemble_member(ens, i), got)
        w = (mdl.g.w * mdl.g.r)[:, None, None] * mdl.sp.cm[None, :, None]
        err = max(np.sqrt(np.sum(w * np.abs(got[f] - X[f]) ** 2) / np.sum(w * np.abs(X[f]) ** 2))
                  for f in range(X.shape[0]))
        assert err <= 1e-10, (i, err)
    tc.tc_ensemble_destroy(ens)


def test_ensemble_graph_follows_member_options(tc):
    """Changing a member's option after the graph was captured re-captures it:
    the member then steps exactly like a run with that option."""
    members = [w.scaled(Nr=20, Ntheta=24, Nz=24) for w in ensemble_members(2)]
    ens = tc.tc_ensemble_create(members, autotune_tiles=False)
    tc.tc_ensemble_set_mode(ens, 0)
    dts, shapes = [], []
    for i, wl in enumerate(members):
        dt, shape = _init(tc, tc.tc_ensemble_member(ens, i), wl)
        dts.append(dt)
        shapes.append(shape)
    tc.tc_ensemble_step(ens, 2, dts)
    tc.tc_set_option(tc.tc_ensemble_member(ens, 0), "n_corr", 2)
    tc.tc_ensemble_step(ens, 3, dts)
    X = np.empty(shapes[0], dtype=np.complex128)
    tc.tc_get_state(tc.tc_ensemble_member(ens, 0), X)
    tc.tc_ensemble_destroy(ens)
    run = tc.Run.from_workload(members[0])
    _init(tc, run.ctx, members[0])
    run.step(2, dts[0])
    run.set_option("n_corr", 2)
    run.step(3, dts[0])
    ref = run.get_state()
    run.close()
    np.testing.assert_array_equal(X, ref)


def test_persistent_unpublished_stage_times_out(tc):
    """Mode 2: the end of member 0's first transform stage is never published,
    so that member never has ready work again; the others finish, every CTA's
    bounded idle wait (2 s) runs out, the kernel ends and the step reports
    TC_ERR_TIMEOUT -- no hang, no fault.  The ensemble then steps normally
    in mode 1."""
    members = [w.scaled(Nr=20, Ntheta=24, Nz=24) for w in ensemble_members(3)]
    ens = tc.tc_ensemble_create(members, autotune_tiles=False)
    dts = [_init(tc, tc.tc_ensemble_member(ens, i), wl)[0] for i, wl in enumerate(members)]
    tc.tc_ensemble_set_mode(ens, 2)
    with pytest.raises(tc.TCError) as e:
        tc.tc_ensemble_step(ens, 1, dts)
    assert e.value.name == "TC_ERR_TIMEOUT"
    tc.tc_ensemble_set_mode(ens, 1)
    tc.tc_ensemble_step(ens, 2, dts)
    for i in range(len(members)):
        info = tc.tc_get_info(tc.tc_ensemble_member(ens, i))
        X = np.empty((info.nfields, info.Nr, info.M + 1, 2 * info.K + 1), dtype=np.complex128)
        tc.tc_get_state(tc.tc_ensemble_member(ens, i), X)
        assert np.all(np.isfinite(X))
    tc.tc_ensemble_destroy(ens)


def test_persistent_mode_steps_unsupported_schemes_as_graph(tc):
    """With a member on a scheme the persistent kernel does not run (n_corr =
    2), the persistent mode steps that call as the graph of member kernels:
    the member then equals the run alone bit for bit."""
    members = [w.scaled(Nr=20, Ntheta=24, Nz=24) for w in ensemble_members(2)]
    ens = tc.tc_ensemble_create(members, autotune_tiles=False)
    assert tc.tc_ensemble_get_mode(ens) == 0
    tc.tc_ensemble_set_mode(ens, 1)
    dts, shapes = [], []
    for i, wl in enumerate(members):
        dt, shape = _init(tc, tc.tc_ensemble_member(ens, i), wl)
        dts.append(dt)
        shapes.append(shape)
    tc.tc_set_option(tc.tc_ensemble_member(ens, 0), "n_corr", 2)
    tc.tc_ensemble_step(ens, 3, dts)
    X = np.empty(shapes[0], dtype=np.complex128)
    tc.tc_get_state(tc.tc_ensemble_member(ens, 0), X)
    tc.tc_ensemble_destroy(ens)
    run = tc.Run.from_workload(members[0])
    _init(tc, run.ctx, members[0])
    run.set_option("n_corr", 2)
    run.step(3, dts[0])
    np.testing.assert_array_equal(X, run.get_state())
    run.close()
