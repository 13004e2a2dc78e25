"""Mixed precision (FP32 transforms of the perturbation, FP64 elsewhere)
against the FP64 oracle.

The FP32 part only carries u'.grad u' of the perturbation u' = u - U(r); the
products with the mean mode are FP64.  So the error is FP32 rounding times
the size of the quadratic perturbation term, which these tests measure on a
random state (no mean flow: plain FP32 level) and on the seeded runs.
"""
import numpy as np
import pytest

from inputs import WORKLOADS, Workload, psi_coefficients, random_state, temperature_coefficients
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


def rel_l2(mdl, a, b):
    w = (mdl.g.w * mdl.g.r)[:, None, None] * mdl.sp.cm[None, :, None]
    return max(float(np.sqrt(np.sum(w * np.abs(a[f] - b[f]) ** 2) / np.sum(w * np.abs(b[f]) ** 2)))
               for f in range(a.shape[0]))


@pytest.mark.parametrize("Nr,Nt,Nz,Ra", [(20, 36, 40, 0.0), (20, 36, 40, 700.0),
                                         (10, 128, 256, 300.0)])   # compile-time plans 128, 256
def test_mixed_nonlinear_random_state(tc, Nr, Nt, Nz, Ra):
    wl = Workload("mx", Nr=Nr, Ntheta=Nt, Nz=Nz, eta=0.6, Lz=1.5, Re_i=80.0, Ra=Ra, Pr=0.9,
                  precision=1)
    mdl = Model(wl)
    X = random_state(900, mdl.nf, wl.Nr, mdl.M, mdl.K)
    ref, rate = mdl.nonlinear(X)
    run = tc.Run.from_workload(wl)
    out = dev(np.zeros_like(X))
    got_rate = tc.tc_nonlinear(run.ctx, dev(X), out)
    got = out.cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err            # FP32 transforms of O(1) fields
    assert abs(got_rate - rate) < 1e-5 * rate
    run.close()


def test_mixed_nonlinear_mean_flow_split(tc):
    """Couette flow + small perturbation: the FP64 mean-flow products dominate,
    so the FP32 part contributes far below FP32 resolution of the total."""
    wl = WORKLOADS["tc_fp64_nr32_n32"].scaled(precision=1)
    mdl = Model(wl)
    X = mdl.initial_state(psi_coefficients(wl.seed, wl.mp, wl.kp))
    ref, _ = mdl.nonlinear(X)
    run = tc.Run.from_workload(wl)
    out = dev(np.zeros_like(X))
    tc.tc_nonlinear(run.ctx, dev(X), out)
    got = out.cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < 1e-11, err
    run.close()


def _run(tc, wl, nsteps):
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    tco = temperature_coefficients(wl.seed, wl.mp, wl.kp) if wl.Ra else None
    run = tc.Run.from_workload(wl)
    run.init_perturbation(psi, wl.amp, tco, wl.amp_T)
    run.step(nsteps, wl.dt)
    out = run.get_state()
    run.close()
    return out, psi, tco


def test_mixed_run_error_vs_oracle(tc):
    """Stated error of the mixed path: 100 steps of the 32^3 run."""
    wl = WORKLOADS["tc_fp64_nr32_n32"].scaled(precision=1)
    got, psi, _ = _run(tc, wl, 100)
    mdl = Model(wl, "fft")
    X, _ = mdl.run(mdl.initial_state(psi), 100, wl.dt)
    err = rel_l2(mdl, got, X)
    pert = rel_l2(mdl, got - mdl.base, X - mdl.base)
    print(f"mixed 32^3 100 steps: rel L2 {err:.3e}, perturbation {pert:.3e}")
    assert err < 1e-10
    assert pert < 1e-5


def test_mixed_shrunken_large_workload_vs_oracle(tc):
    """The 256 x 512^2 mixed workload's parameters (eta = 0.875, Re_i = 1e4,
    amplitude 0.1, dt = 2e-6) at 48 x 64^2, 50 steps, against the FP64
    oracle at the FP64 path's own gate, relative L2 <= 1e-10 per field.

    Why the gate holds for the mixed form: only u'.grad u' of the
    perturbation goes through FP32; its rounding, about 2^-24 of |N'| per
    evaluation, enters the state multiplied by dt.  With |N'| ~ |u'|^2 / gap
    ~ 1e-2 .. 1 here, 50 steps of dt = 2e-6 move the state by at most
    ~1e-4 |N'| and the FP32 part of that is ~1e-11 of |u'| ~ 0.1.  Measured
    against the perturbation itself the FP32 rounding is visible: ~2^-24 of
    u'.grad u' per evaluation, 100 evaluations, ~1e-6 of u' (bound 1e-5)."""
    wl = WORKLOADS["tc_mixed_nr256_n512"].scaled(Nr=48, Ntheta=64, Nz=64, mp=8, kp=8)
    got, psi, _ = _run(tc, wl, 50)
    mdl = Model(wl, "fft")
    X, _ = mdl.run(mdl.initial_state(psi), 50, wl.dt)
    w = (mdl.g.w * mdl.g.r)[:, None, None] * mdl.sp.cm[None, :, None]
    per_field = [float(np.sqrt(np.sum(w * np.abs(got[f] - X[f]) ** 2) / np.sum(w * np.abs(X[f]) ** 2)))
                 for f in range(got.shape[0])]
    pert = rel_l2(mdl, got - mdl.base, X - mdl.base)
    print(f"mixed eta=0.875 Re=1e4 48x64x64 50 steps: rel L2 per field {per_field}, "
          f"perturbation {pert:.3e}")
    assert max(per_field) <= 1e-10, per_field
    assert pert < 1e-5


def test_mixed_vs_fp64_full_size(tc):
    """Stated error at full size (256 x 512 x 512, eta = 0.875, Re_i = 1e4):
    relative L2 per field of the mixed path against the FP64 GPU path after
    50 steps of dt = 2e-6 (the FP64 GPU path itself is pinned to the oracle by
    test_gpu_parity)."""
    wl = WORKLOADS["tc_mixed_nr256_n512"]
    mixed, _, _ = _run(tc, wl, wl.steps)
    full, _, _ = _run(tc, wl.scaled(precision=0), wl.steps)
    mdl = Model(wl.scaled(Ntheta=8, Nz=8), "fft")     # radial weights only
    w = (mdl.g.w * mdl.g.r)[:, None, None] * np.where(np.arange(mixed.shape[2]) == 0, 1.0, 2.0)[None, :, None]
    errs = []
    for f in range(mixed.shape[0]):
        errs.append(float(np.sqrt(np.sum(w * np.abs(mixed[f] - full[f]) ** 2)
                                  / np.sum(w * np.abs(full[f]) ** 2))))
    print("mixed vs FP64, 256x512x512, 50 steps, rel L2 per field:", errs)
    assert max(errs) < 1e-8
