"""GPU parity of the optional scheme settings against the FP64 oracle.

* ``n_corr`` corrector passes: state after the run and the last corrector
  difference (diagnostics ``corr_diff``);
* ``flux_constraint``: basic state, state after the run, zero axial flux;
* ``eps_centrifugal``: the nonlinear stage on a random state and a whole run;
* the combinations that the library does not support are refused.
Whole runs: relative L2 <= 1e-10 per field (weights c_m w_j r_j).
"""
import math

import numpy as np
import pytest

from inputs import Workload, psi_coefficients, random_state, temperature_coefficients
from oracle import Model

pytestmark = pytest.mark.gpu

PLAIN = Workload("opt_plain", Nr=20, Ntheta=24, Nz=30, eta=0.5, Lz=2 * math.pi / 3.16,
                 Re_i=150.0, amp=5e-2, mp=3, kp=3, seed=31, dt=1e-3)
HEATED = Workload("opt_heated", Nr=17, Ntheta=24, Nz=20, eta=0.6, Lz=2 * math.pi,
                  Re_i=80.0, Re_o=-20.0, Ra=3000.0, Pr=0.7, amp=5e-2, mp=3, kp=3,
                  amp_T=5e-2, seed=32, dt=1e-3)


@pytest.fixture(scope="module")
def tc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1908_00587_gb300 import tc as mod
    return mod


def rel_l2(mdl, a, b):
    w = (mdl.g.w * mdl.g.r)[:, None, None] * mdl.sp.cm[None, :, None]
    return max(float(np.sqrt(np.sum(w * np.abs(a[f] - b[f]) ** 2) / np.sum(w * np.abs(b[f]) ** 2)))
               for f in range(a.shape[0]))


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _run_both(tc, wl, nsteps, options, oracle_kw):
    mdl = Model(wl, "fft", **oracle_kw)
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    tco = temperature_coefficients(wl.seed, wl.mp, wl.kp) if wl.Ra else None
    run = tc.Run.from_workload(wl)
    for k, v in options.items():
        run.set_option(k, v)
    run.init_perturbation(psi, wl.amp, tco, wl.amp_T)
    X0 = run.get_state()
    run.step(nsteps, wl.dt)
    got = run.get_state()
    diag = run.diagnostics()
    run.close()
    X = mdl.initial_state(psi, tco)
    assert np.abs(X0 - X).max() <= 1e-13 * np.abs(X).max()
    for _ in range(nsteps):
        X, _, _, _ = mdl.step(X, wl.dt)
    return mdl, got, X, diag


@pytest.mark.parametrize("n_corr", [2, 3])
def test_corrector_passes_match_oracle(tc, n_corr):
    mdl, got, ref, diag = _run_both(tc, PLAIN, 20, {"n_corr": n_corr}, {"n_corr": n_corr})
    assert rel_l2(mdl, got, ref) <= 1e-10
    # the difference of two O(Re) iterates: its own round-off is ~1e-14 Re
    assert abs(diag["corr_diff"] - mdl.last_corr_diff) <= 1e-6 * mdl.last_corr_diff + 1e-13 * PLAIN.Re_i
    assert mdl.last_corr_diff > 0.0


def test_corrector_difference_default_scheme(tc):
    mdl, got, ref, diag = _run_both(tc, PLAIN, 5, {}, {})
    assert rel_l2(mdl, got, ref) <= 1e-10
    assert abs(diag["corr_diff"] - mdl.last_corr_diff) <= 1e-6 * mdl.last_corr_diff + 1e-13 * PLAIN.Re_i


def test_flux_constraint_matches_oracle(tc):
    mdl, got, ref, diag = _run_both(tc, HEATED, 20, {"flux_constraint": 1},
                                       {"flux_constraint": True})
    assert rel_l2(mdl, got, ref) <= 1e-10
    assert abs(mdl.axial_flux(got[2, :, 0, 0])) <= 1e-12 * np.abs(got[2]).max()


def test_flux_constrained_basic_state(tc):
    mdl = Model(HEATED, "fft", flux_constraint=True)
    run = tc.Run.from_workload(HEATED)
    run.set_option("flux_constraint", 1)
    run.init_perturbation(psi_coefficients(1, 0, 0), 0.0,
                          temperature_coefficients(1, 0, 0), 0.0)   # zero amplitude: the base
    X0 = run.get_state()
    assert np.abs(X0 - mdl.base).max() <= 1e-12 * np.abs(mdl.base).max()
    run.step(50, 1e-3)
    X = run.get_state()
    run.close()
    assert np.abs(X - X0).max() <= 1e-12 * np.abs(X0).max()


def test_centrifugal_nonlinear_matches_oracle(tc):
    mdl = Model(HEATED, "fft", eps_c=0.25)
    X = random_state(33, mdl.nf, HEATED.Nr, mdl.M, mdl.K)
    X[3, :, 0, 0] += 0.4          # a temperature with a mean, so 1 - eps T varies
    ref, rate = mdl.nonlinear(X)
    run = tc.Run.from_workload(HEATED)
    run.set_option("eps_centrifugal", 0.25)
    out = dev(np.zeros_like(X))
    got_rate = tc.tc_nonlinear(run.ctx, dev(X), out)
    run.close()
    got = out.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert abs(got_rate - rate) <= 1e-13 * rate


def test_centrifugal_run_matches_oracle(tc):
    mdl, got, ref, _ = _run_both(tc, HEATED, 20, {"eps_centrifugal": 0.3}, {"eps_c": 0.3})
    assert rel_l2(mdl, got, ref) <= 1e-10
    plain = Model(HEATED, "fft")
    X = plain.initial_state(psi_coefficients(HEATED.seed, HEATED.mp, HEATED.kp),
                            temperature_coefficients(HEATED.seed, HEATED.mp, HEATED.kp))
    for _ in range(20):
        X, _, _, _ = plain.step(X, HEATED.dt)
    assert rel_l2(mdl, got - mdl.base, X - mdl.base) > 1e-6   # the option changes the run


def test_unsupported_combinations_refused(tc):
    st = {v: k for k, v in tc.STATUS.items()}
    UNSUP, ARG = st["TC_ERR_UNSUPPORTED"], st["TC_ERR_ARG"]
    run = tc.Run.from_workload(PLAIN)              # no temperature
    assert tc._lib.tc_set_option(run.ctx, b"eps_centrifugal", 0.1) == UNSUP
    assert tc._lib.tc_set_option(run.ctx, b"n_corr", 0.0) == ARG
    assert tc._lib.tc_set_option(run.ctx, b"n_corr", 2.5) == ARG
    run.close()
    run = tc.Run.from_workload(HEATED)
    run.set_option("eps_centrifugal", 0.2)
    assert tc._lib.tc_set_option(run.ctx, b"precision", 1.0) == UNSUP
    X = dev(run.get_state())
    lam = dev(np.zeros(run.shape, dtype=np.complex128))
    assert tc._lib.tc_adjoint_step(run.ctx, X.data_ptr(), 1e-3,
                                   lam.data_ptr()) == UNSUP
    run.set_option("eps_centrifugal", 0.0)
    run.set_option("n_corr", 2)
    assert tc._lib.tc_adjoint_step(run.ctx, X.data_ptr(), 1e-3,
                                   lam.data_ptr()) == UNSUP
    run.close()
