"""Pins of the whole oracle step against physics and mathematics.

* the basic state of Sec. 4 (circular Couette flow, conductive temperature)
  is a steady solution and is kept to round-off; its discrete form converges to
  the analytic profiles; dissipation and torque match their closed forms;
* the Nusselt number of the conductive state is 1 (Sec. 4);
* the initial perturbation is divergence-free (Sec. 2.1), the influence matrix
  makes the wall divergence vanish, and the interior divergence falls at about
  stencil order under radial refinement;
* the energy budget dE/dt = P_wall - eps + buoyancy work holds;
* the time stepper's growth rate of axisymmetric vortices matches an
  independent eigenvalue solve and changes sign at the classical onset;
* symmetries of the equations are kept.
"""
import math
import os

import numpy as np
import pytest

from inputs import Workload, WORKLOADS, psi_coefficients, temperature_coefficients
from oracle import Model
from oracle.grid import conductive_T, couette_AB
from oracle.stability import critical_reynolds, leading_eigenvalue

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CFG1 = WORKLOADS["tc_fp64_nr32_n32"]


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


def test_couette_preserved_to_roundoff():
    mdl = Model(CFG1, "fft")
    X0 = mdl.base.copy()
    X = X0
    for _ in range(100):
        X, _, _, _ = mdl.step(X, 1e-3)
    assert np.abs(X - X0).max() <= 1e-12 * np.abs(X0).max()


def test_discrete_couette_converges_to_analytic():
    errs = []
    for Nr in (16, 32):
        mdl = Model(CFG1.scaled(Nr=Nr), "fft")
        A, B = couette_AB(CFG1.eta, CFG1.Re_i, CFG1.Re_o)
        ut = mdl.base[1, :, 0, 0].real
        errs.append(np.abs(ut - (A * mdl.g.r + B / mdl.g.r)).max())
    assert errs[1] < 1e-6 * CFG1.Re_i
    assert errs[0] / errs[1] > 2 ** 6


def test_couette_closed_forms():
    mdl = Model(CFG1, "fft")
    A, B = couette_AB(CFG1.eta, CFG1.Re_i, CFG1.Re_o)
    d = mdl.diagnostics(mdl.base)
    Lz, g = CFG1.Lz, mdl.g
    eps = 4 * math.pi * Lz * B ** 2 * (g.r_i ** -2 - g.r_o ** -2)
    assert abs(d["eps"] - eps) < 1e-8 * eps
    G = 4 * math.pi * Lz * B
    assert abs(d["torque_i"] + G) < 1e-5 * G
    assert abs(d["torque_o"] + G) < 1e-5 * G
    assert abs(d["P_wall"] - eps) < 1e-5 * eps
    assert abs(d["E_pert"]) == 0.0


def test_conductive_state_kept_and_nusselt_one():
    wl = Workload("T", Nr=32, Ntheta=16, Nz=16, eta=0.71, Lz=2 * math.pi,
                  Re_i=300.0, Re_o=-100.0, Ra=1e4, Pr=0.7)
    mdl = Model(wl, "fft")
    X0 = mdl.base.copy()
    d0 = mdl.diagnostics(X0)
    assert abs(d0["Nu_i"] - 1.0) < 1e-13 and abs(d0["Nu_o"] - 1.0) < 1e-13
    X = X0
    for _ in range(20):
        X, _, _, _ = mdl.step(X, 1e-3)
    assert np.abs(X - X0).max() <= 1e-12 * np.abs(X0).max()
    # analytic ln r profile: Nu = 1 up to truncation
    Tan = conductive_T(mdl.g.r, wl.eta)
    assert np.abs(X0[3, :, 0, 0].real - Tan).max() < 1e-7
    Xa = X0.copy()
    Xa[3, :, 0, 0] = Tan
    d = mdl.diagnostics(Xa)
    assert abs(d["Nu_i"] - 1.0) < 1e-6 and abs(d["Nu_o"] - 1.0) < 1e-6


def test_initial_condition_divergence_free_and_scaled():
    mdl = Model(CFG1)
    X = mdl.initial_state(psi_coefficients(1, 4, 4))
    u = X[:3] - mdl.base[:3]
    ph = [mdl.sp.to_physical(u[c]) for c in range(3)]
    assert abs(np.sqrt(sum(p ** 2 for p in ph)).max() - CFG1.amp) < 1e-15
    d = mdl.diagnostics(X)
    gu = np.abs(mdl.g.dr(u[0])).max()
    assert d["div_max"] < 1e-13 * gu
    # only the excited modes are non-zero
    assert np.abs(u[:, :, 5:, :]).max() == 0.0


def test_divergence_at_walls_and_refinement():
    rel = []
    for Nr in (24, 48):
        mdl = Model(CFG1.scaled(Nr=Nr), "fft")
        X = mdl.initial_state(psi_coefficients(1, 4, 4))
        for _ in range(3):
            X, _, _, _ = mdl.step(X, 1e-3)
        g, sp = mdl.g, mdl.sp
        r = g.r[:, None, None]
        div = g.dr(r * X[0]) / r + 1j * sp.m[None, :, None] * X[1] / r \
            + 1j * sp.beta[None, None, :] * X[2]
        gu = np.abs(g.dr(X[0])).max()
        assert np.abs(div[0]).max() < 1e-12 * gu
        assert np.abs(div[-1]).max() < 1e-12 * gu
        rel.append(np.abs(div).max() / gu)
    assert rel[0] / rel[1] > 2 ** 5


def test_energy_budget():
    mdl = Model(CFG1, "fft")
    X = mdl.initial_state(psi_coefficients(1, 4, 4))
    dt = 1e-3
    E, rhs = [], []
    for _ in range(4):
        d = mdl.diagnostics(X)
        E.append(d["E"])
        rhs.append(d["P_wall"] - d["eps"] + d["buoy_work"])
        X, _, _, _ = mdl.step(X, dt)
    for n in (1, 2):
        dEdt = (E[n + 1] - E[n - 1]) / (2 * dt)
        assert abs(dEdt - rhs[n]) < 1e-5 * mdl.diagnostics(mdl.base)["eps"]


@pytest.mark.parametrize("fixture", ["taylor_onset_eta05.txt", "taylor_onset_eta0875.txt"])
def test_taylor_onset_eigenvalue(fixture):
    gold = _golden(fixture)
    beta = gold["beta_c"]
    lo = leading_eigenvalue(32, gold["eta"], gold["Re_stable"], 0.0, 0, beta).real
    hi = leading_eigenvalue(32, gold["eta"], gold["Re_unstable"], 0.0, 0, beta).real
    assert lo < 0 < hi
    rec = critical_reynolds(32, gold["eta"], beta, gold["Re_stable"], gold["Re_unstable"],
                            tol=1e-3)
    assert abs(rec - gold["Re_c"]) < 0.02
    # beta_c is the minimum of the neutral curve: 0.1 to either side needs a
    # larger Reynolds number
    for b in (beta - 0.1, beta + 0.1):
        assert critical_reynolds(32, gold["eta"], b, gold["Re_stable"], gold["Re_unstable"],
                                 tol=1e-3) > rec + 0.02


def _growth_rate(mdl, dt, t_end=0.8, t_fit=0.2):
    X = mdl.initial_state(psi_coefficients(7, 0, 1))
    amps = []
    n = int(round(t_end / dt))
    for _ in range(n):
        X, _, _, _ = mdl.step(X, dt)
        d = X[:3, :, 0, 1]
        amps.append(math.sqrt(mdl.radial_integral(sum(np.abs(d[c]) ** 2 for c in range(3)))))
    nf = int(round(t_fit / dt))
    return math.log(amps[-1] / amps[-1 - nf]) / (nf * dt), X


def _onset_model(Re):
    gold = _golden("taylor_onset_eta05.txt")
    wl = Workload("onset", Nr=32, Ntheta=4, Nz=8, eta=gold["eta"],
                  Lz=2 * math.pi / gold["beta_c"], Re_i=Re, amp=1e-6, mp=0, kp=1)
    return Model(wl, "fft"), gold


def test_stepper_growth_rate_matches_eigenvalue():
    errs = []
    for Re in (66.0, 70.0):
        mdl, gold = _onset_model(Re)
        lam = leading_eigenvalue(32, gold["eta"], Re, 0.0, 0, gold["beta_c"]).real
        rate, X = _growth_rate(mdl, 2e-3)
        assert np.sign(rate) == np.sign(lam)
        errs.append(abs(rate - lam) / abs(lam))
        # axisymmetric start: m != 0 modes stay at round-off
        assert np.abs(X[:, :, 1:, :]).max() < 1e-14 * np.abs(X).max()
    assert max(errs) < 2e-3
    # second order in time: halving dt cuts the mismatch ~4x
    mdl, gold = _onset_model(70.0)
    lam = leading_eigenvalue(32, gold["eta"], 70.0, 0.0, 0, gold["beta_c"]).real
    rate, _ = _growth_rate(mdl, 1e-3)
    assert errs[1] / (abs(rate - lam) / lam) > 3.0


def test_planted_curvature_sign_error_is_caught(monkeypatch):
    """A sign error in the centrifugal term must break the onset pin."""
    mdl, gold = _onset_model(70.0)
    orig = mdl.physical_fields

    def flipped(X):
        f = orig(X)
        # (u_theta/r) d(u_r)/dtheta gains 2 u_theta^2/r, which turns the
        # centrifugal term -u_theta^2/r of N_r into +u_theta^2/r
        f["ur_t"] = f["ur_t"] + 2.0 * f["ut"]
        return f

    monkeypatch.setattr(mdl, "physical_fields", flipped)
    lam = leading_eigenvalue(32, gold["eta"], 70.0, 0.0, 0, gold["beta_c"]).real
    rate, _ = _growth_rate(mdl, 2e-3, t_end=0.4, t_fit=0.1)
    assert abs(rate - lam) / abs(lam) > 1e-2


def test_z_reflection_symmetry_kept():
    mdl = Model(CFG1, "fft")
    X = mdl.initial_state(psi_coefficients(1, 4, 4))
    K = mdl.K

    def reflect(Y):
        R = Y.copy()
        idx = [0] + list(range(2 * K, 0, -1))     # k -> -k in FFT order
        R = R[..., idx]
        R[2] = -R[2]
        return R

    X = 0.5 * (X + reflect(X))
    for _ in range(5):
        X, _, _, _ = mdl.step(X, 1e-3)
    assert np.abs(X - reflect(X)).max() < 1e-13 * np.abs(X).max()


def test_hermitian_m0_column_kept():
    wl = WORKLOADS["tc_fp64T_nr64_n128"].scaled(Nr=24, Ntheta=24, Nz=24, mp=4, kp=4)
    mdl = Model(wl, "fft")
    X = mdl.initial_state(psi_coefficients(2, 4, 4), temperature_coefficients(2, 4, 4))
    dts = []
    dt = 0.0
    for _ in range(3):
        X, _, dt, _ = mdl.step(X, 0.0, dt)
        dts.append(dt)
    K = mdl.K
    for f in X:
        np.testing.assert_allclose(f[:, 0, 1:K + 1], np.conj(f[:, 0, K + 1:][:, ::-1]),
                                   atol=1e-12 * np.abs(f).max())
        assert np.abs(f[:, 0, 0].imag).max() < 1e-12 * np.abs(f).max()
    assert all(0 < d <= wl.dt_max for d in dts)


def test_dt_policy():
    mdl = Model(CFG1)
    wl = CFG1
    assert mdl.dt_policy(0.0, 0.0) == wl.dt_max
    assert mdl.dt_policy(0.0, 1e4) == pytest.approx(wl.cfl / 1e4)
    dt = wl.cfl / 1e4
    assert mdl.dt_policy(dt, 1.01e4) == pytest.approx(wl.cfl / 1.01e4)   # decrease now
    assert mdl.dt_policy(dt, 0.95e4) == dt                                # small increase held
    assert mdl.dt_policy(dt, 0.8e4) == pytest.approx(wl.cfl / 0.8e4)     # > 1.1x: increase
    assert mdl.dt_policy(dt, 1.0) == wl.dt_max
