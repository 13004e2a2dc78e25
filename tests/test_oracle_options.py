"""Pins of the oracle's optional scheme settings.

* corrector passes (``n_corr``): the iterates contract and their limit solves
  the implicit (Crank-Nicolson on every term) stage equation;
* axial-flux constraint: zero axial volume flux after every step; the
  constrained basic state is kept to round-off and converges to the closed
  form of the zero-flux convective axial flow of a radially heated annulus
  (and, without the constraint, to the closed form with no pressure gradient);
* centrifugal buoyancy (density factor 1 - eps T on the advective
  acceleration): with a uniform temperature the momentum advection scales by
  exactly 1 - eps T0 while buoyancy and heat advection stay; the terms are
  affine in eps; the basic state stays steady.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from inputs import Workload, psi_coefficients, random_state, temperature_coefficients
from oracle import Model

SMALL = Workload("opt_small", Nr=16, Ntheta=12, Nz=12, eta=0.5, Lz=2 * math.pi / 3.16,
                 Re_i=150.0, amp=5e-2, mp=3, kp=3, seed=11, dt=1e-3)
HEATED = Workload("opt_heated", Nr=16, Ntheta=12, Nz=12, eta=0.6, Lz=2 * math.pi,
                  Re_i=80.0, Ra=3000.0, Pr=0.7, amp=5e-2, mp=3, kp=3, amp_T=5e-2, seed=12,
                  dt=1e-3)


def _perturbed(mdl, wl):
    T_raw = temperature_coefficients(wl.seed, wl.mp, wl.kp) if mdl.has_T else None
    return mdl.initial_state(psi_coefficients(wl.seed, wl.mp, wl.kp), T_raw)


# ----------------------------------------------------------------- correctors
def test_corrector_iterates_contract_to_implicit_stage():
    diffs = []
    for n in (1, 2, 3, 4):
        mdl = Model(SMALL, "fft", n_corr=n)
        X0 = _perturbed(mdl, SMALL)
        mdl.step(X0, 2e-3)
        diffs.append(mdl.last_corr_diff)
    assert diffs[0] > 0.0
    for a, b in zip(diffs, diffs[1:]):
        assert b < 0.5 * a, diffs
    # the limit X* satisfies (I/dt - c L) X* = X^n/dt + (1-c) L X^n + (1-c) N^n
    # + c N(X*) with grad p and the wall conditions, i.e. one more stage with
    # N(X*) returns X* itself
    dt = 2e-3
    mdl = Model(SMALL, "fft", n_corr=40)
    X0 = _perturbed(mdl, SMALL)
    Xs, _, _, _ = mdl.step(X0, dt)
    assert mdl.last_corr_diff < 1e-13 * np.abs(Xs).max()
    N0, _ = mdl.nonlinear(X0)
    Ns, _ = mdl.nonlinear(Xs)
    Xpm, Npm0, Npms = mdl.to_pm(X0), mdl.to_pm(N0), mdl.to_pm(Ns)
    LX = mdl.explicit_linear(Xpm)
    c = 0.5
    R = [Xpm[i] / dt + (1 - c) * LX[i] + (1 - c) * Npm0[i] + c * Npms[i] for i in range(mdl.nf)]
    Xchk, _ = mdl.stage_solve(R, dt)
    assert np.abs(Xchk - Xs).max() <= 1e-12 * np.abs(Xs).max()
    # one corrector is not the limit at this amplitude
    m1 = Model(SMALL, "fft")
    X1, _, _, _ = m1.step(X0, dt)
    assert np.abs(X1 - Xs).max() > 1e3 * np.abs(Xchk - Xs).max()


# ----------------------------------------------------------------- axial flux
def _closed_form_axial_flow(wl, zero_flux, r_nodes):
    """Continuous steady u_z(r) of the conductive state, (1/r)(r u')' = -Gr T - G.

    T = a + b ln r with T(r_i) = 1/2, T(r_o) = -1/2.  Integrating twice,
    u = phi0 + G phiG + C1 ln r + C2 with phi0 = -Gr a r^2/4 - Gr b (r^2/4)(ln r - 1)
    and phiG = -r^2/4; C1, C2 (and G when the flux is constrained) from
    u(r_i) = u(r_o) = 0 and int u r dr = 0 (adaptive quadrature).
    """
    ri, ro = wl.eta / (1 - wl.eta), 1 / (1 - wl.eta)
    Gr = wl.Ra / wl.Pr
    b = -1.0 / math.log(ro / ri)
    a = 0.5 - b * math.log(ri)
    phi0 = lambda r: -Gr * a * r * r / 4 - Gr * b * (r * r / 4) * (math.log(r) - 1)
    basis = [lambda r: -r * r / 4, lambda r: math.log(r), lambda r: 1.0]
    if zero_flux:
        A = np.array([[f(ri) for f in basis], [f(ro) for f in basis],
                      [quad(lambda r: f(r) * r, ri, ro, epsabs=0, epsrel=1e-13)[0] for f in basis]])
        rhs = -np.array([phi0(ri), phi0(ro), quad(lambda r: phi0(r) * r, ri, ro,
                                                  epsabs=0, epsrel=1e-13)[0]])
        G, C1, C2 = np.linalg.solve(A, rhs)
    else:
        A = np.array([[f(ri) for f in basis[1:]], [f(ro) for f in basis[1:]]])
        C1, C2 = np.linalg.solve(A, -np.array([phi0(ri), phi0(ro)]))
        G = 0.0
    return np.array([phi0(r) + G * basis[0](r) + C1 * math.log(r) + C2 for r in r_nodes])


@pytest.mark.parametrize("zero_flux", [False, True])
def test_axial_base_flow_matches_closed_form(zero_flux):
    errs = []
    for Nr in (24, 48):
        wl = HEATED.scaled(Nr=Nr)
        mdl = Model(wl, "fft", flux_constraint=zero_flux)
        uz = mdl.base[2, :, 0, 0].real
        ref = _closed_form_axial_flow(wl, zero_flux, mdl.g.r)
        errs.append(np.abs(uz - ref).max() / np.abs(ref).max())
    assert errs[1] < 1e-10, errs
    assert errs[0] / errs[1] > 50, errs     # about stencil order under refinement
    mdl = Model(HEATED, "fft", flux_constraint=zero_flux)
    if zero_flux:
        assert abs(mdl.axial_flux(mdl.base[2, :, 0, 0])) < 1e-13 * np.abs(mdl.base[2]).max()
    else:
        assert abs(mdl.axial_flux(mdl.base[2, :, 0, 0])) > 1e-3 * np.abs(mdl.base[2]).max()


def test_flux_constrained_base_state_kept():
    mdl = Model(HEATED, "fft", flux_constraint=True)
    X0 = mdl.base.copy()
    X = X0
    for _ in range(20):
        X, _, _, _ = mdl.step(X, 1e-3)
    assert np.abs(X - X0).max() <= 1e-12 * np.abs(X0).max()


def test_flux_zero_after_every_step():
    mdl = Model(HEATED, "fft", flux_constraint=True)
    free = Model(HEATED, "fft")
    X = _perturbed(mdl, HEATED)
    # a perturbation with net axial flux, so the constraint has work to do
    X[2, 1:-1, 0, 0] += 0.3 * np.sin(np.pi * np.linspace(0, 1, HEATED.Nr))[1:-1]
    Xf = X.copy()
    scale = np.abs(X[2]).max()
    for _ in range(5):
        X, _, _, _ = mdl.step(X, 1e-3)
        Xf, _, _, _ = free.step(Xf, 1e-3)
        assert abs(mdl.axial_flux(X[2, :, 0, 0])) < 1e-13 * scale
    assert abs(free.axial_flux(Xf[2, :, 0, 0])) > 1e-3 * scale
    # only the (0,0) u_z column carries the constraint's uniform forcing; the
    # other columns see it only through the nonlinear coupling
    assert np.abs(X[0] - Xf[0]).max() < np.abs(X[2, :, 0, 0] - Xf[2, :, 0, 0]).max()


# ---------------------------------------------------------------- centrifugal
def test_centrifugal_uniform_temperature_scales_momentum_advection():
    mdl0 = Model(HEATED, "fft")
    M, K = mdl0.M, mdl0.K
    X = random_state(21, 4, HEATED.Nr, M, K, scale=[1.0, 1.0, 1.0, 0.0])
    T0 = 0.3
    X[3, :, 0, 0] = T0          # uniform temperature: only the (0,0) mode
    eps = 0.2
    N0, _ = mdl0.nonlinear(X)
    Ne, _ = Model(HEATED, "fft", eps_c=eps).nonlinear(X)
    buoy = np.zeros_like(N0[2])
    buoy[:, 0, 0] = mdl0.Gr * T0
    for c in range(3):
        adv0 = N0[c] - (buoy if c == 2 else 0.0)
        adve = Ne[c] - (buoy if c == 2 else 0.0)
        assert np.abs(adve - (1 - eps * T0) * adv0).max() <= 1e-13 * np.abs(adv0).max(), c
    assert np.abs(Ne[3] - N0[3]).max() <= 1e-14 * np.abs(N0[3]).max()


def test_centrifugal_terms_affine_in_eps():
    mdl = Model(HEATED, "fft")
    X = random_state(22, 4, HEATED.Nr, mdl.M, mdl.K)
    N = [Model(HEATED, "fft", eps_c=e).nonlinear(X)[0] for e in (0.0, 0.1, 0.2)]
    d1, d2 = N[1] - N[0], N[2] - N[1]
    assert np.abs(d1).max() > 1e-3 * np.abs(N[0]).max()
    assert np.abs(d2 - d1).max() <= 1e-12 * np.abs(N[0]).max()


def test_centrifugal_base_state_kept():
    mdl = Model(HEATED, "fft", eps_c=0.3)
    X0 = mdl.base.copy()
    X = X0
    for _ in range(20):
        X, _, _, _ = mdl.step(X, 1e-3)
    assert np.abs(X - X0).max() <= 1e-12 * np.abs(X0).max()


def test_centrifugal_needs_temperature():
    with pytest.raises(ValueError):
        Model(SMALL, "fft", eps_c=0.1)
