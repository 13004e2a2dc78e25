"""Pins of the oracle's tangent and dense adjoint (differentiation form).

The tangent is pinned to central differences of the oracle step; the dense
adjoint P_H J^T is pinned to the derivative of <lambda, step(X + eps v)> along
Hermitian directions, so both rest on the forward map alone.
"""
import numpy as np

from inputs import Workload, psi_coefficients, random_state, temperature_coefficients
from oracle import Model
from oracle.adjoint import (adjoint_step_dense, from_real, hermitian_projection,
                            objective, objective_gradient, step_jacobian, step_tangent, to_real)

WL = Workload("adj", Nr=9, Ntheta=6, Nz=6, eta=0.6, Lz=1.7, Re_i=40.0, Re_o=-10.0, Ra=300.0,
              Pr=0.8, amp=0.3, mp=1, kp=1, amp_T=0.1, seed=3, dt=2e-3)


def _state(mdl):
    return mdl.initial_state(psi_coefficients(WL.seed, WL.mp, WL.kp),
                             temperature_coefficients(WL.seed, WL.mp, WL.kp))


def test_tangent_matches_central_differences():
    mdl = Model(WL)
    X = _state(mdl)
    d = hermitian_projection(random_state(31, mdl.nf, WL.Nr, mdl.M, mdl.K))
    jv = step_tangent(mdl, X, d, WL.dt)
    eps = 1e-5
    fd = (mdl.step(X + eps * d, WL.dt)[0] - mdl.step(X - eps * d, WL.dt)[0]) / (2 * eps)
    assert np.abs(fd - jv).max() <= 1e-7 * np.abs(jv).max()


def test_dense_adjoint_is_the_transposed_step():
    mdl = Model(WL)
    X = _state(mdl)
    J = step_jacobian(mdl, X, WL.dt)
    lam = hermitian_projection(random_state(32, mdl.nf, WL.Nr, mdl.M, mdl.K))
    adj = adjoint_step_dense(mdl, X, lam, WL.dt, J)
    for seed in (33, 34):
        v = hermitian_projection(random_state(seed, mdl.nf, WL.Nr, mdl.M, mdl.K))
        eps = 1e-5
        lhs = (np.dot(to_real(lam), to_real(mdl.step(X + eps * v, WL.dt)[0]))
               - np.dot(to_real(lam), to_real(mdl.step(X - eps * v, WL.dt)[0]))) / (2 * eps)
        rhs = np.dot(to_real(v), to_real(adj))
        assert abs(lhs - rhs) <= 1e-7 * abs(rhs)
    # the adjoint is Hermitian by construction
    np.testing.assert_allclose(adj, hermitian_projection(adj), atol=0)


def test_objective_gradient_matches_differences():
    mdl = Model(WL)
    X = _state(mdl)
    g = objective_gradient(mdl, X)
    v = hermitian_projection(random_state(35, mdl.nf, WL.Nr, mdl.M, mdl.K))
    eps = 1e-6
    fd = (objective(mdl, X + eps * v) - objective(mdl, X - eps * v)) / (2 * eps)
    assert abs(fd - np.dot(to_real(g), to_real(v))) <= 1e-7 * abs(fd)
