"""Tangent and dense adjoint of the oracle step (test infrastructure only).

The differentiation form asks for the gradient of a final-time perturbation
energy with respect to the initial field; its reference is the exact
transpose of the discrete step, built here densely on tiny grids.

Tangent (exact, no finite differences):
* the nonlinear term is quadratic plus the linear buoyancy, N(X) = Q(X, X) +
  Gr T e_z, so dN(X)[d] = N(X + d) - N(X) - N(d) + Gr dT e_z (a polynomial
  identity);
* each implicit stage is affine in its right-hand side (the wall values are
  the constant part), so its linear part is stage(R) - stage(0);
* the explicit right-hand side is linear.

Conventions: a state is the real vector of (Re, Im) of every stored
coefficient [field][r][m][kk]; the inner product is the plain Euclidean one
on that vector.  The stored m = 0 column is redundant (u(0,-k) = conj u(0,k)),
so the adjoint of a step is defined as P_H J^T, with P_H the orthogonal
projection onto that Hermitian subspace; gradients with respect to any
parameters that enter through Hermitian states (the psi coefficients) are
unchanged by it.
"""
from __future__ import annotations

import numpy as np

from .model import CN


def to_real(X: np.ndarray) -> np.ndarray:
    return np.stack([X.real, X.imag], axis=-1).ravel()


def from_real(v: np.ndarray, shape) -> np.ndarray:
    a = v.reshape(tuple(shape) + (2,))
    return a[..., 0] + 1j * a[..., 1]


def hermitian_projection(X: np.ndarray) -> np.ndarray:
    """Orthogonal projection (real Euclidean metric) onto u(0,-k) = conj u(0,k)."""
    out = X.copy()
    NK = X.shape[-1]
    K = (NK - 1) // 2
    for k in range(1, K + 1):
        a = 0.5 * (X[..., 0, k] + np.conj(X[..., 0, NK - k]))
        out[..., 0, k] = a
        out[..., 0, NK - k] = np.conj(a)
    out[..., 0, 0] = X[..., 0, 0].real
    return out


def nonlinear_tangent(mdl, X, d):
    N_xd, _ = mdl.nonlinear(X + d)
    N_x, _ = mdl.nonlinear(X)
    N_d, _ = mdl.nonlinear(d)
    out = N_xd - N_x - N_d
    if mdl.has_T:
        out[2] = out[2] + mdl.Gr * d[3]
    return out


def stage_tangent(mdl, dR, dt):
    X1, _ = mdl.stage_solve(dR, dt)
    X0, _ = mdl.stage_solve([np.zeros_like(r) for r in dR], dt)
    return X1 - X0


def step_tangent(mdl, X, d, dt):
    """J(X) d for one predictor-corrector step at fixed dt."""
    N0, _ = mdl.nonlinear(X)
    Xpm = mdl.to_pm(X)
    base = [Xpm[i] / dt + (1.0 - CN) * mdl.explicit_linear(Xpm)[i] + (1.0 - CN) * mdl.to_pm(N0)[i]
            for i in range(mdl.nf)]
    Xp, _ = mdl.stage_solve([base[i] + CN * mdl.to_pm(N0)[i] for i in range(mdl.nf)], dt)
    # tangent
    dN0 = nonlinear_tangent(mdl, X, d)
    dpm = mdl.to_pm(d)
    Ld = mdl.explicit_linear(dpm)
    dN0pm = mdl.to_pm(dN0)
    dbase = [dpm[i] / dt + (1.0 - CN) * Ld[i] + (1.0 - CN) * dN0pm[i] for i in range(mdl.nf)]
    dXp = stage_tangent(mdl, [dbase[i] + CN * dN0pm[i] for i in range(mdl.nf)], dt)
    dN1 = nonlinear_tangent(mdl, Xp, dXp)
    dN1pm = mdl.to_pm(dN1)
    return stage_tangent(mdl, [dbase[i] + CN * dN1pm[i] for i in range(mdl.nf)], dt)


def step_jacobian(mdl, X, dt):
    """Dense real Jacobian of one step (columns: unit (Re, Im) perturbations)."""
    n = 2 * X.size
    J = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        J[:, c] = to_real(step_tangent(mdl, X, from_real(e, X.shape), dt))
    return J


def adjoint_step_dense(mdl, X, lam, dt, J=None):
    """P_H J(X)^T lam, the reference for the GPU adjoint step."""
    if J is None:
        J = step_jacobian(mdl, X, dt)
    return hermitian_projection(from_real(J.T @ to_real(lam), X.shape))


def objective(mdl, X):
    """J = E_pert = (1/2) int |u - u_base|^2 dV (velocity only)."""
    return mdl.diagnostics(X)["E_pert"]


def objective_gradient(mdl, X):
    """dJ/dX in the real Euclidean convention: V w_j r_j c_m (u - u_base)."""
    V = 2.0 * np.pi * mdl.wl.Lz
    w = (mdl.g.w * mdl.g.r)[:, None, None] * mdl.sp.cm[None, :, None]
    g = np.zeros_like(X)
    g[:3] = V * w[None] * (X[:3] - mdl.base[:3])
    return g
