"""Linear stability of circular Couette flow on the oracle's radial grid.

Test infrastructure only.  Used to pin the time stepper against the classical
onset of Taylor vortices: the basic state of Sec. 4 (circular Couette flow)
loses stability to axisymmetric vortices when Re_i passes a critical value.

For a perturbation (u_r, u_theta, u_z, p) exp(i m theta + i beta z + lambda t)
about u_theta = V(r), linearising the convective term with its curvature terms
gives
  lambda u_r     = L(m) u_r - u_r/r^2 - (2im/r^2) u_theta - (im V/r) u_r
                   + 2 V u_theta / r - D1 p
  lambda u_theta = L(m) u_theta - u_theta/r^2 + (2im/r^2) u_r - (im V/r) u_theta
                   - (V' + V/r) u_r - (im/r) p
  lambda u_z     = L(m) u_z - (im V/r) u_z - i beta p
  0              = (1/r) D1(r u_r) + (im/r) u_theta + i beta u_z
with L(m) = D2 + D1/r - m^2/r^2 - beta^2, no-slip rows at both walls, and
continuity imposed at every node.  Solved as a dense generalised eigenproblem.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .grid import Grid, couette_AB


def leading_eigenvalue(Nr: int, eta: float, Re_i: float, Re_o: float,
                       m: int, beta: float) -> complex:
    g = Grid(Nr, eta)
    r = g.r
    A_, B_ = couette_AB(eta, Re_i, Re_o)
    V = A_ * r + B_ / r
    dV = A_ - B_ / r ** 2
    I = np.eye(Nr)
    L = g.D2 + g.D1 / r[:, None] - np.diag(m * m / r ** 2 + beta ** 2)
    R = np.diag(1.0 / r)
    R2 = np.diag(1.0 / r ** 2)
    adv = np.diag(1j * m * V / r)
    Z = np.zeros((Nr, Nr))
    # blocks: rows (r, theta, z, continuity), columns (u_r, u_theta, u_z, p)
    A = np.block([
        [L - R2 - adv, -2j * m * R2 + 2.0 * np.diag(V / r), Z, -g.D1],
        [2j * m * R2 - np.diag(dV + V / r), L - R2 - adv, Z, -1j * m * R],
        [Z, Z, L - adv, -1j * beta * I],
        [R @ g.D1 @ np.diag(r), 1j * m * R, 1j * beta * I, Z],
    ]).astype(complex)
    B = np.zeros_like(A)
    for blk in range(3):
        for j in range(1, Nr - 1):
            B[blk * Nr + j, blk * Nr + j] = 1.0
        # no-slip rows
        for j in (0, Nr - 1):
            row = blk * Nr + j
            A[row, :] = 0.0
            A[row, row] = 1.0
    w = sla.eig(A, B, right=False)
    w = w[np.isfinite(w)]
    return complex(w[np.argmax(w.real)])


def critical_reynolds(Nr: int, eta: float, beta: float, lo: float, hi: float,
                      tol: float = 1e-4) -> float:
    """Bisection on Re_i (outer cylinder at rest) for Re(lambda) = 0, m = 0."""
    f = lambda re: leading_eigenvalue(Nr, eta, re, 0.0, 0, beta).real
    flo, fhi = f(lo), f(hi)
    if flo * fhi > 0:
        raise ValueError("no sign change in bracket")
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if fm * flo > 0:
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)
