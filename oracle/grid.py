"""Radial grid, finite-difference weights and radial quadrature (oracle).

Sec. 2.1: the radial direction is the only inhomogeneous one and is discretised
by high-order finite differences on a runtime-selectable point distribution,
with a 9-point stencil by default.

Readings (the paper gives no formulas):
* the gap is [r_i, r_o] with d = r_o - r_i = 1, r_i = eta/(1-eta);
* the radial points are Chebyshev-Gauss-Lobatto points, wall nodes included,
  r_j = r_i + (1 - cos(pi j/(Nr-1)))/2, ascending;
* the stencil of node j is the 9 nodes [s, s+8], s = clamp(j-4, 0, Nr-9):
  centred where it fits, one-sided next to the walls;
* weights come from Fornberg's recursion (Math. Comp. 51, 1988), written
  here from the published recursion for the Lagrange-interpolant derivatives.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

STENCIL = 9


def cgl_radii(Nr: int, eta: float) -> np.ndarray:
    """Chebyshev-Gauss-Lobatto radii on [r_i, r_i + 1], ascending."""
    r_i = eta / (1.0 - eta)
    j = np.arange(Nr, dtype=np.float64)
    return r_i + 0.5 * (1.0 - np.cos(np.pi * j / (Nr - 1)))


def fornberg_weights(x0: float, x: np.ndarray, order: int) -> np.ndarray:
    """Finite-difference weights at x0 on nodes x, derivatives 0..order.

    Returns w of shape (order+1, len(x)) with sum_j w[d, j] f(x_j) ~ f^(d)(x0).
    Fornberg's recursion builds the weights of the Lagrange interpolant on
    x[0..i] from those on x[0..i-1], one node at a time.
    """
    n = len(x)
    w = np.zeros((order + 1, n))
    w[0, 0] = 1.0
    prod_prev = 1.0
    dx_prev = x[0] - x0
    for i in range(1, n):
        top = min(i, order)
        prod = 1.0
        dx_i = x[i] - x0
        for j in range(i):
            diff = x[i] - x[j]
            prod *= diff
            if j == i - 1:
                # weights of the newly added node i
                for d in range(top, 0, -1):
                    w[d, i] = prod_prev * (d * w[d - 1, i - 1] - dx_prev * w[d, i - 1]) / prod
                w[0, i] = -prod_prev * dx_prev * w[0, i - 1] / prod
            # update the weights of the old node j
            for d in range(top, 0, -1):
                w[d, j] = (dx_i * w[d, j] - d * w[d - 1, j]) / diff
            w[0, j] = dx_i * w[0, j] / diff
        prod_prev = prod
        dx_prev = dx_i
    return w


def stencil_start(j: int, Nr: int) -> int:
    return min(max(j - STENCIL // 2, 0), Nr - STENCIL)


def fd_matrices(r: np.ndarray):
    """Dense first- and second-derivative matrices D1, D2 (Nr x Nr)."""
    Nr = len(r)
    D1 = np.zeros((Nr, Nr))
    D2 = np.zeros((Nr, Nr))
    for j in range(Nr):
        s = stencil_start(j, Nr)
        w = fornberg_weights(r[j], r[s:s + STENCIL], 2)
        D1[j, s:s + STENCIL] = w[1]
        D2[j, s:s + STENCIL] = w[2]
    return D1, D2


def cc_weights(Nr: int) -> np.ndarray:
    """Clenshaw-Curtis weights on the CGL points of [-1, 1].

    Plain definition: the weights integrate every Chebyshev polynomial T_n,
    n <= Nr-1, exactly (int_{-1}^{1} T_n = 2/(1-n^2) for even n, 0 for odd n).
    Solved as a linear system in the Chebyshev basis (well conditioned on
    these points).
    """
    N = Nr - 1
    x = -np.cos(np.pi * np.arange(Nr) / N)
    n = np.arange(Nr)
    T = np.cos(np.outer(n, np.arccos(np.clip(x, -1.0, 1.0))))  # T[n, j] = T_n(x_j)
    mom = np.zeros(Nr)
    even = n % 2 == 0
    mom[even] = 2.0 / (1.0 - n[even].astype(np.float64) ** 2)
    return np.linalg.solve(T, mom)


@dataclass
class Grid:
    """Radial grid of one run: nodes, D1/D2, quadrature on [r_i, r_o]."""

    Nr: int
    eta: float

    def __post_init__(self):
        self.r_i = self.eta / (1.0 - self.eta)
        self.r_o = 1.0 / (1.0 - self.eta)
        self.r = cgl_radii(self.Nr, self.eta)
        self.D1, self.D2 = fd_matrices(self.r)
        # dr = dx/2 on the map x = 2(r - r_i) - 1
        self.w = 0.5 * cc_weights(self.Nr)
        self.x = 2.0 * (self.r - self.r_i) - 1.0

    def dr(self, f: np.ndarray) -> np.ndarray:
        """D1 applied along axis 0."""
        return np.tensordot(self.D1, f, axes=(1, 0))

    def drr(self, f: np.ndarray) -> np.ndarray:
        return np.tensordot(self.D2, f, axes=(1, 0))

    def min_spacing(self) -> np.ndarray:
        """Distance from each node to its nearest neighbour."""
        d = np.diff(self.r)
        out = np.empty(self.Nr)
        out[0] = d[0]
        out[-1] = d[-1]
        out[1:-1] = np.minimum(d[:-1], d[1:])
        return out


def couette_AB(eta: float, Re_i: float, Re_o: float):
    """Analytic circular Couette profile u_theta = A r + B / r (Sec. 4).

    Viscous units (d = 1): u_theta(r_i) = Re_i, u_theta(r_o) = Re_o.
    """
    A = (Re_o - eta * Re_i) / (1.0 + eta)
    B = eta * (Re_i - eta * Re_o) / ((1.0 - eta) * (1.0 - eta ** 2))
    return A, B


def conductive_T(r: np.ndarray, eta: float) -> np.ndarray:
    """Analytic conductive temperature, T(r_i) = +1/2, T(r_o) = -1/2 (Sec. 4)."""
    r_o = 1.0 / (1.0 - eta)
    return np.log(r / r_o) / math.log(eta) - 0.5
