"""Pins of the oracle's radial discretisation (Sec. 2.1: 9-point FD in r).

Each check compares against something other than the oracle itself: textbook
weights, the Vandermonde definition of FD weights, exact differentiation of
polynomials, the convergence order, and closed-form quadrature rules.
"""
import math
import os

import numpy as np
import pytest

from oracle.grid import (Grid, cc_weights, cgl_radii, conductive_T, couette_AB,
                         fd_matrices, fornberg_weights)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _textbook():
    rows = []
    with open(os.path.join(GOLDEN, "fd_textbook_weights.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            d, nodes, w = line.split()
            rows.append((int(d), [float(v) for v in nodes.split(",")],
                         [float(v) for v in w.split(",")]))
    return rows


@pytest.mark.parametrize("row", _textbook())
def test_fornberg_textbook_weights(row):
    d, nodes, w = row
    got = fornberg_weights(0.0, np.array(nodes), d)[d]
    np.testing.assert_allclose(got, w, rtol=0, atol=1e-14)


def test_fornberg_matches_vandermonde_definition():
    """Weights solve sum_j w_j (x_j - x0)^p = p! [p == d] (definition)."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        x = np.sort(rng.uniform(0, 1, 9))
        x0 = rng.uniform(x[0], x[-1])
        h = x[-1] - x[0]
        s = (x - x0) / h
        V = np.vander(s, 9, increasing=True).T       # V[p, j] = s_j^p
        for d in (1, 2):
            rhs = np.zeros(9)
            rhs[d] = math.factorial(d)
            ref = np.linalg.solve(V, rhs) / h ** d
            got = fornberg_weights(x0, x, 2)[d]
            np.testing.assert_allclose(got, ref, rtol=1e-8,
                                       atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("Nr", [9, 16, 32, 64])
def test_fd_exact_on_polynomials(Nr):
    r = cgl_radii(Nr, 0.5)
    D1, D2 = fd_matrices(r)
    for p in range(9):
        f = r ** p
        d1 = p * r ** (p - 1) if p >= 1 else 0 * r
        d2 = p * (p - 1) * r ** (p - 2) if p >= 2 else 0 * r
        sc = max(1.0, np.abs(d1).max(), np.abs(d2).max())
        assert np.abs(D1 @ f - d1).max() <= 1e-9 * sc * Nr ** 2
        assert np.abs(D2 @ f - d2).max() <= 1e-8 * sc * Nr ** 4


def test_fd_not_exact_beyond_degree_8():
    """A 9-point stencil is exact only up to degree 8 (sanity of the pin)."""
    r = cgl_radii(32, 0.5)
    D1, _ = fd_matrices(r)
    x = r - r.mean()
    f = x ** 12
    assert np.abs(D1 @ f - 12 * x ** 11).max() > 1e-10


def test_fd_convergence_order():
    errs = []
    for Nr in (24, 48):
        r = cgl_radii(Nr, 0.5)
        D1, D2 = fd_matrices(r)
        f = np.sin(3 * r)
        errs.append((np.abs(D1 @ f - 3 * np.cos(3 * r)).max(),
                     np.abs(D2 @ f + 9 * np.sin(3 * r)).max()))
    o1 = math.log(errs[0][0] / errs[1][0]) / math.log(2)
    o2 = math.log(errs[0][1] / errs[1][1]) / math.log(2)
    assert o1 > 6.5 and o2 > 5.5, (o1, o2)


def test_stencil_layout():
    """Stencil of node j is [clamp(j-4, 0, Nr-9), +8]: centred inside."""
    Nr = 20
    D1, _ = fd_matrices(cgl_radii(Nr, 0.5))
    for j in range(Nr):
        nz = np.nonzero(D1[j])[0]
        s = min(max(j - 4, 0), Nr - 9)
        assert nz.min() >= s and nz.max() <= s + 8


def test_cgl_radii():
    r = cgl_radii(5, 0.5)
    np.testing.assert_allclose(r, [1.0, 1.0 + (1 - math.sqrt(0.5)) / 2, 1.5,
                                   1.0 + (1 + math.sqrt(0.5)) / 2, 2.0], atol=1e-15)


def test_clenshaw_curtis_simpson_and_exactness():
    np.testing.assert_allclose(cc_weights(3), [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    for Nr in (9, 17, 32):
        w = cc_weights(Nr)
        x = -np.cos(np.pi * np.arange(Nr) / (Nr - 1))
        assert np.all(w > 0)
        for p in range(Nr):
            exact = 0.0 if p % 2 else 2.0 / (p + 1)
            assert abs(w @ x ** p - exact) < 1e-13


def test_grid_quadrature_on_gap():
    g = Grid(32, 0.71)
    # int r dr over [r_i, r_o] = (r_o^2 - r_i^2)/2
    assert abs(np.sum(g.w * g.r) - 0.5 * (g.r_o ** 2 - g.r_i ** 2)) < 1e-13


def test_couette_closed_form():
    for eta, ri_, ro_ in ((0.5, 100.0, 0.0), (0.71, 3000.0, -1000.0)):
        A, B = couette_AB(eta, ri_, ro_)
        r_i, r_o = eta / (1 - eta), 1 / (1 - eta)
        assert abs(A * r_i + B / r_i - ri_) < 1e-10 * abs(ri_)
        assert abs(A * r_o + B / r_o - ro_) < 1e-10 * max(1.0, abs(ro_))
    A, B = couette_AB(0.5, 100.0, 0.0)
    assert abs(A + 100 / 3) < 1e-12 and abs(B - 400 / 3) < 1e-12


def test_conductive_profile_closed_form():
    r = cgl_radii(16, 0.71)
    T = conductive_T(r, 0.71)
    assert abs(T[0] - 0.5) < 1e-14 and abs(T[-1] + 0.5) < 1e-14
    # harmonic in the plane: (r T')' = 0
    D1, _ = fd_matrices(r)
    assert np.abs(D1 @ (r * (D1 @ T))).max() < 1e-6
