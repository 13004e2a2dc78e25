"""Pins of the oracle's restart with a change of resolution (Sec. 2.1).

* radial interpolation reproduces every polynomial of degree < Nr_src at the
  new nodes, is the identity on the same grid, and coarse -> fine -> coarse
  returns the original values;
* the Fourier part keeps the trigonometric interpolant: the regridded field on
  the new (theta, z) grid equals the source series summed term by term at
  those points (padding), and modes the target cannot hold are dropped
  (truncation);
* wall values are copied exactly; the coarse basic state lands on the fine
  one to finite-difference accuracy; a run without T gets the conductive T.
"""
import math

import numpy as np

from inputs import Workload, random_state
from oracle import Model
from oracle.grid import cgl_radii
from oracle.regrid import lagrange_matrix, regrid

WL = Workload("rg", Nr=12, Ntheta=12, Nz=18, eta=0.6, Lz=2.5, Re_i=70.0, Re_o=-10.0)


def test_lagrange_reproduces_polynomials_below_node_count():
    xs = cgl_radii(12, WL.eta)
    xd = cgl_radii(31, WL.eta)
    rng = np.random.Generator(np.random.PCG64(3))
    c = rng.standard_normal(12)
    P = lagrange_matrix(xs, xd)
    poly = lambda x: np.polyval(c, x - 1.7)          # degree 11, centred in the gap
    assert np.abs(P @ poly(xs) - poly(xd)).max() <= 1e-11 * np.abs(poly(xd)).max()
    c13 = np.append(c, 1.0)                           # degree 12: not reproduced
    poly13 = lambda x: np.polyval(c13, x - 1.7)
    assert np.abs(P @ poly13(xs) - poly13(xd)).max() > 1e-8
    np.testing.assert_array_equal(lagrange_matrix(xs, xs), np.eye(12))


def test_regrid_identity_and_round_trip():
    coarse = Model(WL)
    fine = Model(WL.scaled(Nr=25, Ntheta=24, Nz=30))
    X = random_state(5, coarse.nf, WL.Nr, coarse.M, coarse.K)
    np.testing.assert_array_equal(regrid(X, WL.eta, coarse), X)
    back = regrid(regrid(X, WL.eta, fine), WL.eta, coarse)
    assert np.abs(back - X).max() <= 1e-12 * np.abs(X).max()


def _series(X1, M, K, Lz, theta, z):
    """Real field sum_{m,k} c_m Re(X(m,k) e^{i(m theta + beta z)}) term by term."""
    NK = 2 * K + 1
    out = np.zeros((X1.shape[0], theta.size, z.size))
    for m in range(M + 1):
        for k in range(-K, K + 1):
            a = X1[:, m, k % NK]
            ph = np.exp(1j * (m * theta[:, None] + 2 * math.pi * k / Lz * z[None, :]))
            w = 1.0 if m == 0 else 2.0
            out += w * np.real(a[:, None, None] * ph[None])
    return out


def test_regrid_keeps_trigonometric_interpolant():
    coarse = Model(WL)
    fine = Model(WL.scaled(Nr=WL.Nr, Ntheta=24, Nz=30))
    X = random_state(6, coarse.nf, WL.Nr, coarse.M, coarse.K)
    Y = regrid(X, WL.eta, fine)
    th = 2 * math.pi * np.arange(24) / 24
    z = WL.Lz * np.arange(30) / 30
    direct = _series(X[0], coarse.M, coarse.K, WL.Lz, th, z)
    assert np.abs(fine.sp.to_physical(Y[0]) - direct).max() <= 1e-12 * np.abs(direct).max()
    # truncation: fine -> coarse drops the modes the coarse run cannot hold
    Xf = random_state(7, fine.nf, WL.Nr, fine.M, fine.K)
    Xc = regrid(Xf, WL.eta, coarse)
    for m in range(coarse.M + 1):
        for k in range(-coarse.K, coarse.K + 1):
            np.testing.assert_array_equal(Xc[:, :, m, k % (2 * coarse.K + 1)],
                                          Xf[:, :, m, k % (2 * fine.K + 1)])


def test_regrid_walls_base_state_and_temperature():
    coarse = Model(WL.scaled(Nr=24))
    fine = Model(WL.scaled(Nr=48, Ntheta=24, Nz=30))
    Y = regrid(coarse.base, WL.eta, fine)
    # the wall nodes of both grids coincide: wall values are copied exactly
    np.testing.assert_array_equal(Y[:, [0, -1], :, :][..., :coarse.K + 1][:, :, :coarse.M + 1],
                                  coarse.base[:, [0, -1], :, :][..., :coarse.K + 1])
    err = np.abs(Y[1, :, 0, 0] - fine.base[1, :, 0, 0]).max()
    assert err <= 1e-8 * WL.Re_i
    heated = Model(WL.scaled(Nr=48, Ntheta=24, Nz=30, Ra=1500.0, Pr=0.7))
    Yt = regrid(coarse.base, WL.eta, heated)
    np.testing.assert_array_equal(Yt[3, :, 0, 0], heated.base[3, :, 0, 0])
    assert np.abs(Yt[3]).sum() == np.abs(Yt[3, :, 0, 0]).sum()
