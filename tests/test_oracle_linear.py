"""Pins of the oracle's radial stage (per-mode Helmholtz / Poisson solves).

Sec. 2.2: Fourier modes are independent in the linear terms.  The stage solve
is checked by substituting its output back into the equations it must satisfy
(the definition), mode by mode, with dense matrices built independently here.
"""
import numpy as np
import pytest

from inputs import Workload
from oracle.model import CN, Model


def _model(Ra=0.0):
    wl = Workload("lin", Nr=20, Ntheta=12, Nz=15, eta=0.6, Lz=1.9,
                  Re_i=50.0, Re_o=-10.0, Ra=Ra, Pr=0.8)
    return Model(wl)


def _random_R(mdl, rng):
    sh = (mdl.wl.Nr, mdl.M + 1, mdl.NK)
    R = [mdl.sp.hermitian_fix(rng.standard_normal(sh) + 1j * rng.standard_normal(sh))
         for _ in range(mdl.nf)]
    # R+ and R- of a real field: R+(0,-k) = conj R-(0,k)
    Rr = mdl.sp.hermitian_fix(rng.standard_normal(sh) + 1j * rng.standard_normal(sh))
    Rt = mdl.sp.hermitian_fix(rng.standard_normal(sh) + 1j * rng.standard_normal(sh))
    R[0], R[1] = Rr + 1j * Rt, Rr - 1j * Rt
    return R


@pytest.mark.parametrize("Ra", [0.0, 500.0])
def test_stage_solve_satisfies_its_equations(Ra):
    mdl = _model(Ra)
    rng = np.random.default_rng(7)
    R = _random_R(mdl, rng)
    dt = 3e-3
    X, p = mdl.stage_solve(R, dt)
    g = mdl.g
    r = g.r
    D1, D2 = g.D1, g.D2
    I = np.eye(g.Nr)
    scale = max(np.abs(Ri).max() for Ri in R)
    for im in range(mdl.M + 1):
        for ik in range(mdl.NK):
            m = float(im)
            beta = mdl.sp.beta[ik]

            def L(q):
                return D2 + D1 / r[:, None] - np.diag(q * q / r ** 2) - beta ** 2 * I

            ur, ut, uz = X[0][:, im, ik], X[1][:, im, ik], X[2][:, im, ik]
            up, um = ur + 1j * ut, ur - 1j * ut
            pp = p[:, im, ik]
            Rp, Rm, Rz = R[0][:, im, ik], R[1][:, im, ik], R[2][:, im, ik]
            inner = slice(1, -1)
            if (im, ik) == (0, 0):
                assert np.abs(ur).max() == 0.0
                Rt = (Rp - Rm) / 2j
                res = (I / dt - CN * L(1.0)) @ ut - Rt
                assert np.abs(res[inner]).max() < 1e-10 * scale
                assert abs(ut[0] - mdl.wl.Re_i) < 1e-12 and abs(ut[-1] - mdl.wl.Re_o) < 1e-12
                res = (I / dt - CN * L(0.0)) @ uz - Rz
                assert np.abs(res[inner]).max() < 1e-10 * scale
                continue
            # momentum rows at interior nodes
            gp = D1 @ pp
            res_p = (I / dt - CN * L(m + 1)) @ up - (Rp - (gp - m * pp / r))
            res_m = (I / dt - CN * L(m - 1)) @ um - (Rm - (gp + m * pp / r))
            res_z = (I / dt - CN * L(m)) @ uz - (Rz - 1j * beta * pp)
            for res in (res_p, res_m, res_z):
                assert np.abs(res[inner]).max() < 1e-9 * scale
            # no-slip rows
            for f in (ur, ut, uz):
                assert abs(f[0]) < 1e-13 * scale and abs(f[-1]) < 1e-13 * scale
            # Poisson rows: L p = div R inside
            Rr, Rt = (Rp + Rm) / 2, (Rp - Rm) / 2j
            divR = (D1 @ (r * Rr)) / r + 1j * m * Rt / r + 1j * beta * Rz
            resP = L(m) @ pp - divR
            assert np.abs(resP[inner]).max() < 1e-8 * scale
            # continuity at both wall nodes (influence matrix)
            div = (D1 @ (r * ur)) / r + 1j * m * ut / r + 1j * beta * uz
            gu = np.abs(D1 @ ur).max() + 1e-300
            assert abs(div[0]) < 1e-10 * gu and abs(div[-1]) < 1e-10 * gu
    if Ra:
        T = X[3]
        for im in range(mdl.M + 1):
            for ik in range(mdl.NK):
                beta = mdl.sp.beta[ik]
                Lm = D2 + D1 / r[:, None] - np.diag(im * im / r ** 2) - beta ** 2 * I
                res = (I / dt - CN * mdl.kappa_T * Lm) @ T[:, im, ik] - R[3][:, im, ik]
                assert np.abs(res[1:-1]).max() < 1e-10 * scale
                wall = (0.5, -0.5) if (im, ik) == (0, 0) else (0.0, 0.0)
                assert abs(T[0, im, ik] - wall[0]) < 1e-13
                assert abs(T[-1, im, ik] - wall[1]) < 1e-13


def test_stage_solve_keeps_hermitian_m0_column():
    mdl = _model(300.0)
    rng = np.random.default_rng(8)
    X, _ = mdl.stage_solve(_random_R(mdl, rng), 1e-3)
    for f in X:
        np.testing.assert_allclose(f[:, 0, 1:mdl.K + 1],
                                   np.conj(f[:, 0, mdl.K + 1:][:, ::-1]), atol=1e-12)


def test_influence_matrix_is_nonsingular_and_real():
    mdl = _model()
    ops = mdl.operators(1e-3)
    A = ops["A"]
    assert np.abs(A.imag).max() < 1e-12 * np.abs(A).max()
    assert np.min(np.abs(np.linalg.det(A.real))) > 0


def test_explicit_operator_decouples_in_pm_form():
    """L+- of u+- equals the cylindrical vector Laplacian (closed form).

    For a single mode, (lap u)_r = L u_r - u_r/r^2 - (2im/r^2) u_theta and
    (lap u)_theta = L u_theta - u_theta/r^2 + (2im/r^2) u_r.
    """
    mdl = _model()
    g = mdl.g
    rng = np.random.default_rng(9)
    sh = (g.Nr, mdl.M + 1, mdl.NK)
    ur = rng.standard_normal(sh) + 1j * rng.standard_normal(sh)
    ut = rng.standard_normal(sh) + 1j * rng.standard_normal(sh)
    m = mdl.sp.m[:, None].astype(float)
    r = g.r[:, None, None]
    Lpm = mdl.explicit_linear([ur + 1j * ut, ur - 1j * ut, ur])
    lap_r = mdl.apply_lap(ur, m) - ur / r ** 2 - 2j * m * ut / r ** 2
    lap_t = mdl.apply_lap(ut, m) - ut / r ** 2 + 2j * m * ur / r ** 2
    np.testing.assert_allclose(Lpm[0], lap_r + 1j * lap_t, atol=1e-8 * np.abs(Lpm[0]).max())
    np.testing.assert_allclose(Lpm[1], lap_r - 1j * lap_t, atol=1e-8 * np.abs(Lpm[1]).max())
