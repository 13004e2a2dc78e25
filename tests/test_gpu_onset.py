"""Physics check of the CUDA path on its own: near the Taylor-vortex onset the
growth rate of an axisymmetric perturbation of circular Couette flow is the
leading eigenvalue of the linearised problem (classical onset Re_c = 118.16
at beta_c = 3.13 for eta = 0.875, outer cylinder at rest).  The eigenvalue
comes from the oracle's linear-stability solver, which the CPU tests pin to
the classical onset values; the stepper compared here is the GPU one."""
import math

import numpy as np
import pytest

from inputs import psi_coefficients

pytestmark = pytest.mark.gpu

ETA, BETA = 0.875, 3.13


@pytest.fixture(scope="module")
def tc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1908_00587_gb300 import tc as mod
    return mod


def _amp(X):
    # the (m = 0, k = 1) column of u_r, u_theta, u_z; any fixed norm serves
    # once the leading eigenmode dominates
    return math.sqrt(float(np.sum(np.abs(X[:3, :, 0, 1]) ** 2)))


@pytest.mark.parametrize("Re", [115.0, 121.0])
def test_growth_rate_is_the_leading_eigenvalue(tc, Re):
    from oracle.stability import leading_eigenvalue
    lam = leading_eigenvalue(32, ETA, Re, 0.0, 0, BETA).real
    dt, t1, t2 = 2e-3, 0.6, 0.8
    run = tc.Run(32, 4, 8, ETA, 2 * math.pi / BETA, Re, 0.0, 0.0, 1.0)
    run.init_perturbation(psi_coefficients(7, 0, 1), 1e-6)
    run.step(int(round(t1 / dt)), dt)
    a1 = _amp(run.get_state())
    run.step(int(round((t2 - t1) / dt)), dt)
    X = run.get_state()
    run.close()
    rate = math.log(_amp(X) / a1) / (t2 - t1)
    assert np.sign(rate) == np.sign(lam)
    assert abs(rate - lam) <= 2e-3 * abs(lam), (rate, lam)
    # an axisymmetric start keeps m != 0 at round-off
    assert np.abs(X[:, :, 1:, :]).max() <= 1e-14 * np.abs(X).max()
