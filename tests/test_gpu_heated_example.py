"""The illustrative heated example (Sec. 4) behaves as described there.

Qualitative, not a parity target (the paper omits eta, Pr, Lz and the grid):
at Re_i = 50, Ra = 2130 the run starts with purely conductive heat transfer
(Nu_i = 1), and after about two viscous times the single-harmonic disturbance
has grown into a convective state with Nu_i above 1 and a time-dependent
u_theta at the mid-gap probe.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def example():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1908_00587_gb300 import heated_example
    return heated_example


def test_heated_example_first_transition(example):
    rows = np.array(example.run(t_stage=3.0, ras=(2130.0,), verbose=False))
    t, nu, probe = rows[:, 1], rows[:, 2], rows[:, 3]
    assert abs(nu[0] - 1.0) < 1e-6                       # conductive start
    assert np.all(np.abs(nu[t < 1.0] - 1.0) < 1e-3)      # still conductive early on
    assert nu[-1] > 1.002                                 # convective after ~2 viscous times
    late = probe[t > 2.5]
    assert late.std() > 1e-3 * abs(late.mean())           # time-dependent flow at the probe
    assert np.all(np.isfinite(rows))
