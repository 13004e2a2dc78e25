"""The inverse axial transforms on the tensor cores (k_zinv_tc) against the
FP64 FFT path (k_zinv) of the same library and against the oracle.

k_zinv_tc forms the inverse z transforms (of the state, its d/dr stencil and
its z derivative) as products of the folded axial DFT matrix (cosine rows
over sine rows) with 7 BF16 slices per operand, exact FP32 level sums and an
exact integer combination of a cosine and a sine row per output, so it must
agree with the FP64 transforms to FP64 round-off: 1e-13 of the largest
nonlinear term, at the benchmark's size and at ragged sizes with even and
odd Nz, alone and together with the tensor-core azimuthal stage; and a
whole run through it must meet the oracle gate (option tensor_z; the default
path is the FP64 FFT)."""
import numpy as np
import pytest

from inputs import WORKLOADS, Workload, psi_coefficients, random_state, temperature_coefficients
from oracle import Model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_1908_00587_gb300 import tc as mod
    return mod


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


CASES = [
    WORKLOADS["tc_fp64T_nr64_n128"],
    Workload("zt1", Nr=17, Ntheta=96, Nz=45, eta=0.6, Lz=1.3, Re_i=70.0, Ra=0.0),
    Workload("zt2", Nr=12, Ntheta=30, Nz=24, eta=0.7, Lz=2.1, Re_i=40.0, Re_o=-9.0, Ra=400.0,
             Pr=0.9),
    Workload("zt3", Nr=9, Ntheta=8, Nz=5, eta=0.5, Lz=1.0, Re_i=20.0, Ra=0.0),
    Workload("zt4", Nr=20, Ntheta=64, Nz=75, eta=0.8, Lz=3.0, Re_i=90.0, Ra=1e3, Pr=0.7),
    Workload("zt5", Nr=10, Ntheta=12, Nz=128, eta=0.5, Lz=2.0, Re_i=30.0, Ra=0.0),
]


@pytest.mark.parametrize("wl", CASES, ids=[w.name for w in CASES])
def test_tensor_z_matches_fft_z(tc, wl):
    run = tc.Run.from_workload(wl)
    X = random_state(700 + wl.Nr, run.nf, wl.Nr, run.M, run.K)
    outs, rates = {}, {}
    for tz, tt in ((1, 0), (0, 0), (1, 1)):
        tc.tc_set_option(run.ctx, "tensor_z", tz)
        tc.tc_set_option(run.ctx, "tensor_theta", tt)
        info = tc.tc_get_info(run.ctx)
        # the tensor path is available at these sizes (table built)
        assert info.tensor_z == tz
        out = dev(np.zeros_like(X))
        rates[tz, tt] = tc.tc_nonlinear(run.ctx, dev(X), out)
        outs[tz, tt] = out.cpu().numpy()
    run.close()
    b = outs[0, 0]
    for key in ((1, 0), (1, 1)):
        rel = np.abs(outs[key] - b).max() / np.abs(b).max()
        print(f"{wl.name}: tensor z (tensor theta {key[1]}) vs FFT, max rel difference {rel:.2e}")
        assert rel <= 1e-13, (key, rel)
        assert abs(rates[key] - rates[0, 0]) <= 1e-13 * rates[0, 0]


def test_tensor_z_step_matches_oracle(tc):
    """A whole heated run with the dynamic step, both tensor-core stages on,
    against the oracle."""
    wl = WORKLOADS["tc_fp64T_nr64_n128"].scaled(Nr=24, Ntheta=48, Nz=45, mp=4, kp=4)
    mdl = Model(wl, "fft")
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    tco = temperature_coefficients(wl.seed, wl.mp, wl.kp)
    run = tc.Run.from_workload(wl)
    tc.tc_set_option(run.ctx, "tensor_z", 1)
    tc.tc_set_option(run.ctx, "tensor_theta", 1)
    run.init_perturbation(psi, wl.amp, tco, wl.amp_T)
    dts = run.step(30, wl.dt)
    got = run.get_state()
    run.close()
    X = mdl.initial_state(psi, tco)
    dtp, ref_dts = 0.0, []
    for _ in range(30):
        X, _, dtp, _ = mdl.step(X, wl.dt, dtp)
        ref_dts.append(dtp)
    assert np.all(np.abs(dts - np.array(ref_dts)) <= 1e-8 * np.array(ref_dts))
    w = (mdl.g.w * mdl.g.r)[:, None, None] * mdl.sp.cm[None, :, None]
    err = max(float(np.sqrt(np.sum(w * np.abs(got[f] - X[f]) ** 2) / np.sum(w * np.abs(X[f]) ** 2)))
              for f in range(X.shape[0]))
    assert err <= 1e-10, err


def test_tensor_z_wait_timeout_is_reported(tc):
    """k_zinv_tc waits on its DFT-slice copies with a 1 s bound: with the
    copies never started (test hook) the waits run out, the CTAs free their
    tensor memory and return, tc_nonlinear reports TC_ERR_TIMEOUT, and the
    same context then computes the stage correctly."""
    wl = CASES[3]
    run = tc.Run.from_workload(wl)
    X = dev(random_state(78, run.nf, wl.Nr, run.M, run.K))
    out = dev(np.zeros(X.shape, dtype=np.complex128))
    tc.tc_set_option(run.ctx, "tensor_z", 1)
    tc.tc_set_option(run.ctx, "selftest_no_copy", 1)
    with pytest.raises(tc.TCError) as e:
        tc.tc_nonlinear(run.ctx, X, out)
    assert e.value.name == "TC_ERR_TIMEOUT"
    tc.tc_set_option(run.ctx, "selftest_no_copy", 0)
    tc.tc_nonlinear(run.ctx, X, out)
    a = out.cpu().numpy()
    tc.tc_set_option(run.ctx, "tensor_z", 0)
    tc.tc_nonlinear(run.ctx, X, out)
    b = out.cpu().numpy()
    run.close()
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
