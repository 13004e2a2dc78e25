"""GPU discrete adjoint (differentiation form) against the oracle and
against finite differences of the GPU forward map.

Inner product: real Euclidean on stored (Re, Im) coefficients,
<a, b> = sum Re(conj(a) b).  The step adjoint is P_H J^T (see
tc_adjoint_step); the stage adjoints are checked by the dot-product identity
<A v, w> = <v, A^T w> with the forward maps of the same library.
"""
import numpy as np
import pytest

from inputs import WORKLOADS, Workload, psi_coefficients, random_state, temperature_coefficients
from oracle import Model
from oracle.adjoint import adjoint_step_dense, hermitian_projection, objective

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


def host(t):
    return t.cpu().numpy()


def dot(a, b):
    return float(np.sum((np.conj(a) * b).real))


TINY = Workload("adjt", Nr=12, Ntheta=12, Nz=12, eta=0.6, Lz=1.7, Re_i=40.0, Re_o=-10.0,
                Ra=300.0, Pr=0.8, amp=0.3, mp=2, kp=2, amp_T=0.1, seed=3, dt=2e-3)


@pytest.mark.parametrize("Ra", [0.0, 300.0])
def test_nonlinear_adjoint_dot_product(tc, Ra):
    wl = TINY.scaled(Ra=Ra, Nr=20, Ntheta=24, Nz=30)
    run = tc.Run.from_workload(wl)
    nf = run.nf
    X = random_state(41, nf, wl.Nr, run.M, run.K)
    v = random_state(42, nf, wl.Nr, run.M, run.K)
    w = random_state(43, nf, wl.Nr, run.M, run.K)

    def N(a):
        out = dev(np.zeros_like(a))
        tc.tc_nonlinear(run.ctx, dev(a), out)
        return host(out)

    Jv = N(X + v) - N(X) - N(v)
    if nf == 4:
        Jv[2] += (wl.Ra / wl.Pr) * v[3]
    xb = dev(np.zeros_like(X))
    tc.tc_nonlinear_adjoint(run.ctx, dev(X), dev(w), xb)
    lhs, rhs = dot(w, Jv), dot(host(xb), v)
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs)), (lhs, rhs)
    run.close()


@pytest.mark.parametrize("Ra", [0.0, 300.0])
def test_stage_adjoint_dot_product(tc, Ra):
    wl = TINY.scaled(Ra=Ra, Nr=33, Ntheta=18, Nz=24)
    run = tc.Run.from_workload(wl)
    nf = run.nf
    v = random_state(51, nf, wl.Nr, run.M, run.K)     # +- right-hand side
    w = random_state(52, nf, wl.Nr, run.M, run.K)     # primitive cotangent
    dt = 3e-3

    def A(r):
        out = dev(np.zeros_like(r))
        tc.tc_stage_solve(run.ctx, dev(r), dt, out)
        return host(out)

    Av = A(v) - A(np.zeros_like(v))
    rb = dev(np.zeros_like(w))
    tc.tc_stage_solve_adjoint(run.ctx, dev(w), dt, rb)
    lhs, rhs = dot(w, Av), dot(host(rb), v)
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs)), (lhs, rhs)
    run.close()


def test_adjoint_step_matches_oracle_dense_gpu(tc):
    wl = TINY.scaled(Nr=10, Ntheta=8, Nz=8, mp=1, kp=1)
    mdl = Model(wl)
    X = mdl.initial_state(psi_coefficients(wl.seed, 1, 1), temperature_coefficients(wl.seed, 1, 1))
    lam = hermitian_projection(random_state(61, mdl.nf, wl.Nr, mdl.M, mdl.K))
    ref = adjoint_step_dense(mdl, X, lam, wl.dt)
    run = tc.Run.from_workload(wl)
    adj = dev(lam)
    tc.tc_adjoint_step(run.ctx, dev(X), wl.dt, adj)
    got = host(adj)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    run.close()


def test_gradient_matches_oracle_differences(tc):
    """d E_pert(X^N) / d psi through the whole chain on a tiny grid vs central
    differences of the oracle with the same frozen initial-condition scales."""
    import torch
    from paper_1908_00587_gb300.autograd import perturbation_energy
    wl = TINY
    nsteps = 4
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    tco = temperature_coefficients(wl.seed, wl.mp, wl.kp)
    mdl = Model(wl, "fft")
    # the oracle fixes its own scales (max|u'| = amp, max|T'| = amp_T); the
    # library's, found by its own kernels, must agree with them
    su, sT = mdl.ic_scales(psi, tco)
    run = tc.Run.from_workload(wl)
    run.init_perturbation(psi, wl.amp, tco, wl.amp_T)
    su_gpu, sT_gpu = tc.tc_get_ic_scales(run.ctx)
    assert abs(su_gpu - su) <= 1e-12 * su and abs(sT_gpu - sT) <= 1e-12 * sT
    pt = torch.from_numpy(psi.copy()).requires_grad_(True)
    tt = torch.from_numpy(tco.copy()).requires_grad_(True)
    J = perturbation_energy(run, pt, nsteps, wl.dt, -su, tt, -sT, checkpoint=3)
    J.backward()
    gpsi, gt = pt.grad.numpy(), tt.grad.numpy()
    run.close()

    def Jor(p, t):
        X = mdl.initial_state(p, t, scales=(su, sT))
        X, _ = mdl.run(X, nsteps, wl.dt)
        return objective(mdl, X)

    Jv = float(J.detach())
    assert abs(Jv - Jor(psi, tco)) <= 1e-10 * abs(Jv)
    rng = np.random.default_rng(7)
    for _ in range(3):
        dp = rng.standard_normal(psi.shape) + 1j * rng.standard_normal(psi.shape)
        dtc = rng.standard_normal(tco.shape) + 1j * rng.standard_normal(tco.shape)
        eps = 1e-6
        fd = (Jor(psi + eps * dp, tco + eps * dtc) - Jor(psi - eps * dp, tco - eps * dtc)) / (2 * eps)
        ad = dot(gpsi, dp) + dot(gt, dtc)
        assert abs(fd - ad) <= 1e-6 * abs(fd), (fd, ad)


def test_gradient_vs_central_differences_adjoint_workload(tc):
    """64^3, eta = 0.5, Re_i = 120, 200 steps of dt = 2e-4, checkpoints every
    20 steps: the adjoint gradient against central differences of the GPU
    forward map on 16 seeded directions, at eps = 1e-3 and eps = 1e-6.

    J is the energy of a 1e-3 perturbation riding on an O(120) base flow.  The
    step works on the whole field, so every step rounds the state at ~1e-16 of
    the base flow, i.e. ~1e-13 of the perturbation; which way each rounding
    goes depends on the last bits of the coefficients.  J(psi + t d) is
    therefore a smooth function plus a deterministic but irregular floor
    sigma_J (measured on GB300: about 1e-12 of J).  Here the floor is
    measured, not assumed:
      * repeated identical runs give bit-identical J (no run-to-run jitter);
      * along each of two directions, J at 9 points t in [-4e-6, 4e-6] is fit
        by a quadratic; the residual RMS is sigma_J;
      * a central difference at eps then carries an error of about
        sqrt(2) sigma_J / (2 eps |J'|), and the measured eps = 1e-6 error
        must agree with that prediction (within 5x either way allowed above,
        it may be smaller) -- at eps = 1e-6 the difference quotient measures
        the floor, not the gradient;
      * at eps = 1e-3 the floor's share is 1000x smaller and J is close to
        quadratic in the coefficients, so the central difference meets the
        1e-6 criterion there.
    """
    import torch
    from paper_1908_00587_gb300.autograd import perturbation_energy
    wl = WORKLOADS["tc_adjoint_nr64_n64"]
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    su, _ = Model(wl, "fft").ic_scales(psi)
    run = tc.Run.from_workload(wl)
    run.init_perturbation(psi, wl.amp)
    su_gpu, _ = tc.tc_get_ic_scales(run.ctx)
    assert abs(su_gpu - su) <= 1e-12 * su
    pt = torch.from_numpy(psi.copy()).requires_grad_(True)
    J = perturbation_energy(run, pt, wl.steps, wl.dt, -su, None, 0.0, checkpoint=20)
    J.backward()
    g = pt.grad.numpy()

    def Jgpu(p):
        run.init_perturbation(p, -su)
        run.step(wl.steps, wl.dt)
        return tc.tc_objective(run.ctx)

    J0 = Jgpu(psi)
    assert Jgpu(psi) == J0          # deterministic: identical runs, identical J
    rng = np.random.default_rng(16)
    dirs = [rng.standard_normal(psi.shape) + 1j * rng.standard_normal(psi.shape)
            for _ in range(16)]
    worst = {1e-3: 0.0, 1e-6: 0.0}
    err6 = []
    for d in dirs:
        ad = dot(g, d)
        for eps in worst:
            fd = (Jgpu(psi + eps * d) - Jgpu(psi - eps * d)) / (2 * eps)
            e = abs(fd - ad) / abs(fd)
            worst[eps] = max(worst[eps], e)
            if eps == 1e-6:
                err6.append(e)
    # the floor along the first two directions
    ts = np.linspace(-4e-6, 4e-6, 9)
    floors, predicted = [], []
    for d in dirs[:2]:
        Js = np.array([Jgpu(psi + t * d) for t in ts])
        coef = np.polyfit(ts, Js - J0, 2)
        resid = (Js - J0) - np.polyval(coef, ts)
        sigma = float(np.sqrt(np.sum(resid ** 2) / (len(ts) - 3)))
        slope = abs(dot(g, d))
        floors.append(sigma / abs(J0))
        predicted.append(np.sqrt(2.0) * sigma / (2e-6 * slope))
    run.close()
    print("adjoint 64^3 200 steps: worst rel diff vs central FD over 16 directions:",
          {k: f"{v:.2e}" for k, v in worst.items()},
          f"| J floor sigma_J/J {floors[0]:.2e} {floors[1]:.2e}",
          f"| predicted eps=1e-6 error {predicted[0]:.2e} {predicted[1]:.2e},"
          f" measured on those directions {err6[0]:.2e} {err6[1]:.2e}")
    assert worst[1e-3] <= 1e-6
    # the eps = 1e-6 error is the floor: it agrees with the floor's prediction
    for meas, pred in zip(err6[:2], predicted):
        assert meas <= 5.0 * pred + 1e-6, (meas, pred)
    # and the floor is round-off of the whole field, ~1e-10 of J, not larger
    assert max(floors) <= 1e-9


def test_recorded_segment_matches_step_by_step(tc):
    """tc_adjoint_steps over tc_step_record's records equals chained
    tc_adjoint_step calls on the same states (the records hold the forward
    run's own predictor states; the single-step entry point recomputes them,
    which differs only by round-off)."""
    import torch
    wl = TINY.scaled(Nr=20, Ntheta=24, Nz=24, mp=3, kp=3)
    run = tc.Run.from_workload(wl)
    run.init_perturbation(psi_coefficients(wl.seed, wl.mp, wl.kp), wl.amp,
                          temperature_coefficients(wl.seed, wl.mp, wl.kp), wl.amp_T)
    n = 6
    per = tc.tc_record_bytes_per_step(run.ctx)
    rec = torch.empty(n * per, dtype=torch.uint8, device="cuda")
    X0 = run.get_state()
    tc.tc_step_record(run.ctx, n, wl.dt, rec)
    X_rec = run.get_state()
    # the recorded run advanced the state like tc_step
    ref = tc.Run.from_workload(wl)
    ref.set_state(X0)
    ref.step(n, wl.dt)
    X_plain = ref.get_state()
    ref.close()
    assert np.abs(X_rec - X_plain).max() <= 1e-12 * np.abs(X_plain).max()
    lam0 = hermitian_projection(random_state(71, run.nf, wl.Nr, run.M, run.K))
    lam_a = dev(lam0)
    tc.tc_adjoint_steps(run.ctx, n, rec, wl.dt, lam_a)
    nstate = int(np.prod(run.shape)) * 16
    states = [rec[k * per:k * per + nstate].view(torch.complex128).reshape(run.shape)
              for k in range(n)]
    lam_b = dev(lam0)
    for k in reversed(range(n)):
        tc.tc_adjoint_step(run.ctx, states[k], wl.dt, lam_b)
    run.close()
    a, b = host(lam_a), host(lam_b)
    assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()
    np.testing.assert_array_equal(host(states[0]), X0)


def test_gradient_recorded_and_recomputed_agree(tc):
    import torch
    from paper_1908_00587_gb300.autograd import perturbation_energy
    wl = TINY.scaled(Nr=20, Ntheta=24, Nz=24, mp=3, kp=3)
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    grads = []
    for budget in (4 << 30, 0):
        run = tc.Run.from_workload(wl)
        run.init_perturbation(psi, wl.amp)
        su, _ = tc.tc_get_ic_scales(run.ctx)
        pt = torch.from_numpy(psi.copy()).requires_grad_(True)
        J = perturbation_energy(run, pt, 9, wl.dt, -su, None, 0.0, checkpoint=4,
                                record_budget=budget)
        J.backward()
        grads.append(pt.grad.numpy().copy())
        run.close()
    assert np.abs(grads[0] - grads[1]).max() <= 1e-9 * np.abs(grads[1]).max()
