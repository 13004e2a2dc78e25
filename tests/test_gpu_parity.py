"""GPU parity: every stage of the CUDA path against the FP64 oracle.

All inputs come from the seeded generators in ``inputs``; expected values come
only from ``oracle``.  Tolerances: single stages 1e-12 relative to the largest
output coefficient (they differ only by rounding order); whole runs relative
L2 <= 1e-10 per field after 100 steps, weighted by c_m w_j r_j.
"""
import math

import numpy as np
import pytest

from inputs import (WORKLOADS, Workload, psi_coefficients, random_state,
                    temperature_coefficients)
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


def rel_l2(mdl, a, b):
    w = (mdl.g.w * mdl.g.r)[:, None, None] * mdl.sp.cm[None, :, None]
    out = []
    for f in range(a.shape[0]):
        num = np.sum(w * np.abs(a[f] - b[f]) ** 2)
        den = np.sum(w * np.abs(b[f]) ** 2)
        out.append(float(np.sqrt(num / den)))
    return max(out)


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


SIZES = [
    # Nr, Ntheta, Nz, Ra : several tiles, ragged tails, radices 2/3/5
    (12, 24, 30, 500.0),
    (20, 32, 32, 0.0),
    (9, 48, 40, 0.0),
    (16, 20, 12, 800.0),
    (33, 36, 18, 0.0),
    (10, 64, 64, 300.0),   # twiddled radix-8 passes (plan 8 x 8) in both directions
]


def _wl(Nr, Nt, Nz, Ra):
    return Workload("p", Nr=Nr, Ntheta=Nt, Nz=Nz, eta=0.62, Lz=1.7, Re_i=60.0, Re_o=-15.0,
                    Ra=Ra, Pr=0.8)


@pytest.mark.parametrize("Nr,Nt,Nz,Ra", SIZES)
def test_nonlinear_matches_oracle(tc, Nr, Nt, Nz, Ra):
    wl = _wl(Nr, Nt, Nz, Ra)
    mdl = Model(wl)
    X = random_state(100 + Nr, mdl.nf, Nr, mdl.M, mdl.K)
    ref, rate = mdl.nonlinear(X)
    run = tc.Run.from_workload(wl)
    out = dev(np.zeros_like(X))
    got_rate = tc.tc_nonlinear(run.ctx, dev(X), out)
    got = out.cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-12 * scale
    assert abs(got_rate - rate) <= 1e-13 * rate
    run.close()


@pytest.mark.parametrize("Nr,Nt,Nz,Ra", SIZES)
def test_stage_solve_matches_oracle(tc, Nr, Nt, Nz, Ra):
    wl = _wl(Nr, Nt, Nz, Ra)
    mdl = Model(wl)
    Rr, Rt = random_state(200 + Nr, 2, Nr, mdl.M, mdl.K)
    R = [Rr + 1j * Rt, Rr - 1j * Rt]
    if mdl.nf == 4:
        R += list(random_state(300 + Nr, 2, Nr, mdl.M, mdl.K))
    else:
        R += [random_state(300 + Nr, 1, Nr, mdl.M, mdl.K)[0]]
    R = np.stack(R)
    dt = 2.5e-3
    Xref, Pref = mdl.stage_solve(list(R), dt)
    run = tc.Run.from_workload(wl)
    xo = dev(np.zeros_like(R))
    po = dev(np.zeros(R.shape[1:], dtype=np.complex128))
    tc.tc_stage_solve(run.ctx, dev(R), dt, xo, po)
    X, P = xo.cpu().numpy(), po.cpu().numpy()
    for f in range(mdl.nf):
        assert np.abs(X[f] - Xref[f]).max() <= 1e-11 * np.abs(Xref[f]).max(), f
    assert np.abs(P - Pref).max() <= 1e-11 * np.abs(Pref).max()
    run.close()


def _stage_backward_errors(mdl, R, dt, X, P):
    """Worst componentwise backward error |A x - b|_i / (|A| |x| + |b|)_i over
    the interior rows of each stage equation, and of the influence-matrix
    continuity condition at both walls, for a stage solution (X, P)."""
    from oracle.model import CN
    g = mdl.g
    r, D1, D2, I = g.r, g.D1, g.D2, np.eye(g.Nr)
    inner = slice(1, -1)

    def berr(A, x, b):
        res = A @ x - b
        den = np.abs(A) @ np.abs(x) + np.abs(b)
        return float((np.abs(res[inner]) / den[inner]).max())

    worst = {"momentum": 0.0, "poisson": 0.0, "T": 0.0, "continuity": 0.0}
    for im in range(mdl.M + 1):
        for ik in range(mdl.NK):
            m, beta = float(im), mdl.sp.beta[ik]

            def L(q):
                return D2 + D1 / r[:, None] - np.diag(q * q / r ** 2) - beta ** 2 * I

            ur, ut, uz = X[0][:, im, ik], X[1][:, im, ik], X[2][:, im, ik]
            up, um, pp = ur + 1j * ut, ur - 1j * ut, P[:, im, ik]
            Rp, Rm, Rz = R[0][:, im, ik], R[1][:, im, ik], R[2][:, im, ik]
            worst["T"] = max(worst["T"], berr(I / dt - CN * mdl.kappa_T * L(m), X[3][:, im, ik],
                                              R[3][:, im, ik]))
            if (im, ik) == (0, 0):
                worst["momentum"] = max(worst["momentum"],
                                        berr(I / dt - CN * L(1.0), ut, (Rp - Rm) / 2j),
                                        berr(I / dt - CN * L(0.0), uz, Rz))
                continue
            gp = D1 @ pp
            worst["momentum"] = max(worst["momentum"],
                                    berr(I / dt - CN * L(m + 1), up, Rp - (gp - m * pp / r)),
                                    berr(I / dt - CN * L(m - 1), um, Rm - (gp + m * pp / r)),
                                    berr(I / dt - CN * L(m), uz, Rz - 1j * beta * pp))
            Rrr, Rtt = (Rp + Rm) / 2, (Rp - Rm) / 2j
            divR = (D1 @ (r * Rrr)) / r + 1j * m * Rtt / r + 1j * beta * Rz
            worst["poisson"] = max(worst["poisson"], berr(L(m), pp, divR))
            div = (D1 @ (r * ur)) / r + 1j * m * ut / r + 1j * beta * uz
            den = ((np.abs(D1) @ np.abs(r * ur)) / r + abs(m) * np.abs(ut) / r
                   + abs(beta) * np.abs(uz))
            worst["continuity"] = max(worst["continuity"], float(abs(div[0]) / den[0]),
                                      float(abs(div[-1]) / den[-1]))
    return worst


@pytest.mark.parametrize("Nr", [512, 1024])
def test_stage_solve_largest_radial_sizes(tc, Nr):
    """The largest radial grids: the Chebyshev-Gauss-Lobatto points cluster at
    the walls (smallest spacing about 1e-6 of the gap at Nr = 1024, second
    derivative weights near 1e12), so two correct FP64 solvers differ by the
    operators' condition number times the rounding in the forward sense (here
    up to ~1e-8).  The GPU solution is checked in the backward sense instead:
    it satisfies every stage equation (momentum, Poisson and temperature rows
    inside, continuity at both walls) with a componentwise backward error
    within 10x of the oracle's pivoted dense solution, measured the same way.
    The forward difference is bounded loosely as a sanity check."""
    wl = Workload("bigr", Nr=Nr, Ntheta=8, Nz=8, eta=0.62, Lz=1.7, Re_i=60.0, Re_o=-15.0,
                  Ra=300.0, Pr=0.8)
    mdl = Model(wl)
    Rr, Rt = random_state(200 + Nr, 2, Nr, mdl.M, mdl.K)
    R = np.stack([Rr + 1j * Rt, Rr - 1j * Rt]
                 + list(random_state(300 + Nr, 2, Nr, mdl.M, mdl.K)))
    dt = 2.5e-3
    run = tc.Run.from_workload(wl)
    xo = dev(np.zeros_like(R))
    po = dev(np.zeros(R.shape[1:], dtype=np.complex128))
    tc.tc_stage_solve(run.ctx, dev(R), dt, xo, po)
    run.close()
    X, P = xo.cpu().numpy(), po.cpu().numpy()
    Xref, Pref = mdl.stage_solve(list(R), dt)
    gpu = _stage_backward_errors(mdl, R, dt, X, P)
    ref = _stage_backward_errors(mdl, R, dt, Xref, Pref)
    fwd = max(float(np.abs(X[f] - Xref[f]).max() / np.abs(Xref[f]).max()) for f in range(mdl.nf))
    print(f"Nr={Nr} backward errors GPU {gpu} oracle {ref}, forward difference {fwd:.2e}")
    for k in gpu:
        assert gpu[k] <= 10.0 * max(ref[k], 1e-14), (k, gpu[k], ref[k])
    assert fwd < 1e-7


def test_initial_perturbation_matches_oracle(tc):
    wl = WORKLOADS["tc_fp64T_nr64_n128"].scaled(Nr=24, Ntheta=32, Nz=48, mp=5, kp=6)
    mdl = Model(wl)
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    tco = temperature_coefficients(wl.seed, wl.mp, wl.kp)
    ref = mdl.initial_state(psi, tco)
    run = tc.Run.from_workload(wl)
    base = run.get_state()            # the library's own discrete basic state
    run.init_perturbation(psi, wl.amp, tco, wl.amp_T)
    got = run.get_state()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    pert = got - base
    pref = ref - mdl.base
    assert np.abs(pert - pref).max() <= 1e-12 * np.abs(pref).max()
    run.close()


def test_basic_state_preserved(tc):
    wl = WORKLOADS["tc_fp64_nr32_n32"]
    mdl = Model(wl)
    run = tc.Run.from_workload(wl)
    X0 = run.get_state()
    assert np.abs(X0 - mdl.base).max() <= 1e-13 * np.abs(mdl.base).max()
    run.step(100, wl.dt)
    X = run.get_state()
    assert np.abs(X - X0).max() <= 1e-12 * np.abs(X0).max()
    run.close()


_ORACLE_RUNS = {}


def _run_both(tc, wl, nsteps, transform="naive", tuned=False):
    """The CUDA run and the oracle's run of the same seeded case.  tuned: the
    launch configuration the benchmark times (tc_autotune after the initial
    state: tiles and the azimuthal path).  The oracle's run is kept for the
    next call with the same case."""
    mdl = Model(wl, transform)
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    tco = temperature_coefficients(wl.seed, wl.mp, wl.kp) if wl.Ra else None
    run = tc.Run.from_workload(wl)
    run.init_perturbation(psi, wl.amp, tco, wl.amp_T)
    if tuned:
        tc.tc_autotune(run.ctx)
        info = tc.tc_get_info(run.ctx)
        print(f"{wl.name}: tuned tiles {info.tile_mb, info.tile_lb, info.tile_mbf}, "
              f"tensor_theta {info.tensor_theta}, tensor_z {info.tensor_z}")
    dts = run.step(nsteps, wl.dt)
    got = run.get_state()
    dg = run.diagnostics()
    pg = run.get_pressure()
    run.close()
    key = (repr(wl), nsteps, transform)
    if key not in _ORACLE_RUNS:
        X = mdl.initial_state(psi, tco)
        ref_dts = []
        dt_prev = 0.0
        p = None
        rate = 0.0
        for _ in range(nsteps):
            X, p, used, rate = mdl.step(X, wl.dt, dt_prev)
            ref_dts.append(used)
            dt_prev = used
        _ORACLE_RUNS[key] = (X, np.array(ref_dts), mdl.diagnostics(X, ref_dts[-1], rate), p)
    X, rdts, dr, p = _ORACLE_RUNS[key]
    return mdl, got, X, dts, rdts, dg, dr, pg, p


def test_step_parity_100_steps(tc):
    wl = WORKLOADS["tc_fp64_nr32_n32"]
    mdl, got, ref, dts, rdts, dg, dr, pg, pr = _run_both(tc, wl, 100, "fft")
    err = rel_l2(mdl, got, ref)
    assert err <= 1e-10, err
    # perturbation part (informational bound): the O(Re) basic state carries
    # round-off of ~1e-13 Re, magnified by Re/amp relative to the perturbation
    pert = rel_l2(mdl, got - mdl.base, ref - mdl.base)
    assert pert <= 1e-6, pert
    np.testing.assert_array_equal(dts, rdts)
    sel = np.ones(pr.shape, bool)
    sel[:, 0, 0] = False
    assert np.abs(pg - pr)[sel].max() <= 1e-9 * np.abs(pr[sel]).max()
    for k in ("E", "E_pert", "torque_i", "torque_o", "P_wall", "eps"):
        assert abs(dg[k] - dr[k]) <= 1e-9 * abs(dr[k]) + 1e-300, (k, dg[k], dr[k])
    # the divergence is a cancellation of O(Re_i) gradients: bound it on that scale
    for k in ("div_rms", "div_max"):
        assert abs(dg[k] - dr[k]) <= 1e-13 * wl.Re_i, (k, dg[k], dr[k])


def test_step_parity_temperature_dynamic_dt(tc):
    wl = WORKLOADS["tc_fp64T_nr64_n128"].scaled(Nr=24, Ntheta=24, Nz=36, mp=4, kp=4)
    mdl, got, ref, dts, rdts, dg, dr, _, _ = _run_both(tc, wl, 30, "fft")
    assert np.all(np.abs(dts - rdts) <= 1e-8 * rdts)
    err = rel_l2(mdl, got, ref)
    assert err <= 1e-10, err
    for k in ("E", "E_pert", "eps", "buoy_work", "Nu_i", "Nu_o", "P_wall", "cfl"):
        assert abs(dg[k] - dr[k]) <= 1e-9 * abs(dr[k]) + 1e-300, (k, dg[k], dr[k])


@pytest.mark.parametrize("Nr,Nt,Nz", [(17, 30, 20), (40, 48, 24), (9, 16, 60)])
def test_step_parity_ragged_sizes(tc, Nr, Nt, Nz):
    wl = Workload("rag", Nr=Nr, Ntheta=Nt, Nz=Nz, eta=0.71, Lz=2.3, Re_i=150.0, Re_o=-40.0,
                  amp=5e-2, mp=min(3, (Nt - 1) // 3), kp=min(3, (Nz - 1) // 3), seed=5,
                  dt=1e-3)
    mdl, got, ref, *_ = _run_both(tc, wl, 20, "fft")
    assert rel_l2(mdl, got, ref) <= 1e-10


def test_bench_workload_parity(tc):
    """The benchmarked configuration itself (64 x 128 x 128, temperature, CFL
    step), a few steps against the oracle."""
    wl = WORKLOADS["tc_fp64T_nr64_n128"]
    mdl, got, ref, dts, rdts, dg, dr, _, _ = _run_both(tc, wl, 2, "fft")
    assert np.all(np.abs(dts - rdts) <= 1e-8 * rdts)
    assert rel_l2(mdl, got, ref) <= 1e-10
    assert rel_l2(mdl, got - mdl.base, ref - mdl.base) <= 1e-6


# Whole runs of the configured workloads at their own sizes, element by
# element against the oracle in the weighted relative L2 of each field
# (c_m w_j r_j weights), gate 1e-10:
#   64 x 128 x 128 with temperature and the dynamic CFL step, 200 steps (the
#     two step sequences compared separately to 1e-8);
#   64^3, eta = 0.5, Re_i = 120, dt = 2e-4, 100 steps (the forward run of the
#     differentiation workload);
#   the 256 x 512^2 mixed workload's physics (eta = 0.875, Re_i = 1e4,
#     amplitude 0.1, modes up to 16, dt = 2e-6) shrunk to 64 x 128^2 and run
#     in FP64 for 50 steps.
# The benchmark's workload runs twice against the same oracle run: with the
# default launch configuration (FFT azimuthal stage) and with the one the
# benchmark times (tc_autotune: tiles, and the tensor-core azimuthal stage
# where it is the faster).
FULL_RUNS = [
    ("tc_fp64T_nr64_n128", {}, 200, False),
    ("tc_fp64T_nr64_n128", {}, 200, True),
    ("tc_adjoint_nr64_n64", {}, 100, False),
    ("tc_mixed_nr256_n512", dict(Nr=64, Ntheta=128, Nz=128, precision=0), 50, False),
]


@pytest.mark.parametrize("name,shrink,nsteps,tuned", FULL_RUNS,
                         ids=["fp64T_64x128x128_200", "fp64T_64x128x128_200_tuned",
                              "adjoint_fwd_64cubed_100", "eta0875_Re1e4_64x128x128_fp64_50"])
def test_workload_full_run_parity(tc, name, shrink, nsteps, tuned):
    wl = WORKLOADS[name].scaled(**shrink)
    mdl, got, ref, dts, rdts, dg, dr, _, _ = _run_both(tc, wl, nsteps, "fft", tuned)
    per_field = []
    w = (mdl.g.w * mdl.g.r)[:, None, None] * mdl.sp.cm[None, :, None]
    for f in range(got.shape[0]):
        per_field.append(float(np.sqrt(np.sum(w * np.abs(got[f] - ref[f]) ** 2)
                                       / np.sum(w * np.abs(ref[f]) ** 2))))
    pert = rel_l2(mdl, got - mdl.base, ref - mdl.base)
    print(f"{name} {shrink} {nsteps} steps: rel L2 per field {per_field}, "
          f"perturbation {pert:.2e}, dt range {rdts.min():.4e}..{rdts.max():.4e}")
    assert np.all(np.abs(dts - rdts) <= 1e-8 * rdts)
    assert max(per_field) <= 1e-10, per_field
    for k in ("E", "E_pert", "eps"):
        assert abs(dg[k] - dr[k]) <= 1e-9 * abs(dr[k]) + 1e-300, (k, dg[k], dr[k])
    # the wall power is a wall derivative of the O(Re) mean flow: the 9-point
    # one-sided stencil at the first Chebyshev node amplifies a relative state
    # difference by kappa = (|D1| |u| + |u|/r) / |D1 u - u/r| (about 1e4 at
    # eta = 0.875, Re_i = 1e4); gate it at that conditioning times the field
    # difference
    kappa = _wall_shear_condition(mdl, ref)
    tol = max(1e-9, 10.0 * kappa * max(per_field))
    assert abs(dg["P_wall"] - dr["P_wall"]) <= tol * abs(dr["P_wall"]), (dg["P_wall"], dr["P_wall"],
                                                                        kappa)


def _wall_shear_condition(mdl, X):
    """Relative condition number of the wall shear d u_theta/dr - u_theta/r of
    the (0,0) mode with respect to the nodal values (worst wall)."""
    g = mdl.g
    u = X[1][:, 0, 0].real
    worst = 1.0
    for w in (0, -1):
        row = g.D1[w]
        sig = row @ u - u[w] / g.r[w]
        worst = max(worst, float((np.abs(row) @ np.abs(u) + abs(u[w]) / g.r[w]) / abs(sig)))
    return worst


def test_set_state_validation(tc):
    wl = WORKLOADS["tc_fp64_nr32_n32"]
    run = tc.Run.from_workload(wl)
    X = run.get_state()
    Y = X.copy()
    Y[0, 3, 0, 1] += 1.0          # breaks u(0,-1) = conj u(0,1)
    with pytest.raises(tc.TCError) as e:
        run.set_state(Y)
    assert e.value.name == "TC_ERR_STATE"
    Y = X.copy()
    Y[1, 2, 2, 2] = np.nan
    with pytest.raises(tc.TCError) as e:
        run.set_state(Y)
    assert e.value.name == "TC_ERR_NONFINITE"
    run.set_state(X)                 # the valid state is accepted again
    assert np.array_equal(run.get_state(), X)
    with pytest.raises(tc.TCError):
        run.set_option("bogus", 1.0)
    run.close()


def test_cfl_limit_reports(tc):
    wl = WORKLOADS["tc_fp64_nr32_n32"]
    run = tc.Run.from_workload(wl)
    run.set_option("cfl_limit", 1e-6)
    with pytest.raises(tc.TCError) as e:
        run.step(1, 1e-3)
    assert e.value.name == "TC_ERR_CFL"
    run.close()


def test_sweep_wait_timeout_is_reported(tc):
    """The radial sweeps wait on shared-memory copies with a 1 s bound; with
    the copies never started (test hook) every wait runs out, the kernels
    return, and the step reports TC_ERR_TIMEOUT instead of hanging."""
    wl = Workload("to", Nr=16, Ntheta=12, Nz=12, eta=0.5, Lz=1.0, Re_i=50.0)
    run = tc.Run.from_workload(wl)
    run.set_option("selftest_no_copy", 1)
    with pytest.raises(tc.TCError) as e:
        run.step(1, 1e-3)
    assert e.value.name == "TC_ERR_TIMEOUT"
    run.close()
    # a fresh context on the same device works normally afterwards
    run = tc.Run.from_workload(wl)
    run.step(2, 1e-3)
    assert np.all(np.isfinite(run.get_state()))
    run.close()


def test_non_blocking_stream_gives_identical_results(tc):
    """Every host copy is ordered on the context's stream: a run on a
    non-blocking stream must match a run on the legacy stream bit for bit."""
    import torch
    wl = WORKLOADS["tc_fp64T_nr64_n128"].scaled(Nr=20, Ntheta=24, Nz=24, mp=3, kp=3)
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    tco = temperature_coefficients(wl.seed, wl.mp, wl.kp)
    out = []
    for use_stream in (False, True):
        run = tc.Run.from_workload(wl)
        if use_stream:
            s = torch.cuda.Stream()
            run.set_stream(s.cuda_stream)
        run.init_perturbation(psi, wl.amp, tco, wl.amp_T)
        run.step(5, wl.dt)
        out.append((run.get_state(), run.get_pressure()))
        run.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_nonlinear_identical_for_every_tile(tc):
    """Tiles change only which CTA computes a transform: the nonlinear terms
    are bitwise the same for every (tile_mb, tile_lb, tile_mbf), including
    widths that are not powers of two and a ragged last block."""
    wl = _wl(12, 24, 30, 500.0)
    mdl = Model(wl)
    X = random_state(321, mdl.nf, wl.Nr, mdl.M, mdl.K)
    outs = []
    for mb, lb, mbf in [(0, 0, 0), (1, 1, 1), (3, 2, 5), (2, 3, 1), (5, 4, 3), (8, 8, 8)]:
        run = tc.Run.from_workload(wl)
        tc.tc_set_option(run.ctx, "tile_mb", mb)
        tc.tc_set_option(run.ctx, "tile_lb", lb)
        tc.tc_set_option(run.ctx, "tile_mbf", mbf)
        info = tc.tc_get_info(run.ctx)
        if mbf:
            assert info.tile_mbf == min(mbf, mdl.M + 1)
        out = dev(np.zeros_like(X))
        tc.tc_nonlinear(run.ctx, dev(X), out)
        outs.append(out.cpu().numpy())
        run.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_fp64_rate_probe(tc):
    """The FP64 FMA rate the roofline quotes: positive, and not above the
    nominal 4 flop/clk/SM of 152 SMs at the 2.07 GHz maximum clock (a probe
    that read above it would not be doing the work)."""
    r = tc.tc_measure_fp64_rate(50.0)
    assert 0.2 < r <= 152 * 2.07e9 * 4 / 1e12


def test_zero_and_negative_step_counts(tc):
    """tc_step with no steps is a no-op that leaves the state bit for bit;
    a negative count is an argument error that changes nothing."""
    wl = WORKLOADS["tc_fp64_nr32_n32"].scaled(Nr=12, Ntheta=12, Nz=12, mp=2, kp=2)
    run = tc.Run.from_workload(wl)
    run.init_perturbation(psi_coefficients(wl.seed, wl.mp, wl.kp), wl.amp)
    before = run.get_state()
    assert len(run.step(0, wl.dt)) == 0
    assert np.array_equal(run.get_state(), before)
    with pytest.raises(tc.TCError) as e:
        run.step(-1, wl.dt)
    assert e.value.name == "TC_ERR_ARG"
    assert np.array_equal(run.get_state(), before)
    run.step(1, wl.dt)                      # the context is still usable
    assert not np.array_equal(run.get_state(), before)
    run.close()


def test_create_size_limits(tc):
    """The azimuthal size limit that the shared-memory transforms impose."""
    st = {v: k for k, v in tc.STATUS.items()}

    def create(Nt, Ra):
        h = tc.ctypes.c_void_p()
        code = tc._lib.tc_create(9, Nt, 8, 0.5, 1.0, 10.0, 0.0, Ra, 1.0, tc.ctypes.byref(h))
        if code == 0:
            tc._lib.tc_destroy(h)
        return code

    assert create(1000, 0.0) == 0
    assert create(750, 100.0) == 0
    assert create(1024, 0.0) == st["TC_ERR_UNSUPPORTED"]
    assert create(768, 100.0) == st["TC_ERR_UNSUPPORTED"]
    assert create(1030, 0.0) == st["TC_ERR_ARG"]          # not 2^a 3^b 5^c / above 1024


@pytest.mark.parametrize("Nr,Nt,Nz,Ra", [(9, 750, 8, 400.0),     # largest azimuthal size with T
                                         (11, 1000, 6, 0.0),      # largest without T
                                         (9, 512, 16, 0.0),       # plan 8 x 8 x 8 in theta
                                         (9, 256, 16, 300.0),     # plan 8 x 8 x 4 in theta
                                         (10, 16, 256, 0.0),      # plan 8 x 8 x 4 in z
                                         (9, 8, 1024, 300.0),     # largest axial size
                                         (9, 4, 4, 300.0)])       # smallest: M = K = 1
def test_nonlinear_extreme_sizes(tc, Nr, Nt, Nz, Ra):
    wl = _wl(Nr, Nt, Nz, Ra)
    mdl = Model(wl, "fft")
    X = random_state(200 + Nt, mdl.nf, Nr, mdl.M, mdl.K)
    ref, rate = mdl.nonlinear(X)
    run = tc.Run.from_workload(wl)
    out = dev(np.zeros_like(X))
    got_rate = tc.tc_nonlinear(run.ctx, dev(X), out)
    run.close()
    got = out.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert abs(got_rate - rate) <= 1e-13 * rate


def test_step_parity_smallest_grid(tc):
    """Nr = 9 (one stencil spans the gap), Ntheta = Nz = 4 (M = K = 1), with T."""
    wl = Workload("tiny", Nr=9, Ntheta=4, Nz=4, eta=0.5, Lz=2.0, Re_i=40.0, Ra=200.0, Pr=1.0,
                  amp=1e-2, mp=1, kp=1, amp_T=1e-2, seed=9, dt=1e-3)
    mdl, got, ref, *_ = _run_both(tc, wl, 30, "fft")
    assert rel_l2(mdl, got, ref) <= 1e-10


def test_quiescent_state_stays_at_rest(tc):
    """Re_i = Re_o = 0, no heating: the basic state is zero and stays exactly zero."""
    wl = Workload("rest", Nr=12, Ntheta=12, Nz=12, eta=0.5, Lz=2.0, Re_i=0.0)
    run = tc.Run.from_workload(wl)
    run.step(10, 1e-3)
    X = run.get_state()
    d = run.diagnostics()
    run.close()
    assert np.abs(X).max() == 0.0
    assert d["E"] == 0.0 and d["corr_diff"] == 0.0


def test_rhs_from_stage_equation_matches_stencil(tc):
    """After a corrector, the explicit part takes L X from that stage's
    equation; with the state re-entered before every step (which forgets the
    stage) it takes the 9-point stencil.  Both runs must agree to round-off,
    and both stay on the oracle."""
    # fixed dt near the CFL step of this flow (its dynamic step is about 5e-5)
    wl = WORKLOADS["tc_fp64T_nr64_n128"].scaled(Nr=24, Ntheta=24, Nz=30, mp=4, kp=4, dt=5e-5)
    psi = psi_coefficients(wl.seed, wl.mp, wl.kp)
    tco = temperature_coefficients(wl.seed, wl.mp, wl.kp)
    a = tc.Run.from_workload(wl)
    a.init_perturbation(psi, wl.amp, tco, wl.amp_T)
    a.step(20, wl.dt)
    Xa = a.get_state()
    a.close()
    b = tc.Run.from_workload(wl)
    b.init_perturbation(psi, wl.amp, tco, wl.amp_T)
    for _ in range(20):
        b.step(1, wl.dt)
        b.set_state(b.get_state())
    Xb = b.get_state()
    b.close()
    mdl = Model(wl, "fft")
    # the two forms of L X differ by round-off of the stage solve divided by
    # c dt: ~1e-16 |X| / dt per step, against a perturbation ~1e-5 of |X|
    assert rel_l2(mdl, Xa, Xb) <= 1e-11
    assert rel_l2(mdl, Xa - mdl.base, Xb - mdl.base) <= 1e-9
    X = mdl.initial_state(psi, tco)
    X, _ = mdl.run(X, 20, wl.dt)
    assert rel_l2(mdl, Xa, X) <= 1e-10
