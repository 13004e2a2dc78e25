"""Illustrative heated example (Sec. 4), run through the library's public API.

A hot inner cylinder rotating at Re_i = 50 inside a cooled stationary outer
cylinder.  Three runs at increasing Rayleigh number, Ra = 2130, 2840, 3550,
each started from the final state of the one before (the first from the
basic state plus a small single-harmonic disturbance).  Recorded over time:
the Nusselt number at the inner wall, Nu_i (heat flux over that of the
conductive basic state, so 1 while the heat transfer is purely conductive),
and u_theta at a mid-gap probe.

Sec. 4 gives Re_i and the Ra sequence but not eta, Pr, the axial period or the
resolution.  The values used here -- eta = 0.5, Pr = 0.7, Lz = pi (axial
wavenumber 2), a 32^3 grid, dynamic CFL step capped at 5e-4 -- were chosen so
that the basic state at Ra = 2130 is unstable and the disturbance reaches the
nonlinear regime after about two viscous times, as described there.  It is a
qualitative demonstration, not a reproduction of the paper's figure.

    python -m paper_1908_00587_gb300.heated_example [--t-stage 4.0] [--csv out.csv]
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np

from . import tc

RE_I = 50.0
RAS = (2130.0, 2840.0, 3550.0)
ETA, PR, LZ = 0.5, 0.7, math.pi
GRID = (32, 32, 32)


def probe_u_theta(X: np.ndarray, j: int) -> float:
    """u_theta at (r_j, theta = 0, z = 0): sum over modes of c_m Re(u_theta(m, k))."""
    col = X[1, j]
    return float(np.real(col[0]).sum() + 2.0 * np.real(col[1:]).sum())


def single_harmonic_psi(m: int = 3, k: int = -1) -> np.ndarray:
    """Vector-potential draws with one nonzero entry: psi_r of mode (m, k).

    (3, -1) is the spiral mode that grows fastest at these parameters (found
    by starting from random draws over m <= 3, |k| <= 3 and following the
    modal energies)."""
    kp = abs(k)
    psi = np.zeros((3, m + 1, 2 * kp + 1), dtype=np.complex128)
    psi[0, m, kp + k] = 1.0
    return psi


def run(t_stage: float = 4.0, record_every: float = 0.05, amp: float = 1e-3,
        ras=RAS, grid=GRID, dt_max: float = 5e-4, verbose: bool = True):
    """Returns a list of (Ra, t, Nu_i, u_theta_probe) rows."""
    Nr, Nt, Nz = grid
    rows = []
    X = None
    j_mid = Nr // 2
    steps_total, t0 = 0, time.time()
    for Ra in ras:
        r = tc.Run(Nr, Nt, Nz, ETA, LZ, RE_I, 0.0, Ra, PR)
        r.set_option("dt_max", dt_max)
        if X is None:
            r.init_perturbation(single_harmonic_psi(), amp)
        else:
            r.set_state(X)
        t = 0.0
        while True:
            d = r.diagnostics()
            X = r.get_state()
            rows.append((Ra, d["t"], d["Nu_i"], probe_u_theta(X, j_mid)))
            if d["t"] >= t_stage - 1e-12:
                break
            # steps until the next record time (dynamic dt: count from dt_max)
            n = max(1, int(round(record_every / dt_max)))
            r.step(n, 0.0)
            steps_total += n
        r.close()
        if verbose:
            nu = [x[2] for x in rows if x[0] == Ra]
            print(f"Ra={Ra:7.1f}: Nu_i {nu[0]:.6f} -> {nu[-1]:.6f} (max {max(nu):.6f})",
                  flush=True)
    if verbose:
        el = time.time() - t0
        pts = Nr * Nt * Nz
        print(f"{steps_total} steps of {Nr}x{Nt}x{Nz} in {el:.1f} s "
              f"({steps_total * pts / el:.3g} grid-point-steps/s incl. host I/O)", flush=True)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--t-stage", type=float, default=4.0, help="viscous times per Ra")
    ap.add_argument("--csv", default=None, help="write Ra,t,Nu_i,u_theta_probe rows here")
    a = ap.parse_args(argv)
    rows = run(a.t_stage)
    if a.csv:
        with open(a.csv, "w") as f:
            f.write("Ra,t,Nu_i,u_theta_probe\n")
            for row in rows:
                f.write(",".join(f"{v:.10g}" for v in row) + "\n")


if __name__ == "__main__":
    main()
