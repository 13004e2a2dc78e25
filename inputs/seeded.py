"""Seeded random draws and the workload definitions.

The initial perturbation of every run is u' = curl(psi) with psi a vector
potential whose Fourier coefficients are drawn here (Sec. 2.1: divergence-free
initial conditions exciting selected Fourier modes).  Only the raw normal draws
are produced; building psi's radial profile, the curl, the Hermitian fix-up of
the m = 0 column and the amplitude scaling are the method's arithmetic and are
done separately by each consumer.

Draw order (NumPy ``Generator(PCG64(seed))``, one ``standard_normal`` call per
array, C order): component (r, theta, z) -> m ascending (0..mp) -> k ascending
(-kp..kp) -> (re, im).  The temperature draws, when present, come next from the
same stream: m ascending -> k ascending -> (re, im).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np


@dataclass(frozen=True)
class Workload:
    """Physical and numerical parameters of one Taylor-Couette run.

    Lengths are in units of the gap d, times in d^2/nu, velocities in nu/d.
    ``Ntheta`` and ``Nz`` are the physical (3/2-padded) grid sizes.
    """

    name: str
    Nr: int
    Ntheta: int
    Nz: int
    eta: float
    Lz: float
    Re_i: float
    Re_o: float = 0.0
    Ra: float = 0.0
    Pr: float = 1.0
    amp: float = 1e-3      # max over the grid of |u'|
    mp: int = 4            # excited azimuthal modes 0..mp
    kp: int = 4            # excited axial modes -kp..kp
    amp_T: float = 0.0     # max over the grid of |T'| (0: no T')
    seed: int = 1
    steps: int = 100
    dt: float = 1e-3       # > 0 fixed step, <= 0 dynamic CFL step
    dt_max: float = 1e-3
    cfl: float = 0.25
    precision: int = 0     # 0: FP64 throughout; 1: FP32 transforms of u' (mixed)

    @property
    def points(self) -> int:
        return self.Nr * self.Ntheta * self.Nz

    def scaled(self, **kw) -> "Workload":
        return replace(self, **kw)


WORKLOADS = {
    # Plain FP64 run, outer cylinder at rest.
    "tc_fp64_nr32_n32": Workload(
        "tc_fp64_nr32_n32", Nr=32, Ntheta=32, Nz=32, eta=0.5,
        Lz=2 * math.pi / 3.16, Re_i=100.0, amp=1e-3, mp=4, kp=4, seed=1,
        steps=100, dt=1e-3),
    # FP64 with Boussinesq temperature and dynamic CFL time step.
    "tc_fp64T_nr64_n128": Workload(
        "tc_fp64T_nr64_n128", Nr=64, Ntheta=128, Nz=128, eta=0.71,
        Lz=2 * math.pi, Re_i=3000.0, Re_o=-1000.0, Ra=1e4, Pr=0.7,
        amp=1e-2, mp=8, kp=8, amp_T=1e-2, seed=2, steps=200, dt=0.0,
        dt_max=1e-3, cfl=0.25),
    # Mixed precision, ~67 M grid points.
    "tc_mixed_nr256_n512": Workload(
        "tc_mixed_nr256_n512", Nr=256, Ntheta=512, Nz=512, eta=0.875,
        Lz=2 * math.pi / 3.16, Re_i=1e4, amp=0.1, mp=16, kp=16, seed=3,
        steps=50, dt=2e-6, precision=1),
    # Discrete adjoint.  dt = 2e-4 keeps the advective CFL number at the inner
    # wall near 0.25 (at 1e-3 it is 1.22 and the explicit predictor-corrector
    # amplifies round-off in the highest azimuthal modes).
    "tc_adjoint_nr64_n64": Workload(
        "tc_adjoint_nr64_n64", Nr=64, Ntheta=64, Nz=64, eta=0.5,
        Lz=2 * math.pi / 3.16, Re_i=120.0, amp=1e-3, mp=4, kp=4, seed=4,
        steps=200, dt=2e-4),
}


def psi_coefficients(seed: int, mp: int, kp: int) -> np.ndarray:
    """Raw vector-potential draws, complex128 of shape (3, mp+1, 2*kp+1).

    Axis 2 is in natural order k = -kp..kp.  The Hermitian constraint of the
    m = 0 column is NOT applied here.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((3, mp + 1, 2 * kp + 1, 2))
    return d[..., 0] + 1j * d[..., 1]


def temperature_coefficients(seed: int, mp: int, kp: int) -> np.ndarray:
    """Raw temperature draws, complex128 (mp+1, 2*kp+1), natural k order.

    They follow the psi draws in the same stream.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    rng.standard_normal((3, mp + 1, 2 * kp + 1, 2))
    d = rng.standard_normal((mp + 1, 2 * kp + 1, 2))
    return d[..., 0] + 1j * d[..., 1]


def ensemble_members(n: int = 64, seed: int = 5000) -> list:
    """Uneven-size ensemble: n independent runs with drawn sizes and Re_i.

    Member i uses seed ``seed + i`` for its own perturbation draws.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nrs = rng.choice([32, 48, 64], size=n)
    ns = rng.choice([32, 64, 96], size=n)
    etas = rng.choice([0.5, 0.71, 0.875], size=n)
    res = rng.uniform(80.0, 400.0, size=n)
    out = []
    for i in range(n):
        out.append(Workload(
            f"ens{i}", Nr=int(nrs[i]), Ntheta=int(ns[i]), Nz=int(ns[i]),
            eta=float(etas[i]), Lz=2 * math.pi / 3.16, Re_i=float(res[i]),
            amp=1e-3, mp=4, kp=4, seed=seed + i, steps=100, dt=1e-3))
    return out


def random_state(seed: int, nf: int, Nr: int, M: int, K: int, scale=1.0) -> np.ndarray:
    """Random spectral coefficients of real fields, complex128 (nf, Nr, M+1, 2K+1).

    Axis 3 is in FFT order (0..K, -K..-1).  Entries are N(0,1) draws in C
    order (re, im) times ``scale`` (scalar or per-field sequence); the m = 0
    column is then given the structure every real field has, u(0,-k) =
    conj(u(0,k)) with a real (0,0) entry, so the array is a valid input.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((nf, Nr, M + 1, 2 * K + 1, 2))
    a = d[..., 0] + 1j * d[..., 1]
    a *= np.asarray(scale, dtype=np.float64).reshape(-1, 1, 1, 1) if np.ndim(scale) else scale
    for k in range(1, K + 1):
        a[:, :, 0, 2 * K + 1 - k] = np.conj(a[:, :, 0, k])
    a[:, :, 0, 0] = a[:, :, 0, 0].real
    return a
