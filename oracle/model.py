"""The discrete Taylor-Couette time step, written out plainly (oracle).

Test infrastructure only (see the package docstring).  Sections cited are those
of the nsCouette paper (arXiv:1908.00587).

Equations (viscous units: length d = r_o - r_i, time d^2/nu, velocity nu/d):
    du/dt + u.grad u = -grad p + lap u + Gr T e_z,   div u = 0,
    dT/dt + u.grad T = (1/Pr) lap T,                 Gr = Ra / Pr,
with u_theta(r_i) = Re_i, u_theta(r_o) = Re_o, T(r_i) = +1/2, T(r_o) = -1/2
(Sec. 2.1: differentially heated, independently rotating cylinders; a negative
radial temperature gradient and gravity along z, Boussinesq-like buoyancy).
Temperature is carried only when Ra != 0.

Options of the scheme (all off by default):
* ``n_corr`` corrector passes (default 1), each c N(X_prev) + (1-c) N^n with
  the same explicit part; the last difference max |X_corr - X_prev| over the
  stored coefficients is kept as ``last_corr_diff``;
* ``flux_constraint``: a uniform axial pressure gradient G in the (0,0) u_z
  equation, solved with the stage so that the axial volume flux
  int u_z r dr (Clenshaw-Curtis quadrature) is zero after every stage;
* ``eps_c`` (centrifugal buoyancy, Sec. 2.1 cites a Boussinesq-like
  approximation for rotating flows and leaves other buoyancy set-ups open):
  the advective acceleration of the momentum equation is weighted by the
  density factor (1 - eps_c T), so N_u = -(1 - eps_c T)(u.grad u + curvature
  terms) + Gr T e_z.  The temperature equation is unchanged.

Readings of the scheme (the paper defers its details to other papers):
* nonlinear term in convective form with the cylindrical curvature terms,
    N_r = -(u.grad u_r - u_theta^2/r),  N_theta = -(u.grad u_theta + u_r u_theta/r),
    N_z = -u.grad u_z + Gr T,           N_T = -u.grad T,
  u.grad = u_r d/dr + (u_theta/r) d/dtheta + u_z d/dz, formed on the 3/2 grid;
* radial and azimuthal velocities are solved as u+- = u_r +- i u_theta, whose
  viscous operators decouple: L+- = D2 + D1/r - (m+-1)^2/r^2 - beta^2;
  u_z and T use L = D2 + D1/r - m^2/r^2 - beta^2;
* predictor-corrector (Sec. 2.1): Crank-Nicolson weight c = 1/2 on the
  viscous/diffusive terms, pressure implicit, Euler predictor with N^n, then
  one corrector with c N(X*) + (1-c) N^n;
* pressure by an influence-matrix method: Poisson with homogeneous Neumann
  rows for a particular solution, two homogeneous Poisson solutions with unit
  wall flux, and a 2x2 system per mode so that div u = 0 at both wall nodes;
* mode (m, k) = (0, 0): no pressure solve, u_r = 0, u_theta and u_z solved
  directly with their wall values;
* dynamic time step from a CFL bound on the start-of-step state, with
  hysteresis (see ``dt_policy``).
"""
from __future__ import annotations

import math

import numpy as np
from .grid import Grid, couette_AB
from .spectral import Spectral

CN = 0.5  # implicit weight c of the predictor-corrector


def _dirichlet_rows(A: np.ndarray) -> np.ndarray:
    """Replace first and last rows of a (..., Nr, Nr) batch by identity rows."""
    A[..., 0, :] = 0.0
    A[..., -1, :] = 0.0
    A[..., 0, 0] = 1.0
    A[..., -1, -1] = 1.0
    return A


class _Factored:
    """A batch of real matrices solved by LAPACK gesv (LU, partial pivoting)."""

    def __init__(self, A: np.ndarray):
        self.A = A

    def solve(self, b: np.ndarray) -> np.ndarray:
        """b complex (n, Nr): solve real and imaginary parts together."""
        rhs = np.stack([b.real, b.imag], axis=-1)
        x = np.linalg.solve(self.A, rhs)
        return x[..., 0] + 1j * x[..., 1]


class Model:
    """One run: grid, transforms, operators, base state, step, diagnostics."""

    def __init__(self, wl, transform: str = "naive", n_corr: int = 1,
                 flux_constraint: bool = False, eps_c: float = 0.0):
        if n_corr < 1:
            raise ValueError("n_corr >= 1")
        self.n_corr = int(n_corr)
        self.flux_constraint = bool(flux_constraint)
        self.eps_c = float(eps_c)
        self.last_corr_diff = 0.0
        self.wl = wl
        self.g = Grid(wl.Nr, wl.eta)
        self.sp = Spectral(wl.Ntheta, wl.Nz, wl.Lz, transform)
        self.has_T = wl.Ra != 0.0
        self.Gr = wl.Ra / wl.Pr if self.has_T else 0.0
        self.kappa_T = 1.0 / wl.Pr
        self.nf = 4 if self.has_T else 3
        if self.eps_c != 0.0 and not self.has_T:
            raise ValueError("centrifugal buoyancy needs the temperature (Ra != 0)")
        self.M, self.K = self.sp.M, self.sp.K
        self.NK = 2 * self.K + 1
        mm, kk = np.meshgrid(self.sp.m, self.sp.kk, indexing="ij")
        self.mv = mm.ravel().astype(np.float64)          # (nmodes,)
        self.bv = self.sp.alpha * kk.ravel()              # axial wavenumber
        self.nmodes = self.mv.size
        self.sel = np.arange(1, self.nmodes)              # all but (0, 0)
        self._ops_dt = None
        self.base = self.base_state()
        self.Tb_disc = self.base[3].copy() if self.has_T else None

    # ------------------------------------------------------------------ layout
    def cols(self, f: np.ndarray) -> np.ndarray:
        """(Nr, M+1, NK) -> (nmodes, Nr)."""
        return f.reshape(self.wl.Nr, self.nmodes).T

    def uncols(self, c: np.ndarray) -> np.ndarray:
        return c.T.reshape(self.wl.Nr, self.M + 1, self.NK)

    # --------------------------------------------------------------- operators
    def lap(self, q: np.ndarray, beta: np.ndarray) -> np.ndarray:
        """Batch of D2 + D1/r - q^2/r^2 - beta^2 (nmodes, Nr, Nr)."""
        g = self.g
        base = g.D2 + g.D1 / g.r[:, None]
        A = np.broadcast_to(base, (q.size,) + base.shape).copy()
        idx = np.arange(g.Nr)
        A[:, idx, idx] -= q[:, None] ** 2 / g.r[None, :] ** 2 + beta[:, None] ** 2
        return A

    def apply_lap(self, f: np.ndarray, q: np.ndarray) -> np.ndarray:
        """L(q) f for f (Nr, M+1, NK) spectral, q broadcastable to (M+1, 1)."""
        g = self.g
        r = g.r[:, None, None]
        beta = self.sp.beta[None, None, :]
        return g.drr(f) + g.dr(f) / r - (q ** 2 / r ** 2 + beta ** 2) * f

    def poisson_matrix(self, m, beta):
        """Pressure operator: L(m) inside, D1 (Neumann) rows at both walls."""
        P = self.lap(m, beta)
        P[:, 0, :] = self.g.D1[0]
        P[:, -1, :] = self.g.D1[-1]
        return P

    def helmholtz_matrix(self, q, beta, dt, kappa):
        """I/dt - c kappa L(q) inside, Dirichlet rows at both walls."""
        H = -CN * kappa * self.lap(q, beta)
        idx = np.arange(self.g.Nr)
        H[:, idx, idx] += 1.0 / dt
        return _dirichlet_rows(H)

    def div_cols(self, up, um, uz, m, beta):
        """Discrete divergence of a field given in +- form, per mode column.

        div u = (1/r) D1(r u_r) + (i m / r) u_theta + i beta u_z,
        u_r = (u+ + u-)/2, u_theta = (u+ - u-)/(2i).  Arrays (n, Nr).
        """
        r = self.g.r[None, :]
        ur = 0.5 * (up + um)
        ut = (up - um) / 2j
        return ((r * ur) @ self.g.D1.T) / r + 1j * m[:, None] * ut / r \
            + 1j * beta[:, None] * uz

    # --------------------------------------------------- per-dt factorisations
    def operators(self, dt: float):
        """Factor every radial operator and build the influence matrices."""
        if self._ops_dt == dt:
            return self._ops
        s = self.sel
        m, b = self.mv[s], self.bv[s]
        ops = {}
        ops["P"] = _Factored(self.poisson_matrix(m, b))
        ops["Hp"] = _Factored(self.helmholtz_matrix(m + 1, b, dt, 1.0))
        ops["Hm"] = _Factored(self.helmholtz_matrix(m - 1, b, dt, 1.0))
        ops["Hz"] = _Factored(self.helmholtz_matrix(m, b, dt, 1.0))
        if self.has_T:
            ops["HT"] = _Factored(self.helmholtz_matrix(m, b, dt, self.kappa_T))
        # (0,0): u_theta uses L(1), u_z and T use L(0)
        z = np.zeros(1)
        ops["H00_t"] = _Factored(self.helmholtz_matrix(z + 1, z, dt, 1.0))
        ops["H00_z"] = _Factored(self.helmholtz_matrix(z, z, dt, 1.0))
        if self.has_T:
            ops["H00_T"] = _Factored(self.helmholtz_matrix(z, z, dt, self.kappa_T))
        # homogeneous solutions: unit Neumann flux at r_i (a) or r_o (b)
        Nr = self.g.Nr
        n = s.size
        homog = []
        for wall in (0, Nr - 1):
            e = np.zeros((n, Nr), dtype=complex)
            e[:, wall] = 1.0
            p = ops["P"].solve(e)
            up, um, uz = self._velocity_solve(ops, -self._grad_pm(p, m, b, +1),
                                              -self._grad_pm(p, m, b, -1),
                                              -1j * b[:, None] * p)
            homog.append((p, up, um, uz))
        divs = [self.div_cols(h[1], h[2], h[3], m, b) for h in homog]
        A = np.empty((n, 2, 2), dtype=complex)
        for j, h in enumerate(divs):
            A[:, 0, j] = h[:, 0]
            A[:, 1, j] = h[:, -1]
        ops["homog"] = homog
        ops["A"] = A
        self._ops, self._ops_dt = ops, dt
        return ops

    def _grad_pm(self, p, m, b, sign):
        """(grad p)_r +- i (grad p)_theta = D1 p -+ (m/r) p, per column."""
        r = self.g.r[None, :]
        return p @ self.g.D1.T - sign * m[:, None] * p / r

    def _velocity_solve(self, ops, fp, fm, fz):
        """Helmholtz solves with homogeneous Dirichlet rows."""
        fp, fm, fz = fp.copy(), fm.copy(), fz.copy()
        for f in (fp, fm, fz):
            f[:, 0] = 0.0
            f[:, -1] = 0.0
        return ops["Hp"].solve(fp), ops["Hm"].solve(fm), ops["Hz"].solve(fz)

    # ------------------------------------------------------------- stage solve
    def stage_solve(self, R, dt: float):
        """Solve (I/dt - c L) X = R - grad p, div X = 0, for every mode.

        R: list of spectral arrays [R+, R-, R_z, (R_T)] (Nr, M+1, NK), the full
        explicit right-hand side evaluated at every radial node.  Returns the
        new primitive state (nf, Nr, M+1, NK) and the pressure (Nr, M+1, NK).
        """
        ops = self.operators(dt)
        s = self.sel
        m, b = self.mv[s], self.bv[s]
        Rp, Rm, Rz = (self.cols(R[i])[s] for i in range(3))
        r = self.g.r[None, :]
        # particular pressure: Poisson of div R, homogeneous Neumann rows
        divR = self.div_cols(Rp, Rm, Rz, m, b)
        divR[:, 0] = 0.0
        divR[:, -1] = 0.0
        p0 = ops["P"].solve(divR)
        up, um, uz = self._velocity_solve(
            ops, Rp - self._grad_pm(p0, m, b, +1), Rm - self._grad_pm(p0, m, b, -1),
            Rz - 1j * b[:, None] * p0)
        # influence-matrix correction: div u = 0 at both wall nodes
        d0 = self.div_cols(up, um, uz, m, b)
        rhs = -np.stack([d0[:, 0], d0[:, -1]], axis=-1)
        alpha = np.linalg.solve(ops["A"], rhs[..., None])[..., 0]
        p = p0.copy()
        for j, (ph, uph, umh, uzh) in enumerate(ops["homog"]):
            a = alpha[:, j:j + 1]
            p = p + a * ph
            up = up + a * uph
            um = um + a * umh
            uz = uz + a * uzh
        Nr = self.g.Nr
        out = np.zeros((self.nf, self.nmodes, Nr), dtype=complex)
        pres = np.zeros((self.nmodes, Nr), dtype=complex)
        out[0, s] = 0.5 * (up + um)
        out[1, s] = (up - um) / 2j
        out[2, s] = uz
        pres[s] = p
        # mode (0,0): u_r = 0; u_theta, u_z (and T) with their wall values
        Rt00 = ((self.cols(R[0])[0] - self.cols(R[1])[0]) / 2j)[None, :]
        Rt00 = Rt00.copy()
        Rt00[:, 0], Rt00[:, -1] = self.wl.Re_i, self.wl.Re_o
        out[1, 0] = ops["H00_t"].solve(Rt00)[0]
        Rz00 = self.cols(R[2])[0][None, :].copy()
        Rz00[:, 0] = Rz00[:, -1] = 0.0
        out[2, 0] = ops["H00_z"].solve(Rz00)[0]
        if self.flux_constraint:
            # uniform forcing G (interior rows) chosen so that the flux is zero
            e = np.ones((1, Nr), dtype=complex)
            e[:, 0] = e[:, -1] = 0.0
            ug = ops["H00_z"].solve(e)[0]
            G = -self.axial_flux(out[2, 0]) / self.axial_flux(ug)
            out[2, 0] = out[2, 0] + G * ug
        if self.has_T:
            RT = self.cols(R[3]).copy()
            RT[:, 0] = RT[:, -1] = 0.0
            out[3, s] = ops["HT"].solve(RT[s])
            RT00 = RT[0][None, :].copy()
            RT00[:, 0], RT00[:, -1] = 0.5, -0.5
            out[3, 0] = ops["H00_T"].solve(RT00)[0]
        X = np.stack([self.uncols(out[i]) for i in range(self.nf)])
        return X, self.uncols(pres)

    # --------------------------------------------------------------- nonlinear
    def physical_fields(self, X):
        """Physical values of each component and its r, theta, z derivatives.

        Returns dict name -> (Nr, Ntheta, Nz) for names c, c_r, c_t, c_z with
        c in (ur, ut, uz[, T]).
        """
        sp, g = self.sp, self.g
        m = sp.m[None, :, None]
        beta = sp.beta[None, None, :]
        names = ["ur", "ut", "uz", "T"][: self.nf]
        out = {}
        for c, nm in enumerate(names):
            xh = X[c]
            out[nm] = sp.to_physical(xh)
            out[nm + "_r"] = sp.to_physical(g.dr(xh))
            out[nm + "_t"] = sp.to_physical(1j * m * xh)
            out[nm + "_z"] = sp.to_physical(1j * beta * xh)
        return out

    def nonlinear(self, X):
        """Dealiased nonlinear terms [N_r, N_theta, N_z, (N_T)] and CFL rate.

        The CFL rate is max over the grid of
        max(|u_r|/dr_j, |u_theta|/(r_j dtheta), |u_z|/dz), dr_j the distance
        from node j to its nearest neighbour.
        """
        f = self.physical_fields(X)
        r = self.g.r[:, None, None]
        ur, ut, uz = f["ur"], f["ut"], f["uz"]

        def adv(c):
            return ur * f[c + "_r"] + (ut / r) * f[c + "_t"] + uz * f[c + "_z"]

        Nph = [-(adv("ur") - ut * ut / r),
               -(adv("ut") + ur * ut / r),
               -adv("uz")]
        if self.eps_c != 0.0:
            rho = 1.0 - self.eps_c * f["T"]
            Nph = [rho * a for a in Nph]
        if self.has_T:
            Nph[2] = Nph[2] + self.Gr * f["T"]
            Nph.append(-adv("T"))
        N = np.stack([self.sp.to_spectral(a) for a in Nph])
        dr = self.g.min_spacing()[:, None, None]
        dth = 2.0 * math.pi / self.wl.Ntheta
        dz = self.wl.Lz / self.wl.Nz
        rate = max(np.max(np.abs(ur) / dr), np.max(np.abs(ut) / (r * dth)),
                   np.max(np.abs(uz) / dz))
        return N, float(rate)

    # ------------------------------------------------------------------- step
    def to_pm(self, X):
        out = [X[0] + 1j * X[1], X[0] - 1j * X[1], X[2]]
        if self.has_T:
            out.append(X[3])
        return out

    def explicit_linear(self, Xpm):
        """L X in +- form: [L+ u+, L- u-, L u_z, (1/Pr) L T]."""
        m = self.sp.m[:, None].astype(np.float64)
        out = [self.apply_lap(Xpm[0], m + 1), self.apply_lap(Xpm[1], m - 1),
               self.apply_lap(Xpm[2], m)]
        if self.has_T:
            out.append(self.kappa_T * self.apply_lap(Xpm[3], m))
        return out

    def dt_policy(self, dt_prev: float, rate: float) -> float:
        """Dynamic step (Sec. 2.1 names dynamic control; the rule is a reading).

        dt* = min(dt_max, C / rate); take dt* at once when it is smaller than
        the current step, and only when it exceeds 1.1 x the current step when
        larger.  The first step takes dt*.
        """
        dt_star = self.wl.dt_max if rate <= 0.0 else min(self.wl.dt_max,
                                                          self.wl.cfl / rate)
        if dt_prev <= 0.0 or dt_star < dt_prev or dt_star > 1.1 * dt_prev:
            return dt_star
        return dt_prev

    def step(self, X, dt: float, dt_prev: float = 0.0):
        """One predictor-corrector step.  dt <= 0 selects the dynamic step.

        Returns (X_new, pressure, dt_used, cfl_rate).
        """
        N0, rate = self.nonlinear(X)
        if dt <= 0.0:
            dt = self.dt_policy(dt_prev, rate)
        Xpm = self.to_pm(X)
        Npm0 = self.to_pm(N0)
        LX = self.explicit_linear(Xpm)
        base = [Xpm[i] / dt + (1.0 - CN) * LX[i] + (1.0 - CN) * Npm0[i]
                for i in range(self.nf)]
        Xc, _ = self.stage_solve([base[i] + CN * Npm0[i] for i in range(self.nf)], dt)
        for _ in range(self.n_corr):
            Xprev = Xc
            N1, _ = self.nonlinear(Xprev)
            Npm1 = self.to_pm(N1)
            Xc, p = self.stage_solve([base[i] + CN * Npm1[i] for i in range(self.nf)], dt)
        self.last_corr_diff = float(max(np.max(np.abs((Xc - Xprev).real)),
                                        np.max(np.abs((Xc - Xprev).imag))))
        return Xc, p, dt, rate

    def run(self, X, nsteps: int, dt: float):
        """nsteps steps; returns (X, list of dt used)."""
        dts = []
        dt_prev = 0.0
        for _ in range(nsteps):
            X, _, used, _ = self.step(X, dt, dt_prev)
            dts.append(used)
            dt_prev = used
        return X, dts

    # ------------------------------------------------------------- base state
    def base_state(self):
        """Discrete steady basic state (Sec. 4: u_theta(r), T(r) analytic).

        Circular Couette u_theta solves L(1) u = 0 with the wall speeds; the
        conductive T solves L(0) T = 0 with T = +-1/2; with buoyancy the steady
        axial flow solves L(0) u_z = -Gr T (no mean axial pressure gradient).
        All with the same discrete D1/D2, so the scheme keeps them exactly.
        """
        Nr = self.g.Nr
        z = np.zeros(1)
        X = np.zeros((self.nf, Nr, self.M + 1, self.NK), dtype=complex)

        def dsolve(q, rhs, lo, hi):
            A = _dirichlet_rows(self.lap(z + q, z))[0]
            b = rhs.copy()
            b[0], b[-1] = lo, hi
            return np.linalg.solve(A, b)

        X[1, :, 0, 0] = dsolve(1.0, np.zeros(Nr), self.wl.Re_i, self.wl.Re_o)
        if self.has_T:
            T = dsolve(0.0, np.zeros(Nr), 0.5, -0.5)
            X[3, :, 0, 0] = T
            uz = dsolve(0.0, -self.Gr * T, 0.0, 0.0)
            if self.flux_constraint:
                # L(0) u_z = -Gr T - G with G such that the axial flux is zero
                ones = dsolve(0.0, -np.ones(Nr), 0.0, 0.0)
                uz = uz - (self.axial_flux(uz) / self.axial_flux(ones)) * ones
            X[2, :, 0, 0] = uz
        return X

    def axial_flux(self, uz_profile) -> float:
        """int u_z r dr over the gap (Clenshaw-Curtis weights), real part."""
        return float(np.sum(self.g.w * self.g.r * np.real(uz_profile)))

    # -------------------------------------------------------- initial states
    def place(self, raw: np.ndarray, profile: np.ndarray) -> np.ndarray:
        """Radial profile x raw coefficients (mp+1, 2kp+1 natural k) ->
        spectral (Nr, M+1, NK) with the m = 0 Hermitian fix."""
        mp = raw.shape[0] - 1
        kp = (raw.shape[1] - 1) // 2
        if mp > self.M or kp > self.K:
            raise ValueError("excited modes exceed the resolved ones")
        out = np.zeros((self.g.Nr, self.M + 1, self.NK), dtype=complex)
        for m in range(mp + 1):
            for k in range(-kp, kp + 1):
                out[:, m, k % self.NK] = profile * raw[m, k + kp]
        return self.sp.hermitian_fix(out)

    def curl(self, psi):
        """Discrete curl of a spectral vector field (3, Nr, M+1, NK).

        (curl psi)_r = (i m/r) psi_z - i beta psi_theta
        (curl psi)_theta = i beta psi_r - D1 psi_z
        (curl psi)_z = (1/r) D1(r psi_theta) - (i m/r) psi_r
        Its discrete divergence (same D1) vanishes identically.
        """
        g = self.g
        r = g.r[:, None, None]
        m = self.sp.m[None, :, None]
        beta = self.sp.beta[None, None, :]
        pr, pt, pz = psi
        return np.stack([1j * m * pz / r - 1j * beta * pt,
                         1j * beta * pr - g.dr(pz),
                         g.dr(r * pt) / r - 1j * m * pr / r])

    def _perturbation_shapes(self, psi_raw, T_raw=None):
        """Unscaled u' = curl(psi) (zeroed at the wall nodes) and T' (Sec. 2.1).

        psi = (1 - x^2)^2 x raw coefficients, T' = (1 - x^2) x raw
        coefficients (None without temperature or raw T draws).
        """
        x = self.g.x
        prof = (1.0 - x * x) ** 2
        psi = np.stack([self.place(psi_raw[c], prof) for c in range(3)])
        u = self.curl(psi)
        u[:, 0] = 0.0
        u[:, -1] = 0.0
        t = None
        if self.has_T and T_raw is not None:
            t = self.place(T_raw, 1.0 - x * x)
        return u, t

    def ic_scales(self, psi_raw, T_raw=None):
        """The constants s_u, s_T that scale curl(psi) to max|u'| = amp and T'
        to max |T'| = amp_T on the physical grid (Sec. 2.1 initial conditions;
        s_T = 0 without temperature draws or with amp_T = 0)."""
        u, t = self._perturbation_shapes(psi_raw, T_raw)
        ph = [self.sp.to_physical(u[c]) for c in range(3)]
        mag = np.sqrt(ph[0] ** 2 + ph[1] ** 2 + ph[2] ** 2).max()
        s_u = self.wl.amp / mag
        s_T = 0.0
        if t is not None and self.wl.amp_T > 0:
            s_T = self.wl.amp_T / np.abs(self.sp.to_physical(t)).max()
        return s_u, s_T

    def initial_state(self, psi_raw, T_raw=None, scales=None):
        """Basic state + u' = curl(psi) scaled to max|u'| = amp (Sec. 2.1).

        psi = (1 - x^2)^2 x raw coefficients; u' is zeroed at the wall nodes
        and scaled by a constant so that the largest Euclidean norm of u' over
        the physical grid equals ``amp``.  With temperature, T' = (1 - x^2) x
        raw coefficients scaled so that max |T'| = amp_T.  ``scales`` = (s_u,
        s_T) applies fixed factors instead (the map is then linear in the
        coefficients, as the gradient of the differentiation form assumes).
        """
        u, t = self._perturbation_shapes(psi_raw, T_raw)
        X = self.base.copy()
        if scales is None:
            scales = self.ic_scales(psi_raw, T_raw)
            if self.wl.amp_T <= 0:
                t = None
        X[:3] += scales[0] * u
        if t is not None:
            X[3] += scales[1] * t
        return X

    # ------------------------------------------------------------ diagnostics
    def radial_integral(self, f: np.ndarray) -> float:
        """int f r dr over the gap with the Clenshaw-Curtis weights."""
        return float(np.sum(self.g.w * self.g.r * f))

    def diagnostics(self, X, dt: float = 0.0, rate: float = 0.0):
        """Global quantities of a state.

        E = (1/2) int |u|^2 dV; E_pert with u - u_base; torque_w =
        2 pi Lz r_w^2 (d u_theta/dr - u_theta/r) of the mean flow at wall w;
        P_wall = work of the walls on the fluid; eps = int 2 S:S dV;
        buoy_work = Gr int u_z T dV; Nu_w = mean dT/dr at wall w over the same
        quantity of the discrete conductive state (Sec. 4); div_max = max
        |div u| over all stored coefficients; div_rms = (int |div u|^2 dV / V)^1/2.
        """
        g, sp, wl = self.g, self.sp, self.wl
        V = 2.0 * math.pi * wl.Lz
        r = g.r[:, None, None]
        m = sp.m[None, :, None]
        beta = sp.beta[None, None, :]
        ur, ut, uz = X[0], X[1], X[2]
        pd = sp.plane_dot
        E = 0.5 * V * self.radial_integral(pd(ur, ur) + pd(ut, ut) + pd(uz, uz))
        d = X[:3] - self.base[:3]
        E_pert = 0.5 * V * self.radial_integral(sum(pd(d[c], d[c]) for c in range(3)))
        Srr = g.dr(ur)
        Stt = 1j * m * ut / r + ur / r
        Szz = 1j * beta * uz
        Srt = 0.5 * (g.dr(ut) - ut / r + 1j * m * ur / r)
        Srz = 0.5 * (1j * beta * ur + g.dr(uz))
        Stz = 0.5 * (1j * beta * ut + 1j * m * uz / r)
        ss = 2.0 * (pd(Srr, Srr) + pd(Stt, Stt) + pd(Szz, Szz)) \
            + 4.0 * (pd(Srt, Srt) + pd(Srz, Srz) + pd(Stz, Stz))
        eps = V * self.radial_integral(ss)
        ut00 = ut[:, 0, 0].real
        sig = g.D1 @ ut00 - ut00 / g.r
        torque_i = V * g.r_i ** 2 * sig[0]
        torque_o = V * g.r_o ** 2 * sig[-1]
        P_wall = V * (g.r_o * wl.Re_o * sig[-1] - g.r_i * wl.Re_i * sig[0])
        buoy = Nu_i = Nu_o = 0.0
        if self.has_T:
            buoy = self.Gr * V * self.radial_integral(pd(uz, X[3]))
            dT = g.D1 @ X[3][:, 0, 0].real
            dTb = g.D1 @ self.Tb_disc[:, 0, 0].real
            Nu_i, Nu_o = dT[0] / dTb[0], dT[-1] / dTb[-1]
        div = (g.dr(r * ur) / r + 1j * m * ut / r + 1j * beta * uz)
        div_max = float(np.abs(div).max())
        div_rms = math.sqrt(self.radial_integral(pd(div, div))
                            / self.radial_integral(np.ones(g.Nr)))
        return dict(dt=dt, E=E, E_pert=E_pert, torque_i=torque_i,
                    torque_o=torque_o, P_wall=P_wall, eps=eps, buoy_work=buoy,
                    Nu_i=Nu_i, Nu_o=Nu_o, div_max=div_max, div_rms=div_rms,
                    cfl=rate * dt)

    # ----------------------------------------------------- analytic reference
    def couette_analytic(self):
        return couette_AB(self.wl.eta, self.wl.Re_i, self.wl.Re_o)
