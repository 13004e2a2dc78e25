"""Fourier transforms in (theta, z) with the 3/2 dealiasing rule (oracle).

Sec. 2.1: Fourier-Galerkin ansatz in theta and z, periodic in z; the products
of the nonlinear term are formed on the physical grid (pseudospectral).

Readings:
* u(r, theta, z) = sum_{|m|<=M} sum_{|k|<=K} u_{m,k}(r) exp(i(m theta + k a z)),
  a = 2 pi / Lz, real fields so u_{-m,-k} = conj(u_{m,k});
* the physical grid is theta_j = 2 pi j / Ntheta, z_l = Lz l / Nz, and it is
  already the padded grid: M = floor((Ntheta-1)/3), K = floor((Nz-1)/3), so a
  quadratic product has no aliasing inside |m| <= M, |k| <= K (3/2 rule) and
  Nyquist modes are never kept;
* stored coefficients are m = 0..M (Hermitian half) and k in FFT order
  (0..K, -K..-1), array shape (..., M+1, 2K+1);
* forward transform normalised by 1/(Ntheta Nz), inverse unnormalised.

Two transform modes: ``naive`` evaluates the sums above as explicit DFT
matrices (the definition); ``fft`` uses ``scipy.fft`` and is only a faster
route to the same numbers (tests check the two agree).
"""
from __future__ import annotations

import numpy as np
import scipy.fft


def k_order(K: int) -> np.ndarray:
    """Axial wavenumber index of each stored column, FFT order."""
    return np.concatenate([np.arange(0, K + 1), np.arange(-K, 0)])


class Spectral:
    def __init__(self, Ntheta: int, Nz: int, Lz: float, mode: str = "naive"):
        if mode not in ("naive", "fft"):
            raise ValueError(mode)
        self.Nt, self.Nz, self.Lz, self.mode = Ntheta, Nz, Lz, mode
        self.M = (Ntheta - 1) // 3
        self.K = (Nz - 1) // 3
        self.alpha = 2.0 * np.pi / Lz
        self.kk = k_order(self.K)                     # (2K+1,)
        self.m = np.arange(self.M + 1)                # (M+1,)
        self.beta = self.alpha * self.kk              # axial wavenumbers
        # weight of each stored m in a full-plane sum (Parseval)
        self.cm = np.where(self.m == 0, 1.0, 2.0)
        if mode == "naive":
            th = 2.0 * np.pi * np.arange(Ntheta) / Ntheta
            mm = np.arange(-self.M, self.M + 1)
            self.Et = np.exp(1j * np.outer(th, mm))                  # (Nt, 2M+1)
            kn = np.arange(-self.K, self.K + 1)
            zl = 2.0 * np.pi * np.arange(Nz) / Nz                    # a * z_l
            self.Ez = np.exp(1j * np.outer(zl, kn))                  # (Nz, 2K+1)

    # -- helpers -----------------------------------------------------------
    def _natural(self, uh: np.ndarray) -> np.ndarray:
        """(..., M+1, 2K+1) FFT-order -> (..., 2M+1, 2K+1), m and k natural."""
        K, M = self.K, self.M
        nat = np.concatenate([uh[..., K + 1:], uh[..., :K + 1]], axis=-1)  # k=-K..K
        full = np.empty(uh.shape[:-2] + (2 * M + 1, 2 * K + 1), dtype=complex)
        full[..., M:, :] = nat
        # u_{-m,-k} = conj(u_{m,k})
        full[..., :M, :] = np.conj(nat[..., :0:-1, ::-1])
        return full

    # -- transforms ---------------------------------------------------------
    def to_physical(self, uh: np.ndarray) -> np.ndarray:
        """Spectral (..., M+1, 2K+1) -> physical real (..., Ntheta, Nz)."""
        if self.mode == "naive":
            full = self._natural(uh)
            u = np.einsum("tm,...mk,zk->...tz", self.Et, full, self.Ez,
                          optimize=True)
            return u.real
        Nt, Nz, M, K = self.Nt, self.Nz, self.M, self.K
        spec = np.zeros(uh.shape[:-2] + (Nz, Nt // 2 + 1), dtype=complex)
        ks = self.kk % Nz
        spec[..., ks, :M + 1] = np.swapaxes(uh, -1, -2)
        u = scipy.fft.irfft2(spec, s=(Nz, Nt), axes=(-2, -1), workers=-1)
        return np.swapaxes(u, -1, -2) * (Nt * Nz)

    def to_spectral(self, u: np.ndarray) -> np.ndarray:
        """Physical (..., Ntheta, Nz) -> truncated spectral (..., M+1, 2K+1)."""
        Nt, Nz, M, K = self.Nt, self.Nz, self.M, self.K
        if self.mode == "naive":
            full = np.einsum("tm,...tz,zk->...mk", np.conj(self.Et), u,
                             np.conj(self.Ez), optimize=True) / (Nt * Nz)
            nat = full[..., M:, :]                     # m = 0..M, k = -K..K
            return np.concatenate([nat[..., K:], nat[..., :K]], axis=-1)
        spec = scipy.fft.rfft2(np.swapaxes(u, -1, -2), axes=(-2, -1), workers=-1)
        ks = self.kk % Nz
        return np.swapaxes(spec[..., ks, :M + 1], -1, -2) / (Nt * Nz)

    # -- inner products -------------------------------------------------------
    def plane_dot(self, ah: np.ndarray, bh: np.ndarray) -> np.ndarray:
        """(1/(2 pi Lz)) int int a b dtheta dz for real fields, per leading index.

        Parseval over the stored half plane: sum_m c_m sum_k Re(a conj(b)).
        """
        return np.einsum("m,...mk->...", self.cm, (ah * np.conj(bh)).real)

    def hermitian_fix(self, uh: np.ndarray) -> np.ndarray:
        """Impose u_{0,-k} = conj(u_{0,k}) and a real (0,0) coefficient.

        The k > 0 entries of the m = 0 column are kept; k < 0 are overwritten.
        """
        out = uh.copy()
        K = self.K
        pos = out[..., 0, 1:K + 1]
        out[..., 0, K + 1:] = np.conj(pos[..., ::-1])
        out[..., 0, 0] = out[..., 0, 0].real
        return out
