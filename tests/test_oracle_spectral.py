"""Pins of the oracle's (theta, z) transforms and 3/2-rule dealiasing.

Sec. 2.1: Fourier-Galerkin ansatz in theta and z with products formed on the
physical grid.  The naive matrix DFT is the definition; the scipy.fft mode
must agree with it; single modes have closed forms; the dealiased product
equals the brute-force truncated convolution of the coefficients.
"""
import math

import numpy as np
import pytest
from scipy.signal import convolve2d

from oracle.spectral import Spectral, k_order


def _random_hermitian(sp, rng, lead=()):
    uh = (rng.standard_normal(lead + (sp.M + 1, 2 * sp.K + 1))
          + 1j * rng.standard_normal(lead + (sp.M + 1, 2 * sp.K + 1)))
    return sp.hermitian_fix(uh)


@pytest.mark.parametrize("Nt,Nz", [(32, 32), (48, 64), (12, 30)])
def test_naive_matches_fft(Nt, Nz):
    rng = np.random.default_rng(1)
    a = Spectral(Nt, Nz, 2.0, "naive")
    b = Spectral(Nt, Nz, 2.0, "fft")
    uh = _random_hermitian(a, rng, (3,))
    np.testing.assert_allclose(a.to_physical(uh), b.to_physical(uh), atol=1e-12)
    u = rng.standard_normal((2, Nt, Nz))
    np.testing.assert_allclose(a.to_spectral(u), b.to_spectral(u), atol=1e-14)


def test_round_trip():
    rng = np.random.default_rng(2)
    sp = Spectral(32, 48, 1.7)
    uh = _random_hermitian(sp, rng, (4,))
    np.testing.assert_allclose(sp.to_spectral(sp.to_physical(uh)), uh, atol=1e-13)


def test_single_mode_closed_form():
    Nt, Nz, Lz = 24, 36, 2 * math.pi / 3.16
    sp = Spectral(Nt, Nz, Lz)
    th = 2 * math.pi * np.arange(Nt)[:, None] / Nt
    z = Lz * np.arange(Nz)[None, :] / Nz
    a = 2 * math.pi / Lz
    m, k, c = 3, -2, 0.7 - 0.4j
    u = 2 * (c * np.exp(1j * (m * th + k * a * z))).real
    uh = sp.to_spectral(u)
    ref = np.zeros_like(uh)
    ref[m, k % (2 * sp.K + 1)] = c
    np.testing.assert_allclose(uh, ref, atol=1e-14)
    # derivatives as multipliers
    dth = sp.to_physical(1j * sp.m[:, None] * uh)
    dz = sp.to_physical(1j * sp.beta[None, :] * uh)
    np.testing.assert_allclose(dth, 2 * (1j * m * c * np.exp(1j * (m * th + k * a * z))).real,
                               atol=1e-12)
    np.testing.assert_allclose(dz, 2 * (1j * k * a * c * np.exp(1j * (m * th + k * a * z))).real,
                               atol=1e-12)


def test_truncation_sizes():
    sp = Spectral(32, 32, 1.0)
    assert (sp.M, sp.K) == (10, 10)
    sp = Spectral(128, 128, 1.0)
    assert (sp.M, sp.K) == (42, 42)
    sp = Spectral(512, 512, 1.0)
    assert (sp.M, sp.K) == (170, 170)
    assert list(k_order(2)) == [0, 1, 2, -2, -1]


@pytest.mark.parametrize("Nt,Nz", [(32, 32), (48, 24), (30, 45)])
def test_dealiased_product_equals_truncated_convolution(Nt, Nz):
    rng = np.random.default_rng(3)
    sp = Spectral(Nt, Nz, 1.3)
    ah = _random_hermitian(sp, rng)
    bh = _random_hermitian(sp, rng)
    prod = sp.to_spectral(sp.to_physical(ah) * sp.to_physical(bh))
    A = sp._natural(ah)
    B = sp._natural(bh)
    C = convolve2d(A, B)               # exact coefficients of the product
    M, K = sp.M, sp.K
    Cc = C[2 * M - M:2 * M + M + 1, 2 * K - K:2 * K + K + 1]   # |m|<=M, |k|<=K
    ref = np.concatenate([Cc[M:, K:], Cc[M:, :K]], axis=1)
    np.testing.assert_allclose(prod, ref, atol=1e-12 * np.abs(ref).max())


def test_aliasing_would_appear_without_padding():
    """The 3/2 grid matters: on an unpadded grid the same product aliases."""
    rng = np.random.default_rng(4)
    sp = Spectral(32, 32, 1.0)
    ah = _random_hermitian(sp, rng)
    small = Spectral(21, 21, 1.0)       # 2M+1 points: no room for products
    assert small.M < sp.M               # truncation changes with the grid
    A = sp._natural(ah)
    C = convolve2d(A, A)
    # the product has energy beyond |m| <= M that a 2M+1 grid would fold back
    M = sp.M
    assert np.abs(C[:M, :]).max() > 1e-3


def test_parseval_plane_dot():
    rng = np.random.default_rng(5)
    sp = Spectral(24, 30, 1.0)
    ah = _random_hermitian(sp, rng)
    bh = _random_hermitian(sp, rng)
    mean = np.mean(sp.to_physical(ah) * sp.to_physical(bh))
    assert abs(sp.plane_dot(ah, bh) - mean) < 1e-12 * abs(mean) + 1e-13


def test_hermitian_fix():
    rng = np.random.default_rng(6)
    sp = Spectral(12, 12, 1.0)
    uh = sp.hermitian_fix(rng.standard_normal((4, 7)) + 1j * rng.standard_normal((4, 7)))
    K = sp.K
    for k in range(1, K + 1):
        assert uh[0, -k] == np.conj(uh[0, k])
    assert uh[0, 0].imag == 0.0
