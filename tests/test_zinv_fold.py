"""Arithmetic of the tensor-core inverse axial stage (k_zinv_tc), restated in
Python and checked on the CPU:

* the folded axial DFT matrix: cosine rows j = 0 .. Nz/2 stacked over sine
  rows j = 1 .. (Nz-1)/2, Nz rows in all.  With P_j and Q_j the products of
  a complex column with a cosine and a sine row, v_j = P_j + i Q_j and
  v_(Nz-j) = P_j - i Q_j reproduce v_l = sum_k a_k e^(2 pi i k l / Nz) for
  every l, at even and odd Nz;
* through the 7-slice split (exact level sums, Horner in 64-bit integers in
  units of 2^(E-56), E the exponent of the complex column), the integer sum
  of a cosine and a sine row gives v_j and v_(Nz-j) to within a few units of
  2^(E-56), and stays inside the signed 64-bit range.

The CUDA kernel itself is checked on the GPU against the FFT path and the
oracle (tests/test_gpu_zinv_tc.py)."""
import math
import random
from fractions import Fraction

import numpy as np

from test_theta_split import S, split


def folded_matrix(Nz, K):
    """Rows 0 .. Nz-1 of the kernel's table (the padding rows and columns are
    zero and left out); column kk is the stored axial index."""
    NK, h = 2 * K + 1, Nz // 2
    A = np.zeros((Nz, NK))
    for row in range(Nz):
        for kk in range(NK):
            k = kk if kk <= K else kk - NK
            sine = row > h
            j = row - h if sine else row
            ang = 2.0 * math.pi * ((k * j) % Nz) / Nz
            A[row, kk] = math.sin(ang) if sine else math.cos(ang)
    return A


def unfold(D, Nz):
    """v (Nz values) from the Nz rows of D = A a, as the kernel's last phase."""
    h, hq = Nz // 2, (Nz - 1) // 2
    v = np.zeros(Nz, dtype=complex)
    for j in range(h + 1):
        P = D[j]
        Q = D[h + j] if 1 <= j <= hq else 0.0
        v[j] = P + 1j * Q
        if 1 <= j <= hq:
            v[Nz - j] = P - 1j * Q
    return v


def test_folded_matrix_reproduces_the_inverse_transform():
    rng = np.random.default_rng(11)
    for Nz in (128, 96, 75, 45, 40, 10, 8, 5):
        K = (Nz - 1) // 3
        NK = 2 * K + 1
        assert Nz <= 128 and NK <= 96
        A = folded_matrix(Nz, K)
        a = rng.standard_normal(NK) + 1j * rng.standard_normal(NK)
        ks = np.array([kk if kk <= K else kk - NK for kk in range(NK)])
        ref = np.exp(2j * np.pi * np.outer(np.arange(Nz), ks) / Nz) @ a
        # real and imaginary parts as two real data columns
        D = A @ a.real + 1j * (A @ a.imag)
        got = unfold(D, Nz)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(a).sum(), Nz


def levels_int(Arow, Bcol):
    """The kernel's integer of one row times one data column: exact level
    sums, Horner in units of 2^-40 of level 0, the last level rounded."""
    levels = [sum(Arow[k][i] * Bcol[k][L - i] for k in range(len(Arow)) for i in range(L + 1))
              for L in range(S)]
    assert all(abs(s) < 2 ** 24 for s in levels)
    I = levels[0]
    for L in range(1, S - 1):
        I = I * 256 + levels[L]
    return I + round(Fraction(levels[S - 1], 256))


def test_split_fold_sum_matches_exact_values():
    rng = random.Random(5)
    Nz, K = 128, 42
    NK, h = 2 * K + 1, Nz // 2
    A = folded_matrix(Nz, K)
    for trial in range(4):
        j = rng.randrange(1, h)   # a row with a mirror
        scale = 10 ** rng.uniform(-8, 2)
        re = [Fraction(rng.uniform(-1, 1) * scale) for _ in range(NK)]
        im = [Fraction(rng.uniform(-1, 1) * scale) for _ in range(NK)]
        # one exponent for the complex column: max |x| < 2^E
        E = max(math.frexp(float(abs(v)))[1] for v in re + im if v != 0)
        crow = [split(Fraction(float(x)), 0) for x in A[j]]
        srow = [split(Fraction(float(x)), 0) for x in A[h + j]]
        Bre = [split(v, E) for v in re]
        Bim = [split(v, E) for v in im]
        Pr, Pi = levels_int(crow, Bre), levels_int(crow, Bim)
        Qr, Qi = levels_int(srow, Bre), levels_int(srow, Bim)
        unit = Fraction(2) ** (E - 56)
        # the same table rows: v_j = P_j + i Q_j, v_(Nz-j) = P_j - i Q_j
        c = [Fraction(float(x)) for x in A[j]]
        sn = [Fraction(float(x)) for x in A[h + j]]
        Pre = sum(ci * r for ci, r in zip(c, re))
        Pim = sum(ci * m for ci, m in zip(c, im))
        Qre = sum(si * r for si, r in zip(sn, re))
        Qim = sum(si * m for si, m in zip(sn, im))
        exact = {j: (Pre - Qim, Pim + Qre), Nz - j: (Pre + Qim, Pim - Qre)}
        got = {j: (Pr - Qi, Pi + Qr), Nz - j: (Pr + Qi, Pi - Qr)}
        for l in (j, Nz - j):
            for part in range(2):
                I = got[l][part]
                assert abs(I) < 2 ** 63
                # the error of the split: the roundings of the table entries
                # and of the data to 2^-56 of their scales, and of the last level
                err = abs(Fraction(I) * unit - exact[l][part]) / unit
                assert err <= 16, (trial, l, part, float(err))
