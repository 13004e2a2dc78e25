"""Arithmetic of the 7-slice BF16 split that the tensor-core azimuthal stage
uses (Ozaki et al., Numer. Algorithms 59, 2012), restated in Python
integers and checked on the CPU:

* the balanced base-256 digits come from the bytes of q + 0x0080808080808080
  (the carry of each added 0x80 lands where a balanced digit borrows): they
  sum back to q, the six low ones lie in [-128, 127] and the top one in
  [-128, 256], and each is exact in BF16 (at most 8 significant bits);
* a level of the slice products (all pairs i + j = L over K = 96
  coefficients) stays below 2^24, so FP32 accumulation of it is exact;
* a DFT row times a data column through the split (levels 0..6 kept, level 6
  rounded to units of 2^-40 as the kernel does) equals the exact product to
  within a few units of 2^-56 of the column scale.

The CUDA kernel itself is checked on the GPU against the FFT path and the
oracle (tests/test_gpu_theta_tc.py)."""
import math
import random
from fractions import Fraction

S = 7


def digits_from_bytes(q):
    """Balanced digits (least significant first) of 0 <= q < 2^56."""
    t = q + 0x0080808080808080
    d = [((t >> (8 * j)) & 0xFF) - 128 for j in range(6)]
    d.append((t >> 48) - 128)   # bytes 6 and 7
    return d


def bf16_exact(v):
    """True if the integer v is exactly representable in BF16."""
    if v == 0:
        return True
    a = abs(v)
    while a % 2 == 0:
        a //= 2
    return a < 256   # at most 8 significant bits


def test_byte_digits_reconstruct_and_bound():
    rng = random.Random(7)
    cases = [0, 1, 127, 128, 255, 256, (1 << 56) - 1, (1 << 55), 0x0080808080808080,
             0x7F7F7F7F7F7F7F]
    cases += [rng.getrandbits(rng.randint(1, 56)) for _ in range(20000)]
    for q in cases:
        d = digits_from_bytes(q)
        assert sum(dj * 256 ** j for j, dj in enumerate(d)) == q
        assert all(-128 <= dj <= 127 for dj in d[:6]), (q, d)
        assert -128 <= d[6] <= 256, (q, d)
        assert all(bf16_exact(dj) and bf16_exact(-dj) for dj in d)


def test_level_sums_below_2_to_24():
    # |a_0|, |b_0| <= 256, the other digits <= 128: level L has at most
    # two pairs with a top digit and L - 1 pairs of lower digits
    K = 96
    for L in range(S):
        top = (2 * 256 * 128 if L >= 1 else 256 * 256)
        low = max(L - 1, 0) * 128 * 128
        assert K * (top + low) < 2 ** 24, L
    # the closed form used in the kernel's comment, K 2^14 (L + 3) for L >= 1
    for L in range(1, S):
        assert K * (2 * 256 * 128 + (L - 1) * 128 * 128) == K * 2 ** 14 * (L + 3)


def split(y, E):
    """Digits (most significant first) of y / 2^E, |y| < 2^E: y / 2^E =
    2^-8 sum_j b_j 2^-8j with q = round(|y| 2^(56 - E))."""
    q = round(abs(y) * Fraction(2) ** (56 - E))
    d = digits_from_bytes(int(q))[::-1]
    return [-x for x in d] if y < 0 else d


def test_split_product_matches_exact_dft_product():
    rng = random.Random(3)
    Nt, M = 128, 42
    for trial in range(6):
        j = rng.randrange(Nt)
        # row j of F/2: 1/2, 0, cos(m theta_j), -sin(m theta_j) (interleaved)
        row = [Fraction(1, 2), Fraction(0)]
        for m in range(1, M + 1):
            ang = 2.0 * math.pi * ((m * j) % Nt) / Nt
            row += [Fraction(math.cos(ang)), Fraction(-math.sin(ang))]
        x = [Fraction(rng.uniform(-1, 1) * 10 ** rng.uniform(-6, 0)) for _ in row]
        x[1] = Fraction(0)
        E = max(math.frexp(float(abs(v)))[1] for v in x if v != 0)   # max |x| < 2^E
        A = [split(a, 0) for a in row]   # |F/2| <= 1 < 2^1, scaled as 2^0 (the kernel's choice)
        B = [split(v, E) for v in x]
        levels = [sum(A[k][i] * B[k][L - i] for k in range(len(row)) for i in range(L + 1))
                  for L in range(S)]
        assert all(abs(s) < 2 ** 24 for s in levels)
        I = levels[0]
        for L in range(1, S - 1):
            I = I * 256 + levels[L]
        I += round(Fraction(levels[S - 1], 256))
        approx = Fraction(I) * Fraction(2) ** (E - 56)           # (F/2) x
        exact = sum(a * v for a, v in zip(row, x))
        assert abs(approx - exact) <= 8 * Fraction(2) ** (E - 56), (trial, float(approx - exact))


def mag_of(x):
    """|x| = mag 2^eu with mag < 2^53 an integer (the kernels' mag_of)."""
    m, e = math.frexp(abs(x))           # |x| = m 2^e, 0.5 <= m < 1
    if x == 0:
        return 0, -1074
    eu = max(e - 53, -1074)
    return int(Fraction(abs(x)) / Fraction(2) ** eu), eu


def scaled_int(mag, eu, E):
    """round(mag 2^(eu + 56 - E)), ties away from zero (the kernels' scaled_int)."""
    sh = eu + 56 - E
    if sh >= 0:
        return mag << sh
    rs = -sh
    if rs >= 63:
        return 0
    return (mag + (1 << (rs - 1))) >> rs


def test_derivative_magnitudes_exact_before_the_split():
    """The theta derivative's coefficients m |x| are formed as the integer
    significand times m (below 2^59) and rounded once, at the split, to
    units of 2^(E - 56): the result is round(m |x| 2^(56 - E)) of the exact
    product, ties away from zero."""
    rng = random.Random(11)
    for _ in range(5000):
        x = rng.uniform(-1, 1) * 10 ** rng.uniform(-300, 300)
        m = rng.randrange(0, 48)
        mag, eu = mag_of(x)
        assert Fraction(mag) * Fraction(2) ** eu == abs(Fraction(x))
        mm = mag * m
        assert mm < 2 ** 59
        if mm == 0:
            continue
        top = eu + mm.bit_length() - 1                       # 2^top <= m |x| < 2^(top+1)
        for E in (top + 1, top + 2, top + 9):                # the column maximum may be larger
            got = scaled_int(mm, eu, E)
            exact = m * abs(Fraction(x)) * Fraction(2) ** (56 - E)
            want = int(exact + Fraction(1, 2))               # ties away from zero (exact >= 0)
            assert got == want, (x, m, E)
            assert got < 2 ** 56
