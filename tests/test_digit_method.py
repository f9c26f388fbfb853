"""The arithmetic behind the tensor-core products (PCV_ALGO_FACTOR_TC),
restated with exact Python integers and rationals: the error-free splitting
of Ozaki, Ogita, Oishi and Rump (2012) as this library applies it.  These
tests pin the facts the kernels rely on, not the kernels themselves (those
are checked against the oracle on the GPU):

* the balanced base-128 digits D_i = field_i(X + C) - 64, C = 64 in every
  7-bit field, give back X exactly, with |D_i| <= 64;
* each diagonal i + j = d of digit-pair sums over K <= 512 sign vectors stays
  within 2^24 in magnitude, so an FP32 accumulator never rounds it;
* keeping the 36 pairs with i + j <= 7 (and the splitting itself) leaves an
  error within K 2^{-54} of the row x column scale, the order of FP64
  summation's own worst case;
* combining the diagonals as Z = sum_d acc_d 128^{7-d} and scaling by
  2^{E_row + E_col - 63} gives the product sum of the split values.
"""
import math
import random
from fractions import Fraction

import pytest

C = sum(64 << (7 * k) for k in range(8))          # 64 in every 7-bit field


def exponent(values):
    """Smallest E with max |x| <= 2^{E-1} (None for an all-zero row)."""
    m = max(abs(v) for v in values)
    if m == 0:
        return None
    E = math.frexp(m)[1] + 1                       # m < 2^{frexp}, so m <= 2^{E-1}
    while m <= 2.0 ** (E - 2):
        E -= 1
    return E


def fixed(x, E):
    """round(x 2^{56-E}), the magnitude rounded half up, sign restored
    (0 for an all-zero row, E = None)."""
    if E is None:
        return 0
    v = abs(Fraction(x)) * Fraction(2) ** (56 - E)
    r = math.floor(v + Fraction(1, 2))
    return -r if x < 0 else r


def digits(X):
    """Balanced base-128 digits of X, most significant first."""
    P = X + C
    assert 0 <= P < 1 << 57
    out = [(P >> 49) - 64]
    for i in range(1, 8):
        out.append(((P >> (7 * (7 - i))) & 127) - 64)
    return out


def test_digits_reconstruct_and_stay_small():
    rng = random.Random(1)
    cases = [0, 1, -1, 1 << 55, -(1 << 55), (1 << 55) - 1, 64, -64, 63, -65]
    cases += [rng.randrange(-(1 << 55), (1 << 55) + 1) for _ in range(20000)]
    for X in cases:
        D = digits(X)
        assert sum(d * 128 ** (7 - i) for i, d in enumerate(D)) == X
        assert all(abs(d) <= 64 for d in D)


def test_worst_case_diagonal_fits_fp32():
    # every digit at its extreme: 8 pairs per diagonal, K = 512 sign vectors
    K, worst = 512, 64 * 64
    for d in range(8):
        pairs = d + 1
        assert pairs * K * worst <= 1 << 24
    assert 8 * K * worst == 1 << 24              # the bound is tight only at d = 7


@pytest.mark.parametrize("K", [1, 64, 512])
def test_truncated_digit_products_match_the_exact_sum(K):
    rng = random.Random(K)
    for trial in range(4):
        # rows with a spread of magnitudes, like products of row sums
        a = [rng.gauss(0, 1) * 2.0 ** rng.randint(-30, 3) for _ in range(K)]
        b = [rng.gauss(0, 1) * 2.0 ** rng.randint(-12, 8) for _ in range(K)]
        if trial == 3:
            a[0], b[-1] = 0.0, 0.0
        Ea, Eb = exponent(a), exponent(b)
        Da = [digits(fixed(x, Ea)) for x in a]
        Db = [digits(fixed(x, Eb)) for x in b]
        acc = [0] * 8
        for da, db in zip(Da, Db):
            for i in range(8):
                for j in range(8 - i):
                    acc[i + j] += da[i] * db[j]
        assert all(abs(v) <= 1 << 24 for v in acc)
        Z = sum(acc[d] * 128 ** (7 - d) for d in range(8))
        exact = sum(Fraction(x) * Fraction(y) for x, y in zip(a, b))
        if Ea is None or Eb is None:             # an all-zero row: the product is 0
            assert Z == 0 and exact == 0
            continue
        got = Fraction(Z) * Fraction(2) ** (Ea + Eb - 63)
        scale = Fraction(2) ** (Ea + Eb)
        # splitting (half a unit of 2^{E-56} per value) and the dropped pairs
        # (diagonals 8..14, weight <= 2^{-63} each) together stay below
        # K 2^{-54} of the row x column scale 2^{Ea + Eb}
        assert abs(got - exact) <= K * scale / 2 ** 54


def test_fp64_scaling_of_the_combined_diagonals():
    # hi 2^28 + lo with hi, lo from the two halves of the diagonals equals Z
    rng = random.Random(5)
    for _ in range(2000):
        acc = [rng.randrange(-(1 << 24), (1 << 24) + 1) for _ in range(8)]
        hi = sum(acc[d] * 128 ** (3 - d) for d in range(4))
        lo = sum(acc[d] * 128 ** (7 - d) for d in range(4, 8))
        assert abs(hi) < 1 << 46 and abs(lo) < 1 << 46
        assert hi * (1 << 28) + lo == sum(acc[d] * 128 ** (7 - d) for d in range(8))


def fixed_by_shift(x, E):
    """The kernels' branch-free recipe for fixed(x, E): with the 53-bit
    mantissa m of x and sh = e - 1019 - E <= 3 (e its exponent field; any E
    with |x| <= 2^{E-1}), one right shift by s = 4 - sh >= 1 of 16 m, rounded
    half up."""
    if E is None or x == 0:
        return 0
    bits = int.from_bytes(__import__("struct").pack(">d", x), "big")
    e = (bits >> 52) & 0x7FF
    m = (bits & ((1 << 52) - 1)) | (1 << 52)
    s = 4 - (e - 1019 - E)
    assert s >= 1
    M = ((m << 4) + (1 << (s - 1))) >> s if s < 64 else 0
    return -M if x < 0 else M


def test_branch_free_fixed_point_matches_rounding_half_up():
    rng = random.Random(11)
    for _ in range(400):
        row = [rng.gauss(0, 1) * 2.0 ** rng.randint(-70, 10) for _ in range(16)]
        row.append(2.0 ** rng.randint(-20, 20))          # an exact power of two as the row maximum
        for extra in (0, 1):                             # the row's own exponent, and one bit coarser
            E = exponent(row) + extra
            for x in row + [0.0, -row[0]]:
                assert fixed_by_shift(x, E) == fixed(x, E)


@pytest.mark.parametrize("K", [1, 64, 512])
def test_common_exponent_for_real_and_imaginary_parts(K):
    """One exponent per row for re and im, one bit above their largest: then
    |X_re|, |X_im| <= 2^54, the re + im operand is the integer X_re + X_im
    (|.| <= 2^55, so its balanced digits exist), Re = t1 - t2 and
    Im = t3 - t1 - t2 hold exactly in integers before the single scaling, and
    the result is within K 2^{-53} of the row x column scale."""
    rng = random.Random(100 + K)
    for trial in range(3):
        ar = [rng.gauss(0, 1) * 2.0 ** rng.randint(-30, 3) for _ in range(K)]
        ai = [rng.gauss(0, 1) * 2.0 ** rng.randint(-30, 3) for _ in range(K)]
        br = [rng.gauss(0, 1) * 2.0 ** rng.randint(-12, 8) for _ in range(K)]
        bi = [rng.gauss(0, 1) * 2.0 ** rng.randint(-12, 8) for _ in range(K)]
        Ea, Eb = exponent(ar + ai) + 1, exponent(br + bi) + 1
        Xa = [(fixed(r, Ea), fixed(i, Ea)) for r, i in zip(ar, ai)]
        Xb = [(fixed(r, Eb), fixed(i, Eb)) for r, i in zip(br, bi)]
        assert all(abs(v) <= 1 << 54 for p in Xa + Xb for v in p)

        def product(f, g):
            acc = [0] * 8
            for x, y in zip(f, g):
                dx, dy = digits(x), digits(y)
                for i in range(8):
                    for j in range(8 - i):
                        acc[i + j] += dx[i] * dy[j]
            assert all(abs(v) <= 1 << 24 for v in acc)
            return sum(acc[d] * 128 ** (7 - d) for d in range(8))

        t1 = product([x for x, _ in Xa], [y for y, _ in Xb])
        t2 = product([x for _, x in Xa], [y for _, y in Xb])
        t3 = product([x + y for x, y in Xa], [x + y for x, y in Xb])
        sc = Fraction(2) ** (Ea + Eb - 63)
        re, im = (t1 - t2) * sc, (t3 - t1 - t2) * sc
        ex_re = sum(Fraction(p) * Fraction(q) - Fraction(r) * Fraction(s) for p, r, q, s in zip(ar, ai, br, bi))
        ex_im = sum(Fraction(p) * Fraction(s) + Fraction(r) * Fraction(q) for p, r, q, s in zip(ar, ai, br, bi))
        scale = Fraction(2) ** (Ea + Eb)
        assert abs(re - ex_re) <= K * scale / 2 ** 53
        assert abs(im - ex_im) <= K * scale / 2 ** 53


def floor_rd(x):
    """RD(x + 2^23) - 2^23 for 0 <= x < 2^22 with x on a grid of 2^-23 or
    coarser: FP32 addition rounded down leaves the integer part exactly."""
    assert 0 <= x < 2 ** 22
    return math.floor(x)


def digits_by_pieces(P):
    """The kernels' FP32 recipe for the balanced digits of P = X + C: the
    15-bit piece P >> 42 holds fields 0 and 1, and the 21-bit pieces
    (P >> 21) mod 2^21 and P mod 2^21 three fields each; every field comes
    from floor(v 2^-14) or floor(r 2^-7) and fused multiply-adds whose
    operands and results are integers below 2^24 (exact in FP32)."""
    out = []
    a = P >> 42
    d0 = floor_rd(Fraction(a, 128)) - 64
    out += [d0, (a - 8256) - 128 * d0]
    for v in ((P >> 21) & ((1 << 21) - 1), P & ((1 << 21) - 1)):
        da = floor_rd(Fraction(v, 1 << 14)) - 64
        r = (v - (1 << 20)) - 16384 * da
        db = floor_rd(Fraction(r, 128)) - 64
        out += [da, db, (r - 8256) - 128 * db]
    # every intermediate the recipe forms is an integer of magnitude < 2^24
    return out


def test_digits_from_fp32_pieces_equal_the_field_digits():
    rng = random.Random(21)
    cases = [0, 1, -1, 1 << 55, -(1 << 55), (1 << 55) - 1, 64, -64, 63, -65, (1 << 54) + 12345]
    cases += [rng.randrange(-(1 << 55), (1 << 55) + 1) for _ in range(20000)]
    for X in cases:
        assert digits_by_pieces(X + C) == digits(X)
