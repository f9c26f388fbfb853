"""The output blocks of the tensor-core distribution, checked on the CPU
against brute force.

With the modes split at h into a low side [0, h) and a high side [h, m), e =
min(3, n / 2) and k the photons on the low side, every output S is computed
exactly once:
  * k = e+1 .. n-e-1: low-side multiset P (k photons) times high-side Q;
  * k >= n-e: S = R ++ E, R the n-e smallest modes (all low), E the rest;
  * k <= e (k < e when n = 2e): S = E ++ R, R the n-e largest modes (all high).
The index of S in the canonical (lexicographic) order splits into a part of R
and a part of E, and the amplitude of S is the sum over the sign vectors of
the product of the entries of R and E, times 1/sqrt(C(mu_R + mu_E, mu_E)) when
they share the seam mode.  The first test enumerates every pair and compares
with the rank of the merged mode list; the second builds the amplitudes from
the Glynn factors (Eq. of the permanent as a sum over sign vectors) and
compares with the oracle's permanents.
"""
import itertools
import math

import numpy as np
import pytest

import oracle


def msets(w, k):
    return 1 if k == 0 else (0 if w <= 0 else math.comb(w + k - 1, k))


def rank(m, s):
    """Lexicographic rank of the non-decreasing mode list s over m modes."""
    r, prev, n = 0, 0, len(s)
    for p, x in enumerate(s):
        r += sum(msets(m - v, n - p - 1) for v in range(prev, x))
        prev = x
    return r


def blocks(m, n, h):
    """Every (kind, R, E) pair the blocks compute, with the two index parts."""
    e = max(1, min(3, n // 2))
    L = n - e
    phi = lambda z: sum(msets(m - v, e - 1) for v in range(z))
    psi = lambda z: sum(msets(m - v, L - 1) for v in range(z))
    for R in itertools.combinations_with_replacement(range(h), L):
        t = R[-1]
        rb = rank(m, R + (t,) * e) - phi(t)
        for E in itertools.combinations_with_replacement(range(m), e):
            if E[0] >= t:
                yield "low", R, E, rb, rank(m, E)
    for R in itertools.combinations_with_replacement(range(h, m), L):
        rb = rank(m, (0,) * e + R)
        for E in itertools.combinations_with_replacement(range(m), e):
            if E[-1] <= R[0] and not (n == 2 * e and E[-1] < h):
                yield "high", R, E, rb, rank(m, E + (E[-1],) * L) - psi(E[-1])


@pytest.mark.parametrize("m,n", [(2, 2), (3, 2), (2, 3), (5, 4), (6, 3), (7, 4), (9, 5), (8, 6),
                                 (10, 7), (8, 9), (7, 10), (6, 2), (4, 5)])
def test_every_output_once_at_the_index_of_its_parts(m, n):
    h = max(1, m // 2)
    e = max(1, min(3, n // 2))
    seen = {}
    for s in itertools.combinations_with_replacement(range(m), n):
        k = sum(x < h for x in s)
        if e + 1 <= k <= n - e - 1:
            seen[s] = 1
    for kind, R, E, rb, cb in blocks(m, n, h):
        S = tuple(sorted(R + E))
        assert rank(m, S) == rb + cb, (kind, R, E)
        seen[S] = seen.get(S, 0) + 1
    assert len(seen) == msets(m, n)
    assert set(seen.values()) == {1}


@pytest.mark.parametrize("m,n,seed", [(4, 2, 1), (5, 3, 2), (6, 4, 3), (4, 6, 4), (6, 5, 5), (5, 6, 6),
                                      (3, 7, 7)])
def test_amplitudes_from_the_factors_of_each_pair(m, n, seed):
    h = max(1, m // 2)
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)))[0]
    cols = [i % m for i in range(n)]
    t = np.bincount(cols, minlength=m)
    K = 2 ** (n - 1)
    signs = np.ones((K, n))
    for d in range(K):
        for i in range(1, n):
            signs[d, i] = -1.0 if (d >> (i - 1)) & 1 else 1.0
    sigma = signs.prod(axis=1)
    Y = signs @ U[:, cols].T                          # y_r(d) = sum_i s_i(d) U[r, col_i]
    lead = 2.0 ** (-(n - 1)) / math.sqrt(math.prod(math.factorial(x) for x in t))

    def entry(P):
        v = np.ones(K, complex)
        for x in set(P):
            v = v * Y[:, x] ** P.count(x) / math.sqrt(math.factorial(P.count(x)))
        return v

    got, occ = [], []
    for kind, R, E, _, _ in blocks(m, n, h):
        a = np.sum(lead * sigma * entry(R) * entry(E))
        key = R[-1] if kind == "low" else R[0]
        if (E[0] if kind == "low" else E[-1]) == key:
            a /= math.sqrt(math.comb(R.count(key) + E.count(key), E.count(key)))
        got.append(a)
        occ.append(np.bincount(R + E, minlength=m))
    want = oracle.amplitudes(U, t.astype(np.uint8), np.array(occ, np.uint8))
    assert np.max(np.abs(np.array(got) - want)) <= 1e-13
