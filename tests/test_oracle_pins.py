"""Pins of the oracle against what the paper and elementary algebra fix.

No GPU.  Each test names the passage it checks.  The checks are chosen so
that a plausible slip anywhere in the oracle (a wrong root, a dropped
correction term, a swapped butterfly output, a wrong tree step, a bad half)
fails at least one of them:

* the brute-force definition F^_s = F(omega_s) and Gaussian elimination;
* the textbook FFT at n = 2^k and truncation of the zero-padded FFT;
* Figure 1 and the omega table of Section 2.2, transcribed under
  tests/golden/;
* Proposition 3.2's visit counts and Section 4's reverse-path statement;
* schoolbook products and Schwartz-Zippel evaluation of large products.
"""

import os
import random

import numpy as np
import pytest

from oracle import field as F
from oracle import native as NV
from oracle import tft as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PRIMES = F.PRIME_BY_ID


def _rand_vec(rng, pr, n):
    return [rng.randrange(pr.p) for _ in range(n)]


# --------------------------------------------------------------------------
# Section 2: the ring and the roots of unity
# --------------------------------------------------------------------------

@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_generator_and_two_adicity(pr):
    # Section 2.1: 2^K | p - 1 and the root of order 2^K exists.
    assert (pr.p - 1) % (1 << pr.K) == 0
    assert ((pr.p - 1) >> pr.K) % 2 == 1
    odd = (pr.p - 1) >> pr.K
    for f in pr.odd_factors:
        while odd % f == 0:
            odd //= f
    assert odd == 1, "odd_factors must factor (p-1)/2^K completely"
    assert F.is_primitive_root(pr)
    wK = F.omega_k(pr, pr.K)
    # primitive 2^K-th root: order exactly 2^K
    assert pow(wK, 1 << pr.K, pr.p) == 1
    assert pow(wK, 1 << (pr.K - 1), pr.p) == pr.p - 1


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_compatible_roots(pr):
    # Section 2.2: omega_[k+1]^2 = omega_[k]; omega_[0] = 1, omega_[1] = -1.
    assert F.omega_k(pr, 0) == 1
    assert F.omega_k(pr, 1) == pr.p - 1
    for k in range(pr.K):
        assert pow(F.omega_k(pr, k + 1), 2, pr.p) == F.omega_k(pr, k)


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_omega_sequence_identities(pr):
    # Section 2.2: omega_{2s+1} = -omega_{2s}, omega_{2s}^2 = omega_{2s+1}^2
    # = omega_s.  Exhaustive for s < 2^12 (cheap through the C oracle) plus
    # the Python definition on a prefix.
    p = pr.p
    om = [NV.omega(pr, s) for s in range(1 << 13)]
    for s in range(1 << 12):
        assert om[2 * s + 1] == (p - om[2 * s]) % p
        assert om[2 * s] * om[2 * s] % p == om[s]
        assert om[2 * s + 1] * om[2 * s + 1] % p == om[s]
    for s in range(64):
        assert F.omega(pr, s) == om[s]


def test_omega_table_of_section_2_2():
    rows = [l.split() for l in open(os.path.join(GOLDEN,
                                                 "omega_table_sec2_2.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 8
    for pr in PRIMES:
        for s, j, e in rows:
            assert F.omega(pr, int(s)) == pow(F.omega_k(pr, int(j)), int(e),
                                               pr.p)


def test_root_values_match_c_oracle():
    # Python and C compute the convention independently.
    for pr in PRIMES:
        for k in range(pr.K + 1):
            assert NV.omega_k(pr, k) == F.omega_k(pr, k)
        for s in (0, 1, 2, 3, 5, 1000, 123456, (1 << pr.K) - 1):
            assert NV.omega(pr, s) == F.omega(pr, s)


# --------------------------------------------------------------------------
# Section 3: the tree (Figure 1)
# --------------------------------------------------------------------------

def test_figure1_tree_n6():
    rows = []
    for line in open(os.path.join(GOLDEN, "fig1_tree_n6.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        left, right = line.split(":")
        q, r = map(int, left.split())
        rows.append(((q, r), [int(v) for v in right.split()]))
    t = T.Tree(6)
    for S, idx in rows:
        assert t.indices(S) == idx, S
        assert t.is_leaf(S) == (len(idx) == 1)
    # the figure's edges: each internal node's children are Even and Odd
    table = dict(rows)
    for S, idx in rows:
        if len(idx) > 1:
            assert t.even(S) in table and t.odd(S) in table
            assert sorted(table[t.even(S)] + table[t.odd(S)]) == idx
            assert t.parent(t.even(S)) == S and t.parent(t.odd(S)) == S
    assert t.leftmost_leaf((0, 0)) == (0, 3)
    # Section 4: Parent(RP(N2)) = N1 when LeftmostLeaf(Odd(N1)) = N2
    for S, idx in rows:
        if len(idx) > 1:
            N2 = t.leftmost_leaf(t.odd(S))
            assert t.parent(t.rightmost_parent(N2)) == S


@pytest.mark.parametrize("n", [1, 2, 3, 6, 7, 11, 16, 33, 100, 257])
def test_rightmost_parent_inverts_descent(n):
    t = T.Tree(n)
    stack = [(0, 0)]
    while stack:
        S = stack.pop()
        if t.is_leaf(S):
            continue
        N2 = t.leftmost_leaf(t.odd(S))
        assert t.parent(t.rightmost_parent(N2)) == S
        stack += [t.even(S), t.odd(S)]


# --------------------------------------------------------------------------
# Algorithms 1 and 2 against the definition
# --------------------------------------------------------------------------

@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_alg1_equals_definition_all_n_le_64(pr):
    # Proposition 3.2 vs the definition, every n <= 64, three seeds.
    for seed in range(3):
        rng = random.Random(1000 * seed + pr.K)
        for n in range(1, 65):
            x = _rand_vec(rng, pr, n)
            assert T.alg1_tft(pr, x) == T.naive_tft(pr, x), (seed, n)


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_alg2_equals_gaussian_elimination(pr):
    # Proposition 4.2 vs solving the Vandermonde system directly.
    rng = random.Random(7 + pr.K)
    sizes = list(range(1, 33)) + [40, 47, 64]
    for n in sizes:
        X = _rand_vec(rng, pr, n)
        assert T.alg2_itft(pr, X) == T.naive_itft(pr, X), n


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_power_of_two_is_the_textbook_fft(pr):
    # n = 2^k: Algorithm 1 == definition == textbook radix-2 FFT (Section 1).
    rng = random.Random(3)
    for k in range(0, 8):
        x = _rand_vec(rng, pr, 1 << k)
        ref = T.fft_pow2(pr, x)
        assert T.naive_tft(pr, x) == ref
        assert T.alg1_tft(pr, x) == ref
    for k in (10, 12, 14):
        x = np.array(_rand_vec(rng, pr, 1 << k), dtype=np.uint64)
        assert (NV.alg1_tft(pr, x) == NV.fft_pow2(pr, x)).all()
        assert (NV.fft_pow2(pr, x) ==
                np.array(T.fft_pow2(pr, [int(v) for v in x]),
                         dtype=np.uint64)).all()


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_truncation_of_padded_fft(pr):
    # Section 1.2: the TFT of length n <= 2^k is the first n outputs of the
    # length-2^k FFT of the zero-padded input, for any admissible k.
    rng = random.Random(11)
    for n in [1, 2, 3, 5, 9, 31, 33, 63, 65, 100, 129, 255]:
        x = _rand_vec(rng, pr, n)
        mine = T.alg1_tft(pr, x)
        k0 = max(0, (n - 1).bit_length())
        for k in (k0, k0 + 1, k0 + 2):
            padded = T.fft_pow2(pr, x + [0] * ((1 << k) - n))
            assert mine == padded[:n], (n, k)
    for n in [1000, 3001, 4097, 12345]:
        x = np.array(_rand_vec(rng, pr, n), dtype=np.uint64)
        k = (n - 1).bit_length()
        padded = np.zeros(1 << k, dtype=np.uint64)
        padded[:n] = x
        assert (NV.alg1_tft(pr, x) == NV.fft_pow2(pr, padded)[:n]).all()


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_roundtrip_every_n_up_to_4096(pr):
    # Proposition 4.2: ITFT(TFT(x)) = x for every n <= 2^12 (C oracle), and
    # the C and Python oracles agree bit for bit on n <= 48 and a sample of
    # larger n.
    rng = np.random.default_rng(pr.K)
    for n in range(1, 4097):
        x = rng.integers(0, pr.p, n, dtype=np.uint64)
        X = NV.alg1_tft(pr, x)
        assert (NV.alg2_itft(pr, X) == x).all(), n
        if n <= 48 or (n <= 600 and n % 97 == 0):
            xl = [int(v) for v in x]
            assert [int(v) for v in X] == T.alg1_tft(pr, xl), n
            assert T.alg2_itft(pr, [int(v) for v in X]) == xl, n


@pytest.mark.slow
@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_roundtrip_random_large_n(pr):
    rng = np.random.default_rng(99 + pr.K)
    for n in [5000, 65537, 100003, (1 << 20) + 1, 3 * (1 << 19) - 7]:
        x = rng.integers(0, pr.p, n, dtype=np.uint64)
        X = NV.alg1_tft(pr, x)
        assert (NV.alg2_itft(pr, X) == x).all(), n
        # the definition at sampled points (Horner, O(n) each)
        s = rng.integers(0, n, 6, dtype=np.uint64)
        s[0], s[1] = 0, n - 1
        assert (NV.eval_tft_points(pr, x, s) == X[s.astype(np.int64)]).all()


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_linearity(pr):
    # The TFT is a linear map (Section 1.1, the DFT is linear).
    rng = random.Random(5)
    p = pr.p
    for n in [1, 7, 30, 64, 99]:
        x, y = _rand_vec(rng, pr, n), _rand_vec(rng, pr, n)
        al, be = rng.randrange(p), rng.randrange(p)
        z = [(al * u + be * v) % p for u, v in zip(x, y)]
        X, Y, Z = T.alg1_tft(pr, x), T.alg1_tft(pr, y), T.alg1_tft(pr, z)
        assert Z == [(al * u + be * v) % p for u, v in zip(X, Y)]


def test_corrections_are_needed():
    # A plain pruned radix-2 network without the odd-length correction is
    # NOT the TFT for odd node lengths: dropping line "S_{m-1} += v w_{m-1}"
    # must break agreement with the definition (guards against a silent
    # no-op correction).
    pr = F.P998244353
    rng = random.Random(0)
    x = _rand_vec(rng, pr, 7)
    good = T.alg1_tft(pr, x)
    assert good == T.naive_tft(pr, x)
    saved = T._odd_child_value
    try:
        T._odd_child_value = lambda *a: 0
        bad = T.alg1_tft(pr, x)
    finally:
        T._odd_child_value = saved
    assert bad != good


# --------------------------------------------------------------------------
# Proposition 3.2 and Section 4: the walk
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 8, 13, 31, 64, 100, 333])
def test_visit_counts_and_reverse_path(n):
    t = T.Tree(n)
    internal = leaves = 0
    stack = [(0, 0)]
    while stack:
        S = stack.pop()
        if t.is_leaf(S):
            leaves += 1
        else:
            internal += 1
            stack += [t.even(S), t.odd(S)]
    assert leaves == n
    pr = F.P2013265921
    x = list(range(1, n + 1))
    trace, ev1, ev2 = [], [], []
    X = T.alg1_tft(pr, x, trace=trace, events=ev1)
    # Proposition 3.2: each leaf once, each internal node twice
    assert len(trace) == leaves + 2 * internal
    from collections import Counter
    c = Counter(trace)
    assert all(c[S] == (1 if t.is_leaf(S) else 2) for S in c)
    # Section 4: the ITFT's path is the exact reverse of the TFT's
    T.alg2_itft(pr, X, events=ev2)
    assert ev2 == list(reversed(ev1))


@pytest.mark.parametrize("n", list(range(1, 70)) + [1000, 4096, 5000])
def test_butterfly_count(n):
    # The multiply count used by the roofline equals the number of
    # butterflies Algorithm 1 actually performs; (n/2) k at n = 2^k.
    t = T.Tree(n)
    total = 0
    stack = [(0, 0)]
    while stack:
        S = stack.pop()
        if not t.is_leaf(S):
            total += t.len(S) // 2
            stack += [t.even(S), t.odd(S)]
    assert T.butterfly_multiplies(n) == total
    if n & (n - 1) == 0:
        assert total == (n // 2) * (n.bit_length() - 1)


# --------------------------------------------------------------------------
# Section 5: products
# --------------------------------------------------------------------------

@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_tft_polymul_equals_schoolbook_small(pr):
    rng = random.Random(17)
    for na in range(1, 13):
        for nb in range(1, 13):
            a, b = _rand_vec(rng, pr, na), _rand_vec(rng, pr, nb)
            assert T.tft_polymul(pr, a, b) == T.schoolbook(pr, a, b)


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_tft_polymul_equals_schoolbook_all_sizes_to_64(pr):
    # every (na, nb) <= 64 through the C oracle
    rng = np.random.default_rng(23)
    for na in range(1, 65):
        for nb in range(1, 65):
            a = rng.integers(0, pr.p, na, dtype=np.uint64)
            b = rng.integers(0, pr.p, nb, dtype=np.uint64)
            assert (NV.tft_polymul(pr, a, b) ==
                    NV.schoolbook(pr, a, b)).all(), (na, nb)
    # C and Python agree
    a = [int(v) for v in rng.integers(0, pr.p, 37, dtype=np.uint64)]
    b = [int(v) for v in rng.integers(0, pr.p, 29, dtype=np.uint64)]
    assert [int(v) for v in NV.tft_polymul(pr, a, b)] == \
        T.tft_polymul(pr, a, b)


def _exact_product(a, b, p):
    # numpy's convolution over Python integers (object arrays): the exact
    # integer product of the two polynomials, reduced mod p afterwards.
    c = np.convolve(np.array([int(v) for v in a], dtype=object),
                    np.array([int(v) for v in b], dtype=object))
    return [int(v) % p for v in c]


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_conv_coeff_every_t_all_sizes_to_64(pr):
    # orc_conv_coeff, the per-coefficient checker of the full-size GPU
    # product tests: c_t = sum_i a_i b_{t-i} over the index pairs inside
    # both operands (Section 5's product), for every t of every
    # (na, nb) <= 64, against numpy's exact integer convolution; positions
    # at and past r = na + nb - 1 are zero.  The first and last terms of the
    # sum (lo and hi) are exercised by t = 0, t < min(na, nb), t in the
    # middle band and t > max(na, nb).
    rng = np.random.default_rng(53)
    for na in range(1, 65):
        for nb in range(1, 65):
            a = rng.integers(0, pr.p, na, dtype=np.uint64)
            b = rng.integers(0, pr.p, nb, dtype=np.uint64)
            want = _exact_product(a, b, pr.p)
            got = [NV.conv_coeff(pr, a, b, t) for t in range(na + nb + 1)]
            assert got == want + [0, 0], (na, nb)


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_conv_coeff_random_t_large(pr):
    rng = np.random.default_rng(59)
    for na, nb in ((4096, 3), (1, 4096), (2500, 4096), (4096, 4096),
                   (3001, 1777)):
        a = rng.integers(0, pr.p, na, dtype=np.uint64)
        b = rng.integers(0, pr.p, nb, dtype=np.uint64)
        want = _exact_product(a, b, pr.p)
        r = na + nb - 1
        ts = {0, 1, na - 1, na, nb - 1, nb, r - 2, r - 1} | \
            {int(t) for t in rng.integers(0, r, 40)}
        for t in sorted(x for x in ts if 0 <= x < r):
            assert NV.conv_coeff(pr, a, b, t) == want[t], (na, nb, t)


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_tft_polymul_random_sizes(pr):
    rng = np.random.default_rng(31)
    for _ in range(6):
        na, nb = (int(v) for v in rng.integers(1, 4097, 2))
        a = rng.integers(0, pr.p, na, dtype=np.uint64)
        b = rng.integers(0, pr.p, nb, dtype=np.uint64)
        assert (NV.tft_polymul(pr, a, b) == NV.schoolbook(pr, a, b)).all()


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_product_through_any_longer_tft_length(pr):
    # Section 1.2: a polynomial of degree < n' is determined by its TFT of
    # length n' (the transform is invertible), so the product of degree < r
    # comes out of transforms of any length n' >= r -- the GPU product runs
    # them at r rounded up to a multiple of its row length.  The inverse of
    # the pointwise product returns the r product coefficients followed by
    # n' - r zeros; a length below r loses information.
    rng = np.random.default_rng(37)
    for na, nb in ((5, 9), (100, 157), (300, 4), (513, 512)):
        a = rng.integers(0, pr.p, na, dtype=np.uint64)
        b = rng.integers(0, pr.p, nb, dtype=np.uint64)
        r = na + nb - 1
        want = [int(v) for v in NV.schoolbook(pr, a, b)]
        for n2 in sorted({r, r + 1, r + 37, -(-r // 64) * 64,
                          1 << (r - 1).bit_length()}):
            A = NV.alg1_tft(pr, np.concatenate(
                [a, np.zeros(n2 - na, dtype=np.uint64)]))
            B = NV.alg1_tft(pr, np.concatenate(
                [b, np.zeros(n2 - nb, dtype=np.uint64)]))
            Cp = np.array([int(x) * int(y) % pr.p for x, y in zip(A, B)],
                          dtype=np.uint64)
            c = [int(v) for v in NV.alg2_itft(pr, Cp)]
            assert c[:r] == want and c[r:] == [0] * (n2 - r), (na, nb, n2)
        # one position short of r: the top coefficient is lost
        n2 = r - 1
        if n2 >= max(na, nb):
            A = NV.alg1_tft(pr, np.concatenate(
                [a, np.zeros(n2 - na, dtype=np.uint64)]))
            B = NV.alg1_tft(pr, np.concatenate(
                [b, np.zeros(n2 - nb, dtype=np.uint64)]))
            Cp = np.array([int(x) * int(y) % pr.p for x, y in zip(A, B)],
                          dtype=np.uint64)
            assert [int(v) for v in NV.alg2_itft(pr, Cp)] != want[:n2]


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_polymul_random_point_large(pr):
    # Schwartz-Zippel: C(z) = A(z) B(z) at random z, independent of the TFT.
    rng = np.random.default_rng(41)
    na, nb = 70001, 50000
    a = rng.integers(0, pr.p, na, dtype=np.uint64)
    b = rng.integers(0, pr.p, nb, dtype=np.uint64)
    c = NV.tft_polymul(pr, a, b)
    for z in rng.integers(2, pr.p - 1, 4, dtype=np.uint64):
        lhs = NV.eval_at(pr, c, int(z))
        rhs = NV.eval_at(pr, a, int(z)) * NV.eval_at(pr, b, int(z)) % pr.p
        assert lhs == rhs


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_alg3_product_and_invariants(pr):
    # Proposition 5.1: Algorithm 3 computes AB; the intervals [q_i, q_i+L_i)
    # partition [0, r-1); L_i | q_i; each L appears at most twice; the loop
    # runs at most 2 lg r times.
    rng = random.Random(43)
    for m in list(range(1, 10)) + [17, 64, 100]:
        for n in (1, 2, 5, 31, 64, 77):
            A, B = _rand_vec(rng, pr, m), _rand_vec(rng, pr, n)
            tr = []
            assert T.alg3_polymul(pr, A, B, trace=tr) == \
                T.schoolbook(pr, A, B)
            r = m + n - 1
            covered = []
            for q, L in tr:
                assert q % L == 0
                assert q + 2 * L <= r
                covered += list(range(q, q + L))
            assert covered == list(range(r - 1))
            Ls = [L for _, L in tr]
            assert all(Ls.count(L) <= 2 for L in set(Ls))
            if r > 1:
                assert len(tr) <= 2 * (r.bit_length())


def test_config1_product_golden():
    # tests/golden/config1_product.txt is written by tests/golden/make_golden.py
    # from the oracle's schoolbook product (no GPU path involved).
    from workloads import config1_inputs
    a, b, _ = config1_inputs()
    ref = [int(l) for l in open(os.path.join(GOLDEN, "config1_product.txt"))
           if l.strip() and not l.startswith("#")]
    assert len(ref) == 999
    assert T.schoolbook(F.P998244353, [int(v) for v in a],
                        [int(v) for v in b]) == ref
    assert [int(v) for v in NV.tft_polymul(F.P998244353, a, b)] == ref
