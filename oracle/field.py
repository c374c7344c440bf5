"""Rings Z/p and compatible roots of unity (oracle; test infrastructure only).

Section 2.1 asks for a ring R in which 2 is not a zero-divisor and that holds
2^k-th roots of unity for every k needed.  We instantiate R = Z/p for three
primes p = c*2^K + 1.  Section 2.2 asks for primitive 2^k-th roots omega_[k]
chosen compatibly, omega_[k+1]^2 = omega_[k]; the paper does not say which
ones.  Reading adopted here: omega_[K] = g^((p-1)/2^K) for the generator g
listed below, and omega_[k] = omega_[K]^(2^(K-k)) for k <= K.  The product of
two polynomials does not depend on this choice; transform values do.

Everything is plain Python integers reduced with ``%``.
"""

from dataclasses import dataclass


@dataclass(frozen=True)
class Prime:
    name: str
    p: int          # the modulus
    K: int          # two-adicity: 2^K divides p - 1
    g: int          # a generator of (Z/p)^*
    odd_factors: tuple  # distinct odd prime factors of p - 1 (for checking g)
    word_bits: int  # storage width of one element (32 or 64)


P998244353 = Prime("p998244353", 998244353, 23, 3, (7, 17), 32)
P2013265921 = Prime("p2013265921", 2013265921, 27, 31, (3, 5), 32)
PGOLDILOCKS = Prime("goldilocks", 2**64 - 2**32 + 1, 32, 7,
                    (3, 5, 17, 257, 65537), 64)

PRIMES = {pr.name: pr for pr in (P998244353, P2013265921, PGOLDILOCKS)}
# Integer ids shared, as plain numbers, with the C library's enum (0, 1, 2).
PRIME_BY_ID = (P998244353, P2013265921, PGOLDILOCKS)


def get(prime):
    """Accept a Prime, its name, its integer id or its modulus."""
    if isinstance(prime, Prime):
        return prime
    if isinstance(prime, str):
        return PRIMES[prime]
    if isinstance(prime, int):
        if prime in (0, 1, 2):
            return PRIME_BY_ID[prime]
        for pr in PRIME_BY_ID:
            if pr.p == prime:
                return pr
    raise KeyError(prime)


def rev(s, k):
    """Length-k bit reversal rev_k(s) of Section 2.2 (requires s < 2^k)."""
    assert 0 <= s < (1 << k)
    out = 0
    for _ in range(k):
        out = (out << 1) | (s & 1)
        s >>= 1
    return out


def omega_k(prime, k):
    """omega_[k]: the compatible primitive 2^k-th root of unity (Section 2.2)."""
    pr = get(prime)
    if not 0 <= k <= pr.K:
        raise ValueError(f"k={k} exceeds the two-adicity {pr.K} of {pr.name}")
    top = pow(pr.g, (pr.p - 1) >> pr.K, pr.p)      # omega_[K]
    return pow(top, 1 << (pr.K - k), pr.p)


def omega(prime, s):
    """omega_s = omega_[K]^(rev_K s) (Section 2.2).

    The paper allows any k >= ceil(lg(s+1)); with compatible roots the value
    does not depend on k, and we use k = K.
    """
    pr = get(prime)
    return pow(omega_k(pr, pr.K), rev(s, pr.K), pr.p)


def inv(prime, a):
    pr = get(prime)
    if a % pr.p == 0:
        raise ZeroDivisionError("0 has no inverse")
    return pow(a, pr.p - 2, pr.p)


def is_primitive_root(prime):
    """g generates (Z/p)^*: g^((p-1)/f) != 1 for every prime f | p-1."""
    pr = get(prime)
    for f in (2,) + tuple(pr.odd_factors):
        if pow(pr.g, (pr.p - 1) // f, pr.p) == 1:
            return False
    return True
