"""Oracle transforms and products (test infrastructure only).

Plain Python integers; every list is a list of ints in [0, p).  Each function
names the passage of Harvey & Roche (2010) it follows.

Definitions (written out, O(n^2)):
  naive_tft      F^_s = F(omega_s) for 0 <= s < n           (Section 2.2)
  naive_itft     solve the n x n system V[s][j] = omega_s^j by Gaussian
                 elimination mod p (the inverse map, Section 4's output)
  eval_at        Horner evaluation F(z)
  schoolbook     c_t = sum_i a_i b_{t-i}

Algorithms (the paper's steps, in its order and notation):
  alg1_tft       Algorithm 1, InplaceTFT (Section 3)
  alg2_itft      Algorithm 2, InplaceITFT (Section 4)
  fft_pow2       a textbook radix-2 FFT, natural order in, bit-reversed
                 order out: the FFT subroutine of Algorithm 3 (Section 5)
  tft_polymul    TFT of both operands, pointwise product, ITFT (Section 1.2
                 and the first paragraph of Section 5)
  alg3_polymul   Algorithm 3, the space-restricted product (Section 5)
"""

from . import field as _f


# ----------------------------------------------------------------------------
# Definitions
# ----------------------------------------------------------------------------

def eval_at(prime, coeffs, z):
    """F(z) by Horner's rule."""
    p = _f.get(prime).p
    acc = 0
    for c in reversed(coeffs):
        acc = (acc * z + c) % p
    return acc


def naive_tft(prime, x):
    """F^_s = F(omega_s) for s < n, the definition of Section 2.2."""
    n = len(x)
    return [eval_at(prime, x, _f.omega(prime, s)) for s in range(n)]


def naive_itft(prime, X):
    """Inverse of naive_tft by Gaussian elimination mod p (small n only).

    Solves sum_j omega_s^j F_j = X_s for s < n.  The points omega_s, s < n,
    are distinct (distinct bit reversals of a primitive root's exponent), so
    the Vandermonde matrix is invertible.
    """
    pr = _f.get(prime)
    p = pr.p
    n = len(X)
    rows = []
    for s in range(n):
        w = _f.omega(pr, s)
        rows.append([pow(w, j, p) for j in range(n)] + [X[s] % p])
    for col in range(n):
        piv = next(r for r in range(col, n) if rows[r][col] % p)
        rows[col], rows[piv] = rows[piv], rows[col]
        inv = pow(rows[col][col], p - 2, p)
        rows[col] = [(v * inv) % p for v in rows[col]]
        for r in range(n):
            if r != col and rows[r][col]:
                f = rows[r][col]
                rows[r] = [(a - f * b) % p for a, b in zip(rows[r], rows[col])]
    return [rows[j][n] for j in range(n)]


def schoolbook(prime, a, b):
    """c_t = sum_i a_i b_{t-i} mod p; length len(a) + len(b) - 1."""
    p = _f.get(prime).p
    out = [0] * (len(a) + len(b) - 1)
    for i, ai in enumerate(a):
        if ai:
            for j, bj in enumerate(b):
                out[i + j] = (out[i + j] + ai * bj) % p
    return out


# ----------------------------------------------------------------------------
# The implicit recursion tree of Section 3 (Figure 1)
# ----------------------------------------------------------------------------

class Tree:
    """Node S = (q, r): offset q, stride 2^r, S_i = X_{q + i 2^r} (Section 3)."""

    def __init__(self, n):
        if n < 1:
            raise ValueError("the tree needs n >= 1")
        self.n = n

    def len(self, S):
        q, r = S
        return -(-(self.n - q) // (1 << r))          # ceil((n - q) / 2^r)

    def is_leaf(self, S):
        return self.len(S) == 1

    def even(self, S):
        q, r = S
        return (q, r + 1)

    def odd(self, S):
        q, r = S
        return (q + (1 << r), r + 1)

    def parent(self, S):
        q, r = S
        half = 1 << (r - 1)
        return (q, r - 1) if q < half else (q - half, r - 1)

    def leftmost_leaf(self, S):
        while not self.is_leaf(S):
            S = self.even(S)
        return S

    def rightmost_parent(self, S):
        # Section 4: RP(S) = S if S = Odd(Parent(S)), else RP(Parent(S)).
        while S != self.odd(self.parent(S)):
            S = self.parent(S)
        return S

    def indices(self, S):
        q, r = S
        return [q + i * (1 << r) for i in range(self.len(S))]


# ----------------------------------------------------------------------------
# Algorithm 1 and Algorithm 2
# ----------------------------------------------------------------------------

def _butterfly_roots(pr, m, inverse):
    """The pairs (j, omega_{2j}) (or omega_{2j}^{-1}), 0 <= j < floor(m/2)."""
    for j in range(m // 2):
        w = _f.omega(pr, 2 * j)
        yield j, (_f.inv(pr, w) if inverse else w)


def _odd_child_value(pr, X, tree, S, m):
    """v = sum_{i=0}^{(m-3)/2} S_{2i+1} (omega_{(m-1)/2})^i (Alg. 1 and 2)."""
    q, r = S
    z = _f.omega(pr, (m - 1) // 2)
    v = 0
    zi = 1
    for i in range((m - 3) // 2 + 1):
        v = (v + X[q + (2 * i + 1) * (1 << r)] * zi) % pr.p
        zi = (zi * z) % pr.p
    return v


def alg1_tft(prime, x, trace=None, events=None):
    """InplaceTFT, Algorithm 1 (Section 3), on a copy of x.

    If ``trace`` is a list, the node S at the top of every while-loop
    iteration is appended to it (pins the visit counts of Proposition 3.2).
    If ``events`` is a list, ("bfly", S) is appended whenever a node with
    len(S) >= 2 runs its butterfly loop and ("corr", S) whenever the
    odd-length correction runs (pins the reverse-path claim of Section 4).
    """
    pr = _f.get(prime)
    p = pr.p
    X = [v % p for v in x]
    n = len(X)
    if n == 0:
        raise ValueError("InplaceTFT needs n >= 1")
    t = Tree(n)
    S = t.leftmost_leaf((0, 0))
    prev = None
    while True:
        if trace is not None:
            trace.append(S)
        m = t.len(S)
        q, r = S
        step = 1 << r
        if t.is_leaf(S) or prev == t.odd(S):
            if events is not None and m >= 2:
                events.append(("bfly", S))
            for i, theta in _butterfly_roots(pr, m, inverse=False):
                a = X[q + 2 * i * step]
                b = X[q + (2 * i + 1) * step]
                X[q + 2 * i * step] = (a + theta * b) % p
                X[q + (2 * i + 1) * step] = (a - theta * b) % p
            if S == (0, 0):
                return X
            prev = S
            S = t.parent(S)
        elif prev == t.even(S):
            if m % 2 == 1:
                if events is not None:
                    events.append(("corr", S))
                v = _odd_child_value(pr, X, t, S, m)
                last = q + (m - 1) * step
                X[last] = (X[last] + v * _f.omega(pr, m - 1)) % p
            prev = S
            S = t.leftmost_leaf(t.odd(S))
        else:  # pragma: no cover - Lemma 3.1 rules this out
            raise AssertionError("unreachable state in Algorithm 1")


def alg2_itft(prime, X_hat, trace=None, events=None):
    """InplaceITFT, Algorithm 2 (Section 4), on a copy of X_hat.

    Division by 2 is exact in Z/p: a/2 = a * (p+1)/2.  ``trace`` and
    ``events`` record the walk as in alg1_tft.
    """
    pr = _f.get(prime)
    p = pr.p
    half = (p + 1) // 2
    X = [v % p for v in X_hat]
    n = len(X)
    if n == 0:
        raise ValueError("InplaceITFT needs n >= 1")
    t = Tree(n)
    S = (0, 0)
    stop = t.leftmost_leaf((0, 0))
    while S != stop:
        if trace is not None:
            trace.append(S)
        if t.is_leaf(S):
            S = t.parent(t.rightmost_parent(S))
            m = t.len(S)
            q, r = S
            if m % 2 == 1:
                if events is not None:
                    events.append(("corr", S))
                v = _odd_child_value(pr, X, t, S, m)
                last = q + (m - 1) * (1 << r)
                X[last] = (X[last] - v * _f.omega(pr, m - 1)) % p
            S = t.even(S)
        else:
            m = t.len(S)
            q, r = S
            step = 1 << r
            if events is not None:
                events.append(("bfly", S))
            for i, theta in _butterfly_roots(pr, m, inverse=True):
                a = X[q + 2 * i * step]
                b = X[q + (2 * i + 1) * step]
                X[q + 2 * i * step] = ((a + b) * half) % p
                X[q + (2 * i + 1) * step] = (theta * (a - b) * half) % p
            S = t.odd(S)
    if trace is not None:
        trace.append(S)
    return X


# ----------------------------------------------------------------------------
# Textbook FFT (natural order in, bit-reversed order out)
# ----------------------------------------------------------------------------

def fft_pow2(prime, x):
    """Radix-2 decimation-in-frequency FFT of length N = 2^k.

    The textbook Gentleman-Sande loop with twiddles in natural order: after
    it, position s holds sum_i x_i w^(i * rev_k(s)) with w = omega_[k], which
    Section 2.2 writes as F(omega_s).  This is the FFT subroutine that
    Algorithm 3 calls (same interface as the TFT, power-of-two lengths).
    """
    pr = _f.get(prime)
    p = pr.p
    X = [v % p for v in x]
    N = len(X)
    k = N.bit_length() - 1
    if N != 1 << k:
        raise ValueError("fft_pow2 needs a power-of-two length")
    length = N // 2
    while length >= 1:
        w_len = _f.omega_k(pr, (2 * length).bit_length() - 1)  # 2len-th root
        for start in range(0, N, 2 * length):
            w = 1
            for j in range(length):
                u = X[start + j]
                v = X[start + j + length]
                X[start + j] = (u + v) % p
                X[start + j + length] = ((u - v) * w) % p
                w = (w * w_len) % p
        length //= 2
    return X


# ----------------------------------------------------------------------------
# Products
# ----------------------------------------------------------------------------

def tft_polymul(prime, a, b):
    """C = A B through the TFT: zero-extend both operands to r = len(a) +
    len(b) - 1, InplaceTFT both, multiply pointwise (C^_s = A^_s B^_s), then
    InplaceITFT (Sections 1.2 and 5)."""
    p = _f.get(prime).p
    if not a or not b:
        raise ValueError("empty operand")
    r = len(a) + len(b) - 1
    A = alg1_tft(prime, list(a) + [0] * (r - len(a)))
    B = alg1_tft(prime, list(b) + [0] * (r - len(b)))
    return alg2_itft(prime, [(u * v) % p for u, v in zip(A, B)])


def alg3_polymul(prime, A, B, trace=None):
    """Algorithm 3, the space-restricted product (Section 5).

    Follows the names of the algorithm box: deg A < m, deg B < n, output
    buffer X of length r = n + m - 1.  If ``trace`` is a list, each loop
    iteration appends (q, L).
    """
    pr = _f.get(prime)
    p = pr.p
    m, n = len(A), len(B)
    if m == 0 or n == 0:
        raise ValueError("empty operand")
    r = n + m - 1
    X = [0] * r
    q = 0
    while q < r - 1:
        ell = (r - q).bit_length() - 1 - 1          # floor(lg(r - q)) - 1
        L = 1 << ell
        if trace is not None:
            trace.append((q, L))
        for i in range(2 * L):
            X[q + i] = 0
        wq = _f.omega(pr, q)
        wi = 1
        for i in range(m):
            X[q + i % L] = (X[q + i % L] + wi * A[i]) % p
            wi = (wi * wq) % p
        X[q:q + L] = fft_pow2(pr, X[q:q + L])
        wi = 1
        for i in range(n):
            X[q + L + i % L] = (X[q + L + i % L] + wi * B[i]) % p
            wi = (wi * wq) % p
        X[q + L:q + 2 * L] = fft_pow2(pr, X[q + L:q + 2 * L])
        for i in range(L):
            X[q + i] = (X[q + i] * X[q + L + i]) % p
        q += L
    w_last = _f.omega(pr, r - 1)
    X[r - 1] = (eval_at(pr, A, w_last) * eval_at(pr, B, w_last)) % p
    return alg2_itft(pr, X)


def butterfly_multiplies(n):
    """Number of butterflies (one twiddle multiply each) that Algorithm 1
    performs for length n: sum over the internal nodes of floor(len/2).

    Equivalently, summed per level r of the tree, sum_{q < 2^r} floor(len(q,r)/2).
    This is the algorithmic multiply count used by the roofline (corrections
    are overhead and are not counted).
    """
    total = 0
    r = 0
    while (1 << r) < n:
        step = 1 << r
        # nodes (q, r) for q < min(2^r, n)
        full, rem = divmod(n, step)
        # len(q, r) = full + 1 for q < rem, full otherwise
        total += rem * ((full + 1) // 2) + (step - rem) * (full // 2)
        r += 1
    return total
