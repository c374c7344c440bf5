/*
 * Oracle, plain C (test infrastructure only; never linked into the library).
 *
 * The same definitions and algorithms as oracle/tft.py, for sizes that the
 * Python loops cannot reach in seconds.  Every element is stored in a
 * uint64_t whatever the prime; every product is reduced with
 * (unsigned __int128)a * b % p.  No Montgomery form, no special reduction,
 * no tables: roots are computed by modular exponentiation or, inside the
 * butterfly loops, by the bit-reversed counter that Section 2.2 describes.
 *
 *   orc_alg1_tft     Algorithm 1 (InplaceTFT), Section 3
 *   orc_alg2_itft    Algorithm 2 (InplaceITFT), Section 4
 *   orc_tft_polymul  zero-extend, Algorithm 1 twice, pointwise, Algorithm 2
 *                    (Sections 1.2 and 5)
 *   orc_eval         F(z) by Horner
 *   orc_eval_tft_points   F(omega_s) for chosen s (the definition, Sec. 2.2)
 *   orc_schoolbook   c_t = sum_i a_i b_{t-i}
 *   orc_conv_coeff   one coefficient c_t of the product, by that sum
 *   orc_fft_pow2     textbook radix-2 DIF FFT, natural in, bit-reversed out
 *
 * Prime ids: 0 -> 998244353 (g = 3), 1 -> 2013265921 (g = 31),
 * 2 -> 2^64 - 2^32 + 1 (g = 7); omega_[K] = g^((p-1)/2^K) with K the
 * two-adicity (23, 27, 32).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

typedef struct {
    uint64_t p;
    int K;
    uint64_t g;
} orc_prime;

static const orc_prime PRIMES[3] = {
    {998244353ull, 23, 3},
    {2013265921ull, 27, 31},
    {0xFFFFFFFF00000001ull, 32, 7},
};

static int valid_id(int id) { return id >= 0 && id < 3; }

static uint64_t mulm(uint64_t a, uint64_t b, uint64_t p) {
    return (uint64_t)(((u128)a * b) % p);
}
static uint64_t addm(uint64_t a, uint64_t b, uint64_t p) {
    return (uint64_t)(((u128)a + b) % p);
}
static uint64_t subm(uint64_t a, uint64_t b, uint64_t p) {
    return (uint64_t)(((u128)a + p - b) % p);
}
static uint64_t powm(uint64_t a, uint64_t e, uint64_t p) {
    uint64_t r = 1 % p;
    a %= p;
    while (e) {
        if (e & 1) r = mulm(r, a, p);
        a = mulm(a, a, p);
        e >>= 1;
    }
    return r;
}
static uint64_t invm(uint64_t a, uint64_t p) { return powm(a, p - 2, p); }

static uint64_t rev_bits(uint64_t s, int k) {
    uint64_t out = 0;
    for (int i = 0; i < k; i++) {
        out = (out << 1) | (s & 1);
        s >>= 1;
    }
    return out;
}

/* omega_[k] = omega_[K]^(2^(K-k)). */
static uint64_t omega_k(const orc_prime *pr, int k) {
    uint64_t top = powm(pr->g, (pr->p - 1) >> pr->K, pr->p);
    for (int i = 0; i < pr->K - k; i++) top = mulm(top, top, pr->p);
    return top;
}

/* omega_s = omega_[K]^(rev_K s), Section 2.2. */
static uint64_t omega_s(const orc_prime *pr, uint64_t s) {
    return powm(omega_k(pr, pr->K), rev_bits(s, pr->K), pr->p);
}

uint64_t orc_omega(int id, uint64_t s) {
    if (!valid_id(id)) return 0;
    return omega_s(&PRIMES[id], s);
}

uint64_t orc_omega_k(int id, int k) {
    if (!valid_id(id) || k < 0 || k > PRIMES[id].K) return 0;
    return omega_k(&PRIMES[id], k);
}

/* ------------------------------------------------------------------------ */
/* The implicit tree of Section 3: S = (q, r), S_i = X[q + i 2^r].           */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t q;
    int r;
} node;

static uint64_t node_len(uint64_t n, node S) {
    uint64_t step = (uint64_t)1 << S.r;
    return (n - S.q + step - 1) >> S.r;
}
static int is_leaf(uint64_t n, node S) { return node_len(n, S) == 1; }
static node even_child(node S) { node c = {S.q, S.r + 1}; return c; }
static node odd_child(node S) {
    node c = {S.q + ((uint64_t)1 << S.r), S.r + 1};
    return c;
}
static node parent_of(node S) {
    uint64_t half = (uint64_t)1 << (S.r - 1);
    node c;
    c.r = S.r - 1;
    c.q = S.q < half ? S.q : S.q - half;
    return c;
}
static int same(node a, node b) { return a.q == b.q && a.r == b.r; }
static node leftmost_leaf(uint64_t n, node S) {
    while (!is_leaf(n, S)) S = even_child(S);
    return S;
}
static node rightmost_parent(node S) {
    while (!same(S, odd_child(parent_of(S)))) S = parent_of(S);
    return S;
}

/* Butterflies over the pairs (S_2j, S_2j+1) with theta = omega_2j (or its
 * inverse times 1/2), j < floor(m/2).  The roots are produced the way
 * Section 2.2 describes: powers of omega_[t+1] in natural order while the
 * index runs through a t-bit bit-reversed counter, where 2^t >= floor(m/2).
 * (omega_2j = omega_[t+1]^(rev_t j) for j < 2^t.) */
static void butterflies(const orc_prime *pr, uint64_t *X, node S, uint64_t m,
                        int inverse) {
    const uint64_t p = pr->p;
    uint64_t h = m / 2;
    if (h == 0) return;
    int t = 0;
    while (((uint64_t)1 << t) < h) t++;
    uint64_t base = omega_k(pr, t + 1);
    if (inverse) base = invm(base, p);
    const uint64_t half = (p + 1) / 2;
    const uint64_t step = (uint64_t)1 << S.r;
    uint64_t w = 1;  /* base^e */
    uint64_t j = 0;  /* rev_t(e) */
    uint64_t count = (uint64_t)1 << t;
    for (uint64_t e = 0; e < count; e++) {
        if (j < h) {
            uint64_t ia = S.q + 2 * j * step, ib = ia + step;
            uint64_t a = X[ia], b = X[ib];
            if (!inverse) {
                uint64_t tb = mulm(w, b, p);
                X[ia] = addm(a, tb, p);
                X[ib] = subm(a, tb, p);
            } else {
                X[ia] = mulm(addm(a, b, p), half, p);
                X[ib] = mulm(mulm(w, subm(a, b, p), p), half, p);
            }
        }
        w = mulm(w, base, p);
        /* bit-reversed increment of j (t bits) */
        if (t > 0) {
            uint64_t mask = (uint64_t)1 << (t - 1);
            while (mask && (j & mask)) {
                j ^= mask;
                mask >>= 1;
            }
            j |= mask;
        }
    }
}

/* v = sum_{i=0}^{(m-3)/2} S_{2i+1} (omega_{(m-1)/2})^i, by Horner. */
static uint64_t odd_child_value(const orc_prime *pr, const uint64_t *X, node S,
                                uint64_t m) {
    const uint64_t p = pr->p;
    uint64_t z = omega_s(pr, (m - 1) / 2);
    uint64_t step = (uint64_t)1 << S.r;
    uint64_t top = (m - 3) / 2;
    uint64_t v = 0;
    for (uint64_t i = top + 1; i-- > 0;)
        v = addm(mulm(v, z, p), X[S.q + (2 * i + 1) * step], p);
    return v;
}

int orc_alg1_tft(int id, uint64_t *X, uint64_t n) {
    if (!valid_id(id) || n == 0 || !X) return -1;
    const orc_prime *pr = &PRIMES[id];
    const uint64_t p = pr->p;
    node root = {0, 0};
    node S = leftmost_leaf(n, root);
    node prev = {~(uint64_t)0, -1};
    for (;;) {
        uint64_t m = node_len(n, S);
        if (is_leaf(n, S) || same(prev, odd_child(S))) {
            butterflies(pr, X, S, m, 0);
            if (same(S, root)) return 0;
            prev = S;
            S = parent_of(S);
        } else if (same(prev, even_child(S))) {
            if (m % 2 == 1) {
                uint64_t v = odd_child_value(pr, X, S, m);
                uint64_t last = S.q + (m - 1) * ((uint64_t)1 << S.r);
                X[last] = addm(X[last], mulm(v, omega_s(pr, m - 1), p), p);
            }
            prev = S;
            S = leftmost_leaf(n, odd_child(S));
        } else {
            return -2; /* unreachable by Lemma 3.1 */
        }
    }
}

int orc_alg2_itft(int id, uint64_t *X, uint64_t n) {
    if (!valid_id(id) || n == 0 || !X) return -1;
    const orc_prime *pr = &PRIMES[id];
    const uint64_t p = pr->p;
    node root = {0, 0};
    node S = root;
    node stop = leftmost_leaf(n, root);
    while (!same(S, stop)) {
        if (is_leaf(n, S)) {
            S = parent_of(rightmost_parent(S));
            uint64_t m = node_len(n, S);
            if (m % 2 == 1) {
                uint64_t v = odd_child_value(pr, X, S, m);
                uint64_t last = S.q + (m - 1) * ((uint64_t)1 << S.r);
                X[last] = subm(X[last], mulm(v, omega_s(pr, m - 1), p), p);
            }
            S = even_child(S);
        } else {
            uint64_t m = node_len(n, S);
            butterflies(pr, X, S, m, 1);
            S = odd_child(S);
        }
    }
    return 0;
}

int orc_tft_polymul(int id, const uint64_t *a, uint64_t na, const uint64_t *b,
                    uint64_t nb, uint64_t *out, uint64_t *work) {
    if (!valid_id(id) || !a || !b || !out || !work || na == 0 || nb == 0)
        return -1;
    const uint64_t p = PRIMES[id].p;
    uint64_t r = na + nb - 1;
    memset(out, 0, r * sizeof(uint64_t));
    memset(work, 0, r * sizeof(uint64_t));
    memcpy(out, a, na * sizeof(uint64_t));
    memcpy(work, b, nb * sizeof(uint64_t));
    int rc = orc_alg1_tft(id, out, r);
    if (rc) return rc;
    rc = orc_alg1_tft(id, work, r);
    if (rc) return rc;
    for (uint64_t s = 0; s < r; s++) out[s] = mulm(out[s], work[s], p);
    return orc_alg2_itft(id, out, r);
}

uint64_t orc_eval(int id, const uint64_t *x, uint64_t n, uint64_t z) {
    if (!valid_id(id)) return 0;
    const uint64_t p = PRIMES[id].p;
    uint64_t acc = 0;
    for (uint64_t i = n; i-- > 0;) acc = addm(mulm(acc, z, p), x[i], p);
    return acc;
}

int orc_eval_tft_points(int id, const uint64_t *x, uint64_t n,
                        const uint64_t *s, uint64_t ns, uint64_t *out) {
    if (!valid_id(id)) return -1;
    for (uint64_t i = 0; i < ns; i++)
        out[i] = orc_eval(id, x, n, omega_s(&PRIMES[id], s[i]));
    return 0;
}

int orc_schoolbook(int id, const uint64_t *a, uint64_t na, const uint64_t *b,
                   uint64_t nb, uint64_t *out) {
    if (!valid_id(id) || na == 0 || nb == 0) return -1;
    const uint64_t p = PRIMES[id].p;
    uint64_t r = na + nb - 1;
    memset(out, 0, r * sizeof(uint64_t));
    for (uint64_t i = 0; i < na; i++)
        for (uint64_t j = 0; j < nb; j++)
            out[i + j] = addm(out[i + j], mulm(a[i], b[j], p), p);
    return 0;
}

int orc_fft_pow2(int id, uint64_t *X, uint64_t N) {
    if (!valid_id(id) || N == 0 || (N & (N - 1))) return -1;
    const orc_prime *pr = &PRIMES[id];
    const uint64_t p = pr->p;
    for (uint64_t len = N / 2; len >= 1; len /= 2) {
        int lg = 0;
        while (((uint64_t)1 << lg) < 2 * len) lg++;
        uint64_t wl = omega_k(pr, lg);
        for (uint64_t start = 0; start < N; start += 2 * len) {
            uint64_t w = 1;
            for (uint64_t j = 0; j < len; j++) {
                uint64_t u = X[start + j], v = X[start + j + len];
                X[start + j] = addm(u, v, p);
                X[start + j + len] = mulm(subm(u, v, p), w, p);
                w = mulm(w, wl, p);
            }
        }
    }
    return 0;
}

/* c_t = sum_{i} a_i b_{t-i} over 0 <= i < na, 0 <= t-i < nb. */
uint64_t orc_conv_coeff(int id, const uint64_t *a, uint64_t na,
                        const uint64_t *b, uint64_t nb, uint64_t t) {
    if (!valid_id(id)) return 0;
    const uint64_t p = PRIMES[id].p;
    uint64_t lo = t + 1 > nb ? t + 1 - nb : 0;
    uint64_t hi = t < na - 1 ? t : na - 1;
    uint64_t acc = 0;
    for (uint64_t i = lo; i <= hi && i < na; i++)
        acc = addm(acc, mulm(a[i], b[t - i], p), p);
    return acc;
}
