"""The five synthetic workloads (no public dataset exists for this method).

Values are uniform residues in [0, p), drawn as
``numpy.random.default_rng(seed).integers(0, p, size, dtype=uint64)`` and
narrowed to uint32 for the two 32-bit primes.  Draw order is fixed per
configuration and documented on each function, so that any consumer (the
oracle, the CUDA path, a reader) regenerates the same arrays.

Prime ids match the library's enum: 0 -> 998244353, 1 -> 2013265921,
2 -> 2^64 - 2^32 + 1.  The moduli below are data (the ring each workload
lives in), not arithmetic of the method.
"""

from dataclasses import dataclass, field

import numpy as np

_MODULI = {0: 998244353, 1: 2013265921, 2: 2**64 - 2**32 + 1}


def modulus(prime_id):
    return _MODULI[prime_id]


def elem_dtype(prime_id):
    return np.uint64 if prime_id == 2 else np.uint32


@dataclass(frozen=True)
class Config:
    key: str
    prime_id: int
    seed: int
    description: str
    params: dict = field(default_factory=dict)


CONFIGS = {
    "polymul_p998244353_500x500": Config(
        "polymul_p998244353_500x500", 0, 0,
        "TFT product of two length-500 polynomials over Z/998244353 "
        "(r = 999) plus an ITFT(TFT(x)) round trip on a length-1000 vector",
        {"na": 500, "nb": 500, "roundtrip_n": 1000}),
    "tft_goldilocks_n17838137": Config(
        "tft_goldilocks_n17838137", 2, 1,
        "one forward and one inverse TFT of length n = 2^24 + 2^20 + 12345 "
        "(k = 25) over Z/(2^64 - 2^32 + 1)",
        {"n": 2**24 + 2**20 + 12345, "k": 25}),
    "polymul_goldilocks_3000000x5000001": Config(
        "polymul_goldilocks_3000000x5000001", 2, 2,
        "TFT product of lengths 3,000,000 and 5,000,001 over "
        "Z/(2^64 - 2^32 + 1) (r = 8,000,000, k = 23)",
        {"na": 3_000_000, "nb": 5_000_001}),
    "batched_polymul_p2013265921_4096": Config(
        "batched_polymul_p2013265921_4096", 1, 3,
        "4096 independent products over Z/2013265921, each operand length "
        "log-uniform in [64, 65536]",
        {"count": 4096, "lo": 64, "hi": 65536}),
    "served_polymul_goldilocks_20000rps": Config(
        "served_polymul_goldilocks_20000rps", 2, 4,
        "Poisson arrivals at 20,000 requests/s for 10 s over "
        "Z/(2^64 - 2^32 + 1), operand lengths log-uniform in [256, 2^20]",
        {"rate": 20000.0, "duration_s": 10.0, "lo": 256, "hi": 2**20}),
}


def uniform_residues(rng, prime_id, size):
    """``size`` residues uniform in [0, p), in the element dtype of the prime."""
    p = _MODULI[prime_id]
    v = rng.integers(0, p, size=size, dtype=np.uint64)
    return v.astype(elem_dtype(prime_id), copy=False)


def config1_inputs():
    """(a, b, x): a then b (500 each), then the 1000-vector, one stream."""
    c = CONFIGS["polymul_p998244353_500x500"]
    rng = np.random.default_rng(c.seed)
    a = uniform_residues(rng, c.prime_id, c.params["na"])
    b = uniform_residues(rng, c.prime_id, c.params["nb"])
    x = uniform_residues(rng, c.prime_id, c.params["roundtrip_n"])
    return a, b, x


def config2_input():
    c = CONFIGS["tft_goldilocks_n17838137"]
    rng = np.random.default_rng(c.seed)
    return uniform_residues(rng, c.prime_id, c.params["n"])


def config3_inputs(scale=1.0):
    """(a, b), a drawn first.  ``scale`` < 1 gives a proportionally smaller
    instance of the same shape (used for bounded CPU samples)."""
    c = CONFIGS["polymul_goldilocks_3000000x5000001"]
    rng = np.random.default_rng(c.seed)
    na = max(1, int(round(c.params["na"] * scale)))
    nb = max(1, int(round(c.params["nb"] * scale)))
    a = uniform_residues(rng, c.prime_id, na)
    b = uniform_residues(rng, c.prime_id, nb)
    return a, b


def _log_uniform_lengths(rng, count, lo, hi):
    """L = floor(lo * (hi/lo)^u), u ~ U[0, 1), clipped to [lo, hi]."""
    u = rng.random(count)
    L = np.floor(lo * (hi / lo) ** u).astype(np.int64)
    return np.clip(L, lo, hi)


def config4_lengths(count=None):
    """(na, nb): all a-lengths, then all b-lengths, before any coefficient."""
    c = CONFIGS["batched_polymul_p2013265921_4096"]
    rng = np.random.default_rng(c.seed)
    count = count or c.params["count"]
    na = _log_uniform_lengths(rng, count, c.params["lo"], c.params["hi"])
    nb = _log_uniform_lengths(rng, count, c.params["lo"], c.params["hi"])
    return na, nb, rng


def config4_inputs(count=None):
    """Lengths first, then for each product i in order: a_i, then b_i."""
    na, nb, rng = config4_lengths(count)
    c = CONFIGS["batched_polymul_p2013265921_4096"]
    A, B = [], []
    for i in range(na.size):
        A.append(uniform_residues(rng, c.prime_id, int(na[i])))
        B.append(uniform_residues(rng, c.prime_id, int(nb[i])))
    return A, B


def config5_schedule(duration_s=None, rate=None):
    """Arrival times (s) and operand lengths of the served stream.

    Exponential inter-arrival times at ``rate`` per second until
    ``duration_s``; then, for the requests that arrived, all a-lengths and
    all b-lengths (log-uniform in [256, 2^20]).
    """
    c = CONFIGS["served_polymul_goldilocks_20000rps"]
    rng = np.random.default_rng(c.seed)
    rate = rate or c.params["rate"]
    duration_s = duration_s or c.params["duration_s"]
    expected = int(rate * duration_s * 1.2) + 16
    gaps = rng.exponential(1.0 / rate, size=expected)
    t = np.cumsum(gaps)
    t = t[t < duration_s]
    na = _log_uniform_lengths(rng, t.size, c.params["lo"], c.params["hi"])
    nb = _log_uniform_lengths(rng, t.size, c.params["lo"], c.params["hi"])
    return t, na, nb
