"""GPU parity: the CUDA library (through its C ABI) against the oracle.

Every comparison is bit-exact (all arithmetic is exact mod p; tolerance 0).
Inputs come from seeded generators; expected values from oracle/ only.
Sizes span the single-CTA path, the two-pass path with several column tiles
and a ragged last row, b = 0 plans, powers of two, and the full benchmark
sizes (checked on sampled outputs the oracle computes one by one, plus
properties that hold at any size).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import field as F  # noqa: E402
from oracle import native as NV  # noqa: E402
from workloads import (config1_inputs, config2_input,  # noqa: E402
                       config3_inputs, config4_inputs)

PRIMES = F.PRIME_BY_ID


def _lib():
    from paper_1001_5272_gb300 import tft
    return tft


@pytest.fixture(scope="module")
def ctxs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tft = _lib()
    # the largest lengths each field's plans admit (products up to r = 2^27
    # need the work buffer of the 32-bit contexts)
    out = {pr.name: tft.Context(i, 0, max_len=(1 << 25) if pr.word_bits == 64
                                else (1 << 27))
           for i, pr in enumerate(PRIMES)}
    yield out
    for c in out.values():
        c.close()


def _tdtype(pr):
    return torch.int64 if pr.word_bits == 64 else torch.int32


def to_dev(pr, arr):
    a = np.ascontiguousarray(arr)
    if pr.word_bits == 64:
        t = torch.from_numpy(a.astype(np.uint64).view(np.int64))
    else:
        t = torch.from_numpy(a.astype(np.uint32).view(np.int32))
    return t.cuda()


def to_host(pr, t):
    a = t.cpu().numpy()
    return a.view(np.uint64) if pr.word_bits == 64 else \
        a.view(np.uint32).astype(np.uint64)


def rand(pr, n, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, pr.p, n, dtype=np.uint64)


def gpu_forward(ctxs, pr, x, k=None):
    tft = _lib()
    t = to_dev(pr, x)
    tft.tft_forward(ctxs[pr.name], t, k)
    torch.cuda.synchronize()
    return to_host(pr, t)


def gpu_inverse(ctxs, pr, X, k=None):
    tft = _lib()
    t = to_dev(pr, X)
    tft.tft_inverse(ctxs[pr.name], t, k)
    torch.cuda.synchronize()
    return to_host(pr, t)


def gpu_polymul(ctxs, pr, a, b):
    tft = _lib()
    ta, tb = to_dev(pr, a), to_dev(pr, b)
    out = torch.empty(a.size + b.size - 1, dtype=_tdtype(pr), device="cuda")
    tft.tft_polymul(ctxs[pr.name], ta, tb, out)
    torch.cuda.synchronize()
    return to_host(pr, out)


# ---------------------------------------------------------------------------
# Transforms, element by element against Algorithm 1 / Algorithm 2
# ---------------------------------------------------------------------------

SMALL = list(range(1, 130)) + [255, 256, 257, 511, 512, 513, 999, 1000,
                                1023, 1024, 1025, 2047, 2048, 2049, 4095,
                                4096]
TWO_PASS = [4097, 5000, 8191, 8192, 8193, 12345, 16384, 20001, 65536, 65537,
            100003, (1 << 18) - 1, (1 << 18) + 1, 3 * (1 << 17) + 5,
            (1 << 20) + 12345]


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_forward_inverse_small(ctxs, pr):
    for n in SMALL:
        x = rand(pr, n, n)
        ref = NV.alg1_tft(pr, x)
        got = gpu_forward(ctxs, pr, x)
        assert np.array_equal(got, ref), f"forward n={n}"
        back = gpu_inverse(ctxs, pr, ref)
        assert np.array_equal(back, x), f"inverse n={n}"


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
@pytest.mark.parametrize("n", TWO_PASS)
def test_forward_inverse_two_pass(ctxs, pr, n):
    x = rand(pr, n, 1000 + n)
    ref = NV.alg1_tft(pr, x)
    got = gpu_forward(ctxs, pr, x)
    assert np.array_equal(got, ref), f"forward n={n}"
    back = gpu_inverse(ctxs, pr, ref)
    assert np.array_equal(back, x), f"inverse n={n}"


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_k_does_not_change_the_result(ctxs, pr):
    # Compatible roots: the TFT of length n does not depend on k >= lg n.
    n = 3001
    x = rand(pr, n, 5)
    base = gpu_forward(ctxs, pr, x, k=12)
    for k in (13, 20, pr.K):
        assert np.array_equal(gpu_forward(ctxs, pr, x, k=k), base)


def test_every_plan_boundary_u32(ctxs):
    # Lengths around each change of (lr, c) for the 32-bit prime.
    tft = _lib()
    pr = F.P2013265921
    seen = set()
    for e in range(12, 21):
        for n in ((1 << e) - 1, 1 << e, (1 << e) + 1):
            plan = tft.tft_describe_plan(1, n)
            seen.add((plan["small"], plan["lr"], plan["c"]))
            x = rand(pr, n, n + 7)
            ref = NV.alg1_tft(pr, x)
            assert np.array_equal(gpu_forward(ctxs, pr, x), ref), n
            assert np.array_equal(gpu_inverse(ctxs, pr, ref), x), n
    assert len(seen) >= 5


# ---------------------------------------------------------------------------
# Products against schoolbook / Algorithm 1-2 products
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_polymul_small_sizes(ctxs, pr):
    rng = np.random.default_rng(77)
    pairs = [(1, 1), (1, 7), (7, 1), (2, 2), (3, 5), (31, 33), (64, 64),
             (100, 1), (500, 500), (1000, 3000), (2048, 2049), (4000, 97)]
    pairs += [tuple(int(v) for v in rng.integers(1, 2500, 2))
              for _ in range(6)]
    for na, nb in pairs:
        a = rand(pr, na, na * 31 + nb)
        b = rand(pr, nb, nb * 17 + na)
        assert np.array_equal(gpu_polymul(ctxs, pr, a, b),
                              NV.schoolbook(pr, a, b)), (na, nb)


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_polymul_two_pass_sizes(ctxs, pr):
    for na, nb in [(3000, 2000), (4096, 4097), (10000, 20000),
                   (65536, 65536), (70001, 50000), (1, 100000),
                   (123457, 9)]:
        a = rand(pr, na, na + 3)
        b = rand(pr, nb, nb + 5)
        ref = NV.tft_polymul(pr, a, b)
        assert np.array_equal(gpu_polymul(ctxs, pr, a, b), ref), (na, nb)


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_polymul_rounded_length_edges(ctxs, pr):
    # the product's transforms run at length (a + 1) R when r = a R + b with
    # b > 0 (the R - b positions past r in the context's scratch).  Edges: b
    # = 0, 1, R/2 and R - 1; a + 1 a power of two (each column's inverse is
    # a full network), just above one, and odd
    tft = _lib()
    cases = []
    for lr, a_vals in ((8, (127, 128, 155)), (9, (255, 256, 301))):
        R = 1 << lr
        for a_rows in a_vals:
            for b_len in (0, 1, R // 2, R - 1):
                r = a_rows * R + b_len
                P = tft.tft_describe_plan(pr.name, r)
                if P["small"] or P["lr"] != lr:
                    continue
                assert (P["a"], P["b"]) == (a_rows, b_len)
                cases.append(r)
    assert len(cases) >= 12
    for r in cases:
        na = r // 3 + 1
        nb = r - na + 1
        a = rand(pr, na, r)
        b = rand(pr, nb, r + 1)
        assert np.array_equal(gpu_polymul(ctxs, pr, a, b),
                              NV.tft_polymul(pr, a, b)), r


def test_polymul_aliased_operands(ctxs):
    # a and b may be the same buffer (squaring)
    tft = _lib()
    pr = F.PGOLDILOCKS
    a = rand(pr, 9000, 3)
    ta = to_dev(pr, a)
    out = torch.empty(2 * a.size - 1, dtype=torch.int64, device="cuda")
    tft.tft_polymul(ctxs[pr.name], ta, ta, out)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(pr, out), NV.tft_polymul(pr, a, a))


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def test_config1_exact(ctxs):
    import os
    pr = F.P998244353
    a, b, x = config1_inputs()
    golden = os.path.join(os.path.dirname(__file__), "golden",
                          "config1_product.txt")
    ref = np.array([int(l) for l in open(golden)
                    if l.strip() and not l.startswith("#")], dtype=np.uint64)
    assert np.array_equal(gpu_polymul(ctxs, pr, a, b), ref)
    X = gpu_forward(ctxs, pr, x)
    assert np.array_equal(X, NV.alg1_tft(pr, x))
    assert np.array_equal(gpu_inverse(ctxs, pr, X), x.astype(np.uint64))


def _sample_indices(n, rng, extra=()):
    s = set(int(v) for v in rng.integers(0, n, 10))
    s |= {0, 1, n - 1, n - 2} | {v for v in extra if 0 <= v < n}
    return np.array(sorted(s), dtype=np.uint64)


def test_config2_full_size(ctxs):
    # n = 2^24 + 2^20 + 12345 over 2^64 - 2^32 + 1, in the launch
    # configuration the benchmark times: every output element against the
    # oracle's Algorithm 1 (run on a host thread while the GPU works),
    # sampled outputs against the definition (one Horner evaluation each),
    # and the inverse exactly (the round trip returns the input).
    from concurrent.futures import ThreadPoolExecutor
    tft = _lib()
    pr = F.PGOLDILOCKS
    x = config2_input()
    n = x.size
    with ThreadPoolExecutor(1) as pool:
        ref_fut = pool.submit(NV.alg1_tft, pr, x)
        plan = tft.tft_describe_plan(2, n)
        R = 1 << plan["lr"]
        t = to_dev(pr, x)
        tft.tft_forward(ctxs[pr.name], t, 25)
        torch.cuda.synchronize()
        X = to_host(pr, t)
        rng = np.random.default_rng(123)
        # include the last row (s >= aR) and a row boundary
        s = _sample_indices(n, rng, extra=(plan["a"] * R, plan["a"] * R - 1,
                                           R, R - 1))
        ref = NV.eval_tft_points(pr, x, s)
        assert np.array_equal(X[s.astype(np.int64)], ref)
        tft.tft_inverse(ctxs[pr.name], t, 25)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(pr, t), x)
        full = ref_fut.result()
    bad = np.flatnonzero(X != full)
    assert bad.size == 0, f"{bad.size} outputs differ, first at {bad[:8]}"


def test_config3_full_size(ctxs):
    # 3,000,000 x 5,000,001 over 2^64 - 2^32 + 1: every coefficient against
    # the oracle's TFT product (Algorithm 1 on both zero-extended operands,
    # pointwise product, Algorithm 2; run on a host thread while the GPU
    # works), C(z) = A(z) B(z) at random z (Schwartz-Zippel) and sampled
    # coefficients by their defining sums.
    from concurrent.futures import ThreadPoolExecutor
    pr = F.PGOLDILOCKS
    a, b = config3_inputs()
    with ThreadPoolExecutor(1) as pool:
        ref_fut = pool.submit(NV.tft_polymul, pr, a, b)
        c = gpu_polymul(ctxs, pr, a, b)
        rng = np.random.default_rng(321)
        for z in rng.integers(2, pr.p - 1, 2, dtype=np.uint64):
            z = int(z)
            assert NV.eval_at(pr, c, z) == \
                NV.eval_at(pr, a, z) * NV.eval_at(pr, b, z) % pr.p
        r = c.size
        for t_ in [0, 1, 2, r - 1, r - 2, 2_999_999, 4_000_000]:
            assert int(c[t_]) == NV.conv_coeff(pr, a, b, t_), t_
        full = ref_fut.result()
    bad = np.flatnonzero(c != full)
    assert bad.size == 0, f"{bad.size} coefficients differ, first at {bad[:8]}"


@pytest.mark.parametrize("pid,na,nb", [
    (2, (1 << 24) + 3, (1 << 24) - 7),   # r just below 2^25: rows of 2^13
    (1, (1 << 26) - 5, (1 << 26) + 1),   # r = 2^27 - 5: rows of 2^14
])
def test_polymul_longest_rows(ctxs, pid, na, nb):
    # the largest products each field admits, which run the fused row pass
    # on rows of 2^13 (64-bit) and 2^14 (32-bit) elements: sampled
    # coefficients against their defining sums, and C(z) = A(z) B(z)
    pr = PRIMES[pid]
    a, b = rand(pr, na, 17), rand(pr, nb, 18)
    c = gpu_polymul(ctxs, pr, a, b)
    r = c.size
    for t_ in [0, 1, r // 3, na - 1, nb, r - 2, r - 1]:
        assert int(c[t_]) == NV.conv_coeff(pr, a, b, t_), t_
    z = 987654321
    assert NV.eval_at(pr, c, z) == \
        NV.eval_at(pr, a, z) * NV.eval_at(pr, b, z) % pr.p


def test_config4_subset(ctxs):
    # The batched workload's products through the single-call path
    # (every 64th product).
    pr = F.P2013265921
    A, B = config4_inputs()
    for i in range(0, len(A), 64):
        a, b = A[i].astype(np.uint64), B[i].astype(np.uint64)
        ref = NV.tft_polymul(pr, a, b)
        assert np.array_equal(gpu_polymul(ctxs, pr, a, b), ref), i


# ---------------------------------------------------------------------------
# Edge cases and the C ABI's argument checks (nothing is launched on error)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_maximum_size_roundtrip(pr, ctxs):
    # the largest length each prime and plan admit: 2^25 words for
    # 2^64 - 2^32 + 1, 2^K = 2^23 for 998244353, a ragged 2^25 + 12345 for
    # 2013265921 (the context was created with max_len 2^27)
    tft = _lib()
    n = {"goldilocks": 1 << 25, "p998244353": 1 << 23,
         "p2013265921": (1 << 25) + 12345}[pr.name]
    x = rand(pr, n, 99)
    t = to_dev(pr, x)
    ctx = ctxs[pr.name]
    tft.tft_forward(ctx, t)
    torch.cuda.synchronize()
    X = to_host(pr, t)
    rng = np.random.default_rng(5)
    s = _sample_indices(n, rng)
    assert np.array_equal(X[s.astype(np.int64)], NV.eval_tft_points(pr, x, s))
    tft.tft_inverse(ctx, t)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(pr, t), x)


def test_argument_errors(ctxs):
    tft = _lib()
    ctx = ctxs["goldilocks"]
    x = torch.zeros(1024, dtype=torch.int64, device="cuda")
    with pytest.raises(tft.TFTError) as e:
        tft.tft_forward(ctx, x, k=9)                    # n > 2^k
    assert e.value.status == tft.TFT_EINVAL
    with pytest.raises(tft.TFTError) as e:
        tft.tft_forward(ctx, x, k=33)                   # k > K
    assert e.value.status == tft.TFT_EINVAL
    with pytest.raises(tft.TFTError) as e:
        tft.tft_forward(ctx, x[1:], k=10)               # misaligned
    assert e.value.status == tft.TFT_EINVAL
    with pytest.raises(tft.TFTError) as e:
        tft.tft_forward(ctx, x[:0], k=10)               # n = 0
    assert e.value.status == tft.TFT_EINVAL
    big = torch.zeros((1 << 25) + 2, dtype=torch.int64, device="cuda")
    with pytest.raises(tft.TFTError) as e:
        tft.tft_forward(ctx, big, k=26)                 # beyond max_len
    assert e.value.status == tft.TFT_ERANGE
    out = torch.zeros(2047, dtype=torch.int64, device="cuda")
    with pytest.raises(tft.TFTError) as e:
        tft.tft_polymul(ctx, out[:1024], x, out)        # out aliases a
    assert e.value.status == tft.TFT_EINVAL
    assert tft.tft_last_error(ctx) == tft.TFT_OK


def test_host_buffer_entry_points():
    tft = _lib()
    pr = F.PGOLDILOCKS
    with tft.Context(2, 0, max_len=1 << 16, host_staging=True) as ctx:
        a, b = rand(pr, 20000, 1), rand(pr, 30000, 2)
        out = np.zeros(a.size + b.size - 1, dtype=np.uint64)
        tft.tft_polymul_host(ctx, a, b, out)
        assert np.array_equal(out, NV.tft_polymul(pr, a, b))
        x = rand(pr, 50000, 3)
        y = x.copy()
        tft.tft_forward_host(ctx, y)
        assert np.array_equal(y, NV.alg1_tft(pr, x))
        tft.tft_inverse_host(ctx, y)
        assert np.array_equal(y, x)
    # an odd max_len must still give 16-byte aligned staging slots
    with tft.Context(2, 0, max_len=70001, host_staging=True) as ctx:
        a, b = rand(pr, 30001, 4), rand(pr, 40000, 5)
        out = np.zeros(a.size + b.size - 1, dtype=np.uint64)
        tft.tft_polymul_host(ctx, a, b, out)
        assert np.array_equal(out, NV.tft_polymul(pr, a, b))
