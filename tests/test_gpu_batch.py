"""GPU parity of the batched product (tft_polymul_batch and its plan/run
split) against the oracle, bit for bit.

Each product of a batch is the Section 5 product of its own operands, so
the expected value of every product is the oracle's TFT product of that
pair alone: the batch must not change any result.  Batches mix the
single-CTA class and the row/column class, ragged and exact last rows,
every admissible schedule parameter, and the full log-uniform workload of
4096 products over 2013265921 (checked completely through Schwartz-Zippel
evaluations plus every 32nd product element by element).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import field as F  # noqa: E402
from oracle import native as NV  # noqa: E402
from workloads import config4_inputs  # noqa: E402

PRIMES = F.PRIME_BY_ID


def _lib():
    from paper_1001_5272_gb300 import tft
    return tft


@pytest.fixture(scope="module")
def ctxs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tft = _lib()
    out = {pr.name: tft.Context(i, 0, max_len=1 << 20)
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


def run_batch(ctx, pr, pairs, params=None, seed=0, reserve=True):
    """Batched product of random operands of the given lengths; returns the
    host operands and the host results."""
    tft = _lib()
    A = [rand(pr, na, seed * 7919 + 2 * i) for i, (na, nb) in enumerate(pairs)]
    B = [rand(pr, nb, seed * 7919 + 2 * i + 1)
         for i, (na, nb) in enumerate(pairs)]
    prods = []
    for a, b in zip(A, B):
        prods.append((to_dev(pr, a), to_dev(pr, b),
                      torch.empty(a.size + b.size - 1, dtype=_tdtype(pr),
                                  device="cuda")))
    if reserve:
        words = tft.tft_batch_work_words(ctx.prime, pairs, params)
        tft.tft_ctx_reserve_batch(ctx, len(pairs), words)
    tft.tft_polymul_batch(ctx, prods, params)
    torch.cuda.synchronize()
    return A, B, [to_host(pr, o) for _, _, o in prods]


# lengths spanning both classes: r = na + nb - 1 at and around 2^13 (the
# 32-bit default small-class bound) and 2^12 (64-bit), exact multiples of
# the row length (no last row), one-row-plus-one, long thin products
MIXED = [(1, 1), (1, 9), (3, 5), (100, 200), (257, 256), (2048, 2049),
         (4000, 4193), (4097, 4096), (4097, 4097), (2048, 2050), (2049, 2049),
         (513, 8000), (1, 20000), (20000, 1), (10000, 20000), (65536, 65536),
         (70001, 50000), (5000, 5000), (8193, 8192), (1024, 1025),
         (6145, 10240), (123457, 9)]


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_batch_mixed_classes(ctxs, pr):
    A, B, C = run_batch(ctxs[pr.name], pr, MIXED, seed=1)
    for i, (a, b, c) in enumerate(zip(A, B, C)):
        assert np.array_equal(c, NV.tft_polymul(pr, a, b)), MIXED[i]


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
@pytest.mark.parametrize("params", [
    {"lr": 8, "small_log": 8, "clog": 0},
    {"lr": 8, "small_log": 10, "clog": 3},
    {"lr": 9, "small_log": 9, "clog": 4},
    {"lr": 10, "small_log": 12, "clog": 2},
    {"lr": 11, "small_log": 11, "clog": 1},
    {"lr": 12, "small_log": 12, "clog": 4},
    {"lr": 8, "small_log": 12, "clog": 5},
    {"lr": 8, "small_log": 9, "clog": 3, "clog_lo": 5},
    {"lr": 9, "small_log": 9, "clog": 4, "clog_lo": 1},
    {"lr": 10, "small_log": 10, "clog": 2, "clog_lo": 0},
], ids=lambda d: "lr{lr}-s{small_log}-c{clog}-clo{}".format(
    d.get("clog_lo", "-"), **d))
def test_batch_schedules(ctxs, pr, params):
    pairs = [(300, 200), (256, 1), (257, 1), (1000, 3000), (4096, 4097),
             (9000, 7001), (30000, 40000), (2, 70000), (12345, 12345)]
    A, B, C = run_batch(ctxs[pr.name], pr, pairs, params, seed=2)
    for i, (a, b, c) in enumerate(zip(A, B, C)):
        assert np.array_equal(c, NV.tft_polymul(pr, a, b)), (pairs[i], params)


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_batch_rounded_length_edges(ctxs, pr):
    # one batch on rows of 2^8 whose large products have r = a 2^8 + b with
    # b = 0, 1, 128, 255 and a + 1 a power of two, just above one, or odd
    # (a product with b > 0 runs its transforms at length (a + 1) 2^8)
    pairs = []
    for a_rows in (31, 32, 63, 64, 155):
        for b_len in (0, 1, 128, 255):
            r = a_rows * 256 + b_len
            na = r // 2 + 1
            pairs.append((na, r - na + 1))
    params = {"lr": 8, "small_log": 9, "clog": 3}
    A, B, C = run_batch(ctxs[pr.name], pr, pairs, params, seed=4)
    for i, (a, b, c) in enumerate(zip(A, B, C)):
        assert np.array_equal(c, NV.tft_polymul(pr, a, b)), pairs[i]


def test_batch_only_small_and_only_large(ctxs):
    pr = F.P998244353
    ctx = ctxs[pr.name]
    for pairs in ([(10, 20), (4096, 4097), (1, 1)],
                  [(4097, 4097), (30000, 2), (16384, 16385)]):
        A, B, C = run_batch(ctx, pr, pairs, seed=3)
        for a, b, c in zip(A, B, C):
            assert np.array_equal(c, NV.tft_polymul(pr, a, b))


def test_batch_many_equal_products(ctxs):
    # 600 products of the same shape: more tasks than persistent CTAs in
    # every phase, so each CTA walks several products
    pr = F.PGOLDILOCKS
    pairs = [(1500, 1500)] * 300 + [(9000, 3000)] * 300
    A, B, C = run_batch(ctxs[pr.name], pr, pairs, seed=4)
    for i in range(0, 600, 37):
        assert np.array_equal(C[i], NV.tft_polymul(pr, A[i], B[i])), i
    z = 123456789
    for i in range(600):
        assert NV.eval_at(pr, C[i], z) == \
            NV.eval_at(pr, A[i], z) * NV.eval_at(pr, B[i], z) % pr.p, i


def test_batch_matches_single_calls(ctxs):
    tft = _lib()
    pr = F.P2013265921
    ctx = ctxs[pr.name]
    pairs = [(700, 900), (5000, 7000), (40000, 3)]
    A, B, C = run_batch(ctx, pr, pairs, seed=5)
    for a, b, c in zip(A, B, C):
        out = torch.empty(a.size + b.size - 1, dtype=torch.int32,
                          device="cuda")
        tft.tft_polymul(ctx, to_dev(pr, a), to_dev(pr, b), out)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(pr, out), c)


def test_batch_graph_replay(ctxs):
    # plan once, capture tft_batch_run into a CUDA graph, then replay it on
    # new operand values written into the same buffers
    tft = _lib()
    pr = F.P2013265921
    ctx = ctxs[pr.name]
    pairs = [(64, 64), (3000, 5000), (20000, 20001), (4096, 1)]
    prods = [(torch.empty(na, dtype=torch.int32, device="cuda"),
              torch.empty(nb, dtype=torch.int32, device="cuda"),
              torch.empty(na + nb - 1, dtype=torch.int32, device="cuda"))
             for na, nb in pairs]
    tft.tft_ctx_reserve_batch(ctx, len(pairs),
                              tft.tft_batch_work_words(ctx.prime, pairs))
    tft.tft_batch_plan(ctx, prods)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        tft.tft_batch_run(ctx, s)  # warm-up outside capture
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            tft.tft_batch_run(ctx, s)
    for rep in range(3):
        A = [rand(pr, na, 100 * rep + i) for i, (na, _) in enumerate(pairs)]
        B = [rand(pr, nb, 100 * rep + i + 50)
             for i, (_, nb) in enumerate(pairs)]
        for (ta, tb, _), a, b in zip(prods, A, B):
            ta.copy_(to_dev(pr, a))
            tb.copy_(to_dev(pr, b))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        for (_, _, to), a, b in zip(prods, A, B):
            assert np.array_equal(to_host(pr, to), NV.tft_polymul(pr, a, b))


def test_batch_full_log_uniform_workload(ctxs):
    # 4096 products, lengths log-uniform in [64, 65536], over 2013265921:
    # every product checked at a random point (Schwartz-Zippel: a wrong
    # product of degree < 2^17 passes with probability < 2^17 / p), every
    # 32nd product element by element
    tft = _lib()
    pr = F.P2013265921
    ctx = ctxs[pr.name]
    A, B = config4_inputs()
    prods = [(to_dev(pr, a), to_dev(pr, b),
              torch.empty(a.size + b.size - 1, dtype=torch.int32,
                          device="cuda")) for a, b in zip(A, B)]
    pairs = [(a.size, b.size) for a, b in zip(A, B)]
    tft.tft_ctx_reserve_batch(ctx, len(pairs),
                              tft.tft_batch_work_words(ctx.prime, pairs))
    tft.tft_polymul_batch(ctx, prods)
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    for i, ((_, _, to), a, b) in enumerate(zip(prods, A, B)):
        c = to_host(pr, to)
        z = int(rng.integers(2, pr.p))
        assert NV.eval_at(pr, c, z) == \
            NV.eval_at(pr, a, z) * NV.eval_at(pr, b, z) % pr.p, i
        if i % 32 == 0:
            assert np.array_equal(c, NV.tft_polymul(pr, a, b)), i


def _served_range_pairs():
    # operand lengths of the served workload's range: log-uniform in
    # [256, 2^20] (products up to r = 2^21 - 1), plus the extremes
    rng = np.random.default_rng(61)
    u = rng.random((2, 20))
    L = np.clip(np.floor(256 * 4096.0 ** u), 256, 1 << 20).astype(np.int64)
    pairs = [(int(x), int(y)) for x, y in zip(L[0], L[1])]
    return pairs + [(1 << 20, 1 << 20), (1 << 20, 256), (256, 1 << 20),
                    (256, 256), ((1 << 19) + 1, (1 << 19) + 3)]


@pytest.mark.parametrize("params", [
    None, {"small_log": 12, "lr": 11, "clog": 4}],
    ids=["default", "sl12-lr11-c4"])
def test_batch_goldilocks_served_length_range(ctxs, params):
    # the served stream's products over 2^64 - 2^32 + 1 at full length
    # range, under the default schedule and the one the serving benchmark
    # runs: every product checked at a random point (Schwartz-Zippel), 24
    # sampled coefficients of each by their defining sums, and the longest
    # product (r = 2^21 - 1) plus three others element by element against
    # the oracle's TFT product
    pr = F.PGOLDILOCKS
    pairs = _served_range_pairs()
    A, B, C = run_batch(ctxs[pr.name], pr, pairs, params, seed=6)
    rng = np.random.default_rng(67)
    for i, (a, b, c) in enumerate(zip(A, B, C)):
        r = c.size
        z = int(rng.integers(2, pr.p - 1, dtype=np.uint64))
        assert NV.eval_at(pr, c, z) == \
            NV.eval_at(pr, a, z) * NV.eval_at(pr, b, z) % pr.p, pairs[i]
        ts = {0, r - 1, a.size - 1, b.size - 1} | \
            {int(t) for t in rng.integers(0, r, 20)}
        for t in sorted(ts):
            assert int(c[t]) == NV.conv_coeff(pr, a, b, t), (pairs[i], t)
    for i in (len(pairs) - 5, len(pairs) - 4, len(pairs) - 1, 0):
        assert np.array_equal(C[i], NV.tft_polymul(pr, A[i], B[i])), pairs[i]


def test_batch_argument_errors(ctxs):
    tft = _lib()
    pr = F.PGOLDILOCKS
    ctx = tft.Context(2, 0, max_len=1 << 12)
    try:
        a = torch.zeros(5000, dtype=torch.int64, device="cuda")
        b = torch.zeros(5000, dtype=torch.int64, device="cuda")
        out = torch.zeros(9999, dtype=torch.int64, device="cuda")
        # nothing reserved yet
        with pytest.raises(tft.TFTError) as e:
            tft.tft_batch_plan(ctx, [(a, b, out)])
        assert e.value.status == tft.TFT_EINVAL
        with pytest.raises(tft.TFTError) as e:
            tft.tft_batch_run(ctx)
        assert e.value.status == tft.TFT_EINVAL
        tft.tft_ctx_reserve_batch(ctx, 2, 100)
        # work area too small for a large product
        with pytest.raises(tft.TFTError) as e:
            tft.tft_batch_plan(ctx, [(a, b, out)])
        assert e.value.status == tft.TFT_ERANGE
        tft.tft_ctx_reserve_batch(
            ctx, 2, tft.tft_batch_work_words(2, [(5000, 5000)]))
        # more products than reserved
        with pytest.raises(tft.TFTError) as e:
            tft.tft_batch_plan(ctx, [(a, b, out)] * 3)
        assert e.value.status == tft.TFT_ERANGE
        # out overlapping an operand
        with pytest.raises(tft.TFTError) as e:
            tft.tft_batch_plan(ctx, [(a, b, out), (a[:10], b[:10], a[:19])])
        assert e.value.status == tft.TFT_EINVAL
        # misaligned operand
        with pytest.raises(tft.TFTError) as e:
            tft.tft_batch_plan(ctx, [(a[1:11], b[:10], out[:19])])
        assert e.value.status == tft.TFT_EINVAL
        # schedule out of range (row length below 2^8; small class above
        # the shared-memory bound; small class below the row length)
        for bad in ({"lr": 7}, {"lr": 13}, {"small_log": 13},
                    {"lr": 11, "small_log": 10}, {"clog": 6},
                    {"clog_lo": 6}):
            with pytest.raises(tft.TFTError) as e:
                tft.tft_batch_plan(ctx, [(a, b, out)], bad)
            assert e.value.status == tft.TFT_EINVAL, bad
        # a product whose columns are too long for the row length
        big_a = torch.zeros(1 << 22, dtype=torch.int64, device="cuda")
        big_o = torch.zeros((1 << 22) + 4999, dtype=torch.int64,
                            device="cuda")
        with pytest.raises(tft.TFTError) as e:
            tft.tft_batch_plan(ctx, [(big_a, b, big_o)], {"lr": 8})
        assert e.value.status == tft.TFT_ERANGE
        # a valid plan after the errors still runs correctly
        ha, hb = rand(pr, 5000, 1), rand(pr, 5000, 2)
        a.copy_(to_dev(pr, ha))
        b.copy_(to_dev(pr, hb))
        tft.tft_polymul_batch(ctx, [(a, b, out)])
        torch.cuda.synchronize()
        assert np.array_equal(to_host(pr, out), NV.tft_polymul(pr, ha, hb))
    finally:
        ctx.close()
