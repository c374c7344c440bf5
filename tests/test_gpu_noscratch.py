"""GPU parity of the transforms without global scratch (tft_forward_noscratch,
tft_inverse_noscratch): element by element against Algorithm 1 of the
oracle, the round trip, and bit-for-bit agreement with the context-based
transforms at the full n = 2^24 + 2^20 + 12345 of the benchmark.  Lengths
cover the single-CTA plans, rows of fewer than 2^8 and of at least 2^8,
b = 0 (no ragged row), b = 1, b = R - 1 and random b."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import field as F  # noqa: E402
from oracle import native as NV  # noqa: E402
from workloads import config2_input  # noqa: E402

pytestmark = pytest.mark.gpu

PRIMES = F.PRIME_BY_ID


def _lib():
    from paper_1001_5272_gb300 import tft
    return tft


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


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


def lengths(pr):
    """Single-CTA, short-row and long-row plans with b = 0, 1, R - 1 and
    random b (R from the library's own plan for each length)."""
    tft = _lib()
    out = [1, 2, 100, 4095, 4097, 5000, 8193, 12345, 20001, 65537, 100003,
           262145, 1000003]
    for base in (5000, 40000, 300000):
        P = tft.tft_describe_plan(pr.name, base)
        if P["small"]:
            continue
        R = 1 << P["lr"]
        a = P["a"]
        for b in (0, 1, R - 1):
            n = a * R + b
            Q = tft.tft_describe_plan(pr.name, n)
            if not Q["small"] and Q["lr"] == P["lr"]:
                out.append(n)
    return sorted(set(out))


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_noscratch_matches_algorithm_1_and_round_trips(pr):
    tft = _lib()
    for i, n in enumerate(lengths(pr)):
        x = rand(pr, n, 1000 + i)
        t = to_dev(pr, x)
        tft.tft_forward_noscratch(pr.name, t)
        torch.cuda.synchronize()
        X = to_host(pr, t)
        assert np.array_equal(X, NV.alg1_tft(pr, x)), n
        tft.tft_inverse_noscratch(pr.name, t)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(pr, t), x), n


@pytest.mark.parametrize("pr", PRIMES, ids=lambda p: p.name)
def test_noscratch_inverse_of_given_values(pr):
    # the inverse on arbitrary transform values (not only on outputs of the
    # forward) against Algorithm 2
    tft = _lib()
    for i, n in enumerate((4097, 20001, 65537, 262145)):
        X = rand(pr, n, 2000 + i)
        t = to_dev(pr, X)
        tft.tft_inverse_noscratch(pr.name, t)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(pr, t), NV.alg2_itft(pr, X)), n


def test_noscratch_full_size_matches_context_transforms():
    # n = 2^24 + 2^20 + 12345 over 2^64 - 2^32 + 1: the same outputs as the
    # context-based transforms (themselves checked against the definition)
    tft = _lib()
    pr = F.PGOLDILOCKS
    x = config2_input()
    n = x.size
    ref = to_dev(pr, x)
    with tft.Context(2, 0, max_len=n) as ctx:
        tft.tft_forward(ctx, ref, 25)
    t = to_dev(pr, x)
    tft.tft_forward_noscratch(2, t, 25)
    torch.cuda.synchronize()
    assert torch.equal(t, ref)
    tft.tft_inverse_noscratch(2, t, 25)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(pr, t), x)


def test_noscratch_argument_errors():
    tft = _lib()
    t = torch.zeros(10, dtype=torch.int64, device="cuda")
    with pytest.raises(tft.TFTError):
        tft.tft_forward_noscratch(2, t, 3)       # n > 2^k
    with pytest.raises(tft.TFTError):
        tft.tft_inverse_noscratch(2, t[1:])      # misaligned
