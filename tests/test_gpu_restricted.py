"""GPU parity of the space-restricted product (Algorithm 3, Section 5) on
the device: bit-exact against the oracle's product (the product is unique,
so the oracle's TFT product and schoolbook are both references) over sizes
that exercise no chunk (tail only), one and several chunks, chunk sizes
repeating, tails that cross an aligned 2^15 block, and the full benchmark
size (sampled coefficients, and equality with tft_polymul)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import field as F  # noqa: E402
from oracle import native as NV  # noqa: E402
from workloads import config3_inputs  # noqa: E402

PRIMES = F.PRIME_BY_ID


def _lib():
    from paper_1001_5272_gb300 import tft
    return tft


@pytest.fixture(scope="module")
def ctxs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tft = _lib()
    # max_len is irrelevant to the restricted product (no work area)
    out = {i: tft.Context(i, 0, max_len=1 << 12) for i in range(3)}
    yield out
    for c in out.values():
        c.close()


def to_dev(pid, arr):
    a = np.ascontiguousarray(arr)
    if pid == 2:
        return torch.from_numpy(a.astype(np.uint64).view(np.int64)).cuda()
    return torch.from_numpy(a.astype(np.uint32).view(np.int32)).cuda()


def to_host(pid, t):
    a = t.cpu().numpy()
    return a.view(np.uint64) if pid == 2 else a.view(np.uint32).astype(
        np.uint64)


def rand(pid, n, seed):
    return np.random.default_rng(seed).integers(0, PRIMES[pid].p, n,
                                                dtype=np.uint64)


def restricted(ctx, pid, a, b):
    tft = _lib()
    out = torch.empty(a.size + b.size - 1,
                      dtype=torch.int64 if pid == 2 else torch.int32,
                      device="cuda")
    tft.tft_polymul_restricted(ctx, to_dev(pid, a), to_dev(pid, b), out)
    torch.cuda.synchronize()
    return to_host(pid, out)


@pytest.mark.parametrize("pid", [0, 1, 2])
def test_restricted_small_sizes_against_schoolbook(ctxs, pid):
    for na, nb in [(1, 1), (1, 2), (2, 1), (3, 5), (16, 17), (100, 1),
                   (500, 500), (1000, 3000), (2048, 2049)]:
        a, b = rand(pid, na, na + 7), rand(pid, nb, nb + 11)
        assert np.array_equal(restricted(ctxs[pid], pid, a, b),
                              NV.schoolbook(pid, a, b)), (na, nb)


@pytest.mark.parametrize("pid", [0, 1, 2])
def test_restricted_chunked_sizes(ctxs, pid):
    # r = 2^14 - 1 .. 2^14 + 1 (first chunk appears), 30000 (two chunks of
    # 8192 and a tail inside one block), 2^15 + 1, 100000 (tail crossing a
    # 2^15 boundary), 131071, and lopsided operands
    for na, nb in [(8192, 8192), (8192, 8193), (8193, 8193), (15000, 15001),
                   (16384, 16386), (50000, 50001), (65536, 65536),
                   (1, 100000), (123457, 9), (70001, 50000)]:
        a, b = rand(pid, na, na * 3 + 1), rand(pid, nb, nb * 5 + 2)
        assert np.array_equal(restricted(ctxs[pid], pid, a, b),
                              NV.tft_polymul(pid, a, b)), (na, nb)


def test_restricted_full_size_goldilocks(ctxs):
    # the 3,000,000 x 5,000,001 benchmark product: equal to the two-buffer
    # product, and sampled coefficients equal to their defining sums
    tft = _lib()
    pid = 2
    a, b = config3_inputs()
    ta, tb = to_dev(pid, a), to_dev(pid, b)
    r = a.size + b.size - 1
    out_r = torch.empty(r, dtype=torch.int64, device="cuda")
    tft.tft_polymul_restricted(ctxs[pid], ta, tb, out_r)
    ctx_full = tft.Context(2, 0, max_len=r)
    out_s = torch.empty(r, dtype=torch.int64, device="cuda")
    tft.tft_polymul(ctx_full, ta, tb, out_s)
    torch.cuda.synchronize()
    ctx_full.close()
    assert torch.equal(out_r, out_s)
    c = to_host(pid, out_r)
    for t in [0, 1, r // 2, r - 2, r - 1, 4_000_000, 7_999_000]:
        assert int(c[t]) == NV.conv_coeff(pid, a, b, t), t


def test_restricted_largest_998244353(ctxs):
    # r = 2^23 - 1, the largest product 998244353 admits (K = 23)
    pid = 0
    a, b = rand(pid, 1 << 22, 1), rand(pid, 1 << 22, 2)
    c = restricted(ctxs[pid], pid, a, b)
    rng = np.random.default_rng(3)
    for t in [0, 5, (1 << 22) - 1, (1 << 23) - 2] + \
            [int(v) for v in rng.integers(0, (1 << 23) - 1, 4)]:
        assert int(c[t]) == NV.conv_coeff(pid, a, b, t), t
    z = 123456
    p = PRIMES[pid].p
    assert NV.eval_at(pid, c, z) == \
        NV.eval_at(pid, a, z) * NV.eval_at(pid, b, z) % p


def test_restricted_argument_errors(ctxs):
    tft = _lib()
    ctx = ctxs[2]
    a = torch.zeros(100, dtype=torch.int64, device="cuda")
    out = torch.zeros(199, dtype=torch.int64, device="cuda")
    with pytest.raises(tft.TFTError) as e:  # out overlapping an operand
        tft.tft_polymul_restricted(ctx, out[:100], a, out)
    assert e.value.status == tft.TFT_EINVAL
    with pytest.raises(tft.TFTError) as e:  # misaligned operand
        tft.tft_polymul_restricted(ctx, a[1:], a[:10], out[:108])
    assert e.value.status == tft.TFT_EINVAL
