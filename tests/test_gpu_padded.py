"""GPU parity of the padded power-of-two product (the comparison path):
bit-exact against the oracle's product, for r below, at and just above
powers of two, and on a full-size product sampled against the defining
sums."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import field as F  # noqa: E402
from oracle import native as NV  # noqa: E402

PRIMES = F.PRIME_BY_ID


def _lib():
    from paper_1001_5272_gb300 import tft
    return tft


@pytest.fixture(scope="module")
def ctxs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tft = _lib()
    out = {i: tft.Context(i, 0, max_len=1 << 12) for i in range(3)}
    yield out
    for c in out.values():
        c.close()


def dt(pid):
    return torch.int64 if pid == 2 else torch.int32


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


def padded(ctx, pid, a, b):
    tft = _lib()
    r = a.size + b.size - 1
    N = 1 << (r - 1).bit_length()
    out = torch.empty(r, dtype=dt(pid), device="cuda")
    scratch = torch.empty(2 * N, dtype=dt(pid), device="cuda")
    tft.tft_polymul_padded(ctx, to_dev(pid, a), to_dev(pid, b), out, scratch)
    torch.cuda.synchronize()
    return to_host(pid, out)


@pytest.mark.parametrize("pid", [0, 1, 2])
def test_padded_against_oracle(ctxs, pid):
    for na, nb in [(1, 1), (3, 5), (2048, 2049), (4096, 4097), (8192, 8193),
                   (8193, 8192), (16384, 16385), (70001, 50000),
                   (65536, 65537), (1, 100000)]:
        a, b = rand(pid, na, na + 1), rand(pid, nb, nb + 2)
        assert np.array_equal(padded(ctxs[pid], pid, a, b),
                              NV.tft_polymul(pid, a, b)), (na, nb)


def test_padded_full_size_just_above_power_of_two(ctxs):
    # r = 2^22 + 1: the padded transforms have length 2^23
    pid = 2
    a, b = rand(pid, (1 << 21) + 1, 5), rand(pid, (1 << 21) + 1, 6)
    c = padded(ctxs[pid], pid, a, b)
    r = c.size
    for t in [0, 1, 1 << 21, r - 2, r - 1, 3_000_000]:
        assert int(c[t]) == NV.conv_coeff(pid, a, b, t), t


def test_padded_argument_errors(ctxs):
    # raw C calls: scratch overlapping out, and a null scratch, are rejected
    # before any launch
    tft = _lib()
    ctx = ctxs[2]
    a = torch.zeros(100, dtype=torch.int64, device="cuda")
    out = torch.zeros(199, dtype=torch.int64, device="cuda")
    sc = torch.zeros(512, dtype=torch.int64, device="cuda")
    L = tft.load()
    assert L.tft_polymul_padded(ctx.handle, a.data_ptr(), 100, a.data_ptr(),
                                100, sc.data_ptr(), sc.data_ptr(),
                                None) == tft.TFT_EINVAL
    assert L.tft_polymul_padded(ctx.handle, a.data_ptr(), 100, a.data_ptr(),
                                100, out.data_ptr(), None,
                                None) == tft.TFT_EINVAL
