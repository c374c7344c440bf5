"""Batched transforms of uneven lengths (tft_transform_batch) against the
oracle: every buffer's forward TFT equals Algorithm 1 on it alone and the
batched inverse returns every input, bit for bit, with single-CTA lengths
(one persistent launch) and row/column lengths (one after another) mixed in
one batch."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import field as F  # noqa: E402
from oracle import native as NV  # noqa: E402


@pytest.fixture(scope="module")
def tft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_5272_gb300 import tft as lib
    return lib


def _dev(pid, x):
    if pid == 2:
        return torch.from_numpy(x.view(np.int64).copy()).cuda()
    return torch.from_numpy(x.astype(np.uint32).view(np.int32)).cuda()


def _host(pid, t):
    a = t.cpu().numpy()
    return a.view(np.uint64) if pid == 2 else \
        a.view(np.uint32).astype(np.uint64)


@pytest.mark.parametrize("pid", [2, 1, 0])
def test_batched_transforms_match_the_oracle(tft, pid):
    p = F.PRIME_BY_ID[pid].p
    rng = np.random.default_rng(80 + pid)
    lens = [1, 2, 3, 17, 64, 255, 1000, 4095, 4096, 4097, 8191, 8192, 8193,
            12345, 70001, 100003]
    lens += [int(v) for v in np.floor(64 * 1024.0 ** rng.random(40))]
    xs = [rng.integers(0, p, n, dtype=np.uint64) for n in lens]
    with tft.Context(pid, 0, max_len=max(lens)) as ctx:
        tft.tft_ctx_reserve_batch(ctx, len(lens), 0)
        ts = [_dev(pid, x) for x in xs]
        tft.tft_transform_batch(ctx, ts)
        torch.cuda.synchronize()
        for n, x, t in zip(lens, xs, ts):
            assert np.array_equal(_host(pid, t), NV.alg1_tft(pid, x)), n
        tft.tft_transform_batch(ctx, ts, inverse=True)
        torch.cuda.synchronize()
        for n, x, t in zip(lens, xs, ts):
            assert np.array_equal(_host(pid, t), x), n


def test_batched_transforms_equal_single_calls_and_errors(tft):
    pid = 2
    rng = np.random.default_rng(5)
    lens = [int(v) for v in np.floor(64 * 1024.0 ** rng.random(300))]
    xs = [rng.integers(0, F.PRIME_BY_ID[pid].p, n, dtype=np.uint64)
          for n in lens]
    with tft.Context(pid, 0, max_len=max(lens)) as ctx:
        ts = [_dev(pid, x) for x in xs]
        with pytest.raises(tft.TFTError) as e:     # nothing reserved
            tft.tft_transform_batch(ctx, ts)
        assert e.value.status == tft.TFT_ERANGE
        tft.tft_ctx_reserve_batch(ctx, len(lens), 0)
        tft.tft_transform_batch(ctx, ts)
        for x, t in zip(xs, ts):
            one = _dev(pid, x)
            tft.tft_forward(ctx, one)
            assert torch.equal(one, t)
        big = torch.zeros(max(lens) + 16, dtype=torch.int64, device="cuda")
        with pytest.raises(tft.TFTError) as e:     # beyond max_len
            tft.tft_transform_batch(ctx, [big])
        assert e.value.status == tft.TFT_ERANGE
        buf = torch.zeros(4096, dtype=torch.int64, device="cuda")
        with pytest.raises(tft.TFTError) as e:     # overlapping buffers
            tft.tft_transform_batch(ctx, [buf[:2048], buf[1024:3072]])
        assert e.value.status == tft.TFT_EINVAL
        assert tft.tft_last_error(ctx) == tft.TFT_OK
