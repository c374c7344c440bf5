"""The sharded transform on one GPU: every part's device steps through the
C ABI (tft_shard_columns / tft_shard_rows / tft_shard_last_row), the parts
held in one process and the exchanges done as copies (the host code of
paper_1001_5272_gb300/shard.py, whose distributed driver the CPU tests run
on gloo ranks).  No kernel waits on another; the steps are ordered by the
host.  Results must equal the oracle's Algorithm 1 / Algorithm 2 and the
unsharded tft_forward / tft_inverse bit for bit."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import field as F  # noqa: E402
from oracle import native as NV  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_5272_gb300 import shard, tft
    return tft, shard


def _x(pid, n, seed):
    p = F.PRIME_BY_ID[pid].p
    return np.random.default_rng(seed).integers(0, p, n, dtype=np.uint64)


def _dev(pid, x):
    if pid == 2:
        return torch.from_numpy(x.view(np.int64).copy()).cuda()
    return torch.from_numpy(x.astype(np.uint32).view(np.int32)).cuda()


def _host(pid, t):
    a = t.cpu().numpy()
    return a.view(np.uint64) if pid == 2 else \
        a.view(np.uint32).astype(np.uint64)


def _run(lib, pid, n, parts, seed, check_oracle=True):
    tft, shard = lib
    x = _x(pid, n, seed)
    L = shard.Layout.for_plan(tft.tft_describe_plan(pid, n), n, parts)
    with tft.Context(pid, 0, max_len=n) as ctx:
        ops = shard.GpuOps(ctx, L)
        xd = _dev(pid, x)
        rows, last = shard.forward_local(L, ops, [L.block_of(xd, p)
                                                  for p in range(parts)])
        X = L.vector_of_rows(rows, last)
        want = xd.clone()
        tft.tft_forward(ctx, want)
        torch.cuda.synchronize()
        assert torch.equal(X, want), (n, parts)
        if check_oracle:
            assert np.array_equal(_host(pid, X), NV.alg1_tft(pid, x))
        blocks = shard.inverse_local(L, ops, [L.rows_piece(X, p)
                                              for p in range(parts)],
                                     L.last_piece(X) if L.b else None)
        back = L.vector_of_blocks(blocks)
        torch.cuda.synchronize()
        assert np.array_equal(_host(pid, back), x), (n, parts)


@pytest.mark.parametrize("pid", [2, 1, 0])
@pytest.mark.parametrize("n", [70001, 70144, 300001, (1 << 20) + 12345])
@pytest.mark.parametrize("parts", [1, 2, 4, 8])
def test_sharded_transform_matches_oracle(lib, pid, n, parts):
    _run(lib, pid, n, parts, n + parts)


@pytest.mark.parametrize("parts", [2, 8, 64])
def test_sharded_transform_full_size(lib, parts):
    # n = 2^24 + 2^20 + 12345 over 2^64 - 2^32 + 1 (rows of 2^13, a ragged
    # last row of 4153 outputs) in 2, 8 and 64 parts, against the unsharded
    # transform
    _run(lib, 2, (1 << 24) + (1 << 20) + 12345, parts, 1, check_oracle=False)


def test_shard_argument_errors(lib):
    tft, _ = lib
    with tft.Context(2, 0, max_len=1 << 16) as ctx:
        blk = torch.zeros(137 * 128, dtype=torch.int64, device="cuda")
        E = torch.zeros(128, dtype=torch.int64, device="cuda")
        for bad in ((3, 0), (4, 4), (0, 0)):       # parts, part
            with pytest.raises(tft.TFTError) as e:
                tft.tft_shard_columns(ctx, 0, 0, blk, 70001, bad[0], bad[1],
                                      E)
            assert e.value.status == tft.TFT_EINVAL
        with pytest.raises(tft.TFTError) as e:     # single-CTA plan
            tft.tft_shard_columns(ctx, 0, 0, blk, 3000, 2, 0, E)
        assert e.value.status == tft.TFT_EINVAL
        with pytest.raises(tft.TFTError) as e:     # short columns need E
            tft.tft_shard_columns(ctx, 0, 0, blk, 70001, 4, 3, None)
        assert e.value.status == tft.TFT_EINVAL
        rows = torch.zeros(512 * 3, dtype=torch.int64, device="cuda")
        with pytest.raises(tft.TFTError) as e:     # rows beyond a = 136
            tft.tft_shard_rows(ctx, 0, rows.view(3, 512), 70001, 134, 3)
        assert e.value.status == tft.TFT_EINVAL
        assert tft.tft_last_error(ctx) == tft.TFT_OK
