"""The allocation-free forward TFT entry point, against the context one and
against the oracle.

Some callers cannot allocate device memory once they are running -- a
serving loop whose device memory is reserved at start-up, or code inside an
allocator callback -- so they cannot create a context.  tft_forward_noalloc
serves them with a fixed device array as scratch.  These tests call it
through the C ABI and require bit-for-bit the result of tft_forward and of
the oracle's Algorithm 1 (the tolerance of every parity test here is zero:
the arithmetic is exact), on two calls in a row that reuse the shared array
with different lengths.  The file is named to be collected last; the last
test runs the others again in a fresh Python process, so that they also
pass when the entry point's first call is the process's first.
"""

import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import native as NV  # noqa: E402

P_GOLD = 2**64 - 2**32 + 1


def _rand(n, seed):
    return np.random.default_rng(seed).integers(0, P_GOLD, n, dtype=np.uint64)


def _dev(x):
    return torch.from_numpy(x.view(np.int64).copy()).cuda()


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_5272_gb300 import tft
    return tft


def test_noalloc_matches_context_path_on_consecutive_calls(lib):
    # Both lengths use the two-pass plan with a ragged last row, so the
    # fixed scratch is written and read on each call; the second call sees
    # the first call's leftovers.
    sizes = [(1 << 20) + 12345, 3 * (1 << 17) + 5]
    with lib.Context(2, 0, max_len=max(sizes)) as ctx:
        for i, n in enumerate(sizes):
            x = _rand(n, 40 + i)
            want = _dev(x)
            lib.tft_forward(ctx, want)
            got = _dev(x)
            lib.tft_forward_noalloc(2, got)
            torch.cuda.synchronize()
            assert torch.equal(got, want), f"call {i} (n={n}) differs"
            ref = NV.alg1_tft(2, x)
            assert np.array_equal(got.cpu().numpy().view(np.uint64), ref), \
                f"call {i} (n={n}) differs from Algorithm 1"


def test_noalloc_small_and_32bit_prime(lib):
    # a single-CTA length and a two-pass length of a 32-bit prime, back to
    # back, against the context path and the oracle
    p = 2013265921
    for pid, n, seed in ((1, 3001, 7), (1, 200003, 8)):
        x = np.random.default_rng(seed).integers(0, p, n, dtype=np.uint64)
        x32 = x.astype(np.uint32).view(np.int32)
        with lib.Context(pid, 0, max_len=n) as ctx:
            want = torch.from_numpy(x32.copy()).cuda()
            lib.tft_forward(ctx, want)
        got = torch.from_numpy(x32.copy()).cuda()
        lib.tft_forward_noalloc(pid, got)
        torch.cuda.synchronize()
        assert torch.equal(got, want), n
        got64 = got.cpu().numpy().view(np.uint32).astype(np.uint64)
        assert np.array_equal(got64, NV.alg1_tft(pid, x)), n


def test_noalloc_rejects_sizes_beyond_its_limit(lib):
    big = torch.zeros((1 << 25) + 16, dtype=torch.int64, device="cuda")
    with pytest.raises(lib.TFTError) as e:
        lib.tft_forward_noalloc(2, big, k=26)         # beyond 2^25 words
    assert e.value.status == lib.TFT_ERANGE
    x = torch.zeros(1024, dtype=torch.int64, device="cuda")
    with pytest.raises(lib.TFTError) as e:
        lib.tft_forward_noalloc(2, x, k=9)            # n > 2^k
    assert e.value.status == lib.TFT_EINVAL
    with pytest.raises(lib.TFTError) as e:
        lib.tft_forward_noalloc(2, x[1:], k=10)       # misaligned
    assert e.value.status == lib.TFT_EINVAL


@pytest.mark.skipif(os.environ.get("TFT_NOALLOC_CHILD") == "1",
                    reason="already the fresh process")
def test_noalloc_tests_pass_in_a_fresh_process(lib):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, TFT_NOALLOC_CHILD="1")
    res = subprocess.run(
        [sys.executable, "-m", "pytest", os.path.abspath(__file__), "-q",
         "-m", "gpu", "-p", "no:cacheprovider"],
        cwd=root, env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-2000:]
    assert "3 passed" in res.stdout, res.stdout[-2000:]
