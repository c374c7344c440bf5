"""Failure handling on the host: device and pinned-host allocation failures
at context creation, batch reservation and server creation.

The failures are made on the host (the library's allocation wrapper is told
to fail one allocation without calling CUDA), or by asking for more memory
than the device has, which the CUDA runtime refuses without touching the
GPU's state.  Each failing call must return TFT_ENOMEM, release whatever it
had allocated (the library's live-allocation count returns to where it
was), and leave the library usable: a context, batch or server created
afterwards computes bit-exact products (checked against the oracle).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import native as NV  # noqa: E402

P_GOLD = 2**64 - 2**32 + 1


@pytest.fixture(scope="module")
def tft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_5272_gb300 import tft as lib
    yield lib
    lib.tft_debug_fail_allocation(-1)


def _rand(n, seed):
    return np.random.default_rng(seed).integers(0, P_GOLD, n, dtype=np.uint64)


def _dev(x):
    return torch.from_numpy(x.view(np.int64).copy()).cuda()


def _check_product(tft, ctx, seed):
    a, b = _rand(3000, seed), _rand(5001, seed + 1)
    out = torch.empty(a.size + b.size - 1, dtype=torch.int64, device="cuda")
    tft.tft_polymul(ctx, _dev(a), _dev(b), out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint64),
                          NV.tft_polymul(2, a, b))


def test_context_creation_allocation_failures(tft):
    # a context with host staging makes three device allocations (scratch,
    # product work buffer, staging); failing each in turn gives TFT_ENOMEM
    # and leaks nothing
    base = tft.tft_debug_live_allocations()
    failed = 0
    for n in range(6):
        tft.tft_debug_fail_allocation(n)
        try:
            ctx = tft.Context(2, 0, max_len=1 << 16, host_staging=True)
        except tft.TFTError as e:
            assert e.status == tft.TFT_ENOMEM, n
            assert tft.tft_debug_live_allocations() == base, n
            failed += 1
            continue
        tft.tft_debug_fail_allocation(-1)
        assert tft.tft_debug_live_allocations() == base + 3
        _check_product(tft, ctx, 10 + n)
        ctx.close()
        assert tft.tft_debug_live_allocations() == base
    assert failed == 3


def test_batch_reservation_allocation_failures(tft):
    with tft.Context(2, 0, max_len=1 << 16) as ctx:
        base = tft.tft_debug_live_allocations()
        pairs = [(3000, 5001), (20000, 30000), (100, 7)]
        words = tft.tft_batch_work_words(2, pairs)
        for n in (0, 1):
            tft.tft_debug_fail_allocation(n)
            with pytest.raises(tft.TFTError) as e:
                tft.tft_ctx_reserve_batch(ctx, len(pairs), words)
            assert e.value.status == tft.TFT_ENOMEM
            assert tft.tft_debug_live_allocations() == base
        tft.tft_debug_fail_allocation(-1)
        # nothing reserved after the failures: planning is refused
        A = [_rand(na, 20 + i) for i, (na, _) in enumerate(pairs)]
        B = [_rand(nb, 30 + i) for i, (_, nb) in enumerate(pairs)]
        prods = [(_dev(a), _dev(b),
                  torch.empty(a.size + b.size - 1, dtype=torch.int64,
                              device="cuda")) for a, b in zip(A, B)]
        with pytest.raises(tft.TFTError) as e:
            tft.tft_batch_plan(ctx, prods)
        assert e.value.status == tft.TFT_EINVAL
        # a reservation that succeeds, and the batch is exact
        tft.tft_ctx_reserve_batch(ctx, len(pairs), words)
        assert tft.tft_debug_live_allocations() == base + 2
        tft.tft_polymul_batch(ctx, prods)
        torch.cuda.synchronize()
        for (_, _, o), a, b in zip(prods, A, B):
            assert np.array_equal(o.cpu().numpy().view(np.uint64),
                                  NV.tft_polymul(2, a, b))
        _check_product(tft, ctx, 40)


def _serve_and_check(tft, ctx, srv, first_id):
    ids = np.arange(first_id, first_id + 24)
    rng = np.random.default_rng(first_id)
    na = rng.integers(256, 5000, 24)
    nb = rng.integers(256, 5000, 24)
    t = np.cumsum(rng.exponential(1 / 20000.0, 24))
    keep = {i: torch.empty(int(na[i] + nb[i] - 1), dtype=torch.int64,
                           device="cuda") for i in range(24)}
    done, st = srv.replay(ids, na, nb, t, seed=4, keep=keep)
    torch.cuda.synchronize()
    assert st["completed"] == 24
    for i in range(0, 24, 5):
        a = NV.gen_operand(2, 4, int(ids[i]), 0, int(na[i]))
        b = NV.gen_operand(2, 4, int(ids[i]), 1, int(nb[i]))
        assert np.array_equal(keep[i].cpu().numpy().view(np.uint64),
                              NV.tft_polymul(2, a, b)), i


def test_server_creation_allocation_failures(tft):
    # a server allocates its budget, then per slot a device and a pinned
    # host table (two slots): five allocations, each failed in turn
    with tft.Context(2, 0, max_len=1 << 16) as ctx:
        base = tft.tft_debug_live_allocations()
        failed = 0
        for n in range(7):
            tft.tft_debug_fail_allocation(n)
            try:
                srv = tft.Server(ctx, 64 << 20, max_batch=64)
            except tft.TFTError as e:
                assert e.status == tft.TFT_ENOMEM, n
                assert tft.tft_debug_live_allocations() == base, n
                failed += 1
                continue
            tft.tft_debug_fail_allocation(-1)
            _serve_and_check(tft, ctx, srv, 100 * n)
            srv.close()
            assert tft.tft_debug_live_allocations() == base
        assert failed == 5


def test_budget_larger_than_the_device(tft):
    # a real allocation failure: a budget of 2^50 bytes; the runtime's error
    # is cleared, so the next launches are not reported as failed
    with tft.Context(2, 0, max_len=1 << 16) as ctx:
        base = tft.tft_debug_live_allocations()
        with pytest.raises(tft.TFTError) as e:
            tft.Server(ctx, 1 << 50, max_batch=64)
        assert e.value.status == tft.TFT_ENOMEM
        assert tft.tft_debug_live_allocations() == base
        _check_product(tft, ctx, 50)
        with tft.Server(ctx, 64 << 20, max_batch=64) as srv:
            _serve_and_check(tft, ctx, srv, 7000)
        assert tft.tft_last_error(ctx) == tft.TFT_OK
