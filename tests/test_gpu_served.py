"""GPU parity of the served path: the device operand generator against the
oracle's, and every served product against the product of the same
request computed alone (single call) and by the oracle, bit for bit.

A request served inside a mix of other requests (continuous batching,
shared budget, other products in the same launches) must give exactly the
result it gives alone.
"""

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
    out = {i: tft.Context(i, 0, max_len=1 << 18) for i in range(3)}
    yield out
    for c in out.values():
        c.close()


def _tdtype(pid):
    return torch.int64 if pid == 2 else torch.int32


def to_host(pid, t):
    a = t.cpu().numpy()
    return a.view(np.uint64) if pid == 2 else a.view(np.uint32).astype(
        np.uint64)


def schedule(n, rate, lo, hi, seed):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    u = rng.random((2, n))
    L = np.clip(np.floor(lo * (hi / lo) ** u), lo, hi).astype(np.int64)
    return t, L[0], L[1]


@pytest.mark.parametrize("pid", [0, 1, 2])
def test_generator_matches_oracle(ctxs, pid):
    tft = _lib()
    ctx = ctxs[pid]
    for req, operand, n in [(0, 0, 1), (5, 1, 1000), (123456789, 0, 4099),
                            ((3 << 32) + 17, 1, 70001)]:
        t = torch.empty(n, dtype=_tdtype(pid), device="cuda")
        tft.tft_generate(ctx, 4, req, operand, t)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(pid, t),
                              NV.gen_operand(pid, 4, req, operand, n)), \
            (req, operand, n)


@pytest.mark.parametrize("pid", [2, 1])
def test_served_mix_equals_alone_and_oracle(ctxs, pid):
    # 400 requests at 20,000/s, lengths log-uniform in [256, 2^14]: every
    # product kept and checked at a random point; every 16th also element
    # by element against the oracle and against the same request computed
    # alone through the single-call product
    tft = _lib()
    ctx = ctxs[pid]
    t, na, nb = schedule(400, 20000.0, 256, 1 << 14, 40 + pid)
    ids = np.arange(1000, 1400)
    keep = {i: torch.empty(int(na[i] + nb[i] - 1), dtype=_tdtype(pid),
                           device="cuda") for i in range(400)}
    with tft.Server(ctx, 1 << 30, max_batch=512) as srv:
        done, st = srv.replay(ids, na, nb, t, seed=4, keep=keep)
    torch.cuda.synchronize()
    assert st["completed"] == 400 and st["batches"] >= 1
    assert np.all(done >= t - 1e-3)  # no request completes before it arrives
    p = PRIMES[pid].p
    rng = np.random.default_rng(7)
    for i in range(400):
        a = NV.gen_operand(pid, 4, int(ids[i]), 0, int(na[i]))
        b = NV.gen_operand(pid, 4, int(ids[i]), 1, int(nb[i]))
        c = to_host(pid, keep[i])
        z = int(rng.integers(2, p, dtype=np.uint64))
        assert NV.eval_at(pid, c, z) == \
            NV.eval_at(pid, a, z) * NV.eval_at(pid, b, z) % p, i
        if i % 16 == 0:
            assert np.array_equal(c, NV.tft_polymul(pid, a, b)), i
            ta = torch.empty(int(na[i]), dtype=_tdtype(pid), device="cuda")
            tb = torch.empty(int(nb[i]), dtype=_tdtype(pid), device="cuda")
            tft.tft_generate(ctx, 4, int(ids[i]), 0, ta)
            tft.tft_generate(ctx, 4, int(ids[i]), 1, tb)
            alone = torch.empty_like(keep[i])
            tft.tft_polymul(ctx, ta, tb, alone)
            torch.cuda.synchronize()
            assert torch.equal(alone, keep[i]), i


@pytest.mark.parametrize("params", [
    None, {"small_log": 12, "lr": 11, "clog": 4}],
    ids=["default", "sl12-lr11-c4"])
def test_served_full_length_range(params):
    # 64 requests of the served workload's shape over 2^64 - 2^32 + 1:
    # 20,000 requests/s, operand lengths log-uniform in [256, 2^20], one
    # request at the longest (r = 2^21 - 1), an 8 GB budget, under the
    # default schedule and the one the serving benchmark runs.  Every
    # product is checked at a random point (Schwartz-Zippel) and on sampled
    # coefficients by their defining sums; the longest and every 16th
    # element by element against the oracle and against the same request
    # computed alone through the single-call product.
    tft = _lib()
    pid = 2
    p = PRIMES[pid].p
    t, na, nb = schedule(64, 20000.0, 256, 1 << 20, 71)
    na[5] = nb[5] = 1 << 20
    ids = np.arange(5000, 5064)
    with tft.Context(pid, 0, max_len=1 << 21) as ctx:
        keep = {i: torch.empty(int(na[i] + nb[i] - 1), dtype=torch.int64,
                               device="cuda") for i in range(64)}
        with tft.Server(ctx, 8 << 30, max_batch=4096, params=params) as srv:
            done, st = srv.replay(ids, na, nb, t, seed=4, keep=keep)
        torch.cuda.synchronize()
        assert st["completed"] == 64
        rng = np.random.default_rng(73)
        for i in range(64):
            a = NV.gen_operand(pid, 4, int(ids[i]), 0, int(na[i]))
            b = NV.gen_operand(pid, 4, int(ids[i]), 1, int(nb[i]))
            c = to_host(pid, keep[i])
            r = c.size
            z = int(rng.integers(2, p, dtype=np.uint64))
            assert NV.eval_at(pid, c, z) == \
                NV.eval_at(pid, a, z) * NV.eval_at(pid, b, z) % p, i
            for t_ in {0, r - 1} | {int(v) for v in rng.integers(0, r, 6)}:
                assert int(c[t_]) == NV.conv_coeff(pid, a, b, t_), (i, t_)
            if i % 16 == 0 or i == 5:
                assert np.array_equal(c, NV.tft_polymul(pid, a, b)), i
                ta = torch.empty(int(na[i]), dtype=torch.int64, device="cuda")
                tb = torch.empty(int(nb[i]), dtype=torch.int64, device="cuda")
                tft.tft_generate(ctx, 4, int(ids[i]), 0, ta)
                tft.tft_generate(ctx, 4, int(ids[i]), 1, tb)
                alone = torch.empty_like(keep[i])
                tft.tft_polymul(ctx, ta, tb, alone)
                torch.cuda.synchronize()
                assert torch.equal(alone, keep[i]), i


def test_one_by_one_equals_batched_and_budget_holds(ctxs):
    # the comparison path gives the same products; a small budget forces
    # many batches and its peak stays within it
    tft = _lib()
    pid = 2
    ctx = ctxs[pid]
    t, na, nb = schedule(300, 50000.0, 256, 1 << 15, 9)
    ids = np.arange(300) + 77
    budget = 24 << 20
    keep_b = {i: torch.empty(int(na[i] + nb[i] - 1), dtype=torch.int64,
                             device="cuda") for i in range(300)}
    keep_p = {i: torch.empty_like(keep_b[i]) for i in range(300)}
    with tft.Server(ctx, budget, max_batch=64) as srv:
        done_b, st_b = srv.replay(ids, na, nb, t, seed=4, keep=keep_b)
        done_p, st_p = srv.replay(ids, na, nb, t, seed=4, mode="one_by_one",
                                  keep=keep_p)
    torch.cuda.synchronize()
    for i in range(300):
        assert torch.equal(keep_b[i], keep_p[i]), i
    assert st_b["completed"] == st_p["completed"] == 300
    assert st_b["peak_bytes"] <= budget
    assert st_b["max_batch"] <= 64 and st_b["batches"] >= 300 // 64
    assert st_p["batches"] == 300
    assert np.all(done_b >= t - 1e-3) and np.all(done_p >= t - 1e-3)
    # completion in arrival order for the one-by-one path
    assert np.all(np.diff(done_p) >= 0)


def test_server_argument_errors(ctxs):
    tft = _lib()
    ctx = ctxs[2]
    with tft.Server(ctx, 1 << 20, max_batch=8) as srv:
        with pytest.raises(tft.TFTError) as e:  # arrivals not sorted
            srv.replay([1, 2], [300, 300], [300, 300], [0.002, 0.001], 4)
        assert e.value.status == tft.TFT_EINVAL
        with pytest.raises(tft.TFTError) as e:  # larger than the budget
            srv.replay([1], [1 << 17], [1 << 17], [0.0], 4)
        assert e.value.status == tft.TFT_ERANGE
        with pytest.raises(tft.TFTError) as e:  # empty operand
            srv.replay([1], [0], [5], [0.0], 4)
        assert e.value.status == tft.TFT_EINVAL
        # still usable afterwards
        keep = {0: torch.empty(599, dtype=torch.int64, device="cuda")}
        done, st = srv.replay([3], [300], [300], [0.0], 4, keep=keep)
        torch.cuda.synchronize()
        a = NV.gen_operand(2, 4, 3, 0, 300)
        b = NV.gen_operand(2, 4, 3, 1, 300)
        assert np.array_equal(to_host(2, keep[0]), NV.tft_polymul(2, a, b))
