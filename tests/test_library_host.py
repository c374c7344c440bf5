"""CPU-only checks of the C library: it builds, loads, exports every symbol
that include/tft.h declares, and its host-side logic (planning, footprint,
argument checks that need no device) behaves.  No kernel is launched."""

import ctypes

import pytest

from paper_1001_5272_gb300 import build as B
from paper_1001_5272_gb300 import tft


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def test_exports_every_declared_symbol():
    declared = tft._header_functions()
    assert len(declared) >= 13
    L = tft.load()
    missing = [n for n in declared if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings():
    assert tft.status_string(0) == "ok"
    assert tft.status_string(1) == "invalid argument"
    assert tft.status_string(5) == "device wait timed out"


@pytest.mark.parametrize("pid", [0, 1, 2])
def test_plan_invariants(pid):
    w = 8 if pid == 2 else 4
    for e in range(0, 26 if w == 8 else 28):
        for n in {(1 << e) - 1, 1 << e, (1 << e) + 1, 3 << max(0, e - 2),
                  (1 << e) + 12345}:
            if n < 1:
                continue
            try:
                P = tft.tft_describe_plan(pid, n)
            except tft.TFTError as err:
                assert err.status == tft.TFT_ERANGE
                assert n > ((1 << 25) if w == 8 else (1 << 27))
                continue
            if P["small"]:
                assert n <= 1 << P["l"] and (P["l"] == 0 or n > 1 << (P["l"] - 1))
                continue
            R = 1 << P["lr"]
            assert P["a"] * R + P["b"] == n and 0 <= P["b"] < R
            assert P["a"] >= 1
            rows = P["a"] + (1 if P["b"] else 0)
            assert rows <= 1 << P["c"]
            assert (1 << P["clog"]) <= R
            assert 1 <= P["row_ctas_per_sm"] <= 4


def test_footprint_against_padded():
    # n = 2^24 + 2^20 + 12345 words of 8 bytes plus one R-word scratch,
    # against a padded 2^25 buffer.
    n = 2**24 + 2**20 + 12345
    inplace, padded = tft.tft_footprint(2, n, 25, 0)
    P = tft.tft_describe_plan(2, n)
    assert inplace == (n + (1 << P["lr"])) * 8
    assert padded == (1 << 25) * 8
    assert inplace < 0.54 * padded
    # product r = 8,000,000: out + work (+ two R-word scratches) vs 2 x 2^23
    inplace, padded = tft.tft_footprint(2, 8_000_000, 0, 1)
    P = tft.tft_describe_plan(2, 8_000_000)
    assert inplace == (2 * 8_000_000 + 2 * (1 << P["lr"])) * 8
    assert padded == 2 * (1 << 23) * 8
    with pytest.raises(tft.TFTError):
        tft.tft_footprint(2, 0, 0, 0)
    with pytest.raises(tft.TFTError):
        tft.tft_footprint(0, 1025, 10, 0)         # n > 2^k


def test_null_arguments_rejected_without_a_device():
    L = tft.load()
    assert L.tft_forward(None, ctypes.c_void_p(16), 4, 2, None) == tft.TFT_EINVAL
    assert L.tft_ctx_destroy(None) == tft.TFT_EINVAL
    h = ctypes.c_void_p()
    assert L.tft_ctx_create(7, 0, 16, 0, ctypes.byref(h)) == tft.TFT_EINVAL
    assert L.tft_ctx_create(0, 0, 0, 0, ctypes.byref(h)) == tft.TFT_EINVAL
    assert L.tft_ctx_create(2, 0, (1 << 25) + 1, 0,
                            ctypes.byref(h)) == tft.TFT_ERANGE
    assert L.tft_element_bytes(0) == 4 and L.tft_element_bytes(2) == 8
    assert L.tft_element_bytes(9) == 0


def test_noscratch_arguments_rejected_without_a_device():
    # argument errors come back before any CUDA call
    L = tft.load()
    for fn in (L.tft_forward_noscratch, L.tft_inverse_noscratch):
        assert fn(7, ctypes.c_void_p(16), 4, 2, None) == tft.TFT_EINVAL
        assert fn(2, None, 4, 2, None) == tft.TFT_EINVAL
        assert fn(2, ctypes.c_void_p(16), 0, 2, None) == tft.TFT_EINVAL
        assert fn(2, ctypes.c_void_p(16), 5, 2, None) == tft.TFT_EINVAL  # n > 2^k
        assert fn(2, ctypes.c_void_p(16), 4, 33, None) == tft.TFT_EINVAL  # k > K
        assert fn(2, ctypes.c_void_p(24), 4, 2, None) == tft.TFT_EINVAL  # alignment


def test_context_creation_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = tft.load()
    h = ctypes.c_void_p()
    st = L.tft_ctx_create(2, 0, 1024, 0, ctypes.byref(h))
    assert st in (tft.TFT_ECUDA, tft.TFT_EINVAL)
    assert not h.value


@pytest.mark.parametrize("pid", [0, 1, 2])
def test_batch_work_words(pid):
    # host-only sizing of the batched product's work area: each product of
    # the row/column class takes r words for B' plus two R-word E buffers,
    # each slot rounded up to 16 bytes; the single-CTA class takes none
    w = 8 if pid == 2 else 4
    small_log, lr = (12, 10) if w == 8 else (13, 9)
    al = 16 // w

    def up(x):
        return (x + al - 1) // al * al

    rng = __import__("random").Random(pid)
    pairs = [(1, 1), (1 << (small_log - 1), (1 << (small_log - 1)) + 1),
             (1 << (small_log - 1), (1 << (small_log - 1)) + 2),
             (65536, 65536)] + [(rng.randint(1, 40000), rng.randint(1, 40000))
                                for _ in range(20)]
    expect = 0
    for na, nb in pairs:
        r = na + nb - 1
        if r > (1 << small_log):
            expect += up(r) + 2 * up(1 << lr)
    assert tft.tft_batch_work_words(pid, pairs) == expect
    # an explicit schedule: everything above 2^8 in the row/column class
    expect8 = sum(up(na + nb - 1) + 2 * up(1 << 8) for na, nb in pairs
                  if na + nb - 1 > 256)
    assert tft.tft_batch_work_words(pid, pairs,
                                    {"lr": 8, "small_log": 8}) == expect8
    assert tft.tft_batch_work_words(pid, []) == 0
    with pytest.raises(tft.TFTError):
        tft.tft_batch_work_words(pid, [(0, 5)])


def test_batch_entry_points_reject_null_context():
    L = tft.load()
    assert L.tft_ctx_reserve_batch(None, 4, 100) == tft.TFT_EINVAL
    assert L.tft_batch_plan(None, None, 0, None) == tft.TFT_EINVAL
    assert L.tft_batch_run(None, None) == tft.TFT_EINVAL
    assert L.tft_polymul_batch(None, None, 0, None, None) == tft.TFT_EINVAL
    w = ctypes.c_uint64()
    assert L.tft_batch_work_words(7, None, 0, None, ctypes.byref(w)) == \
        tft.TFT_EINVAL


def test_autotune_grid_is_admissible():
    # every candidate schedule satisfies the constraints tft_batch_plan
    # checks, and the sizing entry point accepts it
    from paper_1001_5272_gb300 import autotune
    for pid in (0, 1, 2):
        grid = autotune.candidates(pid)
        assert grid
        for g in grid:
            assert 8 <= g["lr"] <= 12
            assert g["lr"] <= g["small_log"] <= (12 if pid == 2 else 13)
            assert 0 <= g["clog"] <= 5
            tft.tft_batch_work_words(pid, [(5000, 7000)], g)
    assert autotune.mix_signature([(1, 1), (2, 3), (3, 2), (64, 65)]) == \
        "0:1,2:2,7:1"


def test_restricted_schedule_follows_algorithm_3():
    # the chunk loop of Algorithm 3 (Section 5), checked through the
    # properties its proof states: the chunks partition [0, tail), L_i is a
    # power of two dividing q_i with q_i + 2 L_i <= r and is the largest such
    # power (so each L appears at most twice, in non-increasing order); the
    # device stops before the first chunk with L <= 2^16, so the tail holds
    # fewer than 2^18 positions
    import random
    rng = random.Random(5)
    sizes = [1, 2, 3, 2 ** 17, 2 ** 18 - 1, 2 ** 18, 2 ** 18 + 1, 8_000_000,
             2 ** 22 + 1, 2 ** 25] + [rng.randint(1, 2 ** 25) for _ in range(200)]
    for r in sizes:
        chunks, tail = tft.tft_restricted_schedule(r)
        q = 0
        seen = {}
        prevL = None
        for qi, L in chunks:
            assert qi == q and L & (L - 1) == 0 and qi % L == 0, (r, qi, L)
            assert qi + 2 * L <= r and qi + 4 * L > r, (r, qi, L)
            assert L > 2 ** 16
            assert prevL is None or L <= prevL
            seen[L] = seen.get(L, 0) + 1
            assert seen[L] <= 2
            prevL = L
            q += L
        assert tail == q and r - tail < 2 ** 18, (r, tail)
    with pytest.raises(tft.TFTError):
        tft.tft_restricted_schedule(0)


def test_allocation_injection_hooks_without_a_device():
    # the hooks are host state only: nothing is allocated here, and arming
    # and disarming an injected failure touches no device
    assert tft.tft_debug_live_allocations() == 0
    tft.tft_debug_fail_allocation(2)
    tft.tft_debug_fail_allocation(-1)
    assert tft.tft_debug_live_allocations() == 0
