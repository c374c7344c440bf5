"""CPU-only checks of the server's host logic: the arena's first-fit
policy against a plain model, its coalescing, and the admission footprint of
a request.  No device is used."""

import random

import pytest

from paper_1001_5272_gb300 import build as B
from paper_1001_5272_gb300 import tft


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


class ModelArena:
    """First fit over the sorted free ranges, merging neighbours on free."""

    def __init__(self, size, align):
        self.align = align
        self.size = size // align * align
        self.free = [(0, self.size)]
        self.live = {}

    def alloc(self, n):
        need = (max(n, 1) + self.align - 1) // self.align * self.align
        for k, (o, ln) in enumerate(self.free):
            if ln >= need:
                if ln > need:
                    self.free[k] = (o + need, ln - need)
                else:
                    del self.free[k]
                self.live[o] = need
                return o
        return None

    def release(self, o):
        ln = self.live.pop(o)
        self.free.append((o, ln))
        self.free.sort()
        merged = []
        for a, b in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + b)
            else:
                merged.append((a, b))
        self.free = merged


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_arena_matches_first_fit_model(seed):
    rng = random.Random(seed)
    size, align = 1 << 24, 256
    a = tft.Arena(size, align)
    m = ModelArena(size, align)
    live = []
    peak = 0
    for step in range(4000):
        if live and (rng.random() < 0.45 or len(live) > 200):
            o = live.pop(rng.randrange(len(live)))
            a.free(o)
            m.release(o)
        else:
            n = int(2 ** rng.uniform(0, 20))
            got, want = a.alloc(n), m.alloc(n)
            assert got == want, (step, n)
            if got is not None:
                live.append(got)
        used = sum(m.live.values())
        peak = max(peak, used)
        u = a.usage()
        assert u["used"] == used
        assert u["free_ranges"] == len(m.free)
        # live ranges are aligned and disjoint
        spans = sorted((o, m.live[o]) for o in m.live)
        for (o1, l1), (o2, _) in zip(spans, spans[1:]):
            assert o1 % align == 0 and o1 + l1 <= o2
    assert a.usage()["peak"] == peak
    for o in live:
        a.free(o)
    assert a.usage()["used"] == 0 and a.usage()["free_ranges"] == 1
    a.close()


def test_arena_errors_and_exhaustion():
    a = tft.Arena(4096, 256)
    offs = [a.alloc(1000) for _ in range(4)]
    assert offs == [0, 1024, 2048, 3072]
    assert a.alloc(1) is None  # full
    with pytest.raises(tft.TFTError):
        a.free(5)  # not an allocated offset
    a.free(1024)
    a.free(2048)  # neighbours merge into one 2048-byte range
    assert a.usage()["free_ranges"] == 1
    assert a.alloc(2048) == 1024
    a.close()
    with pytest.raises(tft.TFTError):
        tft.Arena(4096, 100)  # alignment not a power of two


@pytest.mark.parametrize("pid", [0, 1, 2])
def test_request_bytes(pid):
    # a | b | out | work, each rounded up to 256 bytes; work only for the
    # row/column class (r above 2^small_log)
    w = 8 if pid == 2 else 4
    small_log, lr = (12, 10) if w == 8 else (13, 9)
    al = 16 // w

    def up(x):
        return (x + 255) // 256 * 256

    for na, nb in [(1, 1), (256, 256), (1000, 3097), (4096, 4097),
                   (70000, 1 << 20), (1 << 20, 1 << 20)]:
        r = na + nb - 1
        work = 0
        if r > (1 << small_log):
            rw = (r + al - 1) // al * al
            Rw = ((1 << lr) + al - 1) // al * al
            work = (rw + 2 * Rw) * w
        want = up(na * w) + up(nb * w) + up(r * w) + up(work)
        assert tft.tft_request_bytes(pid, na, nb) == want, (na, nb)
    with pytest.raises(tft.TFTError):
        tft.tft_request_bytes(pid, 0, 5)
