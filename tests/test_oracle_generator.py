"""Pins of the oracle's served-workload generator (oracle/gen_c.c).

The generator is a workload convention, not part of the paper's method:
what matters is that the oracle and the device produce the same operands
(checked in the GPU tests) and that the stream is Philox4x32-10's.  Pinned
here, independently of the C code's own structure:
  * the round function against the generator's published known-answer
    vectors (tests/golden/philox4x32_10_kat.txt), which fix it exactly: a
    wrong constant, round count, key schedule or word order fails them;
  * the packing of the four words into v and the reduction mod p, against
    Python integers;
  * the counter layout (element index, operand, request split in two words)
    and the key layout, through which inputs change which outputs;
  * the round function is a bijection of the counter for a fixed key (no
    collisions on 2^16 counters), the output bits are balanced, and one
    flipped input bit changes about half of the output bits (a dropped
    multiplication or XOR term breaks these).
"""

import os

import numpy as np
import pytest

from oracle import field as F
from oracle import native as NV


GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def words_to_int(x):
    return x[0] | (x[1] << 32) | (x[2] << 64) | (x[3] << 96)


@pytest.mark.parametrize("pr", F.PRIME_BY_ID, ids=lambda p: p.name)
def test_gen_operand_is_packed_words_mod_p(pr):
    pid = F.PRIME_BY_ID.index(pr)
    seed, req = 4, (7 << 32) + 123
    for operand in (0, 1):
        got = NV.gen_operand(pid, seed, req, operand, 300)
        for i in (0, 1, 2, 150, 299):
            x = NV.philox4x32_10((i, operand, req & 0xFFFFFFFF, req >> 32),
                                 (seed & 0xFFFFFFFF, seed >> 32))
            assert int(got[i]) == words_to_int(x) % pr.p
        assert (got < pr.p).all()


def test_counter_and_key_layout_select_distinct_streams():
    a0 = NV.gen_operand(2, 4, 9, 0, 64)
    assert not np.array_equal(a0, NV.gen_operand(2, 4, 9, 1, 64))   # operand
    assert not np.array_equal(a0, NV.gen_operand(2, 4, 10, 0, 64))  # request
    assert not np.array_equal(a0, NV.gen_operand(2, 5, 9, 0, 64))   # seed
    assert not np.array_equal(a0,
                              NV.gen_operand(2, 4, 9 + (1 << 32), 0, 64))
    # a prefix of a longer operand is the shorter operand
    assert np.array_equal(a0[:10], NV.gen_operand(2, 4, 9, 0, 10))


def test_philox_is_injective_on_counters():
    seen = set()
    for i in range(1 << 16):
        out = NV.philox4x32_10((i, 0, 3, 0), (4, 0))
        seen.add(out)
    assert len(seen) == 1 << 16


def test_philox_bit_balance_and_avalanche():
    rng = np.random.default_rng(1)
    counts = np.zeros(128)
    flips = []
    n = 4096
    for _ in range(n):
        c = [int(v) for v in rng.integers(0, 1 << 32, 4, dtype=np.uint64)]
        k = [int(v) for v in rng.integers(0, 1 << 32, 2, dtype=np.uint64)]
        v = words_to_int(NV.philox4x32_10(c, k))
        counts += [(v >> b) & 1 for b in range(128)]
        bit = int(rng.integers(0, 192))
        if bit < 128:
            c2 = list(c)
            c2[bit // 32] ^= 1 << (bit % 32)
            v2 = words_to_int(NV.philox4x32_10(c2, k))
        else:
            k2 = list(k)
            k2[(bit - 128) // 32] ^= 1 << ((bit - 128) % 32)
            v2 = words_to_int(NV.philox4x32_10(c, k2))
        flips.append(bin(v ^ v2).count("1"))
    # each output bit: mean 1/2, standard deviation 1/(2 sqrt(n)) ~ 0.0078
    assert np.all(np.abs(counts / n - 0.5) < 0.04)
    # one input bit flips 64 of 128 output bits on average (binomial sd 5.7)
    assert abs(np.mean(flips) - 64) < 1.0
    assert min(flips) > 25


def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN,
                                                 "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        w = [int(v, 16) for v in row]
        assert NV.philox4x32_10(w[0:4], w[4:6]) == tuple(w[6:10]), row
