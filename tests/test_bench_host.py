"""Host-side pieces of bench.py (no GPU): the algorithmic work behind the
roofline figure must be the butterfly count of Algorithm 1's tree (Section 3),
which the oracle counts from its own tree walk."""

import pytest

import bench
from oracle import tft as T


@pytest.mark.parametrize("n", [2, 3, 5, 17, 64, 100, 1000, 4097, 65537,
                               8_000_000])
def test_level_butterflies_sum_to_the_tree_count(n):
    assert sum(bench.tree_level_butterflies(n)) == T.butterfly_multiplies(n)


def test_level_butterflies_of_a_power_of_two():
    # every level of a full tree of 2^k leaves has 2^(k-1) butterflies
    for k in range(1, 16):
        assert bench.tree_level_butterflies(1 << k) == [1 << (k - 1)] * k


def test_kernel_modmuls_split_rows_and_columns():
    # the row pass takes the lr lowest levels of three transforms plus the
    # r pointwise products; the column passes the levels from lr up
    r = 8_000_000
    plan = {"lr": 12}
    bf = bench.tree_level_butterflies(r)
    w = bench.kernel_modmuls(plan, r)
    assert w["k_row_mul"] == 3 * sum(bf[:12]) + r
    assert w["k_col_fwd"] == sum(bf[12:])
    assert w["k_col_inv"] == sum(bf[12:])
    assert sum(bf) == T.butterfly_multiplies(r)
