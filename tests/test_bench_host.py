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


def test_leg_roofline_picks_the_slower_bound():
    pk = bench.modmul_peaks()[2]["peak_modmul_per_s"]
    bw, _ = bench.hbm_peak_gbs()
    # 1 G modmuls in 10 ms: multiply-bound unless the bytes dominate
    r = bench.leg_roofline(10.0, 10**9, 10**6, 2)
    assert r["bound"] == "alu" and r["unit"] == "Gmodmul/s"
    assert r["frac"] == pytest.approx((10**9 / pk) / 0.010)
    assert r["achieved"] == pytest.approx(100.0)
    # few modmuls, many bytes: HBM-bound
    r = bench.leg_roofline(10.0, 10**3, 10**10, 2)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx((10**10 / (bw * 1e9)) / 0.010)


def test_kernel_keys_of_ncu_names():
    k = bench.kernel_key
    assert k("void tftgb::k_row_mul2<tftgb::Goldilocks, 12>(T1::T *, "
             "const T1::T *)") == "k_row_mul2<goldilocks>"
    assert k("void <unnamed>::k_calib_modmul<tftgb::Mont32<2013265921, "
             "2013265919, 1172168163, 268435454, 27, 1>>(T1::T *, unsigned "
             "int)") == "k_calib_modmul<p2013265921>"
    assert k("<unnamed>::k_calib_mad32(unsigned int *, unsigned int)") == \
        "k_calib_mad32"
    assert k("k_gen_pair(unsigned long *, unsigned long)") == "k_gen_pair"


def test_ncu_summary_of_a_csv(tmp_path):
    # two launches of one kernel with DRAM counters, one calibration launch
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name",
           "Context", "Stream", "Metric Name", "Metric Unit",
           "Metric Value"]
    rows = []
    for i, (rd, wr, t) in enumerate(((100, 50, 1000), (300, 150, 3000))):
        name = "void tftgb::k_row_mul2<tftgb::Goldilocks, 12>(T1::T *)"
        for m, v in (("dram__bytes_read.sum", rd),
                     ("dram__bytes_write.sum", wr),
                     ("gpu__time_duration.sum", t)):
            rows.append([str(i), "1", "py", "h", name, "1", "7", m, "x",
                         f"{v:,}"])
    for m, v in (("launch__grid_size", 2), ("gpu__time_duration.sum", 4000),
                 ("sm__pipe_fmaheavy_cycles_active.sum", 4096)):
        rows.append(["2", "1", "py", "h",
                     "<unnamed>::k_calib_mad32(unsigned int *, unsigned int)",
                     "1", "7", m, "x", str(v)])
    p = tmp_path / "n.csv"
    import csv
    with open(p, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(hdr)
        w.writerows(rows)
    s = bench.ncu_summary(str(p), calib_iters=1)
    rm = s["kernels"]["k_row_mul2<goldilocks>"]
    assert rm["launches"] == 2
    assert rm["dram_bytes_per_launch"] == pytest.approx((150 + 450) / 2)
    assert rm["share"] == pytest.approx(4000 / 8000)
    cm = s["kernels"]["k_calib_mad32"]
    # 2 CTAs x 256 threads x 8 operations / 32 = 128 warp-wide operations
    assert cm["per_warp_op"]["sm__pipe_fmaheavy_cycles_active.sum"] == \
        pytest.approx(4096 / 128)
    assert s["sources_sha16"] == bench.sources_sha16(bench.CALIB_SOURCES)


def test_committed_profiles_parse():
    cal = bench.profile_json(bench.CALIB_PROFILE)
    assert set(cal["c_mul_fmaheavy_cycles_per_warp_modmul"]) == \
        {"goldilocks", "p2013265921", "p998244353"}
    tr = bench.profile_json(bench.TRAFFIC_PROFILE)
    assert tr["kernels"]["k_row_mul2<goldilocks>"]["dram_bytes_per_launch"] > 0
    pk = bench.modmul_peaks()
    assert all(pk[p]["peak_modmul_per_s"] > 0 for p in (0, 1, 2))
