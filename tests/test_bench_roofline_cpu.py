"""Host logic of the benchmark's roofline entry: which kernel is dominant,
how its achieved rate follows from the algorithmic work and the live event
timings, and which peak it is divided by.  No GPU: kernel timings are given
as the (timed ms, timed launches, all launches) triples the library reports."""
import pytest

import bench

N, S, M = 128 * 128 * 8, 32, 5000
PEAKS = {"hbm_gbs": 6788.3}


def test_dominant_kernel_is_ranked_by_estimated_share_not_timed_ms():
    # spmm_gram: 10 ms over 100 timed launches of 1600 -> 160 ms estimated;
    # apply_fields: 50 ms over its only 50 launches -> 50 ms.
    kt = {"spmm_gram": (10.0, 100, 1600), "apply_fields": (50.0, 50, 50)}
    r = bench.roofline(kt, N, S, M, PEAKS)
    assert r["kernel"] == "spmm_gram"
    assert r["share_of_kernel_time"] == pytest.approx(160.0 / 210.0, abs=1e-3)
    assert r["launches"] == 1600 and r["timed_launches"] == 100


def test_alu_kernel_rate_and_fraction():
    kt = {"spmm_gram": (6.0, 100, 100)}   # 60 us per launch
    r = bench.roofline(kt, N, S, M, PEAKS)
    flop = N * (13 * 32 + 4 * 32 * 32)
    achieved = flop / 60e-6 / 1e12
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(achieved, abs=1e-3)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2.070 / 1000, abs=0.1)
    assert r["frac"] == pytest.approx(achieved / bench.FP32_PEAK_TFLOPS, abs=1e-4)
    assert r["avg_launch_us"] == pytest.approx(60.0)


def test_hbm_kernel_uses_the_measured_copy_peak():
    kt = {"apply_fields": (1.0, 1, 1)}   # 1 ms: read T and write q, float32
    r = bench.roofline(kt, N, S, M, PEAKS)
    gbs = 8 * N * M / 1e-3 / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(gbs, abs=1e-2)
    assert r["peak"] == pytest.approx(6788.3)
    assert r["frac"] == pytest.approx(gbs / 6788.3, abs=1e-4)
    assert "measured" in r["peak_source"]


def test_kernels_without_a_cost_model_or_timed_launch_are_skipped():
    # the small solves have no per-cell cost model; a kernel never timed has no rate
    kt = {"alpha_solve": (900.0, 10, 10), "p_update": (0.0, 0, 500), "update_gram": (3.0, 10, 10)}
    assert bench.roofline(kt, N, S, M, PEAKS)["kernel"] == "update_gram"
    assert bench.roofline({"alpha_solve": (1.0, 1, 1)}, N, S, M, PEAKS) is None


def test_cost_model_follows_the_preconditioner():
    # the two-step z-line form moves W = Q^T Z from the update kernel to the second step
    z2 = bench.algorithmic("update_gram", N, S, M, "zline2")[1]
    z1 = bench.algorithmic("update_gram", N, S, M, "zline")[1]
    assert z1 - z2 == N * 2 * S * S
    second = bench.algorithmic("zline_second", N, S, M, "zline2")[1]
    assert second == N * (13 * S + 2 * S + 5 * S + 2 * S * S)
    # the padded width: s = 20 is computed as S = 32
    assert bench.algorithmic("p_update", N, 20, M)[1] == N * 2 * 32 * 32


def test_clock_rows_summary():
    lines = [
        "0, 1965, 2070, 1012.34, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 1890, 2070, 1388.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 1920, 2070, 1290.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]\n",   # unparsable sample: skipped
        "garbage\n",
    ]
    out = bench.ClockSampler.summarize(lines)
    assert out == {"sm_mhz": 1920.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.ClockSampler.summarize(["x, y\n"]) is None
    hw = bench.ClockSampler.summarize(["0, 900, 2070, 700, 0x8, Active, Active, Not Active, Not Active\n"])
    assert hw["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_kernel_timing_separates_noop_launches():
    # the graph launched 32 iterations' worth of loop kernels for 23 real iterations
    kt = {"spmm_gram": (4.0, 2, 32), "apply_fields": (1.0, 1, 1)}
    out = bench.kernel_timing_report(kt, {"spmm_gram": 23})
    assert out["spmm_gram"]["launches_with_work"] == 23 and out["spmm_gram"]["noop_launches"] == 9
    assert out["spmm_gram"]["est_total_ms"] == pytest.approx(2.0 * 23)
    assert out["apply_fields"]["est_total_ms"] == pytest.approx(1.0)
    r = bench.roofline(kt, N, S, M, PEAKS, real_launches={"spmm_gram": 23})
    assert r["launches_with_work"] == 23 and r["share_of_kernel_time"] == pytest.approx(46.0 / 47.0, abs=1e-3)


def test_fused_entry_counts_both_field_writes():
    kt = {"combine_apply": (2.0, 2, 2)}   # 1 ms per launch
    e = bench.hbm_entry("combine_apply", kt, N, S, M, PEAKS)
    assert e["achieved"] == pytest.approx(8 * N * M / 1e-3 / 1e9, abs=0.1)
    assert bench.hbm_entry("combine_apply", {}, N, S, M, PEAKS) is None


def test_fno_flop_model_pieces():
    from paper_2510_23221_gb300 import fno
    # no Fourier layers: lifting and projection only
    sh = fno.FnoShape(nx=8, ny=4, nz=2, c_in=5, width=32, hidden=128, layers=0, mx=4, my=4, mz=2)
    n = 8 * 4 * 2
    assert bench.fno_flops(sh) == n * 32 * 5 * 2 + n * (32 * 128 * 2 + 128 * 2)
    # each layer adds the same amount, which grows with the retained modes
    one = bench.fno_flops(fno.FnoShape(nx=8, ny=4, nz=2, layers=1, mx=4, my=4, mz=2))
    two = bench.fno_flops(fno.FnoShape(nx=8, ny=4, nz=2, layers=2, mx=4, my=4, mz=2))
    more = bench.fno_flops(fno.FnoShape(nx=8, ny=4, nz=2, layers=1, mx=8, my=4, mz=2))
    assert two - one == one - bench.fno_flops(fno.FnoShape(nx=8, ny=4, nz=2, layers=0, mx=4, my=4, mz=2))
    assert more > one


def test_spread_fields():
    f = bench.spread(5000, 32, shift=37)
    assert len(f) == 32 and f.min() >= 0 and f.max() < 5000
    assert len(bench.spread(10, 32)) == 10


def test_loop_kernel_streaming_bandwidth():
    # 4,194,304 cells at s = 64 (S = 64): spmm_gram reads P and R and writes
    # Q (12 S bytes per cell) plus 16 B of coefficients
    n, s = 4_194_304, 64
    kt = {"spmm_gram": (4.0, 2, 2), "p_update": (1.0, 1, 1), "alpha_solve": (1.0, 1, 1)}
    out = bench.loop_hbm(kt, n, s, {"hbm_gbs": 7000.0})
    assert set(out) == {"spmm_gram", "p_update"}
    b = n * (12 * 64 + 16)
    assert out["spmm_gram"]["bytes"] == b
    assert abs(out["spmm_gram"]["GBps"] - b / 2e-3 / 1e9) < 0.1
    assert abs(out["p_update"]["frac"] - n * 12 * 64 / 1e-3 / 1e9 / 7000.0) < 1e-4
