"""bench.py's roofline arithmetic (no GPU): algorithmic bytes per zone and
stage launch (the streaming model: 100 B per zone-cycle in FP32, 200 B in
FP64), the ghost shell the stages write on periodic meshes reported as
overhead beside them, and the binding roof with the other one beside it."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    import bench as B
    return B


def test_ghost_shell_words_per_zone(bench):
    # (n+4)^3 - n^3 ghost cells of 5 words per n^3 zones
    assert bench.ghost_words_per_zone(32) == pytest.approx(5 * 13888 / 32768)
    assert bench.ghost_words_per_zone(16) == pytest.approx(5 * (20 ** 3 - 16 ** 3) / 16 ** 3)


def test_fp32_roofline_counts_algorithmic_bytes_only(bench):
    pk = {"hbm_gbs": 1000.0}
    zones = bench.MESH ** 3
    v = {"precision": "fp32", "block": 32, "stage_ms_avg": 1.0, "launches_per_cycle": 3}
    r = bench.roofline_for(v, pk, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    # 12.5 words of 4 bytes per zone and launch = 100 B per zone-cycle
    assert r["algorithmic_bytes_per_zone_launch"] == pytest.approx(50.0)
    assert r["achieved"] == pytest.approx(50.0 * zones / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 1000.0)
    # the pushed ghost shell is overhead, beside the algorithmic bytes
    assert r["ghost_bytes_per_zone_launch"] == pytest.approx(4 * 5 * 13888 / 32768)
    # the FP32 arithmetic roof beside it
    assert r["alu"]["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert r["alu"]["frac"] == pytest.approx(bench.FLOPS_PER_ZONE_CYCLE / 2 * zones / 1e-3 / 1e12 / r["alu"]["peak"])
    v["launches_per_cycle"] = 5
    r5 = bench.roofline_for(v, pk, "measured")
    assert r5["ghost_bytes_per_zone_launch"] == 0.0 and r5["frac"] == pytest.approx(r["frac"])


def test_fp64_roofline_is_the_fp64_pipe_with_hbm_beside_it(bench):
    pk = {"hbm_gbs": 1000.0}
    zones = bench.MESH ** 3
    v = {"precision": "fp64", "block": 32, "stage_ms_avg": 10.0, "launches_per_cycle": 3}
    r = bench.roofline_for(v, pk, "measured", fp64_measured=1.2)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(bench.FLOPS_PER_ZONE_CYCLE / 2 * zones / 1e-2 / 1e12)
    assert r["peak"] == pytest.approx(152 * 2 * 2 * 2070e6 / 1e12)
    assert r["peak_measured"] == 1.2
    assert r["frac_of_measured"] == pytest.approx(r["achieved"] / 1.2)
    assert r["hbm"]["algorithmic_bytes_per_zone_launch"] == pytest.approx(100.0)
    assert r["hbm"]["frac"] == pytest.approx(100.0 * zones / 1e-2 / 1e9 / 1000.0)
    assert "peak_measured" not in bench.roofline_for(v, pk, "measured")
