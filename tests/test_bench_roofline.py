"""bench.py's roofline arithmetic (no GPU): algorithmic bytes per zone and
stage launch, the ghost shell the stages write on periodic meshes, and the
binding roof with the other one beside it."""
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


def test_fp32_roofline_counts_the_pushed_ghost_shell(bench):
    pk = {"hbm_gbs": 1000.0}
    zones = bench.MESH ** 3
    v = {"precision": "fp32", "block": 32, "stage_ms_avg": 1.0, "launches_per_cycle": 3}
    r = bench.roofline_for(v, pk, "measured")
    words = 12.5 + 5 * 13888 / 32768
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["algorithmic_bytes_per_zone_launch"] == pytest.approx(4 * words)
    assert r["achieved"] == pytest.approx(4 * words * zones / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 1000.0)
    # with a separate exchange launch the stage writes interiors only
    v["launches_per_cycle"] = 5
    assert bench.roofline_for(v, pk, "measured")["algorithmic_bytes_per_zone_launch"] == pytest.approx(50.0)


def test_fp64_roofline_is_the_fp64_pipe_with_hbm_beside_it(bench):
    pk = {"hbm_gbs": 1000.0}
    zones = bench.MESH ** 3
    v = {"precision": "fp64", "block": 32, "stage_ms_avg": 10.0, "launches_per_cycle": 3}
    r = bench.roofline_for(v, pk, "measured")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(bench.FLOPS_PER_ZONE_CYCLE / 2 * zones / 1e-2 / 1e12)
    assert r["peak"] == pytest.approx(152 * 2 * 2 * 2070e6 / 1e12)
    words = 12.5 + 5 * 13888 / 32768
    assert r["hbm"]["algorithmic_bytes_per_zone_launch"] == pytest.approx(8 * words)
    assert r["hbm"]["frac"] == pytest.approx(8 * words * zones / 1e-2 / 1e9 / 1000.0)
