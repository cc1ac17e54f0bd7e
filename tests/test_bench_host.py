"""Host arithmetic of bench.py (no GPU): the raster leg's roofline figures."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_raster_line_roofline_arithmetic():
    pk = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1700.0}
    r = dict(workload="w", points=5120 * 5120, ms=0.125, tiles=1600, scattered_eval_same_points_ms=0.9)
    d = bench.raster_line(r, pk, "measured")
    sec = 0.125e-3
    assert math.isclose(d["points_per_s"], 5120 * 5120 / sec)
    gbs = 12.0 * 5120 * 5120 / sec / 1e9
    assert math.isclose(d["roofline"]["achieved"], gbs) and math.isclose(d["roofline"]["frac"], gbs / 6000.0)
    assert d["roofline"]["traffic"] == bench.RASTER_DRAM_BYTES  # measured on this raster size
    tf = bench.RASTER_TILE_FLOPS * 1600 / sec / 1e12
    assert math.isclose(d["tensor"]["achieved"], tf) and math.isclose(d["tensor"]["frac"], tf / 2000.0)
    assert math.isclose(d["speedup_over_scattered_eval"], 0.9 / 0.125)
    # a raster of another size has no measured traffic
    r2 = dict(r, points=1000 * 1000, tiles=64)
    assert bench.raster_line(r2, pk, "measured")["roofline"]["traffic"] is None
    assert bench.raster_line(None, pk, "measured") is None


def test_max_over_ranks_without_a_group_is_identity():
    assert bench.max_over_ranks(3.5, None) == 3.5
