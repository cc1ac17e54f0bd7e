"""Host arithmetic of bench.py (no GPU): the roofline figures of its legs."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_raster_tile_flops_by_hand():
    # 32-node window: stage 1 is two 128 x 32 x 32 products (2 x 262,144 flops),
    # stage 2 three 128 x 128 x 32 products (3 x 1,048,576 flops): 3,670,016.
    assert bench.raster_tile_flops(32) == 3_670_016
    # 64-node window: 2 x 1,048,576 + 3 x 2,097,152 = 8,388,608
    assert bench.raster_tile_flops(64) == 8_388_608
    # the 5 mm raster on the paper's 0.07 m mesh (sigma = 0.04, radius 0.16 m)
    # spans 0.635 + 0.32 = 0.955 m <= 28.5 x 0.07 = 1.995 m: 32-node windows
    assert bench.raster_window(0.005, 0.07, 0.16) == 32
    assert bench.raster_window(0.015, 0.07, 0.16) == 64


def test_raster_line_roofline_arithmetic():
    pk = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1700.0}
    r = dict(workload="w", points=5120 * 5120, ms=0.125, tiles=1600, scattered_eval_same_points_ms=0.9, kw=32)
    d = bench.raster_line(r, pk, "measured")
    sec = 0.125e-3
    assert math.isclose(d["points_per_s"], 5120 * 5120 / sec)
    gbs = 12.0 * 5120 * 5120 / sec / 1e9
    assert math.isclose(d["roofline"]["achieved"], gbs) and math.isclose(d["roofline"]["frac"], gbs / 6000.0)
    assert d["roofline"]["traffic"] == bench.RASTER_DRAM_BYTES  # measured on this raster size
    tf = 3_670_016 * 1600 / sec / 1e12     # 46.98 TFLOP/s of the method's products
    assert math.isclose(d["tensor"]["achieved"], tf) and math.isclose(d["tensor"]["frac"], tf / 2000.0)
    assert math.isclose(d["tensor"]["issued_frac"], 3 * tf / 2000.0)
    assert math.isclose(d["speedup_over_scattered_eval"], 0.9 / 0.125)
    # a raster of another size has no measured traffic
    r2 = dict(r, points=1000 * 1000, tiles=64)
    assert bench.raster_line(r2, pk, "measured")["roofline"]["traffic"] is None
    assert bench.raster_line(None, pk, "measured") is None


def test_eval_alu_line():
    # 65 G queries/s, K = pi 0.36 / 0.04 = 28.27 neighbours, 16 instructions each:
    # 29.4 T instr/s against 152 x 128 x 2.07 GHz = 40.27 T instr/s
    d = bench.eval_alu_line(65e9, {"sm_max_mhz": 2070.0})
    assert math.isclose(d["peak"], 40.27392, rel_tol=1e-6)
    assert math.isclose(d["achieved"], 65e9 * 16 * 28.274333882308138 / 1e12, rel_tol=1e-9)
    assert 0.72 < d["frac"] < 0.74


def test_max_over_ranks_without_a_group_is_identity():
    assert bench.max_over_ranks(3.5, None) == 3.5


def test_batch_work_by_hand():
    # one patch: M = 64 centers on rows of nx = 8, n = Q = 100; K = 9 pi = 28.274
    # in-support centers; half-bandwidth b = min(5 x 9, 64) = 45:
    #   Gram 100 (28.274 x 29.274 + 2 x 28.274) = 88,426
    #   Cholesky 64 x 45^2 = 129,600; solves 6 x 2 x 64 x 45 = 34,560;
    #   residuals 4 x 64 x 91 = 23,296; evaluation 100 x 16 x 28.274 = 45,239
    f, b = bench.batch_work([(64, 8, 100, 100)])
    assert math.isclose(f, 88426 + 129600 + 34560 + 23296 + 45239, rel_tol=1e-4)
    assert b == 12 * 100 + 20 * 100 + 8 * 64
