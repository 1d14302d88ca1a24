"""Host arithmetic of bench.py's roofline entries (no GPU): the HBM view of a
spectrum pass from its algorithmic bytes, and the FP32-pipe view that the
double-float passes add, on the free 256^3 geometry of the headline."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


@pytest.fixture(scope="module")
def P():
    return bench.pass_geometry(synth.Grid(256, 256, 256, 0.3, 0.3, 0.3, synth.BC_FREE))


def test_geometry_free_256(P):
    assert (P["Px"], P["Py"], P["Pz"], P["Hx"]) == (512, 512, 512, 257)


def test_z_df64_views(P):
    ms = 1.137
    r = bench.kernel_roofline("z_df64", ms, P, {"hbm_gbs": 6770.1})
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(r["algorithmic_bytes"] / (ms * 1e-3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6770.1)
    a = r["alu_view"]
    # 257 x 512 columns, two length-512 transforms each (5 L log2 L flops)
    # and 2 flops per point for the real table; the FFT flops at 6.4 FP32
    # instructions each, the table's at 4
    cols = 257 * 512
    fft = cols * 2 * 5 * 512 * 9
    table = cols * 2 * 512
    assert a["fp32_instructions"] == pytest.approx(fft * 6.4 + table * 4)
    assert a["peak"] == pytest.approx(152 * 128 * 2.07e9 / 1e12)
    assert a["achieved"] == pytest.approx(a["fp32_instructions"] / (ms * 1e-3) / 1e12)
    assert 0.5 < a["frac"] < 1.0


def test_alu_view_only_for_df64_passes(P):
    assert "alu_view" in bench.kernel_roofline("x_inv_df64", 0.41, P, {"hbm_gbs": 6770.1})
    assert "alu_view" not in bench.kernel_roofline("z_fp32", 0.38, P, {"hbm_gbs": 6770.1})
    assert "alu_view" not in bench.kernel_roofline("update_p", 0.17, P, {"hbm_gbs": 6770.1})
    assert bench.kernel_roofline("z", 6.9, P, {"hbm_gbs": 6770.1})["bound"] == "alu"


def test_config_is_the_workload_only():
    """Both arms print config_dict() as `config` and report how they compute
    beside it, so the two lines name the same workload."""
    c = bench.config_dict()
    assert c["workload"] == bench.WORKLOAD and c["grid"] == [256, 256, 256]
    assert "precision" not in c and "pcg_iters_per_solve" not in c
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert src.count('"config": config_dict(), "precision": ') == 2
