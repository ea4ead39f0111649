"""Host-side helpers of bench.py (no GPU): the kernel models behind the roofline fields."""
import math

import bench


def test_issue_floor_of_the_ssor_kernel():
    # 66.6 M warp instructions on 64 SMs at 4 per cycle and 2070 MHz: 125.7 us per launch
    r = bench.issue_model("ssor", 0.2486, 2070.0)
    assert math.isclose(r["floor_ms"], 66.6e6 / (64 * 4 * 2070e6) * 1e3, rel_tol=1e-12)
    assert math.isclose(r["floor_ms"], 0.1257, rel_tol=1e-3)
    assert math.isclose(r["frac"], r["floor_ms"] / 0.2486, rel_tol=1e-12)
    assert bench.issue_model("dslash32", 0.1, 2070.0) is None
    assert bench.issue_model("ssor", 0.0, 2070.0) is None


def test_ssor_flop_model_counts_table1_flops_per_update():
    peaks = {"hbm_gbs": 6764.0, "sm_max_mhz": 2070.0, "source": "measured"}
    V = 12 * 12 * 12 * 24
    bound, units, unit, peak = bench.kernel_model("ssor", V, 1, {"nsweep": 4}, peaks)
    assert (bound, unit) == ("alu", "TFLOP/s")
    # one launch: V/2 sites x 2 passes x 4 sweeps x 1896 flop
    assert math.isclose(units, V / 2 * 2 * 4 * 1896 / 1e12, rel_tol=1e-12)
    assert math.isclose(peak, 152 * 128 * 2 * 2070e6 / 1e12, rel_tol=1e-12)
    bound, units, unit, peak = bench.kernel_model("dslash32", V, 1, {"nsweep": 4}, peaks)
    assert (bound, unit, peak) == ("hbm", "GB/s", 6764.0)
    assert math.isclose(units, V * 768 / 1e9, rel_tol=1e-12)
