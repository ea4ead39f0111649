"""Host-side helpers of bench.py (no GPU): the kernel models behind the roofline fields and the
scaling of the bounded oracle sample."""
import math

import bench


def test_sap_flop_model_counts_table1_flops_per_update():
    peaks = {"hbm_gbs": 6789.0, "sm_max_mhz": 2070.0, "source": "measured", "fp32_tflops": 70.0,
             "fp32_source": "measured"}
    V = 48 * 48 * 48 * 96
    bound, units, unit, peak, src = bench.kernel_model("ssor", V, 4, {"nsweep": 2, "nsap": 2}, peaks)
    assert (bound, unit, peak) == ("alu", "TFLOP/s", 70.0)
    # a 2-cycle application: 4 launches of V/2 sites x 4 right-hand sides x 2 passes x 2 sweeps,
    # the first two also the residual's in-block operator; x 1896 flop, averaged per launch
    assert math.isclose(units, V / 2 * 4 * (4 + 2 / 4) * 1896 / 1e12, rel_tol=1e-12)
    # one cycle: no launch keeps a residual
    _, units, _, _, _ = bench.kernel_model("ssor", V, 4, {"nsweep": 2, "nsap": 1}, peaks)
    assert math.isclose(units, V / 2 * 4 * 4 * 1896 / 1e12, rel_tol=1e-12)
    bound, units, unit, peak, src = bench.kernel_model("dslash32", V, 1, {"nsweep": 2}, peaks)
    assert (bound, unit, peak) == ("hbm", "GB/s", 6789.0)
    assert math.isclose(units, V * 768 / 1e9, rel_tol=1e-12)
    # k right-hand sides: both spinors each, links and clover once
    _, units, _, _, _ = bench.kernel_model("dslash32", V, 12, {"nsweep": 2}, peaks)
    assert math.isclose(units, V * (12 * 192 + 576) / 1e9, rel_tol=1e-12)
    assert bench.kernel_model("blas", V, 1, {"nsweep": 2}, peaks) is None


def test_derived_fp32_peak_and_oracle_scale():
    p = bench.read_peaks()
    assert math.isclose(p["fp32_tflops"], 152 * 128 * 2 * p["sm_max_mhz"] * 1e6 / 1e12, rel_tol=1e-12)
    # 48^3 x 96 has 1296 times the sites of 8^3 x 16; 12 sources
    assert bench.oracle_scale() == 1296 * 12


def test_sap_shared_memory_model():
    V = 24 * 24 * 24 * 48
    # FP16 storage, 2 sweeps, 2 cycles: per (site, right-hand side) 4 x 11 + 1 (x += y) + 9 in half of
    # the launches (the kept residual) + 1 (source) + the y copy-out in 3 of 4 launches, 48 B each
    assert math.isclose(bench.sap_smem_bytes_per_launch(V, 4, 2, 2), V / 2 * 4 * (44 + 1 + 4.5 + 1 + 0.75) * 48,
                        rel_tol=1e-12)
    # one cycle: no residual, y copied out by the first of the two launches
    assert math.isclose(bench.sap_smem_bytes_per_launch(V, 4, 2, 1), V / 2 * 4 * (44 + 1 + 1 + 0.5) * 48,
                        rel_tol=1e-12)
    # FP32 storage keeps f in global memory: 4 x 10 + 1 + 4.5 spinors of 96 B
    assert math.isclose(bench.sap_smem_bytes_per_launch(V, 4, 2, 2, half=False), V / 2 * 4 * 45.5 * 96,
                        rel_tol=1e-12)


def test_sap_traffic_needs_the_captured_application():
    t = {"nsap": 1, "nsweep": 2, "per_launch": [900.0, 1100.0]}
    assert math.isclose(bench.sap_traffic_per_site_rhs(t, 1, 2), 1000.0, rel_tol=1e-12)
    # other launch types (kept residuals, more sweeps): no figure
    assert bench.sap_traffic_per_site_rhs(t, 2, 2) is None
    assert bench.sap_traffic_per_site_rhs(t, 1, 3) is None
    assert bench.sap_traffic_per_site_rhs({"nsap": 1, "nsweep": 2, "per_launch": None}, 1, 2) is None


def test_headline_params_keep_every_tuned_knob():
    """The timed chosen set-up is the tuner's result as a whole, outer operator form included;
    the plain set-up keeps the FP64 outer operator."""
    import paper_1210_7398_gb300 as q
    tuned = q.make_params(0.122, 1.6, (4, 4, 4, 4), (2, 2, 2, 2), omega=1.4, nsweep=2, nsap=1,
                          sap_storage=q.QCD_F16, sap_ctas=-2, outer_precision=q.QCD_F32X2)
    plain, chosen = bench.headline_params(q, tuned)
    for f in ("omega", "nsweep", "nsap", "sap_storage", "sap_ctas", "outer_precision"):
        assert getattr(chosen, f) == getattr(tuned, f), f
    assert tuple(chosen.block) == (4, 4, 4, 4) and tuple(chosen.subblock) == (2, 2, 2, 2)
    assert plain.outer_precision == q.QCD_F64
