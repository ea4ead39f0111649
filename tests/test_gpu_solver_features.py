"""GPU tests of solver features around the method: right-hand-side groups, the tuning cache,
the breakdown path of the outer BiCGStab (Sec. 2) under a breakdown made on the host, and the
FP32 peak measurement hook."""
import json
import os

import numpy as np
import pytest

import oracle
import qcd_inputs as qi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1210_7398_gb300 as q  # noqa: E402

CSW = 1.6


def make_solver(dims, kappa, seed):
    U = qi.gauge_field(dims, 0.3, seed=seed)
    s = q.Solver(dims)
    s.load_gauge(torch.from_numpy(U).cuda())
    s.build_clover(kappa, CSW)
    return s, U


def test_rhs_groups_give_the_batched_solutions_bit_for_bit():
    """Each right-hand side's iterates do not depend on which others share its batch, so solving
    five sources in groups of 1, 2 or all at once gives identical solutions."""
    dims, kappa = (8, 8, 8, 8), 0.12
    s, U = make_solver(dims, kappa, seed=1011)
    b = torch.from_numpy(qi.gaussian_spinor(dims, seed=2011, nrhs=5)).cuda()
    outs = []
    for g in (0, 5, 2, 1):
        prm = q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), nsweep=2, nsap=2, tol=1e-10,
                            sap_storage=q.QCD_F16, sap_ctas=-2, rhs_group=g)
        x = torch.zeros_like(b)
        st = s.solve(x, b, prm, nrhs=5)
        assert st["true_rel_res"] <= 1e-10
        outs.append(x)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    with pytest.raises(q.QcdError) as e:
        s.solve(torch.zeros_like(b), b, q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), rhs_group=-1), nrhs=5)
    assert e.value.code == q.QCD_ERR_ARG
    s.close()


def test_tuning_cache_round_trip(tmp_path):
    dims, kappa = (8, 8, 8, 8), 0.12
    s, _ = make_solver(dims, kappa, seed=1012)
    b = torch.from_numpy(qi.gaussian_spinor(dims, seed=2012, nrhs=2)).cuda()
    base = q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), tol=1e-10)
    path = str(tmp_path / "tune.jsonl")
    q.qcd_set_tune_cache(path)
    try:
        best1, ms1 = q.qcd_autotune(s.ctx, b, base, nrhs=2, max_candidates=6)
        lines = open(path).read().splitlines()
        assert len(lines) == 1
        rec = json.loads(lines[0])
        assert rec["block"] == list(best1.block) and rec["rhs_group"] == best1.rhs_group
        assert rec["omega"] == best1.omega and rec["nsap"] == best1.nsap
        best2, ms2 = q.qcd_autotune(s.ctx, b, base, nrhs=2, max_candidates=6)  # served from the file
        assert q.params_dict(best2) == q.params_dict(best1)
        assert abs(ms2 - ms1) <= 1e-6 * max(1.0, ms1)
        assert len(open(path).read().splitlines()) == 1
        # another key (nrhs) is tuned and appended
        q.qcd_autotune(s.ctx, b[:1].contiguous(), base, nrhs=1, max_candidates=4)
        assert len(open(path).read().splitlines()) == 2
    finally:
        q.qcd_set_tune_cache(None)
    s.close()


def test_breakdown_made_on_the_host_restarts_and_converges():
    """rho = 0 at the start of the first outer iteration: the solver takes the breakdown path
    (true residual, restart from it) and still reaches 1e-10 under the oracle's D."""
    dims, kappa = (4, 4, 4, 4), 0.12
    s, U = make_solver(dims, kappa, seed=1000)
    b = qi.gaussian_spinor(dims, seed=2000, nrhs=2)
    prm = q.make_params(kappa, CSW, (2, 2, 2, 2), (1, 1, 1, 1), nsweep=4, nsap=4, tol=1e-10)
    q.qcd_debug_inject_breakdown(s.ctx, 1)
    x = np.zeros_like(b)
    st = s.solve(x, b, prm, nrhs=2)
    assert st["status"] == q.QCD_OK and st["restarts"] >= 2  # one per right-hand side
    _, F = oracle.clover(dims, U, CSW, kappa)
    for k in range(2):
        r = b[k] - oracle.apply_D(dims, U, F, kappa, x[k])
        assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1e-10
    s.close()


def test_persistent_breakdown_ends_in_qcd_err_breakdown():
    """Breakdowns at every outer iteration: after 5 restarts the solve reports
    QCD_ERR_BREAKDOWN, x stays finite, and the context keeps working."""
    dims, kappa = (4, 4, 4, 4), 0.12
    s, U = make_solver(dims, kappa, seed=1000)
    b = qi.gaussian_spinor(dims, seed=2000)
    prm = q.make_params(kappa, CSW, (2, 2, 2, 2), (1, 1, 1, 1), nsweep=4, nsap=4, tol=1e-10)
    q.qcd_debug_inject_breakdown(s.ctx, 1000)
    x = np.zeros_like(b)
    st = s.solve(x, b, prm, check=False)
    assert st["rc"] == q.QCD_ERR_BREAKDOWN and st["status"] == q.QCD_ERR_BREAKDOWN
    assert st["restarts"] == 6
    assert np.all(np.isfinite(x))
    q.qcd_debug_inject_breakdown(s.ctx, 0)
    x[...] = 0
    st = s.solve(x, b, prm)
    assert st["true_rel_res"] <= 1e-10
    s.close()


def test_fp32_peak_hook():
    s = q.Solver((4, 4, 4, 4))
    t = q.qcd_bench_fp32_peak(s.ctx, 8)
    assert 10.0 < t < 200.0, t  # GB300: 152 SMs x 128 lanes x 2 flop x about 2 GHz
    s.close()


def test_plain_c_client_computes_through_the_abi(tmp_path):
    """tests/c/abi_compute.c (C99, warnings as errors): D and a full solve on the free field
    through the C ABI with host buffers, checked against the closed forms in C."""
    import shutil
    import subprocess
    from paper_1210_7398_gb300 import build as qbuild
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(qbuild.LIB)
    exe = str(tmp_path / "abi_compute")
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(root, "include"),
                           os.path.join(root, "tests", "c", "abi_compute.c"), "-L", libdir, "-lqcd", "-lm",
                           "-Wl,-rpath," + libdir, "-o", exe])
    res = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr
    assert res.stdout.strip() == "ok"


def test_stats_report_kernel_time_when_profiling():
    dims, kappa = (8, 8, 8, 8), 0.12
    s, _ = make_solver(dims, kappa, seed=1013)
    b = torch.from_numpy(qi.gaussian_spinor(dims, seed=2013)).cuda()
    prm = q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), tol=1e-10)
    st = s.solve(torch.zeros_like(b), b, prm)
    assert st["ms_dslash"] == 0 and st["ms_sap"] == 0
    q.qcd_set_profiling(s.ctx, True)
    st = s.solve(torch.zeros_like(b), b, prm)
    q.qcd_set_profiling(s.ctx, False)
    assert 0 < st["ms_dslash"] < st["ms_total"] and 0 < st["ms_sap"] < st["ms_total"]
    s.close()


def test_fp32_outer_operator_reaches_tolerance_through_restarts():
    """outer_precision = QCD_F32: v = D p^ and t = D s^ in FP32, FP64 only for the true residual,
    the dots and x.  The recursive residual drifts by the FP32 error of D, so the solve restarts
    from the true residual and still ends at 1e-10 under the oracle's D; the default FP64 outer
    needs no restart here."""
    dims, kappa = (8, 8, 8, 8), 0.12
    s, U = make_solver(dims, kappa, seed=1014)
    b = qi.gaussian_spinor(dims, seed=2014, nrhs=2)
    _, F = oracle.clover(dims, U, CSW, kappa)
    stats = {}
    for name, op in (("f64", q.QCD_F64), ("f32", q.QCD_F32)):
        prm = q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), nsweep=2, nsap=2, tol=1e-10,
                            outer_precision=op)
        x = np.zeros_like(b)
        st = s.solve(x, b, prm, nrhs=2)
        assert st["status"] == q.QCD_OK and st["true_rel_res"] <= 1e-10
        for k in range(2):
            r = b[k] - oracle.apply_D(dims, U, F, kappa, x[k])
            assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1e-10
        stats[name] = st
    assert stats["f64"]["restarts"] == 0
    assert stats["f32"]["outer_iters"] >= stats["f64"]["outer_iters"]
    with pytest.raises(q.QcdError) as e:
        s.solve(np.zeros_like(b), b, q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), outer_precision=2), nrhs=2)
    assert e.value.code == q.QCD_ERR_ARG
    s.close()



def test_pair_fp32_outer_operator_matches_fp64_outer():
    """outer_precision = QCD_F32X2: the outer v = D p^ and t = D s^ in pair-of-FP32 arithmetic on
    the inner solver's FP32 output.  Its error (about 1e-14 of D) is far below the tolerance, so the
    solve takes the FP64 outer's iterations, needs no restart, and ends at 1e-10 under the oracle's
    D, with a solution within the tolerance of the FP64-outer one."""
    dims, kappa = (8, 8, 8, 8), 0.12
    s, U = make_solver(dims, kappa, seed=1014)
    b = qi.gaussian_spinor(dims, seed=2014, nrhs=2)
    _, F = oracle.clover(dims, U, CSW, kappa)
    xs, stats = {}, {}
    for name, op in (("f64", q.QCD_F64), ("x2", q.QCD_F32X2)):
        prm = q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), nsweep=2, nsap=2, tol=1e-10,
                            outer_precision=op)
        x = np.zeros_like(b)
        st = s.solve(x, b, prm, nrhs=2)
        assert st["status"] == q.QCD_OK and st["true_rel_res"] <= 1e-10
        for k in range(2):
            r = b[k] - oracle.apply_D(dims, U, F, kappa, x[k])
            assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1e-10
        xs[name], stats[name] = x, st
    assert stats["x2"]["restarts"] == 0
    assert stats["x2"]["outer_iters"] == stats["f64"]["outer_iters"]
    assert abs(stats["x2"]["inner_iters"] - stats["f64"]["inner_iters"]) <= 2
    for k in range(2):
        assert np.linalg.norm(xs["x2"][k] - xs["f64"][k]) <= 1e-8 * np.linalg.norm(xs["f64"][k])
    assert q.params_dict(q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2),
                                       outer_precision=q.QCD_F32X2))["outer_precision"] == "f32x2"
    s.close()

def test_smem_peak_hook():
    s = q.Solver((4, 4, 4, 4))
    t = q.qcd_bench_smem_peak(s.ctx, 64)
    assert 5000.0 < t < 100000.0, t  # GB300: 152 SMs x 128 B per cycle x about 2 GHz is about 40 TB/s
    s.close()
