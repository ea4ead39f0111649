"""The allocation-free SAP entry point against the allocating one.

qcd_sap_precondition_noalloc exists for callers that must not allocate device
memory when they call the library (a framework allocator already holds the
GPU's free memory, or a serving loop with a fixed memory budget); it keeps
its scratch in a fixed device array.  This file runs last (pytest collects
files in name order) so that a failure here leaves every other test already
run.  It also passes alone in a fresh process.
"""
import numpy as np
import pytest

import qcd_inputs as qi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1210_7398_gb300 as q  # noqa: E402

CSW = 1.6
SAP_TOL = 1e-5  # the SAP parity tolerance used by the other GPU tests


def rel_norm(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def solver(dims, kappa, seed):
    s = q.Solver(dims)
    s.load_gauge(torch.from_numpy(qi.gauge_field(dims, 0.3, seed=seed)).cuda())
    s.build_clover(kappa, CSW)
    return s


@pytest.mark.parametrize("dims,block,sub", [((12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6)),
                                            ((8, 8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2))])
def test_noalloc_matches_allocating_entry_point_twice(dims, block, sub):
    kappa = 0.12
    s = solver(dims, kappa, seed=1001)
    prm = q.make_params(kappa, CSW, block, sub, omega=1.0, nsweep=4, nsap=4)
    for seed in (3001, 3002):  # two calls in a row, different inputs
        v = torch.from_numpy(qi.gaussian_spinor(dims, seed=seed)[0].astype(np.complex64)).cuda()
        ref = torch.empty_like(v)
        s.sap_precondition(ref, v, prm)
        out = torch.full_like(v, float("nan"))
        q.qcd_sap_precondition_noalloc(s.ctx, out, v, prm)
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(out)).all()
        assert rel_norm(out, ref) <= SAP_TOL
    s.close()


@pytest.mark.parametrize("ctas", [0, 2, -2])
def test_noalloc_kernel_forms_and_no_device_allocation(ctas):
    """The kernel form follows params.sap_ctas as for the allocating entry point (0: the
    context's setting); a repeated call reuses what the fixed array holds and leaves the
    device's free memory unchanged."""
    dims, kappa = (12, 12, 12, 24), 0.12
    s = solver(dims, kappa, seed=1002)
    prm = q.make_params(kappa, CSW, (3, 3, 3, 6), (1, 1, 1, 2), omega=1.0, nsweep=2, nsap=2, sap_ctas=ctas)
    v = torch.from_numpy(qi.gaussian_spinor(dims, seed=3003)[0].astype(np.complex64)).cuda()
    ref = torch.empty_like(v)
    s.sap_precondition(ref, v, prm)
    out = torch.empty_like(v)
    q.qcd_sap_precondition_noalloc(s.ctx, out, v, prm)  # first call: builds the tables and records
    torch.cuda.synchronize()
    assert rel_norm(out, ref) <= SAP_TOL
    out2 = torch.empty_like(v)  # allocated before the measured call
    torch.cuda.synchronize()
    reserved0 = torch.cuda.memory_reserved()
    free0, _ = torch.cuda.mem_get_info()
    q.qcd_sap_precondition_noalloc(s.ctx, out2, v, prm)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0
    assert torch.equal(out2, out)
    bad = q.make_params(kappa, CSW, (3, 3, 3, 6), (1, 1, 1, 2), sap_ctas=17)
    with pytest.raises(q.QcdError) as e:
        q.qcd_sap_precondition_noalloc(s.ctx, out2, v, bad)
    assert e.value.code == q.QCD_ERR_ARG
    s.close()


def test_noalloc_rejects_lattices_above_its_limit():
    dims = (16, 16, 16, 16)  # 65,536 sites > 41,472
    s = solver(dims, 0.12, seed=7)
    prm = q.make_params(0.12, CSW, (8, 8, 8, 8), (4, 4, 4, 4))
    v = torch.zeros((qi.volume(dims), 4, 3), dtype=torch.complex64, device="cuda")
    with pytest.raises(q.QcdError) as e:
        q.qcd_sap_precondition_noalloc(s.ctx, torch.empty_like(v), v, prm)
    assert e.value.code == q.QCD_ERR_ARG
    assert "41472" in str(e.value)
    s.close()
