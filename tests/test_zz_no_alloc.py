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
