"""GPU parity of the right-hand-side tiled thread form of the SSOR block solve
(sap_ctas = -2): SAP against the FP64 oracle (Eq. 4, Algorithm 1, ll-SSOR of
Sec. 3), batched against single right-hand sides, and a full solve.

The tile form keeps the transport matrices as their first two rows (Table 1's
12-real form) and rebuilds the third, so FP32 results differ from the other
forms in rounding but not beyond the SAP tolerance of 1e-5.  Each right-hand
side's arithmetic is the same whatever the tile size, so a batched call equals
single calls bit for bit.
"""
import numpy as np
import pytest

import oracle
import qcd_inputs as qi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1210_7398_gb300 as q  # noqa: E402

CSW = 1.6
SAP_F16_TOL = 5e-3  # as for the other FP16 forms: 10 half-precision units in norm

TILE_CASES = [
    # dims, block, subblock, omega, nsweep, nsap, storages
    ((4, 4, 4, 4), (2, 2, 2, 2), (1, 1, 1, 1), 1.0, 4, 4, ("f32", "f16")),
    ((8, 4, 4, 8), (4, 2, 2, 4), (2, 1, 2, 2), 1.2, 2, 3, ("f32", "f16")),
    ((8, 8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2), 1.0, 3, 2, ("f32", "f16")),
    ((12, 12, 12, 24), (6, 6, 6, 6), (3, 3, 3, 3), 1.0, 4, 4, ("f32", "f16")),  # the paper's split
    ((12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6), 1.0, 4, 4, ("f16",)),  # does not fit: the cluster form stands in
    ((12, 12, 12, 24), (3, 3, 3, 6), (1, 1, 1, 2), 0.9, 2, 2, ("f32", "f16")),
    # block grids of 6 x 2 x 2 x 4 and 4 x 2 x 2 x 2: the cross hops find the neighbouring block
    # of the other colour in each direction, across the periodic wrap; one and two SAP cycles
    ((24, 4, 4, 8), (4, 2, 2, 2), (2, 1, 1, 1), 1.4, 2, 1, ("f32", "f16")),
    ((16, 8, 8, 12), (4, 4, 4, 6), (2, 2, 2, 3), 1.3, 2, 2, ("f16",)),
]


def rel_norm(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def make_solver(dims, kappa, seed):
    U = qi.gauge_field(dims, 0.3, seed=seed)
    s = q.Solver(dims)
    s.load_gauge(torch.from_numpy(U).cuda())
    s.build_clover(kappa, CSW)
    _, F = oracle.clover(dims, U, CSW, kappa)
    return s, U, F


def storage(name):
    return q.QCD_F32 if name == "f32" else q.QCD_F16


@pytest.mark.parametrize("case", TILE_CASES, ids=lambda c: "x".join(map(str, c[0])) + "_b" + "x".join(map(str, c[1])))
def test_tile_sap_vs_oracle(case):
    dims, b, sb, omega, nsweep, nsap, stores = case
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1001)
    v = qi.gaussian_spinor(dims, seed=2001)[0]
    ref = oracle.sap(dims, U, F, kappa, b, sb, omega, nsweep, nsap, v)
    vin = torch.from_numpy(v.astype(np.complex64)).cuda()
    for st in stores:
        prm = q.make_params(kappa, CSW, b, sb, omega=omega, nsweep=nsweep, nsap=nsap, sap_storage=storage(st),
                            sap_ctas=-2)
        out = torch.empty_like(vin)
        s.sap_precondition(out, vin, prm)
        torch.cuda.synchronize()
        err = rel_norm(out.cpu().numpy().astype(np.complex128), ref)
        if st == "f32":
            assert err <= 1e-5, err
        else:
            assert 1e-7 < err <= SAP_F16_TOL, err
    s.close()


def test_tile_falls_back_where_the_block_does_not_fit():
    """A 6^3 x 12 block's FP32 spinor (249 KB) exceeds a CTA's shared memory: sap_ctas = -2 then
    runs the automatic cluster form, bit for bit."""
    dims, kappa = (12, 12, 12, 24), 0.12
    s, _, _ = make_solver(dims, kappa, seed=1001)
    v = qi.gaussian_spinor(dims, seed=2001)[0]
    vin = torch.from_numpy(v.astype(np.complex64)).cuda()
    outs = []
    for ctas in (-2, 0):
        prm = q.make_params(kappa, CSW, (6, 6, 6, 12), (3, 3, 3, 6), nsweep=2, nsap=2, sap_ctas=ctas)
        out = torch.empty_like(vin)
        s.sap_precondition(out, vin, prm)
        outs.append(out)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])
    s.close()


@pytest.mark.parametrize("st", ["f32", "f16"])
def test_tile_batched_equals_single(st):
    """nrhs = 12 runs tiles of 8 right-hand sides (the second tile half empty), nrhs = 3 tiles
    of 2; every right-hand side equals its single call bit for bit."""
    dims, b, sb = (8, 8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2)
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1007)
    v = qi.gaussian_spinor(dims, seed=2007, nrhs=12)
    prm = q.make_params(kappa, CSW, b, sb, omega=1.1, nsweep=3, nsap=2, sap_storage=storage(st), sap_ctas=-2)
    vin = torch.from_numpy(v.astype(np.complex64)).cuda()
    singles = []
    for k in range(12):
        one = torch.empty_like(vin[k:k + 1])
        s.sap_precondition(one, vin[k:k + 1].contiguous(), prm)
        singles.append(one)
    for n in (12, 3, 5):
        out = torch.empty_like(vin[:n])
        s.sap_precondition(out, vin[:n].contiguous(), prm, nrhs=n)
        torch.cuda.synchronize()
        for k in range(n):
            assert torch.equal(singles[k][0], out[k]), (n, k)
    ref = oracle.sap(dims, U, F, kappa, b, sb, 1.1, 3, 2, v[7])
    tol = 1e-5 if st == "f32" else SAP_F16_TOL
    assert rel_norm(singles[7][0].cpu().numpy().astype(np.complex128), ref) <= tol
    s.close()


@pytest.mark.parametrize("st", ["f32", "f16"])
def test_tile_solve_true_residual_under_oracle(st):
    dims, kappa = (8, 8, 8, 16), 0.12
    s, U, F = make_solver(dims, kappa, seed=1001)
    b = qi.gaussian_spinor(dims, seed=2001, nrhs=3)
    prm = q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), nsweep=2, nsap=2, tol=1e-10,
                        sap_storage=storage(st), sap_ctas=-2)
    x = np.zeros_like(b)
    st_ = s.solve(x, b, prm, nrhs=3)
    for k in range(3):
        r = b[k] - oracle.apply_D(dims, U, F, kappa, x[k])
        assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1e-10, (k, st_)
    s.close()
