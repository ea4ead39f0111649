"""Several independent lattices solved concurrently (qcd_solve_multi): each instance gives the same
solution, bit for bit, as its own qcd_solve, and the FP64 residual under the oracle's D meets the
tolerance.  Uneven sizes and kappas, one instance with FP16 SAP storage and two right-hand sides."""
import numpy as np
import pytest

import oracle
import qcd_inputs as qi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1210_7398_gb300 as q  # noqa: E402

CSW = 1.6
INSTANCES = [  # dims, kappa, block, sub-block, storage, nrhs
    ((4, 4, 4, 4), 0.118, (2, 2, 2, 2), (1, 1, 1, 1), q.QCD_F32, 1),
    ((4, 4, 4, 8), 0.120, (2, 2, 2, 2), (2, 2, 2, 2), q.QCD_F16, 2),
    ((8, 8, 8, 8), 0.122, (4, 4, 4, 4), (2, 2, 2, 2), q.QCD_F32, 1),
]


def make(dims, kappa, seed):
    stream = torch.cuda.Stream()
    s = q.Solver(dims, stream=stream.cuda_stream)
    U = qi.gauge_field(dims, 0.3, seed=seed)
    s.load_gauge(torch.from_numpy(U).cuda())
    s.build_clover(kappa, CSW)
    torch.cuda.synchronize()
    return s, stream, U


def test_multi_matches_single_solves():
    solvers, streams, Us, bs, prms = [], [], [], [], []
    for i, (dims, kappa, blk, sub, sto, nr) in enumerate(INSTANCES):
        s, st, U = make(dims, kappa, 1002 + i)
        solvers.append(s)
        streams.append(st)
        Us.append(U)
        bs.append(torch.from_numpy(qi.gaussian_spinor(dims, seed=2002 + i, nrhs=nr)).cuda())
        prms.append(q.make_params(kappa, CSW, blk, sub, nsweep=2, nsap=2, tol=1e-10, sap_storage=sto))
    ref = []
    for s, b, p, inst in zip(solvers, bs, prms, INSTANCES):
        x = torch.zeros_like(b)
        st = s.solve(x, b, p, nrhs=inst[5])
        ref.append((x.clone(), st))
    torch.cuda.synchronize()
    xs = [torch.zeros_like(b) for b in bs]
    rc, stats = q.qcd_solve_multi([s.ctx for s in solvers], xs, bs, prms, [inst[5] for inst in INSTANCES])
    torch.cuda.synchronize()
    assert rc == q.QCD_OK
    for (xr, sr), x, st in zip(ref, xs, stats):
        assert torch.equal(x, xr)
        assert st["outer_iters"] == sr["outer_iters"] and st["inner_iters"] == sr["inner_iters"]
        assert st["true_rel_res"] <= 1e-10
    # the FP64 residual of each instance under the oracle's D
    for (dims, kappa, *_), U, b, x in zip(INSTANCES, Us, bs, xs):
        F = oracle.clover(dims, U, CSW, kappa)[1]
        for k in range(b.shape[0]):
            bk = b.cpu().numpy()[k]
            r = bk - oracle.apply_D(dims, U, F, kappa, x.cpu().numpy()[k])
            assert np.linalg.norm(r) / np.linalg.norm(bk) <= 1e-10
    for s in solvers:
        s.close()


def test_multi_rejects_shared_streams():
    dims = (4, 4, 4, 4)
    stream = torch.cuda.Stream()
    a = q.Solver(dims, stream=stream.cuda_stream)
    b = q.Solver(dims, stream=stream.cuda_stream)
    for s in (a, b):
        s.load_gauge(torch.from_numpy(qi.gauge_field(dims, 0.3, seed=1002)).cuda())
        s.build_clover(0.12, CSW)
    src = torch.from_numpy(qi.gaussian_spinor(dims, seed=2002)).cuda()
    p = q.make_params(0.12, CSW, (2, 2, 2, 2), (1, 1, 1, 1), nsweep=2, nsap=2, tol=1e-10)
    xs = [torch.zeros_like(src), torch.zeros_like(src)]
    rc, _ = q.qcd_solve_multi([a.ctx, b.ctx], xs, [src, src], [p, p], [1, 1], check=False)
    assert rc == q.QCD_ERR_ARG
    a.close()
    b.close()
