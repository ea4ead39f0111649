"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances: FP64 D <= 1e-13 relative (max abs error / max abs value), FP32 D
<= 2e-6 relative in norm, SAP output <= 1e-5 relative in norm, solutions at a
true relative residual <= 1e-10 under the oracle's D.
"""
import numpy as np
import pytest

import oracle
import qcd_inputs as qi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1210_7398_gb300 as q  # noqa: E402

CSW = 1.6


def rel_max(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def rel_norm(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def make_solver(dims, kappa, seed, bc_t=1, eps=0.3):
    U = qi.gauge_field(dims, eps, seed=seed)
    s = q.Solver(dims)
    if bc_t != 1:
        s.set_boundary(bc_t)
    s.load_gauge(torch.from_numpy(U).cuda())
    s.build_clover(kappa, CSW)
    _, F = oracle.clover(dims, U, CSW, kappa)
    return s, U, F


@pytest.mark.parametrize("dims,bc_t", [((4, 4, 4, 4), 1), ((6, 4, 4, 6), -1), ((8, 8, 8, 16), 1),
                                       ((2, 6, 4, 2), -1)])
def test_dslash_fp64_fp32_vs_oracle(dims, bc_t):
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1000, bc_t=bc_t)
    psi = qi.gaussian_spinor(dims, seed=2000, nrhs=2)
    ref = np.stack([oracle.apply_D(dims, U, F, kappa, psi[k], bc_t=bc_t) for k in range(2)])
    dev = torch.from_numpy(psi).cuda()
    out = torch.empty_like(dev)
    s.apply_D(out, dev, q.QCD_F64, nrhs=2)
    torch.cuda.synchronize()
    assert rel_max(out.cpu().numpy(), ref) <= 1e-13
    dev32 = dev.to(torch.complex64)
    out32 = torch.empty_like(dev32)
    s.apply_D(out32, dev32, q.QCD_F32, nrhs=2)
    torch.cuda.synchronize()
    assert rel_norm(out32.cpu().numpy().astype(np.complex128), ref) <= 2e-6
    # host buffers through the same entry point
    host_out = np.empty_like(psi)
    s.apply_D(host_out, psi, q.QCD_F64, nrhs=2)
    assert rel_max(host_out, ref) <= 1e-13
    s.close()



@pytest.mark.parametrize("dims,bc_t", [((4, 4, 4, 4), 1), ((6, 4, 4, 6), -1), ((8, 8, 8, 16), 1),
                                       ((2, 6, 4, 2), -1)])
def test_dslash_pair_fp32_vs_oracle(dims, bc_t):
    """QCD_F32X2: D of an FP32 input in pair-of-FP32 arithmetic, against the oracle's FP64 D of the
    same (exactly widened) input.  Hi + lo links and clover carry 2^-48 of each FP64 entry; every
    product keeps its FMA error and every leading sum its TwoSum error, so what is lost is the FP32
    rounding of the low parts (about 2^-24 of 2^-24 per term, over some 200 terms a site): the same
    1e-13 bound as the FP64 D.  Ragged volumes (96 and 576 sites), three right-hand sides, and the
    hi + lo copies following a change of the clover field."""
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1000, bc_t=bc_t)
    psi32 = qi.gaussian_spinor(dims, seed=2000, nrhs=3).astype(np.complex64)
    psi = psi32.astype(np.complex128)
    ref = np.stack([oracle.apply_D(dims, U, F, kappa, psi[k], bc_t=bc_t) for k in range(3)])
    dev = torch.from_numpy(psi32).cuda()
    out = torch.empty(dev.shape, dtype=torch.complex128, device="cuda")
    s.apply_D(out, dev, q.QCD_F32X2, nrhs=3)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for k in range(3):
        assert rel_max(got[k], ref[k]) <= 1e-13
        assert rel_norm(got[k], ref[k]) <= 1e-13
    # far closer than the FP32 D: the low parts carry the FP64 fields
    out32 = torch.empty_like(dev)
    s.apply_D(out32, dev, q.QCD_F32, nrhs=3)
    torch.cuda.synchronize()
    assert rel_norm(got[0], ref[0]) < 1e-5 * rel_norm(out32[0].cpu().numpy().astype(np.complex128), ref[0])
    # host buffers, and the copies made again after the fields change
    s.build_clover(0.11, CSW)
    _, F2 = oracle.clover(dims, U, CSW, 0.11)
    host_out = np.empty(psi.shape, dtype=np.complex128)
    s.apply_D(host_out, psi32, q.QCD_F32X2, nrhs=3)
    ref2 = oracle.apply_D(dims, U, F2, 0.11, psi[1], bc_t=bc_t)
    assert rel_max(host_out[1], ref2) <= 1e-13
    s.close()

# FP16 storage of links and clover (FP32 arithmetic and spinors): each stored
# value carries a relative rounding of at most 2^-11 = 4.9e-4; the hop sum and
# the clover product add a few of them, so 2e-3 relative in norm.
D_F16_TOL = 2e-3


@pytest.mark.parametrize("dims,bc_t", [((4, 4, 4, 4), 1), ((6, 4, 4, 6), -1), ((8, 8, 8, 16), 1)])
def test_dslash_odd_rhs_counts_and_fp16_storage(dims, bc_t):
    """Three right-hand sides take the two-per-thread kernel and a single tail;
    the FP16-storage operator stays within its rounding bound; the SU(3)
    12-real link form keeps FP32 accuracy."""
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1000, bc_t=bc_t)
    psi = qi.gaussian_spinor(dims, seed=2000, nrhs=3)
    ref = np.stack([oracle.apply_D(dims, U, F, kappa, psi[k], bc_t=bc_t) for k in range(3)])
    dev32 = torch.from_numpy(psi).cuda().to(torch.complex64)
    out32 = torch.empty_like(dev32)
    s.apply_D(out32, dev32, q.QCD_F32, nrhs=3)
    torch.cuda.synchronize()
    for k in range(3):
        assert rel_norm(out32[k].cpu().numpy().astype(np.complex128), ref[k]) <= 2e-6
    out16 = torch.empty_like(dev32)
    s.apply_D(out16, dev32, q.QCD_F16, nrhs=3)
    torch.cuda.synchronize()
    for k in range(3):
        assert rel_norm(out16[k].cpu().numpy().astype(np.complex128), ref[k]) <= D_F16_TOL
    # SU(3) 12-real links (two rows stored, the third rebuilt): FP32 accuracy
    out12 = torch.empty_like(dev32)
    s.apply_D(out12, dev32, q.QCD_F32_SU3, nrhs=3)
    torch.cuda.synchronize()
    for k in range(3):
        assert rel_norm(out12[k].cpu().numpy().astype(np.complex128), ref[k]) <= 2e-6
    # the FP16 copies follow a change of the fields
    s.build_clover(0.11, CSW)
    _, F2 = oracle.clover(dims, U, CSW, 0.11)
    s.apply_D(out16, dev32, q.QCD_F16, nrhs=3)
    torch.cuda.synchronize()
    ref2 = oracle.apply_D(dims, U, F2, 0.11, psi[0], bc_t=bc_t)
    assert rel_norm(out16[0].cpu().numpy().astype(np.complex128), ref2) <= D_F16_TOL
    s.close()


def test_dslash_free_field_plane_wave():
    """U = 1: D e^{ipn} u = [1 - kappa sum(2cos p - 2i gamma sin p)] e^{ipn} u (closed form)."""
    dims, kappa = (8, 4, 4, 8), 0.11
    s = q.Solver(dims)
    s.load_gauge(torch.from_numpy(qi.unit_gauge(dims)).cuda())
    s.build_clover(kappa, CSW)
    p = 2 * np.pi * np.array([1, 1, 0, 3]) / np.array(dims)
    x = np.array(np.unravel_index(np.arange(qi.volume(dims)), dims, order="F")).T
    rng = np.random.default_rng(3)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    ph = np.exp(1j * x @ p)
    psi = (ph[:, None, None] * u[None])[None]
    g = [oracle.gamma(m) for m in range(4)]
    Mp = np.eye(4) * (1 - kappa * np.sum(2 * np.cos(p))) + sum(kappa * 2j * np.sin(p[m]) * g[m] for m in range(4))
    expect = ph[:, None, None] * (Mp @ u)[None]
    out = np.empty_like(psi)
    s.apply_D(out, psi, q.QCD_F64)
    assert rel_max(out[0], expect) <= 1e-14
    s.close()


SAP_CASES = [
    # dims, block, subblock, omega, nsweep, nsap
    ((4, 4, 4, 4), (2, 2, 2, 2), (1, 1, 1, 1), 1.0, 4, 4),   # the 4^4 configuration
    ((8, 4, 4, 8), (4, 2, 2, 4), (2, 1, 2, 2), 1.2, 2, 3),
    ((8, 8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2), 1.0, 3, 2),
    ((12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6), 1.0, 4, 4),  # the 12^3 x 24 configuration
    ((12, 12, 12, 24), (6, 6, 6, 6), (3, 3, 3, 3), 1.0, 4, 4),   # the paper's 6^4 blocks, 3^4 sub-blocks (Sec. 3)
]


@pytest.mark.parametrize("case", SAP_CASES, ids=lambda c: "x".join(map(str, c[0])) + "_b" + "x".join(map(str, c[1])))
def test_sap_vs_oracle(case):
    dims, b, sb, omega, nsweep, nsap = case
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1001)
    v = qi.gaussian_spinor(dims, seed=2001)[0]
    ref = oracle.sap(dims, U, F, kappa, b, sb, omega, nsweep, nsap, v)
    prm = q.make_params(kappa, CSW, b, sb, omega=omega, nsweep=nsweep, nsap=nsap)
    vin = torch.from_numpy(v.astype(np.complex64)).cuda()
    out = torch.empty_like(vin)
    s.sap_precondition(out, vin, prm)
    torch.cuda.synchronize()
    assert rel_norm(out.cpu().numpy().astype(np.complex128), ref) <= 1e-5
    # the thread form of the block solve (one thread per site update), where the block fits a CTA
    q.qcd_set_sap_ctas(s.ctx, -1)
    out_t = torch.empty_like(vin)
    s.sap_precondition(out_t, vin, prm)
    torch.cuda.synchronize()
    assert rel_norm(out_t.cpu().numpy().astype(np.complex128), ref) <= 1e-5
    s.close()


def test_solve_4x4_matches_oracle_and_dense_lu():
    dims, kappa = (4, 4, 4, 4), 0.12
    s, U, F = make_solver(dims, kappa, seed=1000)
    b = qi.gaussian_spinor(dims, seed=2000)
    prm = q.make_params(kappa, CSW, (2, 2, 2, 2), (1, 1, 1, 1), omega=1.0, nsweep=4, nsap=4, tol=1e-10)
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    st = s.solve(x, torch.from_numpy(b).cuda(), prm)
    xg = x.cpu().numpy()[0]
    r = b[0] - oracle.apply_D(dims, U, F, kappa, xg)
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= 1e-10
    assert st["true_rel_res"] <= 1e-10
    xo, status, _ = oracle.solve(dims, U, F, kappa, (2, 2, 2, 2), (1, 1, 1, 1), 1.0, 4, 4, b[0], tol=1e-10)
    assert status == 0
    assert rel_norm(xg, xo) <= 1e-8
    s.close()


@pytest.mark.parametrize("dims,block,sub", [((12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6)),
                                            ((8, 8, 8, 16), (4, 4, 4, 4), (2, 2, 2, 2))])
def test_solve_true_residual_under_oracle(dims, block, sub):
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1001)
    b = qi.gaussian_spinor(dims, seed=2001)
    prm = q.make_params(kappa, CSW, block, sub, omega=1.0, nsweep=4, nsap=4, tol=1e-10)
    x = np.zeros_like(b)
    st = s.solve(x, b, prm)  # host buffers
    r = b[0] - oracle.apply_D(dims, U, F, kappa, x[0])
    rel = np.linalg.norm(r) / np.linalg.norm(b[0])
    assert rel <= 1e-10, (rel, st)
    assert st["outer_iters"] >= 1 and st["inner_iters"] >= 1
    s.close()


def test_solve_is_deterministic():
    dims, kappa = (8, 8, 8, 8), 0.12
    s, U, F = make_solver(dims, kappa, seed=1002)
    b = torch.from_numpy(qi.gaussian_spinor(dims, seed=2002)).cuda()
    prm = q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), tol=1e-10)
    x1 = torch.zeros_like(b)
    x2 = torch.zeros_like(b)
    s.solve(x1, b, prm)
    s.solve(x2, b, prm)
    assert torch.equal(x1, x2)
    s.close()


def test_errors_are_reported_not_fatal():
    dims = (4, 4, 4, 4)
    s = q.Solver(dims)
    psi = torch.zeros((1, 256, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(q.QcdError) as e:
        s.apply_D(torch.empty_like(psi), psi, q.QCD_F64)
    assert e.value.code == q.QCD_ERR_STATE
    s.load_gauge(torch.from_numpy(qi.gauge_field(dims, 0.3, seed=5)).cuda())
    s.build_clover(0.12, CSW)
    bad = q.make_params(0.12, CSW, (4, 2, 2, 2), (1, 1, 1, 1))  # one block along x
    with pytest.raises(q.QcdError) as e:
        s.solve(torch.zeros_like(psi), psi, bad)
    assert e.value.code == q.QCD_ERR_ARG
    # misaligned device pointer
    flat = torch.zeros(256 * 12 + 1, dtype=torch.complex64, device="cuda")
    with pytest.raises(q.QcdError) as e:
        s.apply_D(flat[1:], flat[:-1], q.QCD_F32)
    assert e.value.code == q.QCD_ERR_ARG
    # out-of-range settings and arguments are rejected with QCD_ERR_ARG
    with pytest.raises(q.QcdError) as e:
        q.qcd_set_sap_ctas(s.ctx, 17)
    assert e.value.code == q.QCD_ERR_ARG
    with pytest.raises(q.QcdError) as e:
        q.qcd_set_sap_form(s.ctx, 3)
    assert e.value.code == q.QCD_ERR_ARG
    with pytest.raises(q.QcdError) as e:
        s.apply_D(torch.empty_like(psi), psi, 7)  # no such precision
    assert e.value.code == q.QCD_ERR_ARG
    wrong_kappa = q.make_params(0.11, CSW, (2, 2, 2, 2), (1, 1, 1, 1))  # differs from the clover built
    with pytest.raises(q.QcdError) as e:
        s.solve(torch.zeros_like(psi), psi, wrong_kappa)
    assert e.value.code == q.QCD_ERR_ARG
    bad_omega = q.make_params(0.12, CSW, (2, 2, 2, 2), (1, 1, 1, 1), omega=2.0)
    with pytest.raises(q.QcdError) as e:
        s.solve(torch.zeros_like(psi), psi, bad_omega)
    assert e.value.code == q.QCD_ERR_ARG
    # the context is still usable
    out = torch.empty_like(psi)
    s.apply_D(out, psi, q.QCD_F64)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out) == 0
    s.close()


def test_sap_identical_for_every_cluster_width():
    """The SSOR kernel may split a block over 1..16 CTAs (a thread-block cluster);
    the arithmetic and its order do not change, so the output is bitwise equal."""
    dims, b, sb = (12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6)
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1003)
    v = qi.gaussian_spinor(dims, seed=2003)[0]
    prm = q.make_params(kappa, CSW, b, sb, omega=1.0, nsweep=2, nsap=2)
    vin = torch.from_numpy(v.astype(np.complex64)).cuda()
    outs = []
    for ctas in (0, 1, 2, 3, 4, 5, 6, 8, 12, 16):
        q.qcd_set_sap_ctas(s.ctx, ctas)
        out = torch.empty_like(vin)
        s.sap_precondition(out, vin, prm)
        torch.cuda.synchronize()
        outs.append(out)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    ref = oracle.sap(dims, U, F, kappa, b, sb, 1.0, 2, 2, v)
    assert rel_norm(outs[0].cpu().numpy().astype(np.complex128), ref) <= 1e-5
    # FP16 storage: one scale per CTA, so not bitwise across widths, but each within its bound;
    # widths that do not divide the level sizes leave the CTAs unequal shares
    prm16 = q.make_params(kappa, CSW, b, sb, omega=1.0, nsweep=2, nsap=2, sap_storage=q.QCD_F16)
    for ctas in (1, 3, 5, 12, 16):
        q.qcd_set_sap_ctas(s.ctx, ctas)
        out = torch.empty_like(vin)
        s.sap_precondition(out, vin, prm16)
        torch.cuda.synchronize()
        assert rel_norm(out.cpu().numpy().astype(np.complex128), ref) <= SAP_F16_TOL, ctas
    s.close()


# FP16 storage inside the SAP block solve (FP32 arithmetic): the block spinor is
# kept as half2 scaled by the slab's largest source component, links and clover
# rows as half2.  Unit roundoff 2^-11 = 4.9e-4 per stored value; a few sweeps
# accumulate a few units, so the tolerance is 10 units in norm.
SAP_F16_TOL = 5e-3


@pytest.mark.parametrize("case", [SAP_CASES[0], SAP_CASES[2], SAP_CASES[3]], ids=lambda c: "x".join(map(str, c[0])))
def test_sap_fp16_storage_vs_oracle(case):
    dims, b, sb, omega, nsweep, nsap = case
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1001)
    v = qi.gaussian_spinor(dims, seed=2001)[0]
    ref = oracle.sap(dims, U, F, kappa, b, sb, omega, nsweep, nsap, v)
    prm = q.make_params(kappa, CSW, b, sb, omega=omega, nsweep=nsweep, nsap=nsap, sap_storage=q.QCD_F16)
    vin = torch.from_numpy(v.astype(np.complex64)).cuda()
    out = torch.empty_like(vin)
    s.sap_precondition(out, vin, prm)
    torch.cuda.synchronize()
    err = rel_norm(out.cpu().numpy().astype(np.complex128), ref)
    assert err <= SAP_F16_TOL
    assert err > 1e-7  # really stored in half precision
    s.close()


@pytest.mark.parametrize("storage", [q.QCD_F32, q.QCD_F16], ids=["f32", "f16"])
@pytest.mark.parametrize("geo", [((8, 8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2)),
                                 ((12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6))], ids=["8^4", "12^3x24"])
def test_sap_batched_equals_single_per_rhs(geo, storage):
    """Three right-hand sides through one batched SAP call equal, bitwise, three single
    calls, for the automatic cluster width and for 1, 2 and 4 CTAs per block."""
    dims, b, sb = geo
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1007)
    v = qi.gaussian_spinor(dims, seed=2007, nrhs=3)
    prm = q.make_params(kappa, CSW, b, sb, omega=1.1, nsweep=3, nsap=2, sap_storage=storage)
    vin = torch.from_numpy(v.astype(np.complex64)).cuda()
    for ctas in (0, 1, 2, 4):
        q.qcd_set_sap_ctas(s.ctx, ctas)
        out = torch.empty_like(vin)
        s.sap_precondition(out, vin, prm, nrhs=3)
        for k in range(3):
            one = torch.empty_like(vin[k:k + 1])
            s.sap_precondition(one, vin[k:k + 1].contiguous(), prm)
            torch.cuda.synchronize()
            assert torch.equal(one[0], out[k]), (ctas, k)
    ref = oracle.sap(dims, U, F, kappa, b, sb, 1.1, 3, 2, v[2])
    tol = 1e-5 if storage == q.QCD_F32 else SAP_F16_TOL
    assert rel_norm(out[2].cpu().numpy().astype(np.complex128), ref) <= tol
    s.close()


FORM_CASES = [
    # dims, block, subblock, storage, cluster width (0: automatic), right-hand sides
    ((8, 8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2), q.QCD_F32, 0, 1),
    ((8, 8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2), q.QCD_F16, 2, 3),
    ((12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6), q.QCD_F32, 0, 1),
    ((12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6), q.QCD_F16, 5, 1),
    ((12, 12, 12, 24), (3, 3, 3, 6), (1, 1, 1, 2), q.QCD_F16, 0, 12),
    ((12, 12, 12, 24), (3, 3, 3, 6), (1, 1, 1, 2), q.QCD_F32, 1, 4),
]


@pytest.mark.parametrize("case", FORM_CASES, ids=lambda c: "%s-%s-c%d-n%d" % (
    "x".join(map(str, c[1])), "f16" if c[3] == q.QCD_F16 else "f32", c[4], c[5]))
def test_sap_lane_forms_identical(case):
    """The 32-lane and the 8-lane site updates of the SSOR kernel perform the same
    rounding steps in the same order: their SAP outputs are equal bit for bit (and the
    automatic choice, per launch, equals both)."""
    dims, b, sb, storage, ctas, nrhs = case
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1008)
    v = qi.gaussian_spinor(dims, seed=2008, nrhs=nrhs)
    prm = q.make_params(kappa, CSW, b, sb, omega=1.1, nsweep=2, nsap=2, sap_storage=storage)
    q.qcd_set_sap_ctas(s.ctx, ctas)
    vin = torch.from_numpy(v.astype(np.complex64)).cuda()
    outs = []
    for form in (1, 2, 0):
        q.qcd_set_sap_form(s.ctx, form)
        out = torch.empty_like(vin)
        s.sap_precondition(out, vin, prm, nrhs=nrhs)
        torch.cuda.synchronize()
        outs.append(out)
    assert torch.equal(outs[0], outs[1])
    assert torch.equal(outs[0], outs[2])
    ref = oracle.sap(dims, U, F, kappa, b, sb, 1.1, 2, 2, v[0])
    tol = 1e-5 if storage == q.QCD_F32 else SAP_F16_TOL
    assert rel_norm(outs[1][0].cpu().numpy().astype(np.complex128), ref) <= tol
    s.close()


EO_CASES = [
    # dims, block, MR steps, N_SAP
    ((4, 4, 4, 4), (2, 2, 2, 2), 3, 2),
    ((8, 8, 8, 8), (4, 4, 4, 4), 5, 2),
    ((12, 12, 12, 24), (6, 6, 6, 12), 7, 2),
    ((12, 12, 12, 24), (3, 3, 3, 6), 4, 3),  # blocks with unequal even and odd site counts
]


@pytest.mark.parametrize("case", EO_CASES, ids=lambda c: "x".join(map(str, c[0])) + "-" + "x".join(map(str, c[1])))
def test_sap_even_odd_block_solver_vs_oracle(case):
    """The even-odd minimal-residual block inverse (block_solver = 1) against the oracle's,
    and two right-hand sides in one call equal to single calls bit for bit."""
    dims, b, nmr, nsap = case
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1009)
    v = qi.gaussian_spinor(dims, seed=2009, nrhs=2)
    ref = oracle.sap(dims, U, F, kappa, b, (1, 1, 1, 1), 1.0, nmr, nsap, v[0], block_solver=1)
    prm = q.make_params(kappa, CSW, b, (1, 1, 1, 1), nsweep=nmr, nsap=nsap, block_solver=1)
    vin = torch.from_numpy(v.astype(np.complex64)).cuda()
    out = torch.empty_like(vin)
    s.sap_precondition(out, vin, prm, nrhs=2)
    one = torch.empty_like(vin[:1])
    s.sap_precondition(one, vin[1:].contiguous(), prm)
    torch.cuda.synchronize()
    assert rel_norm(out[0].cpu().numpy().astype(np.complex128), ref) <= 1e-5
    assert torch.equal(one[0], out[1])
    # it is a different block inverse from the SSOR one
    ssor = oracle.sap(dims, U, F, kappa, b, (1, 1, 1, 1), 1.0, nmr, nsap, v[0])
    assert rel_norm(ssor, ref) > 1e-3
    s.close()


def test_solve_with_even_odd_block_solver():
    dims, block = (12, 12, 12, 24), (6, 6, 6, 12)
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1001)
    b = qi.gaussian_spinor(dims, seed=2001)
    prm = q.make_params(kappa, CSW, block, (3, 3, 3, 6), nsweep=7, nsap=4, tol=1e-10, block_solver=1)
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    st = s.solve(x, torch.from_numpy(b).cuda(), prm)
    r = b[0] - oracle.apply_D(dims, U, F, kappa, x.cpu().numpy()[0])
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= 1e-10, st
    for bad in (q.make_params(kappa, CSW, block, (3, 3, 3, 6), block_solver=2),
                q.make_params(kappa, CSW, block, (3, 3, 3, 6), block_solver=1, sap_storage=q.QCD_F16)):
        with pytest.raises(q.QcdError) as e:
            s.solve(x, torch.from_numpy(b).cuda(), bad)
        assert e.value.code == q.QCD_ERR_ARG
    s.close()


def test_solve_with_fp16_sap_reaches_fp64_tolerance():
    dims, block, sub = (12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6)
    kappa = 0.12
    s, U, F = make_solver(dims, kappa, seed=1001)
    b = qi.gaussian_spinor(dims, seed=2001)
    prm = q.make_params(kappa, CSW, block, sub, tol=1e-10, sap_storage=q.QCD_F16)
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    st = s.solve(x, torch.from_numpy(b).cuda(), prm)
    r = b[0] - oracle.apply_D(dims, U, F, kappa, x.cpu().numpy()[0])
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= 1e-10, st
    s.close()


def test_batched_point_sources_equal_single_solves():
    """12 spin-colour point sources solved together: every solution reaches 1e-10 under
    the oracle's D, and equals (bitwise) the solve of that source alone."""
    dims, kappa = (8, 8, 8, 8), 0.12
    s, U, F = make_solver(dims, kappa, seed=1004)
    b = qi.point_sources(dims)
    prm = q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), tol=1e-10)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st = s.solve(x, bd, prm, nrhs=12)
    xs = x.cpu().numpy()
    for k in range(12):
        r = b[k] - oracle.apply_D(dims, U, F, kappa, xs[k])
        assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1e-10, (k, st)
    for k in (0, 7):
        x1 = torch.zeros_like(bd[k:k + 1])
        s.solve(x1, bd[k:k + 1].contiguous(), prm, nrhs=1)
        assert torch.equal(x1[0], x[k])
    s.close()


def test_non_finite_rhs_is_reported_and_isolated():
    """A right-hand side holding a NaN (a fault made on the host) never enters the iteration:
    the call reports QCD_ERR_NOCONV, the other right-hand sides of the batch still reach 1e-10
    under the oracle's D, and the context stays usable."""
    dims, kappa = (8, 8, 8, 8), 0.12
    s, U, F = make_solver(dims, kappa, seed=1010)
    b = qi.gaussian_spinor(dims, seed=2010, nrhs=3)
    b[1, 5, 2, 1] = np.nan
    prm = q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), tol=1e-10)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st = s.solve(x, bd, prm, nrhs=3, check=False)
    assert st["status"] == q.QCD_ERR_NOCONV, st
    xs = x.cpu().numpy()
    for k in (0, 2):
        assert np.all(np.isfinite(xs[k]))
        r = b[k] - oracle.apply_D(dims, U, F, kappa, xs[k])
        assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1e-10
    x1 = torch.zeros_like(bd[:1])
    st1 = s.solve(x1, bd[2:].contiguous(), prm)
    assert st1["status"] == q.QCD_OK
    assert torch.equal(x1[0], x[2])  # batched = single, also next to a failed right-hand side
    s.close()


@pytest.mark.parametrize("ctas,storage", [(0, "f32"), (-2, "f16")])
def test_graph_replay_equals_direct_launches(ctas, storage):
    """The inner solve run as one CUDA graph whose while node the device ends (non-default
    stream) gives the same solution, bitwise, as direct launches with the host deciding each
    iteration; the graph path launches one condition kernel per iteration on top."""
    dims, kappa = (8, 8, 8, 8), 0.12
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        s, U, F = make_solver(dims, kappa, seed=1005)
        b = torch.from_numpy(qi.gaussian_spinor(dims, seed=2005, nrhs=2)).cuda()
        prm = q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), tol=1e-10, sap_ctas=ctas,
                            sap_storage=q.QCD_F16 if storage == "f16" else q.QCD_F32)
        xg = torch.zeros_like(b)
        l0 = q.qcd_launch_count(s.ctx)
        stg = s.solve(xg, b, prm, nrhs=2)
        l1 = q.qcd_launch_count(s.ctx)
        q.qcd_set_graphs(s.ctx, False)
        xd = torch.zeros_like(b)
        std = s.solve(xd, b, prm, nrhs=2)
        l2 = q.qcd_launch_count(s.ctx)
    torch.cuda.synchronize()
    assert torch.equal(xg, xd)
    assert stg["inner_iters"] == std["inner_iters"] and stg["outer_iters"] == std["outer_iters"]
    # the device loop adds its condition kernel to every iteration: strictly more launches
    assert l1 - l0 > l2 - l1 > 0
    s.close()


def test_autotune_returns_a_converging_setup():
    dims, kappa = (8, 8, 8, 16), 0.12
    s, U, F = make_solver(dims, kappa, seed=1006)
    b = torch.from_numpy(qi.gaussian_spinor(dims, seed=2006)).cuda()
    base = q.make_params(kappa, CSW, (4, 4, 4, 4), (2, 2, 2, 2), tol=1e-10)
    best, ms = q.qcd_autotune(s.ctx, b, base, max_candidates=12)
    assert ms > 0
    assert oracle.check_geometry(dims, tuple(best.block), tuple(best.subblock))
    x = torch.zeros_like(b)
    s.solve(x, b, best)
    r = b.cpu().numpy()[0] - oracle.apply_D(dims, U, F, kappa, x.cpu().numpy()[0])
    assert np.linalg.norm(r) / np.linalg.norm(b.cpu().numpy()[0]) <= 1e-10
    s.close()
