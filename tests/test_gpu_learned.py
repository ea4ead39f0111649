"""GPU learned correction against the FP64 oracle (a project addition, not in the paper).

BF16 tensor-core layers with FP32 accumulation: forward <= 2e-2 relative in norm
(BF16 unit roundoff 3.9e-3 times the square root of the ~9 x 8 x 4 terms summed,
times a safety factor), gradients <= 5e-2.
"""
import numpy as np
import pytest

import oracle
import qcd_inputs as qi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1210_7398_gb300 as q  # noqa: E402

CSW, KAPPA = 1.6, 0.12
CH = q.LEARNED_CHANS


def rel_norm(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def setup(dims, seed=1007):
    U = qi.gauge_field(dims, 0.3, seed=seed)
    s = q.Solver(dims)
    s.load_gauge(torch.from_numpy(U).cuda())
    s.build_clover(KAPPA, CSW)
    return s, U


def test_weight_count_matches_oracle():
    assert q.qcd_learned_weight_count() == oracle.learned_weight_count(CH)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8), (6, 4, 4, 6)])
def test_forward_vs_oracle(dims):
    s, U = setup(dims)
    W = q.learned_init_weights(11, scale_last=1.0)
    q.qcd_learned_set_weights(s.ctx, W)
    x = qi.gaussian_spinor(dims, seed=12)
    out = np.empty((qi.volume(dims), 4, 3), dtype=np.complex64)
    q.qcd_learned_apply(s.ctx, out, x[0].astype(np.complex64))
    ref = oracle.learned_forward(dims, U, CH, W.astype(np.complex128), x)[0]
    assert rel_norm(out.astype(np.complex128), ref) <= 2e-2
    s.close()


def test_hop_special_case():
    """Layer weights (1 -+ gamma_mu) on the transports reproduce the Wilson hop; with
    identity first and last layers the network is H itself."""
    dims = (8, 4, 4, 8)
    s, U = setup(dims)
    W = np.zeros(q.qcd_learned_weight_count(), dtype=np.complex64)
    n1 = 9 * 8 * 1 * 16
    n2 = 9 * 8 * 8 * 16
    W1 = W[:n1].reshape(9, 8, 1, 4, 4)
    W2 = W[n1:n1 + n2].reshape(9, 8, 8, 4, 4)
    W3 = W[n1 + n2:].reshape(9, 1, 8, 4, 4)
    W1[0, 0, 0] = np.eye(4)   # channel 0 copies the input
    for mu in range(4):
        g = oracle.gamma(mu)
        W2[1 + 2 * mu, 0, 0] = np.eye(4) - g
        W2[2 + 2 * mu, 0, 0] = np.eye(4) + g
    W3[0, 0, 0] = np.eye(4)
    q.qcd_learned_set_weights(s.ctx, W)
    x = qi.gaussian_spinor(dims, seed=13)[0]
    out = np.empty_like(x, dtype=np.complex64)
    q.qcd_learned_apply(s.ctx, out, x.astype(np.complex64))
    ref = oracle.hop(dims, U, x)
    assert rel_norm(out.astype(np.complex128), ref) <= 2e-2
    s.close()


def test_loss_and_gradient_vs_oracle():
    dims = (4, 4, 4, 8)
    s, U = setup(dims)
    W = q.learned_init_weights(14, scale_last=0.5)
    q.qcd_learned_set_weights(s.ctx, W)
    rho = qi.gaussian_spinor(dims, seed=15)
    eps = qi.gaussian_spinor(dims, seed=16)
    loss, grad = q.qcd_learned_loss_grad(s.ctx, rho[0].astype(np.complex64), eps[0].astype(np.complex64))
    rloss, rgrad = oracle.learned_loss_grad(dims, U, CH, W.astype(np.complex128), rho, eps)
    assert abs(loss - rloss) <= 2e-2 * rloss
    assert rel_norm(grad.astype(np.float64), rgrad) <= 5e-2
    # per layer too (the small first and last layers are not hidden by the big middle one)
    n1 = 2 * 9 * 8 * 16
    n3 = 2 * 9 * 8 * 16
    assert rel_norm(grad[:n1].astype(np.float64), rgrad[:n1]) <= 5e-2
    assert rel_norm(grad[-n3:].astype(np.float64), rgrad[-n3:]) <= 5e-2
    s.close()


def test_training_reduces_loss_and_solver_converges():
    dims = (8, 8, 8, 8)
    s, U = setup(dims)
    prm = q.make_params(KAPPA, CSW, (4, 4, 4, 4), (2, 2, 2, 2), nsweep=2, nsap=2, tol=1e-10)
    q.qcd_learned_set_weights(s.ctx, q.learned_init_weights(17))
    src = torch.from_numpy(qi.gaussian_spinor(dims, seed=18, nrhs=16).astype(np.complex64)).cuda()
    hist = q.qcd_learned_train(s.ctx, src, 16, prm, epochs=6, batch=4, lr=3e-3)
    assert np.all(np.isfinite(hist))
    assert hist[-1] < hist[0]
    b = torch.from_numpy(qi.gaussian_spinor(dims, seed=19)).cuda()
    x = torch.zeros_like(b)
    prm_l = q.make_params(KAPPA, CSW, (4, 4, 4, 4), (2, 2, 2, 2), nsweep=2, nsap=2, tol=1e-10)
    prm_l.learned = 1
    st = s.solve(x, b, prm_l)
    F = oracle.clover(dims, U, CSW, KAPPA)[1]
    r = b.cpu().numpy()[0] - oracle.apply_D(dims, U, F, KAPPA, x.cpu().numpy()[0])
    assert np.linalg.norm(r) / np.linalg.norm(b.cpu().numpy()[0]) <= 1e-10, st
    s.close()


def test_trained_correction_gain_and_fallback():
    """What the trained network gains over plain SAP on a 12^3 x 24 field with small SAP blocks
    (2^3 x 3, 2 sweeps, 2 cycles): fewer inner iterations at the same FP64 accuracy.  The
    verdict picks the faster method, and learned = 1 follows it (the fallback)."""
    dims = (12, 12, 12, 24)
    s, U = setup(dims, seed=1001)
    prm = q.make_params(KAPPA, CSW, (2, 2, 2, 3), (2, 2, 2, 3), nsweep=2, nsap=2, tol=1e-10)
    q.qcd_learned_set_weights(s.ctx, q.learned_init_weights(4000))
    src = qi.gaussian_spinor_torch(dims, 3000, 64, "cuda").to(torch.complex64).contiguous()
    hist = q.qcd_learned_train(s.ctx, src, 64, prm, epochs=8, batch=8, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0], hist
    b = torch.from_numpy(qi.gaussian_spinor(dims, seed=2001)).cuda()
    v = q.qcd_learned_evaluate(s.ctx, b, 1, prm)
    print("learned-correction verdict:", v)
    assert v["plain_relres"] <= 1e-10 and v["learned_relres"] <= 1e-10, v
    assert v["learned_inner"] < v["plain_inner"], v
    assert v["use_learned"] == (1 if v["learned_ms"] < v["plain_ms"] else 0)
    # learned = 1 uses the correction exactly when the verdict favours it
    prm_l = q.make_params(KAPPA, CSW, (2, 2, 2, 3), (2, 2, 2, 3), nsweep=2, nsap=2, tol=1e-10)
    prm_l.learned = 1
    q.qcd_set_profiling(s.ctx, True)
    q.qcd_kernel_stats(s.ctx, 6, reset=True)
    x = torch.zeros_like(b)
    st = s.solve(x, b, prm_l)
    n_learned, _ = q.qcd_kernel_stats(s.ctx, 6, reset=True)
    q.qcd_set_profiling(s.ctx, False)
    assert (n_learned > 0) == bool(v["use_learned"]), (n_learned, v)
    assert st["inner_iters"] == (v["learned_inner"] if v["use_learned"] else v["plain_inner"])
    F = oracle.clover(dims, U, CSW, KAPPA)[1]
    r = b.cpu().numpy()[0] - oracle.apply_D(dims, U, F, KAPPA, x.cpu().numpy()[0])
    assert np.linalg.norm(r) / np.linalg.norm(b.cpu().numpy()[0]) <= 1e-10, st
    s.close()


def test_weights_file_round_trip(tmp_path):
    """qcd_learned_save / qcd_learned_load: the weights come back bit for bit (and with them the
    correction's output); a file for another network is refused."""
    dims = (4, 4, 4, 4)
    s, U = setup(dims)
    with pytest.raises(q.QcdError) as e:
        q.qcd_learned_save(s.ctx, tmp_path / "none.bin")
    assert e.value.code == q.QCD_ERR_STATE
    W = q.learned_init_weights(21, scale_last=1.0)
    q.qcd_learned_set_weights(s.ctx, W)
    path = tmp_path / "w.bin"
    q.qcd_learned_save(s.ctx, path)
    head = open(path, "rb").readline()
    assert b'"count": %d' % q.qcd_learned_weight_count() in head
    s2, _ = setup(dims)
    q.qcd_learned_load(s2.ctx, path)
    assert np.array_equal(q.qcd_learned_get_weights(s2.ctx), q.qcd_learned_get_weights(s.ctx))
    x = qi.gaussian_spinor(dims, seed=22)[0].astype(np.complex64)
    o1, o2 = np.empty_like(x), np.empty_like(x)
    q.qcd_learned_apply(s.ctx, o1, x)
    q.qcd_learned_apply(s2.ctx, o2, x)
    assert np.array_equal(o1, o2)
    bad = tmp_path / "bad.bin"
    bad.write_bytes(open(path, "rb").read()[:-8])  # truncated
    with pytest.raises(q.QcdError) as e:
        q.qcd_learned_load(s2.ctx, bad)
    assert e.value.code == q.QCD_ERR_ARG
    s.close()
    s2.close()


def test_tensor_core_layer_wait_runs_out_cleanly():
    """The tcgen05 8 -> 8 layer with its MMA commits withheld (a test hook; no device fault):
    its bounded mbarrier waits run out, it frees its tensor memory and returns, the call reports
    QCD_ERR_TIMEOUT, and the same context then computes the correction exactly as before."""
    dims = (8, 8, 8, 8)
    s, _ = setup(dims)
    q.qcd_learned_set_weights(s.ctx, q.learned_init_weights(3))
    v = torch.from_numpy(qi.gaussian_spinor(dims, seed=2017)[0].astype(np.complex64)).cuda()
    y0 = torch.empty_like(v)
    q.qcd_learned_apply(s.ctx, y0, v)
    q.qcd_debug_tc_skip_commit(s.ctx, True)
    with pytest.raises(q.QcdError) as e:
        q.qcd_learned_apply(s.ctx, torch.empty_like(v), v)
    assert e.value.code == q.QCD_ERR_TIMEOUT
    q.qcd_debug_tc_skip_commit(s.ctx, False)
    y1 = torch.empty_like(v)
    q.qcd_learned_apply(s.ctx, y1, v)
    torch.cuda.synchronize()
    assert torch.equal(y1, y0)
    s.close()
