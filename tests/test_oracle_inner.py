"""Pins of the oracle's inner BiCGStab alone (Sec. 2: the FP32 solver of D y = q,
right-preconditioned by M_SAP), independent of the outer flexible solve that
would converge even with a wrong alpha, beta or omega.

* Finite termination: BiCGStab's residual is Q_k(B) P_k(B) q with P_k the BiCG
  polynomial of B = D M_SAP; when the Krylov space of q under B has dimension
  m, P_m(B) q = 0 and the m-th iterate is exact.  On the free field of the 2^4
  lattice with single-site blocks m = 3 (measured here from the Krylov vectors
  by their singular values, not assumed).  A wrong beta or alpha breaks the
  BiCG biorthogonality and with it the termination.
* First step: r_1 is s - omega B s with s the residual of the form q - a B q
  orthogonal to r_hat = q (the BiCG step), and omega minimising |s - omega B s|
  (the stabilising step): r_1 is orthogonal to B s.  A conjugated omega still
  terminates but fails this.
* A near-exact preconditioner: M_SAP with 60 sweeps and 120 cycles is D^{-1}
  up to 1e-12, so one iteration gives the dense LU solution.
* A rough field: solved to 1e-12 the iterate equals the dense LU solution.
"""
import numpy as np
import pytest

import oracle
import qcd_inputs as qi

KAPPA = 0.12


def free_field(dims):
    U = np.zeros((qi.volume(dims), 4, 3, 3), dtype=np.complex128)
    U[:, :] = np.eye(3)
    return U


def ops(dims, U, F, block, sub, omega, nsweep, nsap, kappa=KAPPA):
    V = qi.volume(dims)

    def D(v):
        return oracle.apply_D(dims, U, F, kappa, v.reshape(V, 4, 3)).reshape(-1)

    def M(v):
        return oracle.sap(dims, U, F, kappa, block, sub, omega, nsweep, nsap, v.reshape(V, 4, 3)).reshape(-1)

    return D, M


def krylov_dimension(B, q, kmax=12, rel=1e-9):
    """Numerical rank of [q, Bq, B^2 q, ...] (columns normalised)."""
    K = [q / np.linalg.norm(q)]
    for _ in range(kmax):
        w = B(K[-1])
        K.append(w / np.linalg.norm(w))
    sv = np.linalg.svd(np.array(K).T, compute_uv=False)
    return int(np.sum(sv > rel * sv[0]))


def inner(dims, U, F, block, sub, omega, nsweep, nsap, q, maxit, tol=0.0):
    V = qi.volume(dims)
    y, it = oracle.inner_bicgstab(dims, U, F, KAPPA, block, sub, omega, nsweep, nsap, tol, maxit,
                                  q.reshape(V, 4, 3))
    return y.reshape(-1), it


@pytest.mark.parametrize("nsap", [1, 2])
def test_inner_bicgstab_finite_termination(nsap):
    dims = (2, 2, 2, 2)
    U = free_field(dims)
    _, F = oracle.clover(dims, U, 1.6, KAPPA)
    blk = (1, 1, 1, 1)
    D, M = ops(dims, U, F, blk, blk, 1.0, 1, nsap)
    q = qi.gaussian_spinor(dims, seed=5)[0].reshape(-1)
    m = krylov_dimension(lambda v: D(M(v)), q)
    assert 2 <= m <= 6
    y, it = inner(dims, U, F, blk, blk, 1.0, 1, nsap, q, m)
    assert it == m
    assert np.linalg.norm(q - D(y)) / np.linalg.norm(q) < 1e-12
    y, _ = inner(dims, U, F, blk, blk, 1.0, 1, nsap, q, m - 1)
    assert np.linalg.norm(q - D(y)) / np.linalg.norm(q) > 1e-6


def test_inner_bicgstab_first_step_is_bicg_then_minimal_residual():
    dims = (4, 4, 4, 4)
    U = qi.gauge_field(dims, 0.3, seed=1000)
    _, F = oracle.clover(dims, U, 1.6, KAPPA)
    blk, sub = (2, 2, 2, 2), (1, 1, 1, 1)
    D, M = ops(dims, U, F, blk, sub, 1.0, 2, 2)
    q = qi.gaussian_spinor(dims, seed=2000)[0].reshape(-1)
    y, it = inner(dims, U, F, blk, sub, 1.0, 2, 2, q, 1)
    assert it == 1
    r1 = q - D(y)
    Bq = D(M(q))
    # the BiCG half step: s in q + span{Bq}, orthogonal to r_hat = q
    a = np.vdot(q, q) / np.vdot(q, Bq)
    s = q - a * Bq
    assert abs(np.vdot(q, s)) < 1e-12 * np.linalg.norm(q) * np.linalg.norm(s)
    Bs = D(M(s))
    # r_1 = s - omega Bs for the omega minimising the norm: r_1 orthogonal to Bs
    om = np.vdot(Bs, s) / np.vdot(Bs, Bs)
    assert np.linalg.norm(r1 - (s - om * Bs)) / np.linalg.norm(r1) < 1e-11
    assert abs(np.vdot(Bs, r1)) < 1e-11 * np.linalg.norm(Bs) * np.linalg.norm(r1)
    # and y_1 is the matching combination of preconditioned vectors
    assert np.linalg.norm(y - (a * M(q) + om * M(s))) / np.linalg.norm(y) < 1e-11


def test_inner_bicgstab_exact_preconditioner_one_step():
    dims = (4, 4, 4, 4)
    U = qi.gauge_field(dims, 0.3, seed=1000)
    _, F = oracle.clover(dims, U, 1.6, KAPPA)
    blk, sub = (2, 2, 2, 2), (1, 1, 1, 1)
    D, M = ops(dims, U, F, blk, sub, 1.0, 60, 120)
    q = qi.gaussian_spinor(dims, seed=2000)[0].reshape(-1)
    Dm = np.column_stack([D(e) for e in np.eye(12 * qi.volume(dims), dtype=np.complex128)])
    exact = np.linalg.solve(Dm, q)
    assert np.linalg.norm(M(q) - exact) / np.linalg.norm(exact) < 1e-12  # the premise
    y, it = inner(dims, U, F, blk, sub, 1.0, 60, 120, q, 1)
    assert it == 1
    assert np.linalg.norm(y - exact) / np.linalg.norm(exact) < 1e-11


def test_inner_bicgstab_solves_to_dense_lu():
    dims = (4, 4, 4, 4)
    U = qi.gauge_field(dims, 0.3, seed=1000)
    _, F = oracle.clover(dims, U, 1.6, KAPPA)
    blk, sub = (2, 2, 2, 2), (1, 1, 1, 1)
    D, _ = ops(dims, U, F, blk, sub, 1.0, 4, 4)
    q = qi.gaussian_spinor(dims, seed=2000)[0].reshape(-1)
    Dm = np.column_stack([D(e) for e in np.eye(12 * qi.volume(dims), dtype=np.complex128)])
    exact = np.linalg.solve(Dm, q)
    y, it = inner(dims, U, F, blk, sub, 1.0, 4, 4, q, 200, tol=1e-12)
    assert it < 200
    assert np.linalg.norm(q - D(y)) / np.linalg.norm(q) <= 1e-12
    assert np.linalg.norm(y - exact) / np.linalg.norm(exact) <= 1e-10
