"""Pins of the oracle's operator D = 1 - kappa F H (Eq. (2)) and its clover term.

Each test checks the oracle against something the paper or the mathematics
fixes independently of the oracle's own code: textbook gamma-matrix
identities, the free-field plane-wave closed form, gauge covariance,
gamma_5-hermiticity, and the clover term of a constant abelian field.
"""
import itertools

import numpy as np
import pytest

import oracle
import qcd_inputs as qi

KAPPA = 0.12
CSW = 1.6


def site_coords(dims):
    V = qi.volume(dims)
    return np.array(np.unravel_index(np.arange(V), dims, order="F")).T  # x fastest


# ---------------------------------------------------------------------------
# gamma matrices (Sec. 3: Dirac representation, gamma_4 diagonal)
# ---------------------------------------------------------------------------

def textbook_dirac_gammas():
    s = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    z = np.zeros((2, 2))
    g = [np.block([[z, -1j * sk], [1j * sk, z]]) for sk in s]
    g.append(np.diag([1.0, 1.0, -1.0, -1.0]).astype(complex))
    return g


def test_gamma_identities():
    g = [oracle.gamma(m) for m in range(4)]
    for mu, nu in itertools.product(range(4), range(4)):
        anti = g[mu] @ g[nu] + g[nu] @ g[mu]
        assert np.allclose(anti, 2 * (mu == nu) * np.eye(4), atol=1e-15)
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T, atol=1e-15)
    # gamma_4 diagonal (Dirac representation) and the stated phase convention
    assert np.allclose(g[3], np.diag([1, 1, -1, -1]))
    for mine, ref in zip(g, textbook_dirac_gammas()):
        assert np.allclose(mine, ref, atol=1e-15)
    g5 = oracle.gamma(4)
    assert np.allclose(g5, g[0] @ g[1] @ g[2] @ g[3], atol=1e-15)
    assert np.allclose(g5, -np.block([[np.zeros((2, 2)), np.eye(2)], [np.eye(2), np.zeros((2, 2))]]))
    for mu in range(4):
        assert np.allclose(g5 @ g[mu] + g[mu] @ g5, 0, atol=1e-15)


# ---------------------------------------------------------------------------
# free field U = 1: plane waves diagonalise D
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bc_t", [1, -1])
@pytest.mark.parametrize("k", [(0, 0, 0, 0), (1, 0, 2, 3), (3, 1, 1, 0), (2, 3, 0, 1)])
def test_free_field_plane_wave(k, bc_t):
    dims = (4, 4, 6, 8)
    U = qi.unit_gauge(dims)
    A, F = oracle.clover(dims, U, CSW, KAPPA)
    assert np.abs(F - np.eye(12)).max() == 0.0  # F_{mu nu} = 0 so the clover term is 1
    L = np.array(dims, dtype=float)
    p = 2 * np.pi * np.array(k) / L
    if bc_t == -1:
        p[3] = (2 * k[3] + 1) * np.pi / L[3]
    rng = np.random.default_rng(7)
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    phase = np.exp(1j * site_coords(dims) @ p)
    psi = phase[:, None, None] * u[None]
    out = oracle.apply_D(dims, U, F, KAPPA, psi, bc_t=bc_t)
    g = textbook_dirac_gammas()
    Mp = np.eye(4) * (1 - KAPPA * np.sum(2 * np.cos(p)))
    for mu in range(4):
        Mp = Mp + KAPPA * 2j * np.sin(p[mu]) * g[mu]
    expect = phase[:, None, None] * (Mp @ u)[None]
    assert np.abs(out - expect).max() <= 1e-14 * np.abs(expect).max()


# ---------------------------------------------------------------------------
# gauge covariance of D and of the clover term
# ---------------------------------------------------------------------------

def gauge_transform(dims, U, g):
    V = qi.volume(dims)
    x = site_coords(dims)
    Ug = np.empty_like(U)
    for mu in range(4):
        xs = x.copy()
        xs[:, mu] = (xs[:, mu] + 1) % dims[mu]
        nf = xs[:, 0] + dims[0] * (xs[:, 1] + dims[1] * (xs[:, 2] + dims[2] * xs[:, 3]))
        Ug[:, mu] = g @ U[:, mu] @ g[nf].conj().transpose(0, 2, 1)
    return Ug


@pytest.mark.parametrize("bc_t", [1, -1])
def test_gauge_covariance(bc_t):
    dims = (4, 4, 4, 6)
    U = qi.gauge_field(dims, 0.3, seed=11)
    g = qi.random_gauge_transform(dims, seed=12)
    Ug = gauge_transform(dims, U, g)
    _, F = oracle.clover(dims, U, CSW, KAPPA)
    _, Fg = oracle.clover(dims, Ug, CSW, KAPPA)
    # F(n) -> (1 (x) g(n)) F(n) (1 (x) g(n))^dag
    G12 = np.einsum("ab,ncd->nacbd", np.eye(4), g).reshape(-1, 12, 12)
    assert np.abs(Fg - G12 @ F @ G12.conj().transpose(0, 2, 1)).max() < 1e-13
    psi = qi.gaussian_spinor(dims, seed=13)[0]
    psig = np.einsum("nab,nsb->nsa", g, psi)
    lhs = oracle.apply_D(dims, Ug, Fg, KAPPA, psig, bc_t=bc_t)
    rhs = np.einsum("nab,nsb->nsa", g, oracle.apply_D(dims, U, F, KAPPA, psi, bc_t=bc_t))
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()


# ---------------------------------------------------------------------------
# gamma_5-hermiticity of M = A - kappa H, and D = A^{-1} M
# ---------------------------------------------------------------------------

def test_gamma5_hermiticity_and_clover_structure():
    dims = (4, 4, 4, 4)
    U = qi.gauge_field(dims, 0.3, seed=21)
    A, F = oracle.clover(dims, U, CSW, KAPPA)
    g5 = np.kron(oracle.gamma(4), np.eye(3))
    # A hermitian, commutes with gamma_5, and A F = 1
    assert np.abs(A - A.conj().transpose(0, 2, 1)).max() < 1e-15
    assert np.abs(g5 @ A - A @ g5).max() < 1e-15
    assert np.abs(A @ F - np.eye(12)).max() < 1e-13
    phi = qi.gaussian_spinor(dims, seed=22)[0]
    chi = qi.gaussian_spinor(dims, seed=23)[0]
    G5 = lambda v: (v.reshape(-1, 12) @ g5.T).reshape(v.shape)
    lhs = np.vdot(phi, G5(oracle.apply_M(dims, U, A, KAPPA, chi)))
    rhs = np.conj(np.vdot(chi, G5(oracle.apply_M(dims, U, A, KAPPA, phi))))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    # D = A^{-1} M = F M
    Dpsi = oracle.apply_D(dims, U, F, KAPPA, chi)
    FMpsi = oracle.site_matrix(F, oracle.apply_M(dims, U, A, KAPPA, chi))
    assert np.abs(Dpsi - FMpsi).max() < 1e-13


# ---------------------------------------------------------------------------
# constant abelian field in one plane: closed form of the clover term
# ---------------------------------------------------------------------------

def abelian_field(dims, mu, nu, kq):
    """Every (mu,nu) plaquette equals diag(e^{i phi}, e^{-i phi}, 1), phi = 2 pi k/(L_mu L_nu)."""
    V = qi.volume(dims)
    x = site_coords(dims)
    Lm, Ln = dims[mu], dims[nu]
    phi = 2 * np.pi * kq / (Lm * Ln)
    U = qi.unit_gauge(dims)
    ph = np.exp(1j * phi * x[:, mu])
    U[:, nu, 0, 0] = ph
    U[:, nu, 1, 1] = np.conj(ph)
    edge = x[:, mu] == Lm - 1
    tw = np.exp(-1j * phi * Lm * x[:, nu])
    U[edge, mu, 0, 0] = tw[edge]
    U[edge, mu, 1, 1] = np.conj(tw[edge])
    return U, phi


@pytest.mark.parametrize("plane", list(itertools.combinations(range(4), 2)))
def test_abelian_clover_closed_form(plane):
    mu, nu = plane
    dims = (4, 6, 4, 6)
    U, phi = abelian_field(dims, mu, nu, kq=1)
    A, F = oracle.clover(dims, U, CSW, KAPPA)
    g = textbook_dirac_gammas()
    sigma = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
    Fmn = np.diag([np.sin(phi), -np.sin(phi), 0.0])
    # all-pairs sum with c_SW kappa / 2 equals c_SW kappa times the mu<nu term
    expect = np.eye(12) - CSW * KAPPA * np.kron(sigma, Fmn)
    assert np.abs(A - expect[None]).max() < 1e-14
    assert np.abs(F - np.linalg.inv(expect)[None]).max() < 1e-13
    if plane == (0, 1):
        # sigma_12 = diag(-1, 1, -1, 1): spin 0, colour 0 sees 1 + c_SW kappa sin(phi)
        assert abs(A[0, 0, 0] - (1 + CSW * KAPPA * np.sin(phi))) < 1e-15
    ev = np.sort(np.linalg.eigvalsh(A[0]))
    s = CSW * KAPPA * np.sin(phi)
    assert np.allclose(ev, np.sort([1 - s] * 4 + [1 + s] * 4 + [1.0] * 4), atol=1e-14)
