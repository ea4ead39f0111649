"""Pins of the oracle's learned correction (a linear gauge-covariant network of
parallel-transport layers; a project addition, not in the paper).

* A single layer with on-site weight 0 and spin weights (1 -+ gamma_mu) on the
  forward/backward transports is exactly the Wilson hop H of Eq. (2).
* Gauge covariance N[U^g](g x) = g N[U](x), and linearity.
* The analytic gradient equals central finite differences of the loss.
"""
import numpy as np
import pytest

import oracle
import qcd_inputs as qi
from test_oracle_operator import gauge_transform

CHANS = (1, 3, 2, 1)


def random_weights(chans, seed, scale=0.3):
    n = oracle.learned_weight_count(chans)
    r = qi.normals(seed, 2 * n)
    return scale * (r[0::2] + 1j * r[1::2])


@pytest.mark.parametrize("bc_t", [1, -1])
def test_hop_is_a_special_layer(bc_t):
    dims = (4, 4, 4, 6)
    U = qi.gauge_field(dims, 0.3, seed=41)
    W = np.zeros((9, 1, 1, 4, 4), dtype=np.complex128)
    for mu in range(4):
        g = oracle.gamma(mu)
        W[1 + 2 * mu, 0, 0] = np.eye(4) - g
        W[2 + 2 * mu, 0, 0] = np.eye(4) + g
    x = qi.gaussian_spinor(dims, seed=42)
    y = oracle.learned_forward(dims, U, (1, 1), W.reshape(-1), x, bc_t=bc_t)
    h = oracle.hop(dims, U, x[0], bc_t=bc_t)
    assert np.abs(y[0] - h).max() < 1e-13 * np.abs(h).max()


def test_gauge_covariance_and_linearity():
    dims = (4, 4, 4, 4)
    U = qi.gauge_field(dims, 0.3, seed=43)
    g = qi.random_gauge_transform(dims, seed=44)
    Ug = gauge_transform(dims, U, g)
    W = random_weights(CHANS, 45)
    x = qi.gaussian_spinor(dims, seed=46)
    xg = np.einsum("nab,cnsb->cnsa", g, x)
    lhs = oracle.learned_forward(dims, Ug, CHANS, W, xg)
    rhs = np.einsum("nab,cnsb->cnsa", g, oracle.learned_forward(dims, U, CHANS, W, x))
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()
    x2 = qi.gaussian_spinor(dims, seed=47)
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    lin = oracle.learned_forward(dims, U, CHANS, W, a * x + b * x2)
    sep = a * oracle.learned_forward(dims, U, CHANS, W, x) + b * oracle.learned_forward(dims, U, CHANS, W, x2)
    assert np.abs(lin - sep).max() < 1e-12 * np.abs(sep).max()


def test_gradient_matches_finite_differences():
    dims = (2, 2, 2, 4)
    U = qi.gauge_field(dims, 0.3, seed=48)
    W = random_weights(CHANS, 49)
    rho = qi.gaussian_spinor(dims, seed=50)
    eps = qi.gaussian_spinor(dims, seed=51)
    loss, grad = oracle.learned_loss_grad(dims, U, CHANS, W, rho, eps)
    assert loss > 0
    rng = np.random.default_rng(0)
    h = 1e-6
    idx = rng.choice(len(W), size=12, replace=False)
    for i in idx:
        for part, unit in ((0, 1.0), (1, 1j)):
            Wp, Wm = W.copy(), W.copy()
            Wp[i] += h * unit
            Wm[i] -= h * unit
            fd = (oracle.learned_loss_grad(dims, U, CHANS, Wp, rho, eps)[0] -
                  oracle.learned_loss_grad(dims, U, CHANS, Wm, rho, eps)[0]) / (2 * h)
            an = grad[2 * i + part]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (i, part, fd, an)
