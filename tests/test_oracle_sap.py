"""Pins of the oracle's block decomposition, ll ordering, SSOR, SAP and nested BiCGStab.

* ll ordering (Sec. 3): special cases s = 1^4 and s = b reduce to natural
  lexicographic order; a tuple-sort restatement of the definition; brute force
  non-adjacency of the sites that share a local position.
* SSOR (Sec. 3): the site loop equals the matrix form of forward/backward
  substitution with the strictly lower / upper split of the dense D_BB in ll
  order, and converges to the dense block inverse.
* SAP (Eq. (4), Alg. 1): the recurrence equals K sum_j (1-DK)^j built from
  dense matrices; with exact block inverses the odd part of (1-DK)v vanishes;
  M_SAP v approaches D^{-1} v as N_SAP grows.
* Nested BiCGStab (Sec. 2): the solution equals a dense LU solve.
* Colour blocks (Eq. 3): they sum to D and are the dense D restricted to one block (diagonal
  blocks) or to neighbouring blocks (off-diagonal blocks).
* Even-odd block inverse: odd rows exact, monotone residual, the one-step least-squares
  optimum, the dense block inverse in the limit.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import qcd_inputs as qi

KAPPA = 0.12
CSW = 1.6


def dense_D(dims, U, F, bc_t=1, kappa=KAPPA):
    V = qi.volume(dims)
    N = 12 * V
    cols = np.empty((N, N), dtype=np.complex128)
    e = np.zeros((V, 4, 3), dtype=np.complex128)
    flat = e.reshape(-1)
    for j in range(N):
        flat[:] = 0
        flat[j] = 1.0
        cols[:, j] = oracle.apply_D(dims, U, F, kappa, e, bc_t=bc_t).reshape(-1)
    return cols


def site_coords(dims):
    V = qi.volume(dims)
    return np.array(np.unravel_index(np.arange(V), dims, order="F")).T


# ---------------------------------------------------------------------------
# ll ordering
# ---------------------------------------------------------------------------

def ll_order_by_tuple_sort(b, s):
    """Definition restated: sort by local position (t,z,y,x major..minor), then sub-block."""
    vol = int(np.prod(b))
    keys = []
    for yl in range(vol):
        y = np.unravel_index(yl, b, order="F")
        l = [y[m] % s[m] for m in range(4)]
        q = [y[m] // s[m] for m in range(4)]
        keys.append(((l[3], l[2], l[1], l[0]), (q[3], q[2], q[1], q[0]), yl))
    return np.array([k[2] for k in sorted(keys)], dtype=np.int32)


@pytest.mark.parametrize("b", [(2, 2, 2, 2), (4, 2, 4, 2), (6, 6, 6, 12)])
def test_ll_order_special_cases(b):
    vol = int(np.prod(b))
    assert np.array_equal(oracle.ll_order(b, (1, 1, 1, 1)), np.arange(vol))
    assert np.array_equal(oracle.ll_order(b, b), np.arange(vol))


@pytest.mark.parametrize("b,s", [((4, 4, 4, 4), (2, 2, 2, 2)), ((6, 6, 6, 12), (3, 3, 3, 6)),
                                 ((6, 6, 6, 6), (3, 3, 3, 3)), ((4, 2, 4, 2), (2, 1, 2, 1)),
                                 ((4, 4, 2, 6), (2, 4, 1, 3))])
def test_ll_order_definition_and_independence(b, s):
    order = oracle.ll_order(b, s)
    assert np.array_equal(np.sort(order), np.arange(int(np.prod(b))))
    assert np.array_equal(order, ll_order_by_tuple_sort(b, s))
    if (b, s) == ((4, 4, 4, 4), (2, 2, 2, 2)):
        # the first 16 sites are the sub-block origins (local position 0)
        origins = [2 * qx + 4 * (2 * qy + 4 * (2 * qz + 4 * 2 * qt))
                   for qt, qz, qy, qx in itertools.product(range(2), repeat=4)]
        assert list(order[:16]) == origins
    if min(s) >= 2:
        nsb = int(np.prod(np.array(b) // np.array(s)))
        y = np.array(np.unravel_index(order, b, order="F")).T
        for g in range(len(order) // nsb):
            grp = y[g * nsb:(g + 1) * nsb]
            d = np.abs(grp[:, None, :] - grp[None, :, :]).sum(-1)
            assert not np.any(d == 1), "sites sharing a local position must not be neighbours"


def test_colours_checkerboard():
    dims, b = (4, 4, 4, 8), (2, 2, 2, 2)
    col = oracle.colours(dims, b)
    x = site_coords(dims)
    assert np.array_equal(col, (x // np.array(b)).sum(1) % 2)
    assert not oracle.check_geometry((6, 4, 4, 4), (2, 2, 2, 2))  # 3 blocks along x: odd
    assert not oracle.check_geometry((4, 4, 4, 4), (4, 2, 2, 2))  # 1 block along x
    assert oracle.check_geometry((12, 12, 12, 24), (6, 6, 6, 12), (3, 3, 3, 6))


# ---------------------------------------------------------------------------
# SSOR: site loop vs matrix form on 2^4 blocks of a 4^4 lattice
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def field44():
    dims = (4, 4, 4, 4)
    U = qi.gauge_field(dims, 0.3, seed=1000)
    _, F = oracle.clover(dims, U, CSW, KAPPA)
    return dims, U, F, dense_D(dims, U, F)


def block_sites_ll(dims, b, B, s):
    """Global site indices of block B (block coordinates), in ll order."""
    order = ll_order_by_tuple_sort(b, s)
    y = np.array(np.unravel_index(order, b, order="F")).T
    xg = np.array(B)[None] * np.array(b)[None] + y
    return xg[:, 0] + dims[0] * (xg[:, 1] + dims[1] * (xg[:, 2] + dims[2] * xg[:, 3]))


def dof(sites):
    return (np.asarray(sites)[:, None] * 12 + np.arange(12)[None]).reshape(-1)


def ssor_matrix(DBB, omega, nsweep):
    """Matrix of f -> x after nsweep SSOR sweeps from x = 0 (forward then backward
    substitution on D_BB = 1 - L - U split in the given order)."""
    n = DBB.shape[0]
    Lm = -np.tril(DBB, -1)
    Um = -np.triu(DBB, 1)
    I = np.eye(n)
    X = np.zeros((n, n), dtype=complex)
    for _ in range(nsweep):
        Xh = sla.solve_triangular(I - omega * Lm, ((1 - omega) * I + omega * Um) @ X + omega * I,
                                  lower=True)
        X = sla.solve_triangular(I - omega * Um, ((1 - omega) * I + omega * Lm) @ Xh + omega * I,
                                 lower=False)
    return X


@pytest.mark.parametrize("s", [(1, 1, 1, 1), (2, 2, 2, 2), (2, 1, 2, 1)])
@pytest.mark.parametrize("omega", [1.0, 1.2])
def test_ssor_site_loop_equals_matrix_form(field44, s, omega):
    dims, U, F, Dm = field44
    b = (2, 2, 2, 2)
    nsweep = 3
    f = qi.gaussian_spinor(dims, seed=5)[0]
    x = oracle.ssor(dims, U, F, KAPPA, b, s, omega, nsweep, 0, f)
    fl, xl = f.reshape(-1), x.reshape(-1)
    for B in itertools.product(range(2), repeat=4):
        sites = block_sites_ll(dims, b, B, s)
        idx = dof(sites)
        DBB = Dm[np.ix_(idx, idx)]
        # unit site diagonal: no diagonal solve in the substitutions
        for k in range(len(sites)):
            assert np.allclose(DBB[12 * k:12 * k + 12, 12 * k:12 * k + 12], np.eye(12), atol=1e-15)
        if sum(B) % 2 == 0:
            X = ssor_matrix(DBB, omega, nsweep)
            expect = X @ fl[idx]
            assert np.abs(xl[idx] - expect).max() < 1e-13 * np.abs(expect).max()
            # combined one-step form x_{k+1} = x_k + w(2-w)(1-wU)^-1(1-wL)^-1 (f - D x_k)
            n = len(idx)
            Minv = omega * (2 - omega) * np.linalg.inv(np.eye(n) + omega * np.triu(DBB, 1)) @ \
                np.linalg.inv(np.eye(n) + omega * np.tril(DBB, -1))
            Y = np.zeros((n, n), dtype=complex)
            for _ in range(nsweep):
                Y = Y + Minv @ (np.eye(n) - DBB @ Y)
            assert np.abs(Y - X).max() < 1e-12
        else:
            assert np.all(xl[idx] == 0)  # other colour untouched


def test_ssor_converges_to_block_inverse(field44):
    dims, U, F, Dm = field44
    b, s = (2, 2, 2, 2), (2, 2, 2, 2)
    f = qi.gaussian_spinor(dims, seed=6)[0]
    x = oracle.ssor(dims, U, F, KAPPA, b, s, 1.0, 60, 1, f).reshape(-1)
    fl = f.reshape(-1)
    errs = []
    for B in itertools.product(range(2), repeat=4):
        if sum(B) % 2 != 1:
            continue
        idx = dof(block_sites_ll(dims, b, B, s))
        exact = np.linalg.solve(Dm[np.ix_(idx, idx)], fl[idx])
        errs.append(np.abs(x[idx] - exact).max() / np.abs(exact).max())
    assert max(errs) < 1e-12
    # error falls with the sweep count
    prev = np.inf
    for ns in (1, 2, 4, 8):
        xs = oracle.ssor(dims, U, F, KAPPA, b, s, 1.0, ns, 1, f).reshape(-1)
        e = np.linalg.norm(xs - x)
        assert e < prev
        prev = e


# ---------------------------------------------------------------------------
# SAP: recurrence vs dense algebra; exact block inverses; limit N_SAP -> inf
# ---------------------------------------------------------------------------

def dense_sap(dims, Dm, b, s, omega, nsweep, nsap):
    V = qi.volume(dims)
    N = 12 * V
    col = oracle.colours(dims, b)
    PE = np.repeat(col == 0, 12).astype(float)
    PO = 1.0 - PE
    A = {0: np.zeros((N, N), dtype=complex), 1: np.zeros((N, N), dtype=complex)}
    nb = [dims[m] // b[m] for m in range(4)]
    for B in itertools.product(*[range(n) for n in nb]):
        c = sum(B) % 2
        idx = dof(block_sites_ll(dims, b, B, s))
        A[c][np.ix_(idx, idx)] = ssor_matrix(Dm[np.ix_(idx, idx)], omega, nsweep)
    D_OE = PO[:, None] * Dm * PE[None, :]
    K = A[0] + A[1] - A[1] @ D_OE @ A[0]
    I = np.eye(N)
    T = I - Dm @ K
    S = np.zeros((N, N), dtype=complex)
    P = I.copy()
    for _ in range(nsap):
        S += P
        P = T @ P
    return K @ S, K, PE, PO


@pytest.mark.parametrize("s,nsweep,nsap,omega", [((1, 1, 1, 1), 2, 3, 1.0), ((2, 2, 2, 2), 1, 2, 1.1)])
def test_sap_recurrence_equals_dense(field44, s, nsweep, nsap, omega):
    dims, U, F, Dm = field44
    b = (2, 2, 2, 2)
    Msap, _, _, _ = dense_sap(dims, Dm, b, s, omega, nsweep, nsap)
    v = qi.gaussian_spinor(dims, seed=8)[0]
    out = oracle.sap(dims, U, F, KAPPA, b, s, omega, nsweep, nsap, v).reshape(-1)
    expect = Msap @ v.reshape(-1)
    assert np.abs(out - expect).max() < 1e-12 * np.abs(expect).max()


def test_sap_exact_blocks_and_limit(field44):
    dims, U, F, Dm = field44
    b, s = (2, 2, 2, 2), (2, 2, 2, 2)
    v = qi.gaussian_spinor(dims, seed=9)[0].reshape(-1)
    col = np.repeat(oracle.colours(dims, b), 12)
    # nsweep large: A_BB = D_BB^{-1}; then DK is block triangular and the odd
    # component of (1 - DK) v vanishes
    Kv = oracle.sap(dims, U, F, KAPPA, b, s, 1.0, 60, 1, v.reshape(-1, 4, 3)).reshape(-1)
    res = v - Dm @ Kv
    assert np.abs(res[col == 1]).max() < 1e-12 * np.abs(v).max()
    assert np.abs(res[col == 0]).max() > 1e-3
    # M_SAP v -> D^{-1} v as N_SAP grows (|1 - DK| < 1 comfortably at kappa = 0.10)
    k2 = 0.10
    _, F2 = oracle.clover(dims, U, CSW, k2)
    D2 = dense_D(dims, U, F2, kappa=k2)
    exact = np.linalg.solve(D2, v)
    errs = []
    for nsap in (1, 2, 4, 8, 16, 32):
        m = oracle.sap(dims, U, F2, k2, b, s, 1.0, 4, nsap, v.reshape(-1, 4, 3)).reshape(-1)
        errs.append(np.linalg.norm(m - exact) / np.linalg.norm(exact))
    assert all(e2 < e1 for e1, e2 in zip(errs[:-1], errs[1:-1]))
    assert errs[-1] < 1e-12


# ---------------------------------------------------------------------------
# nested BiCGStab vs dense LU
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["2^4", "4^4"])
def test_nested_bicgstab_matches_dense_lu(field44, case):
    if case == "2^4":
        dims = (2, 2, 2, 2)
        U = qi.gauge_field(dims, 0.3, seed=31)
        _, F = oracle.clover(dims, U, CSW, KAPPA)
        Dm = dense_D(dims, U, F)
        b, s = (1, 1, 1, 1), (1, 1, 1, 1)
    else:
        dims, U, F, Dm = field44
        b, s = (2, 2, 2, 2), (1, 1, 1, 1)
    src = qi.gaussian_spinor(dims, seed=2000)[0]
    x, status, st = oracle.solve(dims, U, F, KAPPA, b, s, 1.0, 4, 4, src, tol=1e-10)
    assert status == 0
    exact = np.linalg.solve(Dm, src.reshape(-1))
    assert st["true_rel_res"] <= 1e-10
    r = src.reshape(-1) - Dm @ x.reshape(-1)
    assert np.linalg.norm(r) / np.linalg.norm(src) <= 1e-10
    assert np.linalg.norm(x.reshape(-1) - exact) / np.linalg.norm(exact) <= 1e-9


# ---------------------------------------------------------------------------
# even-odd minimal-residual block inverse (the alternative block solver that
# Sec. 3 compares ll-SSOR with): pinned to the dense D of the 4^4 lattice
# ---------------------------------------------------------------------------

def parity_dof(dims):
    return np.repeat(site_coords(dims).sum(axis=1) % 2, 12)


def colour1_blocks(dims, b):
    nb = [dims[m] // b[m] for m in range(4)]
    return [B for B in itertools.product(*[range(n) for n in nb]) if sum(B) % 2 == 1]


def test_eo_mr_odd_rows_exact_and_residual_monotone(field44):
    """The odd sites are solved exactly after any number of steps (x_o is rebuilt from
    x_e), and the block residual, which then lives on the even sites, never grows."""
    dims, U, F, Dm = field44
    b = (2, 2, 2, 2)
    f = qi.gaussian_spinor(dims, seed=11)[0]
    fl = f.reshape(-1)
    col = np.repeat(oracle.colours(dims, b), 12)
    par = parity_dof(dims)
    prev = np.inf
    for nmr in (1, 2, 3, 5, 8, 13):
        x = oracle.eo_mr(dims, U, F, KAPPA, b, nmr, 1, f).reshape(-1)
        assert np.all(x[col == 0] == 0)  # other colour untouched
        res = fl - Dm @ np.where(col == 1, x, 0)  # blocks of one colour are not neighbours
        assert np.abs(res[(col == 1) & (par == 1)]).max() < 1e-12 * np.abs(fl).max()
        e = np.linalg.norm(res[col == 1])
        assert e <= prev * (1 + 1e-12)
        prev = e
    assert prev < 0.5 * np.linalg.norm(fl[col == 1])


def test_eo_mr_one_step_is_the_least_squares_step(field44):
    """One step: x_e = alpha fhat with alpha minimising |fhat - alpha S fhat| for the
    Schur complement S = 1 - D_eo D_oe of each dense block (D_ee = D_oo = 1)."""
    dims, U, F, Dm = field44
    b = (2, 2, 2, 2)
    f = qi.gaussian_spinor(dims, seed=12)[0]
    fl = f.reshape(-1)
    x = oracle.eo_mr(dims, U, F, KAPPA, b, 1, 1, f).reshape(-1)
    par = parity_dof(dims)
    for B in colour1_blocks(dims, b):
        idx = dof(block_sites_ll(dims, b, B, (1, 1, 1, 1)))
        ev, od = idx[par[idx] == 0], idx[par[idx] == 1]
        assert np.abs(Dm[np.ix_(ev, ev)] - np.eye(len(ev))).max() < 1e-15
        Deo, Doe = Dm[np.ix_(ev, od)], Dm[np.ix_(od, ev)]
        S = np.eye(len(ev)) - Deo @ Doe
        fhat = fl[ev] - Deo @ fl[od]
        alpha = np.linalg.lstsq((S @ fhat)[:, None], fhat, rcond=None)[0][0]
        xe = alpha * fhat
        assert np.abs(x[ev] - xe).max() < 1e-12 * np.abs(xe).max()
        xo = fl[od] - Doe @ xe
        assert np.abs(x[od] - xo).max() < 1e-12 * np.abs(xo).max()


def test_eo_mr_converges_to_block_inverse(field44):
    dims, U, F, Dm = field44
    b = (2, 2, 2, 2)
    f = qi.gaussian_spinor(dims, seed=13)[0]
    fl = f.reshape(-1)
    x = oracle.eo_mr(dims, U, F, KAPPA, b, 80, 1, f).reshape(-1)
    for B in colour1_blocks(dims, b):
        idx = dof(block_sites_ll(dims, b, B, (1, 1, 1, 1)))
        exact = np.linalg.solve(Dm[np.ix_(idx, idx)], fl[idx])
        assert np.abs(x[idx] - exact).max() < 1e-10 * np.abs(exact).max()


def test_sap_with_eo_blocks_limit_equals_ssor_limit(field44):
    """With many steps both block solvers give the exact block inverse, so the two SAP
    variants agree; with few steps they differ."""
    dims, U, F, Dm = field44
    b, s = (2, 2, 2, 2), (1, 1, 1, 1)
    v = qi.gaussian_spinor(dims, seed=14)[0]
    a = oracle.sap(dims, U, F, KAPPA, b, s, 1.0, 80, 2, v, block_solver=1)
    c = oracle.sap(dims, U, F, KAPPA, b, s, 1.0, 60, 2, v, block_solver=0)
    assert np.abs(a - c).max() < 1e-10 * np.abs(c).max()
    a2 = oracle.sap(dims, U, F, KAPPA, b, s, 1.0, 2, 2, v, block_solver=1)
    assert np.abs(a2 - c).max() > 1e-4 * np.abs(c).max()


def test_eo_mr_larger_blocks_matrix_free():
    """4^4 blocks of an 8^4 lattice (and 3^3 x 6 blocks of 6^3 x 12, where a block holds
    unequal numbers of even and odd sites): odd rows exact, residual non-increasing,
    checked with the block-restricted operator."""
    for dims, b in (((8, 8, 8, 8), (4, 4, 4, 4)), ((6, 6, 6, 12), (3, 3, 3, 6))):
        U = qi.gauge_field(dims, 0.3, seed=1002)
        _, F = oracle.clover(dims, U, CSW, KAPPA)
        f = qi.gaussian_spinor(dims, seed=15)[0]
        col = np.repeat(oracle.colours(dims, b), 12)
        par = parity_dof(dims)
        prev = np.inf
        for nmr in (1, 3, 9, 27):
            x = oracle.eo_mr(dims, U, F, KAPPA, b, nmr, 0, f)
            Dx = oracle.apply_D_colour(dims, U, F, KAPPA, b, 0, 0, x).reshape(-1)
            res = (f.reshape(-1) - Dx)[col == 0]
            assert np.abs(res[par[col == 0] == 1]).max() < 1e-12 * np.abs(f).max()
            e = np.linalg.norm(res)
            assert e <= prev * (1 + 1e-12)
            prev = e
        assert prev < 0.1 * np.linalg.norm(f.reshape(-1)[col == 0])


def test_colour_blocks_of_D(field44):
    """Eq. 3: the four colour blocks P_r D P_c sum to D; D_EE and D_OO are D restricted to
    pairs of sites in one block (blocks of one colour are never neighbours), D_OE and D_EO
    to pairs in neighbouring blocks of opposite colour."""
    dims, U, F, Dm = field44
    b = (2, 2, 2, 2)
    psi = qi.gaussian_spinor(dims, seed=16)[0]
    parts = {(r, c): oracle.apply_D_colour(dims, U, F, KAPPA, b, r, c, psi).reshape(-1)
             for r in (0, 1) for c in (0, 1)}
    full = oracle.apply_D(dims, U, F, KAPPA, psi).reshape(-1)
    assert np.abs(sum(parts.values()) - full).max() < 1e-13 * np.abs(full).max()
    x = site_coords(dims)
    blk = np.ravel_multi_index(tuple((x // np.array(b)).T), [dims[m] // b[m] for m in range(4)], order="F")
    col = oracle.colours(dims, b)
    same_block = np.repeat(np.repeat(blk[:, None] == blk[None, :], 12, axis=0), 12, axis=1)
    cd = np.repeat(col, 12)
    v = psi.reshape(-1)
    for c in (0, 1):
        rows = cd == c
        expect = (Dm * same_block)[rows] @ np.where(cd == c, v, 0)
        assert np.abs(parts[(c, c)][rows] - expect).max() < 1e-13 * np.abs(expect).max()
        assert np.all(parts[(c, c)][~rows] == 0)
    cross = (Dm * ~same_block)[cd == 1] @ np.where(cd == 0, v, 0)
    assert np.abs(parts[(1, 0)][cd == 1] - cross).max() < 1e-13 * np.abs(cross).max()
