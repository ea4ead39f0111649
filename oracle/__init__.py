"""Python binding of the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it to check and time the CUDA path.  The
CUDA library never imports, links or calls it, and it shares no code with it.

Every array is complex128 in the canonical layout (links [V,4,3,3],
spinors [V,4,3], dense site matrices [V,12,12] with index spin*3+colour).
Parity of the Krylov iteration counts and timings is not pinned by the paper
(it prints none); the operator, the clover term, the ll ordering, SSOR, the
even-odd block inverse, SAP, the inner BiCGStab on its own and the final
solution are pinned by the tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=gnu11"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no CPU-specific flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i, d = ctypes.c_int, ctypes.c_double
            L.orc_gamma.argtypes = [i, P]
            L.orc_hop.argtypes = [P, i, P, P, P]
            L.orc_clover.argtypes = [P, P, d, d, P, P]
            L.orc_clover.restype = i
            L.orc_site_matrix.argtypes = [ctypes.c_long, P, P, P]
            L.orc_apply_D.argtypes = [P, i, P, P, d, P, P]
            L.orc_apply_M.argtypes = [P, i, P, P, d, P, P]
            L.orc_check_geometry.argtypes = [P, P, P]
            L.orc_colours.argtypes = [P, P, P]
            L.orc_apply_D_colour.argtypes = [P, i, P, P, P, d, i, i, P, P]
            L.orc_ll_order.argtypes = [P, P, P]
            L.orc_ssor.argtypes = [P, i, P, P, d, P, P, d, i, i, P, P]
            L.orc_ssor.restype = i
            L.orc_sap.argtypes = [P, i, P, P, d, P, P, d, i, i, P, P]
            L.orc_sap.restype = i
            L.orc_sap_bs.argtypes = [P, i, P, P, d, P, P, d, i, i, i, P, P]
            L.orc_sap_bs.restype = i
            L.orc_eo_mr.argtypes = [P, i, P, P, d, P, i, i, P, P]
            L.orc_eo_mr.restype = i
            L.orc_inner_bicgstab.argtypes = [P, i, P, P, d, P, P, d, i, i, d, i, P, P]
            L.orc_inner_bicgstab.restype = i
            L.orc_solve.argtypes = [P, i, P, P, d, P, P, d, i, i, d, d, i, i, P, P, P]
            L.orc_solve.restype = i
            L.orc_learned_layer.argtypes = [P, i, P, i, i, P, P, P]
            L.orc_learned_forward.argtypes = [P, i, P, i, P, P, P, P]
            L.orc_learned_loss_grad.argtypes = [P, i, P, i, P, P, P, P, P]
            L.orc_learned_loss_grad.restype = d
            _lib = L
    return _lib


def _c(a, dtype=np.complex128):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _ivec(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _vol(dims):
    return int(np.prod(dims))


def gamma(mu: int) -> np.ndarray:
    """gamma_{mu+1} (mu = 0..3) or gamma_5 (mu = 4) as the oracle defines them."""
    out = np.zeros((4, 4), dtype=np.complex128)
    lib().orc_gamma(mu, out.ctypes.data_as(ctypes.c_void_p))
    return out


def hop(dims, U, psi, bc_t: int = 1):
    Lk, Lp = _ivec(dims)
    U, Up = _c(U)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    lib().orc_hop(Lp, bc_t, Up, pp, out.ctypes.data_as(ctypes.c_void_p))
    return out


def clover(dims, U, csw: float, kappa: float):
    """Returns (A, F) with A = 1 - (c_SW kappa/2) sigma.F and F = A^-1, [V,12,12]."""
    Lk, Lp = _ivec(dims)
    U, Up = _c(U)
    V = _vol(dims)
    A = np.empty((V, 12, 12), dtype=np.complex128)
    F = np.empty((V, 12, 12), dtype=np.complex128)
    st = lib().orc_clover(Lp, Up, csw, kappa, A.ctypes.data_as(ctypes.c_void_p),
                          F.ctypes.data_as(ctypes.c_void_p))
    if st != 0:
        raise ArithmeticError("clover term singular")
    return A, F


def site_matrix(M, psi):
    M, Mp = _c(M)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    lib().orc_site_matrix(M.shape[0], Mp, pp, out.ctypes.data_as(ctypes.c_void_p))
    return out


def apply_D(dims, U, F, kappa, psi, bc_t: int = 1):
    Lk, Lp = _ivec(dims)
    U, Up = _c(U)
    F, Fp = _c(F)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    lib().orc_apply_D(Lp, bc_t, Up, Fp, kappa, pp, out.ctypes.data_as(ctypes.c_void_p))
    return out


def apply_M(dims, U, A, kappa, psi, bc_t: int = 1):
    Lk, Lp = _ivec(dims)
    U, Up = _c(U)
    A, Ap = _c(A)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    lib().orc_apply_M(Lp, bc_t, Up, Ap, kappa, pp, out.ctypes.data_as(ctypes.c_void_p))
    return out


def colours(dims, block):
    Lk, Lp = _ivec(dims)
    bk, bp = _ivec(block)
    out = np.empty(_vol(dims), dtype=np.int32)
    lib().orc_colours(Lp, bp, out.ctypes.data_as(ctypes.c_void_p))
    return out


def check_geometry(dims, block, sub=None) -> bool:
    Lk, Lp = _ivec(dims)
    bk, bp = _ivec(block)
    if sub is None:
        return lib().orc_check_geometry(Lp, bp, None) == 0
    sk, sp = _ivec(sub)
    return lib().orc_check_geometry(Lp, bp, sp) == 0


def apply_D_colour(dims, U, F, kappa, block, row_c, col_c, psi, bc_t: int = 1):
    Lk, Lp = _ivec(dims)
    bk, bp = _ivec(block)
    U, Up = _c(U)
    F, Fp = _c(F)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    lib().orc_apply_D_colour(Lp, bc_t, bp, Up, Fp, kappa, row_c, col_c, pp,
                             out.ctypes.data_as(ctypes.c_void_p))
    return out


def ll_order(block, sub) -> np.ndarray:
    bk, bp = _ivec(block)
    sk, sp = _ivec(sub)
    out = np.empty(_vol(block), dtype=np.int32)
    if lib().orc_ll_order(bp, sp, out.ctypes.data_as(ctypes.c_void_p)) != 0:
        raise ValueError("sub-block must divide block")
    return out


def ssor(dims, U, F, kappa, block, sub, omega, nsweep, colour, f, x=None, bc_t: int = 1):
    """x = A_BB f on every block of ``colour`` (other sites of x unchanged)."""
    Lk, Lp = _ivec(dims)
    bk, bp = _ivec(block)
    sk, sp = _ivec(sub)
    U, Up = _c(U)
    F, Fp = _c(F)
    f, fp = _c(f)
    x = np.zeros_like(f) if x is None else np.ascontiguousarray(x, dtype=np.complex128).copy()
    st = lib().orc_ssor(Lp, bc_t, Up, Fp, kappa, bp, sp, omega, nsweep, colour, fp,
                        x.ctypes.data_as(ctypes.c_void_p))
    if st != 0:
        raise ValueError("bad SAP geometry")
    return x


def eo_mr(dims, U, F, kappa, block, nmr, colour, f, x=None, bc_t: int = 1):
    """x = the even-odd block inverse of f (nmr minimal-residual steps on the Schur complement
    of D_BB on the even sites, then the odd sites) on every block of ``colour``."""
    Lk, Lp = _ivec(dims)
    bk, bp = _ivec(block)
    U, Up = _c(U)
    F, Fp = _c(F)
    f, fp = _c(f)
    x = np.zeros_like(f) if x is None else np.ascontiguousarray(x, dtype=np.complex128).copy()
    st = lib().orc_eo_mr(Lp, bc_t, Up, Fp, kappa, bp, nmr, colour, fp, x.ctypes.data_as(ctypes.c_void_p))
    if st != 0:
        raise ValueError("bad SAP geometry or nmr")
    return x


def sap(dims, U, F, kappa, block, sub, omega, nsweep, nsap, v, bc_t: int = 1, block_solver: int = 0):
    """M_SAP v (Eq. (4)).  block_solver 0: ll-ordered SSOR block inverses (nsweep sweeps);
    1: even-odd minimal-residual block inverses (nsweep steps, omega and sub unused)."""
    Lk, Lp = _ivec(dims)
    bk, bp = _ivec(block)
    sk, sp = _ivec(sub)
    U, Up = _c(U)
    F, Fp = _c(F)
    v, vp = _c(v)
    out = np.empty_like(v)
    st = lib().orc_sap_bs(Lp, bc_t, Up, Fp, kappa, bp, sp, omega, nsweep, nsap, block_solver, vp,
                          out.ctypes.data_as(ctypes.c_void_p))
    if st != 0:
        raise ValueError("bad SAP geometry")
    return out


def inner_bicgstab(dims, U, F, kappa, block, sub, omega, nsweep, nsap, tol, maxit, q, bc_t: int = 1):
    Lk, Lp = _ivec(dims)
    bk, bp = _ivec(block)
    sk, sp = _ivec(sub)
    U, Up = _c(U)
    F, Fp = _c(F)
    q, qp = _c(q)
    y = np.empty_like(q)
    it = lib().orc_inner_bicgstab(Lp, bc_t, Up, Fp, kappa, bp, sp, omega, nsweep, nsap, tol,
                                  maxit, qp, y.ctypes.data_as(ctypes.c_void_p))
    return y, it


def solve(dims, U, F, kappa, block, sub, omega, nsweep, nsap, b, tol=1e-10, inner_tol=1e-5,
          max_outer=100, max_inner=500, x0=None, bc_t: int = 1):
    """Nested flexible BiCGStab (FP64 outer, FP64 inner, M_SAP right preconditioner).

    Returns (x, status, stats) with stats = dict(outer, inner, restarts, true_rel_res).
    """
    Lk, Lp = _ivec(dims)
    bk, bp = _ivec(block)
    sk, sp = _ivec(sub)
    U, Up = _c(U)
    F, Fp = _c(F)
    b, bpp = _c(b)
    x = np.zeros_like(b) if x0 is None else np.ascontiguousarray(x0, dtype=np.complex128).copy()
    st = np.zeros(4)
    status = lib().orc_solve(Lp, bc_t, Up, Fp, kappa, bp, sp, omega, nsweep, nsap, tol, inner_tol,
                             max_outer, max_inner, bpp, x.ctypes.data_as(ctypes.c_void_p),
                             st.ctypes.data_as(ctypes.c_void_p))
    return x, status, dict(outer=int(st[0]), inner=int(st[1]), restarts=int(st[2]),
                           true_rel_res=float(st[3]))


# ---------------------------------------------------------------------------
# learned correction (a project addition): linear gauge-covariant network
# ---------------------------------------------------------------------------

def learned_weight_count(chans) -> int:
    """Complex weights of a network with channel counts chans[0..nl]: 9 x cout x cin x 4 x 4 per layer."""
    return sum(9 * chans[l + 1] * chans[l] * 16 for l in range(len(chans) - 1))


def learned_forward(dims, U, chans, W, x, bc_t: int = 1):
    """N(x): x complex [chans[0]][V][4][3], W complex (layer-concatenated [9][cout][cin][4][4])."""
    Lk, Lp = _ivec(dims)
    ck, cp = _ivec(chans)
    U, Up = _c(U)
    W, Wp = _c(W)
    x, xp = _c(x)
    V = _vol(dims)
    y = np.empty((chans[-1], V, 4, 3), dtype=np.complex128)
    lib().orc_learned_forward(Lp, bc_t, Up, len(chans) - 1, cp, Wp, xp, y.ctypes.data_as(ctypes.c_void_p))
    return y


def learned_loss_grad(dims, U, chans, W, rho, eps, bc_t: int = 1):
    """(loss, grad) for one pair; grad is real [2 * nweights] = 2 (Re, Im) of dL/dW*."""
    Lk, Lp = _ivec(dims)
    ck, cp = _ivec(chans)
    U, Up = _c(U)
    W, Wp = _c(W)
    rho, rp = _c(rho)
    eps, ep = _c(eps)
    g = np.empty(2 * learned_weight_count(chans))
    loss = lib().orc_learned_loss_grad(Lp, bc_t, Up, len(chans) - 1, cp, Wp, rp, ep,
                                       g.ctypes.data_as(ctypes.c_void_p))
    return loss, g
