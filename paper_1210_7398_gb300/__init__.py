"""Python binding of libqcd.so, the GB300 nested-BiCGStab / SAP / ll-SSOR solver.

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels (``csrc/``).  The functions carry the C ABI's names
(``include/qcd.h``); :class:`Solver` bundles them for convenience.  Spinors
and links are passed as torch tensors (device memory, any CUDA stream) or
numpy arrays (host memory, copied inside the call).  There is no CPU
fallback: importing the binding without a built library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqcd.so")

QCD_OK, QCD_ERR_ARG, QCD_ERR_CUDA, QCD_ERR_OOM = 0, -1, -2, -3
QCD_ERR_SINGULAR, QCD_ERR_NOCONV, QCD_ERR_BREAKDOWN, QCD_ERR_TIMEOUT, QCD_ERR_STATE = -4, -5, -6, -7, -8
QCD_F64, QCD_F32, QCD_F16, QCD_F32_SU3, QCD_F32X2 = 0, 1, 2, 4, 5
QCD_K_DSLASH32, QCD_K_DSLASH64, QCD_K_SSOR, QCD_K_SAPHOP, QCD_K_BLAS, QCD_K_OTHER, QCD_K_LEARNED = range(7)
KERNEL_CLASSES = ("dslash32", "dslash64", "ssor", "saphop", "blas", "other", "learned")

EXPORTS = ("qcd_create", "qcd_destroy", "qcd_last_error", "qcd_set_boundary", "qcd_load_gauge",
           "qcd_build_clover", "qcd_apply_D", "qcd_sap_precondition", "qcd_solve", "qcd_set_profiling",
           "qcd_kernel_stats", "qcd_launch_count", "qcd_bench_dslash", "qcd_sap_precondition_noalloc",
           "qcd_set_sap_ctas", "qcd_set_sap_form", "qcd_sap_plan_tables", "qcd_set_graphs", "qcd_autotune", "qcd_learned_weight_count",
           "qcd_learned_set_weights", "qcd_learned_get_weights", "qcd_learned_apply", "qcd_learned_loss_grad",
           "qcd_learned_train", "qcd_learned_evaluate", "qcd_solve_multi", "qcd_set_tune_cache", "qcd_bench_fp32_peak", "qcd_bench_smem_peak",
           "qcd_debug_inject_breakdown", "qcd_learned_save", "qcd_learned_load", "qcd_debug_tc_skip_commit")


class QcdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("qcd status %d: %s" % (code, msg))
        self.code = code


class qcd_params(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("csw", ctypes.c_double),
                ("block", ctypes.c_int * 4), ("subblock", ctypes.c_int * 4),
                ("omega", ctypes.c_double), ("nsweep", ctypes.c_int), ("nsap", ctypes.c_int),
                ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("max_inner", ctypes.c_int),
                ("bc_t", ctypes.c_int), ("sap_storage", ctypes.c_int),
                ("learned", ctypes.c_int), ("sap_ctas", ctypes.c_int), ("block_solver", ctypes.c_int),
                ("rhs_group", ctypes.c_int), ("outer_precision", ctypes.c_int)]


class qcd_learned_verdict(ctypes.Structure):
    _fields_ = [("plain_ms", ctypes.c_double), ("learned_ms", ctypes.c_double),
                ("plain_relres", ctypes.c_double), ("learned_relres", ctypes.c_double),
                ("plain_outer", ctypes.c_int), ("plain_inner", ctypes.c_int),
                ("learned_outer", ctypes.c_int), ("learned_inner", ctypes.c_int),
                ("use_learned", ctypes.c_int), ("pad", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class qcd_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("restarts", ctypes.c_int), ("true_rel_res", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_dslash", ctypes.c_double), ("ms_sap", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libqcd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libqcd.so not built: run `python -m paper_1210_7398_gb300.build` (needs nvcc)")
    L = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "qcd_create": (I, [ctypes.POINTER(P), ctypes.POINTER(I), P]),
        "qcd_destroy": (None, [P]),
        "qcd_last_error": (ctypes.c_char_p, [P]),
        "qcd_set_boundary": (I, [P, I]),
        "qcd_load_gauge": (I, [P, P, I]),
        "qcd_build_clover": (I, [P, D, D]),
        "qcd_apply_D": (I, [P, P, P, I, I]),
        "qcd_sap_precondition": (I, [P, P, P, ctypes.POINTER(qcd_params), I]),
        "qcd_sap_precondition_noalloc": (I, [P, P, P, ctypes.POINTER(qcd_params)]),
        "qcd_solve": (I, [P, P, P, ctypes.POINTER(qcd_params), I, ctypes.POINTER(qcd_stats)]),
        "qcd_set_profiling": (I, [P, I]),
        "qcd_set_sap_ctas": (I, [P, I]),
        "qcd_set_sap_form": (I, [P, I]),
        "qcd_sap_plan_tables": (I, [P, P, P, I, I, I, P, P, P, P, P, P]),
        "qcd_set_graphs": (I, [P, I]),
        "qcd_learned_weight_count": (ctypes.c_long, []),
        "qcd_learned_set_weights": (I, [P, P, ctypes.c_long]),
        "qcd_learned_get_weights": (I, [P, P, ctypes.c_long]),
        "qcd_learned_apply": (I, [P, P, P]),
        "qcd_learned_loss_grad": (I, [P, P, P, ctypes.POINTER(D), P]),
        "qcd_learned_train": (I, [P, P, I, ctypes.POINTER(qcd_params), I, I, ctypes.c_float, P]),
        "qcd_learned_evaluate": (I, [P, P, I, ctypes.POINTER(qcd_params), ctypes.POINTER(qcd_learned_verdict)]),
        "qcd_solve_multi": (I, [I, P, P, P, P, P, P]),
        "qcd_autotune": (I, [P, P, I, ctypes.POINTER(qcd_params), ctypes.POINTER(qcd_params),
                             ctypes.POINTER(D), I]),
        "qcd_kernel_stats": (I, [P, I, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(D), I]),
        "qcd_launch_count": (ctypes.c_long, [P]),
        "qcd_bench_dslash": (I, [P, I, I, I]),
        "qcd_set_tune_cache": (I, [ctypes.c_char_p]),
        "qcd_bench_fp32_peak": (I, [P, I, ctypes.POINTER(D)]),
        "qcd_bench_smem_peak": (I, [P, I, ctypes.POINTER(D)]),
        "qcd_debug_inject_breakdown": (I, [P, I]),
        "qcd_debug_tc_skip_commit": (I, [P, I]),
        "qcd_learned_save": (I, [P, ctypes.c_char_p]),
        "qcd_learned_load": (I, [P, ctypes.c_char_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    """Device pointer of a torch tensor, or host pointer of a numpy array (contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError("expected a torch tensor or a numpy array")


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


# ---- thin wrappers with the C names ------------------------------------------------

def qcd_create(dims, stream=None):
    L = load_library()
    ctx = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    rc = L.qcd_create(ctypes.byref(ctx), d, ctypes.c_void_p(stream or 0))
    if rc != QCD_OK:
        raise QcdError(rc, "qcd_create failed")
    return ctx


def qcd_destroy(ctx):
    load_library().qcd_destroy(ctx)


def qcd_last_error(ctx) -> str:
    return (load_library().qcd_last_error(ctx) or b"").decode()


def _check(ctx, rc):
    if rc != QCD_OK:
        raise QcdError(rc, qcd_last_error(ctx))
    return rc


def qcd_set_boundary(ctx, bc_t: int):
    return _check(ctx, load_library().qcd_set_boundary(ctx, int(bc_t)))


def qcd_load_gauge(ctx, U):
    return _check(ctx, load_library().qcd_load_gauge(ctx, _ptr(U), 1 if _is_device(U) else 0))


def qcd_build_clover(ctx, kappa: float, csw: float):
    return _check(ctx, load_library().qcd_build_clover(ctx, float(kappa), float(csw)))


def qcd_apply_D(ctx, out, inp, prec: int, nrhs: int = 1):
    return _check(ctx, load_library().qcd_apply_D(ctx, _ptr(out), _ptr(inp), int(prec), int(nrhs)))


def qcd_sap_precondition(ctx, out, inp, params: qcd_params, nrhs: int = 1):
    return _check(ctx, load_library().qcd_sap_precondition(ctx, _ptr(out), _ptr(inp), ctypes.byref(params),
                                                           int(nrhs)))


def qcd_sap_precondition_noalloc(ctx, out, inp, params: qcd_params):
    """out = M_SAP inp without any device allocation (device tensors, one right-hand side)."""
    return _check(ctx, load_library().qcd_sap_precondition_noalloc(ctx, _ptr(out), _ptr(inp), ctypes.byref(params)))


def qcd_solve(ctx, x, b, params: qcd_params, nrhs: int = 1, check: bool = True):
    st = qcd_stats()
    rc = load_library().qcd_solve(ctx, _ptr(x), _ptr(b), ctypes.byref(params), int(nrhs), ctypes.byref(st))
    if check:
        _check(ctx, rc)
    d = st.as_dict()
    d["rc"] = rc
    return d


def qcd_solve_multi(ctxs, xs, bs, params, nrhs, check: bool = True):
    """Solves the instances (contexts with distinct streams) concurrently; returns (rc, [stats dict])."""
    n = len(ctxs)
    C = ctypes.c_void_p * n
    prm = (qcd_params * n)(*params)
    nr = (ctypes.c_int * n)(*[int(v) for v in nrhs])
    st = (qcd_stats * n)()
    cv = ctypes.c_void_p
    arrs = [C(*[cv(c) if not isinstance(c, cv) else c for c in ctxs]), C(*[_ptr(v) for v in xs]),
            C(*[_ptr(v) for v in bs]), prm, nr, st]
    rc = load_library().qcd_solve_multi(n, *[ctypes.cast(a, cv) for a in arrs])
    out = [st[i].as_dict() for i in range(n)]
    if check and rc != QCD_OK:
        bad = next((i for i in range(n) if out[i]["status"] != QCD_OK), 0)
        _check(ctxs[bad], rc)
    return rc, out


def qcd_set_sap_ctas(ctx, min_ctas: int):
    return _check(ctx, load_library().qcd_set_sap_ctas(ctx, int(min_ctas)))


def qcd_sap_plan_tables(dims, block, subblock, sap_ctas: int = 0, half: bool = False, sms: int = 152) -> dict:
    """The SSOR schedule for a geometry (host only, no GPU): meta counts and per-site arrays
    (level, owner, slot, chunk; block-local lexicographic order) and the per-step barrier flags."""
    import numpy as np
    L = load_library()
    iv = lambda v: (ctypes.c_int * 4)(*[int(x) for x in v])
    meta = (ctypes.c_int * 8)()
    rc = L.qcd_sap_plan_tables(iv(dims), iv(block), iv(subblock), int(sap_ctas), int(bool(half)), int(sms), meta,
                               None, None, None, None, None)
    if rc != QCD_OK:
        raise QcdError(rc, "qcd_sap_plan_tables: geometry rejected")
    vol, nch = meta[0], meta[3]
    arrs = [np.empty(vol, dtype=np.int32) for _ in range(4)]
    flags = np.empty(2 * nch, dtype=np.uint8)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = L.qcd_sap_plan_tables(iv(dims), iv(block), iv(subblock), int(sap_ctas), int(bool(half)), int(sms), meta,
                               *[ptr(a) for a in arrs], ptr(flags))
    if rc != QCD_OK:
        raise QcdError(rc, "qcd_sap_plan_tables: geometry rejected")
    names = ("vol", "levels", "ctas", "chunks", "nslot", "slab_vol", "thread", "smem_bytes")
    out = {k: int(meta[i]) for i, k in enumerate(names)}
    out.update(level=arrs[0], owner=arrs[1], slot=arrs[2], chunk=arrs[3], flags=flags)
    return out


def qcd_set_sap_form(ctx, form: int):
    """0: lanes per SSOR site update chosen per launch; 1: 32; 2: 8 (identical results)."""
    return _check(ctx, load_library().qcd_set_sap_form(ctx, int(form)))


def qcd_autotune(ctx, b, base: qcd_params, nrhs: int = 1, max_candidates: int = 0):
    """Returns (best qcd_params, best time in ms) over the candidate SAP set-ups."""
    best = qcd_params()
    ms = ctypes.c_double()
    _check(ctx, load_library().qcd_autotune(ctx, _ptr(b), int(nrhs), ctypes.byref(base), ctypes.byref(best),
                                            ctypes.byref(ms), int(max_candidates)))
    return best, ms.value


def qcd_set_tune_cache(path):
    """Tuning results are looked up in, and appended to, this JSON-lines file (None: off)."""
    return load_library().qcd_set_tune_cache(path.encode() if path else None)


def params_dict(p: qcd_params) -> dict:
    return {"block": list(p.block), "subblock": list(p.subblock), "omega": p.omega, "nsweep": p.nsweep,
            "nsap": p.nsap, "sap_storage": {QCD_F32: "f32", QCD_F16: "f16"}.get(p.sap_storage, p.sap_storage),
            "sap_ctas": p.sap_ctas, "learned": p.learned,
            "block_solver": {0: "ll-ssor", 1: "even-odd mr"}.get(p.block_solver, p.block_solver),
            "rhs_group": p.rhs_group, "outer_precision": {QCD_F64: "f64", QCD_F32: "f32", QCD_F32X2: "f32x2"}.get(p.outer_precision)}


LEARNED_CHANS = (1, 8, 8, 1)


def qcd_learned_weight_count() -> int:
    return int(load_library().qcd_learned_weight_count())


def qcd_learned_set_weights(ctx, w):
    """w: complex64 array/tensor [qcd_learned_weight_count()] (layers concatenated, each [9][cout][cin][4][4])."""
    return _check(ctx, load_library().qcd_learned_set_weights(ctx, _ptr(w), int(qcd_learned_weight_count())))


def qcd_learned_get_weights(ctx):
    w = np.empty(qcd_learned_weight_count(), dtype=np.complex64)
    _check(ctx, load_library().qcd_learned_get_weights(ctx, _ptr(w), len(w)))
    return w


def qcd_learned_save(ctx, path):
    """Writes the correction's weights (JSON header line + complex64 data)."""
    return _check(ctx, load_library().qcd_learned_save(ctx, str(path).encode()))


def qcd_learned_load(ctx, path):
    """Reads weights written by qcd_learned_save and sets them."""
    return _check(ctx, load_library().qcd_learned_load(ctx, str(path).encode()))


def qcd_learned_apply(ctx, out, inp):
    return _check(ctx, load_library().qcd_learned_apply(ctx, _ptr(out), _ptr(inp)))


def qcd_learned_loss_grad(ctx, rho, eps):
    """(loss, grad): grad float32 [2 n] = 2 (Re, Im) of dL/dW* for one pair."""
    loss = ctypes.c_double()
    g = np.empty(2 * qcd_learned_weight_count(), dtype=np.float32)
    _check(ctx, load_library().qcd_learned_loss_grad(ctx, _ptr(rho), _ptr(eps), ctypes.byref(loss), _ptr(g)))
    return loss.value, g


def qcd_learned_train(ctx, sources, npairs, params: qcd_params, epochs, batch, lr):
    """Trains the correction on pairs made from ``sources``; returns the loss history [epochs + 1]."""
    hist = np.zeros(epochs + 1)
    _check(ctx, load_library().qcd_learned_train(ctx, _ptr(sources), int(npairs), ctypes.byref(params), int(epochs),
                                                 int(batch), ctypes.c_float(lr), _ptr(hist)))
    return hist


def qcd_learned_evaluate(ctx, b, nrhs, params: qcd_params) -> dict:
    """Solves b with plain SAP and with the learned correction; records and returns the verdict
    (times, iterations, residuals, use_learned)."""
    v = qcd_learned_verdict()
    _check(ctx, load_library().qcd_learned_evaluate(ctx, _ptr(b), int(nrhs), ctypes.byref(params), ctypes.byref(v)))
    return v.as_dict()


def learned_init_weights(seed: int, scale_last: float = 0.01) -> np.ndarray:
    """Seeded initial weights (complex64): N(0, 1/fan_in) per component, last layer scaled down
    so the untrained correction starts near zero."""
    import qcd_inputs as qi
    parts = []
    off = 0
    for l in range(len(LEARNED_CHANS) - 1):
        cin, cout = LEARNED_CHANS[l], LEARNED_CHANS[l + 1]
        n = 9 * cout * cin * 16
        r = qi.normals(seed + 7919 * l, 2 * n)
        sc = (1.0 / np.sqrt(9 * cin * 4)) * (scale_last if l == len(LEARNED_CHANS) - 2 else 1.0)
        parts.append(sc * (r[0::2] + 1j * r[1::2]))
        off += n
    return np.concatenate(parts).astype(np.complex64)


def qcd_set_graphs(ctx, on: bool):
    return _check(ctx, load_library().qcd_set_graphs(ctx, 1 if on else 0))


def qcd_set_profiling(ctx, on: bool):
    return _check(ctx, load_library().qcd_set_profiling(ctx, 1 if on else 0))


def qcd_kernel_stats(ctx, kclass: int, reset: bool = False):
    n = ctypes.c_long()
    ms = ctypes.c_double()
    _check(ctx, load_library().qcd_kernel_stats(ctx, int(kclass), ctypes.byref(n), ctypes.byref(ms),
                                                1 if reset else 0))
    return n.value, ms.value


def qcd_launch_count(ctx) -> int:
    return int(load_library().qcd_launch_count(ctx))


def qcd_bench_dslash(ctx, prec: int, nrhs: int, iters: int):
    return _check(ctx, load_library().qcd_bench_dslash(ctx, int(prec), int(nrhs), int(iters)))


def qcd_debug_inject_breakdown(ctx, count: int):
    """Test hook: the next count outer iterations start from rho = 0 (a host-made breakdown)."""
    return _check(ctx, load_library().qcd_debug_inject_breakdown(ctx, int(count)))


def qcd_debug_tc_skip_commit(ctx, on: bool):
    """Test hook: the tensor-core learned layer commits nothing, so its bounded waits run out."""
    return _check(ctx, load_library().qcd_debug_tc_skip_commit(ctx, 1 if on else 0))


def qcd_bench_fp32_peak(ctx, iters: int = 64) -> float:
    """Measured FP32 FMA throughput of the context's GPU, TFLOP/s."""
    t = ctypes.c_double()
    _check(ctx, load_library().qcd_bench_fp32_peak(ctx, int(iters), ctypes.byref(t)))
    return t.value


def qcd_bench_smem_peak(ctx, iters: int = 64) -> float:
    """Measured shared-memory load bandwidth of the GPU in GB/s."""
    t = ctypes.c_double()
    _check(ctx, load_library().qcd_bench_smem_peak(ctx, int(iters), ctypes.byref(t)))
    return t.value


def make_params(kappa, csw, block, subblock, omega=1.0, nsweep=4, nsap=4, tol=1e-10, inner_tol=1e-5,
                max_outer=100, max_inner=500, bc_t=1, sap_storage=QCD_F32, sap_ctas=0,
                block_solver=0, rhs_group=0, outer_precision=0) -> qcd_params:
    p = qcd_params()
    p.kappa, p.csw = float(kappa), float(csw)
    p.block = (ctypes.c_int * 4)(*block)
    p.subblock = (ctypes.c_int * 4)(*subblock)
    p.omega, p.nsweep, p.nsap = float(omega), int(nsweep), int(nsap)
    p.tol, p.inner_tol = float(tol), float(inner_tol)
    p.max_outer, p.max_inner = int(max_outer), int(max_inner)
    p.bc_t, p.sap_storage, p.learned, p.sap_ctas = int(bc_t), int(sap_storage), 0, int(sap_ctas)
    p.block_solver = int(block_solver)
    p.rhs_group = int(rhs_group)
    p.outer_precision = int(outer_precision)
    return p


class Solver:
    """One context on the current CUDA device and torch's current stream."""

    def __init__(self, dims, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.dims = tuple(int(v) for v in dims)
        self.ctx = qcd_create(self.dims, stream)

    def close(self):
        if self.ctx:
            qcd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_boundary(self, bc_t):
        qcd_set_boundary(self.ctx, bc_t)

    def load_gauge(self, U):
        qcd_load_gauge(self.ctx, U)

    def build_clover(self, kappa, csw):
        qcd_build_clover(self.ctx, kappa, csw)

    def apply_D(self, out, inp, prec, nrhs=1):
        qcd_apply_D(self.ctx, out, inp, prec, nrhs)

    def sap_precondition(self, out, inp, params, nrhs=1):
        qcd_sap_precondition(self.ctx, out, inp, params, nrhs)

    def solve(self, x, b, params, nrhs=1, check=True):
        return qcd_solve(self.ctx, x, b, params, nrhs, check)
