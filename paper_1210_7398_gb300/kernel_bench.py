"""Kernel micro-benchmarks of the library: one SAP application (M_SAP v, Eq. (4) with the
ll-SSOR block inverse of Sec. 3), one application of D (Eq. (2)) or one application of the
learned correction N (three gauge-covariant layers) on a synthetic lattice, repeated, with
per-class device times from the library's profiler.  For tuning by hand and for profilers (ncu),
which need a short program that runs one kernel family on a small case.

    python -m paper_1210_7398_gb300.kernel_bench sap --dims 24x24x24x48 --block 4x4x4x6 \\
        --subblock 2x2x2x3 --nrhs 4 --storage f16 --ctas -2 --reps 3
    python -m paper_1210_7398_gb300.kernel_bench dslash --dims 24x24x24x48 --prec f32 --nrhs 1
    python -m paper_1210_7398_gb300.kernel_bench learned --dims 24x24x24x48 --reps 3

Prints one JSON line.  Links: exp(i 0.3 X) from the seeded generator; sources Gaussian.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def dims_arg(s):
    v = tuple(int(t) for t in s.lower().split("x"))
    if len(v) != 4:
        raise argparse.ArgumentTypeError("four extents, e.g. 24x24x24x48")
    return v


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("what", choices=["sap", "dslash", "learned"])
    ap.add_argument("--dims", type=dims_arg, default=(24, 24, 24, 48))
    ap.add_argument("--kappa", type=float, default=0.122)
    ap.add_argument("--csw", type=float, default=1.6)
    ap.add_argument("--seed", type=int, default=1003)
    ap.add_argument("--block", type=dims_arg, default=(4, 4, 4, 4))
    ap.add_argument("--subblock", type=dims_arg, default=(2, 2, 2, 2))
    ap.add_argument("--nsweep", type=int, default=2)
    ap.add_argument("--nsap", type=int, default=2)
    ap.add_argument("--storage", choices=["f32", "f16"], default="f16")
    ap.add_argument("--ctas", type=int, default=-2, help="SSOR kernel form (qcd_set_sap_ctas)")
    ap.add_argument("--prec", choices=["f64", "f32", "f16", "su3", "x2"], default="f32")
    ap.add_argument("--nrhs", type=int, default=4)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)

    import torch

    import paper_1210_7398_gb300 as q
    import qcd_inputs as qi

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        U = qi.gauge_field(a.dims, 0.3, seed=a.seed, device="cuda")
        torch.cuda.synchronize()
        s = q.Solver(a.dims, stream=stream.cuda_stream)
        s.load_gauge(U)
        del U
        s.build_clover(a.kappa, a.csw)
        out = {"what": a.what, "dims": list(a.dims), "nrhs": a.nrhs, "reps": a.reps}
        if a.what == "sap":
            prm = q.make_params(a.kappa, a.csw, a.block, a.subblock, nsweep=a.nsweep, nsap=a.nsap,
                                sap_storage=q.QCD_F16 if a.storage == "f16" else q.QCD_F32, sap_ctas=a.ctas)
            v = qi.gaussian_spinor_torch(a.dims, 2003, a.nrhs, "cuda").to(torch.complex64).contiguous()
            y = torch.empty_like(v)
            torch.cuda.synchronize()
            s.sap_precondition(y, v, prm, nrhs=a.nrhs)  # builds the plan and the records
            q.qcd_set_profiling(s.ctx, True)
            for k in range(len(q.KERNEL_CLASSES)):
                q.qcd_kernel_stats(s.ctx, k, reset=True)
            for _ in range(a.reps):
                s.sap_precondition(y, v, prm, nrhs=a.nrhs)
            out["params"] = q.params_dict(prm)
        elif a.what == "learned":
            q.qcd_learned_set_weights(s.ctx, q.learned_init_weights(7))
            v = qi.gaussian_spinor_torch(a.dims, 2004, 1, "cuda")[0].to(torch.complex64).contiguous()
            y = torch.empty_like(v)
            q.qcd_learned_apply(s.ctx, y, v)
            q.qcd_set_profiling(s.ctx, True)
            for k in range(len(q.KERNEL_CLASSES)):
                q.qcd_kernel_stats(s.ctx, k, reset=True)
            for _ in range(a.reps):
                q.qcd_learned_apply(s.ctx, y, v)
            out["nrhs"] = 1
        else:
            pc = {"f32": q.QCD_F32, "f64": q.QCD_F64, "f16": q.QCD_F16, "su3": q.QCD_F32_SU3,
                  "x2": q.QCD_F32X2}[a.prec]
            q.qcd_bench_dslash(s.ctx, pc, a.nrhs, 1)
            q.qcd_set_profiling(s.ctx, True)
            for k in range(len(q.KERNEL_CLASSES)):
                q.qcd_kernel_stats(s.ctx, k, reset=True)
            q.qcd_bench_dslash(s.ctx, pc, a.nrhs, a.reps)
            out["prec"] = a.prec
        stats = {}
        for k, nm in enumerate(q.KERNEL_CLASSES):
            n, ms = q.qcd_kernel_stats(s.ctx, k, reset=True)
            if n:
                stats[nm] = {"launches": n, "ms": ms, "ms_per_launch": ms / n}
        q.qcd_set_profiling(s.ctx, False)
        out["kernels"] = stats
        s.close()
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
