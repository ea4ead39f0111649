"""Runs the oracle's full nested solve on the 12^3 x 24 workload (kappa 0.12,
c_SW 1.6, eps 0.3, gauge seed 1001, source seed 2001, SAP blocks 6^3 x 12,
sub-blocks 3^3 x 6, omega 1, 4 sweeps, 4 cycles, tol 1e-10) and records its
iteration counts in solve_counts.json.

The counts are a record of the FP64 method's convergence on this workload
(the paper prints none); the GPU solver's counts are reported beside them.
The file is written by this script only (it calls nothing but the oracle).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import qcd_inputs as qi  # noqa: E402

WORKLOAD = dict(dims=(12, 12, 12, 24), kappa=0.12, csw=1.6, eps=0.3, gauge_seed=1001, source_seed=2001,
                block=(6, 6, 6, 12), subblock=(3, 3, 3, 6), omega=1.0, nsweep=4, nsap=4, tol=1e-10,
                inner_tol=1e-5)


def main():
    w = WORKLOAD
    U = qi.gauge_field(w["dims"], w["eps"], seed=w["gauge_seed"])
    _, F = oracle.clover(w["dims"], U, w["csw"], w["kappa"])
    b = qi.gaussian_spinor(w["dims"], seed=w["source_seed"])[0]
    t0 = time.time()
    x, status, st = oracle.solve(w["dims"], U, F, w["kappa"], w["block"], w["subblock"], w["omega"], w["nsweep"],
                                 w["nsap"], b, tol=w["tol"], inner_tol=w["inner_tol"])
    st["status"] = status
    st["seconds_on_writer_host"] = round(time.time() - t0, 1)
    st["workload"] = {k: list(v) if isinstance(v, tuple) else v for k, v in w.items()}
    with open(os.path.join(HERE, "solve_counts.json"), "w") as f:
        json.dump({"12x12x12x24": st}, f, indent=1)
    print(st)


if __name__ == "__main__":
    main()
