"""Benchmark: time to solve D x = b to a true relative residual of 1e-10 on
the 12^3 x 24 lattice (plain method: FP64 outer / FP32 inner nested BiCGStab,
SAP blocks 6^3 x 12, ll sub-blocks 3^3 x 6, SSOR omega = 1, 4 sweeps, 4 SAP
cycles), plus the bandwidth of the operator D on lattices larger than L2.

One step = one full solve from x0 = 0 (every kernel of the solver runs in
the step).  Prints one JSON line.  ``--impl reference`` times the FP64 CPU
oracle instead: each step is one full oracle solve of the same workload on
the host cores (10-20 s of CPU work).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solve time to rel. residual 1e-10, chosen vs plain; D GB/s vs HBM peak"
WORKLOAD = dict(name="12^3x24 plain nested BiCGStab + SAP(6^3x12 blocks, 3^3x6 ll sub-blocks)",
                dims=(12, 12, 12, 24), kappa=0.12, csw=1.6, eps=0.3, gauge_seed=1001, source_seed=2001,
                block=(6, 6, 6, 12), subblock=(3, 3, 3, 6), omega=1.0, nsweep=4, nsap=4, tol=1e-10,
                inner_tol=1e-5)
TABLE1_FLOP_PER_SITE = 1896  # flop per site of the clover hopping matrix without SU(3) reconstruction (Table 1)
D_BYTES_PER_SITE = {"f32": 768, "f64": 1536, "f16": 480, "su3": 672}  # in + out spinor, 4 links (each shared by 2 sites), clover
L2_FLUSH_BYTES = 512 << 20
# DRAM bytes (read + write) per launch of a kernel class on this workload, from one ncu capture
# of the current kernel (dram__bytes_read.sum + dram__bytes_write.sum); None where not captured
NCU_TRAFFIC = {"ssor": 28918016 + 0}
# warp instructions per launch and SMs the launch occupies, from the ncu capture of the plain
# workload's SSOR kernel (profiles/ssor_level_12x12x12x24_c8.md): 64 CTAs, one per SM
NCU_ISSUE = {"ssor": (66.6e6, 64)}


def issue_model(cls, avg_ms, sm_mhz):
    """The instruction-issue floor of a kernel class: its warp instructions per launch issued at
    4 per cycle (one per SM sub-partition) on the SMs it occupies, against the measured launch
    time.  None when the class has no instruction count."""
    if cls not in NCU_ISSUE or not avg_ms or not sm_mhz:
        return None
    instr, sms = NCU_ISSUE[cls]
    floor_ms = instr / (sms * 4.0 * sm_mhz * 1e6) * 1e3
    return {"warp_instructions_per_launch": instr, "sms": sms, "issue_per_cycle_per_sm": 4,
            "floor_ms": floor_ms, "avg_launch_ms": avg_ms, "frac": floor_ms / avg_ms}


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return dict(hbm_gbs=float(p["hbm_gbs"]), sm_max_mhz=float(p.get("sm_max_mhz", 2070.0)), source="measured")
    except Exception:
        return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, source="fallback")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smmax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smmax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smmax) if smmax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device: str = "cuda") -> float:
    """The largest of every rank's value (the slowest replica decides the step time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------

def oracle_setup():
    import oracle
    import qcd_inputs as qi
    w = WORKLOAD
    U = qi.gauge_field(w["dims"], w["eps"], seed=w["gauge_seed"])
    _, F = oracle.clover(w["dims"], U, w["csw"], w["kappa"])
    b = qi.gaussian_spinor(w["dims"], seed=w["source_seed"])[0]
    return U, F, b


def oracle_solve_seconds(U, F, b):
    """Wall seconds of one full oracle solve of the workload (FP64 outer and inner)."""
    import oracle
    w = WORKLOAD
    t0 = time.perf_counter()
    _, status, st = oracle.solve(w["dims"], U, F, w["kappa"], w["block"], w["subblock"], w["omega"], w["nsweep"],
                                 w["nsap"], b, tol=w["tol"], inner_tol=w["inner_tol"])
    return time.perf_counter() - t0, status, st


def cores_used():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    U, F, b = oracle_setup()
    for _ in range(args.warmup):
        oracle_solve_seconds(U, F, b)
    vals = []
    for _ in range(args.steps):
        t, status, st = oracle_solve_seconds(U, F, b)
        vals.append(t)
    v = statistics.mean(vals)
    sample = ("per step: one full FP64 oracle solve of the 12^3x24 workload from x0 = 0 to 1e-10 "
              "(outer %d, inner %d iterations, true rel. residual %.1e)" % (st["outer"], st["inner"],
                                                                             st["true_rel_res"]))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000 * v, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD["name"], "lattice": "12x12x12x24", "kappa": WORKLOAD["kappa"],
                      "csw": WORKLOAD["csw"], "tol": WORKLOAD["tol"]},
           "cpu_baseline": {"value": v, "unit": "s", "cores": cores_used(), "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def kernel_model(cls, V, nrhs_steps, prm, peaks):
    """(bound, algorithmic units per launch, unit, peak) for a kernel class."""
    fp32_tflops = 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
    if cls == "dslash32":
        return "hbm", V * D_BYTES_PER_SITE["f32"] / 1e9, "GB/s", peaks["hbm_gbs"]
    if cls == "dslash64":
        return "hbm", V * D_BYTES_PER_SITE["f64"] / 1e9, "GB/s", peaks["hbm_gbs"]
    if cls == "ssor":
        # one launch: the V/2 sites of one colour, 2 passes per sweep, Table-1 flops per site update
        return "alu", (V / 2) * 2 * prm["nsweep"] * TABLE1_FLOP_PER_SITE / 1e12, "TFLOP/s", fp32_tflops
    if cls == "saphop":
        return "hbm", V * D_BYTES_PER_SITE["f32"] / 1e9, "GB/s", peaks["hbm_gbs"]
    return None


def dslash_bandwidth(q, torch, dims, iters, peaks, seed=1002, variants=(("f32", 1),)):
    """GB/s of the operator D (K1) on internal-layout buffers, CUDA events on the context stream,
    for each (precision, right-hand sides) variant."""
    import qcd_inputs as qi
    V = qi.volume(dims)
    U = qi.gauge_field(dims, 0.3, seed=seed, device="cuda")
    s = q.Solver(dims)
    s.load_gauge(U)
    del U
    s.build_clover(0.12, 1.6)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = []
    for prec, nrhs in variants:
        pc = {"f32": q.QCD_F32, "f64": q.QCD_F64, "f16": q.QCD_F16, "su3": q.QCD_F32_SU3}[prec]
        q.qcd_bench_dslash(s.ctx, pc, nrhs, 3)
        times = []
        for _ in range(iters):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            q.qcd_bench_dslash(s.ctx, pc, nrhs, 1)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        ms = statistics.median(times)
        # per right-hand side: both spinors; links and clover once per launch
        spin = 384 if prec == "f64" else 192  # FP16 storage keeps FP32 spinors
        field = D_BYTES_PER_SITE[prec] - spin
        byts = V * (spin * nrhs + field)
        gbs = byts / (ms * 1e-3) / 1e9
        out.append({"lattice": "x".join(map(str, dims)), "V": V, "prec": prec, "nrhs": nrhs, "ms": ms, "GB_s": gbs,
                    "GFLOP_s": V * nrhs * TABLE1_FLOP_PER_SITE / (ms * 1e-3) / 1e9,
                    "frac_measured": gbs / peaks["hbm_gbs"], "frac_nominal_8TBs": gbs / 8000.0,
                    "bytes_per_launch": byts, "timing": "median of %d launches, L2 flushed before each" % iters})
    s.close()
    del flush
    torch.cuda.empty_cache()
    return out


def learned_section(q, qi, torch, s, dims, prm, b, nrhs, npairs, epochs, lr=3e-3, batch=8):
    """Trains the learned correction on npairs (residual, error) pairs of the plain SAP set-up prm
    (sources seed 3000, weights seed 4000), then lets qcd_learned_evaluate assess it on b."""
    t0 = time.perf_counter()
    q.qcd_learned_set_weights(s.ctx, q.learned_init_weights(4000))
    src = qi.gaussian_spinor_torch(dims, 3000, npairs, "cuda").to(torch.complex64).contiguous()
    hist = q.qcd_learned_train(s.ctx, src, npairs, prm, epochs=epochs, batch=batch, lr=lr)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del src
    v = q.qcd_learned_evaluate(s.ctx, b, nrhs, prm)
    return {"pairs": npairs, "epochs": epochs, "lr": lr, "batch": batch, "train_s": t_train,
            "loss_first": float(hist[0]), "loss_last": float(hist[-1]), "params": q.params_dict(prm),
            "nrhs": nrhs, "verdict": v,
            "inner_iter_ratio": v["learned_inner"] / max(1, v["plain_inner"]),
            "time_ratio": v["learned_ms"] / v["plain_ms"],
            "fallback": "plain SAP" if not v["use_learned"] else None}


def timed(torch, fn):
    """Wall time of fn() on the device, synchronised on both sides (seconds)."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, r


def point_sources_torch(torch, dims, first, count):
    """Spin-colour point sources first..first+count-1 at the origin, complex128 on the device."""
    V = 1
    for L in dims:
        V *= L
    b = torch.zeros((count, V, 4, 3), dtype=torch.complex128, device="cuda")
    for j in range(count):
        k = first + j
        b[j, 0, k // 3, k % 3] = 1.0
    return b


def batched_section(q, qi, torch, csw, eps, tol, inner_tol, candidates):
    """Uneven instances solved one after the other and then concurrently (qcd_solve_multi):
    24^3x48 with 12 point sources and 8^3x16, 12^3x24, 16^3x32 with one Gaussian source each;
    each instance's SAP set-up autotuned on its own source (FP16 storage among the candidates)."""
    specs = [((24, 24, 24, 48), 0.120, 12), ((8, 8, 8, 16), 0.118, 1), ((12, 12, 12, 24), 0.120, 1),
             ((16, 16, 16, 32), 0.122, 1)]
    solvers, streams, bs, prms, nr, info = [], [], [], [], [], []
    for i, (dims, kappa, nrhs) in enumerate(specs):
        st = torch.cuda.Stream()
        sv = q.Solver(dims, stream=st.cuda_stream)
        Ug = qi.gauge_field(dims, eps, seed=1002 + i, device="cuda")
        torch.cuda.synchronize()  # made on torch's stream, read on the context's
        sv.load_gauge(Ug)
        del Ug
        sv.build_clover(kappa, csw)
        b = point_sources_torch(torch, dims, 0, 12) if nrhs == 12 else \
            qi.gaussian_spinor_torch(dims, 2002 + i, 1, "cuda").contiguous()
        base = q.make_params(kappa, csw, tuple(L // 2 for L in dims), tuple(L // 2 for L in dims), tol=tol,
                             inner_tol=inner_tol)
        torch.cuda.synchronize()  # inputs made on torch's stream are complete before the context's stream reads them
        best, ms = q.qcd_autotune(sv.ctx, b[:1].contiguous(), base, max_candidates=candidates)
        solvers.append(sv)
        streams.append(st)
        bs.append(b)
        prms.append(best)
        nr.append(nrhs)
        info.append({"lattice": "x".join(map(str, dims)), "kappa": kappa, "nrhs": nrhs, "params": q.params_dict(best)})
    # warm both ways once, then time
    xs = [torch.zeros_like(b) for b in bs]
    q.qcd_solve_multi([sv.ctx for sv in solvers], xs, bs, prms, nr)
    seq = []
    for sv, x, b, p, n, inf in zip(solvers, xs, bs, prms, nr, info):
        x.zero_()
        t, st = timed(torch, lambda: sv.solve(x, b, p, nrhs=n))
        seq.append(t)
        inf.update({"seconds_alone": t, "outer_iters": st["outer_iters"], "inner_iters": st["inner_iters"],
                    "true_rel_res": st["true_rel_res"]})
    for x in xs:
        x.zero_()
    t_multi, (rc, sts) = timed(torch, lambda: q.qcd_solve_multi([sv.ctx for sv in solvers], xs, bs, prms, nr))
    for inf, st in zip(info, sts):
        inf["true_rel_res_multi"] = st["true_rel_res"]
    for sv in solvers:
        sv.close()
    return {"instances": info, "seconds_sequential": sum(seq), "seconds_concurrent": t_multi,
            "speedup_concurrent": sum(seq) / t_multi,
            "note": "concurrent = qcd_solve_multi: one host thread and one stream per instance; "
                    "each instance replays its captured inner iteration"}


def ll_levels(b, s):
    """Dependent steps per SSOR pass of the ll order on a b block with s sub-blocks: the longest
    chain of in-block neighbours in increasing ll key (the level schedule the kernel runs)."""
    nq = [b[m] // s[m] for m in range(4)]
    nsb = nq[0] * nq[1] * nq[2] * nq[3]
    vol = b[0] * b[1] * b[2] * b[3]

    def coords(yl):
        y = []
        for m in range(4):
            y.append(yl % b[m])
            yl //= b[m]
        return y

    key = [0] * vol
    for yl in range(vol):
        y = coords(yl)
        lam = sig = 0
        for m in (3, 2, 1, 0):
            lam = lam * s[m] + y[m] % s[m]
            sig = sig * nq[m] + y[m] // s[m]
        key[yl] = lam * nsb + sig
    level = [0] * vol
    for yl in sorted(range(vol), key=lambda v: key[v]):
        y = coords(yl)
        lv, stride = 0, 1
        for m in range(4):
            for dd in (-1, 1):
                if 0 <= y[m] + dd < b[m]:
                    nb = yl + dd * stride
                    if key[nb] < key[yl]:
                        lv = max(lv, level[nb] + 1)
            stride *= b[m]
        level[yl] = lv
    return max(level) + 1


def geometry_section(q, qi, torch, s, w, b):
    """SAP block and sub-block geometries on the plain 12^3 x 24 solve (FP32 storage, the
    workload's omega, sweeps and cycles): time to solution, iterations, SSOR launch time."""
    geoms = [((6, 6, 6, 12), (3, 3, 3, 6)), ((6, 6, 6, 6), (3, 3, 3, 3)), ((6, 6, 6, 12), (2, 2, 2, 4)),
             ((6, 6, 6, 12), (6, 6, 6, 12)), ((6, 6, 6, 6), (2, 2, 2, 2)), ((6, 6, 6, 6), (6, 6, 6, 6)),
             ((3, 3, 3, 6), (3, 3, 3, 6)), ((3, 3, 3, 6), (1, 1, 1, 2)), ((3, 3, 3, 3), (1, 1, 1, 1)),
             ((2, 2, 2, 2), (1, 1, 1, 1))]
    out = []
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()
    for blk, sub in geoms:
        p = q.make_params(w["kappa"], w["csw"], blk, sub, omega=w["omega"], nsweep=w["nsweep"], nsap=w["nsap"],
                          tol=w["tol"], inner_tol=w["inner_tol"])
        x.zero_()
        s.solve(x, b, p)
        x.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        st = s.solve(x, b, p)
        ev[1].record(stream)
        torch.cuda.synchronize()
        q.qcd_set_profiling(s.ctx, True)
        q.qcd_kernel_stats(s.ctx, q.KERNEL_CLASSES.index("ssor"), reset=True)
        x.zero_()
        s.solve(x, b, p)
        n, ms = q.qcd_kernel_stats(s.ctx, q.KERNEL_CLASSES.index("ssor"), reset=True)
        q.qcd_set_profiling(s.ctx, False)
        out.append({"block": list(blk), "subblock": list(sub), "levels_per_pass": ll_levels(blk, sub),
                    "ms": ev[0].elapsed_time(ev[1]), "outer_iters": st["outer_iters"], "inner_iters": st["inner_iters"],
                    "ssor_ms_per_launch": ms / max(1, n), "true_rel_res": st["true_rel_res"]})
    return out


def block_solver_section(q, qi, torch, s, w, b):
    """The two block inverses of SAP at equal cost: ll-SSOR with nsweep sweeps against the even-odd
    minimal-residual solver with 2 nsweep - 1 steps (and twice that).  Cost in block-restricted D
    applications per block inverse: an SSOR sweep is 2 (forward and backward pass over every
    site), an MR step 1 (two half-lattice hops), plus 1 for the even-odd set-up and the odd sites.
    Workloads: the plain 12^3 x 24 solve, and 24^3 x 48 at kappa 0.122 with 4^4 blocks (2^4
    sub-blocks), 4 sweeps, N_SAP 4 (many more iterations)."""
    def compare(sv, bb, kappa, block, sub, nsweep, nsap):
        rows = []
        x = torch.zeros_like(bb)
        stream = torch.cuda.current_stream()
        for solver, steps in ((0, nsweep), (1, 2 * nsweep - 1), (1, 4 * nsweep - 1)):
            p = q.make_params(kappa, w["csw"], block, sub, omega=w["omega"], nsweep=steps, nsap=nsap, tol=w["tol"],
                              inner_tol=w["inner_tol"], block_solver=solver)
            x.zero_()
            sv.solve(x, bb, p)
            x.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            st = sv.solve(x, bb, p)
            ev[1].record(stream)
            torch.cuda.synchronize()
            q.qcd_set_profiling(sv.ctx, True)
            q.qcd_kernel_stats(sv.ctx, q.KERNEL_CLASSES.index("ssor"), reset=True)
            x.zero_()
            sv.solve(x, bb, p)
            n, ms = q.qcd_kernel_stats(sv.ctx, q.KERNEL_CLASSES.index("ssor"), reset=True)
            q.qcd_set_profiling(sv.ctx, False)
            rows.append({"block_solver": "ll-ssor" if solver == 0 else "even-odd mr", "steps": steps,
                         "cost_D_per_block_inverse": 2 * steps if solver == 0 else steps + 1,
                         "ms": ev[0].elapsed_time(ev[1]), "outer_iters": st["outer_iters"],
                         "inner_iters": st["inner_iters"], "block_kernel_ms_per_launch": ms / max(1, n),
                         "true_rel_res": st["true_rel_res"]})
        return rows

    out = {"12x12x12x24": compare(s, b, w["kappa"], w["block"], w["subblock"], w["nsweep"], w["nsap"])}
    dl = (24, 24, 24, 48)
    sl = q.Solver(dl)
    sl.load_gauge(qi.gauge_field(dl, w["eps"], seed=1003, device="cuda"))
    sl.build_clover(0.122, w["csw"])
    bl = qi.gaussian_spinor_torch(dl, 2003, 1, "cuda").contiguous()
    torch.cuda.synchronize()
    out["24x24x24x48_kappa0.122_4x4x4x4"] = compare(sl, bl, 0.122, (4, 4, 4, 4), (2, 2, 2, 2), 4, 4)
    sl.close()
    del bl
    torch.cuda.empty_cache()
    return out


def headline_section(q, qi, torch, w, group, candidates):
    """48^3 x 96, kappa 0.122, the 12 spin-colour point sources in right-hand-side groups of `group`:
    plain FP32 SAP (the workload's literal set-up) against the autotuned set-up."""
    dims = (48, 48, 48, 96)
    st = torch.cuda.Stream()
    sv = q.Solver(dims, stream=st.cuda_stream)
    Ug = qi.gauge_field(dims, w["eps"], seed=1004, device="cuda")
    torch.cuda.synchronize()  # made on torch's stream, read on the context's
    sv.load_gauge(Ug)
    del Ug
    torch.cuda.empty_cache()
    sv.build_clover(0.122, w["csw"])
    plain = q.make_params(0.122, w["csw"], w["block"], w["subblock"], omega=w["omega"], nsweep=w["nsweep"],
                          nsap=w["nsap"], tol=w["tol"], inner_tol=w["inner_tol"])
    g = qi.gaussian_spinor_torch(dims, 2004, 1, "cuda").contiguous()
    torch.cuda.synchronize()
    t_tune, (best, _) = timed(torch, lambda: q.qcd_autotune(sv.ctx, g, plain, max_candidates=candidates))
    del g
    out = {"lattice": "48x48x48x96", "kappa": 0.122, "sources": 12, "rhs_group": group,
           "tuning_seconds": t_tune, "chosen_params": q.params_dict(best)}
    for name, p in (("plain", plain), ("chosen", best)):
        total, iters, res = 0.0, [], 0.0
        for k0 in range(0, 12, group):
            b = point_sources_torch(torch, dims, k0, group)
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t, stt = timed(torch, lambda: sv.solve(x, b, p, nrhs=group))
            total += t
            iters.append((stt["outer_iters"], stt["inner_iters"]))
            res = max(res, stt["true_rel_res"])
            del b, x
            torch.cuda.empty_cache()
        out[name] = {"seconds": total, "seconds_per_source": total / 12, "iters_per_group": iters,
                     "true_rel_res_max": res}
    out["speedup_chosen_vs_plain"] = out["plain"]["seconds"] / out["chosen"]["seconds"]
    sv.close()
    torch.cuda.empty_cache()
    return out


def run_gpu(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1210_7398_gb300 import build as qbuild
    if not os.path.exists(qbuild.LIB):
        qbuild.build()
    import paper_1210_7398_gb300 as q
    import qcd_inputs as qi

    peaks = read_peaks()
    # all work of this run on one non-default stream: the library replays its captured inner
    # iteration only there, and torch's fills and copies stay ordered with the solves
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        return run_gpu_on_stream(args, q, qi, torch, np, peaks, rank, world, local)


def run_gpu_on_stream(args, q, qi, torch, np, peaks, rank, world, local):
    if args.only_dslash:  # profiling aid: the FP32 D on 24^3 x 48 alone
        print(json.dumps({"dslash": dslash_bandwidth(q, torch, (24, 24, 24, 48), 5, peaks)}))
        return 0
    if args.only_learned:  # profiling aid: the learned correction's three layers on 24^3 x 48
        dl = (24, 24, 24, 48)
        sl = q.Solver(dl)
        sl.load_gauge(qi.gauge_field(dl, 0.3, seed=1003, device="cuda"))
        sl.build_clover(0.122, 1.6)
        q.qcd_learned_set_weights(sl.ctx, q.learned_init_weights(4000, scale_last=1.0))
        xin = qi.gaussian_spinor_torch(dl, 2003, 1, "cuda").to(torch.complex64).contiguous()
        yout = torch.empty_like(xin)
        for _ in range(3):
            q.qcd_learned_apply(sl.ctx, yout, xin)
        q.qcd_set_profiling(sl.ctx, True)
        for k in range(len(q.KERNEL_CLASSES)):
            q.qcd_kernel_stats(sl.ctx, k, reset=True)
        for _ in range(5):
            q.qcd_learned_apply(sl.ctx, yout, xin)
        n, ms = q.qcd_kernel_stats(sl.ctx, q.KERNEL_CLASSES.index("learned"), reset=True)
        q.qcd_set_profiling(sl.ctx, False)
        sl.close()
        print(json.dumps({"learned_layers_24x24x24x48": {"launches": n, "ms": ms, "ms_per_application": ms / 5}}))
        return 0
    if args.only_ssor_forms:  # profiling aid: SAP on 24^3 x 48 with the 32-lane, then the 8-lane SSOR
        dl = (24, 24, 24, 48)
        sl = q.Solver(dl)
        sl.load_gauge(qi.gauge_field(dl, 0.3, seed=1003, device="cuda"))
        sl.build_clover(0.122, 1.6)
        prm = q.make_params(0.122, 1.6, (4, 4, 4, 4), (2, 2, 2, 2), nsweep=2, nsap=1, sap_storage=q.QCD_F16)
        xin = qi.gaussian_spinor_torch(dl, 2003, 4, "cuda").to(torch.complex64).contiguous()
        yout = torch.empty_like(xin)
        torch.cuda.synchronize()  # made on torch's stream, read on the context's
        res = {}
        for form in (1, 2):  # two SSOR launches (one per colour) per application
            q.qcd_set_sap_form(sl.ctx, form)
            q.qcd_set_profiling(sl.ctx, True)
            q.qcd_kernel_stats(sl.ctx, q.QCD_K_SSOR, reset=True)
            sl.sap_precondition(yout, xin, prm, nrhs=4)
            n, ms = q.qcd_kernel_stats(sl.ctx, q.QCD_K_SSOR, reset=True)
            q.qcd_set_profiling(sl.ctx, False)
            res["lanes_%d" % (32 if form == 1 else 8)] = {"launches": n, "ms_per_launch": ms / max(n, 1)}
        sl.close()
        print(json.dumps({"ssor_forms_24x24x24x48_4x4x4x4_f16_nrhs4": res}))
        return 0
    w = WORKLOAD
    dims = w["dims"]
    V = qi.volume(dims)
    U = qi.gauge_field(dims, w["eps"], seed=w["gauge_seed"])
    b = qi.gaussian_spinor(dims, seed=w["source_seed"])
    s = q.Solver(dims)
    s.load_gauge(torch.from_numpy(U).cuda())
    s.build_clover(w["kappa"], w["csw"])
    prm = q.make_params(w["kappa"], w["csw"], w["block"], w["subblock"], omega=w["omega"], nsweep=w["nsweep"],
                        nsap=w["nsap"], tol=w["tol"], inner_tol=w["inner_tol"])
    stream = torch.cuda.current_stream()
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        x.zero_()
        s.solve(x, bd, prm)
    torch.cuda.synchronize()

    # ---- timed region: K solves, L2 flushed between them ----
    q.qcd_set_profiling(s.ctx, True)
    for k in range(len(q.KERNEL_CLASSES)):
        q.qcd_kernel_stats(s.ctx, k, reset=True)
    launches0 = q.qcd_launch_count(s.ctx)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    step_ms, stats = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        x.zero_()
        ev_a = torch.cuda.Event(enable_timing=True)
        ev_b = torch.cuda.Event(enable_timing=True)
        ev_a.record(stream)
        st = s.solve(x, bd, prm)
        ev_b.record(stream)
        torch.cuda.synchronize()
        step_ms.append(ev_a.elapsed_time(ev_b))
        stats.append(st)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches = q.qcd_launch_count(s.ctx) - launches0
    kstats = {}
    for k, nm in enumerate(q.KERNEL_CLASSES):
        n, ms = q.qcd_kernel_stats(s.ctx, k, reset=True)
        kstats[nm] = {"launches": n, "ms": ms}
    q.qcd_set_profiling(s.ctx, False)
    ms_step = max_over_ranks(sum(step_ms) / len(step_ms), world)

    # true residual of the last solve, checked with the library's FP64 D
    xr = x.cpu().numpy()

    # ---- end to end: host buffers through the C ABI, copies inside the timed region ----
    b_host = torch.from_numpy(b).pin_memory().numpy()
    x_host = torch.zeros(b.shape, dtype=torch.complex128).pin_memory().numpy()
    e2e = []
    for _ in range(max(1, min(args.steps, 3))):
        x_host[...] = 0
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.solve(x_host, b_host, prm)
        e2e.append(time.perf_counter() - t0)
    # ---- chosen: the autotuned SAP set-up, timed like the plain one ----
    chosen = None
    if not args.skip_chosen:
        best, tune_ms = q.qcd_autotune(s.ctx, bd, prm, max_candidates=args.tune_candidates)
        for _ in range(2):
            x.zero_()
            s.solve(x, bd, best)
        torch.cuda.synchronize()
        ch_ms, ch_st = [], None
        for _ in range(args.steps):
            flush.fill_(1.0)
            x.zero_()
            ev_a = torch.cuda.Event(enable_timing=True)
            ev_b = torch.cuda.Event(enable_timing=True)
            ev_a.record(stream)
            ch_st = s.solve(x, bd, best)
            ev_b.record(stream)
            torch.cuda.synchronize()
            ch_ms.append(ev_a.elapsed_time(ev_b))
        chosen = {"value": sum(ch_ms) / len(ch_ms) / 1000.0, "unit": "s", "params": q.params_dict(best),
                  "outer_iters": ch_st["outer_iters"], "inner_iters": ch_st["inner_iters"],
                  "true_rel_res": ch_st["true_rel_res"], "speedup_vs_plain": ms_step / (sum(ch_ms) / len(ch_ms)),
                  "tuning": "qcd_autotune over block/sub-block splits, then FP16 storage, 2 CTAs per block "
                            "and (nsweep, nsap) in {2,4}^2 for the 3 fastest; best of timed full solves"}
        # 12 spin-colour point sources solved together, with the set-up tuned for that batch
        pts = torch.from_numpy(qi.point_sources(dims)).cuda()
        torch.cuda.synchronize()
        best12, _ = q.qcd_autotune(s.ctx, pts, prm, nrhs=12, max_candidates=args.tune_candidates)
        xp = torch.zeros_like(pts)
        s.solve(xp, pts, best12, nrhs=12)
        torch.cuda.synchronize()
        xp.zero_()
        ev_a = torch.cuda.Event(enable_timing=True)
        ev_b = torch.cuda.Event(enable_timing=True)
        ev_a.record(stream)
        bst = s.solve(xp, pts, best12, nrhs=12)
        ev_b.record(stream)
        torch.cuda.synchronize()
        tb = ev_a.elapsed_time(ev_b) / 1000.0
        chosen["batched_12_point_sources"] = {"seconds": tb, "seconds_per_source": tb / 12,
                                              "params": q.params_dict(best12),
                                              "outer_iters": bst["outer_iters"], "inner_iters": bst["inner_iters"],
                                              "true_rel_res_max": bst["true_rel_res"]}
        # the learned correction on top of the chosen set-up; kept only when it is faster
        lr_sec = learned_section(q, qi, torch, s, dims, best, bd, 1, 64, 8)
        chosen["learned"] = lr_sec
        if lr_sec["verdict"]["use_learned"] and lr_sec["verdict"]["learned_ms"] < chosen["value"] * 1000.0:
            chosen["value"] = lr_sec["verdict"]["learned_ms"] / 1000.0
            chosen["params"]["learned"] = 1
            chosen["speedup_vs_plain"] = ms_step / lr_sec["verdict"]["learned_ms"]
    block_solvers = None
    if not args.skip_chosen:
        block_solvers = block_solver_section(q, qi, torch, s, w, bd)
    geometry = None
    if args.geometry_sweep:
        geometry = geometry_section(q, qi, torch, s, w, bd)
    batched = None
    if args.batched_full:
        batched = batched_section(q, qi, torch, w["csw"], w["eps"], w["tol"], w["inner_tol"], 16)
    headline = None
    if args.headline:
        headline = headline_section(q, qi, torch, w, args.rhs_group, 20)
    learned_full = None
    if args.learned_full:
        # 24^3 x 48, kappa 0.122, 12 point sources, 256 training pairs, plain SAP with 4 sweeps
        dl = (24, 24, 24, 48)
        sl = q.Solver(dl)
        sl.load_gauge(qi.gauge_field(dl, w["eps"], seed=1003, device="cuda"))
        sl.build_clover(0.122, w["csw"])
        pl = q.make_params(0.122, w["csw"], (4, 4, 4, 4), (2, 2, 2, 2), nsweep=4, nsap=4, tol=w["tol"],
                           inner_tol=w["inner_tol"])
        pts = torch.from_numpy(qi.point_sources(dl)).cuda()
        learned_full = learned_section(q, qi, torch, sl, dl, pl, pts, 12, 256, 8)
        learned_full["lattice"] = "24x24x24x48"
        sl.close()
        del pts
    s.close()
    del flush
    torch.cuda.empty_cache()

    out = None
    if rank == 0:
        # dominant kernel and its roofline
        dom = max((nm for nm in kstats if kstats[nm]["launches"]), key=lambda nm: kstats[nm]["ms"])
        model = kernel_model(dom, V, 1, w, peaks)
        roof = None
        if model:
            bound, units, unit, peak = model
            avg_ms = kstats[dom]["ms"] / kstats[dom]["launches"]
            achieved = units / (avg_ms * 1e-3)
            roof = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                    "frac": achieved / peak, "traffic": NCU_TRAFFIC.get(dom), "avg_launch_ms": avg_ms,
                    "peak_source": peaks["source"] if bound == "hbm" else "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}
            sm_mhz = clk.get("sm_mhz") if isinstance(clk, dict) else None
            iss = issue_model(dom, avg_ms, sm_mhz or peaks["sm_max_mhz"])
            if iss is not None:
                roof["issue"] = iss
        tot_k = sum(v["ms"] for v in kstats.values())
        for v in kstats.values():
            v["share"] = v["ms"] / tot_k if tot_k else 0.0
        dsl = []
        if not args.skip_dslash:
            dsl += dslash_bandwidth(q, torch, (24, 24, 24, 48), 20, peaks,
                                    variants=(("f32", 1), ("f32", 12), ("f16", 1), ("f16", 12), ("su3", 1), ("su3", 12),
                                              ("f64", 1)))
            dsl += dslash_bandwidth(q, torch, (48, 48, 48, 96), 20, peaks)
        cpu = None
        if world == 1 and not args.skip_cpu:
            try:
                Uo, Fo, bo = oracle_setup()
                t, status, st_o = oracle_solve_seconds(Uo, Fo, bo)
                cpu = {"value": t, "unit": "s", "cores": cores_used(), "kind": "oracle",
                       "sample": "one full FP64 oracle solve of the same workload (outer %d, inner %d, "
                                 "true rel. residual %.1e)" % (st_o["outer"], st_o["inner"], st_o["true_rel_res"])}
            except Exception as e:  # the baseline is reported, not required
                cpu = {"value": None, "unit": "s", "cores": cores_used(), "kind": "oracle", "sample": "failed: %s" % e}
        last = stats[-1]
        out = {"metric": METRIC, "value": ms_step / 1000.0, "unit": "s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
               "config": {"workload": WORKLOAD["name"], "lattice": "12x12x12x24", "kappa": w["kappa"],
                          "csw": w["csw"], "omega": w["omega"], "nsweep": w["nsweep"], "nsap": w["nsap"],
                          "tol": w["tol"], "inner_tol": w["inner_tol"], "l2": "flushed (512 MiB write) between steps",
                          "parallelism": "replicas" if world > 1 else "single GPU"},
               "solve": {"outer_iters": last["outer_iters"], "inner_iters": last["inner_iters"],
                         "restarts": last["restarts"], "true_rel_res": last["true_rel_res"],
                         "solves_per_s_all_gpus": world / (ms_step / 1000.0), "wall_s_timed_region": wall},
               "e2e": {"value": statistics.mean(e2e), "unit": "s", "h2d_bytes_per_step": 2 * 16 * 12 * V,
                       "d2h_bytes_per_step": 16 * 12 * V,
                       "note": "qcd_solve with pinned host x and b; copies inside the call"},
               "gpu_launches": launches, "kernels": kstats, "clocks": clk, "roofline": roof,
               "dslash": dsl, "chosen": chosen, "cpu_baseline": cpu}
        if learned_full is not None:
            out["learned_24x24x24x48"] = learned_full
        if batched is not None:
            out["batched_uneven"] = batched
        if geometry is not None:
            out["geometry_sweep"] = geometry
        if block_solvers is not None:
            out["block_solvers"] = block_solvers
        if headline is not None:
            out["headline_48x48x48x96"] = headline
        print(json.dumps(out))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--skip-dslash", action="store_true", help="skip the D bandwidth measurement")
    ap.add_argument("--skip-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--skip-chosen", action="store_true", help="skip the autotuned (chosen) measurement")
    ap.add_argument("--tune-candidates", type=int, default=48, help="solves the autotuner may time")
    ap.add_argument("--batched-full", action="store_true",
                    help="also solve 24^3x48 (12 point sources) + 8^3x16, 12^3x24, 16^3x32 alone and concurrently")
    ap.add_argument("--geometry-sweep", action="store_true",
                    help="also time the plain 12^3x24 solve over SAP block / sub-block geometries")
    ap.add_argument("--headline", action="store_true",
                    help="also solve 48^3x96 with 12 point sources, plain and autotuned")
    ap.add_argument("--rhs-group", type=int, default=4, help="right-hand sides per 48^3x96 solve")
    ap.add_argument("--only-dslash", action="store_true", help="profiling aid: time only the FP32 D on 24^3x48")
    ap.add_argument("--only-ssor-forms", action="store_true",
                    help="profiling aid: one SAP application (24^3x48, 4^4 blocks, FP16, 4 RHS) with the "
                         "32-lane and then the 8-lane SSOR kernel")
    ap.add_argument("--only-learned", action="store_true",
                    help="profiling aid: time only the learned correction's layers on 24^3x48")
    ap.add_argument("--learned-full", action="store_true",
                    help="also train and assess the learned correction on 24^3 x 48 with 12 point sources")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
