#!/usr/bin/env python
"""Benchmark: time to relative residual 1e-10 of the two-level SFC Schwarz PCG
solve (setup + solve), on seeded synthetic inputs, through the C-ABI library.

A step is one pass of the whole path over one right-hand side: Hilbert keys,
radix sort, partition, local and coarse assembly + Cholesky, then PCG to
rtol = 1e-10 (stencil, restriction, batched substitutions, prolongation,
fused reductions).  Default workload: the 1023 x 31 x 7 anisotropic grid
(levels 10,5,3; N = 221,991), P = 128, gamma = 1, FP64 local factors.

`--impl reference` times the oracle (plain FP64 CPU implementation) on the
host cores instead, on a bounded sample of the same workload.
Multi-GPU (torchrun): every rank solves its own replica (independent problems,
no data-path collective); the time is the max over ranks.
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

from paper_2110_11211_gb300 import inputs  # noqa: E402

METRIC = "time to rel. residual 1e-10 (ms) & precond applies/s; FP64 vs mixed/batched"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="aniso3d_l10x5x3_P128", choices=list(inputs.WORKLOADS))
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "fp32", "bf16"])
    ap.add_argument("--rtol", type=float, default=1e-10)
    ap.add_argument("--no-variants", action="store_true", help="skip the FP32/BF16 comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=4, help="local subdomains the oracle factors")
    ap.add_argument("--levels", default=None, help="custom grid levels, e.g. 8,5,3 (profiling runs)")
    ap.add_argument("--shapes", default=None,
                    help="substitution shapes slabs_local,slabs_coarse instead of autotuning "
                         "(profiling runs: the timings under a profiler mislead the tuner); "
                         "write --shapes=-1,2 for whole-matrix local items")
    ap.add_argument("--P", type=int, default=None, help="custom subdomain count")
    ap.add_argument("--gamma", type=float, default=None, help="custom overlap")
    ap.add_argument("--stencil-levels", default=None,
                    help="time only the curve-order stencil on this grid (e.g. 9,9,9)")
    ap.add_argument("--ct", default=None,
                    help="time the combination technique d,L,P_hat (e.g. 4,10,4): batched "
                         "solve of the full layer set + eq. combi at 2^16 points")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


# FP64 and FP32 CUDA-core peaks from unit counts and clocks: 152 SMs x 2070 MHz
# x 2 flops per FMA x (FP64: 1.25e12 nominal GPU total; FP32: 128 lanes per SM).
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        load = [r for r in rows if (num(r[4]) or 0) >= 50] or rows
        sm = [num(r[1]) for r in load if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max((num(r[2]) or 0) for r in rows),
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(load)}


def dist_setup():
    """One process per GPU (NCCL); without a GPU the same calls run on gloo, so
    the replica logic is testable on the host."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_args(name, precision, args=None):
    w = inputs.WORKLOADS[name]
    if w["levels"] is None:
        raise SystemExit(f"{name} is a batched set, not a single-solve workload")
    out = dict(levels=w["levels"], P=w["P"], gamma=w["gamma"],
               precision=precision or w["precision"], coeffs=inputs.coefficients(name))
    if args is not None and args.levels:
        out["levels"] = tuple(int(v) for v in args.levels.split(","))
        out["coeffs"] = None
    if args is not None and args.P:
        out["P"] = args.P
    if args is not None and args.gamma:
        out["gamma"] = args.gamma
    return out


def cpu_baseline(name, wl, iters, sample):
    """The oracle as it stands, on a bounded sample of the workload, projected to
    the whole solve.  Measured in full: grid operator, curve, partition and the
    coarse FP64 Cholesky; one coarse correction, one operator apply and the PCG
    vector updates.  Measured on `sample` of the P subdomains and scaled by P:
    the local Cholesky factorization, and the oracle's own per-subdomain step of
    the preconditioner apply (index set, gather, solve, weighted scatter).  The
    iteration count is the oracle's own full run (tests/golden).
    time = setup + iters * (P * local step + coarse + operator + vectors)."""
    import numpy as np
    from oracle import schwarz
    levels, P, gamma = wl["levels"], wl["P"], wl["gamma"]
    t0 = time.perf_counter()
    S = schwarz.Schwarz(levels, P, gamma, coeffs=wl["coeffs"], cache_factors=True)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    S.coarse_factor()
    t_coarse_fac = time.perf_counter() - t0
    f = inputs.rhs(name, levels)
    idx = np.linspace(0, P - 1, sample).round().astype(int)
    t_fac = t_loc = 0.0
    h = np.zeros(S.N)
    for i in idx:
        t0 = time.perf_counter()
        S.local_factor(int(i))
        t_fac += time.perf_counter() - t0
        t0 = time.perf_counter()
        ids = S.local_ids(int(i))
        h[ids] += S.omega[int(i)] * S.local_solve(int(i), f[ids])
        t_loc += time.perf_counter() - t0
    t0 = time.perf_counter()
    z = S.coarse_correction(f)
    y = S.A @ f
    # the five vector updates of one PCG iteration (x, r, two dots, p)
    x = np.zeros(S.N)
    x += 0.5 * z
    r = f - 0.5 * y
    rz = float(r @ z)
    pq = float(z @ y)
    p = z + (rz / (pq or 1.0)) * z
    t_iter_other = time.perf_counter() - t0
    setup = t_build + t_coarse_fac + t_fac / len(idx) * P
    per_it = t_loc / len(idx) * P + t_iter_other
    total_ms = 1e3 * (setup + iters * per_it)
    measured = t_build + t_coarse_fac + t_fac + t_loc + t_iter_other
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    del y, p, x
    return {"value": round(total_ms, 1), "unit": "ms", "cores": cores, "kind": "oracle",
            "estimate": "projection from a measured sample (not a full oracle run)",
            "sample": (f"measured in full: operator, curve, partition, coarse FP64 Cholesky, one "
                       f"coarse correction + operator + vector updates; measured on {len(idx)} of "
                       f"{P} subdomains and scaled to {P}: local Cholesky and the apply's "
                       f"per-subdomain step; {iters} iterations (the oracle's own count)"),
            "measured_s": round(measured, 2),
            "measured_fraction": round(measured / (total_ms / 1e3), 6)}


def cpu_full_solve(name="poisson2d_l6x6_P8", rtol=1e-10):
    """A complete oracle run, nothing projected: setup and PCG to rtol on the
    small 63 x 63 workload (P = 8), wall clock on the host cores."""
    from oracle import krylov, schwarz
    w = inputs.WORKLOADS[name]
    t0 = time.perf_counter()
    S = schwarz.Schwarz(w["levels"], w["P"], w["gamma"], coeffs=inputs.coefficients(name))
    for i in range(S.P):
        S.local_factor(i)
    S.coarse_factor()
    t1 = time.perf_counter()
    f = inputs.rhs(name)
    _, its, hist = krylov.pcg(lambda v: S.A @ v, S.apply, f, rtol=rtol)
    t2 = time.perf_counter()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"workload": name, "ms": round(1e3 * (t2 - t0), 2), "setup_ms": round(1e3 * (t1 - t0), 2),
            "solve_ms": round(1e3 * (t2 - t1), 2), "iters": its, "rel_res": hist[-1],
            "cores": cores, "kind": "oracle (complete run, not projected)"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload_args(args.workload, args.precision)
    # the oracle's own PCG iteration count for this workload (full oracle run,
    # written by tests/golden/make_oracle_pcg.py)
    gpath = os.path.join(ROOT, "tests", "golden", f"oracle_pcg_{args.workload}.json")
    if not os.path.exists(gpath):
        print(json.dumps({"impl": "reference", "unavailable":
                          f"no oracle iteration count stored for {args.workload}"}), flush=True)
        return
    with open(gpath) as fh:
        iters = int(json.load(fh)["iters"])
    from oracle import partition
    q_ref = int(partition.paper_q(inputs.grid_size(wl["levels"]), wl["P"]))
    vals, meas = [], []
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(args.workload, wl, iters, max(1, min(args.cpu_sample, 2)))
        if k >= args.warmup:
            vals.append(cb["value"])
            meas.append(cb["measured_s"])
    v = statistics.mean(vals)
    cb["value"] = round(v, 1)
    cb["measured_s"] = round(statistics.mean(meas), 2)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(v, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "step": ("one projection of the whole solve from a measured sample (the oracle "
                     "needs about 3000 s for the full solve); value = mean over the steps"),
            "config": {"workload": args.workload, "levels": list(wl["levels"]),
                       "N": inputs.grid_size(wl["levels"]), "P": wl["P"],
                       "gamma": wl["gamma"], "q": q_ref, "N0": q_ref * wl["P"], "precision": "fp64",
                       "rtol": args.rtol},
            "cpu_baseline": cb,
            "cpu_full_solve": cpu_full_solve(),
            "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# source files whose kernels make up each class with a committed DRAM record
TRAFFIC_SOURCES = {
    "trsv_fwd": ["trsv.cu"],
    "trsv_bwd": ["trsv.cu"],
    "coarse_factor": ["factor.cu", "oz_tile.cuh"],
}


def traffic_sources_sha(kernel):
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2110_11211_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(kernel, workload, precision, shapes=None):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu
    record, or None when there is none for this workload, precision and
    substitution shapes, or the kernels' source changed since the counters were
    taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh).get(kernel)
        sha = traffic_sources_sha(kernel) if kernel in TRAFFIC_SOURCES else None
    except (OSError, ValueError):
        return None
    if not rec or sha is None or rec.get("workload") != workload or rec.get("precision") != precision:
        return None
    if "substitution_slabs" in rec and shapes is not None and rec["substitution_slabs"] != shapes:
        return None
    if rec.get("kernel_source_sha256") != sha:
        return None
    return rec["dram_bytes_per_launch"]


def measure_fp64_rate(stream):
    """The library's in-register FMA probe: the measured FP64 ceiling."""
    import ctypes as C
    from paper_2110_11211_gb300 import _lib
    tf, ms = C.c_double(), C.c_double()
    rc = _lib.lib().sfcdd_measure_fp64_rate(5, C.byref(tf), C.byref(ms),
                                              C.c_void_p(stream.cuda_stream))
    _lib.check("sfcdd_measure_fp64_rate", rc)
    return {"tflops": round(tf.value, 4), "ms_per_launch": round(ms.value, 3),
            "how": "sfcdd_measure_fp64_rate: 8 independent FMA chains per thread, 4 CTAs per SM"}


def oracle_iters(name, fallback):
    """The oracle's own PCG iteration count for the workload (tests/golden, a
    complete oracle run), else the GPU's."""
    gpath = os.path.join(ROOT, "tests", "golden", f"oracle_pcg_{name}.json")
    if os.path.exists(gpath):
        with open(gpath) as fh:
            return int(json.load(fh)["iters"])
    return int(round(fallback))


def gpu_small_solve(name, stream, reps=5):
    """GPU setup + solve of a small workload (CUDA events, mean of reps after one warm-up)."""
    import torch
    from paper_2110_11211_gb300.solver import Solver
    w = inputs.WORKLOADS[name]
    f = torch.tensor(inputs.rhs(name), device="cuda")
    times = []
    for k in range(reps + 1):
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a0.record(stream)
        with Solver(w["levels"], w["P"], w["gamma"]) as s:
            s.solve(f, rtol=1e-10)
        a1.record(stream)
        torch.cuda.synchronize()
        if k:
            times.append(a0.elapsed_time(a1))
    return round(statistics.mean(times), 3)


def single_variant(levels, P, gamma, prec, coeffs, f, u_ref, rtol, stream, steps=3, variant="additive",
                   hbm_peak=None, tensor_cores=-1):
    """Tuned shapes, then `steps` timed setup + solve passes (CUDA events, after one
    warm-up) and one profiled pass for the substitution rates."""
    import torch
    from paper_2110_11211_gb300.solver import Solver
    with Solver(levels, P, gamma, precision=prec, coeffs=coeffs, variant=variant,
                tensor_cores=tensor_cores) as s:
        vt = s.autotune(reps=3)
    shapes = dict(slabs_local=vt["slabs_local"], slabs_coarse=vt["slabs_coarse"],
                  tensor_cores=tensor_cores)
    times = []
    for k in range(steps + 1):
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        s = Solver(levels, P, gamma, precision=prec, coeffs=coeffs, variant=variant, **shapes)
        u, st = s.solve(f, rtol=rtol)
        s.close()
        a1.record(stream)
        torch.cuda.synchronize()
        if k >= 1:
            times.append(a0.elapsed_time(a1))
    out = {"ms": round(statistics.mean(times), 2), "iters": st.iters,
           "setup_ms": round(st.setup_ms, 2), "solve_ms": round(st.solve_ms, 2),
           "applies_per_s": round(st.iters / (st.solve_ms / 1e3), 1),
           "true_rel_res": st.true_rel_res, "substitution_slabs": shapes}
    if u_ref is not None:
        out["rel_err_vs_exact"] = float(torch.linalg.norm(u - u_ref) / torch.linalg.norm(u_ref))
    s = Solver(levels, P, gamma, precision=prec, coeffs=coeffs, variant=variant, profile=True,
               **shapes)
    s.solve(f, rtol=rtol)
    ks = s.kernel_stats()
    for k in ("trsv_fwd", "trsv_bwd"):
        ms, n = ks[k]
        if n:
            gbs = s.kernel_work(k) / (ms / n * 1e-3) / 1e9
            out[k] = {"us_per_launch": round(1e3 * ms / n, 2), "GB/s": round(gbs, 1)}
            if hbm_peak:
                out[k]["frac_hbm"] = round(gbs / hbm_peak, 4)
    out["factor_bytes"] = s.get_info().factor_bytes
    s.close()
    return u, out


def aniso6d_variants(stream, hbm_peak, rtol=1e-10):
    """The d = 6 workload (31 x 15 x 7 x 7 x 3 x 3, P = 256, gamma = 1/4, f ~ N(0,1)):
    local factors in FP64, FP32 and BF16; error against the exact solution."""
    import torch
    from oracle import exact
    name = "aniso6d_l5x4x3x3x2x2_P256"
    w = inputs.WORKLOADS[name]
    f_np = inputs.rhs(name)
    u_ref = torch.tensor(exact.solve_sine(w["levels"], f_np), device="cuda")
    f = torch.tensor(f_np, device="cuda")
    out = {}
    for prec in ("fp64", "fp32", "bf16"):
        _, out[prec] = single_variant(w["levels"], w["P"], w["gamma"], prec, None, f, u_ref, rtol,
                                      stream, hbm_peak=hbm_peak)
    # the FP32-accurate factorization rounded to bf16 afterwards, for comparison
    # with the BF16 factorization (bf16 tensor-core operands) above
    _, out["bf16_fp32_factorization"] = single_variant(
        w["levels"], w["P"], w["gamma"], "bf16", None, f, u_ref, rtol, stream, hbm_peak=hbm_peak,
        tensor_cores=2)
    out["iteration_penalty"] = {p: out[p]["iters"] - out["fp64"]["iters"] for p in ("fp32", "bf16")}
    out["speedup_vs_fp64"] = {p: round(out["fp64"]["ms"] / out[p]["ms"], 3) for p in ("fp32", "bf16")}
    return out


def combi4d_batch(stream, rtol=1e-10, steps=3):
    """The batched combination set: all 385 d = 4 subgrids with |l|_1 in {12, 13},
    P = 64 each, gamma = 1/2, one setup and one CUDA-graph launch (conditional
    while node) for all of them; FP32 and FP64 local factors with autotuned
    shapes, against a loop of single-problem FP64 setups and solves."""
    import torch
    from paper_2110_11211_gb300.solver import BatchSolver, Solver
    name = "combi4d_l12-13_P64"
    w = inputs.WORKLOADS[name]
    levels = inputs.combi_levels(4, (12, 13))
    P, gamma = w["P"], w["gamma"]
    ntot = sum(inputs.grid_size(lv) for lv in levels)
    f = torch.tensor(inputs.uniform(inputs.workload_seed(name), ntot), device="cuda")
    res = {"subgrids": len(levels), "N_total": ntot, "P": P, "gamma": gamma, "rtol": rtol}
    sols = {}
    for prec in ("fp32", "fp64"):
        with BatchSolver(levels, P, gamma, precision=prec) as b:
            tuning = b.autotune(reps=3)
        shapes = dict(slabs_local=tuning["slabs_local"], slabs_coarse=tuning["slabs_coarse"])
        times, st = [], None
        for k in range(steps + 1):
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            b = BatchSolver(levels, P, gamma, precision=prec, **shapes)
            u, tot, per = b.solve(f, rtol=rtol)
            b.close()
            a1.record(stream)
            torch.cuda.synchronize()
            if k >= 1:
                times.append(a0.elapsed_time(a1))
        it = [p.iters for p in per]
        sols[prec] = u
        res[f"batched_{prec}"] = {
            "ms": round(statistics.mean(times), 2), "setup_ms": round(tot.setup_ms, 2),
            "solve_ms": round(tot.solve_ms, 2),
            "iters": {"min": int(min(it)), "max": int(max(it)), "sum": int(sum(it))},
            "worst_true_rel_res": max(p.true_rel_res for p in per),
            "substitution_slabs": shapes}
    offs = [0]
    for lv in levels:
        offs.append(offs[-1] + inputs.grid_size(lv))
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    loop_it = 0
    for k, lv in enumerate(levels):
        s = Solver(lv, P, gamma)
        _, st = s.solve(f[offs[k]:offs[k + 1]], rtol=rtol)
        loop_it += st.iters
        s.close()
    t1.record(stream)
    torch.cuda.synchronize()
    res["looped_fp64"] = {"ms": round(t0.elapsed_time(t1), 2), "iters_sum": loop_it,
                          "mode": "one setup + solve per subgrid, 385 handles in a loop"}
    res["speedup_batched_fp32_vs_looped_fp64"] = round(res["looped_fp64"]["ms"] /
                                                       res["batched_fp32"]["ms"], 2)
    res["speedup_batched_fp32_vs_batched_fp64"] = round(res["batched_fp64"]["ms"] /
                                                        res["batched_fp32"]["ms"], 3)
    res["max_rel_diff_fp32_vs_fp64"] = float(torch.linalg.norm(sols["fp32"] - sols["fp64"]) /
                                             torch.linalg.norm(sols["fp64"]))
    return res


def run_ours(args):
    import numpy as np
    import torch
    from paper_2110_11211_gb300.solver import Solver

    world, rank, local = dist_setup()
    wl = workload_args(args.workload, args.precision, args)
    levels, P, gamma, prec, coeffs = wl["levels"], wl["P"], wl["gamma"], wl["precision"], wl["coeffs"]
    f_np = inputs.rhs(args.workload, levels)
    N = f_np.size
    f = torch.tensor(f_np, device="cuda")
    stream = torch.cuda.current_stream()

    # substitution tile shapes: tuned once (sfcdd_autotune) before the warm-up,
    # then passed to every step's setup like any other option
    if args.shapes:
        sl, sc = (int(v) for v in args.shapes.split(","))
        shapes = dict(slabs_local=sl, slabs_coarse=sc)
    else:
        with Solver(levels, P, gamma, precision=prec, coeffs=coeffs) as s:
            tuning = s.autotune(reps=5)
        shapes = dict(slabs_local=tuning["slabs_local"], slabs_coarse=tuning["slabs_coarse"])

    def step(profile):
        s = Solver(levels, P, gamma, precision=prec, coeffs=coeffs, profile=profile, **shapes)
        u, st = s.solve(f, rtol=args.rtol)
        ks = s.kernel_stats()
        work = {k: s.kernel_work(k) for k in ("trsv_fwd", "trsv_bwd", "stencil", "potrf", "trsm",
                                              "syrk", "coarse_factor")}
        info = s.get_info()
        s.close()
        return u, st, ks, work, info

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    barrier(world)
    clocks = Clocks(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    iters, setup_ms, solve_ms = [], [], []
    nlaunch = 0
    for _ in range(args.steps):
        u, st, ks, work, info = step(False)
        iters.append(st.iters)
        setup_ms.append(st.setup_ms)
        solve_ms.append(st.solve_ms)
        nlaunch += sum(n for (_, n) in ks.values())
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms_step = e0.elapsed_time(e1) / args.steps
    ms_step = max_over_ranks(world, ms_step)
    u64 = u.detach()

    # profiled region: the same steps with a CUDA event pair around every launch
    # (eager launches instead of the iteration graph), for the per-class device
    # times and the roofline; kept out of the timed region above
    prof_steps = max(1, min(2, args.steps))
    agg = {}
    for _ in range(prof_steps):
        _, _, ks, work, _ = step(True)
        for k, (ms, n) in ks.items():
            a = agg.setdefault(k, [0.0, 0])
            a[0] += ms
            a[1] += n

    # end to end through the public C-ABI with host buffers (pinned), same metric
    f_pin = torch.tensor(f_np).pin_memory()
    e2e_ms = []
    for k in range(1 + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = Solver(levels, P, gamma, precision=prec, coeffs=coeffs, **shapes)
        uh, st_h = s.solve_host(f_pin.numpy(), rtol=args.rtol)
        s.close()
        t1 = time.perf_counter()
        if k >= 1:
            e2e_ms.append(1e3 * (t1 - t0))
    e2e = max_over_ranks(world, statistics.mean(e2e_ms))

    # mixed-precision variants of the same workload, and the balanced operator
    variants = {}
    bal_shapes = {}
    if not args.no_variants and rank == 0:
        for vp, var in (("fp32", "additive"), ("bf16", "additive"), (prec, "balanced")):
            if vp == prec and var == "additive":
                continue
            # each variant with its own tuned substitution shapes, like the main arm
            with Solver(levels, P, gamma, precision=vp, coeffs=coeffs, variant=var) as s:
                vt = s.autotune(reps=3)
            vshapes = dict(slabs_local=vt["slabs_local"], slabs_coarse=vt["slabs_coarse"])
            if var == "balanced":
                bal_shapes = vshapes
            times = []
            for k in range(3):
                torch.cuda.synchronize()
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                s = Solver(levels, P, gamma, precision=vp, coeffs=coeffs, variant=var, **vshapes)
                uv, stv = s.solve(f, rtol=args.rtol)
                s.close()
                a1.record(stream)
                torch.cuda.synchronize()
                if k >= 1:
                    times.append(a0.elapsed_time(a1))
            err = float(torch.linalg.norm(uv - u64) / torch.linalg.norm(u64))
            key = vp if var == "additive" else f"{var}_{vp}"
            variants[key] = {"ms": round(statistics.mean(times), 2), "iters": stv.iters,
                            "setup_ms": round(stv.setup_ms, 2), "solve_ms": round(stv.solve_ms, 2),
                            "applies_per_s": round(stv.iters / (stv.solve_ms / 1e3), 1),
                            "rel_diff_vs_fp64_solution": err, "true_rel_res": stv.true_rel_res,
                            "substitution_slabs": vshapes}

    # Algorithm 3 with the balanced operator, damping from the Lanczos estimate
    if not args.no_variants and rank == 0:
        s = Solver(levels, P, gamma, precision=prec, coeffs=coeffs, variant="balanced", **bal_shapes)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        lo, hi = s.estimate_spectrum(f, steps=200)
        xi = 2.0 / (lo + hi)
        ur, str_ = s.richardson(f, xi, rtol=args.rtol, maxit=100000, check_status=False)
        a1.record(stream)
        torch.cuda.synchronize()
        s.close()
        variants[f"richardson_balanced_{prec}"] = {
            "ms": round(a0.elapsed_time(a1), 2), "iters": str_.iters, "lambda_min": lo,
            "lambda_max": hi, "xi": xi, "status": str_.status,
            "true_rel_res": str_.true_rel_res,
            "rel_diff_vs_pcg_solution": float(torch.linalg.norm(ur - u64) / torch.linalg.norm(u64))}

    # the combination technique around the batched solver (eq. combi, Sec. 4.3 problem)
    if not args.no_variants and rank == 0:
        variants["combination_d4_L10_Phat4_fp32"] = ct_measure(4, 10, 4, "fp32", 2)
    # the other workloads of the metric: d = 6 in FP64 / FP32 / BF16, and the
    # 385-subgrid batch (one graph, FP32 and FP64 factors) against a loop
    hbm_peak0 = load_peaks()[0]
    if not args.no_variants and rank == 0 and not args.levels:
        variants["aniso6d_l5x4x3x3x2x2_P256"] = aniso6d_variants(stream, hbm_peak0, args.rtol)
        variants["combi4d_l12-13_P64"] = combi4d_batch(stream, args.rtol)

    hbm_peak, bf16_peak, peak_src = load_peaks()
    fp64_probe = measure_fp64_rate(stream) if rank == 0 else None
    kernels = {}
    for k, (ms, n) in agg.items():
        if n == 0:
            continue
        kernels[k] = {"ms_per_step": round(ms / prof_steps, 3), "launches_per_step": n / prof_steps}
    timed = {k: v for k, v in agg.items() if v[0] > 0}
    d = len(levels)
    # roofline of the per-iteration dominant kernel: one launch of k_trsv
    # (backward sweep over every local matrix and the coarse matrix) per PCG
    # iteration.  FP64 factors: one FMA per 8-byte element = 0.25 FMA/B, which
    # needs 1.7 T FMA/s at full HBM rate; GB300 has 0.63 -> FP64-ALU bound.
    # FP32 / BF16 factors: HBM bound.
    dom = "trsv_bwd"
    dom_ms, dom_n = timed[dom]
    if prec == "fp64":
        per_launch = 2.0 * work[dom] / 8.0
        achieved = per_launch / (dom_ms / dom_n * 1e-3) / 1e12
        roof = {"bound": "alu", "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "peak_source": "nominal (unit counts x clock)",
                "peak_measured_probe": fp64_probe,
                "frac_of_probe": (round(achieved / fp64_probe["tflops"], 4)
                                  if fp64_probe else None)}
    else:
        per_launch = work[dom]
        achieved = per_launch / (dom_ms / dom_n * 1e-3) / 1e9
        roof = {"bound": "hbm", "peak": hbm_peak, "unit": "GB/s", "peak_source": peak_src}
    roof.update({"kernel": "k_trsv backward (class trsv_bwd: one launch per iteration)",
                 "achieved": round(achieved, 3), "frac": round(achieved / roof["peak"], 4),
                 "traffic": recorded_traffic(dom, args.workload if not args.levels else "custom",
                                             prec, shapes),
                 "algorithmic_bytes_per_launch": work[dom],
                 "work_per_launch": per_launch, "avg_launch_ms": round(dom_ms / dom_n, 4),
                 "timing": (f"CUDA events on the launching stream around every launch over "
                            f"{prof_steps} profiled steps")})
    # setup: the coarse factorization (one matrix, a chain of tile steps on a
    # side stream) and the local factorization classes, against the FP64 peak
    setup_roof = {}
    if "coarse_factor" in timed and work.get("coarse_factor"):
        ms, n = timed["coarse_factor"]
        tf = work["coarse_factor"] / (ms / prof_steps * 1e-3) / 1e12
        setup_roof["coarse_factor"] = {
            "TFLOPs": round(tf, 3), "ms_per_step": round(ms / prof_steps, 3),
            "flop_per_step": work["coarse_factor"], "frac_fp64_nominal": round(tf / FP64_PEAK_TFLOPS, 4),
            "note": "128-step chain of diagonal-tile factorizations on a side stream"}
    # the local factorization's classes together: the diagonal-tile
    # factorizations run inside the trailing-update launches (potrf launches
    # only the first tile), so only the sum of the three classes is meaningful
    lk = [k for k in ("potrf", "trsm", "syrk") if k in timed]
    if lk:
        ms = sum(timed[k][0] for k in lk) / prof_steps
        fl = sum(work.get(k, 0.0) for k in lk)
        tf = fl / (ms * 1e-3) / 1e12
        setup_roof["local_factor"] = {"TFLOPs": round(tf, 3), "ms_per_step": round(ms, 3),
                                      "flop_per_step": fl,
                                      "frac_fp64_nominal" if prec == "fp64" else "frac_fp32_nominal":
                                          round(tf / (FP64_PEAK_TFLOPS if prec == "fp64"
                                                      else FP32_PEAK_TFLOPS), 4)}
    # substitution and stencil rates (the per-iteration kernels)
    trsv = {}
    for k in ("trsv_fwd", "trsv_bwd"):
        if k in timed:
            ms, n = timed[k]
            gbs = work[k] / (ms / n * 1e-3) / 1e9
            trsv[k] = {"GB/s": round(gbs, 1), "frac_hbm": round(gbs / hbm_peak, 4),
                       "bytes_per_launch": work[k], "avg_launch_ms": round(ms / n, 4),
                       "traffic": recorded_traffic(k, args.workload if not args.levels else "custom",
                                                   prec, shapes)}
            if prec == "fp64":
                tf = 2.0 * work[k] / 8.0 / (ms / n * 1e-3) / 1e12
                trsv[k].update({"fp64_TFLOPs": round(tf, 3), "frac_fp64": round(tf / FP64_PEAK_TFLOPS, 4)})
    if "stencil" in timed:
        ms, n = timed["stencil"]
        tf = (1 + 3 * d) * N / (ms / n * 1e-3) / 1e12
        trsv["stencil"] = {"GB/s_algorithmic": round(work["stencil"] / (ms / n * 1e-3) / 1e9, 1),
                           "fp64_TFLOPs": round(tf, 3), "frac_fp64": round(tf / FP64_PEAK_TFLOPS, 4),
                           "avg_launch_ms": round(ms / n, 4)}
    if "pcg_vector" in timed:
        # the whole vector phase of an iteration is one cooperative launch
        ms, n = timed["pcg_vector"]
        trsv["vector_phase_us_per_iteration"] = round(ms / n * 1e3, 2)
    else:
        vec_us = sum(timed[k][0] / timed[k][1] * 1e3
                     for k in ("stencil", "update", "restrict", "prolong") if k in timed)
        trsv["vector_phase_us_per_iteration"] = round(vec_us, 2)
    launches = nlaunch / args.steps
    it = statistics.mean(iters)
    sol = statistics.mean(solve_ms)
    line = {
        "metric": METRIC, "value": round(ms_step, 2), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 2),
        "profiled_steps": prof_steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32+f64", "bf16": "bf16+f32+f64"}[prec],
        "data": "synthetic",
        "config": {"workload": args.workload if not args.levels else "custom",
                   "levels": list(levels), "N": N, "P": P,
                   "gamma": gamma, "q": int(info.q), "N0": int(info.N0), "precision": prec,
                   "rtol": args.rtol, "rhs": inputs.WORKLOADS[args.workload]["rhs"],
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "substitution_slabs": shapes,
                   "l2": (f"working set > L2: {info.factor_bytes / 1e9:.1f} GB of factors "
                          "re-streamed every apply; every step re-assembles and re-factors")},
        "iters": it, "setup_ms": round(statistics.mean(setup_ms), 2), "solve_ms": round(sol, 2),
        "applies_per_s": round(it / (sol / 1e3), 1),
        "clocks": clk,
        "e2e": {"value": round(e2e, 2), "unit": "ms", "h2d_bytes_per_step": 8 * N,
                "d2h_bytes_per_step": 8 * N},
        "gpu_launches": int(round(launches)),
        "roofline": roof,
        "setup_roofline": setup_roof,
        "kernels": kernels,
        "hot_loop": trsv,
        "variants": variants,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, wl, oracle_iters(args.workload, it),
                                            args.cpu_sample)
        full = cpu_full_solve()
        full["gpu_ms_same_workload"] = gpu_small_solve(full["workload"], stream)
        line["cpu_full_solve"] = full
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_stencil(args):
    """The matrix-free stencil alone, y = A x in curve order, on a grid whose
    vectors exceed L2; algorithmic bytes 16 N per launch (read x, write y)."""
    import torch
    from paper_2110_11211_gb300.solver import Solver
    torch.cuda.set_device(0)
    levels = tuple(int(v) for v in args.stencil_levels.split(","))
    s = Solver(levels, 64, 0.5, variant="coarse_only", q=1)
    N = s.N
    x = torch.tensor(inputs.uniform(1, N), device="cuda")
    for _ in range(max(args.warmup, 3)):
        s.apply_operator(x, curve_order=True)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.apply_operator(x, curve_order=True)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    hbm, _, src = load_peaks()
    gbs = 16.0 * N / (ms * 1e-3) / 1e9
    # 1 + 3 d FP64 flops per 16 bytes: above GB300's FP64/HBM balance (1.25 TF /
    # 6.8 TB/s = 0.18 flop/B), so the FP64 ALU is the roofline
    tf = (1 + 3 * len(levels)) * N / (ms * 1e-3) / 1e12
    print(json.dumps({"kernel": "stencil", "levels": list(levels), "N": N,
                      "vector_bytes": 8 * N, "ms_per_launch": round(ms, 4),
                      "roofline": {"bound": "alu", "achieved": round(tf, 3),
                                   "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                   "frac": round(tf / FP64_PEAK_TFLOPS, 4),
                                   "peak_source": "nominal (unit counts x clock)"},
                      "algorithmic_GBps": round(gbs, 1), "frac_hbm": round(gbs / hbm, 4),
                      "peak_source": src}), flush=True)
    s.close()


def ct_measure(d, L, P_hat, prec, steps, rtol=1e-8, npts=1 << 16):
    """Combination technique on the Sec. 4.3 Poisson test problem: batched setup
    and one-graph solve of every subgrid of the full layer set (eq. Pchoice
    subdomain counts), then eq. combi at npts seeded points; error against the
    closed-form solution.  Times are CUDA-event device times (mean of `steps`)."""
    import numpy as np
    import torch
    from paper_2110_11211_gb300.combination import Combination
    stream = torch.cuda.current_stream()
    pts = torch.tensor(inputs.unit_points(44, npts, d), device="cuda")
    ue = inputs.ct_exact(pts.cpu().numpy())
    rows = []
    for k in range(steps + 1):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        ct = Combination(d, L, P_hat, precision=prec)
        ev[1].record(stream)
        ct.solve(rtol=rtol)
        ev[2].record(stream)
        out = ct.evaluate(pts)
        ev[3].record(stream)
        torch.cuda.synchronize()
        tot, per = ct.stats
        it = [p.iters for p in per]
        nsub, ntot = len(ct.levels), ct.batch.N
        dev_setup = ct.batch.info()["setup_ms"]
        corners = sum(2 ** sum(1 for l in lv if l > 1) for lv in ct.levels)
        ct.close()
        if k == 0:
            continue  # first pass warms the library and the allocator
        rows.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]),
                     ev[2].elapsed_time(ev[3]), dev_setup])
    m = np.mean(np.array(rows), axis=0)
    err = float(np.abs(out.cpu().numpy() - ue).max())
    return {"d": d, "L": L, "P_hat": P_hat, "precision": prec, "subgrids": nsub,
            "N_total": ntot, "rtol": rtol, "setup_ms": round(float(m[3]), 2),
            "construct_ms": round(float(m[0]), 2),
            "solve_ms": round(float(m[1]), 2), "combine_ms": round(float(m[2]), 3),
            "points": npts, "interior_corner_loads_per_point_max": corners,
            "iters": {"min": int(min(it)), "max": int(max(it)),
                      "mean": round(float(np.mean(it)), 2)},
            "max_abs_error_vs_exact": err,
            "timing": "CUDA events, mean of %d; setup_ms is the library's device time, "
                      "construct_ms adds the host evaluation of f on every subgrid" % steps}


def run_ct_bench(args):
    import torch
    torch.cuda.set_device(0)
    d, L, P_hat = (int(v) for v in args.ct.split(","))
    prec = args.precision or "fp32"
    r = ct_measure(d, L, P_hat, prec, max(args.steps, 1))
    print(json.dumps({"metric": "combination technique: setup + solve + combine (ms)",
                      "value": round(r["construct_ms"] + r["solve_ms"] + r["combine_ms"], 2),
                      "unit": "ms", "higher_is_better": False, "data": "synthetic",
                      "config": {"workload": f"combination_d{d}_L{L}_Phat{P_hat}"}, **r}),
          flush=True)


def run_batch_bench(args):
    """Combination-technique set (all d = 4 level vectors with |l|_1 in {12, 13},
    385 subgrids, P = 64 each, gamma = 1/2): batched setup + one-graph solve of
    every subgrid to rtol, against a loop of single-problem setups and solves."""
    import torch
    from paper_2110_11211_gb300.solver import BatchSolver, Solver
    torch.cuda.set_device(0)
    w = inputs.WORKLOADS[args.workload]
    prec = args.precision or w["precision"]
    levels = inputs.combi_levels(4, (12, 13))
    P, gamma = w["P"], w["gamma"]
    ntot = sum(inputs.grid_size(lv) for lv in levels)
    f = torch.tensor(inputs.uniform(inputs.workload_seed(args.workload), ntot), device="cuda")
    stream = torch.cuda.current_stream()

    with BatchSolver(levels, P, gamma, precision=prec) as b:
        tuning = b.autotune(reps=3)
    shapes = dict(slabs_local=tuning["slabs_local"], slabs_coarse=tuning["slabs_coarse"])

    def step():
        b = BatchSolver(levels, P, gamma, precision=prec, **shapes)
        u, tot, per = b.solve(f, rtol=args.rtol)
        info = b.info()
        b.close()
        return u, tot, per, info

    for _ in range(max(args.warmup, 3)):
        step()
    clocks = Clocks(0)
    clocks.start()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    setups, solves, iters = [], [], []
    for _ in range(args.steps):
        u, tot, per, info = step()
        setups.append(tot.setup_ms)
        solves.append(tot.solve_ms)
        iters.append([p.iters for p in per])
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # loop over single-problem handles (same method, one subgrid at a time)
    offs = [0]
    for lv in levels:
        offs.append(offs[-1] + inputs.grid_size(lv))
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k, lv in enumerate(levels):
        s = Solver(lv, P, gamma, precision=prec)
        s.solve(f[offs[k]:offs[k + 1]], rtol=args.rtol)
        s.close()
    t1.record(stream)
    torch.cuda.synchronize()
    looped = t0.elapsed_time(t1)
    it = np.array(iters[-1])
    hbm, _, src = load_peaks()
    print(json.dumps({
        "metric": METRIC, "value": round(ms, 2), "unit": "ms", "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 2),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32+f64", "bf16": "bf16+f32+f64"}[prec],
        "data": "synthetic",
        "config": {"workload": args.workload, "subgrids": len(levels), "N_total": ntot, "P": P,
                   "gamma": gamma, "precision": prec, "rtol": args.rtol,
                   "mode": "batched setup + one CUDA-graph launch (conditional while node)",
                   "substitution_slabs": shapes},
        "setup_ms": round(statistics.mean(setups), 2), "solve_ms": round(statistics.mean(solves), 2),
        "iters": {"min": int(it.min()), "max": int(it.max()), "mean": round(float(it.mean()), 2)},
        "factor_bytes": info["factor_bytes"],
        "looped_ms": round(looped, 2), "speedup_vs_looped": round(looped / ms, 2),
        "clocks": clk}), flush=True)


def main():
    args = parse()
    if args.workload == "combi4d_l12-13_P64" and args.impl == "ours":
        import numpy as np  # noqa: F401
        globals()["np"] = np
        run_batch_bench(args)
        return
    if args.stencil_levels:
        run_stencil(args)
        return
    if args.ct and args.impl == "ours":
        run_ct_bench(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
