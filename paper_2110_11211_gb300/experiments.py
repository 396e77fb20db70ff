"""Iteration counts of the convergence and scaling studies of Sec. 4, run on the
GPU path through the C-ABI.

Protocol (Sec. 4): the Laplacian (c = 1) with f = 0 and zero Dirichlet data,
so the solution is 0 and every iterate is its own error.  x_0 has entries drawn
from U[-1, 1]; the solvers stop once ||x_K||_A <= 1e-8 ||x_0||_A, and K is the
recorded count.  The damped Richardson iteration (Algorithm 3) uses the
optimal xi* = 2 / (lambda_min + lambda_max) of eq. (redrate), with the extreme
eigenvalues of C^{-1} A estimated from the Lanczos tridiagonal of a PCG run.
Weak scaling keeps N/P ~ 2^S: d = 1 uses the level S + log2 P, d > 1 the
isotropic levels floor((S + log2 P) / d) of Sec. 4.2.

The paper runs CG and Richardson on the diagonally rescaled system
T A T with T = diag(A)^{-1/2}; the Laplacian's diagonal is constant, so that
rescaling is a multiple of the identity and changes neither count.  The D_i
weighting of eq. (Di) coincides with the omega_i weighting for gamma = 1/2
(Lemma on the weightings), so the studies at gamma = 1/2 cover it.

E8 (Sec. 4.3, on one GPU): the combination technique on the Poisson problem
with u = ||x||_2 prod sin(pi x_i), d = 2..6, growing L, P_hat = 2^{L-8} (at least 1):
the error of the combined solution at seeded points against u, with the number
of subgrids, unknowns and PCG iterations (FP32 local factors, FP64 outer
iteration to relative residual 1e-8, as the study stops).

Usage: python -m paper_2110_11211_gb300.experiments [E1 ... E8 | all]
           [--pmax P] [--json FILE]
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import torch

from . import inputs

TOL = 1e-8
X0_SEED = 20211021
RHS_SEED = 20211022


def weak_levels(d: int, S: int, P: int) -> tuple[int, ...]:
    lg = int(round(math.log2(P)))
    if d == 1:
        return (S + lg,)
    return ((S + lg) // d,) * d


def grid_size(levels) -> int:
    return inputs.grid_size(levels)


def run_one(levels, P, gamma, q, variant="balanced", weighting="omega",
            methods=("pcg", "richardson"), spectrum_steps=500, maxit=200000):
    """Counts for one configuration, as a dict; a configuration the partition
    does not admit (q P > N, or 2 floor(gamma) + 1 >= P) is returned with a
    'skipped' reason instead."""
    from .solver import Solver
    N = grid_size(levels)
    row = dict(levels=list(levels), d=len(levels), N=N, P=P, gamma=gamma, q=q,
               variant=variant, weighting=weighting)
    if q * P > N or P > N:
        row["skipped"] = "q P > N"
        return row
    if 2 * math.floor(gamma) + 1 >= P:
        row["skipped"] = "2 floor(gamma) + 1 >= P"
        return row
    x0 = torch.tensor(inputs.uniform(X0_SEED, N), device="cuda")
    t0 = time.perf_counter()
    with Solver(levels, P, gamma, q=q, variant=variant, weighting=weighting) as s:
        if "pcg" in methods:
            _, st = s.solve_homogeneous(x0, "pcg", tol=TOL, maxit=maxit)
            row["pcg"] = st.iters
            row["pcg_energy"] = st.true_rel_res
        if "richardson" in methods:
            f = torch.tensor(inputs.uniform(RHS_SEED, N), device="cuda")
            lo, hi = s.estimate_spectrum(f, steps=spectrum_steps)
            xi = 2.0 / (lo + hi)
            _, st = s.solve_homogeneous(x0, "richardson", xi=xi, tol=TOL, maxit=maxit)
            row.update(lmin=lo, lmax=hi, xi=xi, richardson=st.iters,
                       richardson_energy=st.true_rel_res)
    row["wall_s"] = time.perf_counter() - t0
    return row


def powers(lo, hi):
    p = lo
    while p <= hi:
        yield p
        p *= 2


def configs(name: str, pmax: int):
    """(levels, P, gamma, q, variant, weighting) of each study."""
    out = []
    if name == "E1":  # Sec. 4.1: d = 1, S = 8, q = 16, gamma = 1/2, both operators
        for variant in ("additive", "balanced"):
            for weighting in ("none", "omega"):
                for P in powers(2, pmax):
                    out.append((weak_levels(1, 8, P), P, 0.5, 16, variant, weighting))
    elif name in ("E2", "E3"):  # Sec. 4.1: vary gamma, d = 1 or 3, S = 8, q = 16
        d = 1 if name == "E2" else 3
        for weighting in ("none", "omega"):
            for gamma in (0.2, 0.25, 0.5, 0.75, 1.0, 1.5, 2.0, 5.0):
                for P in powers(4, pmax):
                    out.append((weak_levels(d, 8, P), P, gamma, 16, "balanced", weighting))
    elif name == "E4":  # Sec. 4.2: vary S with q = 16 fixed, d = 1
        for S in (6, 8, 10, 12):
            for P in powers(2, pmax):
                out.append((weak_levels(1, S, P), P, 0.5, 16, "balanced", "omega"))
    elif name == "E5":  # Sec. 4.2: q = 2^{S-4}, d = 1
        for S in (6, 8, 10, 12):
            for P in powers(2, pmax):
                out.append((weak_levels(1, S, P), P, 0.5, 2 ** (S - 4), "balanced", "omega"))
    elif name == "E6":  # Sec. 4.2: d = 1..6 isotropic, S = 8, q = 2^{S-4}
        for d in range(1, 7):
            for P in powers(2, pmax):
                out.append((weak_levels(d, 8, P), P, 0.5, 16, "balanced", "omega"))
    elif name == "E7":  # Sec. 4.2: strong scaling, d = 1, q = 2^{L-12} or P-dependent
        for L in (16, 18, 20):
            N = 2 ** L - 1
            Ps = sorted({p for p in [2, 3, 4, 5, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192,
                                     256, 384, 512, 768, 1024, 1536, 2048, 4096] if p <= pmax})
            for P in Ps:
                qv = 2 ** max(int(math.floor(math.log2(N / P))) - 4, 0)
                for q in sorted({2 ** (L - 12), qv}):
                    out.append(((L,), P, 0.5, q, "balanced", "omega"))
    else:
        raise ValueError(f"unknown study {name}")
    return out


CT_LEVELS = {2: range(6, 17), 3: range(6, 14), 4: range(6, 12), 5: range(7, 11), 6: range(7, 9)}


def run_ct(d, L, npts=1 << 14):
    """One combination-technique solve of the Sec. 4.3 problem (E8)."""
    from .combination import Combination
    P_hat = max(1, 2 ** (L - 8))
    pts = torch.tensor(inputs.unit_points(44, npts, d), device="cuda")
    ue = inputs.ct_exact(pts.cpu().numpy())
    t0 = time.perf_counter()
    with Combination(d, L, P_hat, precision="fp32") as ct:
        ct.solve(rtol=1e-8, maxit=20000)
        out = ct.evaluate(pts).cpu().numpy()
        tot, per = ct.stats
        its = [p.iters for p in per]
        row = dict(study="E8", d=d, L=L, P_hat=P_hat, subgrids=len(ct.levels), N=ct.batch.N,
                   iters_max=max(its), iters_mean=float(sum(its)) / len(its),
                   failed=tot.fail_index)
    row["max_error"] = float(abs(out - ue).max())
    row["wall_s"] = time.perf_counter() - t0
    return row


def fmt(row) -> str:
    if row.get("study") == "E8":
        return (f"d={row['d']} L={row['L']} P_hat={row['P_hat']} subgrids={row['subgrids']} "
                f"N={row['N']} iters max/mean={row['iters_max']}/{row['iters_mean']:.1f} "
                f"max error={row['max_error']:.3e} ({row['wall_s']:.2f} s)")
    if "skipped" in row:
        return (f"d={row['d']} levels={row['levels']} P={row['P']} gamma={row['gamma']} "
                f"q={row['q']} {row['variant']}/{row['weighting']}: skipped ({row['skipped']})")
    return (f"d={row['d']} levels={row['levels']} N={row['N']} P={row['P']} "
            f"gamma={row['gamma']} q={row['q']} {row['variant']}/{row['weighting']}: "
            f"pcg={row.get('pcg')} richardson={row.get('richardson')} "
            f"kappa={row['lmax'] / row['lmin']:.2f} ({row['wall_s']:.2f} s)"
            if "lmin" in row else
            f"d={row['d']} levels={row['levels']} P={row['P']}: pcg={row.get('pcg')}")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("studies", nargs="*", default=["all"])
    ap.add_argument("--pmax", type=int, default=1024)
    ap.add_argument("--json", default=None, help="write the rows (after every row)")
    ap.add_argument("--budget", type=float, default=0.0,
                    help="stop starting new configurations after this many seconds")
    a = ap.parse_args(argv)
    if not torch.cuda.is_available():
        raise SystemExit("the iteration-count studies run on the GPU path: no CUDA device")
    names = ["E1", "E2", "E3", "E4", "E5", "E6", "E7", "E8"] if "all" in a.studies else a.studies
    rows = []
    t0 = time.perf_counter()
    for name in names:
        if name == "E8":
            for d, Ls in CT_LEVELS.items():
                for L in Ls:
                    if a.budget > 0 and time.perf_counter() - t0 > a.budget:
                        print("time budget reached", flush=True)
                        return rows
                    row = run_ct(d, L)
                    rows.append(row)
                    print(name, fmt(row), flush=True)
                    if a.json:
                        with open(a.json, "w") as fh:
                            json.dump(rows, fh, indent=1)
            continue
        for cfg in configs(name, a.pmax):
            if a.budget > 0 and time.perf_counter() - t0 > a.budget:
                print("time budget reached", flush=True)
                return rows
            row = run_one(*cfg)
            row["study"] = name
            rows.append(row)
            print(name, fmt(row), flush=True)
            if a.json:
                with open(a.json, "w") as fh:
                    json.dump(rows, fh, indent=1)
    return rows


if __name__ == "__main__":
    main(sys.argv[1:])
