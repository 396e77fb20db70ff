"""Writes the oracle's PCG iteration count and residual history endpoints for
the benchmarked workloads (calls only oracle/ and the seeded input generator).

    python tests/golden/make_oracle_pcg.py aniso3d_l10x5x3_P128

Output: tests/golden/oracle_pcg_<workload>.json with the additive, omega-weighted
two-level Schwarz PCG (x_0 = 0, stop at ||r|| <= 1e-10 ||f||) on the seeded
right-hand side of the workload.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import krylov, schwarz  # noqa: E402
from paper_2110_11211_gb300 import inputs  # noqa: E402


def main(name, rtol=1e-10):
    w = inputs.WORKLOADS[name]
    t0 = time.time()
    S = schwarz.Schwarz(w["levels"], w["P"], w["gamma"], coeffs=inputs.coefficients(name))
    f = inputs.rhs(name)
    x, its, hist = krylov.pcg(lambda v: S.A @ v, S.apply, f, rtol=rtol)
    res = float(((f - S.A @ x) ** 2).sum() ** 0.5 / (f ** 2).sum() ** 0.5)
    out = {"workload": name, "levels": list(w["levels"]), "P": w["P"], "gamma": w["gamma"],
           "q": S.q, "N": S.N, "N0": S.N0, "rtol": rtol, "iters": its,
           "rel_res": hist[-1], "true_rel_res": res, "oracle_seconds": round(time.time() - t0, 1)}
    path = os.path.join(HERE, f"oracle_pcg_{name}.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "aniso3d_l10x5x3_P128")
