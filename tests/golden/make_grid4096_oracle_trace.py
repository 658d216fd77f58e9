"""Writes grid4096_oracle_trace.json: the FP64 oracle's MDOT (Alg. 1) run on the
64 x 64 grid workload (seed 0, squared-Euclidean cost stored as float32 and
promoted exactly, gamma 2^4 -> 2^14, tol 1e-6), recording its schedule, operation
counts, final marginal error and transport cost. Calls only oracle/ and
workloads/. Run from the repository root:  python tests/golden/make_grid4096_oracle_trace.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import eot_oracle as O  # noqa: E402


def main():
    out = {}
    for kind in ("sqeuclid",):
        p = W.grid_problem_4096(0, kind)
        C = p["C"].astype(np.float64)
        t0 = time.time()
        res = O.mdot(C, p["r"], p["c"], gamma_i=16.0, gamma_f=16384.0, tol_final=1e-6)
        P = O.plan(res.u, res.v, res.gamma, C)
        out[kind] = {
            "stages": res.stages, "newton_steps": res.newton_steps, "cg_iters": res.cg_iters,
            "ls_trials": res.ls_trials, "sinkhorn_iters": res.sinkhorn_iters,
            "gammas": res.gammas, "ok": res.ok,
            "marg_err_l1": float(np.abs(P.sum(1) - p["r"]).sum() + np.abs(P.sum(0) - p["c"]).sum()),
            "transport_cost": float((P * C).sum()),
            "oracle_seconds": round(time.time() - t0, 1),
        }
    out["source"] = ("oracle.eot_oracle.mdot on workloads.grid_problem_4096(0, kind), "
                     "float64, written by tests/golden/make_grid4096_oracle_trace.py")
    with open(os.path.join(ROOT, "tests", "golden", "grid4096_oracle_trace.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
