"""Write tests/golden/oracle_cg_iterations.json by running the CPU oracle only.

For each workload, the FP64 CG iteration count that the oracle needs to
reach the relative residual 1e-10 on the seeded synthetic input, and the
wall time of that full oracle solve on this host.  The CPU baseline of the
benchmark times a bounded sample of oracle iterations and scales it by
these counts to a per-solve time.
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1411_5219_gb300 import synthetic as syn  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_cg_iterations.json")


def main():
    res = {}
    for name, solve in [("4^4", "mdagm"), ("24^3x8", "eo")]:
        w = syn.WORKLOADS[name]
        U = syn.gauge_field(w["dims"], w["eps"], w["seed"])
        b = syn.gaussian_spinor(w["dims"], w["seed"])
        t0 = time.time()
        if solve == "eo":
            _, st = oracle.solve_eo(U, b, w["kappa"], w["mu"], tol=1e-10)
        else:
            _, st = oracle.solve_mdagm(U, b, w["kappa"], w["mu"], tol=1e-10)
        res[name] = {"system": "Mhat^dag Mhat (even-odd)" if solve == "eo" else "M^dag M (full lattice)",
                     "kappa": w["kappa"], "mu": w["mu"], "tol": 1e-10, "iterations": int(st[0]),
                     "true_rel_residual": float(st[1]), "seconds": round(time.time() - t0, 2),
                     "threads": oracle.get_threads()}
        print(name, res[name], flush=True)
    with open(OUT, "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
