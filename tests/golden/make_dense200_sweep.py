"""Writes dense200_sweep.json: the oracle's Framework 1 on the n = 200 dense
conditioning family (kappa_2(A) = 10^k, k = 0..6) with dense direct shifted solves
(Section 5.1's configuration), FP64 and FP32 inner precision, tau_R = 1e-12, and
the error of Z Z^T against the dense Newton solution.  Calls only ``oracle/`` and
the seeded inputs.  The GPU conditioning-sweep test reads the stored outcomes.

    python tests/golden/make_dense200_sweep.py
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))

import care_inputs as ci  # noqa: E402
from oracle import dense as od  # noqa: E402
from oracle import lowrank as ol  # noqa: E402


def main():
    out = {}
    for k in range(7):
        p = ci.config_dense_conditioning(k)
        A = p.A.to_dense()
        X = od.newton_care(A, p.B, p.C)["X"]
        for inner in ("fp64", "fp32"):
            tol = 1e-5 if inner == "fp32" else 1e-12
            Z, info = ol.framework1(A, p.B, p.C, tau_R=1e-12, dense=True, inner=inner, tol_lyap=tol,
                                    tol_newton=tol)
            err = float(np.linalg.norm(Z @ Z.T - X) / np.linalg.norm(X))
            out[f"{k}/{inner}"] = {"status": info["status"], "rel_res": float(info["rel_res"]),
                                   "res_paper": float(info["res_paper"]), "err": err,
                                   "iter": [int(v) for v in info["iter"]], "rank": int(info["rank"])}
            print(k, inner, out[f"{k}/{inner}"], flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dense200_sweep.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
