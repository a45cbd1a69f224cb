"""Conditioning sweep of Section 5.1 (Table 1, Example 1) with the oracle: FP64 and
FP32 inner solves (dense direct shifted solves), Algorithms 1-2 in FP64.

Test infrastructure (see ``oracle/__init__.py``): prints one markdown table row per
kappa_2(A) = 10^q and inner precision for the design notes; nothing here is used
by the GPU path.

    python -m oracle.table1_fp32_sweep [q ...]
"""
from __future__ import annotations

import sys
import time

import care_inputs as ci
from oracle import lowrank as ol


def run(q: float, inner: str):
    p = ci.paper_example1(q=q)
    A = p.A.to_dense()
    tol = 1e-5 if inner == "fp32" else 1e-12
    t = time.time()
    _, info = ol.framework1(A, p.B, p.C, tau_R=1e-14, dense=True, inner=inner, tol_lyap=tol, tol_newton=tol)
    return info, time.time() - t


def main(qs):
    print("| kappa_2(A) | inner | status | Res | rel. residual | Iter0 | Iter | rank | s |")
    print("|---|---|---|---:|---:|---|---|---:|---:|")
    for q in qs:
        for inner in ("fp64", "fp32"):
            info, s = run(q, inner)
            i0, it = info["iter0"], info["iter"]
            print(f"| 1e{q:g} | {inner} | {info['status']} | {info['res_paper']:.2e} | {info['rel_res']:.1e} | "
                  f"{i0[0]}({i0[1]}) | {it[0]}({it[1]}) | {info['rank']} | {s:.0f} |", flush=True)


if __name__ == "__main__":
    main([float(x) for x in sys.argv[1:]] or [1, 2, 3, 4, 5, 6, 7, 8])
