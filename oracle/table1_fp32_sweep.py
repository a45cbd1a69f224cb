"""Conditioning sweeps with the oracle: FP64 and FP32 inner solves (dense direct
shifted solves), Algorithms 1-2 in FP64.

  * Section 5.1 (Table 1, Example 1, n = 1000): kappa_2(A) = 10^q.
  * ``--dense200``: the n = 200 dense conditioning family of ``care_inputs``
    (kappa_2(A) ~ 10^k), with the error against the dense Newton solution.

Test infrastructure (see ``oracle/__init__.py``): prints markdown table rows for the
design notes; nothing here is used by the GPU path.

    python -m oracle.table1_fp32_sweep [q ...]
    python -m oracle.table1_fp32_sweep --inners bf16,fp16 [q ...]
    python -m oracle.table1_fp32_sweep --dense200 [k ...]

bf16 / fp16 are the storage-rounding model of ``oracle.lowrank.storage_rounding``
(FP32 arithmetic, results rounded to the narrow format); their inner tolerances are
1e-2 and 1e-3 (a few units of u_s), FP32's is the paper's 1e-5.
"""
from __future__ import annotations

import sys
import time

import numpy as np

import care_inputs as ci
from oracle import dense as od
from oracle import lowrank as ol


INNER_TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-3, "bf16": 1e-2}


def run(q: float, inner: str):
    p = ci.paper_example1(q=q)
    A = p.A.to_dense()
    tol = INNER_TOL[inner]
    t = time.time()
    _, info = ol.framework1(A, p.B, p.C, tau_R=1e-14, dense=True, inner=inner, tol_lyap=tol, tol_newton=tol)
    return info, time.time() - t


def main(qs, inners=("fp64", "fp32")):
    print("| kappa_2(A) | inner | status | Res | rel. residual | Iter0 | Iter | rank | s |")
    print("|---|---|---|---:|---:|---|---|---:|---:|")
    for q in qs:
        for inner in inners:
            try:
                info, s = run(q, inner)
            except (np.linalg.LinAlgError, FloatingPointError, ValueError) as e:
                print(f"| 1e{q:g} | {inner} | failed ({type(e).__name__}: overflow/non-finite) | | | | | | |",
                      flush=True)
                continue
            i0, it = info["iter0"], info["iter"]
            print(f"| 1e{q:g} | {inner} | {info['status']} | {info['res_paper']:.2e} | {info['rel_res']:.1e} | "
                  f"{i0[0]}({i0[1]}) | {it[0]}({it[1]}) | {info['rank']} | {s:.0f} |", flush=True)


def main_dense200(ks):
    print("| k | kappa_2(A) | inner | status | Res | rel. residual | error vs dense Newton | Iter | rank |")
    print("|---|---:|---|---|---:|---:|---:|---|---:|")
    for k in ks:
        p = ci.config_dense_conditioning(k)
        A = p.A.to_dense()
        X = od.newton_care(A, p.B, p.C)["X"]
        for inner in ("fp64", "fp32"):
            tol = 1e-5 if inner == "fp32" else 1e-12
            Z, info = ol.framework1(A, p.B, p.C, tau_R=1e-12, dense=True, inner=inner, tol_lyap=tol, tol_newton=tol)
            err = np.linalg.norm(Z @ Z.T - X) / np.linalg.norm(X)
            print(f"| {k} | {np.linalg.cond(A):.1e} | {inner} | {info['status']} | {info['res_paper']:.1e} | "
                  f"{info['rel_res']:.1e} | {err:.1e} | {info['iter'][0]}({info['iter'][1]}) | {info['rank']} |",
                  flush=True)


if __name__ == "__main__":
    args = sys.argv[1:]
    if args and args[0] == "--dense200":
        main_dense200([int(x) for x in args[1:]] or list(range(7)))
    elif args and args[0] == "--inners":
        main([float(x) for x in args[2:]] or [1, 2, 3, 4], inners=tuple(args[1].split(",")))
    else:
        main([float(x) for x in args] or [1, 2, 3, 4, 5, 6, 7, 8])
