"""Benchmark: time to relative residual 1e-10 for the large sparse CARE, mixed
precision (FP32 NLR-ADI / LR-ADI inner solves, FP64 residual factorisation and
update) vs the all-FP64 path of the same code, on one B300; plus the SpMM
roofline.  Prints one JSON line.

Workload: 2D convection-diffusion -Lap(u) + 10 u_x + 100 u_y on a 500 x 500
interior grid (n = 250,000, nnz = 1,248,000), A = -L, B n x 5 and C 5 x n with
U[0,1) entries from the seeded generator.  A step is one complete care_solve
(NLR-ADI + refinement to ||R||_F / ||C^T C||_F <= 1e-10) with the inputs
resident in HBM; L2 is flushed (a 256 MB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU FP64 oracle (the program the GPU results are
checked against) on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to rel. residual 1e-10, mixed vs all-FP64 on 1 B300; SpMM HBM GB/s vs peak"
TOL = 1e-10
GRID = 500
MP = 5
R_CAP = 1536


def workload_config(prob):
    return {"workload": f"2D convection-diffusion CARE, {GRID}x{GRID} grid (n={prob.n}, nnz={prob.A.nnz}), "
                        f"m=p={MP}, tol {TOL:g}, mixed FP32-inner/FP64-outer",
            "n": prob.n, "nnz": prob.A.nnz, "m": MP, "p": MP, "tol": TOL,
            "l2": "flushed by a 256 MB write before each timed step"}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampler (SM clock and throttle reasons) for the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, path):
        self.path = path
        self.p = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", "0"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [l.split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return out
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
        if mx:
            out["sm_max_mhz"] = max(mx)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(sm)
        return out


def run_reference(args):
    """CPU FP64 oracle on the host cores: a bounded sample of the same workload."""
    import numpy as np
    import care_inputs as ci
    from oracle import lowrank as ol
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob = ci.config_fdm2d(GRID, MP, MP)
    As = prob.A.to_scipy()
    cores = os.cpu_count()
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        v, sample = oracle_sample(prob, As)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(v)
    val = statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": val * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(prob),
            "cpu_baseline": {"value": val, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def oracle_sample(prob, As, shifted_solves=None):
    """Time the oracle's FP64 LR-ADI shifted solve (SuperLU factorisation of
    M_p = (A + pI)^T and an SMW block solve with p + m right-hand sides) for three
    shifts, and scale to a full solve by the number of shifted solves a full
    FP64 Framework-1 run performs (the GPU run's count, or 150 if unknown)."""
    import numpy as np
    from oracle import lowrank as ol
    solver = ol.ShiftedSolver(As)
    W = np.hstack([prob.C.T, np.zeros((prob.n, MP))])
    K = 1e-3 * prob.B
    shifts = [-3000.0, -3.0e4, -3.0e5]
    t0 = time.perf_counter()
    for p in shifts:
        ol.smw_solve(solver, prob.B, K, p, W)
    per = (time.perf_counter() - t0) / len(shifts)
    count = shifted_solves or 150
    return per * count, (f"3 FP64 SMW shifted solves (SuperLU of (A+pI)^T, {2 * MP} RHS) on the n={prob.n} "
                         f"operator, {per:.3f} s each, scaled x{count} shifted solves per full solve")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host buffers) solve")
    ap.add_argument("--only", default="all", choices=["all", "spmm", "gram"],
                    help="spmm / gram: only the SpMM or Gram microbenchmark cases (the profiling cases "
                         "for k_spmm and k_gram)")
    ap.add_argument("--summarize-launches", metavar="CSV",
                    help="summarise an ncu --csv launch list (gpu__time_duration.sum) per kernel and exit")
    args = ap.parse_args()
    if args.summarize_launches:
        return summarize_launches(args.summarize_launches)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import care_inputs as ci
    import paper_2607_14742_b300 as pb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    prob = ci.config_fdm2d(GRID, MP, MP)
    if args.only == "spmm":
        print(json.dumps(spmm_roofline(pb, torch, prob, dev)))
        return
    if args.only == "gram":
        print(json.dumps(gram_cases(pb, torch, dev)))
        return
    A = pb.CSR.from_arrays(prob.n, prob.A.rowptr, prob.A.colind, prob.A.val, device=dev)
    B = torch.tensor(prob.B, device=dev)
    C = torch.tensor(prob.C, device=dev)
    ws = pb.Workspace()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # shifted-solve configuration chosen by the library's autotuner (outside the timed region)
    t_tune = time.perf_counter()
    tuned, tune_ms = pb.autotune(pb.Operator(A), MP, 2 * MP, prec="mixed")
    t_tune = time.perf_counter() - t_tune
    tuned64, _ = pb.autotune(pb.Operator(A), MP, 2 * MP, prec="fp64")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def solve(prec):
        return pb.care_solve(A, B, C, tol=TOL, prec=prec, r_cap=R_CAP, workspace=ws,
                             opts=pb.default_options(krylov_chunk=(tuned if prec == "mixed" else tuned64).krylov_chunk,
                                                     tri_sweeps=(tuned if prec == "mixed" else tuned64).tri_sweeps,
                                                     precond=(tuned if prec == "mixed" else tuned64).precond))

    for _ in range(args.warmup):
        Z, info = solve("mixed")
    stream = torch.cuda.current_stream()
    ts = []
    infos = []
    launches0 = pb.kernel_launches()
    clocks = Clocks(os.path.join(ROOT, "gpurun_out", "bench_clocks.csv")
                    if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else "/tmp/bench_clocks.csv")
    barrier()
    # the timed steps sit in an NVTX range so that a profiler can be restricted to them
    torch.cuda.nvtx.range_push("bench_timed")
    with clocks:
        for _ in range(args.steps):
            flush.fill_(1.0)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            Z, info = solve("mixed")
            e1.record(stream)
            barrier()
            ts.append(e0.elapsed_time(e1) / 1e3)
            infos.append(info)
    torch.cuda.nvtx.range_pop()
    launches = pb.kernel_launches() - launches0
    t = statistics.mean(ts)
    if world > 1:
        tt = torch.tensor([t], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    info = infos[-1]
    # the all-FP64 path of the same code
    fp64 = None
    if args.fp64_steps > 0:
        Z64, i64 = solve("fp64")
        t64 = []
        for _ in range(args.fp64_steps):
            flush.fill_(1.0)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            Z64, i64 = solve("fp64")
            e1.record(stream)
            barrier()
            t64.append(e0.elapsed_time(e1) / 1e3)
        fp64 = {"s_per_solve": statistics.mean(t64), "status": i64["status"], "rank": i64["rank"],
                "res_rel_CtC": i64["res_rel_CtC"], "iter0": i64["iter0"], "iter": i64["iter"],
                "speedup_mixed_vs_fp64": statistics.mean(t64) / t}
    # end to end through the public API: host inputs -> device, Z -> host, every step
    hA = [torch.from_numpy(prob.A.rowptr).pin_memory(), torch.from_numpy(prob.A.colind).pin_memory(),
          torch.from_numpy(prob.A.val).pin_memory()]
    hB = torch.from_numpy(prob.B).pin_memory()
    hC = torch.from_numpy(prob.C).pin_memory()
    h2d = sum(x.numel() * x.element_size() for x in hA + [hB, hC])
    e2e_t = []
    d2h = 0
    for _ in range(0 if args.no_e2e else max(1, args.steps)):
        flush.fill_(1.0)
        barrier()
        t0 = time.perf_counter()
        dA = pb.CSR(prob.n, hA[0].to(dev, non_blocking=True), hA[1].to(dev, non_blocking=True),
                    hA[2].to(dev, non_blocking=True))
        dB = hB.to(dev, non_blocking=True)
        dC = hC.to(dev, non_blocking=True)
        Ze, ie = pb.care_solve(dA, dB, dC, tol=TOL, prec="mixed", r_cap=R_CAP, workspace=ws,
                               opts=pb.default_options(krylov_chunk=tuned.krylov_chunk, tri_sweeps=tuned.tri_sweeps,
                                                       precond=tuned.precond))
        Zh = Ze.cpu()
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
        d2h = Zh.numel() * Zh.element_size()
    # SpMM roofline: the fused BiCGStab SpMM shape (b = 2*(p+m) FP32 columns) and a
    # cold operator + blocks larger than L2 (the 3D 100^3 operator, 20 columns)
    spmm = spmm_roofline(pb, torch, prob, dev)
    pk = peaks()
    line = {
        "metric": METRIC, "value": t, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic (seeded; see care_inputs)", "config": workload_config(prob),
        "status": info["status"], "res_rel_CtC": info["res_rel_CtC"], "res_paper": info["res_paper"],
        "rank": info["rank"], "iter0": info["iter0"], "iter": info["iter"], "krylov_iters": info["krylov_iters"],
        "ms_phase": {"nlradi": info["ms_phase"][0], "alg1": info["ms_phase"][1], "inner_lradi": info["ms_phase"][2],
                     "alg2": info["ms_phase"][3]},
        "fp64_path": fp64,
        "autotune": {"krylov_chunk": tuned.krylov_chunk, "tri_sweeps": tuned.tri_sweeps, "precond": tuned.precond,
                     "best_ms": tune_ms, "seconds": t_tune},
        "e2e": ({"value": statistics.mean(e2e_t), "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
                if e2e_t else None),
        "gpu_launches": launches // max(1, args.steps),
        "roofline": gram_roofline(info, t),
        "spmm": spmm,
        "clocks": clocks.summary(),
        "peaks_source": "MEASURED_PEAKS.json" if pk else "fallback 6400 GB/s",
    }
    if rank == 0 and not args.no_cpu_baseline:
        v, sample = oracle_sample(prob, prob.A.to_scipy(), shifted_solves=(info["iter0"][1] + info["iter"][1]))
        line["cpu_baseline"] = {"value": v, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": sample}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def summarize_launches(path):
    """Per-kernel launches, total device time and share from an ncu launch list
    (``ncu --metrics gpu__time_duration.sum --csv --log-file PATH``); prints a
    markdown table.  ncu serialises launches and runs them cold, so the shares,
    not the absolute times, are what carry over to the timed run."""
    import csv
    import re
    with open(path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]
    rd = csv.reader(lines)
    head = next(rd)
    ik, im, iu, iv = (head.index(k) for k in ("Kernel Name", "Metric Name", "Metric Unit", "Metric Value"))
    scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}

    def short(name):
        # drop "void " and the trailing (argument list)
        name = re.sub(r"^void ", "", name)
        if name.endswith(")"):
            depth = 0
            for i in range(len(name) - 1, -1, -1):
                depth += name[i] == ")"
                depth -= name[i] == "("
                if depth == 0:
                    return name[:i]
        return name

    agg = {}
    nrows = 0
    for r in rd:
        if len(r) <= iv or r[im] != "gpu__time_duration.sum":
            continue
        name = short(r[ik])
        us = float(r[iv].replace(",", "")) * scale.get(r[iu], 1.0)
        c, t = agg.get(name, (0, 0.0))
        agg[name] = (c + 1, t + us)
        nrows += 1
    total = sum(t for _, t in agg.values())
    print(f"{nrows} launches, {total / 1e3:.1f} ms summed device time\n")
    print("| kernel | launches | total ms | share | mean us |")
    print("|---|---:|---:|---:|---:|")
    for name, (c, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"| `{name}` | {c} | {t / 1e3:.1f} | {100 * t / total:.1f}% | {t / c:.1f} |")
    fam = {}
    for name, (c, t) in agg.items():
        k = name.split("<")[0]
        fc, ft = fam.get(k, (0, 0.0))
        fam[k] = (fc + c, ft + t)
    print("\n| kernel family | launches | total ms | share |")
    print("|---|---:|---:|---:|")
    for k, (c, t) in sorted(fam.items(), key=lambda kv: -kv[1][1]):
        print(f"| `{k}` | {c} | {t / 1e3:.1f} | {100 * t / total:.1f}% |")


FP64_PEAK_TFLOPS = 1.25  # nominal B300 FP64 (CUDA cores): ~2 FMA/clk/SM x 148 SMs x 2.03 GHz x 2


def gram_roofline(info, step_s):
    """Roofline of the dominant FP64 kernel family of the mixed solve, measured live:
    the library brackets every FP64 Gram product X^T Y (k_gram<double> + its split-K
    reduction) and every FP64 tall-skinny product X S (k_gemm_ts) with CUDA events on
    the solve's stream during the timed step and sums their algorithmic FLOP (2 n a b;
    n a (a+1) for X^T X) and device time.  The family with the larger device time is
    reported; both are listed.  Bound by the FP64 FMA pipe of the CUDA cores."""
    fams = {
        "gram": {"kernel": "k_gram<double> + k_gram_reduce: FP64 X^T Y of Algorithms 1-2",
                 "device_s": info["gram_ms"][0] / 1e3, "gflop": info["gram_gflop"][0],
                 "launches": info["gram_calls"][0]},
        "gemm_ts": {"kernel": "k_gemm_ts<double, *>: FP64 X S of Algorithms 1-2 (CGS2, Cholesky QR, factor updates)",
                    "device_s": info.get("gemm_ms", [0, 0])[0] / 1e3, "gflop": info.get("gemm_gflop", [0, 0])[0],
                    "launches": info.get("gemm_calls", [0, 0])[0]},
    }
    for f in fams.values():
        f["TFLOPs"] = f["gflop"] / f["device_s"] / 1e3 if f["device_s"] > 0 else 0.0
        f["share_of_step"] = f["device_s"] / step_s
    name = max(fams, key=lambda k: fams[k]["device_s"])
    top = fams[name]
    ach = top["TFLOPs"]
    return {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
            "kernel": top["kernel"] + " (n=250000, widths up to ~2600 columns), measured live in the timed step "
                      "with CUDA events on its stream",
            "launches": top["launches"], "device_s": top["device_s"], "share_of_step": top["share_of_step"],
            "fp64_families": fams,
            "peak_note": "nominal FP64 rate (no measured FP64 peak); FP32 Gram products of the inner solves: "
                         f"{info['gram_gflop'][1] / max(info['gram_ms'][1], 1e-9):.2f} TFLOP/s over "
                         f"{info['gram_ms'][1] / 1e3:.2f} s"}


def gram_cases(pb, torch, dev):
    """Gram microbenchmark (CUDA events on the launching stream, inputs > L2)."""
    stream = torch.cuda.current_stream()
    out = {}
    for name, dt, n, a, b in (("f64_sym_n250000_a512", torch.float64, 250000, 512, None),
                              ("f64_n250000_256x512", torch.float64, 250000, 256, 512),
                              ("f32_sym_n250000_a1024", torch.float32, 250000, 1024, None)):
        X = torch.randn(n, a, dtype=dt, device=dev)
        Y = X if b is None else torch.randn(n, b, dtype=dt, device=dev)
        flop = n * a * (a + 1) if b is None else 2 * n * a * b
        ms = []
        for it in range(7):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pb.gram(X, Y)
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= 2:
                ms.append(e0.elapsed_time(e1))
        m = statistics.median(ms)
        out[name] = {"ms": m, "gflop": flop / 1e9, "TFLOPs": flop / m / 1e9}
        del X, Y
    return out


def spmm_roofline(pb, torch, prob, dev):
    """Time the SpMM kernel live with CUDA events on the launching stream."""
    import care_inputs as ci
    pk = peaks()
    peak = float(pk.get("hbm_gbs", 6400.0))
    out = {}
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timeit(op, X, reps=20):
        Y = None
        for _ in range(3):
            Y = pb.spmm(op, X, -1000.0)
        ms = []
        for _ in range(reps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pb.spmm(op, X, -1000.0)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    cases = {}

    def alg_bytes(n, nnz, b, vb):
        # A^T values + column indices, row pointers, row sums, X read once, Y written once
        return nnz * (vb + 4) + 4 * (n + 1) + vb * n + 2 * n * b * vb

    op2 = pb.Operator(pb.CSR.from_arrays(prob.n, prob.A.rowptr, prob.A.colind, prob.A.val, device=dev))
    for b in (16, 32):
        X2 = torch.randn(prob.n, b, device=dev, dtype=torch.float32)
        ms2 = timeit(op2, X2)
        by = alg_bytes(prob.n, prob.A.nnz, b, 4)
        cases[f"fdm2d_500_b{b}_f32"] = {"ms": ms2, "alg_bytes": by, "GBs": by / ms2 / 1e6}
    p3 = ci.convection_diffusion(100, (10.0, 50.0, 100.0))
    op3 = pb.Operator(pb.CSR.from_arrays(p3.n, p3.rowptr, p3.colind, p3.val, device=dev))
    for b in (16, 32):
        X3 = torch.randn(p3.n, b, device=dev, dtype=torch.float32)
        ms3 = timeit(op3, X3)
        by = alg_bytes(p3.n, p3.nnz, b, 4)
        cases[f"fdm3d_100_b{b}_f32"] = {"ms": ms3, "alg_bytes": by, "GBs": by / ms3 / 1e6}
    main = cases["fdm3d_100_b32_f32"]
    out["cases"] = cases
    out["roofline"] = {"bound": "hbm", "achieved": main["GBs"], "peak": peak, "unit": "GB/s",
                       "frac": main["GBs"] / peak, "traffic": 289.7e6,
                       "traffic_note": "dram read+write bytes per launch from ncu --set full of this case "
                                       "(bench.py --only spmm): 191.5 MB read, 98.1 MB written; about 30 MB "
                                       "of Y is still in L2 when the kernel ends",
                       "kernel": "k_spmm: Y = (A^T + pI) X, CSR, 7-point 100^3 operator (n=1e6, nnz=6.94e6), "
                                 "32 FP32 columns, difference form, L2 flushed; measured on the launching stream"}
    return out


if __name__ == "__main__":
    main()
