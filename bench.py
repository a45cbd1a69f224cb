"""Benchmark: time to relative residual 1e-10 for the large sparse CARE, mixed
precision (FP32 NLR-ADI / LR-ADI inner solves, FP64 residual factorisation and
update) vs the all-FP64 path of the same code, on one B300; plus the rooflines.
Prints one JSON line.

Workload: 2D convection-diffusion -Lap(u) + 10 u_x + 100 u_y on a 500 x 500
interior grid (n = 250,000, nnz = 1,248,000), A = -L, B n x 5 and C 5 x n with
U[0,1) entries from the seeded generator.  A step is one complete solve through
the public API with host buffers: the pinned host inputs (A in CSR, B, C) are
copied to the device, care_solve runs (NLR-ADI + refinement to
||R||_F / ||C^T C||_F <= 1e-10), and Z is copied back.  CUDA events on the
solve's stream split every step: `value` is the device time of care_solve with
its inputs resident in HBM, `e2e` the whole step including both copies.  L2 is
flushed (a 256 MB write) before every step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU FP64 oracle (the program the GPU results are
checked against) on the host cores, one FP64 SMW shifted solve of the same
workload per step.  One solve takes tens of seconds on the GPU, so the timed
work is kept inside a wall-clock budget (--budget, default 1500 s): if the
requested warm-up and steps cannot fit, fewer are run (at least 3 warm-up
steps) and the line reports the counts actually run.
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

METRIC = "time to rel. residual 1e-10, mixed vs all-FP64 on 1 B300; SpMM HBM GB/s vs peak"
TOL = 1e-10
GRID = 500
MP = 5
R_CAP = 1536
SLICE_PAIRS = 43  # BF16 slice products per FP64 multiply-add in the FP64-accurate tensor-core path
SLICE_PAIRS_F32 = 10  # the same for the FP32-accurate path


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

    def __init__(self):
        fd, self.path = tempfile.mkstemp(prefix="care_bench_clocks_", suffix=".csv")
        os.close(fd)
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
        try:
            os.unlink(self.path)
        except OSError:
            pass
        return out


# ---------------------------------------------------------------- oracle arm --
SHIFTS = (-3000.0, -3.0e4, -3.0e5)


def oracle_shifted_solve(prob, As, shift):
    """One FP64 SMW shifted solve of the oracle on the workload's operator: SuperLU
    factorisation of M_p = (A + pI)^T and the solve for the block [C^T, K] (p + m
    right-hand sides) with the Sherman-Morrison-Woodbury correction (Section 4)."""
    import numpy as np
    from oracle import lowrank as ol
    solver = ol.ShiftedSolver(As)
    W = np.hstack([prob.C.T, np.zeros((prob.n, MP))])
    K = 1e-3 * prob.B
    t0 = time.perf_counter()
    ol.smw_solve(solver, prob.B, K, shift, W)
    return time.perf_counter() - t0


SAMPLE = (f"one FP64 SMW shifted solve per step (SuperLU of (A+pI)^T, {2 * MP} right-hand sides, shifts "
          f"cycling through {SHIFTS}) on the n=250000 operator of the workload")


def run_reference(args):
    """CPU FP64 oracle on the host cores, one shifted solve per step (measured)."""
    import care_inputs as ci
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob = ci.config_fdm2d(GRID, MP, MP)
    As = prob.A.to_scipy()
    times = []
    for it in range(args.warmup + args.steps):
        dt = oracle_shifted_solve(prob, As, SHIFTS[it % len(SHIFTS)])
        if it >= args.warmup:
            times.append(dt)
    val = statistics.mean(times)
    unit = "s per FP64 shifted solve"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": val * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(prob),
            "cpu_baseline": {"value": val, "unit": unit, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": SAMPLE},
            "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "note": "a full oracle solve of this workload takes several hundred shifted solves (tens of minutes "
                    "on the host); the timed unit is one of them"}
    print(json.dumps(line))


# ------------------------------------------------------------------ our arm --
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--budget", type=float, default=1500.0, help="wall-clock seconds for the whole run")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", default="all", choices=["all", "spmm", "gram", "batched"],
                    help="spmm / gram: only the SpMM or Gram microbenchmark cases (the profiling cases "
                         "for k_spmm and k_tc_gemm / k_gram); batched: the serving sweep of many "
                         "independent CAREs (aggregate CAREs/s of the batched paths and of single solves)")
    ap.add_argument("--autotune", action="store_true",
                    help="run the solves with care_autotune's choice instead of the default options")
    ap.add_argument("--batch-count", type=int, default=32)
    ap.add_argument("--batch-side-hi", type=int, default=192)
    ap.add_argument("--summarize-launches", metavar="CSV",
                    help="summarise an ncu --csv launch list (gpu__time_duration.sum) per kernel and exit")
    args = ap.parse_args()
    if args.summarize_launches:
        return summarize_launches(args.summarize_launches)
    if args.impl == "reference":
        return run_reference(args)
    t_start = time.perf_counter()

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
    if args.only == "batched":
        print(json.dumps(batched_cases(pb, torch, dev, args.batch_count, args.batch_side_hi)))
        return

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # the SpMM roofline and the FP64 peak first (cheap; they survive a cut run)
    spmm = spmm_roofline(pb, torch, prob, dev)
    fp64_peak = pb.fp64_peak()
    # pinned host inputs: every step copies them to the device and Z back
    hA = [torch.from_numpy(prob.A.rowptr).pin_memory(), torch.from_numpy(prob.A.colind).pin_memory(),
          torch.from_numpy(prob.A.val).pin_memory()]
    hB = torch.from_numpy(np.ascontiguousarray(prob.B)).pin_memory()
    hC = torch.from_numpy(np.ascontiguousarray(prob.C)).pin_memory()
    h2d = sum(x.numel() * x.element_size() for x in hA + [hB, hC])
    ws = pb.Workspace()
    # The solves run with the library's default options (BiCGStab + sweep ILU(0), chunks
    # of 64 columns, one vector per SpMM thread).  --autotune uses care_autotune's choice
    # per precision instead (outside the timed region): its objective, two shifted solves
    # at one mid-spectrum shift, picked configurations that made this workload's full
    # solve slower (37.7 s against 22.4 s with the defaults), so it is not the default.
    tuned = {}
    tune_ms = {}
    t_tune = 0.0
    if args.autotune:
        dA0 = pb.CSR(prob.n, hA[0].to(dev), hA[1].to(dev), hA[2].to(dev))
        op0 = pb.Operator(dA0)
        t_tune = time.perf_counter()
        for pr in (("fp64", "mixed") if args.fp64_steps > 0 else ("mixed",)):
            tuned[pr], tune_ms[pr] = pb.autotune(op0, MP, 2 * MP, prec=pr)
        t_tune = time.perf_counter() - t_tune

    def use(prec):
        """The options of prec (tuned ones set their launch shape when applied again)."""
        if not args.autotune:
            return pb.default_options()
        t = tuned[prec]
        pb.autotune(op0, MP, 2 * MP, prec=prec)
        return pb.default_options(krylov=t.krylov, krylov_chunk=t.krylov_chunk, tri_sweeps=t.tri_sweeps,
                                  precond=t.precond)

    run_opts = {}

    def step(prec):
        """One end-to-end solve; returns (device solve s, whole step s, info, d2h bytes)."""
        flush.fill_(1.0)
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        dA = pb.CSR(prob.n, hA[0].to(dev, non_blocking=True), hA[1].to(dev, non_blocking=True),
                    hA[2].to(dev, non_blocking=True))
        dB = hB.to(dev, non_blocking=True)
        dC = hC.to(dev, non_blocking=True)
        ev[1].record(stream)
        Z, info = pb.care_solve(dA, dB, dC, tol=TOL, prec=prec, r_cap=R_CAP, workspace=ws, opts=run_opts[prec])
        ev[2].record(stream)
        Zh = Z.to("cpu", non_blocking=False)
        ev[3].record(stream)
        barrier()
        return (ev[1].elapsed_time(ev[2]) / 1e3, ev[0].elapsed_time(ev[3]) / 1e3, info,
                Zh.numel() * Zh.element_size())

    # the all-FP64 path of the same code (same end-to-end step, its own autotuned
    # options), first, so that the budget of the mixed steps is known
    fp64 = None
    if args.fp64_steps > 0:
        t64 = []
        i64 = None
        for _ in range(args.fp64_steps):
            if "fp64" not in run_opts:
                run_opts["fp64"] = use("fp64")
            v64, _, i64, _ = step("fp64")
            t64.append(v64)
        fp64 = {"s_per_solve": statistics.mean(t64), "status": i64["status"], "rank": i64["rank"],
                "res_rel_CtC": i64["res_rel_CtC"], "iter0": i64["iter0"], "iter": i64["iter"],
                "ms_phase": i64["ms_phase"]}
    # warm-up, with a budget check after the first step
    warm_done = 0
    t0 = time.perf_counter()
    run_opts["mixed"] = use("mixed")
    step("mixed")
    warm_done = 1
    t_step = time.perf_counter() - t0
    reserve = 30.0 + (30.0 if not args.no_cpu_baseline else 0.0)
    left = args.budget - (time.perf_counter() - t_start) - reserve
    warmup = max(1, args.warmup)
    steps = max(1, args.steps)
    while (warmup - warm_done + steps) * t_step > left and warmup > 3:
        warmup -= 1
    while (warmup - warm_done + steps) * t_step > left and steps > 1:
        steps -= 1
    for _ in range(warmup - warm_done):
        step("mixed")

    clocks = Clocks()
    vals, e2es, infos = [], [], []
    d2h = 0
    launches0 = pb.kernel_launches()
    barrier()
    torch.cuda.nvtx.range_push("bench_timed")
    with clocks:
        for _ in range(steps):
            v, e, info, d2h = step("mixed")
            vals.append(v)
            e2es.append(e)
            infos.append(info)
    torch.cuda.nvtx.range_pop()
    launches = (pb.kernel_launches() - launches0) // steps
    t = statistics.mean(vals)
    te = statistics.mean(e2es)
    if world > 1:
        t, te = max_over_ranks([t, te], dev)
    info = infos[-1]
    if fp64 is not None:
        fp64["speedup_mixed_vs_fp64"] = fp64["s_per_solve"] / t
    pk = peaks()
    line = {
        "metric": METRIC, "value": t, "unit": "s", "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": t * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic (seeded; see care_inputs)", "config": workload_config(prob),
        "steps_requested": args.steps, "warmup_requested": args.warmup,
        "status": info["status"], "res_rel_CtC": info["res_rel_CtC"], "res_paper": info["res_paper"],
        "rank": info["rank"], "iter0": info["iter0"], "iter": info["iter"], "krylov_iters": info["krylov_iters"],
        "s_per_step_all": vals,
        "ms_phase": {"nlradi": info["ms_phase"][0], "alg1": info["ms_phase"][1], "inner_lradi": info["ms_phase"][2],
                     "alg2": info["ms_phase"][3]},
        "host_syncs": info["host_syncs"],
        "fp64_path": fp64,
        "options": "autotuned" if args.autotune else "library defaults",
        "autotune": {pr: {"krylov": t.krylov, "krylov_chunk": t.krylov_chunk, "tri_sweeps": t.tri_sweeps,
                          "precond": t.precond, "best_ms": tune_ms[pr]} for pr, t in tuned.items()},
        "launch_shape_mixed": {"spmm_vectors_per_thread_by_width_class": pb.launch_shape()[0],
                               "ctas_per_sm": pb.launch_shape()[1], "spmm_row_blocks": pb.launch_shape()[2]},
        "autotune_seconds": t_tune,
        "e2e": {"value": te, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roofline(info, t, pk, fp64_peak),
        "spmm": spmm,
        "clocks": clocks.summary(),
        "peaks_source": "MEASURED_PEAKS.json" if pk else "fallback 6400 GB/s, 1800 TFLOP/s bf16",
    }
    if rank == 0 and not args.no_cpu_baseline:
        As = prob.A.to_scipy()
        ts = [oracle_shifted_solve(prob, As, SHIFTS[i % len(SHIFTS)]) for i in range(4)]
        per = statistics.mean(ts[1:])
        nsolves = info["iter0"][1] + info["iter"][1]
        line["cpu_baseline"] = {"value": per, "unit": "s per FP64 shifted solve", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": SAMPLE + " (3 timed after 1 untimed)",
                                "full_solve_estimate_s": per * nsolves,
                                "full_solve_estimate_note": f"extrapolation, not a timing: the measured time per "
                                                            f"shifted solve x the {nsolves} LR-ADI shifted solves "
                                                            f"of the timed GPU solve"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def roofline(info, step_s, pk, fp64_peak):
    """Roofline of the kernel family with the largest device time in the timed step,
    all measured live (CUDA events on the solve's stream around every launch or
    solve of the family, summed by the library into care_info):
      - tensor: FP64-accurate sliced products (k_tc_gemm and its slicing passes);
        achieved = 43 BF16 slice-pair FLOPs per FP64 FLOP (2 n a b, or n a (a+1) for
        X^T X) / device time, against the sustained bf16 peak;
      - hbm: FP32 block Krylov solves (k_spmm, k_bicg_*, k_trisweep, ILU setup);
        achieved = algorithmic bytes (pass count per iteration, see DESIGN) / time;
      - alu: FP64 products left on the CUDA cores, against the measured FP64 FMA peak."""
    hbm = float(pk.get("hbm_gbs", 6400.0))
    bf16 = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1800.0)))
    fams = {
        "tc_f64_slices": {"device_s": info["tc_ms"][0] / 1e3, "bound": "tensor", "unit": "TFLOP/s", "peak": bf16,
                          "work": info["tc_gflop"][0] * SLICE_PAIRS * 1e-3, "launches": info["tc_calls"][0],
                          "kernel": "k_tc_gemm<0> + slicing: FP64-accurate X^T Y and X S of Algorithms 1-2 "
                                    "(BF16 slices, tcgen05, TMA), n=250000, widths up to ~3000"},
        "tc_f32_slices": {"device_s": info["tc_ms"][1] / 1e3, "bound": "tensor", "unit": "TFLOP/s", "peak": bf16,
                          "work": info["tc_gflop"][1] * SLICE_PAIRS_F32 * 1e-3, "launches": info["tc_calls"][1],
                          "kernel": "k_tc_gemm<3> + slicing: FP32-accurate X^T Y and X S of the inner solves "
                                    "(4 BF16 slices, tcgen05, TMA), n=250000"},
        "krylov_f32": {"device_s": info["krylov_ms"] / 1e3, "bound": "hbm", "unit": "GB/s", "peak": hbm,
                       "work": info["krylov_gbyte"], "launches": None,
                       "kernel": "block BiCGStab shifted solves (k_spmm, k_bicg_*, k_trisweep, ILU(0) setup), "
                                 "FP32, n=250000"},
        "fp64_cuda_cores": {"device_s": (info["gram_ms"][0] + info["gemm_ms"][0]) / 1e3, "bound": "alu",
                            "unit": "TFLOP/s", "peak": fp64_peak,
                            "work": (info["gram_gflop"][0] + info["gemm_gflop"][0]) * 1e-3,
                            "launches": info["gram_calls"][0] + info["gemm_calls"][0],
                            "kernel": "k_gram<double>, k_gemm_ts<double,*>: FP64 products below the tensor-core "
                                      "size threshold"},
    }
    for f in fams.values():
        f["achieved"] = f["work"] / f["device_s"] if f["device_s"] > 0 else 0.0
        f["frac"] = f["achieved"] / f["peak"] if f["peak"] else None
        f["share_of_step"] = f["device_s"] / step_s
    name = max(fams, key=lambda k: fams[k]["device_s"])
    top = fams[name]
    return {"bound": top["bound"], "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
            "frac": top["frac"], "traffic": None, "family": name, "kernel": top["kernel"],
            "device_s": top["device_s"], "share_of_step": top["share_of_step"],
            "peak_note": {"tensor": "bf16_tflops_sustained of measured", "hbm": "hbm_gbs of measured",
                          "alu": "FP64 FMA peak measured in this run (care_fp64_peak)"}[top["bound"]],
            "traffic_note": "not captured live; the per-kernel ncu DRAM bytes are in profiles/",
            "families": fams, "fp64_fma_peak_tflops": fp64_peak}


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


def max_over_ranks(values, device):
    """Element-wise maximum of `values` over the ranks of the default process group
    (every rank gets the result): the job's time is its slowest replica's.  The
    single-CARE path does not shard, so N GPUs run N independent replicas and this
    is the only collective of the bench."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def batched_cases(pb, torch, dev, count, side_hi):
    """Serving sweep: `count` independent 2D convection-diffusion CAREs, grid sides
    U{64..side_hi}, m, p U{1..8}, mixed precision to 1e-10, solved (a) by the serving
    mode (shifted solves of all instances in shared persistent launches), (b) by host
    workers overlapping whole solves, (c) one after another; plus the FP64 single
    solves of a sample.  Wall time per variant (one untimed run first)."""
    import care_inputs as ci
    probs = ci.config_batched(count=count, side_lo=64, side_hi=side_hi, mp_hi=8)
    dA = [(pb.CSR.from_arrays(p.n, p.A.rowptr, p.A.colind, p.A.val, device=dev), p.B, p.C) for p in probs]
    o = pb.default_options(adi_cap=512)
    out = {"workload": f"{count} 2D convection-diffusion CAREs, grid sides U{{64..{side_hi}}} "
                       f"(n {min(p.n for p in probs)}..{max(p.n for p in probs)}), m, p U{{1..8}}, mixed, tol 1e-10",
           "total_unknowns": int(sum(p.n for p in probs))}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, r

    def progress(key):  # each variant as it completes (stderr), so a cut run keeps them
        print(json.dumps({key: out[key]}), file=sys.stderr, flush=True)

    stats = {}
    t, (Z, infos, st) = timed(lambda: pb.care_solve_batched(dA, tol=1e-10, prec="mixed", r_cap=512, opts=o,
                                                            persistent=True, stats=stats, allow=(4, 5, 6)))
    out["persistent"] = {"s": t, "cares_per_s": count / t, "batch_launches": stats.get("batch_launches"),
                         "ok": sum(i["status"] == "CARE_OK" for i in infos),
                         "worst_res": max(i["res_rel_CtC"] for i in infos)}
    progress("persistent")
    t, (Z, infos, st) = timed(lambda: pb.care_solve_batched(dA, tol=1e-10, prec="mixed", r_cap=512, opts=o,
                                                            workers=8, allow=(4, 5, 6)))
    out["host_workers_8"] = {"s": t, "cares_per_s": count / t, "ok": sum(i["status"] == "CARE_OK" for i in infos),
                             "worst_res": max(i["res_rel_CtC"] for i in infos)}
    progress("host_workers_8")

    def loop(prec, items):
        res = []
        for A, B, C in items:
            res.append(pb.care_solve(A, B, C, tol=1e-10, prec=prec, r_cap=512, opts=o, allow=(4, 5, 6))[1])
        return res
    t, infos = timed(lambda: loop("mixed", dA))
    out["single_mixed_loop"] = {"s": t, "cares_per_s": count / t, "ok": sum(i["status"] == "CARE_OK" for i in infos)}
    progress("single_mixed_loop")
    sample = dA[:8]
    t0 = time.perf_counter()
    infos = loop("fp64", sample)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    out["single_fp64_sample"] = {"instances": len(sample), "s": t, "cares_per_s": len(sample) / t,
                                 "ok": sum(i["status"] == "CARE_OK" for i in infos)}
    return out


def gram_cases(pb, torch, dev):
    """Gram microbenchmark (CUDA events on the launching stream, inputs > L2):
    FP64 X^T X on the tensor cores (sliced) and on the CUDA cores."""
    stream = torch.cuda.current_stream()
    out = {}
    for name, n, a in (("f64_sym_n250000_a512", 250000, 512), ("f64_sym_n250000_a2048", 250000, 2048)):
        X = torch.randn(n, a, dtype=torch.float64, device=dev)
        flop = n * a * (a + 1)
        for impl, f in (("tc", lambda: pb.gram_tc(X, X, "f64")), ("cuda_cores", lambda: pb.gram(X, X))):
            ms = []
            for it in range(5):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                f()
                e1.record(stream)
                torch.cuda.synchronize()
                if it >= 2:
                    ms.append(e0.elapsed_time(e1))
            m = statistics.median(ms)
            out[f"{name}_{impl}"] = {"ms": m, "gflop_fp64": flop / 1e9, "TFLOPs_fp64_equiv": flop / m / 1e9}
        del X
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
        for _ in range(3):
            pb.spmm(op, X, -1000.0)
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

    # every case is timed with the launch shape the autotuner's first stage would pick
    # for it (vectors per thread x CTAs per SM x row order, fastest median); the
    # library's default shape is set again afterwards (the solves are autotuned later)
    shapes = [(v, c, b) for b in (0, 1) for c in (4, 8) for v in (1, 2, 4)]

    def best_shape(op, X):
        best = None
        for sh in shapes:
            pb.set_launch_shape(*sh)
            t = timeit(op, X, reps=7)
            if best is None or t < best[0]:
                best = (t, sh)
        pb.set_launch_shape(*best[1])
        return timeit(op, X), best[1]

    op2 = pb.Operator(pb.CSR.from_arrays(prob.n, prob.A.rowptr, prob.A.colind, prob.A.val, device=dev))
    for b in (16, 32):
        X2 = torch.randn(prob.n, b, device=dev, dtype=torch.float32)
        ms2, sh = best_shape(op2, X2)
        by = alg_bytes(prob.n, prob.A.nnz, b, 4)
        cases[f"fdm2d_500_b{b}_f32"] = {"ms": ms2, "alg_bytes": by, "GBs": by / ms2 / 1e6, "shape": sh}
    p3 = ci.convection_diffusion(100, (10.0, 50.0, 100.0))
    op3 = pb.Operator(pb.CSR.from_arrays(p3.n, p3.rowptr, p3.colind, p3.val, device=dev))
    for b in (16, 32):
        X3 = torch.randn(p3.n, b, device=dev, dtype=torch.float32)
        ms3, sh = best_shape(op3, X3)
        by = alg_bytes(p3.n, p3.nnz, b, 4)
        cases[f"fdm3d_100_b{b}_f32"] = {"ms": ms3, "alg_bytes": by, "GBs": by / ms3 / 1e6, "shape": sh}
    pb.set_launch_shape(1, 8, 0)
    main = cases["fdm3d_100_b32_f32"]
    out["cases"] = cases
    out["roofline"] = {"bound": "hbm", "achieved": main["GBs"], "peak": peak, "unit": "GB/s",
                       "frac": main["GBs"] / peak, "traffic": None,
                       "traffic_note": "DRAM bytes per launch of this case are in profiles/k_spmm_fdm3d_100_b32.md "
                                       "(ncu, not captured live)",
                       "kernel": "k_spmm: Y = (A^T + pI) X, CSR, 7-point 100^3 operator (n=1e6, nnz=6.94e6), "
                                 "32 FP32 columns, difference form, L2 flushed; measured on the launching stream "
                                 f"with launch shape (vectors/thread, CTAs/SM, row blocks) = {main['shape']}"}
    return out


if __name__ == "__main__":
    main()
