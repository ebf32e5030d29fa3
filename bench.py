"""Benchmark: INLA f + grad evaluations per second on one GB300.

Workload: univariate spatio-temporal model on a 32x32 grid (b = 1024),
n_t = 50 time blocks, a = 6 fixed effects, d = 4, 1e5 observations
(seeded synthetic data).  One step = one call of inla_value_and_grad (all
of the hot path: assembly of Q_p and Q_c, both BTA factorisations, the
solve for x*, f, both in-place selected inversions with the fused Phase A/C
traces, Phase B and the explicit terms).  The working set (two factors of
0.84 GB each) is far larger than L2, so no flush is needed between steps.

Also reported: the 2d+1 central finite-difference gradient (value-only
evaluations) on the same GPU, the FP64 efficiency of the whole step, the
roofline of the dominant kernel (the FP64 tile GEMM at the sweep's block
shape, timed live), and the FP64 CPU oracle on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "INLA f+∇f evals/s on 1 GB300: AD vs 2d+1 FD; % FP64 TC peak; rel err vs FP64"
UNIT = "gradient evaluations/s"
WORKLOAD = "st_medium"
# FP64 peak of the arithmetic unit the path uses (DFMA, "alu"): 152 SMs x 2 FP64
# FMA/clock/SM x 2 flop x 2.07 GHz maximum SM clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def reduce_replicas(times, dist=None, device="cpu"):
    """Replica timing over ranks: each entry becomes its maximum over all ranks
    (the slowest replica sets the step time).  Without a process group the
    times are returned unchanged."""
    if dist is None or dist.get_world_size() == 1:
        return [float(t) for t in times]
    import torch
    tt = torch.tensor([float(t) for t in times], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return [float(v) for v in tt.tolist()]


def _flops_model(b, n, a):
    """Algorithmic FP64 flops of one f+grad and of one value-only evaluation
    with the block kernels as implemented (per matrix and block: factor
    8/3 b^3 = SYRK b^3 + POTRF b^3/3 + TRTRI b^3/3 + TRMM b^3; selected
    inversion 13/3 b^3), arrow terms O(a b^2) included."""
    b3 = float(b) ** 3
    fwd = 2 * n * (8.0 / 3.0) * b3 + n * (4 * a * b * b)
    bwd = 2 * n * (13.0 / 3.0) * b3 + n * (6 * a * b * b)
    return fwd + bwd, fwd


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self):
        self.rows = []
        self._stop = threading.Event()
        self._proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            idx = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", idx, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self._proc = None

    def _read(self):
        for line in self._proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, nm in enumerate(names):
                if len(r) > 4 + i and r[4 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def cpu_baseline(seconds_hint: float = 20.0):
    """The FP64 oracle's block sweep (f and gradient) on a bounded sample of
    the workload: the same 32x32-grid model with 6 of its 50 time blocks;
    the per-block cost is constant, so the full-size time is the sample's
    time x 50/6."""
    import workloads
    from oracle import bta
    prob = workloads.make_problem("st_medium_nt6")
    t0 = time.perf_counter()
    bta.evaluate(prob)
    dt = time.perf_counter() - t0
    full = workloads.WORKLOADS[WORKLOAD]["nt"]
    t_full = dt * full / prob.nt
    return {"value": 1.0 / t_full, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"oracle f+grad on the {WORKLOAD} model cut to nt={prob.nt} of {full} "
                      f"time blocks ({dt:.1f} s), scaled by {full}/{prob.nt}",
            "seconds_per_gradient": t_full}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times = []
    cb = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline()
        if i >= args.warmup:
            times.append(cb["seconds_per_gradient"])
    t = float(np.mean(times))
    line = {"impl": "reference", "metric": METRIC, "value": 1.0 / t, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": "32x32", "b": 1024, "nt": 50, "a": 6,
                       "d": 4, "n_obs": 100000},
            "cpu_baseline": {"value": 1.0 / t, "unit": UNIT, "cores": cb["cores"],
                             "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": 1.0 / t, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def gemm_roofline(P, torch, b, reps=5, mixed=0):
    """Average duration of the FP64 tile GEMM (mixed=1: the split-TF32
    tensor-core GEMM with its operand splitting; mixed=2: the FP64 GEMM
    emulated from 8 BF16 slices, splitting included) at the sweep's dense
    block shape (b x b x b, the Z_B = -Z_D,i+1 F_B product of the selected
    inversion), timed with CUDA events on its launch stream."""
    import ctypes as C
    from paper_2605_06392_gb300._capi import lib
    A = torch.randn(b, b, dtype=torch.float64, device="cuda")
    B = torch.randn(b, b, dtype=torch.float64, device="cuda")
    Cm = torch.zeros(b, b, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()

    def one():
        if not mixed:
            P.bta_gemm(A, B, Cm, stream=s)
        elif mixed == 2:
            lib().bta_gemm_emulated(b, b, b, 1.0, C.c_void_p(A.data_ptr()), b, 0,
                                    C.c_void_p(B.data_ptr()), b, 0, 0.0,
                                    C.c_void_p(Cm.data_ptr()), b, 8, C.c_void_p(st.data_ptr()),
                                    C.c_void_p(s.cuda_stream))
        else:
            lib().bta_gemm_mixed(b, b, b, 1.0, C.c_void_p(A.data_ptr()), b, 0,
                                 C.c_void_p(B.data_ptr()), b, 0, 0.0, C.c_void_p(Cm.data_ptr()),
                                 b, C.c_void_p(st.data_ptr()), C.c_void_p(s.cuda_stream))
    for _ in range(2):
        one()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        one()
    e1.record(s)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flops = 2.0 * b ** 3
    return ms, flops / (ms * 1e-3) / 1e12


def run_batch(args, P, torch, workloads):
    """Independent coregionalised models of uneven block size (3 responses,
    grid side drawn from --grids, --batch-nt time blocks, d = 15), each at
    its own theta: one CUDA graph for all of them against one call per
    model.  Prints one JSON line."""
    grids = tuple(int(v) for v in args.grids.split(","))
    probs = workloads.make_batch(args.instances, grids=grids, nt=args.batch_nt)
    models = [P.InlaModel(p) for p in probs]
    thetas = [p.theta for p in probs]
    prec = args.precision
    for m, p in zip(models, probs):                 # capture each model's graph
        m.value_and_grad(p.theta, precision=prec)
    batch = P.InlaBatch(models)
    batch.value_and_grad(thetas, precision=prec)    # capture the batch graph
    torch.cuda.synchronize()
    reps = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(reps):
        fs = [m.value_and_grad(p.theta, precision=prec)[0] for m, p in zip(models, probs)]
    t_seq = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        fb, gb = batch.value_and_grad(thetas, precision=prec)
    t_batch = (time.perf_counter() - t0) / reps
    same = bool(np.all(np.array(fs) == fb))
    b_list = [int(p.b) for p in probs]
    flops = sum(14.0 * b ** 3 * p.nt for b, p in zip(b_list, probs))
    print(json.dumps({
        "mode": "batch", "instances": len(probs), "grids": list(grids), "nt": args.batch_nt,
        "b_values": sorted(set(b_list)), "b_counts": {str(v): b_list.count(v) for v in set(b_list)},
        "precision": {0: "f64", 1: "mixed", 2: "emulated f64"}[prec], "reps": reps,
        "seconds_sequential": t_seq, "seconds_one_graph": t_batch,
        "speedup_one_graph": t_seq / t_batch, "gradients_per_s_one_graph": len(probs) / t_batch,
        "identical_results": same, "algorithmic_tflop": flops / 1e12,
        "achieved_tflops_one_graph": flops / t_batch / 1e12}), flush=True)
    batch.close()
    for m in models:
        m.close()


def run_step(args, prob, model, theta, torch, stream):
    """Value-and-gradient steps at one precision (0 FP64, 1 mixed, 2 emulated
    FP64), the timed ones inside the profiler range (for launch lists); then,
    outside it, the 2d+1 value-only evaluations of the FD gradient."""
    for _ in range(args.warmup):
        model.value_and_grad(theta, precision=args.precision)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.cudart().cudaProfilerStart()
    e0.record(stream)
    for _ in range(args.steps):
        f, g = model.value_and_grad(theta, precision=args.precision)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    ms = e0.elapsed_time(e1) / args.steps
    flops, fwd = _flops_model(prob.b, prob.nt, prob.a)
    out = {"mode": "step", "workload": args.workload, "b": prob.b, "nt": prob.nt,
           "low_memory": bool(args.low_memory),
           "precision": args.precision, "ms_per_step": ms, "f": f,
           "algorithmic_tflop_per_step": flops / 1e12,
           "tflops_fp64_equivalent": flops / ms / 1e9,
           "frac_of_fp64_peak": flops / ms / 1e9 / FP64_PEAK_TFLOPS}
    if args.step_fd:
        d = len(theta)
        pts = [theta] + [theta + s * 1e-3 * np.eye(d)[j] for j in range(d) for s in (1.0, -1.0)]
        model.value_and_grad(theta, grad=False, precision=args.precision)
        torch.cuda.synchronize()
        e0.record(stream)
        for q in pts:
            model.value_and_grad(q, grad=False, precision=args.precision)
        e1.record(stream)
        e1.synchronize()
        fd_ms = e0.elapsed_time(e1)
        out.update({"fd_ms_per_gradient": fd_ms, "speedup_ad_vs_fd": fd_ms / ms,
                    "c_ad": ms / (fd_ms / len(pts))})
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fd-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--nt", type=int, default=0,
                    help="override the number of time blocks (profiling a shorter copy of "
                         "the same model: identical per-block kernels)")
    ap.add_argument("--instances", type=int, default=31, help="batch mode: number of models")
    ap.add_argument("--grids", default="16,24,32", help="batch mode: grid sides drawn per model")
    ap.add_argument("--batch-nt", type=int, default=40, help="batch mode: time blocks per model")
    ap.add_argument("--precision", type=int, default=0,
                    help="batch / gemm / step modes: 0 FP64, 1 mixed, 2 emulated FP64")
    ap.add_argument("--mode", default="full", choices=["full", "gemm", "batch", "step"],
                    help="gemm: only the dominant kernel at the sweep's block shape "
                         "(the small case used for ncu captures); step: only the timed "
                         "value-and-gradient steps at --precision, inside the profiler range")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="step mode: the synthetic model (a name from workloads.WORKLOADS)")
    ap.add_argument("--gemm-n", type=int, default=0,
                    help="gemm mode: the product's size n (n x n x n; default the block size)")
    ap.add_argument("--low-memory", action="store_true",
                    help="step mode: the model keeps only the diagonal factors (low-memory sweeps)")
    ap.add_argument("--step-fd", action="store_true",
                    help="step mode: also time the 2d+1 value-only evaluations of FD")
    args = ap.parse_args()
    if args.warmup < 3 and args.mode == "full":
        args.warmup = 3
    args.warmup = max(args.warmup, 1)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    import paper_2605_06392_gb300 as P
    import workloads

    if args.mode == "batch":
        return run_batch(args, P, torch, workloads)
    if args.mode == "gemm":
        b = args.gemm_n or workloads.WORKLOADS[WORKLOAD]["nx"] * workloads.WORKLOADS[WORKLOAD]["ny"]
        ms, tf = gemm_roofline(P, torch, b, reps=args.steps, mixed=args.precision)
        name = {0: "gemm_f64_kernel", 1: "tc_gemm_tf32x3_kernel (+ split)",
                2: "ozaki_gemm_kernel<8> (+ split)"}[args.precision]
        print(json.dumps({"kernel": name, "shape": [b, b, b], "launch_ms": ms,
                          "tflops_fp64_equivalent": tf}), flush=True)
        return

    prob = workloads.make_problem(args.workload if args.mode == "step" else WORKLOAD,
                                  **({"nt": args.nt} if args.nt else {}))
    model = P.InlaModel(prob, low_memory=args.low_memory and args.mode == "step")
    theta = prob.theta.copy()
    stream = torch.cuda.current_stream()
    if args.mode == "step":
        return run_step(args, prob, model, theta, torch, stream)
    # warm-up (also captures the CUDA graphs)
    for _ in range(args.warmup):
        f, g = model.value_and_grad(theta)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # --- timed region: K gradient evaluations, device time by CUDA events
    clocks = ClockSampler()
    clocks.start()
    barrier()
    k0 = model.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    host_times = []
    torch.cuda.cudart().cudaProfilerStart()         # profiler range = the timed steps
    e0.record(stream)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        f, g = model.value_and_grad(theta)          # host theta in, host f/grad out
        host_times.append(time.perf_counter() - t0)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    barrier()
    clocks.stop()
    launches = model.kernel_launches() - k0
    ms = e0.elapsed_time(e1) / args.steps
    t_step = ms * 1e-3
    t_step, t_host = reduce_replicas([t_step, float(np.mean(host_times))], dist, device="cuda")
    value = world / t_step
    e2e = world / t_host

    # --- FD baseline: 2d+1 value-only evaluations per gradient, same GPU
    pts = workloads.fd_stencil(theta, 1e-3)
    t_fd, g_fd, t_fdb = float("nan"), np.full(prob.d, np.nan), float("nan")
    if args.fd_steps > 0:
        model.value_and_grad(pts[:2], grad=False)       # warm the value-only graph
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.fd_steps):
            fv, _ = model.value_and_grad(pts, grad=False)
        t_fd = (time.perf_counter() - t0) / args.fd_steps
        g_fd = (fv[1::2] - fv[2::2]) / 2e-3
        # batched: all 2d+1 evaluations swept together in the same launches
        model.value_and_grad(pts, grad=False, concurrent=pts.shape[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.fd_steps):
            fvb, _ = model.value_and_grad(pts, grad=False, concurrent=pts.shape[0])
        t_fdb = (time.perf_counter() - t0) / args.fd_steps

    # --- mixed precision (tensor-core split-TF32 Schur products, FP64 diagonal
    # factors / log-dets / refinement): time and error against the FP64 path
    f, g = model.value_and_grad(theta)              # FP64 at theta (after the FD points)
    x64 = model.mode().cpu().numpy()
    parts64 = model.last_parts()
    for _ in range(2):
        fm, gm = model.value_and_grad(theta, precision=1)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        fm, gm = model.value_and_grad(theta, precision=1)
    e1.record(stream)
    e1.synchronize()
    t_mixed = e0.elapsed_time(e1) / args.steps * 1e-3
    xm = model.mode().cpu().numpy()
    pm = model.last_parts()
    gscale = np.maximum(np.abs(g), np.abs(parts64["phase_a"]) + np.abs(parts64["phase_b"]) +
                        np.abs(parts64["phase_c"]))
    mixed = {"ms_per_step": 1e3 * t_mixed, "gradients_per_s": 1.0 / t_mixed,
             "speedup_vs_fp64": t_step / t_mixed,
             "rel_err_f": abs(fm - f) / abs(f),
             "rel_err_x": float(np.max(np.abs(xm - x64)) / np.max(np.abs(x64))),
             "rel_err_grad": [float(v) for v in np.abs(gm - g) / gscale],
             "reference": "FP64 GPU path of this run (itself within 1e-10 of the FP64 oracle)"}
    del pm

    # --- emulated FP64 (the b x b products from 8 BF16 slices on the tensor
    # cores, everything else FP64): time and difference from the FP64 path
    emulated = None
    if prob.b <= 5120:
        for _ in range(2):
            fe, ge = model.value_and_grad(theta, precision=2)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            fe, ge = model.value_and_grad(theta, precision=2)
        e1.record(stream)
        e1.synchronize()
        t_emu = e0.elapsed_time(e1) / args.steps * 1e-3
        xe = model.mode().cpu().numpy()
        emulated = {"ms_per_step": 1e3 * t_emu, "gradients_per_s": 1.0 / t_emu,
                    "speedup_vs_fp64": t_step / t_emu,
                    "rel_err_f": abs(fe - f) / abs(f),
                    "rel_err_x": float(np.max(np.abs(xe - x64)) / np.max(np.abs(x64))),
                    "rel_err_grad": [float(v) for v in np.abs(ge - g) / gscale],
                    "reference": "FP64 GPU path of this run"}

    # --- dominant kernel roofline
    gemm_ms, gemm_tf = gemm_roofline(P, torch, prob.b)

    parts = parts64          # the FP64 evaluation at theta
    flops_grad, flops_val = _flops_model(prob.b, prob.nt, prob.a)
    step_tf = flops_grad / t_step / 1e12
    out = None
    if rank == 0:
        cpu = None if args.no_cpu else cpu_baseline()
        if cpu is not None:
            cpu.pop("seconds_per_gradient", None)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if not args.nt else f"{WORKLOAD}_nt{args.nt}",
                       "grid": "32x32", "b": prob.b, "ld": model.ld,
                       "nt": prob.nt, "a": prob.a, "d": prob.d, "n_obs": prob.n_obs,
                       "l2": "working set 1.7 GB > L2, no flush", "parallelism": "replicas"},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * prob.d,
                    "d2h_bytes_per_step": 8 * (1 + prob.d + 8 + 4 * prob.d)},
            "gpu_launches": int(launches),
            "fd_baseline": {"seconds_per_gradient": t_fd, "evals_per_gradient": pts.shape[0],
                            "gradients_per_s": 1.0 / t_fd,
                            "speedup_ad_vs_fd": t_fd / t_step,
                            "c_ad": t_step / (t_fd / pts.shape[0]),
                            "batched_seconds_per_gradient": t_fdb,
                            "speedup_ad_vs_batched_fd": t_fdb / t_step,
                            "max_rel_diff_fd_vs_ad": float(np.max(np.abs(g_fd - g) /
                                                                  np.maximum(np.abs(g), 1.0)))},
            "mixed_precision": mixed,
            "emulated_fp64": emulated,
            "fp64_step": {"algorithmic_tflop_per_step": flops_grad / 1e12,
                          "achieved_tflops": step_tf, "frac_of_peak": step_tf / FP64_PEAK_TFLOPS},
            "roofline": {"bound": "alu", "kernel": "gemm_f64_kernel<32,32> at b x b x b",
                         "achieved": gemm_tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": gemm_tf / FP64_PEAK_TFLOPS, "traffic": 16.8e6,
                         "traffic_source": "ncu dram__bytes_read+write per launch, "
                                           "profiles/gemm_f64_block1024.md",
                         "launch_ms": gemm_ms,
                         "peak_source": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz"},
            "clocks": clocks.summary(),
            "result": {"f": f, "grad": [float(v) for v in g], "logdet_c": parts["logdet_c"],
                       "logdet_p": parts["logdet_p"]},
        }
        if cpu is not None:
            out["cpu_baseline"] = cpu
        print(json.dumps(out), flush=True)
    model.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
