#!/usr/bin/env python
"""Leaf DtN build throughput on one GB300: boxes/s and algorithmic TFLOP/s.

Workload: the 8 x 8 x 8 grid of leaf boxes of the unit cube (h = 1/8) at
p = 16 (n = 2744 interior, m = 1176 face nodes per box), kappa = 40, b a
seeded sum of 16 random Fourier modes clipped to [0.5, 1.5] (seed 20250304).
One step = hps_leaf_build_dtn over all 512 boxes: operator assembly, FP32 LU
with tcgen05 tensor-core update products, FP64 iterative refinement of
S = -A_ii^{-1} A_ib, and the FP64 D_n product T = A_bb + A_bi S.  Inputs are
resident in HBM; the working set (~90 GB) is far larger than L2, so no L2
flush is needed between steps.

Also reported: the plain FP64 GPU path on a 32-box sample of the same
workload (speedup and max relative difference), the end-to-end rate through
the C ABI with host buffers (b uploaded from pinned memory and T written by
the call into pinned host memory, both inside the timed region; the same
with an explicit T download beside it),
per-kernel-class CUDA-event timings with the roofline of the dominant class,
and the FP64 CPU oracle's rate on a bounded sample of boxes.

``--impl reference`` times the FP64 CPU oracle (the only reference this
paper has; it has no code) on the same workload and metric.

Other workloads (``--workload``), each printing its own JSON line: ``uneven``
(1024 boxes of mixed p and kappa with 32 loads), ``learned`` (the learned
low-rank DtN correction at p = 12), ``factored`` (stored factorisations, 32
loads per box), ``timestep`` (Crank-Nicolson steps with every stage on the
GPU, or the interface on the host with ``--interface host``), ``dirichlet``
(the two-stage solve of 8 x 8 x 8 boxes at p = 12 with the GPU interface
factorisation), ``accuracy`` (the Sec. 4.1 Green's-function study) and
``leaf2d`` (the 2-D leaf reduction).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import hps_inputs as hi  # noqa: E402

P, NBOX, KAPPA, GRID = 16, 512, 40.0, (8, 8, 8)
WORKLOAD = ("8x8x8 leaf boxes of the unit cube, p=16 Chebyshev-Lobatto (n=2744, m=1176), kappa=40, "
            "b = clip(1 + 0.5 * sum of 16 seeded Fourier modes |k|<=4, [0.5, 1.5]), seed 20250304")
METRIC = "leaf DtN builds/s at p=16 (FP32 tcgen05 LU + FP64 refinement, rel err <= 1e-10 vs FP64)"

# TF32 dense tensor peak derived from the measured BF16 peak and NVIDIA's
# nominal TF32:BF16 ratio (1.1 : 2.25 PFLOP/s dense).
TF32_OVER_BF16 = 1.1 / 2.25


def operand_format(prec, opts):
    """(name, MMA rate relative to BF16, MMAs per product) of the tensor-core
    update products for a precision and the --opt settings."""
    import paper_2503_04033_gb300 as H
    if prec == H.HPS_BF16_IR:
        return "3 x BF16", 1.0, 6
    if float(opts.get("FP16_OPERANDS", 1)) != 0:
        return "scaled 2 x FP16", 1.0, 3
    return "3 x TF32", TF32_OVER_BF16, 3
# FP64 issue rate: 152 SMs x 2070 MHz x 2 FP64 FMA/clk/SM x 2 flop (1.26
# TFLOP/s, the part's nominal 1.25 TFLOP/s); used only where a run has not
# measured its own FP64 matmul rate.
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 2 * 2 / 1e12
# DRAM bytes per launch of the tensor-core update products at 512 boxes, by
# operand format: dram__bytes_read.sum + dram__bytes_write.sum of one ncu
# capture of the factorisation phase at 32 boxes, per launch, times 16 (the
# traffic grows with the boxes).  None when not captured for the current
# kernel: every change to the product kernel resets it to None until it is
# captured again.
NCU_TRAFFIC_PER_LAUNCH = {("update_tcgen05", "scaled 2 x FP16"): 2.2486e9, ("update_tcgen05", "3 x TF32"): None}


def dtype_label(prec, opts):
    """Arithmetic of the path: the split operand format of the tensor-core
    products (FP32 accumulation) plus the FP64 refinement and D_n."""
    import paper_2503_04033_gb300 as H
    if prec == H.HPS_FP64:
        return "f64"
    fmt = operand_format(prec, opts)[0]
    return {"scaled 2 x FP16": "fp16x2 (f32 accumulate)+f64", "3 x TF32": "tf32x2 (f32 accumulate)+f64",
            "3 x BF16": "bf16x3 (f32 accumulate)+f64"}[fmt]


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("fp32ir", "bf16ir", "fp64"), default="fp32ir")
    ap.add_argument("--nbox", type=int, default=NBOX)
    ap.add_argument("--fp64-sample", type=int, default=32)
    ap.add_argument("--cpu-sample", type=int, default=32)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-alt", action="store_true", help="skip timing the other mixed precision")
    ap.add_argument("--no-uneven", action="store_true", help="skip the uneven-batch measurement in the headline run")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-correction measurement in the headline run")
    ap.add_argument("--opt", action="append", default=[], metavar="NAME=VALUE",
                    help="hps_set_option before timing, e.g. LU_UNIT=2 (name without HPS_OPT_)")
    ap.add_argument("--workload", choices=("fourier16", "uneven", "learned", "factored", "timestep", "dirichlet",
                                                 "accuracy", "leaf2d", "cross", "iti"),
                    default="fourier16",
                    help="fourier16: the p=16 headline workload; uneven: 1024 boxes of mixed p/kappa with 32 "
                         "loads; learned: the learned DtN correction at p=12")
    ap.add_argument("--train-boxes", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--gate-tol", type=float, default=3e-3)
    ap.add_argument("--nb", type=int, default=8, help="dirichlet workload: boxes per axis")
    ap.add_argument("--leaf-prec", choices=("fp32ir", "fp64"), default="fp32ir",
                    help="timestep workload: precision of the stored leaf factors")
    ap.add_argument("--interface", choices=("gpu", "host"), default="gpu",
                    help="timestep workload: interface solve on the GPU (nested dissection) or a host sparse LU")
    ap.add_argument("--ir-tol", type=float, default=None,
                    help="refinement tolerance (HPS_OPT_IR_TOL); library default when omitted")
    return ap.parse_args()


def aggregate_step_ms(ms: float, world: int, device) -> float:
    """The step time the job reports: the maximum over ranks (every rank
    processes its own boxes; no data crosses ranks)."""
    if world == 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def box_lows():
    lows, h = hi.box_grid_lo(GRID)
    return lows, h


def flops_per_box(p: int) -> float:
    """The dense method's count: LU 2/3 n^3 + TRSM 2 n^2 m + structured D_n 2 q m^2."""
    q = p - 2
    n, m = q ** 3, 6 * q * q
    return 2.0 / 3.0 * n ** 3 + 2.0 * n * n * m + 2.0 * q * m * m


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def measured_matmul_peaks(dev):
    """Dense matmul rates measured here with torch (cuBLAS): FP64 at 4096^3
    and FP16 / BF16 at 8192^3, best of 5 after a warm-up, CUDA events.  The
    FP64 figure is the peak of the plain FP64 GPU path and the FP64 kernels;
    the FP16 one checks that FP16 runs at the BF16 rate."""
    import torch
    out = {}
    for name, dt, nn, reps in (("fp64_tflops", torch.float64, 4096, 3), ("fp16_tflops", torch.float16, 8192, 5),
                               ("bf16_tflops", torch.bfloat16, 8192, 5)):
        a = torch.randn(nn, nn, dtype=dt, device=dev)
        bm = torch.randn(nn, nn, dtype=dt, device=dev)
        c = a @ bm
        best = 1e30
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c = a @ bm
            e1.record()
            torch.cuda.synchronize(dev)
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[name] = 2.0 * nn ** 3 / best / 1e12
        del a, bm, c
    torch.cuda.empty_cache()
    out["how"] = "torch.matmul best of several, CUDA events; FP64 4096^3, FP16/BF16 8192^3 (burst)"
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.out is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.out.seek(0)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.out.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def oracle_rate(nbox_sample: int, threads: int | None = None):
    """Boxes/s of the FP64 CPU oracle (as it stands) on the first boxes of the workload."""
    import oracle
    lows, h = box_lows()
    field = hi.fourier_b_field()
    sel = np.linspace(0, NBOX - 1, nbox_sample).astype(int)
    bs = [field.b(oracle.node_coords(P, lows[i], h)) for i in sel]
    t0 = time.perf_counter()
    for b in bs:
        _, _, info = oracle.leaf_dtn(P, h, KAPPA, b, want_S=False)
        assert info == 0
    dt = time.perf_counter() - t0
    return nbox_sample / dt, dt, oracle.max_threads()


def lapack_rate(nbox_sample: int):
    """Boxes/s of a LAPACK-based CPU path on the first boxes of the workload:
    the oracle's collocation matrix, then numpy's threaded LU solve for S and
    one product for T = A_bb + A_bi S (a second, stronger CPU baseline for
    context; the oracle is the one the contract names)."""
    import oracle
    lows, h = box_lows()
    field = hi.fourier_b_field()
    n, m = oracle.sizes(P)
    sel = np.linspace(0, NBOX - 1, nbox_sample).astype(int)
    bs = [field.b(oracle.node_coords(P, lows[i], h)) for i in sel]
    t0 = time.perf_counter()
    for b in bs:
        A = oracle.leaf_matrix(P, h, KAPPA, b)
        S = np.linalg.solve(A[:n, :n], -A[:n, n:])
        T = A[n:, n:] + A[n:, :n] @ S
        assert np.isfinite(T).all()
    dt = time.perf_counter() - t0
    return nbox_sample / dt, dt


def run_reference(args):
    """The oracle on the host cores: each step is one box of the workload (the
    oracle's LU and solves use every core), W untimed, K timed."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    lows, h = box_lows()
    field = hi.fourier_b_field()
    for i in range(args.warmup):
        oracle.leaf_dtn(P, h, KAPPA, field.b(oracle.node_coords(P, lows[i], h)), want_S=False)
    times = []
    for s in range(args.steps):
        b = field.b(oracle.node_coords(P, lows[(7 * s + 3) % NBOX], h))
        t0 = time.perf_counter()
        _, _, info = oracle.leaf_dtn(P, h, KAPPA, b, want_S=False)
        times.append(time.perf_counter() - t0)
        assert info == 0
    ms = 1e3 * sum(times) / len(times)
    value = 1e3 / ms
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "boxes/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nbox_per_step": 1, "p": P, "kappa": KAPPA},
        "tflops": value * flops_per_box(P) / 1e12,
        "cpu_baseline": {"value": value, "unit": "boxes/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} boxes of the workload, one per step, FP64 oracle LU + solves "
                                   f"with OpenMP over {cores} threads"},
        "e2e": {"value": value, "unit": "boxes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist
    import paper_2503_04033_gb300 as H

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    def allmax(x: float) -> float:
        return aggregate_step_ms(x, world, dev)

    nbox = args.nbox
    lows, h = box_lows()
    lows = lows[np.arange(nbox) % NBOX]
    field = hi.fourier_b_field()
    b_np = np.stack([field.b(H.hps_leaf_nodes(P, lo, h)) for lo in lows])
    n, m = H.hps_leaf_sizes(P)
    prec = {"fp32ir": H.HPS_FP32_IR, "bf16ir": H.HPS_BF16_IR, "fp64": H.HPS_FP64}[args.precision]
    kind = H.LeafKind(P, h, KAPPA)
    ctx = H.hps_create(local, 0)
    if args.ir_tol is not None:
        H.hps_set_option(ctx, H.HPS_OPT_IR_TOL, args.ir_tol)
    opts = dict(o.split("=") for o in args.opt)
    for name, val in opts.items():
        H.hps_set_option(ctx, getattr(H, "HPS_OPT_" + name), float(val))
    stream = torch.cuda.current_stream(dev)
    b = torch.from_numpy(b_np).to(dev)
    T = torch.empty(nbox, m, m, dtype=torch.float64, device=dev)
    st = torch.zeros(nbox, dtype=torch.int32, device=dev)

    def step():
        H.hps_leaf_build_dtn(ctx, kind, nbox, b, T, None, prec, st, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    bad = int((st != 0).sum().item())

    # ---- timed region (device-resident inputs), per-kernel events on the stream
    H.hps_profile_enable(ctx, True)
    H.hps_profile_reset(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    with ClockSampler(local) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    barrier()
    ms = allmax(e0.elapsed_time(e1) / args.steps)
    H.hps_profile_enable(ctx, False)
    prof = {}
    launches_total = 0
    for cls, name in enumerate(H.KERNEL_CLASSES):
        nl, kms, fl, by = H.hps_profile_get(ctx, cls)
        if nl:
            prof[name] = {"launches": nl // args.steps, "ms_per_step": kms / args.steps, "flops": fl / args.steps,
                          "bytes": by / args.steps}
            launches_total += nl
    value = world * nbox / (ms / 1e3)
    it, rel = H.hps_last_refinement(ctx, nbox)

    line = {
        "metric": METRIC, "value": value, "unit": "boxes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype_label(prec, opts), "data": "synthetic",
        "config": {"workload": WORKLOAD, "nbox_per_gpu": nbox, "p": P, "kappa": KAPPA,
                   "precision": args.precision, "ir_tol": args.ir_tol, "options": args.opt, "l2": "inputs larger than L2 (~90 GB working set), no flush",
                   "step": "hps_leaf_build_dtn over all boxes (T out, S not stored)"},
        "tflops": value * flops_per_box(P) / 1e12,
        "wall_ms_per_step": 1e3 * wall / args.steps,
        "box_failures": bad,
        "refinement": {"corrections_max": int(it.max()), "corrections_mean": float(it.mean()),
                       "corrections_hist": {int(v): int((it == v).sum()) for v in np.unique(it)},
                       "rel_correction_max": float(rel.max())},
        "gpu_launches": launches_total // args.steps * args.steps,
        "kernels": prof,
        "clocks": clocks.summary(),
    }

    # ---- roofline of the dominant contraction (the mixed path is
    # tensor-bound).  The tensor-core update products do the method's LU and
    # triangular solves: their algorithmic work is 2/3 n^3 + 2 n^2 m per box,
    # counted once (the split operand formats issue several MMAs per product),
    # less the panel factorisation's share, which runs on CUDA cores.
    peaks, src = measured_peaks()
    mm = measured_matmul_peaks(dev)
    line["measured_matmul_peaks"] = mm
    fmt_name, rate, nmma = operand_format(prec, opts)
    if prec == H.HPS_FP64:
        tpeak, tsrc = mm["fp64_tflops"], "torch float64 matmul measured in this run (4096^3)"
    else:
        tpeak = peaks["bf16_tflops_sustained"] * rate
        tsrc = (f"{src} sustained BF16 dense peak" + (" (FP16 has the same nominal rate)" if rate == 1.0 else
                                                       f" x {rate:.3f} (nominal TF32:BF16)"))
    qh = P - 2
    n_, m_ = qh ** 3, 6 * qh * qh
    lu_trsm = nbox * (2.0 / 3.0 * n_ ** 3 + 2.0 * n_ * n_ * m_)
    tc_cls = "update_tcgen05" if "update_tcgen05" in prof else ("update_cudacore" if "update_cudacore" in prof else None)
    if tc_cls is not None:
        d = prof[tc_cls]
        panel_fl = prof.get("panel", {}).get("flops", 0.0)
        alg = lu_trsm - panel_fl
        sec = d["ms_per_step"] / 1e3
        ach = alg / sec / 1e12
        traffic = (NCU_TRAFFIC_PER_LAUNCH.get((tc_cls, fmt_name))
                   if (nbox == NBOX and prec == H.HPS_FP32_IR and not opts) else None)
        line["roofline"] = {
            "kernel": tc_cls, "bound": "tensor", "achieved": ach, "peak": tpeak, "unit": "TFLOP/s",
            "frac": ach / tpeak, "traffic": traffic,
            "algorithmic_flops_per_launch": alg / max(d["launches"], 1), "launches_per_step": d["launches"],
            "ms_per_step": d["ms_per_step"],
            "flops_definition": "(2/3 n^3 + 2 n^2 m) per box x boxes, counted once, less the panel kernel's "
                                "CUDA-core flops; per launch = that / launches",
            "peak_source": tsrc + "; of measured",
            "mma_issue_frac": ach * nmma / tpeak,
            "mma_issue_note": f"{fmt_name}: {nmma} MMAs per product, so the tensor pipe issues {nmma}x the "
                              "algorithmic rate",
            "hbm_view": {"achieved_gbs": d["bytes"] / sec / 1e9, "peak_gbs": peaks["hbm_gbs"],
                         "frac": d["bytes"] / sec / 1e9 / peaks["hbm_gbs"],
                         "note": "bytes the products move by construction (split operands, source and output "
                                 "tiles), not the method's algorithmic bytes"},
            "traffic_source": ("dram__bytes_read.sum + dram__bytes_write.sum per launch from an ncu capture of "
                               "32 boxes, scaled by the box count to 512 (traffic grows with the boxes)"
                               if traffic is not None else "not captured for this configuration"),
        }
    line["roofline_step"] = {
        "achieved": line["tflops"], "peak": tpeak, "unit": "TFLOP/s", "frac": line["tflops"] / tpeak,
        "definition": "2/3 n^3 + 2 n^2 m + 2 q m^2 per box x boxes / ms_per_step (LU of A_ii, the solves for "
                      "S and the product A_bi S), against the same tensor peak",
        "algorithmic_bytes_per_box": 8.0 * P ** 3 + 8.0 * m_ * m_,
        "hbm_frac": nbox * (8.0 * P ** 3 + 8.0 * m_ * m_) / (ms / 1e3) / 1e9 / peaks["hbm_gbs"]}

    # ---- the FP64 residual (its launches skip converged boxes, so its work is
    # counted from the refinement histogram):
    # FP64 pipe instructions per (point, column) of the even/odd line form,
    # 3 (h + 2) + 3 with h = (p - 2) // 2 at even p - 2, against the issue
    # rate of the FP64 pipes (2 per clock per SM at the SM clock sampled).
    if "residual_fp64" in prof and prec != H.HPS_FP64 and float(opts.get("RESIDUAL_DF", 3)) in (0.0, 1.0, 2.0):
        q = P - 2
        per_entry = 3 * (q // 2 + 2) + 3 + (6 if q % 2 else 0)
        # FP64 residual evaluations per step (every step alike); with the
        # double-float first residual (on unless switched off) each box's
        # first evaluation runs on the FP32 pipes instead
        # FP64 evaluations: the launches skip converged boxes, so the work is
        # counted from the refinement histogram (less each box's double-float
        # first residual); only meaningful when every later residual is FP64
        df = float(opts.get("RESIDUAL_DF", 3)) != 0 and float(opts.get("IR_MAX_ITERS", 8)) >= 2
        box_its = float(it.sum()) - (nbox if df else 0)
        instr = box_its * n * m * per_entry
        rms = prof["residual_fp64"]["ms_per_step"]
        sm_mhz = (line.get("clocks") or {}).get("sm_mhz") or 2070.0
        peak_ips = 2.0 * torch.cuda.get_device_properties(dev).multi_processor_count * sm_mhz * 1e6
        line["roofline_fp64_residual"] = {
            "kernel": "residual_fp64", "bound": "alu", "achieved": instr / (rms / 1e3) / 1e9,
            "peak": peak_ips / 1e9, "unit": "G FP64-pipe instr/s", "frac": instr / (rms / 1e3) / peak_ips,
            "instr_per_entry": per_entry, "box_iterations_per_step": box_its,
            "peak_source": "2 FP64 instructions per clock per SM x SMs x sampled SM clock"}
    # ---- the double-float first residual (every box, one launch a step):
    # FP32 operations per (point, column) as written in the kernel: per axis
    # and output 12 h + 6 (exact butterfly, TwoProduct/TwoSum multiply-adds,
    # the even/odd recombination), 12 h + 12 at odd q, plus 28 to accumulate
    # the axes, the kappa^2 b term and round; against 128 FP32 lanes per SM.
    if "residual_df" in prof:
        q = P - 2
        hq = q // 2
        per_df = 3 * (12 * hq + (12 if q % 2 else 6)) + 28
        ops = float(nbox) * n * m * per_df
        rms = prof["residual_df"]["ms_per_step"]
        sm_mhz = (line.get("clocks") or {}).get("sm_mhz") or 2070.0
        peak_ops = 128.0 * torch.cuda.get_device_properties(dev).multi_processor_count * sm_mhz * 1e6
        line["roofline_df_residual"] = {
            "kernel": "residual_df", "bound": "alu", "achieved": ops / (rms / 1e3) / 1e9,
            "peak": peak_ops / 1e9, "unit": "G FP32 ops/s", "frac": ops / (rms / 1e3) / peak_ops,
            "ops_per_entry": per_df,
            "peak_source": "128 FP32 lanes per SM x SMs x sampled SM clock"}

    # ---- plain FP64 GPU path on a sample of the same boxes
    if not args.no_fp64 and prec != H.HPS_FP64 and args.fp64_sample > 0:
        k = min(args.fp64_sample, nbox)
        # half evenly spaced, half the boxes whose refinement ended with the
        # largest corrections (the hardest ones)
        worst = np.argsort(-(np.asarray(rel) * 10.0 ** np.asarray(it)))[: k // 2]
        even = np.linspace(0, nbox - 1, k).astype(np.int64)
        sel_np = np.unique(np.concatenate([worst, [i for i in even if i not in set(worst)][: k - len(worst)]]))
        k = len(sel_np)
        sel = torch.from_numpy(sel_np.astype(np.int64)).to(dev)
        b64 = b.index_select(0, sel).contiguous()
        T64 = torch.empty(k, m, m, dtype=torch.float64, device=dev)
        st64 = torch.zeros(k, dtype=torch.int32, device=dev)
        H.hps_leaf_build_dtn(ctx, kind, 2, b64, T64, None, H.HPS_FP64, st64, stream)   # warm
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        H.hps_leaf_build_dtn(ctx, kind, k, b64, T64, None, H.HPS_FP64, st64, stream)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        fp64_rate = k / (f0.elapsed_time(f1) / 1e3)
        Ts = T.index_select(0, sel)
        relerr = ((Ts - T64).flatten(1).norm(dim=1) / T64.flatten(1).norm(dim=1)).max().item()
        line["fp64_path"] = {"value": fp64_rate, "unit": "boxes/s", "sample_boxes": k,
                             "sample": "half evenly spaced, half the most-refined boxes",
                             "tflops": fp64_rate * flops_per_box(P) / 1e12,
                             "failures": int((st64 != 0).sum().item())}
        line["speedup_vs_fp64_path"] = value / world / fp64_rate
        line["rel_err_vs_fp64_path"] = relerr
        del T64, b64

    # ---- the other mixed precision on the same boxes (timed the same way)
    if prec != H.HPS_FP64 and not args.no_alt:
        alt = H.HPS_BF16_IR if prec == H.HPS_FP32_IR else H.HPS_FP32_IR
        Ta = torch.empty_like(T)
        sta = torch.zeros_like(st)
        for _ in range(2):
            H.hps_leaf_build_dtn(ctx, kind, nbox, b, Ta, None, alt, sta, stream)
        torch.cuda.synchronize(dev)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        a0.record(stream)
        for _ in range(args.steps):
            H.hps_leaf_build_dtn(ctx, kind, nbox, b, Ta, None, alt, sta, stream)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        alt_ms = allmax(a0.elapsed_time(a1) / args.steps)
        ita, rela = H.hps_last_refinement(ctx, nbox)
        rel_ab = ((Ta - T).flatten(1).norm(dim=1) / T.flatten(1).norm(dim=1)).max().item()
        line["other_precision"] = {
            "precision": "bf16ir" if alt == H.HPS_BF16_IR else "fp32ir", "value": world * nbox / (alt_ms / 1e3),
            "unit": "boxes/s", "ms_per_step": alt_ms, "box_failures": int((sta != 0).sum().item()),
            "corrections_mean": float(ita.mean()), "corrections_max": int(ita.max()),
            "max_rel_diff_vs_headline_T": rel_ab}
        del Ta, sta

    # ---- the same precision with every residual in FP64 (the double-float
    # first residual switched off), timed the same way
    if prec != H.HPS_FP64 and not args.no_alt and float(opts.get("RESIDUAL_DF", 3)) != 0:
        H.hps_set_option(ctx, H.HPS_OPT_RESIDUAL_DF, 0)
        Tf = torch.empty_like(T)
        stf = torch.zeros_like(st)
        for _ in range(2):
            H.hps_leaf_build_dtn(ctx, kind, nbox, b, Tf, None, prec, stf, stream)
        torch.cuda.synchronize(dev)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        a0.record(stream)
        for _ in range(args.steps):
            H.hps_leaf_build_dtn(ctx, kind, nbox, b, Tf, None, prec, stf, stream)
        a1.record(stream)
        torch.cuda.synchronize(dev)
        f_ms = allmax(a0.elapsed_time(a1) / args.steps)
        itf, _ = H.hps_last_refinement(ctx, nbox)
        rel_f = ((Tf - T).flatten(1).norm(dim=1) / T.flatten(1).norm(dim=1)).max().item()
        H.hps_set_option(ctx, H.HPS_OPT_RESIDUAL_DF, float(opts.get("RESIDUAL_DF", 3)))
        line["all_fp64_residuals"] = {
            "value": world * nbox / (f_ms / 1e3), "unit": "boxes/s", "ms_per_step": f_ms,
            "box_failures": int((stf != 0).sum().item()), "corrections_mean": float(itf.mean()),
            "max_rel_diff_vs_headline_T": rel_f,
            "note": "HPS_OPT_RESIDUAL_DF = 0: every residual in FP64 (the strict form of the refinement)"}
        del Tf, stf

    # ---- end to end through the C ABI with host buffers.  Every step uploads
    # its b from pinned host memory on a copy stream (double-buffered, events
    # order each buffer's uses) and its T reaches pinned host memory: in the
    # headline form the call writes T there itself (the D_n products store
    # across the host link, zero-copy), in the second form a download on its
    # own stream overlaps the next solve.
    if not args.no_e2e:
        b_host = torch.from_numpy(b_np).pin_memory()
        T_host = [torch.empty(nbox, m, m, dtype=torch.float64, pin_memory=True) for _ in range(2)]
        b_dev = [b, torch.empty_like(b)]
        T_dev = [T, torch.empty_like(T)]
        cs = torch.cuda.Stream(dev)    # uploads
        cd = torch.cuda.Stream(dev)    # downloads (explicit-copy form)

        def e2e_run(zero_copy):
            ev_in = [torch.cuda.Event() for _ in range(2)]    # b[j] is on the device
            ev_out = [torch.cuda.Event() for _ in range(2)]   # T[j] is computed (and, zero-copy, on the host)
            ev_free = [torch.cuda.Event() for _ in range(2)]  # T[j] has reached the host
            solve_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                        for _ in range(args.steps + 2)]

            def e2e_step(i, k):
                j = i & 1
                with torch.cuda.stream(cs):
                    cs.wait_event(ev_out[j])                   # the solve that last read b[j] is done
                    b_dev[j].copy_(b_host, non_blocking=True)
                    ev_in[j].record(cs)
                stream.wait_event(ev_in[j])
                stream.wait_event(ev_free[j])                  # T[j]'s previous copy has left the device
                solve_ev[k][0].record(stream)
                H.hps_leaf_build_dtn(ctx, kind, nbox, b_dev[j], T_host[j] if zero_copy else T_dev[j], None, prec,
                                     st, stream)
                ev_out[j].record(stream)
                solve_ev[k][1].record(stream)
                if zero_copy:
                    ev_free[j].record(stream)
                else:
                    with torch.cuda.stream(cd):
                        cd.wait_event(ev_out[j])
                        T_host[j].copy_(T_dev[j], non_blocking=True)
                        ev_free[j].record(cd)

            for i in range(2):
                ev_out[i].record(stream)
                ev_free[i].record(stream)
            e2e_step(0, 0)
            e2e_step(1, 1)
            torch.cuda.synchronize(dev)
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            with ClockSampler(local) as e2e_clocks:
                g0.record(stream)
                for i in range(args.steps):
                    e2e_step(i, i + 2)
                cd_done = torch.cuda.Event()
                cd_done.record(cd)
                stream.wait_event(cd_done)                      # the last T is on the host
                g1.record(stream)
                torch.cuda.synchronize(dev)
            e2e_ms = allmax(g0.elapsed_time(g1) / args.steps)
            solve_ms = statistics.median(a.elapsed_time(b) for a, b in solve_ev[2:])
            return e2e_ms, solve_ms, e2e_clocks.summary()

        e2e_ms, solve_ms, e2e_clk = e2e_run(True)
        Tz = T_host[(args.steps + 1) & 1].clone()
        cp_ms, cp_solve_ms, _ = e2e_run(False)
        same = bool(torch.equal(Tz, T_host[(args.steps + 1) & 1]))
        line["e2e"] = {"value": world * nbox / (e2e_ms / 1e3), "unit": "boxes/s",
                       "h2d_bytes_per_step": b_host.numel() * 8, "d2h_bytes_per_step": T_host[0].numel() * 8,
                       "ms_per_step": e2e_ms, "solve_ms_median": solve_ms, "clocks": e2e_clk,
                       "pipelining": "b uploads on a second stream overlap the previous solve; T is written by "
                                     "the call straight into pinned host memory (the D_n products store across "
                                     "the host link), so no download follows the solve",
                       "explicit_copy": {"value": world * nbox / (cp_ms / 1e3), "ms_per_step": cp_ms,
                                         "solve_ms_median": cp_solve_ms, "T_equal_to_zero_copy": same,
                                         "how": "T into device memory, then a cudaMemcpyAsync download on a "
                                                "third stream that overlaps the next solve"}}
        del T_host, b_host, b_dev, T_dev, Tz

    H.hps_destroy(ctx)   # the embedded measurements below make their own contexts
    torch.cuda.empty_cache()

    # ---- the uneven batch (mixed p, kappa per box, 32 loads), timed after the
    # headline on the same GPU, with its own schedule tuning
    if not args.no_uneven and world == 1:
        import tempfile as _tf
        tune_dir = _tf.mkdtemp()
        os.environ["HPS_TUNE_CACHE"] = os.path.join(tune_dir, "tune.txt")
        line["uneven_batch"] = uneven_measurement(3, 2, dev)
        del os.environ["HPS_TUNE_CACHE"]

    # ---- the learned correction at p = 12 (train on exact maps, serve gated)
    if not args.no_learned and world == 1:
        line["learned_surrogate"] = learned_measurement(args.train_boxes, args.epochs, args.gate_tol, 3, dev)

    # ---- the oracle on this host's cores (rank 0 at N = 1 only)
    if rank == 0 and world == 1 and not args.no_cpu and args.cpu_sample > 0:
        rate, dt, cores = oracle_rate(args.cpu_sample)
        line["cpu_baseline"] = {"value": rate, "unit": "boxes/s", "cores": cores, "kind": "oracle",
                                "sample": f"{args.cpu_sample} boxes spread over the workload, FP64 oracle "
                                          f"(LU, solves, A_bb + A_bi S) with OpenMP over {cores} threads, "
                                          f"{dt:.1f} s"}
        lrate, ldt = lapack_rate(8)
        line["cpu_lapack_baseline"] = {"value": lrate, "unit": "boxes/s", "cores": os.cpu_count(), "kind": "lapack",
                                       "sample": f"8 boxes spread over the workload: the oracle's collocation "
                                                 f"matrix, numpy's threaded LAPACK solve for S and one product for "
                                                 f"T, {ldt:.1f} s (context)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


LEARNED = ("p=12 boxes of side 1/8, kappa=20, one random Fourier-law b field per box; 20000 training boxes "
           "(seed 1) with exact DtN maps from the FP32+refinement path, 4096 held-out boxes (seed 2); MLP "
           "1728->512->512->2*600*32 (rank-32 factors), BF16 weights, FP32 accumulate, Adam")


def fourier_fields_torch(fields, xyz, dev):
    """[nfield, N] values of per-box b fields at the node coordinates [N, 3]
    of a box at the origin, evaluated on the GPU (input generation only)."""
    import torch
    K = torch.tensor(np.stack([f.k for f in fields]), dtype=torch.float64, device=dev)     # [F, 16, 3]
    A = torch.tensor(np.stack([f.a for f in fields]), dtype=torch.float64, device=dev)     # [F, 16]
    Ph = torch.tensor(np.stack([f.phi for f in fields]), dtype=torch.float64, device=dev)  # [F, 16]
    x = torch.from_numpy(xyz).to(dev)
    out = []
    for i in range(0, len(fields), 1024):
        ph = 2 * math.pi * torch.einsum("nd,fqd->fnq", x, K[i:i + 1024]) + Ph[i:i + 1024, None, :]
        out.append(torch.clamp(1.0 + 0.5 * (torch.cos(ph) * A[i:i + 1024, None, :]).sum(-1), 0.5, 1.5))
    return torch.cat(out).contiguous()


def run_learned(args):
    """The learned DtN correction as its own JSON line."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    print(json.dumps(learned_measurement(args.train_boxes, args.epochs, args.gate_tol, args.steps, dev)), flush=True)


def learned_step_flops(B, dims, m, r):
    """Flops of one training step's products (forward, loss, back propagation
    and weight gradients) for a batch of B boxes."""
    d0, d1, d2, d3 = dims
    fwd = 2.0 * B * (d0 * d1 + d1 * d2 + d2 * d3)
    loss = 6.0 * B * m * m * r                      # E = U V^T, E V, E^T U
    bwd = 2.0 * B * (2 * d2 * d3 + 2 * d1 * d2 + d0 * d1)
    return fwd + loss + bwd


def learned_measurement(train_boxes: int, epochs: int, gate_tol: float, steps: int, dev) -> dict:
    """Train the learned DtN correction on exact maps, then serve the held-out
    boxes through it (with the gate and exact fallback) and through the exact
    reduction alone."""
    import torch
    import paper_2503_04033_gb300 as H
    from paper_2503_04033_gb300.learned import LearnedDtN
    p, h, kappa, rank, batch = 12, 0.125, 20.0, 32, 256
    xyz = H.hps_leaf_nodes(p, (0.0, 0.0, 0.0), (h, h, h))
    ctx = H.hps_create(0, 0)
    model = LearnedDtN(ctx, p, h, kappa, hidden=(512, 512), rank=rank, seed=3)
    b_tr = fourier_fields_torch(hi.fourier_b_per_box(train_boxes, hi.SEED_TRAIN), xyz, dev)
    b_te = fourier_fields_torch(hi.fourier_b_per_box(4096, hi.SEED_HELDOUT), xyz, dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
    ev[0].record()
    T_tr = model.targets(b_tr)
    ev[1].record()
    losses = model.fit(b_tr, T_tr, epochs=epochs, batch=batch, lr=1e-3)
    ev[2].record()
    del T_tr
    T_te = model.targets(b_te)                        # reference maps for the error report
    torch.cuda.synchronize()
    t_data, t_fit = ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3
    n_steps = epochs * ((train_boxes + batch - 1) // batch)
    m = model.m
    dims = [p ** 3, 512, 512, 2 * m * rank]
    fit_flops = epochs * sum(learned_step_flops(min(batch, train_boxes - i), dims, m, rank)
                             for i in range(0, train_boxes, batch))

    def rel(A, B):
        return ((A - B).flatten(1).norm(dim=1) / B.flatten(1).norm(dim=1)).cpu().numpy()

    That = model.predict(b_te)
    e_net, e_t0 = rel(That, T_te), rel(model.T0.expand_as(T_te), T_te)
    tol = gate_tol
    for _ in range(2):                                 # warm both paths
        model.serve(b_te[:64], tol)
        model.exact(b_te[:64])
    torch.cuda.synchronize()
    ev[3].record()
    for _ in range(steps):
        T_ex = model.exact(b_te)
    ev[4].record()
    for _ in range(steps):
        T_sv, acc, err = model.serve(b_te, tol)
    ev[5].record()
    for _ in range(steps):
        model.predict(b_te)
    ev[6].record()
    torch.cuda.synchronize()
    ms_ex = ev[3].elapsed_time(ev[4]) / steps
    ms_sv = ev[4].elapsed_time(ev[5]) / steps
    ms_pr = ev[5].elapsed_time(ev[6]) / steps
    acc_np = acc.cpu().numpy()
    e_out = rel(T_sv, T_te)
    line = {"metric": "learned DtN correction: held-out boxes/s served (surrogate + gate + exact fallback)",
            "value": 4096 / (ms_sv / 1e3), "unit": "boxes/s", "n_gpus": 1, "steps": steps, "warmup": 2,
            "ms_per_step": ms_sv, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16 operands (tcgen05), f32 accumulate; exact path f32+f64", "data": "synthetic",
            "config": {"workload": LEARNED, "train_boxes": train_boxes, "epochs": epochs,
                       "gate_tol": tol, "gate_probes": 4},
            "exact_path": {"value": 4096 / (ms_ex / 1e3), "unit": "boxes/s", "ms_per_step": ms_ex},
            "surrogate_only": {"value": 4096 / (ms_pr / 1e3), "unit": "boxes/s", "ms_per_step": ms_pr,
                               "what": "MLP forward + T0 + s U V^T (no gate)"},
            "accept_rate": float(acc_np.mean()),
            "rel_err": {"T0_median": float(np.median(e_t0)), "surrogate_median": float(np.median(e_net)),
                        "surrogate_p90": float(np.quantile(e_net, 0.9)), "served_max": float(e_out.max()),
                        "served_max_accepted": float(e_out[acc_np == 1].max()) if acc_np.any() else None},
            "gain": {"median_error_ratio_T0_over_surrogate": float(np.median(e_t0) / np.median(e_net)),
                     "served_speedup_over_exact": ms_ex / ms_sv},
            "training": {"data_s": t_data, "fit_s": t_fit, "loss_first": losses[0], "loss_last": losses[-1],
                         "steps": n_steps, "ms_per_step": 1e3 * t_fit / n_steps,
                         "train_boxes_per_s": train_boxes * epochs / t_fit,
                         "product_tflops": fit_flops / t_fit / 1e12,
                         "note": "every product on tcgen05 (BF16 operands, FP32 accumulation); the step also "
                                 "holds the elementwise, loss and Adam kernels and the batch gathers"}}
    model.close()
    H.hps_destroy(ctx)
    return line


UNEVEN = ("1024 leaf boxes (h=1/8) with p drawn from {8,12,16,20} and kappa from {10,20,40,60}, "
          "b = the seeded Fourier law, 32 Gaussian random smooth loads per box (seed 20250305); "
          "one hps_leaf_groups call: DtN map + 32 particular solutions per box from one factorisation")


def load_field_torch(loads, xyz, dev):
    """[nbox, nloads, p^3] values of the load fields at node coordinates
    [nbox, p^3, 3], evaluated on the GPU (input generation only)."""
    import torch
    K = torch.tensor(np.stack([L.k for L in loads]), dtype=torch.float64, device=dev)        # [L, 16, 3]
    A = torch.tensor(np.stack([L.a for L in loads]), dtype=torch.float64, device=dev)        # [L, 16]
    Ph = torch.tensor(np.stack([L.phi for L in loads]), dtype=torch.float64, device=dev)     # [L, 16]
    out = []
    for i in range(xyz.shape[0]):
        x = torch.from_numpy(xyz[i]).to(dev)                                                 # [N, 3]
        ph = 2 * math.pi * torch.einsum("nd,lqd->lnq", x, K) + Ph[:, None, :]
        out.append((torch.cos(ph) * A[:, None, :]).sum(-1))
    return torch.stack(out).contiguous()


def run_uneven(args):
    """The uneven batch as its own JSON line."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    print(json.dumps(uneven_measurement(args.steps, args.warmup, dev)), flush=True)


def uneven_measurement(steps: int, warmup: int, dev) -> dict:
    """The uneven batch (1024 boxes, p from {8, 12, 16, 20}, kappa from
    {10, 20, 40, 60}, 32 loads per box): per p, one group; graphs and the
    schedule autotuner on."""
    import torch
    import paper_2503_04033_gb300 as H
    d = hi.uneven_batch(nbox=1024, nloads=32)
    h = d["h"]
    groups, flops = [], 0.0
    for p in (8, 12, 16, 20):
        sel = np.nonzero(d["p"] == p)[0]
        n, m = H.hps_leaf_sizes(p)
        xyz = np.stack([H.hps_leaf_nodes(p, lo, h) for lo in d["lo"][sel]])
        b = torch.from_numpy(d["b_field"].b(xyz)).to(dev)
        f = load_field_torch(d["loads"], xyz, dev)
        nb = len(sel)
        groups.append({"p": p, "h": h, "kappa": d["kappa"][sel], "b": b,
                       "T": torch.empty(nb, m, m, dtype=torch.float64, device=dev), "f": f,
                       "v": torch.empty(nb, 32, n, dtype=torch.float64, device=dev),
                       "hflux": torch.empty(nb, 32, m, dtype=torch.float64, device=dev),
                       "box_status": torch.zeros(nb, dtype=torch.int32, device=dev)})
        q = p - 2
        flops += nb * (flops_per_box(p) + 2.0 * n * n * 32 + 2.0 * q * m * 32)
    ctx = H.hps_create(0, 0)
    H.hps_set_option(ctx, H.HPS_OPT_AUTOTUNE, 1)
    H.hps_set_option(ctx, H.HPS_OPT_GRAPHS, 1)
    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        H.hps_leaf_groups(ctx, groups, H.HPS_FP32_IR, stream)
    torch.cuda.synchronize(dev)
    fails = sum(int((g["box_status"] != 0).sum().item()) for g in groups)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index or 0) as clocks:
        e0.record(stream)
        for _ in range(steps):
            H.hps_leaf_groups(ctx, groups, H.HPS_FP32_IR, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    # one more call, outside the timed region, with per-kernel events (graphs off)
    H.hps_set_option(ctx, H.HPS_OPT_GRAPHS, 0)
    H.hps_profile_enable(ctx, True)
    H.hps_profile_reset(ctx)
    H.hps_leaf_groups(ctx, groups, H.HPS_FP32_IR, stream)
    torch.cuda.synchronize(dev)
    H.hps_profile_enable(ctx, False)
    prof = {}
    for cls, name in enumerate(H.KERNEL_CLASSES):
        nl, kms, fl, by = H.hps_profile_get(ctx, cls)
        if nl:
            prof[name] = {"launches": nl, "ms": kms}
    H.hps_destroy(ctx)
    tuned = {}
    cache = os.environ.get("HPS_TUNE_CACHE")
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            for ln in fh:
                v = ln.split()
                if len(v) == 6:
                    tuned[f"p{v[0]}"] = {"nb": int(v[3]), "unit": int(v[4]), "tile": int(v[5])}
    del groups
    torch.cuda.empty_cache()
    return {"metric": "uneven leaf batch: boxes/s (DtN + 32 particular solutions per box, mixed p)",
            "value": 1024 / (ms / 1e3), "unit": "boxes/s", "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_label(H.HPS_FP32_IR, {}), "data": "synthetic",
            "config": {"workload": UNEVEN, "boxes_per_p": {str(p): int((d["p"] == p).sum()) for p in (8, 12, 16, 20)},
                       "graphs": True, "autotune": True},
            "tflops": flops / (ms / 1e3) / 1e12, "box_failures": fails, "clocks": clocks.summary(),
            "tuned_schedule": tuned, "kernels_one_call": prof}


def run_factored(args):
    """Factor once, solve many: the p = 16 workload's 512 boxes factored once
    (hps_leaf_factor), then every step solves 32 new loads per box with the
    stored factors (hps_leaf_solve_factored) -- the reuse of the build stage
    that time stepping relies on.  Beside it: the same loads through the
    one-shot hps_leaf_particular (which factors again), and the difference
    from the plain FP64 path on a sample of boxes."""
    import torch
    import paper_2503_04033_gb300 as H
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    nbox, nl = args.nbox, 32
    lows, h = box_lows()
    lows = lows[np.arange(nbox) % NBOX]
    field = hi.fourier_b_field()
    xyz = np.stack([H.hps_leaf_nodes(P, lo, h) for lo in lows])
    b = torch.from_numpy(field.b(xyz)).to(dev)
    f = load_field_torch(hi.fourier_b_per_box(nl, 20250306), xyz, dev)
    n, m = H.hps_leaf_sizes(P)
    kind = H.LeafKind(P, h, KAPPA)
    v = torch.empty(nbox, nl, n, dtype=torch.float64, device=dev)
    hf = torch.empty(nbox, nl, m, dtype=torch.float64, device=dev)
    st = torch.zeros(nbox, dtype=torch.int32, device=dev)
    ctx = H.hps_create(0, 0)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    F = H.hps_leaf_factor(ctx, kind, nbox, b, nl, H.HPS_FP32_IR, st, stream)
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    factor_ms = ev[0].elapsed_time(ev[1])
    fact_fail = int((st != 0).sum().item())
    for _ in range(args.warmup):
        H.hps_leaf_solve_factored(F, nl, f, v, hf, st, stream)
    torch.cuda.synchronize(dev)
    with ClockSampler(0) as clocks:
        ev[0].record(stream)
        for _ in range(args.steps):
            H.hps_leaf_solve_factored(F, nl, f, v, hf, st, stream)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    fails = int((st != 0).sum().item())
    # one more solve, outside the timed region, with per-kernel events
    H.hps_profile_enable(ctx, True)
    H.hps_profile_reset(ctx)
    H.hps_leaf_solve_factored(F, nl, f, v, hf, st, stream)
    torch.cuda.synchronize(dev)
    H.hps_profile_enable(ctx, False)
    prof = {}
    for cls, name in enumerate(H.KERNEL_CLASSES):
        nlaunch, kms, _, _ = H.hps_profile_get(ctx, cls)
        if nlaunch:
            prof[name] = {"launches": nlaunch, "ms": kms}
    H.hps_leaf_factors_destroy(F)
    # the one-shot call on the same loads (factors again), timed once after a warm call
    v1, h1 = torch.empty_like(v), torch.empty_like(hf)
    H.hps_leaf_particular(ctx, kind, nbox, nl, b, f, v1, h1, H.HPS_FP32_IR, st, stream)
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    H.hps_leaf_particular(ctx, kind, nbox, nl, b, f, v1, h1, H.HPS_FP32_IR, st, stream)
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    once_ms = ev[0].elapsed_time(ev[1])
    rel_once = ((v1 - v).flatten(1).norm(dim=1) / v1.flatten(1).norm(dim=1)).max().item()
    del v1, h1
    # the plain FP64 path on a sample of boxes
    k = min(16, nbox)
    sel = torch.from_numpy(np.linspace(0, nbox - 1, k).astype(np.int64)).to(dev)
    v64 = torch.empty(k, nl, n, dtype=torch.float64, device=dev)
    h64 = torch.empty(k, nl, m, dtype=torch.float64, device=dev)
    st64 = torch.zeros(k, dtype=torch.int32, device=dev)
    H.hps_leaf_particular(ctx, kind, k, nl, b.index_select(0, sel).contiguous(), f.index_select(0, sel).contiguous(),
                          v64, h64, H.HPS_FP64, st64, stream)
    torch.cuda.synchronize(dev)
    vs = v.index_select(0, sel)
    rel64 = ((vs - v64).flatten(1).norm(dim=1) / v64.flatten(1).norm(dim=1)).max().item()
    H.hps_destroy(ctx)
    flops = nbox * (4.0 * n * n * nl + 2.0 * (P - 2) * m * nl)   # forward + backward solves and A_bi v
    line = {"metric": "particular solutions/s at p=16 with stored factors (32 loads per box, FP32 LU + FP64 refinement)",
            "value": nbox * nl / (ms / 1e3), "unit": "solutions/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{nbox} boxes of the p=16 workload (kappa=40, Fourier-law b), {nl} Gaussian "
                                   f"random smooth loads per box (seed 20250306); factors kept between steps"},
            "factor_ms": factor_ms, "factor_failures": fact_fail, "box_failures": fails,
            "tflops_solves": flops / (ms / 1e3) / 1e12,
            "one_shot_particular": {"ms": once_ms, "value": nbox * nl / (once_ms / 1e3), "unit": "solutions/s",
                                    "max_rel_diff_v": rel_once},
            "rel_err_vs_fp64_path": rel64, "fp64_sample_boxes": k, "clocks": clocks.summary(),
            "kernels_one_solve": prof}
    print(json.dumps(line), flush=True)


def run_dirichlet(args):
    """The whole two-stage solve of an nb x nb x nb grid of boxes (default
    8 x 8 x 8: 134,400 interface unknowns) at p = 12 (kappa = 20,
    b = 1 - 0.5 exp(-|x - c|^2 / 0.04), f = 1, g = 0) on the GPU: build stage = leaf DtN maps (FP32 LU + FP64
    refinement) and the interface factorisation (nested dissection; FP32
    factors refined in FP64 in each solve, and FP64 factors for comparison);
    solve stage = particular solutions, the interface solve and the interior
    reconstruction (Algorithms 1 and 2).  Checked by the flux-continuity
    residual of the interface equations (Eq. 4) at every shared face node."""
    import torch
    import paper_2503_04033_gb300 as H
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    p, nbx, kappa = 12, args.nb, 20.0
    nb = (nbx, nbx, nbx)
    nbox = nbx ** 3
    lows, h = hi.box_grid_lo(nb)
    n, m = H.hps_leaf_sizes(p)
    qq = (p - 2) ** 2
    kind = H.LeafKind(p, h, kappa)
    b = torch.from_numpy(np.stack([hi.gaussian_dip_b(H.hps_leaf_nodes(p, lo, h)) for lo in lows])).to(dev)
    f = torch.ones(nbox, 1, p ** 3, dtype=torch.float64, device=dev)
    ctx = H.hps_create(0, 0)
    stream = torch.cuda.current_stream(dev)
    T = torch.empty(nbox, m, m, dtype=torch.float64, device=dev)
    S = torch.empty(nbox, n, m, dtype=torch.float64, device=dev)
    v = torch.empty(nbox, 1, n, dtype=torch.float64, device=dev)
    hf = torch.empty(nbox, 1, m, dtype=torch.float64, device=dev)
    ub = torch.empty(nbox, 1, m, dtype=torch.float64, device=dev)
    ui = torch.empty(nbox, 1, n, dtype=torch.float64, device=dev)
    st = torch.zeros(nbox, dtype=torch.int32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    # interface numbering for the flux-continuity check
    gid = np.full((nbox, m), -1, dtype=np.int64)
    Fx = (nbx - 1) * nbx * nbx
    for bx in range(nbox):
        c = (bx % nbx, (bx // nbx) % nbx, bx // (nbx * nbx))
        for f_ in range(6):
            axis, side = f_ // 2, f_ % 2
            plane = c[axis] + side
            if plane == 0 or plane == nbx:
                continue
            if axis == 0:
                fid = (plane - 1) + (nbx - 1) * (c[1] + nbx * c[2])
            elif axis == 1:
                fid = Fx + c[0] + nbx * ((plane - 1) + (nbx - 1) * c[2])
            else:
                fid = 2 * Fx + c[0] + nbx * (c[1] + nbx * (plane - 1))
            gid[bx, f_ * qq:(f_ + 1) * qq] = fid * qq + np.arange(qq)
    sel = np.flatnonzero(gid.reshape(-1) >= 0)
    ni = 3 * Fx * qq
    gid_d = torch.from_numpy(gid.reshape(-1)[sel]).to(dev)
    sel_d = torch.from_numpy(sel).to(dev)

    def flux_residual():
        flux = torch.bmm(T, ub[:, 0, :, None])[:, :, 0] + hf[:, 0, :]
        tot = torch.zeros(ni, dtype=torch.float64, device=dev)
        tot.index_add_(0, gid_d, flux.reshape(-1)[sel_d])
        scale = torch.bmm(T.abs(), ub[:, 0, :, None].abs())[:, :, 0].max().item()
        return tot.abs().max().item() / scale

    results = {}
    for iprec, name in ((H.HPS_FP32_IR, "fp32ir"), (H.HPS_FP64, "fp64")):
        for rep in range(2):   # the first pass warms up (workspace, tables)
            ev[0].record(stream)
            H.hps_leaf_build_dtn(ctx, kind, nbox, b, T, S, H.HPS_FP32_IR, st, stream)
            ev[1].record(stream)
            FI = H.hps_interface_factor(ctx, p, nb, T, 1, iprec, stream=stream)
            ev[2].record(stream)
            H.hps_leaf_particular(ctx, kind, nbox, 1, b, f, v, hf, H.HPS_FP32_IR, st, stream)
            ev[3].record(stream)
            H.hps_interface_solve(FI, 1, hf, None, ub, stream)
            ev[4].record(stream)
            H.hps_leaf_reconstruct(ctx, kind, nbox, 1, b, S, v, ub, ui, H.HPS_FP32_IR, st, stream)
            ev[5].record(stream)
            torch.cuda.synchronize(dev)
            info = H.hps_interface_info(FI)
            refine = H.hps_interface_last_refinement(FI)
            H.hps_interface_destroy(FI)
        stages = {"leaf_dtn_ms": ev[0].elapsed_time(ev[1]), "interface_factor_ms": ev[1].elapsed_time(ev[2]),
                  "particular_ms": ev[2].elapsed_time(ev[3]), "interface_solve_ms": ev[3].elapsed_time(ev[4]),
                  "reconstruct_ms": ev[4].elapsed_time(ev[5])}
        results[name] = {"stages_ms": stages,
                         "build_ms": stages["leaf_dtn_ms"] + stages["interface_factor_ms"],
                         "solve_ms": stages["particular_ms"] + stages["interface_solve_ms"] + stages["reconstruct_ms"],
                         "flux_residual_rel": flux_residual(),
                         "interface_refinement": {"corrections": refine[0], "last_rel_correction": refine[1]},
                         "interface_factor": {"merges": info[0], "levels": info[1], "largest_separator": info[2],
                                              "device_bytes": info[3]},
                         "ui": ui[:, 0, :].cpu().numpy()}
    fails = int((st != 0).sum().item())
    H.hps_destroy(ctx)
    head, other = results["fp32ir"], results["fp64"]
    diff = float(np.abs(head["ui"] - other["ui"]).max() / np.abs(other["ui"]).max())
    for r in results.values():
        r.pop("ui")
    total = head["build_ms"] + head["solve_ms"]
    line = {"metric": f"two-stage Dirichlet solve on the GPU, {nbx}x{nbx}x{nbx} boxes at p=12 (build stage, then solve "
                      f"stage)",
            "value": 1e3 / total, "unit": "solves/s (build + solve)", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": total, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64 leaves, f32+f64 interface", "data": "synthetic",
            "config": {"workload": f"{nbox} boxes of the unit cube, p = {p}, kappa = {kappa}, b = 1 - 0.5 exp(-|x - c|^2 "
                                   f"/ 0.04), f = 1, g = 0; {ni} interface unknowns"},
            "build_ms": head["build_ms"], "solve_ms": head["solve_ms"], "interface_fp32ir": head,
            "interface_fp64": other, "u_int_rel_diff_fp32ir_vs_fp64": diff, "box_failures": fails}
    print(json.dumps(line), flush=True)


def run_accuracy(args):
    """The accuracy study of Sec. 4.1 run entirely on the GPU: Lap u +
    kappa^2 u = 0 on [-1.1, 0.1] x [1, 2] x [1.2, 2.2] with the Green's
    function cos(kappa |x|) / (4 pi |x|) as exact solution and its boundary
    values as g, under p- and h-refinement (kappa = 0, 16, 30).  Leaf maps,
    particular solutions and reconstruction in FP64 (S stored), the interface
    factorised on the GPU in FP64.  Relative l2 error over the interior nodes
    and, once each, the shared face nodes."""
    import time as _time
    import torch
    import paper_2503_04033_gb300 as H
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ctx = H.hps_create(0, 0)
    stream = torch.cuda.current_stream(dev)
    table = {}
    best = {}
    t_all = _time.time()
    for kappa in (0.0, 16.0, 30.0):
        for p in (6, 8, 10, 12):
            for nbx in (2, 4, 8):
                nb = (nbx, nbx, nbx)
                lows, h = hi.box_grid_lo(nb, L=hi.GREEN_L, lo=hi.GREEN_LO)
                nbox = len(lows)
                n, m = H.hps_leaf_sizes(p)
                q = p - 2
                qq = q * q
                kind = H.LeafKind(p, h, kappa)
                xyz = np.stack([H.hps_leaf_nodes(p, lo, h) for lo in lows])
                r1 = np.arange(1, q + 1)
                kk, jj, ii_ = np.meshgrid(r1, r1, r1, indexing="ij")
                ii = (ii_ + p * jj + p * p * kk).reshape(-1)
                fi, fid = [], []
                for f_ in range(6):
                    axis, sv = f_ // 2, (0 if f_ % 2 == 0 else p - 1)
                    for bb in range(1, q + 1):
                        for aa in range(1, q + 1):
                            i3 = [aa, bb]
                            i3.insert(axis, sv)
                            fi.append(i3[0] + p * i3[1] + p * p * i3[2])
                            fid.append(f_)
                fi, fid = np.asarray(fi), np.asarray(fid)
                b = torch.ones(nbox, p ** 3, dtype=torch.float64, device=dev)
                f = torch.zeros(nbox, 1, p ** 3, dtype=torch.float64, device=dev)
                g = torch.from_numpy(hi.green(xyz[:, fi, :], kappa)[:, None, :].copy()).to(dev)
                T = torch.empty(nbox, m, m, dtype=torch.float64, device=dev)
                S = torch.empty(nbox, n, m, dtype=torch.float64, device=dev)
                v = torch.empty(nbox, 1, n, dtype=torch.float64, device=dev)
                hf = torch.empty(nbox, 1, m, dtype=torch.float64, device=dev)
                ub = torch.empty(nbox, 1, m, dtype=torch.float64, device=dev)
                ui = torch.empty(nbox, 1, n, dtype=torch.float64, device=dev)
                st = torch.zeros(nbox, dtype=torch.int32, device=dev)
                H.hps_leaf_build_dtn(ctx, kind, nbox, b, T, S, H.HPS_FP64, st, stream)
                H.hps_leaf_particular(ctx, kind, nbox, 1, b, f, v, hf, H.HPS_FP64, st, stream)
                FI = H.hps_interface_factor(ctx, p, nb, T, 1, H.HPS_FP64, stream=stream)
                H.hps_interface_solve(FI, 1, hf, g, ub, stream)
                H.hps_leaf_reconstruct(ctx, kind, nbox, 1, b, S, v, ub, ui, H.HPS_FP64, st, stream)
                torch.cuda.synchronize(dev)
                H.hps_interface_destroy(FI)
                ok = int((st != 0).sum().item()) == 0
                cell = np.rint((lows - np.asarray(hi.GREEN_LO)) / h).astype(int)
                upper = cell + 1 < np.asarray(nb)[None, :]
                keep = np.stack([upper[:, fid[r] // 2] & (fid[r] % 2 == 1) for r in range(m)], axis=1)
                ue_i = hi.green(xyz[:, ii, :], kappa)
                ue_b = hi.green(xyz[:, fi, :], kappa)[keep]
                err = np.concatenate([(ui[:, 0, :].cpu().numpy() - ue_i).reshape(-1),
                                      ub[:, 0, :].cpu().numpy()[keep] - ue_b])
                rel = float(np.linalg.norm(err) / np.linalg.norm(np.concatenate([ue_i.reshape(-1), ue_b])))
                table.setdefault(f"kappa={kappa:g}", {}).setdefault(f"p={p}", {})[f"{nbx}^3"] = rel if ok else None
                if ok:
                    best[kappa] = min(best.get(kappa, 1.0), rel)
                del T, S
    wall = _time.time() - t_all
    H.hps_destroy(ctx)
    line = {"metric": "Sec. 4.1 accuracy study on the GPU: smallest relative l2 error vs the Green's function (Poisson)",
            "value": best.get(0.0), "unit": "relative l2 error", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 * wall, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (analytic Green's function)",
            "config": {"workload": "Lap u + kappa^2 u = 0 on [-1.1, 0.1] x [1, 2] x [1.2, 2.2], u = g = cos(kappa |x|) "
                                   "/ (4 pi |x|); p in {6, 8, 10, 12}, 2^3 / 4^3 / 8^3 boxes, kappa in {0, 16, 30}"},
            "best": {f"kappa={k:g}": v for k, v in best.items()},
            "paper_floors": {"kappa=0": "about 1e-13", "kappa=16": "about 1e-11", "kappa=30": "about 1e-10"},
            "errors": table}
    print(json.dumps(line), flush=True)


def run_leaf2d(args):
    """The 2-D form of the leaf reduction (FP64): 64 x 64 boxes of the unit
    square at p = 16 (n = 196 interior, m = 56 edge nodes per box), kappa =
    40, b = 1 + 0.4 sin(6 x) cos(4 y), one load f = cos(3 x + y); a step is one
    hps_leaf2d_solve (T, S, v, h of every box).  Inputs resident; the working
    set (about 2 GB) exceeds L2."""
    import torch
    import paper_2503_04033_gb300 as H
    import oracle
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    p, nbx, kappa = 16, 64, 40.0
    nbox = nbx * nbx
    h = (1.0 / nbx, 1.0 / nbx)
    n, m = H.hps_leaf2d_sizes(p)
    q = p - 2
    lows = [((bx % nbx) * h[0], (bx // nbx) * h[1]) for bx in range(nbox)]
    xy = np.stack([H.hps_leaf_nodes(p, (lo[0], lo[1], 0.0), (h[0], h[1], 1.0))[:p * p, :2] for lo in lows])
    bfn = lambda x: 1.0 + 0.4 * np.sin(6 * x[..., 0]) * np.cos(4 * x[..., 1])
    ffn = lambda x: np.cos(3 * x[..., 0] + x[..., 1])
    b = torch.from_numpy(bfn(xy)).to(dev)
    f = torch.from_numpy(ffn(xy)[:, None, :].copy()).to(dev)
    T = torch.empty(nbox, m, m, dtype=torch.float64, device=dev)
    S = torch.empty(nbox, n, m, dtype=torch.float64, device=dev)
    v = torch.empty(nbox, 1, n, dtype=torch.float64, device=dev)
    hf = torch.empty(nbox, 1, m, dtype=torch.float64, device=dev)
    st = torch.zeros(nbox, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        H.hps_leaf2d_solve(p, h, kappa, nbox, b, 1, f, T, S, v, hf, st, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    fails = int((st != 0).sum().item())
    # the dense method's flops per box: LU 2/3 n^3, solves with m + 1 right-hand sides, D_n products
    flops = 2.0 / 3.0 * n ** 3 + 2.0 * n * n * (m + 1) + 2.0 * q * m * (m + 1)
    value = nbox / (ms / 1e3)
    tflops = value * flops / 1e12
    # parity on a sample against the oracle, and the oracle's rate
    sel = np.linspace(0, nbox - 1, 16).astype(int)
    worst = 0.0
    t0 = time.perf_counter()
    for bx in sel:
        xo = oracle.node_coords_2d(p, lows[bx], h)
        To, _, info = oracle.leaf_dtn_2d(p, h, kappa, bfn(xo), want_S=False)
        worst = max(worst, float(np.linalg.norm(T[bx].cpu().numpy() - To) / np.linalg.norm(To)))
    cpu_s = time.perf_counter() - t0
    line = {"metric": "2-D leaf DtN builds/s at p=16 (FP64; T, S, v, h per box)", "value": value, "unit": "boxes/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{nbx}x{nbx} boxes of the unit square, p = {p} (n = {n}, m = {m}), kappa = {kappa}, "
                                   "b = 1 + 0.4 sin(6x) cos(4y), one load f = cos(3x + y)",
                       "l2": "inputs and workspace larger than L2, no flush"},
            "tflops": tflops,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tflops / FP64_PEAK_TFLOPS, "traffic": None,
                         "peak_source": "FP64 issue rate 152 SMs x 2.07 GHz x 2 FMA/clk (the whole call, its LU "
                                        "on the CUDA-core FP64 path)"},
            "rel_err_vs_oracle_max": worst, "box_failures": fails, "clocks": clocks.summary(),
            "cpu_baseline": {"value": len(sel) / cpu_s, "unit": "boxes/s", "cores": oracle.max_threads(),
                             "kind": "oracle", "sample": f"{len(sel)} boxes spread over the grid, 2-D FP64 oracle "
                                                         "(T only), one box at a time"}}
    print(json.dumps(line), flush=True)


def _fp64_leaf_line(metric, value, ms, args, workload, flops_per_box, worst, fails, clocks, cpu_rate, cpu_n,
                    extra=None):
    tflops = value * flops_per_box / 1e12
    import oracle
    line = {"metric": metric, "value": value, "unit": "boxes/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "l2": "inputs and workspace larger than L2, no flush"},
            "tflops": tflops,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tflops / FP64_PEAK_TFLOPS, "traffic": None,
                         "peak_source": "FP64 issue rate 152 SMs x 2.07 GHz x 2 FMA/clk (the whole call, its LU "
                                        "on the CUDA-core FP64 path)"},
            "rel_err_vs_oracle_max": worst, "box_failures": fails, "clocks": clocks.summary(),
            "cpu_baseline": {"value": cpu_rate, "unit": "boxes/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"{cpu_n} boxes spread over the batch, FP64 oracle, one box at a time"}}
    if extra:
        line.update(extra)
    return line


def _timed_steps(step, args, dev):
    import torch
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / args.steps, clocks


def run_cross(args):
    """Leaves of the curved domain of Sec. 4.3 on Legendre face grids (FP64,
    cross-term operator through the parameter map): 512 boxes at p = 10
    (n = 512, m = 486), kappa = |k|; a step is one hps_leaf_cross_solve (T and
    S of every box).  Parity on a sample against the oracle."""
    import torch
    import paper_2503_04033_gb300 as H
    import oracle
    from oracle import cross as cx
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    p, nbx = 10, 8
    kappa = float(np.linalg.norm(hi.CURVED_K))
    h = np.asarray(hi.CURVED_L, dtype=np.float64) / nbx
    lows = np.stack([np.asarray(hi.CURVED_LO) + h * np.array([i % nbx, (i // nbx) % nbx, i // (nbx * nbx)])
                     for i in range(nbx ** 3)])
    nbox = len(lows)
    n, m = H.hps_leaf_cross_sizes(p)
    Cs, ds = [], []
    for lo in lows:
        Cx, dx = hi.curved_coefficients(H.hps_leaf_nodes(p, lo, h))
        Cs.append(Cx)
        ds.append(dx)
    C = torch.from_numpy(np.ascontiguousarray(np.stack(Cs))).to(dev)
    d = torch.from_numpy(np.ascontiguousarray(np.stack(ds))).to(dev)
    bb = torch.ones(nbox, p ** 3, dtype=torch.float64, device=dev)
    T = torch.empty(nbox, m, m, dtype=torch.float64, device=dev)
    S = torch.empty(nbox, n, m, dtype=torch.float64, device=dev)
    st = torch.zeros(nbox, dtype=torch.int32, device=dev)

    def step():
        H.hps_leaf_cross_solve(p, h, kappa, nbox, C, d, bb, 0, None, T, S, None, None, st)

    ms, clocks = _timed_steps(step, args, dev)
    sel = np.linspace(0, nbox - 1, 6).astype(int)
    worst, t0 = 0.0, time.perf_counter()
    for bx in sel:
        Cx, dx = hi.curved_coefficients(oracle.node_coords(p, lows[bx], h))
        To, _, _, _ = cx.leaf_cross(p, h, kappa, Cx, dx, np.ones(p ** 3), None)
        worst = max(worst, float(np.abs(T[bx].cpu().numpy() - To).max() / np.abs(To).max()))
    cpu_s = time.perf_counter() - t0
    flops = 2.0 / 3.0 * n ** 3 + 2.0 * n * n * m
    line = _fp64_leaf_line("cross-term leaf DtN builds/s at p=10 on Legendre face grids (FP64; T and S per box)",
                           nbox / (ms / 1e3), ms, args,
                           f"{nbx}^3 boxes of the curved domain of Sec. 4.3 (parameter map of the box "
                           f"{tuple(hi.CURVED_LO)} + {tuple(hi.CURVED_L)}), p = {p} (n = {n}, m = {m} Legendre face "
                           f"nodes), kappa = {kappa:.4f}, full-tensor coefficients of the map",
                           flops, worst, int((st != 0).sum().item()), clocks, len(sel) / cpu_s, len(sel))
    print(json.dumps(line), flush=True)


def run_iti(args):
    """Leaf impedance-to-impedance maps (FP64): 512 boxes (8^3, h = 1/8) at
    p = 8, kappa = 20, eta = kappa, b from the seeded Fourier law; a step is
    one hps_leaf_iti (R of every box).  Parity on a sample against the
    oracle."""
    import torch
    import paper_2503_04033_gb300 as H
    import oracle
    from oracle import iti
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    p, kappa = 8, 20.0
    lows, h = hi.box_grid_lo((8, 8, 8))
    field = hi.fourier_b_field()
    b_np = np.stack([field.b(H.hps_leaf_nodes(p, lo, h)) for lo in lows])
    nbox = len(lows)
    n, m = H.hps_leaf_sizes(p)
    kind = H.LeafKind(p, h, kappa)
    b = torch.from_numpy(b_np).to(dev)
    R = torch.empty(nbox, m, m, dtype=torch.complex128, device=dev)
    st = torch.zeros(nbox, dtype=torch.int32, device=dev)

    def step():
        H.hps_leaf_iti(kind, kappa, nbox, b, R, st)

    ms, clocks = _timed_steps(step, args, dev)
    sel = np.linspace(0, nbox - 1, 8).astype(int)
    worst, t0 = 0.0, time.perf_counter()
    for bx in sel:
        Ro = iti.leaf_iti(p, h, kappa, b_np[bx], kappa)
        worst = max(worst, float(np.abs(R[bx].cpu().numpy() - Ro).max() / np.abs(Ro).max()))
    cpu_s = time.perf_counter() - t0
    N2 = 2 * (n + m)
    flops = 2.0 / 3.0 * N2 ** 3 + 2.0 * N2 * N2 * m
    line = _fp64_leaf_line("leaf ItI maps/s at p=8 (FP64; the real form of the impedance system, size 2(n+m))",
                           nbox / (ms / 1e3), ms, args,
                           f"8x8x8 leaf boxes (h=1/8), p = {p} (n = {n}, m = {m}), kappa = {kappa}, eta = kappa, "
                           "b = the seeded Fourier law (seed 20250304)",
                           flops, worst, int((st != 0).sum().item()), clocks, len(sel) / cpu_s, len(sel),
                           {"flops_definition": "2/3 (2N)^3 + 2 (2N)^2 m per box, N = n + m"})
    print(json.dumps(line), flush=True)


def run_timestep(args):
    """Crank-Nicolson steps of the heat equation u_t = kappa_d Lap u on the unit
    cube (u = 0 on its boundary), 4 x 4 x 4 boxes at p = 12, as in Sec. 4.4:
    T, the interior factorisations and the interface factorisation built once;
    per step one hps_leaf_apply, one particular solve with the stored factors,
    one interface solve and one reconstruction, all on the GPU and enqueued on
    one stream (no host round trip inside a step).  --interface host runs the
    interface solve with a host sparse LU of the assembled system instead (the
    paper's arrangement, MUMPS there).  The final state is compared with the
    exact decaying solution."""
    import time as _time
    import torch
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import paper_2503_04033_gb300 as H
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    p, nbx, kd, dt = 12, 4, 0.05, 0.01
    nbox = nbx ** 3
    h = np.full(3, 1.0 / nbx)
    n, m = H.hps_leaf_sizes(p)
    q, qq = p - 2, (p - 2) ** 2
    c = 2.0 / (dt * kd)
    kind = H.LeafKind(p, h, float(np.sqrt(c)))
    lows = np.array([[i % nbx, (i // nbx) % nbx, i // (nbx * nbx)] for i in range(nbox)], dtype=np.float64) * h
    xyz = np.stack([H.hps_leaf_nodes(p, lo, h) for lo in lows])
    b = torch.full((nbox, p ** 3), -1.0, dtype=torch.float64, device=dev)
    ctx = H.hps_create(0, 0)
    H.hps_set_option(ctx, H.HPS_OPT_GRAPHS, 1)     # every step replays the same solves
    stream = torch.cuda.current_stream(dev)
    gpu_iface = args.interface == "gpu"
    t0 = _time.time()
    T = torch.empty(nbox, m, m, dtype=torch.float64, device=dev)
    lprec = {"fp32ir": H.HPS_FP32_IR, "fp64": H.HPS_FP64}[args.leaf_prec]
    H.hps_leaf_build_dtn(ctx, kind, nbox, b, T, None, H.HPS_FP32_IR, None, stream)
    F = H.hps_leaf_factor(ctx, kind, nbox, b, 1, lprec, None, stream)
    torch.cuda.synchronize(dev)
    t_gpu_setup = _time.time() - t0
    t0 = _time.time()
    FI = H.hps_interface_factor(ctx, p, (nbx, nbx, nbx), T, 1, stream=stream) if gpu_iface else None
    t_iface_setup = _time.time() - t0
    # node index sets: interior (x fastest) and face nodes (face order)
    r = np.arange(1, q + 1)
    kk, jj, ii_ = np.meshgrid(r, r, r, indexing="ij")
    ii = (ii_ + p * jj + p * p * kk).reshape(-1)
    fi = []
    for f in range(6):
        axis, sv = f // 2, (0 if f % 2 == 0 else p - 1)
        for bb in range(1, q + 1):
            for aa in range(1, q + 1):
                i3 = [aa, bb]
                i3.insert(axis, sv)
                fi.append(i3[0] + p * i3[1] + p * p * i3[2])
    fi = np.asarray(fi)
    u0 = np.sin(np.pi * xyz[..., 0]) * np.sin(np.pi * xyz[..., 1]) * np.sin(np.pi * xyz[..., 2])
    u = torch.from_numpy(u0[:, None, :].copy()).to(dev)
    Au = torch.empty_like(u)
    f = torch.empty_like(u)
    ub = torch.zeros(nbox, 1, m, dtype=torch.float64, device=dev)
    v = torch.empty(nbox, 1, n, dtype=torch.float64, device=dev)
    hf = torch.empty(nbox, 1, m, dtype=torch.float64, device=dev)
    ui = torch.empty(nbox, 1, n, dtype=torch.float64, device=dev)
    st = torch.zeros(nbox, dtype=torch.int32, device=dev)
    ii_d, fi_d = torch.from_numpy(ii).to(dev), torch.from_numpy(fi).to(dev)

    # host sparse LU of the assembled interface system: the --interface host
    # loop uses it, and the GPU loop times a few of its solves for comparison
    t0 = _time.time()
    rows, cols, vals, _, _, _, ni, _ = H.hps_assemble_interface_blocks(p, (nbx, nbx, nbx), T.cpu().numpy())
    lu = spla.splu(sp.coo_matrix((vals, (rows, cols)), shape=(ni, ni)).tocsc())
    t_host_setup = _time.time() - t0
    # interface numbering of each box's face nodes (faces of each normal axis
    # in turn, box-column order, q^2 nodes per face)
    Fx = (nbx - 1) * nbx * nbx
    gid = np.full((nbox, m), -1, dtype=np.int64)
    for bx in range(nbox):
        cxyz = (bx % nbx, (bx // nbx) % nbx, bx // (nbx * nbx))
        for f_ in range(6):
            axis, side = f_ // 2, f_ % 2
            plane = cxyz[axis] + side
            if plane == 0 or plane == nbx:
                continue
            if axis == 0:
                fid = (plane - 1) + (nbx - 1) * (cxyz[1] + nbx * cxyz[2])
            elif axis == 1:
                fid = Fx + cxyz[0] + nbx * ((plane - 1) + (nbx - 1) * cxyz[2])
            else:
                fid = 2 * Fx + cxyz[0] + nbx * (cxyz[1] + nbx * (plane - 1))
            gid[bx, f_ * qq:(f_ + 1) * qq] = fid * qq + np.arange(qq)
    isi = gid >= 0
    gid_t = torch.from_numpy(np.where(isi, gid, 0)).to(dev)
    isi_t = torch.from_numpy(isi).to(dev)
    pos = torch.from_numpy(np.flatnonzero(isi)).to(dev)       # face slots that are interface nodes
    gid_pos = torch.from_numpy(gid.reshape(-1)[np.flatnonzero(isi)]).to(dev)
    rhs_d = torch.zeros(ni, dtype=torch.float64, device=dev)

    def host_interface():
        rhs_d.zero_()
        rhs_d.index_add_(0, gid_pos, hf[:, 0, :].reshape(-1)[pos], alpha=-1.0)   # -sum of the boxes' fluxes
        rhs = rhs_d.cpu().numpy()
        t1 = _time.time()
        u_if = lu.solve(rhs)
        dt_host = _time.time() - t1
        u_if_d = torch.from_numpy(u_if).to(dev)
        ub[:, 0, :] = torch.where(isi_t, u_if_d[gid_t], 0.0)
        return dt_host

    nsteps = args.steps * 10
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    leaf_ms, iface_ms, host_s = 0.0, 0.0, 0.0
    for step in range(args.warmup + nsteps):
        if step == args.warmup:   # the warm-up steps (graph capture, first loads) are not timed
            torch.cuda.synchronize(dev)
            leaf_ms, iface_ms, host_s = 0.0, 0.0, 0.0
            t_all = _time.time()
            ev[4].record(stream)
        ev[0].record(stream)
        H.hps_leaf_apply(ctx, kind, nbox, 1, b, u, Au, stream)
        torch.mul(u, 2.0 * c, out=f)
        f.sub_(Au)
        H.hps_leaf_solve_factored(F, 1, f, v, hf, st, stream)
        ev[1].record(stream)
        if gpu_iface:
            H.hps_interface_solve(FI, 1, hf, None, ub, stream)
        else:
            host_s += host_interface()
        ev[2].record(stream)
        H.hps_leaf_reconstruct_factored(F, 1, v, ub, ui, st, stream)
        u.zero_()
        u[:, 0, ii_d] = ui[:, 0, :]
        u[:, 0, fi_d] = ub[:, 0, :]
        ev[3].record(stream)
        if not gpu_iface:
            torch.cuda.synchronize(dev)
            leaf_ms += ev[0].elapsed_time(ev[1]) + ev[2].elapsed_time(ev[3])
    torch.cuda.synchronize(dev)
    wall = _time.time() - t_all
    loop_ms = ev[4].elapsed_time(ev[3])
    tend = dt * (args.warmup + nsteps)
    exact = np.exp(-3 * np.pi ** 2 * kd * tend) * u0[:, ii]
    err = float(np.abs(ui[:, 0, :].cpu().numpy() - exact).max())
    fails = int((st != 0).sum().item())
    if gpu_iface:
        # per-stage times of one more step (events read after it), then a few
        # host sparse-LU solves of its right-hand side for comparison
        ev[0].record(stream)
        H.hps_leaf_apply(ctx, kind, nbox, 1, b, u, Au, stream)
        torch.mul(u, 2.0 * c, out=f)
        f.sub_(Au)
        H.hps_leaf_solve_factored(F, 1, f, v, hf, st, stream)
        ev[1].record(stream)
        H.hps_interface_solve(FI, 1, hf, None, ub, stream)
        ev[2].record(stream)
        H.hps_leaf_reconstruct_factored(F, 1, v, ub, ui, st, stream)
        ev[3].record(stream)
        torch.cuda.synchronize(dev)
        leaf_ms = (ev[0].elapsed_time(ev[1]) + ev[2].elapsed_time(ev[3])) * nsteps
        iface_ms = ev[1].elapsed_time(ev[2]) * nsteps
        for _ in range(5):
            host_s += host_interface()
        host_s *= nsteps / 5.0
        torch.cuda.synchronize(dev)
    info = H.hps_interface_info(FI) if gpu_iface else None
    if FI is not None:
        H.hps_interface_destroy(FI)
    H.hps_leaf_factors_destroy(F)
    H.hps_destroy(ctx)
    where = "GPU" if gpu_iface else "host sparse LU"
    line = {"metric": f"Crank-Nicolson heat-equation steps/s (4x4x4 boxes, p=12; leaf work on the GPU, "
                      f"interface solve: {where})",
            "value": nsteps / (loop_ms / 1e3) if gpu_iface else nsteps / wall, "unit": "steps/s", "n_gpus": 1,
            "steps": nsteps, "warmup": args.warmup,
            "ms_per_step": loop_ms / nsteps if gpu_iface else 1e3 * wall / nsteps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.leaf_prec == "fp32ir" else "f64",
            "data": "synthetic",
            "config": {"workload": f"u_t = {kd} Lap u on the unit cube, u = 0 on the boundary, u0 = sin(pi x) sin(pi y) "
                                   f"sin(pi z); {nbox} boxes, p = {p}, dt = {dt}, {args.warmup} + {nsteps} steps (the "
                                   f"first untimed); stored leaf factors ({args.leaf_prec}); {ni} interface "
                                   f"unknowns, interface solve: {where}", "interface": args.interface,
                       "leaf_factors": args.leaf_prec},
            "wall_ms_per_step": 1e3 * wall / nsteps,
            "gpu_leaf_ms_per_step": leaf_ms / nsteps,
            "interface_ms_per_step": (iface_ms / nsteps) if gpu_iface else 1e3 * host_s / nsteps,
            "host_sparse_lu_solve_ms": 1e3 * host_s / nsteps,
            "graphs": True,
            "setup": {"gpu_dtn_and_factor_s": t_gpu_setup, "gpu_interface_factor_s": t_iface_setup,
                      "host_assembly_and_lu_s": t_host_setup},
            "max_abs_err_vs_exact": err, "box_failures": fails}
    if info is not None:
        line["interface_factor"] = {"merges": info[0], "levels": info[1], "largest_separator": info[2],
                                    "device_bytes": info[3]}
        # algorithmic bytes of one solve: every stored W^-1, S and E read once
        # (levels padded to their largest separator s and boundary e)
        nodes, _ = H.hps_interface_plan(p, (nbx, nbx, nbx))
        sbytes = 0.0
        for hgt in range(1, int(nodes[:, 2].max()) + 1):
            sel = nodes[nodes[:, 2] == hgt]
            s_, e_ = int(sel[:, 5].max()) * qq, int((sel[:, 4] + sel[:, 6]).max()) * qq
            sbytes += 8.0 * len(sel) * (s_ * s_ + 2 * s_ * e_)
        peaks, src = measured_peaks()
        gbs = sbytes / (iface_ms / nsteps / 1e3) / 1e9
        line["interface_solve"] = {"bound": "hbm", "bytes_per_solve": sbytes, "achieved": gbs, "unit": "GB/s",
                                   "peak": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"],
                                   "peak_source": src}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "uneven":
        run_uneven(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "factored":
        run_factored(args)
    elif args.workload == "timestep":
        run_timestep(args)
    elif args.workload == "dirichlet":
        run_dirichlet(args)
    elif args.workload == "accuracy":
        run_accuracy(args)
    elif args.workload == "leaf2d":
        run_leaf2d(args)
    elif args.workload == "cross":
        run_cross(args)
    elif args.workload == "iti":
        run_iti(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
