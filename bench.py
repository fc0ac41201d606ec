#!/usr/bin/env python3
"""Reaction-step throughput (cells/s) of the GB300 library on a seeded synthetic field.

One step = one df_chem_step over the whole field (a0 compaction, a1-a5 EoS and inputs,
a6-a7 network, a8-a10 de-normalisation, Newton T recovery, write-back). Default workload:
the 2^20-cell 1D supercritical mixing layer with the 30-species mechanism and the
32-1600-800-400-30 network, every cell reacting, network in BF16 on tcgen05.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32|fp8]
                  [--impl ours|reference]

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank advances its own field of
the same size (weak scaling, no collective on the data path); value = all cells / max time.
At N = 1 the line also carries shortened runs of the 16M-cell, 30 %-reacting FP8 workload and
of the 64M-cell (400^3) 3D field under "configs", each with its errors against the FP64
oracle and the BDF truth.
--impl reference times the FP64 CPU oracle (the only reference this method has) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reaction-step cells/s (BF16/FP8 vs FP32) at stated dY/T error vs FP64 oracle"
UNIT = "cells/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="step", choices=["step", "train", "jacobian", "solver", "propnet"],
                    help="step: the reaction step (headline); train: Adam steps on training "
                         "states; jacobian: the step's Jacobian")
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32", "fp8"])
    ap.add_argument("--workload", default="layer1d-30sp-1m")
    ap.add_argument("--cells", type=int, default=0, help="override the workload's cell count")
    ap.add_argument("--fp32-steps", type=int, default=3, help="timed steps of the FP32 comparison")
    ap.add_argument("--cpu-sample", type=int, default=131072, help="cells of the CPU oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the shortened runs of the 16M-cell FP8 and 64M-cell workloads")
    ap.add_argument("--batch", type=int, default=0, help="reacting cells per internal batch")
    ap.add_argument("--gelu", default="tanh", choices=["tanh", "table"],
                    help="hidden activation: hardware tanh form, or the paper's tabulation")
    ap.add_argument("--fit-steps", type=int, default=2000,
                    help="propnet mode: Adam steps of each property network before timing")
    ap.add_argument("--solver-arith", default="fp64", choices=["fp64", "f2"],
                    help="solver mode: FP64 FMAs or double-float pairs on the FP32 pipes")
    ap.add_argument("--part-cells", type=int, default=0,
                    help="solver mode: cells per block row (default: the workload's)")
    ap.add_argument("--autotune", action="store_true",
                    help="time every tile width per layer (df_autotune) instead of the cost model")
    ap.add_argument("--no-autotune", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args=None, backend=None):
    """(world, rank, local) from the torchrun environment; joins the process group when
    world > 1 (NCCL when CUDA is available, else gloo: the CPU path the tests use)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v, local):
    """Maximum of v over all ranks (the slowest rank's time bounds the whole job)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = f"cuda:{local}" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world, cells_per_rank, ms_max):
    """Whole-job cells/s: every rank advances its own field of cells_per_rank cells, and the
    job takes as long as its slowest rank."""
    return world * cells_per_rank / (ms_max * 1e-3)


# DRAM traffic per row (dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture divided
# by the rows of that launch; summaries in profiles/), keyed by kernel family and network, valid
# only for the kernel source the counters were taken on (SHA-256 prefix of the file): once the
# kernel changes, the bench reports traffic as null until it is measured again. Where a file also
# holds kernels that are not the measured ones, the hash leaves out their sections (each from a
# start marker up to, not including, an end marker), so that editing them keeps the figure.
_EOS_OTHER = (("// ---------------------------------------------------------------- transport properties",
               "// ---------------------------------------------------------------- Jacobian of the step"),
              ("// ---------------------------------------------------------------- Jacobian of the step",
               "cudaError_t smem_optin()"),
              ("template <int NM>\ncudaError_t transport_nm(", "template <int NM>\ncudaError_t props_nm("),
              ("  if (e == cudaSuccess) e = smem_optin<transport_kernel<NM>>();\n",
               "  return e;\n}\n\ncudaError_t prepare_eos("),
              ("cudaError_t launch_jac_scale(", "cudaError_t launch_eos_post("),
              ("cudaError_t launch_transport(", "}  // namespace dfgb"))
MEASURED_TRAFFIC = {
    ("layer0", "32-1600-800-400-30"): ("paper_2508_18969_gb300/csrc/mlp_tc.cu", "c22bd239ff26b709", 3157.2),
    ("layer1", "32-1600-800-400-30"): ("paper_2508_18969_gb300/csrc/mlp_tc.cu", "c22bd239ff26b709", 4751.2),
    ("layer2", "32-1600-800-400-30"): ("paper_2508_18969_gb300/csrc/mlp_tc.cu", "c22bd239ff26b709", 2340.1),
    ("layer3", "32-1600-800-400-30"): ("paper_2508_18969_gb300/csrc/mlp_tc.cu", "c22bd239ff26b709", 1062.8),
    ("eos_pre", "32-1600-800-400-30"): ("paper_2508_18969_gb300/csrc/eos.cu", "c12e4383ce9da4a2", 292.1,
                                        _EOS_OTHER),
    ("eos_post", "32-1600-800-400-30"): ("paper_2508_18969_gb300/csrc/eos.cu", "c12e4383ce9da4a2", 578.5,
                                         _EOS_OTHER),
    # one block Gauss-Seidel sweep (gs_rhs_kernel + gs_sweep_kernel), per cell, FP64, 512 cells
    # per block row (profiles/solver_kernels_mesh-2m.md)
    ("gauss_seidel", "mesh-512"): ("paper_2508_18969_gb300/csrc/solver.cu", "bdf796170bcbf319", 128.1),
}


def measured_traffic(family, network, rows_per_launch):
    import hashlib
    entry = MEASURED_TRAFFIC.get((family, network))
    if entry is None:
        return None
    path, digest, per_row = entry[:3]
    others = entry[3] if len(entry) > 3 else ()
    try:
        with open(os.path.join(ROOT, path), "rb") as f:
            src = f.read()
    except OSError:
        return None
    for start, end in others:
        i = src.find(start.encode())
        j = src.find(end.encode(), i) if i >= 0 else -1
        if j < 0:
            return None
        src = src[:i] + src[j:]
    if hashlib.sha256(src).hexdigest()[:16] != digest:
        return None
    return per_row * rows_per_launch


def layer_flops(widths, rows):
    return [2.0 * widths[l] * widths[l + 1] * rows for l in range(len(widths) - 1)]


def eos_fp64_flops(n, iters_per_cell):
    """Algorithmic FP64 flops per cell of the two EoS kernels (counted from the equations:
    per composition 2n(n-1) for the three pair forms, ~20n for the species sums; ~140 per
    evaluation of Z, h, cp at one temperature)."""
    pre = 2 * n * (n - 1) + 20 * n + 140
    post = 2 * n * (n - 1) + 27 * n + 140 * iters_per_cell
    return pre, post


def cpu_oracle_leg(mech, net, T, p, Y, sel, T_react, gpu_after=None):
    """Times the FP64 oracle step on the sampled cells; if the GPU's results for the same
    cells are given, also states the GPU's error against it."""
    from oracle import step as ostep
    t0 = time.perf_counter()
    To, Yo, so = ostep.chem_step(mech, net, T[sel], p[sel], Y[:, sel], net.dt, T_react=T_react)
    dt = time.perf_counter() - t0
    out = {"value": sel.shape[0] / dt, "unit": UNIT, "cores": len(os.sched_getaffinity(0)),
           "kind": "oracle", "sample": f"{sel.shape[0]} evenly strided cells of the field, one "
           "FP64 numpy step (EoS, MLP, Newton), BLAS threads = numpy default",
           "seconds": dt}
    err = None
    if gpu_after is not None:
        err = error_stats(gpu_after[0], gpu_after[1], To, Yo)
    return out, err


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.mode == "solver":
        return run_reference_solver(args, world)
    if args.mode == "propnet":
        return run_reference_propnet(args, world)
    import synth
    from oracle import step as ostep
    w = synth.configs.WORKLOADS[args.workload]
    N = args.cells or w.n_cells
    S = min(4096, N)
    # the sample: S cells of the workload's field recipe, spread evenly over the field
    mech, net, Ts, ps, Ys = synth.configs.build(args.workload, n_cells=S)
    for _ in range(args.warmup):
        ostep.chem_step(mech, net, Ts, ps, Ys, net.dt, T_react=w.T_react)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Ts, Ys, _ = ostep.chem_step(mech, net, Ts, ps, Ys, net.dt, T_react=w.T_react)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    v = S / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "n_cells": N,
                                            "sample_cells_per_step": S},
            "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle",
                             "cores": len(os.sched_getaffinity(0)),
                             "sample": f"{S} cells of the workload's field recipe, evenly spread, per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_solver(args, world):
    """The FP64 oracle's sparse-solver step on a 64^3 instance of the mesh recipe per step."""
    name = args.workload if args.workload in SOLVER_WORKLOADS else "mesh-8m"
    sweeps = SOLVER_WORKLOADS[name]["sweeps"]
    n, own, nei, pp, g, s, b = solver_problem("mesh-256k")
    for _ in range(args.warmup):
        solver_oracle_step(n, own, nei, pp, g, s, b, sweeps)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solver_oracle_step(n, own, nei, pp, g, s, b, sweeps)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    v = n / dt
    unit = "cells/s"
    line = {"impl": "reference",
            "metric": "sparse-solver step cells/s (assembly, conversion, block Gauss-Seidel, residual)",
            "value": v, "unit": unit, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "sample_cells_per_step": n},
            "cpu_baseline": {"value": v, "unit": unit, "kind": "oracle",
                             "cores": len(os.sched_getaffinity(0)),
                             "sample": f"the mesh recipe at 64^3 ({n} cells) per step"},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_propnet(args, world):
    """The FP64 oracle's property networks (Sec. 4.1 sizes, seeded weights) on 4096 cells of the
    training-workload recipe per step."""
    import synth
    from oracle import propnet as opn
    S = 4096
    mech, _, T, p, Y = synth.configs.build("train30-1m", n_cells=S, field_seed=31)
    h, props = opn.exact(mech, T, p, Y)
    nets = [synth.make_propnet(w, mech.n, seed=41 + k, lam=0.1) for k, w in enumerate(PROPNET_WIDTHS.values())]
    for _ in range(args.warmup):
        for net in nets:
            opn.infer(net, h, p, Y)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for net in nets:
            opn.infer(net, h, p, Y)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    v = S / dt
    unit = "cells/s"
    line = {"impl": "reference",
            "metric": "property-network cells/s (rho and T networks of Sec. 4.1 sizes, BF16)",
            "value": v, "unit": unit, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "train30-1m states", "sample_cells_per_step": S},
            "cpu_baseline": {"value": v, "unit": unit, "kind": "oracle",
                             "cores": len(os.sched_getaffinity(0)),
                             "sample": f"{S} cells of the training-workload recipe per step, both networks"},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measure_peaks_live(torch, dev):
    """Dense GEMM rates of this GPU for the types MEASURED_PEAKS.json does not cover, taken the
    way it takes BF16: square library products (cuBLAS / cuBLASLt), best of several, CUDA
    events. FP8 e4m3 (torch._scaled_mm, FP32 unit scales, BF16 output) at 8192^3, FP32 without
    TF32 at 8192^3 (the plain FP32 path's ceiling), FP64 at 4096^3."""
    out = {"how": "torch._scaled_mm e4m3 8192^3 best of 10; torch.matmul fp32 (TF32 off) 8192^3 "
                  "best of 5; torch.matmul fp64 4096^3 best of 5; CUDA events"}

    def best(fn, flops, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return flops / (min(ts) * 1e-3) / 1e12

    g = torch.Generator(device=dev)
    g.manual_seed(5)
    try:
        n = 8192
        A = torch.randn(n, n, device=dev, generator=g).to(torch.float8_e4m3fn)
        B = torch.randn(n, n, device=dev, generator=g).to(torch.float8_e4m3fn).t()
        one = torch.ones((), device=dev, dtype=torch.float32)
        out["fp8_tflops"] = best(lambda: torch._scaled_mm(A, B, scale_a=one, scale_b=one,
                                                           out_dtype=torch.bfloat16), 2.0 * n ** 3, 10)
        del A, B
    except Exception as e:  # noqa: BLE001 (reported, not hidden)
        out["fp8_tflops"] = None
        out["fp8_error"] = str(e)[:200]
    old = torch.backends.cuda.matmul.allow_tf32
    try:
        torch.backends.cuda.matmul.allow_tf32 = False
        n = 8192
        A = torch.randn(n, n, device=dev, generator=g)
        B = torch.randn(n, n, device=dev, generator=g)
        out["fp32_tflops"] = best(lambda: A @ B, 2.0 * n ** 3, 5)
        n = 4096
        A = torch.randn(n, n, device=dev, dtype=torch.float64, generator=g)
        B = torch.randn(n, n, device=dev, dtype=torch.float64, generator=g)
        out["fp64_tflops"] = best(lambda: A @ B, 2.0 * n ** 3, 5)
        del A, B
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    torch.cuda.empty_cache()
    return out


# Measured pipe utilisation of the EoS kernels (ncu sm__inst_executed_pipe_* / issue active, one
# capture; summaries in profiles/), valid for the kernel source they were taken on (hash as for
# MEASURED_TRAFFIC).
MEASURED_PIPES = {
    # profiles/eos_kernels_layer1d-30sp-512k_bf16.md (full capture, 512K rows, first step)
    ("eos_pre", "32-1600-800-400-30"): ("paper_2508_18969_gb300/csrc/eos.cu", "c12e4383ce9da4a2",
                                        {"binding": "issue (FP32 double-float arithmetic)",
                                         "fma_pipe": 0.484, "alu_pipe": 0.197, "fp64_pipe": 0.012,
                                         "issue_active": 0.740, "warps_per_sm": 20.9}, _EOS_OTHER),
    ("eos_post", "32-1600-800-400-30"): ("paper_2508_18969_gb300/csrc/eos.cu", "c12e4383ce9da4a2",
                                         {"binding": "issue (FP32 double-float arithmetic)",
                                          "fma_pipe": 0.323, "alu_pipe": 0.527, "fp64_pipe": 0.037,
                                          "issue_active": 0.722, "warps_per_sm": 22.3}, _EOS_OTHER),
}


def measured_pipes(family, network):
    import hashlib
    entry = MEASURED_PIPES.get((family, network))
    if entry is None:
        return None
    path, digest, pipes = entry[:3]
    others = entry[3] if len(entry) > 3 else ()
    try:
        with open(os.path.join(ROOT, path), "rb") as f:
            src = f.read()
    except OSError:
        return None
    for start, end in others:
        i = src.find(start.encode())
        j = src.find(end.encode(), i) if i >= 0 else -1
        if j < 0:
            return None
        src = src[:i] + src[j:]
    if hashlib.sha256(src).hexdigest()[:16] != digest:
        return None
    return pipes


# algorithmic bytes per reacting cell of the EoS kernels (FP64 state, n species, K0 = n + 2
# network inputs in the network precision, FP32 network outputs):
#   eos_pre  reads T, p, Y (8 (2 + n)), writes x (K0 elements), h0 (8) and a status word (4);
#   eos_post reads O (4 n), h0 (8), T, p, Y (8 (2 + n)), writes T, Y (8 (1 + n)), status (4)
def eos_bytes(n, x_bytes):
    pre = 8 * (2 + n) + (n + 2) * x_bytes + 8 + 4
    post = 4 * n + 8 + 8 * (2 + n) + 8 * (1 + n) + 4
    return pre, post


def error_stats(Tg, Yg, Tr, Yr):
    """max / mean / p99 of |dY| (over every species of every cell) and |dT| (K)."""
    dY = np.abs(Yg - Yr)
    dT = np.abs(Tg - Tr)
    return {"max_abs_dY": float(dY.max()), "mean_abs_dY": float(dY.mean()),
            "p99_abs_dY": float(np.quantile(dY, 0.99)), "max_abs_dT_K": float(dT.max()),
            "mean_abs_dT_K": float(dT.mean()), "p99_abs_dT_K": float(np.quantile(dT, 0.99)),
            "cells": int(Tg.shape[0])}


def bdf_error_leg(mech, net, T, p, Y, sel, gpu_after):
    """The stiff-chemistry integration the network stands in for (the C BDF of the oracle, one
    thread per cell over the host cores) on the given reacting cells, timed, and the GPU step's
    error against it on the same cells (the paper's accuracy check against its stiff reference,
    Sec. 5.1, here on this project's synthetic mechanism and untrained or trained network)."""
    from oracle import truth
    t0 = time.perf_counter()
    Tb, Yb, ok, steps, _ = truth.advance(mech, T[sel], p[sel], Y[:, sel], net.dt)
    dt = time.perf_counter() - t0
    timing = {"value": sel.size / dt, "unit": UNIT, "cells": int(sel.size), "seconds": dt,
              "cores": len(os.sched_getaffinity(0)), "ok_fraction": float(np.mean(ok)),
              "mean_bdf_steps": float(np.mean(steps)),
              "what": "C BDF (orders 1-5, rtol 1e-10, atol 1e-14) of the cell chemistry over dt"}
    err = None
    if gpu_after is not None and ok.any():
        Tg, Yg = gpu_after
        err = error_stats(Tg[ok], Yg[:, ok], Tb[ok], Yb[:, ok])
        err["bdf_change_max_abs_dY"] = float(np.abs(Yb[:, ok] - Y[:, sel][:, ok]).max())
        err["what"] = ("GPU step vs the BDF-integrated state over the network's dt, on reacting "
                       "cells the BDF integrated (ok)")
    return timing, err


def step_leg(df, torch, args, name, precision, *, steps, warmup, local, world, rank,
             fp32_steps=0, e2e_steps=0, cpu_sample=0, bdf_cells=0, graph=False, cells=0):
    """Times df_chem_step on one workload and states its errors; returns a dict of results
    (rank 0's view; times are the maximum over ranks)."""
    import synth
    dev = torch.device("cuda", local)
    w = synth.configs.WORKLOADS[name]
    N = cells or w.n_cells
    t_gen = time.perf_counter()
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N, field_seed=w.seed + rank)
    t_gen = time.perf_counter() - t_gen
    prec = {"bf16": df.DF_BF16, "fp32": df.DF_FP32, "fp8": df.DF_FP8_E4M3}[precision]
    batch = args.batch or min(N, 1 << 22)
    gm = df.DF_GELU_TABLE if args.gelu == "table" else df.DF_GELU_TANH
    st = df.State(mech, net, precision=prec, T_react=w.T_react, device=local, batch_cells=batch,
                  gelu_mode=gm)
    tiles = st.autotune(n_rows=min(N, batch)) if args.autotune else st.tiles()
    tiles = [f"{t & ~df.DF_TILE_PAIR} pair" if t & df.DF_TILE_PAIR else str(t) for t in tiles]
    Td = torch.tensor(T, device=dev)
    pd = torch.tensor(p, device=dev)
    Yd = torch.tensor(Y, device=dev).contiguous()
    status = torch.empty(N, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    # cells whose first-step results are checked: an evenly strided sample for the FP64 oracle,
    # evenly spaced reacting cells for the BDF truth
    from oracle import step as ostep
    sel = np.linspace(0, N - 1, min(cpu_sample, N)).astype(np.int64) if cpu_sample else None
    act = ostep.active_cells(T, w.T_react) if bdf_cells else np.zeros(0, np.int64)
    sel_b = act[np.linspace(0, act.size - 1, min(bdf_cells, act.size)).astype(np.int64)] \
        if act.size else None
    st.chem_step(Td, pd, Yd, status=status)
    torch.cuda.synchronize()

    def gather(ix):
        if ix is None:
            return None
        d = torch.tensor(ix, device=dev)
        return Td[d].cpu().numpy(), Yd[:, d].cpu().numpy()

    first, first_b = gather(sel), gather(sel_b)

    for _ in range(warmup):
        st.chem_step(Td, pd, Yd, status=status)
    torch.cuda.synchronize()
    st.profile_read()
    st.profile_enable(True)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(steps):
            st.chem_step(Td, pd, Yd, status=status)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    st.profile_enable(False)
    prof = st.profile_read()
    rc, n_act, n_flag, iters = st.step_summary()
    ms = max_over_ranks(world, e0.elapsed_time(e1) / steps, local)
    r = {"workload": name, "precision": precision, "N": N, "mech": mech, "net": net, "w": w,
         "batch": batch, "tiles": tiles, "ms": ms, "value": weak_scaling_value(world, N, ms),
         "timed_s": e0.elapsed_time(e1) * 1e-3, "clocks": clk.summary(), "prof": prof,
         "n_act": int(n_act), "n_flag": int(n_flag), "iters": int(iters), "steps": steps,
         "field_seconds": t_gen}

    if graph:
        g = st.graph(Td, pd, Yd, status=status)
        for _ in range(2):
            g.launch()
        torch.cuda.synchronize()
        barrier(world)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for a, b in ev:
            a.record(stream)
            g.launch()
            b.record(stream)
        torch.cuda.synchronize()
        per = sorted(a.elapsed_time(b) for a, b in ev)
        r["graph_ms"] = max_over_ranks(world, float(np.mean(per)), local)
        r["graph_median_ms"] = max_over_ranks(world, float(per[len(per) // 2]), local)
        g.close()

    # end to end: the fields live in host (pinned) memory; every step goes through the C ABI's
    # host entry point (df_chem_step_host), which uploads T, p, Y, steps and downloads T, Y in
    # chunks whose copies overlap the steps of other chunks
    if e2e_steps > 0:
        Th = torch.tensor(T).pin_memory()
        ph = torch.tensor(p).pin_memory()
        Yh = torch.tensor(Y).pin_memory()
        for _ in range(2):
            st.chem_step_host(Th, ph, Yh)
        torch.cuda.synchronize()
        barrier(world)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(e2e_steps):
            st.chem_step_host(Th, ph, Yh)
        a1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(world, a0.elapsed_time(a1) / e2e_steps, local)
        r["e2e"] = {"value": world * N / (ems * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": int(8 * N * (2 + mech.n)),
                    "d2h_bytes_per_step": int(8 * N * (1 + mech.n)), "ms_per_step": ems}
        del Th, ph, Yh

    # plain FP32 step (SIMT network): the comparison the method is judged by
    if prec != df.DF_FP32 and fp32_steps > 0:
        s32 = df.State(mech, net, precision=df.DF_FP32, T_react=w.T_react, device=local,
                       batch_cells=batch)
        s32.chem_step(Td, pd, Yd, status=status)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s32.profile_enable(True)
        f0.record(stream)
        for _ in range(fp32_steps):
            s32.chem_step(Td, pd, Yd, status=status)
        f1.record(stream)
        torch.cuda.synchronize()
        p32 = s32.profile_read()
        fms = max_over_ranks(world, f0.elapsed_time(f1) / fp32_steps, local)
        r["fp32"] = {"value": world * N / (fms * 1e-3), "ms_per_step": fms,
                     "kernels_ms_per_step": {k: v[1] / fp32_steps for k, v in p32.items()}}
        s32.close()
    st.close()
    del Td, pd, Yd, status
    torch.cuda.empty_cache()

    if rank == 0 and sel is not None:
        r["cpu_baseline"], r["error_vs_fp64_oracle"] = cpu_oracle_leg(mech, net, T, p, Y, sel,
                                                                      w.T_react, first)
    if rank == 0 and sel_b is not None:
        r["bdf_truth_cpu"], r["error_vs_bdf_truth"] = bdf_error_leg(mech, net, T, p, Y, sel_b, first_b)
    return r


def roofline_families(r, pk, pk_src, live, df, steps_timed_s):
    """Roofline of every kernel family of one step leg: algorithmic flops or bytes per step over
    the family's device time per step (the library's CUDA events on the launch stream)."""
    w, mech, prec = r["w"], r["mech"], r["precision"]
    rows = r["n_act"]
    fl = layer_flops(w.widths, rows)
    iters_per_cell = r["iters"] / max(rows, 1)
    pre_f, post_f = eos_fp64_flops(mech.n, iters_per_cell)
    xb = {"bf16": 2, "fp8": 1, "fp32": 4}[prec]
    pre_b, post_b = eos_bytes(mech.n, xb)
    # the timed region is short (well under the seconds a power-capped loop needs to settle), so
    # tensor kernels are held to the burst BF16 figure; FP8 to the live-measured FP8 GEMM rate
    burst = steps_timed_s < 2.0
    bf16_peak = pk["bf16_tflops"] if burst else pk["bf16_tflops_sustained"]
    bf16_src = f"bf16_tflops ({pk_src}, burst: timed region {steps_timed_s:.2f} s)" if burst \
        else f"bf16_tflops_sustained ({pk_src}, timed region {steps_timed_s:.2f} s)"
    fams = {k: (v[0], v[1]) for k, v in r["prof"].items()}
    roofs = {}
    net_str = "-".join(str(x) for x in w.widths)
    rows_per_launch = min(rows, r["batch"])
    for fam, (launches, tot) in fams.items():
        avg_s = tot / r["steps"] * 1e-3
        if fam.startswith("layer") and prec != "fp32":
            ls = [int(v) for v in fam[5:].split("+")]   # "layer0+1": layers 0 and 1 fused
            if prec == "fp8" and live.get("fp8_tflops"):
                peak, src = live["fp8_tflops"], "fp8 e4m3 GEMM measured live (torch._scaled_mm 8192^3)"
            else:
                peak, src = bf16_peak, bf16_src
            ach = sum(fl[l] for l in ls) / avg_s / 1e12
            roofs[fam] = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                          "frac": ach / peak, "peak_source": src,
                          "kernel": f"tc_gemm {fam}" if len(ls) == 1 else
                          f"fused01 (layers {ls[0]} and {ls[-1]}; algorithmic flops, the recomputed "
                          "layer-0 blocks not counted)"}
        elif fam.startswith("layer"):
            l = int(fam[5:])
            peak = live.get("fp32_tflops") or 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e-6
            ach = fl[l] / avg_s / 1e12
            roofs[fam] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                          "frac": ach / peak, "kernel": f"sgemm {fam}",
                          "peak_source": "fp32 GEMM (TF32 off) measured live" if live.get("fp32_tflops")
                          else "FP32 FMA: 152 SMs x 128 lanes x 2 flop x max SM clock"}
        elif fam in ("eos_pre", "eos_post"):
            per_b = pre_b if fam == "eos_pre" else post_b
            per_f = pre_f if fam == "eos_pre" else post_f
            ach = per_b * rows / avg_s / 1e9
            e = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "frac": ach / pk["hbm_gbs"], "kernel": fam, "peak_source": f"hbm_gbs ({pk_src})",
                 "algorithmic_bytes_per_cell": per_b}
            f64 = live.get("fp64_tflops")
            e["fp64_equivalent"] = {
                "flop_per_cell": per_f, "achieved_tflops": per_f * rows / avg_s / 1e12,
                "fp64_peak_tflops": f64, "frac": (per_f * rows / avg_s / 1e12 / f64) if f64 else None,
                "note": "the state is evaluated in double-float on the FP32 pipes (no FP64 "
                        "arithmetic in the hot loops), so this can exceed 1"}
            e["ncu_pipes"] = measured_pipes(fam, net_str)
            roofs[fam] = e
        else:
            ach = (12.0 * r["N"]) / avg_s / 1e9
            roofs[fam] = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                          "frac": ach / pk["hbm_gbs"], "kernel": fam,
                          "peak_source": f"hbm_gbs ({pk_src})"}
    for fam_name, e in roofs.items():
        e["traffic"] = measured_traffic(fam_name, net_str, rows_per_launch)
        if e["traffic"] is not None:
            e["traffic_source"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum per row x rows per launch"
    # whole step: sum over phases of the larger of (tensor flops / tensor peak) and
    # (algorithmic bytes / HBM): the network's flops, the EoS kernels' state traffic and the
    # compaction's reads, against the step's measured time
    tpk = roofs.get("layer1", {}).get("peak") if prec != "fp32" else None
    ph = {"compact": 12.0 * r["N"] / (pk["hbm_gbs"] * 1e9),
          "eos_pre": pre_b * rows / (pk["hbm_gbs"] * 1e9),
          "eos_post": post_b * rows / (pk["hbm_gbs"] * 1e9)}
    for l in range(len(fl)):
        if tpk:
            ph[f"layer{l}"] = fl[l] / (tpk * 1e12)
    bound_ms = sum(ph.values()) * 1e3
    step = {"bound_ms": bound_ms, "achieved_ms": r["ms"], "frac": bound_ms / r["ms"],
            "phases_ms": {k: v * 1e3 for k, v in ph.items()},
            "what": "sum over phases of max(tensor flops / tensor peak, algorithmic bytes / HBM) "
                    "over the measured step time"} if tpk else None
    return roofs, step


def run_ours(args):
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2508_18969_gb300 as df

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cpu_sample = 0 if args.no_cpu_baseline else args.cpu_sample
    bdf_cells = 0 if args.no_cpu_baseline else 2048
    r = step_leg(df, torch, args, args.workload, args.precision, steps=args.steps,
                 warmup=args.warmup, local=local, world=world, rank=rank,
                 fp32_steps=args.fp32_steps, e2e_steps=0 if args.no_e2e else max(3, args.steps // 2),
                 cpu_sample=cpu_sample, bdf_cells=bdf_cells, graph=True, cells=args.cells)
    live = measure_peaks_live(torch, dev) if rank == 0 else {}

    # the larger workloads, each in a shortened run (one GPU only: their fields are per rank)
    configs = {}
    if world == 1 and not args.no_configs:
        for key, name, prec, steps, e2e_steps, smp in (
                ("react30-16m_fp8", "react30-16m", "fp8", 10, 3, 4096),
                ("mix3d-30sp-64m_bf16", "mix3d-30sp-64m", "bf16", 4, 2, 4096)):
            try:
                c = step_leg(df, torch, args, name, prec, steps=steps, warmup=3, local=local,
                             world=world, rank=rank, e2e_steps=e2e_steps,
                             cpu_sample=0 if args.no_cpu_baseline else smp,
                             bdf_cells=0 if args.no_cpu_baseline else 512)
            except Exception as e:  # noqa: BLE001 (the line states the omission)
                configs[key] = {"omitted": f"{type(e).__name__}: {str(e)[:200]}"}
                continue
            pk, pk_src = peaks()
            roofs, step_roof = roofline_families(c, pk, pk_src, live, df, c["timed_s"])
            dom = max(roofs, key=lambda k: c["prof"][k][1])
            configs[key] = {
                "workload": name, "precision": prec, "n_cells": c["N"], "reacting_cells": c["n_act"],
                "T_react_K": c["w"].T_react, "steps": steps, "value": c["value"], "unit": UNIT,
                "ms_per_step": c["ms"], "active_cells_per_s": c["n_act"] / (c["ms"] * 1e-3),
                "e2e": c.get("e2e"), "clocks": c["clocks"], "tile_widths": c["tiles"],
                "roofline": roofs[dom], "step_roofline": step_roof,
                "kernels_ms_per_step": {k: v[1] / steps for k, v in c["prof"].items()},
                "error_vs_fp64_oracle": c.get("error_vs_fp64_oracle"),
                "error_vs_bdf_truth": c.get("error_vs_bdf_truth"),
                "flagged_cells": c["n_flag"], "field_seconds": c["field_seconds"],
                "fp32_step": "not run for this workload (the FP32 comparison is the 2^20-cell line's)"}
    if rank != 0:
        return 0

    pk, pk_src = peaks()
    roofs, step_roof = roofline_families(r, pk, pk_src, live, df, r["timed_s"])
    dom = max(roofs, key=lambda k: r["prof"][k][1])
    w, mech = r["w"], r["mech"]
    N, batch = r["N"], r["batch"]
    kpl = len(w.widths) - 1 + 2            # per batch: eos_pre + layers + eos_post
    nb = (N + batch - 1) // batch
    fp32 = r.get("fp32")
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"bf16": "bf16+f64", "fp32": "f32+f64", "fp8": "fp8e4m3+f64"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, "n_cells": N, "n_species": mech.n, "batch_cells": batch,
                   "network": "-".join(str(x) for x in w.widths), "precision": args.precision,
                   "reacting_cells": r["n_act"], "T_react_K": w.T_react, "tile_widths": r["tiles"],
                   "gelu": args.gelu,
                   "l2": "inputs larger than L2 (fields 8*(2+n)*N bytes, activations GBs)"},
        "clocks": r["clocks"],
        "e2e": r.get("e2e"),
        "gpu_launches": int((3 + kpl * nb) * args.steps),
        "graph_ms_per_step": r["graph_ms"],
        "graph_median_ms_per_step": r["graph_median_ms"],
        "graph_value": world * N / (r["graph_ms"] * 1e-3),
        "roofline": roofs[dom],
        "roofline_by_family": roofs,
        "step_roofline": step_roof,
        "measured_peaks_live": live,
        "cpu_baseline": r.get("cpu_baseline"),
        "bdf_truth_cpu": r.get("bdf_truth_cpu"),
        "kernels_ms_per_step": {k: v[1] / args.steps for k, v in r["prof"].items()},
        "newton_iterations_per_cell": r["iters"] / max(r["n_act"], 1),
        "flagged_cells": r["n_flag"],
        "fp32_step": fp32,
        "speedup_vs_fp32": (r["value"] / fp32["value"]) if fp32 else None,
        "error_vs_fp64_oracle": r.get("error_vs_fp64_oracle"),
        "error_vs_bdf_truth": r.get("error_vs_bdf_truth"),
        "configs": configs if world == 1 else "larger workloads run at N = 1 only",
    }
    print(json.dumps(line), flush=True)
    return 0


def _boxcox(y, lam):
    return (np.maximum(y, 0.0) ** lam - 1.0) / lam


def run_train(args):
    """Training (the differentiation configuration): the 30-species network is taught the change
    that a stiff (BDF) integration of each state's chemistry makes over the network's dt, with
    BF16 compute and FP32 masters, Adam, full batches of 65,536 states. The BDF integration of
    the training and held-out states is this mode's CPU baseline (timed on the host cores); its
    results are the targets. After the timed steps the fit continues to --fit-steps, and the
    trained network's reaction step on held-out states is compared with their BDF-integrated
    state in FP32, BF16 and FP8, beside the untrained network and the no-change prediction."""
    import copy
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2508_18969_gb300 as df
    import synth
    from oracle import truth
    from oracle import step as ostep
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name = "train30-1m" if args.workload == "layer1d-30sp-1m" else args.workload
    w = synth.configs.WORKLOADS[name]
    B = args.batch or 65536
    S_test = 8192
    S = B + S_test
    mech, net0, T, p, Y = synth.configs.build(name, n_cells=S, field_seed=w.seed + rank)
    t0 = time.perf_counter()
    Tb, Yb, ok, bdf_steps, _ = truth.advance(mech, T, p, Y, net0.dt)
    bdf_s = time.perf_counter() - t0
    bdf = {"value": S / bdf_s, "unit": "states/s", "cores": len(os.sched_getaffinity(0)),
           "kind": "oracle", "seconds": bdf_s, "ok_fraction": float(np.mean(ok)),
           "mean_bdf_steps": float(np.mean(bdf_steps)),
           "sample": f"{S} states of the {name} recipe, each integrated over dt = {net0.dt:g} s by "
                     "the C BDF (orders 1-5, rtol 1e-10, atol 1e-14): the training targets"}
    keep = np.flatnonzero(ok)
    tr, te = keep[keep < B], keep[keep >= B]
    # a trained network's outputs are normalised by the statistics of its targets
    du = _boxcox(Yb[:, tr], net0.lam) - _boxcox(Y[:, tr], net0.lam)
    net = copy.copy(net0)
    net.out_mean = du.mean(axis=1)
    net.out_std = du.std(axis=1) + 1e-12
    prec = df.DF_BF16 if args.precision != "fp32" else df.DF_FP32
    st = df.State(mech, net, precision=prec, T_react=0.0, device=local)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    batch = (d(T[tr]), d(p[tr]), d(Y[:, tr]), d(Yb[:, tr]))
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    lr = 1e-3
    for i in range(args.warmup):
        st.train_step(*batch, lr=lr, loss=loss)
    torch.cuda.synchronize()
    first_loss = float(loss.item())
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st.profile_read()
    st.profile_enable(True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for i in range(args.steps):
            st.train_step(*batch, lr=lr, loss=loss)
        e1.record(stream)
        torch.cuda.synchronize()
    st.profile_enable(False)
    prof = st.profile_read()
    ms = max_over_ranks(world, e0.elapsed_time(e1) / args.steps, local)
    # the fit continues (untimed): constant step size, then a tenth of it for the last quarter
    losses = []
    done = args.warmup + args.steps
    for i in range(done, max(args.fit_steps, done)):
        st.train_step(*batch, lr=lr if i < 0.75 * args.fit_steps else 0.1 * lr, loss=loss)
        if i % 100 == 0:
            losses.append(float(loss.item()))
    torch.cuda.synchronize()
    last_loss = float(loss.item())
    if rank != 0:
        return 0

    # held-out states: the reaction step with the trained network against the BDF truth
    trained = copy.copy(net)
    trained.W, trained.b = [], []
    for l in range(net.n_layers):
        Wl, bl = st.params(l, widths=net.widths)
        trained.W.append(Wl.cpu().numpy().astype(np.float64))
        trained.b.append(bl.cpu().numpy().astype(np.float64))

    def held_out(nw_, P):
        s2 = df.State(mech, nw_, precision=P, T_react=0.0, device=local)
        Td, Yd = d(T[te]), d(Y[:, te])
        s2.chem_step(Td, d(p[te]), Yd)
        torch.cuda.synchronize()
        out = error_stats(Td.cpu().numpy(), Yd.cpu().numpy(), Tb[te], Yb[:, te])
        s2.close()
        return out

    ident = error_stats(T[te], Y[:, te], Tb[te], Yb[:, te])
    To, Yo, _ = ostep.chem_step(mech, trained, T[te], p[te], Y[:, te], net.dt, T_react=0.0)
    errs = {"what": f"{te.size} held-out states (not trained on): reaction step vs their BDF-integrated "
                    "state over dt",
            "no_change_prediction": ident,
            "untrained_network_bf16": held_out(net, df.DF_BF16),
            "trained_fp64_oracle": error_stats(To, Yo, Tb[te], Yb[:, te]),
            "trained_fp32": held_out(trained, df.DF_FP32),
            "trained_bf16": held_out(trained, df.DF_BF16),
            "trained_fp8": held_out(trained, df.DF_FP8_E4M3)}
    pk, pk_src = peaks()
    flops = 3.0 * sum(layer_flops(w.widths, B))   # forward, input gradients, weight gradients
    fam = {k: v[1] / args.steps for k, v in prof.items()}
    gemm_ms = fam.get("train_forward", 0.0) + fam.get("train_backward", 0.0)
    ach = flops / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else None
    burst = e0.elapsed_time(e1) * 1e-3 < 2.0
    tpk = pk["bf16_tflops"] if burst else pk["bf16_tflops_sustained"]
    line = {"metric": "training states/s (Adam steps)", "value": weak_scaling_value(world, B, ms),
            "unit": "states/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16+f32 master" if prec == df.DF_BF16 else "f32", "data": "synthetic",
            "config": {"workload": name, "states": int(tr.size), "held_out": int(te.size), "batch": B,
                       "network": "-".join(map(str, w.widths)), "targets": "BDF over dt",
                       "fit_steps": max(args.fit_steps, done),
                       "optimizer": "Adam lr 1e-3 (1e-4 for the last quarter) betas (0.9, 0.999) eps 1e-8"},
            "clocks": clk.summary(), "kernels_ms_per_step": fam,
            "roofline": {"bound": "tensor", "achieved": ach, "peak": tpk, "unit": "TFLOP/s",
                         "frac": (ach / tpk) if ach else None, "traffic": None,
                         "kernel": "training forward + backward GEMMs (3 x forward flops)",
                         "peak_source": ("bf16_tflops" if burst else "bf16_tflops_sustained") + f" ({pk_src})"},
            "cpu_baseline": bdf,
            "loss_first": first_loss, "loss_last": last_loss, "loss_every_100_steps": losses,
            "held_out_error_vs_bdf_truth": errs}
    print(json.dumps(line), flush=True)
    return 0


def run_jacobian(args):
    """Jacobian throughput: d(Y' - Y)/d(T, Y) and dT'/d(T, Y) of every cell of the field, with
    the relative Frobenius error per cell against the oracle's central differences on a strided
    1024-cell subset."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2508_18969_gb300 as df
    import synth
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name = "train30-1m" if args.workload == "layer1d-30sp-1m" else args.workload
    w = synth.configs.WORKLOADS[name]
    N = args.cells or w.n_cells
    mech, net, T, p, Y = synth.configs.build(name, n_cells=N, field_seed=w.seed + rank)
    prec = {"bf16": df.DF_BF16, "fp32": df.DF_FP32, "fp8": df.DF_BF16}[args.precision]
    st = df.State(mech, net, precision=prec, T_react=0.0, device=local)
    Td, pd, Yd = (torch.tensor(a, device=dev) for a in (T, p, Y))
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        J, dT = st.chem_jacobian(Td, pd, Yd)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            J, dT = st.chem_jacobian(Td, pd, Yd)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(world, e0.elapsed_time(e1) / args.steps, local)
    # the step's reverse-mode product (df_chem_step_vjp): each batch's Jacobian, then its
    # contraction with the cotangents of (T', Y')
    rng = np.random.default_rng(1 + rank)
    gTd = torch.tensor(rng.uniform(-1e-3, 1e-3, N), device=dev)
    gYd = torch.tensor(rng.uniform(-1.0, 1.0, Y.shape), device=dev)
    for _ in range(args.warmup):
        st.chem_step_vjp(Td, pd, Yd, gTd, gYd)
    torch.cuda.synchronize()
    barrier(world)
    e0.record(stream)
    for _ in range(args.steps):
        st.chem_step_vjp(Td, pd, Yd, gTd, gYd)
    e1.record(stream)
    torch.cuda.synchronize()
    vjp_ms = max_over_ranks(world, e0.elapsed_time(e1) / args.steps, local)
    if rank != 0:
        return 0
    err = None
    if not args.no_cpu_baseline:
        from oracle import step as ostep
        sel = np.linspace(0, N - 1, min(1024, N)).astype(np.int64)
        Jo, dTo = ostep.chem_step_jacobian_fd(mech, net, T[sel], p[sel], Y[:, sel], dY_rel=1e-4)
        Jg = J[torch.tensor(sel, device=dev)].cpu().numpy().astype(np.float64)
        # columns of species below the difference floor are NaN in the reference: compare the
        # finite columns of each cell
        fin = np.isfinite(Jo) & np.isfinite(Jg)
        num = np.sqrt(np.where(fin, (Jg - Jo) ** 2, 0.0).sum(axis=(1, 2)))
        den = np.sqrt(np.where(fin, Jo ** 2, 0.0).sum(axis=(1, 2)))
        ok = den > 0
        rel = num[ok] / den[ok]
        err = {"cells": int(ok.sum()), "finite_columns_fraction": float(fin.mean()),
               "median_rel_frobenius": float(np.median(rel)),
               "p99_rel_frobenius": float(np.quantile(rel, 0.99)), "max_rel_frobenius": float(rel.max()),
               "reference": "oracle central differences (dT 1e-6 T, dY 1e-4 Y)"}
    ntan = mech.n + 1
    flops = ntan * sum(layer_flops(w.widths, 1)) + sum(layer_flops(w.widths, 1))
    line = {"metric": "step Jacobians cells/s", "value": weak_scaling_value(world, N, ms),
            "unit": "cells/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if prec == df.DF_BF16 else "f32", "data": "synthetic",
            "config": {"workload": name, "n_cells": N, "network": "-".join(map(str, w.widths)),
                       "tangents_per_cell": ntan},
            "clocks": clk.summary(),
            "network_tflops": flops * N / (ms * 1e-3) / 1e12,
            "error_vs_finite_differences": err,
            "reverse_mode_product": {"entry_point": "df_chem_step_vjp", "ms_per_step": vjp_ms,
                                     "cells_per_s": weak_scaling_value(world, N, vjp_ms),
                                     "over_jacobian": vjp_ms / ms}}
    print(json.dumps(line), flush=True)
    return 0


# Sparse-solver workload (Sec. 3.2): a seeded 256 x 256 x 128 hexahedral mesh with random
# extra diagonal faces, randomly numbered, decomposed into block rows of 512 cells.
SOLVER_WORKLOADS = {
    "mesh-8m": dict(dims=(256, 256, 128), part_cells=512, seed=7, p_extra=0.15, sweeps=2),
    "mesh-2m": dict(dims=(128, 128, 128), part_cells=512, seed=7, p_extra=0.15, sweeps=2),
    "mesh-256k": dict(dims=(64, 64, 64), part_cells=512, seed=7, p_extra=0.15, sweeps=2),
}


def solver_problem(name, seed_offset=0, part_cells=0):
    """Mesh of the named workload, decomposed and renumbered by the library's host code:
    (n, owner, neighbour, part_ptr, face coefficients, cell sources, right-hand side)."""
    import synth
    from paper_2508_18969_gb300 import solver as sol
    w = SOLVER_WORKLOADS[name]
    m = synth.mesh.grid_mesh(*w["dims"], seed=w["seed"] + seed_offset, p_extra=w["p_extra"])
    parts = max(1, m.n_cells // (part_cells or w["part_cells"]))
    new_of_old, pp = sol.mesh_decompose(m.n_cells, m.owner, m.neighbour, parts)
    own, nei, face_old, _ = sol.mesh_renumber(m.n_cells, m.owner, m.neighbour, new_of_old)
    s = np.empty(m.n_cells)
    s[new_of_old] = m.cell_source
    b = synth.mesh.rhs_vector(m.n_cells, seed=w["seed"] + seed_offset + 4)
    return m.n_cells, own, nei, pp, np.ascontiguousarray(m.face_coeff[face_old]), s, b


def solver_bytes(info, sweeps):
    """Algorithmic bytes per launch of each sparse kernel: every array of the block format,
    every vector and every LDU array moved once (the halo values once per halo cell)."""
    n, nf, nnz_o, nh = info["n_cells"], info["n_faces"], info["nnz_offblock"], info["n_halo"]
    nnz_b = 2 * nf - nnz_o
    return {
        "laplacian": 32 * nf + 20 * n,
        "convert": 40 * nf + 24 * n,
        "spmv": 32 * n + 10 * nnz_b + 12 * nnz_o,
        "residual": 40 * n + 10 * nnz_b + 12 * nnz_o,
        "gauss_seidel": 41 * n + 10 * nnz_b + 12 * nnz_o + 16 * nh,
    }


def solver_oracle_step(n, own, nei, pp, g, s, b, sweeps):
    """One solver step of the FP64 oracle: assemble, build the matrix, sweep, residual."""
    from oracle import solver as osol
    lo, d, up = osol.fv_laplacian(n, own, nei, g, s)
    A = osol.ldu_matrix(n, own, nei, lo, d, up)
    x = osol.gauss_seidel(A, b, np.zeros(n), pp, sweeps)
    return x, osol.residual(A, b, x)


def solver_cpu_leg(sweeps, name="mesh-2m"):
    import time
    n, own, nei, pp, g, s, b = solver_problem(name)
    t0 = time.perf_counter()
    solver_oracle_step(n, own, nei, pp, g, s, b, sweeps)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "cells/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": f"the same recipe at {name} ({n} cells), one oracle step (scipy sparse; BLAS "
                      "threads = default)", "seconds": dt}


def run_solver(args):
    """Sparse-solver step throughput (Sec. 3.2) on one GPU: face-to-cell assembly of the
    finite-volume Laplacian, LDU -> block conversion, block Gauss-Seidel sweeps from x = 0 and
    the residual, per step. Cells/s = cells / step time."""
    import torch
    import __graft_entry__ as g_
    g_.build()
    from paper_2508_18969_gb300 import solver as sol
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    name = args.workload if args.workload in SOLVER_WORKLOADS else "mesh-8m"
    sweeps = SOLVER_WORKLOADS[name]["sweeps"]
    part_cells = args.part_cells or SOLVER_WORKLOADS[name]["part_cells"]
    n, own, nei, pp, gf, sc, b = solver_problem(name, seed_offset=rank, part_cells=part_cells)
    arith = 1 if args.solver_arith == "f2" else 0
    S = sol.Solver(n, own, nei, pp, device=local, arithmetic=arith)
    info = S.info()
    f64 = dict(dtype=torch.float64, device=dev)
    gd, sd, bd = (torch.tensor(a, **f64) for a in (gf, sc, b))
    lo, dg, up = torch.empty(own.size, **f64), torch.empty(n, **f64), torch.empty(own.size, **f64)
    x, r = torch.zeros(n, **f64), torch.empty(n, **f64)
    stream = torch.cuda.current_stream()

    def step():
        S.fv_laplacian(gd, sd, out=(lo, dg, up))
        S.convert(lo, dg, up)
        x.zero_()
        S.gauss_seidel(bd, x, sweeps)
        S.residual(bd, x, r)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(world, e0.elapsed_time(e1) / args.steps, local)
    # per kernel: each launched alone, back to back, CUDA events on the launch stream
    reps = 20
    kern = {}
    y = torch.empty(n, **f64)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        z.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(z) / reps

    kern["laplacian"] = timed(lambda: S.fv_laplacian(gd, sd, out=(lo, dg, up)))
    kern["convert"] = timed(lambda: S.convert(lo, dg, up))
    kern["spmv"] = timed(lambda: S.spmv(x, y))
    kern["residual"] = timed(lambda: S.residual(bd, x, r))
    kern["gauss_seidel"] = timed(lambda: S.gauss_seidel(bd, x, 1))   # halo gather + one sweep
    resid = float(torch.linalg.vector_norm(r).item()) / float(np.linalg.norm(b))
    if rank != 0:
        return 0
    pk, pk_src = peaks()
    by = solver_bytes(info, sweeps)
    fam = {k: {"ms": v, "GB/s": by[k] / (v * 1e-3) / 1e9,
               "frac": by[k] / (v * 1e-3) / 1e9 / pk["hbm_gbs"]} for k, v in kern.items()}
    gs = fam["gauss_seidel"]
    e2e = None
    if not args.no_e2e:
        hp = {k: torch.tensor(a, dtype=torch.float64).pin_memory() for k, a in
              (("g", gf), ("s", sc), ("b", b))}
        xh = torch.empty(n, dtype=torch.float64).pin_memory()

        def e2e_step():
            gd.copy_(hp["g"], non_blocking=True)
            sd.copy_(hp["s"], non_blocking=True)
            bd.copy_(hp["b"], non_blocking=True)
            step()
            xh.copy_(x, non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            e2e_step()
        z.record(stream)
        torch.cuda.synchronize()
        ems = a.elapsed_time(z) / args.steps
        e2e = {"value": n / (ems * 1e-3), "unit": "cells/s", "ms_per_step": ems,
               "h2d_bytes_per_step": 8 * (own.size + 2 * n), "d2h_bytes_per_step": 8 * n}
    cpu = None if args.no_cpu_baseline else solver_cpu_leg(sweeps)
    line = {"metric": "sparse-solver step cells/s (assembly, conversion, block Gauss-Seidel, residual)",
            "value": weak_scaling_value(world, n, ms), "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if arith == 0 else "f64 storage, double-float (2 x f32) arithmetic",
            "data": "synthetic",
            "config": {"workload": name, "n_cells": n, "n_faces": int(own.size),
                       "arithmetic": args.solver_arith,
                       "block_rows": int(info["n_parts"]), "cells_per_block_row": part_cells,
                       "offblock_fraction_of_nnz": info["nnz_offblock"] / info["nnz"],
                       "gauss_seidel_runs": int(info["n_runs"]), "sweeps_per_step": sweeps,
                       "l2": "matrix and vectors larger than L2 (block format + LDU arrays ~1 GB)"},
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": 4 + 2 * sweeps,
            "roofline": {"bound": "hbm", "achieved": gs["GB/s"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": gs["frac"],
                         "traffic": measured_traffic("gauss_seidel", f"mesh-{part_cells}", n)
                         if arith == 0 else None,
                         "kernel": "gauss_seidel (halo gather + one sweep)",
                         "peak_source": f"hbm_gbs ({pk_src})"},
            "kernels": fam, "algorithmic_bytes": by,
            "relative_residual_after_step": resid,
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


# Property networks of Sec. 4.1's sizes (PRNet-style surrogates of the real-fluid state) on the
# 30-species mechanism: density (hidden 1024-512-256) and temperature (hidden 2048-1024-512),
# one output each; transport outputs are not modelled.
PROPNET_WIDTHS = {"rho": [32, 1024, 512, 256, 1], "T": [32, 2048, 1024, 512, 4]}
# rows of the property stack each network learns: density; temperature and the logarithms of
# viscosity, thermal conductivity and thermal diffusivity (the transport properties span
# decades, so the network regresses their logarithms)
PROPNET_ROWS = {"rho": [0], "T": [1, 2, 3, 4]}


def run_propnet(args):
    """Property-network throughput and accuracy: the density network and the temperature-and-
    transport network (T, viscosity, thermal conductivity, thermal diffusivity) trained (BF16,
    Adam, batch 65536) on 2^20 states of the training workload whose exact properties the GPU
    equation of state and transport model give, then run on 2^20 other cells; the explicit path
    (T from h by Newton on the Peng-Robinson h(T), the reaction step's a9, from a start 10 % off,
    and df_transport_props) is timed beside it. A step = both networks on all cells."""
    import torch
    import __graft_entry__ as g_
    g_.build()
    import paper_2508_18969_gb300 as df
    import synth
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N = args.cells or (1 << 20)
    mech, chem_net, T, p, Y = synth.configs.build("train30-1m", n_cells=2 * N, field_seed=31 + rank)
    chem = df.State(mech, chem_net, precision=df.DF_BF16, T_react=0.0, device=local)
    Td, pd, Yd = (torch.tensor(a, device=dev) for a in (T, p, Y))
    rho, h, _, _ = chem.real_fluid_props(Td, pd, Yd)
    mu, lam, alp = chem.transport_props(Td, pd, Yd)
    props = torch.stack([rho, Td, mu.log(), lam.log(), alp.log()])
    tr, te = slice(0, N), slice(N, 2 * N)
    bc = (Yd[:, tr].clamp(min=0.0) ** 0.1 - 1.0) / 0.1
    v = torch.cat([h[None, tr], pd[None, tr], bc], dim=0)
    in_mean, in_std = v.mean(dim=1).cpu().numpy(), v.std(dim=1).cpu().numpy() + 1e-3
    nets, pns = {}, {}
    for k, (name, widths) in enumerate(PROPNET_WIDTHS.items()):
        rows = PROPNET_ROWS[name]
        nets[name] = synth.make_propnet(widths, mech.n, seed=41 + k, lam=0.1, in_mean=in_mean,
                                        in_std=in_std,
                                        out_mean=[float(props[r, tr].mean()) for r in rows],
                                        out_std=[float(props[r, tr].std()) for r in rows])
        pns[name] = df.PropNet(nets[name], precision=df.DF_BF16, device=local)
    B = 65536
    batches = [(h[i:i + B], pd[i:i + B], Yd[:, i:i + B].contiguous(), props[:, i:i + B].contiguous())
               for i in range(0, N - B + 1, B)]
    fit = {}
    for k, name in enumerate(PROPNET_WIDTHS):
        loss = None
        first = None
        for step in range(args.fit_steps):
            hb, pb, Yb, tb = batches[step % len(batches)]
            loss = pns[name].fit_step(hb, pb, Yb, tb[PROPNET_ROWS[name]].contiguous(),
                                      lr=1e-3 if step < args.fit_steps // 2 else 3e-4)
            if step == 0:
                first = float(loss.item())
        fit[name] = {"steps": args.fit_steps, "batch": B, "loss_first": first,
                     "loss_last": float(loss.item())}
    he, pe, Ye = h[te].contiguous(), pd[te].contiguous(), Yd[:, te].contiguous()
    outs = {name: torch.empty(len(PROPNET_ROWS[name]), N, dtype=torch.float64, device=dev)
            for name in PROPNET_WIDTHS}

    def step():
        for name in PROPNET_WIDTHS:
            pns[name].infer(he, pe, Ye, out=outs[name])

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    for name in PROPNET_WIDTHS:
        pns[name].profile_read()
        pns[name].profile_enable(True)
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(world, e0.elapsed_time(e1) / args.steps, local)
    fam = {}
    for name in PROPNET_WIDTHS:
        pns[name].profile_enable(False)
        for f, (launches, tot) in pns[name].profile_read().items():
            fam[f"{name}:{f}"] = tot / args.steps
    # accuracy on the held-out cells
    rho_abs = (outs["rho"][0] - props[0, te]).abs().cpu().numpy()
    rho_err = rho_abs / props[0, te].cpu().numpy()
    T_err = (outs["T"][0] - props[1, te]).abs().cpu().numpy()
    tr_err = {nm: ((outs["T"][r] - props[1 + r, te]).exp() - 1.0).abs().cpu().numpy()
              for r, nm in ((1, "mu"), (2, "lambda"), (3, "alpha"))}
    # explicit path: Newton on h(T) from a start 10 % off (eos_post with a zero network output)
    O0 = torch.zeros(N, mech.n, dtype=torch.float32, device=dev)
    u = torch.tensor(synth.Stream(7, "propnet-start").uniform(N, -0.1, 0.1), device=dev)
    T_start = (props[1, te] * (1.0 + u)).contiguous()
    Tx, Yx = T_start.clone(), Ye.clone()
    chem.eos_post(O0, he, Tx, pe, Yx)
    torch.cuda.synchronize()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        Tx.copy_(T_start)
        chem.eos_post(O0, he, Tx, pe, Yx)
    z.record(stream)
    torch.cuda.synchronize()
    explicit_ms = a.elapsed_time(z) / args.steps
    Tx.copy_(T_start)
    xst = chem.eos_post(O0, he, Tx, pe, Yx)
    ok = xst == 0
    dTx = (Tx - props[1, te]).abs()
    explicit_flagged = int((~ok).sum().item())
    explicit_T_err = float(dTx[ok].max().item()) if bool(ok.any()) else None
    # explicit transport: df_transport_props at the cells' (T, p, Y)
    Te = props[1, te].contiguous()
    tp_out = chem.transport_props(Te, pe, Ye)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(args.steps):
        chem.transport_props(Te, pe, Ye)
    z.record(stream)
    torch.cuda.synchronize()
    transport_ms = a.elapsed_time(z) / args.steps
    del tp_out
    if rank != 0:
        return 0
    pk, pk_src = peaks()
    gemm = {f: t for f, t in fam.items() if ":layer" in f}
    dom = max(gemm, key=gemm.get)
    name, lay = dom.split(":")
    l = int(lay[5:])
    wd = PROPNET_WIDTHS[name]
    ach = 2.0 * wd[l] * wd[l + 1] * N / (gemm[dom] * 1e-3) / 1e12
    burst = e0.elapsed_time(e1) * 1e-3 < 2.0
    tpk = pk["bf16_tflops"] if burst else pk["bf16_tflops_sustained"]
    cpu = None
    if not args.no_cpu_baseline:
        import time as _t
        from oracle import propnet as opn
        S = 16384
        sel = np.linspace(N, 2 * N - 1, S).astype(np.int64)
        hs, ps_, Ys = h[sel].cpu().numpy(), p[sel], Y[:, sel]
        t0 = _t.perf_counter()
        for nm in PROPNET_WIDTHS:
            opn.infer(nets[nm], hs, ps_, Ys)
        dt = _t.perf_counter() - t0
        cpu = {"value": S / dt, "unit": "cells/s", "cores": len(os.sched_getaffinity(0)),
               "kind": "oracle", "sample": f"{S} evenly strided cells, both networks in FP64 numpy",
               "seconds": dt}
    e2e = None
    if not args.no_e2e:
        hh, ph, Yh = (t.cpu().pin_memory() for t in (he, pe, Ye))
        oh = {nm: torch.empty(len(PROPNET_ROWS[nm]), N, dtype=torch.float64).pin_memory()
              for nm in PROPNET_WIDTHS}

        def e2e_step():
            he.copy_(hh, non_blocking=True)
            pe.copy_(ph, non_blocking=True)
            Ye.copy_(Yh, non_blocking=True)
            step()
            for nm in PROPNET_WIDTHS:
                oh[nm].copy_(outs[nm], non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            e2e_step()
        z.record(stream)
        torch.cuda.synchronize()
        ems = a.elapsed_time(z) / args.steps
        e2e = {"value": N / (ems * 1e-3), "unit": "cells/s", "ms_per_step": ems,
               "h2d_bytes_per_step": 8 * N * (2 + mech.n), "d2h_bytes_per_step": 8 * N * 5}
    q = lambda a_, f: float(np.quantile(a_, f))
    line = {"metric": "property-network cells/s (rho and T + transport networks of Sec. 4.1 sizes, BF16)",
            "value": weak_scaling_value(world, N, ms), "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": "train30-1m states, 2^20 training + 2^20 evaluation cells",
                       "n_cells": N, "networks": {k: "-".join(map(str, w)) for k, w in PROPNET_WIDTHS.items()},
                       "inputs": "h, p, Box-Cox(Y) of 30 species, Z-scored",
                       "l2": "inputs larger than L2 (fields 8*(2+n)*N bytes, activations GBs)"},
            "clocks": clk.summary(), "e2e": e2e, "gpu_launches": 2 * (2 + 4),
            "roofline": {"bound": "tensor", "achieved": ach, "peak": tpk,
                         "unit": "TFLOP/s", "frac": ach / tpk, "traffic": None,
                         "kernel": f"tc_gemm {name} network {lay} ({wd[l]} -> {wd[l + 1]})",
                         "peak_source": ("bf16_tflops" if burst else "bf16_tflops_sustained") + f" ({pk_src})"},
            "kernels_ms_per_step": fam, "fit": fit,
            "error_vs_peng_robinson": {
                "rho_rel_median": q(rho_err, 0.5), "rho_rel_p99": q(rho_err, 0.99), "rho_rel_max": float(rho_err.max()),
                "rho_abs_kg_m3_median": q(rho_abs, 0.5), "rho_abs_kg_m3_p99": q(rho_abs, 0.99),
                "rho_true_kg_m3_range": [float(props[0, te].min()), float(props[0, te].max())],
                "T_abs_K_median": q(T_err, 0.5), "T_abs_K_p99": q(T_err, 0.99), "T_abs_K_max": float(T_err.max()),
                **{f"{nm}_rel_{w}": (q(e, f) if f < 1 else float(e.max()))
                   for nm, e in tr_err.items() for w, f in (("median", 0.5), ("p99", 0.99), ("max", 1.0))},
                "transport_reference": "df_transport_props (Chung et al. 1988 at the Peng-Robinson density)",
                "cells": N},
            "explicit_pr_newton": {"ms_per_step": explicit_ms, "cells_per_s": N / (explicit_ms * 1e-3),
                                   "T_abs_K_max_converged": explicit_T_err,
                                   "flagged_cells": explicit_flagged,
                                   "what": "eos_post: T from h by safeguarded Newton on the PR h(T), start 10 % off",
                                   "transport_ms_per_step": transport_ms,
                                   "transport_cells_per_s": N / (transport_ms * 1e-3)},
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "train":
        return run_train(args)
    if args.mode == "jacobian":
        return run_jacobian(args)
    if args.mode == "solver":
        return run_solver(args)
    if args.mode == "propnet":
        return run_propnet(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
