#!/usr/bin/env python3
"""Benchmark: PW momentum advection (MONC, Sec. 2.1) on GB300.

Headline step: one FP64 forward pass (su, sv, sw from u, v, w) over the
2048 x 2048 x 64 grid (268M points, 12.9 GB of fields), inputs resident in
HBM, timed with CUDA events on the launching stream.  Also reported on the
same line: the end-to-end rate through the host-buffer C-ABI call, the
roofline of the forward kernel, the FP32 / FP16-storage variants with their
error against the FP64 result, the adjoint, the ensemble, the GPU clocks
during the timed region, and the CPU oracle on this machine's host cores.

``--impl reference`` times the CPU oracle (test infrastructure; the only
other place this script runs it is the cpu_baseline leg).

Multi-GPU: the grid does not need more than one GPU, so ``--gpus N`` runs N
independent replicas (weak scaling, no collective on the data path); rank 0
prints the whole-job rate over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "advection grid points/s (FP64 vs FP32/FP16-storage) and % of HBM roofline"
UNIT = "points/s"
SHAPE = (2048, 2048, 64)
FLOP_PER_POINT = 53           # the paper's count for su, sv, sw (Sec. 2.3)
# The fewest binary64 operations that evaluate su, sv, sw at one point: 9 face
# sums (each two-point sum is shared with the neighbouring point that also
# reads it) and, per field, 10 multiplies / fused multiply-adds (2 per
# direction for a*S1 - b*S2, 2 to combine tcx*X + tcy*Y, 4 for the two
# per-level vertical products) -- the paper's 53 flops fused.
FP64_OPS_PER_POINT = 39
BYTES_PER_POINT = {"f64": 48, "f32": 24, "f16s": 12}       # 3 fields in + 3 out
ADJ_BYTES_PER_POINT = {"f64": 72, "f32": 36, "f64ff": 72}   # 6 in + 3 out
ADJ_SHAPE = (1024, 1024, 128)
# binary64 operations of the gather-form adjoint per point, as its three sums
# are written (each multiply-add fused; no sums shared between points): 28 for
# du, 28 for dv, 30 for dw and the three doublings 2u, 2v, 2w
FP64_ADJ_OPS_PER_POINT = 89
FP64_DFMA_PER_CLK_PER_SM = 2   # GB300 nominal (1.25 TFLOP/s FP64)
N_SM = 152


# ----------------------------------------------------------------- helpers
def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def profile_traffic(kernel_name, src_hash):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_name}_f64_2048x2048x64.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha1") != src_hash:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# The files that define the forward sweep kernel (tile selection lives elsewhere).
FWD_KERNEL_SOURCES = ("bulk.cuh", "common.cuh", "ff.cuh", "fwd_sweep.cu", "fwd_sweep.cuh", "kernels.h",
                      "sweep_core.cuh")


def _code_only(text: str) -> str:
    """Source text without comments and whitespace (a comment edit does not
    change the kernel)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "".join(text.split())


def kernel_source_hash():
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2010_01545_gb300", "csrc")
    for name in FWD_KERNEL_SOURCES:
        with open(os.path.join(csrc, name)) as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def fp64_pipe_rate():
    """The binary64 pipe's measured rate on this GPU (G fused multiply-adds
    per second) from the in-tree probe kernel (probe/fp64_rate.cu), timed
    with CUDA events: best of three runs of ~10 ms each."""
    import ctypes
    from paper_2010_01545_gb300 import build
    lib = ctypes.CDLL(build.PROBE_LIB)
    f = lib.advect_probe_fp64_fma_rate
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                  ctypes.POINTER(ctypes.c_double)]
    f.restype = ctypes.c_int
    best = None
    for _ in range(3):
        g, ms = ctypes.c_double(), ctypes.c_double()
        rc = f(2048, 4, 5, ctypes.byref(g), ctypes.byref(ms))
        if rc != 0:
            raise RuntimeError(f"fp64 probe failed (CUDA error {rc})")
        if best is None or g.value > best[0]:
            best = (g.value, ms.value)
    return {"gops": best[0], "kernel_ms": best[1],
            "how": "8 independent DFMA chains per thread, 4 x 256-thread CTAs per SM, 2048 iterations; "
                   "best of 3 runs of 5 launches (CUDA events)"}


# ----------------------------------------------------------------- oracle legs
def oracle_sample_rate(winds, grid, planes, repeats=1, openmp=False):
    import oracle
    c = oracle.coefficients(grid)
    sub = [np.ascontiguousarray(a[: planes + 2]) for a in winds]   # planes + x-halo
    best = None
    for _ in range(repeats):
        t0 = time.perf_counter()
        oracle.forward(*sub, c, i_range=(1, planes + 1), openmp=openmp)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return planes * SHAPE[1] * SHAPE[2] / best, best


def oracle_all_cores(winds, grid, planes):
    """The same oracle loop built with -fopenmp (x-planes shared among all
    host cores; bitwise the same results), timed on the same sample."""
    import subprocess as sp
    import oracle
    try:
        oracle.build(openmp=True)
    except (sp.CalledProcessError, OSError) as e:
        return {"unavailable": f"gcc -fopenmp build failed: {e}"}
    oracle_sample_rate(winds, grid, min(8, planes), openmp=True)    # thread-pool start
    rate, dt = oracle_sample_rate(winds, grid, planes, repeats=2, openmp=True)
    return {"value": rate, "unit": UNIT, "cores": oracle.threads(openmp=True), "kind": "oracle",
            "sample": f"the same {planes} x-planes, OpenMP parallel-for over x ({dt:.2f} s, best of 2)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import workload
    grid = workload.vertical_grid(SHAPE[2])
    planes = 128
    winds = [workload.wind_field(planes + 2, SHAPE[1], SHAPE[2], f) for f in range(3)]
    import oracle
    c = oracle.coefficients(grid)
    for _ in range(args.warmup):
        oracle.forward(*winds, c, i_range=(1, planes + 1))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.forward(*winds, c, i_range=(1, planes + 1))
    dt = time.perf_counter() - t0
    pts = planes * SHAPE[1] * SHAPE[2]
    value = pts * args.steps / dt
    sample = (f"{planes} x-planes ({pts} points) of the 2048x2048x64 FP64 forward per step, "
              "single-threaded plain C oracle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(workload_config(world), sample_points_per_step=pts),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU legs
def workload_config(world):
    """The benchmarked workload (both arms report it)."""
    return {"workload": "pw_advection_fwd_2048x2048x64_f64", "nx": SHAPE[0], "ny": SHAPE[1], "nz": SHAPE[2],
            "points": SHAPE[0] * SHAPE[1] * SHAPE[2], "l2": "inputs (6.4 GB) larger than L2; no flush",
            "parallelism": f"replicas x{world}"}


def whole_job_rate(local_units, local_seconds, device):
    """Units of all ranks over the slowest rank's time (the timed regions are
    bracketed by barriers, so the slowest rank bounds the job)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local_units / local_seconds, local_seconds
    t = torch.tensor([float(local_seconds), float(local_units)], dtype=torch.float64, device=device)
    secs = t[:1].clone()
    dist.all_reduce(secs, op=dist.ReduceOp.MAX)
    units = t[1:].clone()
    dist.all_reduce(units, op=dist.ReduceOp.SUM)
    return units.item() / secs.item(), secs.item()


def time_calls(fn, steps, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def normwise_errors(got, ref):
    import torch
    out = []
    for g, r in zip(got, ref):
        g = g.to(torch.float64)
        d = g - r
        m = torch.max(torch.abs(r)).item()
        out.append({"max_rel": torch.max(torch.abs(d)).item() / m,
                    "rms_rel": (torch.linalg.vector_norm(d) / torch.linalg.vector_norm(r)).item()})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-variants", action="store_true", help="headline only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    ap.add_argument("--shape", default=None,
                    help="nx,ny,nz of a smaller forward case (profiling); not a bench line")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "f16s", "f64ff"],
                    help="element type of the --shape case")
    ap.add_argument("--adjoint", action="store_true", help="--shape case runs the adjoint")
    ap.add_argument("--integrate", action="store_true",
                    help="--shape case runs the forward fused with the integration step")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="run only an ensemble of this many members (FP32, forward, or adjoint with "
                         "--adjoint; the default tiles), for profiling")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.ensemble:
        return run_ensemble_case(args)
    if args.shape:
        return run_case(args)

    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()

    import workload
    from paper_2010_01545_gb300 import build, torch_api
    build.build()

    grid = workload.vertical_grid(SHAPE[2])
    coeffs = torch_api.coefficients_from_grid(grid)
    n_pts = SHAPE[0] * SHAPE[1] * SHAPE[2]
    winds = workload.winds(*SHAPE, seed=workload.DEFAULT_SEED + rank)
    op = torch_api.Advect(*SHAPE, coeffs, "f64")
    d_in = [torch.from_numpy(a).cuda() for a in winds]
    d_out = [op.empty() for _ in range(3)]

    def step():
        op.forward(*d_in, out=d_out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        secs = time_calls(step, args.steps, stream)
    value, secs = whole_job_rate(n_pts * args.steps, secs, "cuda")
    per_launch = secs / args.steps
    fwd_name = op.kernel_name()

    hbm_gbs, sm_max_mhz, peak_kind = peaks()
    nominal_gops = FP64_DFMA_PER_CLK_PER_SM * N_SM * sm_max_mhz * 1e6 / 1e9
    probe = fp64_pipe_rate()
    fp64_peak_gops = probe["gops"]
    achieved_gops = FP64_OPS_PER_POINT * n_pts / per_launch / 1e9
    achieved_gflops = FLOP_PER_POINT * n_pts / per_launch / 1e9
    achieved_gbs = BYTES_PER_POINT["f64"] * n_pts / per_launch / 1e9
    src_hash = kernel_source_hash()
    traffic = profile_traffic(fwd_name, src_hash)
    roofline = {"bound": "alu", "achieved": achieved_gops, "peak": fp64_peak_gops,
                "unit": "G FP64 op/s", "frac": achieved_gops / fp64_peak_gops, "traffic": traffic,
                "kernel": fwd_name, "tile": op.tuned_config(),
                "peak_kind": "measured: binary64 pipe throughput probe on this GPU (one op per DFMA)",
                "peak_probe": probe,
                "peak_nominal": nominal_gops,
                "frac_of_nominal": achieved_gops / nominal_gops,
                "nominal_kind": "2 add/mul/fma per clk per SM x 152 SM x max SM clock",
                "ops_per_point": FP64_OPS_PER_POINT,
                "flops": {"achieved": achieved_gflops, "peak": 2 * fp64_peak_gops, "unit": "GFLOP/s",
                          "frac": achieved_gflops / (2 * fp64_peak_gops),
                          "note": "53 flop/point (paper); the peak counts every operation as an FMA"},
                "hbm": {"achieved": achieved_gbs, "peak": hbm_gbs, "unit": "GB/s",
                        "frac": achieved_gbs / hbm_gbs, "peak_kind": peak_kind}}

    # end to end through the host-buffer C-ABI call (pinned host memory)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, torch, op, winds, world, n_pts)

    ref_out = [t.clone() for t in d_out]
    variants = {}
    if not args.no_variants:
        variants = run_variants(args, torch, torch_api, workload, winds, coeffs, ref_out, stream,
                                hbm_gbs, grid, fp64_peak_gops)

    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle  # noqa: F401  (CPU baseline leg)
        rate, dt = oracle_sample_rate(winds, grid, SHAPE[0] - 2)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"FP64 forward over {SHAPE[0] - 2} of the 2048 x-planes of the same grid "
                         f"({dt:.1f} s, single-threaded plain C, -O2 -ffp-contract=off)",
               "all_cores": oracle_all_cores(winds, grid, SHAPE[0] - 2)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * per_launch, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(world),
                "roofline": roofline, "e2e": e2e, "gpu_launches": args.steps,
                "clocks": clk.summary(), "cpu_baseline": cpu,
                "cpu_baseline_all_cores": cpu.get("all_cores") if cpu else None,
                "variants": variants, "kernel_source": src_hash}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_e2e(args, torch, op, winds, world, n_pts):
    """Forward through advect_forward_host: pinned host buffers in and out, the
    library's chunked copy/kernel pipeline inside the timed region.  The link
    bound is measured on the same buffers right after: the inputs copied to the
    device while the outputs come back, on two streams, with no kernel."""
    h_in = [torch.from_numpy(a).pin_memory() for a in winds]
    h_out = [torch.empty(SHAPE, dtype=torch.float64).pin_memory() for _ in range(3)]
    e2e_steps = max(3, min(args.steps, 20))
    for _ in range(args.warmup):
        op.forward_host(*h_in, h_out)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    t0 = time.perf_counter()
    per_step = []
    for _ in range(e2e_steps):
        t1 = time.perf_counter()
        op.forward_host(*h_in, h_out)  # returns with the results in h_out
        per_step.append(time.perf_counter() - t1)
    # all ranks' points over the slowest rank's time
    value, total = whole_job_rate(n_pts * e2e_steps, time.perf_counter() - t0, "cuda")
    e2e_secs = total / e2e_steps
    link_secs = measure_link(torch, h_in, h_out)
    moved = 6 * n_pts * 8
    return {"value": value, "unit": UNIT,
            "h2d_bytes_per_step": 3 * n_pts * 8, "d2h_bytes_per_step": 3 * n_pts * 8,
            "ms_per_step": 1e3 * e2e_secs,
            "ms_per_step_min": 1e3 * min(per_step), "ms_per_step_median": 1e3 * statistics.median(per_step),
            "ms_steps": [round(1e3 * x, 2) for x in per_step],
            "link_bound_ms": 1e3 * link_secs, "link_gbs": moved / link_secs / 1e9,
            "link_frac": link_secs / e2e_secs}


def measure_link(torch, h_in, h_out, reps=3):
    """Seconds for the copies alone (best of reps): h_in to the device and, at
    the same time, the device to h_out (pinned, one stream each way)."""
    d_in = [torch.empty(h.shape, dtype=h.dtype, device="cuda") for h in h_in]
    d_out = [torch.zeros(h.shape, dtype=h.dtype, device="cuda") for h in h_out]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def once():
        with torch.cuda.stream(s_in):
            for h, d in zip(h_in, d_in):
                d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s_out):
            for h, d in zip(h_out, d_out):
                h.copy_(d, non_blocking=True)
        torch.cuda.synchronize()

    once()
    secs = float("inf")
    for _ in range(reps):  # best of reps: the link's capability, not its noise
        t0 = time.perf_counter()
        once()
        secs = min(secs, time.perf_counter() - t0)
    del d_in, d_out
    torch.cuda.empty_cache()
    return secs


def run_case(args):
    """One kernel on another shape / type, for profiling: the forward, the
    adjoint (--adjoint) or the forward fused with the integration step
    (--integrate: a separate base updated in place, dt = 0.5)."""
    import torch

    import workload
    from paper_2010_01545_gb300 import build, torch_api
    build.build()
    shape = tuple(int(x) for x in args.shape.split(","))
    n_pts = shape[0] * shape[1] * shape[2]
    grid = workload.vertical_grid(shape[2])
    op = torch_api.Advect(*shape, torch_api.coefficients_from_grid(grid), args.dtype)
    winds = workload.winds(*shape)
    scales = None
    if args.dtype == "f16s":
        s_in = [float(2.0 ** np.ceil(np.log2(np.max(np.abs(a))))) for a in winds]
        scales = s_in + op.output_scales(s_in)
        d = [(torch.from_numpy(a).cuda() / s).to(torch.float16) for a, s in zip(winds, s_in)]
    else:
        d = [torch.from_numpy(a).to("cuda", op.torch_dtype) for a in winds]
    out = [op.empty() for _ in range(3)]
    if args.adjoint:
        lam = [torch.from_numpy(a).to("cuda", op.torch_dtype) for a in workload.cotangents(*shape)]
        call = lambda: op.adjoint(*d, *lam, out=out)  # noqa: E731
    elif args.integrate:
        if args.dtype == "f16s":
            raise SystemExit("--integrate takes f64, f32 or f64ff")
        base = [t.clone() for t in d]
        call = lambda: op.integrate(*d, 0.5, base=base, out=base)  # noqa: E731
    else:
        call = lambda: op.forward(*d, out=out, scales=scales)  # noqa: E731
    for _ in range(args.warmup):
        call()
    secs = time_calls(call, args.steps, torch.cuda.current_stream()) / args.steps
    kind = "adj" if args.adjoint else ("int" if args.integrate else "fwd")
    print(json.dumps({"case": f"{kind}_{args.dtype}_{shape[0]}x{shape[1]}x{shape[2]}",
                      "kernel": op.kernel_name(args.adjoint), "tile": op.tuned_config(args.adjoint),
                      "ms": 1e3 * secs, "points_per_s": n_pts / secs, "steps": args.steps,
                      "warmup": args.warmup}), flush=True)
    return 0


def run_variants(args, torch, torch_api, workload, winds, coeffs, ref_out, stream, hbm_gbs, grid,
                 fp64_peak_gops):
    out = {}
    n_pts = SHAPE[0] * SHAPE[1] * SHAPE[2]
    steps = max(3, min(args.steps, 10))
    # FP32 storage + arithmetic
    op32 = torch_api.Advect(*SHAPE, coeffs, "f32")
    d32 = [torch.from_numpy(a).to("cuda", torch.float32) for a in winds]
    o32 = [op32.empty() for _ in range(3)]
    for _ in range(args.warmup):
        op32.forward(*d32, out=o32)
    secs = time_calls(lambda: op32.forward(*d32, out=o32), steps, stream) / steps
    errs = normwise_errors(o32, ref_out)
    out["f32"] = {"value": n_pts / secs, "unit": UNIT, "ms": 1e3 * secs, "kernel": op32.kernel_name(),
                  "tile": op32.tuned_config(),
                  "hbm_frac": BYTES_PER_POINT["f32"] * n_pts / secs / 1e9 / hbm_gbs,
                  "error_vs_f64": dict(zip(("su", "sv", "sw"), errs))}
    del d32, o32, op32
    # binary64 storage, double-float arithmetic on the binary32 pipes
    opff = torch_api.Advect(*SHAPE, coeffs, "f64ff")
    dff = [torch.from_numpy(a).cuda() for a in winds]
    off = [opff.empty() for _ in range(3)]
    for _ in range(args.warmup):
        opff.forward(*dff, out=off)
    secs = time_calls(lambda: opff.forward(*dff, out=off), steps, stream) / steps
    errs = normwise_errors(off, ref_out)
    out["f64ff"] = {"value": n_pts / secs, "unit": UNIT, "ms": 1e3 * secs, "kernel": opff.kernel_name(),
                    "tile": opff.tuned_config(),
                    "hbm_frac": BYTES_PER_POINT["f64"] * n_pts / secs / 1e9 / hbm_gbs,
                    "error_vs_f64": dict(zip(("su", "sv", "sw"), errs)),
                    "note": "binary64 in memory, pairs of binary32 in arithmetic"}
    del dff, off, opff
    # FP16 storage with per-field power-of-two scales
    op16 = torch_api.Advect(*SHAPE, coeffs, "f16s")
    s_in = [float(2.0 ** np.ceil(np.log2(np.max(np.abs(a))))) for a in winds]
    s_out = op16.output_scales(s_in)
    d16 = [(torch.from_numpy(a).cuda() / s).to(torch.float16) for a, s in zip(winds, s_in)]
    o16 = [op16.empty() for _ in range(3)]
    sc = s_in + s_out
    for _ in range(args.warmup):
        op16.forward(*d16, out=o16, scales=sc)
    secs = time_calls(lambda: op16.forward(*d16, out=o16, scales=sc), steps, stream) / steps
    errs = normwise_errors([o.to(torch.float64) * s for o, s in zip(o16, s_out)], ref_out)
    out["f16s"] = {"value": n_pts / secs, "unit": UNIT, "ms": 1e3 * secs, "kernel": op16.kernel_name(),
                   "tile": op16.tuned_config(),
                   "hbm_frac": BYTES_PER_POINT["f16s"] * n_pts / secs / 1e9 / hbm_gbs,
                   "error_vs_f64": dict(zip(("su", "sv", "sw"), errs)),
                   "note": "error includes the fp16 quantisation of the inputs"}
    del d16, o16, op16
    torch.cuda.empty_cache()
    # forward fused with the integration step: one explicit step (u + dt su,
    # binary64) and a leapfrog-form step on a separate base updated in place
    # (binary32); the source terms never reach memory
    dt = 0.5
    for name, tdt, with_base in (("f64", torch.float64, False), ("f32", torch.float32, True)):
        opi = torch_api.Advect(*SHAPE, coeffs, name)
        x = [torch.from_numpy(a).to("cuda", tdt) for a in winds]
        if with_base:
            b = [t.clone() for t in x]
            call = lambda: opi.integrate(*x, dt, base=b, out=b)  # noqa: E731
        else:
            o = [opi.empty() for _ in range(3)]
            call = lambda: opi.integrate(*x, dt, out=o)  # noqa: E731
        for _ in range(args.warmup):
            call()
        secs = time_calls(call, steps, stream) / steps
        bpp = BYTES_PER_POINT[name] * (3 if with_base else 2) // 2
        out[f"integrate_{name}"] = {
            "value": n_pts / secs, "unit": UNIT, "ms": 1e3 * secs, "kernel": opi.kernel_name(),
            "hbm_frac": bpp * n_pts / secs / 1e9 / hbm_gbs, "bytes_per_point": bpp,
            "step": "u_base + dt * su in place on a separate base" if with_base else "u + dt * su",
            # forward writing su, sv, sw, then a pass reading base and source terms
            "unfused_bytes_per_point": BYTES_PER_POINT[name] * 5 // 2}
        del x, opi
        if with_base:
            del b
        else:
            del o
        torch.cuda.empty_cache()
    # adjoint on the 1024 x 1024 x 128 differentiation grid (inputs drawn on
    # the device: U(-10, 10) winds and N(0, 1) cotangents from a seeded
    # torch generator)
    agrid = workload.vertical_grid(ADJ_SHAPE[2])
    acoef = torch_api.coefficients_from_grid(agrid)
    an = ADJ_SHAPE[0] * ADJ_SHAPE[1] * ADJ_SHAPE[2]
    gen = torch.Generator(device="cuda")
    for name, tdt in (("f64", torch.float64), ("f32", torch.float32), ("f64ff", torch.float64)):
        gen.manual_seed(workload.DEFAULT_SEED)
        opa = torch_api.Advect(*ADJ_SHAPE, acoef, name)
        x = [torch.rand(ADJ_SHAPE, generator=gen, device="cuda", dtype=tdt) * 20 - 10 for _ in range(3)]
        lam = [torch.randn(ADJ_SHAPE, generator=gen, device="cuda", dtype=tdt) for _ in range(3)]
        g = [opa.empty() for _ in range(3)]
        for _ in range(args.warmup):
            opa.adjoint(*x, *lam, out=g)
        secs = time_calls(lambda: opa.adjoint(*x, *lam, out=g), steps, stream) / steps
        rec = out[f"adjoint_{name}_1024x1024x128"] = {
            "value": an / secs, "unit": UNIT, "ms": 1e3 * secs, "kernel": opa.kernel_name(True),
            "tile": opa.tuned_config(True),
            "hbm_frac": ADJ_BYTES_PER_POINT[name] * an / secs / 1e9 / hbm_gbs}
        if name == "f64":
            gops = FP64_ADJ_OPS_PER_POINT * an / secs / 1e9
            rec["alu"] = {"bound": "alu", "ops_per_point": FP64_ADJ_OPS_PER_POINT, "achieved": gops,
                          "peak": fp64_peak_gops, "unit": "G FP64 op/s", "frac": gops / fp64_peak_gops,
                          "peak_kind": "measured: binary64 pipe throughput probe on this GPU"}
        del x, lam, g, opa
        torch.cuda.empty_cache()
    out["ensemble_f32_48"] = run_ensemble(args, torch, torch_api, workload, stream, hbm_gbs)
    return out


def run_ensemble_case(args):
    """The first N members of the benchmark's ensemble (FP32), forward or
    adjoint, for profiling the persistent ensemble kernel on a small case."""
    import torch

    import workload
    from paper_2010_01545_gb300 import build, torch_api
    build.build()
    shapes = workload.ensemble_shapes(48)[: args.ensemble]
    pts = sum(a * b * c for a, b, c in shapes)
    coeffs = [torch_api.coefficients_from_grid(workload.vertical_grid(s[2])) for s in shapes]
    ens = torch_api.AdvectEnsemble(shapes, coeffs, "f32")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(workload.DEFAULT_SEED)
    x = [[torch.rand(s, generator=gen, device="cuda") * 20 - 10 for s in shapes] for _ in range(3)]
    lam = [[torch.randn(s, generator=gen, device="cuda") for s in shapes] for _ in range(3)]
    out = [ens.empty() for _ in range(3)]
    if args.adjoint:
        call = lambda: ens.adjoint(*x, *lam, out=out)  # noqa: E731
    else:
        call = lambda: ens.forward(*x, out=out)  # noqa: E731
    for _ in range(args.warmup):
        call()
    secs = time_calls(call, args.steps, torch.cuda.current_stream()) / args.steps
    print(json.dumps({"case": f"ensemble_{'adj' if args.adjoint else 'fwd'}_f32_{len(shapes)}_members",
                      "points": pts, "tile": ens.tuned_config(bool(args.adjoint)), "ms": 1e3 * secs,
                      "points_per_s": pts / secs, "steps": args.steps, "warmup": args.warmup}), flush=True)
    return 0


def run_ensemble(args, torch, torch_api, workload, stream, hbm_gbs):
    """48 members of uneven shape, FP32, forward and adjoint, autotuned tiles."""
    shapes = workload.ensemble_shapes(48)
    pts = sum(a * b * c for a, b, c in shapes)
    coeffs = [torch_api.coefficients_from_grid(workload.vertical_grid(s[2])) for s in shapes]
    ens = torch_api.AdvectEnsemble(shapes, coeffs, "f32")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(workload.DEFAULT_SEED)
    x = [[torch.rand(s, generator=gen, device="cuda") * 20 - 10 for s in shapes] for _ in range(3)]
    lam = [[torch.randn(s, generator=gen, device="cuda") for s in shapes] for _ in range(3)]
    y = [ens.empty() for _ in range(3)]
    g = [ens.empty() for _ in range(3)]
    ens.autotune(True)
    ens.forward(*x, out=y)          # tunes on these buffers, then runs the winner
    ens.adjoint(*x, *lam, out=g)
    steps = max(3, min(args.steps, 10))
    res = {"members": len(shapes), "points": pts}
    for name, fn, bpp in (("forward", lambda: ens.forward(*x, out=y), 24),
                          ("adjoint", lambda: ens.adjoint(*x, *lam, out=g), 36)):
        for _ in range(args.warmup):
            fn()
        secs = time_calls(fn, steps, stream) / steps
        res[name] = {"value": pts / secs, "unit": UNIT, "ms": 1e3 * secs,
                     "hbm_frac": bpp * pts / secs / 1e9 / hbm_gbs,
                     "tile": ens.tuned_config(name == "adjoint"),
                     "launch": "one persistent kernel, CUDA graph replay"}
    del x, lam, y, g
    ens.close()
    torch.cuda.empty_cache()
    return res


if __name__ == "__main__":
    sys.exit(main())
