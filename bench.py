#!/usr/bin/env python
"""Throughput of the hybrid LBM step (Renard et al., arXiv 2002.03644) on GB300.

Workload: isentropic vortex convected at Ma 1.2 in a periodic 1024 x 1024
box (vortex strength 0.2, radius 32 cells, gamma 1.4, Pr 0.71, sigma 0,
seeded +-1e-6 density noise), FP32 storage and arithmetic.  One bench step is
one time step of Algorithm 1 over the whole grid (one launch of the fused
kernel).  The state (2 x 54.5 MB) fits in L2, so L2 is flushed between timed
steps (a write of one buffer and a read of another, each larger than L2) and
each step is timed alone with CUDA events on the library's stream.

Prints one JSON line.  Beside the headline step it carries, on one GPU, the
end-to-end figure through the C ABI with host buffers (per step, and
amortised over 100 steps per call), the FP64 oracle on the host cores as the
CPU baseline, and two sub-objects for the forms grown from the step:
`batched` (the 64-case vortex sweep advanced together against the same
cases one after another, with both compared to the FP64 oracle) and
`surrogate` (the K = 16 learned surrogate trained in the run, one call
against 16 solver steps, and a hybrid rollout judged by the solver at a
sweep of tolerances).  --impl reference times the FP64 CPU oracle on the
host cores on the same workload.  Under torchrun every rank runs an
independent replica on its own GPU (the method has no exchange step in this
single-GPU build); value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# 9 populations + s + 3 a1 read and written once per cell-update
BYTES_PER_CELL = {"fp32": 104, "fp64": 208, "fp16pop": 68, "bf16pop": 68, "moments": 56}
# the FP64 marching kernel also reads and writes each cell's level rho, u_x,
# u_y, theta (4 FP64 planes kept so that no step recomputes them)
FP64_MARCH_BYTES_PER_CELL = 272


def bytes_per_cell(precision, cells):
    """Bytes one cell-update reads and writes in the fused-step kernel the
    library launches (kernel choice as in kernel_name)."""
    if precision == "fp64":
        march = int(os.environ.get("HLBM_MARCH", "-1" if cells <= 768 * 768 else "0"))
        if 0 <= march < 4:
            return FP64_MARCH_BYTES_PER_CELL
    return BYTES_PER_CELL[precision]
METRIC, UNIT = "MLUPS", "MLUPS"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16pop", "bf16pop", "moments"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--workload", default="vortex", choices=["vortex", "quadrant"],
                    help="vortex: the isentropic vortex (default); quadrant: the four-quadrant Riemann problem on its "
                         "longest-running setting (FD Phi, sigma 0.1, C_0 10, mu 0.01; zero-gradient sides)")
    ap.add_argument("--e2e-inner", type=int, default=100)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--surrogate", action="store_true",
                    help="only the surrogate leg: train the K=16 conv surrogate on HLBM rollouts and compare "
                         "it with the HLBM step")
    ap.add_argument("--sur-samples", type=int, default=2000)
    ap.add_argument("--sur-epochs", type=int, default=30)
    ap.add_argument("--sur-noise", type=float, default=0.1,
                    help="standard deviation of the Gaussian noise added to the normalised training inputs")
    ap.add_argument("--sur-pushforward", type=float, default=0.0,
                    help="fraction of training inputs replaced by the network's own prediction from the previous "
                         "snapshot (second half of the epochs)")
    ap.add_argument("--sur-rollout", type=int, default=2,
                    help="calls chained through the network per training sample from --sur-rollout-from on "
                         "(1: one call; k > 1: the loss of k calls, back-propagated through the chain)")
    ap.add_argument("--sur-rollout-from", type=float, default=0.8,
                    help="fraction of the epochs after which the chained training starts")
    ap.add_argument("--sur-tol", type=float, default=1.0,
                    help="judged-error tolerance of the hybrid rollout (max-abs, normalised fields)")
    ap.add_argument("--batched", action="store_true",
                    help="only the batched leg: the 64-case batched vortex sweep (one launch per step over all "
                         "cases, replayed from CUDA graphs) against the same cases run one after another")
    ap.add_argument("--batched-steps", type=int, default=200)
    ap.add_argument("--batched-cases", type=int, default=64,
                    help="cases of the sweep (the first ones of the seeded draw); the configured sweep has 64")
    ap.add_argument("--no-batched", action="store_true", help="leave the batched leg out of the default line")
    ap.add_argument("--no-surrogate", action="store_true", help="leave the surrogate leg out of the default line")
    return ap.parse_args()


def workload(n, kind="vortex"):
    from paper_2002_03644_gb300 import inputs
    if kind == "quadrant":
        case = inputs.four_quadrant(n=n, C0=10.0, mu=0.01, sigma=0.1)
        case.phi_mode = 1
        return case
    return inputs.vortex(n=n)


def describe(case, precision):
    if case.name == "four_quadrant":
        text = (f"four-quadrant Riemann problem {case.nx}x{case.ny}, zero-gradient sides, C_0 10, mu 0.01, "
                f"sigma 0.1, finite-difference Phi")
    else:
        text = (f"isentropic vortex {case.nx}x{case.ny} periodic, Ma 1.2, strength 0.2, radius 32, "
                f"gamma 1.4, Pr 0.71, sigma 0, mu 1.5e-6, +-1e-6 seeded rho noise")
    return {"workload": text, "nx": case.nx, "ny": case.ny, "precision": precision,
            "l2": "flushed between timed steps" + (" (state smaller than L2)" if case.nx * case.ny <= 1 << 20 else "")}


# ---- distributed plumbing ------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws):
    """Largest value of x over the ranks (the job's time is its slowest rank)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, seconds_this_rank, ws):
    """Whole-job throughput: every rank processes units_per_rank in its own
    time; the job takes the slowest rank's time."""
    return ws * units_per_rank / max_over_ranks(seconds_this_rank, ws)


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---- clocks ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"hlbm_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        try:
            self.f.close()
        except Exception:
            pass

    def summary(self):
        if not self.proc:
            return None
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
            os.remove(self.path)
        except Exception:
            return None
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        mx = max(num(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        loaded = [s for s in sm if not math.isnan(s)]
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


# ---- roofline helpers ------------------------------------------------------------------
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("hlbm_device.cuh", "hlbm_tma.cuh", "hlbm_march.cuh", "hlbm_pack.cuh", "hlbm_api.cu"):
        h.update(open(os.path.join(ROOT, "paper_2002_03644_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def kernel_name(precision, cells, sigma=0.0, phi_mode=0, periodic=False):
    """The fused-step kernel the library launches for this precision: the
    row-marching kernel on grids of more than 768^2 cells unless
    HLBM_MARCH=-1 (then the tiled kernels, chosen for FP32 by HLBM_FP32_TMA /
    HLBM_FP32_TILE), the tiled kernel on small grids unless HLBM_MARCH
    selects a marching variant."""
    if precision == "moments":
        return "march_moment_kernel<64,8,%s,%s%s>" % (str(sigma > 0).lower(), str(phi_mode == 0).lower(),
                                                      ",true" if periodic else "")
    march = int(os.environ.get("HLBM_MARCH", "-1" if cells <= 768 * 768 else "0"))
    if 0 <= march < 4:
        t = {"fp64": "double,FullStore<double>", "fp16pop": "float,HalfStore", "bf16pop": "float,BF16Store"}
        f64 = precision == "fp64"
        nt, minb = [(64, 8), (96, 5), (128, 4), (64, 1)][march]
        # the default FP32-arithmetic kernel has an instantiation for all-periodic grids
        per = ",true" if (march == 0 and not f64 and periodic) else ""
        return "march_pair_kernel<%s,%d,%d,%s,%s%s>" % (t.get(precision, "float,FullStore<float>"), nt,
                                                        1 if f64 else minb, str(sigma > 0).lower(),
                                                        str(phi_mode == 0).lower(), per)
    if precision == "fp64":
        return "fused_step_kernel<double,FullStore<double>,32,8,256>"
    if precision in ("fp16pop", "bf16pop"):
        st = "HalfStore" if precision == "fp16pop" else "BF16Store"
        return f"fused_step_kernel<float,{st},32,32,512>"
    tma = int(os.environ.get("HLBM_FP32_TMA", "0" if cells > 2048 * 2048 else "-1"))
    if tma >= 0:
        return ["fused_step_tma_kernel<32,16,512>", "fused_step_tma_kernel<32,16,256>",
                "fused_step_tma_kernel<64,16,512>", "fused_step_tma_kernel<32,32,512>"][tma]
    tile = int(os.environ.get("HLBM_FP32_TILE", "4"))
    return "fused_step_kernel<float,FullStore<float>,%s>" % ["32,16,256", "64,16,256", "32,8,128", "64,32,512",
                                                             "32,32,512"][tile]


FP64_NOMINAL_TFLOPS = 1.25


def profiled_fp64_counts(n):
    """FP64 operations (add, mul, 2 per fma) and FP64 instructions per
    cell-update of the FP64 fused kernel from the committed ncu count, if it
    was taken on the current kernel source; (None, None) otherwise."""
    path = os.path.join(ROOT, "profiles", "fused_step_vortex_traffic.json")
    try:
        e = json.load(open(path)).get(f"fp64_{n}")
    except Exception:
        return None, None
    if not e or e.get("kernel_source_hash") != kernel_source_hash():
        return None, None
    return e.get("fp64_flops_per_cell"), e.get("fp64_instructions_per_cell")


def profiled_traffic(precision, n):
    """dram bytes per launch of the fused kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "fused_step_vortex_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get(f"{precision}_{n}")
    if not e or e.get("kernel_source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


# ---- CPU oracle timing -----------------------------------------------------------------
def oracle_mlups(case, seconds, rows=None, threads=1):
    """Time the FP64 oracle on the host with its per-cell passes split over
    `threads` threads.  With rows, a periodic strip of that many rows of the
    workload is used as the sample."""
    from oracle.oracle import Oracle
    if rows:
        sl = slice(case.ny // 2 - rows // 2, case.ny // 2 - rows // 2 + rows)
        f = [np.ascontiguousarray(a[sl]) for a in case.fields()]
        nx, ny = case.nx, rows
    else:
        f = list(case.fields())
        nx, ny = case.nx, case.ny
    o = Oracle(nx, ny, **case.params())
    o.set_threads(threads)
    o.init(*f)
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t0
    k = max(1, int(seconds / max(t1, 1e-6)))
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    return nx * ny * k / dt / 1e6, k, dt, nx, ny


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    case = workload(args.n, args.workload)
    from oracle.oracle import Oracle, max_threads
    threads = max_threads()
    o = Oracle(case.nx, case.ny, **case.params())
    o.set_threads(threads)
    o.init(*case.fields())
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    cells = case.nx * case.ny
    v = cells * args.steps / dt / 1e6
    sample = (f"the full {case.nx}x{case.ny} workload, one time step per bench step, rows of each per-cell pass "
              f"split over {threads} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": describe(case, "fp64"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---- the GPU arm ------------------------------------------------------------------------
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__ as g
    if rank == 0 or ws == 1:
        g.build()
    barrier(ws)
    from paper_2002_03644_gb300 import hlbm

    prec = {"fp32": hlbm.HLBM_FP32, "fp64": hlbm.HLBM_FP64, "fp16pop": hlbm.HLBM_FP32_F16POP,
            "bf16pop": hlbm.HLBM_FP32_BF16POP, "moments": hlbm.HLBM_FP32_MOMENTS}[args.precision]
    case = workload(args.n, args.workload)
    cells = case.nx * case.ny
    # a dedicated stream: torch's default stream has handle 0, which the C ABI
    # reads as "create your own stream"; events and flushes must share the
    # library's stream
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s = hlbm.Solver(case.nx, case.ny, stream=stream.cuda_stream, precision=prec, **case.params())
    s.init(*case.fields())
    # the FP64 pipe's rate, for the FP64 form's roofline (outside the timed region)
    fp64_fma_rate = hlbm.hlbm_selftest_fp64_rate(stream=stream.cuda_stream) if args.precision == "fp64" else None

    flush_w = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush_r = torch.ones(64 << 20, dtype=torch.float32, device="cuda")

    def flush():
        flush_w.zero_()
        flush_r.sum()

    # clocks are sampled from the first warm-up step to the end of the last
    # GPU leg (the timed steps alone are shorter than the sampling period)
    clk = ClockSampler(local).__enter__()
    try:
        for _ in range(args.warmup):
            flush()
            s.step(1)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier(ws)
        torch.cuda.synchronize()
        for a, b in ev:
            flush()
            a.record(stream)
            s.step(1)
            b.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        step_ms = [a.elapsed_time(b) for a, b in ev]
        own_s = sum(step_ms) / 1e3
        value = job_throughput(cells * args.steps, own_s, ws) / 1e6
        ms_per_step = max_over_ranks(own_s, ws) / args.steps * 1e3

        # back-to-back steps (L2 warm), reported for context only
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.step(args.steps)
        b.record(stream)
        torch.cuda.synchronize()
        b2b = cells * args.steps / (a.elapsed_time(b) / 1e3) / 1e6

        d = s.diagnostics()
        if d[7] != 0:
            raise RuntimeError("non-finite state after the timed steps")

        # end to end through the C ABI with pinned host buffers: every e2e step
        # initialises the state from the host fields, advances it by one time
        # step and reads rho, u, theta back to the host (so the copies are per
        # step); the same with 100 time steps per call is reported beside it
        pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in case.fields()]
        outs = [torch.empty((case.ny, case.nx), dtype=torch.float64).pin_memory() for _ in range(4)]

        def e2e_leg(inner, iters):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(iters):
                hlbm.hlbm_init_fields(s.h, *pin, n=cells)
                s.step(inner)
                hlbm.hlbm_get_macros(s.h, rho=outs[0], ux=outs[1], uy=outs[2], theta=outs[3], n=cells)
            return job_throughput(cells * inner * iters, time.perf_counter() - t0, ws) / 1e6

        e2e_leg(1, 2)
        copy_bytes = 4 * 8 * cells
        e2e = {"value": e2e_leg(1, max(args.steps, 3)), "unit": UNIT, "h2d_bytes_per_step": copy_bytes,
               "d2h_bytes_per_step": copy_bytes, "steps_per_call": 1,
               "note": "one e2e step = hlbm_init_fields(pinned host rho, u_x, u_y, theta) + hlbm_step(1) + "
                       "hlbm_get_macros(pinned host rho, u_x, u_y, theta)",
               "amortised": {"value": e2e_leg(args.e2e_inner, 3), "unit": UNIT, "steps_per_call": args.e2e_inner,
                             "h2d_bytes_per_step": copy_bytes / args.e2e_inner,
                             "d2h_bytes_per_step": copy_bytes / args.e2e_inner}}
        s.close()
        del flush_w, flush_r

        batched = surr = None
        if ws == 1 and not args.no_batched:
            batched = batched_leg(args, stream, cpu=not args.no_cpu_baseline)
        if ws == 1 and not args.no_surrogate:
            surr = surrogate_leg(args, stream)
    finally:
        clk.__exit__(None, None, None)

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    peaks = measured_peaks()
    bpc = bytes_per_cell(args.precision, cells)
    mean_launch_s = statistics.mean(step_ms) / 1e3
    achieved = bpc * cells / mean_launch_s / 1e9
    if args.precision != "fp64":
        peak = peaks["hbm_gbs"] if peaks else 6800.0
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": profiled_traffic(args.precision, args.n) if args.workload == "vortex" else None,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback",
                "kernel": kernel_name(args.precision, cells, case.sigma, case.phi_mode,
                                      all(b == 0 for b in case.bc) and case.ny >= 4
                                      and os.environ.get("HLBM_MARCH_GENERAL", "0") != "1"),
                "algorithmic_bytes_per_launch": bpc * cells}
    else:
        # FP64 is bound by GB300's FP64 pipe: FP64 operations (add, mul, 2 per
        # fma) executed per cell-update, counted by ncu, against this GPU's
        # FP64 rate measured in the same run by the library's FMA-chain probe.
        # An add or a multiply occupies the pipe like an FMA but counts one
        # flop, so the FP64 instruction rate against the probe's FMA rate
        # (pipe_instruction_frac) is the tighter measure.
        fpc, ipc = profiled_fp64_counts(args.n)
        tf = None if fpc is None else fpc * cells / mean_launch_s / 1e12
        peak = 2.0 * fp64_fma_rate / 1e12
        roof = {"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                "frac": None if tf is None else tf / peak,
                "pipe_instruction_frac": None if ipc is None else ipc * cells / mean_launch_s / fp64_fma_rate,
                "traffic": profiled_traffic(args.precision, args.n) if args.workload == "vortex" else None,
                "peak_source": "measured in this run: hlbm_selftest_fp64_rate, FP64 FMA chains on every SM "
                               f"(nominal {FP64_NOMINAL_TFLOPS} TFLOP/s)",
                "fp64_flops_per_cell": fpc, "fp64_instructions_per_cell": ipc, "hbm_gbs_achieved": achieved,
                "kernel": kernel_name(args.precision, cells, case.sigma, case.phi_mode),
                "algorithmic_bytes_per_launch": bpc * cells}

    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        # the oracle on all host cores (rows of each per-cell pass split over
        # threads), and on one core
        from oracle.oracle import max_threads
        threads = max_threads()
        v, k, dt, nx, ny = oracle_mlups(case, args.cpu_seconds, threads=threads)
        v1, k1, dt1, _, _ = oracle_mlups(case, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"FP64 oracle, full {nx}x{ny} grid, {k} time steps after init ({dt:.1f} s), "
                         f"rows split over {threads} threads",
               "single_core": {"value": v1, "unit": UNIT, "cores": 1,
                               "sample": f"the same, one thread, {k1} time steps ({dt1:.1f} s)"}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic", "config": dict(describe(case, args.precision), parallelism=f"replicas{ws}",
                                            back_to_back_mlups=b2b),
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
        "gpu_launches": args.steps,
    }
    if batched is not None:
        line["batched"] = batched
    if surr is not None:
        line["surrogate"] = surr
    print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def field_errors(got, ref, gamma):
    """max |got - ref| per field over the parity tests' field scales (rho:
    max rho; u: max |u| + max sound speed; theta: max theta; a1: max p), and
    a1 at its own scale (max |a1_ref|)."""
    c = np.sqrt(gamma * np.abs(ref["theta"]) / 3.0).max()
    um = np.sqrt(ref["ux"] ** 2 + ref["uy"] ** 2).max()
    sc = {"rho": np.abs(ref["rho"]).max(), "ux": um + c, "uy": um + c, "theta": np.abs(ref["theta"]).max(),
          "s": np.abs(ref["s"]).max(), "a1": (ref["rho"] * ref["theta"] / 3.0).max()}
    e = {k: float(np.abs(got[k] - ref[k]).max() / sc[k]) for k in sc}
    e["a1_own"] = float(np.abs(got["a1"] - ref["a1"]).max() / max(np.abs(ref["a1"]).max(), 1e-300))
    return e


def batched_leg(args, stream, cpu=True, ncmp=4):
    """The 64-case vortex sweep (128^2 .. 1024^2, Mach 0.1-1.5, three gammas)
    advanced together (autotuned work shape, CUDA-graph replay), against the
    same cases stepped one after another by the default single-case kernel.
    With cpu, the FP64 oracle runs the `ncmp` smallest cases over the same
    steps on the host cores (timed: the leg's CPU baseline) and both GPU
    forms are compared with it field by field."""
    import torch
    from paper_2002_03644_gb300 import hlbm, inputs
    cases = inputs.batch_sweep(ncase=args.batched_cases)
    steps, warm = args.batched_steps, max(args.warmup, 3)
    cells = sum(c.nx * c.ny for c in cases)
    spec = [dict(nx=c.nx, ny=c.ny, precision=hlbm.HLBM_FP32, **c.params()) for c in cases]
    b = hlbm.Batch(spec, stream=stream.cuda_stream)
    for v, c in zip(b.cases, cases):
        v.init(*c.fields())
    tile = b.autotune()
    b.step(warm)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    bad = sum(int(v.diagnostics()[7]) for v in b.cases)
    order = sorted(range(len(cases)), key=lambda i: (cases[i].nx * cases[i].ny, i))
    cmp_idx = order[:ncmp]
    final_b = {i: b.cases[i].macros() for i in cmp_idx}
    fields = ("rho", "ux", "uy", "theta")
    all_b = [{k: m[k].astype(np.float32) for k in fields} for m in (v.macros() for v in b.cases)]
    b.close()
    t_sep, err_sep, final_s = 0.0, 0.0, {}
    for i, (c, fb) in enumerate(zip(cases, all_b)):
        s = hlbm.Solver(c.nx, c.ny, stream=stream.cuda_stream, precision=hlbm.HLBM_FP32, **c.params())
        s.init(*c.fields())
        s.step(warm)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        t_sep += e0.elapsed_time(e1) / 1e3
        m = s.macros()
        if i in cmp_idx:
            final_s[i] = m
        for k in fields:
            err_sep = max(err_sep, float(np.abs(m[k] - fb[k]).max() / max(np.abs(m[k]).max(), 1e-30)))
        s.close()
    v_batch = cells * steps / t_batch / 1e6
    v_sep = cells * steps / t_sep / 1e6
    nc = len(cases)
    state_gb = 2 * 52 * cells / 1e9
    out = {"metric": f"MLUPS (batched {nc}-case vortex sweep)", "value": v_batch, "unit": UNIT,
           "steps": steps, "warmup": warm, "ms_per_step": t_batch / steps * 1e3,
           "workload": f"{nc} vortex cases, N from {{128,256,512,1024}}, Ma U[0.1,1.5], gamma from {{1.4,1.3,1.67}}, "
                       "CFL 0.7, seed 2002, FP32", "cells": cells, "autotuned_tile_index": tile,
           "separate_runs_mlups": v_sep, "speedup_vs_separate": v_batch / v_sep,
           "batch_vs_separate_max_rel": err_sep, "nonfinite_cells": bad,
           "l2": f"state ({cells / 1e6:.1f} M cells, {state_gb:.1f} GB) "
                 + ("larger than L2" if state_gb * 1e9 > 129e6 else "smaller than L2")}
    if cpu:
        from oracle.oracle import Oracle, max_threads
        threads = max_threads()
        errs_b, errs_s, work, t_cpu = [], [], 0, 0.0
        for i in cmp_idx:
            c = cases[i]
            o = Oracle(c.nx, c.ny, **c.params())
            o.set_threads(threads)
            o.init(*c.fields())
            t0 = time.perf_counter()
            o.step(warm + steps)
            t_cpu += time.perf_counter() - t0
            work += c.nx * c.ny * (warm + steps)
            ref = o.macros()
            errs_b.append(field_errors(final_b[i], ref, c.gamma))
            errs_s.append(field_errors(final_s[i], ref, c.gamma))

        def worst(es):
            return {k: max(e[k] for e in es) for k in es[0]}
        out["field_error_vs_oracle"] = {
            "batched": worst(errs_b), "separate": worst(errs_s), "bound": 1e-4,
            "cases": [cases[i].name for i in cmp_idx], "steps": warm + steps,
            "note": "max |GPU - FP64 oracle| over the parity tests' field scales after the leg's steps; a1_own: "
                    "a1 over max |a1_oracle|"}
        out["cpu_baseline"] = {"value": work / t_cpu / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": f"FP64 oracle on the {ncmp} smallest cases of the sweep, "
                                         f"{warm + steps} time steps each ({t_cpu:.1f} s)"}
    return out


def run_batched(args):
    """The batched leg alone, as its own JSON line."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = batched_leg(args, stream, cpu=not args.no_cpu_baseline)
    out.update(n_gpus=1, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic")
    print(json.dumps(out))
    return 0


def surrogate_leg(args, stream):
    """Learned K = 16 surrogate: 6 periodic 3x3 conv layers (4 -> 64 x 5 -> 4,
    GELU), BF16 operands with FP32 accumulation, trained by the library's own
    kernels on HLBM snapshot pairs of 256^2 random-Fourier fields (8 lowest
    modes, amplitude 0.05, Mach 0.3-1.2).  Reports training throughput, the
    held-out error, the time of one surrogate call against 16 HLBM steps on
    the same grid, and a hybrid rollout of held-out initial states (the HLBM
    judging every 8th call, falling back above the tolerance) against the
    plain FP32 HLBM over the same steps."""
    import torch
    from paper_2002_03644_gb300 import hlbm, inputs, surrogate
    n, K, batch, judge_every, calls = 256, 16, 16, 8, 16
    sh = stream.cuda_stream
    t0 = time.perf_counter()
    X, Y = surrogate.make_dataset_device(args.sur_samples, n=n, K=K, pairs_per_run=4, seed=2002, stream=sh)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    ntrain = int(0.9 * X.shape[0]) // batch * batch
    norm = surrogate.DeviceNormaliser(X[:ntrain])
    Xn, Yn = norm.fwd(X).contiguous(), norm.fwd(Y).contiguous()
    del X, Y
    widths = (4, 64, 64, 64, 64, 64, 4)
    sur = surrogate.Surrogate(widths, n, n, batch_max=batch, seed=0, stream=sh)
    fwd_flops = sum(2 * 9 * a * b * n * n for a, b in zip(widths[:-1], widths[1:]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = sur.fit(Xn[:ntrain], Yn[:ntrain], epochs=args.sur_epochs, batch=batch, lr=2e-3, lr_final=5e-5,
                   noise=args.sur_noise, pushforward=args.sur_pushforward, pairs_per_run=4,
                   rollout=args.sur_rollout, rollout_from=args.sur_rollout_from)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    samples = sur.fit_calls  # one forward and one backward pass of one sample each
    errs, errs_id, mse, mse_id = [], [], [], []
    for b0 in range(ntrain, Xn.shape[0] - batch + 1, batch):
        pred = sur.predict(Xn[b0:b0 + batch].contiguous())
        d, d0 = pred - Yn[b0:b0 + batch], Xn[b0:b0 + batch] - Yn[b0:b0 + batch]
        errs.append(float(d.abs().max())); errs_id.append(float(d0.abs().max()))
        mse.append(float((d * d).mean())); mse_id.append(float((d0 * d0).mean()))
    del Xn, Yn
    # one call per sample (batch of 16) against 16 FP32 HLBM steps per sample
    x = torch.from_numpy(np.random.default_rng(1).normal(size=(batch, n, n, 4)).astype(np.float32)).cuda()
    y = torch.empty_like(x)
    for _ in range(3):
        sur.predict(x, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record(stream)
    for _ in range(reps):
        sur.predict(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    sur.synchronize()  # raises if a tensor-core kernel reported a timeout
    t_sur = e0.elapsed_time(e1) / 1e3 / (reps * batch)
    held = [inputs.random_fourier(n=n, seed=10 ** 6 + k) for k in range(batch)]
    s = hlbm.Solver(n, n, stream=sh, precision=hlbm.HLBM_FP32, **held[0].params())
    s.init(*held[0].fields())
    s.step(K)
    s.synchronize()
    e0.record(stream)
    s.step(K * 50)
    e1.record(stream)
    torch.cuda.synchronize()
    t_hlbm = e0.elapsed_time(e1) / 1e3 / 50
    s.close()
    # hybrid rollout of 16 held-out states over calls * K steps, end to end
    # through the library's API (device buffers), against the plain FP32 HLBM
    x0 = torch.stack([torch.from_numpy(np.stack(c.fields(), axis=-1)) for c in held]).float().cuda()
    judge = surrogate.FieldJudge(n, held[0].params(), stream=sh)
    surrogate.hybrid_rollout_device(sur, norm, judge, x0.clone(), calls=judge_every, K=K,
                                    judge_every=judge_every, tol=args.sur_tol)  # warm-up
    plain = torch.empty_like(x0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for bi in range(batch):
        judge.advance(x0[bi], calls * K, plain[bi])
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0

    def hybrid(tol):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, lg = surrogate.hybrid_rollout_device(sur, norm, judge, x0.clone(), calls=calls, K=K,
                                                 judge_every=judge_every, tol=tol)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        d = norm.fwd(st) - norm.fwd(plain)
        return st, lg, dt, d

    st_h, log, t_hyb, dn = hybrid(args.sur_tol)
    sweep = []
    for tol in (0.5, 1.0, 2.0, 4.0, 8.0, None):
        _, lg, dt, d = hybrid(tol)
        sweep.append({"tolerance": tol, "accepted": sum(1 for *_, b in lg if not b), "judged": len(lg),
                      "final_error_vs_plain_hlbm_max": float(d.abs().max()),
                      "final_error_vs_plain_hlbm_rms": float(d.pow(2).mean().sqrt()),
                      "speedup_vs_plain_hlbm": t_plain / dt})
    judge.close()
    sur.close()
    jerr = [e for _, _, e, _ in log if math.isfinite(e)]
    return {
        "metric": "surrogate K=16 call vs 16 HLBM steps (256^2)", "value": t_hlbm / t_sur, "unit": "x",
        "dtype": "bf16 operands, f32 accumulate",
        "workload": "256^2 periodic random-Fourier fields (8 lowest modes, amplitude 0.05, Mach 0.3-1.2), K = 16, "
                    "net 4-64x5-4 3x3 periodic conv, GELU",
        "samples": int(args.sur_samples), "train": ntrain, "epochs": args.sur_epochs, "batch": batch,
        "input_noise": args.sur_noise, "pushforward": args.sur_pushforward,
        "rollout_training": {"calls": args.sur_rollout, "from_epoch_fraction": args.sur_rollout_from},
        "surrogate_s_per_sample": t_sur, "hlbm_s_per_16_steps": t_hlbm,
        "train_samples_per_s": samples / t_train, "train_tflops": 3 * fwd_flops * samples / t_train / 1e12,
        "data_generation_s": t_data, "loss_first_last": [hist[0], hist[-1]],
        "heldout_mse_normalised": float(np.mean(mse)) if mse else None,
        "heldout_mse_identity": float(np.mean(mse_id)) if mse_id else None,
        "heldout_maxabs_err_normalised": max(errs) if errs else None,
        "heldout_maxabs_err_identity": max(errs_id) if errs_id else None,
        "hybrid_rollout": {
            "samples": batch, "calls": calls, "steps": calls * K, "judge_every": judge_every,
            "tolerance": args.sur_tol, "judged": len(log), "accepted": sum(1 for *_, b in log if not b),
            "judged_nonfinite": len(log) - len(jerr),
            "judged_error_mean": float(np.mean(jerr)) if jerr else None,
            "judged_error_median": float(np.median(jerr)) if jerr else None,
            "judged_error_max": float(np.max(jerr)) if jerr else None,
            "final_error_vs_plain_hlbm_max": float(dn.abs().max()),
            "final_error_vs_plain_hlbm_rms": float(dn.pow(2).mean().sqrt()),
            "seconds": t_hyb, "plain_hlbm_seconds": t_plain, "speedup_vs_plain_hlbm": t_plain / t_hyb,
            "tolerance_sweep": sweep,
            "note": "both legs through the library's API with device buffers: per sample, the plain leg "
                    "initialises the FP32 solver, advances calls*K steps and reads the fields back; the hybrid "
                    "runs the surrogate on all samples per call and the judge (the same solver, K steps) every "
                    "judge_every-th call; a rejected sample is re-run by the solver over its whole window. "
                    "Errors: max-abs of the normalised fields (judged: one call against the judge; final: the "
                    "hybrid's state after all calls against the plain HLBM's)"},
        "field_error_bound_note": "errors in units of the per-channel standard deviation of the training inputs"}


def run_surrogate(args):
    """The surrogate leg alone, as its own JSON line."""
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = surrogate_leg(args, stream)
    out.update(n_gpus=1, higher_is_better=True, data="synthetic")
    print(json.dumps(out))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.surrogate:
        return run_surrogate(args)
    if args.batched:
        return run_batched(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
