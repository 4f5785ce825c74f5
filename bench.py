#!/usr/bin/env python
"""Benchmark of the super-potential GS/FFT free-space Poisson solve on GB300.

Metric: grid points per second (output points n^3 per second) of the solve phase
(Alg. 2; the one-time precompute of Alg. 1 is excluded, as in the paper's timings) on
the 256^3 workload: the C-infinity bump density exp(-1/(1 - r^2/0.64)) on [-1,1]^3.
The value is the FP64-accuracy path (FP64 in and out, double-float passes on the FP32
pipes, within 1e-12 of the FP64 oracle); native FP64 passes and the FP32 path are
reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 the script runs under torch.distributed.run, one rank per GPU; each rank
solves its own copy of the workload (independent solves, no collective besides the
timing barrier and the max-over-ranks reduction), so the scaling is weak.

Timing: W untimed solves, then a barrier and a device synchronise, then exactly K
solves bracketed by CUDA events on the launching stream, a synchronise, a barrier; the
step time is the maximum over ranks.  Three rho/u buffer pairs rotate, each larger
than the 129 MB L2 (with a 537 MB workspace), so no step starts with its input in L2.
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 256
BOX = (-1.0, 1.0)
# the headline metric, printed identically by both arms
METRIC = "grid pts/s at 256\u00b3 (FP64 1e-12 vs FP32 1e-5), % HBM roofline; served p50/p99"


def workload_config(n, world=1):
    """The workload both arms time: one solve (Alg. 2) of the bump density on [-1,1]^3."""
    return {"workload": f"bump exp(-1/(1-r^2/0.64)) density on [-1,1]^3, {n}^3 grid, padded {2 * n}^3, "
                        f"solve phase (Alg. 2), one independent solve per GPU",
            "grid": n, "box": list(BOX), "precision": "FP64 in/out at the 1e-12 bar",
            "l2": "inputs larger than L2: 3 rotating rho/u pairs of "
                  f"{8 * n ** 3 / 1e6:.0f} MB plus the workspace",
            "parallelism": f"replicas x{world}"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--grid", type=int, default=N_GRID, help="grid points per axis of the workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--no-configs", action="store_true", help="skip the per-configuration legs")
    ap.add_argument("--profile", nargs=3, metavar=("N", "PRECISION", "SOLVES"),
                    help="only build one plan and run SOLVES solves (a small target for ncu)")
    ap.add_argument("--ingest-ncu", nargs="+", metavar="CSV",
                    help="write profiles/ncu_counts.txt from ncu launch lists launches_<n>_<prec>.csv")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate (CUDA cores; the tensor path is no faster)


def pass_model(n, prec):
    """Algorithmic bytes and flops per launch of each pass of the five-pass solve.

    Bytes: the pass's compulsory reads and writes (real in/out at 8 or 4 B, complex
    workspace at 16 or 8 B, the multiplier octant once).  Flops: 5 N log2 N per complex
    length-N line transform (2.5 N log2 N per real line) plus 2 per multiplier use.
    """
    c = 16 if prec in ("fp64", "df32") else 8
    r = 8 if prec in ("fp64", "mixed", "df32") else 4
    m = 8 if prec in ("fp64", "df32") else 4
    n0 = n1 = n2 = n
    N = 2 * n
    lg = math.log2(N)
    half = n0 * n1 * (n2 + 1)
    full = n0 * 2 * n1 * (n2 + 1)
    out = {
        "z_forward": (r * n0 * n1 * n2 + c * half, n0 * n1 * 2.5 * N * lg),
        "y_forward": (c * half + c * full, n0 * (n2 + 1) * 5 * N * lg),
        "x_multiply": (2 * c * full + m * (n0 + 1) * (n1 + 1) * (n2 + 1),
                       2 * n1 * (n2 + 1) * (10 * N * lg + 2 * N)),
        "y_inverse": (c * full + c * half, n0 * (n2 + 1) * 5 * N * lg),
        "z_inverse": (c * half + r * n0 * n1 * n2, n0 * n1 * 2.5 * N * lg),
    }
    return out


def minimal_bytes_per_point(prec):
    """Bytes per output point of the minimal three-pass schedule (forward plane pass,
    x-pencil pass with the multiplier, inverse plane pass)."""
    return 152.0 if prec in ("fp64", "df32") else 76.0


# Sources of the solve-pass kernels (the plan, setup, graph and API files do not change
# what a pass executes); ncu counts are valid while their hash is unchanged.
PASS_SOURCES = ("sp_common.cuh", "sp_df32.cuh", "sp_fft.cuh", "sp_v2.cuh", "sp_plane.cuh", "sp_passes.cu",
                "sp_v2_df.cu", "sp_v2_df_lines.cu", "sp_v2_df_alt.cu", "sp_v2_f32.cu", "sp_v2_f32_lines.cu",
                "sp_v2_f32_alt.cu", "sp_v2_f64.cu", "sp_v2_f64_lines.cu")


def source_hash():
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_2506_04489_gb300", "csrc")
    for name in PASS_SOURCES:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:12]


COUNTS_FILE = os.path.join(ROOT, "profiles", "ncu_counts.txt")
PASS_OF_KERNEL = (("k2_z_fwd", "z_forward"), ("k2_z_inv", "z_inverse"), ("k3_line<", None), ("k2_line<", None))
LINE_MODES = {"0": "y_forward", "1": "y_inverse", "2": "x_multiply"}


def ncu_count(kernel, workload, metric):
    """Per-launch count `metric` of pass `kernel` on `workload` from the committed ncu
    summary, if it was taken on the current kernel sources; else None."""
    try:
        cur = source_hash()
        with open(COUNTS_FILE) as f:
            for line in f:
                t = line.split()
                if (len(t) == 5 and not line.startswith("#") and t[0] == kernel and t[1] == workload
                        and t[2] == metric and t[4] == cur):
                    return float(t[3])
    except OSError:
        pass
    return None


def _pass_name(kernel_name, seen):
    """Solve pass of an ncu kernel name (line passes carry their mode as the third
    template argument; y passes come before and after the x pass in launch order)."""
    for prefix, name in PASS_OF_KERNEL:
        if kernel_name.startswith("void " + prefix) or kernel_name.startswith(prefix):
            if name:
                return name
            mode = kernel_name.split("<", 1)[1].split(",")[2].strip().rstrip(">").split(">")[0]
            return LINE_MODES.get(mode)
    return None


def ingest_ncu(paths):
    """Turn ncu launch lists (--csv, one file per workload, named launches_<n>_<prec>.csv;
    metrics gpu__time_duration, dram bytes and the FP32 instruction counts) into the
    per-launch counts that bench.py reads, tagged with the current source hash, and print
    a markdown table per workload."""
    import collections
    import csv
    cur = source_hash()
    keep = []
    try:
        with open(COUNTS_FILE) as f:
            keep = [ln for ln in f if not ln.startswith("#") and ln.split() and ln.split()[-1] == cur]
    except OSError:
        pass
    rows_out = {}
    for path in paths:
        base = os.path.basename(path)[:-4].split("_")  # launches, n, prec
        workload = f"n{base[1]}_{base[2]}"
        launches = collections.OrderedDict()
        with open(path) as f:
            for r in csv.DictReader(ln for ln in f if not ln.startswith("==")):
                launches.setdefault(r["ID"], {"kernel": r["Kernel Name"]})[r["Metric Name"]] = float(
                    r["Metric Value"].replace(",", ""))
        agg = collections.OrderedDict()
        for m in launches.values():
            name = _pass_name(m["kernel"], agg)
            if name is None:
                continue
            a = agg.setdefault(name, {"kernel": m["kernel"], "n": 0, "time_ns": 0.0, "dram": 0.0, "fp32_ops": 0.0})
            a["n"] += 1
            a["time_ns"] += m.get("gpu__time_duration.sum", 0.0)
            a["dram"] += m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0)
            one = sum(m.get(f"smsp__sass_thread_inst_executed_op_{op}_pred_on.sum", 0.0) for op in ("fadd", "fmul", "ffma"))
            two = sum(m.get(f"smsp__sass_thread_inst_executed_op_{op}2_pred_on.sum", 0.0) for op in ("fadd", "fmul", "ffma"))
            a["fp32_ops"] += one + 2.0 * two
        tot = sum(a["time_ns"] for a in agg.values()) or 1.0
        print(f"\n## {workload}\n\n| pass | kernel | launches | avg ms | share | DRAM MB/launch | FP32 lane-ops/launch |")
        print("|---|---|---|---|---|---|---|")
        for name, a in agg.items():
            k = a["n"]
            print(f"| {name} | {a['kernel'].replace('void ', '').rsplit('(', 1)[0]} | {k} | {a['time_ns'] / k / 1e6:.3f} | "
                  f"{a['time_ns'] / tot:.3f} | {a['dram'] / k / 1e6:.1f} | {a['fp32_ops'] / k:.4g} |")
            rows_out[(name, workload, "dram_bytes")] = a["dram"] / k
            if a["fp32_ops"] > 0:
                rows_out[(name, workload, "fp32_lane_ops")] = a["fp32_ops"] / k
    keep = [ln for ln in keep if tuple(ln.split()[:3]) not in rows_out]
    with open(COUNTS_FILE, "w") as f:
        f.write("# per-launch counts from ncu launch lists of the bench workload (python bench.py --ingest-ncu)\n"
                "# pass workload metric value source-hash (bench.py uses a row only while the hash matches)\n")
        f.writelines(keep)
        for (name, workload, metric), v in rows_out.items():
            f.write(f"{name} {workload} {metric} {v:.6g} {cur}\n")
    return 0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_id)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        time.sleep(0.05)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            t = [x.strip() for x in line.split(",")]
            if len(t) < 9:
                continue
            try:
                sm.append(float(t[1]))
                mx.append(float(t[2]))
            except ValueError:
                continue
            for name, v in zip(names, t[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- dist
def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        # one process per GPU over NCCL; the host-side logic also runs over gloo (CPU tests)
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- oracle leg
def host_cpu():
    """Model name and logical core count of the host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"model": model, "logical_cpus": os.cpu_count()}


def oracle_solves(n, steps=1, warmup=0):
    """The FP64 CPU oracle (Alg. 2, its own FFT, the full (2n)^3 padded grid) on the bump
    density at n^3 on [-1,1]^3, all host threads: `warmup` untimed solves, then `steps`
    timed ones (solve phase only; its tables are built first, untimed, as the paper's
    timings exclude the precompute)."""
    import oracle
    from paper_2506_04489_gb300 import workloads as W
    oracle.set_threads(os.cpu_count() or 1)
    _, _, M = oracle.plan_tables(n, *BOX)
    rho = W.bump_profile(n, *BOX)
    for _ in range(warmup):
        oracle.solve(M, rho)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.solve(M, rho)
        times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    cpu = host_cpu()
    return {"value": n ** 3 / mean, "unit": "grid pts/s", "cores": oracle.get_threads(), "kind": "oracle",
            "cpu_model": cpu["model"], "logical_cpus": cpu["logical_cpus"],
            "sample": f"{steps} full oracle solves of the bump density at {n}^3 on [-1,1]^3 (the benchmark "
                      f"workload itself; solve phase only, tables built first), mean {mean:.2f} s"}, mean


def run_reference(args, world, rank):
    """The reference arm: the FP64 oracle itself on the benchmark workload (the paper
    gives no implementation to run), one full 256^3 solve per step on the host cores."""
    if rank != 0:
        return 0
    cpu, mean = oracle_solves(args.grid, steps=args.steps, warmup=args.warmup)
    line = {"impl": "reference", "metric": METRIC,
            "value": cpu["value"], "unit": "grid pts/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.grid, args.gpus),
            "cpu_baseline": cpu,
            "e2e": {"value": cpu["value"], "unit": "grid pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU leg
def time_solves(plan, rhos, outs, steps, warmup, world, stream, instrument=False):
    """W untimed solves, then K solves between CUDA events on `stream` (barrier and device
    synchronise on both sides), max over ranks.  With `instrument`, every solve also
    records an event between its passes (events created before the timed region), and
    the per-pass totals are returned; the headline region runs without them."""
    import torch
    if instrument:
        plan.set_timing(True, reserve=max(steps, warmup, 1))
    for i in range(warmup):
        plan.solve(rhos[i % len(rhos)], outs[i % len(outs)], stream)
    barrier(world)
    torch.cuda.synchronize()
    if instrument:
        plan.pass_times()  # drop the warm-up record (its events return to the pool)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(steps):
        plan.solve(rhos[i % len(rhos)], outs[i % len(outs)], stream)
    end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = start.elapsed_time(end)
    passes = None
    if instrument:
        passes = plan.pass_times()
        plan.set_timing(False)
    return max_over_ranks(ms, world), passes


# FP32 pipe of the chip: 152 SMs x 128 FP32 lanes, one operation per lane per clock
# (an FMA counts once) at the 2070 MHz maximum SM clock
FP32_LANE_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12


def roofline_for(prec, n, passes, solve_ms, hbm_peak, peak_kind):
    """Roofline of the dominant pass: its algorithmic bytes per launch (pass_model) over its
    average launch duration (CUDA events between the passes of an instrumented timed
    region) against the measured HBM bandwidth, for every precision.  Beside it: what
    actually bounds the pass (FP32 pipe for double-float, FP64 pipe for native FP64: the
    executed FP32 lane operations from ncu over the same duration, labelled as executed
    work) and the whole solve's fraction on the minimal three-pass byte count."""
    model = pass_model(n, prec)
    name = max(passes, key=lambda k: passes[k][0])
    tot_ms, launches = passes[name]
    avg_s = tot_ms / max(launches, 1) / 1e3
    nbytes, nflops = model[name]
    workload = f"n{n}_{prec}"
    traffic = ncu_count(name, workload, "dram_bytes")
    achieved = nbytes / avg_s / 1e9
    roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
            "traffic": traffic, "avg_launch_ms": avg_s * 1e3, "algorithmic_bytes": nbytes,
            "algorithmic_flops": nflops,
            "solve_frac": minimal_bytes_per_point(prec) * n ** 3 / (solve_ms / 1e3) / 1e9 / hbm_peak,
            "solve_frac_note": "minimal three-pass bytes per output point x n^3 / solve time / measured HBM"}
    if prec == "df32":
        ops = ncu_count(name, workload, "fp32_lane_ops")
        roof["limiter"] = "FP32 pipe (double-float arithmetic)"
        roof["fp32_issue_frac"] = ops / avg_s / 1e12 / FP32_LANE_PEAK_TOPS if ops else None
        roof["fp32_issue_note"] = ("EXECUTED FP32 lane operations of this kernel (ncu fadd/fmul/ffma, f32x2 forms "
                                   "twice, profiles/ncu_counts.txt) / avg launch / 152 SMs x 128 lanes x 2.07 GHz; "
                                   "executed work, not the method's")
        roof["fp64_class_tflops"] = nflops / avg_s / 1e12
    elif prec == "fp64":
        roof["limiter"] = "FP64 pipe"
        roof["fp64_pipe_frac"] = nflops / avg_s / 1e12 / FP64_PEAK_TFLOPS
        roof["fp64_pipe_note"] = "algorithmic flops (5 N log2 N per line) / avg launch / nominal 1.25 TFLOP/s"
    share = {k: round(v[0] / sum(x[0] for x in passes.values()), 4) for k, v in passes.items()}
    roof["pass_share"] = share
    return roof


def run_served(args):
    """Served stream: Poisson arrivals (mean 200/s, seed 0) of solves with n drawn from
    {32, 64, 96, 128, 192, 256} and accuracy from {1e-6 (FP32), 1e-12 (double-float)}, bump
    densities, device-resident plans (built before traffic) under a 120 GB budget; p50/p99
    latency and solves/s over the requests arriving in 30 s after a 2 s warm-up; results go
    to pinned buffers the client owns and reuses."""
    import torch

    from paper_2506_04489_gb300 import serve, workloads as W
    sizes = (32, 64, 96, 128, 192, 256)
    dens = {}
    for n in sizes:
        b = W.bump_profile(n, *BOX)
        for prec, dt in (("fp32", torch.float32), ("df32", torch.float64)):
            dens[(n, prec)] = torch.from_numpy(b).to(dt).pin_memory()
    srv = serve.Server(BOX[0], BOX[1], budget_bytes=120e9, max_batch=8, slots=4)
    srv.prepare(dens.keys())  # resident plans for every key before traffic starts
    # the client's own result buffers (pinned), reused as results are consumed
    outputs = {k: [v.new_empty(v.shape).pin_memory() for _ in range(4)] for k, v in dens.items()}
    srv.start()
    warm = 2.0
    t0 = time.monotonic() + 0.05
    # the library submits each request at its arrival time (sp_server_replay)
    serve.poisson_stream(srv, rate=200.0, duration=args.serve_seconds, sizes=sizes, accuracies=(1e-6, 1e-12),
                         seed=0, densities=dens, warmup=warm, outputs=outputs, t0=t0)
    summary = serve.latency_summary(srv, t0 + warm, t0 + warm + args.serve_seconds)
    srv.stop()
    if summary is not None:
        summary.update({"rate_per_s": 200.0, "seconds": args.serve_seconds, "warmup_s": warm,
                        "sizes": list(sizes), "accuracies": [1e-6, 1e-12], "budget_bytes": 120e9,
                        "latency": "completion (host callback once the result is in host memory) minus scheduled "
                                   "arrival, host monotonic clock; requests submitted at their arrival times by the "
                                   "library's native server"})
    return summary


def run_cufft_comparison(n, rho_np, m_octant, ref_u, steps, warmup, stream):
    """The same padded convolution (Alg. 2) with torch.fft, i.e. cuFFT, in FP64 and in
    FP32: pad into a zeroed (2n)^3 buffer, real-to-complex FFT, multiply by the plan's own
    multiplier (expanded from its octant by evenness), complex-to-real FFT, crop.  A
    comparison for the hand-written passes only; the library never calls it."""
    import torch
    N = 2 * n
    k = torch.arange(N)
    fold = torch.minimum(k, N - k)
    m64 = torch.from_numpy(m_octant)  # [|kx|][|ky|][kz], already divided by Ntilde
    out = {}
    for prec, rdt in (("fp64", torch.float64), ("fp32", torch.float32)):
        mult = m64[fold][:, fold].to("cuda", dtype=rdt).contiguous()
        pad = torch.zeros((N, N, N), dtype=rdt, device="cuda")
        rho = torch.from_numpy(rho_np).to("cuda", dtype=rdt)
        u = torch.empty_like(rho)

        def solve():
            pad[:n, :n, :n].copy_(rho)
            spec = torch.fft.rfftn(pad)
            spec.mul_(mult)
            u.copy_(torch.fft.irfftn(spec, s=(N, N, N), norm="forward")[:n, :n, :n])

        for _ in range(max(warmup, 3)):
            solve()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for _ in range(steps):
            solve()
        e.record(stream)
        torch.cuda.synchronize()
        ms = s.elapsed_time(e) / steps
        dev = float((u.double() - ref_u).abs().max() / ref_u.abs().max())
        out[prec] = {"ms_per_step": ms, "value": n ** 3 / (ms / 1e3), "unit": "grid pts/s",
                     "max_rel_dev_from_fp64": dev}
        del mult, pad, rho, u
        torch.cuda.empty_cache()
    out["note"] = ("torch.fft (cuFFT) running the same padded convolution with the same multiplier: "
                   "a comparison only, not the product path")
    return out


def _time_on(stream, fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(steps):
        fn()
    e.record(stream)
    torch.cuda.synchronize()
    return s.elapsed_time(e) / steps


def run_configs():
    """The other benchmark configurations, each timed with CUDA events on its own stream
    (a few steps each, after warm-up):
      c1  32^3 normalised Gaussian (sigma 0.1) on [-1,1]^3, FP64: time and max-norm error
          against the closed form erf(r/(sigma sqrt 2))/(4 pi r);
      c2  128^3 bump and cos-Gaussian on [-1,1]^3: double-float and native FP64;
      c3  512^3 bump: double-float, mixed (FP32 passes) and native FP64, with the mixed
          path's deviation from the double-float one and its speedup over native FP64;
      c4  64 right-hand sides of 128^3 (seeded Gaussian mixtures) in one batched solve
          replayed from a captured CUDA graph, double-float and FP32: the persistent single
          launch and the five launches with autotuned tiles, the faster one reported."""
    import numpy as np
    import torch

    from paper_2506_04489_gb300 import Plan, workloads as W
    st = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(st):
        # c1
        n, sig = 32, 0.1
        plan = Plan(n, BOX[0], BOX[1], precision="fp64")
        rho = torch.from_numpy(W.gaussian(n, BOX[0], BOX[1], sig)).cuda()
        u = torch.empty_like(rho)
        ms = _time_on(st, lambda: plan.solve(rho, u, st), 20, 3)
        X, Y, Z = W.mesh(n, BOX[0], BOX[1])
        r = np.sqrt(X * X + Y * Y + Z * Z)
        exact = np.vectorize(math.erf)(r / (sig * math.sqrt(2.0))) / (4.0 * math.pi * r)
        err = float(np.abs(u.cpu().numpy() - exact).max() / np.abs(exact).max())
        out["c1_gaussian_32_fp64"] = {"ms_per_solve": ms, "max_rel_err_vs_closed_form": err}
        plan.close()
        # c2
        n = 128
        c2 = {}
        for name, dens in (("bump", W.bump_profile(n, *BOX)), ("cos_gaussian", W.cos_gaussian(n, *BOX))):
            ref = None
            for prec in ("fp64", "df32"):
                plan = Plan(n, BOX[0], BOX[1], precision=prec)
                plan.autotune(1)
                rho = torch.from_numpy(dens).cuda()
                u = torch.empty_like(rho)
                ms = _time_on(st, lambda: plan.solve(rho, u, st), 20, 3)
                rec = {"ms_per_solve": ms, "value": n ** 3 / (ms / 1e3), "unit": "grid pts/s"}
                if ref is None:
                    ref = u.clone()
                else:
                    rec["max_rel_dev_from_fp64"] = float((u - ref).abs().max() / ref.abs().max())
                c2[f"{name}_{prec}"] = rec
                plan.close()
        out["c2_128"] = c2
        # c3
        n = 512
        c3 = {}
        dens = W.bump_profile(n, *BOX)
        ref = None
        for prec, steps, tune in (("df32", 5, True), ("mixed", 5, True), ("fp64", 2, False)):
            plan = Plan(n, BOX[0], BOX[1], precision=prec)
            if tune:
                plan.autotune(1)
            rho = torch.from_numpy(dens).cuda()
            u = torch.empty_like(rho)
            ms = _time_on(st, lambda: plan.solve(rho, u, st), steps, 1)
            rec = {"ms_per_solve": ms, "value": n ** 3 / (ms / 1e3), "unit": "grid pts/s"}
            if ref is None:
                ref = u.clone()
            else:
                rec["max_rel_dev_from_df32"] = float((u - ref).abs().max() / ref.abs().max())
            c3[prec] = rec
            plan.close()
            del rho, u
            torch.cuda.empty_cache()
        c3["mixed_speedup_over_fp64"] = c3["fp64"]["ms_per_solve"] / c3["mixed"]["ms_per_solve"]
        c3["df32_speedup_over_fp64"] = c3["fp64"]["ms_per_solve"] / c3["df32"]["ms_per_solve"]
        out["c3_bump_512"] = c3
        del ref
        torch.cuda.empty_cache()
        # c4
        n, nb = 128, 64
        c4 = {}
        host = np.stack([W.gaussian_mixture(n, BOX[0], BOX[1], s) for s in range(nb)])
        for prec in ("df32", "fp32"):
            plan = Plan(n, BOX[0], BOX[1], precision=prec, max_batch=nb)
            plan.autotune(nb)
            rho = torch.from_numpy(host).to("cuda", dtype=plan.dtype)
            u = torch.empty_like(rho)
            rec = {}
            # one persistent cooperative launch (all five passes, grid barriers between
            # them) captured in a graph, and the graph of five launches with autotuned tiles
            for mode in ("persistent", "five_launches"):
                plan.set_persistent(mode == "persistent")
                graph = plan.capture(rho, u, st)
                ms = _time_on(st, lambda: graph.launch(st), 10, 2)
                plan.sync()
                rec[mode] = {"ms_per_batch": ms, "solves_per_s": nb / (ms / 1e3), "value": nb * n ** 3 / (ms / 1e3),
                             "unit": "grid pts/s"}
                graph.close()
            best = min(rec, key=lambda k: rec[k]["ms_per_batch"])
            c4[prec] = dict(rec[best], launch=best, launch_config=plan.launch_config(), modes=rec)
            plan.close()
            del rho, u
            torch.cuda.empty_cache()
        out["c4_batched_64x128_graph"] = c4
    return out


def run_ours(args, world, rank, local):
    import torch

    from paper_2506_04489_gb300 import Plan, workloads as W
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.grid
    hbm_peak, peak_kind = peaks()
    stream = torch.cuda.current_stream()
    rho_np = W.bump_profile(n, *BOX)
    results = {}
    clocks = None
    ref_u = None
    # clocks sampled from the native FP64 run through the end of the double-float timed
    # region (the headline), i.e. around and during it
    sampler = ClockSampler(local)
    for prec in ("fp64", "df32", "fp32"):
        plan = Plan(n, BOX[0], BOX[1], precision=prec)
        launch_config = plan.autotune(1)  # the library's own autotuner (tiles, radix plans; setup, not timed)
        dt = plan.dtype
        base = torch.from_numpy(rho_np).to(dev, dtype=dt)
        rhos = [base.clone() for _ in range(3)]
        outs = [torch.empty_like(base) for _ in range(3)]
        # the headline region: plain solves, nothing recorded between the passes
        ms, _ = time_solves(plan, rhos, outs, args.steps, args.warmup, world, stream)
        if prec == "df32":
            clocks = sampler.stop()
        ms_step = ms / args.steps
        value = world * n ** 3 / (ms_step / 1e3)
        # a second timed region of the same K solves with an event between passes (events
        # created beforehand): per-pass durations for the roofline of the dominant pass
        ms_i, passes = time_solves(plan, rhos, outs, args.steps, 2, world, stream, instrument=True)
        roof = roofline_for(prec, n, passes, ms_step, hbm_peak, peak_kind)
        roof["instrumented_ms_per_step"] = ms_i / args.steps
        hbm_frac = minimal_bytes_per_point(prec) * n ** 3 / (ms_step / 1e3) / 1e9 / hbm_peak
        launches = sum(v[1] for v in passes.values())
        # live accuracy guard: deviation of this path from the native FP64 solve of the
        # same input (the FP64 path itself is checked against the oracle in tests/)
        u_dev = outs[(args.steps - 1) % len(outs)].double()
        if prec == "fp64":
            ref_u = u_dev.clone()
            rel_dev = 0.0
            m_octant = plan.tables(0)["M"]  # multiplier / Ntilde, for the cuFFT comparison
        else:
            rel_dev = float((u_dev - ref_u).abs().max() / ref_u.abs().max())
        roof["launch_config"] = launch_config
        results[prec] = {"value": value, "ms_per_step": ms_step, "roofline": roof,
                         "max_rel_dev_from_fp64": rel_dev,
                         "hbm_roofline": {"frac": hbm_frac, "bytes_per_point": minimal_bytes_per_point(prec),
                                          "peak_gbs": hbm_peak, "note": "bytes of the minimal 3-pass schedule / "
                                          "solve time / measured HBM bandwidth"},
                         "gpu_launches": launches}
        # end to end through the C ABI's host-buffer entry (sp_solve_host): pinned host
        # densities -> device -> solve -> pinned host potentials, each step's copies
        # overlapped with its neighbours' solves
        if prec == "df32":
            e2e_steps = max(10, args.steps)
            host_in = [torch.from_numpy(rho_np).to(dtype=dt).pin_memory() for _ in range(2)]
            host_out = [torch.empty(host_in[0].shape, dtype=dt, pin_memory=True) for _ in range(2)]
            ins = [host_in[i % 2] for i in range(e2e_steps)]
            outs_h = [host_out[i % 2] for i in range(e2e_steps)]
            plan.solve_host_stream(ins[:4], outs_h[:4], stream)  # warm-up (streams, staging buffers)
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            plan.solve_host_stream(ins, outs_h, stream)
            torch.cuda.synchronize()
            e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, world) / e2e_steps
            barrier(world)
            host_in = host_in[0]
            host_out = host_out[0]
            results["e2e"] = {"value": world * n ** 3 / (e2e_ms / 1e3), "unit": "grid pts/s",
                              "ms_per_step": e2e_ms, "h2d_bytes_per_step": host_in.numel() * host_in.element_size(),
                              "d2h_bytes_per_step": host_out.numel() * host_out.element_size()}
        plan.close()
        del rhos, outs, base
        torch.cuda.empty_cache()
    # the served stream (part of the headline metric) right after the headline legs, before
    # the other configurations' large allocations
    served = None
    if world == 1 and not args.no_serve:
        try:
            served = run_served(args)
        except Exception as e:  # a served stream that fails or stalls is reported, not fatal
            served = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()
    cufft = run_cufft_comparison(n, rho_np, m_octant, ref_u, args.steps, args.warmup, stream)
    configs = run_configs() if (world == 1 and not args.no_configs) else None
    del ref_u
    torch.cuda.empty_cache()
    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu, _ = oracle_solves(n, steps=2, warmup=0)
    r64 = results["df32"]
    line = {
        "metric": METRIC,
        "value": r64["value"], "unit": "grid pts/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r64["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2 (double-float)", "data": "synthetic",
        "accuracy_path": "double-float passes (hi+lo FP32 pairs) meet the FP64 bar: oracle parity <= 1e-12 "
                         "in tests/; live max deviation from the native FP64 solve reported below",
        "config": workload_config(n, world),
        "roofline": r64["roofline"],
        "hbm_roofline": r64["hbm_roofline"],
        "max_rel_dev_from_fp64": r64["max_rel_dev_from_fp64"],
        "fp64_native": {"value": results["fp64"]["value"], "unit": "grid pts/s",
                        "ms_per_step": results["fp64"]["ms_per_step"], "roofline": results["fp64"]["roofline"],
                        "hbm_roofline": results["fp64"]["hbm_roofline"]},
        "fp32": {"value": results["fp32"]["value"], "unit": "grid pts/s",
                 "ms_per_step": results["fp32"]["ms_per_step"], "roofline": results["fp32"]["roofline"],
                 "hbm_roofline": results["fp32"]["hbm_roofline"],
                 "max_rel_dev_from_fp64": results["fp32"]["max_rel_dev_from_fp64"]},
        "e2e": results["e2e"],
        "cufft_comparison": cufft,
        "configs": configs,
        "served": served,
        "gpu_launches": r64["gpu_launches"],
        "clocks": clocks,
        "cpu_baseline": cpu,
        "kernel_sources": source_hash(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_profile_case(args):
    """One plan of grid N^3 and the given precision, autotuned as in the bench, then
    SOLVES solves of the bump density inside an NVTX range named "solves" (ncu
    --nvtx --nvtx-include solves/ captures just those launches): the launch sequence
    that the ncu summaries under profiles/ capture."""
    import torch

    from paper_2506_04489_gb300 import Plan, workloads as W
    n, prec, k = int(args.profile[0]), args.profile[1], int(args.profile[2])
    plan = Plan(n, BOX[0], BOX[1], precision=prec)
    plan.autotune(1)
    rho = torch.from_numpy(W.bump_profile(n, *BOX)).cuda().to(plan.dtype)
    out = torch.empty_like(rho)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("solves")
    for _ in range(k):
        plan.solve(rho, out)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": {"n": n, "precision": prec, "solves": k, "launch_config": plan.launch_config()}}))
    plan.close()
    return 0


def main():
    args = parse()
    if args.ingest_ncu:
        return ingest_ncu(args.ingest_ncu)
    if args.profile:
        return run_profile_case(args)
    if args.impl == "reference":
        # host-only arm: rank 0 times the oracle, the other ranks exit without work
        return run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
    world, rank, local = dist_init()
    rc = run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
