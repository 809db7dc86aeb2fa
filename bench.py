#!/usr/bin/env python3
"""LJ pair interactions/s on one GB300: FP64, mixed precision and double-float.

Workload: the paper's benchmark (section "Benchmark Conditions"): an FCC
crystal of N = 119,164 = 4*31^3 atoms at density 1.0, cutoff 3.0 sigma,
search length 3.3 sigma (bookkeeping margin 0.3), jitter 0.05 sigma,
particle order randomly permuted, half list (i < j), dt = 0.01.

One step = one pass of the hot path: build the sorted CSR Verlet list on
the GPU (cell binning, count, scan, fill) and then run the force 100 times
on it, the paper's protocol ("the time to calculate the force 100 times").
A pair interaction is one unique list entry processed in one force call,
so each step credits 100 * nnz(half list).

Timing: inputs resident in HBM; L2 flushed (256 MiB write) before every
step, outside the timed events; each step timed with CUDA events on the
launching stream (three events a step: start, list built, end; the force
call's duration is the span after the list over the 100 calls); W warm-up
steps; the max over ranks of the summed step times.  `e2e` repeats the step with the positions and momenta copied from
pinned host memory and the momenta copied back inside the timed region.

`--impl reference` times the CPU oracle (the plain double-precision C
implementation the tests compare against) on the same workload: each step
is one oracle cell-list build plus 10 oracle force calls, single thread.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "LJ pair interactions/s on 1 GB300, FP64 vs mixed at stated error; % HBM roofline"
UNIT = "pair interactions/s"
FORCE_CALLS = 100
DT, RC, MARGIN = 0.01, 3.0, 0.3
CPU_FORCE_CALLS = 10
L2_FLUSH_BYTES = 256 << 20
# FP64 peak derived from unit counts and clock: 152 SMs x 2 FP64 FMA/clk/SM
# (4 flop) x 2070 MHz (the nominal 1.25 TFLOP/s FP64 of GB300).
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 256 * 2.07e9 / 1e12
# DRAM bytes (read + write) per launch of the FP64 force kernel, by
# schedule, from one ncu capture of the kernel as it stands on this workload
# (profiles/force_fp64_images_tpi8_half_N119164.md); a schedule without an
# entry reports null.
# DRAM bytes (read + write) of one launch of the FP64 force kernel per
# schedule, from ncu (cold cache), with the profile that records them.
# L2 read and reduction sectors per launch of the FP64 force kernel from the
# same ncu capture (the gathered-bytes view), per schedule.
LTS_SECTORS_PER_LAUNCH = {
    2056: (11254023, 24806804, "profiles/force_fp64_fixed_tpi8_half_N119164.md"),
}
TRAFFIC_PER_LAUNCH = {
    1032: (41903872.0 + 1280.0, "profiles/force_fp64_images_tpi8_half_N119164.md"),
    2056: (41910784.0 + 5632.0, "profiles/force_fp64_fixed_tpi8_half_N119164.md"),
    4104: (41915904.0, "profiles/force_fp64_compact_tpi8_half_N119164.md"),
}


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--order", choices=["random", "cell"], default="random")
    ap.add_argument("--no-variants", action="store_true", help="skip the per-variant table")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads (1M atoms, 512-system batch, 64-replica adjoint)")
    ap.add_argument("--profile", choices=["fp64", "fp64-full", "mixed", "mixed-full", "dfloat",
                                          "dfloat-full", "list", "vjp", "vjp-dfloat", "batched",
                                          "batched-mixed", "batched-dfloat"],
                    help="no timing: build the list and run a few calls of one kernel (for ncu)")
    ap.add_argument("--schedule", type=int, default=0,
                    help="FP64 schedule for the timed steps (0 = the library's autotuner picks)")
    ap.add_argument("--peaks", action="store_true",
                    help="only measure the FP64 / FP32 / packed-FP32 / L2-read ceilings and print them")
    ap.add_argument("--profile-atoms", choices=["paper", "million"], default="paper")
    ap.add_argument("--profile-tpi", type=int, default=0, help="schedule for --profile (0 = auto)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback (profiling recipe)"


def measure_ceilings(lj, dev, target_ms: float = 40.0, reps: int = 3):
    """The roofline denominators of the force kernels, measured on this GPU
    with the library's probe kernels (lj_measure_peak): DFMA, FFMA and
    packed-FFMA throughput (TFLOP/s) and L2 read bandwidth of a 32 MiB
    resident buffer (GB/s).  Each probe is sized to run ~target_ms and the
    best of `reps` runs is kept."""
    import torch
    buf = torch.zeros(32 << 20, dtype=torch.uint8, device=dev)
    out = {}
    for name, kind, scale in (("fp64_fma_tflops", lj.LJ_PEAK_DFMA, 1e12),
                              ("fp32_fma_tflops", lj.LJ_PEAK_FFMA, 1e12),
                              ("fp32x2_fma_tflops", lj.LJ_PEAK_FFMA2, 1e12),
                              ("l2_read_gbs", lj.LJ_PEAK_L2_READ, 1e9)):
        b = buf if kind == lj.LJ_PEAK_L2_READ else None
        work = 4
        _, ms = lj.lj_measure_peak(kind, work, b)
        work = max(1, int(work * target_ms / max(ms, 1e-3)))
        best, best_ms = 0.0, 0.0
        for _ in range(reps):
            rate, ms = lj.lj_measure_peak(kind, work, b)
            if rate > best:
                best, best_ms = rate, ms
        out[name] = best / scale
        out[name.rsplit("_", 1)[0] + "_ms"] = best_ms
    del buf
    return out


def run_peaks(args):
    import torch
    from paper_1806_05713_gb300 import build as lib_build
    from paper_1806_05713_gb300 import lj
    lib_build.build()
    dev = torch.device("cuda", 0)
    lj.load()
    with ClockSampler(0) as clk:
        res = measure_ceilings(lj, dev)
    res["clocks"] = clk.summary()
    res["sm_count"] = torch.cuda.get_device_properties(dev).multi_processor_count
    res["derived_fp64_tflops"] = FP64_PEAK_TFLOPS
    res["derived_fp32_tflops"] = FP32_PEAK_TFLOPS
    print(json.dumps(res))


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None or not self.path:
            out["reasons"] = ["nvidia-smi unavailable"]
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over all ranks (all-reduce MAX); x itself when world = 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return units_per_rank * world / (max_ms / 1e3)


def workload(rank: int, order: str):
    from paper_1806_05713_gb300 import inputs
    return inputs.fcc_system(31, 1.0, 0.05, seed=rank, order=order, rc=RC, margin=MARGIN)


def workload_name(order: str) -> str:
    return f"fcc-31^3 N=119164 rho=1.0 rc=3.0 rs=3.3 jitter=0.05 {order}-order half-list dt=0.01"


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and --impl reference)
# ---------------------------------------------------------------------------

def oracle_sample(s, calls: int):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    rp, col = oracle.pairlist(s.q, s.box, s.rs, True, "cells")
    p = np.zeros((s.n, 3))
    for _ in range(calls):
        p = oracle.force(s.q, p, rp, col, True, DT, s.rc, s.box)
    dt = time.perf_counter() - t0
    return dt, int(col.size)


def run_reference(args, world, rank):
    if rank != 0:
        return
    s = workload(0, args.order)
    for _ in range(max(0, args.warmup)):
        oracle_sample(s, 1)
    times, nnz = [], 0
    for _ in range(args.steps):
        t, nnz = oracle_sample(s, CPU_FORCE_CALLS)
        times.append(t)
    total = sum(times)
    value = args.steps * CPU_FORCE_CALLS * nnz / total
    sample = (f"each step: 1 oracle cell-list build + {CPU_FORCE_CALLS} oracle force calls on "
              f"N={s.n} ({nnz} half-list entries), single thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args.order), "n_atoms": s.n, "pairs_per_call": nnz,
                   "force_calls_per_step": CPU_FORCE_CALLS, "list_builds_per_step": 1,
                   "parallelism": "one CPU thread"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def count_in_cutoff(q, pl, box, rc):
    """Entries with r < r_c (for the flop count), with torch on the GPU at
    set-up time; not part of the timed path."""
    import torch
    rp = pl.row_ptr.long()
    rows = torch.repeat_interleave(torch.arange(pl.n, device=q.device), rp[1:] - rp[:-1])
    col = pl.col_view.long()
    d = q[col, :3] - q[rows, :3]
    L = torch.tensor(box, device=q.device, dtype=torch.float64)
    d = d - L * torch.round(d / L)
    return int(((d * d).sum(1) < rc * rc).sum().item())


def run_profile(args):
    """A short, fixed launch sequence for a profiler: 2 list builds, then
    5 calls of the chosen force kernel (or 3 more list builds)."""
    import torch
    from paper_1806_05713_gb300 import build as lib_build
    from paper_1806_05713_gb300 import inputs, lj
    lib_build.build()
    k = 31 if args.profile_atoms == "paper" else 64
    s = inputs.fcc_system(k, 1.0, 0.05, seed=0, order=args.order, rc=RC, margin=MARGIN)
    box = [float(x) for x in s.box]
    q = torch.from_numpy(s.q).cuda()
    p = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
    half = not args.profile.endswith("full")
    if args.profile.startswith("batched"):
        from paper_1806_05713_gb300.batch import Batch
        systems = inputs.batched_systems(nsys=64, seed=0)
        prec = {"batched": lj.LJ_FP64, "batched-mixed": lj.LJ_MIXED,
                "batched-dfloat": lj.LJ_DFLOAT}[args.profile]
        b = Batch(systems, DT, prec, True, tpi=8 if prec == lj.LJ_FP64 else 4, rows_per_item=16)
        for _ in range(5):
            b.force()
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "systems": len(systems), "atoms": b.total_atoms}))
        return
    if args.profile.startswith("vjp"):
        half = False
    pl = lj.lj_build_pairlist(q, box, s.rs, half)
    pl = lj.lj_build_pairlist(q, box, s.rs, half, reuse=pl)
    if args.profile.startswith("vjp"):
        R = torch.ones((s.n, 4), dtype=torch.float64, device="cuda")
        prec = lj.LJ_DFLOAT if args.profile == "vjp-dfloat" else lj.LJ_FP64
        for _ in range(5):
            lj.lj_force_vjp(q, R, pl, s.rc, box, 1.1, 0.97, prec)
    elif args.profile == "list":
        for _ in range(3):
            lj.lj_build_pairlist(q, box, s.rs, half, reuse=pl)
    else:
        prec = (lj.LJ_MIXED if args.profile.startswith("mixed") else
                lj.LJ_DFLOAT if args.profile.startswith("dfloat") else lj.LJ_FP64)
        tpi = args.profile_tpi
        fn = lj.lj_force_prepared(q, p, pl, DT, s.rc, box, precision=prec, tpi=tpi)
        for _ in range(5):
            fn()
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "n": s.n, "nnz": pl.nnz,
                      "launches": int(lj.load().lj_kernel_launch_count())}))


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.profile:
        run_profile(args)
        return
    if args.peaks:
        run_peaks(args)
        return

    import torch
    import torch.distributed as dist
    from paper_1806_05713_gb300 import build as lib_build
    from paper_1806_05713_gb300 import lj

    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    if rank == 0:
        lib_build.build()
    if world > 1:
        dist.barrier()
    lib = lj.load()

    s = workload(rank, args.order)
    box = [float(x) for x in s.box]
    q = torch.from_numpy(s.q).to(dev)
    p = torch.zeros((s.n, 4), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    pl = lj.lj_build_pairlist(q, box, s.rs, True)
    # schedule picked by the library's autotuner on this system and list
    if args.schedule:
        best_tpi, tune_table = args.schedule, {}
    else:
        best_tpi, _, tune_table = lj.lj_autotune_force(q, pl, DT, s.rc, box, reps=5)
    force = lj.lj_force_prepared(q, p, pl, DT, s.rc, box, precision=lj.LJ_FP64, tpi=best_tpi)
    nnz = pl.nnz
    n_cut = count_in_cutoff(q, pl, box, s.rc)

    def one_step(list_done):
        lj.lj_build_pairlist(q, box, s.rs, True, reuse=pl)
        list_done.record(stream)
        for c in range(FORCE_CALLS):
            force()

    def new_events():
        return [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    for _ in range(args.warmup):
        flush.zero_()
        one_step(new_events()[1])
    torch.cuda.synchronize()

    step_ms, list_ms, force_ms = [], [], []
    launches0 = lib.lj_kernel_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0, e_list, e1 = new_events()
            e0.record(stream)
            one_step(e_list)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            list_ms.append(e0.elapsed_time(e_list))
            # the average force call (fixed-point pre-pass + force kernel)
            force_ms.append(e_list.elapsed_time(e1) / FORCE_CALLS)
        torch.cuda.synchronize()
    launches = lib.lj_kernel_launch_count() - launches0
    if world > 1:
        dist.barrier()
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    pairs_rank = FORCE_CALLS * nnz * args.steps
    value = whole_job_rate(pairs_rank, world, total_ms)

    # ---- end to end through the public API, host buffers --------------------
    q_host = torch.from_numpy(s.q).pin_memory()
    p_host = torch.zeros((s.n, 4), dtype=torch.float64).pin_memory()
    p_back = torch.empty_like(p_host).pin_memory()
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        q.copy_(q_host, non_blocking=True)
        p.copy_(p_host, non_blocking=True)
        lj.lj_build_pairlist(q, box, s.rs, True, reuse=pl)
        for _ in range(FORCE_CALLS):
            force()
        p_back.copy_(p, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if it >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_total = max_over_ranks(sum(e2e_ms), world, dev)
    e2e_value = whole_job_rate(pairs_rank, world, e2e_total)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (the FP64 force) -------------------
    hbm_peak, hbm_src = measured_peaks()
    t_force = statistics.mean(force_ms) / 1e3
    flops = 28.0 * n_cut + 8.0 * (nnz - n_cut)     # paper: 27 add/mul + 1 div per pair
    alg_bytes = 4.0 * nnz + 4.0 * (s.n + 1) + 32.0 * s.n + 64.0 * s.n
    roof = {"bound": "alu", "achieved": flops / t_force / 1e12, "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": flops / t_force / 1e12 / FP64_PEAK_TFLOPS,
            "traffic": TRAFFIC_PER_LAUNCH.get(best_tpi, (None, None))[0],
            "traffic_source": (TRAFFIC_PER_LAUNCH.get(best_tpi, (None, "not profiled"))[1] +
                               " (ncu dram__bytes_read.sum + dram__bytes_write.sum, cold cache)"),
            "kernel": f"FP64 force kernel, {schedule_name(best_tpi)}, half list",
            "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2.07 GHz (nominal 1.25 TFLOP/s)",
            "flops_per_launch": flops, "launch_ms": t_force * 1e3}
    hbm_view = {"achieved": alg_bytes / t_force / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": alg_bytes / t_force / 1e9 / hbm_peak, "peak_source": hbm_src,
                "bytes_per_pair": alg_bytes / nnz}
    # the gathered-bytes view: what the kernel asks of L2 -- per entry its
    # column index and q_j record, per row its row pointers and q_i, and the
    # FP64 reductions (p_j per interacting entry, p_i per lane and row)
    gathered_reads = 36.0 * nnz + 40.0 * s.n
    reductions = 3.0 * n_cut + 3.0 * 8 * s.n
    lts = LTS_SECTORS_PER_LAUNCH.get(best_tpi)
    l2_view = {"gathered_read_bytes": gathered_reads, "reductions": reductions,
               "gathered_read_GBps": gathered_reads / t_force / 1e9,
               "reductions_per_s": reductions / t_force,
               "lts_read_sectors": None if lts is None else lts[0],
               "lts_red_sectors": None if lts is None else lts[1],
               "lts_source": None if lts is None else lts[2]}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.order), "n_atoms": s.n, "pairs_per_call": nnz,
                   "pairs_in_cutoff": n_cut, "force_calls_per_step": FORCE_CALLS,
                   "list_builds_per_step": 1, "schedule": schedule_name(best_tpi),
                   "l2": "flushed before every step (256 MiB write, outside the timed events)",
                   "parallelism": f"replicas x{world}"},
        "list_build_ms": statistics.mean(list_ms),
        "force_ms_per_call": t_force * 1e3,
        "force_only_pairs_per_s": nnz / t_force,
        "roofline": roof, "hbm_roofline": hbm_view, "l2_gather_view": l2_view,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 32 * s.n,
                "d2h_bytes_per_step": 32 * s.n},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }

    out["autotune_ms"] = {schedule_name(k): v for k, v in tune_table.items()}
    out["forms"] = forms(lj, q, pl, box, s, best_tpi, flops, dev, stream, flush)
    if not args.no_variants:
        out["variants"] = variants(lj, s, q, pl, box, dev, stream, flush)
    if not args.no_extra:
        del p, q, pl, force
        torch.cuda.empty_cache()
        out["other_configs"] = {
            "million_fp64_vs_mixed": extra_million(lj, dev, stream, flush),
            "batched_512_systems": extra_batched(lj, dev, stream, flush),
            "adjoint_64_replicas": extra_adjoint(lj, dev, stream, flush),
            "md_velocity_verlet": extra_md(lj, dev, stream),
        }
    if world == 1 and not args.no_cpu:
        t, m = oracle_sample(s, CPU_FORCE_CALLS)
        out["cpu_baseline"] = {
            "value": CPU_FORCE_CALLS * m / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 oracle cell-list build + {CPU_FORCE_CALLS} oracle force calls on the "
                      f"same N={s.n} system, single thread ({t:.1f} s)"}
    print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def schedule_name(tpi: int) -> str:
    t = tpi & 63
    name = f"{max(t, 1)} lanes/row"
    if tpi & 256:
        name = f"lane-queue, {name}"
    if tpi & 64:
        name = f"group-refill, {name}"
    if tpi & 128:
        name += ", 2 entries/lane (software-pipelined)"
    if tpi & 512:
        name += ", rows by length"
    if tpi & 1024:
        name += ", image-selected displacement"
    if tpi & 2048:
        name += ", exact fixed-point displacement"
    if tpi & 4096:
        name += ", exact fixed-point displacement, margin entries compacted away"
    return name


def extra_million(lj, dev, stream, flush):
    """N = 1,048,576 (64^3 FCC): FP64 vs mixed, per call (L2 flushed), the
    mixed error against the FP64 result."""
    import torch
    from paper_1806_05713_gb300 import inputs
    s = inputs.workload_million()
    box = [float(x) for x in s.box]
    q = torch.from_numpy(s.q).to(dev)
    t_list = time_calls(lambda: lj.lj_build_pairlist(q, box, s.rs, True), stream, flush, 3, 1)
    pl = lj.lj_build_pairlist(q, box, s.rs, True)
    res = {"n_atoms": s.n, "pairs_per_call": pl.nnz, "list_build_ms": t_list}
    best, _, _ = lj.lj_autotune_force(q, pl, DT, s.rc, box, reps=3)
    out = {}
    for name, prec, tpis in (("fp64", lj.LJ_FP64, (best,)), ("mixed", lj.LJ_MIXED, (4, 8, 16)),
                             ("dfloat", lj.LJ_DFLOAT, (136, 132))):
        for t in tpis:
            pp = torch.zeros((s.n, 4), dtype=torch.float64, device=dev)
            fn = lj.lj_force_prepared(q, pp, pl, DT, s.rc, box, precision=prec, tpi=t)
            ms = time_calls(fn, stream, flush, 10, 2)
            pp.zero_()
            fn()
            out[(name, t)] = (ms, pp[:, :3].clone())
    ms64, ref = out[("fp64", best)]
    res["fp64"] = {"schedule": schedule_name(best), "ms": ms64, "pairs_per_s": pl.nnz / (ms64 / 1e3)}
    mk = min((k for k in out if k[0] == "mixed"), key=lambda k: out[k][0])
    msm, pm = out[mk]
    err = pm - ref
    res["mixed"] = {"schedule": schedule_name(mk[1]), "ms": msm, "pairs_per_s": pl.nnz / (msm / 1e3),
                    "max_err_rel_vs_fp64": float(err.abs().max() / ref.abs().max()),
                    "rms_err_rel_vs_fp64": float(err.pow(2).mean().sqrt() / ref.pow(2).mean().sqrt())}
    res["speedup_mixed_vs_fp64"] = ms64 / msm
    dk = min((k for k in out if k[0] == "dfloat"), key=lambda k: out[k][0])
    msd, pd = out[dk]
    err = pd - ref
    res["dfloat"] = {"schedule": schedule_name(dk[1]), "ms": msd, "pairs_per_s": pl.nnz / (msd / 1e3),
                     "max_err_rel_vs_fp64": float(err.abs().max() / ref.abs().max()),
                     "rms_err_rel_vs_fp64": float(err.pow(2).mean().sqrt() / ref.pow(2).mean().sqrt())}
    res["speedup_dfloat_vs_fp64"] = ms64 / msd
    return res


def extra_batched(lj, dev, stream, flush):
    """512 systems, N log-uniform in 500..32000, rho in 0.8..1.2, rc 2.5 or
    3.0: one persistent launch replayed from a CUDA graph vs one launch per
    system, FP64, mixed and double-float; the autotuner picks lanes per row,
    rows per work item and the list layout (half list with atomics or full
    list without)."""
    import torch
    from paper_1806_05713_gb300 import inputs
    from paper_1806_05713_gb300.batch import Batch
    systems = inputs.batched_systems(nsys=512, seed=0)
    res = {"n_systems": len(systems), "total_atoms": int(sum(s.n for s in systems))}
    for name, prec in (("fp64", lj.LJ_FP64), ("mixed", lj.LJ_MIXED), ("dfloat", lj.LJ_DFLOAT)):
        b = Batch(systems, DT, prec, True, tpi=8, rows_per_item=64, plan_rows_min=16)
        tpi, rows, _ = b.autotune(tpis=(4, 8, 16), rows=(16, 32, 64, 128), reps=3,
                                  layouts=(True, False))
        g = b.capture_graph()
        t_graph = time_calls(g.replay, stream, flush, 10, 2)
        t_sep = time_calls(lambda: b.force_per_system(tpi=lj.LJ_TPI_AUTO),
                           stream, flush, 5, 1)
        res[name] = {"tpi": tpi, "rows_per_item": rows, "list": "half" if b.half else "full",
                     "pairs_per_call": b.pairs,
                     "graph_persistent_ms": t_graph,
                     "graph_persistent_pairs_per_s": b.pairs / (t_graph / 1e3),
                     "per_system_launches_ms": t_sep,
                     "per_system_pairs_per_s": b.pairs / (t_sep / 1e3),
                     "speedup": t_sep / t_graph}
        del b, g
    return res


def extra_adjoint(lj, dev, stream, flush):
    """64 replicas of N = 16,384 (16^3 FCC, rho 1, jitter 0.1): forces with
    (eps, sigma) = (1.1, 0.97) against targets at (1, 1), mean squared force
    error, gradient w.r.t. positions, eps and sigma through the autograd
    wrapper (forward kernel + hand-written adjoint kernel)."""
    import torch
    from paper_1806_05713_gb300 import inputs
    from paper_1806_05713_gb300.autograd import lj_forces
    reps = inputs.workload_replicas(64, 16, seed=0)
    L = float(reps[0].box[0])
    box = [L, L, L]
    n1 = reps[0].n
    q = torch.from_numpy(np.concatenate([r.q for r in reps])).to(dev)
    rows, cols, off = [torch.zeros(1, dtype=torch.int32, device=dev)], [], 0
    for k, r in enumerate(reps):  # block-diagonal list over replicas sharing one box size
        pl = lj.lj_build_pairlist(q[k * n1:(k + 1) * n1].contiguous(), box, r.rs, False)
        rows.append(pl.row_ptr[1:] + off)
        cols.append(pl.col_view + k * n1)
        off += pl.nnz
    big = lj.PairList(torch.cat(rows).contiguous(), torch.cat(cols).contiguous(), q.shape[0], off,
                      False, reps[0].rs, 0)
    Ft = torch.zeros_like(q)
    lj.lj_force(q, Ft, big, 1.0, reps[0].rc, box, 1.0, 1.0)
    res = {"replicas": len(reps), "atoms": int(q.shape[0]), "pairs": off // 2}
    for name, prec in (("fp64", lj.LJ_FP64), ("mixed", lj.LJ_MIXED), ("dfloat", lj.LJ_DFLOAT)):
        eps = torch.tensor(1.1, dtype=torch.float64, device=dev, requires_grad=True)
        sig = torch.tensor(0.97, dtype=torch.float64, device=dev, requires_grad=True)

        def step():
            qq = q.detach().requires_grad_(True)
            eps.grad = None
            sig.grad = None
            F = lj_forces(qq, eps, sig, big, reps[0].rc, box, prec)
            loss = ((F - Ft) ** 2)[:, :3].mean()
            loss.backward()
            return qq.grad
        ms = time_calls(step, stream, flush, 5, 1)
        res[name] = {"forward_backward_ms": ms, "grad_eps": float(eps.grad), "grad_sigma": float(sig.grad)}
    return res


def extra_md(lj, dev, stream):
    """Velocity Verlet on the N = 119,164 workload with random initial momenta
    (T ~ 1): one drift and one force call per step, the list rebuilt by the
    fastest-atom bookkeeping rule; reports steps/s and pairs/s including the
    rebuilds, with the FP64 and the double-float force.  The default driver
    queues steps through lj_md_steps (validity test on the device); the
    host-checked loop (one host read per step) is timed beside it, and so is
    the displacement criterion (rebuild when 2 max |q - q_build| reaches the
    margin) beside the paper's fastest-atom bound."""
    import torch
    from paper_1806_05713_gb300 import inputs
    from paper_1806_05713_gb300.md import VelocityVerlet
    s = inputs.workload_paper()
    g = np.random.default_rng(0).normal(size=(s.n, 4))
    g[:, 3] = 0.0
    g[:, :3] -= g[:, :3].mean(axis=0)
    res = {"n_atoms": s.n, "dt": 0.005}
    for name, prec, driver, crit in (
            ("fp64", lj.LJ_FP64, "device", "fastest_atom"),
            ("dfloat", lj.LJ_DFLOAT, "device", "fastest_atom"),
            ("fp64_host_driver", lj.LJ_FP64, "host", "fastest_atom"),
            ("dfloat_host_driver", lj.LJ_DFLOAT, "host", "fastest_atom"),
            ("fp64_displacement_criterion", lj.LJ_FP64, "device", "displacement"),
            ("dfloat_displacement_criterion", lj.LJ_DFLOAT, "device", "displacement")):
        q = torch.from_numpy(s.q).to(dev)
        p = torch.from_numpy(g).to(dev)
        vv = VelocityVerlet(q, p, s.box, s.rc, s.margin, 0.005, precision=prec, driver=driver,
                            criterion=crit)
        vv.run(20)
        e0 = vv.kinetic_energy() + vv.potential_energy()
        r0 = vv.rebuilds
        steps = 200
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        vv.run(steps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        e1 = vv.kinetic_energy() + vv.potential_energy()
        res[name] = {"steps": steps, "ms_per_step": ms / steps, "list_rebuilds": vv.rebuilds - r0,
                     "pairs_per_s": vv.plist.nnz * steps / (ms / 1e3),
                     "energy_drift_rel": abs(e1 - e0) / abs(e0)}
    return res


FORM_NAMES = {0: "fp64", 1: "mixed", 2: "dfloat"}


def forms(lj, q, pl, box, s, best_tpi, flops, dev, stream, flush):
    """The three arithmetic forms on the headline workload (half list, one
    force call, L2 flushed): time, pair interactions/s, FP64-equivalent
    TFLOP/s (the paper's 28 flops per in-cutoff pair), error vs the FP64
    kernel (itself within 1e-12 of the oracle in the tests); and each form
    again with the list layout (half or full) chosen by measurement, its
    pairs still counted as unique half-list entries."""
    import torch
    res, ref = {}, None
    for name, prec, tpis in (("fp64", lj.LJ_FP64, (best_tpi,)), ("mixed", lj.LJ_MIXED, (8, 16)),
                             ("dfloat", lj.LJ_DFLOAT, (136, 132))):
        best = None
        for t in tpis:
            pp = torch.zeros((s.n, 4), dtype=torch.float64, device=dev)
            fn = lj.lj_force_prepared(q, pp, pl, DT, s.rc, box, precision=prec, tpi=t)
            ms = time_calls(fn, stream, flush)
            if best is None or ms < best[0]:
                best = (ms, t, fn, pp)
        ms, t, fn, pp = best
        pp.zero_()
        fn()
        torch.cuda.synchronize()
        r = {"schedule": schedule_name(t), "ms_per_call": ms, "pairs_per_s": pl.nnz / (ms / 1e3),
             "fp64_equivalent_tflops": flops / (ms / 1e3) / 1e12}
        if ref is None:
            ref = pp[:, :3].clone()
        else:
            err = pp[:, :3] - ref
            r["max_err_rel_vs_fp64"] = float(err.abs().max() / ref.abs().max())
            r["rms_err_rel_vs_fp64"] = float(err.pow(2).mean().sqrt() / ref.pow(2).mean().sqrt())
            r["speedup_vs_fp64"] = res["fp64"]["ms_per_call"] / ms
        res[name] = r
    # each form with the list layout and schedule chosen by measurement
    # (lj_autotune_layout: half list with p_j atomics, or full list)
    for name, prec in (("fp64", lj.LJ_FP64), ("mixed", lj.LJ_MIXED), ("dfloat", lj.LJ_DFLOAT)):
        plb, t, _, _ = lj.lj_autotune_layout(q, box, s.rs, DT, s.rc, precision=prec, reps=3)
        pp = torch.zeros((s.n, 4), dtype=torch.float64, device=dev)
        ms = time_calls(lj.lj_force_prepared(q, pp, plb, DT, s.rc, box, precision=prec, tpi=t),
                        stream, flush)
        res[name]["best_layout"] = {"list": "half" if plb.half else "full",
                                    "schedule": schedule_name(t), "ms_per_call": ms,
                                    "pairs_per_s": pl.nnz / (ms / 1e3)}
        del plb, pp
    res["note"] = ("dfloat: pair arithmetic in double-float on the FP32 pipe, exact fixed-point "
                   "displacement; mixed: FP32 pair arithmetic; both add into FP64 momenta")
    return res


def time_calls(fn, stream, flush, calls=20, warm=3):
    import torch
    for _ in range(warm):
        fn()
    ms = []
    for _ in range(calls):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def variants(lj, s, q, pl_half, box, dev, stream, flush):
    """Force-only time per call of each schedule, list kind, precision and
    particle order (config 'paper size: two orderings, half and full'), with
    L2 flushed before each call, plus list-build times and mixed-form error."""
    import torch
    from paper_1806_05713_gb300 import inputs
    res = {}
    for order in ("random", "cell"):
        if order == "random":
            qq, sys_ = q, s
        else:
            sys_ = inputs.fcc_system(31, 1.0, 0.05, seed=0, order="cell", rc=RC, margin=MARGIN)
            qq = torch.from_numpy(sys_.q).to(dev)
        for half in (True, False):
            kind = "half" if half else "full"
            t_list = time_calls(lambda: lj.lj_build_pairlist(qq, box, sys_.rs, half), stream, flush, 5, 1)
            pl = lj.lj_build_pairlist(qq, box, sys_.rs, half)
            m_half = pl.nnz if half else pl.nnz // 2
            res[f"list_build_ms/{order}/{kind}"] = t_list
            ref = None
            for prec, tpis in ((lj.LJ_FP64, (1032, 1028, 1544, 1160, 2056, 2052, 2568, 4104, 4100, 4112)),
                               (lj.LJ_MIXED, (4, 8, 16)),
                               (lj.LJ_DFLOAT, (136, 132, 144, 648, 8))):
                for tpi in tpis:
                    pp = torch.zeros((sys_.n, 4), dtype=torch.float64, device=dev)
                    fn = lj.lj_force_prepared(qq, pp, pl, DT, sys_.rc, box, precision=prec, tpi=tpi)
                    ms = time_calls(fn, stream, flush)
                    name = f"{FORM_NAMES[prec]}/{order}/{kind}/tpi{tpi}"
                    res[name] = {"ms": ms, "pairs_per_s": m_half / (ms / 1e3)}
                    # error of one call vs the FP64 result (itself within 1e-12 of the oracle)
                    pp.zero_()
                    fn()
                    if prec == lj.LJ_FP64 and ref is None:
                        ref = pp[:, :3].clone()
                    elif prec != lj.LJ_FP64 and ref is not None:
                        err = pp[:, :3] - ref
                        res[name]["max_err_rel"] = float(err.abs().max() / ref.abs().max())
                        res[name]["rms_err_rel"] = float(err.pow(2).mean().sqrt() / ref.pow(2).mean().sqrt())
    # the paper's layout question on GB300: AoS4 vs AoS8 vs SoA, FP64, 8 lanes/row
    for half in (True, False):
        kind = "half" if half else "full"
        pl = lj.lj_build_pairlist(q, box, s.rs, half)
        m_half = pl.nnz if half else pl.nnz // 2
        n = s.n
        rec = torch.zeros((n, 8), dtype=torch.float64, device=dev)
        rec[:, :3] = q[:, :3]
        qs = q[:, :3].t().contiguous()
        ps = torch.zeros_like(qs)
        p4 = torch.zeros_like(q)
        for name, fn in (("aos4", lambda: lj.lj_force_strided(q, p4, n, 4, 1, pl, DT, s.rc, box)),
                         ("aos8", lambda: lj.lj_force_strided(rec, rec, n, 8, 1, pl, DT, s.rc, box,
                                                              p_offset=4)),
                         ("soa", lambda: lj.lj_force_strided(qs, ps, n, 1, n, pl, DT, s.rc, box))):
            ms = time_calls(fn, stream, flush)
            res[f"layout/fp64/random/{kind}/{name}"] = {"ms": ms, "pairs_per_s": m_half / (ms / 1e3)}
    return res


if __name__ == "__main__":
    main()
