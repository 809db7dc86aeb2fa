#!/usr/bin/env python3
"""LJ pair interactions/s on one GB300: FP64 vs mixed precision at stated error.

Headline workload (the precision configuration of this benchmark, the largest
single system): an FCC crystal of N = 1,048,576 = 4*64^3 atoms at density
1.0, cutoff 3.0 sigma, search length 3.3 sigma (bookkeeping margin 0.3),
jitter 0.05 sigma, particle order randomly permuted, half list (i < j),
dt = 0.01.  The FP64 kernel gives the headline value; the mixed and
double-float forms are timed beside it and every form's force error is
stated against the FP64 oracle.

One step = one pass of the hot path, the paper's protocol (section
"Benchmark Conditions": the force computed 100 times): build the sorted CSR
Verlet list on the GPU (cell binning, scan, walk, row sort), then run the
force 100 times on it.  A pair interaction is one unique half-list entry
processed in one force call, so each step credits 100 * nnz(half list).

Timing: inputs resident in HBM and larger than L2 (the list alone is
~300 MB); L2 also flushed (256 MiB write) before every step, outside the
timed events; each step timed with CUDA events on the launching stream; W
warm-up steps; the max over ranks of the summed step times.  `e2e` repeats
the step with positions and momenta copied from pinned host memory and the
momenta copied back inside the timed region.

The other configurations (the paper-size system in both orderings with
half and full lists, the 4,000-atom system, 512 uneven systems in one
persistent launch, the 64-replica adjoint) are reported in
`other_configs`, each with its error against the oracle.  The CPU oracle,
the plain double-precision C implementation the tests check against, is
timed on the host's cores as `cpu_baseline` (one core, the paper's setting,
and all cores).  `--impl reference` times the oracle alone on a bounded
sample of the headline workload (the comparison arm).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
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
DT, RC, MARGIN, RHO, JITTER = 0.01, 3.0, 0.3, 1.0, 0.05
HEADLINE_K = 64          # 64^3 FCC cells: N = 1,048,576
PAPER_K = 31             # 31^3 FCC cells: N = 119,164 (the paper's benchmark size)
L2_FLUSH_BYTES = 256 << 20
# The FP64 and FP32 ceilings derived from unit counts and the 2070 MHz clock
# (152 SMs x 2 FP64 FMA/clk, x 128 FP32 FMA/clk); the bench reports the
# measured ones (lj_measure_peak) and keeps these beside them.
FP64_PEAK_DERIVED = 152 * 4 * 2.07e9 / 1e12
FP32_PEAK_DERIVED = 152 * 256 * 2.07e9 / 1e12
# CPU samples of the headline workload (bounded so the default run stays in
# minutes): one core walks the middle block of rows of the half list; each
# of the P all-core workers a block of rows of the full list.
CPU_ROWS_ONE_CORE = 16384
CPU_ROWS_PER_WORKER = 1024
ORACLE_SAMPLE_ATOMS = 512
# ncu counters per launch of the dominant kernel (the FP64 force kernel),
# keyed by (schedule, list, atoms): DRAM bytes read + written, L2 read and
# reduction sectors, and the summary that records them.  A schedule or
# workload without an entry reports no traffic figure ("not profiled").
PROFILED = {
    (2056, "half", 119164): {"dram_bytes": 41910784.0 + 768.0, "lts_read_sectors": 10565312,
                             "lts_red_sectors": 24809860,
                             "source": "profiles/force_fp64_fixed_tpi8_half_N119164.md"},
    (10272, "half", 1048576): {"dram_bytes": 488836608.0 + 55444224.0,
                               "lts_read_sectors": 106171089, "lts_red_sectors": 199342661,
                               "source": "profiles/force_fp64_stream_r32_half_N1048576.md"},
}
ERROR_DEFINITION = ("max_err_rel = max |dp_gpu - dp_oracle| / max |dp_oracle|; rms_err_rel = "
                    "RMS(dp_gpu - dp_oracle) / RMS(dp_oracle), over the x, y, z components of "
                    "the atoms compared (dp = the momentum change of one call from p = 0)")


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--order", choices=["random", "cell"], default="random")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline legs")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other configurations (paper size, 4,000 atoms, batch, adjoint, MD)")
    ap.add_argument("--cpu-workers", type=int, default=0,
                    help="processes for the oracle (0 = every core this process may use)")
    ap.add_argument("--schedule", type=int, default=0,
                    help="FP64 schedule for the timed steps (0 = the library's autotuner picks)")
    ap.add_argument("--peaks", action="store_true",
                    help="only measure the FP64 / FP32 / packed-FP32 / L2-read ceilings and print them")
    ap.add_argument("--profile", choices=["fp64", "fp64-full", "mixed", "mixed-full", "dfloat",
                                          "dfloat-full", "list", "vjp", "vjp-half", "vjp-dfloat",
                                          "batched",
                                          "batched-mixed", "batched-dfloat"],
                    help="no timing: build the list and run a few calls of one kernel (for ncu)")
    ap.add_argument("--profile-atoms", choices=["paper", "million"], default="paper",
                    help="--profile workload: N = 119,164 (paper) or N = 1,048,576 (million)")
    ap.add_argument("--profile-tpi", type=int, default=0, help="schedule for --profile (0 = auto)")
    return ap.parse_args()


def cpu_count() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json, STREAM-style copy)"
    except Exception:
        return 6800.0, "fallback (profiling recipe)"


# ---------------------------------------------------------------------------
# Workloads (regenerated from their seeds in every process that needs them)
# ---------------------------------------------------------------------------

_SYSTEMS: dict = {}


def system_from_spec(spec):
    """("fcc", k, rho, jitter, seed, order) | ("batch", nsys, seed, index) |
    ("replica", replicas, k, seed, index) -> LJSystem (cached per process)."""
    if spec in _SYSTEMS:
        return _SYSTEMS[spec]
    from paper_1806_05713_gb300 import inputs
    kind = spec[0]
    if kind == "fcc":
        _, k, rho, jit, seed, order = spec
        s = inputs.fcc_system(k, rho, jit, seed=seed, order=order, rc=RC, margin=MARGIN)
    elif kind == "batch":
        _, nsys, seed, idx = spec
        key = ("batch-all", nsys, seed)
        if key not in _SYSTEMS:
            _SYSTEMS[key] = inputs.batched_systems(nsys=nsys, seed=seed)
        s = _SYSTEMS[key][idx]
    elif kind == "replica":
        _, reps, k, seed, idx = spec
        key = ("replica-all", reps, k, seed)
        if key not in _SYSTEMS:
            _SYSTEMS[key] = inputs.workload_replicas(reps, k, seed=seed)
        s = _SYSTEMS[key][idx]
    else:
        raise ValueError(spec)
    _SYSTEMS[spec] = s
    return s


def headline_spec(seed: int, order: str):
    return ("fcc", HEADLINE_K, RHO, JITTER, seed, order)


def headline_config(n_atoms: int, order: str) -> dict:
    """The workload as both arms state it (same dict in both lines)."""
    return {"workload": f"fcc-64^3 N={n_atoms} rho=1.0 rc=3.0 rs=3.3 jitter=0.05 {order}-order "
                        f"half-list dt=0.01",
            "n_atoms": n_atoms, "list": "half (i < j), CSR int32, rows sorted",
            "force_calls_per_step": FORCE_CALLS, "list_builds_per_step": 1,
            "l2": "inputs larger than the 129 MB L2 (list ~300 MB, q and p 33.5 MB each)"}


# ---------------------------------------------------------------------------
# CPU oracle: tasks for a process pool, and a team of timing processes
# ---------------------------------------------------------------------------

def _oracle_task(task):
    """One oracle computation in a pool worker (spawned; loads no GPU code)."""
    import oracle
    kind = task[0]
    if kind == "atoms":       # per-atom momentum change from the definition
        _, spec, idx = task
        s = system_from_spec(spec)
        return oracle.force_atoms(s.q, idx, DT, s.rc, s.box)
    if kind == "force":       # whole-system momentum change over the oracle's own list
        _, spec = task
        s = system_from_spec(spec)
        rp, col = oracle.pairlist(s.q, s.box, s.rs, True)
        return oracle.force(s.q, np.zeros((s.n, 3)), rp, col, True, DT, s.rc, s.box)
    if kind == "grad":        # one replica's share of the force-matching gradient
        _, spec, eps, sig, inv_count = task
        s = system_from_spec(spec)
        rp, col = oracle.pairlist(s.q, s.box, s.rs, False)
        Ft = oracle.forces(s.q, rp, col, False, s.rc, s.box, 1.0, 1.0)
        F = oracle.forces(s.q, rp, col, False, s.rc, s.box, eps, sig)
        R = 2.0 * (F - Ft) * inv_count
        gq, ge, gs = oracle.force_vjp(s.q, R, rp, col, False, s.rc, s.box, eps, sig)
        return gq, ge, gs, float(np.sum((F - Ft) ** 2) * inv_count)
    raise ValueError(kind)


class OraclePool:
    """A spawned process pool for the oracle (spawn: safe next to a CUDA
    context, and the workers import no GPU code)."""

    def __init__(self, workers: int):
        import oracle
        oracle.build()                      # compile once, before the workers load it
        self.workers = workers
        self.pool = mp.get_context("spawn").Pool(workers)

    def submit(self, tasks):
        return self.pool.map_async(_oracle_task, tasks, chunksize=1)

    def close(self):
        self.pool.close()
        self.pool.join()


def _team_worker(w, nworkers, spec, cmd_q, res_q, barrier):
    import oracle
    s = system_from_spec(spec)
    oracle.force_rows(s.q, np.zeros((s.n, 3)), np.zeros(1, dtype=np.int32), np.zeros(0, np.int32),
                      False, DT, s.rc, s.box, 0, 0)           # load the library before timing
    while True:
        msg = cmd_q.get()
        if msg[0] == "stop":
            return
        _, i0, i1, half, calls = msg
        a = i0 + (i1 - i0) * w // nworkers
        b = i0 + (i1 - i0) * (w + 1) // nworkers
        p = np.zeros((s.n, 3))
        barrier.wait()
        t0 = time.monotonic()
        rp, col = oracle.pairlist_rows(s.q, s.box, s.rs, half, a, b)
        for _ in range(calls):
            oracle.force_rows(s.q, p, rp, col, half, DT, s.rc, s.box, a, b, inplace=True)
        t1 = time.monotonic()
        res_q.put((w, t0, t1, int(col.size)))


class CpuTeam:
    """P spawned processes that each time the oracle on their block of rows,
    released together by a barrier: the all-cores leg of the CPU baseline.
    Each worker builds its rows of the list and runs the force calls over
    them (full list: a row updates only its own atom, so the workers share
    nothing and need no reduction)."""

    def __init__(self, workers: int, spec):
        ctx = mp.get_context("spawn")
        import oracle
        oracle.build()
        self.workers = workers
        self.cmd = [ctx.Queue() for _ in range(workers)]
        self.res = ctx.Queue()
        self.barrier = ctx.Barrier(workers + 1)
        self.procs = [ctx.Process(target=_team_worker,
                                  args=(w, workers, spec, self.cmd[w], self.res, self.barrier),
                                  daemon=True) for w in range(workers)]
        for p in self.procs:
            p.start()

    def step(self, i0: int, i1: int, half: bool, calls: int):
        """One timed step; returns (wall seconds, list entries walked)."""
        for q in self.cmd:
            q.put(("step", i0, i1, half, calls))
        self.barrier.wait(timeout=900)
        t0 = time.monotonic()
        res = [self.res.get(timeout=900) for _ in range(self.workers)]
        return max(r[2] for r in res) - t0, sum(r[3] for r in res)

    def close(self):
        for q in self.cmd:
            q.put(("stop",))
        for p in self.procs:
            p.join(timeout=60)


def cpu_one_core_leg(s, calls: int = FORCE_CALLS):
    """One step of the paper's setting on one core: the oracle builds the
    middle CPU_ROWS_ONE_CORE rows of the half list and runs `calls` force
    calls over them.  Returns (pairs/s, seconds, entries, description)."""
    import oracle
    oracle.build()
    i0 = s.n // 2 - CPU_ROWS_ONE_CORE // 2
    i1 = i0 + CPU_ROWS_ONE_CORE
    p = np.zeros((s.n, 3))
    t0 = time.monotonic()
    rp, col = oracle.pairlist_rows(s.q, s.box, s.rs, True, i0, i1)
    for _ in range(calls):
        oracle.force_rows(s.q, p, rp, col, True, DT, s.rc, s.box, i0, i1, inplace=True)
    t = time.monotonic() - t0
    desc = (f"1 core: oracle list rows {i0}..{i1 - 1} of the half list ({col.size} entries) "
            f"built, then {calls} oracle force calls over them ({t:.1f} s)")
    return calls * col.size / t, t, int(col.size), desc


def cpu_all_cores_leg(team: CpuTeam, n: int, calls: int = FORCE_CALLS):
    """One step on every core: P workers, each the oracle over its own block
    of CPU_ROWS_PER_WORKER rows of the full list (list rows built, then
    `calls` force calls).  A full-list entry is half a pair interaction, as
    for the GPU's full-list kernels.  Returns (pairs/s, seconds, entries,
    description)."""
    rows = CPU_ROWS_PER_WORKER * team.workers
    i0 = n // 2 - rows // 2
    t, entries = team.step(i0, i0 + rows, False, calls)
    desc = (f"{team.workers} processes (one per core): oracle list rows {i0}..{i0 + rows - 1} of "
            f"the full list ({entries} entries = {entries // 2} pair interactions) built, then "
            f"{calls} oracle force calls, each process over its {CPU_ROWS_PER_WORKER} rows "
            f"({t:.2f} s wall)")
    return calls * (entries / 2.0) / t, t, entries, desc


# ---------------------------------------------------------------------------
# Device-side helpers
# ---------------------------------------------------------------------------

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


def time_calls(fn, stream, flush, calls=20, warm=3):
    """Median device time (ms) of fn over `calls` launches, L2 flushed before
    each, CUDA events on the launching stream."""
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


def count_in_cutoff(q, pl, box, rc, chunk: int = 1 << 24):
    """List entries with r < r_c (for the flop count), by the definition:
    d = q_j - q_i, per axis the branchy minimum image (d > L/2: d - L;
    d < -L/2: d + L), r^2 = (dx*dx + dy*dy) + dz*dz in separately rounded
    double operations; torch elementwise ops at set-up time, not timed."""
    import torch
    rp = pl.row_ptr.long()
    rows = torch.repeat_interleave(torch.arange(pl.n, device=q.device), rp[1:] - rp[:-1])
    col = pl.col_view.long()
    rc2 = float(rc) * float(rc)
    total = 0
    for k0 in range(0, col.numel(), chunk):
        i, j = rows[k0:k0 + chunk], col[k0:k0 + chunk]
        sq = []
        for a in range(3):
            L = float(box[a])
            d = q[j, a] - q[i, a]
            d = torch.where(d > 0.5 * L, d - L, torch.where(d < -0.5 * L, d + L, d))
            sq.append(d * d)
        r2 = (sq[0] + sq[1]) + sq[2]
        total += int((r2 < rc2).sum().item())
    return total


def err_stats(got: np.ndarray, want: np.ndarray) -> dict:
    d = got - want
    return {"max_err_rel_vs_oracle": float(np.max(np.abs(d)) / np.max(np.abs(want))),
            "rms_err_rel_vs_oracle": float(np.sqrt(np.mean(d ** 2)) / np.sqrt(np.mean(want ** 2)))}


def schedule_name(tpi: int) -> str:
    t = tpi & 63
    name = f"{max(t, 1)} lanes/row"
    if tpi & 128:
        name += ", 2 entries/lane (software-pipelined)"
    if tpi & 512:
        name += ", rows by length"
    if tpi & 16384:
        name += ", rows in cell order"
    if tpi & 1024:
        name += ", image-selected displacement"
    if tpi & 2048:
        name += ", exact fixed-point displacement"
    if tpi & 8192:
        name = f"{max(t, 1)} rows/warp, their entries in one chunk per lane, exact fixed-point displacement"
    return name


FORMS = (("fp64", 0), ("mixed", 1), ("dfloat", 2))
FORM_CANDIDATES = {1: (4, 8, 16, 132, 136, 144), 2: (132, 136, 144)}


def best_form_call(lj, q, pl, box, rc, prec, tpis, stream, flush, dev, calls=10):
    """Fastest schedule of one form on one list: (ms, tpi, dp of one call
    from zero on the GPU)."""
    import torch
    best = None
    for t in tpis:
        pp = torch.zeros((pl.n, 4), dtype=torch.float64, device=dev)
        fn = lj.lj_force_prepared(q, pp, pl, DT, rc, box, precision=prec, tpi=t)
        ms = time_calls(fn, stream, flush, calls, 2)
        if best is None or ms < best[0]:
            best = (ms, t, fn, pp)
    ms, t, fn, pp = best
    pp.zero_()
    fn()
    torch.cuda.synchronize()
    return ms, t, pp


# ---------------------------------------------------------------------------
# Reference arm: the oracle alone
# ---------------------------------------------------------------------------

def run_reference(args, world, rank):
    if rank != 0:
        return
    spec = headline_spec(0, args.order)
    s = system_from_spec(spec)
    workers = args.cpu_workers or cpu_count()
    team = CpuTeam(workers, spec)
    try:
        for _ in range(max(0, args.warmup)):
            cpu_all_cores_leg(team, s.n)
        times, pairs, desc = [], [], ""
        for _ in range(args.steps):
            r, t, _, desc = cpu_all_cores_leg(team, s.n)
            times.append(t)
            pairs.append(r * t)
    finally:
        team.close()
    one_rate, _, _, one_desc = cpu_one_core_leg(s)
    value = sum(pairs) / sum(times)
    sample = ("each step: " + desc + "; the same FP64 oracle the tests compare against, "
              "unchanged, in spawned processes")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "ms_per_step_median": 1e3 * statistics.median(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": headline_config(s.n, args.order),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": sample,
                         "single_core": {"value": one_rate, "cores": 1, "sample": one_desc}},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---------------------------------------------------------------------------
# Clocks and ranks
# ---------------------------------------------------------------------------

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


# ---------------------------------------------------------------------------
# Profiling and peak modes
# ---------------------------------------------------------------------------

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
    res["derived_fp64_tflops"] = FP64_PEAK_DERIVED
    res["derived_fp32_tflops"] = FP32_PEAK_DERIVED
    print(json.dumps(res))


def run_profile(args):
    """A short, fixed launch sequence for a profiler: 2 list builds, then
    5 calls of the chosen force kernel (or 3 more list builds)."""
    import torch
    from paper_1806_05713_gb300 import build as lib_build
    from paper_1806_05713_gb300 import inputs, lj
    lib_build.build()
    k = PAPER_K if args.profile_atoms == "paper" else HEADLINE_K
    s = inputs.fcc_system(k, RHO, JITTER, seed=0, order=args.order, rc=RC, margin=MARGIN)
    box = [float(x) for x in s.box]
    q = torch.from_numpy(s.q).cuda()
    p = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
    half = not args.profile.endswith("full")
    if args.profile.startswith("batched"):
        from paper_1806_05713_gb300.batch import Batch
        systems = inputs.batched_systems(nsys=64, seed=0)
        prec = {"batched": lj.LJ_FP64, "batched-mixed": lj.LJ_MIXED,
                "batched-dfloat": lj.LJ_DFLOAT}[args.profile]
        tpi = args.profile_tpi or (8 if prec == lj.LJ_FP64 else 4)
        b = Batch(systems, DT, prec, True, tpi=tpi,
                  rows_per_item=64 if tpi == lj.LJ_SCHED_STREAM else 16)
        for _ in range(5):
            b.force()
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "systems": len(systems), "atoms": b.total_atoms}))
        return
    if args.profile.startswith("vjp"):
        half = args.profile == "vjp-half"
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
        fn = lj.lj_force_prepared(q, p, pl, DT, s.rc, box, precision=prec, tpi=args.profile_tpi)
        for _ in range(5):
            fn()
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "n": s.n, "nnz": pl.nnz,
                      "launches": int(lj.load().lj_kernel_launch_count())}))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

BATCH_SAMPLE = tuple(range(0, 512, 32))   # 16 of the 512 systems checked against the oracle
ADJ_REPLICAS, ADJ_K, ADJ_EPS, ADJ_SIGMA = 64, 16, 1.1, 0.97


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

    spec = headline_spec(rank, args.order)
    s = system_from_spec(spec)
    box = [float(x) for x in s.box]
    q = torch.from_numpy(s.q).to(dev)
    p = torch.zeros((s.n, 4), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    pl = lj.lj_build_pairlist(q, box, s.rs, True)
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
        for _ in range(FORCE_CALLS):
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

    workers = args.cpu_workers or cpu_count()
    pool = OraclePool(workers)
    sample = np.sort(np.random.default_rng(7).choice(s.n, ORACLE_SAMPLE_ATOMS, replace=False))
    chunks = np.array_split(sample, workers)
    jobs = {"headline_atoms": pool.submit([("atoms", spec, c) for c in chunks if c.size])}
    if not args.no_extra:
        jobs["paper"] = pool.submit([("force", ("fcc", PAPER_K, RHO, JITTER, 0, o))
                                     for o in ("random", "cell")])
        jobs["small"] = pool.submit([("force", ("fcc", 10, RHO, JITTER, 0, "random"))])
        jobs["batch"] = pool.submit([("force", ("batch", 512, 0, int(k))) for k in BATCH_SAMPLE])
        inv = 1.0 / (3.0 * ADJ_REPLICAS * 4 * ADJ_K ** 3)
        jobs["adjoint"] = pool.submit([("grad", ("replica", ADJ_REPLICAS, ADJ_K, 0, r), ADJ_EPS,
                                        ADJ_SIGMA, inv) for r in range(ADJ_REPLICAS)])

    # ---- ceilings and the roofline of the dominant kernel ------------------
    ceil = measure_ceilings(lj, dev)
    hbm_peak, hbm_src = measured_hbm()
    t_force = statistics.mean(force_ms) / 1e3
    flops = 28.0 * n_cut + 8.0 * (nnz - n_cut)     # paper: 27 add/mul + 1 div per pair
    alg_bytes = 4.0 * nnz + 4.0 * (s.n + 1) + 32.0 * s.n + 64.0 * s.n
    achieved = flops / t_force / 1e12
    prof = PROFILED.get((best_tpi, "half", s.n))
    roof = {"bound": "alu", "achieved": achieved, "peak": ceil["fp64_fma_tflops"],
            "unit": "TFLOP/s", "frac": achieved / ceil["fp64_fma_tflops"],
            "traffic": None if prof is None else prof["dram_bytes"],
            "traffic_note": ("not profiled: no ncu capture of this schedule on this workload"
                             if prof is None else
                             prof["source"] + " (ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                                              "one launch, cold cache)"),
            "kernel": f"FP64 force kernel, {schedule_name(best_tpi)}, half list",
            "peak_source": ("measured live: lj_measure_peak DFMA probe (of measured; method and "
                            "clocks in profiles/pipe_peaks_gb300.md)"),
            "peak_derived": FP64_PEAK_DERIVED,
            "frac_of_derived": achieved / FP64_PEAK_DERIVED,
            "flops_per_launch": flops, "launch_ms": t_force * 1e3,
            "flops_basis": "28 per in-cutoff entry (27 add/mul + 1 div), 8 per margin entry"}
    hbm_view = {"achieved": alg_bytes / t_force / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": alg_bytes / t_force / 1e9 / hbm_peak, "peak_source": hbm_src,
                "bytes_per_pair": alg_bytes / nnz}
    gathered_reads = 36.0 * nnz + 40.0 * s.n
    # p_i partial sums: one per lane and row for a grid over rows (t lanes);
    # for r rows per warp in 32 per-lane chunks, one per row plus one per
    # chunk boundary (32 per r rows)
    t_lanes = best_tpi & 63
    flushes = (s.n + 32.0 * s.n / t_lanes) if best_tpi & 8192 else float(t_lanes * s.n)
    reductions = 3.0 * n_cut + 3.0 * flushes
    l2_view = {"gathered_read_bytes": gathered_reads, "reductions": reductions,
               "gathered_read_GBps": gathered_reads / t_force / 1e9,
               "gathered_read_frac_of_l2_read_peak": gathered_reads / t_force / 1e9 / ceil["l2_read_gbs"],
               "reductions_per_s": reductions / t_force,
               "lts_read_sectors": None if prof is None else prof["lts_read_sectors"],
               "lts_red_sectors": None if prof is None else prof["lts_red_sectors"]}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "ms_per_step_median": statistics.median(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(s.n, args.order),
        "l2_flush": "256 MiB write before every step, outside the timed events",
        "parallelism": f"replicas x{world}",
        "schedule": schedule_name(best_tpi), "pairs_per_call": nnz, "pairs_in_cutoff": n_cut,
        "list_build_ms": statistics.mean(list_ms),
        "force_ms_per_call": t_force * 1e3,
        "force_only_pairs_per_s": nnz / t_force,
        "roofline": roof, "hbm_roofline": hbm_view, "l2_gather_view": l2_view,
        "ceilings_measured": ceil,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 32 * s.n,
                "d2h_bytes_per_step": 32 * s.n},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "error_definition": ERROR_DEFINITION,
        "autotune_ms": {schedule_name(k): v for k, v in tune_table.items()},
    }

    # ---- the three forms on the headline workload, errors vs the oracle ----
    want_atoms = np.concatenate(jobs["headline_atoms"].get(timeout=1800))
    out["forms"] = headline_forms(lj, q, pl, box, s, best_tpi, flops, dev, stream, flush, sample,
                                  want_atoms, ceil)
    del p, force
    if not args.no_extra:
        oc = {}
        oc["paper_119164"] = extra_paper(lj, dev, stream, flush, jobs["paper"].get(timeout=1800))
        oc["small_4000"] = extra_small(lj, dev, stream, flush, jobs["small"].get(timeout=1800)[0])
        oc["batched_512_systems"] = extra_batched(lj, dev, stream, flush,
                                                  jobs["batch"].get(timeout=1800))
        oc["adjoint_64_replicas"] = extra_adjoint(lj, dev, stream, flush,
                                                  jobs["adjoint"].get(timeout=3600))
        oc["md_velocity_verlet"] = extra_md(lj, dev, stream)
        out["other_configs"] = oc
    pool.close()

    if world == 1 and not args.no_cpu:
        one_rate, _, _, one_desc = cpu_one_core_leg(s)
        team = CpuTeam(workers, spec)
        try:
            cpu_all_cores_leg(team, s.n)               # warm-up step
            all_rate, _, _, all_desc = cpu_all_cores_leg(team, s.n)
        finally:
            team.close()
        out["cpu_baseline"] = {
            "value": all_rate, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": all_desc + "; a bounded sample of the headline workload",
            "single_core": {"value": one_rate, "unit": UNIT, "cores": 1, "sample": one_desc}}
    print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def headline_forms(lj, q, pl, box, s, best_tpi, flops, dev, stream, flush, sample, want, ceil):
    """FP64, mixed and double-float on the headline workload: time per call
    (L2 flushed), pair interactions/s, and each form's error against the
    oracle on the sampled atoms (the oracle's per-atom sums over all atoms);
    then each form on the list layout chosen by measurement (half list with
    p_j atomics or full list without), its pairs still counted as unique
    half-list entries."""
    import torch
    idx = torch.from_numpy(sample).to(dev)
    res, fp64_ms = {}, None
    for name, prec in FORMS:
        tpis = (best_tpi,) if prec == 0 else FORM_CANDIDATES[prec]
        ms, t, pp = best_form_call(lj, q, pl, box, s.rc, prec, tpis, stream, flush, dev)
        got = pp[idx, :3].cpu().numpy()
        r = {"schedule": schedule_name(t), "list": "half", "ms_per_call": ms,
             "pairs_per_s": pl.nnz / (ms / 1e3),
             "fp64_equivalent_tflops": flops / (ms / 1e3) / 1e12,
             "oracle_atoms": int(sample.size), **err_stats(got, want)}
        if prec == 0:
            fp64_ms = ms
        else:
            r["speedup_vs_fp64"] = fp64_ms / ms
        res[name] = r
        del pp
    for name, prec in FORMS:
        plb, t, _, _ = lj.lj_autotune_layout(q, box, s.rs, DT, s.rc, precision=prec, reps=3)
        ms, t, pp = best_form_call(lj, q, plb, box, s.rc, prec, (t,), stream, flush, dev)
        got = pp[idx, :3].cpu().numpy()
        res[name]["best_layout"] = {"list": "half" if plb.half else "full",
                                    "schedule": schedule_name(t), "ms_per_call": ms,
                                    "pairs_per_s": pl.nnz / (ms / 1e3), **err_stats(got, want)}
        del plb, pp
    res["note"] = ("fp64: IEEE double; mixed: FP32 pair arithmetic, FP64/compensated sums; "
                   "dfloat: double-float pair arithmetic on the FP32 pipe, exact fixed-point "
                   "displacement; all add into FP64 momenta.  Errors against the oracle on "
                   f"{sample.size} sampled atoms (seeded choice); ceilings: FP32 FMA "
                   f"{ceil['fp32_fma_tflops']:.1f} TFLOP/s, packed {ceil['fp32x2_fma_tflops']:.1f}, "
                   f"L2 read {ceil['l2_read_gbs']:.0f} GB/s (measured)")
    return res


# ---------------------------------------------------------------------------
# Other configurations
# ---------------------------------------------------------------------------

def extra_paper(lj, dev, stream, flush, oracle_dp):
    """N = 119,164 (31^3 FCC, the paper's benchmark size): random and
    cell-sorted particle order, half and full lists, list-build time, every
    form's fastest schedule with its error against the oracle (whole
    system); the FP64 schedules timed one by one; and the paper's layout
    question (AoS4 / AoS8 / SoA)."""
    import torch
    res = {"n_atoms": 4 * PAPER_K ** 3, "schedules_fp64_ms": {}}
    for order, want in zip(("random", "cell"), oracle_dp):
        s = system_from_spec(("fcc", PAPER_K, RHO, JITTER, 0, order))
        box = [float(x) for x in s.box]
        q = torch.from_numpy(s.q).to(dev)
        for half in (True, False):
            kind = "half" if half else "full"
            t_list = time_calls(lambda: lj.lj_build_pairlist(q, box, s.rs, half), stream, flush, 5, 1)
            pl = lj.lj_build_pairlist(q, box, s.rs, half)
            m_half = pl.nnz if half else pl.nnz // 2
            entry = {"list_build_ms": t_list, "pairs_per_call": m_half}
            for name, prec in FORMS:
                tpis = (10272, 10256, 10248, 2056, 2052, 2064, 2568, 1032) if prec == 0 else FORM_CANDIDATES[prec]
                if prec == 0:
                    for t in tpis:
                        pp = torch.zeros((s.n, 4), dtype=torch.float64, device=dev)
                        fn = lj.lj_force_prepared(q, pp, pl, DT, s.rc, box, precision=0, tpi=t)
                        res["schedules_fp64_ms"][f"{order}/{kind}/{schedule_name(t)}"] = \
                            time_calls(fn, stream, flush, 10, 2)
                        del pp
                ms, t, pp = best_form_call(lj, q, pl, box, s.rc, prec, tpis, stream, flush, dev)
                entry[name] = {"schedule": schedule_name(t), "ms_per_call": ms,
                               "pairs_per_s": m_half / (ms / 1e3),
                               **err_stats(pp[:, :3].cpu().numpy(), want)}
                del pp
            res[f"{order}/{kind}"] = entry
            del pl
    # the paper's layout question on GB300: AoS4 vs AoS8 vs SoA, FP64
    s = system_from_spec(("fcc", PAPER_K, RHO, JITTER, 0, "random"))
    box = [float(x) for x in s.box]
    q = torch.from_numpy(s.q).to(dev)
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


def extra_small(lj, dev, stream, flush, want):
    """N = 4,000 (10^3 FCC): the parity configuration -- every form's error
    against the oracle, and its time per call."""
    import torch
    s = system_from_spec(("fcc", 10, RHO, JITTER, 0, "random"))
    box = [float(x) for x in s.box]
    q = torch.from_numpy(s.q).to(dev)
    pl = lj.lj_build_pairlist(q, box, s.rs, True)
    res = {"n_atoms": s.n, "pairs_per_call": pl.nnz}
    for name, prec in FORMS:
        tpis = (2056, 2052) if prec == 0 else FORM_CANDIDATES[prec]
        ms, t, pp = best_form_call(lj, q, pl, box, s.rc, prec, tpis, stream, flush, dev)
        res[name] = {"schedule": schedule_name(t), "ms_per_call": ms,
                     **err_stats(pp[:, :3].cpu().numpy(), want)}
    return res


def extra_batched(lj, dev, stream, flush, oracle_dp):
    """512 systems, N log-uniform in 500..32000, rho in 0.8..1.2, rc 2.5 or
    3.0: one persistent launch replayed from a CUDA graph, against (a) one
    lj_force call per system issued from the host and (b) the same per-system
    calls replayed from one CUDA graph (no host work between launches, so
    (b) against the persistent launch is the GPU-side difference and (a)
    against (b) the host's).  FP64, mixed and double-float; the autotuner
    picks lanes per row, rows per work item and the list layout.  Errors
    against the oracle on 16 sampled systems."""
    import torch
    from paper_1806_05713_gb300.batch import Batch
    systems = [system_from_spec(("batch", 512, 0, k)) for k in range(512)]
    res = {"n_systems": len(systems), "total_atoms": int(sum(x.n for x in systems)),
           "oracle_systems": list(BATCH_SAMPLE)}
    for name, prec in FORMS:
        b = Batch(systems, DT, prec, True, tpi=8, rows_per_item=64, plan_rows_min=16)
        tpis = (4, 8, 16, lj.LJ_SCHED_STREAM) if prec == lj.LJ_FP64 else (4, 8, 16)
        tpi, rows, _ = b.autotune(tpis=tpis, rows=(16, 32, 64, 128), reps=3,
                                  layouts=(True, False))
        g = b.capture_graph()
        t_graph = time_calls(g.replay, stream, flush, 10, 2)
        t_host = time_calls(lambda: b.force_per_system(tpi=lj.LJ_TPI_AUTO), stream, flush, 5, 1)
        g_sep = b.capture_per_system_graph(tpi=lj.LJ_TPI_AUTO)
        t_sep_graph = time_calls(g_sep.replay, stream, flush, 10, 2)
        b.p4.zero_()
        b.force()
        torch.cuda.synchronize()
        out_p = b.p4.cpu().numpy()
        errs = [err_stats(out_p[int(b.atom_offset[k]):int(b.atom_offset[k]) + systems[k].n, :3], w)
                for k, w in zip(BATCH_SAMPLE, oracle_dp)]
        res[name] = {"tpi": "stream" if tpi == lj.LJ_SCHED_STREAM else tpi,
                     "rows_per_item": rows, "list": "half" if b.half else "full",
                     "pairs_per_call": b.pairs,
                     "graph_persistent_ms": t_graph,
                     "graph_persistent_pairs_per_s": b.pairs / (t_graph / 1e3),
                     "per_system_graph_ms": t_sep_graph,
                     "per_system_host_launches_ms": t_host,
                     "speedup_persistent_vs_per_system_graph": t_sep_graph / t_graph,
                     "speedup_per_system_graph_vs_host_launches": t_host / t_sep_graph,
                     "max_err_rel_vs_oracle": max(e["max_err_rel_vs_oracle"] for e in errs),
                     "rms_err_rel_vs_oracle": max(e["rms_err_rel_vs_oracle"] for e in errs),
                     "error_note": "worst of the sampled systems, each relative to its own scale"}
        del b, g, g_sep
    return res


def extra_adjoint(lj, dev, stream, flush, oracle_parts):
    """64 replicas of N = 16,384 (16^3 FCC, rho 1, jitter 0.1): forces with
    (eps, sigma) = (1.1, 0.97) against targets at (1, 1), loss = mean squared
    force error over all replicas, atoms and components; gradient w.r.t.
    positions, eps and sigma through the autograd wrapper (forward kernel +
    hand-written adjoint kernel).  Each form's gradient against the oracle's
    (its adjoint summed over replicas), and the FP64 adjoint against central
    differences (h = 1e-6) of the FP64 loss for eps, sigma and four
    coordinates."""
    import torch
    from paper_1806_05713_gb300.autograd import lj_forces
    reps = [system_from_spec(("replica", ADJ_REPLICAS, ADJ_K, 0, r)) for r in range(ADJ_REPLICAS)]
    L = float(reps[0].box[0])
    box = [L, L, L]
    n1 = reps[0].n
    q = torch.from_numpy(np.concatenate([r.q for r in reps])).to(dev)

    def block_list(half):  # block-diagonal list over replicas sharing one box size
        rows, cols, off = [torch.zeros(1, dtype=torch.int32, device=dev)], [], 0
        for k, r in enumerate(reps):
            pl = lj.lj_build_pairlist(q[k * n1:(k + 1) * n1].contiguous(), box, r.rs, half)
            rows.append(pl.row_ptr[1:] + off)
            cols.append(pl.col_view + k * n1)
            off += pl.nnz
        return lj.PairList(torch.cat(rows).contiguous(), torch.cat(cols).contiguous(), q.shape[0],
                           off, half, reps[0].rs, 0)
    lists = {"full": block_list(False), "half": block_list(True)}
    big = lists["full"]
    off = big.nnz
    Ft = torch.zeros_like(q)
    lj.lj_force(q, Ft, big, 1.0, reps[0].rc, box, 1.0, 1.0)
    want_q = np.concatenate([o[0] for o in oracle_parts])
    want_e = float(sum(o[1] for o in oracle_parts))
    want_s = float(sum(o[2] for o in oracle_parts))
    want_loss = float(sum(o[3] for o in oracle_parts))
    res = {"replicas": len(reps), "atoms": int(q.shape[0]), "pairs": off // 2,
           "oracle_loss": want_loss, "oracle_grad_eps": want_e, "oracle_grad_sigma": want_s}

    def loss_of(qq, e, sg, prec, plist=big):
        F = lj_forces(qq, e, sg, plist, reps[0].rc, box, prec)
        return ((F - Ft) ** 2)[:, :3].mean()

    for name, prec in FORMS:
        eps = torch.tensor(ADJ_EPS, dtype=torch.float64, device=dev, requires_grad=True)
        sig = torch.tensor(ADJ_SIGMA, dtype=torch.float64, device=dev, requires_grad=True)
        last = {}

        def step(plist):
            qq = q.detach().requires_grad_(True)
            eps.grad = None
            sig.grad = None
            loss = loss_of(qq, eps, sig, prec, plist)
            loss.backward()
            last["q"], last["loss"] = qq.grad, loss
            return qq.grad
        # half list (atomics) or full list (gathers), chosen by measurement
        layout_ms = {k: time_calls(lambda: step(pl), stream, flush, 5, 1) for k, pl in lists.items()}
        layout = min(layout_ms, key=layout_ms.get)
        ms = layout_ms[layout]
        step(lists[layout])
        gq = last["q"][:, :3].cpu().numpy()
        d = gq - want_q
        res[name] = {"forward_backward_ms": ms, "list": layout,
                     "forward_backward_ms_by_list": layout_ms,
                     "loss": float(last["loss"].detach()),
                     "grad_eps": float(eps.grad), "grad_sigma": float(sig.grad),
                     "grad_eps_rel_err_vs_oracle": abs(float(eps.grad) - want_e) / abs(want_e),
                     "grad_sigma_rel_err_vs_oracle": abs(float(sig.grad) - want_s) / abs(want_s),
                     "grad_q_max_err_rel_vs_oracle": float(np.max(np.abs(d)) / np.max(np.abs(want_q))),
                     "grad_q_rms_err_rel_vs_oracle": float(np.sqrt(np.mean(d ** 2)) /
                                                           np.sqrt(np.mean(want_q ** 2)))}
    # central differences of the FP64 loss
    h = 1e-6
    coords = [(0, 0), (12345, 1), (n1 * 7 + 3, 2), (q.shape[0] - 1, 0)]
    with torch.no_grad():
        def loss64(qq=q, e=ADJ_EPS, sg=ADJ_SIGMA):
            te = torch.tensor(e, dtype=torch.float64, device=dev)
            ts = torch.tensor(sg, dtype=torch.float64, device=dev)
            return float(loss_of(qq, te, ts, 0))
        fd = {"eps": (loss64(e=ADJ_EPS + h) - loss64(e=ADJ_EPS - h)) / (2 * h),
              "sigma": (loss64(sg=ADJ_SIGMA + h) - loss64(sg=ADJ_SIGMA - h)) / (2 * h)}
        for (i, a) in coords:
            qp, qm = q.clone(), q.clone()
            qp[i, a] += h
            qm[i, a] -= h
            fd[f"q[{i},{a}]"] = (loss64(qq=qp) - loss64(qq=qm)) / (2 * h)
    adj = {"eps": res["fp64"]["grad_eps"], "sigma": res["fp64"]["grad_sigma"]}
    eps = torch.tensor(ADJ_EPS, dtype=torch.float64, device=dev, requires_grad=True)
    sig = torch.tensor(ADJ_SIGMA, dtype=torch.float64, device=dev, requires_grad=True)
    qq = q.detach().requires_grad_(True)
    loss_of(qq, eps, sig, 0).backward()
    for (i, a) in coords:
        adj[f"q[{i},{a}]"] = float(qq.grad[i, a])
    res["fp64_vs_central_differences"] = {
        k: {"adjoint": adj[k], "central_difference": fd[k],
            "rel_diff": abs(adj[k] - fd[k]) / max(abs(fd[k]), 1e-300)} for k in fd}
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
    from paper_1806_05713_gb300.md import VelocityVerlet
    s = system_from_spec(("fcc", PAPER_K, RHO, JITTER, 0, "random"))
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


if __name__ == "__main__":
    main()
