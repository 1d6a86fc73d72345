"""Benchmark of the GB300 Ant System (one JSON line on stdout).

A step is one full Ant System iteration of the workload (tour construction,
iteration best, deposit, evaporation and choice_info), replayed from a CUDA
graph through the C ABI with all state resident in HBM.  Between timed steps
L2 is flushed by writing a 256 MB buffer (outside the timed region); each step
is timed with CUDA events on the stream the library launches on.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload n1002]
                  [--deposit sym|gather|u64|f32] [--impl ours|reference]

--impl reference times the CPU oracle (the slow, plain restatement of the
method used by the tests) on a bounded sample of the same workload.
With N > 1 (torchrun) every rank runs an independent replica of the workload
(no data-path collective: the instances are independent); the reported value
is the sum over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
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

METRIC = "ant-steps/s (tour constr.) & edges/s (pheromone) vs roofline; batched solves/s, p99"
WORKLOADS = {
    "n48": "workload_n48",
    "n1002": "workload_n1002",
    "n2392": "workload_n2392",
    "batched": None,
    "served": None,
}
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="n1002", choices=sorted(WORKLOADS))
    ap.add_argument("--deposit", default="sym", choices=["gather", "u64", "f32", "sym", "sort"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dist-timeout", type=float, default=600.0,
                    help="seconds a rank waits in a barrier or collective for the others")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--warps-per-ant", type=int, default=0, help="0 = library default")
    ap.add_argument("--ants-per-cta", type=int, default=0, help="0 = library default")
    ap.add_argument("--lanes-per-ant", type=int, default=0, help="0 = library default (32)")
    ap.add_argument("--staging", type=int, default=-1,
                    help="row staging of the construction kernel: 0 bulk copy (TMA), "
                         "1 lane copies; -1 = library default")
    ap.add_argument("--nn", type=int, default=0,
                    help="nearest-neighbour list length (0 = every unvisited city)")
    ap.add_argument("--variant", default="as", choices=["as", "mmas", "acs"],
                    help="as: the Ant System update (Eqs. 2-4); mmas: the MAX-MIN Ant System "
                         "update (p_best 0.05, iteration-best deposit); acs: the Ant Colony "
                         "System (q0 0.9, xi 0.1; m = min(m, 10))")
    ap.add_argument("--selection", default="eq1", choices=["eq1", "data-parallel", "exp-race"],
                    help="eq1: Eq. 1 by the integer roulette (default); data-parallel: the "
                         "paper's product-argmax kernel; exp-race: the exponential race "
                         "(per-candidate exponentials, samples Eq. 1)")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--batch-iterations", type=int, default=0,
                    help="0 = the workload's 100; fewer for profiling runs")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched: default tiling for every class (profiling runs)")
    ap.add_argument("--no-loop-baseline", action="store_true",
                    help="skip the per-instance loop (profiling runs)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the Poisson arrival window for --workload served")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-step-work", type=float, default=1e11,
                    help="served: candidate evaluations one step may hold (admission bound)")
    ap.add_argument("--serve-nn", type=int, default=0,
                    help="served: nearest-neighbour lists of this length for every request "
                         "(0: dense Eq. 1, the configured workload)")
    ap.add_argument("--no-multirate", action="store_true",
                    help="served: one iteration per step for every request (no multi-rate "
                         "stepping)")
    ap.add_argument("--serve-loop-sample", type=int, default=16,
                    help="requests solved one at a time for the loop comparison")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ---------------------------------------------------------------------------
def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import datetime
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        # a replica that dies makes the others' next barrier fail after this
        # long instead of waiting forever
        dist.init_process_group("nccl", timeout=datetime.timedelta(seconds=args.dist_timeout))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    """Largest v over all ranks (the slowest rank's time sets the job's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, my_seconds: float, world: int) -> float:
    """Whole-job throughput of `world` independent replicas: all ranks' units
    divided by the slowest rank's time (every rank does the same work)."""
    return units_per_rank * world / max_over_ranks(my_seconds, world)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measure_l2_copy_gbs(reps: int = 64, mib: int = 24, trials: int = 5) -> float:
    """L2 copy bandwidth: torch copies between two L2-resident buffers.

    Same method as the HBM figure of MEASURED_PEAKS.json (read + write bytes
    of b.copy_(a), CUDA events), but on 2 x `mib` MiB, which stay in the
    129 MB L2, with `reps` back-to-back copies replayed from one CUDA graph
    so launch gaps do not count; best of `trials`."""
    import torch
    a = torch.empty(mib << 18, dtype=torch.float32, device="cuda").normal_()
    b = torch.empty_like(a)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(3):
            b.copy_(a)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            b.copy_(a)
    g.replay()
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(trials):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        if ms > 0:
            best = max(best, reps * 2 * a.numel() * 4 / (ms / 1e3) / 1e9)
    return best


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample(w, ants: int):
    """Time the oracle on `ants` ants of iteration 0 plus one full update.

    Returns (ant_steps_per_s, seconds, description)."""
    import numpy as np
    from oracle import oracle as orc
    d = w["inst"].dist
    n, m = d.shape[0], w["m"]
    t0 = time.perf_counter()
    h = orc.heta(d, w["beta"])
    tau = np.full((n, n), orc.tau0(d, m), np.float32)
    np.fill_diagonal(tau, 0)
    ch = orc.choice(tau, h, w["alpha"])
    t_setup = time.perf_counter() - t0
    ants = max(1, min(ants, m))
    t0 = time.perf_counter()
    tours = np.zeros((m, n + 1), np.int32)
    lens = np.zeros(m, np.int64)
    for k in range(ants):
        tours[k], lens[k] = orc.construct_ant(ch, d, w["seed"], 0, k)
    t_con = time.perf_counter() - t0
    # the other ants' tours are copies for the update (same work per edge)
    for k in range(ants, m):
        tours[k], lens[k] = tours[k % ants], lens[k % ants]
    t0 = time.perf_counter()
    tau = orc.update_mirror(tau, tours, lens, w["rho"])
    ch = orc.choice(tau, h, w["alpha"])
    t_upd = time.perf_counter() - t0
    per_iter = t_con / ants * m + t_upd
    value = m * (n - 1) / per_iter
    desc = (f"oracle (C, 1 thread): {ants} of {m} ants of iteration 0 constructed plus one "
            f"full pheromone update and choice_info; iteration time extrapolated as "
            f"t_ant*m + t_update (setup {t_setup:.2f}s not counted)")
    return value, t_con + t_upd, desc


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    import numpy as np  # noqa: F401
    from oracle import oracle as orc
    orc.build()
    d = w["inst"].dist
    n, m = d.shape[0], w["m"]
    ants = max(1, min(m, int(2.0 / max(_oracle_ant_seconds(w), 1e-6))))
    for _ in range(args.warmup):
        oracle_sample(w, max(1, ants // 4))
    vals, secs = [], 0.0
    for _ in range(args.steps):
        v, s, desc = oracle_sample(w, ants)
        vals.append(v)
        secs += s
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ant-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": m * (n - 1) / value * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["name"], "n": n, "m": m, "iterations": w["iterations"],
                   "parallelism": "cpu-1-thread", "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": "ant-steps/s", "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "ant-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _oracle_ant_seconds(w):
    import numpy as np
    from oracle import oracle as orc
    d = w["inst"].dist
    n, m = d.shape[0], w["m"]
    h = orc.heta(d, w["beta"])
    tau = np.full((n, n), orc.tau0(d, m), np.float32)
    ch = orc.choice(tau, h, w["alpha"])
    t0 = time.perf_counter()
    orc.construct_ant(ch, d, w["seed"], 0, 0)
    return time.perf_counter() - t0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args, w, rank, world, local):
    import numpy as np
    import torch

    from paper_1101_2678_gb300 import aco

    torch.cuda.set_device(local)
    aco.load()
    d = w["inst"].dist
    n, m = d.shape[0], w["m"]
    if args.variant == "acs":
        m = min(m, 10)  # the Ant Colony System's usual colony (one CTA, m <= 32)
    dep = {"gather": aco.ACO_DEPOSIT_GATHER, "u64": aco.ACO_DEPOSIT_ATOMIC_U64,
           "f32": aco.ACO_DEPOSIT_ATOMIC_F32, "sym": aco.ACO_DEPOSIT_SYMMETRIC,
           "sort": aco.ACO_DEPOSIT_SORT}[args.deposit]
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    def configure(h):
        """The run's options and update rule (the timed handle and the e2e solve)."""
        aco.aco_set_option(h, aco.ACO_OPT_DEPOSIT, dep)
        if args.warps_per_ant:
            aco.aco_set_option(h, aco.ACO_OPT_WARPS_PER_ANT, args.warps_per_ant)
        if args.selection != "eq1":
            aco.aco_set_option(h, aco.ACO_OPT_SELECTION,
                               {"data-parallel": aco.ACO_SELECT_DATA_PARALLEL,
                                "exp-race": aco.ACO_SELECT_EXP_RACE}[args.selection])
        if args.nn:
            aco.aco_set_option(h, aco.ACO_OPT_NN_LIST, args.nn)
        if args.staging >= 0:
            aco.aco_set_option(h, aco.ACO_OPT_STAGING, args.staging)
        if args.variant == "mmas":
            aco.aco_set_mmas(h, 0.05, False)
        elif args.variant == "acs":
            aco.aco_set_acs(h, 0.9, 0.1)
        if args.lanes_per_ant:
            aco.aco_set_option(h, aco.ACO_OPT_LANES_PER_ANT, args.lanes_per_ant)
        if args.ants_per_cta:
            aco.aco_set_option(h, aco.ACO_OPT_ANTS_PER_CTA, args.ants_per_cta)

    col = aco.Colony(d, m, seed=w["seed"] + rank, alpha=w["alpha"], beta=w["beta"], rho=w["rho"])
    h = col.h
    aco.aco_set_option(h, aco.ACO_OPT_STREAM, stream.cuda_stream)
    aco.aco_set_option(h, aco.ACO_OPT_PROFILE, 1)
    configure(h)
    tiling = (aco.aco_get_option(h, aco.ACO_OPT_WARPS_PER_ANT),
              aco.aco_get_option(h, aco.ACO_OPT_ANTS_PER_CTA),
              aco.aco_get_option(h, aco.ACO_OPT_LANES_PER_ANT))
    launches = aco.aco_kernel_launches_per_iteration(h)
    staging = aco.aco_get_option(h, aco.ACO_OPT_STAGING)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            aco.aco_iterate(h, 1)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        clocks = ClockSampler(local) if rank == 0 else None
        if clocks:
            clocks.start()
        step_ms, phase_ms = [], np.zeros(aco.ACO_NUM_PHASES)
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            aco.aco_iterate(h, 1)
            e1.record(stream)
            phase_ms += aco.aco_get_kernel_times(h)  # synchronises the stream
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
    aco.aco_synchronize(h)
    best_tour, best_len = aco.aco_best_tour(h, n)
    col.close()

    steps = args.steps
    value = replica_throughput(m * (n - 1) * steps, sum(step_ms) / 1e3, world)
    total_ms = m * (n - 1) * steps * world / value * 1e3
    con_ms = phase_ms[aco.ACO_PHASE_CONSTRUCT] / steps
    upd_ms = (phase_ms[aco.ACO_PHASE_DEPOSIT] + phase_ms[aco.ACO_PHASE_UPDATE]) / steps
    best_ms = phase_ms[aco.ACO_PHASE_BEST] / steps

    # e2e: a whole solve through the public API from host memory.
    e2e = None
    if not args.no_e2e:
        e2e = e2e_solve(aco, w, rank, m, configure)

    if rank != 0:
        return
    peaks, peak_kind = measured_peaks()
    if args.variant == "acs":
        kernel = "acs_construct_kernel"
    elif args.nn:
        kernel = "construct_nn_kernel"
    else:
        kernel = "construct_kernel"
    roof = construct_roofline(n, m, con_ms, peaks, peak_kind, kernel=kernel, nn=args.nn)
    if not (args.nn or args.selection != "eq1" or args.lanes_per_ant or args.warps_per_ant
            or args.ants_per_cta or args.variant != "as"):
        roof["traffic"], roof["traffic_source"] = recorded_traffic(w["name"])
    l2_gbs = measure_l2_copy_gbs()
    algo = roof["algorithmic_bytes_per_launch"]
    # bytes the kernel stages per launch: whole rows for the Eq. 1 kernels,
    # one 128-byte line of list values plus the list for the NN-list kernel
    dense = 4.0 * m * (n - 1) * n if not args.nn else 256.0 * m * (n - 1)
    roof_l2 = {"bound": "l2", "peak": l2_gbs, "unit": "GB/s",
               "peak_kind": "L2 copy bandwidth measured in this run (64 graph-replayed torch copies, 2 x 24 MiB)",
               "achieved_algorithmic": algo / (con_ms / 1e3) / 1e9,
               "frac_algorithmic": algo / (con_ms / 1e3) / 1e9 / l2_gbs,
               "achieved_dense_rows": dense / (con_ms / 1e3) / 1e9,
               "frac_dense_rows": dense / (con_ms / 1e3) / 1e9 / l2_gbs}
    line = {
        "metric": METRIC, "value": value, "unit": "ant-steps/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": total_ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w["name"], "n": n, "m": m, "alpha": w["alpha"],
                   "beta": w["beta"], "rho": w["rho"], "deposit": args.deposit,
                   "warps_per_ant": tiling[0], "ants_per_cta": tiling[1],
                   "lanes_per_ant": tiling[2], "selection": args.selection, "nn_list": args.nn,
                   "variant": args.variant,
                   "staging": staging,
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "flushed between steps (256 MB write)"},
        "construct_ant_steps_per_s": m * (n - 1) / (con_ms / 1e3),
        "pheromone_edges_per_s": m * n / (upd_ms / 1e3),
        "phase_ms": {"construct": con_ms, "best": best_ms, "pheromone": upd_ms},
        "best_len": best_len,
        "roofline": roof,
        "roofline_l2": roof_l2,
        "gpu_launches": launches * steps,
        "clocks": clk,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        v, s, desc = oracle_sample(w, max(1, int(10.0 / max(_oracle_ant_seconds(w), 1e-6))))
        line["cpu_baseline"] = {"value": v, "unit": "ant-steps/s", "cores": 1, "kind": "oracle",
                                "sample": desc}
    print(json.dumps(line), flush=True)


CONSTRUCT_SOURCES = ("aco_device.cuh", "construct.cuh", "construct_g1h8.cu", "construct_g1h16.cu",
                     "construct_g1h32.cu", "construct_g2h32.cu", "construct_g4h32.cu",
                     "construct_rule.cuh", "construct_rule1.cu", "construct_rule2.cu")


def construct_sources_sha256() -> str:
    """SHA-256 over the construction kernel's sources, in a fixed order."""
    import hashlib
    h = hashlib.sha256()
    for f in CONSTRUCT_SOURCES:
        with open(os.path.join(ROOT, "paper_1101_2678_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(workload: str):
    """DRAM bytes (read + write) per construct launch from a committed ncu capture.

    The summaries under profiles/ carry a line
    `traffic-record: workload=<name> dram_bytes_per_launch=<B> sources_sha256=<H>`;
    the figure is used only if H equals the hash of the current sources (else
    the counters describe another kernel and traffic is null)."""
    import glob
    sha = construct_sources_sha256()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "construct_kernel_*.md"))):
        with open(path) as fh:
            for line in fh:
                if not line.startswith("traffic-record:"):
                    continue
                kv = dict(x.split("=", 1) for x in line.split()[1:])
                if kv.get("workload") == workload and kv.get("sources_sha256") == sha:
                    return float(kv["dram_bytes_per_launch"]), os.path.relpath(path, ROOT)
    return None, None


def construct_roofline(n, m, con_ms, peaks, peak_kind, kernel="construct_kernel", nn=0):
    """Roofline entry for the construction kernel (the dominant kernel).

    Algorithmic bytes per launch: every ant reads, at each of its n-1 steps,
    the 4-byte choice_info entries of the cities it has not visited yet:
    4 * m * sum_{s=1}^{n-1} (n - s) = 4 m n (n-1) / 2.  With nearest-neighbour
    lists a step needs the current city's nn list entries and their
    list-ordered choice_info values: 8 * nn bytes, m (n-1) steps."""
    if nn:
        algo = 8.0 * nn * m * (n - 1)
    else:
        algo = 4.0 * m * n * (n - 1) / 2.0
    achieved = algo / (con_ms / 1e3) / 1e9
    peak = float(peaks["hbm_gbs"])
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None,
            "peak_kind": f"{peak_kind} HBM copy bandwidth",
            "kernel": kernel, "algorithmic_bytes_per_launch": algo,
            "avg_launch_ms": con_ms}


def e2e_solve(aco, w, rank, m, configure):
    """create (uploads dist) + the run's options + iterate + best tour to the host,
    wall-clock timed."""
    import numpy as np
    import torch
    d = np.ascontiguousarray(w["inst"].dist, dtype=np.int32)
    n, iters = d.shape[0], w["iterations"]
    pinned = torch.from_numpy(d).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = aco.aco_create(pinned, w["alpha"], w["beta"], w["rho"], m, w["seed"] + rank)
    configure(h)
    aco.aco_iterate(h, iters)
    tour, length = aco.aco_best_tour(h, n)
    t1 = time.perf_counter()
    aco.aco_destroy(h)
    h2d = d.nbytes
    d2h = tour.nbytes + 8
    return {"value": m * (n - 1) * iters / (t1 - t0), "unit": "ant-steps/s",
            "h2d_bytes_per_step": h2d / iters, "d2h_bytes_per_step": d2h / iters,
            "what": f"aco_create from pinned host dist + aco_iterate({iters}) + aco_best_tour "
                    f"to host, wall clock; bytes amortised over the {iters} iterations",
            "seconds": t1 - t0}


def run_batched(args, rank, world, local):
    """256 independent instances x 100 iterations: one pool (graph per step) vs the
    plain per-instance loop over the same kernels."""
    import numpy as np
    import torch
    from paper_1101_2678_gb300 import aco, instances
    torch.cuda.set_device(local)
    aco.load()
    w = instances.workload_batched(args.batch_count)
    insts, ms, seeds, iters = w["insts"], w["ms"], w["seeds"], w["iterations"]
    if args.batch_iterations:
        iters = args.batch_iterations
    dists = [x.dist for x in insts]
    # warm-up (module load, graph code paths)
    b = aco.aco_batch_create(dists[:4], ms[:4], seeds[:4])
    if args.no_autotune:
        aco.aco_pool_set_autotune(b, False)
    aco.aco_batch_iterate(b, 3)
    aco.aco_pool_synchronize(b)
    aco.aco_batch_destroy(b)
    barrier(world)
    b = aco.aco_batch_create(dists, ms, seeds)
    aco.aco_pool_synchronize(b)
    if args.no_autotune:
        aco.aco_pool_set_autotune(b, False)
    # choose each class's construction tiling before the timed run (the
    # choice does not change any result); reported in config
    t_tune = time.perf_counter()
    aco.aco_pool_autotune(b)
    aco.aco_pool_synchronize(b)
    t_tune = time.perf_counter() - t_tune
    tilings = {}
    for i, x in enumerate(insts):
        g, hh, c, sg = aco.aco_pool_tiling(b, i)
        key = f"G{g}H{hh}C{c}S{sg}"
        tilings[key] = tilings.get(key, 0) + 1
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    t0 = time.perf_counter()
    aco.aco_batch_iterate(b, iters)
    aco.aco_pool_synchronize(b)
    t_batch = time.perf_counter() - t0
    clk = clocks.stop() if clocks else None
    launches = aco.aco_pool_stats(b)["launches_last_step"]
    best_batch = [aco.aco_batch_best(b, i, x.n)[1] for i, x in enumerate(insts)]
    aco.aco_batch_destroy(b)
    # per-instance loop
    t_loop = 0.0
    best_loop = []
    for i, x in enumerate([] if args.no_loop_baseline else insts):
        c = aco.Colony(x.dist, ms[i], seed=seeds[i])
        aco.aco_synchronize(c.h)
        t0 = time.perf_counter()
        aco.aco_iterate(c.h, iters)
        aco.aco_synchronize(c.h)
        t_loop += time.perf_counter() - t0
        best_loop.append(aco.aco_best_tour(c.h, x.n)[1])
        c.close()
    t_batch = max_over_ranks(t_batch, world)
    if rank != 0:
        return
    ant_steps = sum(m * (x.n - 1) for m, x in zip(ms, insts)) * iters
    line = {
        "metric": "batched solves/s", "value": world * len(insts) / t_batch, "unit": "solves/s",
        "n_gpus": world, "steps": iters, "warmup": 3, "ms_per_step": t_batch / iters * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w["name"], "instances": len(insts), "n_min": min(x.n for x in insts),
                   "n_max": max(x.n for x in insts), "iterations": iters,
                   "l2": "not flushed (one continuous 100-step run)",
                   "autotuned_tilings": tilings, "autotune_seconds": t_tune},
        "per_instance_loop_solves_per_s": len(insts) / t_loop if t_loop else None,
        "speedup_vs_loop": t_loop / t_batch if t_loop else None,
        "identical_best_lengths": best_batch == best_loop,
        "ant_steps_per_s": ant_steps / t_batch,
        "gpu_launches": launches * iters, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_batched_rule(args, rank, world, local):
    """The batched workload's instances under another update rule, in one pool
    vs the plain per-instance loop over the single-handle kernels:
    acs: Ant Colony System colonies (m = 10, q0 0.9, xi 0.1, rho 0.1), one
    launch for all colonies per step; mmas: the MAX-MIN Ant System (m = n,
    rho 0.02, p_best 0.05, iteration-best deposit), construction classes
    shared with the Ant System path and its own row update."""
    import torch
    from paper_1101_2678_gb300 import aco, instances
    torch.cuda.set_device(local)
    aco.load()
    w = instances.workload_batched(args.batch_count)
    insts, seeds, iters = w["insts"], w["seeds"], w["iterations"]
    if args.batch_iterations:
        iters = args.batch_iterations
    acs = args.variant == "acs"
    ms = [10] * len(insts) if acs else list(w["ms"])
    rho = 0.1 if acs else 0.02
    q0, xi, p_best = 0.9, 0.1, 0.05

    def admit(p, i, x, iterations):
        if acs:
            return aco.aco_pool_admit_acs(p, x.dist, 1.0, 2.0, rho, ms[i], seeds[i], iterations,
                                          q0, xi)
        return aco.aco_pool_admit_mmas(p, x.dist, 1.0, 2.0, rho, ms[i], seeds[i], iterations,
                                       p_best, False)

    def pool_run(subset, iterations):
        need = sum(aco.aco_pool_bytes_needed(x.n, ms[i]) for i, x in enumerate(subset))
        p = aco.aco_pool_create(len(subset), need + (1 << 20))
        if args.no_autotune:
            aco.aco_pool_set_autotune(p, False)
        slots = [admit(p, i, x, iterations) for i, x in enumerate(subset)]
        aco.aco_pool_synchronize(p)
        return p, slots

    p, _ = pool_run(insts[:4], 3)  # warm-up (module load, graph code paths)
    while aco.aco_pool_step(p) > 0:
        pass
    aco.aco_pool_synchronize(p)
    aco.aco_pool_destroy(p)
    barrier(world)
    p, slots = pool_run(insts, iters)
    # the construction tilings of the MAX-MIN classes are chosen before the
    # timed run (the choice changes no result)
    t_tune = time.perf_counter()
    aco.aco_pool_autotune(p)
    aco.aco_pool_synchronize(p)
    t_tune = time.perf_counter() - t_tune
    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
    t0 = time.perf_counter()
    launches = steps = 0
    while True:
        live = aco.aco_pool_step(p)
        launches += aco.aco_pool_stats(p)["launches_last_step"]
        steps += 1
        if live == 0:
            break
    aco.aco_pool_synchronize(p)
    t_batch = time.perf_counter() - t0
    clk = clocks.stop() if clocks else None
    best_batch = [aco.aco_pool_result(p, s, x.n)[1] for s, x in zip(slots, insts)]
    aco.aco_pool_destroy(p)
    t_loop = 0.0
    best_loop = []
    for i, x in enumerate([] if args.no_loop_baseline else insts):
        c = aco.Colony(x.dist, ms[i], seed=seeds[i], rho=rho)
        if acs:
            aco.aco_set_acs(c.h, q0, xi)
        else:
            aco.aco_set_mmas(c.h, p_best, False)
        aco.aco_synchronize(c.h)
        t0 = time.perf_counter()
        aco.aco_iterate(c.h, iters)
        aco.aco_synchronize(c.h)
        t_loop += time.perf_counter() - t0
        best_loop.append(aco.aco_best_tour(c.h, x.n)[1])
        c.close()
    t_batch = max_over_ranks(t_batch, world)
    if rank != 0:
        return
    ant_steps = sum(m * (x.n - 1) for m, x in zip(ms, insts)) * iters
    rule = ({"variant": "acs", "m": 10, "q0": q0, "xi": xi, "rho": rho} if acs else
            {"variant": "mmas", "m": "n", "p_best": p_best, "deposit": "iteration best",
             "rho": rho, "autotune_seconds": t_tune})
    line = {
        "metric": "batched solves/s", "value": world * len(insts) / t_batch, "unit": "solves/s",
        "n_gpus": world, "steps": iters, "warmup": 3, "ms_per_step": t_batch / iters * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w["name"].replace("as-", args.variant + "-"), **rule,
                   "instances": len(insts), "n_min": min(x.n for x in insts),
                   "n_max": max(x.n for x in insts), "iterations": iters, "pool_steps": steps,
                   "l2": "not flushed (one continuous run)"},
        "per_instance_loop_solves_per_s": len(insts) / t_loop if t_loop else None,
        "speedup_vs_loop": t_loop / t_batch if t_loop else None,
        "identical_best_lengths": best_batch == best_loop if best_loop else None,
        "ant_steps_per_s": ant_steps / t_batch,
        "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_served(args, rank, world, local):
    """Poisson arrivals (n log-uniform in [48, 4096], m = min(n, 1024), 200 iterations)
    through the continuous-batching server with a 64 GB HBM budget."""
    import numpy as np
    import torch
    from paper_1101_2678_gb300 import aco, instances, serve
    torch.cuda.set_device(local)
    aco.load()
    arrivals = instances.poisson_arrivals(args.serve_rate, args.serve_seconds)
    reqs = []
    for r in range(len(arrivals)):
        q = instances.served_request(r)
        reqs.append(serve.Request(q["inst"].coords, q["m"], q["iterations"], q["seed"],
                                  nn=args.serve_nn))
    mr = not args.no_multirate
    work = int(args.serve_step_work)
    with serve.Server(budget_bytes=64 << 30, max_slots=4096, multirate=mr,
                      max_step_work=work) as srv:
        # configured stream: stop admitting/stepping at the end of the arrival window
        outs, st = srv.run(reqs, arrivals, deadline=args.serve_seconds)
    with serve.Server(budget_bytes=64 << 30, max_slots=4096, multirate=mr,
                      max_step_work=work) as srv:
        # sustainable stream at 0.7x the measured completion rate
        cap = max(st["solves_per_s"], 0.5)
        rate = 0.7 * cap
        arr2 = instances.poisson_arrivals(rate, args.serve_seconds, seed=6)
        reqs2 = [reqs[i % len(reqs)] for i in range(len(arr2))]
        outs2, st2 = srv.run(reqs2, arr2, deadline=3 * args.serve_seconds)
    # the same requests one at a time through the single-instance API (the plain
    # per-request loop) against the server on the same sample, all admitted at once
    sample = reqs[:args.serve_loop_sample]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loop_lens = []
    for r in sample:
        h = aco.aco_create_coords(r.coords, r.alpha, r.beta, r.rho, r.m, r.seed)
        if r.nn:
            aco.aco_set_option(h, aco.ACO_OPT_NN_LIST, r.nn)
        aco.aco_iterate(h, r.iterations)
        loop_lens.append(aco.aco_best_tour(h, r.n)[1])
        aco.aco_destroy(h)
    t_loop = time.perf_counter() - t0
    loop = None
    if sample:
        with serve.Server(budget_bytes=64 << 30, max_slots=4096, max_step_work=1 << 62,
                          multirate=mr) as srv:
            outs3, st3 = srv.run(sample, np.zeros(len(sample)), realtime=False)
        same = sorted((o.index, o.best_len) for o in outs3) == list(enumerate(loop_lens))
        loop = {
            "requests": len(sample), "per_request_loop_solves_per_s": len(sample) / t_loop,
            "server_solves_per_s": st3["solves_per_s"],
            "speedup_vs_loop": st3["solves_per_s"] * t_loop / len(sample),
            "identical_best_lengths": same,
            "what": "the first requests of the stream solved one at a time (aco_create_coords "
                    "+ aco_iterate(200) + aco_best_tour) vs the server with all of them "
                    "admitted at once"}
    if rank != 0:
        return
    line = {
        "metric": "served solves/s, p50/p99 latency", "value": st["solves_per_s"],
        "unit": "solves/s", "n_gpus": world, "steps": st["steps"], "warmup": 0,
        "ms_per_step": st["elapsed_s"] / max(st["steps"], 1) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "as-served-poisson", "rate_per_s": args.serve_rate,
                   "window_s": args.serve_seconds, "budget_gb": 64, "iterations": 200,
                   "multirate": mr, "max_step_work": work, "nn_list": args.serve_nn},
        "configured_stream": st,
        "sustainable_stream": dict(st2, rate_per_s=rate),
        "loop_comparison": loop,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init(args)
    from paper_1101_2678_gb300 import instances
    if args.workload == "batched" and args.variant != "as":
        run_batched_rule(args, rank, world, local)
        return
    if args.workload == "batched":
        run_batched(args, rank, world, local)
        return
    if args.workload == "served":
        run_served(args, rank, world, local)
        return
    w = getattr(instances, WORKLOADS[args.workload])()
    if args.impl == "reference":
        run_reference(args, w, rank, world)
    else:
        run_ours(args, w, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
