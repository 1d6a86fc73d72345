"""Benchmark of the GB300 Ant System (one JSON line on stdout).

A step is one full Ant System iteration of the workload (tour construction,
iteration best, deposit, evaporation and choice_info), replayed from a CUDA
graph through the C ABI with all state resident in HBM.  Between timed steps
L2 is flushed by writing a 256 MB buffer (outside the timed region); each step
is timed with CUDA events on the stream the library launches on.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload n2392]
                  [--deposit sym|gather|u64|f32] [--impl ours|reference]

The default workload is 2392 clustered cities with m = 2392 ants (the size of
the paper's largest instance, pr2392).  Its line also carries the batched
workload (256 instances in one pool against the per-instance loop) and the
CPU oracle on every host core.  --impl reference times the CPU oracle (the
slow, plain restatement of the method used by the tests) on every host core,
in steps of whole iterations or of a measured sample of ants.
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
    ap.add_argument("--workload", default="n2392", choices=sorted(WORKLOADS))
    ap.add_argument("--deposit", default="sym", choices=["gather", "u64", "f32", "sym", "sort"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dist-timeout", type=float, default=600.0,
                    help="seconds a rank waits in a barrier or collective for the others")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="single-instance workloads: skip the batched line carried in the "
                         "same JSON line (the 256-instance pool against the per-instance loop)")
    ap.add_argument("--ants", type=int, default=0,
                    help="override m (0 = the workload's m); for small profiling captures of "
                         "the same kernel")
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
    ap.add_argument("--single-launch", action="store_true",
                    help="batched: every construction class in one persistent launch")
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


L2_PROBE_MIB = 24


def measure_l2_read_gbs(trials: int = 10, reps: int = 64):
    """Read-only L2 bandwidth, measured in this run with the library's probe.

    A 24 MiB buffer (L2-resident: the L2 holds 129 MB) is read `reps` times per
    launch, either by 16-byte loads that bypass L1 or by 16 KB bulk copies into
    shared memory (the construction kernel's route); each launch is timed with
    CUDA events on its stream, best of `trials`, over a few grid sizes.
    Returns {"float4": GB/s, "bulk": GB/s, "peak": the larger, ...}."""
    import torch
    from paper_1101_2678_gb300 import aco
    nbytes = L2_PROBE_MIB << 20
    buf = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda").uniform_(0.0, 1.0)
    sink = torch.zeros(4, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    out = {}
    with torch.cuda.stream(s):
        for mode, name, grids in ((0, "float4", (2, 4, 8)), (1, "bulk", (2, 3, 6))):
            best = 0.0
            for bps in grids:
                for t in range(trials + 2):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(s)
                    aco.aco_stream_read(buf.data_ptr(), nbytes, reps, mode, bps, s.cuda_stream,
                                        sink.data_ptr(), status.data_ptr())
                    e1.record(s)
                    e1.synchronize()
                    ms = e0.elapsed_time(e1)
                    if t >= 2 and ms > 0:  # the first two launches warm up
                        best = max(best, reps * nbytes / (ms / 1e3) / 1e9)
            out[name] = best
    torch.cuda.synchronize()
    if int(status.item()) != 0:
        raise RuntimeError("the bulk-copy read probe reported a timed-out wait")
    out["peak"] = max(out["float4"], out["bulk"])
    out["how"] = (f"aco_stream_read over a {L2_PROBE_MIB} MiB L2-resident buffer, {reps} "
                  f"passes per launch, CUDA events, best of {trials} over grids of 2-8 CTAs "
                  f"per SM; float4 = 16-byte ld.global.cg loads, bulk = 16 KB cp.async.bulk "
                  f"copies into shared memory")
    return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
class OracleStep:
    """Timed steps of the CPU oracle on a workload.

    A step builds the first `ants` ants of iteration 0 with Eq. 1 (ant k uses
    the same counters as in a whole iteration) on `threads` host threads, then
    runs the pheromone update (Eqs. 2-4) with their tours and choice_info.
    With ants = m a step is one whole iteration.  Setup (eta^beta, tau0, the
    first choice_info) happens once, outside the timed steps."""

    def __init__(self, w):
        import numpy as np
        from oracle import oracle as orc
        orc.build()
        self.orc, self.w = orc, w
        self.d = w["inst"].dist
        self.n, self.m = self.d.shape[0], w["m"]
        self.h = orc.heta(self.d, w["beta"])
        self.tau = np.full((self.n, self.n), orc.tau0(self.d, self.m), np.float32)
        np.fill_diagonal(self.tau, 0)
        self.ch = orc.choice(self.tau, self.h, w["alpha"])

    def run(self, ants: int, threads: int):
        """(seconds, ant-steps) of one step."""
        orc, w = self.orc, self.w
        ants = max(1, min(ants, self.m))
        orc.set_threads(threads)
        try:
            t0 = time.perf_counter()
            tours, lens = orc.construct(self.ch, self.d, ants, w["seed"], 0)
            tau = orc.update_mirror(self.tau, tours, lens, w["rho"])
            orc.choice(tau, self.h, w["alpha"])
            sec = time.perf_counter() - t0
        finally:
            orc.set_threads(1)
        return sec, ants * (self.n - 1)

    def ants_for(self, seconds: float, threads: int) -> int:
        """Ants whose step takes about `seconds` (calibrated on a short step)."""
        probe = min(self.m, 4 * max(threads, 1))
        sec, _ = self.run(probe, threads)
        per_ant = sec / probe
        return max(1, min(self.m, int(seconds / max(per_ant, 1e-9))))

    def describe(self, ants: int, threads: int) -> str:
        what = ("whole iterations" if ants >= self.m else
                f"the first {ants} of {self.m} ants of an iteration")
        return (f"oracle (C, {threads} host thread{'s' if threads > 1 else ''}): {what} built "
                f"with Eq. 1, then the full pheromone update and choice_info over their tours; "
                f"value = ant-steps built / measured step time")


def cpu_baseline(w):
    """The oracle on every host core (whole iterations if one takes under
    ~20 s, else a timed sample of ants of about that length) and on one core
    (a timed sample of about 5 s); each figure is measured, not extrapolated."""
    o = OracleStep(w)
    hw = o.orc.hardware_threads()
    ants = o.ants_for(20.0, hw)
    sec, units = o.run(ants, hw)
    one_ants = o.ants_for(5.0, 1)
    sec1, units1 = o.run(one_ants, 1)
    return {"value": units / sec, "unit": "ant-steps/s", "cores": hw, "kind": "oracle",
            "sample": o.describe(ants, hw), "seconds": sec, "hardware_threads": hw,
            "one_core": {"value": units1 / sec1, "unit": "ant-steps/s", "cores": 1,
                         "sample": o.describe(one_ants, 1), "seconds": sec1}}


def run_reference(args, w, rank, world):
    """--impl reference: the CPU oracle on every host core, K timed steps after
    W warm-up steps, each step sized so the whole run stays within ~3 minutes
    (whole iterations when they fit)."""
    if rank != 0:
        return
    o = OracleStep(w)
    hw = o.orc.hardware_threads()
    budget = 150.0 / max(args.steps + args.warmup, 1)
    ants = o.ants_for(budget, hw)
    for _ in range(args.warmup):
        o.run(ants, hw)
    secs, units = 0.0, 0
    for _ in range(args.steps):
        sec, u = o.run(ants, hw)
        secs += sec
        units += u
    value = units / secs
    n, m = o.n, o.m
    desc = o.describe(ants, hw)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ant-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["name"], "n": n, "m": m, "iterations": w["iterations"],
                   "ants_per_step": ants, "parallelism": f"cpu-{hw}-threads",
                   "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": "ant-steps/s", "cores": hw, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "ant-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


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
    if args.ants:
        m = args.ants
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

    # The batched workload (256 instances in one pool against the per-instance
    # loop), carried in the same line.
    batched = None
    if not args.no_batched and args.variant == "as" and not args.ants:
        batched = batched_measure(args, rank, world, local)

    if rank != 0:
        return
    peaks, peak_kind = measured_peaks()
    if args.variant == "acs":
        kernel = "acs_construct_kernel"
    elif args.nn:
        kernel = "construct_nn_kernel"
    elif args.selection == "eq1" and tiling[0] == 1 and n > 12 * tiling[2]:
        # one warp or segment per ant with at least 20 cities per lane: the
        # walk with compaction
        kernel = "construct_phased_kernel"
    else:
        kernel = "construct_kernel"
    l2 = measure_l2_read_gbs()
    roof = construct_roofline(n, m, con_ms, l2, peaks, peak_kind, kernel=kernel, nn=args.nn)
    if not (args.nn or args.selection != "eq1" or args.lanes_per_ant or args.warps_per_ant
            or args.ants_per_cta or args.variant != "as"):
        rec = recorded_traffic(w["name"], m)
        if rec:
            roof["traffic"] = rec["dram_bytes_per_launch"]
            roof["l2_bytes_per_launch"] = rec.get("l2_bytes_per_launch")
            if rec.get("l2_bytes_per_launch"):
                # L2 bytes the kernel moved (ncu lts__t_bytes, scaled to the
                # full launch) per second of the launch timed here, against
                # the same measured read peak
                l2_gbs = rec["l2_bytes_per_launch"] / (con_ms / 1e3) / 1e9
                roof["achieved_l2_traffic"] = l2_gbs
                roof["frac_l2_traffic"] = l2_gbs / roof["peak"]
            roof["traffic_source"] = rec["source"]
            roof["ncu_capture"] = {"ants": rec["captured_ants"],
                                   "lts_throughput_pct": rec.get("lts_throughput_pct"),
                                   "note": "bytes scaled to m ants; the percentage is the "
                                           "captured launch's own"}
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
        "gpu_launches": launches * steps,
        "clocks": clk,
        "e2e": e2e,
    }
    if batched is not None:
        line["batched"] = {k: batched[k] for k in (
            "value", "unit", "ms_per_step", "per_instance_loop_solves_per_s", "speedup_vs_loop",
            "identical_best_lengths", "ant_steps_per_s", "gpu_launches", "clocks")}
        line["batched"]["config"] = batched["config"]
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)


CONSTRUCT_SOURCES = ("aco_device.cuh", "construct.cuh", "construct_chunks.h", "construct_dispatch.cuh",
                     "construct_phased.cuh", "construct_g1h8.cu", "construct_g1h16.cu", "construct_g1h32.cu",
                     "construct_g2h32.cu", "construct_g4h32.cu", "construct_rule.cuh",
                     "construct_rule1.cu", "construct_rule2.cu")


def construct_sources_sha256() -> str:
    """SHA-256 over the construction kernel's sources, in a fixed order."""
    import hashlib
    h = hashlib.sha256()
    for f in CONSTRUCT_SOURCES:
        with open(os.path.join(ROOT, "paper_1101_2678_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(workload: str, m: int):
    """Memory traffic per construct launch from a committed ncu capture.

    The summaries under profiles/ carry a line
    `traffic-record: workload=<name> ants=<a> dram_bytes_per_launch=<B>
    l2_bytes_per_launch=<L> lts_throughput_pct=<P> sources_sha256=<H>`.
    It is used only if H equals the hash of the current sources (else the
    counters describe another kernel and traffic stays null).  A capture of
    the same kernel with fewer ants (a small case) is scaled to m ants: every
    ant reads its own rows, so the bytes grow in proportion to the ants."""
    import glob
    sha = construct_sources_sha256()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "construct_kernel_*.md"))):
        with open(path) as fh:
            for line in fh:
                if not line.startswith("traffic-record:"):
                    continue
                kv = dict(x.split("=", 1) for x in line.split()[1:])
                if kv.get("workload") != workload or kv.get("sources_sha256") != sha:
                    continue
                ants = int(kv.get("ants", m))
                scale = m / ants
                rec = {"source": os.path.relpath(path, ROOT), "captured_ants": ants,
                       "dram_bytes_per_launch": float(kv["dram_bytes_per_launch"]) * scale}
                if "l2_bytes_per_launch" in kv:
                    rec["l2_bytes_per_launch"] = float(kv["l2_bytes_per_launch"]) * scale
                if "lts_throughput_pct" in kv:
                    rec["lts_throughput_pct"] = float(kv["lts_throughput_pct"])
                return rec
    return None


def construct_roofline(n, m, con_ms, l2, peaks, peak_kind, kernel="construct_kernel", nn=0):
    """Roofline entry for the construction kernel (the dominant kernel).

    Algorithmic bytes per launch: every ant reads, at each of its n-1 steps,
    the 4-byte choice_info entries of the cities it has not visited yet:
    4 * m * sum_{s=1}^{n-1} (n - s) = 4 m n (n-1) / 2.  With nearest-neighbour
    lists a step needs the current city's nn list entries and their
    list-ordered choice_info values: 8 * nn bytes, m (n-1) steps.  The matrix
    stays in L2, so the ceiling is the read-only L2 bandwidth measured in this
    run; the HBM copy peak is given beside it for reference."""
    if nn:
        algo = 8.0 * nn * m * (n - 1)
        dense = 256.0 * m * (n - 1)  # one 128-byte line of values plus the list row
    else:
        algo = 4.0 * m * n * (n - 1) / 2.0
        dense = 4.0 * m * (n - 1) * ((n + 3) // 4 * 4)  # whole padded rows, as staged
    achieved = algo / (con_ms / 1e3) / 1e9
    peak = float(l2["peak"])
    hbm = float(peaks["hbm_gbs"])
    return {"bound": "l2", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None,
            "peak_kind": "read-only L2 bandwidth measured in this run (" + l2["how"] + ")",
            "l2_read_gbs": {"float4": l2["float4"], "bulk": l2["bulk"]},
            "kernel": kernel, "algorithmic_bytes_per_launch": algo,
            "staged_bytes_per_launch": dense,
            "achieved_staged": dense / (con_ms / 1e3) / 1e9,
            "frac_staged": dense / (con_ms / 1e3) / 1e9 / peak,
            "hbm": {"peak": hbm, "peak_kind": f"{peak_kind} HBM copy bandwidth",
                    "frac": achieved / hbm},
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
    line = batched_measure(args, rank, world, local)
    if line is not None:
        print(json.dumps(line), flush=True)


def batched_measure(args, rank, world, local):
    """The batched line's fields (rank 0; None on the other ranks)."""
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
    if args.single_launch:
        aco.aco_pool_set_single_launch(b, True)
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
    return line


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
    loop_lens, loop_times = [], []
    for r in sample:
        t1 = time.perf_counter()
        h = aco.aco_create_coords(r.coords, r.alpha, r.beta, r.rho, r.m, r.seed)
        if r.nn:
            aco.aco_set_option(h, aco.ACO_OPT_NN_LIST, r.nn)
        aco.aco_iterate(h, r.iterations)
        loop_lens.append(aco.aco_best_tour(h, r.n)[1])
        aco.aco_destroy(h)
        loop_times.append(time.perf_counter() - t1)
    t_loop = sum(loop_times)
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
            "loop_seconds_per_request": [round(x, 4) for x in loop_times],
            "request_n": [r.n for r in sample],
            # A request in the mix runs no faster than alone, so the server's
            # makespan on the sample is at least the longest request's time:
            # its speedup over the loop cannot exceed sum / max.
            "makespan_bound_speedup": t_loop / max(loop_times),
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
        # throughput against the loop on the stream's own request mix (the
        # loop's rate from the timed sample)
        "saturated_vs_loop": (st["solves_per_s"] / (len(sample) / t_loop)) if sample else None,
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
