"""Continuous-batching solve server over an aco pool.

Requests (TSP instances given by integer coordinates) arrive over time.  The
server admits them in arrival order whenever the pool has a free slot and
enough of its HBM budget, keeps every admitted instance's state resident on
the device, and runs one iteration for all live instances per step (Ant
System, MAX-MIN Ant System and Ant Colony System requests side by side), so
work from requests that arrived at different times overlaps on the GPU.  A
request finishes after its own number of iterations; its latency is
completion time minus arrival time (queueing included).

All compute happens in the library's kernels (aco_pool_step); this module only
decides which request enters which slot and when.  The host keeps one step
ahead of the device: a step is launched before the results of the previous
step's finished requests are read (each read waits only for the step that
ran the request's last iterations), and admissions and the next step's
graph are prepared while the device runs.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import aco


@dataclass
class Request:
    coords: np.ndarray  # (n, 2) int
    m: int
    iterations: int
    seed: int
    alpha: float = 1.0
    beta: float = 2.0
    rho: float = 0.5
    # "as": the Ant System; "acs": the Ant Colony System with q0 and xi
    # (m <= 32); "mmas": the MAX-MIN Ant System with p_best and best_so_far
    # (rho is then the rule's own rate)
    variant: str = "as"
    q0: float = 0.9
    xi: float = 0.1
    p_best: float = 0.05
    best_so_far: bool = False
    # nearest-neighbour lists of this length (0: every unvisited city); not
    # with the Ant Colony System
    nn: int = 0

    @property
    def n(self) -> int:
        return int(self.coords.shape[0])


@dataclass
class Outcome:
    index: int
    arrival: float
    admitted: float
    finished: float
    best_len: int
    best_tour: np.ndarray = field(repr=False)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def step_work(r: Request) -> int:
    """Candidate evaluations one iteration of request r costs: m ants x n steps x the
    candidates of a step (n cities, or the nn list entries)."""
    return int(r.m) * r.n * (min(r.nn, r.n) if r.nn else r.n)


class Server:
    """Admission is bounded by the pool's HBM budget and by `max_step_work`,
    the candidate evaluations one step may contain (the sum of step_work over
    live requests): a larger batch raises throughput but every live request
    waits for the whole step, so the bound trades throughput for latency.  A
    request larger than the bound is admitted alone.  `max_live` (optional)
    caps the number of live requests as well.  With `multirate`, each
    step runs several iterations of the shorter requests, so they no longer
    wait one step of the longest request per iteration."""

    def __init__(self, budget_bytes: int = 64 << 30, max_slots: int = 2048,
                 max_step_work: int = 20_000_000_000, multirate: bool = False,
                 max_live: int | None = None):
        self.pool = aco.aco_pool_create(max_slots, budget_bytes)
        self.max_live = max_live
        if multirate:
            # short requests run several iterations per step (aco_pool_set_multirate)
            aco.aco_pool_set_multirate(self.pool, True)
        self.budget = budget_bytes
        self.max_slots = max_slots
        self.max_step_work = max_step_work

    def close(self):
        if self.pool is not None:
            aco.aco_pool_destroy(self.pool)
            self.pool = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def run(self, requests, arrivals, deadline: float | None = None, realtime: bool = True):
        """Serve `requests` arriving at `arrivals` (seconds from start).

        realtime=True follows the wall clock (a request is visible once its
        arrival time has passed); realtime=False makes every request available
        immediately in arrival order (a throughput run).  Stops when all
        requests are done or, with `deadline`, at the first step boundary past
        it.  Returns (outcomes, stats)."""
        pool = self.pool
        total = len(requests)
        order = np.argsort(np.asarray(arrivals), kind="stable")
        queue = collections.deque()
        live = {}  # slot -> (request index, admit time)
        live_work = 0
        outcomes = []
        nxt = 0
        steps = 0
        max_live = 0
        # (time, queued, live, HBM bytes in use) about once a second, and
        # per-step queue depth and arena use for the summary
        timeline = []
        next_sample = 0.0
        depth_sum = 0
        depth_max = 0
        bytes_max = 0
        t0 = time.perf_counter()
        seen = set()   # finished slots already noted
        pending = []   # slots whose last step is in flight: read after the next launch

        def drain(slots):
            nonlocal live_work
            for slot in slots:
                ri, tadm = live.pop(slot)
                live_work -= step_work(requests[ri])
                tour, length = aco.aco_pool_result(pool, slot, requests[ri].n)
                tfin = time.perf_counter() - t0
                outcomes.append(Outcome(ri, float(arrivals[ri]), tadm, tfin, length, tour))
                aco.aco_pool_release(pool, slot)
                seen.discard(slot)

        while len(outcomes) < total:
            now = time.perf_counter() - t0
            if deadline is not None and now >= deadline:
                break
            while nxt < total and (not realtime or arrivals[order[nxt]] <= now):
                queue.append(int(order[nxt]))
                nxt += 1
            while queue:
                r = requests[queue[0]]
                w = step_work(r)
                if live and live_work + w > self.max_step_work:
                    break
                if self.max_live is not None and len(live) >= self.max_live:
                    break
                slot = aco.aco_pool_admit_coords(pool, r.coords, r.alpha, r.beta, r.rho, r.m,
                                                 r.seed, r.iterations)
                if slot is None:
                    break
                if r.variant == "acs":
                    aco.aco_pool_set_acs(pool, slot, r.q0, r.xi)
                elif r.variant == "mmas":
                    aco.aco_pool_set_mmas(pool, slot, r.p_best, r.best_so_far)
                if r.nn:
                    aco.aco_pool_set_nn(pool, slot, r.nn)
                live[slot] = (queue.popleft(), time.perf_counter() - t0)
                live_work += w
            running = len(live) - len(pending)
            if running == 0:
                # nothing left to step: collect what the last step finished
                drain(pending)
                pending = []
                if not live and nxt < total:
                    time.sleep(max(0.0, min(0.01, arrivals[order[nxt]] - now)))
                continue
            max_live = max(max_live, running)
            queued_now = len(queue)  # arrived and waiting for admission
            in_use = aco.aco_pool_stats(pool)["bytes_in_use"]
            depth_sum += queued_now
            depth_max = max(depth_max, queued_now)
            bytes_max = max(bytes_max, in_use)
            if now >= next_sample:
                timeline.append([round(now, 3), queued_now, running, round(in_use / 2 ** 30, 3)])
                next_sample = now + 1.0
            aco.aco_pool_step(pool)
            steps += 1
            # the requests that finished in the step before this one: their
            # last step is done or about to be, while this one runs on
            drain(pending)
            pending = [s for s in aco.aco_pool_finished(pool) if s not in seen]
            seen.update(pending)
        drain([s for s in pending if s in live])
        aco.aco_pool_synchronize(pool)
        elapsed = time.perf_counter() - t0
        lat = np.array([o.latency for o in outcomes]) if outcomes else np.zeros(1)
        stats = dict(
            completed=len(outcomes), submitted=nxt, total=total,
            backlog=total - len(outcomes), still_live=len(live), queued=len(queue),
            elapsed_s=elapsed, steps=steps, max_live=max_live,
            solves_per_s=len(outcomes) / elapsed if elapsed > 0 else 0.0,
            p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
            queue_depth_max=depth_max, queue_depth_mean=depth_sum / max(steps, 1),
            hbm_in_use_max_gb=bytes_max / 2 ** 30, timeline=timeline,
        )
        return outcomes, stats
