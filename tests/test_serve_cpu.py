"""Host logic of the solve server (serve.Server) on the CPU.

The server only decides which request enters which pool slot and when; the
pool itself is replaced here by a fake with the same calls, so admission
order, the step-work bound, the HBM budget, rule switches, deadlines and the
statistics are checked without a GPU.
"""
import numpy as np
import pytest

from paper_1101_2678_gb300 import serve


class FakePool:
    """Slots with an iteration budget; one iteration per step."""

    def __init__(self, max_slots, budget):
        self.max_slots, self.budget, self.used = max_slots, budget, 0
        self.slots = {}      # slot -> dict(n, left, bytes, rule)
        self.finished = []
        self.log = []        # ("admit", n) / ("step", live slots) / ("rule", slot, name)
        self.multirate = False

    def bytes_of(self, n):
        return 16 * n * n


class FakeAco:
    def __init__(self):
        self.pools = []

    def aco_pool_create(self, max_slots, budget):
        p = FakePool(max_slots, budget)
        self.pools.append(p)
        return p

    def aco_pool_destroy(self, p):
        p.slots.clear()

    def aco_pool_set_multirate(self, p, on):
        p.multirate = bool(on)

    def aco_pool_admit_coords(self, p, coords, alpha, beta, rho, m, seed, iterations):
        n = len(coords)
        b = p.bytes_of(n)
        free = [s for s in range(p.max_slots) if s not in p.slots and s not in p.finished]
        if not free or p.used + b > p.budget:
            return None
        s = free[0]
        p.slots[s] = dict(n=n, left=iterations, bytes=b, rule="as", seed=seed)
        p.used += b
        p.log.append(("admit", n))
        return s

    def aco_pool_set_acs(self, p, slot, q0, xi):
        p.slots[slot]["rule"] = "acs"
        p.log.append(("rule", slot, "acs"))

    def aco_pool_set_mmas(self, p, slot, p_best, best_so_far):
        p.slots[slot]["rule"] = "mmas"
        p.log.append(("rule", slot, "mmas"))

    def aco_pool_set_nn(self, p, slot, nn):
        p.slots[slot]["nn"] = nn
        p.log.append(("rule", slot, f"nn{nn}"))

    def aco_pool_stats(self, p):
        return dict(live=len(p.slots), finished=len(p.finished), bytes_in_use=p.used,
                    launches_last_step=1)

    def aco_pool_step(self, p):
        p.log.append(("step", sorted(sl["n"] for s, sl in p.slots.items()
                                     if s not in p.finished)))
        p.nsteps = getattr(p, "nsteps", 0) + 1
        for s in list(p.slots):
            p.slots[s]["left"] -= 1
            if p.slots[s]["left"] == 0:
                p.finished.append(s)
                p.slots[s]["finish_step"] = p.nsteps
        return sum(1 for s in p.slots if s not in p.finished)

    def aco_pool_finished(self, p):
        return list(p.finished)

    def aco_pool_result(self, p, slot, n):
        sl = p.slots[slot]
        p.log.append(("result", sl["finish_step"], p.nsteps))
        return np.arange(n + 1, dtype=np.int32) % n, 1000 * sl["n"] + sl["seed"]

    def aco_pool_release(self, p, slot):
        p.used -= p.slots[slot]["bytes"]
        del p.slots[slot]
        p.finished.remove(slot)

    def aco_pool_synchronize(self, p):
        pass


@pytest.fixture
def fake(monkeypatch):
    f = FakeAco()
    monkeypatch.setattr(serve, "aco", f)
    return f


def req(n, iterations=3, seed=0, **kw):
    return serve.Request(np.zeros((n, 2), np.int32), m=min(n, 64), iterations=iterations,
                         seed=seed, **kw)


def test_every_request_completes_in_arrival_order_of_admission(fake):
    reqs = [req(n, 2 + i % 3, seed=i) for i, n in enumerate([50, 80, 30, 120, 60, 40])]
    arrivals = np.array([0.5, 0.1, 0.3, 0.2, 0.4, 0.0])
    with serve.Server(budget_bytes=1 << 30, max_slots=4, max_step_work=10**12) as srv:
        outs, st = srv.run(reqs, arrivals, realtime=False)
    pool = fake.pools[0]
    admitted = [e[1] for e in pool.log if e[0] == "admit"]
    order = np.argsort(arrivals, kind="stable")
    assert admitted == [reqs[i].n for i in order]
    assert st["completed"] == len(reqs) and st["backlog"] == 0 and st["still_live"] == 0
    assert sorted(o.index for o in outs) == list(range(len(reqs)))
    for o in outs:
        assert o.best_len == 1000 * reqs[o.index].n + reqs[o.index].seed
        assert o.finished >= o.admitted >= 0
    assert st["max_live"] <= 4


def test_step_work_bound_and_oversized_request(fake):
    # step_work = m n^2; the bound admits two 100-city requests (m = 64) at a
    # time, and a request above the bound runs alone
    small = [req(100, 2, seed=i) for i in range(4)]
    big = req(300, 2, seed=9)
    bound = 2 * serve.step_work(small[0])
    assert serve.step_work(big) > bound
    with serve.Server(budget_bytes=1 << 30, max_slots=8, max_step_work=bound) as srv:
        outs, st = srv.run(small[:2] + [big] + small[2:], np.zeros(5), realtime=False)
    steps = [e[1] for e in fake.pools[0].log if e[0] == "step"]
    assert st["completed"] == 5
    for live in steps:
        assert len(live) <= 2
        assert 300 not in live or live == [300]
    assert [300] in steps


def test_hbm_budget_limits_admission(fake):
    reqs = [req(100, 2, seed=i) for i in range(5)]
    budget = 2 * 16 * 100 * 100  # room for two instances
    with serve.Server(budget_bytes=budget, max_slots=8, max_step_work=10**12) as srv:
        outs, st = srv.run(reqs, np.zeros(5), realtime=False)
    assert st["completed"] == 5 and st["max_live"] == 2
    assert st["hbm_in_use_max_gb"] <= budget / 2**30


def test_rules_and_multirate_reach_the_pool(fake):
    reqs = [req(40, 2, seed=1, variant="acs", q0=0.8, xi=0.2),
            req(50, 2, seed=2, variant="mmas", p_best=0.1, best_so_far=True, nn=16),
            req(60, 2, seed=3)]
    with serve.Server(budget_bytes=1 << 30, max_slots=8, multirate=True) as srv:
        outs, st = srv.run(reqs, np.zeros(3), realtime=False)
    pool = fake.pools[0]
    assert pool.multirate
    rules = [e[2] for e in pool.log if e[0] == "rule"]
    assert sorted(rules) == ["acs", "mmas", "nn16"]
    assert st["completed"] == 3


def test_deadline_stops_with_a_backlog(fake):
    reqs = [req(100, 10**6, seed=i) for i in range(3)]  # never finish
    with serve.Server(budget_bytes=1 << 30, max_slots=1, max_step_work=10**12) as srv:
        outs, st = srv.run(reqs, np.zeros(3), deadline=0.05, realtime=False)
    assert st["completed"] == 0 and st["backlog"] == 3
    assert st["still_live"] == 1 and st["queued"] == 2
    assert st["queue_depth_max"] == 2 and st["steps"] >= 1


def test_live_cap(fake):
    reqs = [req(30, 3, seed=i) for i in range(7)]
    with serve.Server(budget_bytes=1 << 30, max_slots=16, max_step_work=10**12,
                      max_live=3) as srv:
        outs, st = srv.run(reqs, np.zeros(7), realtime=False)
    steps = [e[1] for e in fake.pools[0].log if e[0] == "step"]
    assert st["completed"] == 7 and st["max_live"] == 3
    assert max(len(s) for s in steps) == 3


def test_results_are_read_while_the_next_step_runs(fake):
    # A request's result is read after the following step has been launched
    # (the host stays a step ahead of the device), unless nothing else was
    # left to run; every request is still read exactly once.
    reqs = [req(40 + 10 * i, 2 + i, seed=i) for i in range(5)]
    with serve.Server(budget_bytes=1 << 30, max_slots=8, max_step_work=10**12) as srv:
        outs, st = srv.run(reqs, np.zeros(5), realtime=False)
    pool = fake.pools[0]
    reads = [e for e in pool.log if e[0] == "result"]
    assert st["completed"] == 5 and len(reads) == 5
    last = max(r[1] for r in reads)
    for _, fin, launched in reads:
        if fin < last:
            assert launched == fin + 1   # read once the next step was in flight
        else:
            assert launched == fin       # the final step: nothing left to overlap
