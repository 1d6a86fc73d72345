"""Many Ant Colony System colonies per launch (aco_pool_admit_acs).

Every live Ant Colony System slot of a pool runs in one launch, one CTA per
colony, beside the Ant System classes.  Each colony keeps its own seed and
iteration counter, and its lockstep steps and local updates stay inside its
own CTA, so a colony's tours, pheromone and best tour must equal the CPU
oracle's run (reading R14) bit for bit in any mix of sizes, ant counts and
admission times.
"""
import numpy as np
import pytest

from paper_1101_2678_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aco():
    from paper_1101_2678_gb300 import build
    build.build()
    from paper_1101_2678_gb300 import aco as a
    a.load()
    return a


def as_alone(aco, dist, m, seed, iters):
    n = dist.shape[0]
    with aco.Colony(dist, m, seed=seed) as c:
        aco.aco_iterate(c.h, iters)
        return aco.aco_get_pheromone(c.h, n), aco.aco_best_tour(c.h, n)


def check_acs_slot(aco, orc, p, slot, dist, m, seed, iters, rho, q0, xi):
    n = dist.shape[0]
    ref = orc.run_acs(dist, m, iters, seed, rho=rho, q0=q0, xi=xi)
    tour, length = aco.aco_pool_result(p, slot, n)
    assert length == ref["best_len"] and np.array_equal(tour, ref["best_tour"]), slot
    assert np.array_equal(aco.aco_pool_pheromone(p, slot, n), ref["tau32"]), slot


def test_mixed_pool_with_staggered_admission(aco, orc):
    # (n, m, seed, iterations, rho, q0, xi) per colony; m from 1 to 32, so the
    # launch's CTA is sized for 32 warps and the others idle through the
    # lockstep barriers
    colonies = [(48, 10, 11, 6, 0.1, 0.9, 0.1), (97, 32, 12, 4, 0.1, 0.5, 0.3),
                (3, 1, 13, 5, 0.2, 0.9, 0.1), (300, 7, 14, 3, 0.1, 0.0, 0.1),
                (31, 16, 15, 7, 0.1, 1.0, 0.2), (130, 10, 16, 2, 0.3, 0.75, 0.1)]
    insts = [I.clustered_instance(c[0], seed=600 + c[0], clusters=5, sigma=150, side=3000)
             for c in colonies]
    as_insts = [I.uniform_instance(n, 1000, seed=700 + n) for n in (200, 64)]
    need = sum(aco.aco_pool_bytes_needed(c[0], c[1]) for c in colonies)
    need += sum(aco.aco_pool_bytes_needed(x.n, x.n) for x in as_insts)
    p = aco.aco_pool_create(16, need + (1 << 20))
    try:
        slots = {}
        sa = aco.aco_pool_admit(p, as_insts[0].dist, 1.0, 2.0, 0.5, 200, 21, 6)
        for i in (0, 1, 2):
            n, m, seed, iters, rho, q0, xi = colonies[i]
            slots[i] = aco.aco_pool_admit_acs(p, insts[i].dist, 1.0, 2.0, rho, m, seed, iters,
                                              q0, xi)
        aco.aco_pool_step(p)
        aco.aco_pool_step(p)
        sb = aco.aco_pool_admit(p, as_insts[1].dist, 1.0, 2.0, 0.5, 64, 22, 3)
        for i in (3, 4, 5):
            n, m, seed, iters, rho, q0, xi = colonies[i]
            slots[i] = aco.aco_pool_admit_acs(p, insts[i].dist, 1.0, 2.0, rho, m, seed, iters,
                                              q0, xi)
        while aco.aco_pool_step(p) > 0:
            pass
        aco.aco_pool_synchronize(p)
        for i, c in enumerate(colonies):
            n, m, seed, iters, rho, q0, xi = c
            check_acs_slot(aco, orc, p, slots[i], insts[i].dist, m, seed, iters, rho, q0, xi)
        for s, x, m, seed, iters in ((sa, as_insts[0], 200, 21, 6), (sb, as_insts[1], 64, 22, 3)):
            tau_a, (tour_a, len_a) = as_alone(aco, x.dist, m, seed, iters)
            tour_p, len_p = aco.aco_pool_result(p, s, x.n)
            assert len_p == len_a and np.array_equal(tour_p, tour_a)
            assert np.array_equal(aco.aco_pool_pheromone(p, s, x.n), tau_a)
    finally:
        aco.aco_pool_destroy(p)


def test_hundreds_of_colonies_in_one_launch(aco, orc):
    # more colonies than the GPU holds CTAs at once (3 per SM at 10 ants)
    count, n, m, iters = 600, 60, 10, 3
    insts = [I.uniform_instance(n, 1000, seed=2000 + i) for i in range(count)]
    p = aco.aco_pool_create(count, count * aco.aco_pool_bytes_needed(n, m) + (1 << 20))
    try:
        slots = [aco.aco_pool_admit_acs(p, x.dist, 1.0, 2.0, 0.1, m, 5000 + i, iters, 0.9, 0.1)
                 for i, x in enumerate(insts)]
        aco.aco_pool_step(p)
        # one construction, one best, one global-update launch for all colonies
        assert aco.aco_pool_stats(p)["launches_last_step"] == 3
        while aco.aco_pool_step(p) > 0:
            pass
        aco.aco_pool_synchronize(p)
        for i in list(range(0, count, 37)) + [count - 1]:
            check_acs_slot(aco, orc, p, slots[i], insts[i].dist, m, 5000 + i, iters, 0.1, 0.9,
                           0.1)
    finally:
        aco.aco_pool_destroy(p)


def test_pool_colony_equals_single_handle_at_full_size(aco):
    w = I.workload_n1002()
    d = w["inst"].dist
    with aco.Colony(d, 10, seed=w["seed"], rho=0.1) as c:
        aco.aco_set_acs(c.h, 0.9, 0.1)
        aco.aco_iterate(c.h, 2)
        tau_h, (tour_h, len_h) = aco.aco_get_pheromone(c.h, 1002), aco.aco_best_tour(c.h, 1002)
    p = aco.aco_pool_create(2, 2 * aco.aco_pool_bytes_needed(1002, 10) + (1 << 20))
    try:
        s = aco.aco_pool_admit_acs(p, d, 1.0, 2.0, 0.1, 10, w["seed"], 2, 0.9, 0.1)
        while aco.aco_pool_step(p) > 0:
            pass
        tour_p, len_p = aco.aco_pool_result(p, s, 1002)
        assert len_p == len_h and np.array_equal(tour_p, tour_h)
        assert np.array_equal(aco.aco_pool_pheromone(p, s, 1002), tau_h)
    finally:
        aco.aco_pool_destroy(p)


def test_acs_admission_errors(aco):
    x = I.uniform_instance(20, 100, seed=1)
    p = aco.aco_pool_create(2, 1 << 24)
    try:
        for kw in [dict(m=33), dict(m=0), dict(q0=1.5), dict(q0=-0.1), dict(xi=2.0),
                   dict(rho=0.0), dict(iterations=0)]:
            args = dict(alpha=1.0, beta=2.0, rho=0.1, m=10, seed=1, iterations=2, q0=0.9, xi=0.1)
            args.update(kw)
            with pytest.raises(aco.AcoError) as e:
                aco.aco_pool_admit_acs(p, x.dist, **args)
            assert e.value.code == aco.ACO_EINVAL
        s = aco.aco_pool_admit_acs(p, x.dist, 1.0, 2.0, 0.1, 10, 1, 2, 0.9, 0.1)
        aco.aco_pool_step(p)
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_tiling(p, s)
        assert e.value.code == aco.ACO_EINVAL
    finally:
        aco.aco_pool_destroy(p)


def test_server_mixes_ant_system_and_colony_system_requests(aco, orc):
    # Requests of both update rules through serve.Server, by coordinates, in a
    # step-work budget small enough to stagger admission; each Ant Colony
    # System result equals the oracle's run, each Ant System result its run
    # alone.
    from paper_1101_2678_gb300 import serve
    reqs = []
    for i, (n, variant) in enumerate([(90, "acs"), (300, "as"), (48, "acs"), (200, "acs"),
                                      (150, "as"), (33, "acs")]):
        inst = I.clustered_instance(n, seed=90 + i, clusters=6, side=4000)
        if variant == "acs":
            reqs.append(serve.Request(inst.coords, m=10 + i, iterations=3 + i, seed=850 + i,
                                      rho=0.1, variant="acs", q0=0.9, xi=0.1))
        else:
            reqs.append(serve.Request(inst.coords, m=min(n, 128), iterations=3 + i,
                                      seed=850 + i))
    arrivals = np.array([0.001 * i for i in range(len(reqs))])
    with serve.Server(budget_bytes=1 << 30, max_slots=8, max_step_work=300 * 300 * 128) as srv:
        outs, st = srv.run(reqs, arrivals, realtime=False)
    assert st["completed"] == len(reqs) and st["backlog"] == 0
    for o in outs:
        r = reqs[o.index]
        d = I.distance_matrix(r.coords)
        if r.variant == "acs":
            ref = orc.run_acs(d, r.m, r.iterations, r.seed, rho=r.rho, q0=r.q0, xi=r.xi)
            assert o.best_len == ref["best_len"], o.index
            assert np.array_equal(o.best_tour, ref["best_tour"]), o.index
        else:
            with aco.Colony(d, r.m, seed=r.seed) as c:
                aco.aco_iterate(c.h, r.iterations)
                tour, length = aco.aco_best_tour(c.h, r.n)
            assert o.best_len == length and np.array_equal(o.best_tour, tour), o.index
