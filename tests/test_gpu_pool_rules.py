"""The Ant Colony System and the MAX-MIN Ant System in a pool
(aco_pool_set_acs / aco_pool_set_mmas).

Every live Ant Colony System slot of a pool runs in one launch, one CTA per
colony, beside the Ant System classes; MAX-MIN slots construct with the Ant
System slots and take their own update in the row-update launch.  Each slot
keeps its own seed and iteration counter, and nothing of one slot's step
reads another slot's state, so a slot's tours, pheromone and best tour must
equal the CPU oracle's run (readings R13 and R14) bit for bit in any mix of
sizes, ant counts, rules and admission times.
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
        # the rule is chosen once, before the slot's first step
        for call in (lambda: aco.aco_pool_set_acs(p, s, 0.9, 0.1),
                     lambda: aco.aco_pool_set_mmas(p, s, 0.05, False)):
            with pytest.raises(aco.AcoError) as e:
                call()
            assert e.value.code == aco.ACO_ESTATE
        s2 = aco.aco_pool_admit(p, x.dist, 1.0, 2.0, 0.1, 10, 2, 2)
        for kw in [dict(p_best=0.0), dict(p_best=1.0), dict(best_so_far=2)]:
            args = dict(p_best=0.05, best_so_far=0)
            args.update(kw)
            with pytest.raises(aco.AcoError) as e:
                aco.aco_pool_set_mmas(p, s2, **args)
            assert e.value.code == aco.ACO_EINVAL
        aco.aco_pool_step(p)
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_set_mmas(p, s2, 0.05, False)
        assert e.value.code == aco.ACO_ESTATE
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_tiling(p, s)
        assert e.value.code == aco.ACO_EINVAL
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_set_acs(p, 7, 0.9, 0.1)
        assert e.value.code == aco.ACO_EINVAL
    finally:
        aco.aco_pool_destroy(p)


def check_mmas_slot(aco, orc, p, slot, dist, m, seed, iters, rho, p_best, bsf):
    n = dist.shape[0]
    ref = orc.run_mmas(dist, m, iters, seed, rho=rho, p_best=p_best, best_so_far=bsf)
    tour, length = aco.aco_pool_result(p, slot, n)
    assert length == ref["best_len"] and np.array_equal(tour, ref["best_tour"]), slot
    assert np.array_equal(aco.aco_pool_pheromone(p, slot, n), ref["tau32"]), slot


def test_all_three_rules_in_one_pool(aco, orc):
    # MAX-MIN slots (both deposit choices) share construction classes with
    # Ant System slots of similar n; Ant Colony System colonies run beside them
    mm = [(48, 48, 31, 6, 0.02, 0.05, False), (300, 100, 32, 3, 0.1, 0.05, True),
          (97, 97, 33, 5, 0.2, 0.3, False), (3, 3, 34, 4, 0.02, 0.05, True)]
    ac = [(60, 10, 41, 5, 0.1, 0.9, 0.1), (250, 32, 42, 3, 0.1, 0.5, 0.2)]
    asys = [(290, 120, 51, 4), (50, 50, 52, 6)]
    inst = {}
    for n, *_r in mm + ac + asys:
        inst[n] = I.uniform_instance(n, 1000, seed=3000 + n)
    need = sum(aco.aco_pool_bytes_needed(c[0], c[1]) for c in mm + ac + asys)
    p = aco.aco_pool_create(16, need + (1 << 20))
    try:
        slot = {}
        for i, (n, m, seed, iters, rho, pb, bsf) in enumerate(mm):
            slot["mm", i] = aco.aco_pool_admit_mmas(p, inst[n].dist, 1.0, 2.0, rho, m, seed,
                                                    iters, pb, bsf)
            if i == 1:
                for j, (n2, m2, seed2, iters2) in enumerate(asys):
                    slot["as", j] = aco.aco_pool_admit(p, inst[n2].dist, 1.0, 2.0, 0.5, m2,
                                                       seed2, iters2)
                aco.aco_pool_step(p)
        for i, (n, m, seed, iters, rho, q0, xi) in enumerate(ac):
            slot["ac", i] = aco.aco_pool_admit_acs(p, inst[n].dist, 1.0, 2.0, rho, m, seed, iters,
                                                   q0, xi)
        while aco.aco_pool_step(p) > 0:
            pass
        aco.aco_pool_synchronize(p)
        for i, (n, m, seed, iters, rho, pb, bsf) in enumerate(mm):
            check_mmas_slot(aco, orc, p, slot["mm", i], inst[n].dist, m, seed, iters, rho, pb, bsf)
        for i, (n, m, seed, iters, rho, q0, xi) in enumerate(ac):
            check_acs_slot(aco, orc, p, slot["ac", i], inst[n].dist, m, seed, iters, rho, q0, xi)
        for j, (n, m, seed, iters) in enumerate(asys):
            ref = orc.run(inst[n].dist, m, iters, seed)
            assert np.array_equal(aco.aco_pool_pheromone(p, slot["as", j], n), ref["tau32"])
            assert aco.aco_pool_result(p, slot["as", j], n)[1] == ref["best_len"]
    finally:
        aco.aco_pool_destroy(p)


def test_pool_mmas_equals_single_handle_at_full_size(aco):
    w = I.workload_n1002()
    d = w["inst"].dist
    with aco.Colony(d, 256, seed=w["seed"], rho=0.02) as c:
        aco.aco_set_mmas(c.h, 0.05, False)
        aco.aco_iterate(c.h, 3)
        tau_h, (tour_h, len_h) = aco.aco_get_pheromone(c.h, 1002), aco.aco_best_tour(c.h, 1002)
    p = aco.aco_pool_create(2, 2 * aco.aco_pool_bytes_needed(1002, 256) + (1 << 20))
    try:
        s = aco.aco_pool_admit_mmas(p, d, 1.0, 2.0, 0.02, 256, w["seed"], 3, 0.05, False)
        while aco.aco_pool_step(p) > 0:
            pass
        tour_p, len_p = aco.aco_pool_result(p, s, 1002)
        assert len_p == len_h and np.array_equal(tour_p, tour_h)
        assert np.array_equal(aco.aco_pool_pheromone(p, s, 1002), tau_h)
    finally:
        aco.aco_pool_destroy(p)


def test_server_mixes_all_three_rules(aco, orc):
    # Requests of the three update rules through serve.Server, by
    # coordinates, in a step-work budget small enough to stagger admission;
    # each Ant Colony System and MAX-MIN result equals the oracle's run, each
    # Ant System result its run alone.
    from paper_1101_2678_gb300 import serve
    reqs = []
    for i, (n, variant) in enumerate([(90, "acs"), (300, "as"), (48, "acs"), (200, "mmas"),
                                      (150, "as"), (33, "acs"), (120, "mmas")]):
        inst = I.clustered_instance(n, seed=90 + i, clusters=6, side=4000)
        if variant == "acs":
            reqs.append(serve.Request(inst.coords, m=10 + i, iterations=3 + i, seed=850 + i,
                                      rho=0.1, variant="acs", q0=0.9, xi=0.1))
        elif variant == "mmas":
            reqs.append(serve.Request(inst.coords, m=min(n, 128), iterations=3 + i,
                                      seed=850 + i, rho=0.02, variant="mmas", p_best=0.05,
                                      best_so_far=i % 2 == 1))
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
        if r.variant in ("acs", "mmas"):
            ref = (orc.run_acs(d, r.m, r.iterations, r.seed, rho=r.rho, q0=r.q0, xi=r.xi)
                   if r.variant == "acs" else
                   orc.run_mmas(d, r.m, r.iterations, r.seed, rho=r.rho, p_best=r.p_best,
                                best_so_far=r.best_so_far))
            assert o.best_len == ref["best_len"], o.index
            assert np.array_equal(o.best_tour, ref["best_tour"]), o.index
        else:
            with aco.Colony(d, r.m, seed=r.seed) as c:
                aco.aco_iterate(c.h, r.iterations)
                tour, length = aco.aco_best_tour(c.h, r.n)
            assert o.best_len == length and np.array_equal(o.best_tour, tour), o.index


def test_multirate_steps_keep_every_result(aco, orc):
    # One long instance (n = 1000) beside short ones of all three rules:
    # with multi-rate stepping the short groups run several iterations per
    # step, finish in fewer steps, and every slot still equals its run alone.
    big = I.uniform_instance(1000, 1000, seed=4100)
    small = [(60, "as", 60, 31, 30), (48, "mmas", 48, 32, 25), (90, "acs", 10, 33, 20),
             (130, "as", 64, 34, 12)]
    insts = {n: I.uniform_instance(n, 1000, seed=4100 + n) for n, *_r in small}
    need = aco.aco_pool_bytes_needed(1000, 256) + sum(
        aco.aco_pool_bytes_needed(n, m) for n, _v, m, *_r in small)
    p = aco.aco_pool_create(8, need + (1 << 20))
    try:
        aco.aco_pool_set_multirate(p, True)
        sb = aco.aco_pool_admit(p, big.dist, 1.0, 2.0, 0.5, 256, 30, 4)
        slots = {}
        for n, variant, m, seed, iters in small:
            if variant == "acs":
                slots[n] = aco.aco_pool_admit_acs(p, insts[n].dist, 1.0, 2.0, 0.1, m, seed,
                                                  iters, 0.9, 0.1)
            elif variant == "mmas":
                slots[n] = aco.aco_pool_admit_mmas(p, insts[n].dist, 1.0, 2.0, 0.02, m, seed,
                                                   iters, 0.05, False)
            else:
                slots[n] = aco.aco_pool_admit(p, insts[n].dist, 1.0, 2.0, 0.5, m, seed, iters)
        steps = 0
        aco.aco_pool_step(p)
        steps += 1
        rates = {n: aco.aco_pool_rate(p, s) for n, s in slots.items()}
        assert aco.aco_pool_rate(p, sb) == 1
        assert all(k > 1 for k in rates.values()), rates
        while aco.aco_pool_step(p) > 0:
            steps += 1
        steps += 1
        # one iteration per step would take 30 steps (the longest budget);
        # the colony group runs 3 per step beside the long instance and one
        # per step once it is alone
        assert steps < 20, steps
        aco.aco_pool_synchronize(p)
        for n, variant, m, seed, iters in small:
            d = insts[n].dist
            if variant == "acs":
                ref = orc.run_acs(d, m, iters, seed, rho=0.1, q0=0.9, xi=0.1)
            elif variant == "mmas":
                ref = orc.run_mmas(d, m, iters, seed, rho=0.02, p_best=0.05)
            else:
                ref = orc.run(d, m, iters, seed)
            assert np.array_equal(aco.aco_pool_pheromone(p, slots[n], n), ref["tau32"]), n
            assert aco.aco_pool_result(p, slots[n], n)[1] == ref["best_len"], n
        tau_a, (tour_a, len_a) = as_alone(aco, big.dist, 256, 30, 4)
        assert np.array_equal(aco.aco_pool_pheromone(p, sb, 1000), tau_a)
        assert aco.aco_pool_result(p, sb, 1000)[1] == len_a
    finally:
        aco.aco_pool_destroy(p)


def test_multirate_rate_never_exceeds_the_budget_left(aco, orc):
    # a short instance with 5 iterations beside a long one: its rate is
    # capped at 5, so it finishes after one step and runs exactly 5
    big = I.uniform_instance(700, 1000, seed=4200)
    x = I.uniform_instance(40, 1000, seed=4201)
    p = aco.aco_pool_create(4, aco.aco_pool_bytes_needed(700, 128) +
                            aco.aco_pool_bytes_needed(40, 40) + (1 << 20))
    try:
        aco.aco_pool_set_multirate(p, True)
        aco.aco_pool_admit(p, big.dist, 1.0, 2.0, 0.5, 128, 1, 3)
        s = aco.aco_pool_admit(p, x.dist, 1.0, 2.0, 0.5, 40, 2, 5)
        aco.aco_pool_step(p)
        assert aco.aco_pool_finished(p) == [s]
        ref = orc.run(x.dist, 40, 5, 2)
        assert np.array_equal(aco.aco_pool_pheromone(p, s, 40), ref["tau32"])
        assert aco.aco_pool_rate(p, s) == 5
        s2 = aco.aco_pool_admit(p, x.dist, 1.0, 2.0, 0.5, 40, 3, 2)
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_rate(p, s2)  # no step yet
        assert e.value.code == aco.ACO_ESTATE
    finally:
        aco.aco_pool_destroy(p)
    b = aco.aco_batch_create([x.dist], [40], [2])
    try:
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_set_multirate(b, True)
        assert e.value.code == aco.ACO_EINVAL
    finally:
        aco.aco_batch_destroy(b)


def nn_alone(aco, dist, m, seed, iters, nn, rho=0.5, mmas=False):
    n = dist.shape[0]
    with aco.Colony(dist, m, seed=seed, rho=rho) as c:
        if mmas:
            aco.aco_set_mmas(c.h, 0.05, False)
        aco.aco_set_option(c.h, aco.ACO_OPT_NN_LIST, nn)
        aco.aco_iterate(c.h, iters)
        return aco.aco_get_pheromone(c.h, n), aco.aco_best_tour(c.h, n)


@pytest.mark.parametrize("multirate", [False, True])
def test_nn_list_slots_equal_their_handle_runs(aco, orc, multirate):
    # list slots of several sizes and list lengths (one with the MAX-MIN
    # update) beside dense Ant System slots and a colony; each equals its
    # handle run with ACO_OPT_NN_LIST, and the smallest the oracle's run
    cases = [(10, 9, 12, 5, 41, False), (300, 30, 64, 4, 42, False), (130, 20, 60, 6, 43, True),
             (700, 32, 40, 3, 44, False)]
    insts = {n: I.clustered_instance(n, seed=n + 7, clusters=6, side=4000) for n, *_r in cases}
    dense = I.uniform_instance(200, 1000, seed=46)
    colony = I.uniform_instance(60, 1000, seed=47)
    need = sum(aco.aco_pool_bytes_needed(n, m) for n, _nn, m, *_r in cases)
    need += aco.aco_pool_bytes_needed(200, 100) + aco.aco_pool_bytes_needed(60, 10)
    p = aco.aco_pool_create(8, need + (1 << 20))
    try:
        aco.aco_pool_set_multirate(p, multirate)
        slots = {}
        for n, nn, m, iters, seed, mmas in cases:
            rho = 0.02 if mmas else 0.5
            slots[n] = aco.aco_pool_admit(p, insts[n].dist, 1.0, 2.0, rho, m, seed, iters)
            if mmas:
                aco.aco_pool_set_mmas(p, slots[n], 0.05, False)
            aco.aco_pool_set_nn(p, slots[n], nn)
        sd = aco.aco_pool_admit(p, dense.dist, 1.0, 2.0, 0.5, 100, 48, 4)
        sc = aco.aco_pool_admit_acs(p, colony.dist, 1.0, 2.0, 0.1, 10, 49, 5, 0.9, 0.1)
        while aco.aco_pool_step(p) > 0:
            pass
        aco.aco_pool_synchronize(p)
        for n, nn, m, iters, seed, mmas in cases:
            tau_a, (tour_a, len_a) = nn_alone(aco, insts[n].dist, m, seed, iters, nn,
                                              rho=0.02 if mmas else 0.5, mmas=mmas)
            assert np.array_equal(aco.aco_pool_pheromone(p, slots[n], n), tau_a), n
            tour_p, len_p = aco.aco_pool_result(p, slots[n], n)
            assert len_p == len_a and np.array_equal(tour_p, tour_a), n
        ref = orc.run(insts[10].dist, 12, 5, 41, rule=2, nn=9)
        assert np.array_equal(aco.aco_pool_pheromone(p, slots[10], 10), ref["tau32"])
        tau_a, (_, len_a) = as_alone(aco, dense.dist, 100, 48, 4)
        assert np.array_equal(aco.aco_pool_pheromone(p, sd, 200), tau_a)
        check_acs_slot(aco, orc, p, sc, colony.dist, 10, 49, 5, 0.1, 0.9, 0.1)
    finally:
        aco.aco_pool_destroy(p)


def test_nn_list_slot_errors(aco):
    x = I.uniform_instance(40, 1000, seed=9)
    p = aco.aco_pool_create(4, 4 * aco.aco_pool_bytes_needed(40, 10) + (1 << 20))
    try:
        s = aco.aco_pool_admit(p, x.dist, 1.0, 2.0, 0.5, 10, 1, 3)
        for bad in (-1, 33):
            with pytest.raises(aco.AcoError) as e:
                aco.aco_pool_set_nn(p, s, bad)
            assert e.value.code == aco.ACO_EINVAL
        aco.aco_pool_set_nn(p, s, 8)
        aco.aco_pool_step(p)
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_set_nn(p, s, 4)
        assert e.value.code == aco.ACO_ESTATE
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_tiling(p, s)
        assert e.value.code == aco.ACO_EINVAL
    finally:
        aco.aco_pool_destroy(p)


@pytest.mark.parametrize("multirate", [False, True])
def test_colonies_with_lists_in_a_pool(aco, orc, multirate):
    # colonies with and without lists in one pool (two colony launches per
    # step), lists set before or after the switch, with and without
    # multi-rate stepping: each equals the oracle's R16 / R14 run
    cases = [(60, 10, 8, 5, 51, True), (97, 16, 20, 4, 52, False), (130, 10, 0, 4, 53, True),
             (40, 8, 12, 6, 54, False)]
    insts = {n: I.clustered_instance(n, seed=n + 11, clusters=5, sigma=150, side=3000)
             for n, *_r in cases}
    need = sum(aco.aco_pool_bytes_needed(n, m) for n, m, *_r in cases)
    p = aco.aco_pool_create(8, need + (1 << 20))
    try:
        aco.aco_pool_set_multirate(p, multirate)
        slots = {}
        for n, m, nn, iters, seed, lists_first in cases:
            s = aco.aco_pool_admit(p, insts[n].dist, 1.0, 2.0, 0.1, m, seed, iters)
            if nn and lists_first:
                aco.aco_pool_set_nn(p, s, nn)
            aco.aco_pool_set_acs(p, s, 0.9, 0.1)
            if nn and not lists_first:
                aco.aco_pool_set_nn(p, s, nn)
            slots[n] = s
        aco.aco_pool_step(p)
        if not multirate:
            assert aco.aco_pool_stats(p)["launches_last_step"] == 4
        while aco.aco_pool_step(p) > 0:
            pass
        aco.aco_pool_synchronize(p)
        for n, m, nn, iters, seed, _ in cases:
            ref = orc.run_acs(insts[n].dist, m, iters, seed, rho=0.1, q0=0.9, xi=0.1, nn=nn)
            assert np.array_equal(aco.aco_pool_pheromone(p, slots[n], n), ref["tau32"]), n
            tour, length = aco.aco_pool_result(p, slots[n], n)
            assert length == ref["best_len"] and np.array_equal(tour, ref["best_tour"]), n
    finally:
        aco.aco_pool_destroy(p)


@pytest.mark.parametrize("lists_first", [True, False])
def test_max_min_list_slot_either_order_matches_oracle(aco, orc, lists_first):
    # Lists set before or after the MAX-MIN switch: the slot's first tours
    # come from the list-ordered choice_info of the tau_max trails, so the
    # run equals the oracle's MAX-MIN run with lists (readings R13 + R9).
    n, m, nn, iters, seed = 150, 40, 16, 5, 61
    x = I.clustered_instance(n, seed=67, clusters=6, side=4000)
    p = aco.aco_pool_create(2, aco.aco_pool_bytes_needed(n, m) + (1 << 20))
    try:
        s = aco.aco_pool_admit(p, x.dist, 1.0, 2.0, 0.02, m, seed, iters)
        if lists_first:
            aco.aco_pool_set_nn(p, s, nn)
        aco.aco_pool_set_mmas(p, s, 0.05, False)
        if not lists_first:
            aco.aco_pool_set_nn(p, s, nn)
        while aco.aco_pool_step(p) > 0:
            pass
        aco.aco_pool_synchronize(p)
        ref = orc.run_mmas(x.dist, m, iters, seed, rho=0.02, p_best=0.05, rule=2, nn=nn)
        assert np.array_equal(aco.aco_pool_pheromone(p, s, n), ref["tau32"])
        tour, length = aco.aco_pool_result(p, s, n)
        assert length == ref["best_len"] and np.array_equal(tour, ref["best_tour"])
    finally:
        aco.aco_pool_destroy(p)
