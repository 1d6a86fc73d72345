"""Batched and served instances (aco_pool_* / aco_batch_*) on the GPU.

Every instance in a pool keeps its own seed and iteration counter, and the
pool uses the deterministic gather deposit, so an instance's pheromone and
best tour must be identical bit for bit whether it runs alone, in a static
batch, or admitted mid-stream next to other instances of different sizes.
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


def alone(aco, dist, m, seed, iters):
    n = dist.shape[0]
    with aco.Colony(dist, m, seed=seed) as c:
        aco.aco_iterate(c.h, iters)
        return aco.aco_get_pheromone(c.h, n), aco.aco_best_tour(c.h, n)


def test_static_batch_equals_alone(aco, orc):
    ns = [48, 300, 97, 1024, 5, 130, 517]
    insts = [I.uniform_instance(n, 1000, seed=500 + n) for n in ns]
    ms = [n if n < 1000 else 200 for n in ns]
    seeds = [900 + i for i in range(len(ns))]
    b = aco.aco_batch_create([x.dist for x in insts], ms, seeds)
    try:
        aco.aco_batch_iterate(b, 6)
        for i, x in enumerate(insts):
            tau_a, (tour_a, len_a) = alone(aco, x.dist, ms[i], seeds[i], 6)
            tour_b, len_b = aco.aco_batch_best(b, i, x.n)
            assert len_b == len_a and np.array_equal(tour_b, tour_a), i
            assert np.array_equal(aco.aco_pool_pheromone(b, i, x.n), tau_a), i
    finally:
        aco.aco_batch_destroy(b)
    # and the oracle agrees for the small ones
    for i in [0, 4]:
        ref = orc.run(insts[i].dist, ms[i], 6, seeds[i])
        tau_a, (_, len_a) = alone(aco, insts[i].dist, ms[i], seeds[i], 6)
        assert np.array_equal(tau_a, ref["tau32"]) and len_a == ref["best_len"]


def test_compacting_pool_zero_weights_equal_alone(aco, orc):
    # rho = 1 leaves pheromone only on the last iteration's edges, so the
    # compacted phases of the pool's construction (city-index list entries,
    # one and two warps per ant) often meet the zero-weight rule; every
    # instance must still match its run alone, and the smallest the oracle
    ns = [520, 900, 1000, 2500]
    insts = [I.clustered_instance(n, seed=40 + n, clusters=10, sigma=300, side=20000) for n in ns]
    ms = [24] * len(ns)
    seeds = [70 + i for i in range(len(ns))]
    b = aco.aco_batch_create([x.dist for x in insts], ms, seeds, rho=1.0)
    try:
        aco.aco_pool_set_autotune(b, False)  # default tilings: the compacting walk
        aco.aco_batch_iterate(b, 3)
        for i, x in enumerate(insts):
            g, h, c, _ = aco.aco_pool_tiling(b, i)
            assert c >= 20 and (g, h) == ((1, 32) if x.n <= 2432 else (2, 32)), (i, g, h, c)
            with aco.Colony(x.dist, ms[i], seed=seeds[i], rho=1.0) as col:
                aco.aco_iterate(col.h, 3)
                tau_a = aco.aco_get_pheromone(col.h, x.n)
                tour_a, len_a = aco.aco_best_tour(col.h, x.n)
            tau_b = aco.aco_pool_pheromone(b, i, x.n)
            assert (tau_b == 0).mean() > 0.85, i
            tour_b, len_b = aco.aco_batch_best(b, i, x.n)
            assert len_b == len_a and np.array_equal(tour_b, tour_a), i
            assert np.array_equal(tau_b, tau_a), i
    finally:
        aco.aco_batch_destroy(b)
    ref = orc.run(insts[0].dist, ms[0], 3, seeds[0], rho=1.0)
    with aco.Colony(insts[0].dist, ms[0], seed=seeds[0], rho=1.0) as col:
        aco.aco_iterate(col.h, 3)
        assert np.array_equal(aco.aco_get_pheromone(col.h, ns[0]), ref["tau32"])


def test_coordinates_build_the_same_instance(aco, orc):
    inst = I.clustered_instance(333, seed=4)
    h = aco.aco_create_coords(inst.coords, 1.0, 2.0, 0.5, 64, 3)
    try:
        assert np.array_equal(aco.aco_get_heuristic(h, 333), orc.heta(inst.dist, 2.0))
        assert aco.aco_get_tau0(h)[1] == orc.nn_tour_length(inst.dist)
        aco.aco_iterate(h, 3)
        tau = aco.aco_get_pheromone(h, 333)
    finally:
        aco.aco_destroy(h)
    assert np.array_equal(tau, orc.run(inst.dist, 64, 3, 3)["tau32"])
    with pytest.raises(aco.AcoError) as e:
        aco.aco_create_coords(np.array([[0, 0], [5, 5], [0, 0]]), 1.0, 2.0, 0.5, 3, 1)
    assert e.value.code == aco.ACO_EINVAL


def test_continuous_admission_equals_alone(aco):
    a = I.uniform_instance(400, 1000, seed=41)
    b = I.clustered_instance(150, seed=42, clusters=8, side=3000)
    c = I.uniform_instance(64, 1000, seed=43)
    budget = sum(aco.aco_pool_bytes_needed(x.n, x.n) for x in (a, b, c)) + (1 << 20)
    p = aco.aco_pool_create(8, budget)
    try:
        sa = aco.aco_pool_admit_coords(p, a.coords, 1.0, 2.0, 0.5, a.n, 7, 10)
        for _ in range(3):
            aco.aco_pool_step(p)
        sb = aco.aco_pool_admit_coords(p, b.coords, 1.0, 2.0, 0.5, b.n, 8, 5)
        aco.aco_pool_step(p)
        sc = aco.aco_pool_admit(p, c.dist, 1.0, 2.0, 0.5, c.n, 9, 4)
        steps = 0
        while aco.aco_pool_step(p) > 0:
            steps += 1
            assert steps < 50
        fin = aco.aco_pool_finished(p)
        assert sorted(fin) == sorted([sa, sb, sc])
        for slot, x, seed, iters in [(sa, a, 7, 10), (sb, b, 8, 5), (sc, c, 9, 4)]:
            tau_a, (tour_a, len_a) = alone(aco, x.dist, x.n, seed, iters)
            tour_p, len_p = aco.aco_pool_result(p, slot, x.n)
            assert len_p == len_a and np.array_equal(tour_p, tour_a)
            assert np.array_equal(aco.aco_pool_pheromone(p, slot, x.n), tau_a)
            aco.aco_pool_release(p, slot)
        st = aco.aco_pool_stats(p)
        assert st["live"] == 0 and st["finished"] == 0 and st["bytes_in_use"] == 0
    finally:
        aco.aco_pool_destroy(p)


def test_budget_and_slots_refuse_then_recover(aco):
    x = I.uniform_instance(200, 1000, seed=5)
    need = aco.aco_pool_bytes_needed(200, 200)
    p = aco.aco_pool_create(4, need + need // 2)
    try:
        s0 = aco.aco_pool_admit_coords(p, x.coords, 1.0, 2.0, 0.5, 200, 1, 2)
        assert s0 is not None
        assert aco.aco_pool_admit_coords(p, x.coords, 1.0, 2.0, 0.5, 200, 2, 2) is None
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_admit(p, x.dist, 1.0, 2.0, 0.5, 200, 2, 2)
        assert e.value.code == aco.ACO_EBUSY
        aco.aco_pool_step(p)
        aco.aco_pool_step(p)
        assert aco.aco_pool_finished(p) == [s0]
        aco.aco_pool_release(p, s0)
        s1 = aco.aco_pool_admit_coords(p, x.coords, 1.0, 2.0, 0.5, 200, 2, 1)
        assert s1 is not None
        aco.aco_pool_step(p)
        aco.aco_pool_synchronize(p)
    finally:
        aco.aco_pool_destroy(p)
    p = aco.aco_pool_create(1, 1 << 30)
    try:
        aco.aco_pool_admit_coords(p, x.coords, 1.0, 2.0, 0.5, 10, 1, 1)
        assert aco.aco_pool_admit_coords(p, x.coords, 1.0, 2.0, 0.5, 10, 1, 1) is None
    finally:
        aco.aco_pool_destroy(p)


def test_pool_rejects_bad_arguments(aco):
    p = aco.aco_pool_create(2, 1 << 24)
    try:
        x = I.uniform_instance(10, 100, seed=1)
        for kw in [dict(rho=0.0), dict(m=0), dict(iterations=0)]:
            args = dict(alpha=1.0, beta=2.0, rho=0.5, m=5, seed=1, iterations=3)
            args.update(kw)
            with pytest.raises(aco.AcoError) as e:
                aco.aco_pool_admit(p, x.dist, **args)
            assert e.value.code == aco.ACO_EINVAL
        with pytest.raises(aco.AcoError):
            aco.aco_pool_result(p, 0, 10)
    finally:
        aco.aco_pool_destroy(p)


def test_server_results_equal_alone(aco):
    # Continuous batching through serve.Server: requests of different sizes
    # arrive together and in a small step-work budget (so admission is
    # staggered); each result must be the one the request gets alone.
    from paper_1101_2678_gb300 import serve
    reqs, arrivals = [], []
    for i, (n, kind) in enumerate([(90, "u"), (300, "c"), (48, "u"), (600, "c"), (150, "u")]):
        inst = (I.uniform_instance(n, 1000, seed=70 + i) if kind == "u"
                else I.clustered_instance(n, seed=70 + i, clusters=6, side=4000))
        reqs.append(serve.Request(inst.coords, m=min(n, 128), iterations=3 + i, seed=800 + i))
        arrivals.append(0.001 * i)
    with serve.Server(budget_bytes=1 << 30, max_slots=8, max_step_work=600 * 600 * 128) as srv:
        outs, st = srv.run(reqs, np.array(arrivals), realtime=False)
    assert st["completed"] == len(reqs) and st["backlog"] == 0
    for o in outs:
        r = reqs[o.index]
        d = I.distance_matrix(r.coords)
        with aco.Colony(d, r.m, seed=r.seed) as c:
            aco.aco_iterate(c.h, r.iterations)
            tour, length = aco.aco_best_tour(c.h, r.n)
        assert o.best_len == length and np.array_equal(o.best_tour, tour), o.index


def test_autotuned_tilings_give_identical_results(aco):
    # The tuner picks per class among tilings that all build the same tours;
    # a batch with tuning on and one with it off end in the same state.
    ns = [48, 130, 300, 700, 1000]
    insts = [I.uniform_instance(n, 1000, seed=900 + n) for n in ns]
    ms = ns
    seeds = [31 + i for i in range(len(ns))]
    out = {}
    for on in (True, False):
        b = aco.aco_batch_create([x.dist for x in insts], ms, seeds)
        try:
            aco.aco_pool_set_autotune(b, on)
            aco.aco_pool_autotune(b)
            tilings = [aco.aco_pool_tiling(b, i) for i in range(len(ns))]
            for (g, h, c, sg), n in zip(tilings, ns):
                assert g in (1, 2, 4) and h in (8, 16, 32) and (h == 32 or g == 1)
                assert g * h * c >= n and sg in (0, 1)
                if not on:
                    assert (g, h, sg) == (1, 32, 0)
            aco.aco_batch_iterate(b, 4)
            out[on] = [(aco.aco_pool_pheromone(b, i, n), aco.aco_batch_best(b, i, n))
                       for i, n in enumerate(ns)]
        finally:
            aco.aco_batch_destroy(b)
    for (ta, (tra, la)), (tb, (trb, lb)) in zip(out[True], out[False]):
        assert np.array_equal(ta, tb) and la == lb and np.array_equal(tra, trb)


def test_cancel_mid_flight_and_allocation_failure(aco):
    # A request released while still live (cancelled) frees its memory and
    # leaves the others' results unchanged; a budget the device cannot
    # allocate fails cleanly with ACO_ENOMEM.
    a = I.uniform_instance(120, 1000, seed=61)
    b = I.uniform_instance(90, 1000, seed=62)
    p = aco.aco_pool_create(4, 1 << 28)
    try:
        sa = aco.aco_pool_admit_coords(p, a.coords, 1.0, 2.0, 0.5, 60, 5, 6)
        sb = aco.aco_pool_admit_coords(p, b.coords, 1.0, 2.0, 0.5, 40, 6, 6)
        aco.aco_pool_step(p)
        aco.aco_pool_step(p)
        aco.aco_pool_release(p, sb)  # cancelled after two of its six iterations
        assert aco.aco_pool_stats(p)["live"] == 1
        while aco.aco_pool_step(p) > 0:
            pass
        assert aco.aco_pool_finished(p) == [sa]
        tau_a, (tour_a, len_a) = alone(aco, a.dist, 60, 5, 6)
        tour_p, len_p = aco.aco_pool_result(p, sa, a.n)
        assert len_p == len_a and np.array_equal(tour_p, tour_a)
        assert np.array_equal(aco.aco_pool_pheromone(p, sa, a.n), tau_a)
        aco.aco_pool_release(p, sa)
        assert aco.aco_pool_stats(p)["bytes_in_use"] == 0
    finally:
        aco.aco_pool_destroy(p)
    with pytest.raises(aco.AcoError) as e:
        aco.aco_pool_create(4, 1 << 50)
    assert e.value.code == aco.ACO_ENOMEM


def test_large_instances_in_a_batch_equal_alone(aco):
    # n > 2432 takes two warps per ant; mixed with small instances in one
    # batch, each still ends exactly as when run alone.
    insts = [I.clustered_instance(3000, seed=77, clusters=16, sigma=400, side=20000),
             I.uniform_instance(150, 1000, seed=78), I.uniform_instance(4096, 30000, seed=79)]
    ms, seeds = [48, 150, 32], [5, 6, 7]
    b = aco.aco_batch_create([x.dist for x in insts], ms, seeds)
    try:
        aco.aco_batch_iterate(b, 2)
        for i, x in enumerate(insts):
            tau_a, (tour_a, len_a) = alone(aco, x.dist, ms[i], seeds[i], 2)
            tour_b, len_b = aco.aco_batch_best(b, i, x.n)
            assert len_b == len_a and np.array_equal(tour_b, tour_a), i
            assert np.array_equal(aco.aco_pool_pheromone(b, i, x.n), tau_a), i
    finally:
        aco.aco_batch_destroy(b)


def test_tuning_table_round_trips_through_json(aco, tmp_path):
    ns = [60, 250, 700, 1000]
    insts = [I.uniform_instance(n, 1000, seed=300 + n) for n in ns]
    seeds = [1, 2, 3, 4]
    b = aco.aco_batch_create([x.dist for x in insts], ns, seeds)
    try:
        aco.aco_pool_autotune(b)
        chosen = [aco.aco_pool_tiling(b, i) for i in range(len(ns))]
        table = aco.aco_pool_get_tuning(b)
        assert len(table) == len({tuple(k) for k, _ in table}) >= 3
        path = str(tmp_path / "tuning.json")
        aco.save_tuning(b, path)
    finally:
        aco.aco_batch_destroy(b)
    b = aco.aco_batch_create([x.dist for x in insts], ns, seeds)
    try:
        aco.load_tuning(b, path)
        assert aco.aco_pool_get_tuning(b) == table
        aco.aco_batch_iterate(b, 2)
        assert [aco.aco_pool_tiling(b, i) for i in range(len(ns))] == chosen
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_set_tuning(b, [[[1, 32, 36], [3, 32, 4, 0]]])  # 3 warps per ant
        assert e.value.code == aco.ACO_EINVAL
        assert aco.aco_pool_get_tuning(b) == table
    finally:
        aco.aco_batch_destroy(b)


def test_single_construction_launch_equals_alone(aco):
    # Every class of the batch in one persistent construction launch (items
    # from a global ticket, each with its class's chunk width): the instances
    # end as when run alone, and the step has fewer launches than with one
    # launch per class.
    ns = [48, 130, 300, 517, 700, 1000, 77, 900]
    insts = [I.uniform_instance(n, 1000, seed=700 + n) for n in ns]
    ms = [min(n, 160) for n in ns]
    seeds = [40 + i for i in range(len(ns))]
    launches = {}
    for single in (False, True):
        b = aco.aco_batch_create([x.dist for x in insts], ms, seeds)
        try:
            aco.aco_pool_set_single_launch(b, single)
            aco.aco_batch_iterate(b, 4)
            launches[single] = aco.aco_pool_stats(b)["launches_last_step"]
            for i, x in enumerate(insts):
                tau_a, (tour_a, len_a) = alone(aco, x.dist, ms[i], seeds[i], 4)
                tour_b, len_b = aco.aco_batch_best(b, i, x.n)
                assert len_b == len_a and np.array_equal(tour_b, tour_a), (single, i)
                assert np.array_equal(aco.aco_pool_pheromone(b, i, x.n), tau_a), (single, i)
        finally:
            aco.aco_batch_destroy(b)
    assert launches[True] < launches[False]
    with pytest.raises(aco.AcoError) as e:
        aco.aco_pool_set_single_launch(None, True)
    assert e.value.code == aco.ACO_EINVAL
