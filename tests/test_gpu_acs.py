"""Ant Colony System (aco_set_acs) on the GPU against the CPU oracle.

The colony runs in one CTA, one warp per ant, in lockstep: every step's
choices read the same state, then the local updates of that step are applied
once per crossing (reading R14 of the oracle).  Every operation is integer
or a fixed sequence of IEEE-rounded float operations, so tours, lengths and
tau must match the oracle bit for bit.
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


def run_gpu(aco, dist, m, iters, seed, rho, q0, xi):
    n = dist.shape[0]
    with aco.Colony(dist, m, seed=seed, rho=rho) as c:
        aco.aco_set_acs(c.h, q0, xi)
        start = aco.aco_get_pheromone(c.h, n)
        aco.aco_iterate(c.h, iters - 1)
        tours, lens = aco.aco_construct_tours(c.h, n, m)
        aco.aco_update_pheromone(c.h)
        return dict(start=start, tau=aco.aco_get_pheromone(c.h, n),
                    best=aco.aco_best_tour(c.h, n), tours=tours, lens=lens,
                    launches=aco.aco_kernel_launches_per_iteration(c.h))


def test_acs_n48_hundred_iterations_bit_exact(aco, orc):
    w = I.workload_n48()
    d = w["inst"].dist
    ref = orc.run_acs(d, 10, 100, w["seed"], rho=0.1, q0=0.9, xi=0.1)
    g = run_gpu(aco, d, 10, 100, w["seed"], 0.1, 0.9, 0.1)
    assert np.array_equal(g["tours"], ref["tours"]) and np.array_equal(g["lens"], ref["lens"])
    assert g["best"][1] == ref["best_len"] and np.array_equal(g["best"][0], ref["best_tour"])
    assert np.array_equal(g["tau"], ref["tau32"])
    assert g["launches"] == 3


@pytest.mark.parametrize("n,m,iters,q0,xi", [(3, 1, 3, 0.9, 0.1), (5, 32, 4, 0.5, 0.3),
                                             (31, 7, 6, 0.0, 0.1), (33, 32, 5, 1.0, 0.1),
                                             (97, 10, 8, 0.9, 0.1), (300, 16, 3, 0.75, 0.2)])
def test_acs_runs_bit_exact(aco, orc, n, m, iters, q0, xi):
    inst = I.clustered_instance(n, seed=50 + n, clusters=5, sigma=150, side=3000)
    ref = orc.run_acs(inst.dist, m, iters, 21, rho=0.1, q0=q0, xi=xi)
    g = run_gpu(aco, inst.dist, m, iters, 21, 0.1, q0, xi)
    assert np.array_equal(g["tours"], ref["tours"]) and np.array_equal(g["lens"], ref["lens"])
    assert np.array_equal(g["tau"], ref["tau32"])
    assert g["best"][1] == ref["best_len"]


def test_acs_initial_trails(aco, orc):
    inst = I.uniform_instance(60, 1000, seed=6)
    g = run_gpu(aco, inst.dist, 10, 1, 2, 0.1, 0.9, 0.1)
    tau0 = np.float32(1.0 / (60 * orc.nn_tour_length(inst.dist)))
    off = ~np.eye(60, dtype=bool)
    assert np.all(g["start"][off] == tau0) and np.all(np.diag(g["start"]) == 0)


@pytest.mark.parametrize("wl,iters", [("workload_n1002", 2), ("workload_n2392", 1)])
def test_acs_full_size_bit_exact(aco, orc, wl, iters):
    w = getattr(I, wl)()
    d = w["inst"].dist
    ref = orc.run_acs(d, 10, iters, w["seed"])
    g = run_gpu(aco, d, 10, iters, w["seed"], 0.1, 0.9, 0.1)
    assert np.array_equal(g["tours"], ref["tours"]) and np.array_equal(g["lens"], ref["lens"])
    assert np.array_equal(g["tau"], ref["tau32"])


def test_acs_argument_and_state_errors(aco):
    inst = I.uniform_instance(20, 100, seed=2)
    with aco.Colony(inst.dist, 33, seed=1) as c:
        with pytest.raises(aco.AcoError) as e:
            aco.aco_set_acs(c.h, 0.9, 0.1)
        assert e.value.code == aco.ACO_EINVAL
    with aco.Colony(inst.dist, 10, seed=1) as c:
        for q0, xi in [(-0.1, 0.1), (1.5, 0.1), (0.9, -0.5), (0.9, 2.0)]:
            with pytest.raises(aco.AcoError) as e:
                aco.aco_set_acs(c.h, q0, xi)
            assert e.value.code == aco.ACO_EINVAL
        aco.aco_set_option(c.h, aco.ACO_OPT_SELECTION, aco.ACO_SELECT_DATA_PARALLEL)
        with pytest.raises(aco.AcoError) as e:
            aco.aco_set_acs(c.h, 0.9, 0.1)  # the variant has its own rule
        assert e.value.code == aco.ACO_EINVAL
        aco.aco_set_option(c.h, aco.ACO_OPT_SELECTION, aco.ACO_SELECT_EQ1)
        aco.aco_set_acs(c.h, 0.9, 0.1)
        with pytest.raises(aco.AcoError):
            aco.aco_set_option(c.h, aco.ACO_OPT_SELECTION, aco.ACO_SELECT_EXP_RACE)
        with pytest.raises(aco.AcoError) as e:
            aco.aco_set_mmas(c.h, 0.05, False)
        assert e.value.code == aco.ACO_ESTATE
        aco.aco_iterate(c.h, 2)
        tour, length = aco.aco_best_tour(c.h, 20)
        assert sorted(tour[:-1].tolist()) == list(range(20))


def run_gpu_nn(aco, dist, m, iters, seed, rho, q0, xi, nn, lists_first=True):
    n = dist.shape[0]
    with aco.Colony(dist, m, seed=seed, rho=rho) as c:
        if lists_first:
            aco.aco_set_option(c.h, aco.ACO_OPT_NN_LIST, nn)
        aco.aco_set_acs(c.h, q0, xi)
        if not lists_first:
            aco.aco_set_option(c.h, aco.ACO_OPT_NN_LIST, nn)
        aco.aco_iterate(c.h, iters - 1)
        tours, lens = aco.aco_construct_tours(c.h, n, m)
        aco.aco_update_pheromone(c.h)
        return dict(tau=aco.aco_get_pheromone(c.h, n), best=aco.aco_best_tour(c.h, n),
                    tours=tours, lens=lens,
                    launches=aco.aco_kernel_launches_per_iteration(c.h))


@pytest.mark.parametrize("n,m,nn,iters,q0,xi", [(10, 4, 9, 6, 0.9, 0.1), (97, 10, 10, 8, 0.9, 0.1),
                                                (300, 16, 30, 4, 0.5, 0.2),
                                                (200, 32, 32, 3, 0.0, 0.1),
                                                (150, 7, 20, 5, 1.0, 0.3)])
def test_acs_with_lists_bit_exact(aco, orc, n, m, nn, iters, q0, xi):
    # reading R16: list-restricted exploitation and exploration, the dense
    # argmax when a list is exhausted, the lockstep local updates
    inst = I.clustered_instance(n, seed=80 + n, clusters=5, sigma=150, side=3000)
    ref = orc.run_acs(inst.dist, m, iters, 23, rho=0.1, q0=q0, xi=xi, nn=nn)
    g = run_gpu_nn(aco, inst.dist, m, iters, 23, 0.1, q0, xi, nn, lists_first=n % 2 == 0)
    assert np.array_equal(g["tours"], ref["tours"]) and np.array_equal(g["lens"], ref["lens"])
    assert np.array_equal(g["tau"], ref["tau32"])
    assert g["best"][1] == ref["best_len"] and np.array_equal(g["best"][0], ref["best_tour"])
    assert g["launches"] == 3


def test_acs_with_lists_full_size(aco, orc):
    w = I.workload_n1002()
    d = w["inst"].dist
    ref = orc.run_acs(d, 10, 2, w["seed"], nn=30)
    g = run_gpu_nn(aco, d, 10, 2, w["seed"], 0.1, 0.9, 0.1, 30)
    assert np.array_equal(g["tours"], ref["tours"]) and np.array_equal(g["tau"], ref["tau32"])
