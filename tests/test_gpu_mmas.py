"""MAX-MIN Ant System update (aco_set_mmas) on the GPU against the CPU oracle.

The construction is the Ant System's; the update keeps one depositing tour
and clamps every trail into [tau_min, tau_max] (reading R13 of the oracle).
Every operation is a fixed sequence of IEEE-rounded float or double
operations, so tau, the limits and the tours must match the oracle bit for
bit.
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


def run_gpu(aco, dist, m, iters, seed, rho, p_best, best_so_far, nn=0, rule=0):
    n = dist.shape[0]
    with aco.Colony(dist, m, seed=seed, rho=rho) as c:
        if nn:
            aco.aco_set_option(c.h, aco.ACO_OPT_NN_LIST, nn)
        if rule:
            aco.aco_set_option(c.h, aco.ACO_OPT_SELECTION, rule)
        aco.aco_set_mmas(c.h, p_best, best_so_far)
        start = aco.aco_get_pheromone(c.h, n)
        aco.aco_iterate(c.h, iters - 1)
        tours, lens = aco.aco_construct_tours(c.h, n, m)
        aco.aco_update_pheromone(c.h)
        return dict(start=start, tau=aco.aco_get_pheromone(c.h, n), best=aco.aco_best_tour(c.h, n),
                    limits=aco.aco_get_mmas_limits(c.h), tours=tours, lens=lens,
                    launches=aco.aco_kernel_launches_per_iteration(c.h))


@pytest.mark.parametrize("best_so_far", [False, True])
def test_mmas_n48_hundred_iterations_bit_exact(aco, orc, best_so_far):
    w = I.workload_n48()
    d = w["inst"].dist
    ref = orc.run_mmas(d, 48, 100, w["seed"], rho=0.02, p_best=0.05, best_so_far=best_so_far)
    g = run_gpu(aco, d, 48, 100, w["seed"], 0.02, 0.05, best_so_far)
    assert np.array_equal(g["tours"], ref["tours"]) and np.array_equal(g["lens"], ref["lens"])
    assert g["best"][1] == ref["best_len"] and np.array_equal(g["best"][0], ref["best_tour"])
    assert np.array_equal(g["tau"], ref["tau32"])
    assert g["limits"] == (ref["tau_min"], ref["tau_max"])
    assert g["launches"] == 3
    r64 = ref["tau64"]
    assert np.all(np.abs(g["tau"] - r64) <= 1e-5 * np.abs(r64))


def test_mmas_initial_trails_are_tau_max_of_the_nn_tour(aco, orc):
    inst = I.uniform_instance(77, 1000, seed=4)
    g = run_gpu(aco, inst.dist, 20, 1, 3, 0.1, 0.05, False)
    _, hi = orc.mmas_limits(77, 0.1, 0.05, orc.nn_tour_length(inst.dist))
    off = ~np.eye(77, dtype=bool)
    assert np.all(g["start"][off] == np.float32(hi)) and np.all(np.diag(g["start"]) == 0)


@pytest.mark.parametrize("n,m,iters,rho,p", [(3, 3, 4, 0.1, 0.05), (33, 33, 30, 0.2, 0.05),
                                             (97, 60, 12, 0.2, 0.01), (300, 100, 6, 0.5, 0.05)])
def test_mmas_multi_iteration_bit_exact(aco, orc, n, m, iters, rho, p):
    inst = I.clustered_instance(n, seed=n, clusters=6, sigma=200, side=4000)
    for bsf in (False, True):
        ref = orc.run_mmas(inst.dist, m, iters, 9, rho=rho, p_best=p, best_so_far=bsf)
        g = run_gpu(aco, inst.dist, m, iters, 9, rho, p, bsf)
        assert np.array_equal(g["tau"], ref["tau32"]), bsf
        assert g["best"][1] == ref["best_len"] and g["limits"] == (ref["tau_min"], ref["tau_max"])


def test_mmas_composes_with_other_construction_rules(aco, orc):
    inst = I.uniform_instance(130, 1000, seed=15)
    ref = orc.run_mmas(inst.dist, 50, 8, 4, rho=0.2, rule=2, nn=16)
    g = run_gpu(aco, inst.dist, 50, 8, 4, 0.2, 0.05, False, nn=16)
    assert np.array_equal(g["tau"], ref["tau32"]) and g["best"][1] == ref["best_len"]
    assert g["launches"] == 4  # construct, best, update, list-ordered choice_info
    ref = orc.run_mmas(inst.dist, 50, 8, 4, rho=0.2, rule=1)
    g = run_gpu(aco, inst.dist, 50, 8, 4, 0.2, 0.05, False, rule=1)
    assert np.array_equal(g["tau"], ref["tau32"]) and g["best"][1] == ref["best_len"]


def test_mmas_full_size_n1002(aco, orc):
    # The bench's n = 1002 configuration, two iterations: tau equals the
    # oracle's (sampled rows), the limits follow the best-so-far length, and
    # the trails are symmetric and inside the limits.
    w = I.workload_n1002()
    d, m = w["inst"].dist, w["m"]
    n = d.shape[0]
    ref = orc.run_mmas(d, m, 2, w["seed"], rho=0.02)
    g = run_gpu(aco, d, m, 2, w["seed"], 0.02, 0.05, False)
    rows = np.random.default_rng(0).choice(n, 64, replace=False)
    assert np.array_equal(g["tau"][rows], ref["tau32"][rows])
    assert g["best"][1] == ref["best_len"]
    lo, hi = g["limits"]
    assert (lo, hi) == orc.mmas_limits(n, 0.02, 0.05, g["best"][1])
    off = ~np.eye(n, dtype=bool)
    assert np.all(g["tau"][off] >= lo) and np.all(g["tau"][off] <= hi)
    assert np.array_equal(g["tau"], g["tau"].T)


def test_mmas_argument_and_state_errors(aco):
    inst = I.uniform_instance(20, 100, seed=2)
    with aco.Colony(inst.dist, 10, seed=1) as c:
        with pytest.raises(aco.AcoError) as e:
            aco.aco_get_mmas_limits(c.h)
        assert e.value.code == aco.ACO_ESTATE
        for p in (0.0, 1.0, -0.5, float("nan")):
            with pytest.raises(aco.AcoError) as e:
                aco.aco_set_mmas(c.h, p, False)
            assert e.value.code == aco.ACO_EINVAL
        aco.aco_construct_tours(c.h)
        with pytest.raises(aco.AcoError) as e:
            aco.aco_set_mmas(c.h, 0.05, False)
        assert e.value.code == aco.ACO_ESTATE
