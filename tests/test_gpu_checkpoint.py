"""Checkpoint and resume: a run saved after k iterations and restored into a
fresh handle continues exactly as the uninterrupted run (the random numbers
are counter-based on seed, iteration, ant and step)."""
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


def _final(aco, h, n):
    return aco.aco_get_pheromone(h, n), aco.aco_best_tour(h, n), aco.aco_get_iteration(h)


def _setup(aco, h, variant):
    if variant == "mmas":
        aco.aco_set_mmas(h, 0.05, False)
    elif variant == "acs":
        aco.aco_set_acs(h, 0.9, 0.1)


@pytest.mark.parametrize("variant,m,rho", [("as", 60, 0.5), ("mmas", 60, 0.1), ("acs", 10, 0.1)])
def test_resume_equals_uninterrupted_run(aco, variant, m, rho):
    inst = I.uniform_instance(200, 1000, seed=44)
    n, total, cut = 200, 9, 4
    with aco.Colony(inst.dist, m, seed=12, rho=rho) as c:
        _setup(aco, c.h, variant)
        aco.aco_iterate(c.h, total)
        ref = _final(aco, c.h, n)
    with aco.Colony(inst.dist, m, seed=12, rho=rho) as c:
        _setup(aco, c.h, variant)
        aco.aco_iterate(c.h, cut)
        blob = aco.aco_save_state(c.h)
    with aco.Colony(inst.dist, m, seed=12, rho=rho) as c:
        aco.aco_restore_state(c.h, blob)  # the update rule comes with the checkpoint
        assert aco.aco_get_iteration(c.h) == cut
        aco.aco_iterate(c.h, total - cut)
        got = _final(aco, c.h, n)
    assert np.array_equal(got[0], ref[0])
    assert got[1][1] == ref[1][1] and np.array_equal(got[1][0], ref[1][0])
    assert got[2] == ref[2] == total


def test_checkpoint_rejects_other_instances_and_damage(aco):
    inst = I.uniform_instance(50, 1000, seed=3)
    with aco.Colony(inst.dist, 20, seed=7) as c:
        aco.aco_iterate(c.h, 2)
        blob = aco.aco_save_state(c.h)
    for kw in (dict(m=21, seed=7), dict(m=20, seed=8)):
        with aco.Colony(inst.dist, kw["m"], seed=kw["seed"]) as c:
            with pytest.raises(aco.AcoError) as e:
                aco.aco_restore_state(c.h, blob)
            assert e.value.code == aco.ACO_EINVAL
    with aco.Colony(inst.dist, 20, seed=7) as c:
        for bad in (blob[:100], b"x" * len(blob), blob[:-4]):
            with pytest.raises(aco.AcoError) as e:
                aco.aco_restore_state(c.h, bad)
            assert e.value.code == aco.ACO_EINVAL
        aco.aco_restore_state(c.h, blob)
        aco.aco_iterate(c.h, 1)
        assert aco.aco_get_iteration(c.h) == 3


@pytest.mark.parametrize("variant,m,rho", [("as", 60, 0.5), ("mmas", 60, 0.1), ("acs", 10, 0.1)])
def test_handle_checkpoint_continues_in_a_pool_and_back(aco, variant, m, rho):
    # the same blob format on both sides: a run cut at iteration 4 on a
    # handle continues in a pool slot, and one cut in a pool continues on a
    # handle, both exactly as the uninterrupted run
    inst = I.uniform_instance(200, 1000, seed=45)
    n, total, cut = 200, 9, 4
    with aco.Colony(inst.dist, m, seed=13, rho=rho) as c:
        _setup(aco, c.h, variant)
        aco.aco_iterate(c.h, total)
        ref = _final(aco, c.h, n)
    with aco.Colony(inst.dist, m, seed=13, rho=rho) as c:
        _setup(aco, c.h, variant)
        aco.aco_iterate(c.h, cut)
        blob = aco.aco_save_state(c.h)
    p = aco.aco_pool_create(2, 2 * aco.aco_pool_bytes_needed(n, m) + (1 << 20))
    try:
        s = aco.aco_pool_admit(p, inst.dist, 1.0, 2.0, rho, m, 13, total - cut)
        aco.aco_pool_restore_slot(p, s, blob)
        while aco.aco_pool_step(p) > 0:
            pass
        assert np.array_equal(aco.aco_pool_pheromone(p, s, n), ref[0])
        tour, length = aco.aco_pool_result(p, s, n)
        assert length == ref[1][1] and np.array_equal(tour, ref[1][0])
        # pool -> handle: cut inside the pool this time
        s2 = aco.aco_pool_admit(p, inst.dist, 1.0, 2.0, rho, m, 13, cut)
        if variant == "acs":
            aco.aco_pool_set_acs(p, s2, 0.9, 0.1)
        elif variant == "mmas":
            aco.aco_pool_set_mmas(p, s2, 0.05, False)
        while aco.aco_pool_step(p) > 0:
            pass
        blob2 = aco.aco_pool_save_slot(p, s2)
    finally:
        aco.aco_pool_destroy(p)
    with aco.Colony(inst.dist, m, seed=13, rho=rho) as c:
        aco.aco_restore_state(c.h, blob2)
        assert aco.aco_get_iteration(c.h) == cut
        aco.aco_iterate(c.h, total - cut)
        got = _final(aco, c.h, n)
    assert np.array_equal(got[0], ref[0])
    assert got[1][1] == ref[1][1] and np.array_equal(got[1][0], ref[1][0])


def test_pool_checkpoint_state_errors(aco):
    inst = I.uniform_instance(50, 1000, seed=3)
    with aco.Colony(inst.dist, 20, seed=7) as c:
        aco.aco_iterate(c.h, 2)
        blob = aco.aco_save_state(c.h)
    p = aco.aco_pool_create(4, 4 * aco.aco_pool_bytes_needed(50, 21) + (1 << 20))
    try:
        other = aco.aco_pool_admit(p, inst.dist, 1.0, 2.0, 0.5, 21, 7, 3)
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_restore_slot(p, other, blob)  # another m
        assert e.value.code == aco.ACO_EINVAL
        s = aco.aco_pool_admit(p, inst.dist, 1.0, 2.0, 0.5, 20, 7, 3)
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_restore_slot(p, s, blob[:-8])
        assert e.value.code == aco.ACO_EINVAL
        aco.aco_pool_restore_slot(p, s, blob)
        for call in (lambda: aco.aco_pool_restore_slot(p, s, blob),
                     lambda: aco.aco_pool_set_acs(p, s, 0.9, 0.1)):
            with pytest.raises(aco.AcoError) as e:
                call()
            assert e.value.code == aco.ACO_ESTATE
        aco.aco_pool_step(p)
        late = aco.aco_pool_admit(p, inst.dist, 1.0, 2.0, 0.5, 20, 7, 3)
        aco.aco_pool_step(p)
        with pytest.raises(aco.AcoError) as e:
            aco.aco_pool_restore_slot(p, late, blob)  # it has stepped
        assert e.value.code == aco.ACO_ESTATE
    finally:
        aco.aco_pool_destroy(p)
