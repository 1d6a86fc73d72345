"""The allocation-free pheromone update against the regular entry point.

aco_update_pheromone_noalloc is for callers that cannot allocate device
memory (graph capture by someone else, allocator-less runtimes, hosts that
reserve all device memory up front).  Its scratch lives in one static device
array shared by every call, so two calls in a row must each start from a
clean accumulator.  Both calls here must reproduce, bit for bit, what
aco_update_pheromone computes on the same tours (deterministic fixed-point
deposit), including the per-call clearing of the shared scratch.
"""
import numpy as np
import pytest

from paper_1101_2678_gb300 import instances as I

pytestmark = pytest.mark.gpu


# A size in the middle of the range, and the largest the static scratch holds
# (the whole n x n accumulator, and the per-ant deposits and the scale slot at
# the end of the array).
@pytest.mark.parametrize("n,m", [(300, 257), (1024, 4096)])
def test_noalloc_update_matches_regular_update_twice(n, m):
    torch = pytest.importorskip("torch")
    from paper_1101_2678_gb300 import build
    build.build()
    from paper_1101_2678_gb300 import aco
    aco.load()
    assert n <= aco.ACO_NOALLOC_MAX_N and m <= aco.ACO_NOALLOC_MAX_M
    inst = I.uniform_instance(n, 1000, seed=77)
    dev = torch.device("cuda", torch.cuda.current_device())
    with aco.Colony(inst.dist, m, seed=5) as c:
        aco.aco_set_option(c.h, aco.ACO_OPT_DEPOSIT, aco.ACO_DEPOSIT_ATOMIC_U64)
        heta = torch.from_numpy(aco.aco_get_heuristic(c.h, n)).to(dev)
        tau = torch.from_numpy(aco.aco_get_pheromone(c.h, n)).to(dev)
        choice = torch.empty_like(tau)
        for call in range(2):
            tours_h, lens_h = aco.aco_construct_tours(c.h, n, m)
            tours = torch.from_numpy(tours_h).to(dev)
            lens = torch.from_numpy(lens_h).to(dev)
            torch.cuda.synchronize()
            aco.aco_update_pheromone_noalloc(n, m, tours.data_ptr(), lens.data_ptr(),
                                             heta.data_ptr(), tau.data_ptr(), choice.data_ptr(),
                                             1.0, 0.5, torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            aco.aco_update_pheromone(c.h)
            ref_tau = aco.aco_get_pheromone(c.h, n)
            ref_choice = aco.aco_choice_info(c.h, n)
            assert np.array_equal(tau.cpu().numpy(), ref_tau), call
            assert np.array_equal(choice.cpu().numpy(), ref_choice), call


def test_noalloc_update_rejects_sizes_beyond_the_static_scratch():
    from paper_1101_2678_gb300 import build
    build.build()
    from paper_1101_2678_gb300 import aco
    for n, m in [(aco.ACO_NOALLOC_MAX_N + 1, 10), (100, aco.ACO_NOALLOC_MAX_M + 1), (2, 5)]:
        with pytest.raises(aco.AcoError) as e:
            aco.aco_update_pheromone_noalloc(n, m, 1, 1, 1, 1, 1, 1.0, 0.5)
        assert e.value.code == aco.ACO_EINVAL
