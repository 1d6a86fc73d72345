"""Failure detection on the GPU without a GPU fault.

The library's only device-side spin waits are the bounded mbarrier waits of
the bulk row copies.  The self-test kernel runs the same bounded loop on a
phase that nothing completes: the wait must give up, the call must return
ACO_ETIMEOUT, and the context must stay usable.
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


def test_bounded_wait_gives_up_and_context_survives(aco, orc):
    assert aco.aco_selftest_bounded_wait(1000, True) == aco.ACO_OK
    assert aco.aco_selftest_bounded_wait(1000, False) == aco.ACO_ETIMEOUT
    assert aco.aco_selftest_bounded_wait(1000, True) == aco.ACO_OK
    # a normal run afterwards still matches the oracle
    inst = I.uniform_instance(40, 1000, seed=2)
    ref = orc.run(inst.dist, 20, 3, 4)
    with aco.Colony(inst.dist, 20, seed=4) as c:
        aco.aco_iterate(c.h, 3)
        assert np.array_equal(aco.aco_get_pheromone(c.h, 40), ref["tau32"])



def test_tour_check_option_passes_on_valid_runs(aco, orc):
    # With the check on, every construction is verified on the device; valid
    # runs (all rules) report nothing and end as without the check.
    inst = I.uniform_instance(120, 1000, seed=9)
    ref = orc.run(inst.dist, 40, 4, 2)
    with aco.Colony(inst.dist, 40, seed=2) as c:
        aco.aco_set_option(c.h, aco.ACO_OPT_CHECK, 1)
        assert aco.aco_get_option(c.h, aco.ACO_OPT_CHECK) == 1
        n_launch = aco.aco_kernel_launches_per_iteration(c.h)
        aco.aco_iterate(c.h, 4)
        assert np.array_equal(aco.aco_get_pheromone(c.h, 120), ref["tau32"])
        aco.aco_set_option(c.h, aco.ACO_OPT_CHECK, 0)
        assert aco.aco_kernel_launches_per_iteration(c.h) == n_launch - 1
    for setup in (lambda h: aco.aco_set_option(h, aco.ACO_OPT_NN_LIST, 10),
                  lambda h: aco.aco_set_acs(h, 0.9, 0.1),
                  lambda h: aco.aco_set_option(h, aco.ACO_OPT_SELECTION, 1)):
        with aco.Colony(inst.dist, 10, seed=3) as c:
            setup(c.h)
            aco.aco_set_option(c.h, aco.ACO_OPT_CHECK, 1)
            aco.aco_iterate(c.h, 3)
            aco.aco_synchronize(c.h)


def test_read_probe_runs_both_modes_and_rejects_bad_arguments(aco):
    # The roofline's read-bandwidth probe: both modes complete with a clear
    # status word (the bulk-copy mode's waits are bounded like the
    # construction kernel's), and invalid arguments are refused on the host.
    import torch
    nbytes = 4 << 20
    buf = torch.rand(nbytes // 4, device="cuda")
    sink = torch.zeros(4, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    for mode in (0, 1):
        for bps in (1, 3):
            aco.aco_stream_read(buf.data_ptr(), nbytes, 3, mode, bps, s.cuda_stream,
                                sink.data_ptr(), status.data_ptr())
    s.synchronize()
    assert int(status.item()) == 0
    lib = aco.load()
    assert lib.aco_stream_read(buf.data_ptr() + 4, 64, 1, 0, 1, 0, sink.data_ptr(),
                               status.data_ptr()) == aco.ACO_EINVAL  # misaligned
    assert lib.aco_stream_read(buf.data_ptr(), 1000, 1, 1, 1, 0, sink.data_ptr(),
                               status.data_ptr()) == aco.ACO_EINVAL  # not whole 16 KB chunks
    assert lib.aco_stream_read(buf.data_ptr(), 64, 1, 2, 1, 0, sink.data_ptr(),
                               status.data_ptr()) == aco.ACO_EINVAL  # unknown mode
    assert lib.aco_stream_read(buf.data_ptr(), 64, 0, 0, 1, 0, sink.data_ptr(),
                               status.data_ptr()) == aco.ACO_EINVAL  # no passes
