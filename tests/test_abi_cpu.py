"""The C ABI library loads and exports every entry point of include/aco.h (no GPU).

Only host-side argument validation is exercised here: those paths return
before any CUDA call.  Compute paths are covered by the -m gpu tests.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1101_2678_gb300 import build
    build.build()
    from paper_1101_2678_gb300 import aco
    return aco.load()


def _declared():
    names = set()
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(aco_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["aco_create", "aco_choice_info", "aco_construct_tours", "aco_update_pheromone",
                 "aco_iterate", "aco_best_tour", "aco_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1101_2678_gb300 import aco
    bound = {name for name, _, _ in aco.SIGNATURES}
    assert set(_declared()) <= bound | set(getattr(aco, "EXTRA_SIGNATURE_NAMES", ()))


def test_strerror_names_every_code(lib):
    from paper_1101_2678_gb300 import aco
    for code in [0, -1, -2, -3, -4, -5, -6]:
        assert aco.aco_strerror(code).startswith("ACO_")


def _create(lib, dist, alpha=1.0, beta=2.0, rho=0.5, m=4, seed=1, n=None):
    d = np.ascontiguousarray(dist, np.int32)
    h = C.c_void_p()
    n = d.shape[0] if n is None else n
    rc = lib.aco_create(n, d.ctypes.data_as(C.c_void_p), alpha, beta, rho, m, seed, C.byref(h))
    return rc, h


def test_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    from paper_1101_2678_gb300 import aco
    good = np.array([[0, 1, 2], [1, 0, 3], [2, 3, 0]], np.int32)
    cases = [
        dict(dist=good[:2, :2], n=2),                               # n < 3
        dict(dist=good, m=0),                                       # no ants
        dict(dist=good, m=aco.ACO_MAX_M + 1),
        dict(dist=good, rho=0.0), dict(dist=good, rho=1.5),         # 0 < rho <= 1 (Eq. 2)
        dict(dist=good, alpha=float("nan")), dict(dist=good, beta=-1.0),
        dict(dist=np.array([[0, 1, 2], [1, 0, 3], [2, 4, 0]])),     # not symmetric
        dict(dist=np.array([[1, 1, 2], [1, 0, 3], [2, 3, 0]])),     # d_ii != 0
        dict(dist=np.array([[0, 0, 2], [0, 0, 3], [2, 3, 0]])),     # d_ij = 0: eta undefined
        dict(dist=np.array([[0, -1, 2], [-1, 0, 3], [2, 3, 0]])),
    ]
    for kw in cases:
        rc, h = _create(lib, **kw)
        assert rc == aco.ACO_EINVAL, kw
        assert h.value is None
        assert lib.aco_last_error_message()
    big = np.ones((aco.ACO_MAX_N + 1, 1), np.int32)
    rc, _ = _create(lib, big, n=aco.ACO_MAX_N + 1)
    assert rc == aco.ACO_EINVAL


def test_null_handle_calls_fail_cleanly(lib):
    from paper_1101_2678_gb300 import aco
    assert lib.aco_destroy(None) == aco.ACO_OK
    assert lib.aco_iterate(None, 1) == aco.ACO_EINVAL
    assert lib.aco_update_pheromone(None) == aco.ACO_EINVAL
    assert lib.aco_best_tour(None, None, None) == aco.ACO_EINVAL
    h = C.c_void_p()
    assert lib.aco_create(3, None, 1.0, 2.0, 0.5, 3, 1, C.byref(h)) == aco.ACO_EINVAL
    assert lib.aco_set_mmas(None, 0.05, 0) == aco.ACO_EINVAL
    assert lib.aco_set_acs(None, 0.9, 0.1) == aco.ACO_EINVAL
    assert lib.aco_pool_autotune(None) == aco.ACO_EINVAL
    assert lib.aco_pool_set_tuning(None, None, 0) == aco.ACO_EINVAL
    assert lib.aco_pool_set_acs(None, 0, 0.9, 0.1) == aco.ACO_EINVAL
    assert lib.aco_pool_set_mmas(None, 0, 0.05, 0) == aco.ACO_EINVAL
    assert lib.aco_pool_set_multirate(None, 1) == aco.ACO_EINVAL
    assert lib.aco_pool_set_nn(None, 0, 8) == aco.ACO_EINVAL
    sz = C.c_uint64()
    assert lib.aco_pool_save_slot(None, 0, None, 0, C.byref(sz)) == aco.ACO_EINVAL
    assert lib.aco_pool_restore_slot(None, 0, None, 0) == aco.ACO_EINVAL
    k = C.c_int32()
    assert lib.aco_pool_rate(None, 0, C.byref(k)) == aco.ACO_EINVAL


def test_selftest_rejects_bad_arguments_before_touching_the_gpu(lib):
    from paper_1101_2678_gb300 import aco
    x = np.zeros(4, np.uint32)
    out = np.zeros(4, np.float32)
    assert lib.aco_race_exponential(None, out.ctypes.data, 4) == aco.ACO_EINVAL
    assert lib.aco_race_exponential(x.ctypes.data, out.ctypes.data, 0) == aco.ACO_EINVAL
    assert lib.aco_selftest_bounded_wait(0, 1) == aco.ACO_EINVAL
    assert lib.aco_selftest_bounded_wait((1 << 20) + 1, 1) == aco.ACO_EINVAL
    assert lib.aco_selftest_bounded_wait(100, 2) == aco.ACO_EINVAL
