"""ctypes binding of libaco_gb300.so (include/aco.h), same names as the C ABI.

This module only marshals arguments: every step of the Ant System runs in the
CUDA kernels of the library.  There is no CPU fallback; if the library or a
GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libaco_gb300.so")

ACO_OK = 0
ACO_EINVAL = -1
ACO_ENOMEM = -2
ACO_ECUDA = -3
ACO_ESTATE = -4
ACO_ETIMEOUT = -5
ACO_EBUSY = -6
ACO_MAX_N = 4096
ACO_MAX_M = 16384

ACO_OPT_DEPOSIT = 1
ACO_OPT_STREAM = 2
ACO_OPT_USE_GRAPH = 3
ACO_OPT_PROFILE = 4
ACO_OPT_WARPS_PER_ANT = 5
ACO_OPT_ANTS_PER_CTA = 6
ACO_OPT_LANES_PER_ANT = 7
ACO_OPT_SELECTION = 8
ACO_OPT_NN_LIST = 9
ACO_OPT_STAGING = 10
ACO_OPT_CHECK = 11
ACO_SELECT_EQ1 = 0
ACO_SELECT_DATA_PARALLEL = 1
ACO_SELECT_EXP_RACE = 2

ACO_DEPOSIT_GATHER = 0
ACO_DEPOSIT_ATOMIC_U64 = 1
ACO_DEPOSIT_ATOMIC_F32 = 2
ACO_DEPOSIT_SYMMETRIC = 3
ACO_DEPOSIT_SORT = 4

ACO_PHASE_CONSTRUCT = 0
ACO_PHASE_BEST = 1
ACO_PHASE_DEPOSIT = 2
ACO_PHASE_UPDATE = 3
ACO_NUM_PHASES = 4

# (name, restype, argtypes) of every exported entry point.
_vp = C.c_void_p
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_f32p = C.POINTER(C.c_float)
SIGNATURES = [
    ("aco_strerror", C.c_char_p, [C.c_int]),
    ("aco_last_error_message", C.c_char_p, []),
    ("aco_create", C.c_int, [C.c_int32, _vp, C.c_float, C.c_float, C.c_float, C.c_int32,
                             C.c_uint64, C.POINTER(_vp)]),
    ("aco_destroy", C.c_int, [_vp]),
    ("aco_choice_info", C.c_int, [_vp, _vp]),
    ("aco_construct_tours", C.c_int, [_vp, _vp, _vp]),
    ("aco_update_pheromone", C.c_int, [_vp]),
    ("aco_iterate", C.c_int, [_vp, C.c_int32]),
    ("aco_best_tour", C.c_int, [_vp, _vp, _vp]),
    ("aco_get_pheromone", C.c_int, [_vp, _vp]),
    ("aco_get_heuristic", C.c_int, [_vp, _vp]),
    ("aco_get_iteration", C.c_int, [_vp, _i64p]),
    ("aco_get_tau0", C.c_int, [_vp, _f32p, _i64p]),
    ("aco_set_mmas", C.c_int, [_vp, C.c_double, C.c_int32]),
    ("aco_get_mmas_limits", C.c_int, [_vp, _f32p, _f32p]),
    ("aco_set_acs", C.c_int, [_vp, C.c_double, C.c_float]),
    ("aco_selftest_bounded_wait", C.c_int, [C.c_int32, C.c_int32]),
    ("aco_save_state", C.c_int, [_vp, _vp, C.c_uint64, C.POINTER(C.c_uint64)]),
    ("aco_restore_state", C.c_int, [_vp, _vp, C.c_uint64]),
    ("aco_philox4x32_10", C.c_int, [_vp, _vp, _vp, C.c_int32]),
    ("aco_race_exponential", C.c_int, [_vp, _vp, C.c_int32]),
    ("aco_stream_read", C.c_int, [_vp, C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_uint64,
                                  _vp, _vp]),
    ("aco_set_option", C.c_int, [_vp, C.c_int32, C.c_int64]),
    ("aco_get_option", C.c_int, [_vp, C.c_int32, _i64p]),
    ("aco_get_kernel_times", C.c_int, [_vp, _vp]),
    ("aco_synchronize", C.c_int, [_vp]),
    ("aco_kernel_launches_per_iteration", C.c_int, [_vp, _i32p]),
    ("aco_create_coords", C.c_int, [C.c_int32, _vp, C.c_float, C.c_float, C.c_float, C.c_int32,
                                    C.c_uint64, C.POINTER(_vp)]),
    ("aco_pool_bytes_needed", C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_uint64)]),
    ("aco_pool_create", C.c_int, [C.c_int32, C.c_uint64, C.POINTER(_vp)]),
    ("aco_pool_destroy", C.c_int, [_vp]),
    ("aco_pool_admit", C.c_int, [_vp, C.c_int32, _vp, C.c_float, C.c_float, C.c_float, C.c_int32,
                                 C.c_uint64, C.c_int32, _i32p]),
    ("aco_pool_admit_coords", C.c_int, [_vp, C.c_int32, _vp, C.c_float, C.c_float, C.c_float,
                                        C.c_int32, C.c_uint64, C.c_int32, _i32p]),
    ("aco_pool_set_acs", C.c_int, [_vp, C.c_int32, C.c_double, C.c_float]),
    ("aco_pool_set_mmas", C.c_int, [_vp, C.c_int32, C.c_double, C.c_int32]),
    ("aco_pool_set_multirate", C.c_int, [_vp, C.c_int32]),
    ("aco_pool_rate", C.c_int, [_vp, C.c_int32, _i32p]),
    ("aco_pool_save_slot", C.c_int, [_vp, C.c_int32, _vp, C.c_uint64, C.POINTER(C.c_uint64)]),
    ("aco_pool_restore_slot", C.c_int, [_vp, C.c_int32, _vp, C.c_uint64]),
    ("aco_pool_set_nn", C.c_int, [_vp, C.c_int32, C.c_int32]),
    ("aco_pool_step", C.c_int, [_vp, _i32p]),
    ("aco_pool_set_single_launch", C.c_int, [_vp, C.c_int32]),
    ("aco_pool_finished", C.c_int, [_vp, _vp, C.c_int32, _i32p]),
    ("aco_pool_result", C.c_int, [_vp, C.c_int32, _vp, _vp]),
    ("aco_pool_pheromone", C.c_int, [_vp, C.c_int32, _vp]),
    ("aco_pool_release", C.c_int, [_vp, C.c_int32]),
    ("aco_pool_stats", C.c_int, [_vp, _i32p, _i32p, C.POINTER(C.c_uint64), _i32p]),
    ("aco_pool_synchronize", C.c_int, [_vp]),
    ("aco_pool_set_autotune", C.c_int, [_vp, C.c_int32]),
    ("aco_pool_autotune", C.c_int, [_vp]),
    ("aco_pool_tiling", C.c_int, [_vp, C.c_int32, _i32p, _i32p, _i32p, _i32p]),
    ("aco_pool_get_tuning", C.c_int, [_vp, _vp, C.c_int32, _i32p]),
    ("aco_pool_set_tuning", C.c_int, [_vp, _vp, C.c_int32]),
    ("aco_batch_create", C.c_int, [C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.POINTER(_vp)]),
    ("aco_batch_iterate", C.c_int, [_vp, C.c_int32]),
    ("aco_batch_best", C.c_int, [_vp, C.c_int32, _vp, _vp]),
    ("aco_batch_destroy", C.c_int, [_vp]),
    ("aco_update_pheromone_noalloc", C.c_int, [C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, _vp,
                                               C.c_float, C.c_float, C.c_int64]),
]

_lock = threading.Lock()
_lib = None


class AcoError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {detail} (code {code})")
        self.code = code


def load(path: str | None = None):
    """Load the CUDA library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"{p} is missing: build it with __graft_entry__.build() "
                                   "(the Ant System has no CPU fallback)")
            L = C.CDLL(p)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, where: str) -> None:
    if rc != ACO_OK:
        L = load()
        detail = L.aco_last_error_message().decode() or L.aco_strerror(rc).decode()
        raise AcoError(rc, where, detail)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def aco_strerror(code: int) -> str:
    return load().aco_strerror(code).decode()


def aco_create(dist, alpha: float, beta: float, rho: float, m: int, seed: int):
    """Create an instance from an n x n int32 distance matrix; returns the handle."""
    d = np.ascontiguousarray(dist, dtype=np.int32)
    if d.ndim != 2 or d.shape[0] != d.shape[1]:
        raise ValueError("dist must be a square matrix")
    h = C.c_void_p()
    _check(load().aco_create(d.shape[0], _ptr(d), alpha, beta, rho, m, seed, C.byref(h)),
           "aco_create")
    return h


def aco_destroy(h) -> None:
    _check(load().aco_destroy(h), "aco_destroy")


def aco_choice_info(h, n: int | None = None):
    """Recompute choice_info; with n given, return it as an n x n float32 array."""
    out = None if n is None else np.empty((n, n), np.float32)
    _check(load().aco_choice_info(h, _ptr(out)), "aco_choice_info")
    return out


def aco_construct_tours(h, n: int | None = None, m: int | None = None):
    """Construct tours; with n and m given, return (tours (m, n+1), lens (m,))."""
    tours = lens = None
    if n is not None and m is not None:
        tours = np.empty((m, n + 1), np.int32)
        lens = np.empty(m, np.int64)
    _check(load().aco_construct_tours(h, _ptr(tours), _ptr(lens)), "aco_construct_tours")
    return tours, lens


def aco_update_pheromone(h) -> None:
    _check(load().aco_update_pheromone(h), "aco_update_pheromone")


def aco_iterate(h, iterations: int) -> None:
    _check(load().aco_iterate(h, iterations), "aco_iterate")


def aco_best_tour(h, n: int):
    tour = np.empty(n + 1, np.int32)
    length = np.zeros(1, np.int64)
    _check(load().aco_best_tour(h, _ptr(tour), _ptr(length)), "aco_best_tour")
    return tour, int(length[0])


def aco_get_pheromone(h, n: int) -> np.ndarray:
    out = np.empty((n, n), np.float32)
    _check(load().aco_get_pheromone(h, _ptr(out)), "aco_get_pheromone")
    return out


def aco_get_heuristic(h, n: int) -> np.ndarray:
    out = np.empty((n, n), np.float32)
    _check(load().aco_get_heuristic(h, _ptr(out)), "aco_get_heuristic")
    return out


def aco_get_iteration(h) -> int:
    v = C.c_int64()
    _check(load().aco_get_iteration(h, C.byref(v)), "aco_get_iteration")
    return v.value


def aco_get_tau0(h):
    t = C.c_float()
    nn = C.c_int64()
    _check(load().aco_get_tau0(h, C.byref(t), C.byref(nn)), "aco_get_tau0")
    return float(np.float32(t.value)), nn.value


def aco_set_mmas(h, p_best: float = 0.05, best_so_far: bool = False) -> None:
    """Switch to the MAX-MIN Ant System update (before the first construction)."""
    _check(load().aco_set_mmas(h, float(p_best), int(bool(best_so_far))), "aco_set_mmas")


def aco_philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 words computed on the GPU: ctr (count, 4) uint32, key (2,) uint32."""
    c = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, np.uint32).reshape(2)
    out = np.empty_like(c)
    _check(load().aco_philox4x32_10(_ptr(c), _ptr(k), _ptr(out), c.shape[0]), "aco_philox4x32_10")
    return out


def aco_race_exponential(x) -> np.ndarray:
    """The exponential race's variate E for Philox words x (uint32), computed on the GPU."""
    xs = np.ascontiguousarray(x, np.uint32)
    out = np.empty(xs.shape, np.float32)
    _check(load().aco_race_exponential(_ptr(xs), _ptr(out), xs.size), "aco_race_exponential")
    return out


def aco_stream_read(buf_ptr: int, nbytes: int, reps: int, mode: int, blocks_per_sm: int,
                    stream: int, sink_ptr: int, status_ptr: int) -> None:
    """Launch the read-bandwidth probe on device memory (raw device pointers;
    the caller times the launch on `stream`)."""
    _check(load().aco_stream_read(C.c_void_p(buf_ptr), nbytes, reps, mode, blocks_per_sm, stream,
                                  C.c_void_p(sink_ptr), C.c_void_p(status_ptr)), "aco_stream_read")


def aco_save_state(h) -> bytes:
    """A checkpoint of the run (tau, best tour, iteration counter, update rule)."""
    size = C.c_uint64()
    _check(load().aco_save_state(h, None, 0, C.byref(size)), "aco_save_state")
    buf = np.empty(size.value, np.uint8)
    _check(load().aco_save_state(h, _ptr(buf), size.value, C.byref(size)), "aco_save_state")
    return buf.tobytes()


def aco_restore_state(h, blob: bytes) -> None:
    """Continue a run from a checkpoint written by aco_save_state."""
    buf = np.frombuffer(blob, np.uint8)
    _check(load().aco_restore_state(h, _ptr(buf), buf.size), "aco_restore_state")


def aco_selftest_bounded_wait(polls: int, complete: bool) -> int:
    """Return code of the bounded-wait self-test (ACO_OK or ACO_ETIMEOUT)."""
    return int(load().aco_selftest_bounded_wait(int(polls), int(bool(complete))))


def aco_set_acs(h, q0: float = 0.9, xi: float = 0.1) -> None:
    """Switch to the Ant Colony System (before the first construction; m <= 32)."""
    _check(load().aco_set_acs(h, float(q0), float(xi)), "aco_set_acs")


def aco_get_mmas_limits(h):
    """(tau_min, tau_max) of a MAX-MIN handle."""
    lo = C.c_float()
    hi = C.c_float()
    _check(load().aco_get_mmas_limits(h, C.byref(lo), C.byref(hi)), "aco_get_mmas_limits")
    return float(np.float32(lo.value)), float(np.float32(hi.value))


def aco_set_option(h, key: int, value: int) -> None:
    _check(load().aco_set_option(h, key, value), "aco_set_option")


def aco_get_option(h, key: int) -> int:
    v = C.c_int64()
    _check(load().aco_get_option(h, key, C.byref(v)), "aco_get_option")
    return v.value


def aco_get_kernel_times(h) -> np.ndarray:
    out = np.zeros(ACO_NUM_PHASES, np.float32)
    _check(load().aco_get_kernel_times(h, _ptr(out)), "aco_get_kernel_times")
    return out


def aco_synchronize(h) -> None:
    _check(load().aco_synchronize(h), "aco_synchronize")


def aco_kernel_launches_per_iteration(h) -> int:
    v = C.c_int32()
    _check(load().aco_kernel_launches_per_iteration(h, C.byref(v)),
           "aco_kernel_launches_per_iteration")
    return v.value


def aco_create_coords(xy, alpha: float, beta: float, rho: float, m: int, seed: int):
    """Create an instance from (n, 2) integer coordinates (EUC_2D distances on device)."""
    c = np.ascontiguousarray(xy, dtype=np.int32)
    h = C.c_void_p()
    _check(load().aco_create_coords(c.shape[0], _ptr(c), alpha, beta, rho, m, seed, C.byref(h)),
           "aco_create_coords")
    return h


# ---- pools (batched / served instances) ---------------------------------------------------

def aco_pool_bytes_needed(n: int, m: int) -> int:
    v = C.c_uint64()
    _check(load().aco_pool_bytes_needed(n, m, C.byref(v)), "aco_pool_bytes_needed")
    return v.value


def aco_pool_create(max_slots: int, budget_bytes: int):
    p = C.c_void_p()
    _check(load().aco_pool_create(max_slots, budget_bytes, C.byref(p)), "aco_pool_create")
    return p


def aco_pool_destroy(p) -> None:
    _check(load().aco_pool_destroy(p), "aco_pool_destroy")


def aco_pool_admit(p, dist, alpha, beta, rho, m, seed, iterations):
    """Admit an instance given by its distance matrix; returns the slot (raises AcoError)."""
    d = np.ascontiguousarray(dist, dtype=np.int32)
    slot = C.c_int32()
    _check(load().aco_pool_admit(p, d.shape[0], _ptr(d), alpha, beta, rho, m, seed, iterations,
                                 C.byref(slot)), "aco_pool_admit")
    return slot.value


def aco_pool_save_slot(p, slot: int) -> bytes:
    """A checkpoint of a pool slot (the format of aco_save_state)."""
    size = C.c_uint64()
    _check(load().aco_pool_save_slot(p, slot, None, 0, C.byref(size)), "aco_pool_save_slot")
    buf = np.empty(size.value, np.uint8)
    _check(load().aco_pool_save_slot(p, slot, _ptr(buf), size.value, C.byref(size)),
           "aco_pool_save_slot")
    return buf.tobytes()


def aco_pool_restore_slot(p, slot: int, blob: bytes) -> None:
    """Load a checkpoint into a freshly admitted slot of the same instance."""
    buf = np.frombuffer(blob, np.uint8)
    _check(load().aco_pool_restore_slot(p, slot, _ptr(buf), buf.size), "aco_pool_restore_slot")


def aco_pool_set_nn(p, slot: int, nn: int) -> None:
    _check(load().aco_pool_set_nn(p, slot, nn), "aco_pool_set_nn")


def aco_pool_set_multirate(p, on: bool) -> None:
    _check(load().aco_pool_set_multirate(p, int(on)), "aco_pool_set_multirate")


def aco_pool_rate(p, slot: int) -> int:
    k = C.c_int32()
    _check(load().aco_pool_rate(p, slot, C.byref(k)), "aco_pool_rate")
    return k.value


def aco_pool_set_acs(p, slot: int, q0: float, xi: float) -> None:
    _check(load().aco_pool_set_acs(p, slot, q0, xi), "aco_pool_set_acs")


def aco_pool_set_mmas(p, slot: int, p_best: float, best_so_far: bool) -> None:
    _check(load().aco_pool_set_mmas(p, slot, p_best, int(best_so_far)), "aco_pool_set_mmas")


def aco_pool_admit_acs(p, dist, alpha, beta, rho, m, seed, iterations, q0, xi):
    """aco_pool_admit then aco_pool_set_acs; returns the slot (raises AcoError, and releases
    the slot if the switch is refused)."""
    slot = aco_pool_admit(p, dist, alpha, beta, rho, m, seed, iterations)
    try:
        aco_pool_set_acs(p, slot, q0, xi)
    except AcoError:
        aco_pool_release(p, slot)
        raise
    return slot


def aco_pool_admit_mmas(p, dist, alpha, beta, rho, m, seed, iterations, p_best, best_so_far):
    """aco_pool_admit then aco_pool_set_mmas; returns the slot (raises AcoError, and releases
    the slot if the switch is refused)."""
    slot = aco_pool_admit(p, dist, alpha, beta, rho, m, seed, iterations)
    try:
        aco_pool_set_mmas(p, slot, p_best, best_so_far)
    except AcoError:
        aco_pool_release(p, slot)
        raise
    return slot


def aco_pool_admit_coords(p, xy, alpha, beta, rho, m, seed, iterations):
    """Admit an instance given by integer coordinates; returns the slot or None if busy."""
    c = np.ascontiguousarray(xy, dtype=np.int32)
    slot = C.c_int32()
    rc = load().aco_pool_admit_coords(p, c.shape[0], _ptr(c), alpha, beta, rho, m, seed,
                                      iterations, C.byref(slot))
    if rc == ACO_EBUSY:
        return None
    _check(rc, "aco_pool_admit_coords")
    return slot.value


def aco_pool_set_single_launch(p, on: bool) -> None:
    _check(load().aco_pool_set_single_launch(p, int(bool(on))), "aco_pool_set_single_launch")


def aco_pool_step(p) -> int:
    live = C.c_int32()
    _check(load().aco_pool_step(p, C.byref(live)), "aco_pool_step")
    return live.value


def aco_pool_finished(p):
    cnt = C.c_int32()
    _check(load().aco_pool_finished(p, None, 0, C.byref(cnt)), "aco_pool_finished")
    out = np.zeros(max(cnt.value, 1), np.int32)
    _check(load().aco_pool_finished(p, _ptr(out), len(out), C.byref(cnt)), "aco_pool_finished")
    return out[:cnt.value].tolist()


def aco_pool_result(p, slot: int, n: int):
    tour = np.empty(n + 1, np.int32)
    length = np.zeros(1, np.int64)
    _check(load().aco_pool_result(p, slot, _ptr(tour), _ptr(length)), "aco_pool_result")
    return tour, int(length[0])


def aco_pool_pheromone(p, slot: int, n: int) -> np.ndarray:
    out = np.empty((n, n), np.float32)
    _check(load().aco_pool_pheromone(p, slot, _ptr(out)), "aco_pool_pheromone")
    return out


def aco_pool_release(p, slot: int) -> None:
    _check(load().aco_pool_release(p, slot), "aco_pool_release")


def aco_pool_stats(p) -> dict:
    live, fin, launches = C.c_int32(), C.c_int32(), C.c_int32()
    used = C.c_uint64()
    _check(load().aco_pool_stats(p, C.byref(live), C.byref(fin), C.byref(used), C.byref(launches)),
           "aco_pool_stats")
    return dict(live=live.value, finished=fin.value, bytes_in_use=used.value,
                launches_last_step=launches.value)


def aco_pool_synchronize(p) -> None:
    _check(load().aco_pool_synchronize(p), "aco_pool_synchronize")


def aco_pool_set_autotune(p, on: bool) -> None:
    _check(load().aco_pool_set_autotune(p, int(bool(on))), "aco_pool_set_autotune")


def aco_pool_autotune(p) -> None:
    """Tune the construction tiling of the live set's new classes now."""
    _check(load().aco_pool_autotune(p), "aco_pool_autotune")


def aco_pool_get_tuning(p) -> list:
    """The tuner's table: [[default G, H, C], [chosen G, H, ants per CTA, staging]] entries."""
    cnt = C.c_int32()
    _check(load().aco_pool_get_tuning(p, None, 0, C.byref(cnt)), "aco_pool_get_tuning")
    buf = np.zeros((max(cnt.value, 1), 7), np.int32)
    _check(load().aco_pool_get_tuning(p, _ptr(buf), buf.shape[0], C.byref(cnt)),
           "aco_pool_get_tuning")
    return [[row[:3].tolist(), row[3:].tolist()] for row in buf[:cnt.value]]


def aco_pool_set_tuning(p, table) -> None:
    """Replace the tuner's table (entries as returned by aco_pool_get_tuning)."""
    buf = np.array([list(k) + list(v) for k, v in table], np.int32).reshape(-1, 7)
    _check(load().aco_pool_set_tuning(p, _ptr(np.ascontiguousarray(buf)), buf.shape[0]),
           "aco_pool_set_tuning")


def save_tuning(p, path: str) -> None:
    """Write the pool's tuning table to a JSON file."""
    import json
    with open(path, "w") as f:
        json.dump({"construct_tiling": aco_pool_get_tuning(p)}, f, indent=1)


def load_tuning(p, path: str) -> None:
    """Load a tuning table written by save_tuning into the pool."""
    import json
    with open(path) as f:
        aco_pool_set_tuning(p, json.load(f)["construct_tiling"])


def aco_pool_tiling(p, slot: int):
    """(warps per ant, lanes per ant, cities per lane, staging) of the class of live `slot`."""
    g, h, c, s = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().aco_pool_tiling(p, slot, C.byref(g), C.byref(h), C.byref(c), C.byref(s)),
           "aco_pool_tiling")
    return g.value, h.value, c.value, s.value


def aco_batch_create(dists, ms, seeds, alpha=1.0, beta=2.0, rho=0.5):
    """A static batch: one slot per instance (lists of distance matrices, ant counts, seeds)."""
    count = len(dists)
    ds = [np.ascontiguousarray(d, dtype=np.int32) for d in dists]
    ns = np.array([d.shape[0] for d in ds], np.int32)
    ptrs = (C.c_void_p * count)(*[d.ctypes.data for d in ds])
    al = np.full(count, alpha, np.float32)
    be = np.full(count, beta, np.float32)
    rh = np.full(count, rho, np.float32)
    mm = np.ascontiguousarray(ms, np.int32)
    sd = np.ascontiguousarray(seeds, np.uint64)
    b = C.c_void_p()
    _check(load().aco_batch_create(count, _ptr(ns), ptrs, _ptr(al), _ptr(be), _ptr(rh), _ptr(mm),
                                   _ptr(sd), C.byref(b)), "aco_batch_create")
    return b


def aco_batch_iterate(b, iterations: int) -> None:
    _check(load().aco_batch_iterate(b, iterations), "aco_batch_iterate")


def aco_batch_best(b, idx: int, n: int):
    tour = np.empty(n + 1, np.int32)
    length = np.zeros(1, np.int64)
    _check(load().aco_batch_best(b, idx, _ptr(tour), _ptr(length)), "aco_batch_best")
    return tour, int(length[0])


def aco_batch_destroy(b) -> None:
    _check(load().aco_batch_destroy(b), "aco_batch_destroy")


ACO_NOALLOC_MAX_N = 1024
ACO_NOALLOC_MAX_M = 4096


def aco_update_pheromone_noalloc(n: int, m: int, tours_ptr: int, lens_ptr: int, heta_ptr: int,
                                 tau_ptr: int, choice_ptr: int, alpha: float, rho: float,
                                 stream: int = 0) -> None:
    """Pheromone update on caller-owned device arrays (raw device pointers), no allocation."""
    _check(load().aco_update_pheromone_noalloc(n, m, tours_ptr, lens_ptr, heta_ptr, tau_ptr,
                                               choice_ptr, alpha, rho, stream),
           "aco_update_pheromone_noalloc")


class Colony:
    """Thin owner of one handle (destroys it on close / garbage collection)."""

    def __init__(self, dist, m: int, seed: int, alpha=1.0, beta=2.0, rho=0.5):
        d = np.ascontiguousarray(dist, dtype=np.int32)
        self.n = int(d.shape[0])
        self.m = int(m)
        self.h = aco_create(d, alpha, beta, rho, m, seed)

    def close(self):
        if self.h is not None:
            aco_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
