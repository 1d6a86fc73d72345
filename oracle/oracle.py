"""ctypes front end of the CPU oracle (aco_oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs are the only callers.  The product path (the CUDA
library and its binding) never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "aco_oracle.c")
LIB = os.path.join(HERE, "libaco_oracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, IEEE semantics)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
            u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
            u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
            u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
            f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = C.c_int
            L.orc_get_threads.argtypes = []
            L.orc_get_threads.restype = C.c_int
            L.orc_hardware_threads.argtypes = []
            L.orc_hardware_threads.restype = C.c_int
            L.orc_philox4x32_10.restype = None
            L.orc_ceil_log2.argtypes = [C.c_int64]
            L.orc_ceil_log2.restype = C.c_int
            L.orc_roulette.argtypes = [C.c_int, f32p, u8p, C.c_uint64]
            L.orc_roulette.restype = C.c_int
            L.orc_roulette_weights.argtypes = [C.c_int, f32p, u8p, u64p]
            L.orc_roulette_weights.restype = C.c_uint64
            L.orc_heta.argtypes = [C.c_int, i32p, C.c_double, f32p]
            L.orc_heta.restype = None
            L.orc_nn_tour_length.argtypes = [C.c_int, i32p]
            L.orc_nn_tour_length.restype = C.c_int64
            L.orc_tau0.argtypes = [C.c_int, C.c_int, i32p]
            L.orc_tau0.restype = C.c_float
            L.orc_choice.argtypes = [C.c_int, f32p, f32p, C.c_float, f32p]
            L.orc_choice.restype = None
            L.orc_construct_ant.argtypes = [C.c_int, f32p, i32p, C.c_uint64, C.c_uint32,
                                            C.c_uint32, i32p]
            L.orc_construct_ant.restype = C.c_int64
            L.orc_construct.argtypes = [C.c_int, C.c_int, f32p, i32p, C.c_uint64, C.c_uint32,
                                        i32p, i64p]
            L.orc_construct.restype = None
            L.orc_deposit_scale.argtypes = [C.c_int, i64p]
            L.orc_deposit_scale.restype = C.c_int
            L.orc_update_mirror.argtypes = [C.c_int, C.c_int, i32p, i64p, C.c_float, f32p]
            L.orc_update_mirror.restype = None
            L.orc_update_fp64.argtypes = [C.c_int, C.c_int, i32p, i64p, C.c_double, f64p]
            L.orc_update_fp64.restype = None
            vp = C.c_void_p
            L.orc_run.argtypes = [C.c_int, i32p, C.c_float, C.c_float, C.c_float, C.c_int,
                                  C.c_uint64, C.c_int, vp, vp, vp, vp, vp, vp, vp]
            L.orc_run.restype = C.c_int
            L.orc_candidate_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                                C.c_int]
            L.orc_candidate_uniform.restype = C.c_float
            L.orc_iroulette.argtypes = [C.c_int, f32p, u8p, C.c_uint64, C.c_uint32, C.c_uint32,
                                        C.c_uint32]
            L.orc_iroulette.restype = C.c_int
            L.orc_race_exponentials.argtypes = [C.c_int, vp, vp]
            L.orc_race_exponentials.restype = None
            L.orc_race.argtypes = [C.c_int, f32p, u8p, C.c_uint64, C.c_uint32, C.c_uint32,
                                   C.c_uint32]
            L.orc_race.restype = C.c_int
            L.orc_construct_rule.argtypes = [C.c_int, C.c_int, f32p, i32p, C.c_uint64, C.c_uint32,
                                             C.c_int, i32p, i64p]
            L.orc_construct_rule.restype = None
            L.orc_run_rule.argtypes = [C.c_int, i32p, C.c_float, C.c_float, C.c_float, C.c_int,
                                       C.c_uint64, C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp]
            L.orc_run_rule.restype = C.c_int
            L.orc_nn_lists.argtypes = [C.c_int, i32p, C.c_int, i32p]
            L.orc_nn_lists.restype = None
            L.orc_nn_select.argtypes = [C.c_int, C.c_int, i32p, f32p, u8p, C.c_uint64]
            L.orc_nn_select.restype = C.c_int
            L.orc_construct_nn.argtypes = [C.c_int, C.c_int, f32p, i32p, C.c_uint64, C.c_uint32,
                                           C.c_int, C.c_int, vp, i32p, i64p]
            L.orc_construct_nn.restype = None
            L.orc_run_nn.argtypes = [C.c_int, i32p, C.c_float, C.c_float, C.c_float, C.c_int,
                                     C.c_uint64, C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, vp,
                                     vp, vp]
            L.orc_run_nn.restype = C.c_int
            L.orc_mmas_limits.argtypes = [C.c_int, C.c_float, C.c_double, C.c_int64, f32p, f32p]
            L.orc_mmas_limits.restype = None
            L.orc_update_mmas.argtypes = [C.c_int, i32p, C.c_int64, C.c_float, C.c_float,
                                          C.c_float, f32p]
            L.orc_update_mmas.restype = None
            L.orc_run_mmas.argtypes = [C.c_int, i32p, C.c_float, C.c_float, C.c_float, C.c_int,
                                       C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                                       vp, vp, vp, vp, vp, vp, vp, vp]
            L.orc_run_mmas.restype = C.c_int
            L.orc_acs_threshold.argtypes = [C.c_double]
            L.orc_acs_threshold.restype = C.c_uint64
            L.orc_acs_select.argtypes = [C.c_int, f32p, u8p, C.c_uint64, C.c_uint32, C.c_uint64]
            L.orc_acs_select.restype = C.c_int
            L.orc_acs_select_nn.argtypes = [C.c_int, C.c_int, i32p, f32p, u8p, C.c_uint64,
                                            C.c_uint32, C.c_uint64]
            L.orc_acs_select_nn.restype = C.c_int
            L.orc_acs_local.argtypes = [C.c_float, C.c_float, C.c_float]
            L.orc_acs_local.restype = C.c_float
            L.orc_run_acs.argtypes = [C.c_int, i32p, C.c_float, C.c_float, C.c_float, C.c_int,
                                      C.c_uint64, C.c_int, C.c_double, C.c_float,
                                      vp, vp, vp, vp, vp, vp]
            L.orc_run_acs.restype = C.c_int
            L.orc_run_acs_nn.argtypes = [C.c_int, i32p, C.c_float, C.c_float, C.c_float,
                                         C.c_int, C.c_uint64, C.c_int, C.c_double, C.c_float,
                                         C.c_int, vp, vp, vp, vp, vp, vp]
            L.orc_run_acs_nn.restype = C.c_int
            L.orc_brute_force.argtypes = [C.c_int, i32p, i32p]
            L.orc_brute_force.restype = C.c_int64
            _lib = L
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def set_threads(threads: int) -> int:
    """Host threads for the ants of one construction (1 = the plain loop).
    The results do not depend on it.  Returns the count in effect."""
    return int(lib().orc_set_threads(int(threads)))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def hardware_threads() -> int:
    """Online host cores (sysconf), the count an all-core run uses."""
    return int(lib().orc_hardware_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def ceil_log2(v: int) -> int:
    return int(lib().orc_ceil_log2(int(v)))


def roulette(w, visited, r: int) -> int:
    w = np.ascontiguousarray(w, np.float32)
    v = np.ascontiguousarray(visited, np.uint8)
    return int(lib().orc_roulette(len(w), w, v, C.c_uint64(r)))


def roulette_weights(w, visited):
    w = np.ascontiguousarray(w, np.float32)
    v = np.ascontiguousarray(visited, np.uint8)
    q = np.zeros(len(w), np.uint64)
    Q = lib().orc_roulette_weights(len(w), w, v, q)
    return q, int(Q)


def heta(dist, beta: float) -> np.ndarray:
    d = _i32(dist)
    out = np.zeros(d.shape, np.float32)
    lib().orc_heta(d.shape[0], d, float(beta), out)
    return out


def nn_tour_length(dist) -> int:
    d = _i32(dist)
    return int(lib().orc_nn_tour_length(d.shape[0], d))


def tau0(dist, m: int) -> float:
    d = _i32(dist)
    return float(np.float32(lib().orc_tau0(d.shape[0], int(m), d)))


def choice(tau, heta_, alpha: float) -> np.ndarray:
    tau = np.ascontiguousarray(tau, np.float32)
    h = np.ascontiguousarray(heta_, np.float32)
    out = np.zeros_like(tau)
    lib().orc_choice(tau.shape[0], tau, h, float(alpha), out)
    return out


def construct_ant(choice_, dist, seed: int, iteration: int, ant: int):
    ch = np.ascontiguousarray(choice_, np.float32)
    d = _i32(dist)
    n = d.shape[0]
    tour = np.zeros(n + 1, np.int32)
    length = lib().orc_construct_ant(n, ch, d, C.c_uint64(seed), iteration, ant, tour)
    return tour, int(length)


def construct(choice_, dist, m: int, seed: int, iteration: int, rule: int = 0):
    """rule 0: Eq. 1 by the integer roulette; rule 1: the paper's data-parallel rule;
    rule 3: the exponential race (R15)."""
    ch = np.ascontiguousarray(choice_, np.float32)
    d = _i32(dist)
    n = d.shape[0]
    tours = np.zeros((m, n + 1), np.int32)
    lens = np.zeros(m, np.int64)
    lib().orc_construct_rule(n, m, ch, d, C.c_uint64(seed), iteration, rule, tours, lens)
    return tours, lens


def nn_lists(dist, nn: int) -> np.ndarray:
    d = _i32(dist)
    n = d.shape[0]
    out = np.zeros((n, nn), np.int32)
    lib().orc_nn_lists(n, d, nn, out)
    return out


def nn_select(list_row, w, visited, r: int) -> int:
    lst = np.ascontiguousarray(list_row, np.int32)
    w = np.ascontiguousarray(w, np.float32)
    v = np.ascontiguousarray(visited, np.uint8)
    return int(lib().orc_nn_select(len(w), len(lst), lst, w, v, C.c_uint64(r)))


def construct_nn(choice_, dist, m: int, seed: int, iteration: int, nn: int):
    """Tours by the nearest-neighbour-list rule (reading R9)."""
    ch = np.ascontiguousarray(choice_, np.float32)
    d = _i32(dist)
    n = d.shape[0]
    lists = nn_lists(d, nn)
    tours = np.zeros((m, n + 1), np.int32)
    lens = np.zeros(m, np.int64)
    lib().orc_construct_nn(n, m, ch, d, C.c_uint64(seed), iteration, 2, nn, lists.ctypes.data,
                           tours, lens)
    return tours, lens


def candidate_uniform(seed: int, step: int, ant: int, iteration: int, j: int) -> float:
    return float(np.float32(lib().orc_candidate_uniform(C.c_uint64(seed), step, ant, iteration, j)))


def iroulette(w, visited, seed: int, step: int, ant: int, iteration: int) -> int:
    w = np.ascontiguousarray(w, np.float32)
    v = np.ascontiguousarray(visited, np.uint8)
    return int(lib().orc_iroulette(len(w), w, v, C.c_uint64(seed), step, ant, iteration))


def race_exponentials(v) -> np.ndarray:
    """E = -ln(v 2^-24) in single precision by the series of R15, for integers v in [1, 2^24]."""
    v = np.ascontiguousarray(v, np.uint32)
    out = np.empty(v.shape, np.float32)
    lib().orc_race_exponentials(v.size, v.ctypes.data, out.ctypes.data)
    return out


def race(w, visited, seed: int, step: int, ant: int, iteration: int) -> int:
    """One step of the exponential race (R15) over the row w."""
    w = np.ascontiguousarray(w, np.float32)
    v = np.ascontiguousarray(visited, np.uint8)
    return int(lib().orc_race(len(w), w, v, C.c_uint64(seed), step, ant, iteration))


def deposit_scale(lens) -> int:
    lens = np.ascontiguousarray(lens, np.int64)
    return int(lib().orc_deposit_scale(len(lens), lens))


def update_mirror(tau, tours, lens, rho: float) -> np.ndarray:
    tau = np.array(tau, dtype=np.float32, copy=True, order="C")
    tours = _i32(tours)
    lens = np.ascontiguousarray(lens, np.int64)
    lib().orc_update_mirror(tau.shape[0], tours.shape[0], tours, lens, float(rho), tau)
    return tau


def update_fp64(tau, tours, lens, rho: float) -> np.ndarray:
    tau = np.array(tau, dtype=np.float64, copy=True, order="C")
    tours = _i32(tours)
    lens = np.ascontiguousarray(lens, np.int64)
    lib().orc_update_fp64(tau.shape[0], tours.shape[0], tours, lens, float(rho), tau)
    return tau


def mmas_limits(n: int, rho: float, p_best: float, c_gb: int):
    """(tau_min, tau_max) of the MAX-MIN Ant System for best-so-far length c_gb (R13)."""
    lo = np.zeros(1, np.float32)
    hi = np.zeros(1, np.float32)
    lib().orc_mmas_limits(int(n), float(rho), float(p_best), int(c_gb), lo, hi)
    return float(lo[0]), float(hi[0])


def update_mmas(tau, dep_tour, dep_len: int, rho: float, tau_min: float, tau_max: float):
    """One MMAS update of a copy of tau (float): the tour dep_tour deposits, then the clamp."""
    tau = np.array(tau, dtype=np.float32, copy=True, order="C")
    lib().orc_update_mmas(tau.shape[0], _i32(dep_tour), int(dep_len), float(rho),
                          float(tau_min), float(tau_max), tau)
    return tau


def run_mmas(dist, m: int, iterations: int, seed: int, alpha=1.0, beta=2.0, rho=0.02,
             p_best=0.05, best_so_far=False, rule: int = 0, nn: int = 0) -> dict:
    """A whole MAX-MIN Ant System run (R13), float state with fp64 carried alongside."""
    d = _i32(dist)
    n = d.shape[0]
    best_tour = np.zeros(n + 1, np.int32)
    best_len = np.zeros(1, np.int64)
    tau32 = np.zeros((n, n), np.float32)
    tau64 = np.zeros((n, n), np.float64)
    tours = np.zeros((m, n + 1), np.int32)
    lens = np.zeros(m, np.int64)
    iter_best = np.zeros(max(iterations, 1), np.int64)
    limits = np.zeros(2, np.float32)
    rc = lib().orc_run_mmas(n, d, float(alpha), float(beta), float(rho), int(m),
                            C.c_uint64(seed), int(iterations), int(rule), int(nn),
                            float(p_best), int(bool(best_so_far)),
                            best_tour.ctypes.data, best_len.ctypes.data, tau32.ctypes.data,
                            tau64.ctypes.data, tours.ctypes.data, lens.ctypes.data,
                            iter_best.ctypes.data, limits.ctypes.data)
    if rc != 0:
        raise ValueError("oracle MMAS run failed")
    return dict(best_tour=best_tour, best_len=int(best_len[0]), tau32=tau32, tau64=tau64,
                tours=tours, lens=lens, iter_best=iter_best[:iterations],
                tau_min=float(limits[0]), tau_max=float(limits[1]))


def acs_threshold(q0: float) -> int:
    return int(lib().orc_acs_threshold(float(q0)))


def acs_select(w, visited, r: int, x2: int, q0: float) -> int:
    """One step of the Ant Colony System's pseudo-random proportional rule (R14)."""
    w = np.ascontiguousarray(w, np.float32)
    v = np.ascontiguousarray(visited, np.uint8)
    return int(lib().orc_acs_select(w.shape[0], w, v, C.c_uint64(r), C.c_uint32(x2),
                                    C.c_uint64(acs_threshold(q0))))


def acs_select_nn(w, visited, lst, r: int, x2: int, q0: float) -> int:
    """One step of the Ant Colony System with a nearest-neighbour list (R16)."""
    w = np.ascontiguousarray(w, np.float32)
    v = np.ascontiguousarray(visited, np.uint8)
    lst = np.ascontiguousarray(lst, np.int32)
    return int(lib().orc_acs_select_nn(w.shape[0], lst.shape[0], lst, w, v, C.c_uint64(r),
                                       C.c_uint32(x2), C.c_uint64(acs_threshold(q0))))


def acs_local(tau: float, xi: float, tau0: float) -> float:
    return float(np.float32(lib().orc_acs_local(float(tau), float(xi), float(tau0))))


def run_acs(dist, m: int, iterations: int, seed: int, alpha=1.0, beta=2.0, rho=0.1,
            q0=0.9, xi=0.1, nn: int = 0) -> dict:
    """A whole Ant Colony System run (R14); nn > 0: with nearest-neighbour lists (R16)."""
    d = _i32(dist)
    n = d.shape[0]
    best_tour = np.zeros(n + 1, np.int32)
    best_len = np.zeros(1, np.int64)
    tau = np.zeros((n, n), np.float32)
    tours = np.zeros((m, n + 1), np.int32)
    lens = np.zeros(m, np.int64)
    iter_best = np.zeros(max(iterations, 1), np.int64)
    rc = lib().orc_run_acs_nn(n, d, float(alpha), float(beta), float(rho), int(m),
                              C.c_uint64(seed), int(iterations), float(q0), float(xi), int(nn),
                              best_tour.ctypes.data, best_len.ctypes.data, tau.ctypes.data,
                              tours.ctypes.data, lens.ctypes.data, iter_best.ctypes.data)
    if rc != 0:
        raise ValueError("oracle ACS run failed")
    return dict(best_tour=best_tour, best_len=int(best_len[0]), tau32=tau, tours=tours,
                lens=lens, iter_best=iter_best[:iterations])


def run(dist, m: int, iterations: int, seed: int, alpha=1.0, beta=2.0, rho=0.5,
        rule: int = 0, nn: int = 0) -> dict:
    """A whole Ant System run in mirror mode, with the fp64 pheromone carried alongside.

    rule 0 selects by Eq. 1, rule 1 by the paper's data-parallel rule, rule 2
    by nearest-neighbour lists of length nn, rule 3 by the exponential race."""
    d = _i32(dist)
    n = d.shape[0]
    best_tour = np.zeros(n + 1, np.int32)
    best_len = np.zeros(1, np.int64)
    tau32 = np.zeros((n, n), np.float32)
    tau64 = np.zeros((n, n), np.float64)
    tours = np.zeros((m, n + 1), np.int32)
    lens = np.zeros(m, np.int64)
    iter_best = np.zeros(max(iterations, 1), np.int64)
    rc = lib().orc_run_nn(n, d, float(alpha), float(beta), float(rho), int(m),
                       C.c_uint64(seed), int(iterations), int(rule), int(nn),
                       best_tour.ctypes.data, best_len.ctypes.data,
                       tau32.ctypes.data, tau64.ctypes.data, tours.ctypes.data,
                       lens.ctypes.data, iter_best.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle run failed")
    return dict(best_tour=best_tour, best_len=int(best_len[0]), tau32=tau32, tau64=tau64,
                tours=tours, lens=lens, iter_best=iter_best[:iterations])


def brute_force(dist):
    d = _i32(dist)
    n = d.shape[0]
    tour = np.zeros(n + 1, np.int32)
    best = lib().orc_brute_force(n, d, tour)
    return int(best), tour
