"""Pins of the CPU oracle against what the paper and mathematics fix (no GPU).

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, invariants of Eqs. 1-4, brute force, or a
statistical test against the probabilities of Eq. 1.  The cases are chosen so
that a plausible slip in the oracle (a dropped term, rho in place of 1 - rho, a
transposed operand, >= in place of >, the wrong row) fails at least one test.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1101_2678_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Philox4x32-10 (the random numbers of reading R1)
# --------------------------------------------------------------------------

def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert list(orc.philox4x32_10(ctr, key)) == out


def test_philox_uniformity(orc):
    # 4 * 20000 words: the top 4 bits should be uniform over 16 bins.
    from scipy.stats import chisquare
    words = np.concatenate([orc.philox4x32_10([i, 7, 3, 0], [11, 13]) for i in range(20000)])
    hist = np.bincount((words >> 28).astype(np.int64), minlength=16)
    assert chisquare(hist).pvalue > 1e-3


# --------------------------------------------------------------------------
# Eq. 1: the random proportional rule, sampled by the integer roulette
# --------------------------------------------------------------------------

def test_ceil_log2(orc):
    for v, c in [(1, 0), (2, 1), (3, 2), (4, 2), (5, 3), (48, 6), (1002, 10), (1024, 10),
                 (1025, 11), (2392, 12), (4096, 12)]:
        assert orc.ceil_log2(v) == c


def test_roulette_weights_are_proportional(orc):
    # q_j / Q must equal w_j / sum(w) (Eq. 1) up to the quantisation step,
    # i.e. |q_j/Q - p_j| <= n / 2^(B-1) with B = 46 bits per weight.
    rng = np.random.default_rng(0)
    for n in [3, 6, 48, 1002, 4096]:
        w = rng.lognormal(0.0, 3.0, size=n).astype(np.float32)
        vis = (rng.uniform(size=n) < 0.3).astype(np.uint8)
        vis[int(np.argmax(w))] = 0
        q, Q = orc.roulette_weights(w, vis)
        assert Q == int(q.sum()) and Q < 2**62
        W = sum(Fraction(float(x)) for x, v in zip(w, vis) if not v)
        B = 46
        assert int(q.max()) < 2**B <= 2 * int(q.max())
        for j in range(n):
            if vis[j]:
                assert q[j] == 0
                continue
            p = Fraction(float(w[j])) / W
            assert abs(Fraction(int(q[j]), Q) - p) <= Fraction(n, 2 ** (B - 1))


def test_roulette_boundaries_pick_first_prefix_above_target(orc):
    # T = floor(r Q / 2^64); the chosen city is the first j with prefix_j > T.
    w = np.array([0.5, 0.0, 2.0, 1.25, 0.75, 3.0], np.float32)
    vis = np.array([0, 0, 0, 1, 0, 0], np.uint8)
    q, Q = orc.roulette_weights(w, vis)
    prefix = np.cumsum(q.astype(object))

    def r_for(T):  # smallest r with floor(r Q / 2^64) == T
        return -((-T << 64) // Q)

    for j in range(len(w)):
        if q[j] == 0:
            continue
        lo = int(prefix[j] - q[j])
        hi = int(prefix[j]) - 1
        assert orc.roulette(w, vis, r_for(lo)) == j
        assert orc.roulette(w, vis, r_for(hi)) == j
    assert orc.roulette(w, vis, 0) == 0
    assert orc.roulette(w, vis, 2**64 - 1) == 5


def test_roulette_degenerate_cases(orc):
    w = np.zeros(5, np.float32)
    vis = np.array([1, 1, 0, 0, 1], np.uint8)
    # all unvisited weights zero: the lowest-index unvisited city
    assert orc.roulette(w, vis, 12345) == 2
    # only one unvisited city: always it, whatever r
    vis1 = np.array([1, 1, 1, 0, 1], np.uint8)
    w1 = np.array([5, 5, 5, 1e-30, 5], np.float32)
    for r in [0, 1, 2**63, 2**64 - 1]:
        assert orc.roulette(w1, vis1, r) == 3
    # everything visited
    assert orc.roulette(w1, np.ones(5, np.uint8), 7) == -1
    # subnormal weights are weighted exactly like normal ones
    ws = np.array([2.0**-149, 2.0**-148, 0, 0], np.float32)
    q, Q = orc.roulette_weights(ws, np.zeros(4, np.uint8))
    assert q[1] == 2 * q[0] and Q == 3 * q[0]


@pytest.mark.parametrize("visited", [[], [1, 4]])
def test_roulette_chi_squared_against_eq1(orc, visited):
    # Frequencies of the first move out of city 0 versus p_0j of Eq. 1.
    from scipy.stats import chisquare
    n = 6
    w = np.array([0.0, 0.9, 0.05, 2.5, 0.3, 1.25], np.float32)
    vis = np.zeros(n, np.uint8)
    vis[0] = 1
    vis[visited] = 1
    draws = 100_000
    counts = np.zeros(n, np.int64)
    for i in range(draws):
        x = orc.philox4x32_10([1, i, 0, 0], [99, 0])
        r = (int(x[1]) << 32) | int(x[0])
        counts[orc.roulette(w, vis, r)] += 1
    cand = [j for j in range(n) if not vis[j]]
    p = np.array([w[j] for j in cand], np.float64)
    p /= p.sum()
    assert counts[vis == 1].sum() == 0
    res = chisquare(counts[cand], p * draws)
    assert res.pvalue > 0.01, (counts, p * draws)


def test_first_step_uses_row_of_current_city(orc):
    # With an asymmetric choice matrix the second city of each tour must follow
    # row tour[0] (not the column): per start city, chi-squared against Eq. 1.
    from scipy.stats import chisquare
    n = 4
    ch = np.array([[0, 1, 2, 5],
                   [3, 0, 1, 1],
                   [1, 8, 0, 1],
                   [2, 2, 4, 0]], np.float32)
    d = np.ones((n, n), np.int32) - np.eye(n, dtype=np.int32)
    counts = np.zeros((n, n), np.int64)
    for it in range(60):
        tours, _ = orc.construct(ch, d, 500, seed=5, iteration=it)
        np.add.at(counts, (tours[:, 0], tours[:, 1]), 1)
    for i in range(n):
        row = ch[i].astype(np.float64)
        cand = [j for j in range(n) if j != i]
        p = row[cand] / row[cand].sum()
        assert counts[i, i] == 0
        assert chisquare(counts[i, cand], p * counts[i].sum()).pvalue > 0.01


def test_start_city_is_uniform(orc):
    from scipy.stats import chisquare
    n = 7
    ch = np.ones((n, n), np.float32)
    d = np.ones((n, n), np.int32) - np.eye(n, dtype=np.int32)
    starts = np.concatenate([orc.construct(ch, d, 700, 3, it)[0][:, 0] for it in range(20)])
    assert chisquare(np.bincount(starts, minlength=n)).pvalue > 0.01


# --------------------------------------------------------------------------
# Tours (Section II: each ant visits every city exactly once; C^k = sum of d)
# --------------------------------------------------------------------------

def test_tours_are_closed_permutations_with_summed_lengths(orc):
    inst = I.uniform_instance(37, 1000, seed=9)
    h = orc.heta(inst.dist, 2.0)
    ch = orc.choice(np.where(np.eye(37) > 0, 0, 0.01).astype(np.float32), h, 1.0)
    tours, lens = orc.construct(ch, inst.dist, 29, seed=4, iteration=3)
    for k in range(29):
        t = tours[k]
        assert sorted(t[:-1].tolist()) == list(range(37)) and t[-1] == t[0]
        assert lens[k] == int(inst.dist[t[:-1], t[1:]].astype(np.int64).sum())


# --------------------------------------------------------------------------
# Setup: heuristic (eta = 1/d, Section II), nearest-neighbour tour, tau0
# --------------------------------------------------------------------------

def test_heta_is_inverse_distance_power(orc):
    inst = I.uniform_instance(50, 1000, seed=2)
    d = inst.dist.astype(np.float64)
    off = ~np.eye(50, dtype=bool)
    for beta in [1.0, 2.0, 3.0, 2.5, 0.0]:
        h = orc.heta(inst.dist, beta).astype(np.float64)
        assert np.all(np.diag(h) == 0)
        # h * d^beta == 1 up to one float rounding (plus the double rounding)
        err = np.abs(h[off] * d[off] ** beta - 1.0)
        assert err.max() <= 2.0 ** -23


# --------------------------------------------------------------------------
# choice_info = tau^alpha * eta^beta (Section III-A, the choice kernel)
# --------------------------------------------------------------------------

# (tau, alpha, tau^alpha) with every power exactly representable, so the
# expected value is exact whatever the pow implementation's rounding.
_EXACT_POWERS = [
    (4.0, 0.5, 2.0), (9.0, 0.5, 3.0), (0.25, 0.5, 0.5), (2.0 ** -4, 0.5, 2.0 ** -2),
    (4.0, 1.5, 8.0), (2.0 ** -4, 1.5, 2.0 ** -6), (0.25, 1.5, 0.125), (9.0, 1.5, 27.0),
    (3.0, 2.0, 9.0), (2.0 ** -4, 2.0, 2.0 ** -8), (5.0, 2.0, 25.0),
    (3.0, 3.0, 27.0), (0.5, 3.0, 0.125), (16.0, 0.25, 2.0), (2.0 ** -8, 0.25, 0.25),
]


@pytest.mark.parametrize("alpha", sorted({a for _, a, _ in _EXACT_POWERS}))
def test_choice_info_powers_of_tau(orc, alpha):
    # Cells (i, j) with different tau and heta in the two halves, so that a
    # swapped base and exponent, a dropped exponent, tau and heta read from
    # different cells, or a missing heta factor all change some cell.
    cases = [(t, p) for t, a, p in _EXACT_POWERS if a == alpha]
    n = 2 * len(cases) + 1
    tau = np.zeros((n, n), np.float32)
    heta = np.zeros((n, n), np.float32)
    want = np.zeros((n, n), np.float64)
    hvals = [0.75, 1.25, 0.5, 3.0, 0.375]
    for k, (t, p) in enumerate(cases):
        i, j = 2 * k, 2 * k + 1
        h = hvals[k % len(hvals)]
        tau[i, j], heta[i, j], want[i, j] = t, h, p * h      # exact: p and h have short significands
        tau[j, i], heta[j, i], want[j, i] = 1.0, 2.0 * h, 2.0 * h   # 1^alpha = 1
    ch = orc.choice(tau, heta, alpha).astype(np.float64)
    assert np.array_equal(ch, want)


def test_choice_info_alpha_one_and_zero(orc):
    # alpha = 1: the correctly rounded product tau * heta (the exact product
    # of two floats fits in a double; one rounding to float).  alpha = 0:
    # heta itself, whatever tau is (0^0 = 1 included).
    rng = np.random.default_rng(7)
    n = 64
    tau = rng.uniform(1e-6, 3.0, (n, n)).astype(np.float32)
    tau[0, :8] = 0.0
    heta = rng.uniform(1e-8, 1.0, (n, n)).astype(np.float32)
    exact = tau.astype(np.float64) * heta.astype(np.float64)
    assert np.array_equal(orc.choice(tau, heta, 1.0), exact.astype(np.float32))
    assert np.array_equal(orc.choice(tau, heta, 0.0), heta)


def test_nearest_neighbour_tour_closed_forms(orc):
    # cities on a line at x = 0..n-1: the NN tour walks out and back, 2(n-1)
    n = 12
    coords = np.stack([np.arange(n), np.zeros(n)], axis=1)
    d = I.distance_matrix(coords)
    assert orc.nn_tour_length(d) == 2 * (n - 1)
    assert orc.tau0(d, 30) == np.float32(30 / (2 * (n - 1)))
    # shuffled line: from any start the greedy walk sweeps to one end, jumps
    # back past the start and sweeps to the other end: again 2(n-1)
    for s in range(5):
        perm = np.random.default_rng(s).permutation(n)
        assert orc.nn_tour_length(I.distance_matrix(coords[perm])) == 2 * (n - 1)
    # a tie at the first step: (10,0) and (0,10) are both 10 away from city 0;
    # the lower index (1) gives 10 + 14 + 22 + 32 = 78, the other choice 86
    pts = np.array([[0, 0], [10, 0], [0, 10], [10, 30]])
    assert orc.nn_tour_length(I.distance_matrix(pts)) == 78


# --------------------------------------------------------------------------
# Pheromone update, Eqs. 2-4
# --------------------------------------------------------------------------

def _random_tours(n, m, seed):
    rng = np.random.default_rng(seed)
    tours = np.zeros((m, n + 1), np.int32)
    for k in range(m):
        p = rng.permutation(n)
        tours[k, :n] = p
        tours[k, n] = p[0]
    return tours


def _lens(d, tours):
    return d[tours[:, :-1], tours[:, 1:]].astype(np.int64).sum(axis=1)


@pytest.mark.parametrize("rho", [0.3, 0.5, 1.0])
def test_single_ant_update_closed_form(orc, rho):
    # m = 1: on-tour edges get (1-rho) tau + 1/C, off-tour edges (1-rho) tau (Eqs. 2-4).
    n = 9
    inst = I.uniform_instance(n, 1000, seed=4)
    rng = np.random.default_rng(3)
    tau = rng.uniform(0.1, 2.0, size=(n, n)).astype(np.float32)
    tau = ((tau + tau.T) / 2).astype(np.float32)
    np.fill_diagonal(tau, 0)
    tours = _random_tours(n, 1, 5)
    lens = _lens(inst.dist, tours)
    out = orc.update_mirror(tau, tours, lens, rho)
    keep = np.float32(1.0) - np.float32(rho)
    dk = np.float32(1.0 / float(lens[0]))
    on = np.zeros((n, n), bool)
    t = tours[0]
    on[t[:-1], t[1:]] = True
    on[t[1:], t[:-1]] = True
    expect = (keep * tau).astype(np.float32)
    expect[on] = (expect[on] + dk).astype(np.float32)
    assert np.array_equal(out, expect)
    out64 = orc.update_fp64(tau.astype(np.float64), tours, lens, rho)
    e64 = (1 - rho) * tau.astype(np.float64)
    e64[on] += 1.0 / float(lens[0])
    assert np.allclose(out64, e64, rtol=1e-15, atol=0)


def test_update_invariants(orc):
    # Total deposit = 2 n sum_k 1/C^k (each tour has n edges, each counted in
    # both directions); tau stays symmetric; mirror within 1e-6 of fp64.
    n, m, rho = 31, 40, 0.5
    inst = I.uniform_instance(n, 1000, seed=6)
    tau = np.full((n, n), 0.02, np.float32)
    np.fill_diagonal(tau, 0)
    tours = _random_tours(n, m, 8)
    # make several ants share edges (the converged case)
    tours[10:20] = tours[0]
    lens = _lens(inst.dist, tours)
    out = orc.update_mirror(tau, tours, lens, rho)
    out64 = orc.update_fp64(tau.astype(np.float64), tours, lens, rho)
    assert np.array_equal(out, out.T)
    assert np.allclose(out64, out64.T, rtol=1e-14)
    dep64 = out64 - (1 - rho) * tau.astype(np.float64)
    assert math.isclose(dep64.sum(), 2 * n * float((1.0 / lens).sum()), rel_tol=1e-12)
    rel = np.abs(out.astype(np.float64) - out64) / np.maximum(out64, 1e-300)
    assert rel.max() < 1e-6
    assert np.all(np.diag(out) == 0)


def test_deposit_fixed_point_is_exact_sum(orc):
    # sum_k q_k 2^-S equals sum_k dtau_k up to m * 2^-S, and q never overflows.
    rng = np.random.default_rng(11)
    lens = rng.integers(3, 10**7, size=3000).astype(np.int64)
    S = orc.deposit_scale(lens)
    m = len(lens)
    dts = [Fraction(float(np.float32(1.0 / float(c)))) for c in lens]
    qs = [math.floor(x * 2**S) for x in dts]
    assert max(qs) * m < 2**63
    assert abs(Fraction(sum(qs), 2**S) - sum(dts)) <= Fraction(m, 2**S)
    assert max(qs) >= 2 ** (62 - orc.ceil_log2(m) - 1)


# --------------------------------------------------------------------------
# Whole runs: brute force, FP64 agreement, determinism
# --------------------------------------------------------------------------

def test_brute_force_on_convex_polygon(orc):
    # Points on a circle, shuffled: the optimum visits them in angular order.
    n = 9
    ang = np.linspace(0, 2 * np.pi, n, endpoint=False)
    pts = np.rint(np.stack([5000 + 4000 * np.cos(ang), 5000 + 4000 * np.sin(ang)], 1))
    perm = np.random.default_rng(2).permutation(n)
    d = I.distance_matrix(pts[perm])
    hull = I.distance_matrix(pts)
    perimeter = int(sum(hull[i, (i + 1) % n] for i in range(n)))
    best, tour = orc.brute_force(d)
    assert best == perimeter
    assert int(d[tour[:-1], tour[1:]].sum()) == best


@pytest.mark.parametrize("n,seed", [(8, 21), (9, 22), (10, 23)])
def test_ant_system_reaches_brute_force_optimum(orc, n, seed):
    inst = I.uniform_instance(n, 1000, seed=seed)
    opt, _ = orc.brute_force(inst.dist)
    res = orc.run(inst.dist, m=n, iterations=100, seed=seed)
    assert np.all(res["iter_best"] >= opt)
    assert res["best_len"] == opt
    t = res["best_tour"]
    assert int(inst.dist[t[:-1], t[1:]].sum()) == opt


def test_run_fp32_mirror_tracks_fp64(orc):
    w = I.workload_n48()
    res = orc.run(w["inst"].dist, w["m"], 100, w["seed"])
    r64, r32 = res["tau64"], res["tau32"].astype(np.float64)
    assert np.all(np.abs(r32 - r64) <= 1e-5 * np.abs(r64) + 2.0 ** -126)
    assert res["best_len"] == res["iter_best"].min()
    again = orc.run(w["inst"].dist, w["m"], 100, w["seed"])
    assert np.array_equal(again["tau32"], res["tau32"]) and again["best_len"] == res["best_len"]


# --------------------------------------------------------------------------
# The paper's data-parallel selection rule (Section III-A; reading R8)
# --------------------------------------------------------------------------

def _iroulette_freqs(orc, w, vis, draws):
    counts = np.zeros(len(w), np.int64)
    for i in range(draws):
        counts[orc.iroulette(w, vis, 17, 1 + (i % 997), i // 997, 3)] += 1
    return counts


def test_candidate_uniforms_lie_in_unit_interval_and_are_uniform(orc):
    from scipy.stats import kstest
    u = np.array([orc.candidate_uniform(5, s, 3, 0, j) for s in range(50) for j in range(40)])
    assert u.min() > 0 and u.max() <= 1
    assert np.all(u * 2**24 == np.rint(u * 2**24))
    assert kstest(u, "uniform").pvalue > 0.01


def test_iroulette_two_candidates_closed_form(orc):
    # w1 >= w2: city 2 wins u2 w2 > u1 w1 with probability w2 / (2 w1).
    from scipy.stats import binomtest
    w = np.array([0.0, 3.0, 1.0], np.float32)
    vis = np.array([1, 0, 0], np.uint8)
    counts = _iroulette_freqs(orc, w, vis, 40_000)
    assert counts[0] == 0
    assert binomtest(int(counts[2]), int(counts.sum()), 1.0 / 6.0).pvalue > 0.01


def test_iroulette_chi_squared_against_integral_closed_form(orc):
    # P(j) = int_0^1 prod_{l != j} min(1, x w_j / w_l) dx for independent
    # uniforms u_l; checked on four candidates and one visited city.
    from scipy.integrate import quad
    from scipy.stats import chisquare
    w = np.array([1.0, 2.0, 0.5, 4.0, 3.0], np.float32)
    vis = np.array([0, 0, 0, 0, 1], np.uint8)
    cand = [j for j in range(5) if not vis[j]]
    p = []
    for j in cand:
        f = lambda x, j=j: np.prod([min(1.0, x * w[j] / w[l]) for l in cand if l != j])
        p.append(quad(f, 0, 1, limit=200)[0])
    p = np.array(p)
    assert abs(p.sum() - 1) < 1e-9
    counts = _iroulette_freqs(orc, w, vis, 60_000)
    assert counts[4] == 0
    assert chisquare(counts[cand], p * counts.sum()).pvalue > 0.01


def test_iroulette_degenerate_rows_and_tours(orc):
    w = np.zeros(6, np.float32)
    vis = np.array([1, 0, 1, 0, 0, 0], np.uint8)
    assert orc.iroulette(w, vis, 1, 1, 0, 0) == 1
    inst = I.uniform_instance(23, 1000, seed=3)
    h = orc.heta(inst.dist, 2.0)
    ch = orc.choice(np.where(np.eye(23) > 0, 0, 0.3).astype(np.float32), h, 1.0)
    tours, lens = orc.construct(ch, inst.dist, 11, seed=2, iteration=1, rule=1)
    for k in range(11):
        t = tours[k]
        assert sorted(t[:-1].tolist()) == list(range(23)) and t[-1] == t[0]
        assert lens[k] == int(inst.dist[t[:-1], t[1:]].astype(np.int64).sum())
    # starts are shared with Eq. 1 (same counter), later moves differ in general
    t0, _ = orc.construct(ch, inst.dist, 11, seed=2, iteration=1, rule=0)
    assert np.array_equal(t0[:, 0], tours[:, 0])


# --------------------------------------------------------------------------
# The exponential race (reading R15): a per-candidate random rule for Eq. 1
# --------------------------------------------------------------------------

def test_race_exponential_is_minus_log_of_the_uniform(orc):
    # every one of the 2^24 uniforms: within 3 units in the last place of the
    # float nearest -ln(v 2^-24), exactly 0 at v = 2^24, and non-increasing
    prev_last = np.inf
    for lo in range(1, (1 << 24) + 1, 1 << 22):
        v = np.arange(lo, min(lo + (1 << 22), (1 << 24) + 1), dtype=np.uint32)
        e = orc.race_exponentials(v)
        true = -np.log(v.astype(np.float64) / 2.0**24)
        ulp = np.spacing(np.abs(true).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(e.astype(np.float64) - true) <= 3 * ulp)
        assert e[0] <= prev_last and np.all(np.diff(e) <= 0)
        prev_last = e[-1]
    assert prev_last == 0.0
    assert orc.race_exponentials(np.array([1], np.uint32))[0] == np.float32(24 * math.log(2))


def _race_freqs(orc, w, vis, draws):
    counts = np.zeros(len(w), np.int64)
    for i in range(draws):
        counts[orc.race(w, vis, 23, 1 + (i % 997), i // 997, 5)] += 1
    return counts


def test_race_samples_eq1(orc):
    # the minimum of independent exponentials of rates w_j is j with
    # probability w_j / sum w: Eq. 1, unlike the product rule of R8
    from scipy.stats import binomtest, chisquare
    w = np.array([1.0, 2.0, 0.5, 4.0, 3.0, 0.0], np.float32)
    vis = np.array([0, 0, 0, 0, 1, 0], np.uint8)
    counts = _race_freqs(orc, w, vis, 60_000)
    assert counts[4] == 0 and counts[5] == 0
    cand = [0, 1, 2, 3]
    p = w[cand].astype(np.float64) / float(w[cand].sum())
    assert chisquare(counts[cand], p * counts.sum()).pvalue > 0.01
    # two candidates w1 = 3 w2: city 2 with probability 1/4 (the product
    # rule of R8 gives 1/6)
    w2 = np.array([0.0, 3.0, 1.0], np.float32)
    c2 = _race_freqs(orc, w2, np.array([1, 0, 0], np.uint8), 40_000)
    assert binomtest(int(c2[2]), int(c2.sum()), 0.25).pvalue > 0.01


def test_race_degenerate_rows_and_tours(orc):
    w = np.zeros(6, np.float32)
    vis = np.array([1, 0, 1, 0, 0, 0], np.uint8)
    assert orc.race(w, vis, 1, 1, 0, 0) == 1          # every weight 0: lowest unvisited
    w1 = np.array([5.0, 0.0, 0.0, 1e-3, 0.0, 0.0], np.float32)
    for step in range(1, 200):                         # the only positive weight wins
        assert orc.race(w1, vis, 4, step, 2, 0) == 3
    assert orc.race(np.ones(4, np.float32), np.array([1, 1, 0, 1], np.uint8), 3, 1, 0, 0) == 2
    inst = I.uniform_instance(23, 1000, seed=3)
    h = orc.heta(inst.dist, 2.0)
    ch = orc.choice(np.where(np.eye(23) > 0, 0, 0.3).astype(np.float32), h, 1.0)
    tours, lens = orc.construct(ch, inst.dist, 11, seed=2, iteration=1, rule=3)
    for k in range(11):
        t = tours[k]
        assert sorted(t[:-1].tolist()) == list(range(23)) and t[-1] == t[0]
        assert lens[k] == int(inst.dist[t[:-1], t[1:]].astype(np.int64).sum())
    t0, _ = orc.construct(ch, inst.dist, 11, seed=2, iteration=1, rule=0)
    assert np.array_equal(t0[:, 0], tours[:, 0])


@pytest.mark.parametrize("n,seed", [(8, 1), (9, 2)])
def test_race_ant_system_reaches_brute_force_optimum(orc, n, seed):
    inst = I.uniform_instance(n, 1000, seed=seed)
    opt, _ = orc.brute_force(inst.dist)
    assert orc.run(inst.dist, n, 40, seed, rule=3)["best_len"] == opt


# --------------------------------------------------------------------------
# Nearest-neighbour lists (reading R9; Table 2 versions 4-6 use nn = 30)
# --------------------------------------------------------------------------

def test_nn_lists_on_a_line(orc):
    # cities at x = 0..n-1 in order: list(k) = k-1, k+1, k-2, k+2, ... (the
    # lower index first on equal distance), truncated at the ends
    n, nn = 12, 5
    coords = np.stack([np.arange(n), np.zeros(n)], 1)
    lists = orc.nn_lists(I.distance_matrix(coords), nn)
    for k in range(n):
        expect = []
        for step in range(1, n):
            for j in (k - step, k + step):
                if 0 <= j < n:
                    expect.append(j)
        assert lists[k].tolist() == expect[:nn]


def test_nn_lists_properties(orc):
    inst = I.uniform_instance(60, 100, seed=9)  # small grid: many equal distances
    lists = orc.nn_lists(inst.dist, 20)
    for i in range(60):
        row = lists[i]
        assert i not in row and len(set(row.tolist())) == 20
        dd = inst.dist[i, row]
        assert np.all(np.diff(dd) >= 0)
        # every city outside the list is at least as far as the last entry,
        # and on equal distance has a larger index
        outside = [j for j in range(60) if j != i and j not in row]
        last = (dd[-1], row[-1])
        assert all((inst.dist[i, j], j) > tuple(last) for j in outside)


def test_nn_select_rules(orc):
    from scipy.stats import chisquare
    n = 7
    w = np.array([0.0, 1.0, 4.0, 2.0, 8.0, 0.5, 3.0], np.float32)
    lst = np.array([2, 5, 3], np.int32)
    vis = np.zeros(n, np.uint8)
    vis[0] = 1
    # Eq. 1 restricted to the list: probabilities 4 : 0.5 : 2
    counts = np.zeros(n, np.int64)
    for i in range(30_000):
        x = orc.philox4x32_10([1, i, 0, 0], [3, 0])
        counts[orc.nn_select(lst, w, vis, (int(x[1]) << 32) | int(x[0]))] += 1
    assert counts[[0, 1, 4, 6]].sum() == 0
    p = np.array([4.0, 0.5, 2.0]) / 6.5
    assert chisquare(counts[[2, 5, 3]], p * counts.sum()).pvalue > 0.01
    # all list entries visited: the heaviest unvisited city (4), ties low
    vis2 = vis.copy()
    vis2[[2, 5, 3]] = 1
    assert orc.nn_select(lst, w, vis2, 123) == 4
    w2 = w.copy()
    w2[4] = 3.0
    assert orc.nn_select(lst, w2, vis2, 123) == 4  # 3.0 at 4 and 6: the lower index


def test_nn_construction_tours_and_nn1_walk(orc):
    inst = I.uniform_instance(40, 1000, seed=12)
    h = orc.heta(inst.dist, 2.0)
    ch = orc.choice(np.where(np.eye(40) > 0, 0, 0.1).astype(np.float32), h, 1.0)
    tours, lens = orc.construct_nn(ch, inst.dist, 9, seed=3, iteration=0, nn=8)
    for k in range(9):
        t = tours[k]
        assert sorted(t[:-1].tolist()) == list(range(40)) and t[-1] == t[0]
        assert lens[k] == int(inst.dist[t[:-1], t[1:]].astype(np.int64).sum())
    # nn = 1: the walk goes to the nearest city while it is unvisited and
    # otherwise to the heaviest unvisited one; replay that rule by hand
    lists = orc.nn_lists(inst.dist, 1)
    t1, _ = orc.construct_nn(ch, inst.dist, 4, seed=3, iteration=0, nn=1)
    for k in range(4):
        seen = {int(t1[k, 0])}
        for s in range(1, 40):
            cur = int(t1[k, s - 1])
            nxt = int(lists[cur, 0])
            if nxt in seen:
                cand = [j for j in range(40) if j not in seen]
                nxt = max(cand, key=lambda j: (ch[cur, j], -j))
            assert int(t1[k, s]) == nxt
            seen.add(nxt)


# --------------------------------------------------------------------------
# MAX-MIN Ant System (reading R13: Stutzle and Hoos 2000)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,rho,p,c", [(48, 0.02, 0.05, 33523), (1002, 0.2, 0.05, 259045),
                                       (100, 0.5, 0.005, 21282)])
def test_mmas_limits_properties(orc, n, rho, p, c):
    lo, hi = orc.mmas_limits(n, rho, p, c)
    # tau_max is the limit of repeated deposits of 1/C on one tour under
    # evaporation: x <- (1 - rho) x + 1/C, iterated to its fixed point
    x = 0.0
    for _ in range(20000):
        x = (1.0 - rho) * x + 1.0 / c
    assert abs(hi - x) <= 2.0 ** -23 * x
    # tau_min makes the probability of choosing the tau_max edge at each of
    # n steps among n/2 candidates (the others at tau_min) multiply to p_best
    pdec = hi / (hi + (n / 2.0 - 1.0) * lo)
    assert abs(pdec ** n / p - 1.0) < 1e-5
    assert 0.0 < lo < hi


def test_mmas_limits_collapse_for_tiny_instances(orc):
    # n = 3, p = 0.05: the formula gives tau_min > tau_max; tau_min = tau_max
    lo, hi = orc.mmas_limits(3, 0.1, 0.05, 60)
    assert lo == hi == np.float32(1.0 / (0.1 * 60))
    lo, hi = orc.mmas_limits(12, 0.1, 0.05, 60)
    assert lo < hi


def test_mmas_update_closed_form(orc):
    # Uniform trails c = 0.25 off the diagonal, rho = 1/2, one tour of
    # length 8 deposits 1/8 = 0.125 on its edges (both directions):
    #   unclamped: on-tour 0.125 + 0.125 = 0.25, off-tour 0.125;
    #   [0.15, 0.3]: off-tour raised to 0.15, on-tour 0.25 (a clamp before
    #   the deposit would give 0.275);
    #   [0.15, 0.2]: on-tour lowered to 0.2.
    n = 6
    tour = np.array([0, 3, 1, 5, 2, 4, 0], np.int32)
    on = np.zeros((n, n), bool)
    for a, b in zip(tour[:-1], tour[1:]):
        on[a, b] = on[b, a] = True
    tau = np.full((n, n), 0.25, np.float32)
    np.fill_diagonal(tau, 0)
    off = ~on & ~np.eye(n, dtype=bool)
    for lo, hi, v_on, v_off in [(0.01, 1.0, 0.25, 0.125), (0.15, 0.3, 0.25, 0.15),
                                (0.15, 0.2, 0.2, 0.15)]:
        out = orc.update_mmas(tau, tour, 8, 0.5, lo, hi)
        assert np.all(out[on] == np.float32(v_on)) and np.all(out[off] == np.float32(v_off))
        assert np.all(np.diag(out) == 0)
    # rho = 0.25 keeps 3/4 (catches rho vs 1 - rho): off-tour 0.1875
    out = orc.update_mmas(tau, tour, 8, 0.25, 0.01, 1.0)
    assert np.all(out[off] == np.float32(0.1875)) and np.all(out[on] == np.float32(0.3125))


@pytest.mark.parametrize("best_so_far", [False, True])
def test_mmas_run_bounds_and_depositing_tour(orc, best_so_far):
    n, m, its = 40, 40, 60
    inst = I.uniform_instance(n, 1000, seed=21)
    kw = dict(rho=0.3, p_best=0.05, best_so_far=best_so_far)
    prev = orc.run_mmas(inst.dist, m, its - 1, 5, **kw)
    last = orc.run_mmas(inst.dist, m, its, 5, **kw)
    tau, lo, hi = last["tau32"], last["tau_min"], last["tau_max"]
    offd = ~np.eye(n, dtype=bool)
    assert np.all(tau[offd] >= lo) and np.all(tau[offd] <= hi) and np.all(np.diag(tau) == 0)
    assert np.array_equal(tau, tau.T) and lo > 2.0 ** -126
    assert (lo, hi) == orc.mmas_limits(n, 0.3, 0.05, last["best_len"])
    # cells that changed other than by evaporation and the clamp lie on the
    # depositing tour: the last iteration's best ant, or the best-so-far tour
    evap = np.clip((np.float32(0.7) * prev["tau32"]).astype(np.float32), lo, hi)
    changed = (tau != evap) & offd
    if best_so_far:
        dep = last["best_tour"]
    else:
        dep = last["tours"][int(np.argmin(last["lens"]))]
    on = np.zeros((n, n), bool)
    for a, b in zip(dep[:-1], dep[1:]):
        on[a, b] = on[b, a] = True
    assert changed.any() and not (changed & ~on).any()
    # float state tracks the fp64 recurrence
    r64 = last["tau64"]
    assert np.all(np.abs(tau - r64) <= 1e-5 * np.abs(r64))


@pytest.mark.parametrize("n,seed", [(8, 1), (9, 2), (10, 3)])
def test_mmas_reaches_brute_force_optimum(orc, n, seed):
    inst = I.uniform_instance(n, 1000, seed=seed)
    opt, _ = orc.brute_force(inst.dist)
    r = orc.run_mmas(inst.dist, n, 60, seed, rho=0.1)
    assert r["best_len"] == opt


# --------------------------------------------------------------------------
# Ant Colony System (reading R14: Dorigo and Gambardella 1997)
# --------------------------------------------------------------------------

def _greedy_tour(dist, start):
    n = dist.shape[0]
    tour, seen = [start], {start}
    while len(tour) < n:
        row = [(dist[tour[-1], j], j) for j in range(n) if j not in seen]
        j = min(row)[1]
        tour.append(j)
        seen.add(j)
    return tour + [start]


def test_acs_exploitation_only_is_the_greedy_tour(orc):
    # q0 = 1: every step takes the largest tau * eta^2.  The trails start
    # uniform and the local update moves them by at most an ulp, so on an
    # instance with no equal distances in any row each ant walks the
    # nearest-neighbour tour from its start.
    inst = I.uniform_instance(25, 100000, seed=8)
    d = inst.dist
    for i in range(25):
        row = np.delete(d[i], i)
        assert len(np.unique(row)) == 24
    r = orc.run_acs(d, 6, 1, 3, q0=1.0, xi=0.1)
    for k in range(6):
        assert r["tours"][k].tolist() == _greedy_tour(d, int(r["tours"][k, 0]))


def test_acs_without_exploitation_or_local_update_is_eq1(orc):
    # q0 = 0 and xi = 0: the local update is the identity and every step
    # samples Eq. 1, so the first iteration equals the Ant System's
    # construction on choice_info = tau0 * eta^2.
    inst = I.uniform_instance(40, 1000, seed=4)
    n, m = 40, 12
    r = orc.run_acs(inst.dist, m, 1, 7, q0=0.0, xi=0.0)
    tau0 = np.float32(1.0 / (n * orc.nn_tour_length(inst.dist)))
    tau = np.where(np.eye(n) > 0, 0, tau0).astype(np.float32)
    ch = orc.choice(tau, orc.heta(inst.dist, 2.0), 1.0)
    tours, lens = orc.construct(ch, inst.dist, m, seed=7, iteration=0)
    assert np.array_equal(r["tours"], tours) and np.array_equal(r["lens"], lens)


def test_acs_local_update_closed_form_and_counts(orc):
    # One application with xi = 1/2, tau0 = 1 on tau = 4: 2 + 1/2 = 2.5; a
    # second: 1.25 + 0.5 = 1.75 (all exact in float).
    assert orc.acs_local(4.0, 0.5, 1.0) == 2.5
    assert orc.acs_local(2.5, 0.5, 1.0) == 1.75
    # Over a greedy iteration (q0 = 1) an edge crossed c times (by any ants,
    # at any steps) carries f^c(tau0); the best-so-far tour's edges then get
    # the global update (1 - rho) tau + rho / C_bs.
    inst = I.uniform_instance(7, 100000, seed=3)
    n, m, xi, rho = 7, 20, 0.25, 0.1
    r = orc.run_acs(inst.dist, m, 1, 11, q0=1.0, xi=xi, rho=rho)
    tau0 = np.float32(1.0 / (n * orc.nn_tour_length(inst.dist)))
    count = np.zeros((n, n), int)
    for t in r["tours"]:
        for a, b in zip(t[:-1], t[1:]):
            count[a, b] += 1
            count[b, a] += 1
    expect = np.where(np.eye(n) > 0, 0, tau0).astype(np.float32)
    for a in range(n):
        for b in range(n):
            for _ in range(count[a, b]):
                expect[a, b] = orc.acs_local(expect[a, b], xi, tau0)
    on = np.zeros((n, n), bool)
    bt = r["best_tour"]
    for a, b in zip(bt[:-1], bt[1:]):
        on[a, b] = on[b, a] = True
    assert np.array_equal(r["tau32"][~on], expect[~on])
    dep = np.float32(np.float32(rho) * np.float32(1.0 / r["best_len"]))
    glob = (np.float32(1 - np.float32(rho)) * expect + dep).astype(np.float32)
    assert np.array_equal(r["tau32"][on], glob[on])
    assert r["best_len"] == min(r["lens"])


def test_acs_exploitation_frequency(orc):
    # Weights 5, 1, 1, 1: exploitation always takes city 0, the roulette with
    # probability 5/8, so P(0) = q0 + (1 - q0) 5/8.
    from scipy.stats import binomtest
    w = np.array([5.0, 1.0, 1.0, 1.0], np.float32)
    vis = np.zeros(4, np.uint8)
    for q0 in (0.3, 0.8):
        hits, trials = 0, 20000
        for i in range(trials):
            x = orc.philox4x32_10([i, 1, 2, 0], [99, 0])
            r = (int(x[1]) << 32) | int(x[0])
            hits += orc.acs_select(w, vis, r, int(x[2]), q0) == 0
        assert binomtest(hits, trials, q0 + (1 - q0) * 5 / 8).pvalue > 0.01
    # ties in exploitation go to the lower index; visited cities never win
    w2 = np.array([9.0, 2.0, 7.0, 7.0], np.float32)
    assert orc.acs_select(w2, np.array([1, 0, 0, 0], np.uint8), 0, 0, 1.0) == 2
    assert orc.acs_threshold(0.0) == 0 and orc.acs_threshold(1.0) == 2 ** 32
    assert orc.acs_threshold(0.5) == 2 ** 31


@pytest.mark.parametrize("n,seed", [(8, 1), (9, 2), (10, 3)])
def test_acs_reaches_brute_force_optimum(orc, n, seed):
    inst = I.uniform_instance(n, 1000, seed=seed)
    opt, _ = orc.brute_force(inst.dist)
    r = orc.run_acs(inst.dist, 10, 60, seed)
    assert r["best_len"] == opt


# --------------------------------------------------------------------------
# The Ant Colony System with nearest-neighbour lists (reading R16)
# --------------------------------------------------------------------------

def test_acs_list_step_rules(orc):
    # the heaviest city (7) is outside the list [2, 5, 3]: exploitation takes
    # the heaviest unvisited entry (5, not 7); with 5 visited, the earlier of
    # two equal entries (2 before 3); with every entry visited, the dense
    # argmax (7); exploration samples only list entries, by q_j / Q in list
    # order
    w = np.array([0, 1, 4, 4, 0, 6, 0, 9], np.float32)
    vis = np.zeros(8, np.uint8)
    lst = np.array([2, 5, 3], np.int32)
    assert orc.acs_select_nn(w, vis, lst, 0, 0, 1.0) == 5
    assert orc.acs_select_nn(w, np.array([0, 0, 0, 0, 0, 1, 0, 0], np.uint8), lst, 0, 0, 1.0) == 2
    all_vis = np.array([0, 0, 1, 1, 0, 1, 0, 0], np.uint8)
    assert orc.acs_select_nn(w, all_vis, lst, 0, 0, 1.0) == 7
    assert orc.acs_select_nn(w, all_vis, lst, 0, 0, 0.0) == 7
    # exploring: T at the very start picks the first list entry (2), the top
    # of the range the last (3); never a city outside the list
    assert orc.acs_select_nn(w, vis, lst, 0, 0xffffffff, 0.9) == 2
    assert orc.acs_select_nn(w, vis, lst, 2**64 - 1, 0xffffffff, 0.9) == 3
    rng = np.random.default_rng(1)
    picks = [orc.acs_select_nn(w, vis, lst, int(rng.integers(0, 2**63)) * 2, 0xffffffff, 0.9)
             for _ in range(2000)]
    assert set(picks) == {2, 5, 3}


def test_acs_lists_pure_exploitation_is_the_dense_greedy_walk(orc):
    # q0 = 1, xi = 0: tau stays uniform during the first iteration, so the
    # largest choice_info among unvisited list entries is the nearest
    # unvisited city whenever one of them is unvisited (the list is sorted by
    # distance, ties to the lower index like the dense argmax), and the
    # fallback is the dense argmax itself: the tours equal the dense ones.
    inst = I.uniform_instance(50, 1000, seed=14)
    dense = orc.run_acs(inst.dist, 8, 1, 3, q0=1.0, xi=0.0)
    listed = orc.run_acs(inst.dist, 8, 1, 3, q0=1.0, xi=0.0, nn=6)
    assert np.array_equal(listed["tours"], dense["tours"])


def test_acs_lists_pure_exploration_is_the_list_roulette(orc):
    # q0 = 0, xi = 0: every step is the restricted roulette of R9 on
    # choice_info = tau0 * eta^2, so the first iteration equals the Ant
    # System's list construction on that matrix.
    inst = I.uniform_instance(60, 1000, seed=15)
    n, m, nn = 60, 12, 8
    r = orc.run_acs(inst.dist, m, 1, 7, q0=0.0, xi=0.0, nn=nn)
    tau0 = np.float32(1.0 / (n * orc.nn_tour_length(inst.dist)))
    tau = np.where(np.eye(n) > 0, 0, tau0).astype(np.float32)
    ch = orc.choice(tau, orc.heta(inst.dist, 2.0), 1.0)
    tours, lens = orc.construct_nn(ch, inst.dist, m, seed=7, iteration=0, nn=nn)
    assert np.array_equal(r["tours"], tours) and np.array_equal(r["lens"], lens)
    dense = orc.run_acs(inst.dist, m, 1, 7, q0=0.0, xi=0.0)
    assert not np.array_equal(dense["tours"], r["tours"])  # the lists do restrict


@pytest.mark.parametrize("n,seed", [(8, 1), (9, 2), (10, 3)])
def test_acs_lists_reach_brute_force_optimum(orc, n, seed):
    inst = I.uniform_instance(n, 1000, seed=seed)
    opt, _ = orc.brute_force(inst.dist)
    assert orc.run_acs(inst.dist, 10, 60, seed, nn=5)["best_len"] == opt


def test_threaded_construction_equals_the_plain_loop(orc):
    # Splitting the independent ants of a construction across host threads
    # (the all-core timing mode) changes nothing in a run.
    inst = I.uniform_instance(150, 1000, seed=41)
    try:
        orc.set_threads(1)
        one = orc.run(inst.dist, 150, 3, 5)
        assert orc.set_threads(7) == 7
        many = orc.run(inst.dist, 150, 3, 5)
    finally:
        orc.set_threads(1)
    for k in ("tau32", "tau64", "tours", "lens", "best_tour", "iter_best"):
        assert np.array_equal(one[k], many[k]), k
    assert one["best_len"] == many["best_len"]
    assert orc.hardware_threads() >= 1
