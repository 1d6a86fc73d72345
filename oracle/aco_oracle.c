/*
 * CPU oracle for the Ant System on the symmetric TSP (Cecilia et al.,
 * "Parallelization Strategies for Ant Colony Optimisation on GPUs").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The CUDA
 * path shares no code with it: nothing here is included by, linked into or
 * generated for the kernels, and nothing here reads anything the kernels wrote.
 *
 * It is deliberately plain and slow: loops over cities and ants, in the order
 * the paper states the algorithm (Section II).  Only the independent ants of
 * one construction may be spread over host threads (orc_set_threads; one by
 * default); every other part is single-threaded:
 *
 *   repeat:  choice_info = tau^alpha * eta^beta          (Section III-A, "choice kernel")
 *            every ant builds a tour with Eq. 1          (Section II)
 *            tau <- (1 - rho) tau                        (Eq. 2)
 *            tau <- tau + sum_k dtau^k, dtau^k = 1/C^k   (Eqs. 3-4)
 *
 * Two arithmetic modes:
 *  - "mirror" (FP32 state, the precision the benchmark configurations fix):
 *    tau, eta^beta and choice_info are float, the deposit is summed exactly in
 *    64-bit fixed point and rounded once.  Every value is a fixed function of
 *    the inputs, so this mode is reproducible bit for bit by any correct
 *    implementation that follows the same readings.
 *  - "fp64": the pheromone recurrence of Eqs. 2-4 evaluated in double
 *    precision on the same tours, the reference for the 1e-5 relative
 *    tolerance on tau.
 *
 * Readings of points the paper leaves open (all written out where used):
 *  R1 random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key =
 *     seed, counter = (step, ant, iteration, 0).  Step 0 places the ant:
 *     start = floor(x0 * n / 2^32) ("ants are randomly placed", Section II).
 *     Step s >= 1 draws r = x1 * 2^32 + x0.
 *  R2 Eq. 1 is sampled by an exact integer roulette: with M the largest weight
 *     among unvisited cities and B = 46, each unvisited weight w_j becomes
 *     q_j = floor(w_j * 2^(B-1-ilogb M)) < 2^46; for n <= 4096 = 2^12 cities
 *     Q = sum q_j < 2^58 fits 64 bits.  The target is
 *     T = floor(r * Q / 2^64); the chosen city is the first j (ascending index)
 *     whose inclusive prefix sum of q exceeds T.  P(j) = q_j / Q.  If M = 0
 *     the lowest-index unvisited city is taken.
 *  R3 eta_ij^beta = 1 / d_ij^beta computed in double and rounded to float; for
 *     beta in {1,2,3} d^beta is formed by exact integer-valued products, for
 *     other beta with pow().  The diagonal gets 0.
 *  R4 tau0 = m / C_nn with C_nn the nearest-neighbour tour from city 0 (ties to
 *     the lowest index); tau_ii = 0.
 *  R5 dtau^k = (float)(1 / (double)C^k), added to both (a,b) and (b,a).  In
 *     mirror mode each dtau^k becomes q_k = floor(dtau^k * 2^S) with
 *     S = 62 - ceil(log2 m) - ilogb(max_k dtau^k); the per-cell sum of q_k is
 *     exact, converted to float once (round to nearest) and scaled by 2^-S.
 *     tau' = fl(fl((1-rho) tau) + dep).
 *  R6 choice = tau * eta^beta for alpha = 1, eta^beta for alpha = 0, and
 *     powf(tau, alpha) * eta^beta otherwise.
 *  R7 the best-so-far tour is replaced only by a strictly shorter one; within
 *     an iteration the lowest ant index wins ties.
 *  R8 (optional selection rule) the paper's data-parallel construction
 *     (Section III-A): every unvisited city j draws u_j in (0, 1], its score
 *     is fl(u_j * w_j), and the ant moves to the highest score (ties to the
 *     lower index; if every score is 0, to the lowest unvisited city).  The
 *     paper's "best among the tile winners" is read as the highest score of
 *     the same product, so tiling does not change the choice.  u_j =
 *     (floor(x / 2^8) + 1) * 2^-24 with x word (j mod 4) of Philox counter
 *     (step, ant, iteration, 1 + floor(j / 4)).  This is not Eq. 1: for two
 *     cities with w_1 >= w_2 it picks city 2 with probability w_2 / (2 w_1).
 *  R9 (optional) nearest-neighbour lists (Section II, the construction the
 *     paper's Table 2 versions 4-6 use with nn = 30): list(i) holds the nn
 *     cities j != i with the smallest d_ij, ties to the lower index, in that
 *     order.  An ant at i samples Eq. 1 restricted to the unvisited entries
 *     of list(i) by the integer roulette of R2 in list order; if every entry
 *     is visited it moves to the unvisited city with the largest weight,
 *     ties to the lower index.
 *  R16 (optional) the Ant Colony System of R14 with the nearest-neighbour
 *     lists of R9: at city i, if an entry of list(i) is unvisited, an
 *     exploiting step moves to the unvisited entry of largest choice_info
 *     (ties to the earlier entry) and an exploring step samples Eq. 1 over
 *     the unvisited entries by the integer roulette in list order; if every
 *     entry is visited, either step moves to the unvisited city of largest
 *     choice_info (ties to the lower index).  The weights are the current
 *     choice_info values (after the local updates), read at the list's cities.
 *  R15 (optional selection rule) the exponential race, a per-candidate
 *     random rule that samples Eq. 1: every unvisited city j draws
 *     v_j = floor(x / 2^8) + 1 in [1, 2^24] (x as in R8), E_j = -ln(v_j 2^-24)
 *     is an exponential variate of rate 1, and the ant moves to the smallest
 *     key E_j / w_j (ties to the lower index), which is city j with
 *     probability w_j / sum w (the minimum of independent exponentials of
 *     rates w_j).  Zero weights get the key +inf (so does a key that
 *     overflows); if every key is +inf the lowest unvisited city is taken.  E_j is computed in IEEE
 *     single precision by the range-reduced inverse-hyperbolic-tangent
 *     series of the logarithm: v = 2^e f with f in [1, 2), halved (e + 1)
 *     when f > sqrt 2; s = (f - 1) / (f + 1); ln f = 2 s (1 + z/3 + z^2/5 +
 *     z^3/7 + z^4/9), z = s^2, by Horner from the z^4 term, every operation
 *     rounded on its own (no fused multiply-add); E = (24 - e) ln 2 - ln f;
 *     the key is fl(E / w).  The constants are the floats nearest sqrt 2,
 *     ln 2, 1/3, 1/5, 1/7 and 1/9.
 *
 *  R13 (optional variant) the MAX-MIN Ant System, which the paper cites as an
 *     earlier GPU target (Section II-B) and which stands for the "other ACO
 *     algorithms" of its future work (Section V); the variant is the one of
 *     Stutzle and Hoos, "MAX-MIN Ant System", Future Generation Computer
 *     Systems 16 (2000).  One tour deposits per iteration (the iteration
 *     best, or the best-so-far tour): dtau = (float)(1 / (double)C) on its n
 *     edges, both directions; every tau_ij (i != j) is then clamped into
 *     [tau_min, tau_max].  tau_max = 1 / (rho C_gb), C_gb the best-so-far
 *     length (the limit of repeated deposits on one tour); tau_min =
 *     tau_max * f, f = (1 - p^(1/n)) / ((n/2 - 1) p^(1/n)) with p = p_best,
 *     and tau_min = tau_max where that is larger.  Both limits are computed
 *     in double in this order and rounded to float once; the trails start at
 *     tau_max computed from C_nn.  tau' = clamp(fl(fl((1-rho) tau) + dtau)).
 *
 *  R14 (optional variant) the Ant Colony System, which the paper names as
 *     its next target (Section V); the variant is the one of Dorigo and
 *     Gambardella, IEEE Trans. Evol. Comp. 1(1) (1997).  tau starts at
 *     tau0 = (float)(1 / (n C_nn)).  At step s ant k draws x = Philox (s, k,
 *     iteration, 0): it exploits when x2 < floor(q0 2^32) (compared as
 *     64-bit integers), moving to the unvisited city of largest choice_info
 *     (ties to the lower index), and otherwise samples Eq. 1 by the integer
 *     roulette of R2 with r = x1 2^32 + x0.  The ants move in lockstep: all
 *     ants choose their s-th city from the same state, then every edge
 *     crossed at that step gets the local update tau <- fl(fl((1-xi) tau) +
 *     fl(xi tau0)) in both directions, once per ant that crossed it (the
 *     applications are identical, so their order does not matter), and its
 *     choice_info is recomputed.  The closing edge back to the start is the
 *     n-th such step.  After the tours, only the best-so-far tour's edges get
 *     the global update tau <- fl(fl((1-rho) tau) + fl(rho dtau)), dtau =
 *     (float)(1 / (double)C_bs), both directions; no other cell evaporates.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared -lm.
 * -ffp-contract=off matters: a fused multiply-add would change the rounding of
 * fl(fl(a*b)+c).
 */
#include <pthread.h>
#include <unistd.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, from the published description (Salmon et al., SC'11):     */
/* ten rounds of the 4x32 S-box with multipliers 0xD2511F53 and 0xCD9E8D57,  */
/* key schedule bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85       */
/* between rounds.                                                           */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Philox words for (seed, step, ant, iteration) under reading R1. */
static void draw(uint64_t seed, uint32_t step, uint32_t ant, uint32_t iteration, uint32_t x[4])
{
    uint32_t ctr[4] = {step, ant, iteration, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, x);
}

/* Smallest c with 2^c >= v (v >= 1). */
int orc_ceil_log2(int64_t v)
{
    int c = 0;
    while (((int64_t)1 << c) < v) ++c;
    return c;
}

/* Unbiased binary exponent of a positive finite float (subnormals included). */
static int exponent_of(float x)
{
    int e;
    (void)frexp((double)x, &e); /* x = f * 2^e, f in [0.5, 1) */
    return e - 1;
}

/* ------------------------------------------------------------------------- */
/* Eq. 1 by the integer roulette of reading R2.                               */
/* w: weights of row i (n entries), visited: 1 for cities in the tabu list.  */
/* Returns the chosen city, -1 if every city is visited, -2 if n > 4096.     */
/* ------------------------------------------------------------------------- */
#define ROULETTE_BITS 46
#define ROULETTE_MAX_N 4096

int orc_roulette(int n, const float *w, const uint8_t *visited, uint64_t r)
{
    if (n > ROULETTE_MAX_N) return -2;
    float M = 0.0f;
    int first_unvisited = -1;
    for (int j = 0; j < n; ++j) {
        if (visited[j]) continue;
        if (first_unvisited < 0) first_unvisited = j;
        if (w[j] > M) M = w[j];
    }
    if (first_unvisited < 0) return -1;
    if (M == 0.0f) return first_unvisited;

    int scale = ROULETTE_BITS - 1 - exponent_of(M);
    uint64_t *q = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    uint64_t Q = 0;
    for (int j = 0; j < n; ++j) {
        q[j] = visited[j] ? 0u : (uint64_t)floor(ldexp((double)w[j], scale));
        Q += q[j];
    }
    uint64_t T = (uint64_t)(((unsigned __int128)r * (unsigned __int128)Q) >> 64);
    uint64_t prefix = 0;
    int chosen = -1;
    for (int j = 0; j < n; ++j) {
        prefix += q[j];
        if (prefix > T) { chosen = j; break; }
    }
    free(q);
    return chosen;
}

/* Exposed for tests: the quantised weights q_j and their sum Q of reading R2. */
uint64_t orc_roulette_weights(int n, const float *w, const uint8_t *visited, uint64_t *q)
{
    float M = 0.0f;
    for (int j = 0; j < n; ++j)
        if (!visited[j] && w[j] > M) M = w[j];
    uint64_t Q = 0;
    if (M == 0.0f) {
        for (int j = 0; j < n; ++j) q[j] = 0;
        return 0;
    }
    int scale = ROULETTE_BITS - 1 - exponent_of(M);
    for (int j = 0; j < n; ++j) {
        q[j] = visited[j] ? 0u : (uint64_t)floor(ldexp((double)w[j], scale));
        Q += q[j];
    }
    return Q;
}

/* ------------------------------------------------------------------------- */
/* The paper's data-parallel selection rule (reading R8).                     */
/* ------------------------------------------------------------------------- */
float orc_candidate_uniform(uint64_t seed, uint32_t step, uint32_t ant, uint32_t iteration,
                            int j)
{
    uint32_t ctr[4] = {step, ant, iteration, 1u + (uint32_t)(j / 4)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    return (float)((x[j % 4] >> 8) + 1u) * (1.0f / 16777216.0f);
}

int orc_iroulette(int n, const float *w, const uint8_t *visited, uint64_t seed, uint32_t step,
                  uint32_t ant, uint32_t iteration)
{
    int best = -1, first_unvisited = -1;
    float best_score = 0.0f;
    for (int j = 0; j < n; ++j) {
        if (visited[j]) continue;
        if (first_unvisited < 0) first_unvisited = j;
        float u = orc_candidate_uniform(seed, step, ant, iteration, j);
        float score = u * w[j];
        if (score > best_score) {
            best_score = score;
            best = j;
        }
    }
    return best >= 0 ? best : first_unvisited;
}

/* ------------------------------------------------------------------------- */
/* The exponential race (reading R15).                                        */
/* ------------------------------------------------------------------------- */
/* E = -ln(v 2^-24) for v in [1, 2^24], in single precision (R15). */
float orc_race_exponential(uint32_t v)
{
    int e = 0;
    while (e < 31 && (v >> (e + 1)) != 0u) ++e; /* floor(log2 v) */
    float f = ldexpf((float)v, -e);             /* exact: v < 2^25, f in [1, 2) */
    if (f > 0x1.6a09e6p+0f) {                   /* sqrt 2 */
        f = f * 0.5f;
        e += 1;
    }
    float s = (f - 1.0f) / (f + 1.0f);
    float z = s * s;
    float p = 0x1.c71c72p-4f;                   /* 1/9 */
    p = p * z + 0x1.24924ap-3f;                 /* 1/7 */
    p = p * z + 0x1.99999ap-3f;                 /* 1/5 */
    p = p * z + 0x1.555556p-2f;                 /* 1/3 */
    p = p * z + 1.0f;
    float ln_f = (s + s) * p;
    return (float)(24 - e) * 0x1.62e430p-1f - ln_f; /* ln 2 */
}

void orc_race_exponentials(int count, const uint32_t *v, float *out)
{
    for (int i = 0; i < count; ++i) out[i] = orc_race_exponential(v[i]);
}

int orc_race(int n, const float *w, const uint8_t *visited, uint64_t seed, uint32_t step,
             uint32_t ant, uint32_t iteration)
{
    int best = -1;
    float best_key = 0.0f;
    for (int j = 0; j < n; ++j) {
        if (visited[j]) continue;
        uint32_t ctr[4] = {step, ant, iteration, 1u + (uint32_t)(j / 4)};
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        uint32_t vj = (x[j % 4] >> 8) + 1u;
        float k = w[j] > 0.0f ? orc_race_exponential(vj) / w[j] : INFINITY;
        if (best < 0 || k < best_key) { /* strict: the lower index keeps a tie */
            best = j;
            best_key = k;
        }
    }
    return best;
}

/* ------------------------------------------------------------------------- */
/* Nearest-neighbour lists and the list-restricted step (reading R9).        */
/* ------------------------------------------------------------------------- */
void orc_nn_lists(int n, const int32_t *d, int nn, int32_t *lists)
{
    for (int i = 0; i < n; ++i) {
        /* selection by repeated minimum of (d_ij, j) above the previous pick */
        long long last_d = -1;
        int last_j = -1;
        for (int l = 0; l < nn; ++l) {
            int best = -1;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                long long dj = d[(size_t)i * n + j];
                int after_last = dj > last_d || (dj == last_d && j > last_j);
                if (!after_last) continue;
                if (best < 0 || dj < d[(size_t)i * n + best]) best = j;
            }
            lists[(size_t)i * nn + l] = best;
            last_d = d[(size_t)i * n + best];
            last_j = best;
        }
    }
}

int orc_nn_select(int n, int nn, const int32_t *list, const float *w, const uint8_t *visited,
                  uint64_t r)
{
    float wl[32];
    uint8_t vl[32];
    int any = 0;
    for (int l = 0; l < nn; ++l) {
        wl[l] = w[list[l]];
        vl[l] = visited[list[l]];
        if (!vl[l]) any = 1;
    }
    if (any) return list[orc_roulette(nn, wl, vl, r)];
    int best = -1;
    for (int j = 0; j < n; ++j) {
        if (visited[j]) continue;
        if (best < 0 || w[j] > w[best]) best = j;
    }
    return best;
}

/* ------------------------------------------------------------------------- */
/* Setup: heuristic, nearest-neighbour tour, initial pheromone.              */
/* ------------------------------------------------------------------------- */

/* eta_ij^beta as float (reading R3), n x n row-major. */
void orc_heta(int n, const int32_t *d, double beta, float *heta)
{
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double v;
            if (i == j) {
                v = 0.0;
            } else {
                double dd = (double)d[(size_t)i * n + j];
                if (beta == 0.0) v = 1.0;
                else if (beta == 1.0) v = 1.0 / dd;
                else if (beta == 2.0) v = 1.0 / (dd * dd);
                else if (beta == 3.0) v = 1.0 / (dd * dd * dd);
                else v = pow(dd, -beta);
            }
            heta[(size_t)i * n + j] = (float)v;
        }
    }
}

/* eta_ij^beta in double, for the fp64 mode. */
static void heta64(int n, const int32_t *d, double beta, double *h)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            h[(size_t)i * n + j] = (i == j) ? 0.0 : pow(1.0 / (double)d[(size_t)i * n + j], beta);
}

/* Length of the nearest-neighbour tour from city 0, ties to the lowest index (R4). */
int64_t orc_nn_tour_length(int n, const int32_t *d)
{
    uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
    int cur = 0;
    seen[0] = 1;
    int64_t len = 0;
    for (int s = 1; s < n; ++s) {
        int best = -1;
        for (int j = 0; j < n; ++j) {
            if (seen[j]) continue;
            if (best < 0 || d[(size_t)cur * n + j] < d[(size_t)cur * n + best]) best = j;
        }
        len += d[(size_t)cur * n + best];
        seen[best] = 1;
        cur = best;
    }
    len += d[(size_t)cur * n + 0];
    free(seen);
    return len;
}

float orc_tau0(int n, int m, const int32_t *d)
{
    return (float)((double)m / (double)orc_nn_tour_length(n, d));
}

/* choice_info = tau^alpha * eta^beta in float (reading R6). */
void orc_choice(int n, const float *tau, const float *heta, float alpha, float *choice)
{
    for (size_t e = 0; e < (size_t)n * n; ++e) {
        float t;
        if (alpha == 1.0f) t = tau[e];
        else if (alpha == 0.0f) t = 1.0f;
        else t = powf(tau[e], alpha);
        choice[e] = t * heta[e];
    }
}

/* ------------------------------------------------------------------------- */
/* Tour construction (Section II): one ant.                                  */
/* tour has n+1 entries, tour[n] = tour[0].  Returns C^k.                    */
/* ------------------------------------------------------------------------- */
/* rule 0: Eq. 1 (reading R2); rule 1: the paper's data-parallel rule (R8);
   rule 2: nearest-neighbour lists of length nn (R9); rule 3: the exponential
   race (R15). */
int64_t orc_construct_ant_nn(int n, const float *choice, const int32_t *d, uint64_t seed,
                             uint32_t iteration, uint32_t ant, int rule, int nn,
                             const int32_t *lists, int32_t *tour);

int64_t orc_construct_ant_rule(int n, const float *choice, const int32_t *d, uint64_t seed,
                               uint32_t iteration, uint32_t ant, int rule, int32_t *tour)
{
    return orc_construct_ant_nn(n, choice, d, seed, iteration, ant, rule, 0, NULL, tour);
}

int64_t orc_construct_ant(int n, const float *choice, const int32_t *d, uint64_t seed,
                          uint32_t iteration, uint32_t ant, int32_t *tour)
{
    return orc_construct_ant_rule(n, choice, d, seed, iteration, ant, 0, tour);
}

int64_t orc_construct_ant_nn(int n, const float *choice, const int32_t *d, uint64_t seed,
                             uint32_t iteration, uint32_t ant, int rule, int nn,
                             const int32_t *lists, int32_t *tour)
{
    uint8_t *visited = (uint8_t *)calloc((size_t)n, 1);
    uint32_t x[4];
    draw(seed, 0u, ant, iteration, x);
    int start = (int)(((uint64_t)x[0] * (uint64_t)n) >> 32);
    tour[0] = start;
    visited[start] = 1;
    int cur = start;
    for (int s = 1; s < n; ++s) {
        int next;
        if (rule == 2) {
            draw(seed, (uint32_t)s, ant, iteration, x);
            uint64_t r = ((uint64_t)x[1] << 32) | (uint64_t)x[0];
            next = orc_nn_select(n, nn, lists + (size_t)cur * nn, choice + (size_t)cur * n,
                                 visited, r);
        } else if (rule == 1) {
            next = orc_iroulette(n, choice + (size_t)cur * n, visited, seed, (uint32_t)s, ant,
                                 iteration);
        } else if (rule == 3) {
            next = orc_race(n, choice + (size_t)cur * n, visited, seed, (uint32_t)s, ant,
                            iteration);
        } else {
            draw(seed, (uint32_t)s, ant, iteration, x);
            uint64_t r = ((uint64_t)x[1] << 32) | (uint64_t)x[0];
            next = orc_roulette(n, choice + (size_t)cur * n, visited, r);
        }
        tour[s] = next;
        visited[next] = 1;
        cur = next;
    }
    tour[n] = start;
    free(visited);
    int64_t len = 0;
    for (int s = 0; s < n; ++s) len += d[(size_t)tour[s] * n + tour[s + 1]];
    return len;
}

/* Ants are independent within an iteration (Section II: each builds its tour
   from the same choice_info), so the construction may be split across host
   threads, ant k always computed by the same code and with the same counters:
   the result does not depend on the thread count.  One thread by default. */
static int g_threads = 1;

int orc_set_threads(int threads)
{
    if (threads < 1) threads = 1;
    if (threads > 512) threads = 512;
    g_threads = threads;
    return g_threads;
}

int orc_get_threads(void) { return g_threads; }

int orc_hardware_threads(void)
{
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c < 1 ? 1 : (int)c;
}

struct construct_job {
    int n, rule, nn, k0, k1;
    const float *choice;
    const int32_t *d, *lists;
    uint64_t seed;
    uint32_t iteration;
    int32_t *tours;
    int64_t *lens;
};

static void *construct_worker(void *arg)
{
    struct construct_job *j = (struct construct_job *)arg;
    for (int k = j->k0; k < j->k1; ++k)
        j->lens[k] = orc_construct_ant_nn(j->n, j->choice, j->d, j->seed, j->iteration,
                                          (uint32_t)k, j->rule, j->nn, j->lists,
                                          j->tours + (size_t)k * (j->n + 1));
    return NULL;
}

void orc_construct_nn(int n, int m, const float *choice, const int32_t *d, uint64_t seed,
                      uint32_t iteration, int rule, int nn, const int32_t *lists,
                      int32_t *tours, int64_t *lens)
{
    int t = g_threads < m ? g_threads : m;
    struct construct_job jobs[512];
    pthread_t th[512];
    for (int i = 0; i < t; ++i) {
        jobs[i] = (struct construct_job){n, rule, nn, (int)((int64_t)m * i / t),
                                         (int)((int64_t)m * (i + 1) / t), choice, d, lists,
                                         seed, iteration, tours, lens};
    }
    if (t <= 1) {
        if (m > 0) construct_worker(&jobs[0]);
        return;
    }
    int started = 0;
    for (int i = 1; i < t; ++i) {
        if (pthread_create(&th[i], NULL, construct_worker, &jobs[i]) != 0) break;
        started = i;
    }
    construct_worker(&jobs[0]);
    for (int i = started + 1; i < t; ++i) construct_worker(&jobs[i]);  /* threads not started */
    for (int i = 1; i <= started; ++i) pthread_join(th[i], NULL);
}

void orc_construct_rule(int n, int m, const float *choice, const int32_t *d, uint64_t seed,
                        uint32_t iteration, int rule, int32_t *tours, int64_t *lens)
{
    orc_construct_nn(n, m, choice, d, seed, iteration, rule, 0, NULL, tours, lens);
}

void orc_construct(int n, int m, const float *choice, const int32_t *d, uint64_t seed,
                   uint32_t iteration, int32_t *tours, int64_t *lens)
{
    orc_construct_rule(n, m, choice, d, seed, iteration, 0, tours, lens);
}

/* ------------------------------------------------------------------------- */
/* Pheromone update, Eqs. 2-4.                                               */
/* ------------------------------------------------------------------------- */

/* Deposit scale S of reading R5 for this iteration's tour lengths. */
int orc_deposit_scale(int m, const int64_t *lens)
{
    int64_t cmin = lens[0];
    for (int k = 1; k < m; ++k)
        if (lens[k] < cmin) cmin = lens[k];
    float dmax = (float)(1.0 / (double)cmin);
    return 62 - orc_ceil_log2(m) - exponent_of(dmax);
}

/* Mirror mode: tau (float, n x n) updated in place. */
void orc_update_mirror(int n, int m, const int32_t *tours, const int64_t *lens, float rho,
                       float *tau)
{
    int S = orc_deposit_scale(m, lens);
    uint64_t *acc = (uint64_t *)calloc((size_t)n * n, sizeof(uint64_t));
    for (int k = 0; k < m; ++k) {
        float dk = (float)(1.0 / (double)lens[k]);
        uint64_t qk = (uint64_t)floor(ldexp((double)dk, S));
        const int32_t *t = tours + (size_t)k * (n + 1);
        for (int s = 0; s < n; ++s) {
            int a = t[s], b = t[s + 1];
            acc[(size_t)a * n + b] += qk;
            acc[(size_t)b * n + a] += qk;
        }
    }
    float keep = 1.0f - rho;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            size_t e = (size_t)i * n + j;
            float evaporated = keep * tau[e];                  /* Eq. 2 */
            float dep = ldexpf((float)acc[e], -S);             /* Eqs. 3-4 */
            tau[e] = evaporated + dep;
        }
    }
    free(acc);
}

/* fp64 mode: tau (double) updated in place by Eqs. 2-4 with dtau^k = 1/C^k. */
void orc_update_fp64(int n, int m, const int32_t *tours, const int64_t *lens, double rho,
                     double *tau)
{
    for (size_t e = 0; e < (size_t)n * n; ++e) tau[e] *= (1.0 - rho);
    for (int k = 0; k < m; ++k) {
        double dk = 1.0 / (double)lens[k];
        const int32_t *t = tours + (size_t)k * (n + 1);
        for (int s = 0; s < n; ++s) {
            int a = t[s], b = t[s + 1];
            tau[(size_t)a * n + b] += dk;
            tau[(size_t)b * n + a] += dk;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Whole Ant System run (mirror mode), with the fp64 pheromone carried along  */
/* on the same tours.  Outputs (any may be NULL):                            */
/*   best_tour[n+1], best_len, tau32[n*n], tau64[n*n], last_tours[m*(n+1)],  */
/*   last_lens[m], iter_best[iterations] (shortest C^k of each iteration).   */
/* first_iteration lets a caller continue a run (the counter of R1).         */
/* ------------------------------------------------------------------------- */
int orc_run_rule(int n, const int32_t *d, float alpha, float beta, float rho, int m,
                 uint64_t seed, int iterations, int rule, int32_t *best_tour, int64_t *best_len,
                 float *tau32_out, double *tau64_out, int32_t *last_tours, int64_t *last_lens,
                 int64_t *iter_best);
int orc_run_nn(int n, const int32_t *d, float alpha, float beta, float rho, int m,
               uint64_t seed, int iterations, int rule, int nn, int32_t *best_tour,
               int64_t *best_len, float *tau32_out, double *tau64_out, int32_t *last_tours,
               int64_t *last_lens, int64_t *iter_best);

int orc_run(int n, const int32_t *d, float alpha, float beta, float rho, int m, uint64_t seed,
            int iterations, int32_t *best_tour, int64_t *best_len, float *tau32_out,
            double *tau64_out, int32_t *last_tours, int64_t *last_lens, int64_t *iter_best)
{
    return orc_run_rule(n, d, alpha, beta, rho, m, seed, iterations, 0, best_tour, best_len,
                        tau32_out, tau64_out, last_tours, last_lens, iter_best);
}

int orc_run_rule(int n, const int32_t *d, float alpha, float beta, float rho, int m,
                 uint64_t seed, int iterations, int rule, int32_t *best_tour, int64_t *best_len,
                 float *tau32_out, double *tau64_out, int32_t *last_tours, int64_t *last_lens,
                 int64_t *iter_best)
{
    return orc_run_nn(n, d, alpha, beta, rho, m, seed, iterations, rule, 0, best_tour, best_len,
                      tau32_out, tau64_out, last_tours, last_lens, iter_best);
}

int orc_run_nn(int n, const int32_t *d, float alpha, float beta, float rho, int m,
               uint64_t seed, int iterations, int rule, int nn, int32_t *best_tour,
               int64_t *best_len, float *tau32_out, double *tau64_out, int32_t *last_tours,
               int64_t *last_lens, int64_t *iter_best)
{
    int32_t *lists = NULL;
    if (rule == 2) {
        if (nn < 1 || nn > 32 || nn > n - 1) return -1;
        lists = (int32_t *)malloc((size_t)n * nn * sizeof(int32_t));
        if (!lists) return -2;
        orc_nn_lists(n, d, nn, lists);
    }
    size_t cells = (size_t)n * n;
    float *heta = (float *)malloc(cells * sizeof(float));
    double *h64 = (double *)malloc(cells * sizeof(double));
    float *tau = (float *)malloc(cells * sizeof(float));
    double *tau64 = (double *)malloc(cells * sizeof(double));
    float *choice = (float *)malloc(cells * sizeof(float));
    int32_t *tours = (int32_t *)malloc((size_t)m * (n + 1) * sizeof(int32_t));
    int64_t *lens = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    if (!heta || !h64 || !tau || !tau64 || !choice || !tours || !lens) return -2;

    orc_heta(n, d, (double)beta, heta);
    heta64(n, d, (double)beta, h64);
    int64_t cnn = orc_nn_tour_length(n, d);
    float tau0 = (float)((double)m / (double)cnn);
    double tau0_64 = (double)m / (double)cnn;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            tau[(size_t)i * n + j] = (i == j) ? 0.0f : tau0;
            tau64[(size_t)i * n + j] = (i == j) ? 0.0 : tau0_64;
        }

    int64_t best = INT64_MAX;
    for (int it = 0; it < iterations; ++it) {
        orc_choice(n, tau, heta, alpha, choice);
        orc_construct_nn(n, m, choice, d, seed, (uint32_t)it, rule, nn, lists, tours, lens);
        int kbest = 0;
        for (int k = 1; k < m; ++k)
            if (lens[k] < lens[kbest]) kbest = k;
        if (iter_best) iter_best[it] = lens[kbest];
        if (lens[kbest] < best) {
            best = lens[kbest];
            if (best_tour) memcpy(best_tour, tours + (size_t)kbest * (n + 1), (size_t)(n + 1) * sizeof(int32_t));
        }
        orc_update_mirror(n, m, tours, lens, rho, tau);
        orc_update_fp64(n, m, tours, lens, (double)rho, tau64);
    }
    if (best_len) *best_len = best;
    if (tau32_out) memcpy(tau32_out, tau, cells * sizeof(float));
    if (tau64_out) memcpy(tau64_out, tau64, cells * sizeof(double));
    if (last_tours) memcpy(last_tours, tours, (size_t)m * (n + 1) * sizeof(int32_t));
    if (last_lens) memcpy(last_lens, lens, (size_t)m * sizeof(int64_t));
    (void)h64;
    free(heta); free(h64); free(tau); free(tau64); free(choice); free(tours); free(lens);
    free(lists);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* MAX-MIN Ant System (reading R13).                                          */
/* ------------------------------------------------------------------------- */

/* Trail limits for best-so-far length c_gb, in double, each rounded once.  */
void orc_mmas_limits(int n, float rho, double p_best, int64_t c_gb, float *tau_min,
                     float *tau_max)
{
    double tmax = 1.0 / ((double)rho * (double)c_gb);
    double root = pow(p_best, 1.0 / (double)n);
    double f = (1.0 - root) / (((double)n / 2.0 - 1.0) * root);
    double tmin = tmax * f;
    if (tmin > tmax) tmin = tmax;
    *tau_max = (float)tmax;
    *tau_min = (float)tmin;
}

static void mmas_limits64(int n, double rho, double p_best, int64_t c_gb, double *tau_min,
                          double *tau_max)
{
    double tmax = 1.0 / (rho * (double)c_gb);
    double root = pow(p_best, 1.0 / (double)n);
    double tmin = tmax * ((1.0 - root) / (((double)n / 2.0 - 1.0) * root));
    *tau_max = tmax;
    *tau_min = tmin > tmax ? tmax : tmin;
}

/* One MMAS update in float: evaporation of every cell, dtau on the n edges
 * of dep_tour (n+1 entries, length dep_len) in both directions, then the
 * clamp of every off-diagonal cell.  In a closed tour of n >= 3 cities every
 * edge occurs once, so every cell receives at most one dtau. */
void orc_update_mmas(int n, const int32_t *dep_tour, int64_t dep_len, float rho, float tau_min,
                     float tau_max, float *tau)
{
    float keep = 1.0f - rho;
    float dtau = (float)(1.0 / (double)dep_len);
    for (size_t c = 0; c < (size_t)n * n; ++c) tau[c] = keep * tau[c];
    for (int s = 0; s < n; ++s) {
        int a = dep_tour[s], b = dep_tour[s + 1];
        tau[(size_t)a * n + b] = tau[(size_t)a * n + b] + dtau;
        tau[(size_t)b * n + a] = tau[(size_t)b * n + a] + dtau;
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            if (i == j) continue;
            float *t = &tau[(size_t)i * n + j];
            if (*t < tau_min) *t = tau_min;
            if (*t > tau_max) *t = tau_max;
        }
}

static void update_mmas64(int n, const int32_t *dep_tour, int64_t dep_len, double rho,
                          double tau_min, double tau_max, double *tau)
{
    for (size_t c = 0; c < (size_t)n * n; ++c) tau[c] = (1.0 - rho) * tau[c];
    for (int s = 0; s < n; ++s) {
        int a = dep_tour[s], b = dep_tour[s + 1];
        tau[(size_t)a * n + b] += 1.0 / (double)dep_len;
        tau[(size_t)b * n + a] += 1.0 / (double)dep_len;
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            if (i == j) continue;
            double *t = &tau[(size_t)i * n + j];
            if (*t < tau_min) *t = tau_min;
            if (*t > tau_max) *t = tau_max;
        }
}

/* A whole MMAS run (construction as in orc_run_nn: rule 0/1/2, nn).  Extra
 * output limits[2] = (tau_min, tau_max) after the last iteration. */
int orc_run_mmas(int n, const int32_t *d, float alpha, float beta, float rho, int m,
                 uint64_t seed, int iterations, int rule, int nn, double p_best, int best_so_far,
                 int32_t *best_tour, int64_t *best_len, float *tau32_out, double *tau64_out,
                 int32_t *last_tours, int64_t *last_lens, int64_t *iter_best, float *limits)
{
    if (n < 3) return -1;
    int32_t *lists = NULL;
    if (rule == 2) {
        if (nn < 1 || nn > 32 || nn > n - 1) return -1;
        lists = (int32_t *)malloc((size_t)n * nn * sizeof(int32_t));
        if (!lists) return -2;
        orc_nn_lists(n, d, nn, lists);
    }
    size_t cells = (size_t)n * n;
    float *heta = (float *)malloc(cells * sizeof(float));
    float *tau = (float *)malloc(cells * sizeof(float));
    double *tau64 = (double *)malloc(cells * sizeof(double));
    float *choice = (float *)malloc(cells * sizeof(float));
    int32_t *tours = (int32_t *)malloc((size_t)m * (n + 1) * sizeof(int32_t));
    int64_t *lens = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    int32_t *gb = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    if (!heta || !tau || !tau64 || !choice || !tours || !lens || !gb) return -2;

    orc_heta(n, d, (double)beta, heta);
    int64_t cnn = orc_nn_tour_length(n, d);
    float tmin, tmax;
    double tmin64, tmax64;
    orc_mmas_limits(n, rho, p_best, cnn, &tmin, &tmax);
    mmas_limits64(n, (double)rho, p_best, cnn, &tmin64, &tmax64);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            tau[(size_t)i * n + j] = (i == j) ? 0.0f : tmax;
            tau64[(size_t)i * n + j] = (i == j) ? 0.0 : tmax64;
        }

    int64_t best = INT64_MAX;
    for (int it = 0; it < iterations; ++it) {
        orc_choice(n, tau, heta, alpha, choice);
        orc_construct_nn(n, m, choice, d, seed, (uint32_t)it, rule, nn, lists, tours, lens);
        int kbest = 0;
        for (int k = 1; k < m; ++k)
            if (lens[k] < lens[kbest]) kbest = k;
        if (iter_best) iter_best[it] = lens[kbest];
        if (lens[kbest] < best) {
            best = lens[kbest];
            memcpy(gb, tours + (size_t)kbest * (n + 1), (size_t)(n + 1) * sizeof(int32_t));
        }
        orc_mmas_limits(n, rho, p_best, best, &tmin, &tmax);
        mmas_limits64(n, (double)rho, p_best, best, &tmin64, &tmax64);
        const int32_t *dep = best_so_far ? gb : tours + (size_t)kbest * (n + 1);
        int64_t dep_len = best_so_far ? best : lens[kbest];
        orc_update_mmas(n, dep, dep_len, rho, tmin, tmax, tau);
        update_mmas64(n, dep, dep_len, (double)rho, tmin64, tmax64, tau64);
    }
    if (best_len) *best_len = best;
    if (best_tour && iterations > 0) memcpy(best_tour, gb, (size_t)(n + 1) * sizeof(int32_t));
    if (tau32_out) memcpy(tau32_out, tau, cells * sizeof(float));
    if (tau64_out) memcpy(tau64_out, tau64, cells * sizeof(double));
    if (last_tours) memcpy(last_tours, tours, (size_t)m * (n + 1) * sizeof(int32_t));
    if (last_lens) memcpy(last_lens, lens, (size_t)m * sizeof(int64_t));
    if (limits) {
        limits[0] = tmin;
        limits[1] = tmax;
    }
    free(heta); free(tau); free(tau64); free(choice); free(tours); free(lens); free(gb);
    free(lists);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Ant Colony System (reading R14).                                           */
/* ------------------------------------------------------------------------- */

/* floor(q0 * 2^32): a step exploits when its Philox word x2 is below it. */
uint64_t orc_acs_threshold(double q0)
{
    if (!(q0 > 0.0)) return 0;
    if (q0 >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)floor(q0 * 4294967296.0);
}

/* The pseudo-random proportional rule for one step (w: the row of the
 * current city, visited: the tabu list).  Returns -1 if every city is
 * visited. */
int orc_acs_select(int n, const float *w, const uint8_t *visited, uint64_t r, uint32_t x2,
                   uint64_t threshold)
{
    if ((uint64_t)x2 < threshold) {
        int best = -1;
        for (int j = 0; j < n; ++j)
            if (!visited[j] && (best < 0 || w[j] > w[best])) best = j;
        return best;
    }
    return orc_roulette(n, w, visited, r);
}

/* The same with nearest-neighbour lists (reading R16): list holds the nn
 * cities of list(i). */
int orc_acs_select_nn(int n, int nn, const int32_t *list, const float *w, const uint8_t *visited,
                      uint64_t r, uint32_t x2, uint64_t threshold)
{
    int any = 0;
    for (int l = 0; l < nn; ++l)
        if (!visited[list[l]]) any = 1;
    if (!any || (uint64_t)x2 >= threshold) return orc_nn_select(n, nn, list, w, visited, r);
    int best = -1;
    for (int l = 0; l < nn; ++l) {
        int j = list[l];
        if (!visited[j] && (best < 0 || w[j] > w[best])) best = j;
    }
    return best;
}

/* One local update of one cell. */
float orc_acs_local(float tau, float xi, float tau0)
{
    float keep = 1.0f - xi;
    float add = xi * tau0;
    return keep * tau + add;
}

static float choice_cell(float tau, float heta, float alpha)
{
    if (alpha == 1.0f) return tau * heta;
    if (alpha == 0.0f) return heta;
    return powf(tau, alpha) * heta;
}

static void acs_cross(int n, int a, int b, float xi, float tau0, float alpha, const float *heta,
                      float *tau, float *choice)
{
    size_t ab = (size_t)a * n + b, ba = (size_t)b * n + a;
    tau[ab] = orc_acs_local(tau[ab], xi, tau0);
    tau[ba] = orc_acs_local(tau[ba], xi, tau0);
    choice[ab] = choice_cell(tau[ab], heta[ab], alpha);
    choice[ba] = choice_cell(tau[ba], heta[ba], alpha);
}

/* A whole ACS run.  tau_out (n*n) is the final pheromone; the others as in
 * orc_run_nn.  nn > 0: with nearest-neighbour lists of that length (R16). */
int orc_run_acs_nn(int n, const int32_t *d, float alpha, float beta, float rho, int m,
                   uint64_t seed, int iterations, double q0, float xi, int nn,
                   int32_t *best_tour, int64_t *best_len, float *tau_out, int32_t *last_tours,
                   int64_t *last_lens, int64_t *iter_best)
{
    if (n < 3 || m < 1 || nn < 0 || nn > 32 || nn > n - 1) return -1;
    int32_t *lists = NULL;
    if (nn > 0) {
        lists = (int32_t *)malloc((size_t)n * nn * sizeof(int32_t));
        if (!lists) return -2;
        orc_nn_lists(n, d, nn, lists);
    }
    size_t cells = (size_t)n * n;
    float *heta = (float *)malloc(cells * sizeof(float));
    float *tau = (float *)malloc(cells * sizeof(float));
    float *choice = (float *)malloc(cells * sizeof(float));
    int32_t *tours = (int32_t *)malloc((size_t)m * (n + 1) * sizeof(int32_t));
    int64_t *lens = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    int32_t *gb = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    uint8_t *visited = (uint8_t *)malloc((size_t)m * n);
    int *cur = (int *)malloc((size_t)m * sizeof(int));
    int *next = (int *)malloc((size_t)m * sizeof(int));
    if (!heta || !tau || !choice || !tours || !lens || !gb || !visited || !cur || !next)
        return -2;

    orc_heta(n, d, (double)beta, heta);
    int64_t cnn = orc_nn_tour_length(n, d);
    float tau0 = (float)(1.0 / ((double)n * (double)cnn));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) tau[(size_t)i * n + j] = (i == j) ? 0.0f : tau0;
    orc_choice(n, tau, heta, alpha, choice);
    uint64_t thr = orc_acs_threshold(q0);
    float keep = 1.0f - rho;

    int64_t best = INT64_MAX;
    for (int it = 0; it < iterations; ++it) {
        uint32_t x[4];
        memset(visited, 0, (size_t)m * n);
        for (int k = 0; k < m; ++k) {
            draw(seed, 0u, (uint32_t)k, (uint32_t)it, x);
            int start = (int)(((uint64_t)x[0] * (uint64_t)n) >> 32);
            tours[(size_t)k * (n + 1)] = start;
            visited[(size_t)k * n + start] = 1;
            cur[k] = start;
        }
        for (int s = 1; s < n; ++s) {
            for (int k = 0; k < m; ++k) {
                draw(seed, (uint32_t)s, (uint32_t)k, (uint32_t)it, x);
                uint64_t r = ((uint64_t)x[1] << 32) | (uint64_t)x[0];
                next[k] = nn > 0 ? orc_acs_select_nn(n, nn, lists + (size_t)cur[k] * nn,
                                                     choice + (size_t)cur[k] * n,
                                                     visited + (size_t)k * n, r, x[2], thr)
                                 : orc_acs_select(n, choice + (size_t)cur[k] * n,
                                                  visited + (size_t)k * n, r, x[2], thr);
            }
            for (int k = 0; k < m; ++k) {
                acs_cross(n, cur[k], next[k], xi, tau0, alpha, heta, tau, choice);
                tours[(size_t)k * (n + 1) + s] = next[k];
                visited[(size_t)k * n + next[k]] = 1;
                cur[k] = next[k];
            }
        }
        for (int k = 0; k < m; ++k) {
            int start = tours[(size_t)k * (n + 1)];
            acs_cross(n, cur[k], start, xi, tau0, alpha, heta, tau, choice);
            tours[(size_t)k * (n + 1) + n] = start;
            int64_t len = 0;
            for (int s = 0; s < n; ++s)
                len += d[(size_t)tours[(size_t)k * (n + 1) + s] * n +
                         tours[(size_t)k * (n + 1) + s + 1]];
            lens[k] = len;
        }
        int kbest = 0;
        for (int k = 1; k < m; ++k)
            if (lens[k] < lens[kbest]) kbest = k;
        if (iter_best) iter_best[it] = lens[kbest];
        if (lens[kbest] < best) {
            best = lens[kbest];
            memcpy(gb, tours + (size_t)kbest * (n + 1), (size_t)(n + 1) * sizeof(int32_t));
        }
        float dep = rho * (float)(1.0 / (double)best);
        for (int s = 0; s < n; ++s) {
            int a = gb[s], b = gb[s + 1];
            size_t ab = (size_t)a * n + b, ba = (size_t)b * n + a;
            tau[ab] = keep * tau[ab] + dep;
            tau[ba] = keep * tau[ba] + dep;
            choice[ab] = choice_cell(tau[ab], heta[ab], alpha);
            choice[ba] = choice_cell(tau[ba], heta[ba], alpha);
        }
    }
    if (best_len) *best_len = best;
    if (best_tour && iterations > 0) memcpy(best_tour, gb, (size_t)(n + 1) * sizeof(int32_t));
    if (tau_out) memcpy(tau_out, tau, cells * sizeof(float));
    if (last_tours) memcpy(last_tours, tours, (size_t)m * (n + 1) * sizeof(int32_t));
    if (last_lens) memcpy(last_lens, lens, (size_t)m * sizeof(int64_t));
    free(heta); free(tau); free(choice); free(tours); free(lens); free(gb); free(visited);
    free(cur); free(next); free(lists);
    return 0;
}

int orc_run_acs(int n, const int32_t *d, float alpha, float beta, float rho, int m,
                uint64_t seed, int iterations, double q0, float xi, int32_t *best_tour,
                int64_t *best_len, float *tau_out, int32_t *last_tours, int64_t *last_lens,
                int64_t *iter_best)
{
    return orc_run_acs_nn(n, d, alpha, beta, rho, m, seed, iterations, q0, xi, 0, best_tour,
                          best_len, tau_out, last_tours, last_lens, iter_best);
}

/* ------------------------------------------------------------------------- */
/* Brute-force optimum for tiny instances (n <= 11): city 0 fixed first,     */
/* every permutation of the rest enumerated.                                 */
/* ------------------------------------------------------------------------- */
static void bf_rec(int n, const int32_t *d, int depth, int *perm, uint8_t *used, int64_t acc,
                   int64_t *best, int *best_perm)
{
    if (acc >= *best) return; /* distances are non-negative */
    if (depth == n) {
        int64_t total = acc + d[(size_t)perm[n - 1] * n + perm[0]];
        if (total < *best) {
            *best = total;
            memcpy(best_perm, perm, (size_t)n * sizeof(int));
        }
        return;
    }
    for (int c = 1; c < n; ++c) {
        if (used[c]) continue;
        used[c] = 1;
        perm[depth] = c;
        bf_rec(n, d, depth + 1, perm, used, acc + d[(size_t)perm[depth - 1] * n + c], best, best_perm);
        used[c] = 0;
    }
}

int64_t orc_brute_force(int n, const int32_t *d, int32_t *tour)
{
    if (n < 2 || n > 11) return -1;
    int perm[11], best_perm[11];
    uint8_t used[11] = {0};
    perm[0] = 0;
    used[0] = 1;
    int64_t best = INT64_MAX;
    bf_rec(n, d, 1, perm, used, 0, &best, best_perm);
    if (tour) {
        for (int i = 0; i < n; ++i) tour[i] = best_perm[i];
        tour[n] = best_perm[0];
    }
    return best;
}
