/*
 * aco.h - C ABI of the GB300 (sm_103a) Ant System for the symmetric TSP.
 *
 * The method is the Ant System of Cecilia, Garcia, Ujaldon, Nisbet and Amos,
 * "Parallelization Strategies for Ant Colony Optimisation on GPUs": m ants
 * build tours by the random proportional rule (Section II, Eq. 1) over
 * choice_info = tau^alpha * eta^beta (Section III-A), then the pheromone is
 * evaporated (Eq. 2) and every ant deposits 1/C^k on its tour's edges
 * (Eqs. 3-4).  Everything runs in CUDA kernels on one GPU; there is no CPU
 * fallback.  If the library cannot reach a GPU every call fails with
 * ACO_ECUDA.
 *
 * Conventions for every entry point:
 *  - Return value: ACO_OK (0) or a negative ACO_E* code; no exception or
 *    abort crosses the ABI.  aco_strerror() names the code and
 *    aco_last_error_message() gives the detail of the last failure on the
 *    calling thread.
 *  - Host pointers are plain C arrays owned by the caller; the library copies
 *    what it needs and never keeps a caller pointer after the call returns.
 *  - Matrices are row-major, n x n, without padding.  Tours are arrays of
 *    n+1 city indices with tour[n] == tour[0] (a closed tour, Section II).
 *  - A handle is not thread-safe: calls on one handle must not overlap.
 *    Work on a handle is ordered on its CUDA stream; calls that return data
 *    to the host synchronise that stream.
 *
 * Readings of points the paper leaves open (the same in the CPU oracle):
 *  - eta_ij^beta = 1/d_ij^beta in double rounded to float; d_ij >= 1 is
 *    required for i != j (eta = 1/d is undefined at d = 0).
 *  - tau0 = m / C_nn, C_nn the nearest-neighbour tour from city 0 (ties to
 *    the lower index); tau_ii = 0.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *    counter = (step, ant, iteration, 0); an ant starts at
 *    floor(x0 * n / 2^32) ("ants are randomly placed", Section II).
 *  - Eq. 1 is sampled exactly by an integer roulette: with M the largest
 *    unvisited weight and B = 46, q_j = floor(w_j * 2^(B-1-ilogb M)) for
 *    unvisited j (so Q < 2^58 for n <= 4096), T = floor(r Q / 2^64) with
 *    r = x1 * 2^32 + x0 and Q = sum q_j, and the chosen city is the first j
 *    (ascending) whose prefix sum exceeds T; if M == 0 the lowest unvisited
 *    city.  The result does not depend on how the kernel tiles the row.
 *  - Deposit (Eqs. 3-4): dtau^k = (float)(1/(double)C^k) on both (a,b) and
 *    (b,a).  The deterministic variants sum q_k = floor(dtau^k * 2^S),
 *    S = 62 - ceil(log2 m) - ilogb(max_k dtau^k), exactly in 64-bit
 *    integers, round the sum to float once and scale it by 2^-S;
 *    tau' = fl(fl((1-rho) tau) + dep).
 *  - choice = tau * eta^beta for alpha == 1, eta^beta for alpha == 0, and
 *    powf(tau, alpha) * eta^beta otherwise.
 *  - The best-so-far tour changes only to a strictly shorter tour; within an
 *    iteration the lowest ant index wins ties.
 */
#ifndef ACO_GB300_H
#define ACO_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define ACO_OK 0
#define ACO_EINVAL (-1)   /* an argument is out of range or inconsistent     */
#define ACO_ENOMEM (-2)   /* a device or host allocation failed              */
#define ACO_ECUDA (-3)    /* a CUDA call failed (no GPU, bad launch, ...)    */
#define ACO_ESTATE (-4)   /* the call is not valid in the handle's state     */
#define ACO_ETIMEOUT (-5) /* a bounded device-side wait gave up              */
#define ACO_EBUSY (-6)    /* no free slot or not enough memory budget left   */

/* ---- limits ------------------------------------------------------------- */
#define ACO_MAX_N 4096    /* cities per instance                             */
#define ACO_MAX_M 16384   /* ants per instance                               */

/* ---- options (aco_set_option / aco_get_option) --------------------------- */
#define ACO_OPT_CHECK 11       /* 1: after every construction a kernel checks
                                  each tour (every city once, closed, stored
                                  length = summed distances) and a failure
                                  makes the next synchronising call return
                                  ACO_ECUDA; 0 (default): no check.  A debug
                                  aid: one extra launch per iteration.       */
#define ACO_OPT_DEPOSIT 1      /* ACO_DEPOSIT_* below; default SYMMETRIC (the
                                  fastest measured on GB300)                  */
#define ACO_OPT_STREAM 2       /* cudaStream_t as int64; 0 = the handle's own   */
#define ACO_OPT_USE_GRAPH 3    /* 1 (default): aco_iterate replays a CUDA graph */
#define ACO_OPT_PROFILE 4      /* 1: record CUDA events around every kernel     */
#define ACO_OPT_WARPS_PER_ANT 5 /* 0 (default) = automatic, else 1, 2 or 4      */
#define ACO_OPT_ANTS_PER_CTA 6 /* 0 (default) = automatic, else 1..32; at most 8
                                  warps per CTA                                */
#define ACO_OPT_LANES_PER_ANT 7 /* 0 (default) = 32; 8 or 16: 32/H ants share a
                                  warp (one warp per ant group)                */
#define ACO_OPT_SELECTION 8    /* ACO_SELECT_* below; default ACO_SELECT_EQ1     */
#define ACO_OPT_NN_LIST 9      /* 0 (default): every unvisited city is a
                                  candidate.  k in [1, min(32, n-1)]: the
                                  nearest-neighbour-list construction (Section
                                  II; the paper's Table 2 versions 4-6 use 30):
                                  list(i) = the k nearest cities of i (ties to
                                  the lower index, in that order); an ant at i
                                  samples Eq. 1 among the unvisited entries of
                                  list(i) (the integer roulette in list order)
                                  and, when all are visited, moves to the
                                  unvisited city with the largest choice_info
                                  value (ties to the lower index).  Needs
                                  ACO_SELECT_EQ1; pool slots: aco_pool_set_nn. */
#define ACO_OPT_STAGING 10     /* how the construction kernel brings row
                                  choice[cur] into shared memory at each step:
                                  0 one bulk copy (TMA engine, cp.async.bulk)
                                  completing on an mbarrier; 1 coalesced
                                  16-byte loads by the ant's threads.  Default:
                                  1 for n <= 64, else 0 (the faster measured
                                  on GB300).  Results are identical.          */

#define ACO_SELECT_EQ1 0       /* Eq. 1 (random proportional rule), exact      */
#define ACO_SELECT_DATA_PARALLEL 1 /* the paper's data-parallel kernel (Section
                                  III-A, Fig. 1): every unvisited city j draws
                                  u_j in (0,1] (Philox counter (step, ant,
                                  iteration, 1 + j/4), word j mod 4, u_j =
                                  (floor(x/2^8) + 1) 2^-24), scores fl(u_j w_j),
                                  and the highest score wins (ties to the lower
                                  index; all scores 0: lowest unvisited city).
                                  Not Eq. 1: for two cities with w1 >= w2 it
                                  picks city 2 with probability w2 / (2 w1).
                                  Whole warps per ant only (lanes per ant 32,
                                  warps per ant 1 or 2).                       */
#define ACO_SELECT_EXP_RACE 2  /* the exponential race, a per-candidate random
                                  rule that samples Eq. 1: every unvisited city
                                  j takes v_j = floor(x/2^8) + 1 from the same
                                  counter and word as above, E_j = -ln(v_j
                                  2^-24) in single precision by the range-
                                  reduced inverse-hyperbolic-tangent series
                                  (every operation rounded on its own), and
                                  the smallest key fl(E_j / w_j) wins (ties to
                                  the lower index; zero weights and
                                  overflowing keys are +inf).  City j then wins
                                  with probability w_j / sum w.  Same tilings
                                  as ACO_SELECT_DATA_PARALLEL.                 */

#define ACO_DEPOSIT_GATHER 0   /* atomic-free: edges bucketed per city by the
                                  construction kernel, one warp reduces a row  */
#define ACO_DEPOSIT_ATOMIC_U64 1 /* red.global.add.u64 of the fixed-point q_k  */
#define ACO_DEPOSIT_ATOMIC_F32 2 /* red.global.add.f32 of dtau^k into tau after
                                  evaporation (the paper's atomic kernel; the
                                  order of additions, hence the last bits of
                                  tau, is not deterministic)                   */
#define ACO_DEPOSIT_SYMMETRIC 3  /* the paper's "Reduction" version (Section
                                  III-B): for the symmetric TSP the edge (a,b)
                                  adds q_k once, to the upper-triangle cell
                                  (min, max), with red.global.add.u64 (half the
                                  atomics of ATOMIC_U64); the apply pass reads
                                  tau, eta^beta and the accumulator in the
                                  upper triangle only and writes both halves
                                  of tau and choice_info through shared-memory
                                  tiles.  Results equal GATHER and ATOMIC_U64
                                  bit for bit.                                 */
#define ACO_DEPOSIT_SORT 4     /* atomic-free scatter-to-gather by sorting
                                  (Section III-B's idea without its n^4
                                  loads): each tour edge becomes the key
                                  min(a,b)*n + max(a,b) with its ant as value,
                                  a stable LSD radix sort (8-bit digits) groups
                                  equal edges, one thread per run of equal
                                  keys sums q_k exactly, and the symmetric
                                  apply pass finishes the update.  Bit-exact
                                  with the other deterministic variants.
                                  Allocates 16 bytes per (ant, city) of
                                  scratch when first selected.                */

/* ---- phases reported by aco_get_kernel_times ------------------------------ */
#define ACO_PHASE_CONSTRUCT 0  /* tour construction kernel                      */
#define ACO_PHASE_BEST 1       /* iteration-best / best-so-far kernel          */
#define ACO_PHASE_DEPOSIT 2    /* deposit kernel(s) (0 for the gather variant)  */
#define ACO_PHASE_UPDATE 3     /* evaporation + deposit apply + choice_info     */
#define ACO_NUM_PHASES 4

typedef struct aco_colony *aco_handle;

/* Name of an error code (static string). */
const char *aco_strerror(int code);

/* Detail of the last failure on the calling thread (static per-thread buffer). */
const char *aco_last_error_message(void);

/*
 * aco_create - set up one Ant System instance (Section II; Section III-A for
 * the choice_info table).
 *   n      number of cities, 3 <= n <= ACO_MAX_N
 *   dist   host array, n*n int32, row-major: symmetric, d_ii = 0 and
 *          d_ij >= 1 for i != j.  Copied; the caller keeps ownership.
 *   alpha  pheromone exponent (finite, >= 0)
 *   beta   heuristic exponent (finite, >= 0)
 *   rho    evaporation rate, 0 < rho <= 1 (Eq. 2)
 *   m      number of ants, 1 <= m <= ACO_MAX_M
 *   seed   Philox key
 *   out    receives the handle (owned by the library until aco_destroy)
 * Computes eta^beta, the nearest-neighbour tour, tau0 and the first
 * choice_info on the device.  Errors: ACO_EINVAL (bad argument, dist not
 * symmetric / zero diagonal / positive off-diagonal), ACO_ENOMEM, ACO_ECUDA.
 * On error *out is set to NULL and nothing is leaked.
 */
int aco_create(int32_t n, const int32_t *dist, float alpha, float beta, float rho, int32_t m,
               uint64_t seed, aco_handle *out);

/* aco_destroy - free everything the handle owns; NULL is accepted. */
int aco_destroy(aco_handle h);

/*
 * aco_choice_info - recompute choice_info = tau^alpha * eta^beta from the
 * current tau (Section III-A; idempotent).  If out != NULL, copy it to the
 * host as n*n float (row-major).
 */
int aco_choice_info(aco_handle h, float *out);

/*
 * aco_construct_tours - every ant builds a tour for the current iteration
 * (Section II, Eq. 1), then the iteration-best and best-so-far tours are
 * updated.  The iteration counter does not advance, so calling it twice
 * gives the same tours.  tours (m*(n+1) int32) and lens (m int64, C^k) are
 * host outputs; either may be NULL.
 */
int aco_construct_tours(aco_handle h, int32_t *tours, int64_t *lens);

/*
 * aco_update_pheromone - evaporation (Eq. 2) and deposit (Eqs. 3-4) from the
 * tours of the last aco_construct_tours, then choice_info is recomputed and
 * the iteration counter advances.  ACO_ESTATE if no tours were constructed
 * since the last update.
 */
int aco_update_pheromone(aco_handle h);

/*
 * aco_iterate - `iterations` full Ant System iterations (construct, best,
 * update).  With ACO_OPT_USE_GRAPH the iteration is captured once as a CUDA
 * graph and replayed.  Asynchronous: returns once the work is enqueued.
 */
int aco_iterate(aco_handle h, int32_t iterations);

/*
 * aco_best_tour - best-so-far tour (n+1 int32) and its length; either output
 * may be NULL.  ACO_ESTATE before the first construction.
 */
int aco_best_tour(aco_handle h, int32_t *tour, int64_t *len);

/* aco_get_pheromone - copy tau (n*n float, row-major) to the host. */
int aco_get_pheromone(aco_handle h, float *tau);

/* aco_get_heuristic - copy eta^beta (n*n float, row-major) to the host. */
int aco_get_heuristic(aco_handle h, float *heta);

/* aco_get_iteration - number of completed pheromone updates. */
int aco_get_iteration(aco_handle h, int64_t *iteration);

/* aco_get_tau0 - the initial pheromone m / C_nn and C_nn; either may be NULL. */
int aco_get_tau0(aco_handle h, float *tau0, int64_t *nn_len);

/*
 * aco_set_mmas - switch the handle's update rule to the MAX-MIN Ant System,
 * the ACO variant the paper cites as an earlier GPU target (Section II-B);
 * the paper leaves other variants to future work (Section V) and does not
 * define it, so this follows Stutzle and Hoos, "MAX-MIN Ant System", Future
 * Generation Computer Systems 16 (2000):
 *  - construction is unchanged (Eq. 1, or the rule/lists the options select);
 *  - one tour deposits per iteration: the iteration best (best_so_far = 0)
 *    or the best-so-far tour (best_so_far = 1), dtau = (float)(1/(double)C)
 *    on its n edges in both directions, after evaporation by (1 - rho);
 *  - every off-diagonal tau is then clamped into [tau_min, tau_max], where
 *    tau_max = 1 / (rho C_gb) with C_gb the best-so-far length, and
 *    tau_min = tau_max * f, f = (1 - p^(1/n)) / ((n/2 - 1) p^(1/n)),
 *    p = p_best (tau_min = tau_max where that is larger); both computed in
 *    double, f first, and rounded to float once;
 *  - tau starts at tau_max computed from C_nn, replacing m / C_nn.
 * The ACO_OPT_DEPOSIT variants do not apply (a single tour deposits, without
 * atomics).  Call before the first construction (ACO_ESTATE after it); the
 * switch cannot be undone.  p_best must lie in (0, 1) and best_so_far be 0
 * or 1 (ACO_EINVAL).
 */
int aco_set_mmas(aco_handle h, double p_best, int32_t best_so_far);

/*
 * aco_set_acs - switch the handle to the Ant Colony System, the ACO variant
 * the paper names as its next target (Section V); the paper does not define
 * it, so this follows Dorigo and Gambardella, IEEE Trans. Evol. Comp. 1(1)
 * (1997), with choice_info = tau^alpha * eta^beta as in the Ant System:
 *  - tau starts at tau0 = (float)(1 / (n C_nn)) off the diagonal;
 *  - at step s ant k draws Philox (s, k, iteration, 0); it exploits when
 *    word x2 < floor(q0 * 2^32), moving to the unvisited city of largest
 *    choice_info (ties to the lower index), and otherwise samples Eq. 1 by
 *    the integer roulette;
 *  - the ants move in lockstep: all choose their s-th city from the same
 *    state, then every edge crossed at that step gets the local update
 *    tau <- fl(fl((1-xi) tau) + fl(xi tau0)) in both directions, once per
 *    ant that crossed it, with its choice_info; the closing edge back to the
 *    start is the n-th step;
 *  - after the tours only the best-so-far tour's edges get the global update
 *    tau <- fl(fl((1-rho) tau) + fl(rho / C_bs)) (rho as given to create);
 *    no other cell evaporates.
 * The colony runs in one CTA, so m <= 32 (the variant's usual m is 10).
 * Because construction changes tau, construction calls are not idempotent
 * under this rule.  With ACO_OPT_NN_LIST the steps use the lists (the
 * original variant's candidate lists): at city i, if an entry of list(i) is
 * unvisited, exploitation takes the unvisited entry of largest choice_info
 * (ties to the earlier entry) and exploration samples Eq. 1 over the
 * unvisited entries in list order; if every entry is visited, either takes
 * the unvisited city of largest choice_info.  ACO_OPT_SELECTION does not
 * apply.  Call once, before the first construction (ACO_ESTATE otherwise);
 * q0 and xi must lie in [0, 1] and m <= 32 (ACO_EINVAL).
 */
int aco_set_acs(aco_handle h, double q0, float xi);

/*
 * Checkpoint and resume (library feature; the paper has no counterpart).
 * The state of a run is tau, the best-so-far tour and length, the iteration
 * counter and the update rule with its parameters.  The random numbers are
 * counter-based on (seed, iteration, ant, step), so a run restored from a
 * checkpoint continues exactly as the uninterrupted run would.
 *   aco_save_state: *size = bytes of the checkpoint; with buf != NULL and
 *     capacity >= *size it is written to buf (host memory).
 *   aco_restore_state: load a checkpoint into a handle created with the same
 *     n, distances, alpha, beta, rho, m and seed (the header checks all but
 *     the distances; ACO_EINVAL on a mismatch, a truncated or foreign
 *     buffer).  choice_info is recomputed from tau.  Options (deposit
 *     variant, tiling, staging, lists, selection, stream) are not part of the
 *     state: set them on the new handle as before; a checkpoint of an Ant
 *     Colony System run needs a handle without lists and with Eq. 1.
 */
int aco_save_state(aco_handle h, void *buf, uint64_t capacity, uint64_t *size);
int aco_restore_state(aco_handle h, const void *buf, uint64_t size);

/*
 * aco_get_mmas_limits - the current trail limits tau_min and tau_max of a
 * MAX-MIN handle (either output may be NULL); ACO_ESTATE for an Ant System
 * handle.
 */
int aco_get_mmas_limits(aco_handle h, float *tau_min, float *tau_max);

/* aco_set_option / aco_get_option - ACO_OPT_* keys above. */
int aco_set_option(aco_handle h, int32_t key, int64_t value);
int aco_get_option(aco_handle h, int32_t key, int64_t *value);

/*
 * aco_get_kernel_times - with ACO_OPT_PROFILE on, the device time in ms of
 * each ACO_PHASE_* in the most recent iteration (synchronises the stream).
 * ms must hold ACO_NUM_PHASES floats.
 */
int aco_get_kernel_times(aco_handle h, float *ms);

/* aco_synchronize - wait for the handle's stream and report device-side errors. */
int aco_synchronize(aco_handle h);

/*
 * aco_kernel_launches_per_iteration - how many kernels one iteration launches
 * with the handle's current options.
 */
int aco_kernel_launches_per_iteration(aco_handle h, int32_t *count);

/*
 * aco_create_coords - as aco_create, but the instance is given by integer
 * city coordinates (xy: n pairs x, y, host, copied) and the distance matrix
 * is built on the device with the TSPLIB EUC_2D rounding
 * d = floor(sqrt(dx^2 + dy^2) + 0.5) in IEEE double.  Coordinates must lie in
 * [-2^25, 2^25] and be pairwise distinct (ACO_EINVAL otherwise).
 */
int aco_create_coords(int32_t n, const int32_t *xy, float alpha, float beta, float rho,
                      int32_t m, uint64_t seed, aco_handle *out);

/* ======================================================================== *
 * Batched and served instances: a pool of device-resident slots.
 *
 * A pool owns one HBM arena of `budget_bytes`; every admitted instance gets
 * its own dist / eta^beta / tau / choice_info / tours / best-tour block from
 * it and keeps it until released.  aco_pool_step() runs one iteration for
 * every live slot: one construction launch per tiling class (Ant System and
 * MAX-MIN Ant System instances of similar n), one launch for all Ant Colony
 * System slots, one best launch for all slots, one row-update launch (the
 * gather update, or the MAX-MIN update) and one global-update launch for the
 * Ant Colony System slots, captured as a CUDA graph while the live set is
 * unchanged.  Random numbers use each instance's own seed and iteration
 * counter, so an instance's results are identical alone and in any mix.
 * Pools use the deterministic gather deposit.  A pool is not thread-safe.
 * ======================================================================== */
typedef struct aco_pool *aco_pool_handle;

/* Device bytes one instance of n cities and m ants takes from a pool. */
int aco_pool_bytes_needed(int32_t n, int32_t m, uint64_t *bytes);

/* aco_pool_create - max_slots >= 1 concurrent instances within budget_bytes of HBM. */
int aco_pool_create(int32_t max_slots, uint64_t budget_bytes, aco_pool_handle *out);

/* aco_pool_destroy - free the arena and every slot; NULL is accepted. */
int aco_pool_destroy(aco_pool_handle p);

/*
 * aco_pool_admit / aco_pool_admit_coords - add an instance that will run
 * `iterations` iterations (>= 1) in subsequent aco_pool_step calls.  Same
 * argument rules as aco_create / aco_create_coords.  The upload and setup
 * (eta^beta, nearest-neighbour tour, tau0, choice_info) run on a side stream
 * and overlap with steps already in flight.  A pageable dist / xy buffer may
 * be reused as soon as the call returns; a pinned one must stay unchanged
 * until the next aco_pool_step or aco_pool_synchronize.  *slot receives the
 * slot index.
 * ACO_EBUSY if no slot is free or the arena has no block large enough.
 */
int aco_pool_admit(aco_pool_handle p, int32_t n, const int32_t *dist, float alpha, float beta,
                   float rho, int32_t m, uint64_t seed, int32_t iterations, int32_t *slot);
int aco_pool_admit_coords(aco_pool_handle p, int32_t n, const int32_t *xy, float alpha,
                          float beta, float rho, int32_t m, uint64_t seed, int32_t iterations,
                          int32_t *slot);

/*
 * aco_pool_set_acs / aco_pool_set_mmas - switch a live slot that has not yet
 * taken part in a step to the Ant Colony System or the MAX-MIN Ant System,
 * with the rules and argument ranges of aco_set_acs / aco_set_mmas (rho, as
 * admitted, is then the rule's own rate).  The start trails are written on
 * the side stream after the admission's setup.  A slot's results are those
 * of a handle created with the same arguments and switched the same way.
 * Every aco_pool_step runs all live Ant Colony System slots in one launch,
 * one CTA per colony (m <= 32, ACO_EINVAL otherwise), beside the Ant System
 * classes; MAX-MIN slots construct with the Ant System slots and take the
 * rule's update in the row-update launch.  ACO_ESTATE once the slot has
 * stepped or already switched; aco_pool_tiling answers ACO_EINVAL for an
 * Ant Colony System slot.
 */
int aco_pool_set_acs(aco_pool_handle p, int32_t slot, double q0, float xi);
int aco_pool_set_mmas(aco_pool_handle p, int32_t slot, double p_best, int32_t best_so_far);

/*
 * aco_pool_set_nn - nearest-neighbour-list construction for a live slot
 * before its first step, as ACO_OPT_NN_LIST does for a handle (the
 * construction of the paper's Table 2 versions 4-6, Section II): nn = 1 ..
 * min(n - 1, 32) entries, 0 = dense Eq. 1 again.  Composes with all three
 * rules (the Ant Colony System as with ACO_OPT_NN_LIST on a handle).  All
 * Ant System and MAX-MIN list slots of a pool construct in one launch (one
 * warp per ant) and refresh their list-ordered choice_info after each
 * update; Ant Colony System colonies with lists run in one launch of their
 * own.  ACO_ESTATE after the slot's first step.
 */
int aco_pool_set_nn(aco_pool_handle p, int32_t slot, int32_t nn);

/*
 * aco_pool_save_slot / aco_pool_restore_slot - checkpoints of pool slots, in
 * the format of aco_save_state (library feature; the paper has no
 * counterpart).  A blob from either side restores into the other.
 *   aco_pool_save_slot: *size = bytes of the checkpoint of slot (live or
 *     finished); with buf != NULL and capacity >= *size it is written to buf
 *     (host memory).  Synchronises the pool.
 *   aco_pool_restore_slot: load a checkpoint into a live slot admitted with
 *     the same n, distances, alpha, beta, rho, m and seed, before its first
 *     step and rule switch (ACO_ESTATE otherwise); the slot takes the
 *     checkpoint's update rule and iteration counter, and its own admitted
 *     iteration budget counts from there.  choice_info is recomputed from
 *     tau.  ACO_EINVAL on a mismatch, a truncated or foreign buffer.
 */
int aco_pool_save_slot(aco_pool_handle p, int32_t slot, void *buf, uint64_t capacity,
                       uint64_t *size);
int aco_pool_restore_slot(aco_pool_handle p, int32_t slot, const void *buf, uint64_t size);

/*
 * aco_pool_step - one iteration for every live slot (asynchronous; with
 * multi-rate stepping, each slot's own rate).  A slot whose iteration budget
 * is used up becomes finished and leaves the live set.
 * *live_after (may be NULL) receives the number of slots still live.
 */
int aco_pool_step(aco_pool_handle p, int32_t *live_after);

/*
 * aco_pool_set_single_launch - on = 1: each step builds the tours of every
 * construction class in one persistent launch (warps take (instance, ant)
 * items from a global ticket, widest chunks first, each with its class's
 * chunk width) instead of one launch per class; only when every class uses
 * whole warps with at most 36 cities per lane, one iteration per step and no
 * lists, else the step keeps one launch per class.  Results are identical
 * either way.  on = 0 (default): one launch per class.
 */
int aco_pool_set_single_launch(aco_pool_handle p, int32_t on);

/*
 * aco_pool_finished - slots that are finished but not yet released, in
 * completion order; writes at most `capacity` of them and the total count.
 */
int aco_pool_finished(aco_pool_handle p, int32_t *slots, int32_t capacity, int32_t *count);

/*
 * aco_pool_result - best-so-far tour (n+1 int32) and length of a slot, live
 * or finished.  For a finished slot it waits only for the step that ran the
 * slot's last iterations and reads on a stream of its own, so steps launched
 * since keep running; for a live slot it synchronises the pool.  Either
 * output may be NULL.
 */
int aco_pool_result(aco_pool_handle p, int32_t slot, int32_t *tour, int64_t *len);

/* aco_pool_pheromone - copy a slot's tau (n*n float) to the host. */
int aco_pool_pheromone(aco_pool_handle p, int32_t slot, float *tau);

/*
 * aco_pool_release - return a finished (or live) slot and its memory.  A
 * finished slot waits only for its last step (no later step reads it); a
 * live slot first waits for all work in flight.
 */
int aco_pool_release(aco_pool_handle p, int32_t slot);

/*
 * aco_pool_stats - live and finished slot counts, arena bytes in use, and
 * kernel launches of the last step.  Any output may be NULL.
 */
int aco_pool_stats(aco_pool_handle p, int32_t *live, int32_t *finished, uint64_t *bytes_in_use,
                   int32_t *launches_last_step);

/*
 * Construction tiling of pooled instances.  Live instances are grouped into
 * classes by their default tiling (whole warps, C cities per lane); each
 * class is one construction launch per step.  With autotuning on (the
 * default), the first step that sees a class times each candidate tiling on
 * it (1, 2 or 4 warps per ant, or 8- or 16-lane segments with 4 or 2 ants per
 * warp, leaving out tilings with more than twice the default's city slots per
 * ant; each with either row staging of ACO_OPT_STAGING; the second of two
 * runs) and keeps the fastest for that class from then on.  Every tiling builds the same tours, so tuning never changes a
 * result.
 *   aco_pool_set_autotune: on = 1 (default) or 0 (the default tiling always;
 *     forgets earlier choices).
 *   aco_pool_autotune: run the tuner now for classes of the current live
 *     set not tuned yet (otherwise it runs inside the next aco_pool_step);
 *     it builds tours but advances no iteration.
 *   aco_pool_tiling: the tiling the class of live `slot` uses: warps per ant,
 *     lanes per ant, cities per lane and row staging (0 bulk copy, 1 lane
 *     copies); any output may be NULL;
 *     ACO_ESTATE before the first step after the live set changed.
 */
int aco_pool_set_autotune(aco_pool_handle p, int32_t on);
/*
 * aco_pool_set_multirate (no counterpart in the paper: a serving extension
 * of the batched step) - on = 1: every aco_pool_step runs k iterations for
 * each group of slots (a construction class, or all Ant Colony System
 * colonies), each group on its own stream with its own best and update
 * launches, where k = floor(T_max / T_group) within [1, 64] from a model of
 * one iteration's time alone (about n (0.6 + 0.025 n / 32) us; 4 n us for a
 * colony) and T_max that of the slowest group, and never more than the
 * iterations any slot of the group has left.  Short instances then keep
 * pace with the longest instead of waiting one long step per iteration.
 * Every slot still runs exactly its own iterations, so its results are
 * unchanged.  on = 0 (default): one iteration per step for every slot.
 * ACO_EINVAL for a static batch (aco_batch_*), whose steps count iterations.
 * aco_pool_rate: the iterations the last step ran for `slot` (live or
 * finished; 1 unless multi-rate; ACO_ESTATE before its first step).
 */
int aco_pool_set_multirate(aco_pool_handle p, int32_t on);
int aco_pool_rate(aco_pool_handle p, int32_t slot, int32_t *iterations_per_step);
int aco_pool_autotune(aco_pool_handle p);
int aco_pool_tiling(aco_pool_handle p, int32_t slot, int32_t *warps_per_ant,
                    int32_t *lanes_per_ant, int32_t *cities_per_lane, int32_t *staging);

/*
 * The tuner's table, to keep it across runs (the Python binding saves it as
 * JSON).  One entry is 7 int32: the class's default (warps per ant, lanes
 * per ant, cities per lane) and the chosen (warps per ant, lanes per ant,
 * ants per CTA, staging).
 *   aco_pool_get_tuning: *count = entries in the table; up to `capacity` of
 *     them are written to `entries` (7 * capacity int32) when it is not NULL.
 *   aco_pool_set_tuning: replace the table (count >= 0 entries); classes in
 *     it are not timed again.  ACO_EINVAL if an entry names an unsupported
 *     tiling (the table is then unchanged).  Turns autotuning on.
 */
int aco_pool_get_tuning(aco_pool_handle p, int32_t *entries, int32_t capacity, int32_t *count);
int aco_pool_set_tuning(aco_pool_handle p, const int32_t *entries, int32_t count);

/* aco_pool_synchronize - wait for all pool work and report device-side errors. */
int aco_pool_synchronize(aco_pool_handle p);

/*
 * Static batches (a pool with one slot per instance and no iteration limit).
 *   aco_batch_create: count instances; ns[i] cities, dists[i] (host, n*n,
 *   copied), alpha/beta/rho/ms/seeds per instance.
 *   aco_batch_iterate: `iterations` steps of every instance.
 *   aco_batch_best: best-so-far tour and length of instance idx.
 */
typedef struct aco_pool *aco_batch;
int aco_batch_create(int32_t count, const int32_t *ns, const int32_t *const *dists,
                     const float *alpha, const float *beta, const float *rho, const int32_t *ms,
                     const uint64_t *seeds, aco_batch *out);
int aco_batch_iterate(aco_batch b, int32_t iterations);
int aco_batch_best(aco_batch b, int32_t idx, int32_t *tour, int64_t *len);
int aco_batch_destroy(aco_batch b);

/* ======================================================================== *
 * Allocation-free pheromone update.
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory: code running while someone else is
 * capturing a CUDA graph, runtimes without a device allocator, and hosts
 * that reserve all device memory up front.  It performs the same update as
 * aco_update_pheromone with ACO_DEPOSIT_ATOMIC_U64 (same results bit for
 * bit), but on arrays the caller owns and with its scratch (a 64-bit
 * accumulator of ACO_NOALLOC_MAX_N^2 entries plus ACO_NOALLOC_MAX_M per-ant
 * deposits, about 8.4 MB) in one static device array that the library
 * reserves on every GPU that loads it, until the process exits.
 * ======================================================================== */
#define ACO_NOALLOC_MAX_N 1024
#define ACO_NOALLOC_MAX_M 4096

/*
 * aco_update_pheromone_noalloc - evaporation (Eq. 2), deposit (Eqs. 3-4)
 * and choice_info, on device arrays, without allocating.
 *   n, m    cities (3..ACO_NOALLOC_MAX_N) and ants (1..ACO_NOALLOC_MAX_M);
 *           larger sizes are rejected with ACO_EINVAL.
 *   tours   device, m rows of n+1 int32 cities: closed tours that visit
 *           every city once (tour[n] == tour[0]), as the construction
 *           builds them.  Entries outside [0, n) are ignored.  The deposit
 *           is summed in 64-bit fixed point scaled so that m ants' deposits
 *           on one edge fit; a row that repeats an edge adds it again and
 *           can overflow that sum without an error being reported.
 *   lens    device, m int64 tour lengths C^k (>= 1).
 *   heta    device, n*n float eta^beta, row-major.
 *   tau     device, n*n float, updated in place.
 *   choice  device, n*n float, written with tau'^alpha * eta^beta.
 *   alpha, rho  as in aco_create.
 *   stream  cudaStream_t as int64 (0 = the legacy default stream); the work
 *           is enqueued there and the call returns without synchronising.
 * It calls no cudaMalloc, cudaFree or other allocating routine.  The first
 * call on a device looks up the static array's device address with
 * cudaGetSymbolAddress (the current device must be the one the pointers
 * belong to); make that first call before any stream capture.  Every call
 * shares the one array and each call clears what it uses first, so calls
 * that overlap on the GPU (different streams, or different host threads on
 * one device) race and corrupt each other's results: serialise them.
 */
int aco_update_pheromone_noalloc(int32_t n, int32_t m, const int32_t *tours, const int64_t *lens,
                                 const float *heta, float *tau, float *choice, float alpha,
                                 float rho, int64_t stream);

/*
 * aco_selftest_bounded_wait - exercise the library's bounded device-side
 * wait (no counterpart in the paper).  A one-warp kernel expects 16 bytes on
 * an mbarrier and waits with the loop the construction kernel uses, giving
 * up after `polls` polls (1 <= polls <= 2^20).  complete = 1: a 16-byte bulk
 * copy delivers the bytes, the wait succeeds, ACO_OK.  complete = 0: nothing
 * completes the phase, the wait gives up and the call returns ACO_ETIMEOUT;
 * the kernel still ends normally and the context stays usable.
 */
int aco_selftest_bounded_wait(int32_t polls, int32_t complete);

/*
 * aco_philox4x32_10 - the kernels' counter-based generator (Philox4x32-10,
 * Salmon, Moraes, Dror and Shaw, SC'11), evaluated on the GPU for `count`
 * counters: ctr and out are host arrays of 4 * count uint32 (c0..c3 and
 * x0..x3 per entry), key holds (k0, k1).  The construction kernels draw
 * counter (step, ant, iteration, 0) with key (seed low, seed high) for Eq. 1,
 * and (step, ant, iteration, 1 + j/4) for the data-parallel rule.
 * 1 <= count <= 2^24; ACO_EINVAL on NULL pointers.
 */
int aco_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int32_t count);

/*
 * aco_race_exponential - the exponential race's variate (ACO_SELECT_EXP_RACE,
 * a per-candidate rule that samples Eq. 1 of Section II; no counterpart in
 * the paper's kernels) as the construction kernels compute it, on the GPU:
 * out[i] = E for the Philox word x[i], E = -ln(v 2^-24), v = floor(x[i] /
 * 2^8) + 1, in single precision by the range-reduced inverse-hyperbolic-
 * tangent series.  x and out are host arrays of `count` entries,
 * 1 <= count <= 2^24; ACO_EINVAL on NULL pointers.
 */
int aco_race_exponential(const uint32_t *x, float *out, int32_t count);

/*
 * aco_stream_read - read-bandwidth probe for the construction kernel's
 * roofline (measurement infrastructure; no counterpart in the paper).  The
 * construction of Section III-A reads the rows of choice_info, which stay in
 * L2 at the benchmark sizes, so its ceiling is the rate at which the SMs read
 * an L2-resident buffer.  One launch on `stream` (a cudaStream_t as an
 * integer; 0 = the legacy default stream) reads the caller's device buffer
 * `buf` (16-byte aligned, `bytes` long) `reps` times:
 *   mode 0: 16-byte loads that bypass L1, 256 threads per CTA;
 *   mode 1: 16 KB bulk copies (cp.async.bulk) into shared memory, one warp
 *           per CTA with four stages, as the construction kernel stages rows.
 * The grid is blocks_per_sm (1..32) CTAs per SM.  The call returns after the
 * launch; the caller times it with CUDA events on `stream`.  `sink` (device,
 * one float) keeps the loads live and is written only in a case that does not
 * occur in practice; `status` (device, one uint32) receives bit 1 if a bulk
 * copy's bounded wait gave up (the CTA then waits, again bounded, for its
 * copies in flight and ends).  The caller owns every buffer.
 * ACO_EINVAL: NULL pointers, misalignment, bytes not a positive multiple of
 * 16 (mode 0) or 16384 (mode 1), reps outside [1, 2^20], an unknown mode.
 */
int aco_stream_read(const void *buf, uint64_t bytes, int32_t reps, int32_t mode,
                    int32_t blocks_per_sm, uint64_t stream, float *sink, uint32_t *status);

#ifdef __cplusplus
}
#endif

#endif /* ACO_GB300_H */
