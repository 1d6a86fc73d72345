// Batched and served instances: a pool of device-resident slots
// (include/aco.h, aco_pool_* and aco_batch_*).
//
// Memory: one cudaMalloc'ed arena of the caller's HBM budget, carved by a
// first-fit free list (host side) into one block per instance.  Each step
// runs, for every live slot, the same three phases as a single instance:
//   construct  one launch per tiling class (C cities per lane, G warps per
//              ant), items (slot, ant) listed longest instance first; one
//              launch for all nearest-neighbour-list slots; one launch for
//              all Ant Colony System colonies (a CTA each);
//   best       one CTA per live slot;
//   update     one warp per (slot, row): gather deposit + evaporation +
//              choice_info, fused (the MAX-MIN rule for its slots), then the
//              list-order refresh for list slots; the colonies' global
//              update on their best tours.
// Slots choose their rule, lists and checkpoint before their first step.
// Multi-rate stepping repeats each group's phases k times per step on its
// own stream.  The device-side lists are rebuilt and the step re-captured as
// a CUDA graph only when the live set (or a group's rate) changes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <new>
#include <vector>

#include "../../include/aco.h"
#include "aco_device.cuh"
#include "kernels.h"
#include "runtime.h"
#include "checkpoint.h"

namespace aco {

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct Layout {
  size_t dist, heta, tau, choice, tours, lens, nbr, q, delta, best, dep_nb, nnlist, nnchoice, st,
      total;
};

static Layout layout_of(int n, int m) {
  const size_t ld = (size_t)((n + 3) / 4 * 4), ldt = (size_t)((n + 1 + 3) / 4 * 4),
               ldm = (size_t)((m + 31) / 32 * 32);
  const size_t mat = (size_t)n * ld;
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  L.dist = take(mat * 4);
  L.heta = take(mat * 4);
  L.tau = take(mat * 4);
  L.choice = take(mat * 4);
  L.tours = take((size_t)m * ldt * 4);
  L.lens = take((size_t)m * 8);
  L.nbr = take((size_t)n * ldm * 4);
  L.q = take((size_t)m * 8);
  L.delta = take((size_t)m * 4);
  L.best = take(((size_t)n + 1) * 4);
  L.dep_nb = take((size_t)n * 4);
  L.nnlist = take((size_t)n * kNnStride * 4);
  L.nnchoice = take((size_t)n * kNnStride * 4);
  L.st = take(sizeof(IterState));
  L.total = off;
  return L;
}

static int validate_coords(int32_t n, const int32_t* xy) {
  if (n < 3 || n > ACO_MAX_N) return fail(ACO_EINVAL, "n=%d outside [3, %d]", n, ACO_MAX_N);
  if (!xy) return fail(ACO_EINVAL, "xy is NULL");
  const int32_t lim = 1 << 25;
  std::vector<std::pair<int32_t, int32_t>> pts((size_t)n);
  for (int i = 0; i < n; ++i) {
    const int32_t x = xy[2 * i], y = xy[2 * i + 1];
    if (x < -lim || x > lim || y < -lim || y > lim)
      return fail(ACO_EINVAL, "coordinate of city %d outside [-2^25, 2^25]", i);
    pts[(size_t)i] = {x, y};
  }
  std::sort(pts.begin(), pts.end());
  for (int i = 1; i < n; ++i)
    if (pts[(size_t)i] == pts[(size_t)i - 1])
      return fail(ACO_EINVAL, "duplicate city coordinates: eta = 1/d is undefined at d = 0");
  return ACO_OK;
}

int validate_coords_public(int32_t n, const int32_t* xy) { return validate_coords(n, xy); }

}  // namespace aco

using namespace aco;

struct PoolSlot {
  bool used = false;
  bool live = false;
  bool finished = false;
  int n = 0, m = 0;
  long long iters_left = 0;
  size_t off = 0, bytes = 0;
  Instance I{};
  cudaEvent_t ready = nullptr;  // setup done on the side stream
  bool wait_ready = false;
  bool started = false;  // taken part in a step (the update rule is then fixed)
  bool restored = false; // state loaded from a checkpoint (rule fixed as well)
  int rate = 1;          // iterations per step (multi-rate stepping)
  bool nn_built = false; // nearest-neighbour lists built (aco_pool_set_nn)
  long long finish_step = -1;  // the step that ran the slot's last iterations
};

struct aco_pool {
  int max_slots = 0;
  size_t budget = 0;
  void* arena = nullptr;
  std::map<size_t, size_t> free_blocks;  // offset -> size
  size_t in_use = 0;
  std::vector<PoolSlot> slots;
  std::vector<int> finished_order;
  cudaStream_t stream = nullptr, side = nullptr;
  int sms = 148;
  // device tables
  Instance* d_inst = nullptr;
  int* d_live = nullptr;
  int2* d_items = nullptr;
  int2* d_rows = nullptr;
  int* d_coords = nullptr;  // staging for aco_pool_admit_coords (n pairs)
  int* d_acs = nullptr;     // live Ant Colony System slots
  int* d_cls_slots = nullptr;  // the live slots of each class, class after class
  size_t items_cap = 0, rows_cap = 0;
  // host mirrors of the lists
  std::vector<int> h_live, h_acs, h_cls_slots;
  int acs_max_m = 0, acs_max_n = 0;
  int acs_dense = 0;  // h_acs holds the colonies without lists first, then those with
  // Multi-rate stepping: each class (and the colonies) runs `k` iterations
  // per step, chosen so that short instances keep pace with the longest.
  bool multirate = false;
  int acs_k = 1;
  std::vector<int2> h_items, h_rows;
  struct Class {
    ConstructTiling t;
    int begin, count;               // its items (slot, ant)
    std::tuple<int, int, int> key;  // the default tiling's (G, H, C)
    int max_n;
    int slot_begin, slot_count;     // its slots in h_cls_slots
    int row_begin, row_count, max_ld;  // its rows in h_rows
    int k;                          // iterations per step
    bool nn;                        // nearest-neighbour-list construction
  };
  std::vector<Class> classes;
  // Autotuner: for each default class, the (G, H, ants per CTA) that measured
  // fastest on the first live set that contained the class.
  bool autotune = true;
  bool tuned_pending = false;
  std::map<std::tuple<int, int, int>, std::tuple<int, int, int, int>> tuned;
  int max_ld = 4;
  bool dirty = true;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
  bool unlimited = false;  // static batch: no iteration budget
  // Construction classes run concurrently on these streams (fork/join events
  // inside the captured step graph).
  static constexpr int kClassStreams = 8;
  cudaStream_t class_stream[kClassStreams] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kClassStreams] = {};
  // Completion of recent steps (ring; entry k % kStepEvents is recorded
  // after step k's graph), so a finished slot's result is read as soon as
  // its last step is done, on the io stream, while later steps run.  An
  // entry re-recorded by a later step only makes the wait longer, never
  // wrong: the steps run in order on one stream.
  bool single_launch = false;  // all classes in one construction launch
  int* d_ticket = nullptr;
  static constexpr int kStepEvents = 8;
  cudaEvent_t step_ev[kStepEvents] = {};
  long long steps_launched = 0;
  cudaStream_t io = nullptr;
};

static void pool_drop_graph(aco_pool* p) {
  if (p->exec) {
    cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
  }
}

static bool pool_alloc(aco_pool* p, size_t bytes, size_t* off) {
  for (auto it = p->free_blocks.begin(); it != p->free_blocks.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t noff = it->first + bytes;
      p->free_blocks.erase(it);
      if (rest) p->free_blocks[noff] = rest;
      p->in_use += bytes;
      return true;
    }
  }
  return false;
}

static void pool_free(aco_pool* p, size_t off, size_t bytes) {
  p->in_use -= bytes;
  auto it = p->free_blocks.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != p->free_blocks.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    p->free_blocks.erase(nx);
  }
  if (it != p->free_blocks.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      p->free_blocks.erase(it);
    }
  }
}

static int ensure_capacity(void** ptr, size_t* cap, size_t need, size_t elem) {
  if (need <= *cap) return ACO_OK;
  size_t ncap = std::max(need, *cap * 2 + 64);
  void* np = nullptr;
  cudaError_t e = cudaMalloc(&np, ncap * elem);
  if (e != cudaSuccess) return cuda_fail(e, "pool list");
  if (*ptr) cudaFree(*ptr);
  *ptr = np;
  *cap = ncap;
  return ACO_OK;
}

// Modelled time of one iteration of an instance of n cities run alone, in
// microseconds: n dependent steps, each costing a fixed latency plus the
// per-lane chunk (n / 32 cities); the Ant Colony System's lockstep step is
// about 4 us.  Only ratios matter (they set the iterations per step).
static double iteration_time_model(int n, bool acs, bool nn = false) {
  return acs ? 4.0 * n : nn ? 0.65 * n : n * (0.6 + 0.025 * n / 32.0);
}
constexpr int kMaxRate = 64;  // iterations per step at most

// Iterations per step for a group whose slowest instance takes t (model) in
// a step whose slowest group takes t_max, limited so that no slot of the
// group runs past its iteration budget.
static int group_rate(const aco_pool* p, const int* slots, int count, double t, double t_max) {
  if (!p->multirate) return 1;
  int k = (int)std::floor(t_max / t);
  k = std::max(1, std::min(k, kMaxRate));
  for (int i = 0; i < count; ++i) {
    const long long left = p->slots[(size_t)slots[i]].iters_left;
    if (left > 0 && left < k) k = (int)left;
  }
  return k;
}

// Rebuild the device work lists for the current live set.
static int pool_rebuild(aco_pool* p) {
  p->h_live.clear();
  p->h_acs.clear();
  p->h_cls_slots.clear();
  p->h_items.clear();
  p->h_rows.clear();
  p->classes.clear();
  p->max_ld = 4;
  p->acs_max_m = p->acs_max_n = 0;
  std::vector<int> live;
  for (int s = 0; s < p->max_slots; ++s)
    if (p->slots[(size_t)s].live) live.push_back(s);
  // longest instance first
  std::sort(live.begin(), live.end(), [&](int a, int b) {
    const int na = p->slots[(size_t)a].n, nb = p->slots[(size_t)b].n;
    return na != nb ? na > nb : a < b;
  });
  p->h_live = live;
  // Ant Colony System slots: one CTA per colony in one launch of their own
  // (MAX-MIN Ant System slots construct and update with the Ant System ones:
  // the best and row-update kernels follow each slot's rule)
  for (int pass = 0; pass < 2; ++pass) {
    for (int s : live) {
      const PoolSlot& sl = p->slots[(size_t)s];
      if (sl.I.variant != kVariantAcs || (sl.I.nn > 0) != (pass == 1)) continue;
      p->h_acs.push_back(s);
      p->acs_max_m = std::max(p->acs_max_m, sl.m);
      p->acs_max_n = std::max(p->acs_max_n, sl.n);
    }
    if (pass == 0) p->acs_dense = (int)p->h_acs.size();
  }
  // group the Ant System slots by tiling class, keeping the longest-first
  // order inside a class
  std::map<std::tuple<int, int, int>, std::vector<int>> by_class;
  std::vector<std::tuple<int, int, int>> class_order;
  for (int s : live) {
    if (p->slots[(size_t)s].I.variant == kVariantAcs) continue;
    const ConstructTiling t = batched_construct_tiling(p->slots[(size_t)s].n);
    // nearest-neighbour-list slots: one class of their own (key 0, 0, 0)
    const auto key = p->slots[(size_t)s].I.nn > 0 ? std::make_tuple(0, 0, 0)
                                                  : std::make_tuple(t.G, t.H, t.C);
    if (!by_class.count(key)) class_order.push_back(key);
    by_class[key].push_back(s);
  }
  for (const auto& key : class_order) {
    aco_pool::Class c;
    c.key = key;
    c.nn = key == std::make_tuple(0, 0, 0);
    c.max_n = 0;
    for (int s : by_class[key]) c.max_n = std::max(c.max_n, p->slots[(size_t)s].n);
    c.t = batched_construct_tiling(c.max_n);
    if (p->autotune && !c.nn) {
      auto it = p->tuned.find(key);
      if (it == p->tuned.end()) {
        p->tuned_pending = true;
      } else {
        ConstructTiling t = construct_tiling(c.max_n, std::get<0>(it->second),
                                             std::get<1>(it->second), std::get<2>(it->second));
        t.S = std::get<3>(it->second);
        if (t.C != 0) c.t = t;
      }
    }
    c.begin = (int)p->h_items.size();
    for (int s : by_class[key])
      for (int k = 0; k < p->slots[(size_t)s].m; ++k) p->h_items.push_back(make_int2(s, k));
    c.count = (int)p->h_items.size() - c.begin;
    c.slot_begin = (int)p->h_cls_slots.size();
    c.row_begin = (int)p->h_rows.size();
    c.max_ld = 4;
    for (int s : by_class[key]) {
      const PoolSlot& sl = p->slots[(size_t)s];
      p->h_cls_slots.push_back(s);
      c.max_ld = std::max(c.max_ld, sl.I.ld);
      for (int i = 0; i < sl.n; ++i) p->h_rows.push_back(make_int2(s, i));
    }
    c.slot_count = (int)p->h_cls_slots.size() - c.slot_begin;
    c.row_count = (int)p->h_rows.size() - c.row_begin;
    p->max_ld = std::max(p->max_ld, c.max_ld);
    c.k = 1;
    p->classes.push_back(c);
  }
  // iterations per step of each group (1 unless multi-rate stepping is on)
  double t_max = p->h_acs.empty() ? 0.0 : iteration_time_model(p->acs_max_n, true);
  for (const auto& c : p->classes)
    t_max = std::max(t_max, iteration_time_model(c.max_n, false, c.nn));
  for (auto& c : p->classes) {
    c.k = group_rate(p, p->h_cls_slots.data() + c.slot_begin, c.slot_count,
                     iteration_time_model(c.max_n, false, c.nn), t_max);
    for (int i = 0; i < c.slot_count; ++i)
      p->slots[(size_t)p->h_cls_slots[(size_t)(c.slot_begin + i)]].rate = c.k;
  }
  p->acs_k = p->h_acs.empty() ? 1
                              : group_rate(p, p->h_acs.data(), (int)p->h_acs.size(),
                                           iteration_time_model(p->acs_max_n, true), t_max);
  for (int s : p->h_acs) p->slots[(size_t)s].rate = p->acs_k;
  int rc = ensure_capacity((void**)&p->d_items, &p->items_cap, p->h_items.size(), sizeof(int2));
  if (!rc) rc = ensure_capacity((void**)&p->d_rows, &p->rows_cap, p->h_rows.size(), sizeof(int2));
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (!p->h_items.empty())
    e = cudaMemcpyAsync(p->d_items, p->h_items.data(), p->h_items.size() * sizeof(int2),
                        cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess && !p->h_rows.empty())
    e = cudaMemcpyAsync(p->d_rows, p->h_rows.data(), p->h_rows.size() * sizeof(int2),
                        cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess && !p->h_live.empty())
    e = cudaMemcpyAsync(p->d_live, p->h_live.data(), p->h_live.size() * sizeof(int),
                        cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess && !p->h_acs.empty())
    e = cudaMemcpyAsync(p->d_acs, p->h_acs.data(), p->h_acs.size() * sizeof(int),
                        cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess && !p->h_cls_slots.empty())
    e = cudaMemcpyAsync(p->d_cls_slots, p->h_cls_slots.data(), p->h_cls_slots.size() * sizeof(int),
                        cudaMemcpyHostToDevice, p->stream);
  // The host vectors must outlive the copies: synchronise before they change.
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "pool lists");
  pool_drop_graph(p);
  p->dirty = false;
  return ACO_OK;
}

// The autotuner.  For every class not tuned yet, each candidate tiling
// (whole warps with 1, 2 or 4 warps per ant; 8- or 16-lane segments) builds
// the class's tours twice on the pool stream and the second run is timed;
// the fastest is kept for the class from then on.  Every tiling builds the
// same tours (the selection is exact integer arithmetic), so the trial runs
// change nothing: the step that follows rebuilds the same tours.  A tiling
// with warp segments (several ants per warp) must beat the fastest
// whole-warp tiling by kSegmentMargin: timed alone a class gains from the
// segments' fewer instructions per ant more than it does in the step, where
// the other classes share the SMs (the n 897-1019 class of the batched
// workload: 16-lane segments 0.5 % faster alone, 2 % slower in the step).
static int pool_autotune(aco_pool* p) {
  // (warps per ant, lanes per ant, ants per CTA): CTA widths of 2-8 warps
  static const int kCand[][3] = {{1, 32, 4}, {1, 32, 2}, {1, 32, 8}, {2, 32, 2},
                                 {4, 32, 1}, {1, 16, 8}, {1, 8, 16}};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (auto& c : p->classes) {
    if (e != cudaSuccess) break;
    if (c.nn || p->tuned.count(c.key)) continue;
    constexpr float kSegmentMargin = 0.95f;
    float best_ms = 0.0f, warp_ms = 0.0f;
    int bi = -1, bw = -1;  // fastest overall, fastest with whole warps
    const ConstructTiling d = batched_construct_tiling(c.max_n);
    const int ncand = (int)(sizeof kCand / sizeof kCand[0]);
    for (int i = 0; i < 2 * ncand && e == cudaSuccess; ++i) {
      ConstructTiling t = construct_tiling(c.max_n, kCand[i % ncand][0], kCand[i % ncand][1],
                                           kCand[i % ncand][2]);
      t.S = i / ncand;  // row staging: bulk copy, then lane copies
      if (t.C == 0 || t.W < 1 || t.W > 8 || ants_per_cta(t) < 1) continue;
      // a tiling with more than twice the default's city slots per ant only
      // adds masked-off work: not worth a trial
      if (t.G * t.H * t.C > 2 * d.G * d.H * d.C) continue;
      float ms = 0.0f;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        if (rep == 1) e = cudaEventRecord(e0, p->stream);
        if (e == cudaSuccess)
          e = launch_construct_items(p->d_inst, p->d_items + c.begin, c.count, t, p->stream);
        if (e == cudaSuccess && rep == 1) e = cudaEventRecord(e1, p->stream);
      }
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && (bi < 0 || ms < best_ms)) {
        best_ms = ms;
        bi = i;
      }
      if (e == cudaSuccess && t.H == 32 && (bw < 0 || ms < warp_ms)) {
        warp_ms = ms;
        bw = i;
      }
    }
    if (bi >= 0 && bw >= 0 && kCand[bi % ncand][1] != 32 && best_ms > kSegmentMargin * warp_ms)
      bi = bw;
    if (e == cudaSuccess && bi >= 0) {
      const int* k = kCand[bi % ncand];
      p->tuned[c.key] = std::make_tuple(k[0], k[1], k[2], bi / ncand);
      c.t = construct_tiling(c.max_n, k[0], k[1], k[2]);
      c.t.S = bi / ncand;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  p->tuned_pending = false;
  if (e != cudaSuccess) return cuda_fail(e, "pool autotune");
  return ACO_OK;
}

// Order the pool stream after the setup of newly admitted instances.
static int pool_wait_ready(aco_pool* p) {
  for (int s : p->h_live) {
    PoolSlot& sl = p->slots[(size_t)s];
    if (sl.wait_ready) {
      const cudaError_t e = cudaStreamWaitEvent(p->stream, sl.ready, 0);
      if (e != cudaSuccess) return cuda_fail(e, "wait setup");
      sl.wait_ready = false;
    }
  }
  return ACO_OK;
}

static int pool_enqueue_step(aco_pool* p) {
  cudaError_t e;
  int launches = 0;
  // Fork: every tiling class, and the Ant Colony System colonies, get their
  // own stream so that the tail of one overlaps the others.  One iteration
  // per step: join before the best/update launches, which cover all slots.
  // Multi-rate: each group runs its k iterations (construct, best, update)
  // on its own stream, and the streams join at the end.
  const bool mr = p->multirate;
  const int ncls = (int)p->classes.size();
  const int nacs = (int)p->h_acs.size();
  const int nstreams = std::min(ncls + (nacs > 0 ? 1 : 0), (int)aco_pool::kClassStreams);
  if (nstreams > 1 && (e = cudaEventRecord(p->fork_ev, p->stream)) != cudaSuccess)
    return cuda_fail(e, "pool fork");
  for (int i = 0; i < nstreams && nstreams > 1; ++i)
    if ((e = cudaStreamWaitEvent(p->class_stream[i], p->fork_ev, 0)) != cudaSuccess)
      return cuda_fail(e, "pool fork wait");
  // The colonies (n lockstep steps each) go first, on the first stream.
  const int first = nacs > 0 ? 1 : 0;
  if (nacs > 0) {
    cudaStream_t st = nstreams > 1 ? p->class_stream[0] : p->stream;
    const int nd = p->acs_dense;
    for (int r = 0; r < (mr ? p->acs_k : 1); ++r) {
      e = launch_acs_construct_slots(p->d_inst, p->d_acs, nd, p->acs_max_m, p->acs_max_n, false,
                                     st);
      if (e == cudaSuccess)
        e = launch_acs_construct_slots(p->d_inst, p->d_acs + nd, nacs - nd, p->acs_max_m,
                                       p->acs_max_n, true, st);
      if (e != cudaSuccess) return cuda_fail(e, "pool acs construct");
      launches += (nd > 0 ? 1 : 0) + (nacs > nd ? 1 : 0);
      if (!mr) break;
      if ((e = launch_best_slots(p->d_inst, p->d_acs, nacs, st)) != cudaSuccess)
        return cuda_fail(e, "pool acs best");
      if ((e = launch_acs_global_slots(p->d_inst, p->d_acs, nacs, st)) != cudaSuccess)
        return cuda_fail(e, "pool acs update");
      launches += 2;
    }
  }
  // One launch for every class: only for plain classes (whole warps, one
  // iteration per step, no lists) of supported widths.
  bool single = p->single_launch && !mr && ncls > 0 && ncls <= 8;
  for (int ci = 0; single && ci < ncls; ++ci) {
    const auto& c = p->classes[(size_t)ci];
    single = !c.nn && std::get<0>(c.key) == 1 && std::get<1>(c.key) == 32 &&
             single_launch_supports(std::get<2>(c.key));
  }
  if (single) {
    SingleClasses sc{};
    std::vector<int> order((size_t)ncls);
    for (int ci = 0; ci < ncls; ++ci) order[(size_t)ci] = ci;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
      return std::get<2>(p->classes[(size_t)a].key) > std::get<2>(p->classes[(size_t)b].key);
    });
    int total = 0;
    for (int j = 0; j < ncls; ++j) {
      const auto& c = p->classes[(size_t)order[(size_t)j]];
      sc.begin[j] = c.begin;
      sc.count[j] = c.count;
      sc.C[j] = std::get<2>(c.key);
      sc.lane_copy[j] = c.t.S;
      total += c.count;
    }
    sc.n = ncls;
    cudaStream_t st = nstreams > 1 ? p->class_stream[first % nstreams] : p->stream;
    if ((e = launch_construct_single(p->d_inst, p->d_items, sc, total, p->d_ticket, p->sms, st)) !=
        cudaSuccess)
      return cuda_fail(e, "pool construct (one launch)");
    launches += 2;  // the ticket reset and the kernel
  }
  for (int ci = 0; ci < ncls && !single; ++ci) {
    const auto& c = p->classes[(size_t)ci];
    cudaStream_t st = nstreams > 1 ? p->class_stream[(ci + first) % nstreams] : p->stream;
    for (int r = 0; r < (mr ? c.k : 1); ++r) {
      e = c.nn ? launch_construct_nn_items(p->d_inst, p->d_items + c.begin, c.count, c.max_n, st)
               : launch_construct_items(p->d_inst, p->d_items + c.begin, c.count, c.t, st);
      if (e != cudaSuccess) return cuda_fail(e, "pool construct");
      ++launches;
      if (!mr) break;
      if ((e = launch_best_slots(p->d_inst, p->d_cls_slots + c.slot_begin, c.slot_count, st)) !=
          cudaSuccess)
        return cuda_fail(e, "pool best");
      if ((e = launch_update_rows(p->d_inst, p->d_rows + c.row_begin, c.row_count, c.max_ld,
                                  st)) != cudaSuccess)
        return cuda_fail(e, "pool update");
      launches += 2;
      if (c.nn) {
        if ((e = launch_nn_choice_slots(p->d_inst, p->d_cls_slots + c.slot_begin, c.slot_count,
                                        c.max_n, st)) != cudaSuccess)
          return cuda_fail(e, "pool nn choice");
        ++launches;
      }
    }
  }
  for (int i = 0; i < nstreams && nstreams > 1; ++i) {
    if ((e = cudaEventRecord(p->join_ev[i], p->class_stream[i])) != cudaSuccess)
      return cuda_fail(e, "pool join");
    if ((e = cudaStreamWaitEvent(p->stream, p->join_ev[i], 0)) != cudaSuccess)
      return cuda_fail(e, "pool join wait");
  }
  if (!mr) {
    if ((e = launch_best_slots(p->d_inst, p->d_live, (int)p->h_live.size(), p->stream)) !=
        cudaSuccess)
      return cuda_fail(e, "pool best");
    ++launches;
    if ((e = launch_update_rows(p->d_inst, p->d_rows, (int)p->h_rows.size(), p->max_ld,
                                p->stream)) != cudaSuccess)
      return cuda_fail(e, "pool update");
    launches += p->h_rows.empty() ? 0 : 1;
    if ((e = launch_acs_global_slots(p->d_inst, p->d_acs, nacs, p->stream)) != cudaSuccess)
      return cuda_fail(e, "pool acs update");
    launches += nacs > 0 ? 1 : 0;
    for (const auto& c : p->classes) {
      if (!c.nn) continue;
      if ((e = launch_nn_choice_slots(p->d_inst, p->d_cls_slots + c.slot_begin, c.slot_count,
                                      c.max_n, p->stream)) != cudaSuccess)
        return cuda_fail(e, "pool nn choice");
      ++launches;
    }
  }
  p->launches = launches;
  return ACO_OK;
}

static int pool_admit_common(aco_pool* p, int32_t n, const int32_t* dist, const int32_t* xy,
                             float alpha, float beta, float rho, int32_t m, uint64_t seed,
                             int32_t iterations, int32_t* slot) {
  NvtxRange nvtx_range("aco_pool_admit");
  if (!p || !slot) return fail(ACO_EINVAL, "NULL argument");
  if (!p->unlimited && iterations < 1) return fail(ACO_EINVAL, "iterations must be >= 1");
  int rc = dist ? validate_instance(n, dist, alpha, beta, rho, m)
                : validate_coords_public(n, xy);
  if (rc) return rc;
  if (!dist) {
    if (m < 1 || m > ACO_MAX_M) return fail(ACO_EINVAL, "m=%d outside [1, %d]", m, ACO_MAX_M);
    if (!std::isfinite(alpha) || alpha < 0.0f || !std::isfinite(beta) || beta < 0.0f)
      return fail(ACO_EINVAL, "alpha and beta must be finite and >= 0");
    if (!(rho > 0.0f && rho <= 1.0f)) return fail(ACO_EINVAL, "rho must lie in (0, 1]");
  }
  int s = -1;
  for (int i = 0; i < p->max_slots; ++i)
    if (!p->slots[(size_t)i].used) {
      s = i;
      break;
    }
  if (s < 0) return fail(ACO_EBUSY, "no free slot");
  const Layout L = layout_of(n, m);
  size_t off = 0;
  if (!pool_alloc(p, L.total, &off)) return fail(ACO_EBUSY, "HBM budget exhausted");
  PoolSlot& sl = p->slots[(size_t)s];
  const cudaEvent_t ev = sl.ready;
  sl = PoolSlot{};
  sl.ready = ev;
  sl.used = true;
  sl.n = n;
  sl.m = m;
  sl.iters_left = p->unlimited ? -1 : iterations;
  sl.off = off;
  sl.bytes = L.total;
  Instance& I = sl.I;
  I.n = n;
  I.m = m;
  I.ld = (n + 3) / 4 * 4;
  I.ldt = (n + 1 + 3) / 4 * 4;
  I.ldm = (m + 31) / 32 * 32;
  I.alpha = alpha;
  I.beta = beta;
  I.rho = rho;
  I.seed = seed;
  char* b = (char*)p->arena + off;
  I.dist = (const int32_t*)(b + L.dist);
  I.heta = (float*)(b + L.heta);
  I.tau = (float*)(b + L.tau);
  I.choice = (float*)(b + L.choice);
  I.tours = (int32_t*)(b + L.tours);
  I.lens = (long long*)(b + L.lens);
  I.nbr = (uint32_t*)(b + L.nbr);
  I.q = (unsigned long long*)(b + L.q);
  I.delta = (float*)(b + L.delta);
  I.acc = nullptr;
  I.best_tour = (int32_t*)(b + L.best);
  I.dep_nb = (uint32_t*)(b + L.dep_nb);
  I.nnlist = (int32_t*)(b + L.nnlist);
  I.nnchoice = (float*)(b + L.nnchoice);
  I.nn = 0;
  I.st = (IterState*)(b + L.st);
  cudaError_t e = cudaSuccess;
  // Sources of the asynchronous copies below must outlive this call: the
  // initial state is a static constant and the descriptor lives in the slot.
  static const IterState st0 = [] {
    IterState z{};
    z.best_len = INT64_MAX;
    return z;
  }();
  do {
    if (!sl.ready && (e = cudaEventCreateWithFlags(&sl.ready, cudaEventDisableTiming)) != cudaSuccess)
      break;
    if ((e = cudaMemsetAsync(b, 0, L.total, p->side)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(I.st, &st0, sizeof st0, cudaMemcpyHostToDevice, p->side)) !=
        cudaSuccess)
      break;
    if (dist) {
      e = cudaMemcpy2DAsync((void*)I.dist, (size_t)I.ld * 4, dist, (size_t)n * 4, (size_t)n * 4,
                            (size_t)n, cudaMemcpyHostToDevice, p->side);
    } else {
      // stage the coordinates in the (not yet used) choice_info block
      e = cudaMemcpyAsync(I.choice, xy, (size_t)n * 8, cudaMemcpyHostToDevice, p->side);
      if (e == cudaSuccess) e = launch_dist_from_coords(I, (const int32_t*)I.choice, p->side);
    }
    if (e != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(p->d_inst + s, &sl.I, sizeof sl.I, cudaMemcpyHostToDevice,
                             p->side)) != cudaSuccess)
      break;
    if ((e = launch_setup(I, p->sms, p->side)) != cudaSuccess) break;
    e = cudaEventRecord(sl.ready, p->side);
  } while (0);
  if (e != cudaSuccess) {
    pool_free(p, off, L.total);
    sl.used = false;
    return cuda_fail(e, "pool admit");
  }
  sl.live = true;
  sl.wait_ready = true;
  p->dirty = true;
  *slot = s;
  return ACO_OK;
}

static int pool_check_status(aco_pool* p, int slot, cudaStream_t st = nullptr) {
  if (!st) st = p->stream;
  int status = 0;
  cudaError_t e = cudaMemcpyAsync(&status, &p->slots[(size_t)slot].I.st->status, sizeof(int),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "pool synchronize");
  if (status & kStatusTimeout) return fail(ACO_ETIMEOUT, "a device-side wait gave up");
  if (status) return fail(ACO_ECUDA, "device status 0x%x in slot %d", status, slot);
  return ACO_OK;
}

// Switch a slot admitted but not yet stepped to another update rule: the
// descriptor is uploaded again and the rule's start trails written, both on
// the side stream after the admission's setup.
template <class Apply>
static int pool_switch_rule(aco_pool* p, int32_t slot, Apply apply) {
  PoolSlot& sl = p->slots[(size_t)slot];
  apply(sl.I);
  Instance& I = sl.I;
  cudaError_t e = cudaMemcpyAsync(p->d_inst + slot, &I, sizeof I, cudaMemcpyHostToDevice, p->side);
  if (e == cudaSuccess)
    e = I.variant == kVariantAcs ? launch_acs_init(I, p->sms, p->side)
                                 : launch_mmas_init(I, p->sms, p->side);
  // A slot that already has nearest-neighbour lists builds its first tours
  // from the list-ordered copy of choice_info: refresh it from the new rule's
  // start trails (the Ant Colony System reads the dense row instead).
  if (e == cudaSuccess && I.nn > 0 && I.variant != kVariantAcs) e = launch_nn_choice(I, p->side);
  if (e == cudaSuccess) e = cudaEventRecord(sl.ready, p->side);
  if (e != cudaSuccess) return cuda_fail(e, "pool rule switch");
  sl.wait_ready = true;
  p->dirty = true;
  return ACO_OK;
}

static int pool_rule_slot_check(aco_pool* p, int32_t slot) {
  if (!p) return fail(ACO_EINVAL, "NULL pool");
  if (slot < 0 || slot >= p->max_slots || !p->slots[(size_t)slot].live)
    return fail(ACO_EINVAL, "slot %d is not live", slot);
  const PoolSlot& sl = p->slots[(size_t)slot];
  if (sl.started || sl.restored || sl.I.variant != kVariantAs)
    return fail(ACO_ESTATE, "the update rule is chosen once, before the slot's first step");
  return ACO_OK;
}

extern "C" {

int aco_pool_bytes_needed(int32_t n, int32_t m, uint64_t* bytes) {
  if (!bytes) return fail(ACO_EINVAL, "NULL argument");
  if (n < 3 || n > ACO_MAX_N || m < 1 || m > ACO_MAX_M) return fail(ACO_EINVAL, "n or m out of range");
  *bytes = layout_of(n, m).total;
  return ACO_OK;
}

int aco_pool_create(int32_t max_slots, uint64_t budget_bytes, aco_pool_handle* out) {
  if (!out) return fail(ACO_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_slots < 1 || max_slots > (1 << 20)) return fail(ACO_EINVAL, "max_slots out of range");
  if (budget_bytes < 4096) return fail(ACO_EINVAL, "budget too small");
  aco_pool* p = new (std::nothrow) aco_pool();
  if (!p) return fail(ACO_ENOMEM, "host allocation");
  p->max_slots = max_slots;
  p->budget = align256(budget_bytes);
  p->slots.resize((size_t)max_slots);
  p->sms = device_sms();
  cudaError_t e;
  do {
    if ((e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaMalloc(&p->arena, p->budget)) != cudaSuccess) break;
    if ((e = cudaMalloc(&p->d_inst, sizeof(Instance) * (size_t)max_slots)) != cudaSuccess) break;
    if ((e = cudaMalloc(&p->d_live, sizeof(int) * (size_t)max_slots)) != cudaSuccess) break;
    if ((e = cudaMalloc(&p->d_acs, sizeof(int) * (size_t)max_slots)) != cudaSuccess) break;
    if ((e = cudaMalloc(&p->d_cls_slots, sizeof(int) * (size_t)max_slots)) != cudaSuccess) break;
    if ((e = cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming)) != cudaSuccess) break;
    if ((e = cudaStreamCreateWithFlags(&p->io, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaMalloc(&p->d_ticket, sizeof(int))) != cudaSuccess) break;
    for (int i = 0; i < aco_pool::kStepEvents && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&p->step_ev[i], cudaEventDisableTiming);
    for (int i = 0; i < aco_pool::kClassStreams && e == cudaSuccess; ++i) {
      e = cudaStreamCreateWithFlags(&p->class_stream[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->join_ev[i], cudaEventDisableTiming);
    }
  } while (0);
  if (e != cudaSuccess) {
    const int rc = cuda_fail(e, "pool create");
    aco_pool_destroy(p);
    return rc;
  }
  p->free_blocks[0] = p->budget;
  *out = p;
  return ACO_OK;
}

int aco_pool_destroy(aco_pool_handle p) {
  if (!p) return ACO_OK;
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->side) cudaStreamSynchronize(p->side);
  pool_drop_graph(p);
  for (auto& s : p->slots)
    if (s.ready) cudaEventDestroy(s.ready);
  if (p->arena) cudaFree(p->arena);
  if (p->d_inst) cudaFree(p->d_inst);
  if (p->d_live) cudaFree(p->d_live);
  if (p->d_acs) cudaFree(p->d_acs);
  if (p->d_cls_slots) cudaFree(p->d_cls_slots);
  if (p->d_ticket) cudaFree(p->d_ticket);
  if (p->d_items) cudaFree(p->d_items);
  if (p->d_rows) cudaFree(p->d_rows);
  for (int i = 0; i < aco_pool::kClassStreams; ++i) {
    if (p->class_stream[i]) {
      cudaStreamSynchronize(p->class_stream[i]);
      cudaStreamDestroy(p->class_stream[i]);
    }
    if (p->join_ev[i]) cudaEventDestroy(p->join_ev[i]);
  }
  if (p->fork_ev) cudaEventDestroy(p->fork_ev);
  for (int i = 0; i < aco_pool::kStepEvents; ++i)
    if (p->step_ev[i]) cudaEventDestroy(p->step_ev[i]);
  if (p->io) {
    cudaStreamSynchronize(p->io);
    cudaStreamDestroy(p->io);
  }
  if (p->stream) cudaStreamDestroy(p->stream);
  if (p->side) cudaStreamDestroy(p->side);
  delete p;
  return ACO_OK;
}

int aco_pool_admit(aco_pool_handle p, int32_t n, const int32_t* dist, float alpha, float beta,
                   float rho, int32_t m, uint64_t seed, int32_t iterations, int32_t* slot) {
  if (!dist) return fail(ACO_EINVAL, "dist is NULL");
  return pool_admit_common(p, n, dist, nullptr, alpha, beta, rho, m, seed, iterations, slot);
}

int aco_pool_admit_coords(aco_pool_handle p, int32_t n, const int32_t* xy, float alpha,
                          float beta, float rho, int32_t m, uint64_t seed, int32_t iterations,
                          int32_t* slot) {
  if (!xy) return fail(ACO_EINVAL, "xy is NULL");
  return pool_admit_common(p, n, nullptr, xy, alpha, beta, rho, m, seed, iterations, slot);
}

int aco_pool_set_acs(aco_pool_handle p, int32_t slot, double q0, float xi) {
  int rc = pool_rule_slot_check(p, slot);
  if (rc) return rc;
  if (!(q0 >= 0.0 && q0 <= 1.0)) return fail(ACO_EINVAL, "q0 must lie in [0, 1]");
  if (!(xi >= 0.0f && xi <= 1.0f)) return fail(ACO_EINVAL, "xi must lie in [0, 1]");
  const int m = p->slots[(size_t)slot].m;
  if (m > kAcsMaxAnts)
    return fail(ACO_EINVAL, "the Ant Colony System runs at most %d ants (m=%d)", kAcsMaxAnts, m);
  return pool_switch_rule(p, slot, [&](Instance& I) {
    I.variant = kVariantAcs;
    I.acs_threshold = acs_threshold_of(q0);
    I.acs_xi = xi;
  });
}

int aco_pool_set_mmas(aco_pool_handle p, int32_t slot, double p_best, int32_t best_so_far) {
  int rc = pool_rule_slot_check(p, slot);
  if (rc) return rc;
  if (!(p_best > 0.0 && p_best < 1.0)) return fail(ACO_EINVAL, "p_best must lie in (0, 1)");
  if (best_so_far != 0 && best_so_far != 1) return fail(ACO_EINVAL, "best_so_far must be 0 or 1");
  return pool_switch_rule(p, slot, [&](Instance& I) {
    I.variant = kVariantMmas;
    I.mmas_f = mmas_f_of(I.n, p_best);
    I.mmas_best_so_far = best_so_far;
  });
}

int aco_pool_step(aco_pool_handle p, int32_t* live_after) {
  NvtxRange nvtx_range("aco_pool_step");
  if (!p) return fail(ACO_EINVAL, "NULL pool");
  int rc;
  if (p->dirty && (rc = pool_rebuild(p)) != ACO_OK) return rc;
  cudaError_t e;
  if (!p->h_live.empty()) {
    if ((rc = pool_wait_ready(p)) != ACO_OK) return rc;
    if (p->tuned_pending && (rc = pool_autotune(p)) != ACO_OK) return rc;
    if (!p->exec) {
      cudaGraph_t g = nullptr;
      if ((e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "pool capture");
      rc = pool_enqueue_step(p);
      e = cudaStreamEndCapture(p->stream, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (e != cudaSuccess) return cuda_fail(e, "pool end capture");
      e = cudaGraphInstantiate(&p->exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        p->exec = nullptr;
        return cuda_fail(e, "pool instantiate");
      }
    }
    if ((e = cudaGraphLaunch(p->exec, p->stream)) != cudaSuccess) return cuda_fail(e, "pool launch");
    const long long step = p->steps_launched++;
    if ((e = cudaEventRecord(p->step_ev[step % aco_pool::kStepEvents], p->stream)) != cudaSuccess)
      return cuda_fail(e, "pool step event");
    for (int s : p->h_live) {
      PoolSlot& sl = p->slots[(size_t)s];
      sl.started = true;
      if (sl.iters_left > 0) {
        sl.iters_left -= sl.rate;  // rate <= iters_left by construction
        if (sl.iters_left == 0) {
          sl.live = false;
          sl.finished = true;
          sl.finish_step = step;
          p->finished_order.push_back(s);
          p->dirty = true;
        } else if (sl.iters_left < sl.rate) {
          p->dirty = true;  // the group's rate must shrink to the budget left
        }
      }
    }
  } else {
    p->launches = 0;
  }
  if (live_after) {
    int live = 0;
    for (const auto& sl : p->slots) live += sl.live ? 1 : 0;
    *live_after = live;
  }
  return ACO_OK;
}

int aco_pool_set_single_launch(aco_pool_handle p, int32_t on) {
  if (!p) return fail(ACO_EINVAL, "NULL pool");
  if (on != 0 && on != 1) return fail(ACO_EINVAL, "on must be 0 or 1");
  p->single_launch = on != 0;
  p->dirty = true;
  return ACO_OK;
}

int aco_pool_finished(aco_pool_handle p, int32_t* slots, int32_t capacity, int32_t* count) {
  if (!p || !count) return fail(ACO_EINVAL, "NULL argument");
  const int total = (int)p->finished_order.size();
  for (int i = 0; i < total && i < capacity && slots; ++i) slots[i] = p->finished_order[(size_t)i];
  *count = total;
  return ACO_OK;
}

int aco_pool_result(aco_pool_handle p, int32_t slot, int32_t* tour, int64_t* len) {
  if (!p) return fail(ACO_EINVAL, "NULL pool");
  if (slot < 0 || slot >= p->max_slots || !p->slots[(size_t)slot].used)
    return fail(ACO_EINVAL, "slot %d is not in use", slot);
  const PoolSlot& sl = p->slots[(size_t)slot];
  if (sl.finished && sl.finish_step >= 0) {
    // Its last step is known: wait for that step only and read on the io
    // stream, without waiting for the steps launched since.
    cudaError_t e = cudaStreamWaitEvent(
        p->io, p->step_ev[sl.finish_step % aco_pool::kStepEvents], 0);
    if (e == cudaSuccess && tour)
      e = cudaMemcpyAsync(tour, sl.I.best_tour, ((size_t)sl.n + 1) * 4, cudaMemcpyDeviceToHost,
                          p->io);
    if (e == cudaSuccess && len)
      e = cudaMemcpyAsync(len, &sl.I.st->best_len, 8, cudaMemcpyDeviceToHost, p->io);
    if (e != cudaSuccess) return cuda_fail(e, "pool result");
    return pool_check_status(p, slot, p->io);
  }
  cudaError_t e = cudaStreamSynchronize(p->side);
  if (e == cudaSuccess && tour)
    e = cudaMemcpyAsync(tour, sl.I.best_tour, ((size_t)sl.n + 1) * 4, cudaMemcpyDeviceToHost,
                        p->stream);
  if (e == cudaSuccess && len)
    e = cudaMemcpyAsync(len, &sl.I.st->best_len, 8, cudaMemcpyDeviceToHost, p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "pool result");
  return pool_check_status(p, slot);
}

int aco_pool_set_nn(aco_pool_handle p, int32_t slot, int32_t nn) {
  NvtxRange nvtx_range("aco_pool_set_nn");
  if (!p) return fail(ACO_EINVAL, "NULL pool");
  if (slot < 0 || slot >= p->max_slots || !p->slots[(size_t)slot].live)
    return fail(ACO_EINVAL, "slot %d is not live", slot);
  PoolSlot& sl = p->slots[(size_t)slot];
  if (sl.started) return fail(ACO_ESTATE, "lists are chosen before the slot's first step");
  const int most = std::min(sl.n - 1, kNnStride);
  if (nn < 0 || nn > most)
    return fail(ACO_EINVAL, "nearest-neighbour list length must be in [0, %d]", most);
  Instance& I = sl.I;
  cudaError_t e = cudaSuccess;
  // on the side stream after the admission's setup (and any rule switch)
  if (nn > 0 && !sl.nn_built) e = launch_nn_lists(I, most, p->side);
  I.nn = nn;
  if (e == cudaSuccess && nn > 0) e = launch_nn_choice(I, p->side);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_inst + slot, &I, sizeof I, cudaMemcpyHostToDevice, p->side);
  if (e == cudaSuccess) e = cudaEventRecord(sl.ready, p->side);
  if (e != cudaSuccess) return cuda_fail(e, "pool set nn");
  if (nn > 0) sl.nn_built = true;
  sl.wait_ready = true;
  p->dirty = true;
  return ACO_OK;
}

int aco_pool_save_slot(aco_pool_handle p, int32_t slot, void* buf, uint64_t capacity,
                       uint64_t* size) {
  NvtxRange nvtx_range("aco_pool_save_slot");
  if (!p || !size) return fail(ACO_EINVAL, "NULL argument");
  if (slot < 0 || slot >= p->max_slots || !p->slots[(size_t)slot].used)
    return fail(ACO_EINVAL, "slot %d is not in use", slot);
  const PoolSlot& sl = p->slots[(size_t)slot];
  const int n = sl.n;
  *size = checkpoint_bytes(n);
  if (!buf) return ACO_OK;
  if (capacity < *size) return fail(ACO_EINVAL, "buffer holds %llu bytes, %llu needed",
                                    (unsigned long long)capacity, (unsigned long long)*size);
  char* b = static_cast<char*>(buf);
  char* stp = b + sizeof(CheckpointHeader);
  float* tau = reinterpret_cast<float*>(stp + sizeof(IterState));
  int32_t* best = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(tau) + (size_t)n * n * 4);
  // the slot's steps and setup first
  cudaError_t e = cudaStreamSynchronize(p->side);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(stp, sl.I.st, sizeof(IterState), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(tau, (size_t)n * 4, sl.I.tau, (size_t)sl.I.ld * 4, (size_t)n * 4,
                          (size_t)n, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(best, sl.I.best_tour, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost,
                        p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "pool save slot");
  IterState st{};
  std::memcpy(&st, stp, sizeof st);
  if (st.status & kStatusTimeout) return fail(ACO_ETIMEOUT, "a device-side wait gave up");
  if (st.status) return fail(ACO_ECUDA, "device status 0x%x in slot %d", st.status, slot);
  CheckpointHeader hd = checkpoint_header(sl.I);
  hd.constructed = st.iteration > 0 ? 1 : 0;
  hd.host_iteration = (long long)st.iteration;
  std::memcpy(b, &hd, sizeof hd);
  return ACO_OK;
}

int aco_pool_restore_slot(aco_pool_handle p, int32_t slot, const void* buf, uint64_t size) {
  NvtxRange nvtx_range("aco_pool_restore_slot");
  if (!p || !buf) return fail(ACO_EINVAL, "NULL argument");
  if (slot < 0 || slot >= p->max_slots || !p->slots[(size_t)slot].live)
    return fail(ACO_EINVAL, "slot %d is not live", slot);
  PoolSlot& sl = p->slots[(size_t)slot];
  if (sl.started || sl.restored)
    return fail(ACO_ESTATE, "a slot takes a checkpoint once, before its first step");
  CheckpointHeader hd{};
  IterState st{};
  const float* tau = nullptr;
  const int32_t* best = nullptr;
  int rc = checkpoint_parse(sl.I, buf, size, hd, st, tau, best);
  if (rc) return rc;
  if (hd.variant == kVariantAcs && sl.m > kAcsMaxAnts)
    return fail(ACO_EINVAL, "the Ant Colony System runs at most %d ants", kAcsMaxAnts);
  Instance& I = sl.I;
  I.variant = hd.variant;
  I.mmas_best_so_far = hd.mmas_best_so_far;
  I.mmas_f = hd.mmas_f;
  I.acs_threshold = hd.acs_threshold;
  I.acs_xi = hd.acs_xi;
  const int n = I.n;
  // On the side stream after the admission's setup: the state, tau and best
  // tour, the descriptor with the rule, then choice_info from tau.  The
  // sources are the caller's buffer and locals: synchronise before returning.
  cudaError_t e = cudaMemcpyAsync(I.st, &st, sizeof st, cudaMemcpyHostToDevice, p->side);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(I.tau, (size_t)I.ld * 4, tau, (size_t)n * 4, (size_t)n * 4, (size_t)n,
                          cudaMemcpyHostToDevice, p->side);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(I.best_tour, best, ((size_t)n + 1) * 4, cudaMemcpyHostToDevice, p->side);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_inst + slot, &I, sizeof I, cudaMemcpyHostToDevice, p->side);
  if (e == cudaSuccess) e = launch_choice(I, p->sms, p->side);
  if (e == cudaSuccess && I.nn > 0) e = launch_nn_choice(I, p->side);
  if (e == cudaSuccess) e = cudaEventRecord(sl.ready, p->side);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->side);
  if (e != cudaSuccess) return cuda_fail(e, "pool restore slot");
  sl.restored = true;
  sl.wait_ready = true;
  p->dirty = true;
  return ACO_OK;
}

int aco_pool_set_multirate(aco_pool_handle p, int32_t on) {
  if (!p) return fail(ACO_EINVAL, "NULL pool");
  if (on != 0 && on != 1) return fail(ACO_EINVAL, "on must be 0 or 1");
  if (on && p->unlimited)
    return fail(ACO_EINVAL, "a static batch steps one iteration per aco_batch_iterate step");
  if (p->multirate != (on != 0)) {
    p->multirate = on != 0;
    p->dirty = true;
  }
  return ACO_OK;
}

int aco_pool_rate(aco_pool_handle p, int32_t slot, int32_t* iterations_per_step) {
  if (!p || !iterations_per_step) return fail(ACO_EINVAL, "NULL argument");
  if (slot < 0 || slot >= p->max_slots || !p->slots[(size_t)slot].used)
    return fail(ACO_EINVAL, "slot %d is not in use", slot);
  if (!p->slots[(size_t)slot].started)
    return fail(ACO_ESTATE, "slot %d has not taken part in a step yet", slot);
  *iterations_per_step = p->slots[(size_t)slot].rate;
  return ACO_OK;
}

int aco_pool_set_autotune(aco_pool_handle p, int32_t on) {
  if (!p) return fail(ACO_EINVAL, "NULL pool");
  if (on != 0 && on != 1) return fail(ACO_EINVAL, "on must be 0 or 1");
  p->autotune = on != 0;
  if (!p->autotune) p->tuned.clear();
  p->dirty = true;
  return ACO_OK;
}

int aco_pool_autotune(aco_pool_handle p) {
  NvtxRange nvtx_range("aco_pool_autotune");
  if (!p) return fail(ACO_EINVAL, "NULL pool");
  int rc;
  if (p->dirty && (rc = pool_rebuild(p)) != ACO_OK) return rc;
  if (p->h_live.empty() || !p->tuned_pending) return ACO_OK;
  if ((rc = pool_wait_ready(p)) != ACO_OK) return rc;
  if ((rc = pool_autotune(p)) != ACO_OK) return rc;
  pool_drop_graph(p);
  return ACO_OK;
}

int aco_pool_get_tuning(aco_pool_handle p, int32_t* entries, int32_t capacity, int32_t* count) {
  if (!p || !count) return fail(ACO_EINVAL, "NULL argument");
  *count = (int32_t)p->tuned.size();
  if (!entries) return ACO_OK;
  int i = 0;
  for (const auto& kv : p->tuned) {
    if (i >= capacity) break;
    int32_t* e = entries + 7 * i;
    e[0] = std::get<0>(kv.first);
    e[1] = std::get<1>(kv.first);
    e[2] = std::get<2>(kv.first);
    e[3] = std::get<0>(kv.second);
    e[4] = std::get<1>(kv.second);
    e[5] = std::get<2>(kv.second);
    e[6] = std::get<3>(kv.second);
    ++i;
  }
  return ACO_OK;
}

int aco_pool_set_tuning(aco_pool_handle p, const int32_t* entries, int32_t count) {
  if (!p || (count > 0 && !entries)) return fail(ACO_EINVAL, "NULL argument");
  if (count < 0) return fail(ACO_EINVAL, "count < 0");
  std::map<std::tuple<int, int, int>, std::tuple<int, int, int, int>> table;
  for (int i = 0; i < count; ++i) {
    const int32_t* e = entries + 7 * i;
    // the class key must be a supported (G, H, C) and the choice a supported
    // (G, H, ants per CTA, staging)
    const bool key_ok = construct_supported(e[2], e[0], e[1]);
    const ConstructTiling t = construct_tiling(1, e[3], e[4], e[5]);
    const bool choice_ok = t.C != 0 && t.W >= 1 && t.W <= 8 && ants_per_cta(t) >= 1 &&
                           (e[4] == 32 || e[3] == 1) && (e[6] == 0 || e[6] == 1);
    if (!key_ok || !choice_ok)
      return fail(ACO_EINVAL, "tuning entry %d is not a supported tiling", i);
    table[std::make_tuple(e[0], e[1], e[2])] = std::make_tuple(e[3], e[4], e[5], e[6]);
  }
  p->tuned = table;
  p->autotune = true;
  p->dirty = true;
  return ACO_OK;
}

int aco_pool_tiling(aco_pool_handle p, int32_t slot, int32_t* warps_per_ant,
                    int32_t* lanes_per_ant, int32_t* cities_per_lane, int32_t* staging) {
  if (!p) return fail(ACO_EINVAL, "NULL pool");
  if (slot < 0 || slot >= p->max_slots || !p->slots[(size_t)slot].live)
    return fail(ACO_EINVAL, "slot %d is not live", slot);
  if (p->dirty) return fail(ACO_ESTATE, "no step has run since the live set changed");
  if (p->slots[(size_t)slot].I.variant == kVariantAcs)
    return fail(ACO_EINVAL, "slot %d runs the Ant Colony System (one CTA per colony)", slot);
  if (p->slots[(size_t)slot].I.nn > 0)
    return fail(ACO_EINVAL, "slot %d constructs with nearest-neighbour lists (one warp per ant)",
                slot);
  const int n = p->slots[(size_t)slot].n;
  for (const auto& c : p->classes)
    if (c.key == std::make_tuple(batched_construct_tiling(n).G, batched_construct_tiling(n).H,
                                 batched_construct_tiling(n).C)) {
      if (warps_per_ant) *warps_per_ant = c.t.G;
      if (lanes_per_ant) *lanes_per_ant = c.t.H;
      if (cities_per_lane) *cities_per_lane = c.t.C;
      if (staging) *staging = c.t.S;
      return ACO_OK;
    }
  return fail(ACO_ESTATE, "slot %d has no class", slot);
}

int aco_pool_pheromone(aco_pool_handle p, int32_t slot, float* tau) {
  if (!p || !tau) return fail(ACO_EINVAL, "NULL argument");
  if (slot < 0 || slot >= p->max_slots || !p->slots[(size_t)slot].used)
    return fail(ACO_EINVAL, "slot %d is not in use", slot);
  const PoolSlot& sl = p->slots[(size_t)slot];
  cudaError_t e = cudaStreamSynchronize(p->side);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(tau, (size_t)sl.n * 4, sl.I.tau, (size_t)sl.I.ld * 4, (size_t)sl.n * 4,
                          (size_t)sl.n, cudaMemcpyDeviceToHost, p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "pool pheromone");
  return pool_check_status(p, slot);
}

int aco_pool_release(aco_pool_handle p, int32_t slot) {
  if (!p) return fail(ACO_EINVAL, "NULL pool");
  if (slot < 0 || slot >= p->max_slots || !p->slots[(size_t)slot].used)
    return fail(ACO_EINVAL, "slot %d is not in use", slot);
  // Work that still reads the slot must finish before its memory is reused.
  // A finished slot is read by no step after its last one (its class lists
  // are rebuilt without it), so waiting for that step is enough; other slots
  // wait for everything in flight.
  PoolSlot& sl = p->slots[(size_t)slot];
  cudaError_t e;
  if (sl.finished && sl.finish_step >= 0) {
    e = cudaEventSynchronize(p->step_ev[sl.finish_step % aco_pool::kStepEvents]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->io);
  } else {
    e = cudaStreamSynchronize(p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->side);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->io);
  }
  if (e != cudaSuccess) return cuda_fail(e, "pool release");
  if (sl.live) p->dirty = true;
  pool_free(p, sl.off, sl.bytes);
  cudaEvent_t ev = sl.ready;
  sl = PoolSlot{};
  sl.ready = ev;
  auto& fo = p->finished_order;
  fo.erase(std::remove(fo.begin(), fo.end(), slot), fo.end());
  return ACO_OK;
}

int aco_pool_stats(aco_pool_handle p, int32_t* live, int32_t* finished, uint64_t* bytes_in_use,
                   int32_t* launches_last_step) {
  if (!p) return fail(ACO_EINVAL, "NULL pool");
  int l = 0;
  for (const auto& sl : p->slots) l += sl.live ? 1 : 0;
  if (live) *live = l;
  if (finished) *finished = (int32_t)p->finished_order.size();
  if (bytes_in_use) *bytes_in_use = p->in_use;
  if (launches_last_step) *launches_last_step = p->launches;
  return ACO_OK;
}

int aco_pool_synchronize(aco_pool_handle p) {
  if (!p) return fail(ACO_EINVAL, "NULL pool");
  cudaError_t e = cudaStreamSynchronize(p->side);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(e, "pool synchronize");
  for (int s = 0; s < p->max_slots; ++s)
    if (p->slots[(size_t)s].used) {
      const int rc = pool_check_status(p, s);
      if (rc) return rc;
    }
  return ACO_OK;
}

int aco_batch_create(int32_t count, const int32_t* ns, const int32_t* const* dists,
                     const float* alpha, const float* beta, const float* rho, const int32_t* ms,
                     const uint64_t* seeds, aco_batch* out) {
  if (!out) return fail(ACO_EINVAL, "out is NULL");
  *out = nullptr;
  if (count < 1 || !ns || !dists || !alpha || !beta || !rho || !ms || !seeds)
    return fail(ACO_EINVAL, "bad batch arguments");
  uint64_t total = 0;
  for (int i = 0; i < count; ++i) {
    uint64_t b = 0;
    const int rc = aco_pool_bytes_needed(ns[i], ms[i], &b);
    if (rc) return rc;
    total += b;
  }
  aco_pool* p = nullptr;
  int rc = aco_pool_create(count, total, &p);
  if (rc) return rc;
  p->unlimited = true;
  for (int i = 0; i < count; ++i) {
    int32_t slot = -1;
    rc = aco_pool_admit(p, ns[i], dists[i], alpha[i], beta[i], rho[i], ms[i], seeds[i], 1, &slot);
    if (rc) {
      aco_pool_destroy(p);
      return rc;
    }
  }
  *out = p;
  return ACO_OK;
}

int aco_batch_iterate(aco_batch b, int32_t iterations) {
  if (!b) return fail(ACO_EINVAL, "NULL batch");
  if (iterations < 0) return fail(ACO_EINVAL, "iterations < 0");
  for (int i = 0; i < iterations; ++i) {
    const int rc = aco_pool_step(b, nullptr);
    if (rc) return rc;
  }
  return ACO_OK;
}

int aco_batch_best(aco_batch b, int32_t idx, int32_t* tour, int64_t* len) {
  return aco_pool_result(b, idx, tour, len);
}

int aco_batch_destroy(aco_batch b) { return aco_pool_destroy(b); }

}  // extern "C"
