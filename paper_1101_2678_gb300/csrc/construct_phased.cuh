// Tour construction by Eq. 1 (Section II; the integer roulette of reading R2)
// for one warp, one warp segment or two warps per ant, with the unvisited
// cities compacted up to three times along the walk.
//
// A step of the plain kernel (construct_ant) handles every city of the row,
// visited or not: lane t owns the cities [tC, tC + C), zeroes the visited
// ones and still pays the max, the quantisation and the sum for them.  Half
// way through a tour half of that work is spent on visited cities.  Here the
// walk runs in up to four phases:
//   phase 0  (at most 32*C1 unvisited cities not yet reached): as the plain
//            kernel, lane t owns the contiguous chunk [tC, tC + C) of the row;
//   phase 1  the unvisited cities, in ascending order, are listed in shared
//            memory and dealt out C1 = 4*ceil(C/8) per lane (lane t takes
//            entries [t*C1, t*C1 + C1)); each step reads the entries and
//            then their weights from the staged row through them.  A visited
//            slot's entry is pointed at a float beside the row that stays 0,
//            so these phases keep no tabu bits and mask nothing (entries are
//            byte offsets for a single instance, city indices in pools);
//   phase 2  the same with C2 = 4*ceil(C/16) per lane;
//   phase 3  the same with C3 = 4*ceil(C/32) per lane (when smaller than C2).
// Phase p starts at the first step at which the unvisited cities fit in the
// segment's H*Cp slots.  Every phase keeps the cities of the segment in
// ascending order, lane after lane and slot after slot, so the integer
// roulette (first city whose inclusive prefix sum exceeds T) chooses the same
// city as the plain kernel and the CPU oracle.  With two warps per ant the
// group's 64 threads hold the slots in that order, warp 0 first; the warps
// combine their maxima and totals through shared memory, and the warp whose
// range holds the target runs the second-level search.  The row is still staged
// whole (bulk copy), so the L2 bytes do not change; the per-candidate work
// of the later steps halves, quarters and eighths.
#pragma once

namespace aco {

// The weight bits a list entry points at: entry = city * kUnit (kUnit 1: a
// city index; 4: a byte offset into the staged row).
template <uint32_t kUnit>
__device__ __forceinline__ uint32_t entry_weight(const float* row, uint32_t e) {
  if constexpr (kUnit == 4u)
    return *reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(row) + e);
  else
    return __float_as_uint(row[e]);
}

struct WalkState {
  int cur;       // current city
  int s;         // next step (1 .. n-1)
  int live;      // unvisited cities listed for the current phase (gather phases)
  unsigned long long rwin;  // this lane's Philox words for the steps of the window
  uint32_t parity;          // mbarrier phase of the row copy
  bool waits_ok;
};

// Steps [w.s, s_end) of one phase.  CP: slots per thread.  kGather = false:
// slot i of thread t is city t*C + i (phase 0); true: slot i holds the entry
// ulist[t*CP + i] (its city's weight, or the zero slot once visited).  CPN > 0:
// afterwards, list the unvisited cities for a phase of CPN slots per thread.
template <int C, int CP, int CPN, int G, int H, bool kGather, bool kPool>
__device__ __forceinline__ void eq1_phase(const Instance& I, const int ant, const int tg,
                                          const Seg<H> seg, GroupSmem* gs, const int bar_id,
                                          float* srow, uint16_t* ulist, const int start,
                                          const int s_end, WalkState& w, const bool lane_copy) {
  static_assert(CP % 4 == 0 && CP >= 4 && CP <= 128, "CP must be a multiple of 4 in [4,128]");
  static_assert(kGather || CP == C, "the direct phase reads whole chunks");
  static_assert(G == 1 || (G == 2 && H == 32), "two warps per ant use whole warps");
  constexpr int NT = G * H;  // threads per ant
  constexpr int NW = (CP + 31) / 32;  // tabu words per lane (direct phase)
  constexpr int KW = (CP + H - 1) / H;
  // parts of the thread's slots for the second-level search: one per 32
  // slots (up to four); with the branch-free part choice a split pays for
  // two words too (n = 1002: 1.138 to 1.126 ms)
  constexpr int KP = KW < 4 ? KW : 4;
  constexpr int K = KP < CP / 4 ? KP : CP / 4;
  using Parts = ChunkParts<CP, K>;
  constexpr int PP = (Parts::max_cities() + H - 1) / H;  // cities per lane in the rescan
  constexpr int kListCap = StageLayout<C, G, H>::kListEntries;
  const int n = I.n, ld = I.ld;
  const int hl = seg.hl;          // lane within the segment
  const int wg = G > 1 ? tg >> 5 : 0;  // warp within the group
  const int base = tg * C;        // phase 0: the thread's chunk in the row
  auto group_wait = [&]() {
    if constexpr (G > 1)
      group_sync(bar_id, NT);
    else
      seg.sync();
  };
  const uint32_t iter = (uint32_t)I.st->iteration;
  const unsigned long long seed = I.seed;
  const uint32_t srow_a = smem_u32(srow);
  const uint32_t bar = srow_a + (uint32_t)StageLayout<C, G, H>::kRowFloats * 4u;
  const uint32_t row_bytes = (uint32_t)ld * 4u;
  int32_t* tour = I.tours + (size_t)ant * I.ldt;
  const float* const choice = I.choice;

  // Direct phase: tabu bits (1 = visited, or no city in the slot).  Gather
  // phases keep no tabu bits: a slot's list entry points at its city's
  // weight in the staged row while it is unvisited, and at kZeroSlot (a
  // float beside the row that stays 0) once it is visited or holds no city,
  // so a visited slot reads weight 0 and is never chosen.
  constexpr uint32_t kZeroSlot = StageLayout<C, G, H>::kZeroSlot;
  // A single instance lists byte offsets into the staged row (city * 4: no
  // address arithmetic per read), pools list city indices (measured faster
  // for the batched classes, slower for one instance).
  constexpr uint32_t kUnit = kPool ? 1u : 4u;
  constexpr uint32_t kZeroEntry = kZeroSlot * kUnit;
  static_assert(kZeroEntry <= 0xffffu, "list entries are 16-bit");
  uint32_t vis[kGather ? 1 : NW];
  if constexpr (!kGather) {
#pragma unroll
    for (int wd = 0; wd < NW; ++wd) {
      const int real = n - (base + 32 * wd);  // local cities of word wd below n
      uint32_t word = real <= 0 ? FULL : (real >= 32 ? 0u : (FULL << real));
      const int inchunk = C - 32 * wd;
      if (inchunk < 32) word |= FULL << inchunk;
      vis[wd] = word;
    }
    const int li = start - base;
    if (li >= 0 && li < C) {
#pragma unroll
      for (int wd = 0; wd < NW; ++wd)
        if (wd == (li >> 5)) vis[wd] |= 1u << (li & 31);
    }
  } else {
    // The thread's slots past the listed cities point at the zero weight.
#pragma unroll
    for (int i = 0; i < CP; ++i) {
      const int k = tg * CP + i;
      if (k >= w.live) ulist[k] = (uint16_t)kZeroEntry;
    }
    group_wait();  // other lanes read these entries in the rescan
  }

  for (; w.s < s_end; ++w.s) {
    const int s = w.s;
    const int cur = w.cur;
    // Everyone is done with the previous row (the segment agreed on `cur`).
    if (lane_copy) {
      const float4* src = reinterpret_cast<const float4*>(choice + (size_t)cur * ld);
      float4* dst = reinterpret_cast<float4*>(srow);
      for (int i = tg; i < (ld >> 2); i += NT) dst[i] = src[i];
    } else if (tg == 0) {
      fence_proxy_async_smem();
      bulk_load(srow_a, choice + (size_t)cur * ld, row_bytes, bar);
    }
    const int off = (s - 1) % H;
    if (off == 0) {
      const Philox4 x = step_draw(seed, (uint32_t)(s + hl), (uint32_t)ant, iter);
      w.rwin = ((unsigned long long)x.x1 << 32) | x.x0;
    }
    const unsigned long long r = seg.shfl(w.rwin, off);
    if (lane_copy) {
      group_wait();
    } else {
      if (w.waits_ok && !mbar_wait_bounded(bar, w.parity)) {
        w.waits_ok = false;  // stale data from here on; the status word says so
        if (tg == 0) atomicOr(&I.st->status, kStatusTimeout);
      }
      w.parity ^= 1u;
    }
    const float* row = srow;

    uint32_t v[CP];  // weight bits of the slots; w >= 0 orders like its bit pattern
    if constexpr (!kGather) {
#pragma unroll
      for (int i = 0; i < CP; i += 4) {
        const uint4 t = *reinterpret_cast<const uint4*>(row + base + i);
        v[i] = t.x;
        v[i + 1] = t.y;
        v[i + 2] = t.z;
        v[i + 3] = t.w;
      }
    } else {
      const uint2* lw = reinterpret_cast<const uint2*>(ulist + tg * CP);
#pragma unroll
      for (int i = 0; i < CP; i += 4) {
        const uint2 e = lw[i >> 2];
        v[i] = entry_weight<kUnit>(row, e.x & 0xffffu);
        v[i + 1] = entry_weight<kUnit>(row, e.x >> 16);
        v[i + 2] = entry_weight<kUnit>(row, e.y & 0xffffu);
        v[i + 3] = entry_weight<kUnit>(row, e.y >> 16);
      }
    }
    // The max pass.  A float max equals the integer max of the bit patterns
    // for weights >= 0 (no NaN; subnormals kept: no flush to zero); it
    // measured faster in the compacted phases and for direct chunks of 44
    // cities or more (n = 2392 0.6 %, n = 1002 0.45 %), slower for a direct
    // chunk of 36 (0.6 %).
    constexpr bool kFloatMax = kGather || C >= 44;
    uint32_t mx;
    if constexpr (kFloatMax) {
      float m4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int i = 0; i < CP; ++i) {
        if constexpr (!kGather) {
          if ((vis[i >> 5] >> (i & 31)) & 1u) v[i] = 0u;
        }
        m4[i & 3] = fmaxf(m4[i & 3], __uint_as_float(v[i]));
      }
      mx = seg.max_u32(__float_as_uint(fmaxf(fmaxf(m4[0], m4[1]), fmaxf(m4[2], m4[3]))));
    } else {
      uint32_t m4[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int i = 0; i < CP; ++i) {
        if constexpr (!kGather) {
          if ((vis[i >> 5] >> (i & 31)) & 1u) v[i] = 0u;
        }
        m4[i & 3] = max(m4[i & 3], v[i]);
      }
      mx = seg.max_u32(max(max(m4[0], m4[1]), max(m4[2], m4[3])));
    }
    if constexpr (G > 1) {
      if (hl == 0) gs->wmax[wg] = mx;
      group_wait();
#pragma unroll
      for (int k = 0; k < G; ++k) mx = max(mx, gs->wmax[k]);
    }

    int next;
    int chosen = -1, chosen_slot = 0;  // gather phases: the thread and slot to mark
    if (mx == 0u) {
      // Every unvisited weight is zero: the lowest unvisited city.
      uint32_t cand = 0xffffffffu;
      if constexpr (!kGather) {
#pragma unroll
        for (int wd = NW - 1; wd >= 0; --wd) {
          const uint32_t fr = ~vis[wd];
          if (fr) cand = (uint32_t)(base + 32 * wd + __ffs(fr) - 1);
        }
      } else {
        // the smallest entry: kZeroEntry is above every city's
        const uint2* lw = reinterpret_cast<const uint2*>(ulist + tg * CP);
#pragma unroll
        for (int i = 0; i < CP; i += 4) {
          const uint2 e = lw[i >> 2];
          cand = min(cand, min(min(e.x & 0xffffu, e.x >> 16), min(e.y & 0xffffu, e.y >> 16)));
        }
      }
      cand = seg.min_u32(cand);
      if constexpr (G > 1) {
        if (hl == 0) gs->wmin[wg] = (int)cand;
        group_wait();
#pragma unroll
        for (int k = 0; k < G; ++k) cand = min(cand, (uint32_t)gs->wmin[k]);
      }
      const uint32_t cand_entry = cand;  // gather phases: the list entry
      if constexpr (kGather) cand /= kUnit;
      next = (int)cand;
      if constexpr (kGather) {
        // the thread whose slot holds that city points the slot at the zero
        // weight (no other thread reads the list until the step's end)
#pragma unroll
        for (int i = 0; i < CP; ++i)
          if (ulist[tg * CP + i] == cand_entry) ulist[tg * CP + i] = (uint16_t)kZeroEntry;
      }
    } else {
      const int sc = kRouletteBits - 1 - exponent_of_bits(mx);
      float f1, f1s, f2;
      quant_factors(sc, f1, f1s, f2);
      if (f2 != 1.0f) {
#pragma unroll
        for (int i = 0; i < CP; ++i) v[i] = __float_as_uint(__fmul_rn(__uint_as_float(v[i]), f2));
      }
      uint32_t phi[K], plo[K];
      chunk_sum_parts<CP, K>(v, f1, f1s, phi, plo);
      uint32_t hs = phi[0], ls = plo[0];
#pragma unroll
      for (int k = 1; k < K; ++k) {
        hs += phi[k];
        ls += plo[k];
      }
      // Inclusive sums of the thread's first K - 1 parts (they overlap the
      // scan below; the selected lane's are used for the part choice).
      unsigned long long pincl[K > 1 ? K - 1 : 1];
      if constexpr (K > 1) {
        pincl[0] = part_value<CP, K>(phi, plo, 0);
#pragma unroll
        for (int k = 1; k < K - 1; ++k) pincl[k] = pincl[k - 1] + part_value<CP, K>(phi, plo, k);
      }
      const uint32_t offb = (uint32_t)CP * kTwo23Bits;
      const unsigned long long mine = ((unsigned long long)(hs - offb) << 23) + (ls - offb);
      const unsigned long long incl = seg.inclusive_scan(mine);
      const unsigned long long wtot = seg.shfl(incl, H - 1);
      unsigned long long woff = 0, Q = wtot;
      if constexpr (G > 1) {
        if (hl == 0) gs->wsum[wg] = wtot;
        group_wait();
        Q = 0;
#pragma unroll
        for (int k = 0; k < G; ++k) {
          const unsigned long long u = gs->wsum[k];
          if (k < wg) woff += u;
          Q += u;
        }
      }
      const unsigned long long T = __umul64hi(r, Q);
      // The warp whose range holds T finds the city (every warp when G = 1).
      if (G == 1 || (T >= woff && T - woff < wtot)) {
      const unsigned long long t1 = T - woff;
      const int L = max(__ffs(seg.ballot(incl > t1)) - 1, 0);
      const unsigned long long t2 = t1 - seg.shfl(incl - mine, L);
      // The part of lane L's slots that holds the target: the first whose
      // inclusive sum exceeds t2 (the sums ascend, so it is the count of
      // those at most t2).  Every lane takes lane L's sums and decides alike.
      int part = 0;
      unsigned long long t3 = t2;
      if constexpr (K > 1) {
        unsigned long long before = 0;
#pragma unroll
        for (int k = 0; k < K - 1; ++k) {
          const unsigned long long pk = seg.shfl(pincl[k], L);
          if (pk <= t2) {
            part = k + 1;
            before = pk;
          }
        }
        t3 = t2 - before;
      }
      // The segment rescans that part, PP slots per lane.
      const int pstart = 4 * (part * Parts::NG / K);
      const int psz = 4 * ((part + 1) * Parts::NG / K) - pstart;
      // lane L's tabu bits (direct phase; gather phases read them from the
      // list: a visited slot reads weight 0)
      uint32_t visL[kGather ? 1 : NW];
      if constexpr (!kGather) {
#pragma unroll
        for (int wd = 0; wd < NW; ++wd) visL[wd] = seg.shfl(vis[wd], L);
      }
      unsigned long long qv[PP];
      int cc[PP];
      unsigned long long ps = 0;
#pragma unroll
      for (int p = 0; p < PP; ++p) {
        const int pi = hl * PP + p;  // position within the part
        const int li = pstart + pi;  // slot within lane L's slots
        uint32_t w8 = 0u;
        int c = 0;
        const int tL = wg * 32 + L;  // thread of lane L within the group
        if constexpr (!kGather) {
          uint32_t word = FULL;
#pragma unroll
          for (int wd = 0; wd < NW; ++wd)
            if (wd == (li >> 5)) word = visL[wd];
          const bool open = pi < psz && !((word >> (li & 31)) & 1u);
          c = (G > 1 ? tL : L) * C + li;
          if (open && c < ld) w8 = __float_as_uint(row[c]);
        } else {
          if (pi < psz) {
            const uint32_t e = ulist[(G > 1 ? tL : L) * CP + li];
            w8 = entry_weight<kUnit>(row, e);
            c = (int)(e / kUnit);
          }
        }
        cc[p] = c;
        qv[p] = quant_value(w8, f1, f1s, f2);
        ps += qv[p];
      }
      const unsigned long long incl2 = seg.inclusive_scan(ps);
      const int L2 = max(__ffs(seg.ballot(incl2 > t3)) - 1, 0);
      int pick = 0;
      if constexpr (PP > 1) {
        if (hl == L2) {
          unsigned long long c = incl2 - ps;
          pick = -1;
#pragma unroll
          for (int p = 0; p < PP; ++p) {
            c += qv[p];
            if (pick < 0 && c > t3) pick = p;
          }
        }
        pick = max(seg.shfl(pick, L2), 0);
      }
      int pc = cc[0];
#pragma unroll
      for (int p = 1; p < PP; ++p)
        if (p == pick) pc = cc[p];
      next = seg.shfl(pc, L2);
      chosen = G > 1 ? wg * 32 + L : L;
      chosen_slot = pstart + L2 * PP + pick;
      if constexpr (G > 1) {
        if (hl == 0) {
          gs->next = next;
          gs->wmin[0] = chosen;
          gs->wmin[1] = chosen_slot;
        }
      }
      }
      if constexpr (G > 1) {
        group_wait();
        next = gs->next;
        chosen = gs->wmin[0];
        chosen_slot = gs->wmin[1];
      }
    }

    // A city outside [0, n) can only come from a defect; record it and stay
    // in bounds instead of reading past the matrix.
    if ((unsigned)next >= (unsigned)n) {
      if (tg == 0) atomicOr(&I.st->status, kStatusBadTour);
      next = start;
      chosen = -1;
    }
    if constexpr (!kGather) {
      const int li = next - base;
      if (li >= 0 && li < C) {
#pragma unroll
        for (int wd = 0; wd < NW; ++wd)
          if (wd == (li >> 5)) vis[wd] |= 1u << (li & 31);
      }
    } else if (tg == chosen) {
      // every read of this entry in this step came before the shuffle that
      // decided it
      ulist[tg * CP + chosen_slot] = (uint16_t)kZeroEntry;
    }
    if (tg == 0) tour[s] = next;
    w.cur = next;
    group_wait();
  }

  if constexpr (CPN > 0) {
    // List the unvisited cities for the next phase, ascending: lane after
    // lane, each lane's slots in order.
    uint32_t cnt = 0;
    uint32_t own[kGather ? CP : 1];  // gather phases: the thread's entries
    if constexpr (kGather) {
      const uint2* lw = reinterpret_cast<const uint2*>(ulist + tg * CP);
#pragma unroll
      for (int i = 0; i < CP; i += 4) {
        const uint2 e = lw[i >> 2];
        own[i] = e.x & 0xffffu;
        own[i + 1] = e.x >> 16;
        own[i + 2] = e.y & 0xffffu;
        own[i + 3] = e.y >> 16;
      }
#pragma unroll
      for (int i = 0; i < CP; ++i) cnt += own[i] != kZeroEntry ? 1u : 0u;
    } else {
#pragma unroll
      for (int wd = 0; wd < NW; ++wd) cnt += __popc(~vis[wd]);
    }
    const unsigned long long incl = seg.inclusive_scan((unsigned long long)cnt);
    int total = (int)seg.shfl(incl, H - 1);
    int k = (int)(incl - cnt);
    if constexpr (G > 1) {
      if (hl == 0) gs->wsum[wg] = (unsigned long long)total;
      group_wait();
      total = 0;
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const int u = (int)gs->wsum[q];
        if (q < wg) k += u;
        total += u;
      }
    }
    group_wait();  // the list of this phase is no longer read
#pragma unroll
    for (int i = 0; i < CP; ++i) {
      bool live;
      if constexpr (kGather)
        live = own[i] != kZeroEntry;
      else
        live = !((vis[i >> 5] >> (i & 31)) & 1u);
      if (live) {
        // a defect can leave more entries than the list holds: keep in bounds
        if (k < kListCap) ulist[k] = (uint16_t)(kGather ? own[i] : kUnit * (uint32_t)(base + i));
        ++k;
      }
    }
    w.live = total < NT * CPN ? total : NT * CPN;
    group_wait();
  }
}

// Phase J of the walk and the ones after it.  Phase J runs while the
// unvisited cities do not fit in the next phase's slots, then lists them for
// it; the last phase runs to the end of the tour.
template <int C, int G, int H, bool kPool, int J>
__device__ __forceinline__ void eq1_phases(const Instance& I, const int ant, const int tg,
                                           const Seg<H> seg, GroupSmem* gs, const int bar_id,
                                           float* srow, uint16_t* ulist, const int start,
                                           WalkState& w, const bool lane_copy) {
  using Cm = Compaction<C, G>;
  constexpr int CP = Cm::slots(J);
  constexpr int CPN = Cm::slots(J + 1);
  const int s_end = CPN > 0 ? max(w.s, I.n - G * H * CPN) : I.n;
  eq1_phase<C, CP, CPN, G, H, (J > 0), kPool>(I, ant, tg, seg, gs, bar_id, srow, ulist, start,
                                              s_end, w, lane_copy);
  if constexpr (CPN > 0)
    eq1_phases<C, G, H, kPool, J + 1>(I, ant, tg, seg, gs, bar_id, srow, ulist, start, w,
                                      lane_copy);
}

// The whole walk of one ant (G warps or one H-lane segment) and its length
// and neighbour buckets.
template <int C, int G, int H, bool kPool>
__device__ __forceinline__ void construct_ant_phased(const Instance& I, const int ant,
                                                     const int tg, const Seg<H> seg,
                                                     GroupSmem* gs, const int bar_id, float* srow,
                                                     const bool lane_copy) {
  using Cm = Compaction<C, G>;
  static_assert(Cm::kOn, "compaction needs one or two whole groups per ant and C >= kCompactMinC");
  constexpr int NT = G * H;
  uint16_t* ulist = reinterpret_cast<uint16_t*>(reinterpret_cast<char*>(srow) +
                                                StageLayout<C, G, H>::kListOffset);
  const int n = I.n;
  const int hl = seg.hl;
  const int wg = G > 1 ? tg >> 5 : 0;
  auto group_wait = [&]() {
    if constexpr (G > 1)
      group_sync(bar_id, NT);
    else
      seg.sync();
  };
  const uint32_t iter = (uint32_t)I.st->iteration;
  const Philox4 x0 = step_draw(I.seed, 0u, (uint32_t)ant, iter);
  const int start = (int)__umulhi(x0.x0, (uint32_t)n);
  int32_t* tour = I.tours + (size_t)ant * I.ldt;
  if (tg == 0) tour[0] = start;
  const uint32_t bar = smem_u32(srow) + (uint32_t)StageLayout<C, G, H>::kRowFloats * 4u;
  if (tg == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    srow[StageLayout<C, G, H>::kZeroSlot] = 0.0f;  // the weight of a visited list slot
  }
  group_wait();

  WalkState w{start, 1, 0, 0ull, 0u, true};
  eq1_phases<C, G, H, kPool, 0>(I, ant, tg, seg, gs, bar_id, srow, ulist, start, w, lane_copy);
  if (tg == 0) tour[n] = start;
  group_wait();

  // C^k (Section II) and the per-city neighbour buckets.
  long long len = 0;
  for (int s = tg; s < n; s += NT) {
    const int a = tour[s], b = tour[s + 1];
    const int p = tour[s == 0 ? n - 1 : s - 1];
    len += I.dist[(size_t)a * I.ld + b];
    I.nbr[(size_t)a * I.ldm + ant] = ((uint32_t)p << 16) | (uint32_t)b;
  }
#pragma unroll
  for (int o = H / 2; o > 0; o >>= 1) len += seg.shfl_xor(len, o);
  if constexpr (G > 1) {
    if (hl == 0) gs->wlen[wg] = len;
    group_wait();
    len = 0;
#pragma unroll
    for (int k = 0; k < G; ++k) len += gs->wlen[k];
  }
  if (tg == 0) I.lens[ant] = len;
}

}  // namespace aco
