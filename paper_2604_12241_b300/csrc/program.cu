// Generic interpretation of stage programs (AML_FAM_PROGRAM columns).
//
// A program that no kernel family implements runs the way Alg. 1 writes it:
// the trigger edge, then one loop per stage over a neighbour list, binding
// the stage's node and testing its skip_if and time constraints, and at the
// last stage the Postprocess that reports the binding.  One thread walks the
// bindings of one trigger edge depth first, with an explicit stack of at
// most seven stages; a trigger with more than 64 first-stage candidates is
// queued and walked by a whole warp, lane i taking every 32nd candidate.
// Each stage's loop starts where its time constraints allow
// (Find_Starting_Edge: binary searches in the operand's (t, id)-sorted list
// for the window, the span so far and the order bound) and stops where they
// end; an INTERSECT stage finds its b-side edges by binary search in
// the (counterparty, t, id) copy of the second operand's list.  The exact
// conditions (ties broken by edge id, skip masks, closing onto a bound node,
// amount ranges and ratios, pairwise distinct edges of an instance) are
// tested per candidate.
//
// Aggregates: EDGES stores the number of bindings of each trigger; DISTINCT
// counts bindings first (to size a hash set), then stores the number of
// distinct (trigger, last node) keys each trigger inserts; INSTANCES adds one
// to each edge of every binding with an atomic.  A launch stops after 2^34
// candidate visits and reports it, so a program with an enormous search
// space ends with an error instead of holding the GPU.
#include <cstring>
#include <type_traits>

#include "aml_internal.cuh"
#include "mine.cuh"
#include "profile.cuh"

namespace aml {

namespace {

constexpr unsigned long long PROG_WORK_LIMIT = 1ull << 34;
constexpr int PROG_FLUSH = 1024;  // visits a thread counts before adding them to the total
constexpr int PROG_BLOCK = 128;
constexpr int AGG_COUNT = 0, AGG_SET = 1, AGG_CREDIT = 2;  // kernel modes
constexpr unsigned long long SET_EMPTY = ~0ull;

struct ProgCtl {
  unsigned long long work;  // candidate visits of the launch so far
  uint32_t stop;            // set once the limit is crossed
  uint32_t n_heavy;         // triggers left to a whole warp
  unsigned long long total; // DISTINCT: bindings counted by the first pass
  unsigned long long next;  // next heavy trigger a warp takes
};

// A trigger whose first stage has more candidates than this is walked by a
// whole warp (each lane takes every 32nd first-stage candidate) instead of
// one thread, so hub triggers do not leave one lane working long after the
// rest of the GPU is idle.
constexpr int32_t PROG_HEAVY = 64;
constexpr unsigned long long PROG_DEFERRED = ~0ull;

// one direction's lists: (t, id) order and the (counterparty, t, id) copy
struct ListView {
  const int32_t *ptr, *nbr, *t, *eid, *nnbr, *nt, *neid;
};

__device__ __forceinline__ ListView list_of(const GraphView& g, int dir) {
  return dir == AML_DIR_OUT ? ListView{g.optr, g.onbr, g.ot, g.oeid, g.onnbr, g.ont, g.oneid}
                            : ListView{g.iptr, g.inbr, g.it, g.ieid, g.innbr, g.int_, g.ineid};
}

// first i in [lo, hi) with (nnbr[i], nt[i]) >= (x, tmin)
__device__ __forceinline__ int32_t lower_nbr_t(const int32_t* __restrict__ nnbr,
                                               const int32_t* __restrict__ nt, int32_t lo,
                                               int32_t hi, int32_t x, int64_t tmin) {
  while (lo < hi) {
    const int32_t mid = (int32_t)(((uint32_t)lo + (uint32_t)hi) >> 1);
    const int32_t y = __ldg(nnbr + mid);
    if (y < x || (y == x && (int64_t)__ldg(nt + mid) < tmin)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// SplitMix64's output function (Steele, Lea and Flood), used as a hash
__device__ __forceinline__ uint64_t set_hash(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// open addressing, linear probing; true when the key was not there yet
__device__ bool set_insert(unsigned long long* table, uint64_t mask, unsigned long long key) {
  uint64_t h = set_hash(key) & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const unsigned long long prev = atomicCAS(table + h, SET_EMPTY, key);
    if (prev == SET_EMPTY) return true;
    if (prev == key) return false;
    h = (h + 1) & mask;
  }
  return false;  // not reached: the table holds at least twice the keys
}

// The bindings of trigger e0: returns the trigger's count (EDGES, DISTINCT),
// or PROG_DEFERRED when a single thread (WARP false) finds the first stage
// heavy and queues the trigger for a warp.  With WARP, lane `lane` of the
// warp walks the first-stage candidates lane, lane + 32, ...
// the stage's amount constraints on edge f, whose predecessor on the walk
// is edge prev; ratio * amount in double, the exact product of two floats
__device__ __forceinline__ bool amount_ok(const ProgStage& q, const float* __restrict__ amount,
                                          int32_t f, int32_t prev) {
  if (!q.amt) return true;
  const double a = __ldg(amount + f);
  if ((q.amt & AML_AMT_RANGE) && !(a >= q.amin && a <= q.amax)) return false;
  if (q.amt & AML_AMT_RATIO) {
    const double b = __ldg(amount + prev);
    if (!(a >= (double)q.rmin * b && a <= (double)q.rmax * b)) return false;
  }
  return true;
}

template <int MODE, bool WARP>
__device__ __forceinline__ unsigned long long walk(const GraphView& g, const float* amount,
                                                   const Prog& p, int32_t e0,
                                                   int lane, unsigned long long* __restrict__ out,
                                                   unsigned long long* __restrict__ table,
                                                   uint64_t table_mask, ProgCtl* ctl,
                                                   int32_t* __restrict__ heavy) {
  const int32_t t0 = g.ts[e0];
  const int n = p.n;
  const int64_t delta = p.delta;
  int32_t node[PROG_MAX_STAGES + 1], reach_e[PROG_MAX_STAGES + 1], reach_t[PROG_MAX_STAGES + 1];
  int32_t nb[PROG_MAX_STAGES];  // variables bound before each stage
  int32_t cur[PROG_MAX_STAGES], hi[PROG_MAX_STAGES], bcur[PROG_MAX_STAGES], bhi[PROG_MAX_STAGES];
  int32_t ea[PROG_MAX_STAGES], eb[PROG_MAX_STAGES], xa[PROG_MAX_STAGES], ta[PROG_MAX_STAGES];
  int32_t smin[PROG_MAX_STAGES], smax[PROG_MAX_STAGES];
  node[0] = g.src[e0];
  node[1] = g.dst[e0];
  if (node[0] == node[1]) return 0;  // self-loops are in no list; their rows stay 0
  if (!amount_ok(p.st[0], amount, e0, e0)) return 0;  // not a trigger (range only)
  reach_e[0] = reach_e[1] = e0;
  reach_t[0] = reach_t[1] = t0;
  nb[1] = 2;
  for (int s = 1; s + 1 < n; ++s) nb[s + 1] = nb[s] + (p.st[s].out_var == nb[s] ? 1 : 0);
  int32_t tmin = t0, tmax = t0;  // the span set: e0 and the SPAN stages' edges
  unsigned long long found = 0;
  int work = 0;
  bool stopped = false;
  // bit s: intersection stage s walks its b-side window and searches the
  // a-side (degree-ordered intersection: the shorter window is walked)
  uint32_t swp = 0;

  auto tick = [&]() {
    if (++work < PROG_FLUSH) return;
    work = 0;
    const unsigned long long tot = atomicAdd(&ctl->work, (unsigned long long)PROG_FLUSH);
    if (tot + PROG_FLUSH > PROG_WORK_LIMIT) {
      atomicExch(&ctl->stop, 1u);
      stopped = true;
    } else if (*(volatile uint32_t*)&ctl->stop) {
      stopped = true;
    }
  };
  // f repeats an edge already in the binding (stages before s, and e0)
  auto used = [&](int32_t f, int s) {
    if (f == e0) return true;
    for (int j = 1; j < s; ++j)
      if (ea[j] == f || (p.st[j].op == AML_OP_INTERSECT && eb[j] == f)) return true;
    return false;
  };
  auto node_ok = [&](const ProgStage& q, int s, int32_t x) {
    for (int i = 0; i < nb[s]; ++i)
      if (((q.skip >> i) & 1u) && node[i] == x) return false;
    return q.out_var >= nb[s] || node[q.out_var] == x;
  };
  auto bind = [&](const ProgStage& q, int s, int32_t x, int32_t f, int32_t tf) {
    if (q.out_var == nb[s]) {
      node[q.out_var] = x;
      reach_e[q.out_var] = f;
      reach_t[q.out_var] = tf;
    }
  };
  auto complete = [&](int32_t x_last) {
    if (MODE == AGG_COUNT) {
      ++found;
    } else if (MODE == AGG_SET) {
      const unsigned long long key = ((unsigned long long)(uint32_t)e0 << 32) | (uint32_t)x_last;
      if (set_insert(table, table_mask, key)) ++found;
    } else {
      atomicAdd(out + e0, 1ull);
      for (int j = 1; j < n; ++j) {
        atomicAdd(out + ea[j], 1ull);
        if (p.st[j].op == AML_OP_INTERSECT) atomicAdd(out + eb[j], 1ull);
      }
    }
  };
  // loop bounds of stage s from its window, the span so far and its order
  auto enter = [&](int s) {
    const ProgStage q = p.st[s];
    smin[s] = tmin;
    smax[s] = tmax;
    const ListView L = list_of(g, q.a_dir);
    const int A = q.a_var;
    int64_t tl, th;
    if (q.window == AML_WIN_TRAILING) {
      tl = (int64_t)t0 - delta;
      th = t0;
    } else {
      tl = (int64_t)tmax - delta;
      th = (int64_t)tmin + delta;
    }
    if (q.order == AML_ORDER_AFTER) tl = max(tl, (int64_t)reach_t[A]);
    else if (q.order == AML_ORDER_BEFORE) th = min(th, (int64_t)reach_t[A]);
    else if (q.order == AML_ORDER_AFTER_TRIGGER) tl = max(tl, (int64_t)t0);
    const int32_t lo = L.ptr[node[A]], end = L.ptr[node[A] + 1];
    swp &= ~(1u << s);
    if (tl > th) {
      cur[s] = hi[s] = lo;
    } else {
      cur[s] = lower_t(L.t, lo, end, tl);
      hi[s] = lower_t(L.t, cur[s], end, th + 1);
      // an intersection without order or amount constraints is symmetric in
      // its two sides: walk the shorter window, search the other side's
      // (counterparty, t, id) copy (Sec. 6's degree-ordered intersection);
      // the bindings are the same pairs of edges either way
      if (q.op == AML_OP_INTERSECT && q.order == AML_ORDER_NONE && !q.amt) {
        const ListView LB = list_of(g, q.b_dir);
        const int32_t lob = LB.ptr[node[q.b_var]], endb = LB.ptr[node[q.b_var] + 1];
        const int32_t cb = lower_t(LB.t, lob, endb, tl);
        const int32_t hb = lower_t(LB.t, cb, endb, th + 1);
        if (hb - cb < hi[s] - cur[s]) {
          swp |= 1u << s;
          cur[s] = cb;
          hi[s] = hb;
        }
      }
    }
    bcur[s] = bhi[s] = 0;
  };
  // the next binding of stage s (its bounds set by enter(s)); false when none is left
  auto next = [&](int s) -> bool {
    const ProgStage q = p.st[s];
    const ListView LA = list_of(g, q.a_dir);
    const int A = q.a_var;
    const bool span = q.window == AML_WIN_SPAN;
    if (q.op == AML_OP_FOR_ALL) {
      while (cur[s] < hi[s]) {
        tick();
        if (stopped) return false;
        const int32_t i = cur[s];
        cur[s] += (WARP && s == 1) ? 32 : 1;
        const int32_t f = LA.eid[i], x = LA.nbr[i], tf = LA.t[i];
        if (q.order == AML_ORDER_AFTER && !before(reach_t[A], reach_e[A], tf, f)) continue;
        if (q.order == AML_ORDER_BEFORE && !before(tf, f, reach_t[A], reach_e[A])) continue;
        if (q.order == AML_ORDER_AFTER_TRIGGER && !before(t0, e0, tf, f)) continue;
        if (!span && before(t0, e0, tf, f)) continue;  // trailing: f <= e0
        if (!node_ok(q, s, x)) continue;
        if (!amount_ok(q, amount, f, reach_e[A])) continue;
        if (MODE == AGG_CREDIT && used(f, s)) continue;
        ea[s] = f;
        xa[s] = x;
        tmin = span ? min(smin[s], tf) : smin[s];
        tmax = span ? max(smax[s], tf) : smax[s];
        bind(q, s, x, f, tf);
        return true;
      }
      return false;
    }
    // an intersection: the outer loop walks one side's time window (the
    // a-side, or the b-side when swapped), the inner loop the other side's
    // edges with the outer edge's far end x, from its (counterparty, t, id)
    // copy
    const bool sw = (swp >> s) & 1u;
    const ListView LO = list_of(g, sw ? q.b_dir : q.a_dir);
    const ListView LI = list_of(g, sw ? q.a_dir : q.b_dir);
    const int32_t inode = node[sw ? q.a_var : q.b_var];
    while (true) {
      while (bcur[s] < bhi[s]) {
        tick();
        if (stopped) return false;
        const int32_t j = bcur[s]++;
        const int32_t fi = LI.neid[j], ti = LI.nt[j];
        const int32_t fo = sw ? eb[s] : ea[s], to = ta[s];
        if (!sw) {  // fo = fa (a-side), fi = fb (b-side)
          if ((q.order == AML_ORDER_AFTER || q.order == AML_ORDER_LEG) && !before(to, fo, ti, fi))
            continue;
          if (q.order == AML_ORDER_BEFORE && !before(ti, fi, to, fo)) continue;
          if (q.order == AML_ORDER_AFTER_TRIGGER && !before(t0, e0, ti, fi)) continue;
          if (!amount_ok(q, amount, fi, fo)) continue;
        }
        if (!span && before(t0, e0, ti, fi)) continue;
        if (MODE == AGG_CREDIT && (fi == fo || used(fi, s))) continue;
        if (sw) ea[s] = fi; else eb[s] = fi;
        tmin = span ? min(min(smin[s], to), ti) : smin[s];
        tmax = span ? max(max(smax[s], to), ti) : smax[s];
        // the new variable is reached by the b-side edge
        if (sw) bind(q, s, xa[s], fo, to); else bind(q, s, xa[s], fi, ti);
        return true;
      }
      if (cur[s] >= hi[s]) return false;
      tick();
      if (stopped) return false;
      const int32_t i = cur[s];
      cur[s] += (WARP && s == 1) ? 32 : 1;
      const int32_t fo = LO.eid[i], x = LO.nbr[i], to = LO.t[i];
      bhi[s] = bcur[s] = 0;
      if (!sw) {  // the a-side edge's order and amount constraints
        if (q.order == AML_ORDER_AFTER && !before(reach_t[A], reach_e[A], to, fo)) continue;
        if (q.order == AML_ORDER_BEFORE && !before(to, fo, reach_t[A], reach_e[A])) continue;
        if (q.order == AML_ORDER_AFTER_TRIGGER && !before(t0, e0, to, fo)) continue;
        if (!amount_ok(q, amount, fo, reach_e[A])) continue;
      }
      if (!span && before(t0, e0, to, fo)) continue;
      if (!node_ok(q, s, x)) continue;
      if (MODE == AGG_CREDIT && used(fo, s)) continue;
      if (sw) eb[s] = fo; else ea[s] = fo;
      xa[s] = x;
      ta[s] = to;
      // the inner side's edges: far end x, inside the window with the outer
      // edge in the span
      int64_t tl, th;
      if (span) {
        tl = (int64_t)max(smax[s], to) - delta;
        th = (int64_t)min(smin[s], to) + delta;
      } else {
        tl = (int64_t)t0 - delta;
        th = t0;
      }
      if (!sw) {
        if (q.order == AML_ORDER_AFTER || q.order == AML_ORDER_LEG) tl = max(tl, (int64_t)to);
        else if (q.order == AML_ORDER_BEFORE) th = min(th, (int64_t)to);
        else if (q.order == AML_ORDER_AFTER_TRIGGER) tl = max(tl, (int64_t)t0);
      }
      if (tl > th) continue;
      const int32_t lo = LI.ptr[inode], end = LI.ptr[inode + 1];
      bcur[s] = lower_nbr_t(LI.nnbr, LI.nt, lo, end, x, tl);
      bhi[s] = lower_nbr_t(LI.nnbr, LI.nt, bcur[s], end, x, th + 1);
    }
  };

  if (n == 1) {
    if (!WARP || lane == 0) complete(node[1]);
  } else {
    int s = 1;
    enter(1);
    if (!WARP && heavy && hi[1] - cur[1] > PROG_HEAVY) {
      heavy[atomicAdd(&ctl->n_heavy, 1u)] = e0;
      return PROG_DEFERRED;
    }
    if (WARP) cur[1] += lane;
    while (s >= 1) {
      if (!next(s)) {
        if (stopped) break;
        --s;
        continue;
      }
      if (s == n - 1) {
        complete(xa[s]);
      } else {
        ++s;
        enter(s);
      }
    }
  }
  return found;
}

// one thread per trigger edge; heavy triggers are queued for k_program_warp
template <int MODE>
__global__ void __launch_bounds__(PROG_BLOCK) k_program(GraphView g, const float* amount, Prog p,
                                                        unsigned long long* __restrict__ out,
                                                        unsigned long long* __restrict__ table,
                                                        uint64_t table_mask, ProgCtl* ctl,
                                                        int32_t* __restrict__ heavy) {
  const int64_t e64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e64 >= g.E) return;
  const int32_t e0 = (int32_t)e64;
  const unsigned long long f =
      walk<MODE, false>(g, amount, p, e0, 0, out, table, table_mask, ctl, heavy);
  if (MODE != AGG_CREDIT && f != PROG_DEFERRED) out[e0] = f;
}

// the queued heavy triggers, one warp each, taken from a shared cursor by
// resident warps
template <int MODE>
__global__ void __launch_bounds__(PROG_BLOCK) k_program_warp(GraphView g, const float* amount,
                                                             Prog p,
                                                             unsigned long long* __restrict__ out,
                                                             unsigned long long* __restrict__ table,
                                                             uint64_t table_mask, ProgCtl* ctl,
                                                             const int32_t* __restrict__ heavy) {
  const int lane = threadIdx.x & 31;
  const unsigned long long n_heavy = ctl->n_heavy;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(&ctl->next, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_heavy || *(volatile uint32_t*)&ctl->stop) return;
    const int32_t e0 = heavy[item];
    unsigned long long f =
        walk<MODE, true>(g, amount, p, e0, lane, out, table, table_mask, ctl, nullptr);
    for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
    if (MODE != AGG_CREDIT && lane == 0) out[e0] = f;
  }
}

// v[i] / d for counts that are exact multiples of d (the bindings of an
// instance set each credit it once)
__global__ void k_div_exact(unsigned long long* __restrict__ v, int64_t n, uint32_t d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] /= d;
}

__global__ void k_sum_u64(const unsigned long long* __restrict__ v, int64_t n,
                          unsigned long long* __restrict__ total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long x = i < n ? v[i] : 0ull;
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0 && x) atomicAdd(total, x);
}

}  // namespace

// Counts of one interpreted program into out[E] (uint64; INSTANCES adds to
// it, so it must hold zeros; EDGES and DISTINCT overwrite it).  Waits for
// `s` to read the launch's status.
void run_program(const GraphView& gv, const float* amount, const Prog& p,
                 unsigned long long* out, cudaStream_t s) {
  const int64_t E = gv.E;
  if (E == 0) return;
  DBuf<ProgCtl> ctl(1, s);
  DBuf<int32_t> heavy((size_t)E, s);
  AML_CUDA(cudaMemsetAsync(ctl.p, 0, sizeof(ProgCtl), s));
  const unsigned grid = grid_for(E, PROG_BLOCK);
  const unsigned warp_grid = (unsigned)sm_count() * 8;  // resident warps take the queue
  auto check_stop = [&](unsigned long long* total) {
    ProgCtl h;
    const SmallRead rd{&h, ctl.p, (uint32_t)sizeof(ProgCtl)};
    read_small(&rd, 1, s);
    AML_REQUIRE(!h.stop, AML_EUNSUPPORTED,
                "interpreted stage program stopped at the limit of 2^34 candidate edges");
    if (total) *total = h.total;
  };
  // one pass: a thread per trigger, then a warp per heavy trigger
  auto pass = [&](auto mode, unsigned long long* table, uint64_t mask) {
    constexpr int M = decltype(mode)::value;
    AML_LAUNCH("k_program", s,
               k_program<M><<<grid, PROG_BLOCK, 0, s>>>(gv, amount, p, out, table, mask, ctl.p,
                                                        heavy.p));
    AML_LAUNCH("k_program_warp", s,
               k_program_warp<M><<<warp_grid, PROG_BLOCK, 0, s>>>(gv, amount, p, out, table,
                                                                  mask, ctl.p, heavy.p));
  };
  if (p.agg == AML_AGG_INSTANCES) {
    pass(std::integral_constant<int, AGG_CREDIT>{}, nullptr, 0);
    if (p.div > 1)
      AML_LAUNCH("k_div_exact", s,
                 k_div_exact<<<grid_for(E, 256), 256, 0, s>>>(out, E, (uint32_t)p.div));
  } else if (p.agg == AML_AGG_EDGES) {
    pass(std::integral_constant<int, AGG_COUNT>{}, nullptr, 0);
  } else {
    // bindings first, to size the set of (trigger, last node) keys
    pass(std::integral_constant<int, AGG_COUNT>{}, nullptr, 0);
    AML_LAUNCH("k_sum_u64", s,
               k_sum_u64<<<grid_for(E, 256), 256, 0, s>>>(out, E, &ctl.p->total));
    unsigned long long total = 0;
    check_stop(&total);
    AML_REQUIRE(total < (1ull << 31), AML_EUNSUPPORTED,
                "interpreted DISTINCT program has more than 2^31 bindings");
    uint64_t size = 1024;
    while (size < 2 * total) size <<= 1;
    DBuf<unsigned long long> table((size_t)size, s);
    AML_CUDA(cudaMemsetAsync(table.p, 0xff, (size_t)size * 8, s));
    AML_CUDA(cudaMemsetAsync(ctl.p, 0, sizeof(ProgCtl), s));
    pass(std::integral_constant<int, AGG_SET>{}, table.p, size - 1);
  }
  check_stop(nullptr);
}

}  // namespace aml
