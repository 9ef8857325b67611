// Per-edge pattern counting kernels and the aml_mine pipeline.
//
// Notation: edge e = u->v at time t_e; f < e iff (t_f, f) < (t_e, e).
// A "leg" is a temporal 2-path a = x->h, b = h->y with x != y, a < b and
// t_b - t_a <= delta: the first two stages of both the scatter-gather and
// the cycle programs (trigger N0->N1, for_all N1.out -> N2 skipping N0;
// Sec. 5, Fig. 4), so it is expanded once per window and shared by both.
#include <algorithm>
#include <climits>
#include <cstring>
#include <type_traits>

#include "aml_internal.cuh"
#include "mine.cuh"
#include "profile.cuh"

namespace aml {

// ------------------------------------------------------------------ FAN
//
// FAN_OUT(e) = DEG_OUT(e) - R(p), p = slot of e in out(u), where R(p) is the
// number of slots q in the trailing window [lb(p), p] whose previous
// same-counterparty slot prev(q) is also in the window (repeats).  Moving
// from p-1 to p, the window gains slot p (a repeat iff prev(p) >= lb(p)) and
// drops slots r in [lb(p-1), lb(p)), each of which removes one repeat iff
// next(r) <= p-1.  So R is a per-row prefix sum of per-slot deltas: one pass
// plus one scan, O(list length) in total.

// Per slot p of one direction: DEG(p) = p - lb(p) + 1, lb(p) the start of
// its trailing window, and, when FAN is wanted, the repeat delta above.
// deg_s: DEG per slot; df: (DEG, 0) stored in the edge's 32-byte row of df
// (the DEG-only case: no FAN pass follows).  Each output may be null.
__global__ void __launch_bounds__(512) k_window_slots(const int32_t* __restrict__ rstart,
                                                      const int32_t* __restrict__ t,
                                                      const int32_t* __restrict__ eid,
                                                      const int32_t* __restrict__ prev,
                                                      const int32_t* __restrict__ next,
                                                      int64_t Ev, int32_t delta,
                                                      int32_t* __restrict__ deg_s,
                                                      int32_t* __restrict__ D,
                                                      int2* __restrict__ df) {
  int64_t p64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p64 >= Ev) return;
  int32_t p = (int32_t)p64;
  const int32_t rs = __ldg(rstart + p);
  const int32_t tp = __ldg(t + p);
  const int32_t lbp = lower_t(t, rs, p + 1, (int64_t)tp - delta);
  const int32_t deg = p - lbp + 1;
  if (deg_s) deg_s[p] = deg;
  if (df) {  // the whole 32-byte row: a full-sector store, no read-modify-write
    int4* row = reinterpret_cast<int4*>(df + (int64_t)__ldg(eid + p) * DF_STRIDE);
    row[0] = make_int4(deg, 0, 0, 0);
    row[1] = make_int4(0, 0, 0, 0);
  }
  if (!D) return;
  int32_t d = 0;
  if (p > rs) {
    // lb(p-1) <= min(lb(p), p-1): search only up to there
    int32_t lbq = lower_t(t, rs, min(lbp + 1, p), (int64_t)__ldg(t + p - 1) - delta);
    d = (__ldg(prev + p) >= lbp) ? 1 : 0;
    for (int32_t r = lbq; r < lbp; ++r) d -= (__ldg(next + r) <= p - 1) ? 1 : 0;
  }
  D[p] = d;
}

// ------------------------------------------------------------------ legs

__device__ __forceinline__ void leg_window(const GraphView& g, int32_t a, int32_t& q0,
                                           int32_t& q1, int32_t delta) {
  int32_t h = g.dst[a];
  int32_t hs = g.optr[h], he = g.optr[h + 1];
  int32_t ta = g.ts[a];
  after_edge_upto(g.ot, g.oeid, hs, he, ta, a, (int64_t)ta + delta, q0, q1);
}

// number of slots in [lo, hi) of the (nbr, t, id) copy with nbr == x and
// (t, id) in ((te, e), te + delta]
__device__ __forceinline__ int32_t pair_after(const int32_t* __restrict__ nn,
                                              const int32_t* __restrict__ nt,
                                              const int32_t* __restrict__ ne, int32_t lo,
                                              int32_t hi, int32_t x, int32_t te, int32_t e,
                                              int32_t delta) {
  int32_t r0, r1, b0, b1;
  nbr_range(nn, lo, hi, x, r0, r1);
  if (r1 == r0) return 0;
  after_edge_upto(nt, ne, r0, r1, te, e, (int64_t)te + delta, b0, b1);
  return b1 - b0;
}

// ... with (t, id) in [te - delta, (te, e))
__device__ __forceinline__ int32_t pair_before(const int32_t* __restrict__ nn,
                                               const int32_t* __restrict__ nt,
                                               const int32_t* __restrict__ ne, int32_t lo,
                                               int32_t hi, int32_t x, int32_t te, int32_t e,
                                               int32_t delta) {
  int32_t r0, r1, b0, b1;
  nbr_range(nn, lo, hi, x, r0, r1);
  if (r1 == r0) return 0;
  since_upto_edge(nt, ne, r0, r1, (int64_t)te - delta, te, e, b0, b1);
  return b1 - b0;
}

// legs starting with a (the gather side of GS): later edges out of dst(a)
// inside the window, minus those returning to src(a)
__device__ __forceinline__ int32_t legs_from(const GraphView& g, int32_t a, int32_t delta) {
  int32_t q0, q1;
  leg_window(g, a, q0, q1, delta);
  int32_t h = g.dst[a];
  return (q1 - q0) - pair_after(g.onnbr, g.ont, g.oneid, g.optr[h], g.optr[h + 1], g.src[a],
                                g.ts[a], a, delta);
}

// legs ending with b (the scatter side of GS): earlier edges into src(b)
// inside the window, minus those coming from dst(b)
__device__ __forceinline__ int32_t legs_into(const GraphView& g, int32_t b, int32_t delta) {
  int32_t h = g.src[b];
  int32_t hs = g.iptr[h], he = g.iptr[h + 1];
  int32_t tb = g.ts[b];
  int32_t c0, c1;
  since_upto_edge(g.it, g.ieid, hs, he, (int64_t)tb - delta, tb, b, c0, c1);
  return (c1 - c0) - pair_before(g.innbr, g.int_, g.ineid, hs, he, g.dst[b], tb, b, delta);
}

// slot bound of the legs of a that can start a cycle: its window slots that
// precede the latest edge cl = (t, id) of its closing range (q0 when that
// range is empty)
__device__ __forceinline__ int32_t cycle_bound(const GraphView& g, int2 cr, int2 cl, int32_t q0,
                                               int32_t q1) {
  if (cr.x >= cr.y) return q0;
  return after_edge(g.ot, g.oeid, q0, q1, cl.x, cl.y - 1);  // first slot not before it
}

// The closing range B1 of edge a = x -> h (the slots of x's in-list after a,
// up to t_a + delta; delta counting: only new closing edges) and the (t,
// id) of its latest edge, as (B1 begin, B1 end, t, id); with rec, also
// stored as a's whole 32-byte anchor record (one sector).
__device__ __forceinline__ int4 close_anchor(const GraphView& g, int32_t a, int32_t x, int32_t h,
                                             int32_t ta, int32_t delta, AnchorRec* rec) {
  int2 r = make_int2(0, 0);
  if (x != h) {
    const int32_t is = g.iptr[x], ie = g.iptr[x + 1];
    after_edge_upto(g.it, g.ieid, is, ie, ta, a, (int64_t)ta + delta, r.x, r.y);
    // delta counting: a cycle is new iff its closing (latest) edge is new
    if (g.new_from > 0) r.x = after_edge(g.it, g.ieid, r.x, r.y, g.t_new, g.new_from - 1);
  }
  const bool any = r.x < r.y;
  const int4 an = make_int4(r.x, r.y, any ? __ldg(g.it + r.y - 1) : 0,
                            any ? __ldg(g.ieid + r.y - 1) : 0);
  if (rec) {
    int4* dst = reinterpret_cast<int4*>(rec + a);
    dst[0] = an;
    dst[1] = make_int4(x, h, ta, 0);
  }
  return an;
}

// L[a]: legs from a.  With anc (anchor records): L2[a] = those that can
// start a cycle (slots before the cycle bound, minus returns to src(a) among
// them).
// With L_new (delta counting): L_new[a] = legs from a whose second edge is new.
// qwin[a] = a's window slots [q0, q1) in dst(a)'s out-list and, with anc,
// qcb[a] = its cycle bound, kept for the emission.
// close_here: the anchor record of every edge with legs is computed and
// stored here (no separate k_close_range pass; an edge without legs starts
// no cycle and its record is never read); else it is read from anc.
// Z: the accumulators the emission and later kernels add into, zeroed here
// (element a of each) instead of by separate memsets.
constexpr int LEG_SCAN = 4;  // windows up to this many slots are scanned, not searched
// the leg count of one edge a (every thread of k_leg_count, and the fused
// mine's first phase)
template <int NS>
__device__ __forceinline__ void leg_count_item(const GraphView& g, int32_t delta, int32_t a,
                                               int32_t* __restrict__ L,
                                               AnchorRec* __restrict__ anc, int close_here,
                                               int32_t* __restrict__ L2,
                                               int32_t* __restrict__ L_new,
                                               int2* __restrict__ qwin,
                                               int32_t* __restrict__ qcb,
                                               const SubWindows& sub, const ZeroSink& Z) {
  for (int c = 0; c < Z.n_acc; ++c) Z.acc[(int64_t)c * g.E + a] = 0ull;
  if (Z.gs_in) Z.gs_in[a] = 0;
#pragma unroll
  for (int i = 0; i < NS; ++i)
    if (i < sub.n && sub.gs_in[i]) sub.gs_in[i][a] = 0;
  const int32_t x = g.src[a], h = g.dst[a];
  if (x == h) {
    L[a] = 0;
    qwin[a] = make_int2(0, 0);
#pragma unroll
    for (int i = 0; i < NS; ++i)
      if (i < sub.n && sub.gs_from[i]) sub.gs_from[i][a] = 0;
    if (L2) {
      L2[a] = 0;
      qcb[a] = 0;
    }
    if (L_new) L_new[a] = 0;
    return;
  }
  const int32_t ta = g.ts[a];
  const int32_t hs = g.optr[h], he = g.optr[h + 1];
  int32_t q0, q1;
  after_edge_upto(g.ot, g.oeid, hs, he, ta, a, (int64_t)ta + delta, q0, q1);
  qwin[a] = make_int2(q0, q1);
  const int32_t n = q1 - q0;
  if (n <= LEG_SCAN) {
    // a short window (most are): its slots are read at once and every count
    // is taken from them -- the returns h -> x are the slots whose
    // counterparty is x -- with no search of the (nbr, t, id) copy
    const bool need_id = g.new_from > 0 || L2 != nullptr;
    int32_t y[LEG_SCAN], tq[LEG_SCAN], iq[LEG_SCAN];
#pragma unroll
    for (int k = 0; k < LEG_SCAN; ++k) {
      y[k] = k < n ? __ldg(g.onbr + q0 + k) : -1;
      tq[k] = k < n ? __ldg(g.ot + q0 + k) : 0;
      iq[k] = k < n && need_id ? __ldg(g.oeid + q0 + k) : 0;
    }
    int32_t back = 0;
#pragma unroll
    for (int k = 0; k < LEG_SCAN; ++k) back += y[k] == x ? 1 : 0;
    L[a] = n - back;
    // delta counting: a slot is new when it comes after (t_new, new_from - 1)
    auto is_new = [&](int k) {
      return g.new_from == 0 || before(g.t_new, g.new_from - 1, tq[k], iq[k]);
    };
#pragma unroll
    for (int i = 0; i < NS; ++i)
      if (i < sub.n && sub.gs_from[i]) {
        const int64_t tmax = (int64_t)ta + sub.delta[i];
        int32_t c = 0;
#pragma unroll
        for (int k = 0; k < LEG_SCAN; ++k)
          if (k < n && (int64_t)tq[k] <= tmax && is_new(k) && y[k] != x) ++c;
        sub.gs_from[i][a] = c;
      }
    if (L_new) {
      int32_t c = 0;
#pragma unroll
      for (int k = 0; k < LEG_SCAN; ++k)
        if (k < n && is_new(k) && y[k] != x) ++c;
      L_new[a] = c;
    }
    if (!L2) return;
    if (n == 0) {  // no legs: no cycle starts at a
      qcb[a] = q0;
      L2[a] = 0;
      return;
    }
    const int4 an = close_here ? close_anchor(g, a, x, h, ta, delta, anc)
                               : *reinterpret_cast<const int4*>(anc + a);
    // the cycle bound: the window's slots before the latest closing edge
    int32_t nc = 0, c2 = 0;
    if (an.x < an.y) {
#pragma unroll
      for (int k = 0; k < LEG_SCAN; ++k)
        if (k < n && before(tq[k], iq[k], an.z, an.w)) {
          ++nc;
          if (y[k] != x) ++c2;
        }
    }
    qcb[a] = q0 + nc;
    L2[a] = c2;
    return;
  }
  // returns h -> x inside the window: slots [b0, b1) of x's run [r0, r1) in
  // h's (nbr, t, id) list
  int32_t r0, r1, b0, b1;
  nbr_range(g.onnbr, hs, he, x, r0, r1);
  b0 = b1 = r0;
  if (r1 > r0) after_edge_upto(g.ont, g.oneid, r0, r1, ta, a, (int64_t)ta + delta, b0, b1);
  L[a] = (q1 - q0) - (b1 - b0);
  // smaller windows: the prefix of the window within their delta (delta
  // counting: only the legs whose second edge is new)
#pragma unroll
  for (int i = 0; i < NS; ++i)
    if (i < sub.n && sub.gs_from[i]) {
      const int32_t di = sub.delta[i];
      const int32_t q1i = upper_t(g.ot, q0, q1, (int64_t)ta + di);
      if (g.new_from == 0) {
        sub.gs_from[i][a] = (q1i - q0) - (upper_t(g.ont, b0, b1, (int64_t)ta + di) - b0);
      } else {
        const int32_t qn = after_edge(g.ot, g.oeid, q0, q1i, g.t_new, g.new_from - 1);
        int32_t back = 0;
        if (qn < q1i && b1 > b0) {
          const int32_t bn = after_edge(g.ont, g.oneid, b0, b1, g.t_new, g.new_from - 1);
          back = upper_t(g.ont, bn, b1, (int64_t)ta + di) - bn;
        }
        sub.gs_from[i][a] = (q1i - qn) - back;
      }
    }
  if (L_new) {
    const int32_t qn = after_edge(g.ot, g.oeid, q0, q1, g.t_new, g.new_from - 1);
    int32_t back = 0;
    if (qn < q1 && b1 > b0) back = b1 - after_edge(g.ont, g.oneid, b0, b1, g.t_new, g.new_from - 1);
    L_new[a] = (q1 - qn) - back;
  }
  if (!L2) return;
  const int4 an = close_here ? close_anchor(g, a, x, h, ta, delta, anc)
                             : *reinterpret_cast<const int4*>(anc + a);
  const int2 cr = make_int2(an.x, an.y), cl = make_int2(an.z, an.w);
  const int32_t qc = cycle_bound(g, cr, cl, q0, q1);
  qcb[a] = qc;
  int32_t back = 0;
  if (qc > q0 && b1 > b0)  // returns h -> src(a) among the slots [q0, qc)
    back = after_edge(g.ont, g.oneid, b0, b1, cl.x, cl.y - 1) - b0;
  L2[a] = (qc - q0) - back;
}

template <int NS>
__global__ void __launch_bounds__(512, 4) k_leg_count(GraphView g, int32_t delta,
                                                   int32_t* __restrict__ L,
                                                   AnchorRec* __restrict__ anc,
                                                   int close_here,
                                                   int32_t* __restrict__ L2,
                                                   int32_t* __restrict__ L_new,
                                                   int2* __restrict__ qwin,
                                                   int32_t* __restrict__ qcb,
                                                   SubWindows sub, ZeroSink Z) {
  const int64_t a64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a64 >= g.E) return;
  leg_count_item<NS>(g, delta, (int32_t)a64, L, anc, close_here, L2, L_new, qwin, qcb, sub, Z);
}

// legs ending with each edge, by binary search (when no legs are emitted)
__global__ void __launch_bounds__(512) k_gs_into(GraphView g, int32_t delta,
                                                 int32_t* __restrict__ gs_in) {
  int64_t b64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b64 >= g.E) return;
  int32_t b = (int32_t)b64;
  // delta counting: a leg (a, b) is new iff b is new
  gs_in[b] = (g.src[b] == g.dst[b] || b < g.new_from) ? 0 : legs_into(g, b, delta);
}

// --------------------------------------------------------- leg emission
//
// A leg (a, b) of a scatter-gather candidate is filed under its (source,
// destination) pair s*N + d.  Pairs are spread over `nb` buckets by the top
// bits of a 64-bit mix of the key (MurmurHash3's finalizer, Appleby), so a
// bucket holds about the tuned mean of legs (at most 512 on average) and
// every leg of one pair lands in one bucket.

__device__ __forceinline__ uint64_t mix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ uint32_t bucket_of(uint64_t key, int bucket_bits) {
  return bucket_bits ? (uint32_t)(mix64(key) >> (64 - bucket_bits)) : 0u;
}

__device__ __forceinline__ void put_rec(const LegSink& S, int64_t pos, uint64_t key, int32_t a,
                                        int32_t b) {
  LegRec r;
  r.key = key;
  r.a = a;
  r.b = b;
  S.rec[pos] = r;
}

__device__ __forceinline__ bool in_mask(const uint32_t* mask, int32_t v) {
  return (__ldg(mask + (v >> 5)) >> (v & 31)) & 1u;
}

// SG record of a leg: at the leg's own position, or -- when filtering by the
// destination mask -- compacted with one atomic per warp (all lanes call it)
__device__ __forceinline__ void sg_record(const LegSink& S, bool leg, int64_t pos, int32_t a,
                                          int32_t b, int32_t x, int32_t h, int32_t y, int32_t ta,
                                          int32_t tb, int64_t n_nodes, int bits) {
  const uint64_t key = (uint64_t)x * (uint64_t)n_nodes + (uint64_t)y;
  if (!S.dmask) {
    // buckets are many and the keys of a warp's legs differ, so the
    // histogram takes one plain increment per leg
    if (leg) {
      put_rec(S, pos, key, a, b);
      if (S.hist) atomicAdd(S.hist + bucket_of(key, bits), 1u);
    }
    return;
  }
  const bool keep = leg && in_mask(S.dmask, y);
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  if (!m) return;
  const int lane = threadIdx.x & 31, lead = __ffs(m) - 1;
  unsigned long long base = 0;
  if (lane == lead) base = atomicAdd(S.n_rec, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, lead);
  if (keep) put_rec(S, (int64_t)base + __popc(m & ((1u << lane) - 1u)), key, a, b);
}

// Writes every leg (a, b) of edge a at off[a]...; reciprocal edges b = h->x
// inside the window close 2-cycles (a, b) and are credited directly.  With
// gs_in, also counts the legs ending with each edge (the scatter side of GS);
// with records, also counts them into the SG buckets.  Windows of up to 32
// slots are written by their own lane; longer ones (hub accounts) by the
// whole warp, 32 slots at a time, with ballots keeping the output order.
// smaller windows: GS legs ending with b, and 2-cycles (a slot returning to
// the anchor's source), when the pair spans at most their delta (delta
// counting: when b is new)
template <int NS>
__device__ __forceinline__ void sub_leg_credit(const SubWindows& sub, bool leg, int32_t a,
                                               int32_t b, int32_t span, int32_t new_from) {
  if (b < new_from) return;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    if (i >= sub.n || span > sub.delta[i]) continue;
    if (leg) {
      if (sub.gs_in[i]) atomicAdd(sub.gs_in[i] + b, 1);
    } else if (sub.cyc2[i]) {
      atomicAdd(sub.cyc2[i] + a, 1ull);
      atomicAdd(sub.cyc2[i] + b, 1ull);
    }
  }
}

// The emission of the warp's 32 edges, a64 this lane's (g.E or beyond:
// none).  Every lane of the warp calls it together (k_leg_emit, and the
// fused mine's emission phase).
template <int NS>
__device__ __forceinline__ void leg_emit_warp(const GraphView& g, const int2* __restrict__ qwin,
                                              const int32_t* __restrict__ qcb,
                                              const int64_t* __restrict__ off, const LegSink& S,
                                              unsigned long long* __restrict__ acc_cyc2,
                                              int32_t* __restrict__ gs_in, int32_t own_max,
                                              const SubWindows& sub, int64_t a64) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  int32_t a = (int32_t)a64, x = 0, q0 = 0, q1 = 0, h = 0, ta = 0;
  int64_t o = 0;
  if (a64 < g.E) {
    x = g.src[a];
    h = g.dst[a];
    if (x != h) {
      const int2 w = qwin[a];
      q0 = w.x;
      q1 = w.y;
      o = off[a];
      ta = g.ts[a];
    }
  }
  // legs before the cycle bound can start a cycle: their records go to S.leg at
  // off2[a] + their rank among a's legs
  int32_t qc = q0;
  int64_t o2 = 0;
  if (S.leg && q1 > q0) {
    qc = qcb[a];
    o2 = S.off2[a] - o;
  }
  const bool own = q1 - q0 <= own_max;
  // Short windows (the lanes' own) are flattened over the warp: round r
  // takes slots [32r, 32r + 32) of the concatenated windows, so every lane
  // has a slot in every round but the last.  A slot's leg rank inside its
  // anchor's window = the legs its anchor had in earlier rounds (kept by
  // the anchor's lane) + the legs before it in this round.
  const unsigned full = 0xffffffffu;
  const int32_t own_len = own ? q1 - q0 : 0;
  int32_t incl = own_len;
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t y = __shfl_up_sync(full, incl, d);
    if (lane >= d) incl += y;
  }
  const int32_t excl = incl - own_len;
  const int32_t total = __shfl_sync(full, incl, 31);
  const int64_t c2 = o2 + o;  // first cycle-leg position of this lane's anchor
  int32_t run = 0;            // legs of this lane's anchor in earlier rounds
  for (int32_t base = 0; base < total; base += 32) {
    const int32_t k = base + lane;
    const bool in = k < total;
    // the lane whose window holds flattened slot k: the largest s with
    // excl_s <= k (an empty window shares the next lane's excl)
    int src = 0;
    for (int step = 16; step > 0; step >>= 1) {
      const int t = src + step;
      if (__shfl_sync(full, excl, t) <= k) src = t;
    }
    const int32_t sa = __shfl_sync(full, a, src);
    const int32_t sx = __shfl_sync(full, x, src);
    const int32_t sh = __shfl_sync(full, h, src);
    const int32_t sta = __shfl_sync(full, ta, src);
    const int32_t sqc = __shfl_sync(full, qc, src);
    const int32_t sq = __shfl_sync(full, q0, src) + (k - __shfl_sync(full, excl, src));
    const int64_t so = __shfl_sync(full, o, src);
    const int64_t sc2 = __shfl_sync(full, c2, src);
    const int32_t srun = __shfl_sync(full, run, src);
    const int32_t y = in ? __ldg(g.onbr + sq) : sx;
    const int32_t b = in ? __ldg(g.oeid + sq) : 0;
    const int32_t tb = in ? __ldg(g.ot + sq) : 0;
    const bool leg = in && y != sx;
    const unsigned peers = __match_any_sync(full, in ? src : 32 + lane);
    const unsigned lm = __ballot_sync(full, leg);
    const int32_t rank = srun + __popc(lm & peers & lt);
    if (S.rec) sg_record(S, leg, so + rank, sa, b, sx, sh, y, sta, tb, g.N, S.bits);
    if (NS > 0 && in) sub_leg_credit<NS>(sub, leg, sa, b, tb - sta, g.new_from);
    if (leg) {
      if (gs_in && b >= g.new_from) atomicAdd(gs_in + b, 1);
      if (S.leg && sq < sqc) S.leg[sc2 + rank] = make_int4(sa, b, y, tb);
    } else if (in && acc_cyc2 && b >= g.new_from) {  // a return: a 2-cycle
      atomicAdd(acc_cyc2 + b, 1ull);
      atomicAdd(acc_cyc2 + sa, 1ull);
    }
    // every lane's anchor adds its legs of this round (read from a lane
    // that held one of its slots: the first, at max(excl, base) - base)
    const int32_t cnt = __popc(lm & peers);
    const bool mine = own_len > 0 && excl < base + 32 && incl > base;
    const int32_t add = __shfl_sync(full, cnt, mine ? max(excl, base) - base : lane);
    if (mine) run += add;
  }
  unsigned heavy = __ballot_sync(0xffffffffu, !own);
  while (heavy) {
    const int src = __ffs(heavy) - 1;
    heavy &= heavy - 1;
    const int32_t ha = __shfl_sync(0xffffffffu, a, src);
    const int32_t hx = __shfl_sync(0xffffffffu, x, src);
    const int32_t hh = __shfl_sync(0xffffffffu, h, src);
    const int32_t hta = __shfl_sync(0xffffffffu, ta, src);
    const int32_t hqc = __shfl_sync(0xffffffffu, qc, src);
    const int64_t ho2 = __shfl_sync(0xffffffffu, o2, src);
    const int32_t hq1 = __shfl_sync(0xffffffffu, q1, src);
    int32_t base = __shfl_sync(0xffffffffu, q0, src);
    int64_t ho = __shfl_sync(0xffffffffu, o, src);
    unsigned long long hc2 = 0;
    for (; base < hq1; base += 32) {
      const int32_t q = base + lane;
      const bool in = q < hq1;
      const int32_t y = in ? __ldg(g.onbr + q) : hx;
      const int32_t b = in ? __ldg(g.oeid + q) : 0;
      const bool leg = in && y != hx;
      const unsigned m = __ballot_sync(0xffffffffu, leg);
      const int32_t tb = in ? __ldg(g.ot + q) : 0;
      if (S.rec) sg_record(S, leg, ho + __popc(m & lt), ha, b, hx, hh, y, hta, tb, g.N, S.bits);
      if (NS > 0 && in) sub_leg_credit<NS>(sub, leg, ha, b, tb - hta, g.new_from);
      if (leg) {
        if (gs_in && b >= g.new_from) atomicAdd(gs_in + b, 1);
      } else if (in && acc_cyc2 && b >= g.new_from) {
        atomicAdd(acc_cyc2 + b, 1ull);
        ++hc2;
      }
      if (S.leg && leg && q < hqc) S.leg[ho2 + ho + __popc(m & lt)] = make_int4(ha, b, y, tb);
      ho += __popc(m);
    }
    if (acc_cyc2) {
      for (int sh = 16; sh > 0; sh >>= 1) hc2 += __shfl_down_sync(0xffffffffu, hc2, sh);
      if (lane == 0 && hc2) atomicAdd(acc_cyc2 + ha, hc2);
    }
  }
}

template <int NS>
__global__ void __launch_bounds__(512, 3) k_leg_emit(GraphView g, const int2* __restrict__ qwin,
                                                  const int32_t* __restrict__ qcb,
                                                  const int64_t* __restrict__ off, LegSink S,
                                                  unsigned long long* __restrict__ acc_cyc2,
                                                  int32_t* __restrict__ gs_in, int32_t own_max,
                                                  SubWindows sub) {
  leg_emit_warp<NS>(g, qwin, qcb, off, S, acc_cyc2, gs_in, own_max, sub,
                    (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------- legs for delta counting
//
// A streaming recount counts only the instances whose latest edge is new
// (id >= new_from; the newest edges of every list).  Of anchor a's legs
// (a, b), b in the window [q0, q1) of dst(a)'s out-list:
//   new legs, b in the list's new suffix [qn, q1): GS and 2-cycle credits,
//     sub-window credits, and SG records (their destination is a batch
//     destination by definition);
//   old legs: only SG records into a batch destination (the other leg of
//     the pair may be new), found in the list's marked slots (those whose
//     counterparty is a batch destination) inside [q0, qn);
//   the cycle legs [q0, qc), whose anchors have a new closing edge.
// So the old part of a hub's window is walked only where it can matter.
// Used while the marked slots are a small share of all (few batch
// destinations); otherwise walking every window contiguously (k_leg_emit)
// is faster than visiting most slots through the marked list.

// flag of every out-list slot whose counterparty is in the mask
__global__ void k_mark_slots(const int32_t* __restrict__ nbr, int64_t Ev,
                             const uint32_t* __restrict__ mask, int32_t* __restrict__ flag) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p <= Ev) flag[p] = p < Ev && in_mask(mask, nbr[p]);
}

// marked slots, compacted in slot order, and each node's range of them
__global__ void k_compact_marked(const int32_t* __restrict__ flag_scan, int64_t Ev,
                                 int32_t* __restrict__ mslot) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < Ev && flag_scan[p + 1] != flag_scan[p]) mslot[flag_scan[p]] = (int32_t)p;
}

__global__ void k_marked_ptr(const int32_t* __restrict__ optr, const int32_t* __restrict__ flag_scan,
                             int32_t N, int32_t* __restrict__ mptr) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u <= N) mptr[u] = flag_scan[optr[u]];
}

// first i in [lo, hi) with v[i] >= x
__device__ __forceinline__ int32_t lower_i32(const int32_t* __restrict__ v, int32_t lo, int32_t hi,
                                             int32_t x) {
  while (lo < hi) {
    const int32_t mid = (int32_t)(((uint32_t)lo + (uint32_t)hi) >> 1);
    if (__ldg(v + mid) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// first slot of every out-list holding a new edge (new edges are the
// newest, so they end every list)
__global__ void k_first_new(const int32_t* __restrict__ optr, const int32_t* __restrict__ oeid,
                            int32_t N, int32_t new_from, int32_t* __restrict__ first_new) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < N) first_new[u] = lower_i32(oeid, optr[u], optr[u + 1], new_from);
}

// f(owner lane, position or -1) over every lane's range [lo, hi), called by
// all 32 lanes together: ranges up to own_max long one position per lane per
// round, longer ones by the whole warp, one owner after another
template <typename F>
__device__ __forceinline__ void warp_ranges(int32_t lo, int32_t hi, int32_t own_max, F&& f) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const bool own = hi - lo <= own_max;
  int32_t q = lo;
  while (__any_sync(full, own && q < hi)) {
    const bool in = own && q < hi;
    f(lane, in ? q : -1);
    if (in) ++q;
  }
  unsigned heavy = __ballot_sync(full, !own && hi > lo);
  while (heavy) {
    const int src = __ffs(heavy) - 1;
    heavy &= heavy - 1;
    const int32_t hlo = __shfl_sync(full, lo, src), hhi = __shfl_sync(full, hi, src);
    for (int32_t base = hlo; base < hhi; base += 32) f(src, base + lane < hhi ? base + lane : -1);
  }
}

template <int NS>
__global__ void __launch_bounds__(512, 3) k_leg_emit_delta(
    GraphView g, const int2* __restrict__ qwin, const int32_t* __restrict__ qcb, LegSink S,
    unsigned long long* __restrict__ acc_cyc2, int32_t* __restrict__ gs_in, int32_t own_max,
    SubWindows sub, const int32_t* __restrict__ first_new, const int32_t* __restrict__ mptr,
    const int32_t* __restrict__ mslot) {
  const unsigned full = 0xffffffffu;
  const int64_t a64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  int32_t a = (int32_t)a64, x = 0, h = 0, ta = 0, q0 = 0, q1 = 0, qn = 0, qc = 0, m0 = 0, m1 = 0;
  int64_t c2 = 0;
  if (a64 < g.E) {
    x = g.src[a];
    h = g.dst[a];
    if (x != h) {
      const int2 w = qwin[a];
      q0 = qn = qc = w.x;
      q1 = w.y;
      if (q1 > q0) {
        ta = g.ts[a];
        qn = min(max(__ldg(first_new + h), q0), q1);
        if (S.leg) {
          qc = qcb[a];
          c2 = S.off2[a];
        }
        if (S.rec && qn > q0) {
          const int32_t lo = mptr[h], hi = mptr[h + 1];
          m0 = lower_i32(mslot, lo, hi, q0);
          m1 = lower_i32(mslot, m0, hi, qn);
        }
      }
    }
  }
  // new legs and returns
  warp_ranges(qn, q1, own_max, [&](int src, int32_t q) {
    const int32_t sa = __shfl_sync(full, a, src), sx = __shfl_sync(full, x, src);
    const int32_t sh = __shfl_sync(full, h, src), sta = __shfl_sync(full, ta, src);
    const bool in = q >= 0;
    const int32_t y = in ? __ldg(g.onbr + q) : sx;
    const int32_t b = in ? __ldg(g.oeid + q) : 0;
    const int32_t tb = in ? __ldg(g.ot + q) : 0;
    const bool leg = in && y != sx;
    if (S.rec) sg_record(S, leg, 0, sa, b, sx, sh, y, sta, tb, g.N, S.bits);
    if (NS > 0 && in) sub_leg_credit<NS>(sub, leg, sa, b, tb - sta, g.new_from);
    if (leg) {
      if (gs_in) atomicAdd(gs_in + b, 1);
    } else if (in && acc_cyc2) {  // a return: a 2-cycle
      atomicAdd(acc_cyc2 + b, 1ull);
      atomicAdd(acc_cyc2 + sa, 1ull);
    }
  });
  // old legs into a batch destination
  if (S.rec)
    warp_ranges(m0, m1, own_max, [&](int src, int32_t i) {
      const int32_t sa = __shfl_sync(full, a, src), sx = __shfl_sync(full, x, src);
      const int32_t sh = __shfl_sync(full, h, src), sta = __shfl_sync(full, ta, src);
      const bool in = i >= 0;
      const int32_t q = in ? __ldg(mslot + i) : 0;
      const int32_t y = in ? __ldg(g.onbr + q) : sx;
      const int32_t b = in ? __ldg(g.oeid + q) : 0;
      const int32_t tb = in ? __ldg(g.ot + q) : 0;
      sg_record(S, in && y != sx, 0, sa, b, sx, sh, y, sta, tb, g.N, S.bits);
    });
  if (!S.leg) return;
  // cycle legs: the legs in [q0, qc), at off2[a] + their rank
  const bool own = qc - q0 <= own_max;
  int32_t q = q0;
  int64_t rank = 0;
  while (__any_sync(full, own && q < qc)) {
    if (own && q < qc) {
      const int32_t y = __ldg(g.onbr + q);
      if (y != x) {
        S.leg[c2 + rank] = make_int4(a, __ldg(g.oeid + q), y, __ldg(g.ot + q));
        ++rank;
      }
      ++q;
    }
  }
  unsigned heavy = __ballot_sync(full, !own && qc > q0);
  while (heavy) {
    const int src = __ffs(heavy) - 1;
    heavy &= heavy - 1;
    const int32_t ha = __shfl_sync(full, a, src), hx = __shfl_sync(full, x, src);
    const int32_t hq0 = __shfl_sync(full, q0, src), hqc = __shfl_sync(full, qc, src);
    const int64_t hc2 = __shfl_sync(full, c2, src);
    int64_t r = 0;
    for (int32_t base = hq0; base < hqc; base += 32) {
      const int32_t qq = base + lane;
      const bool in = qq < hqc;
      const int32_t y = in ? __ldg(g.onbr + qq) : hx;
      const bool leg = in && y != hx;
      const unsigned m = __ballot_sync(full, leg);
      if (leg)
        S.leg[hc2 + r + __popc(m & lt)] = make_int4(ha, __ldg(g.oeid + qq), y, __ldg(g.ot + qq));
      r += __popc(m);
    }
  }
}

// --------------------------------------------------------- scatter-gather
//
// Every SG instance is two legs of one (s, d) pair with different
// intermediaries whose four edges span at most delta; it is credited to the
// four edges (each leg credits its own two edges once per partner leg).
// After emission the leg records are moved into their buckets; then one
// block per bucket groups its records by key in a shared-memory hash table
// and counts, for every record of a group of two or more, its partners.

// bucket histogram of compacted records (delta counting)
// Delta counting: a pair of legs counts only with a new gather edge, and
// both legs of a pair share their (s, d) key, so only the records whose key
// has a new leg need grouping.  Those keys go into an open-addressing set
// (linear probing, at least twice the keys' slots, ~0 = empty); the
// histogram and the partition keep only the records whose key it holds.
__device__ __forceinline__ bool keyset_has(const KeySet& ks, uint64_t key) {
  uint64_t h = mix64(key) & ks.mask;
  for (uint64_t probe = 0; probe <= ks.mask; ++probe) {
    const unsigned long long v = __ldg(ks.tab + h);
    if (v == key) return true;
    if (v == ~0ull) return false;
    h = (h + 1) & ks.mask;
  }
  return false;
}

// new legs among the records (to size the key set)
__global__ void __launch_bounds__(256) k_sg_count_new(const LegRec* __restrict__ rec, int64_t n,
                                                      int32_t new_from,
                                                      unsigned long long* __restrict__ count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned m = __ballot_sync(0xffffffffu, i < n && rec[i].b >= new_from);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(count, (unsigned long long)__popc(m));
}

__global__ void __launch_bounds__(256) k_sg_new_keys(const LegRec* __restrict__ rec, int64_t n,
                                                     int32_t new_from, KeySet ks) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || rec[i].b < new_from) return;
  const unsigned long long key = rec[i].key;
  uint64_t h = mix64(key) & ks.mask;
  for (uint64_t probe = 0; probe <= ks.mask; ++probe) {
    const unsigned long long old = atomicCAS(ks.tab + h, ~0ull, key);
    if (old == ~0ull || old == key) return;
    h = (h + 1) & ks.mask;
  }
}

// (ks.tab null: every record)
__global__ void __launch_bounds__(256) k_sg_hist(const LegRec* __restrict__ rec, int64_t n,
                                                 int bits, KeySet ks,
                                                 uint32_t* __restrict__ hist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t key = rec[i].key;
  if (!ks.tab || keyset_has(ks, key)) atomicAdd(hist + bucket_of(key, bits), 1u);
}

// mask bit v set for v = node_of[e], e in [from, E)
__global__ void __launch_bounds__(256) k_mark_nodes(const int32_t* __restrict__ node_of,
                                                    int64_t from, int64_t E,
                                                    uint32_t* __restrict__ mask) {
  const int64_t e = from + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int32_t v = node_of[e];
  atomicOr(mask + (v >> 5), 1u << (v & 31));
}

// SG_PART_ITEMS independent records per thread keep several cursor atomics
// in flight at once (the kernel is bound by their latency)
// (skip: a device error word; when it is set the records may be unwritten
// and nothing is moved)
__global__ void __launch_bounds__(256) k_sg_partition(const LegRec* __restrict__ rec, int64_t n,
                                                      int bits, KeySet ks,
                                                      uint32_t* __restrict__ cursor,
                                                      LegRec* __restrict__ out,
                                                      const uint32_t* __restrict__ skip) {
  if (skip && *(volatile const uint32_t*)skip) return;
  const int64_t base = (int64_t)blockIdx.x * blockDim.x * SG_PART_ITEMS + threadIdx.x;
  LegRec r[SG_PART_ITEMS];
  uint32_t bkt[SG_PART_ITEMS];
  int64_t pos[SG_PART_ITEMS];
#pragma unroll
  for (int k = 0; k < SG_PART_ITEMS; ++k) {
    const int64_t i = base + (int64_t)k * blockDim.x;
    if (i < n) {
      r[k] = rec[i];
      bkt[k] = bucket_of(r[k].key, bits);
    }
  }
  bool take[SG_PART_ITEMS];
#pragma unroll
  for (int k = 0; k < SG_PART_ITEMS; ++k)
    take[k] = base + (int64_t)k * blockDim.x < n && (!ks.tab || keyset_has(ks, r[k].key));
#pragma unroll
  for (int k = 0; k < SG_PART_ITEMS; ++k)
    if (take[k]) pos[k] = atomicAdd(cursor + bkt[k], 1u);
#pragma unroll
  for (int k = 0; k < SG_PART_ITEMS; ++k)
    if (take[k]) out[pos[k]] = r[k];
}


// c instances credited to the leg's two edges
__device__ __forceinline__ void sg_credit(unsigned long long* acc, int32_t a, int32_t b,
                                          unsigned long long c) {
  if (c) {
    atomicAdd(acc + a, c);
    atomicAdd(acc + b, c);
  }
}

// (intermediary, scatter time, gather time, gather edge) of a leg; dts[a] =
// (dst[a], ts[a]), so the scatter edge's two values come in one sector
__device__ __forceinline__ int4 leg_info(const LegRec& r, const int2* dts, const int32_t* ts) {
  const int2 sa = __ldg(dts + r.a);
  return make_int4(sa.x, sa.y, __ldg(ts + r.b), r.b);
}

__global__ void __launch_bounds__(256) k_pack_dst_ts(const int32_t* __restrict__ dst,
                                                     const int32_t* __restrict__ ts, int64_t E,
                                                     int2* __restrict__ dts) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < E) dts[e] = make_int2(dst[e], ts[e]);
}

// two legs of one (s, d) key form an SG instance within a window when their
// intermediaries differ (which also excludes the leg itself) and all four
// edges lie within its delta; delta counting keeps the pairs whose latest
// edge -- one of the two gather edges -- is new.  The span of the pair, or
// INT64_MAX when it is no instance at all.
__device__ __forceinline__ int64_t sg_span(const int4& r, const int4& o, int32_t new_from) {
  if (o.x == r.x || max(r.w, o.w) < new_from) return INT64_MAX;
  return (int64_t)max(r.z, o.z) - (int64_t)min(r.y, o.y);
}

// sg_span in 32-bit arithmetic: the latest minus the earliest of int32 times
// lies in [0, 2^32), exact as uint32; UINT32_MAX when the pair is no
// instance (or spans 2^32 - 1 seconds: above every window either way)
__device__ __forceinline__ uint32_t sg_span32(const int4& r, const int4& o, int32_t new_from) {
  if (o.x == r.x || max(r.w, o.w) < new_from) return 0xffffffffu;
  return (uint32_t)max(r.z, o.z) - (uint32_t)min(r.y, o.y);
}

// partners of `own` among group entries [j0, j1), per window, credited to
// the leg's two edges (DC: delta counting, pairs need a new gather edge)
template <int NS, bool DC>
__device__ __forceinline__ void sg_count_partners(const int4* grp, uint32_t j0, uint32_t j1,
                                                  const int4& own, int32_t a,
                                                  int32_t delta, int32_t new_from,
                                                  unsigned long long* acc,
                                                  const SubWindows& sub) {
  uint32_t k = 0, ks[NS > 0 ? NS : 1] = {};  // at most CAP partners
  for (uint32_t j = j0; j < j1; ++j) {
    const uint32_t span = sg_span32(own, grp[j], DC ? new_from : 0);
    if (span > (uint32_t)delta) continue;
    ++k;
#pragma unroll
    for (int i = 0; i < NS; ++i)
      if (i < sub.n && span <= (uint32_t)sub.delta[i]) ++ks[i];
  }
  if (acc) sg_credit(acc, a, own.w, k);
#pragma unroll
  for (int i = 0; i < NS; ++i)
    if (i < sub.n && sub.sg[i]) sg_credit(sub.sg[i], a, own.w, ks[i]);
}

// table slot of a key inside its bucket: a 32-bit mix of both halves (the
// keys of one bucket already share the top bits of mix64, which picked it)
__device__ __forceinline__ uint32_t slot_hash(uint64_t key) {
  uint32_t h = (uint32_t)key * 0x9e3779b1u ^ (uint32_t)(key >> 32) * 0x85ebca77u;
  return h ^ (h >> 15);
}

// Groups one bucket's records by key in a shared-memory hash table and
// credits every leg of a group of two or more with its partners.  CAP
// records at most; tab = a power of two >= 2n.  The thread that files a key
// first leads its group: once the counts are known it reserves the group's
// range of the group array with one block atomic, so no scan over the
// table is needed.  Then the grouped legs' data are filed group by group
// and consecutive threads take consecutive group members (a warp's threads
// mostly walk the same group).
// Groups are laid out by size class (2-4, 5-16, 17-64, more legs), so that
// the threads of a warp, which take consecutive group entries and walk
// their own group, walk groups of about one length.
constexpr int SG_CLASSES = 4;
__device__ __forceinline__ int sg_class(uint32_t c) {
  return c <= 4 ? 0 : c <= 16 ? 1 : c <= 64 ? 2 : 3;
}

template <int CAP, int TAB>
struct SgSmem {
  int4 grp[CAP];                 // leg_info of grouped legs, by group
  int32_t ga[CAP];               // the scatter edge a of each group entry
  uint16_t gslot[CAP];           // the table slot (group) of each group entry
  unsigned long long key[TAB];   // filed keys; later (as uint32) group cursors
  uint32_t cnt[TAB];             // records per slot
  uint32_t n_grouped;
  uint32_t cls_n[SG_CLASSES];    // grouped legs per size class, then the class's start
  uint32_t n_big;                // groups counted by sorting (sg_sorted_group)
  uint32_t n_valid;              // legs within the window being counted there
  uint32_t big_start[CAP / 64], big_n[CAP / 64];
};

// Groups of more than SG_SORT_MIN legs are counted by sorting instead of
// comparing every pair (overflow buckets, full mines)
constexpr uint32_t SG_SORT_MIN = 64;

// ascending bitonic sort of a[0, n) and, independently, b[0, n) (n a power
// of two), by the whole block; one barrier per stage for both
template <typename T>
__device__ __forceinline__ void bitonic_sort2(T* a, T* b, uint32_t n) {
  for (uint32_t k = 2; k <= n; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const T x = a[i], y = a[l];
          if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
          }
          const T u = b[i], v = b[l];
          if ((u > v) == up) {
            b[i] = v;
            b[l] = u;
          }
        }
      }
      __syncthreads();
    }
}

// first i in [lo, hi) with a[i] >= x (upper: a[i] > x)
template <typename T, typename K>
__device__ __forceinline__ uint32_t bound_in(const T* a, uint32_t lo, uint32_t hi, K x,
                                             bool upper) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const K v = (K)a[mid];
    if (v < x || (upper && v == x)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// an int32 time as an unsigned key of the same order
__device__ __forceinline__ unsigned long long tkey(long long t) {
  return (unsigned long long)((uint32_t)(int32_t)t ^ 0x80000000u);
}

// Partners of every leg of one (s, d) group of c legs, grp[start, start + c),
// without comparing all pairs.  For a window dw and the legs U whose own
// span is within dw, a leg i of U has span(i, j) <= dw with exactly the legs
// j of U that start at or after tb_i - dw, except those that end after
// ta_i + dw (every such leg starts after ta_i, so it was among the former):
// two counts in U's start and end times, sorted.  The legs of U through i's
// own intermediary (i included) are counted the same way in U's (m, start)
// and (m, end) keys, sorted, and subtracted.  Full mines only (no delta
// counting).
template <int CAP, int TAB, int NS>
__device__ __forceinline__ void sg_sorted_group(SgSmem<CAP, TAB>& S, uint32_t start, uint32_t c,
                                                int32_t delta,
                                                unsigned long long* __restrict__ acc,
                                                const SubWindows& sub) {
  static_assert(TAB >= 2 * CAP, "the sort buffers live in the hash table's space");
  int32_t* sa = reinterpret_cast<int32_t*>(S.key);  // start times of U
  int32_t* sb = sa + CAP;                            // end times of U
  unsigned long long* ka = S.key + CAP;               // (m, start) of U, then ~0
  unsigned long long* kb = reinterpret_cast<unsigned long long*>(S.cnt);  // (m, end)
  const int4* grp = S.grp + start;
  constexpr int NT = 1 + NS;
#pragma unroll
  for (int w = 0; w < NT; ++w) {
    if (w > 0 && w - 1 >= sub.n) break;
    unsigned long long* col = w == 0 ? acc : sub.sg[w - 1];
    if (!col) continue;
    const long long dw = w == 0 ? delta : sub.delta[w - 1];
    if (threadIdx.x == 0) S.n_valid = 0;
    __syncthreads();
    // U compacted to the front (any order: it is sorted next), the rest of
    // the next power of two padded with keys that sort last
    for (uint32_t k = threadIdx.x; k < c; k += blockDim.x) {
      const int4 r = grp[k];
      if ((long long)r.z - r.y > dw) continue;
      const uint32_t at = atomicAdd(&S.n_valid, 1u);
      const unsigned long long m = (unsigned long long)(uint32_t)r.x << 32;
      sa[at] = r.y;
      sb[at] = r.z;
      ka[at] = m | tkey(r.y);
      kb[at] = m | tkey(r.z);
    }
    __syncthreads();
    const uint32_t nw = S.n_valid;  // |U|: the first nw entries of every array
    if (nw < 2) continue;           // no pair within this window (uniform: nw is shared)
    uint32_t pw = 1;
    while (pw < nw) pw <<= 1;
    for (uint32_t k = nw + threadIdx.x; k < pw; k += blockDim.x) {
      sa[k] = INT32_MAX;
      sb[k] = INT32_MAX;
      ka[k] = ~0ull;
      kb[k] = ~0ull;
    }
    __syncthreads();
    bitonic_sort2(sa, sb, pw);
    bitonic_sort2(ka, kb, pw);
    for (uint32_t k = threadIdx.x; k < c; k += blockDim.x) {
      const int4 r = grp[k];
      if ((long long)r.z - r.y > dw) continue;
      const long long x = (long long)r.z - dw, y = (long long)r.y + dw;
      // legs of U with start >= x, minus those with end > y
      const uint32_t all = (nw - bound_in<int32_t, long long>(sa, 0, nw, x, false)) -
                           (nw - bound_in<int32_t, long long>(sb, 0, nw, y, true));
      // the same within i's intermediary's run of the (m, time) keys
      const unsigned long long m = (unsigned long long)(uint32_t)r.x << 32;
      const uint32_t a0 = bound_in(ka, 0, nw, m, false);
      const uint32_t a1 = bound_in(ka, a0, nw, m + (1ull << 32), false);
      const uint32_t b0 = bound_in(kb, 0, nw, m, false);
      const uint32_t b1 = bound_in(kb, b0, nw, m + (1ull << 32), false);
      const uint32_t ge = x <= INT32_MIN ? a1 - a0
                        : x > INT32_MAX  ? 0u
                                         : a1 - bound_in(ka, a0, a1, m | tkey(x), false);
      const uint32_t gt = y >= INT32_MAX ? 0u
                        : y < INT32_MIN  ? b1 - b0
                                         : b1 - bound_in(kb, b0, b1, m | tkey(y), true);
      sg_credit(col, S.ga[start + k], r.w, (unsigned long long)(all - (ge - gt)));
    }
    __syncthreads();  // the next window rewrites the buffers
  }
}

template <int CAP, int TAB, int NS, int BS, bool SORT_BIG = false>
__device__ __forceinline__ void sg_group_bucket(SgSmem<CAP, TAB>& S, const LegRec* __restrict__ R, int n,
                                int32_t delta, const int2* __restrict__ dts,
                                const int32_t* __restrict__ ts,
                                unsigned long long* __restrict__ acc, int32_t new_from,
                                const SubWindows& sub) {
  constexpr int PER = (CAP + BS - 1) / BS;  // records per thread (blocks of BS)
  uint32_t* cur = reinterpret_cast<uint32_t*>(S.key);
  // this thread's records stay in registers from the first read on
  LegRec r[PER];
  int any_new = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int i = threadIdx.x + k * BS;
    if (i < n) {
      r[k] = R[i];
      any_new |= r[k].b >= new_from;
    }
  }
  // delta counting: a pair counts only with a new gather edge, and both legs
  // of a pair share a key, hence a bucket: a bucket without new legs has
  // nothing to count
  if (new_from > 0 && !__syncthreads_or(any_new)) return;
  int tab = 64;
  while (tab < 2 * n) tab <<= 1;
  for (int t = threadIdx.x; t < tab; t += BS) {
    S.key[t] = ~0ull;
    S.cnt[t] = 0;
  }
  if (threadIdx.x < SG_CLASSES) S.cls_n[threadIdx.x] = 0;
  if (threadIdx.x == 0) S.n_big = 0;
  __syncthreads();
  // file every record under its key; remember which keys this thread filed
  uint32_t lead = 0;
  uint16_t h[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    if (threadIdx.x + k * BS >= n) break;
    const unsigned long long key = r[k].key;
    uint32_t q = slot_hash(key) & (uint32_t)(tab - 1);
    for (int probe = 0; probe < tab; ++probe) {  // n < tab: a slot is always found
      const unsigned long long cur_key = S.key[q];
      if (cur_key == key) break;
      if (cur_key == ~0ull) {
        const unsigned long long old = atomicCAS(&S.key[q], ~0ull, key);
        if (old == ~0ull) {
          lead |= 1u << k;
          break;
        }
        if (old == key) break;
      }
      q = (q + 1) & (uint32_t)(tab - 1);
    }
    h[k] = (uint16_t)q;
    atomicAdd(&S.cnt[q], 1u);
  }
  __syncthreads();
  // group leaders reserve their group's range inside its size class (keys
  // are no longer read); the classes' starts follow
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    if (threadIdx.x + k * BS >= n) break;
    if ((lead >> k) & 1u) {
      const uint32_t c = S.cnt[h[k]];
      if (c >= 2) cur[h[k]] = atomicAdd(&S.cls_n[sg_class(c)], c);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t at = 0;
    for (int q = 0; q < SG_CLASSES; ++q) {
      const uint32_t m = S.cls_n[q];
      S.cls_n[q] = at;
      at += m;
    }
    S.n_grouped = at;
  }
  __syncthreads();
  const uint32_t n_grouped = S.n_grouped;
  if (n_grouped == 0) return;
  // the grouped legs' data, group by group (cursor ends at the group's end
  // within its class)
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    if (threadIdx.x + k * BS >= n) break;
    const uint32_t c = S.cnt[h[k]];
    if (c >= 2) {
      const uint32_t at = S.cls_n[sg_class(c)] + atomicAdd(&cur[h[k]], 1u);
      S.grp[at] = leg_info(r[k], dts, ts);
      S.ga[at] = r[k].a;
      S.gslot[at] = h[k];
    }
  }
  const bool sort_big = SORT_BIG && new_from == 0;
  if constexpr (NS <= 1 && 2 * CAP <= TAB) {
    // Every unordered pair once: entry i of a group of c walks the entries
    // 1 .. (c-1)/2 places after it, cyclically (and, for even c, the lower
    // half also the one c/2 places on), so a group's threads walk about
    // (c-1)/2 entries each; a pair within a window adds 1 to both entries'
    // counters (the key array's upper half: the cursors use its lower half).
    uint32_t* pk0 = cur + TAB;  // partners within delta
    uint32_t* pk1 = pk0 + CAP;  // partners within the sub-window
    // (the filed entries and the final cursors are read after the barrier
    // below; the counters lie outside both)
    for (uint32_t p = threadIdx.x; p < n_grouped; p += BS) {
      pk0[p] = 0;
      pk1[p] = 0;
    }
    __syncthreads();
    const uint32_t d1 = NS > 0 && sub.n > 0 ? (uint32_t)sub.delta[0] : 0u;
    for (uint32_t p = threadIdx.x; p < n_grouped; p += BS) {
      const uint32_t q = S.gslot[p];
      const uint32_t c = S.cnt[q];
      const uint32_t g0 = S.cls_n[sg_class(c)] + cur[q] - c;
      if (sort_big && c > SG_SORT_MIN) {  // listed by its first entry, counted below
        if (p == g0) {
          const uint32_t k = atomicAdd(&S.n_big, 1u);
          S.big_start[k] = g0;
          S.big_n[k] = c;
        }
        continue;
      }
      const int4 own = S.grp[p];
      const uint32_t i = p - g0;
      const uint32_t steps = (c - 1) / 2 + ((c & 1u) == 0 && i < c / 2 ? 1u : 0u);
      uint32_t k0 = 0, k1 = 0;
      uint32_t j = i;
      for (uint32_t t = 0; t < steps; ++t) {
        if (++j == c) j = 0;
        const uint32_t span = sg_span32(own, S.grp[g0 + j], new_from);
        if (span > (uint32_t)delta) continue;
        ++k0;
        atomicAdd(&pk0[g0 + j], 1u);
        if (NS > 0 && span <= d1) {
          ++k1;
          atomicAdd(&pk1[g0 + j], 1u);
        }
      }
      if (k0) atomicAdd(&pk0[p], k0);
      if (k1) atomicAdd(&pk1[p], k1);
    }
    __syncthreads();
    for (uint32_t p = threadIdx.x; p < n_grouped; p += BS) {
      const uint32_t c = S.cnt[S.gslot[p]];
      if (sort_big && c > SG_SORT_MIN) continue;
      const int32_t a = S.ga[p], b = S.grp[p].w;
      if (acc) sg_credit(acc, a, b, pk0[p]);
      if (NS > 0 && sub.n > 0 && sub.sg[0]) sg_credit(sub.sg[0], a, b, pk1[p]);
    }
  } else {
    __syncthreads();
    for (uint32_t p = threadIdx.x; p < n_grouped; p += BS) {
      const uint32_t q = S.gslot[p];
      const uint32_t c = S.cnt[q];
      const uint32_t end = S.cls_n[sg_class(c)] + cur[q];
      if (sort_big && c > SG_SORT_MIN) {  // listed by its first entry, counted below
        if (p == end - c) {
          const uint32_t k = atomicAdd(&S.n_big, 1u);
          S.big_start[k] = end - c;
          S.big_n[k] = c;
        }
        continue;
      }
      if (new_from > 0)
        sg_count_partners<NS, true>(S.grp, end - c, end, S.grp[p], S.ga[p], delta, new_from,
                                    acc, sub);
      else
        sg_count_partners<NS, false>(S.grp, end - c, end, S.grp[p], S.ga[p], delta, 0, acc,
                                     sub);
    }
  }
  if (!sort_big) return;
  __syncthreads();  // the table's space becomes the sort buffers
  const uint32_t n_big = S.n_big;
  for (uint32_t k = 0; k < n_big; ++k)
    sg_sorted_group<CAP, TAB, NS>(S, S.big_start[k], S.big_n[k], delta, acc, sub);
}

// One block per bucket of up to SG_CAP records; larger buckets are listed
// in overflow (count at overflow[0]) for k_sg_bucket_big.
template <int NS>
__global__ void __launch_bounds__(SG_BLOCK, 8) k_sg_bucket(const LegRec* __restrict__ rec,
                                                   const uint32_t* __restrict__ bend,
                                                   int32_t delta, const int2* __restrict__ dts,
                                                   const int32_t* __restrict__ ts,
                                                   unsigned long long* __restrict__ acc,
                                                   int32_t new_from,
                                                   uint32_t* __restrict__ overflow,
                                                   SubWindows sub,
                                                   const uint32_t* __restrict__ skip) {
  __shared__ SgSmem<SG_CAP, SG_TAB> S;
  // (skip set: the records and bucket ends may be unwritten; nothing is
  // grouped and no bucket is listed for k_sg_bucket_big)
  if (skip && *(volatile const uint32_t*)skip) return;
  const int64_t base = blockIdx.x ? bend[blockIdx.x - 1] : 0;
  const int64_t n = (int64_t)bend[blockIdx.x] - base;
  if (n < 2) return;
  if (n > SG_CAP) {
    if (threadIdx.x == 0) overflow[1 + atomicAdd(overflow, 1u)] = blockIdx.x;
    return;
  }
  sg_group_bucket<SG_CAP, SG_TAB, NS, SG_BLOCK>(S, rec + base, (int)n, delta, dts, ts, acc,
                                                new_from, sub);
}

// The listed buckets, a few blocks looping over the list (the count is read
// on the device); buckets beyond SG_CAP_BIG compare every record with all.
template <int NS>
__global__ void __launch_bounds__(SG_BIG_BLOCK, 1) k_sg_bucket_big(const LegRec* __restrict__ rec,
                                                       const uint32_t* __restrict__ bend,
                                                       int32_t delta,
                                                       const int2* __restrict__ dts,
                                                       const int32_t* __restrict__ ts,
                                                       unsigned long long* __restrict__ acc,
                                                       int32_t new_from,
                                                       const uint32_t* __restrict__ overflow,
                                                       SubWindows sub) {
  extern __shared__ __align__(16) unsigned char sg_big_smem[];
  auto& S = *reinterpret_cast<SgSmem<SG_CAP_BIG, SG_TAB_BIG>*>(sg_big_smem);
  const uint32_t n_over = overflow[0];
  for (uint32_t k = blockIdx.x; k < n_over; k += gridDim.x) {
    const uint32_t b = overflow[1 + k];
    const int64_t base = b ? bend[b - 1] : 0;
    const int64_t n = (int64_t)bend[b] - base;
    const LegRec* R = rec + base;
    if (n <= SG_CAP_BIG) {
      sg_group_bucket<SG_CAP_BIG, SG_TAB_BIG, NS, SG_BIG_BLOCK, true>(S, R, (int)n, delta, dts,
                                                                      ts, acc, new_from, sub);
    } else {
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const LegRec r = R[i];
        const int4 ri = leg_info(r, dts, ts);
        unsigned long long c = 0, cs[NS > 0 ? NS : 1] = {};
        for (int64_t j = 0; j < n; ++j) {
          const LegRec o = R[j];
          if (o.key != r.key) continue;
          const int64_t span = sg_span(ri, leg_info(o, dts, ts), new_from);
          if (span > delta) continue;
          ++c;
#pragma unroll
          for (int q = 0; q < NS; ++q)
            if (q < sub.n && span <= sub.delta[q]) ++cs[q];
        }
        if (acc) sg_credit(acc, r.a, r.b, c);
#pragma unroll
        for (int q = 0; q < NS; ++q)
          if (q < sub.n && sub.sg[q]) sg_credit(sub.sg[q], r.a, r.b, cs[q]);
      }
    }
    __syncthreads();  // the shared table is reused by the next bucket
  }
}


// ---------------------------------------------------------------- cycles
//
// Every cycle is enumerated once, from its earliest edge e1 = u0->u1, as a
// path of later edges that returns to u0 within t(e1) + delta (the cycle
// program of Sec. 5 / Fig. 4b: trigger, for_all expansions, and a closing
// intersection with N0.in).  The closing edges of e1 are the slots of u0's
// in-list after e1 and inside the window: one contiguous range B1, found
// per mine.  The paths are then extended level by level (all paths of j
// edges, then all of j+1), so a hub's large window is split over many
// threads instead of being walked by one.  On the way every path
//   * stops at once when B1 is empty (no cycle can start at e1),
//   * is bounded by the latest edge of B1 (a cycle's intermediate edges all
//     precede its closing edge), and
//   * closes at its end node w by matching w against B1 -- a scan of B1 when
//     it is short, two binary searches in u0's (nbr, t, id) in-list otherwise
//     (the degree-ordered intersection of Sec. 6).

// B1 of every edge a = u0 -> u1: slots of in(u0) after a with t <= t_a + delta,
// into rng and/or, with the (t, id) of B1's latest edge, u0, u1 and t_a, into
// the anchor record anc[a]: a path then reads everything it needs of its
// anchor in one sector, in one round of loads
__global__ void __launch_bounds__(512) k_close_range(GraphView g, int32_t delta,
                                                     int2* __restrict__ rng,
                                                     AnchorRec* __restrict__ anc) {
  int64_t a64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a64 >= g.E) return;
  int32_t a = (int32_t)a64;
  const int32_t u0 = g.src[a], u1 = g.dst[a], ta = g.ts[a];
  const int4 an = close_anchor(g, a, u0, u1, ta, delta, anc);
  if (rng) rng[a] = make_int2(an.x, an.y);
}


// first i in [lo, hi) with t[i] > tmax, for ranges that are usually short:
// the first eight slots are read at once (independent loads, one round of
// latency), and only a range longer than that is bisected further
__device__ __forceinline__ int32_t upper_t_short(const int32_t* __restrict__ t, int32_t lo,
                                                 int32_t hi, int64_t tmax) {
  const int32_t n = hi - lo;
  int32_t c = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (k < n && (int64_t)__ldg(t + lo + k) <= tmax) ++c;  // sorted: a prefix
  if (c < 8 || n <= 8) return lo + c;
  return upper_t(t, lo + 8, hi, tmax);
}

// Rebuilds the path of frontier element i at level j (j edges):
// edges[0..j-1] and nodes[0..j] (nodes[0] = u0 = src of the anchor), and
// *tl = the time of its last edge (read from the slot beside its id, so it
// costs no extra round of loads); with tp, also the latest time among
// edges[1..j-1] (the anchor's own time when j = 1).
// The level J and the base level (2: legs; 1: anchors, window cycles) are
// compile-time constants, so the walk unrolls and the path stays in
// registers.
template <int J, int BASE>
__device__ __forceinline__ void cyc_path(const GraphView& g, const CycFrontier& F, int64_t i,
                                         int32_t (&edges)[J], int32_t (&nodes)[J + 1],
                                         int32_t* tl, int32_t* tp = nullptr) {
  int64_t idx = i;
  int32_t t_late = INT32_MIN;
#pragma unroll
  for (int lev = J; lev > BASE; --lev) {
    const int32_t q = F.slot[lev][idx];
    edges[lev - 1] = __ldg(g.oeid + q);
    nodes[lev] = __ldg(g.onbr + q);
    if (tp || lev == J) {
      const int32_t tq = __ldg(g.ot + q);
      t_late = max(t_late, tq);
      if (lev == J) *tl = tq;
    }
    idx = F.par[lev][idx];
  }
  if constexpr (BASE == 2) {  // the leg record; nodes[0..1] come with the anchor's record
    const int4 lg = F.leg[idx];
    edges[0] = lg.x;
    edges[1] = lg.y;
    nodes[2] = lg.z;
    t_late = max(t_late, lg.w);
    if (J == 2) *tl = lg.w;
  } else {
    edges[0] = F.la[idx];
    nodes[0] = g.src[edges[0]];
    nodes[1] = g.dst[edges[0]];
    if (J == 1) *tl = g.ts[edges[0]];
  }
  if (tp) *tp = J == 1 ? g.ts[edges[0]] : t_late;
}

// One level of the cycle search.  Element i of level j is a path of j
// increasing edges from the anchor e1; the kernel checks that its last hop
// is admissible (new node, before the latest closing edge), credits the
// cycles of length j+1 that close from its end node through B1, and reports
// the window of later hops its children will take.
// WIN (window cycles): the hops only have to come after e1, in any order;
// the frontier starts at level 1 (the anchors); a cycle closes through any
// edge of B1, and a smaller window keeps it only when the path's latest edge
// also lies inside it.
// Ordered cycles read a path's anchor (closing range and bound, its two
// nodes and time) from one anchor record and the path's base leg from one
// leg record; the window of a path's children starts at qwin[last].x (the
// leg window of every edge: its end node's out-slots after it, up to its
// time + delta) with no search, and ends inside it (the latest closing edge
// is at most delta after the anchor, hence after the path's last edge).
// Window cycles read the closing ranges and search both bounds.
// Arguments of one level of the cycle search (see cyc_item).
struct CycLevelArgs {
  GraphView g;
  int32_t delta;
  int K;
  const int2* close_rng;  // window cycles
  const AnchorRec* anc;   // ordered cycles
  const int2* qwin;       // ordered cycles
  CycleSlots slots;
  unsigned long long* acc;
  int32_t close_scan_max;
};

constexpr int CLOSE_BATCH = 4;

// One element i of level j: closes its cycles and returns the window
// [*q0, *q0 + count) of its children's slots (count 0: none).
template <int NS, bool WIN, int J>
__device__ __forceinline__ int32_t cyc_item(const CycLevelArgs& A, const CycFrontier& F,
                                            const SubWindows& sub, int64_t i, int32_t* q0_out) {
  constexpr int j = J;
  const GraphView& g = A.g;
  const int32_t delta = A.delta;
  const int K = A.K;
  const bool has_next = j + 1 <= K - 1;
  int32_t edges[J];
  int32_t nodes[J + 1];
  int32_t tp = 0, tl = 0;
  cyc_path<J, WIN ? 1 : 2>(g, F, i, edges, nodes, &tl, WIN ? &tp : nullptr);
  int2 cr, cl;
  int32_t t1;
  if constexpr (WIN) {
    cr = A.close_rng[edges[0]];
    if (cr.x >= cr.y) return 0;  // e1 starts no cycle
    cl = make_int2(__ldg(g.it + cr.y - 1), __ldg(g.ieid + cr.y - 1));
    t1 = g.ts[edges[0]];
  } else {
    const int4* rec = reinterpret_cast<const int4*>(A.anc + edges[0]);
    const int4 r0 = __ldg(rec), r1 = __ldg(rec + 1);
    cr = make_int2(r0.x, r0.y);
    if (cr.x >= cr.y) return 0;  // e1 starts no cycle
    cl = make_int2(r0.z, r0.w);
    nodes[0] = r1.x;
    nodes[1] = r1.y;
    t1 = r1.z;
  }
  const int32_t t_cl = cl.x, id_cl = cl.y;
  const int32_t last = edges[j - 1];
  if (!WIN && !before(tl, last, t_cl, id_cl)) return 0;  // nothing can close after it
  const int32_t u0 = nodes[0], w = nodes[j];
  if (j >= (WIN ? 2 : 3)) {  // the hop into w must reach a new node
    if (w == u0) return 0;
#pragma unroll
    for (int m = 1; m < j; ++m)
      if (nodes[m] == w) return 0;
  }
  const CycleSlots& slots = A.slots;
  unsigned long long* acc = A.acc;
  const int32_t close_scan_max = A.close_scan_max;
  const int32_t e1 = edges[0];
  // cycles of length j+1: edges w -> u0 in B1 (after `last` unless WIN), for
  // this window and every smaller one whose delta the cycle keeps
  const int k = j + 1;
  if (k <= K && (!WIN || j >= 2)) {
    constexpr int NT = 1 + NS;
    unsigned long long* col[NT];
    int64_t tmax[NT];
    unsigned long long c[NT];
    bool any = false;
    const int64_t ta = t1;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int sl = t == 0 ? slots.slot[k] : (t - 1 < sub.n ? sub.cyc[t - 1].slot[k] : -1);
      col[t] = sl >= 0 ? acc + (int64_t)sl * g.E : nullptr;
      tmax[t] = ta + (t == 0 ? delta : (t - 1 < sub.n ? sub.delta[t - 1] : 0));
      if (WIN && tp > tmax[t]) col[t] = nullptr;  // the path already leaves window t
      c[t] = 0;
      any |= col[t] != nullptr;
    }
    if (any) {
      if (cr.y - cr.x <= close_scan_max) {
        // CLOSE_BATCH counterparties are requested before any is compared,
        // so a scan waits for one round of loads per batch, not per slot
        for (int32_t qb = cr.x; qb < cr.y; qb += CLOSE_BATCH) {
          int32_t nb[CLOSE_BATCH];
#pragma unroll
          for (int k = 0; k < CLOSE_BATCH; ++k) nb[k] = qb + k < cr.y ? __ldg(g.inbr + qb + k) : -1;
#pragma unroll
          for (int k = 0; k < CLOSE_BATCH; ++k) {
            if (nb[k] != w) continue;
            const int32_t q = qb + k;
            const int32_t cid = __ldg(g.ieid + q), tq = __ldg(g.it + q);
            if (!WIN && !before(tl, last, tq, cid)) continue;
#pragma unroll
            for (int t = 0; t < NT; ++t)
              if (col[t] && tq <= tmax[t]) {
                atomicAdd(col[t] + cid, 1ull);
                ++c[t];
              }
          }
        }
      } else {
        const int32_t in_s = g.iptr[u0], in_e = g.iptr[u0 + 1];
        int32_t r0, r1;
        nbr_range(g.innbr, in_s, in_e, w, r0, r1);
        if (r1 > r0) {
          int32_t b0, b1;
          if (WIN) after_edge_upto(g.int_, g.ineid, r0, r1, t1, e1, tmax[0], b0, b1);
          else after_edge_upto(g.int_, g.ineid, r0, r1, tl, last, tmax[0], b0, b1);
          // delta counting: only new closing edges (the scan branch's range already is)
          if (g.new_from > 0) b0 = min(after_edge(g.int_, g.ineid, b0, r1, g.t_new, g.new_from - 1), b1);
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            if (!col[t]) continue;
            const int32_t bt = t == 0 ? b1 : upper_t(g.int_, b0, b1, tmax[t]);
            for (int32_t q = b0; q < bt; ++q) atomicAdd(col[t] + __ldg(g.ineid + q), 1ull);
            c[t] = (unsigned long long)(bt - b0);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (c[t]) {
#pragma unroll
          for (int m = 0; m < j; ++m) atomicAdd(col[t] + edges[m], c[t]);
        }
    }
  }
  if (!has_next) return 0;
  int32_t q0, q1;
  if constexpr (!WIN) {
    const int2 lw = A.qwin[last];
    q0 = lw.x;
    q1 = upper_t_short(g.ot, lw.x, lw.y, t_cl);
  } else {
    const int32_t ws = g.optr[w], we = g.optr[w + 1];
    if (WIN) after_edge_upto(g.ot, g.oeid, ws, we, t1, e1, (int64_t)t1 + delta, q0, q1);
    else after_edge_upto(g.ot, g.oeid, ws, we, tl, last, t_cl, q0, q1);
  }
  *q0_out = q0;
  return q1 - q0;
}

template <int NS, bool WIN, int J>
__global__ void __launch_bounds__(512, 4) k_cyc_level(CycLevelArgs A, CycFrontier F, int64_t n,
                                                   int32_t* __restrict__ cnt,
                                                   int32_t* __restrict__ q0_out,
                                                   SubWindows sub) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t q0 = 0;
  const int32_t c = cyc_item<NS, WIN, J>(A, F, sub, i, &q0);
  if (J + 1 <= A.K - 1) {
    cnt[i] = c;
    if (c) q0_out[i] = q0;
  }
}

// calls f(std::integral_constant<int, j>) for a level j in [1, MAX_CYCLE - 1]
template <typename Fn>
__host__ __device__ __forceinline__ void level_dispatch(int j, Fn&& f) {
  switch (j) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    default: f(std::integral_constant<int, 7>{}); break;
  }
}

template <typename F>
static void nsub_dispatch(int n, F&& f) {
  if (n <= 0)
    f(std::integral_constant<int, 0>{});
  else if (n == 1)
    f(std::integral_constant<int, 1>{});
  else if (n == 2)
    f(std::integral_constant<int, 2>{});
  else
    f(std::integral_constant<int, MAX_SUB>{});
}

// ------------------------------------------- fused persistent cycle search
//
// Every level of the search above in one cooperative launch (AML_MINE_FUSED):
// the blocks stay resident and run, per level j, (1) the elements of their
// own contiguous chunk of level j (cyc_item), (2) after a grid-wide barrier,
// the prefix of their chunk's child count from all blocks' sums, and (3) the
// children of their chunk at their final positions, then a second barrier
// before level j+1 reads them.  It replaces per level the separate level,
// scan and emission launches and the count/offset arrays between them.  Each
// barrier wait is bounded by P.wait_limit SM cycles: a wait that runs out
// sets ERR_TIMEOUT in the graph's error word and the block returns (the
// others then run out at their next barrier), so a stalled launch ends with
// an error status instead of holding the GPU.  A cooperative launch keeps
// every block resident, so in normal operation no wait runs out.

constexpr int FUSED_BLOCK = 512;
constexpr int FUSED_WARP_TILE = 256;  // edges a warp takes from the fused mine's work queues

// Sense-reversing grid barrier: the last block to arrive resets the count
// and advances the generation the others wait on.  False if the wait ran out.
__device__ bool grid_wait(GridBarrier* bar, long long limit, uint32_t* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* gen = &bar->gen;
    const unsigned int g0 = *gen;
    __threadfence();
    if (atomicAdd(&bar->count, 1u) + 1u == gridDim.x) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g0) {
        if (clock64() - t0 > limit) {
          atomicOr(err, ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// sum over the block (every thread gets it)
__device__ __forceinline__ long long fused_block_sum(long long v, long long* s_w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) s_w[warp] = v;
  __syncthreads();
  long long t = 0;
  for (int w = 0; w < FUSED_BLOCK / 32; ++w) t += s_w[w];
  return t;
}

// exclusive prefix over the block in thread order; *total = the block's sum
__device__ __forceinline__ long long fused_block_excl(long long v, long long* s_w,
                                                      long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  long long before = 0, t = 0;
  for (int w = 0; w < FUSED_BLOCK / 32; ++w) {
    if (w < warp) before += s_w[w];
    t += s_w[w];
  }
  *total = t;
  return before + x - v;
}

// every level of the cycle search from the n2 cycle legs of P.F (the fused
// mine's last phase); false if a barrier wait ran out or a level outgrew its
// buffers
template <int NS>
__device__ __forceinline__ bool cyc_fused_levels(const CycLevelArgs& A, const FusedCycles& P,
                                                 const SubWindows& sub, int64_t n2,
                                                 long long* s_w) {
  const int lane = threadIdx.x & 31;
  const unsigned G = gridDim.x;
  CycFrontier F = P.F;
  int64_t n = n2;
  for (int j = 2; j <= A.K - 1 && n > 0; ++j) {
    const bool has_next = j + 1 <= A.K - 1;
    const int64_t C = (n + G - 1) / G;
    const int64_t c0 = min(n, (int64_t)blockIdx.x * C), c1 = min(n, c0 + C);
    // the level's paths from a work queue of warp tiles (the paths of a hub
    // anchor are contiguous, and a static chunk of them would set the
    // level's end); each path's child count and first child slot are stored
    const long long n_wt = (n + FUSED_WARP_TILE - 1) / FUSED_WARP_TILE;
    level_dispatch(j, [&](auto jc) {
      constexpr int JJ = decltype(jc)::value < 2 ? 2 : decltype(jc)::value;
      for (;;) {
        long long t = 0;
        if (lane == 0) t = (long long)atomicAdd(P.ctr + j, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= n_wt) break;
        for (int k = 0; k < FUSED_WARP_TILE / 32; ++k) {
          const int64_t i = t * FUSED_WARP_TILE + k * 32 + lane;
          if (i >= n) continue;
          int32_t q0 = 0;
          const int32_t c = cyc_item<NS, false, JJ>(A, F, sub, i, &q0);
          if (has_next) {
            P.cnt[i] = c;
            P.q0[i] = q0;
          }
        }
      }
    });
    if (!has_next) break;
    // the children of block b's contiguous chunk of paths, once all counts
    // are stored
    if (!grid_wait(P.bar, P.wait_limit, P.err)) return false;
    long long mine = 0;
    for (int64_t i = c0 + threadIdx.x; i < c1; i += FUSED_BLOCK) mine += __ldcg(P.cnt + i);
    mine = fused_block_sum(mine, s_w);
    if (threadIdx.x == 0) P.bsum[blockIdx.x] = mine;
    if (!grid_wait(P.bar, P.wait_limit, P.err)) return false;
    // this chunk's first child position and the level's total
    long long before = 0, total = 0;
    for (unsigned b = threadIdx.x; b < G; b += FUSED_BLOCK) {
      const long long v = __ldcg(P.bsum + b);
      total += v;
      if (b < blockIdx.x) before += v;
    }
    before = fused_block_sum(before, s_w);
    total = fused_block_sum(total, s_w);
    if (total > P.cap[j + 1]) {  // cannot happen for the sizes the capacity came from
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(P.err, ERR_OVERFLOW);
      return false;  // every block sees the same total and leaves here
    }
    int32_t* par = P.par[j + 1];
    int32_t* slot = P.slot[j + 1];
    long long run = before;
    for (int64_t t0 = c0; t0 < c1; t0 += FUSED_BLOCK) {
      const int64_t i = t0 + threadIdx.x;
      const int32_t c = i < c1 ? __ldcg(P.cnt + i) : 0;
      const int32_t b = c ? __ldcg(P.q0 + i) : 0;
      long long tile = 0;
      const long long o = run + fused_block_excl(c, s_w, &tile);
      const bool own = c <= P.own_max;  // short child lists by the lane, long ones by the warp
      if (own)
        for (int32_t k = 0; k < c; ++k) {
          par[o + k] = (int32_t)i;
          slot[o + k] = b + k;
        }
      unsigned heavy = __ballot_sync(0xffffffffu, !own);
      while (heavy) {
        const int src = __ffs(heavy) - 1;
        heavy &= heavy - 1;
        const int64_t hi = __shfl_sync(0xffffffffu, i, src);
        const int32_t hc = __shfl_sync(0xffffffffu, c, src);
        const long long ho = __shfl_sync(0xffffffffu, o, src);
        const int32_t hb = __shfl_sync(0xffffffffu, b, src);
        for (int32_t k = lane; k < hc; k += 32) {
          par[ho + k] = (int32_t)hi;
          slot[ho + k] = hb + k;
        }
      }
      run += tile;
    }
    if (!grid_wait(P.bar, P.wait_limit, P.err)) return false;
    F.par[j + 1] = par;
    F.slot[j + 1] = slot;
    n = total;
  }
  return true;
}

// The fused mine (FusedLegs): P.bar, P.err and P.wait_limit serve every
// barrier; K >= 3 runs the cycle levels after the legs.  3 blocks of 512
// per SM at 40 registers (with spills) measured faster than 2 at 64.
template <int NS>
__global__ void __launch_bounds__(FUSED_BLOCK, 3) k_mine_fused(GraphView g, FusedLegs Q,
                                                             CycLevelArgs A, FusedCycles P,
                                                             SubWindows sub) {
  __shared__ long long s_w[FUSED_BLOCK / 32];
  const unsigned G = gridDim.x;
  const int64_t E = g.E;
  const int64_t C = (E + G - 1) / G;
  const int64_t c0 = min(E, (int64_t)blockIdx.x * C), c1 = min(E, c0 + C);
  const bool cyc = Q.anc != nullptr;
  const int lane = threadIdx.x & 31;
  const long long n_wt = (E + FUSED_WARP_TILE - 1) / FUSED_WARP_TILE;
  // 1. leg count: a work queue of warp tiles (FUSED_WARP_TILE consecutive
  // edges a warp takes from a counter), so the blocks whose edges have long
  // windows do not set the phase's end
  for (;;) {
    long long t = 0;
    if (lane == 0) t = (long long)atomicAdd(Q.ctr, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= n_wt) break;
    for (int k = 0; k < FUSED_WARP_TILE / 32; ++k) {
      const int64_t a = t * FUSED_WARP_TILE + k * 32 + lane;
      if (a < E)
        leg_count_item<NS>(g, Q.delta, (int32_t)a, Q.L, Q.anc, 1, Q.L2, nullptr, Q.qwin, Q.qcb,
                           sub, Q.Z);
    }
  }
  if (!grid_wait(P.bar, P.wait_limit, P.err)) return;
  // 2. the leg offsets: block b sums the legs of its contiguous chunk, meets
  // the others, and places the chunk's legs and cycle legs from every
  // block's sums; the totals go to off[E], off2[E]
  long long nl = 0, nc = 0;
  for (int64_t a = c0 + threadIdx.x; a < c1; a += FUSED_BLOCK) {
    nl += __ldcg(Q.L + a);
    if (cyc) nc += __ldcg(Q.L2 + a);
  }
  nl = fused_block_sum(nl, s_w);
  nc = fused_block_sum(nc, s_w);
  if (threadIdx.x == 0) {
    Q.bsum[2 * blockIdx.x] = nl;
    Q.bsum[2 * blockIdx.x + 1] = nc;
  }
  if (!grid_wait(P.bar, P.wait_limit, P.err)) return;
  long long b1 = 0, b2 = 0, t1 = 0, t2 = 0;
  for (unsigned b = threadIdx.x; b < G; b += FUSED_BLOCK) {
    const long long v1 = __ldcg(Q.bsum + 2 * b), v2 = __ldcg(Q.bsum + 2 * b + 1);
    t1 += v1;
    t2 += v2;
    if (b < blockIdx.x) {
      b1 += v1;
      b2 += v2;
    }
  }
  b1 = fused_block_sum(b1, s_w);
  b2 = fused_block_sum(b2, s_w);
  t1 = fused_block_sum(t1, s_w);
  t2 = fused_block_sum(t2, s_w);
  if (t1 != Q.n_legs || (cyc && t2 != Q.n2)) {  // every block sees the same totals
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(P.err, ERR_OVERFLOW);
    return;
  }
  for (int64_t t0 = c0; t0 < c1; t0 += FUSED_BLOCK) {
    const int64_t a = t0 + threadIdx.x;
    const int32_t l1 = a < c1 ? __ldcg(Q.L + a) : 0;
    const int32_t l2 = cyc && a < c1 ? __ldcg(Q.L2 + a) : 0;
    long long tile1 = 0, tile2 = 0;
    const long long o1 = b1 + fused_block_excl(l1, s_w, &tile1);
    const long long o2 = b2 + fused_block_excl(l2, s_w, &tile2);
    if (a < c1) {
      Q.off[a] = o1;
      if (cyc) Q.off2[a] = o2;
    }
    b1 += tile1;
    b2 += tile2;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Q.off[E] = t1;
    if (cyc) Q.off2[E] = t2;
  }
  // 3. leg emission, from a second work queue of warp tiles once every
  // offset is placed; the accumulators it adds into were zeroed in phase 1
  if (!grid_wait(P.bar, P.wait_limit, P.err)) return;
  for (;;) {
    long long t = 0;
    if (lane == 0) t = (long long)atomicAdd(Q.ctr + 1, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= n_wt) break;
    for (int k = 0; k < FUSED_WARP_TILE / 32; ++k) {
      const int64_t a = t * FUSED_WARP_TILE + k * 32 + lane;
      leg_emit_warp<NS>(g, Q.qwin, Q.qcb, Q.off, Q.S, Q.acc_cyc2, Q.gs_in, Q.own_max, sub,
                        a < E ? a : E);
    }
  }
  if (!cyc || A.K < 3) return;
  // 4. the cycle levels, once every block's cycle legs are written
  if (!grid_wait(P.bar, P.wait_limit, P.err)) return;
  cyc_fused_levels<NS>(A, P, sub, t2, s_w);
}

template <int NS>
static void fused_mine_blocks(int* per_sm) {
  AML_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_mine_fused<NS>, FUSED_BLOCK,
                                                         0));
}

int fused_mine_grid(int n_sub) {
  static int cached[64][MAX_SUB + 1] = {};
  int dev = 0;
  AML_CUDA(cudaGetDevice(&dev));
  int per_sm = 0;
  const int key = n_sub <= 0 ? 0 : n_sub == 1 ? 1 : n_sub == 2 ? 2 : MAX_SUB;
  if (dev < 64 && cached[dev][key]) return cached[dev][key];
  nsub_dispatch(n_sub, [&](auto ns) { fused_mine_blocks<decltype(ns)::value>(&per_sm); });
  AML_REQUIRE(per_sm >= 1, AML_EUNSUPPORTED, "the fused mine kernel cannot be resident");
  const int grid = per_sm * sm_count();
  if (dev < 64) cached[dev][key] = grid;
  return grid;
}

void launch_mine_fused(int grid, cudaStream_t s, const GraphView& g, const FusedLegs& Q, int K,
                       const CycleSlots& slots, unsigned long long* acc, int32_t close_scan_max,
                       const FusedCycles& P, const SubWindows& sub) {
  const CycLevelArgs A{g, Q.delta, K, nullptr, Q.anc, Q.qwin, slots, acc, close_scan_max};
  nsub_dispatch(sub.n, [&](auto ns) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(FUSED_BLOCK);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    AML_LAUNCH("k_mine_fused", s,
               AML_CUDA(cudaLaunchKernelEx(&cfg, k_mine_fused<decltype(ns)::value>, g, Q, A, P,
                                           sub)));
  });
}

// flag[a] = 1 when edge a's closing range is not empty (it anchors cycles)
__global__ void __launch_bounds__(256) k_anchor_flags(const int2* __restrict__ crng, int64_t E,
                                                      int32_t* __restrict__ flag) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < E) {
    const int2 cr = crng[a];
    flag[a] = cr.x < cr.y ? 1 : 0;
  }
}

// items[off[a]] = a for every flagged a
__global__ void __launch_bounds__(256) k_compact_ids(const int32_t* __restrict__ flag,
                                                     const int32_t* __restrict__ off, int64_t E,
                                                     int32_t* __restrict__ items) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < E && flag[a]) items[off[a]] = (int32_t)a;
}

// Writes the children (parent, slot) of every element at off[i]...; short
// windows are written by their own lane, long ones by the whole warp.
__global__ void __launch_bounds__(512) k_cyc_emit(int64_t n, const int32_t* __restrict__ cnt,
                                                  const int32_t* __restrict__ q0,
                                                  const int64_t* __restrict__ off,
                                                  int32_t* __restrict__ par,
                                                  int32_t* __restrict__ slot, int32_t own_max) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int32_t c = i < n ? cnt[i] : 0;
  const int64_t o = c ? off[i] : 0;
  const int32_t b = c ? q0[i] : 0;
  const bool own = c <= own_max;
  if (own)
    for (int32_t k = 0; k < c; ++k) {
      par[o + k] = (int32_t)i;
      slot[o + k] = b + k;
    }
  unsigned heavy = __ballot_sync(0xffffffffu, !own);
  while (heavy) {
    const int src = __ffs(heavy) - 1;
    heavy &= heavy - 1;
    const int64_t hi = __shfl_sync(0xffffffffu, i, src);
    const int32_t hc = __shfl_sync(0xffffffffu, c, src);
    const int64_t ho = __shfl_sync(0xffffffffu, o, src);
    const int32_t hb = __shfl_sync(0xffffffffu, b, src);
    for (int32_t k = lane; k < hc; k += 32) {
      par[ho + k] = (int32_t)hi;
      slot[ho + k] = hb + k;
    }
  }
}

// -------------------------------------------------------------- assemble
//
// One thread per edge computes the edge's whole output row from values the
// earlier kernels left in edge order: DEG and FAN per window and direction
// (a 32-byte row per edge and direction), GS = legs starting + legs ending
// at the edge, SG and CYC from the 64-bit accumulators; saturated at the graph's count limit (2^32-1).  A streamed
// old row adds its new instances to the stored value and saturates the sum:
// min(min(old, B) + new, B) = min(old + new, B), so a clamped row stays
// exact.
// The block's rows are staged in shared memory and stored as one contiguous
// range when the output has no padding (ld = P), so the stores coalesce.

__device__ __forceinline__ uint64_t assemble_value(const AssembleParams& P, const ColDesc cd,
                                                   int32_t e) {
  const int w = cd.didx;
  switch (cd.family) {
    case AML_FAM_DEG_OUT:
      return (uint64_t)P.df_out[w][(int64_t)e * DF_STRIDE].x;
    case AML_FAM_FAN_OUT:
      return (uint64_t)P.df_out[w][(int64_t)e * DF_STRIDE].y;
    case AML_FAM_DEG_IN:
      return (uint64_t)P.df_in[w][(int64_t)e * DF_STRIDE].x;
    case AML_FAM_FAN_IN:
      return (uint64_t)P.df_in[w][(int64_t)e * DF_STRIDE].y;
    case AML_FAM_GS: {
      const int32_t from =
          P.gs_from[w] ? P.gs_from[w][e] : (int32_t)(P.off[w][e + 1] - P.off[w][e]);
      return (uint64_t)from + (uint64_t)P.gs_in[w][e];
    }
    default:  // accumulated families
      return P.acc[(int64_t)cd.acc_slot * P.g.E + e];
  }
}

// a count above the bound is reported as the bound: saturated, never wrapped
__device__ __forceinline__ uint32_t saturate(uint64_t v, uint32_t limit) {
  return v > (uint64_t)limit ? limit : (uint32_t)v;
}

constexpr int ASM_BATCH = 8;
__global__ void __launch_bounds__(ASM_BLOCK) k_assemble(AssembleParams P) {
  extern __shared__ uint32_t s_rows[];  // the block's rows, row-major
  const GraphView& g = P.g;
  const int nc = P.ncols;
  const int64_t e0 = (int64_t)blockIdx.x * ASM_BLOCK;
  const int nrows = g.E - e0 < ASM_BLOCK ? (int)(g.E - e0) : ASM_BLOCK;
  const int tot = nrows * nc;
  uint32_t* out = P.counts + e0 * P.ld;
  const bool dense = P.ld == nc;  // the block's rows are one contiguous range
  if (e0 < P.accumulate_from) {
    // a block with old rows (streaming): an old row keeps what it holds and
    // only its instance columns with new instances change, so the row is
    // updated in place where a count is not zero (most rows get none); the
    // batch rows of the one block that also holds old rows are written
    // whole, row by row
    if ((int)threadIdx.x < nrows) {
      const int64_t e64 = e0 + threadIdx.x;
      const int32_t e = (int32_t)e64;
      uint32_t* orow = out + (int64_t)threadIdx.x * P.ld;
      const bool add = e64 < P.accumulate_from;
      const bool loop = g.src[e] == g.dst[e];
      for (int c = 0; c < nc; ++c) {
        if (add) {
          if (loop || !((P.inst_mask >> c) & 1ull)) continue;  // trailing windows never change
          const uint64_t val = assemble_value(P, P.cols[c], e);
          if (val == 0) continue;
          orow[c] = saturate(val + orow[c], P.limit);
        } else {
          orow[c] = loop ? 0u : saturate(assemble_value(P, P.cols[c], e), P.limit);
        }
      }
    }
    return;
  }
  if ((int)threadIdx.x < nrows) {
    const int32_t e = (int32_t)(e0 + threadIdx.x);
    uint32_t* row = s_rows + threadIdx.x * nc;
    const int32_t u = g.src[e], v = g.dst[e];
    if (u == v) {
      for (int c = 0; c < nc; ++c) row[c] = 0u;
    } else {
      // ASM_BATCH columns' loads are issued before the first of them is
      // used, so a row waits for a few rounds of memory latency, not one
      // per column
      for (int c0 = 0; c0 < nc; c0 += ASM_BATCH) {
        uint64_t val[ASM_BATCH];
#pragma unroll
        for (int k = 0; k < ASM_BATCH; ++k)
          if (c0 + k < nc) val[k] = assemble_value(P, P.cols[c0 + k], e);
#pragma unroll
        for (int k = 0; k < ASM_BATCH; ++k)
          if (c0 + k < nc) row[c0 + k] = saturate(val[k], P.limit);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < tot; i += ASM_BLOCK) {
    const int r = dense ? 0 : i / nc;
    out[dense ? i : r * P.ld + (i - r * nc)] = s_rows[i];
  }
}


// ------------------------------------------------------------- launchers
//
// The kernels that count sub-windows are compiled for 0, 1, 2 and MAX_SUB
// of them, so the per-window counters live in registers.


void launch_leg_count(unsigned grid, int block, cudaStream_t s, const GraphView& g, int32_t delta,
                      int32_t* L, AnchorRec* anc, bool close_here, int32_t* L2, int32_t* L_new,
                      int2* qwin, int32_t* qcb, const SubWindows& sub, const ZeroSink& Z) {
  nsub_dispatch(sub.n, [&](auto ns) {
    AML_LAUNCH("k_leg_count", s,
               k_leg_count<decltype(ns)::value><<<grid, block, 0, s>>>(
                   g, delta, L, anc, close_here ? 1 : 0, L2, L_new, qwin, qcb, sub, Z));
  });
}

void launch_leg_emit_delta(unsigned grid, int block, cudaStream_t s, const GraphView& g,
                           const int2* qwin, const int32_t* qcb, const LegSink& S,
                           unsigned long long* acc_cyc2, int32_t* gs_in, int32_t own_max,
                           const SubWindows& sub, const int32_t* first_new,
                           const int32_t* mptr, const int32_t* mslot) {
  nsub_dispatch(sub.n, [&](auto ns) {
    AML_LAUNCH("k_leg_emit_delta", s,
               k_leg_emit_delta<decltype(ns)::value><<<grid, block, 0, s>>>(
                   g, qwin, qcb, S, acc_cyc2, gs_in, own_max, sub, first_new, mptr, mslot));
  });
}

void launch_leg_emit(unsigned grid, int block, cudaStream_t s, const GraphView& g,
                     const int2* qwin, const int32_t* qcb, const int64_t* off, const LegSink& S,
                     unsigned long long* acc_cyc2, int32_t* gs_in, int32_t own_max,
                     const SubWindows& sub) {
  nsub_dispatch(sub.n, [&](auto ns) {
    AML_LAUNCH("k_leg_emit", s,
               k_leg_emit<decltype(ns)::value><<<grid, block, 0, s>>>(g, qwin, qcb, off, S,
                                                                     acc_cyc2, gs_in, own_max,
                                                                     sub));
  });
}

void launch_sg_buckets(unsigned n_buckets, cudaStream_t s, const LegRec* rec,
                       const uint32_t* bend, int32_t delta, const int2* dts, const int32_t* ts,
                       unsigned long long* acc, int32_t new_from, uint32_t* overflow,
                       const SubWindows& sub, const uint32_t* skip) {
  nsub_dispatch(sub.n, [&](auto ns) {
    constexpr int NS = decltype(ns)::value;
    static bool smem_set[64][MAX_SUB + 1] = {};  // per device and instantiation
    int dev = 0;
    AML_CUDA(cudaGetDevice(&dev));
    const size_t big = sizeof(SgSmem<SG_CAP_BIG, SG_TAB_BIG>);
    if (dev >= 64 || !smem_set[dev][NS]) {
      AML_CUDA(cudaFuncSetAttribute(k_sg_bucket_big<NS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big));
      if (dev < 64) smem_set[dev][NS] = true;
    }
    AML_LAUNCH("k_sg_bucket", s,
               k_sg_bucket<NS><<<n_buckets, SG_BLOCK, 0, s>>>(rec, bend, delta, dts, ts, acc,
                                                         new_from, overflow, sub, skip));
    AML_LAUNCH("k_sg_bucket_big", s,
               k_sg_bucket_big<NS><<<(unsigned)sm_count(), SG_BIG_BLOCK, big, s>>>(
                   rec, bend, delta, dts, ts, acc, new_from, overflow, sub));
  });
}

void launch_cyc_level(unsigned grid, int block, cudaStream_t s, const GraphView& g,
                      int32_t delta, int K, int j, const CycFrontier& F, int64_t n,
                      const int2* close_rng, const AnchorRec* anc, const int2* qwin,
                      const CycleSlots& slots, unsigned long long* acc, int32_t* cnt,
                      int32_t* q0_out, int32_t close_scan_max, const SubWindows& sub,
                      bool window_cycles) {
  AML_REQUIRE(window_cycles ? close_rng != nullptr : (anc != nullptr && qwin != nullptr),
              AML_EINTERNAL, "cycle level without its anchor data");
  const CycLevelArgs A{g, delta, K, close_rng, anc, qwin, slots, acc, close_scan_max};
  AML_REQUIRE(j >= (window_cycles ? 1 : 2) && j <= MAX_CYCLE - 1, AML_EINTERNAL,
              "cycle level out of range");
  nsub_dispatch(sub.n, [&](auto ns) {
    level_dispatch(j, [&](auto jc) {
      constexpr int NSV = decltype(ns)::value, J = decltype(jc)::value;
      if (window_cycles)
        AML_LAUNCH("k_cyc_level_win", s,
                   k_cyc_level<NSV, true, J><<<grid, block, 0, s>>>(A, F, n, cnt, q0_out, sub));
      else if constexpr (J >= 2)
        AML_LAUNCH("k_cyc_level", s,
                   k_cyc_level<NSV, false, J><<<grid, block, 0, s>>>(A, F, n, cnt, q0_out, sub));
    });
  });
}

}  // namespace aml
