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

#include "aml_internal.cuh"
#include "mine.cuh"

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

// Per slot p of one direction: the start lb(p) of its trailing window (so
// DEG = p - lb(p) + 1) and, when FAN is wanted, the repeat delta above.
__global__ void __launch_bounds__(256) k_window_slots(const int32_t* __restrict__ ptr,
                                                      const int32_t* __restrict__ t,
                                                      const int32_t* __restrict__ eid,
                                                      const int32_t* __restrict__ prev,
                                                      const int32_t* __restrict__ next,
                                                      const int32_t* __restrict__ row_of,
                                                      int64_t Ev, int32_t delta,
                                                      int32_t* __restrict__ lb,
                                                      int32_t* __restrict__ D) {
  int64_t p64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p64 >= Ev) return;
  int32_t p = (int32_t)p64;
  int32_t rs = __ldg(ptr + __ldg(row_of + __ldg(eid + p)));
  int32_t tp = __ldg(t + p);
  int32_t lbp = lower_t(t, rs, p + 1, (int64_t)tp - delta);
  lb[p] = lbp;
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
  q0 = after_edge(g.ot, g.oeid, hs, he, ta, a);
  q1 = upper_t(g.ot, q0, he, (int64_t)ta + delta);
}

// number of slots in [lo, hi) of the (nbr, t, id) copy with nbr == x and
// (t, id) in ((te, e), te + delta]
__device__ __forceinline__ int32_t pair_after(const int32_t* __restrict__ nn,
                                              const int32_t* __restrict__ nt,
                                              const int32_t* __restrict__ ne, int32_t lo,
                                              int32_t hi, int32_t x, int32_t te, int32_t e,
                                              int32_t delta) {
  int32_t r0 = lower_nbr(nn, lo, hi, x);
  if (r0 >= hi || __ldg(nn + r0) != x) return 0;
  int32_t r1 = lower_nbr(nn, r0, hi, x + 1);
  int32_t b0 = after_edge(nt, ne, r0, r1, te, e);
  int32_t b1 = upper_t(nt, b0, r1, (int64_t)te + delta);
  return b1 - b0;
}

// ... with (t, id) in [te - delta, (te, e))
__device__ __forceinline__ int32_t pair_before(const int32_t* __restrict__ nn,
                                               const int32_t* __restrict__ nt,
                                               const int32_t* __restrict__ ne, int32_t lo,
                                               int32_t hi, int32_t x, int32_t te, int32_t e,
                                               int32_t delta) {
  int32_t r0 = lower_nbr(nn, lo, hi, x);
  if (r0 >= hi || __ldg(nn + r0) != x) return 0;
  int32_t r1 = lower_nbr(nn, r0, hi, x + 1);
  int32_t b0 = lower_t(nt, r0, r1, (int64_t)te - delta);
  int32_t b1 = after_edge(nt, ne, b0, r1, te, e);
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
  int32_t c0 = lower_t(g.it, hs, he, (int64_t)tb - delta);
  int32_t c1 = after_edge(g.it, g.ieid, c0, he, tb, b);
  return (c1 - c0) - pair_before(g.innbr, g.int_, g.ineid, hs, he, g.dst[b], tb, b, delta);
}

__global__ void __launch_bounds__(256) k_leg_count(GraphView g, int32_t delta,
                                                   int32_t* __restrict__ L) {
  int64_t a64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a64 >= g.E) return;
  int32_t a = (int32_t)a64;
  L[a] = (g.src[a] == g.dst[a]) ? 0 : legs_from(g, a, delta);
}

// legs ending with each edge, by binary search (when no legs are emitted)
__global__ void __launch_bounds__(256) k_gs_into(GraphView g, int32_t delta,
                                                 int32_t* __restrict__ gs_in) {
  int64_t b64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b64 >= g.E) return;
  int32_t b = (int32_t)b64;
  gs_in[b] = (g.src[b] == g.dst[b]) ? 0 : legs_into(g, b, delta);
}

// Writes every leg (a, b) of edge a at off[a]...; reciprocal edges b = h->x
// inside the window close 2-cycles (a, b) and are credited directly.  With
// gs_in, also counts the legs ending with each edge (the scatter side of GS).
__global__ void __launch_bounds__(256) k_leg_emit(GraphView g, int32_t delta,
                                                  const int64_t* __restrict__ off,
                                                  int32_t* __restrict__ la,
                                                  int32_t* __restrict__ lb,
                                                  uint64_t* __restrict__ key, int64_t n_nodes,
                                                  unsigned long long* __restrict__ acc_cyc2,
                                                  int32_t* __restrict__ gs_in) {
  int64_t a64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a64 >= g.E) return;
  int32_t a = (int32_t)a64;
  int32_t x = g.src[a];
  if (x == g.dst[a]) return;
  int32_t q0, q1;
  leg_window(g, a, q0, q1, delta);
  int64_t o = off[a];
  unsigned long long n_cyc2 = 0;
  for (int32_t q = q0; q < q1; ++q) {
    int32_t y = __ldg(g.onbr + q);
    int32_t b = __ldg(g.oeid + q);
    if (y == x) {
      if (acc_cyc2) {
        atomicAdd(acc_cyc2 + b, 1ull);
        ++n_cyc2;
      }
      continue;
    }
    la[o] = a;
    lb[o] = b;
    if (key) key[o] = (uint64_t)x * (uint64_t)n_nodes + (uint64_t)y;
    if (gs_in) atomicAdd(gs_in + b, 1);
    ++o;
  }
  if (n_cyc2) atomicAdd(acc_cyc2 + a, n_cyc2);
}

// --------------------------------------------------------- scatter-gather
//
// Legs sorted by (s, d): each run of equal keys holds all legs between one
// source and one destination.  A leg's partners are the legs of its run with
// another intermediary whose union with it spans at most delta; each partner
// pair is one SG instance, credited to the four edges (a leg credits its own
// two edges once per partner, and the partner credits its two).

__global__ void __launch_bounds__(256) k_sg_group(const uint64_t* __restrict__ key,
                                                  const uint32_t* __restrict__ idx, int64_t n,
                                                  const int32_t* __restrict__ la,
                                                  const int32_t* __restrict__ lb,
                                                  const int32_t* __restrict__ dst,
                                                  const int32_t* __restrict__ ts, int32_t delta,
                                                  unsigned long long* __restrict__ acc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t k = key[i];
  int64_t gs = i, ge = i + 1;
  while (gs > 0 && key[gs - 1] == k) --gs;
  while (ge < n && key[ge] == k) ++ge;
  if (ge - gs < 2) return;
  uint32_t li = idx[i];
  int32_t ai = la[li], bi = lb[li];
  int32_t mi = dst[ai];
  int64_t lo = ts[ai], hi = ts[bi];
  unsigned long long c = 0;
  for (int64_t j = gs; j < ge; ++j) {
    if (j == i) continue;
    uint32_t lj = idx[j];
    int32_t aj = la[lj];
    if (dst[aj] == mi) continue;
    int64_t loj = ts[aj], hij = ts[lb[lj]];
    int64_t span = max(hi, hij) - min(lo, loj);
    c += (span <= delta) ? 1ull : 0ull;
  }
  if (c) {
    atomicAdd(acc + ai, c);
    atomicAdd(acc + bi, c);
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

// B1 of every edge a = u0 -> u1: slots of in(u0) after a with t <= t_a + delta
__global__ void __launch_bounds__(256) k_close_range(GraphView g, int32_t delta,
                                                     int2* __restrict__ rng) {
  int64_t a64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a64 >= g.E) return;
  int32_t a = (int32_t)a64;
  int32_t u0 = g.src[a];
  int2 r = make_int2(0, 0);
  if (u0 != g.dst[a]) {
    int32_t is = g.iptr[u0], ie = g.iptr[u0 + 1];
    int32_t ta = g.ts[a];
    r.x = after_edge(g.it, g.ieid, is, ie, ta, a);
    r.y = upper_t(g.it, r.x, ie, (int64_t)ta + delta);
  }
  rng[a] = r;
}

constexpr int32_t CLOSE_SCAN_MAX = 48;  // B1 longer than this: binary search

// Rebuilds the path of frontier element i at level j (j edges):
// edges[0..j-1] and nodes[0..j] (nodes[0] = u0 = src of the anchor).
__device__ __forceinline__ void cyc_path(const GraphView& g, const CycFrontier& F, int j,
                                         int64_t i, int32_t* edges, int32_t* nodes) {
  int64_t idx = i;
  for (int lev = j; lev >= 3; --lev) {
    const int32_t q = F.slot[lev][idx];
    edges[lev - 1] = __ldg(g.oeid + q);
    nodes[lev] = __ldg(g.onbr + q);
    idx = F.par[lev][idx];
  }
  edges[0] = F.la[idx];
  edges[1] = F.lb[idx];
  nodes[0] = g.src[edges[0]];
  nodes[1] = g.dst[edges[0]];
  nodes[2] = g.dst[edges[1]];
}

// One level of the cycle search.  Element i of level j is a path of j
// increasing edges from the anchor e1; the kernel checks that its last hop
// is admissible (new node, before the latest closing edge), credits the
// cycles of length j+1 that close from its end node through B1, and reports
// the window of later hops its children will take.
__global__ void __launch_bounds__(256) k_cyc_level(GraphView g, int32_t delta, int K, int j,
                                                   CycFrontier F, int64_t n,
                                                   const int2* __restrict__ close_rng,
                                                   CycleSlots slots,
                                                   unsigned long long* __restrict__ acc,
                                                   int32_t* __restrict__ cnt,
                                                   int32_t* __restrict__ q0_out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool has_next = j + 1 <= K - 1;
  if (has_next) cnt[i] = 0;
  int32_t edges[MAX_CYCLE];
  int32_t nodes[MAX_CYCLE + 1];
  cyc_path(g, F, j, i, edges, nodes);
  const int2 cr = close_rng[edges[0]];
  if (cr.x >= cr.y) return;  // e1 starts no cycle
  const int32_t t_cl = __ldg(g.it + cr.y - 1), id_cl = __ldg(g.ieid + cr.y - 1);
  const int32_t last = edges[j - 1], tl = g.ts[last];
  if (!before(tl, last, t_cl, id_cl)) return;  // nothing can close after it
  const int32_t u0 = nodes[0], w = nodes[j];
  if (j >= 3) {  // the hop into w must reach a new node
    if (w == u0) return;
    for (int m = 1; m < j; ++m)
      if (nodes[m] == w) return;
  }
  // cycles of length j+1: edges w -> u0 in B1 after `last`
  const int k = j + 1;
  if (k <= K && slots.slot[k] >= 0) {
    unsigned long long* col = acc + (int64_t)slots.slot[k] * g.E;
    unsigned long long c = 0;
    if (cr.y - cr.x <= CLOSE_SCAN_MAX) {
      for (int32_t q = cr.x; q < cr.y; ++q) {
        if (__ldg(g.inbr + q) != w) continue;
        const int32_t cid = __ldg(g.ieid + q);
        if (!before(tl, last, __ldg(g.it + q), cid)) continue;
        atomicAdd(col + cid, 1ull);
        ++c;
      }
    } else {
      const int32_t in_s = g.iptr[u0], in_e = g.iptr[u0 + 1];
      const int32_t r0 = lower_nbr(g.innbr, in_s, in_e, w);
      if (r0 < in_e && __ldg(g.innbr + r0) == w) {
        const int32_t r1 = lower_nbr(g.innbr, r0, in_e, w + 1);
        const int32_t b0 = after_edge(g.int_, g.ineid, r0, r1, tl, last);
        const int32_t b1 = upper_t(g.int_, b0, r1, (int64_t)g.ts[edges[0]] + delta);
        for (int32_t q = b0; q < b1; ++q) atomicAdd(col + __ldg(g.ineid + q), 1ull);
        c = (unsigned long long)(b1 - b0);
      }
    }
    if (c)
      for (int m = 0; m < j; ++m) atomicAdd(col + edges[m], c);
  }
  if (has_next) {
    const int32_t ws = g.optr[w], we = g.optr[w + 1];
    const int32_t q0 = after_edge(g.ot, g.oeid, ws, we, tl, last);
    const int32_t q1 = upper_t(g.ot, q0, we, t_cl);
    cnt[i] = q1 - q0;
    q0_out[i] = q0;
  }
}

// Writes the children (parent, slot) of every element at off[i]...; short
// windows are written by their own lane, long ones by the whole warp.
__global__ void __launch_bounds__(256) k_cyc_emit(int64_t n, const int32_t* __restrict__ cnt,
                                                  const int32_t* __restrict__ q0,
                                                  const int64_t* __restrict__ off,
                                                  int32_t* __restrict__ par,
                                                  int32_t* __restrict__ slot) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int32_t c = i < n ? cnt[i] : 0;
  const int64_t o = c ? off[i] : 0;
  const int32_t b = c ? q0[i] : 0;
  const bool own = c <= 32;
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
// One thread per edge writes the edge's whole output row from values the
// earlier kernels left in slot or edge order: DEG = pos - lb(pos) + 1, FAN =
// DEG - repeats (prefix-sum difference), GS = legs starting + legs ending at
// the edge, SG and CYC from the 64-bit accumulators; saturated to 32 bits.

__global__ void __launch_bounds__(256) k_assemble(AssembleParams P) {
  int64_t e64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const GraphView& g = P.g;
  if (e64 >= g.E) return;
  int32_t e = (int32_t)e64;
  uint32_t* row = P.counts + e64 * P.ld;
  int32_t u = g.src[e], v = g.dst[e];
  if (u == v) {
    for (int c = 0; c < P.ncols; ++c) row[c] = 0u;
    return;
  }
  int32_t po = g.opos[e], pi = g.ipos[e];
  int32_t os = g.optr[u], is = g.iptr[v];
  for (int c = 0; c < P.ncols; ++c) {
    const ColDesc cd = P.cols[c];
    const int w = cd.didx;
    uint64_t val = 0;
    switch (cd.family) {
      case AML_FAM_DEG_OUT:
        val = (uint64_t)(po - P.lb_out[w][po] + 1);
        break;
      case AML_FAM_FAN_OUT: {
        const int32_t* S = P.S_out[w];
        val = (uint64_t)(po - P.lb_out[w][po] + 1 - (S[po] - (os > 0 ? S[os - 1] : 0)));
        break;
      }
      case AML_FAM_DEG_IN:
        val = (uint64_t)(pi - P.lb_in[w][pi] + 1);
        break;
      case AML_FAM_FAN_IN: {
        const int32_t* S = P.S_in[w];
        val = (uint64_t)(pi - P.lb_in[w][pi] + 1 - (S[pi] - (is > 0 ? S[is - 1] : 0)));
        break;
      }
      case AML_FAM_GS:
        val = (uint64_t)(P.off[w][e + 1] - P.off[w][e]) + (uint64_t)P.gs_in[w][e];
        break;
      default:  // accumulated families
        val = P.acc[(int64_t)cd.acc_slot * g.E + e];
        break;
    }
    row[c] = val > 0xffffffffull ? 0xffffffffu : (uint32_t)val;
  }
}

}  // namespace aml
