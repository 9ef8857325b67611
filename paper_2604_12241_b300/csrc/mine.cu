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

__global__ void __launch_bounds__(256) k_fan_delta(const int32_t* __restrict__ ptr,
                                                   const int32_t* __restrict__ t,
                                                   const int32_t* __restrict__ eid,
                                                   const int32_t* __restrict__ prev,
                                                   const int32_t* __restrict__ next,
                                                   const int32_t* __restrict__ row_of, int64_t Ev,
                                                   int32_t delta, int32_t* __restrict__ D) {
  int64_t p64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p64 >= Ev) return;
  int32_t p = (int32_t)p64;
  int32_t rs = __ldg(ptr + __ldg(row_of + __ldg(eid + p)));
  int32_t d = 0;
  if (p > rs) {
    int32_t tp = __ldg(t + p);
    int32_t lbp = lower_t(t, rs, p + 1, (int64_t)tp - delta);
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

// Writes every leg (a, b) of edge a at off[a]...; reciprocal edges b = h->x
// inside the window close 2-cycles (a, b) and are credited directly.
__global__ void __launch_bounds__(256) k_leg_emit(GraphView g, int32_t delta,
                                                  const int64_t* __restrict__ off,
                                                  int32_t* __restrict__ la, int32_t* __restrict__ lb,
                                                  uint64_t* __restrict__ key, int64_t n_nodes,
                                                  unsigned long long* __restrict__ acc_cyc2) {
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
// Depth-first search from every leg (e1, e2) taken as the first two edges
// of a cycle (e1 is its earliest edge): every hop takes a later edge inside
// t(e1) + delta to a node not yet on the path; an edge back into u0 closes a
// cycle of length depth+1.  At the last level only closing edges can count,
// so they are found by binary search in the (nbr, t, id) copy instead of a
// window scan (the closing intersection of Sec. 6's cycle example).

__device__ __forceinline__ void credit_cycle(unsigned long long* acc, int64_t E, int slot,
                                             const int32_t* edges, int n,
                                             unsigned long long c) {
  unsigned long long* col = acc + (int64_t)slot * E;
  for (int j = 0; j < n; ++j) atomicAdd(col + edges[j], c);
}

__global__ void __launch_bounds__(128) k_cycles(GraphView g, int32_t delta, int K,
                                                const int32_t* __restrict__ la,
                                                const int32_t* __restrict__ lb, int64_t n_legs,
                                                CycleSlots slots,
                                                unsigned long long* __restrict__ acc) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_legs) return;
  int32_t edges[MAX_CYCLE];
  int32_t nodes[MAX_CYCLE];
  int32_t cur[MAX_CYCLE], end[MAX_CYCLE];
  edges[0] = la[i];
  edges[1] = lb[i];
  nodes[0] = g.src[edges[0]];
  nodes[1] = g.dst[edges[0]];
  nodes[2] = g.dst[edges[1]];
  const int32_t u0 = nodes[0];
  const int64_t tmax = (int64_t)g.ts[edges[0]] + delta;
  int L = 2;  // edges on the path; current node nodes[L]
  // opening a level: the window after the last edge, or the closing lookup
  auto open = [&](int lev) -> bool {
    int32_t w = nodes[lev];
    int32_t last = edges[lev - 1];
    int32_t tl = g.ts[last];
    int32_t ws = g.optr[w], we = g.optr[w + 1];
    if (lev == K - 1) {
      // only closing edges matter here
      // tl >= t(e1), so tmax - tl <= delta fits in int32
      int32_t c = pair_after(g.onnbr, g.ont, g.oneid, ws, we, u0, tl, last,
                             (int32_t)(tmax - tl));
      if (c > 0 && slots.slot[K] >= 0) {
        credit_cycle(acc, g.E, slots.slot[K], edges, lev, (unsigned long long)c);
        int32_t r0 = lower_nbr(g.onnbr, ws, we, u0);
        int32_t r1 = lower_nbr(g.onnbr, r0, we, u0 + 1);
        int32_t b0 = after_edge(g.ont, g.oneid, r0, r1, tl, last);
        int32_t b1 = upper_t(g.ont, b0, r1, tmax);
        unsigned long long* col = acc + (int64_t)slots.slot[K] * g.E;
        for (int32_t q = b0; q < b1; ++q) atomicAdd(col + __ldg(g.oneid + q), 1ull);
      }
      return false;
    }
    cur[lev] = after_edge(g.ot, g.oeid, ws, we, tl, last);
    end[lev] = upper_t(g.ot, cur[lev], we, tmax);
    return true;
  };
  if (!open(L)) return;
  while (L >= 2) {
    if (cur[L] >= end[L]) {
      --L;
      continue;
    }
    int32_t q = cur[L]++;
    int32_t x = __ldg(g.onbr + q);
    int32_t f = __ldg(g.oeid + q);
    if (x == u0) {
      int k = L + 1;
      if (slots.slot[k] >= 0) {
        edges[L] = f;
        credit_cycle(acc, g.E, slots.slot[k], edges, k, 1ull);
      }
      continue;
    }
    if (L + 1 >= K) continue;
    bool seen = false;
    for (int j = 1; j <= L; ++j) seen |= (nodes[j] == x);
    if (seen) continue;
    edges[L] = f;
    nodes[L + 1] = x;
    if (open(L + 1)) ++L;
  }
}

// -------------------------------------------------------------- assemble
//
// One thread per edge writes the edge's whole output row: DEG and FAN from
// the window bounds and the repeat prefix sums, GS from binary searches, SG
// and CYC from the 64-bit accumulators, all saturated to 32 bits.

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
  int32_t te = g.ts[e];
  int32_t po = g.opos[e], pi = g.ipos[e];
  int32_t os = g.optr[u], is = g.iptr[v];
  for (int c = 0; c < P.ncols; ++c) {
    const ColDesc cd = P.cols[c];
    uint64_t val = 0;
    switch (cd.family) {
      case AML_FAM_DEG_OUT:
      case AML_FAM_FAN_OUT: {
        int32_t lb = lower_t(g.ot, os, po + 1, (int64_t)te - cd.delta);
        val = (uint64_t)(po - lb + 1);
        if (cd.family == AML_FAM_FAN_OUT) {
          const int32_t* S = P.S_out[cd.didx];
          int32_t rep = S[po] - (os > 0 ? S[os - 1] : 0);
          val -= (uint64_t)rep;
        }
        break;
      }
      case AML_FAM_DEG_IN:
      case AML_FAM_FAN_IN: {
        int32_t lb = lower_t(g.it, is, pi + 1, (int64_t)te - cd.delta);
        val = (uint64_t)(pi - lb + 1);
        if (cd.family == AML_FAM_FAN_IN) {
          const int32_t* S = P.S_in[cd.didx];
          int32_t rep = S[pi] - (is > 0 ? S[is - 1] : 0);
          val -= (uint64_t)rep;
        }
        break;
      }
      case AML_FAM_GS:
        val = (uint64_t)legs_from(g, e, cd.delta) + (uint64_t)legs_into(g, e, cd.delta);
        break;
      default:  // accumulated families
        val = P.acc[(int64_t)cd.acc_slot * g.E + e];
        break;
    }
    row[c] = val > 0xffffffffull ? 0xffffffffu : (uint32_t)val;
  }
}

}  // namespace aml
