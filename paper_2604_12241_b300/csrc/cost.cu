// Cost-binned cycle search (a persistent kernel beside the level-by-level
// search), and the learned cost model that bins it.
//
// Work item = an anchor edge e1 = u0->u1 whose closing range B1 (u0's
// in-slots after e1 inside the window) is not empty.  Its work is the
// depth-first search of every cycle whose earliest edge is e1; the cost of
// that search varies by orders of magnitude between anchors.  The anchors
// are ordered by decreasing estimated cost; the costliest (whole cost
// buckets, about a quarter) are searched level by level from their legs,
// the rest by one persistent launch (grid = SMs x resident blocks) that
// pulls them with an atomic counter, one lane each.  (The kernel drains a
// warp queue first, whose lanes split an anchor's first window; the hybrid
// and the cost probe give it none.)
//
// Estimated cost: degree binning uses the anchor's first window size (the
// number of second edges it can take); learned binning uses the perceptron of
// mlp.cu, trained on clock64 costs measured by this same kernel run one item
// per lane (the probe).  Neither changes any count.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "aml_internal.cuh"
#include "mine.cuh"
#include "mlp.cuh"
#include "profile.cuh"

namespace aml {

// ------------------------------------------------------------- items

// per edge: 1 if it anchors cycle work, and the size of its first window
__global__ void __launch_bounds__(256) k_cyc_item_flags(GraphView g, int32_t delta,
                                                        const int2* __restrict__ crng,
                                                        int32_t* __restrict__ flag,
                                                        int32_t* __restrict__ w2) {
  const int64_t a64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a64 >= g.E) return;
  const int32_t a = (int32_t)a64;
  const int2 cr = crng[a];
  int32_t w = 0;
  if (cr.x < cr.y) {
    const int32_t u1 = g.dst[a];
    const int32_t t_cl = g.it[cr.y - 1];
    const int32_t ws = g.optr[u1], we = g.optr[u1 + 1];
    const int32_t q0 = after_edge(g.ot, g.oeid, ws, we, g.ts[a], a);
    w = upper_t(g.ot, q0, we, t_cl) - q0;
  }
  flag[a] = w > 0 ? 1 : 0;
  w2[a] = w;
}

__global__ void __launch_bounds__(256) k_cyc_compact(const int32_t* __restrict__ flag,
                                                     const int32_t* __restrict__ off, int64_t E,
                                                     int32_t* __restrict__ items) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a < E && flag[a]) items[off[a]] = (int32_t)a;
}

__device__ __forceinline__ float lg(float v) { return log1pf(fmaxf(v, 0.f)); }

// 16 cheap features of an anchor (raw; the model normalizes them)
__global__ void __launch_bounds__(256) k_cyc_features(GraphView g, int32_t delta, int K,
                                                      const int32_t* __restrict__ items,
                                                      const int32_t* __restrict__ n_items,
                                                      const int2* __restrict__ crng,
                                                      const int32_t* __restrict__ w2,
                                                      float* __restrict__ feat) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *n_items) return;
  const int32_t a = items[i];
  const int32_t u0 = g.src[a], u1 = g.dst[a], ta = g.ts[a];
  const int2 cr = crng[a];
  const int32_t t_cl = g.it[cr.y - 1];
  const int32_t do1 = g.optr[u1 + 1] - g.optr[u1], di0 = g.iptr[u0 + 1] - g.iptr[u0];
  const int32_t do0 = g.optr[u0 + 1] - g.optr[u0], di1 = g.iptr[u1 + 1] - g.iptr[u1];
  const int32_t ws = g.optr[u1], we = g.optr[u1 + 1];
  const int32_t q0 = after_edge(g.ot, g.oeid, ws, we, ta, a);
  const int32_t qd = upper_t(g.ot, q0, we, (int64_t)ta + delta);
  const int32_t po = g.opos[a], pi = g.ipos[a];
  const int32_t deg_o = po - lower_t(g.ot, g.optr[u0], po + 1, (int64_t)ta - delta) + 1;
  const int32_t deg_i = pi - lower_t(g.it, g.iptr[u1], pi + 1, (int64_t)ta - delta) + 1;
  // out-degrees of up to 8 second-hop nodes (spread over the first window)
  const int32_t w = w2[a];
  float s_deg = 0.f, m_deg = 0.f;
  const int ns = min(w, 8);
  for (int k = 0; k < ns; ++k) {
    const int32_t x = g.onbr[q0 + (int32_t)((int64_t)k * w / ns)];
    const float d = lg((float)(g.optr[x + 1] - g.optr[x]));
    s_deg += d;
    m_deg = fmaxf(m_deg, d);
  }
  float* f = feat + i * MLP_IN;
  f[0] = lg((float)w);
  f[1] = lg((float)(cr.y - cr.x));
  f[2] = lg((float)do1);
  f[3] = lg((float)di0);
  f[4] = lg((float)do0);
  f[5] = lg((float)di1);
  f[6] = lg((float)(qd - q0));
  f[7] = delta > 0 ? (float)((double)(t_cl - ta) / delta) : 0.f;
  f[8] = lg((float)deg_o);
  f[9] = lg((float)deg_i);
  f[10] = ns ? s_deg / ns : 0.f;
  f[11] = m_deg;
  f[12] = lg((float)w * (float)(cr.y - cr.x));
  f[13] = do1 > 1000 ? 1.f : 0.f;
  f[14] = di0 > 1000 ? 1.f : 0.f;
  f[15] = (float)(K - 2) / 6.f;
}

// ------------------------------------------------------------- binning

constexpr int N_BUCKETS = 128;  // log-spaced cost buckets per queue

__device__ __forceinline__ int cost_bucket(float c) {
  const int b = (int)(log2f(1.f + fmaxf(c, 0.f)) * 4.f);
  return N_BUCKETS - 1 - min(max(b, 0), N_BUCKETS - 1);  // descending cost
}

// hist[q * N_BUCKETS + b]: queue q = 0 (warp) if cost >= thr, else 1 (thread)
__global__ void __launch_bounds__(256) k_bin_hist(const float* __restrict__ cost,
                                                  const int32_t* __restrict__ n_items, float thr,
                                                  int32_t* __restrict__ hist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *n_items) return;
  const float c = cost[i];
  atomicAdd(hist + (c >= thr ? 0 : N_BUCKETS) + cost_bucket(c), 1);
}

// cursor: exclusive prefix of hist (consumed); out = warp queue then thread queue
__global__ void __launch_bounds__(256) k_bin_scatter(const int32_t* __restrict__ items,
                                                     const float* __restrict__ cost,
                                                     const int32_t* __restrict__ n_items,
                                                     float thr, int32_t* __restrict__ cursor,
                                                     int32_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *n_items) return;
  const float c = cost[i];
  out[atomicAdd(cursor + (c >= thr ? 0 : N_BUCKETS) + cost_bucket(c), 1)] = items[i];
}

__global__ void k_gather_w2(const int32_t* __restrict__ items, const int32_t* __restrict__ n,
                            const int32_t* __restrict__ w2, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < *n) out[i] = (float)w2[items[i]];
}

// predicted log1p(cycles) -> cycles
__global__ void k_expm1(float* __restrict__ v, const int32_t* __restrict__ n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < *n) v[i] = expm1f(fmaxf(v[i], 0.f));
}

// ------------------------------------------------- persistent cycle search

struct CycPersist {
  GraphView g;
  int32_t delta;
  int K;
  CycleSlots slots;
  SubWindows sub;             // smaller windows' CYC columns (sub.cyc)
  unsigned long long* acc;
  const int2* crng;
  const int32_t* queue;       // warp items, then thread items
  const int32_t* n_warp;      // device counts of the two queues
  const int32_t* n_total;
  const int32_t* skip;        // queue entries before the warp items (null: none)
  unsigned long long* next;   // [2] zeroed: warp-queue and thread-queue cursors
  uint32_t* probe;            // clock64 cycles per thread item, or null
  int32_t close_scan_max;
};

// cycles of length L+1 closing from nodes[L] after edges[L-1] through B1,
// for the window and every smaller one that keeps the closing edge (an
// ordered cycle's latest edge)
__device__ __forceinline__ void cyc_close(const CycPersist& A, int L, const int32_t* edges,
                                          const int32_t* nodes, int2 cr) {
  const int k = L + 1;
  if (k > A.K) return;
  constexpr int NT = 1 + MAX_SUB;
  const GraphView& g = A.g;
  unsigned long long* col[NT];
  int64_t tmax[NT];
  unsigned long long c[NT];
  bool any = false;
  const int64_t ta = g.ts[edges[0]];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int sl = t == 0 ? A.slots.slot[k]
                          : (t - 1 < A.sub.n ? A.sub.cyc[t - 1].slot[k] : -1);
    col[t] = sl >= 0 ? A.acc + (int64_t)sl * g.E : nullptr;
    tmax[t] = ta + (t == 0 ? A.delta : (t - 1 < A.sub.n ? A.sub.delta[t - 1] : 0));
    c[t] = 0;
    any |= sl >= 0;
  }
  if (!any) return;
  const int32_t w = nodes[L], last = edges[L - 1], tl = g.ts[last];
  if (cr.y - cr.x <= A.close_scan_max) {
    for (int32_t q = cr.x; q < cr.y; ++q) {
      if (__ldg(g.inbr + q) != w) continue;
      const int32_t cid = __ldg(g.ieid + q), tq = __ldg(g.it + q);
      if (!before(tl, last, tq, cid)) continue;
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (col[t] && tq <= tmax[t]) {
          atomicAdd(col[t] + cid, 1ull);
          ++c[t];
        }
    }
  } else {
    const int32_t u0 = nodes[0];
    const int32_t in_s = g.iptr[u0], in_e = g.iptr[u0 + 1];
    int32_t r0, r1;
    nbr_range(g.innbr, in_s, in_e, w, r0, r1);
    if (r1 > r0) {
      int32_t b0, b1;
      after_edge_upto(g.int_, g.ineid, r0, r1, tl, last, tmax[0], b0, b1);
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
    if (c[t])
      for (int m = 0; m < L; ++m) atomicAdd(col[t] + edges[m], c[t]);
}

// every cycle whose earliest edge is e1 and whose second edge is the
// first-window slot q = first, first + step, ...
__device__ void cyc_anchor(const CycPersist& A, int32_t e1, int32_t first, int32_t step) {
  const GraphView& g = A.g;
  const int2 cr = A.crng[e1];
  if (cr.x >= cr.y) return;
  const int32_t t_cl = __ldg(g.it + cr.y - 1), id_cl = __ldg(g.ieid + cr.y - 1);
  int32_t edges[MAX_CYCLE], nodes[MAX_CYCLE + 1], cur[MAX_CYCLE], end[MAX_CYCLE];
  nodes[0] = g.src[e1];
  nodes[1] = g.dst[e1];
  edges[0] = e1;
  const int32_t u0 = nodes[0];
  const int32_t ws = g.optr[nodes[1]], we = g.optr[nodes[1] + 1];
  const int32_t q0 = after_edge(g.ot, g.oeid, ws, we, g.ts[e1], e1);
  const int32_t q1 = upper_t(g.ot, q0, we, t_cl);
  for (int32_t q2 = q0 + first; q2 < q1; q2 += step) {
    const int32_t x2 = __ldg(g.onbr + q2);
    const int32_t f2 = __ldg(g.oeid + q2);
    if (x2 == u0 || !before(__ldg(g.ot + q2), f2, t_cl, id_cl)) continue;
    edges[1] = f2;
    nodes[2] = x2;
    int L = 2;
    bool fresh = true;
    while (L >= 2) {
      if (fresh) {
        fresh = false;
        cyc_close(A, L, edges, nodes, cr);
        if (L + 1 <= A.K - 1) {
          const int32_t w = nodes[L], last = edges[L - 1];
          const int32_t s0 = g.optr[w], s1 = g.optr[w + 1];
          cur[L] = after_edge(g.ot, g.oeid, s0, s1, g.ts[last], last);
          end[L] = upper_t(g.ot, cur[L], s1, t_cl);
        } else {
          cur[L] = end[L] = 0;
        }
      }
      if (cur[L] >= end[L]) {
        --L;
        continue;
      }
      const int32_t q = cur[L]++;
      const int32_t x = __ldg(g.onbr + q);
      if (x == u0) continue;  // closing edges are counted through B1
      const int32_t f = __ldg(g.oeid + q);
      if (!before(__ldg(g.ot + q), f, t_cl, id_cl)) continue;
      bool seen = false;
      for (int m = 1; m <= L; ++m) seen |= (nodes[m] == x);
      if (seen) continue;
      edges[L] = f;
      nodes[L + 1] = x;
      ++L;
      fresh = true;
    }
  }
}

__global__ void __launch_bounds__(256) k_cyc_persistent(CycPersist A) {
  const int lane = threadIdx.x & 31;
  const int64_t n_warp = *A.n_warp, n_total = *A.n_total;
  const int32_t* queue = A.queue + (A.skip ? *A.skip : 0);
  // warp items: the whole warp splits the anchor's first window
  for (;;) {
    unsigned long long i = 0;
    if (lane == 0) i = atomicAdd(A.next, 1ull);
    i = __shfl_sync(0xffffffffu, i, 0);
    if ((int64_t)i >= n_warp) break;
    cyc_anchor(A, queue[i], lane, 32);
  }
  // thread items, 32 per warp pull
  const int64_t n_thread = n_total - n_warp;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(A.next + 1, 32ull);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((int64_t)base >= n_thread) break;
    const int64_t i = (int64_t)base + lane;
    if (i < n_thread) {
      const long long t0 = clock64();
      cyc_anchor(A, queue[n_warp + i], 0, 1);
      if (A.probe) A.probe[i] = (uint32_t)min(clock64() - t0, (long long)UINT32_MAX);
    }
  }
}

static int persistent_grid() {
  static int grid[64] = {0};
  int dev = 0;
  AML_CUDA(cudaGetDevice(&dev));
  if (dev < 64 && grid[dev]) return grid[dev];
  int sms = 0, per = 0;
  AML_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  AML_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cyc_persistent, 256, 0));
  const int gsz = sms * std::max(per, 1);
  if (dev < 64) grid[dev] = gsz;
  return gsz;
}

// ---------------------------------------------------------- the cycle step

// Items of one window: crng must hold the closing ranges.  Writes the item
// list, its device count and the first-window sizes (edge-indexed).
static void cyc_items(aml_graph* g, const GraphView& gv, int32_t delta, const int2* crng,
                      int32_t* items, int32_t* n_items, int32_t* w2, cudaStream_t s) {
  const int64_t E = g->E;
  DBuf<int32_t> flag(E + 1, s), off(E + 1, s);
  AML_LAUNCH("k_cyc_item_flags", s,
             k_cyc_item_flags<<<grid_for(E, 256), 256, 0, s>>>(gv, delta, crng, flag.p, w2));
  AML_CUDA(cudaMemsetAsync(flag.p + E, 0, 4, s));
  scan_i32(flag.p, off.p, E + 1, false, s);
  AML_LAUNCH("k_cyc_compact", s,
             k_cyc_compact<<<grid_for(E, 256), 256, 0, s>>>(flag.p, off.p, E, items));
  AML_CUDA(cudaMemcpyAsync(n_items, off.p + E, 4, cudaMemcpyDeviceToDevice, s));
}

// The hybrid split: about the first 1/HYB_HEAVY of the anchors, in
// descending estimated cost, are searched level by level (their work spread
// over the GPU); the rest, whose costs are small and similar, one lane each
// in the persistent kernel beside them.  Degree and learned binning get the
// same budget of heavy anchors, so the estimate that ranks costs better
// leaves the persistent launch the shorter tail.  The split takes whole cost
// buckets, so which anchors are heavy depends on their costs only, never on
// the order the queue was filled in (the sizes of the heavy anchors' search
// are learned once and reused).
constexpr int HYB_HEAVY = 4;

// ends[b] = end of cost bucket b in the queue (descending cost);
// ctl = {heavy anchors H, light anchors n - H, 0 (no warp items)}, H the
// first bucket end at or past n / HYB_HEAVY
__global__ void k_hyb_split(const int32_t* __restrict__ ends, const int32_t* __restrict__ n_items,
                            int32_t* __restrict__ ctl) {
  const int32_t n = *n_items;
  const int32_t target = n > 0 ? (n + HYB_HEAVY - 1) / HYB_HEAVY : 0;
  int32_t h = n;
  for (int b = 0; b < N_BUCKETS; ++b)
    if (ends[b] >= target) {
      h = ends[b];
      break;
    }
  ctl[0] = h;
  ctl[1] = n - h;
  ctl[2] = 0;
}

// the heavy legs found must be exactly the ones the buffers were sized for
__global__ void k_check_count(const int32_t* __restrict__ total, int64_t expect,
                              uint32_t* __restrict__ err) {
  if (*total != expect) atomicOr(err, ERR_BOUNDS);
}

// heavy[queue[i]] = 1 for the first ctl[0] queue entries
__global__ void __launch_bounds__(256) k_mark_heavy(const int32_t* __restrict__ queue,
                                                    const int32_t* __restrict__ ctl, int64_t cap,
                                                    int32_t* __restrict__ heavy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cap && i < ctl[0]) heavy[queue[i]] = 1;
}

// flag[i] = 1 for the cycle-capable legs of heavy anchors
__global__ void __launch_bounds__(256) k_heavy_legs(const int4* __restrict__ legs, int64_t n,
                                                    const int32_t* __restrict__ heavy,
                                                    int32_t* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = heavy[legs[i].x];
}

__global__ void __launch_bounds__(256) k_gather_legs(const int32_t* __restrict__ flag,
                                                     const int32_t* __restrict__ off, int64_t n,
                                                     const int4* __restrict__ legs,
                                                     int4* __restrict__ legs_h, int64_t cap,
                                                     uint32_t* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) {
    if (off[i] >= cap) {  // never written past the buffers; reported instead
      atomicOr(err, ERR_BOUNDS);
      return;
    }
    legs_h[off[i]] = legs[i];
  }
}

void cycles_hybrid(aml_graph* g, const GraphView& gv, int32_t delta, int K,
                   const CycleSlots& slots, const SubWindows& sub, unsigned long long* acc,
                   const int2* crng, const AnchorRec* anc, const int2* qwin, const int4* legs,
                   bool learned, cudaStream_t s, cudaStream_t side) {
  const int64_t E = g->E;
  LegCache& lc = g->legs[delta];
  const int64_t n2 = lc.n_front[2];  // all cycle-capable legs
  // anchors with cycle work and their estimated costs, one descending queue
  DBuf<int32_t> items(E, s), w2(E, s), nb(4, s), queue(E, s), hist(2 * N_BUCKETS + 1, s);
  cyc_items(g, gv, delta, crng, items.p, nb.p, w2.p, s);
  DBuf<float> cost(E, s);
  const CostModel* cm = nullptr;
  for (const CostModel& m : g->cost_models)
    if (m.delta == delta) cm = &m;
  const bool model = learned && cm;
  if (model) {
    DBuf<float> feat((size_t)E * MLP_IN, s);
    AML_LAUNCH("k_cyc_features", s,
               k_cyc_features<<<grid_for(E, 256), 256, 0, s>>>(gv, delta, K, items.p, nb.p,
                                                               crng, w2.p, feat.p));
    mlp_infer(device_of(*cm), feat.p, E, cost.p, s, nb.p);
    AML_LAUNCH("k_expm1", s, k_expm1<<<grid_for(E, 256), 256, 0, s>>>(cost.p, nb.p));
  } else {
    AML_LAUNCH("k_gather_w2", s,
               k_gather_w2<<<grid_for(E, 256), 256, 0, s>>>(items.p, nb.p, w2.p, cost.p));
  }
  const float no_warp = 3.0e38f;  // every item in the one (descending) queue
  AML_CUDA(cudaMemsetAsync(hist.p, 0, (2 * N_BUCKETS + 1) * 4, s));
  AML_LAUNCH("k_bin_hist", s,
             k_bin_hist<<<grid_for(E, 256), 256, 0, s>>>(cost.p, nb.p, no_warp, hist.p));
  scan_i32(hist.p, hist.p, 2 * N_BUCKETS + 1, false, s);
  AML_LAUNCH("k_bin_scatter", s,
             k_bin_scatter<<<grid_for(E, 256), 256, 0, s>>>(items.p, cost.p, nb.p, no_warp,
                                                            hist.p, queue.p));
  // the heaviest anchors' legs
  DBuf<int32_t> ctl(4, s), heavy(E, s);
  AML_LAUNCH("k_hyb_split", s, k_hyb_split<<<1, 1, 0, s>>>(hist.p + N_BUCKETS, nb.p, ctl.p));
  AML_CUDA(cudaMemsetAsync(heavy.p, 0, (size_t)E * 4, s));
  AML_LAUNCH("k_mark_heavy", s,
             k_mark_heavy<<<grid_for(E, 256), 256, 0, s>>>(queue.p, ctl.p, E, heavy.p));
  int64_t* cache = lc.n_hyb[model ? 1 : 0];
  DBuf<int32_t> fl((size_t)n2 + 1, s), off((size_t)n2 + 1, s);
  if (n2 > 0)
    AML_LAUNCH("k_heavy_legs", s,
               k_heavy_legs<<<grid_for(n2, 256), 256, 0, s>>>(legs, n2, heavy.p, fl.p));
  AML_CUDA(cudaMemsetAsync(fl.p + n2, 0, sizeof(int32_t), s));
  scan_i32(fl.p, off.p, n2 + 1, false, s);
  if (cache[2] < 0) {
    int32_t nh = 0;
    const SmallRead rd{&nh, off.p + n2, 4};
    read_small(&rd, 1, s);
    cache[2] = nh;
  }
  const int64_t cap = std::max<int64_t>(cache[2], 1);
  DBuf<int4> legs_h((size_t)cap, s);
  // valid edge and node ids whatever happens
  AML_CUDA(cudaMemsetAsync(legs_h.p, 0, (size_t)cap * sizeof(int4), s));
  if (n2 > 0)
    AML_LAUNCH("k_gather_legs", s,
               k_gather_legs<<<grid_for(n2, 256), 256, 0, s>>>(fl.p, off.p, n2, legs, legs_h.p,
                                                              cache[2], g->err));
  AML_LAUNCH("k_check_count", s, k_check_count<<<1, 1, 0, s>>>(off.p + n2, cache[2], g->err));
  // the other anchors: one persistent launch beside the level-by-level search
  DBuf<unsigned long long> next(2, s);
  AML_CUDA(cudaMemsetAsync(next.p, 0, 16, s));
  const bool fork = side != s;
  if (fork) {
    AML_CUDA(cudaEventRecord(g->branch_ev[4], s));
    AML_CUDA(cudaStreamWaitEvent(side, g->branch_ev[4], 0));
  }
  CycPersist A;
  A.g = gv;
  A.delta = delta;
  A.K = K;
  A.slots = slots;
  A.sub = sub;
  A.acc = acc;
  A.crng = crng;
  A.queue = queue.p;
  A.n_warp = ctl.p + 2;
  A.n_total = ctl.p + 1;
  A.skip = ctl.p;
  A.next = next.p;
  A.probe = nullptr;
  A.close_scan_max = g->tune.close_scan_max;
  AML_LAUNCH("k_cyc_persistent", side,
             k_cyc_persistent<<<persistent_grid(), 256, 0, side>>>(A));
  level_cycle_search(g, gv, delta, K, slots, sub, acc, anc, qwin, legs_h.p, cache, s);
  if (fork) {  // joined before the buffers above are released on s
    AML_CUDA(cudaEventRecord(g->branch_ev[5], side));
    AML_CUDA(cudaStreamWaitEvent(s, g->branch_ev[5], 0));
  }
}

// ------------------------------------------------------------- training

static double spearman(const std::vector<float>& a, const std::vector<float>& b) {
  const size_t n = a.size();
  auto ranks = [n](const std::vector<float>& v) {
    std::vector<size_t> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](size_t i, size_t j) { return v[i] < v[j]; });
    std::vector<double> r(n);
    for (size_t i = 0; i < n;) {  // average ranks of ties
      size_t j = i;
      while (j + 1 < n && v[idx[j + 1]] == v[idx[i]]) ++j;
      for (size_t k = i; k <= j; ++k) r[idx[k]] = 0.5 * (double)(i + j);
      i = j + 1;
    }
    return r;
  };
  std::vector<double> ra = ranks(a), rb = ranks(b);
  double ma = 0, mb = 0;
  for (size_t i = 0; i < n; ++i) {
    ma += ra[i];
    mb += rb[i];
  }
  ma /= n;
  mb /= n;
  double sab = 0, saa = 0, sbb = 0;
  for (size_t i = 0; i < n; ++i) {
    sab += (ra[i] - ma) * (rb[i] - mb);
    saa += (ra[i] - ma) * (ra[i] - ma);
    sbb += (rb[i] - mb) * (rb[i] - mb);
  }
  return (saa > 0 && sbb > 0) ? sab / std::sqrt(saa * sbb) : 0.0;
}

void cost_train(aml_graph* g, const aml_pattern_set* ps, int64_t max_samples, int epochs,
                uint64_t seed, cudaStream_t s, aml_cost_report* rep) {
  // the window whose cycle search the model will bin: the widest one with cycles
  int32_t delta = -1;
  int K = 0;
  CycleSlots slots;
  for (int k = 0; k <= MAX_CYCLE; ++k) slots.slot[k] = -1;
  for (const Column& c : ps->cols)
    if (c.family == AML_FAM_CYC && c.k >= 3 && c.delta >= delta) delta = c.delta;
  AML_REQUIRE(delta >= 0, AML_EINVAL, "the pattern set has no cycle column of length >= 3");
  int n_acc = 0;
  for (const Column& c : ps->cols)
    if (c.family == AML_FAM_CYC && c.delta == delta && c.k >= 3 && slots.slot[c.k] < 0) {
      slots.slot[c.k] = n_acc++;
      K = std::max(K, (int)c.k);
    }
  const auto t_start = std::chrono::steady_clock::now();
  const int64_t E = g->E;
  GraphView gv = view_of(g);
  DBuf<int2> crng(E, s);
  AML_LAUNCH("k_close_range", s,
             k_close_range<<<grid_for(E, 256), 256, 0, s>>>(gv, delta, crng.p, nullptr));
  DBuf<int32_t> items(E, s), w2(E, s), nb(4, s);
  cyc_items(g, gv, delta, crng.p, items.p, nb.p, w2.p, s);
  int32_t n_items = 0;
  AML_CUDA(cudaMemcpyAsync(&n_items, nb.p, 4, cudaMemcpyDeviceToHost, s));
  AML_CUDA(cudaStreamSynchronize(s));
  AML_REQUIRE(n_items >= 64, AML_EINVAL, "too few cycle work items to train on");
  // sample
  std::vector<int32_t> all(n_items);
  AML_CUDA(cudaMemcpy(all.data(), items.p, (size_t)n_items * 4, cudaMemcpyDeviceToHost));
  std::mt19937_64 rng(seed);
  std::shuffle(all.begin(), all.end(), rng);
  const int64_t n = std::min<int64_t>(n_items, std::max<int64_t>(max_samples, 64));
  all.resize(n);
  DBuf<int32_t> sample(n, s), nsd(4, s);
  int32_t hn[2] = {(int32_t)n, 0};  // n_total, n_warp = 0: every sample is a thread item
  AML_CUDA(cudaMemcpyAsync(sample.p, all.data(), n * 4, cudaMemcpyHostToDevice, s));
  AML_CUDA(cudaMemcpyAsync(nsd.p, hn, 8, cudaMemcpyHostToDevice, s));
  // features of the sample
  DBuf<float> feat((size_t)n * MLP_IN, s);
  AML_LAUNCH("k_cyc_features", s,
             k_cyc_features<<<grid_for(n, 256), 256, 0, s>>>(gv, delta, K, sample.p, nsd.p,
                                                             crng.p, w2.p, feat.p));
  // probe: the persistent kernel, one sample per lane, clock64 per item
  DBuf<unsigned long long> acc((size_t)std::max(n_acc, 1) * E, s), next(2, s);
  DBuf<uint32_t> cyc(n, s);
  AML_CUDA(cudaMemsetAsync(acc.p, 0, (size_t)std::max(n_acc, 1) * E * 8, s));
  AML_CUDA(cudaMemsetAsync(next.p, 0, 16, s));
  CycPersist A;
  std::memset(&A, 0, sizeof(A));  // no smaller windows, no skipped entries
  A.g = gv;
  A.delta = delta;
  A.K = K;
  A.slots = slots;
  A.acc = acc.p;
  A.crng = crng.p;
  A.queue = sample.p;
  A.n_warp = nsd.p + 1;
  A.n_total = nsd.p;
  A.next = next.p;
  A.probe = cyc.p;
  A.close_scan_max = g->tune.close_scan_max;
  const auto t_probe = std::chrono::steady_clock::now();
  AML_LAUNCH("k_cyc_persistent", s, k_cyc_persistent<<<persistent_grid(), 256, 0, s>>>(A));
  AML_CUDA(cudaStreamSynchronize(s));
  const double probe_ms = std::chrono::duration<double, std::milli>(
                              std::chrono::steady_clock::now() - t_probe)
                              .count();
  std::vector<float> hx((size_t)n * MLP_IN), hy(n), hw(n);
  std::vector<uint32_t> hc(n);
  std::vector<int32_t> hw2_all(E);
  AML_CUDA(cudaMemcpy(hx.data(), feat.p, hx.size() * 4, cudaMemcpyDeviceToHost));
  AML_CUDA(cudaMemcpy(hc.data(), cyc.p, n * 4, cudaMemcpyDeviceToHost));
  AML_CUDA(cudaMemcpy(hw2_all.data(), w2.p, E * 4, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < n; ++i) {
    hy[i] = std::log1p((float)hc[i]);
    hw[i] = (float)hw2_all[all[i]];
  }
  // normalization and an 80/20 split
  CostModel cm;
  cm.delta = delta;
  const int64_t n_tr = std::max<int64_t>(1, n * 4 / 5), n_te = n - n_tr;
  for (int k = 0; k < MLP_IN; ++k) {
    double m = 0, v = 0;
    for (int64_t i = 0; i < n_tr; ++i) m += hx[i * MLP_IN + k];
    m /= n_tr;
    for (int64_t i = 0; i < n_tr; ++i) v += (hx[i * MLP_IN + k] - m) * (hx[i * MLP_IN + k] - m);
    v /= n_tr;
    cm.mean[k] = (float)m;
    cm.inv_std[k] = v > 1e-12 ? (float)(1.0 / std::sqrt(v)) : 0.f;
  }
  {
    double m = 0, v = 0;
    for (int64_t i = 0; i < n_tr; ++i) m += hy[i];
    m /= n_tr;
    for (int64_t i = 0; i < n_tr; ++i) v += (hy[i] - m) * (hy[i] - m);
    cm.y_mean = (float)m;
    cm.y_std = (float)std::max(std::sqrt(v / n_tr), 1e-3);
  }
  std::vector<float> xn(hx.size()), yn(n);
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < MLP_IN; ++k)
      xn[i * MLP_IN + k] = (hx[i * MLP_IN + k] - cm.mean[k]) * cm.inv_std[k];
    yn[i] = (hy[i] - cm.y_mean) / cm.y_std;
  }
  // He-style initialization, Adam on minibatches of 4096
  std::vector<float> p(MLP_NPARAM, 0.f);
  std::normal_distribution<float> nd(0.f, 1.f);
  for (int i = 0; i < MLP_H * MLP_IN; ++i) p[MLP_W1 + i] = nd(rng) * std::sqrt(2.f / MLP_IN);
  for (int i = 0; i < MLP_H * MLP_H; ++i) p[MLP_W2 + i] = nd(rng) * std::sqrt(2.f / MLP_H);
  for (int i = 0; i < MLP_H; ++i) p[MLP_W3 + i] = nd(rng) * std::sqrt(1.f / MLP_H);
  void* dparams = dalloc(MLP_NPARAM * 4, s);  // kept with the graph, freed with it
  cm.params = static_cast<float*>(dparams);
  g->allocs.push_back(dparams);
  AML_CUDA(cudaMemcpyAsync(cm.params, p.data(), MLP_NPARAM * 4, cudaMemcpyHostToDevice, s));
  AML_CUDA(cudaStreamSynchronize(s));
  DBuf<float> m(MLP_NPARAM, s), v(MLP_NPARAM, s), grad(MLP_NPARAM, s), loss(1, s);
  AML_CUDA(cudaMemsetAsync(m.p, 0, MLP_NPARAM * 4, s));
  AML_CUDA(cudaMemsetAsync(v.p, 0, MLP_NPARAM * 4, s));
  DBuf<float> dx((size_t)n_tr * MLP_IN, s), dy((size_t)n_tr, s);
  std::vector<int64_t> perm(n_tr);
  std::iota(perm.begin(), perm.end(), 0);
  std::vector<float> bx((size_t)n_tr * MLP_IN), by(n_tr);
  const int64_t B = 4096;
  int step = 0;
  float last_loss = 0.f;
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(perm.begin(), perm.end(), rng);
    for (int64_t i = 0; i < n_tr; ++i) {
      std::memcpy(&bx[i * MLP_IN], &xn[perm[i] * MLP_IN], MLP_IN * 4);
      by[i] = yn[perm[i]];
    }
    AML_CUDA(cudaMemcpyAsync(dx.p, bx.data(), bx.size() * 4, cudaMemcpyHostToDevice, s));
    AML_CUDA(cudaMemcpyAsync(dy.p, by.data(), by.size() * 4, cudaMemcpyHostToDevice, s));
    double ep_loss = 0;
    for (int64_t b0 = 0; b0 < n_tr; b0 += B) {
      const int64_t nb2 = std::min(B, n_tr - b0);
      mlp_grad(cm.params, dx.p + b0 * MLP_IN, dy.p + b0, nb2, 1.f / (float)nb2, grad.p, loss.p,
             s);
      mlp_adam(cm.params, grad.p, m.p, v.p, MLP_NPARAM, ++step, 2e-3f, 0.9f, 0.999f, 1e-8f, s);
      float l = 0;
      AML_CUDA(cudaMemcpyAsync(&l, loss.p, 4, cudaMemcpyDeviceToHost, s));
      AML_CUDA(cudaStreamSynchronize(s));
      ep_loss += l;
    }
    last_loss = (float)(ep_loss / n_tr);
  }
  // held-out evaluation: model vs the degree proxy
  std::vector<float> pred(std::max<int64_t>(n_te, 1));
  if (n_te > 0) {
    DBuf<float> fx((size_t)n_te * MLP_IN, s), fo(n_te, s);
    AML_CUDA(cudaMemcpyAsync(fx.p, hx.data() + n_tr * MLP_IN, n_te * MLP_IN * 4,
                             cudaMemcpyHostToDevice, s));
    mlp_infer(device_of(cm), fx.p, n_te, fo.p, s);
    AML_CUDA(cudaMemcpyAsync(pred.data(), fo.p, n_te * 4, cudaMemcpyDeviceToHost, s));
    AML_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<float> yt(hy.begin() + n_tr, hy.end()), wt(hw.begin() + n_tr, hw.end());
  pred.resize(n_te);
  double mae = 0;
  for (int64_t i = 0; i < n_te; ++i) mae += std::fabs(pred[i] - yt[i]);
  // warp threshold in cycles: the median cost of training items whose first
  // window is about own_max long (where degree binning switches to warps)
  std::vector<float> near;
  const int own = std::max(1, g->tune.own_max);
  for (int64_t i = 0; i < n_tr; ++i)
    if (hw[i] >= own / 2.0f && hw[i] <= own * 2.0f) near.push_back((float)hc[i]);
  if (near.empty()) {
    cm.warp_threshold = 1e30f;
  } else {
    std::nth_element(near.begin(), near.begin() + near.size() / 2, near.end());
    cm.warp_threshold = near[near.size() / 2];
  }
  for (size_t i = 0; i < g->cost_models.size(); ++i)
    if (g->cost_models[i].delta == delta) g->cost_models.erase(g->cost_models.begin() + i);
  g->cost_models.push_back(cm);
  // a new model picks new heavy anchors: forget their frontier sizes and the
  // mines captured with them
  for (auto& kv : g->legs)
    for (int j = 0; j < 16; ++j) kv.second.n_hyb[1][j] = -1;
  drop_captured_mines(g);
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->delta = delta;
    rep->n_items = n_items;
    rep->n_train = n_tr;
    rep->n_test = n_te;
    rep->epochs = epochs;
    rep->final_train_mse = last_loss;
    rep->test_log_mae = n_te ? (float)(mae / n_te) : 0.f;
    rep->test_spearman = n_te > 1 ? (float)spearman(pred, yt) : 0.f;
    rep->degree_spearman = n_te > 1 ? (float)spearman(wt, yt) : 0.f;
    rep->warp_threshold_cycles = cm.warp_threshold;
    rep->probe_ms = (float)probe_ms;
    rep->total_ms = (float)std::chrono::duration<double, std::milli>(
                        std::chrono::steady_clock::now() - t_start)
                        .count();
  }
}

}  // namespace aml

using namespace aml;

extern "C" aml_status aml_cost_train(aml_graph* g, const aml_pattern_set* ps, int64_t max_samples,
                                     int32_t epochs, uint64_t seed, void* stream,
                                     aml_cost_report* report) {
  try {
    AML_REQUIRE(g && ps, AML_EINVAL, "NULL graph or pattern set");
    AML_REQUIRE(max_samples >= 64 && epochs >= 1 && epochs <= 1000, AML_EINVAL,
                "max_samples >= 64 and epochs in [1, 1000]");
    g->note_stream(static_cast<cudaStream_t>(stream));
    cost_train(g, ps, max_samples, epochs, seed, static_cast<cudaStream_t>(stream), report);
    return AML_OK;
  } catch (const Failure& f) {
    set_error(std::string("aml_cost_train: ") + f.msg);
    return f.status;
  } catch (...) {
    set_error("aml_cost_train: unexpected internal error");
    return AML_EINTERNAL;
  }
}
