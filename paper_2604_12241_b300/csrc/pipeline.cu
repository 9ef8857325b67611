// Host side of a mine: plans the per-window work and enqueues the kernels.
#include <algorithm>
#include <climits>
#include <cstring>
#include <set>

#include "aml_internal.cuh"
#include "mine.cuh"

namespace aml {

namespace {

struct WindowPlan {
  int32_t delta = 0;
  bool fan_out = false, fan_in = false, sg = false;
  int sg_slot = -1;
  CycleSlots cyc;
  int K = 0;  // longest cycle wanted
  bool needs_legs() const { return sg || K >= 2; }
};

}  // namespace

// Leg offsets of a window depend only on the graph, so they are computed on
// the first mine that needs them and kept with the graph.
static LegCache& leg_offsets(aml_graph* g, const GraphView& gv, int32_t delta, cudaStream_t s) {
  LegCache& lc = g->legs[delta];
  if (lc.n_legs >= 0) return lc;
  const int64_t E = g->E;
  DBuf<int32_t> L(E + 1, s);
  k_leg_count<<<grid_for(E, 256), 256, 0, s>>>(gv, delta, L.p);
  AML_CUDA(cudaGetLastError());
  AML_CUDA(cudaMemsetAsync(L.p + E, 0, sizeof(int32_t), s));
  void* off = nullptr;
  AML_CUDA(cudaMalloc(&off, (size_t)(E + 1) * sizeof(int64_t)));
  g->allocs.push_back(off);
  g->bytes += (E + 1) * 8;
  scan_i32_to_i64(L.p, static_cast<int64_t*>(off), E + 1, s);
  int64_t total = 0;
  AML_CUDA(cudaMemcpyAsync(&total, static_cast<int64_t*>(off) + E, sizeof(int64_t),
                           cudaMemcpyDeviceToHost, s));
  AML_CUDA(cudaStreamSynchronize(s));
  AML_REQUIRE(total < (int64_t)UINT32_MAX, AML_EUNSUPPORTED,
              "more than 2^32 temporal 2-paths in one window");
  lc.off = static_cast<int64_t*>(off);
  lc.n_legs = total;
  return lc;
}

void mine_plain(aml_graph* g, const aml_pattern_set* ps, uint32_t* counts, int64_t ld,
                cudaStream_t s) {
  const int64_t E = g->E;
  const int ncols = (int)ps->cols.size();
  AML_REQUIRE(ncols <= MAX_COLS, AML_EUNSUPPORTED, "too many columns in one pattern set");
  if (E == 0) return;
  GraphView gv = view_of(g);

  // windows and accumulator columns
  std::vector<WindowPlan> wins;
  AssembleParams P;
  std::memset(&P, 0, sizeof(P));
  int n_acc = 0;
  for (int c = 0; c < ncols; ++c) {
    const Column& col = ps->cols[c];
    int didx = -1;
    for (size_t w = 0; w < wins.size(); ++w)
      if (wins[w].delta == col.delta) didx = (int)w;
    if (didx < 0) {
      AML_REQUIRE(wins.size() < (size_t)MAX_DELTAS, AML_EUNSUPPORTED, "too many windows");
      WindowPlan wp;
      wp.delta = col.delta;
      for (int k = 0; k <= MAX_CYCLE; ++k) wp.cyc.slot[k] = -1;
      wins.push_back(wp);
      didx = (int)wins.size() - 1;
    }
    WindowPlan& wp = wins[didx];
    ColDesc cd{col.family, col.k, col.delta, didx, -1};
    switch (col.family) {
      case AML_FAM_FAN_OUT: wp.fan_out = true; break;
      case AML_FAM_FAN_IN: wp.fan_in = true; break;
      case AML_FAM_SG:
        if (wp.sg_slot < 0) wp.sg_slot = n_acc++;
        wp.sg = true;
        cd.acc_slot = wp.sg_slot;
        break;
      case AML_FAM_CYC:
        AML_REQUIRE(col.k >= 2 && col.k <= MAX_CYCLE, AML_EUNSUPPORTED, "cycle length");
        if (wp.cyc.slot[col.k] < 0) wp.cyc.slot[col.k] = n_acc++;
        wp.K = std::max(wp.K, (int)col.k);
        cd.acc_slot = wp.cyc.slot[col.k];
        break;
      default: break;
    }
    P.cols[c] = cd;
  }
  P.g = gv;
  P.ncols = ncols;
  P.counts = counts;
  P.ld = ld;

  DBuf<unsigned long long> acc((size_t)std::max(n_acc, 1) * E, s);
  if (n_acc) AML_CUDA(cudaMemsetAsync(acc.p, 0, (size_t)n_acc * E * 8, s));
  P.acc = acc.p;

  std::vector<DBuf<int32_t>> fan_bufs;
  fan_bufs.reserve(2 * wins.size());
  const int B = 256;
  for (size_t w = 0; w < wins.size(); ++w) {
    WindowPlan& wp = wins[w];
    for (int dir = 0; dir < 2; ++dir) {
      bool want = dir == 0 ? wp.fan_out : wp.fan_in;
      if (!want || g->Ev == 0) continue;
      const Adj& a = dir == 0 ? g->out : g->in;
      fan_bufs.emplace_back((size_t)g->Ev, s);
      int32_t* D = fan_bufs.back().p;
      k_fan_delta<<<grid_for(g->Ev, B), B, 0, s>>>(a.ptr, a.t, a.eid, a.prev, a.next,
                                                   dir == 0 ? g->src : g->dst, g->Ev, wp.delta, D);
      AML_CUDA(cudaGetLastError());
      scan_i32(D, D, g->Ev, true, s);
      (dir == 0 ? P.S_out : P.S_in)[w] = D;
    }
    if (!wp.needs_legs()) continue;
    LegCache& lc = leg_offsets(g, gv, wp.delta, s);
    const int64_t nl = lc.n_legs;
    DBuf<int32_t> la(nl, s), lb(nl, s);
    DBuf<uint64_t> key(wp.sg ? nl : 0, s);
    unsigned long long* acc2 = wp.cyc.slot[2] >= 0 ? acc.p + (int64_t)wp.cyc.slot[2] * E : nullptr;
    k_leg_emit<<<grid_for(E, B), B, 0, s>>>(gv, wp.delta, lc.off, la.p, lb.p,
                                            wp.sg ? key.p : nullptr, g->N, acc2);
    AML_CUDA(cudaGetLastError());
    if (wp.sg && nl > 1) {
      DBuf<uint32_t> idx(nl, s), itmp(nl, s);
      DBuf<uint64_t> ktmp(nl, s);
      iota_i32(reinterpret_cast<int32_t*>(idx.p), nl, s);
      uint64_t max_key = (uint64_t)g->N * (uint64_t)g->N;
      radix_sort_u64(key.p, idx.p, ktmp.p, itmp.p, nl, bits_for(max_key), s);
      k_sg_group<<<grid_for(nl, B), B, 0, s>>>(key.p, idx.p, nl, la.p, lb.p, g->dst, g->ts,
                                               wp.delta, acc.p + (int64_t)wp.sg_slot * E);
      AML_CUDA(cudaGetLastError());
    }
    if (wp.K >= 3 && nl > 0) {
      k_cycles<<<grid_for(nl, 128), 128, 0, s>>>(gv, wp.delta, wp.K, la.p, lb.p, nl, wp.cyc,
                                                  acc.p);
      AML_CUDA(cudaGetLastError());
    }
  }
  k_assemble<<<grid_for(E, B), B, 0, s>>>(P);
  AML_CUDA(cudaGetLastError());
}

}  // namespace aml
