// Host side of a mine: plans the per-window work and enqueues the kernels.
//
// Per window delta, in order:
//   1. window starts (and FAN repeat deltas + scan) of the out- and in-slots;
//   2. legs: count per edge, scan to offsets, emit (a, b) pairs, crediting
//      2-cycles and counting the legs that end at each edge;
//   3. SG: bucket the leg records by a hash of (s, d), then per bucket group
//      them by (s, d) in shared memory and count partner legs;
//   4. CYC_3..K: closing ranges, then the legs extended level by level;
// and finally one pass writes every output row.  All of it is enqueued on
// the caller's stream; only the first mine of a (graph, window) pair waits
// once for the number of legs, to size the leg buffers.
#include <algorithm>
#include <climits>
#include <cstring>

#include "aml_internal.cuh"
#include "mine.cuh"
#include "profile.cuh"

namespace aml {

namespace {

struct WindowPlan {
  int32_t delta = 0;
  bool deg_out = false, deg_in = false, fan_out = false, fan_in = false;
  bool gs = false, sg = false;
  int sg_slot = -1;
  CycleSlots cyc;
  int K = 0;  // longest cycle wanted
  CycleSlots cycw;  // window cycles
  int Kw = 0;
  bool emit_legs() const { return sg || K >= 2; }
  bool needs_off() const { return gs || emit_legs(); }
};

// Side streams for a mine's independent branches (DEG/FAN beside the leg
// pass; SG beside the cycle search), created outside any capture; false if
// they do not exist and cannot be made now (the mine then runs in order).
bool ensure_branches(aml_graph* g, cudaStream_t s) {
  if (g->side[2] && g->branch_ev[5]) return true;
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  AML_CUDA(cudaStreamIsCapturing(s, &st));
  if (st != cudaStreamCaptureStatusNone) return false;
  for (cudaStream_t& x : g->side)
    if (!x) AML_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
  for (cudaEvent_t& e : g->branch_ev)
    if (!e) AML_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return true;
}

// work enqueued on `to` from now on runs after what `from` holds so far
void branch_wait(cudaEvent_t ev, cudaStream_t from, cudaStream_t to) {
  AML_CUDA(cudaEventRecord(ev, from));
  AML_CUDA(cudaStreamWaitEvent(to, ev, 0));
}

}  // namespace

// Window cycles of one window (and the smaller ones in sw): closing ranges,
// the anchors (edges with one) as level 1, then the paths level by level.
void window_cycle_search(aml_graph* g, const GraphView& gv, int32_t delta, int K,
                         const CycleSlots& slots, const SubWindows& sw,
                         unsigned long long* acc, cudaStream_t s) {
  const int64_t E = g->E;
  const Tuning tn = g->tune;
  const int B = tn.block;
  LegCache& lc = g->legs[delta];
  DBuf<int2> crng((size_t)E, s);
  AML_LAUNCH("k_close_range", s,
             k_close_range<<<grid_for(E, B), B, 0, s>>>(gv, delta, crng.p, nullptr));
  DBuf<int32_t> flag((size_t)E + 1, s), off((size_t)E + 1, s);
  AML_LAUNCH("k_anchor_flags", s,
             k_anchor_flags<<<grid_for(E, 256), 256, 0, s>>>(crng.p, E, flag.p));
  AML_CUDA(cudaMemsetAsync(flag.p + E, 0, sizeof(int32_t), s));
  scan_i32(flag.p, off.p, E + 1, false, s);
  int64_t& n1 = lc.n_wfront[1];
  if (n1 < 0) {
    int32_t n = 0;
    const SmallRead rd{&n, off.p + E, 4};
    read_small(&rd, 1, s);
    n1 = n;
  }
  DBuf<int32_t> anchors((size_t)std::max<int64_t>(n1, 1), s);
  AML_LAUNCH("k_compact_ids", s,
             k_compact_ids<<<grid_for(E, 256), 256, 0, s>>>(flag.p, off.p, E, anchors.p));
  CycFrontier F;
  std::memset(&F, 0, sizeof(F));
  F.base = 1;
  F.la = anchors.p;
  std::vector<DBuf<int32_t>> front;  // par/slot of levels >= 2
  front.reserve(2 * MAX_CYCLE);
  int64_t n = n1;
  for (int j = 1; j <= K - 1 && n > 0; ++j) {
    const bool has_next = j + 1 <= K - 1;
    DBuf<int32_t> cnt(has_next ? n + 1 : 0, s), q0(has_next ? n : 0, s);
    launch_cyc_level(grid_for(n, B), B, s, gv, delta, K, j, F, n, crng.p, nullptr, nullptr,
                     slots, acc, cnt.p, q0.p, tn.close_scan_max, sw, true);  // window cycles
    if (!has_next) break;
    DBuf<int64_t> foff(n + 1, s);
    AML_CUDA(cudaMemsetAsync(cnt.p + n, 0, sizeof(int32_t), s));
    scan_i32_to_i64(cnt.p, foff.p, n + 1, s);
    int64_t& nn = lc.n_wfront[j + 1];
    if (nn < 0) {  // cached only once it is known to fit
      int64_t got = 0;
      const SmallRead rd{&got, foff.p + n, 8};
      read_small(&rd, 1, s);
      AML_REQUIRE(got < (int64_t)INT32_MAX, AML_EUNSUPPORTED,
                  "window-cycle frontier above 2^31 paths");
      nn = got;
    }
    front.emplace_back((size_t)nn, s);
    int32_t* par = front.back().p;
    front.emplace_back((size_t)nn, s);
    int32_t* slot = front.back().p;
    AML_LAUNCH("k_cyc_emit", s,
               k_cyc_emit<<<grid_for(n, B), B, 0, s>>>(n, cnt.p, q0.p, foff.p, par, slot,
                                                       tn.own_max));
    F.par[j + 1] = par;
    F.slot[j + 1] = slot;
    n = nn;
  }
}

// Ordered cycles of length 3..K (and the sub-windows' ones), level by level
// from the n = front_cache[2] cycle-capable legs (la, lb); front_cache[j]
// caches the number of paths of j edges (-1: not known yet, learned once
// with one wait per level).
void level_cycle_search(aml_graph* g, const GraphView& gv, int32_t delta, int K,
                        const CycleSlots& slots, const SubWindows& sub,
                        unsigned long long* acc, const AnchorRec* anc, const int2* qwin,
                        const int4* legs, int64_t* front_cache, cudaStream_t s) {
  const Tuning tn = g->tune;
  const int B = tn.block;
  CycFrontier F;
  std::memset(&F, 0, sizeof(F));
  F.base = 2;
  F.leg = legs;
  std::vector<DBuf<int32_t>> front;  // par/slot of levels >= 3
  front.reserve(2 * MAX_CYCLE);
  int64_t n = front_cache[2];
  for (int j = 2; j <= K - 1 && n > 0; ++j) {
    const bool has_next = j + 1 <= K - 1;
    DBuf<int32_t> cnt(has_next ? n + 1 : 0, s), q0(has_next ? n : 0, s);
    launch_cyc_level(grid_for(n, B), B, s, gv, delta, K, j, F, n, nullptr, anc, qwin, slots, acc,
                     cnt.p, q0.p, tn.close_scan_max, sub);
    if (!has_next) break;
    DBuf<int64_t> foff(n + 1, s);
    AML_CUDA(cudaMemsetAsync(cnt.p + n, 0, sizeof(int32_t), s));
    scan_i32_to_i64(cnt.p, foff.p, n + 1, s);
    int64_t& nn = front_cache[j + 1];
    if (nn < 0) {  // cached only once it is known to fit
      int64_t got = 0;
      const SmallRead rd{&got, foff.p + n, 8};
      read_small(&rd, 1, s);
      AML_REQUIRE(got < (int64_t)INT32_MAX, AML_EUNSUPPORTED, "cycle frontier above 2^31 paths");
      nn = got;
    }
    front.emplace_back((size_t)nn, s);
    int32_t* par = front.back().p;
    front.emplace_back((size_t)nn, s);
    int32_t* slot = front.back().p;
    AML_LAUNCH("k_cyc_emit", s,
               k_cyc_emit<<<grid_for(n, B), B, 0, s>>>(n, cnt.p, q0.p, foff.p, par, slot,
                                                       tn.own_max));
    F.par[j + 1] = par;
    F.slot[j + 1] = slot;
    n = nn;
  }
}

void mine_plain(aml_graph* g, const aml_pattern_set* ps, uint32_t* counts, int64_t ld,
                cudaStream_t s, uint32_t mode, int32_t new_from, int32_t t_new, bool accumulate) {
  const bool persistent = (mode & (AML_MINE_PERSISTENT | AML_MINE_LEARNED)) != 0;
  const int64_t E = g->E;
  const int ncols = (int)ps->cols.size();
  AML_REQUIRE(ncols <= MAX_COLS, AML_EUNSUPPORTED, "too many columns in one pattern set");
  if (E == 0) return;
  GraphView gv = view_of(g);
  gv.new_from = new_from;
  gv.t_new = t_new;

  // windows and accumulator columns
  std::vector<WindowPlan> wins;
  AssembleParams P;
  std::memset(&P, 0, sizeof(P));
  int n_acc = 0;
  std::vector<std::pair<int, int>> programs;  // (accumulator slot, program)
  for (int c = 0; c < ncols; ++c) {
    const Column& col = ps->cols[c];
    int didx = -1;
    for (size_t w = 0; w < wins.size(); ++w)
      if (wins[w].delta == col.delta) didx = (int)w;
    if (didx < 0) {
      AML_REQUIRE(wins.size() < (size_t)MAX_DELTAS, AML_EUNSUPPORTED, "too many windows");
      WindowPlan wp;
      wp.delta = col.delta;
      for (int k = 0; k <= MAX_CYCLE; ++k) wp.cyc.slot[k] = wp.cycw.slot[k] = -1;
      wins.push_back(wp);
      didx = (int)wins.size() - 1;
    }
    WindowPlan& wp = wins[didx];
    ColDesc cd{col.family, col.k, col.delta, didx, -1};
    switch (col.family) {
      case AML_FAM_DEG_OUT: wp.deg_out = true; break;
      case AML_FAM_DEG_IN: wp.deg_in = true; break;
      case AML_FAM_FAN_OUT: wp.fan_out = true; break;
      case AML_FAM_FAN_IN: wp.fan_in = true; break;
      case AML_FAM_GS: wp.gs = true; break;
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
      case AML_FAM_CYCW:
        AML_REQUIRE(col.k >= 3 && col.k <= MAX_CYCLE, AML_EUNSUPPORTED, "cycle length");
        AML_REQUIRE(new_from == 0, AML_EUNSUPPORTED, "window cycles are not counted incrementally");
        if (wp.cycw.slot[col.k] < 0) wp.cycw.slot[col.k] = n_acc++;
        wp.Kw = std::max(wp.Kw, (int)col.k);
        cd.acc_slot = wp.cycw.slot[col.k];
        break;
      case AML_FAM_PROGRAM:
        AML_REQUIRE(new_from == 0, AML_EUNSUPPORTED,
                    "interpreted stage programs are not counted incrementally");
        cd.acc_slot = n_acc++;
        programs.emplace_back(cd.acc_slot, col.prog);
        break;
      default: break;
    }
    P.cols[c] = cd;
  }
  P.g = gv;
  P.ncols = ncols;
  P.counts = counts;
  P.ld = ld;
  P.limit = g->count_limit;
  P.accumulate_from = accumulate && new_from > 0 ? new_from : -1;
  for (int c = 0; c < ncols; ++c) {
    const uint32_t f = ps->cols[c].family;
    if (f == AML_FAM_GS || f == AML_FAM_SG || f == AML_FAM_CYC || f == AML_FAM_CYCW)
      P.inst_mask |= 1ull << c;
  }

  // zeroed by the first leg count (before any kernel adds into it), or
  // below when no window counts legs
  DBuf<unsigned long long> acc((size_t)std::max(n_acc, 1) * E, s);
  bool acc_zeroed = n_acc == 0;
  P.acc = acc.p;

  // Smaller windows whose GS/SG/CYC columns are counted from the largest
  // leg-emitting window's pass (sub-windows; not when they want longer
  // cycles).
  std::vector<int> owner(wins.size(), -1);
  std::vector<std::vector<int>> members(wins.size());
  {
    int lw = -1;
    for (size_t w = 0; w < wins.size(); ++w)
      if (wins[w].emit_legs() && (lw < 0 || wins[w].delta > wins[lw].delta)) lw = (int)w;
    for (size_t w = 0; lw >= 0 && w < wins.size(); ++w) {
      const WindowPlan& wp = wins[w];
      if ((int)w == lw || !wp.needs_off() || wp.delta > wins[lw].delta) continue;
      if (wp.K >= 3 && wp.K > wins[lw].K) continue;
      if (members[lw].size() >= (size_t)MAX_SUB) continue;
      owner[w] = lw;
      members[lw].push_back((int)w);
    }
  }

  std::vector<DBuf<int32_t>> keep32;   // per-window buffers read by k_assemble
  std::vector<DBuf<int64_t>> keep64;
  std::vector<DBuf<int2>> keep_df;
  keep_df.reserve(2 * wins.size());
  keep32.reserve(8 * wins.size());
  keep64.reserve(wins.size());
  const Tuning tn = g->tune;
  const int B = tn.block;
  const int64_t Ev = g->Ev;
  // 1. trailing windows, per direction: (DEG, FAN) of every window at once
  // when any wants FAN (groups of FAN_MAX_W, largest delta first), else DEG
  // alone window by window.  Planned and allocated here, launched below.
  struct DfJob {
    const Adj* a;
    int nw;
    bool fan;
    int32_t deltas[FAN_MAX_W];
    int2* df;
  };
  std::vector<DfJob> df_jobs;
  for (int dir = 0; dir < 2 && Ev > 0; ++dir) {
    std::vector<int> ws;
    bool any_fan = false;
    for (size_t w = 0; w < wins.size(); ++w) {
      const WindowPlan& wp = wins[w];
      const bool fan = dir == 0 ? wp.fan_out : wp.fan_in;
      const bool deg = dir == 0 ? wp.deg_out : wp.deg_in;
      if (fan || deg) ws.push_back((int)w);
      any_fan |= fan;
    }
    std::sort(ws.begin(), ws.end(), [&](int x, int y) { return wins[x].delta > wins[y].delta; });
    const int group = any_fan ? FAN_MAX_W : 1;
    for (size_t g0 = 0; g0 < ws.size(); g0 += group) {
      DfJob job{dir == 0 ? &g->out : &g->in, (int)std::min<size_t>(group, ws.size() - g0),
                any_fan, {}, nullptr};
      keep_df.emplace_back((size_t)E * DF_STRIDE, s);
      job.df = keep_df.back().p;
      for (int k = 0; k < job.nw; ++k) {
        const int w = ws[g0 + k];
        job.deltas[k] = wins[w].delta;
        (dir == 0 ? P.df_out : P.df_in)[w] = job.df + k;
      }
      df_jobs.push_back(job);
    }
  }

  // Independent branches run on side streams (full mines only; not while
  // kernels are timed one by one): buffers used across streams are
  // allocated on s before the fork and freed on s after the join.
  const bool branches = new_from == 0 && !profiling_enabled() && ensure_branches(g, s);
  cudaStream_t s_fan = branches ? g->side[0] : s;
  cudaStream_t s_sg = branches ? g->side[1] : s;
  if (branches) branch_wait(g->branch_ev[0], s, s_fan);
  for (const DfJob& job : df_jobs) {
    if (job.fan) {
      fan_per_edge(*job.a, Ev, E, new_from, job.nw, job.deltas, job.df, s_fan);
    } else {
      AML_LAUNCH("k_window_slots", s_fan,
                 k_window_slots<<<grid_for(Ev, B), B, 0, s_fan>>>(
                     job.a->rstart, job.a->t, job.a->eid, job.a->prev, job.a->next, Ev,
                     job.deltas[0], nullptr, nullptr, job.df));
    }
  }
  if (branches) AML_CUDA(cudaEventRecord(g->branch_ev[1], s_fan));  // joined before assembly

  for (size_t w = 0; w < wins.size(); ++w) {
    WindowPlan& wp = wins[w];
    if (!wp.needs_off() || owner[w] >= 0) continue;
    // sub-windows counted from this window's legs
    SubWindows sub;
    std::memset(&sub, 0, sizeof(sub));
    bool sg_any = wp.sg;
    for (int m : members[w]) {
      const WindowPlan& mp = wins[m];
      const int i = sub.n++;
      sub.delta[i] = mp.delta;
      sub.cyc[i] = mp.cyc;
      if (mp.gs) {
        keep32.emplace_back((size_t)E, s);
        sub.gs_from[i] = keep32.back().p;
        keep32.emplace_back((size_t)E, s);
        sub.gs_in[i] = keep32.back().p;  // zeroed by k_leg_count
        P.gs_from[m] = sub.gs_from[i];
        P.gs_in[m] = sub.gs_in[i];
      }
      if (mp.cyc.slot[2] >= 0) sub.cyc2[i] = acc.p + (int64_t)mp.cyc.slot[2] * E;
      if (mp.sg) sub.sg[i] = acc.p + (int64_t)mp.sg_slot * E;
      sg_any |= mp.sg;
    }
    // 2. legs (and, for the level-by-level cycle search, the legs that can
    // start a cycle: those of anchors with a closing range, before its end)
    const bool level_cycles = wp.K >= 3;
    // closing ranges: anchor records for the level-by-level search (those
    // of the edges with legs, computed by the leg count), and for the
    // persistent modes' kernels the plain ranges of every edge (a pass of
    // their own)
    DBuf<int2> crng;
    DBuf<AnchorRec> anc;
    DBuf<int32_t> L2;
    DBuf<int64_t> off2;
    if (level_cycles) {
      anc = DBuf<AnchorRec>((size_t)E, s);
      if (persistent) {
        crng = DBuf<int2>((size_t)E, s);
        AML_LAUNCH("k_close_range", s,
                   k_close_range<<<grid_for(E, B), B, 0, s>>>(gv, wp.delta, crng.p, anc.p));
      }
      L2 = DBuf<int32_t>((size_t)E + 1, s);
      off2 = DBuf<int64_t>((size_t)E + 1, s);
    }
    // 3. scatter-gather: bucket the n_rec leg records, group each bucket by
    // (s, d) (beside the cycle search: disjoint accumulator columns); true
    // when that runs on the SG branch, which the caller joins back to s.
    // skip: a device error word that, once set, leaves the records alone.
    auto sg_group = [&](const LegRec* recp, uint32_t* histp, int64_t nbk, int bits,
                        int64_t n_rec, KeySet ks, const uint32_t* skip) {
      const bool on_branch = branches && sg_any && n_rec > 1;
      if (on_branch) branch_wait(g->branch_ev[2], s, s_sg);
      if (sg_any && n_rec > 1) {
        cudaStream_t t = on_branch ? s_sg : s;
        // bucket starts (the sizes sum to < 2^32, so the 32-bit scan is exact
        // read as unsigned); the partition leaves the bucket ends
        scan_i32(reinterpret_cast<const int32_t*>(histp), reinterpret_cast<int32_t*>(histp),
                 nbk, false, t);
        DBuf<LegRec> part((size_t)n_rec, t);
        AML_LAUNCH("k_sg_partition", t,
                   k_sg_partition<<<grid_for(n_rec, 256 * SG_PART_ITEMS), 256, 0, t>>>(
                       recp, n_rec, bits, ks, histp, part.p, skip));
        // buckets beyond SG_CAP records: listed by k_sg_bucket, grouped by
        // k_sg_bucket_big (one large-table block per SM)
        DBuf<uint32_t> overflow((size_t)nbk + 1, t);
        AML_CUDA(cudaMemsetAsync(overflow.p, 0, sizeof(uint32_t), t));
        unsigned long long* acc_sg = wp.sg ? acc.p + (int64_t)wp.sg_slot * E : nullptr;
        launch_sg_buckets((unsigned)nbk, t, part.p, histp, wp.delta, g->dts, gv.ts, acc_sg,
                          new_from, overflow.p, sub, skip);
      }
      return on_branch;
    };
    // SG buckets of about sg_bucket_mean records each
    auto bucket_count = [&](int64_t n_records, int* bits) {
      int64_t nbk = 1;
      while (nbk * tn.sg_bucket_mean < n_records) nbk <<= 1;
      *bits = 0;
      while ((1ll << *bits) < nbk) ++*bits;
      return nbk;
    };

    // The fused mine (AML_MINE_FUSED): leg count, leg offsets, leg emission
    // and every cycle level in one cooperative launch, once an earlier mine
    // of this graph has found the sizes of this window's legs and levels;
    // the SG grouping follows it (the DEG/FAN branch runs beside it).
    LegCache& lcf = g->legs[wp.delta];
    bool fused_mine = (mode & AML_MINE_FUSED) && !persistent && new_from == 0 &&
                      wp.emit_legs() && lcf.n_legs >= 0 &&
                      (!level_cycles || lcf.n_front[2] >= 0);
    for (int j = 3; fused_mine && level_cycles && j <= wp.K - 1; ++j)
      fused_mine = lcf.n_front[j] >= 0;
    if (fused_mine) {
      const int64_t nl = lcf.n_legs, n2 = level_cycles ? lcf.n_front[2] : 0;
      DBuf<int32_t> L((size_t)E + 1, s);
      DBuf<int2> qwin((size_t)E, s);
      DBuf<int32_t> qcb(level_cycles ? (size_t)E : 0, s);
      int32_t* gs_in = nullptr;
      if (wp.gs) {  // gather-side GS counts: zeroed by the count, added to by the emission
        keep32.emplace_back((size_t)E, s);
        gs_in = keep32.back().p;
        P.gs_in[w] = gs_in;
      }
      keep64.emplace_back((size_t)(E + 1), s);
      int64_t* off = keep64.back().p;
      P.off[w] = off;
      FusedLegs Q;
      std::memset(&Q, 0, sizeof(Q));
      Q.delta = wp.delta;
      Q.L = L.p;
      Q.qwin = qwin.p;
      Q.qcb = qcb.p;
      Q.Z = ZeroSink{acc_zeroed ? nullptr : acc.p, acc_zeroed ? 0 : n_acc, gs_in};
      acc_zeroed = true;
      Q.off = off;
      DBuf<int4> legs;
      if (level_cycles) {
        legs = DBuf<int4>((size_t)std::max<int64_t>(n2, 1), s);
        Q.anc = anc.p;
        Q.L2 = L2.p;
        Q.off2 = off2.p;
        Q.S.leg = legs.p;
        Q.S.off2 = off2.p;
      }
      DBuf<LegRec> rec;
      DBuf<uint32_t> hist;
      int64_t nb = 1;
      if (sg_any) {
        rec = DBuf<LegRec>((size_t)std::max<int64_t>(nl, 1), s);
        nb = bucket_count(nl, &Q.S.bits);
        hist = DBuf<uint32_t>((size_t)nb + 1, s);
        AML_CUDA(cudaMemsetAsync(hist.p, 0, (size_t)(nb + 1) * 4, s));
        Q.S.rec = rec.p;
        Q.S.hist = hist.p;
      }
      Q.acc_cyc2 = wp.cyc.slot[2] >= 0 ? acc.p + (int64_t)wp.cyc.slot[2] * E : nullptr;
      Q.gs_in = gs_in;
      Q.own_max = tn.own_max;
      Q.n_legs = nl;
      Q.n2 = n2;
      FusedCycles FC;
      std::memset(&FC, 0, sizeof(FC));
      FC.F.base = 2;
      FC.F.leg = legs.p;
      std::vector<DBuf<int32_t>> front;
      front.reserve(2 * MAX_CYCLE);
      int64_t widest = 1;  // the largest level with children
      for (int j = 2; level_cycles && j <= wp.K - 2; ++j) widest = std::max(widest, lcf.n_front[j]);
      for (int j = 3; level_cycles && j <= wp.K - 1; ++j) {
        FC.cap[j] = lcf.n_front[j];
        front.emplace_back((size_t)std::max<int64_t>(lcf.n_front[j], 1), s);
        FC.par[j] = front.back().p;
        front.emplace_back((size_t)std::max<int64_t>(lcf.n_front[j], 1), s);
        FC.slot[j] = front.back().p;
      }
      const int grid = fused_mine_grid(sub.n);
      DBuf<int32_t> cnt((size_t)widest, s), q0b((size_t)widest, s);
      DBuf<long long> bsum((size_t)2 * grid, s);
      DBuf<GridBarrier> bar(1, s);
      AML_CUDA(cudaMemsetAsync(bar.p, 0, sizeof(GridBarrier), s));
      // the work queues' counters: leg count, emission, then one per cycle level
      DBuf<unsigned long long> ctr(2 + MAX_CYCLE + 1, s);
      AML_CUDA(cudaMemsetAsync(ctr.p, 0, (2 + MAX_CYCLE + 1) * sizeof(unsigned long long), s));
      Q.ctr = ctr.p;
      FC.ctr = ctr.p + 2;
      FC.cnt = cnt.p;
      FC.q0 = q0b.p;
      FC.bsum = bsum.p;
      FC.bar = bar.p;
      FC.err = g->err;
      FC.wait_limit = g->wait_limit;
      FC.own_max = tn.own_max;
      Q.bsum = bsum.p;
      launch_mine_fused(grid, s, gv, Q, wp.K, wp.cyc, acc.p, tn.close_scan_max, FC, sub);
      // the records are complete only if every barrier of the launch was met
      if (sg_group(rec.p, hist.p, nb, Q.S.bits, sg_any ? nl : 0, KeySet{nullptr, 0}, g->err))
        branch_wait(g->branch_ev[3], s_sg, s);
      continue;
    }

    DBuf<int32_t> L(E + 1, s);
    int32_t* L_new = nullptr;
    if (new_from > 0 && wp.gs) {
      keep32.emplace_back((size_t)E, s);
      L_new = keep32.back().p;
      P.gs_from[w] = L_new;
    }
    DBuf<int2> qwin((size_t)E, s);
    DBuf<int32_t> qcb(level_cycles ? (size_t)E : 0, s);
    int32_t* gs_in = nullptr;
    if (wp.gs && wp.emit_legs()) {  // gather-side GS counts, added to by the emission
      keep32.emplace_back((size_t)E, s);
      gs_in = keep32.back().p;
      P.gs_in[w] = gs_in;
    }
    ZeroSink Z{acc_zeroed ? nullptr : acc.p, acc_zeroed ? 0 : n_acc, gs_in};
    acc_zeroed = true;
    launch_leg_count(grid_for(E, B), B, s, gv, wp.delta, L.p, level_cycles ? anc.p : nullptr,
                     level_cycles && !persistent, level_cycles ? L2.p : nullptr, L_new, qwin.p,
                     qcb.p, sub, Z);
    AML_CUDA(cudaMemsetAsync(L.p + E, 0, sizeof(int32_t), s));
    keep64.emplace_back((size_t)(E + 1), s);
    int64_t* off = keep64.back().p;
    scan_i32_to_i64(L.p, off, E + 1, s);
    P.off[w] = off;
    if (level_cycles) {
      AML_CUDA(cudaMemsetAsync(L2.p + E, 0, sizeof(int32_t), s));
      scan_i32_to_i64(L2.p, off2.p, E + 1, s);
    }
    if (wp.gs && !wp.emit_legs()) {  // written outright by k_gs_into
      keep32.emplace_back((size_t)E, s);
      gs_in = keep32.back().p;
      P.gs_in[w] = gs_in;
    }
    if (!wp.emit_legs()) {
      AML_LAUNCH("k_gs_into", s, k_gs_into<<<grid_for(E, B), B, 0, s>>>(gv, wp.delta, gs_in));
      continue;
    }
    LegCache& lc = g->legs[wp.delta];
    if (lc.n_legs < 0 || (level_cycles && lc.n_front[2] < 0)) {
      // one wait for both sizes
      int64_t total[2] = {0, 0};
      const SmallRead rd[2] = {{&total[0], off + E, 8}, {&total[1], off2.p + E, 8}};
      read_small(rd, level_cycles ? 2 : 1, s);
      AML_REQUIRE(total[0] < (int64_t)UINT32_MAX, AML_EUNSUPPORTED,
                  "more than 2^32 temporal 2-paths in one window");
      lc.n_legs = total[0];
      if (level_cycles) lc.n_front[2] = total[1];
    }
    const int64_t nl = lc.n_legs;
    LegSink S{nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr};
    DBuf<int4> legs;
    if (level_cycles) {
      const int64_t n2 = lc.n_front[2];
      legs = DBuf<int4>((size_t)std::max<int64_t>(n2, 1), s);
      S.leg = legs.p;
      S.off2 = off2.p;
    }
    DBuf<LegRec> rec;
    DBuf<uint32_t> hist;
    int64_t nb = 1;
    // delta counting: the latest edge of an SG instance is one of its gather
    // edges, so only legs into a destination of a new edge are recorded
    const bool sg_filter = sg_any && new_from > 0;
    DBuf<uint32_t> dmask;
    DBuf<unsigned long long> n_rec;
    auto size_buckets = [&](int64_t n_records) {
      nb = bucket_count(n_records, &S.bits);
      hist = DBuf<uint32_t>((size_t)nb + 1, s);
      AML_CUDA(cudaMemsetAsync(hist.p, 0, (size_t)(nb + 1) * 4, s));
    };
    if (sg_any) {
      rec = DBuf<LegRec>((size_t)std::max<int64_t>(nl, 1), s);
      S.rec = rec.p;
      if (sg_filter) {
        const int64_t words = (g->N + 31) / 32;
        dmask = DBuf<uint32_t>((size_t)std::max<int64_t>(words, 1), s);
        AML_CUDA(cudaMemsetAsync(dmask.p, 0, (size_t)words * 4, s));
        AML_LAUNCH("k_mark_nodes", s,
                   k_mark_nodes<<<grid_for(E - new_from, 256), 256, 0, s>>>(g->dst, new_from, E,
                                                                           dmask.p));
        n_rec = DBuf<unsigned long long>(1, s);
        AML_CUDA(cudaMemsetAsync(n_rec.p, 0, 8, s));
        S.dmask = dmask.p;
        S.n_rec = n_rec.p;
      } else {
        size_buckets(nl);
        S.hist = hist.p;
      }
    }
    unsigned long long* acc2 =
        wp.cyc.slot[2] >= 0 ? acc.p + (int64_t)wp.cyc.slot[2] * E : nullptr;
    // delta counting: old legs matter only as SG legs into a batch
    // destination, found through the out-list slots marked for it -- while
    // those are a small share of the slots (below 40%: measured break-even
    // on the hi-medium shape); otherwise every window is walked
    bool delta_emit = new_from > 0;
    DBuf<int32_t> mflag, mptr, mslot;
    if (delta_emit && sg_filter) {
      mflag = DBuf<int32_t>((size_t)Ev + 1, s);
      AML_LAUNCH("k_mark_slots", s,
                 k_mark_slots<<<grid_for(Ev + 1, 256), 256, 0, s>>>(g->out.nbr, Ev, dmask.p,
                                                                    mflag.p));
      scan_i32(mflag.p, mflag.p, Ev + 1, false, s);
      int32_t n_marked = 0;
      const SmallRead rd{&n_marked, mflag.p + Ev, 4};
      read_small(&rd, 1, s);
      delta_emit = (double)n_marked < 0.4 * (double)Ev;
    }
    if (delta_emit) {
      DBuf<int32_t> first_new((size_t)std::max<int32_t>(g->N, 1), s);
      AML_LAUNCH("k_first_new", s,
                 k_first_new<<<grid_for(g->N, 256), 256, 0, s>>>(g->out.ptr, g->out.eid, g->N,
                                                                 new_from, first_new.p));
      if (sg_filter) {
        mptr = DBuf<int32_t>((size_t)g->N + 1, s);
        mslot = DBuf<int32_t>((size_t)std::max<int64_t>(Ev, 1), s);
        AML_LAUNCH("k_compact_marked", s,
                   k_compact_marked<<<grid_for(Ev, 256), 256, 0, s>>>(mflag.p, Ev, mslot.p));
        AML_LAUNCH("k_marked_ptr", s,
                   k_marked_ptr<<<grid_for((int64_t)g->N + 1, 256), 256, 0, s>>>(
                       g->out.ptr, mflag.p, g->N, mptr.p));
      }
      launch_leg_emit_delta(grid_for(E, B), B, s, gv, qwin.p, qcb.p, S, acc2, gs_in,
                            tn.own_max, sub, first_new.p, mptr.p, mslot.p);
    } else {
      launch_leg_emit(grid_for(E, B), B, s, gv, qwin.p, qcb.p, off, S, acc2, gs_in, tn.own_max,
                      sub);
    }
    int64_t n_sg = nl;  // records to bucket
    DBuf<unsigned long long> key_tab;  // delta counting: the keys with a new leg
    KeySet ks{nullptr, 0};
    if (sg_filter) {
      unsigned long long kept = 0;
      const SmallRead rd{&kept, n_rec.p, 8};
      read_small(&rd, 1, s);
      n_sg = (int64_t)kept;
      if (n_sg > 1) {
        size_buckets(n_sg);
        // the set holds the new legs' keys and must stay in L2 while every
        // record is looked up in it: sized from the record count already on
        // the host (an upper bound on the new legs) while that gives at most
        // 2^23 slots (64 MB), else from the new legs counted on the device
        // (one more wait for the host)
        uint64_t bound = (uint64_t)n_sg;
        if (2 * bound > (1ull << 23)) {
          AML_CUDA(cudaMemsetAsync(n_rec.p, 0, 8, s));
          AML_LAUNCH("k_sg_count_new", s,
                     k_sg_count_new<<<grid_for(n_sg, 256), 256, 0, s>>>(rec.p, n_sg, new_from,
                                                                       n_rec.p));
          unsigned long long n_new_legs = 0;
          const SmallRead rn{&n_new_legs, n_rec.p, 8};
          read_small(&rn, 1, s);
          bound = n_new_legs;
        }
        uint64_t slots = 1024;
        while (slots < 2 * bound) slots <<= 1;
        key_tab = DBuf<unsigned long long>((size_t)slots, s);
        AML_CUDA(cudaMemsetAsync(key_tab.p, 0xff, (size_t)slots * 8, s));
        ks = KeySet{key_tab.p, slots - 1};
        AML_LAUNCH("k_sg_new_keys", s,
                   k_sg_new_keys<<<grid_for(n_sg, 256), 256, 0, s>>>(rec.p, n_sg, new_from, ks));
        AML_LAUNCH("k_sg_hist", s,
                   k_sg_hist<<<grid_for(n_sg, 256), 256, 0, s>>>(rec.p, n_sg, S.bits, ks, hist.p));
      }
    }
    const bool sg_branch = sg_group(rec.p, hist.p, nb, S.bits, n_sg, ks, nullptr);
    // 4. cycles of length >= 3: the cost-binned hybrid (heaviest anchors
    // level by level, the rest in one persistent launch beside them) ...
    if (wp.K >= 3 && persistent) {
      cycles_hybrid(g, gv, wp.delta, wp.K, wp.cyc, sub, acc.p, crng.p, anc.p, qwin.p, legs.p,
                    (mode & AML_MINE_LEARNED) != 0, s, branches ? g->side[2] : s);
    } else if (level_cycles) {  // ... or level by level from the legs
      level_cycle_search(g, gv, wp.delta, wp.K, wp.cyc, sub, acc.p, anc.p, qwin.p, legs.p,
                         lc.n_front, s);
    }
    // the window's buffers (rec, hist, ...) are freed on s after this join
    if (sg_branch) branch_wait(g->branch_ev[3], s_sg, s);
  }
  if (!acc_zeroed) AML_CUDA(cudaMemsetAsync(acc.p, 0, (size_t)n_acc * E * 8, s));
  acc_zeroed = true;
  if (branches) AML_CUDA(cudaStreamWaitEvent(s, g->branch_ev[1], 0));  // DEG/FAN joined
  // window cycles: one level-by-level search per group of windows, largest
  // delta first; its pass counts the smaller windows by span tests
  std::vector<int> wq;
  for (size_t w = 0; w < wins.size(); ++w)
    if (wins[w].Kw >= 3) wq.push_back((int)w);
  std::sort(wq.begin(), wq.end(), [&](int x, int y) { return wins[x].delta > wins[y].delta; });
  std::vector<char> wdone(wins.size(), 0);
  for (int w : wq) {
    if (wdone[w]) continue;
    wdone[w] = 1;
    const WindowPlan& wp = wins[w];
    SubWindows sw;
    std::memset(&sw, 0, sizeof(sw));
    for (int m : wq)
      if (!wdone[m] && wins[m].Kw <= wp.Kw && sw.n < MAX_SUB) {
        sw.delta[sw.n] = wins[m].delta;
        sw.cyc[sw.n] = wins[m].cycw;
        ++sw.n;
        wdone[m] = 1;
      }
    window_cycle_search(g, gv, wp.delta, wp.Kw, wp.cycw, sw, acc.p, s);
  }
  // stage programs no family implements: the generic interpreter
  for (const auto& pr : programs)
    run_program(gv, g->amount, ps->progs[pr.second], acc.p + (int64_t)pr.first * E, s);
  AML_LAUNCH("k_assemble", s,
             k_assemble<<<grid_for(E, ASM_BLOCK), ASM_BLOCK,
                          (size_t)ASM_BLOCK * (ncols | 1) * sizeof(uint32_t), s>>>(P));
}

}  // namespace aml
