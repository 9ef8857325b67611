// Kernel-parameter structs shared by the mining kernels and their host code.
#pragma once

#include "aml_internal.cuh"

namespace aml {

constexpr int MAX_COLS = 64;    // columns per pattern set
constexpr int MAX_DELTAS = 16;  // distinct windows per pattern set
constexpr int MAX_CYCLE = 8;    // longest cycle
constexpr int SG_CAP = 512;        // leg records one SG bucket block groups in shared memory
constexpr int SG_TAB = 1024;       // its hash-table slots (load <= 0.5)
constexpr int SG_BLOCK = 256;      // threads of that block
constexpr int SG_CAP_BIG = 4096;   // the same for the larger buckets (k_sg_bucket_big)
constexpr int SG_TAB_BIG = 8192;
constexpr int SG_BIG_BLOCK = 1024;  // threads of that block (one block per SM)
constexpr int SG_PART_ITEMS = 4;     // records per thread in k_sg_partition
constexpr int ASM_BLOCK = 128;       // rows per k_assemble block

// Read-only view of a device graph, passed by value to kernels.
struct GraphView {
  int64_t E;
  int32_t N;
  // Delta counting: when new_from > 0, only instances whose latest edge has
  // id >= new_from are counted (edges new_from.. are the latest in (t, id)
  // order, the first of them at time t_new).  0 counts every instance.
  int32_t new_from;
  int32_t t_new;
  const int32_t *src, *dst, *ts;
  const int32_t *optr, *onbr, *ot, *oeid, *oprev, *onext, *onnbr, *ont, *oneid, *opos;
  const int32_t *iptr, *inbr, *it, *ieid, *iprev, *inext, *innbr, *int_, *ineid, *ipos;
};

inline GraphView view_of(const aml_graph* g) {
  GraphView v;
  v.E = g->E;
  v.N = g->N;
  v.new_from = 0;
  v.t_new = 0;
  v.src = g->src; v.dst = g->dst; v.ts = g->ts;
  v.optr = g->out.ptr; v.onbr = g->out.nbr; v.ot = g->out.t; v.oeid = g->out.eid;
  v.oprev = g->out.prev; v.onext = g->out.next; v.onnbr = g->out.nnbr; v.ont = g->out.nt;
  v.oneid = g->out.neid; v.opos = g->out.pos;
  v.iptr = g->in.ptr; v.inbr = g->in.nbr; v.it = g->in.t; v.ieid = g->in.eid;
  v.iprev = g->in.prev; v.inext = g->in.next; v.innbr = g->in.nnbr; v.int_ = g->in.nt;
  v.ineid = g->in.neid; v.ipos = g->in.pos;
  return v;
}

struct ColDesc {
  int32_t family;
  int32_t k;
  int32_t delta;
  int32_t didx;      // index of the column's window in the per-window tables
  int32_t acc_slot;  // accumulator column (SG, CYC), else -1
};

struct AssembleParams {
  GraphView g;
  ColDesc cols[MAX_COLS];
  int32_t ncols;
  const int2* df_out[MAX_DELTAS];  // (DEG_OUT, FAN_OUT) of edge e at [e * DF_STRIDE]
  const int2* df_in[MAX_DELTAS];   // (DEG_IN, FAN_IN) likewise
  const int64_t* off[MAX_DELTAS];     // leg offsets per edge (GS gather side)
  const int32_t* gs_from[MAX_DELTAS]; // delta counting: legs from each edge that are new
  const int32_t* gs_in[MAX_DELTAS];   // legs ending with each edge (GS scatter side)
  const unsigned long long* acc;
  uint32_t* counts;
  int64_t ld;
  uint32_t limit;  // saturation bound of every count (2^32-1 unless lowered)
  // streaming: rows below accumulate_from add their new-instance counts to
  // the instance columns already stored (mask bit c set = instance column);
  // -1 writes every row outright
  int64_t accumulate_from;
  uint64_t inst_mask;
};

// One leg a = s->m, b = m->d filed for the SG grouping under key s*N + d;
// 16 bytes (m and the two times are read back from the edges only for the
// legs that share their key with another leg).
struct __align__(16) LegRec {
  uint64_t key;
  int32_t a, b;
};

// Where k_leg_emit writes the legs: one {a, b, dst of b, t_b} record per
// cycle-starting leg for the cycle search and/or records + bucket histogram
// for the SG grouping (null = not wanted).
struct LegSink {
  int4* leg;        // legs that can start a cycle (closing range not empty and the
                    // second edge before its last closing edge), compacted, as
                    // {a, b, dst b, t_b}: what the cycle search reads of a leg
  const int64_t* off2;  // first cycle leg of each edge (scan of k_leg_count's L2)
  LegRec* rec;
  uint32_t* hist;
  int bits;  // log2 of the number of SG buckets
  // delta counting: only legs into a node of this bitmap can be in a new SG
  // instance; they are compacted into rec by n_rec (hist unused)
  const uint32_t* dmask;
  unsigned long long* n_rec;
};

struct CycleSlots {
  int32_t slot[MAX_CYCLE + 1];  // accumulator column of CYC_k, or -1
};

// Smaller windows counted from the legs, SG groups and cycle paths of a
// larger window: an instance within a smaller window is an instance of the
// larger one whose span is that small, so each count only adds a test of
// the span.  Null pointers / -1 slots: column not wanted.
constexpr int MAX_SUB = 4;
struct SubWindows {
  int n;
  int32_t delta[MAX_SUB];
  int32_t* gs_from[MAX_SUB];          // GS: legs starting with each edge
  int32_t* gs_in[MAX_SUB];            // GS: legs ending with each edge
  unsigned long long* cyc2[MAX_SUB];  // CYC2 accumulator
  unsigned long long* sg[MAX_SUB];    // SG accumulator
  CycleSlots cyc[MAX_SUB];            // CYC_k accumulator slots, k >= 3
};

// Frontier of the level-by-level cycle search: the base level is the leg
// records leg (base 2) or, for window cycles, the anchor edges la (base 1);
// element i of a level j above it extends element par[j][i] of level j-1 by
// the out-slot slot[j][i].
struct CycFrontier {
  int base;
  const int32_t* la;   // base 1: the anchor edges
  const int4* leg;     // base 2: the legs {a, b, dst b, t_b}
  const int32_t* par[MAX_CYCLE + 1];
  const int32_t* slot[MAX_CYCLE + 1];
};

// What a cycle path reads of its anchor edge a = u0 -> u1, in one 32-byte
// record (one sector): its closing range B1 = in(u0) slots [cr_x, cr_y),
// the (t, id) of B1's latest edge (when B1 is not empty), u0, u1 and t_a.
struct __align__(32) AnchorRec {
  int32_t cr_x, cr_y, t_cl, id_cl;
  int32_t u0, u1, t1, pad;
};

__global__ void k_window_slots(const int32_t* rstart, const int32_t* t, const int32_t* eid,
                               const int32_t* prev, const int32_t* next, int64_t Ev,
                               int32_t delta, int32_t* deg_s, int32_t* D, int2* df);
// (DEG, FAN) of every edge for nw <= FAN_MAX_W windows of one direction
// (deltas in descending order): df[e * DF_STRIDE + k] for window k, at the
// edge id (self-loop rows untouched); each edge's row is DF_STRIDE pairs =
// 32 bytes, written whole, so that the stores scattered by edge id fill
// whole sectors (a partial sector costs the memory a read-modify-write);
// two launches on s.  new_from > 0: only the edges e >= new_from (delta
// counting), the other rows untouched.
constexpr int FAN_MAX_W = 4;
constexpr int DF_STRIDE = 4;
void fan_per_edge(const Adj& a, int64_t Ev, int64_t E, int64_t new_from, int nw,
                  const int32_t* deltas, int2* df, cudaStream_t s);
__global__ void k_gs_into(GraphView g, int32_t delta, int32_t* gs_in);
// moves every record to its bucket: cursor = exclusive scan of the bucket
// sizes on entry, the bucket ends on exit
// A set of SG keys (delta counting: those with a new leg); tab null = all.
struct KeySet {
  unsigned long long* tab;
  uint64_t mask;  // slots - 1 (a power of two)
};

__global__ void k_sg_partition(const LegRec* rec, int64_t n, int bits, KeySet ks,
                               uint32_t* cursor,
                               LegRec* out, const uint32_t* skip);
__global__ void k_sg_hist(const LegRec* rec, int64_t n, int bits, KeySet ks, uint32_t* hist);
__global__ void k_sg_new_keys(const LegRec* rec, int64_t n, int32_t new_from, KeySet ks);
__global__ void k_sg_count_new(const LegRec* rec, int64_t n, int32_t new_from,
                               unsigned long long* count);
__global__ void k_mark_nodes(const int32_t* node_of, int64_t from, int64_t E, uint32_t* mask);
// closing ranges of every edge: into rng (int2) and/or anc (anchor records);
// either may be null
__global__ void k_close_range(GraphView g, int32_t delta, int2* rng, AnchorRec* anc);
__global__ void k_anchor_flags(const int2* crng, int64_t E, int32_t* flag);
__global__ void k_compact_ids(const int32_t* flag, const int32_t* off, int64_t E, int32_t* items);
// Buffers k_leg_count zeroes per edge: n_acc accumulator columns of E
// entries, and the GS gather-side counts (either may be absent).
struct ZeroSink {
  unsigned long long* acc;
  int n_acc;
  int32_t* gs_in;
};
// Launchers of the kernels that also count sub-windows (instantiated for
// the number of them in sub).
void launch_leg_count(unsigned grid, int block, cudaStream_t s, const GraphView& g, int32_t delta,
                      int32_t* L, AnchorRec* anc, bool close_here, int32_t* L2, int32_t* L_new,
                      int2* qwin, int32_t* qcb, const SubWindows& sub, const ZeroSink& Z);
// Delta counting (new_from > 0): the legs a new instance can use (mine.cu);
// first_new = each out-list's first new slot (k_first_new); mptr/mslot =
// each node's out-list slots whose counterparty is a batch destination
// (k_mark_slots, k_compact_marked, k_marked_ptr).
void launch_leg_emit_delta(unsigned grid, int block, cudaStream_t s, const GraphView& g,
                           const int2* qwin, const int32_t* qcb, const LegSink& S,
                           unsigned long long* acc_cyc2, int32_t* gs_in, int32_t own_max,
                           const SubWindows& sub, const int32_t* first_new,
                           const int32_t* mptr, const int32_t* mslot);
__global__ void k_first_new(const int32_t* optr, const int32_t* oeid, int32_t N, int32_t new_from,
                            int32_t* first_new);
__global__ void k_mark_slots(const int32_t* nbr, int64_t Ev, const uint32_t* mask, int32_t* flag);
__global__ void k_compact_marked(const int32_t* flag_scan, int64_t Ev, int32_t* mslot);
__global__ void k_marked_ptr(const int32_t* optr, const int32_t* flag_scan, int32_t N,
                             int32_t* mptr);
void launch_leg_emit(unsigned grid, int block, cudaStream_t s, const GraphView& g,
                     const int2* qwin, const int32_t* qcb, const int64_t* off, const LegSink& S,
                     unsigned long long* acc_cyc2, int32_t* gs_in, int32_t own_max,
                     const SubWindows& sub);
// (dst[e], ts[e]) of every edge in one int2, for the SG grouping's gathers
__global__ void k_pack_dst_ts(const int32_t* dst, const int32_t* ts, int64_t E, int2* dts);
// k_sg_bucket over all buckets (bucket b = records [bend[b-1], bend[b])),
// then k_sg_bucket_big over the overflow list; dts from k_pack_dst_ts
void launch_sg_buckets(unsigned n_buckets, cudaStream_t s, const LegRec* rec,
                       const uint32_t* bend, int32_t delta, const int2* dts, const int32_t* ts,
                       unsigned long long* acc, int32_t new_from, uint32_t* overflow,
                       const SubWindows& sub,
                       const uint32_t* skip = nullptr);
// Ordered cycles read their anchors from anc and their children's window
// starts from qwin (the leg windows of the same window's leg pass); window
// cycles (base 1) read close_rng and search their windows.
void launch_cyc_level(unsigned grid, int block, cudaStream_t s, const GraphView& g,
                      int32_t delta, int K, int j, const CycFrontier& F, int64_t n,
                      const int2* close_rng, const AnchorRec* anc, const int2* qwin,
                      const CycleSlots& slots, unsigned long long* acc, int32_t* cnt,
                      int32_t* q0_out, int32_t close_scan_max, const SubWindows& sub,
                      bool window_cycles = false);
__global__ void k_cyc_emit(int64_t n, const int32_t* cnt, const int32_t* q0, const int64_t* off,
                           int32_t* par, int32_t* slot, int32_t own_max);

// Grid-wide barrier state of a cooperative launch (zeroed before it).
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};
// The cycle levels of the fused mine.  par/slot of levels 3..K-1 hold
// cap[j] elements; cnt/q0 hold the largest level that has children; bsum
// one value per block.
struct FusedCycles {
  CycFrontier F;  // base level (the legs)
  int64_t cap[MAX_CYCLE + 1];
  int32_t* par[MAX_CYCLE + 1];
  int32_t* slot[MAX_CYCLE + 1];
  int32_t* cnt;
  int32_t* q0;
  long long* bsum;
  GridBarrier* bar;
  unsigned long long* ctr;  // per level, the work queue's counter (zeroed before the launch)
  uint32_t* err;
  long long wait_limit;  // SM clock cycles a barrier wait may take
  int32_t own_max;       // child lists up to this long are written by one lane
};
// The fused mine of one window: the leg pass and the cycle search in one
// cooperative launch (k_mine_fused).  Phases, between grid barriers: leg
// count (warps take tiles of edges from a work queue), the legs of block b's
// contiguous edge chunk summed, the chunk's leg offsets (off, off2 and their
// totals at [E]) from every block's sums, leg emission (a second work
// queue), then every cycle level (FusedCycles).  The
// buffers are sized for n_legs legs and n2 cycle legs (the sizes of an
// earlier mine of the same graph); other totals set ERR_OVERFLOW.
struct FusedLegs {
  int32_t delta;
  int32_t* L;
  AnchorRec* anc;  // null: no cycle search (L2, qcb, off2 unused)
  int32_t* L2;
  int2* qwin;
  int32_t* qcb;
  ZeroSink Z;
  int64_t* off;
  int64_t* off2;
  LegSink S;
  unsigned long long* acc_cyc2;
  int32_t* gs_in;
  int32_t own_max;
  int64_t n_legs, n2;
  long long* bsum;               // two values per block
  unsigned long long* ctr;       // the two work queues' counters, zeroed before the launch
};
// blocks of the fused launches on this device (all resident at once)
int fused_mine_grid(int n_sub);
void launch_mine_fused(int grid, cudaStream_t s, const GraphView& g, const FusedLegs& Q, int K,
                       const CycleSlots& slots, unsigned long long* acc, int32_t close_scan_max,
                       const FusedCycles& P, const SubWindows& sub);
__global__ void k_assemble(AssembleParams P);

// Host pipeline: enqueue a full mine of `ps` on `g` into device `counts`.
// mode: AML_MINE_PERSISTENT / AML_MINE_LEARNED select the cycle search.
// new_from / t_new: delta counting (see GraphView); 0 counts everything.
// accumulate (with new_from > 0): rows below new_from add their counts to the
// stored instance columns, rows from new_from on are written outright.
void mine_plain(aml_graph* g, const aml_pattern_set* ps, uint32_t* counts, int64_t ld,
                cudaStream_t s, uint32_t mode = 0, int32_t new_from = 0, int32_t t_new = 0,
                bool accumulate = false);
// The same, replayed from a CUDA graph captured on first use.
void mine_graph_mode(aml_graph* g, const aml_pattern_set* ps, uint32_t* counts, int64_t ld,
                     cudaStream_t s, uint32_t mode = 0);
// Ordered cycles level by level from the cycle-capable legs (pipeline.cu).
// The generic interpreter of stage programs (program.cu): counts of one
// program into out[E]; waits for `s` to read the launch's status.
void run_program(const GraphView& gv, const float* amount, const Prog& p,
                 unsigned long long* out, cudaStream_t s);

void level_cycle_search(aml_graph* g, const GraphView& gv, int32_t delta, int K,
                        const CycleSlots& slots, const SubWindows& sub,
                        unsigned long long* acc, const AnchorRec* anc, const int2* qwin,
                        const int4* legs, int64_t* front_cache, cudaStream_t s);
// Cycle search of one window split by estimated anchor cost (cost.cu): the
// heaviest anchors' legs level by level on s, the other anchors by the
// persistent kernel on `side` (forked from and joined back to s).
void cycles_hybrid(aml_graph* g, const GraphView& gv, int32_t delta, int K,
                   const CycleSlots& slots, const SubWindows& sub, unsigned long long* acc,
                   const int2* crng, const AnchorRec* anc, const int2* qwin, const int4* legs,
                   bool learned, cudaStream_t s, cudaStream_t side);
void drop_captured_mines(aml_graph* g);

}  // namespace aml
