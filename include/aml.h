/*
 * aml.h -- C ABI of the B300 per-edge AML pattern-counting library.
 *
 * The library counts, for every transaction edge of a temporal transaction
 * graph, how many instances of each multi-stage laundering pattern the edge
 * takes part in, and writes an E x P uint32 feature matrix (one column per
 * pattern).  This is the mining front end of the paper's pipeline (Sec. 1,
 * Fig. 1: "augments each transaction edge with pattern occurrence counts");
 * patterns are given as stage programs in the paper's multi-stage framework
 * (Sec. 5; stage configuration of Alg. 1 and Sec. 6 "Input specification").
 *
 * Conventions for every call:
 *   - No C++ exception, abort or exit crosses this boundary.  Every call
 *     returns an aml_status; on failure aml_last_error() gives a message
 *     (thread-local, valid until the calling thread's next failing call).
 *   - CUDA errors map to AML_ECUDA.  Kernel faults are asynchronous and
 *     surface at aml_sync() or at the next call on the same object.
 *   - "device pointer" = memory of the current CUDA device (cudaMalloc,
 *     cudaMallocAsync, torch.cuda tensors); "host pointer" = ordinary or
 *     pinned host memory.  Pointer arguments are never retained unless
 *     stated: the library copies what it keeps.
 *   - `stream` is a cudaStream_t passed as void*; NULL = the legacy default
 *     stream.  Work is enqueued on it; calls return before it finishes
 *     unless stated.
 *   - The library owns graphs, pattern sets and its scratch memory; the
 *     caller owns its inputs and the output matrix.
 *   - Edge ids are input positions 0..E-1 and E < 2^31; node ids are in
 *     [0, n_nodes).  Timestamps are int32 seconds.
 */
#ifndef AML_H
#define AML_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */

typedef int32_t aml_status;
#define AML_OK 0
#define AML_EINVAL 1        /* bad argument (null pointer, size, id, flag)        */
#define AML_ENOMEM 2        /* device or host allocation failed                   */
#define AML_ECUDA 3         /* a CUDA runtime call or kernel failed               */
#define AML_EUNSUPPORTED 4  /* well-formed stage program no kernel implements     */
#define AML_EUNSORTED 5     /* AML_ASSUME_SORTED given but timestamps decrease     */
#define AML_ELATE 6         /* streamed batch older than the stream's clock        */
#define AML_EADMIT 7        /* streamed batch refused by the memory budget         */
#define AML_ETIMEOUT 8      /* a bounded device-side wait gave up                  */
#define AML_EINTERNAL 9     /* internal invariant violated (device error word)     */

/* Static string naming a status ("AML_OK", ...); never NULL. */
const char* aml_status_str(aml_status s);
/* Message of the calling thread's last failing call ("" if none); never NULL. */
const char* aml_last_error(void);
/* Library version as 10000*major + 100*minor + patch. */
int32_t aml_version(void);

/* ------------------------------------------------------------------- graph */

/* The transaction graph (Sec. 2.3: node = account, edge = transaction with
 * amount and time).  Built on the device: edges ordered by (timestamp, id);
 * per-account out-lists (CSR) and in-lists (CSC) sorted by (t, id) so that
 * every time window is a contiguous range found by binary search (Alg. 1's
 * Find_Starting_Edge; Sec. 6 "sorted neighbor lists and binary search"), plus
 * a second per-account order by (counterparty, t, id) for membership tests
 * in intersections.  Self-loops (src == dst) are kept as edges but belong to
 * no list: every pattern count of a self-loop is 0. */
typedef struct aml_graph aml_graph;

#define AML_PTR_HOST 0x0u       /* src/dst/ts/amount are host pointers            */
#define AML_PTR_DEVICE 0x1u     /* ... are device pointers                         */
#define AML_ASSUME_SORTED 0x2u  /* caller promises ts non-decreasing in id order;  */
                                /* verified on the device (AML_EUNSORTED if not)   */

/* Build a graph from E transactions.
 *   src, dst : int32[E] account ids in [0, n_nodes)
 *   ts       : int32[E] timestamps (seconds); any order unless ASSUME_SORTED
 *   amount   : float[E] transaction amounts, or NULL (stored; no current
 *              pattern constrains amounts)
 *   n_edges  : E, 0 <= E < 2^31;  n_nodes: 1 <= N < 2^31
 *   flags    : AML_PTR_* | AML_ASSUME_SORTED
 *   stream   : stream for the copies and the build; the call synchronizes it
 *              before returning (the graph is ready on return)
 *   out      : receives the graph handle (unchanged on failure)
 * Errors: AML_EINVAL (null pointers, sizes, an id outside [0, N)),
 * AML_EUNSORTED, AML_ENOMEM, AML_ECUDA.  The inputs are copied. */
aml_status aml_graph_create(const int32_t* src, const int32_t* dst, const int32_t* ts,
                            const float* amount, int64_t n_edges, int32_t n_nodes,
                            uint32_t flags, void* stream, aml_graph** out);

/* Free a graph and everything cached on it (NULL is a no-op).  Waits for the
 * work enqueued on the graph: on every stream passed to aml_graph_create,
 * aml_mine, aml_autotune and aml_cost_train for it, and on the graph's own
 * internal streams -- not for unrelated work elsewhere on the device, so a
 * caller may destroy one graph while the next one's transfers and mining are
 * in flight.  Work a caller enqueued on this graph through aml_fan_noalloc
 * on yet another stream must be finished before the call. */
aml_status aml_graph_destroy(aml_graph* g);

typedef struct aml_graph_info {
  int64_t n_edges;        /* E as given                                       */
  int64_t n_list_edges;   /* edges in the lists (E minus self-loops)          */
  int32_t n_nodes;
  int32_t max_out_degree;
  int32_t max_in_degree;
  int32_t reserved;
  int64_t device_bytes;   /* device memory held by the graph                  */
} aml_graph_info;

/* Sizes of a graph.  The first call waits for the graph's build to finish
 * (the degree maxima are read from the device then). */
aml_status aml_graph_get_info(const aml_graph* g, aml_graph_info* info);

/* Work sizes of one window that earlier mines of this graph measured (no
 * paper counterpart; for measurement and capacity planning).
 *   delta    : the window, seconds
 *   n_legs   : out, temporal 2-paths with distinct ends in the window (the
 *              GS instances; also the SG leg records), -1 if no mine has
 *              expanded this window's legs yet
 *   n_front  : out, int64[AML_MAX_CYCLE + 1]; n_front[j] = paths of j edges
 *              the level-by-level cycle search held (j >= 2), -1 where no
 *              mine has built that level; entries 0 and 1 are -1
 * A window counted inside a larger window's pass (see aml_mine) has no
 * sizes of its own.  Both pointers must be non-NULL host pointers. */
#define AML_MAX_CYCLE 8
aml_status aml_graph_window_stats(const aml_graph* g, int32_t delta, int64_t* n_legs,
                                  int64_t* n_front);

/* ----------------------------------------------------------- stage programs */

/* One stage of a multi-stage pattern (Sec. 5; per-stage configuration of
 * Alg. 1: operation, input node set, output variable, skip_if / break_if
 * constraints including the time window).  Node variables N0, N1, ... are
 * numbered in binding order; the trigger binds N0 -> N1. */
#define AML_OP_TRIGGER 0    /* stage 0: the anchor transaction N0 -> N1          */
#define AML_OP_FOR_ALL 1    /* iterate the neighbours of one bound node         */
#define AML_OP_INTERSECT 2  /* nodes in both of two neighbour sets               */

#define AML_DIR_OUT 0       /* Nx.out_neigh: edges leaving Nx                    */
#define AML_DIR_IN 1        /* Nx.in_neigh: edges entering Nx                    */

#define AML_ORDER_NONE 0    /* no ordering constraint on the matched edge(s)     */
#define AML_ORDER_AFTER 1   /* matched edge comes after the edge that reached    */
                            /* the operand's node (causal flow of funds)         */
#define AML_ORDER_BEFORE 2  /* ... comes before it                               */
#define AML_ORDER_LEG 3     /* INTERSECT: a-side edge before b-side edge         */
#define AML_ORDER_AFTER_TRIGGER 4 /* matched edge comes after the trigger edge;  */
                            /* later hops may arrive in any order among         */
                            /* themselves (Sec. 4's anticipatory edges)         */

#define AML_WIN_TRAILING 0  /* edge time in [t_trigger - delta, trigger]         */
#define AML_WIN_SPAN 1      /* all edges of an instance within delta             */

typedef struct aml_stage {
  int32_t op;        /* AML_OP_*                                                */
  int32_t a_var;     /* first operand: node variable ...                        */
  int32_t a_dir;     /* ... and its neighbour set (AML_DIR_*)                   */
  int32_t b_var;     /* second operand (INTERSECT only; else -1)                */
  int32_t b_dir;
  int32_t out_var;   /* variable this stage binds; naming an already bound      */
                     /* variable closes the walk onto that node                 */
  int32_t order;     /* AML_ORDER_*                                             */
  int32_t window;    /* AML_WIN_*                                               */
  uint32_t skip_eq;  /* skip_if: bit i set = drop candidates equal to N_i       */
                     /* (the paper's "differentiate", e.g. N2 != N0)            */
  uint32_t amount_flags;  /* AML_AMT_* constraints on the amounts of the stage's */
                          /* edges (0: none); any makes the program interpreted */
  float amount_min, amount_max;  /* AML_AMT_RANGE: amount_min <= amount <=       */
                                 /* amount_max for every edge of the stage      */
  float ratio_min, ratio_max;    /* AML_AMT_RATIO: each edge's amount within     */
                                 /* [ratio_min, ratio_max] times the amount of   */
                                 /* the edge before it on the walk: reach(A) for */
                                 /* a FOR_ALL edge and an INTERSECT's a-side     */
                                 /* edge, the a-side edge for the b-side edge    */
} aml_stage;

/* Amount constraints of a stage (edge attributes as operands, Sec. 5).  The
 * comparisons are exact: amounts are the float32 values given to
 * aml_graph_create, and ratio * amount is formed in double precision (the
 * exact product of two floats).  On the trigger (stage 0) only RANGE is
 * allowed: it selects the trigger edges. */
#define AML_AMT_RANGE 0x1u
#define AML_AMT_RATIO 0x2u

/* What the final stage's Postprocess reports for each trigger edge. */
#define AML_AGG_EDGES 0      /* # matched edges (windowed degree)               */
#define AML_AGG_DISTINCT 1   /* # distinct matched nodes (fan-in / fan-out)     */
#define AML_AGG_INSTANCES 2  /* # pattern instances containing the edge, each   */
                             /* instance credited to all of its edges           */
                             /* (Sec. 5: an edge "increments counts for all     */
                             /* pattern instances it participates in")          */
#define AML_AGG_SETS 3       /* # distinct edge sets of the instances that      */
                             /* contain the edge: bindings that find one set of */
                             /* edges from other triggers or in another order   */
                             /* of their stages count once.  Counted for the    */
                             /* scatter-gather of n intermediaries, 2 <= n <= 7 */
                             /* (the trigger s->m1, N1.out -> d after it, then  */
                             /* n-1 intersections N0.out with N2.in, each leg   */
                             /* in order (LEG), each intermediary skipping N1   */
                             /* and the ones before, every stage in the span    */
                             /* window, no amount constraints): the exact       */
                             /* n-intermediary motif (Sec. 4's variable number  */
                             /* of intermediaries), n legs with one source and  */
                             /* one destination, on each of its 2n edges; n = 2 */
                             /* is the SG column.  Also counted for the stacked  */
                             /* bipartite read for Sec. 8's "Stack" pattern     */
                             /* (the trigger s1->m1, N0.out -> m2, N1.in        */
                             /* intersected with N2.in -> s2, then N1.out       */
                             /* intersected with N2.out -> r1 and again -> r2,  */
                             /* each new account skipping those bound before    */
                             /* it, no order, every stage in the span window):  */
                             /* each instance of eight edges once on each of    */
                             /* them.  Any other program with this aggregate:   */
                             /* AML_EUNSUPPORTED.                               */

#define AML_PAT_INTERPRET 0x1  /* run the program through the generic        */
                               /* interpreter even when a family matches it    */

typedef struct aml_pattern {
  const aml_stage* stages;   /* read during aml_pattern_set_create only          */
  int32_t n_stages;
  int32_t aggregate;         /* AML_AGG_*                                        */
  int32_t delta;             /* time window in seconds, >= 0                     */
  int32_t flags;             /* AML_PAT_* (other bits: AML_EINVAL)               */
} aml_pattern;

/* Pattern families the planner maps stage programs onto (one output column
 * per pattern).  Exact semantics (e = u->v at time t_e; f < e means
 * (t_f, f) < (t_e, e); counts saturate at 2^32-1):
 *   DEG_OUT  #{f : src f = u, f <= e, t_f >= t_e - delta}   (DEG_IN: dst f = v)
 *   FAN_OUT  #distinct dst f over the same edges             (FAN_IN: distinct src)
 *   GS       gather-scatter 2-paths a = x->h, b = h->y, x != y, a < b,
 *            t_b - t_a <= delta, counted on a and on b
 *   SG       scatter-gather: unordered pairs of legs (s->m1->d, s->m2->d),
 *            s != d, m1 != m2, scatter before gather in each leg, all four
 *            edges within delta, counted on all four (Sec. 5, Fig. 4a)
 *   CYC_k    simple directed k-cycles whose edges increase in time around the
 *            cycle from the earliest, spanning <= delta (Sec. 5, Fig. 4b)
 *   CYCW_k   window cycles, k >= 3: simple directed k-cycles spanning <= delta
 *            whose edges may occur in any time order (Sec. 4: funds that do
 *            not traverse the cycle in cycle order, "anticipatory" edges).
 *            Every hop after the trigger only has to come after the trigger
 *            edge.  (For k = 2 the set equals CYC_2 and is planned as CYC.)
 *            Not supported by aml_stream_open (AML_EUNSUPPORTED).        */
#define AML_FAM_DEG_OUT 0
#define AML_FAM_DEG_IN 1
#define AML_FAM_FAN_OUT 2
#define AML_FAM_FAN_IN 3
#define AML_FAM_GS 4
#define AML_FAM_SG 5
#define AML_FAM_CYC 6
#define AML_FAM_CYCW 7
#define AML_FAM_PROGRAM 8  /* a program no family matches, interpreted (below) */

typedef struct aml_pattern_set aml_pattern_set;

/* Generic interpretation (AML_FAM_PROGRAM columns: programs no family
 * matches, or given AML_PAT_INTERPRET).  Alg. 1's nested loop run as
 * written, for every trigger edge e0 = N0 -> N1 that is not a self-loop
 * (self-loop rows are 0).  reach(N0) = reach(N1) = e0; a variable bound by a
 * stage is reached by that stage's edge (INTERSECT: its b-side edge).  A
 * binding gives every stage after the trigger
 *   FOR_ALL   an edge f of a_var's a_dir list (OUT: f = A -> x, IN: f = x -> A),
 *   INTERSECT an edge fa of a_var's a_dir list and fb of b_var's b_dir list
 *             with the same far end x,
 * subject to: x binds out_var if it is new, else equals it (last stage
 * only); x differs from every N_i whose skip_eq bit is set; the order --
 *   FOR_ALL   AFTER reach(A) < f, BEFORE f < reach(A), AFTER_TRIGGER e0 < f,
 *             NONE no constraint (LEG: AML_EUNSUPPORTED);
 *   INTERSECT AFTER reach(A) < fa < fb, BEFORE fb < fa < reach(A),
 *             LEG fa < fb, AFTER_TRIGGER e0 < fa and e0 < fb, NONE none;
 * and the window -- TRAILING: each of the stage's edges g has
 * t_e0 - delta <= t_g and g <= e0; SPAN: the stage's edges join e0 in the
 * span set, whose times differ by at most delta.  The row of e0 gets
 *   EDGES      the number of bindings,
 *   DISTINCT   the number of distinct last-stage nodes x over them,
 *   INSTANCES  nothing directly: every binding whose edges (e0 and all the
 *              stages') are pairwise distinct adds 1 to the row of each of
 *              its edges, from whichever trigger it is found.
 * Every family is such a program; interpreted, each gives its family's
 * counts except SG, whose pairs of legs are each found twice (from both
 * scatter edges, or both gather edges).  Limits: at most 8 stages; one
 * launch visits at most 2^34 candidate edges (beyond: AML_EUNSUPPORTED and
 * the column is not written).  One thread walks each trigger's bindings
 * depth first (a warp when the first stage has more than 64 candidates).
 * Not available to AML_MINE_GRAPH or aml_stream_open (AML_EUNSUPPORTED). */

/* Validate and plan n patterns; column j of the output is pattern j.
 * Validation (Sec. 6: "validates operand dependencies between stages"):
 * stage 0 is the trigger; every operand names a variable bound by an
 * earlier stage; skip masks name bound variables; windows and orders are in
 * range.  A valid program no family matches becomes an AML_FAM_PROGRAM
 * column (generic interpretation, above), or AML_EUNSUPPORTED when it is
 * outside the interpreter's limits.  Host-only; no device work. */
aml_status aml_pattern_set_create(const aml_pattern* patterns, int32_t n_patterns,
                                  aml_pattern_set** out);
aml_status aml_pattern_set_destroy(aml_pattern_set* ps);

typedef struct aml_column_info {
  int32_t family;   /* AML_FAM_*                          */
  int32_t k;        /* cycle length (CYC), else 0         */
  int32_t delta;    /* window seconds                     */
  int32_t reserved;
  char name[32];    /* e.g. "FAN_OUT@86400", "CYC4@604800" */
} aml_column_info;

aml_status aml_pattern_set_num_columns(const aml_pattern_set* ps, int32_t* n_cols);
aml_status aml_pattern_set_column(const aml_pattern_set* ps, int32_t col,
                                  aml_column_info* info);

/* ------------------------------------------------------------------ mining */

#define AML_MINE_HOST_OUTPUT 0x1u  /* counts is a host pointer (copied back)     */
#define AML_MINE_GRAPH 0x2u        /* replay the whole mine as one CUDA graph:   */
                                   /* the first call with a given (pattern set,  */
                                   /* counts, ld, tuning) mines normally and     */
                                   /* captures the kernel sequence on a private  */
                                   /* stream; later calls are one graph launch.  */
                                   /* Device output only.                        */
#define AML_MINE_PERSISTENT 0x4u   /* cycles split by estimated anchor cost: the  */
                                   /* costliest quarter of the anchors (whole    */
                                   /* cost buckets; degree estimate = the first  */
                                   /* window's size) level by level, the rest    */
                                   /* one lane each in a persistent launch       */
                                   /* beside them                                */
#define AML_MINE_LEARNED 0x8u      /* as PERSISTENT, but the costs come from the */
                                   /* cost model trained by aml_cost_train for   */
                                   /* that window (degree estimate when no model */
                                   /* exists)                                   */
#define AML_MINE_FUSED 0x20u       /* the leg pass and the level-by-level cycle  */
                                   /* search of a window in one persistent       */
                                   /* cooperative launch (Sec. 4: the families   */
                                   /* share their first hop): warps take tiles    */
                                   /* of edges from a work queue and count their  */
                                   /* legs; after a grid-wide barrier each block  */
                                   /* places its chunk's legs from all blocks'    */
                                   /* sums; warps take tiles again and emit the   */
                                   /* legs (GS, 2-cycle and SG records, cycle     */
                                   /* legs); then per cycle level warps close     */
                                   /* tiles of paths and each block places its   */
                                   /* chunk's children, barriers between.  The    */
                                   /* SG grouping follows the launch and the      */
                                   /* DEG/FAN pass runs beside it.  The first     */
                                   /* mine of a (graph, window) runs the plain    */
                                   /* sequence to learn the leg and level sizes.  */
                                   /* Not with PERSISTENT/LEARNED.  A barrier     */
                                   /* wait that runs out (see                     */
                                   /* aml_graph_set_wait_limit) ends the launch:  */
                                   /* AML_ETIMEOUT at aml_sync, that mine's       */
                                   /* counts invalid.  While the graph's error    */
                                   /* word is set (until aml_sync reports it) a   */
                                   /* fused mine also skips its SG grouping.      */
#define AML_MINE_HOST_ASYNC 0x10u  /* with HOST_OUTPUT: counts is page-locked    */
                                   /* host memory (cudaHostAlloc / registered),  */
                                   /* the copy back is enqueued on `stream` and  */
                                   /* the call returns without waiting for it:   */
                                   /* synchronize `stream` before reading counts */
                                   /* (pageable memory: AML_EINVAL)              */

/* Count every pattern of `ps` for every edge of `g`.
 *   counts : uint32, row-major, row e = input edge e, column j = pattern j;
 *            element (e, j) at counts[e * ld + j].  Device pointer unless
 *            AML_MINE_HOST_OUTPUT (then the call synchronizes `stream`,
 *            unless AML_MINE_HOST_ASYNC).
 *            Columns >= n_cols of each row are left untouched.
 *   ld     : row stride in elements, ld >= n_cols
 *   flags  : AML_MINE_* (unknown bits: AML_EINVAL)
 * The first call for a given (graph, window) sizes the intermediate buffers
 * and synchronizes `stream` once; later calls enqueue work only.
 * Errors: AML_EINVAL, AML_ENOMEM, AML_ECUDA. */
aml_status aml_mine(aml_graph* g, const aml_pattern_set* ps, uint32_t* counts, int64_t ld,
                    uint32_t flags, void* stream);

/* Runtime tunables of the mining kernels.  None of them changes any count;
 * they trade work distribution against overhead.  Defaults: 32, 384, 48, 256. */
typedef struct aml_tuning {
  int32_t own_max;         /* windows up to this many slots are walked by one lane,
                              longer ones by a whole warp (degree binning), [0, 4096] */
  int32_t sg_bucket_mean;  /* target leg records per scatter-gather hash bucket, [16, 512] */
  int32_t close_scan_max;  /* cycle closing ranges up to this long are scanned, longer ones
                              binary-searched, [0, 4096]                               */
  int32_t block;           /* threads per block of the per-edge kernels: 64, 128, 256, 512 */
} aml_tuning;

aml_status aml_graph_get_tuning(const aml_graph* g, aml_tuning* out);
/* Replace a graph's tunables (AML_EINVAL outside the ranges above); drops
 * the graph's captured mines. */
aml_status aml_graph_set_tuning(aml_graph* g, const aml_tuning* t);

/* Saturation bound of the counts aml_mine writes for `g` (no paper
 * counterpart: the paper states no range for its counts).  Every column is
 * an exact count; a count above the bound is written as the bound, never
 * wrapped.  The bound is 2^32-1 (UINT32_MAX) from aml_graph_create on, the
 * largest value of the uint32 output; no realistic graph gives one edge
 * 2^32 instances, so this call exists for tests, which lower it to a few
 * units to exercise the clamp on tiny graphs.  limit >= 1 (0: AML_EINVAL).
 * Drops the graph's captured mines (AML_MINE_GRAPH). */
aml_status aml_graph_set_count_limit(aml_graph* g, uint32_t limit);

/* Bound on every device-side wait of the graph's kernels (the grid-wide
 * barriers of AML_MINE_FUSED), in SM clock cycles (no paper counterpart).
 * Default 2^32 (about 2 s at 2 GHz): in normal operation every block of a
 * cooperative launch is resident and a barrier completes in microseconds.
 * A wait that runs out gives up: the kernel records ERR_TIMEOUT in the
 * graph's error word and returns, aml_sync returns AML_ETIMEOUT, and that
 * mine's counts are not valid; the context stays usable.  0 gives up at once
 * unless the wait is already over (tests use it to make a wait run out).
 * cycles >= 0 (else AML_EINVAL).  Drops the graph's captured mines. */
aml_status aml_graph_set_wait_limit(aml_graph* g, int64_t cycles);

/* Autotuner: times real mines of `ps` on `g` (median of `repeats` after one
 * warm-up each, CUDA events on `stream`) while sweeping one tunable at a time
 * over a fixed candidate list, keeps the fastest setting on the graph and
 * reports it (best / best_ms may be NULL).  Synchronizes `stream`; allocates
 * a temporary output.  The replacement for the paper's compile-time choice of
 * evaluation plan from neighbourhood size and selectivity (Sec. 6). */
aml_status aml_autotune(aml_graph* g, const aml_pattern_set* ps, int32_t repeats, void* stream,
                        aml_tuning* best, float* best_ms);

/* ------------------------------------------------------------- cost model */

/* Learned cost binning of the persistent cycle search.  A perceptron
 * 16 -> 64 -> 64 -> 1 (ReLU; bf16 weights, fp32 accumulation; inference on
 * tensor cores) maps 16 cheap features of an anchor edge (first-window size,
 * closing-range size, degrees of its nodes, second-hop degree samples, ...)
 * to log(1 + clock64 cycles) of that anchor's search.  aml_cost_train samples
 * up to max_samples anchors of the widest window with cycle columns,
 * measures their cost with the persistent kernel run one anchor per lane
 * (clock64 probe), trains the model on 80% of them with the library's own
 * forward/backward and Adam kernels (minibatch 4096, lr 2e-3) for `epochs`
 * epochs, and evaluates it on the other 20% against the degree estimate
 * (the first-window size).  The model is kept with the graph and used by
 * AML_MINE_LEARNED.  Synchronizes `stream`.  The paper's optimizer chooses
 * evaluation plans from neighbourhood size and selectivity (Sec. 6); this is
 * a learned replacement for that estimate, not a feature of the paper. */
typedef struct aml_cost_report {
  int32_t delta;               /* window the model serves                        */
  int32_t epochs;
  int64_t n_items;             /* anchors with cycle work in that window          */
  int64_t n_train, n_test;
  float final_train_mse;       /* normalized-label MSE of the last epoch          */
  float test_log_mae;          /* mean |predicted - measured| of log(1 + cycles)  */
  float test_spearman;         /* rank correlation, model vs measured cost        */
  float degree_spearman;       /* rank correlation, first-window size vs cost     */
  float warp_threshold_cycles; /* predicted cost at which an anchor gets a warp   */
  float probe_ms;              /* time of the clock64 probe                       */
  float total_ms;              /* whole call                                      */
} aml_cost_report;

aml_status aml_cost_train(aml_graph* g, const aml_pattern_set* ps, int64_t max_samples,
                          int32_t epochs, uint64_t seed, void* stream, aml_cost_report* report);

/* Building blocks of the cost model, on host arrays (for verification):
 * params = 5313 floats (W1[64][16], b1[64], W2[64][64], b2[64], w3[64], b3),
 * x = n x 16 normalized features, y = n labels.  aml_mlp_loss_grad returns
 * the mean squared error and its gradient (forward with weights rounded to
 * bf16, fp32 arithmetic).  aml_mlp_adam_step applies one Adam step (bias
 * corrected, step >= 1) to params, m and v in place.  aml_mlp_predict runs
 * the tensor-core inference on raw features; norm = 16 means, 16 inverse
 * standard deviations, label mean, label std. */
aml_status aml_mlp_loss_grad(const float* params, const float* x, const float* y, int64_t n,
                             float* grad, float* loss);
aml_status aml_mlp_adam_step(float* params, const float* grad, float* m, float* v, int32_t step,
                             float lr, float beta1, float beta2, float eps);
aml_status aml_mlp_predict(const float* params, const float* norm, const float* feat, int64_t n,
                           float* out);

/* Wait for the graph's enqueued work and report device-side errors
 * (AML_ETIMEOUT, AML_EINTERNAL) recorded by its kernels since the last call. */
aml_status aml_sync(aml_graph* g);

/* --------------------------------------------------------------- streaming */

/* Streaming recount (Sec. 5, streaming use: a new transaction adds to the
 * count of every instance it completes, and only its neighbourhood is
 * re-examined).  Transactions arrive in batches whose timestamps never
 * decrease; edges get global row ids in arrival order.  After every append,
 * each resident row holds the count of its column over the whole history.
 * A batch B is recounted exactly by one mine of B and the window W of
 * resident edges at most delta_max older than B's first edge that counts
 * only the instances whose latest edge is in B (those B creates) and adds
 * them to the stored rows.  An append evicts the rows older than both
 * t_max - resident_window and B's first time - delta_max (no later batch
 * can reach them). */
typedef struct aml_stream aml_stream;

typedef struct aml_stream_batch {
  int64_t first_row;           /* global row id of the batch's first edge        */
  int64_t n_rows;              /* edges appended                                  */
  int64_t rows_recounted;      /* resident rows inside the recount window W       */
  int64_t resident_first_row;  /* oldest resident row after the append           */
  int64_t resident_rows;
} aml_stream_batch;

typedef struct aml_stream_info {
  int64_t resident_first_row;
  int64_t resident_rows;
  int64_t capacity_rows;       /* resident rows the budget allows                 */
  int64_t final_end_row;       /* rows below this will never change again         */
  int64_t device_bytes;        /* resident rows plus the kept window graph        */
  int32_t t_max;               /* latest timestamp appended                        */
  int32_t delta_max;           /* largest window of the pattern set               */
} aml_stream_info;

/* Open a stream counting the columns of `ps` (copied) over accounts
 * [0, n_nodes).  resident_window_s must be >= the largest pattern window.
 * mem_budget_bytes bounds the device memory of the stream: half holds
 * resident rows (16 + 4*P bytes each), half is the working set of one append
 * (estimated at 512 + 16*P bytes per edge of the recount window).
 * Errors: AML_EINVAL, AML_ENOMEM, AML_ECUDA. */
aml_status aml_stream_open(const aml_pattern_set* ps, int32_t n_nodes, int32_t resident_window_s,
                           size_t mem_budget_bytes, aml_stream** out);

/* Append n transactions (host arrays, or device arrays with AML_PTR_DEVICE)
 * and recount.  Synchronous: returns when every count is updated.  The batch
 * must be non-decreasing in time (AML_EUNSORTED) and start no earlier than
 * the latest appended timestamp (AML_ELATE); ids must be in [0, n_nodes)
 * (AML_EINVAL).  A batch that does not fit the budget returns AML_EADMIT.
 * On any error the stream is unchanged.  info may be NULL. */
aml_status aml_stream_append(aml_stream* st, const int32_t* src, const int32_t* dst,
                             const int32_t* ts, const float* amount, int64_t n, uint32_t flags,
                             void* stream, aml_stream_batch* info);

/* Copy the counts of resident rows [row0, row0 + n) into out (row-major,
 * stride ld >= P; device pointer, or host with AML_MINE_HOST_OUTPUT, which
 * synchronizes `stream`).  Rows outside the resident range: AML_EINVAL. */
aml_status aml_stream_read(aml_stream* st, int64_t row0, int64_t n, uint32_t* out, int64_t ld,
                           uint32_t flags, void* stream);

aml_status aml_stream_get_info(const aml_stream* st, aml_stream_info* info);

/* Self-check of the kept window graph.  Between appends the stream keeps the
 * graph of the last recount window and makes the next window's graph by
 * updating it (dropping the rows that left, adding the batch) instead of
 * rebuilding it.  This call rebuilds that window's graph from scratch and
 * compares every array of the two; *n_mismatch = the number of differing
 * elements (0 when they are equal or no graph is kept).  Synchronizes the
 * device.  Errors: AML_EINVAL, AML_ENOMEM, AML_ECUDA. */
aml_status aml_stream_check_graph(aml_stream* st, int64_t* n_mismatch);

/* The stream's saturation bound (as aml_graph_set_count_limit; 2^32-1 from
 * aml_stream_open on).  It applies from the next append on: a stored count
 * plus the instances an append adds is saturated at the bound, which keeps
 * every stored count equal to min(full-history count, bound).  limit >= 1. */
aml_status aml_stream_set_count_limit(aml_stream* st, uint32_t limit);

aml_status aml_stream_close(aml_stream* st);

/* ------------------------------------------------------ allocation-free FAN */

/* FAN_OUT (direction = AML_DIR_OUT) or FAN_IN (AML_DIR_IN) of every edge for
 * one window, computed without any device memory allocation.  The paper has
 * no counterpart of this call: it exists for callers that cannot allocate at
 * the point of use -- code running while a CUDA stream capture is active,
 * serving processes that reserve their whole device-memory budget up front,
 * and latency-critical loops that cannot afford an allocator's implicit
 * synchronization.  aml_mine allocates scratch on every call; this does not.
 *   g      : a graph made earlier by aml_graph_create
 *   delta  : trailing window in seconds, >= 0
 *   out    : device uint32[E], caller-owned; out[e] = the count for edge e,
 *            equal to aml_mine's FAN_OUT / FAN_IN column for the same window
 *   stream : the work is enqueued on it; the call does not wait for it
 * Limit: at most 4,194,304 non-loop edges (aml_graph_info.n_list_edges);
 * larger graphs get AML_EINVAL.  Scratch: one fixed 32 MiB + 8 KiB __device__
 * array, reserved on every GPU that loads the library until the process
 * exits and shared by all calls -- calls that overlap on the GPU (concurrent
 * streams or host threads) race on it and give wrong counts, so serialize
 * them.  Each call writes every scratch word before reading it, so nothing
 * from an earlier call leaks into a result.  The first call on each device
 * resolves the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  No cudaMalloc, cudaFree or other
 * allocating routine is called. */
aml_status aml_fan_noalloc(const aml_graph* g, int32_t delta, int32_t direction, uint32_t* out,
                           void* stream);

/* --------------------------------------------------------------- profiling */

/* Number of kernels the library has launched in this process (all devices,
 * all threads).  The difference across a region counts its launches. */
aml_status aml_launch_count(int64_t* out);

/* Start (on != 0) or stop timing every kernel launch with a pair of CUDA
 * events recorded on the launching stream.  Launches during stream capture
 * are not timed.  Costs two event records per launch while on; mines run
 * their kernels one after another meanwhile (no concurrent branches), so
 * each time is the kernel's own. */
aml_status aml_profile_enable(int32_t on);

typedef struct aml_kernel_stat {
  char name[40];       /* kernel name, e.g. "k_assemble"                     */
  int64_t launches;    /* timed launches                                     */
  double total_ms;     /* summed event-to-event time of those launches       */
} aml_kernel_stat;

/* Wait for the recorded events, fold them into per-kernel totals and copy up
 * to `cap` totals into `stats` (may be NULL); *n_out receives the number of
 * distinct kernels.  reset != 0 clears the totals afterwards. */
aml_status aml_profile_read(aml_kernel_stat* stats, int32_t cap, int32_t* n_out, int32_t reset);

#ifdef __cplusplus
}
#endif
#endif /* AML_H */
