/*
 * CPU oracle for per-edge AML pattern counts -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct C.  Only the test-suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the product library never
 * does.  It shares no code, header or table with the CUDA path.
 *
 * Column definitions (the paper's stage semantics, Sec. 5 and Alg. 1; edge e =
 * (u->v, t_e), id = input index; f < e means (t_f, f) < (t_e, e); self-loops are
 * in no list and their rows are 0; counts saturate at 2^32-1):
 *   DEG_OUT(e)  #{f : src f = u, f <= e, t_f >= t_e - delta}      (DEG_IN: dst f = v)
 *   FAN_OUT(e)  #distinct dst f over that same set                 (FAN_IN: distinct src)
 *   GS(e)       #{(a,b): dst a = src b, src a != dst b, a < b, t_b - t_a <= delta, e in {a,b}}
 *   SG(e)       #{unordered leg pairs {(s->m1, m1->d), (s->m2, m2->d)}: s != d, m1 != m2,
 *                 scatter < gather inside each leg, span of the 4 edges <= delta, e among them}
 *   CYC_k(e)    #{k-edge simple directed cycles, <-increasing cyclically from their
 *                 <-minimum edge, span <= delta, containing e}
 *   CYCW_k(e)   #{k-edge simple directed cycles with span <= delta, their edges in
 *                 any time order, containing e} (Sec. 4: cycles whose edges are not
 *                 observed in cycle order, "anticipatory" edges; window constraint only)
 * Parity with an external reference implementation: unpinned (none exists);
 * every function below is pinned by the brute-force, exact-variant,
 * planted-motif and invariant tests instead.
 */
#ifndef AML_ORACLE_H
#define AML_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum {
  OG_DEG_OUT = 0,
  OG_DEG_IN = 1,
  OG_FAN_OUT = 2,
  OG_FAN_IN = 3,
  OG_GS = 4,
  OG_SG = 5,
  OG_CYC = 6,
  OG_CYCW = 7
};

typedef struct og_col {
  int32_t kind;   /* OG_* */
  int32_t k;      /* cycle length for OG_CYC / OG_CYCW, else ignored */
  int64_t delta;  /* window in seconds, >= 0 */
} og_col;

typedef struct og_graph og_graph;

/* Copies the arrays.  Returns NULL on bad input (ids out of [0,N), E < 0). */
og_graph* og_graph_new(const int32_t* src, const int32_t* dst, const int32_t* ts,
                       int64_t n_edges, int32_t n_nodes);
void og_graph_free(og_graph* g);

/* Canonical enumeration: every instance is found once, from a canonical
 * anchor, and credited to all of its edges.  out: E x ncols row-major. */
int og_count_all(const og_graph* g, const og_col* cols, int32_t ncols,
                 uint32_t* out, int32_t nthreads);

/* Edge-centric query: the counts of the n listed edges, each found by
 * searching outward from that edge in every role it can play (a different
 * enumeration from og_count_all).  out: n x ncols row-major. */
int og_count_edges(const og_graph* g, const og_col* cols, int32_t ncols,
                   const int64_t* eids, int64_t n, uint32_t* out, int32_t nthreads);

/* The same two enumerations with the saturation bound as an argument:
 * every count above `limit` (>= 1) is reported as `limit`.  The plain calls
 * use limit = 2^32-1; tests pass small limits so that the clamp is reached
 * on tiny graphs (no realistic graph reaches 2^32 instances of one edge). */
int og_count_all_limit(const og_graph* g, const og_col* cols, int32_t ncols,
                       uint32_t* out, int32_t nthreads, uint32_t limit);
int og_count_edges_limit(const og_graph* g, const og_col* cols, int32_t ncols,
                         const int64_t* eids, int64_t n, uint32_t* out, int32_t nthreads,
                         uint32_t limit);

/* ---------------- stage programs (Sec. 5; Alg. 1's nested loop per stage) ----------------
 *
 * A program is a trigger (stage 0: the edge e0 = N0 -> N1) and stages
 * 1..n-1, each binding node variables by iterating neighbour lists.  This is
 * the generic interpretation a program gets when no pattern family applies.
 * reach(N0) = reach(N1) = e0; a variable bound by a stage is reached by that
 * stage's edge (INTERSECT: its b-side edge).  A binding gives every stage:
 *   FOR_ALL (a_var = A, a_dir): an edge f of A's list (OUT: f = A -> x,
 *     IN: f = x -> A; self-loops are in no list); x is the stage's node.
 *   INTERSECT (A.a_dir, B.b_dir): edges fa of A's a_dir list and fb of B's
 *     b_dir list whose other ends are the same node x.
 * and every stage must satisfy:
 *   out_var  new: x binds it; already bound (last stage only): x equals it.
 *   skip_eq  x differs from N_i for every set bit i.
 *   order    FOR_ALL: AFTER reach(A) < f, BEFORE f < reach(A), AFTER_TRIGGER
 *            e0 < f, NONE nothing (LEG is not defined for FOR_ALL).
 *            INTERSECT: AFTER reach(A) < fa < fb, BEFORE fb < fa < reach(A),
 *            LEG fa < fb, AFTER_TRIGGER e0 < fa and e0 < fb, NONE nothing.
 *   window   TRAILING: each of the stage's edges g has t_e0 - delta <= t_g
 *            and g <= e0.  SPAN: the stage's edges join e0 in the span set,
 *            whose latest and earliest times differ by at most delta.
 * Aggregate for the row of trigger e0 (self-loop triggers: 0):
 *   EDGES      the number of bindings;
 *   DISTINCT   the number of distinct last-stage nodes x over them;
 *   INSTANCES  a binding whose edges (e0 and all stages') are pairwise
 *              distinct is an instance, and adds 1 to the row of each of its
 *              edges (credited from every trigger it is found from).
 *   SETS       the distinct edge sets of the instances: each set adds 1 to
 *              the row of each of its edges, once, however many bindings
 *              (triggers, orders of its stages) find it.  For the
 *              scatter-gather of n intermediaries (n - 1 intersections, each
 *              a further intermediary) a set is n legs with one source and
 *              one destination: the exact n-intermediary motif.
 * Every family above is one such program; e.g. the chain of AFTER stages
 * closing on N0 counts CYC_k, and SG's program finds each pair of legs
 * twice (once from each scatter edge). */
enum { OG_OP_TRIGGER = 0, OG_OP_FOR_ALL = 1, OG_OP_INTERSECT = 2 };
enum { OG_DIR_OUT = 0, OG_DIR_IN = 1 };
enum { OG_ORD_NONE = 0, OG_ORD_AFTER = 1, OG_ORD_BEFORE = 2, OG_ORD_LEG = 3,
       OG_ORD_AFTER_TRIGGER = 4 };
enum { OG_WIN_TRAILING = 0, OG_WIN_SPAN = 1 };
enum { OG_AGG_EDGES = 0, OG_AGG_DISTINCT = 1, OG_AGG_INSTANCES = 2, OG_AGG_SETS = 3 };

/* Amount constraints (edge attributes as operands): RANGE = every edge g of
 * the stage has amount_min <= amount(g) <= amount_max; RATIO = every edge
 * g has ratio_min * amount(p) <= amount(g) <= ratio_max * amount(p) with p
 * the edge before g on the walk (reach(A) for a FOR_ALL edge and an
 * intersection's fa; fa for its fb), products in double.  On the trigger,
 * RANGE only: it selects the trigger edges.  Amounts come from
 * og_graph_set_amounts (all 0 otherwise). */
enum { OG_AMT_RANGE = 1, OG_AMT_RATIO = 2 };

typedef struct og_stage {
  int32_t op, a_var, a_dir, b_var, b_dir, out_var, order, window;
  uint32_t skip_eq;
  uint32_t amount_flags;
  float amount_min, amount_max, ratio_min, ratio_max;
} og_stage;

/* Copies the n_edges float32 amounts used by amount constraints. */
void og_graph_set_amounts(og_graph* g, const float* amount);

/* Counts of one program for every edge: out[E] (uint32, saturated).
 * Returns 0, or -1 for a program outside the forms defined above (at most
 * 16 stages and 17 variables). */
int og_program_count(const og_graph* g, const og_stage* st, int32_t n_stages,
                     int32_t aggregate, int64_t delta, uint32_t* out, int32_t nthreads);

#ifdef __cplusplus
}
#endif
#endif
