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

#ifdef __cplusplus
}
#endif
#endif
