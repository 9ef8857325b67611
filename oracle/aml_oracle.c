/*
 * CPU oracle for per-edge AML pattern counts -- TEST INFRASTRUCTURE ONLY.
 * Loaded by the tests, the smoke check and the benchmark's CPU-baseline leg;
 * never by the product library.  Plain nested loops in the shape of the
 * paper's per-stage loop (Alg. 1): find the window start by binary search
 * (Find_Starting_Edge), iterate, break when the time window is exceeded,
 * skip excluded nodes, and credit every edge of every instance found.
 * Counts accumulate in uint64 and are clamped to 2^32-1 on output.
 */
#define _GNU_SOURCE /* qsort_r */
#include "aml_oracle.h"

#include <omp.h>
#include <stdlib.h>
#include <string.h>

struct og_graph {
  int64_t E;
  int32_t N;
  int32_t *src, *dst, *ts;
  float* amount;                 /* for amount constraints; 0 unless set    */
  int64_t *out_start, *in_start; /* N+1 row offsets                         */
  int64_t *out_list, *in_list;   /* non-loop edge ids, rows in (t,id) order  */
  int64_t *pos_out, *pos_in;     /* position of e in its rows, -1 for loops  */
};

typedef struct { int32_t t; int64_t id; } tkey;

static int cmp_tkey(const void* a, const void* b) {
  const tkey* x = (const tkey*)a;
  const tkey* y = (const tkey*)b;
  if (x->t != y->t) return x->t < y->t ? -1 : 1;
  return x->id < y->id ? -1 : (x->id > y->id ? 1 : 0);
}

/* f precedes e in the strict total order (t, id) */
static inline int prec(const og_graph* g, int64_t f, int64_t e) {
  return g->ts[f] < g->ts[e] || (g->ts[f] == g->ts[e] && f < e);
}

/* Find_Start: first i in [lo,hi) with t(list[i]) >= tmin */
static int64_t find_start(const og_graph* g, const int64_t* list, int64_t lo, int64_t hi,
                          int64_t tmin) {
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if ((int64_t)g->ts[list[mid]] < tmin) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/* first i in [lo,hi) whose edge comes strictly after e */
static int64_t first_after(const og_graph* g, const int64_t* list, int64_t lo, int64_t hi,
                           int64_t e) {
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (!prec(g, e, list[mid])) lo = mid + 1; else hi = mid;
  }
  return lo;
}

og_graph* og_graph_new(const int32_t* src, const int32_t* dst, const int32_t* ts,
                       int64_t E, int32_t N) {
  if (E < 0 || N < 0) return NULL;
  for (int64_t e = 0; e < E; ++e)
    if (src[e] < 0 || src[e] >= N || dst[e] < 0 || dst[e] >= N) return NULL;
  og_graph* g = (og_graph*)calloc(1, sizeof(og_graph));
  g->E = E;
  g->N = N;
  size_t e4 = (size_t)(E > 0 ? E : 1) * 4, e8 = (size_t)(E > 0 ? E : 1) * 8;
  g->src = (int32_t*)malloc(e4);
  g->dst = (int32_t*)malloc(e4);
  g->ts = (int32_t*)malloc(e4);
  g->amount = (float*)calloc((size_t)(E > 0 ? E : 1), 4);
  if (E) {
    memcpy(g->src, src, (size_t)E * 4);
    memcpy(g->dst, dst, (size_t)E * 4);
    memcpy(g->ts, ts, (size_t)E * 4);
  }
  g->out_start = (int64_t*)calloc((size_t)N + 1, 8);
  g->in_start = (int64_t*)calloc((size_t)N + 1, 8);
  g->out_list = (int64_t*)malloc(e8);
  g->in_list = (int64_t*)malloc(e8);
  g->pos_out = (int64_t*)malloc(e8);
  g->pos_in = (int64_t*)malloc(e8);

  /* global (t, id) order of the non-loop edges */
  tkey* ord = (tkey*)malloc(sizeof(tkey) * (size_t)(E > 0 ? E : 1));
  int64_t nv = 0;
  for (int64_t e = 0; e < E; ++e) {
    g->pos_out[e] = -1;
    g->pos_in[e] = -1;
    if (src[e] == dst[e]) continue;
    ord[nv].t = ts[e];
    ord[nv].id = e;
    ++nv;
  }
  qsort(ord, (size_t)nv, sizeof(tkey), cmp_tkey);
  for (int64_t i = 0; i < nv; ++i) {
    g->out_start[g->src[ord[i].id] + 1]++;
    g->in_start[g->dst[ord[i].id] + 1]++;
  }
  for (int32_t u = 0; u < N; ++u) {
    g->out_start[u + 1] += g->out_start[u];
    g->in_start[u + 1] += g->in_start[u];
  }
  int64_t* fo = (int64_t*)malloc(((size_t)N + 1) * 8);
  int64_t* fi = (int64_t*)malloc(((size_t)N + 1) * 8);
  memcpy(fo, g->out_start, ((size_t)N + 1) * 8);
  memcpy(fi, g->in_start, ((size_t)N + 1) * 8);
  /* walking the global order keeps every row in (t, id) order */
  for (int64_t i = 0; i < nv; ++i) {
    int64_t e = ord[i].id;
    int64_t p = fo[g->src[e]]++;
    g->out_list[p] = e;
    g->pos_out[e] = p;
    int64_t q = fi[g->dst[e]]++;
    g->in_list[q] = e;
    g->pos_in[e] = q;
  }
  free(fo);
  free(fi);
  free(ord);
  return g;
}

void og_graph_set_amounts(og_graph* g, const float* amount) {
  if (g && amount && g->E) memcpy(g->amount, amount, (size_t)g->E * 4);
}

void og_graph_free(og_graph* g) {
  if (!g) return;
  free(g->src); free(g->dst); free(g->ts); free(g->amount);
  free(g->out_start); free(g->in_start);
  free(g->out_list); free(g->in_list);
  free(g->pos_out); free(g->pos_in);
  free(g);
}

static int32_t max_row(const og_graph* g) {
  int64_t m = 1;
  for (int32_t u = 0; u < g->N; ++u) {
    int64_t a = g->out_start[u + 1] - g->out_start[u];
    int64_t b = g->in_start[u + 1] - g->in_start[u];
    if (a > m) m = a;
    if (b > m) m = b;
  }
  return (int32_t)m;
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* ---------------- DEG / FAN (trailing window [t_e - delta, e]) ---------------- */

/* window of e in its out-row (outgoing=1) or in-row: [lo, pos] */
static void trailing_window(const og_graph* g, int64_t e, int outgoing, int64_t delta,
                            int64_t* lo, int64_t* pos, const int64_t** list) {
  int32_t node = outgoing ? g->src[e] : g->dst[e];
  const int64_t* start = outgoing ? g->out_start : g->in_start;
  *list = outgoing ? g->out_list : g->in_list;
  *pos = outgoing ? g->pos_out[e] : g->pos_in[e];
  *lo = find_start(g, *list, start[node], *pos + 1, (int64_t)g->ts[e] - delta);
}

/* canonical FAN: sort the window's counterparties, count distinct values */
static uint64_t fan_sorted(const og_graph* g, int64_t e, int outgoing, int64_t delta,
                           int32_t* buf) {
  int64_t lo, pos;
  const int64_t* list;
  trailing_window(g, e, outgoing, delta, &lo, &pos, &list);
  int64_t n = 0;
  for (int64_t i = lo; i <= pos; ++i)
    buf[n++] = outgoing ? g->dst[list[i]] : g->src[list[i]];
  qsort(buf, (size_t)n, 4, cmp_i32);
  uint64_t d = 0;
  for (int64_t i = 0; i < n; ++i)
    if (i == 0 || buf[i] != buf[i - 1]) ++d;
  return d;
}

/* edge-centric FAN: mark counterparties with a per-query stamp */
static uint64_t fan_stamp(const og_graph* g, int64_t e, int outgoing, int64_t delta,
                          int64_t* stamp, int64_t q) {
  int64_t lo, pos;
  const int64_t* list;
  trailing_window(g, e, outgoing, delta, &lo, &pos, &list);
  uint64_t d = 0;
  for (int64_t i = lo; i <= pos; ++i) {
    int32_t c = outgoing ? g->dst[list[i]] : g->src[list[i]];
    if (stamp[c] != q) { stamp[c] = q; ++d; }
  }
  return d;
}

static uint64_t deg(const og_graph* g, int64_t e, int outgoing, int64_t delta) {
  int64_t lo, pos;
  const int64_t* list;
  trailing_window(g, e, outgoing, delta, &lo, &pos, &list);
  return (uint64_t)(pos - lo + 1);
}

/* ---------------- canonical enumeration ---------------- */

#define ACC(e, c) acc[(size_t)(e) * (size_t)ncols + (size_t)(c)]

static void add(uint64_t* p, uint64_t v) {
#pragma omp atomic
  *p += v;
}

/* GS: each instance (a, b) found once, from its gather leg a */
static void canon_gs(const og_graph* g, int col, int ncols, int64_t delta, uint64_t* acc,
                     int nth) {
#pragma omp parallel for schedule(dynamic, 256) num_threads(nth)
  for (int64_t a = 0; a < g->E; ++a) {
    if (g->pos_out[a] < 0) continue;
    int32_t x = g->src[a], h = g->dst[a];
    int64_t hi = g->out_start[h + 1];
    for (int64_t i = first_after(g, g->out_list, g->out_start[h], hi, a); i < hi; ++i) {
      int64_t b = g->out_list[i];
      if ((int64_t)g->ts[b] - g->ts[a] > delta) break;  /* break_if: window overflow */
      if (g->dst[b] == x) continue;                       /* skip_if: y == x */
      add(&ACC(a, col), 1);
      add(&ACC(b, col), 1);
    }
  }
}

/* SG: trigger a1 = s->m1, expand m1.out -> b1 = m1->d (for_all), then the
 * second leg from the intersection of s.out and d.in: a2 = s->m2, b2 = m2->d.
 * Requiring m2 > m1 finds each unordered pair of legs exactly once. */
static void canon_sg(const og_graph* g, int col, int ncols, int64_t delta, uint64_t* acc,
                     int nth) {
#pragma omp parallel for schedule(dynamic, 64) num_threads(nth)
  for (int64_t a1 = 0; a1 < g->E; ++a1) {
    if (g->pos_out[a1] < 0) continue;
    int32_t s = g->src[a1], m1 = g->dst[a1];
    int64_t lo = g->ts[a1];
    int64_t j_end = g->out_start[m1 + 1];
    for (int64_t j = first_after(g, g->out_list, g->out_start[m1], j_end, a1); j < j_end; ++j) {
      int64_t b1 = g->out_list[j];
      int64_t hi = g->ts[b1];
      if (hi - lo > delta) break;
      int32_t d = g->dst[b1];
      if (d == s) continue;
      int64_t i_end = g->out_start[s + 1];
      for (int64_t i = find_start(g, g->out_list, g->out_start[s], i_end, hi - delta); i < i_end;
           ++i) {
        int64_t a2 = g->out_list[i];
        if ((int64_t)g->ts[a2] > lo + delta) break;
        int32_t m2 = g->dst[a2];
        if (m2 <= m1 || m2 == d) continue;
        int64_t lo2 = lo < g->ts[a2] ? lo : g->ts[a2];
        int64_t q_end = g->out_start[m2 + 1];
        for (int64_t q = first_after(g, g->out_list, g->out_start[m2], q_end, a2); q < q_end; ++q) {
          int64_t b2 = g->out_list[q];
          if ((int64_t)g->ts[b2] > lo2 + delta) break;
          if (g->dst[b2] != d) continue;
          int64_t mx = hi > g->ts[b2] ? hi : g->ts[b2];
          if (mx - lo2 > delta) continue;
          add(&ACC(a1, col), 1);
          add(&ACC(b1, col), 1);
          add(&ACC(a2, col), 1);
          add(&ACC(b2, col), 1);
        }
      }
    }
  }
}

/* CYC: depth-first from each edge taken as the cycle's earliest edge e1 =
 * u0->u1; each hop goes to a later edge inside t(e1)+delta and to a node not
 * yet on the path; an edge back into u0 closes a cycle of length depth+1.
 * CYCW (window cycles, any time order): the same walk, but each hop only has
 * to come after e1 (the cycle's earliest edge), not after the previous hop. */
typedef struct {
  const og_graph* g;
  int K;
  int window; /* CYCW: hops after e1 instead of after the previous hop */
  const int* colmap; /* colmap[k] = column of CYC_k for this delta, or -1 */
  int ncols;
  uint64_t* acc;
  int64_t tmax;
  int64_t edges[16];
  int32_t nodes[17];
} cyc_ctx;

static void cyc_dfs(cyc_ctx* c, int depth) {
  const og_graph* g = c->g;
  int ncols = c->ncols;
  uint64_t* acc = c->acc;
  int32_t w = c->nodes[depth];
  int64_t end = g->out_start[w + 1];
  int64_t after = c->window ? c->edges[0] : c->edges[depth - 1];
  for (int64_t i = first_after(g, g->out_list, g->out_start[w], end, after); i < end; ++i) {
    int64_t f = g->out_list[i];
    if ((int64_t)g->ts[f] > c->tmax) break;
    int32_t x = g->dst[f];
    if (x == c->nodes[0]) {
      int k = depth + 1;
      if (k <= c->K && c->colmap[k] >= 0) {
        for (int j = 0; j < depth; ++j) add(&ACC(c->edges[j], c->colmap[k]), 1);
        add(&ACC(f, c->colmap[k]), 1);
      }
      continue;
    }
    if (depth + 1 >= c->K) continue;
    int seen = 0;
    for (int j = 1; j <= depth; ++j) seen |= (c->nodes[j] == x);
    if (seen) continue;
    c->edges[depth] = f;
    c->nodes[depth + 1] = x;
    cyc_dfs(c, depth + 1);
  }
}

static void canon_cyc(const og_graph* g, int K, const int* colmap, int ncols, int64_t delta,
                      uint64_t* acc, int nth, int window) {
#pragma omp parallel for schedule(dynamic, 64) num_threads(nth)
  for (int64_t e1 = 0; e1 < g->E; ++e1) {
    if (g->pos_out[e1] < 0) continue;
    cyc_ctx c;
    c.g = g;
    c.K = K;
    c.window = window;
    c.colmap = colmap;
    c.ncols = ncols;
    c.acc = acc;
    c.tmax = (int64_t)g->ts[e1] + delta;
    c.edges[0] = e1;
    c.nodes[0] = g->src[e1];
    c.nodes[1] = g->dst[e1];
    cyc_dfs(&c, 1);
  }
}

static int check_cols(const og_col* cols, int32_t ncols) {
  for (int i = 0; i < ncols; ++i) {
    if (cols[i].kind < OG_DEG_OUT || cols[i].kind > OG_CYCW) return -1;
    if (cols[i].delta < 0) return -1;
    if ((cols[i].kind == OG_CYC || cols[i].kind == OG_CYCW) && (cols[i].k < 2 || cols[i].k > 15))
      return -1;
  }
  return 0;
}

/* Saturation: every exact (uint64) count above `limit` is reported as
 * `limit` (2^32-1 unless a test lowers it to reach the clamp with tiny
 * counts); nothing wraps. */
static uint32_t saturate(uint64_t v, uint32_t limit) {
  return v > (uint64_t)limit ? limit : (uint32_t)v;
}

static void clamp_out(const uint64_t* acc, uint32_t* out, size_t n, uint32_t limit) {
  for (size_t i = 0; i < n; ++i) out[i] = saturate(acc[i], limit);
}

int og_count_all(const og_graph* g, const og_col* cols, int32_t ncols, uint32_t* out,
                 int32_t nthreads) {
  return og_count_all_limit(g, cols, ncols, out, nthreads, 0xffffffffu);
}

int og_count_all_limit(const og_graph* g, const og_col* cols, int32_t ncols, uint32_t* out,
                       int32_t nthreads, uint32_t limit) {
  if (!g || ncols <= 0 || check_cols(cols, ncols) || limit == 0) return -1;
  int nth = nthreads > 0 ? nthreads : omp_get_max_threads();
  size_t n = (size_t)g->E * (size_t)ncols;
  uint64_t* acc = (uint64_t*)calloc(n ? n : 1, 8);
  if (!acc) return -2;
  int32_t mr = max_row(g);
  char* done = (char*)calloc((size_t)ncols, 1);
  for (int c = 0; c < ncols; ++c) {
    int kind = cols[c].kind;
    int64_t delta = cols[c].delta;
    if (kind <= OG_FAN_IN) {
      int outgoing = (kind == OG_DEG_OUT || kind == OG_FAN_OUT);
      int is_fan = (kind == OG_FAN_OUT || kind == OG_FAN_IN);
#pragma omp parallel num_threads(nth)
      {
        int32_t* buf = (int32_t*)malloc((size_t)mr * 4);
#pragma omp for schedule(dynamic, 256)
        for (int64_t e = 0; e < g->E; ++e) {
          if (g->pos_out[e] < 0) continue;
          ACC(e, c) = is_fan ? fan_sorted(g, e, outgoing, delta, buf) : deg(g, e, outgoing, delta);
        }
        free(buf);
      }
    } else if (kind == OG_GS) {
      canon_gs(g, c, ncols, delta, acc, nth);
    } else if (kind == OG_SG) {
      canon_sg(g, c, ncols, delta, acc, nth);
    } else if ((kind == OG_CYC || kind == OG_CYCW) && !done[c]) {
      /* one depth-first search serves every cycle length with this delta */
      int colmap[17];
      for (int k = 0; k < 17; ++k) colmap[k] = -1;
      int K = 0;
      for (int c2 = c; c2 < ncols; ++c2) {
        if (cols[c2].kind == kind && cols[c2].delta == delta && !done[c2]) {
          if (colmap[cols[c2].k] < 0) {
            colmap[cols[c2].k] = c2;
            done[c2] = 1;
            if (cols[c2].k > K) K = cols[c2].k;
          }
        }
      }
      canon_cyc(g, K, colmap, ncols, delta, acc, nth, kind == OG_CYCW);
      /* duplicate columns (same k and delta) copy the first one */
      for (int c2 = c; c2 < ncols; ++c2)
        if (cols[c2].kind == kind && cols[c2].delta == delta && !done[c2]) {
          int src_c = colmap[cols[c2].k];
          for (int64_t e = 0; e < g->E; ++e) ACC(e, c2) = ACC(e, src_c);
          done[c2] = 1;
        }
    }
  }
  clamp_out(acc, out, n, limit);
  free(acc);
  free(done);
  return 0;
}

/* ---------------- edge-centric queries ---------------- */

static uint64_t ec_gs(const og_graph* g, int64_t e, int64_t delta) {
  uint64_t cnt = 0;
  /* e as the gather leg a = x->h: later b = h->y, y != x */
  int32_t x = g->src[e], h = g->dst[e];
  int64_t end = g->out_start[h + 1];
  for (int64_t i = first_after(g, g->out_list, g->out_start[h], end, e); i < end; ++i) {
    int64_t b = g->out_list[i];
    if ((int64_t)g->ts[b] - g->ts[e] > delta) break;
    if (g->dst[b] != x) ++cnt;
  }
  /* e as the scatter leg b = h->y: earlier a = x->h, x != y */
  h = g->src[e];
  int32_t y = g->dst[e];
  int64_t lo = find_start(g, g->in_list, g->in_start[h], g->in_start[h + 1],
                          (int64_t)g->ts[e] - delta);
  for (int64_t i = lo; i < g->in_start[h + 1]; ++i) {
    int64_t a = g->in_list[i];
    if (!prec(g, a, e)) break;
    if (g->src[a] != y) ++cnt;
  }
  return cnt;
}

/* number of legs (a2 = s->m2, b2 = m2->d) with m2 != m1, a2 < b2, whose union
 * with the leg spanning [lo, hi] spans at most delta; enumerated gather-first
 * through d.in and m2.in (the canonical pass goes scatter-first) */
static uint64_t ec_partners(const og_graph* g, int32_t s, int32_t d, int32_t m1, int64_t lo,
                            int64_t hi, int64_t delta) {
  uint64_t cnt = 0;
  int64_t end = g->in_start[d + 1];
  for (int64_t i = find_start(g, g->in_list, g->in_start[d], end, hi - delta); i < end; ++i) {
    int64_t b2 = g->in_list[i];
    int64_t tb = g->ts[b2];
    if (tb > lo + delta) break;
    int32_t m2 = g->src[b2];
    if (m2 == m1) continue;
    int64_t mx = hi > tb ? hi : tb;
    int64_t jend = g->in_start[m2 + 1];
    for (int64_t j = find_start(g, g->in_list, g->in_start[m2], jend, mx - delta); j < jend; ++j) {
      int64_t a2 = g->in_list[j];
      if (!prec(g, a2, b2)) break;
      if (g->src[a2] != s) continue;
      int64_t mn = lo < g->ts[a2] ? lo : g->ts[a2];
      if (mx - mn <= delta) ++cnt;
    }
  }
  return cnt;
}

static uint64_t ec_sg(const og_graph* g, int64_t e, int64_t delta) {
  uint64_t cnt = 0;
  /* e = s->m1 as the scatter edge of its leg */
  int32_t s = g->src[e], m1 = g->dst[e];
  int64_t end = g->out_start[m1 + 1];
  for (int64_t j = first_after(g, g->out_list, g->out_start[m1], end, e); j < end; ++j) {
    int64_t b1 = g->out_list[j];
    if ((int64_t)g->ts[b1] - g->ts[e] > delta) break;
    int32_t d = g->dst[b1];
    if (d == s) continue;
    cnt += ec_partners(g, s, d, m1, g->ts[e], g->ts[b1], delta);
  }
  /* e = m1->d as the gather edge of its leg */
  m1 = g->src[e];
  int32_t d = g->dst[e];
  end = g->in_start[m1 + 1];
  for (int64_t j = find_start(g, g->in_list, g->in_start[m1], end, (int64_t)g->ts[e] - delta);
       j < end; ++j) {
    int64_t a1 = g->in_list[j];
    if (!prec(g, a1, e)) break;
    int32_t s2 = g->src[a1];
    if (s2 == d) continue;
    cnt += ec_partners(g, s2, d, m1, g->ts[a1], g->ts[e], delta);
  }
  return cnt;
}

/* cycles through e = x->y: simple paths y -> ... -> x of k-1 edges inside
 * [t_e - delta, t_e + delta]; a closed walk is a temporal cycle iff its edge
 * sequence, read cyclically, has exactly one descent under <, and it spans
 * at most delta (a window cycle: the span alone) */
typedef struct {
  const og_graph* g;
  int k;
  int window;
  int64_t delta, tlo, thi;
  int64_t edges[16];
  int32_t nodes[17];
  uint64_t cnt;
} ec_cyc_ctx;

static void ec_cyc_dfs(ec_cyc_ctx* c, int depth, int64_t mint, int64_t maxt, int ndesc) {
  const og_graph* g = c->g;
  int32_t w = c->nodes[depth];
  int32_t x = c->nodes[0];
  int64_t end = g->out_start[w + 1];
  for (int64_t i = find_start(g, g->out_list, g->out_start[w], end, c->tlo); i < end; ++i) {
    int64_t f = g->out_list[i];
    int64_t tf = g->ts[f];
    if (tf > c->thi) break;
    int32_t z = g->dst[f];
    int nd = ndesc + prec(g, f, c->edges[depth - 1]);
    int64_t mn = mint < tf ? mint : tf, mx = maxt > tf ? maxt : tf;
    if (mx - mn > c->delta) continue;
    if (depth + 1 == c->k) {
      if (z != x) continue;
      nd += prec(g, c->edges[0], f);
      if (nd == 1 || c->window) c->cnt++;
      continue;
    }
    if (z == x || (nd > 1 && !c->window)) continue;
    int seen = 0;
    for (int j = 1; j <= depth; ++j) seen |= (c->nodes[j] == z);
    if (seen) continue;
    c->edges[depth] = f;
    c->nodes[depth + 1] = z;
    ec_cyc_dfs(c, depth + 1, mn, mx, nd);
  }
}

static uint64_t ec_cyc(const og_graph* g, int64_t e, int k, int64_t delta, int window) {
  ec_cyc_ctx c;
  c.g = g;
  c.k = k;
  c.window = window;
  c.delta = delta;
  c.tlo = (int64_t)g->ts[e] - delta;
  c.thi = (int64_t)g->ts[e] + delta;
  c.edges[0] = e;
  c.nodes[0] = g->src[e];
  c.nodes[1] = g->dst[e];
  c.cnt = 0;
  ec_cyc_dfs(&c, 1, g->ts[e], g->ts[e], 0);
  return c.cnt;
}

int og_count_edges(const og_graph* g, const og_col* cols, int32_t ncols, const int64_t* eids,
                   int64_t n, uint32_t* out, int32_t nthreads) {
  return og_count_edges_limit(g, cols, ncols, eids, n, out, nthreads, 0xffffffffu);
}

int og_count_edges_limit(const og_graph* g, const og_col* cols, int32_t ncols,
                         const int64_t* eids, int64_t n, uint32_t* out, int32_t nthreads,
                         uint32_t limit) {
  if (!g || ncols <= 0 || check_cols(cols, ncols) || n < 0 || limit == 0) return -1;
  for (int64_t i = 0; i < n; ++i)
    if (eids[i] < 0 || eids[i] >= g->E) return -1;
  int nth = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel num_threads(nth)
  {
    int64_t* stamp = (int64_t*)malloc(((size_t)g->N + 1) * 8);
    for (int32_t u = 0; u < g->N; ++u) stamp[u] = -1;
    int64_t qid = 0; /* fresh stamp for every window scanned by this thread */
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) {
      int64_t e = eids[i];
      for (int c = 0; c < ncols; ++c) {
        uint64_t v = 0;
        if (g->pos_out[e] >= 0) {
          int64_t delta = cols[c].delta;
          switch (cols[c].kind) {
            case OG_DEG_OUT: v = deg(g, e, 1, delta); break;
            case OG_DEG_IN: v = deg(g, e, 0, delta); break;
            case OG_FAN_OUT: v = fan_stamp(g, e, 1, delta, stamp, ++qid); break;
            case OG_FAN_IN: v = fan_stamp(g, e, 0, delta, stamp, ++qid); break;
            case OG_GS: v = ec_gs(g, e, delta); break;
            case OG_SG: v = ec_sg(g, e, delta); break;
            case OG_CYC: v = ec_cyc(g, e, cols[c].k, delta, 0); break;
            case OG_CYCW: v = ec_cyc(g, e, cols[c].k, delta, 1); break;
          }
        }
        out[(size_t)i * (size_t)ncols + (size_t)c] = saturate(v, limit);
      }
    }
    free(stamp);
  }
  return 0;
}

/* ---------------- stage programs: the nested loop of Alg. 1, stage by stage ----------------
 * Every stage walks its operand's neighbour list from the start of its time
 * range to the end of it (the trailing window, or the span so far widened by
 * delta) and tests each condition as the definition in aml_oracle.h states
 * it; the span is tested again on the completed binding. */

#define OG_MAXST 16
#define OG_MAXVAR (OG_MAXST + 1)

typedef struct {
  const og_graph* g;
  const og_stage* st;
  int n;
  int agg;
  int64_t delta;
  int64_t e0;
  int32_t node[OG_MAXVAR];
  int64_t reach[OG_MAXVAR];
  int64_t edges[2 * OG_MAXST]; /* e0, then each stage's edge(s) in stage order */
  int span[2 * OG_MAXST];      /* the edge takes part in the span test */
  int nedges;
  uint64_t nbind;              /* EDGES */
  int32_t* seen;               /* DISTINCT: last-stage nodes met so far */
  int64_t nseen, capseen;
  uint64_t* acc;               /* INSTANCES: this thread's credits, E entries */
  int64_t* sets;               /* SETS: this thread's instances, each its    */
  int64_t nsets, capsets;      /* edge ids sorted, nedges entries apiece      */
} pg_ctx;

/* the list of node u in direction dir, and the node at the far end of edge f */
static void pg_list(const og_graph* g, int32_t u, int dir, const int64_t** list, int64_t* lo,
                    int64_t* hi) {
  const int64_t* start = dir == OG_DIR_OUT ? g->out_start : g->in_start;
  *list = dir == OG_DIR_OUT ? g->out_list : g->in_list;
  *lo = start[u];
  *hi = start[u + 1];
}

static int32_t pg_far(const og_graph* g, int64_t f, int dir) {
  return dir == OG_DIR_OUT ? g->dst[f] : g->src[f];
}

static int pg_trailing_ok(const pg_ctx* c, int64_t f) {
  const og_graph* g = c->g;
  return (int64_t)g->ts[f] >= (int64_t)g->ts[c->e0] - c->delta && (f == c->e0 || prec(g, f, c->e0));
}

/* all conditions of the completed binding that involve more than one stage:
 * the span set and, for instances, pairwise distinct edges */
static void pg_complete(pg_ctx* c, int32_t x_last) {
  const og_graph* g = c->g;
  int64_t tmin = INT64_MAX, tmax = INT64_MIN;
  for (int i = 0; i < c->nedges; ++i) {
    if (!c->span[i]) continue;
    int64_t t = g->ts[c->edges[i]];
    if (t < tmin) tmin = t;
    if (t > tmax) tmax = t;
  }
  if (tmax - tmin > c->delta) return;
  if (c->agg == OG_AGG_EDGES) {
    c->nbind++;
  } else if (c->agg == OG_AGG_DISTINCT) {
    for (int64_t i = 0; i < c->nseen; ++i)
      if (c->seen[i] == x_last) return;
    if (c->nseen == c->capseen) {
      c->capseen = c->capseen ? 2 * c->capseen : 64;
      c->seen = (int32_t*)realloc(c->seen, (size_t)c->capseen * 4);
    }
    c->seen[c->nseen++] = x_last;
  } else {
    for (int i = 0; i < c->nedges; ++i)
      for (int j = i + 1; j < c->nedges; ++j)
        if (c->edges[i] == c->edges[j]) return;
    if (c->agg == OG_AGG_INSTANCES) {
      for (int i = 0; i < c->nedges; ++i) c->acc[c->edges[i]]++;
      return;
    }
    /* SETS: keep the instance's edge set (sorted ids); duplicates found
     * from other triggers or in other orders are removed at the end */
    if (c->nsets == c->capsets) {
      c->capsets = c->capsets ? 2 * c->capsets : 64;
      c->sets = (int64_t*)realloc(c->sets, (size_t)c->capsets * c->nedges * 8);
    }
    int64_t* r = c->sets + c->nsets * c->nedges;
    for (int i = 0; i < c->nedges; ++i) {
      int j = i;
      for (; j > 0 && r[j - 1] > c->edges[i]; --j) r[j] = r[j - 1];
      r[j] = c->edges[i];
    }
    c->nsets++;
  }
}

/* lexicographic order of two edge sets of *width ids */
static int pg_cmp_set(const void* a, const void* b, void* width) {
  const int64_t* x = (const int64_t*)a;
  const int64_t* y = (const int64_t*)b;
  for (int i = 0; i < *(const int*)width; ++i)
    if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
  return 0;
}

/* node x passes the stage's out_var and skip_eq conditions */
static int pg_node_ok(const pg_ctx* c, const og_stage* s, int32_t x, int bound) {
  for (int i = 0; i < bound; ++i)
    if (((s->skip_eq >> i) & 1u) && c->node[i] == x) return 0;
  if (s->out_var < bound && c->node[s->out_var] != x) return 0;
  return 1;
}

static void pg_stage(pg_ctx* c, int si, int bound);

/* the stage's amount constraints on edge f, whose predecessor on the walk is p */
static int pg_amount_ok(const pg_ctx* c, const og_stage* s, int64_t f, int64_t p) {
  const double a = c->g->amount[f];
  if ((s->amount_flags & OG_AMT_RANGE) && !(a >= s->amount_min && a <= s->amount_max)) return 0;
  if (s->amount_flags & OG_AMT_RATIO) {
    const double b = c->g->amount[p];
    if (!(a >= (double)s->ratio_min * b && a <= (double)s->ratio_max * b)) return 0;
  }
  return 1;
}

static void pg_bind(pg_ctx* c, int si, int bound, int32_t x, int64_t reach_edge) {
  const og_stage* s = &c->st[si];
  int nb = bound;
  if (s->out_var == bound) {
    c->node[bound] = x;
    c->reach[bound] = reach_edge;
    nb = bound + 1;
  }
  if (si == c->n - 1) pg_complete(c, x);
  else pg_stage(c, si + 1, nb);
}

/* earliest and latest time of the span set bound so far */
static void pg_span(const pg_ctx* c, int64_t* tmin, int64_t* tmax) {
  *tmin = INT64_MAX;
  *tmax = INT64_MIN;
  for (int i = 0; i < c->nedges; ++i) {
    if (!c->span[i]) continue;
    int64_t t = c->g->ts[c->edges[i]];
    if (t < *tmin) *tmin = t;
    if (t > *tmax) *tmax = t;
  }
}

/* the times a stage's edge can have: the trailing window, or within delta
 * of every time in the span set; Alg. 1's loop starts at the first edge in
 * range (Find_Start) and breaks at the first one past it */
static void pg_range(const pg_ctx* c, int window, int64_t tmin, int64_t tmax, int64_t* tl,
                     int64_t* th) {
  if (window == OG_WIN_TRAILING) {
    *tl = (int64_t)c->g->ts[c->e0] - c->delta;
    *th = c->g->ts[c->e0];
  } else {
    *tl = tmax - c->delta;
    *th = tmin + c->delta;
  }
}

static void pg_stage(pg_ctx* c, int si, int bound) {
  const og_graph* g = c->g;
  const og_stage* s = &c->st[si];
  const int64_t* la;
  int64_t alo, ahi, tmin, tmax, tl, th;
  pg_list(g, c->node[s->a_var], s->a_dir, &la, &alo, &ahi);
  const int64_t ra = c->reach[s->a_var];
  const int sp = s->window == OG_WIN_SPAN;
  pg_span(c, &tmin, &tmax);
  pg_range(c, s->window, tmin, tmax, &tl, &th);
  for (int64_t i = find_start(g, la, alo, ahi, tl); i < ahi; ++i) {
    const int64_t fa = la[i];
    if ((int64_t)g->ts[fa] > th) break;
    const int32_t x = pg_far(g, fa, s->a_dir);
    if (!pg_node_ok(c, s, x, bound)) continue;
    if (s->window == OG_WIN_TRAILING && !pg_trailing_ok(c, fa)) continue;
    if (!pg_amount_ok(c, s, fa, ra)) continue;
    if (s->op == OG_OP_FOR_ALL) {
      if (s->order == OG_ORD_AFTER && !prec(g, ra, fa)) continue;
      if (s->order == OG_ORD_BEFORE && !prec(g, fa, ra)) continue;
      if (s->order == OG_ORD_AFTER_TRIGGER && !prec(g, c->e0, fa)) continue;
      c->edges[c->nedges] = fa;
      c->span[c->nedges] = sp;
      c->nedges++;
      pg_bind(c, si, bound, x, fa);
      c->nedges--;
    } else {
      const int64_t* lb;
      int64_t blo, bhi, btl, bth;
      pg_list(g, c->node[s->b_var], s->b_dir, &lb, &blo, &bhi);
      const int64_t ta = g->ts[fa];
      pg_range(c, s->window, sp && ta < tmin ? ta : tmin, sp && ta > tmax ? ta : tmax, &btl,
               &bth);
      for (int64_t j = find_start(g, lb, blo, bhi, btl); j < bhi; ++j) {
        const int64_t fb = lb[j];
        if ((int64_t)g->ts[fb] > bth) break;
        if (pg_far(g, fb, s->b_dir) != x) continue;
        if (!pg_amount_ok(c, s, fb, fa)) continue;
        if (s->window == OG_WIN_TRAILING && !pg_trailing_ok(c, fb)) continue;
        if (s->order == OG_ORD_AFTER && !(prec(g, ra, fa) && prec(g, fa, fb))) continue;
        if (s->order == OG_ORD_BEFORE && !(prec(g, fb, fa) && prec(g, fa, ra))) continue;
        if (s->order == OG_ORD_LEG && !prec(g, fa, fb)) continue;
        if (s->order == OG_ORD_AFTER_TRIGGER && !(prec(g, c->e0, fa) && prec(g, c->e0, fb)))
          continue;
        c->edges[c->nedges] = fa;
        c->span[c->nedges] = sp;
        c->edges[c->nedges + 1] = fb;
        c->span[c->nedges + 1] = sp;
        c->nedges += 2;
        pg_bind(c, si, bound, x, fb);
        c->nedges -= 2;
      }
    }
  }
}

static int pg_check(const og_stage* st, int32_t n, int32_t agg) {
  if (n < 1 || n > OG_MAXST || agg < OG_AGG_EDGES || agg > OG_AGG_SETS) return -1;
  if (st[0].op != OG_OP_TRIGGER || st[0].out_var != 1) return -1;
  for (int s = 0; s < n; ++s) {
    const uint32_t allowed = s == 0 ? OG_AMT_RANGE : (OG_AMT_RANGE | OG_AMT_RATIO);
    if (st[s].amount_flags & ~allowed) return -1;
    if ((st[s].amount_flags & OG_AMT_RANGE) && !(st[s].amount_min <= st[s].amount_max)) return -1;
    if ((st[s].amount_flags & OG_AMT_RATIO) && !(st[s].ratio_min <= st[s].ratio_max)) return -1;
  }
  int bound = 2;
  for (int s = 1; s < n; ++s) {
    const og_stage* x = &st[s];
    if (x->op != OG_OP_FOR_ALL && x->op != OG_OP_INTERSECT) return -1;
    if (x->a_var < 0 || x->a_var >= bound || (x->a_dir != OG_DIR_OUT && x->a_dir != OG_DIR_IN))
      return -1;
    if (x->op == OG_OP_INTERSECT &&
        (x->b_var < 0 || x->b_var >= bound || (x->b_dir != OG_DIR_OUT && x->b_dir != OG_DIR_IN)))
      return -1;
    if (x->order < OG_ORD_NONE || x->order > OG_ORD_AFTER_TRIGGER) return -1;
    if (x->op == OG_OP_FOR_ALL && x->order == OG_ORD_LEG) return -1;
    if (x->window != OG_WIN_TRAILING && x->window != OG_WIN_SPAN) return -1;
    if (bound < 32 && (x->skip_eq >> bound) != 0) return -1;
    if (x->out_var < 0 || x->out_var > bound) return -1;
    if (x->out_var == bound) ++bound;
    else if (s != n - 1) return -1;
  }
  return 0;
}

int og_program_count(const og_graph* g, const og_stage* st, int32_t n, int32_t agg,
                     int64_t delta, uint32_t* out, int32_t nthreads) {
  if (!g || !st || !out || delta < 0 || pg_check(st, n, agg)) return -1;
  const int64_t E = g->E;
  if (nthreads <= 0) nthreads = omp_get_max_threads();
  uint64_t* total = (uint64_t*)calloc((size_t)(E > 0 ? E : 1), 8);
  /* SETS: every thread's instances, gathered; every binding of a program
   * has the same number of edges: the trigger, one per FOR_ALL stage, two
   * per INTERSECT stage */
  int width = 1;
  for (int s = 1; s < n; ++s) width += st[s].op == OG_OP_INTERSECT ? 2 : 1;
  int64_t* all_sets = NULL;
  int64_t n_all = 0;
#pragma omp parallel num_threads(nthreads)
  {
    pg_ctx c;
    memset(&c, 0, sizeof(c));
    c.g = g;
    c.st = st;
    c.n = n;
    c.agg = agg;
    c.delta = delta;
    if (agg == OG_AGG_INSTANCES) c.acc = (uint64_t*)calloc((size_t)(E > 0 ? E : 1), 8);
#pragma omp for schedule(dynamic, 64)
    for (int64_t e0 = 0; e0 < E; ++e0) {
      if (g->src[e0] == g->dst[e0]) continue;
      if ((st[0].amount_flags & OG_AMT_RANGE) &&
          !(g->amount[e0] >= st[0].amount_min && g->amount[e0] <= st[0].amount_max))
        continue;  /* not a trigger */
      c.e0 = e0;
      c.node[0] = g->src[e0];
      c.node[1] = g->dst[e0];
      c.reach[0] = c.reach[1] = e0;
      c.edges[0] = e0;
      c.span[0] = 1;
      c.nedges = 1;
      c.nbind = 0;
      c.nseen = 0;
      if (n == 1) pg_complete(&c, c.node[1]);
      else pg_stage(&c, 1, 2);
      if (agg == OG_AGG_EDGES) total[e0] = c.nbind;
      else if (agg == OG_AGG_DISTINCT) total[e0] = (uint64_t)c.nseen;
    }
    if (agg == OG_AGG_INSTANCES) {
#pragma omp critical
      for (int64_t e = 0; e < E; ++e) total[e] += c.acc[e];
      free(c.acc);
    }
    if (agg == OG_AGG_SETS && c.nsets) {
#pragma omp critical
      {
        all_sets = (int64_t*)realloc(all_sets, (size_t)(n_all + c.nsets) * width * 8);
        memcpy(all_sets + n_all * width, c.sets, (size_t)c.nsets * width * 8);
        n_all += c.nsets;
      }
    }
    free(c.sets);
    free(c.seen);
  }
  if (agg == OG_AGG_SETS) {
    /* sort the sets, then credit each distinct one to its edges once */
    qsort_r(all_sets, (size_t)n_all, (size_t)width * 8, pg_cmp_set, &width);
    for (int64_t i = 0; i < n_all; ++i) {
      const int64_t* r = all_sets + i * width;
      if (i > 0 && pg_cmp_set(r - width, r, &width) == 0) continue;
      for (int k = 0; k < width; ++k) total[r[k]]++;
    }
    free(all_sets);
  }
  clamp_out(total, out, (size_t)E, 0xffffffffu);
  free(total);
  return 0;
}
