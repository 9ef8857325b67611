// Stage-program validation and planning (host only).
//
// A pattern is a chain of stages (Sec. 5); each stage applies an operation
// (for_all, intersection) to neighbour sets of node variables bound by
// earlier stages, with skip_if (node inequality) and time constraints
// (Alg. 1's per-stage configuration).  The planner first validates operand
// dependencies (Sec. 6), then maps the program onto one of the families the
// kernels implement by comparing it, stage by stage, with that family's
// canonical programs; a valid program that matches none is run by the
// generic interpreter (program.cu) exactly as its stages say.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "aml_internal.cuh"

namespace aml {

namespace {

aml_stage st(int op, int a_var, int a_dir, int b_var, int b_dir, int out_var, int order,
             int window, uint32_t skip) {
  aml_stage s;
  std::memset(&s, 0, sizeof(s));  // no amount constraints
  s.op = op; s.a_var = a_var; s.a_dir = a_dir; s.b_var = b_var; s.b_dir = b_dir;
  s.out_var = out_var; s.order = order; s.window = window; s.skip_eq = skip;
  return s;
}

aml_stage trigger() { return st(AML_OP_TRIGGER, 0, AML_DIR_OUT, -1, 0, 1, 0, 0, 0); }

uint32_t bits_upto(int n) { return n >= 32 ? 0xffffffffu : ((1u << (n + 1)) - 1u); }

struct Template {
  int family;
  int k;
  int aggregate;
  std::vector<aml_stage> stages;
};

std::vector<Template> templates() {
  std::vector<Template> t;
  const int O = AML_DIR_OUT, I = AML_DIR_IN;
  const int F = AML_OP_FOR_ALL, X = AML_OP_INTERSECT;
  const int TR = AML_WIN_TRAILING, SP = AML_WIN_SPAN;
  // windowed degree / fan: the trigger's own neighbourhood over the trailing window
  t.push_back({AML_FAM_DEG_OUT, 0, AML_AGG_EDGES, {trigger(), st(F, 0, O, -1, 0, 2, 0, TR, 0)}});
  t.push_back({AML_FAM_FAN_OUT, 0, AML_AGG_DISTINCT, {trigger(), st(F, 0, O, -1, 0, 2, 0, TR, 0)}});
  t.push_back({AML_FAM_DEG_IN, 0, AML_AGG_EDGES, {trigger(), st(F, 1, I, -1, 0, 2, 0, TR, 0)}});
  t.push_back({AML_FAM_FAN_IN, 0, AML_AGG_DISTINCT, {trigger(), st(F, 1, I, -1, 0, 2, 0, TR, 0)}});
  // gather-scatter: N0 -> N1 -> N2 (later), N2 != N0; or the mirrored N2 -> N0 -> N1
  t.push_back({AML_FAM_GS, 0, AML_AGG_INSTANCES,
               {trigger(), st(F, 1, O, -1, 0, 2, AML_ORDER_AFTER, SP, 1u << 0)}});
  t.push_back({AML_FAM_GS, 0, AML_AGG_INSTANCES,
               {trigger(), st(F, 0, I, -1, 0, 2, AML_ORDER_BEFORE, SP, 1u << 1)}});
  // scatter-gather, trigger = scatter edge: N1.out -> N2, then N0.out ∩ N2.in -> N3
  t.push_back({AML_FAM_SG, 0, AML_AGG_INSTANCES,
               {trigger(), st(F, 1, O, -1, 0, 2, AML_ORDER_AFTER, SP, 1u << 0),
                st(X, 0, O, 2, I, 3, AML_ORDER_LEG, SP, 1u << 1)}});
  // scatter-gather, trigger = gather edge: N0.in -> N2, then N2.out ∩ N1.in -> N3
  t.push_back({AML_FAM_SG, 0, AML_AGG_INSTANCES,
               {trigger(), st(F, 0, I, -1, 0, 2, AML_ORDER_BEFORE, SP, 1u << 1),
                st(X, 2, O, 1, I, 3, AML_ORDER_LEG, SP, 1u << 0)}});
  // k-cycles: chain of for_all over out-neighbours, each later than the last,
  // skipping bound nodes, closed by an edge back into N0 ...
  for (int k = 2; k <= 15; ++k) {
    Template c{AML_FAM_CYC, k, AML_AGG_INSTANCES, {trigger()}};
    for (int i = 1; i <= k - 2; ++i)
      c.stages.push_back(st(F, i, O, -1, 0, i + 1, AML_ORDER_AFTER, SP, bits_upto(i)));
    c.stages.push_back(st(F, k - 1, O, -1, 0, 0, AML_ORDER_AFTER, SP, 0));
    t.push_back(c);
    // ... or, as in Sec. 6's 4-cycle, by intersecting N(k-2).out with N0.in
    if (k >= 3) {
      Template d{AML_FAM_CYC, k, AML_AGG_INSTANCES, {trigger()}};
      for (int i = 1; i <= k - 3; ++i)
        d.stages.push_back(st(F, i, O, -1, 0, i + 1, AML_ORDER_AFTER, SP, bits_upto(i)));
      d.stages.push_back(st(X, k - 2, O, 0, I, k - 1, AML_ORDER_AFTER, SP, bits_upto(k - 2)));
      t.push_back(d);
    }
    // window cycles: every hop only after the trigger edge (the cycle's
    // earliest edge), the hops among themselves in any order; for k = 2 the
    // one hop is the same as an ordered one
    Template w{k == 2 ? AML_FAM_CYC : AML_FAM_CYCW, k, AML_AGG_INSTANCES, {trigger()}};
    for (int i = 1; i <= k - 2; ++i)
      w.stages.push_back(st(F, i, O, -1, 0, i + 1, AML_ORDER_AFTER_TRIGGER, SP, bits_upto(i)));
    w.stages.push_back(st(F, k - 1, O, -1, 0, 0, AML_ORDER_AFTER_TRIGGER, SP, 0));
    t.push_back(w);
  }
  return t;
}

// The scatter-gather of n intermediaries with the scatter edge as trigger:
// N1.out -> N2 (the destination, after the trigger), then n - 1
// intersections N0.out with N2.in, each a further intermediary skipping N1
// and the intersections' intermediaries before it, each leg in order.
std::vector<aml_stage> scatter_gather_n(int n) {
  const int O = AML_DIR_OUT, I = AML_DIR_IN, SP = AML_WIN_SPAN;
  std::vector<aml_stage> v{trigger(),
                           st(AML_OP_FOR_ALL, 1, O, -1, 0, 2, AML_ORDER_AFTER, SP, 1u << 0)};
  for (int i = 0; i < n - 1; ++i) {
    uint32_t skip = 1u << 1;
    for (int j = 0; j < i; ++j) skip |= 1u << (3 + j);
    v.push_back(st(AML_OP_INTERSECT, 0, O, 2, I, 3 + i, AML_ORDER_LEG, SP, skip));
  }
  return v;
}

// The stacked bipartite ("Stack"): trigger s1 -> m1, s1.out -> m2, then
// s2 from m1.in intersected with m2.in, r1 and r2 from m1.out intersected
// with m2.out, each new account skipping the ones bound before it, every
// stage in the span window, no order.
std::vector<aml_stage> stack_stages() {
  const int O = AML_DIR_OUT, I = AML_DIR_IN, SP = AML_WIN_SPAN;
  const int F = AML_OP_FOR_ALL, X = AML_OP_INTERSECT;
  return {trigger(), st(F, 0, O, -1, 0, 2, AML_ORDER_NONE, SP, bits_upto(1)),
          st(X, 1, I, 2, I, 3, AML_ORDER_NONE, SP, bits_upto(2)),
          st(X, 1, O, 2, O, 4, AML_ORDER_NONE, SP, bits_upto(3)),
          st(X, 1, O, 2, O, 5, AML_ORDER_NONE, SP, bits_upto(4))};
}

bool same_stage(const aml_stage& a, const aml_stage& b) {
  if (a.op != b.op || a.out_var != b.out_var) return false;
  if (a.amount_flags != b.amount_flags) return false;  // families have no amount constraints
  if (a.op == AML_OP_TRIGGER) return true;
  if (a.a_var != b.a_var || a.a_dir != b.a_dir || a.order != b.order || a.window != b.window ||
      a.skip_eq != b.skip_eq)
    return false;
  if (a.op == AML_OP_INTERSECT && (a.b_var != b.b_var || a.b_dir != b.b_dir)) return false;
  return true;
}

std::string where(int p, int s) {
  char buf[64];
  std::snprintf(buf, sizeof(buf), "pattern %d, stage %d: ", p, s);
  return buf;
}

void validate(const aml_pattern& pat, int p) {
  AML_REQUIRE(pat.stages != nullptr && pat.n_stages >= 1 && pat.n_stages <= 32, AML_EINVAL,
              where(p, 0) + "a pattern needs 1..32 stages");
  AML_REQUIRE(pat.delta >= 0, AML_EINVAL, where(p, 0) + "delta must be >= 0");
  AML_REQUIRE((pat.flags & ~AML_PAT_INTERPRET) == 0, AML_EINVAL,
              where(p, 0) + "unknown pattern flag bits");
  AML_REQUIRE(pat.aggregate >= AML_AGG_EDGES && pat.aggregate <= AML_AGG_SETS, AML_EINVAL,
              where(p, 0) + "unknown aggregate");
  const aml_stage& t = pat.stages[0];
  AML_REQUIRE(t.op == AML_OP_TRIGGER && t.out_var == 1, AML_EINVAL,
              where(p, 0) + "stage 0 must be the trigger binding N0 -> N1");
  for (int s = 0; s < pat.n_stages; ++s) {
    const aml_stage& x = pat.stages[s];
    const uint32_t allowed = s == 0 ? AML_AMT_RANGE : (AML_AMT_RANGE | AML_AMT_RATIO);
    AML_REQUIRE((x.amount_flags & ~allowed) == 0, AML_EINVAL,
                where(p, s) + "bad amount flags (the trigger takes AML_AMT_RANGE only)");
    AML_REQUIRE(!(x.amount_flags & AML_AMT_RANGE) || x.amount_min <= x.amount_max, AML_EINVAL,
                where(p, s) + "amount range needs amount_min <= amount_max (no NaN)");
    AML_REQUIRE(!(x.amount_flags & AML_AMT_RATIO) || x.ratio_min <= x.ratio_max, AML_EINVAL,
                where(p, s) + "ratio range needs ratio_min <= ratio_max (no NaN)");
  }
  int bound = 2;  // N0, N1
  for (int s = 1; s < pat.n_stages; ++s) {
    const aml_stage& x = pat.stages[s];
    AML_REQUIRE(x.op == AML_OP_FOR_ALL || x.op == AML_OP_INTERSECT, AML_EINVAL,
                where(p, s) + "op must be FOR_ALL or INTERSECT after the trigger");
    AML_REQUIRE(x.a_var >= 0 && x.a_var < bound, AML_EINVAL,
                where(p, s) + "first operand is not bound by an earlier stage");
    AML_REQUIRE(x.a_dir == AML_DIR_OUT || x.a_dir == AML_DIR_IN, AML_EINVAL,
                where(p, s) + "bad neighbour direction");
    if (x.op == AML_OP_INTERSECT) {
      AML_REQUIRE(x.b_var >= 0 && x.b_var < bound, AML_EINVAL,
                  where(p, s) + "second operand is not bound by an earlier stage");
      AML_REQUIRE(x.b_dir == AML_DIR_OUT || x.b_dir == AML_DIR_IN, AML_EINVAL,
                  where(p, s) + "bad neighbour direction");
    }
    AML_REQUIRE(x.order >= AML_ORDER_NONE && x.order <= AML_ORDER_AFTER_TRIGGER, AML_EINVAL,
                where(p, s) + "bad order");
    AML_REQUIRE(x.window == AML_WIN_TRAILING || x.window == AML_WIN_SPAN, AML_EINVAL,
                where(p, s) + "bad window");
    AML_REQUIRE(bound >= 32 || (x.skip_eq >> bound) == 0, AML_EINVAL,
                where(p, s) + "skip mask names an unbound variable");
    AML_REQUIRE(x.out_var >= 0 && x.out_var <= bound, AML_EINVAL,
                where(p, s) + "output variable must be new (next index) or already bound");
    if (x.out_var == bound) {
      ++bound;
    } else {
      AML_REQUIRE(s == pat.n_stages - 1, AML_EINVAL,
                  where(p, s) + "only the last stage may close onto a bound variable");
    }
  }
}

}  // namespace

// The generic interpreter's form of a valid program, or a Failure naming
// why the interpreter cannot run it.
static Prog interpretable(const aml_pattern& pat, int p) {
  AML_REQUIRE(pat.n_stages <= PROG_MAX_STAGES, AML_EUNSUPPORTED,
              where(p, 0) + "no family matches and the interpreter runs at most 8 stages");
  Prog g;
  std::memset(&g, 0, sizeof(g));
  g.n = pat.n_stages;
  g.agg = pat.aggregate;
  g.delta = pat.delta;
  g.div = 1;
  for (int s = 0; s < pat.n_stages; ++s) {
    const aml_stage& x = pat.stages[s];
    AML_REQUIRE(!(x.op == AML_OP_FOR_ALL && x.order == AML_ORDER_LEG), AML_EUNSUPPORTED,
                where(p, s) + "LEG order is defined for INTERSECT stages only");
    ProgStage& q = g.st[s];
    q.op = (int8_t)x.op;
    q.a_var = (int8_t)x.a_var;
    q.a_dir = (int8_t)x.a_dir;
    q.b_var = (int8_t)(x.op == AML_OP_INTERSECT ? x.b_var : -1);
    q.b_dir = (int8_t)(x.op == AML_OP_INTERSECT ? x.b_dir : 0);
    q.out_var = (int8_t)x.out_var;
    q.order = (int8_t)x.order;
    q.window = (int8_t)x.window;
    q.skip = s == 0 ? 0u : x.skip_eq;
    q.amt = x.amount_flags;
    q.amin = x.amount_min;
    q.amax = x.amount_max;
    q.rmin = x.ratio_min;
    q.rmax = x.ratio_max;
  }
  return g;
}

// Maps every pattern onto a column (a family, else the interpreter); throws
// Failure on error.
std::vector<Column> plan_patterns(const aml_pattern* pats, int n, std::vector<Prog>* progs) {
  AML_REQUIRE(pats != nullptr && n >= 1, AML_EINVAL, "need at least one pattern");
  static const std::vector<Template> tpl = templates();
  std::vector<Column> cols;
  for (int p = 0; p < n; ++p) {
    validate(pats[p], p);
    const aml_pattern& pat = pats[p];
    if (pat.aggregate == AML_AGG_SETS) {
      // the stacked bipartite: every instance (eight edges) is found from
      // each of its four first-layer edges, with its two receivers in both
      // orders: 8 bindings that all credit its eight edges
      {
        const std::vector<aml_stage> t = stack_stages();
        bool is_stack = pat.n_stages == (int)t.size();
        for (int s = 0; s < pat.n_stages && is_stack; ++s) is_stack = same_stage(pat.stages[s], t[s]);
        if (is_stack) {
          Prog g = interpretable(pat, p);
          g.agg = AML_AGG_INSTANCES;
          g.div = 8;
          progs->push_back(g);
          cols.push_back(Column{AML_FAM_PROGRAM, 0, pat.delta, (int32_t)progs->size() - 1});
          continue;
        }
      }
      // the scatter-gather of n intermediaries: every set of n legs is found
      // from each of its n scatter edges with the other n - 1 legs in every
      // order of the intersections, n! bindings that all credit its 2n edges
      // (the distinct intermediaries make the legs of a set of edges unique)
      const int n_int = pat.n_stages - 1;
      bool ok = n_int >= 2 && n_int <= PROG_MAX_STAGES - 1;
      if (ok) {
        const std::vector<aml_stage> t = scatter_gather_n(n_int);
        for (int s = 0; s < pat.n_stages && ok; ++s) ok = same_stage(pat.stages[s], t[s]);
      }
      AML_REQUIRE(ok, AML_EUNSUPPORTED,
                  where(p, 0) + "AML_AGG_SETS is counted for the scatter-gather of n "
                                "intermediaries (2 <= n <= 7) and the stacked bipartite only");
      if (n_int == 2 && !(pat.flags & AML_PAT_INTERPRET)) {
        cols.push_back(Column{AML_FAM_SG, 0, pat.delta});  // a set of two legs: an SG pair
        continue;
      }
      Prog g = interpretable(pat, p);
      g.agg = AML_AGG_INSTANCES;
      for (int i = 2; i <= n_int; ++i) g.div *= i;
      progs->push_back(g);
      cols.push_back(Column{AML_FAM_PROGRAM, 0, pat.delta, (int32_t)progs->size() - 1});
      continue;
    }
    int fam = -1, k = 0;
    for (const Template& t : tpl) {
      if (pat.flags & AML_PAT_INTERPRET) break;
      if ((int)t.stages.size() != pat.n_stages || t.aggregate != pat.aggregate) continue;
      bool ok = true;
      for (int s = 0; s < pat.n_stages && ok; ++s) ok = same_stage(pat.stages[s], t.stages[s]);
      if (ok) {
        fam = t.family;
        k = t.k;
        break;
      }
    }
    if (fam < 0) {
      progs->push_back(interpretable(pat, p));
      cols.push_back(Column{AML_FAM_PROGRAM, 0, pat.delta, (int32_t)progs->size() - 1});
      continue;
    }
    cols.push_back(Column{fam, k, pat.delta});
  }
  return cols;
}

}  // namespace aml
