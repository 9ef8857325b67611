"""Stage programs for the built-in pattern families (multi-stage framework).

Each builder returns a ``Pattern``: a list of stages in the paper's
multi-stage form (Sec. 5, Fig. 4; per-stage configuration of Alg. 1:
operation, operand node sets, output variable, skip_if / time constraints)
plus the final aggregation and the window.  ``aml_pattern_set_create`` maps
each program onto the kernel family that evaluates it.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence

OP_TRIGGER, OP_FOR_ALL, OP_INTERSECT = 0, 1, 2
DIR_OUT, DIR_IN = 0, 1
ORDER_NONE, ORDER_AFTER, ORDER_BEFORE, ORDER_LEG, ORDER_AFTER_TRIGGER = 0, 1, 2, 3, 4
WIN_TRAILING, WIN_SPAN = 0, 1
AGG_EDGES, AGG_DISTINCT, AGG_INSTANCES, AGG_SETS = 0, 1, 2, 3
AMT_RANGE, AMT_RATIO = 1, 2
FAM_NAMES = {0: "DEG_OUT", 1: "DEG_IN", 2: "FAN_OUT", 3: "FAN_IN", 4: "GS", 5: "SG", 6: "CYC",
             7: "CYCW", 8: "PROGRAM"}

DAY = 86400
WEEK = 7 * DAY


@dataclasses.dataclass(frozen=True)
class Stage:
    op: int
    a_var: int = 0
    a_dir: int = DIR_OUT
    b_var: int = -1
    b_dir: int = 0
    out_var: int = 0
    order: int = ORDER_NONE
    window: int = WIN_TRAILING
    skip_eq: int = 0
    # amount constraints on the stage's edges (AMT_RANGE, AMT_RATIO)
    amount_flags: int = 0
    amount_min: float = 0.0
    amount_max: float = 0.0
    ratio_min: float = 0.0
    ratio_max: float = 0.0


@dataclasses.dataclass(frozen=True)
class Pattern:
    stages: tuple
    aggregate: int
    delta: int
    name: str = ""
    # run through the generic interpreter even when a family matches (a
    # program no family matches is interpreted anyway)
    interpret: bool = False


def program(stages, aggregate: int, delta: int, name: str = "",
            interpret: bool = False) -> Pattern:
    """A pattern from (op, a_var, a_dir, b_var, b_dir, out_var, order, window,
    skip_eq[, amount_flags, amount_min, amount_max, ratio_min, ratio_max])
    tuples or Stage objects, stage 0 the trigger."""
    def stage(v):
        v = tuple(v)
        return Stage(*[int(x) for x in v[:10]], *[float(x) for x in v[10:]])
    st = tuple(s if isinstance(s, Stage) else stage(s) for s in stages)
    return Pattern(st, int(aggregate), int(delta), name, interpret)


def interpreted(p: Pattern) -> Pattern:
    """The same program, forced through the generic interpreter."""
    return dataclasses.replace(p, interpret=True)


def _skip(*vars_: int) -> int:
    m = 0
    for v in vars_:
        m |= 1 << v
    return m


TRIGGER = Stage(OP_TRIGGER, 0, DIR_OUT, -1, 0, 1)


def deg_out(delta: int) -> Pattern:
    """Edges out of N0 in the trailing window of the trigger."""
    return Pattern((TRIGGER, Stage(OP_FOR_ALL, 0, DIR_OUT, out_var=2, window=WIN_TRAILING)),
                   AGG_EDGES, delta, f"DEG_OUT@{delta}")


def deg_in(delta: int) -> Pattern:
    return Pattern((TRIGGER, Stage(OP_FOR_ALL, 1, DIR_IN, out_var=2, window=WIN_TRAILING)),
                   AGG_EDGES, delta, f"DEG_IN@{delta}")


def fan_out(delta: int) -> Pattern:
    """Distinct counterparties N0 paid in the trailing window (fan-out)."""
    return Pattern((TRIGGER, Stage(OP_FOR_ALL, 0, DIR_OUT, out_var=2, window=WIN_TRAILING)),
                   AGG_DISTINCT, delta, f"FAN_OUT@{delta}")


def fan_in(delta: int) -> Pattern:
    return Pattern((TRIGGER, Stage(OP_FOR_ALL, 1, DIR_IN, out_var=2, window=WIN_TRAILING)),
                   AGG_DISTINCT, delta, f"FAN_IN@{delta}")


def gather_scatter(delta: int, mirrored: bool = False) -> Pattern:
    """N0 -> N1 -> N2 with the second edge later, N2 != N0 (funds passing a hub)."""
    if mirrored:
        s = Stage(OP_FOR_ALL, 0, DIR_IN, out_var=2, order=ORDER_BEFORE, window=WIN_SPAN,
                  skip_eq=_skip(1))
    else:
        s = Stage(OP_FOR_ALL, 1, DIR_OUT, out_var=2, order=ORDER_AFTER, window=WIN_SPAN,
                  skip_eq=_skip(0))
    return Pattern((TRIGGER, s), AGG_INSTANCES, delta, f"GS@{delta}")


def scatter_gather(delta: int, trigger: str = "scatter") -> Pattern:
    """Sec. 5's scatter-gather: trigger N0 -> N1, expand N1.out -> N2, then
    intersect N0.out with N2.in -> N3 (another intermediary)."""
    if trigger == "scatter":
        stages = (TRIGGER,
                  Stage(OP_FOR_ALL, 1, DIR_OUT, out_var=2, order=ORDER_AFTER, window=WIN_SPAN,
                        skip_eq=_skip(0)),
                  Stage(OP_INTERSECT, 0, DIR_OUT, 2, DIR_IN, out_var=3, order=ORDER_LEG,
                        window=WIN_SPAN, skip_eq=_skip(1)))
    elif trigger == "gather":
        # the same diamond reached from a gather edge (Sec. 6's description)
        stages = (TRIGGER,
                  Stage(OP_FOR_ALL, 0, DIR_IN, out_var=2, order=ORDER_BEFORE, window=WIN_SPAN,
                        skip_eq=_skip(1)),
                  Stage(OP_INTERSECT, 2, DIR_OUT, 1, DIR_IN, out_var=3, order=ORDER_LEG,
                        window=WIN_SPAN, skip_eq=_skip(0)))
    else:
        raise ValueError(trigger)
    return Pattern(stages, AGG_INSTANCES, delta, f"SG@{delta}")


def scatter_gather_n(n: int, delta: int) -> Pattern:
    """Sec. 4's "at least N" placement accounts: a scatter-gather with n
    intermediaries, n >= 2.  Trigger N0 -> N1 (s -> m1), N1.out -> N2 (the
    destination d, later), then n - 1 intersections of N0.out with N2.in,
    each a further intermediary distinct from the ones before, its two edges
    in order; all 2n edges within delta.  Run by the generic interpreter: an
    edge's count is the number of ordered n-tuples of such legs it belongs
    to, n! * C(k - 1, n - 1) on each edge of an isolated k-intermediary
    scatter-gather, so it is nonzero exactly when the edge takes part in a
    scatter-gather with at least n intermediaries."""
    if not 2 <= n <= 7:
        raise ValueError("n must be in [2, 7] (the interpreter runs at most 8 stages)")
    stages = [TRIGGER, Stage(OP_FOR_ALL, 1, DIR_OUT, out_var=2, order=ORDER_AFTER,
                             window=WIN_SPAN, skip_eq=_skip(0))]
    for i in range(n - 1):
        stages.append(Stage(OP_INTERSECT, 0, DIR_OUT, 2, DIR_IN, out_var=3 + i,
                            order=ORDER_LEG, window=WIN_SPAN,
                            skip_eq=_skip(1, *range(3, 3 + i))))
    return Pattern(tuple(stages), AGG_INSTANCES, delta, f"SG{n}@{delta}", interpret=True)


def scatter_gather_exact(n: int, delta: int, interpret: bool = False) -> Pattern:
    """Exact-size scatter-gather bins: the scatter-gather program of n
    intermediaries with the SETS aggregate, which counts every set of n legs
    (one source, one destination, pairwise distinct intermediaries, each leg
    in order, all 2n edges within delta) once on each of its 2n edges.
    n = 2 is the SG column (mined by the SG family unless ``interpret``);
    larger n run through the interpreter, whose ordered count holds every
    set n! times and is divided by it."""
    p = scatter_gather_n(n, delta)
    return Pattern(p.stages, AGG_SETS, delta, f"SG{n}_EXACT@{delta}", interpret=interpret)


def gather_scatter_n(n_in: int, n_out: int, delta: int) -> Pattern:
    """Gather-scatter through a hub with at least n_in senders and n_out
    receivers: the trigger x1 -> h is the latest gather edge, n_in - 1 earlier
    gathers from further distinct senders, then n_out scatters after the
    trigger to distinct receivers that are not senders; all edges within
    delta.  Run by the generic interpreter: an edge's count is the number of
    such bindings (ordered tuples) it belongs to, nonzero exactly when it
    takes part in a gather-scatter of at least that size.  (1, 1) is the GS
    program itself."""
    if n_in < 1 or n_out < 1 or n_in + n_out > 8:
        raise ValueError("need n_in, n_out >= 1 and n_in + n_out <= 8 (at most 8 stages)")
    stages = [TRIGGER]
    senders = [0]
    for i in range(n_in - 1):  # earlier gathers: new variables 2, 3, ...
        v = 2 + i
        stages.append(Stage(OP_FOR_ALL, 1, DIR_IN, out_var=v, order=ORDER_BEFORE,
                            window=WIN_SPAN, skip_eq=_skip(*senders)))
        senders.append(v)
    receivers = []
    for i in range(n_out):
        v = 1 + n_in + i
        stages.append(Stage(OP_FOR_ALL, 1, DIR_OUT, out_var=v, order=ORDER_AFTER,
                            window=WIN_SPAN, skip_eq=_skip(*senders, *receivers)))
        receivers.append(v)
    return Pattern(tuple(stages), AGG_INSTANCES, delta, f"GS{n_in}x{n_out}@{delta}",
                   interpret=True)


def scatter_gather_nodes(delta: int) -> Pattern:
    """The node-level scatter-gather: for each scatter edge s -> m1 (the
    trigger), the number of distinct other intermediaries m2 that complete a
    scatter-gather s -> m1 -> d, s -> m2 -> d with it (any d, each leg in
    order, all four edges within delta): Sec. 5's scatter-gather program
    with the DISTINCT aggregate over its last node, run by the generic
    interpreter.  k - 1 on each scatter edge of an isolated k-intermediary
    scatter-gather, 0 on its gather edges; parallel legs through the same
    intermediary count once."""
    p = scatter_gather(delta)
    return Pattern(p.stages, AGG_DISTINCT, delta, f"SG_NODES@{delta}", interpret=True)


def stack(delta: int) -> Pattern:
    """The "Stack" pattern (benchmarked in Sec. 8, Fig. 9, never defined in
    the text), read as the stacked bipartite of the laundering-pattern
    catalogue that the paper's Fig. 2 draws on: two senders s1, s2 that each
    pay both of two middle accounts m1, m2 (a complete first layer), and
    m1, m2 that each pay both of two receivers r1, r2 (a complete second
    layer); six distinct accounts, eight transfers, all within delta (no
    order inside the instance beyond the window).  The program: trigger
    s1 -> m1, s1's out-edge to m2, s2 from m1.in intersected with m2.in, then
    r1 and r2 from m1.out intersected with m2.out.  With the SETS aggregate
    each instance (its set of eight edges) counts once on each of its edges.
    Every instance is found by 8 bindings (any of its 4 first-layer edges as
    trigger, times the 2 orders of r1, r2), so the interpreter's per-binding
    count is divided by 8."""
    O, I, X, F, SP = DIR_OUT, DIR_IN, OP_INTERSECT, OP_FOR_ALL, WIN_SPAN
    stages = (TRIGGER,
              Stage(F, 0, O, out_var=2, window=SP, skip_eq=_skip(0, 1)),
              Stage(X, 1, I, 2, I, out_var=3, window=SP, skip_eq=_skip(0, 1, 2)),
              Stage(X, 1, O, 2, O, out_var=4, window=SP, skip_eq=_skip(0, 1, 2, 3)),
              Stage(X, 1, O, 2, O, out_var=5, window=SP, skip_eq=_skip(0, 1, 2, 3, 4)))
    return Pattern(stages, AGG_SETS, delta, f"STACK@{delta}", interpret=True)


def cycle(k: int, delta: int, closing: str = "for_all") -> Pattern:
    """k-cycle: trigger N0 -> N1, then N_i.out -> N_{i+1} (later, new node),
    closed by an edge back into N0 -- or, for k >= 3, by intersecting
    N_{k-2}.out with N0.in as in Sec. 5/6's 4-cycle."""
    if k < 2:
        raise ValueError("k >= 2")
    st: List[Stage] = [TRIGGER]
    if closing == "for_all":
        for i in range(1, k - 1):
            st.append(Stage(OP_FOR_ALL, i, DIR_OUT, out_var=i + 1, order=ORDER_AFTER,
                            window=WIN_SPAN, skip_eq=_skip(*range(i + 1))))
        st.append(Stage(OP_FOR_ALL, k - 1, DIR_OUT, out_var=0, order=ORDER_AFTER,
                        window=WIN_SPAN))
    elif closing == "intersect":
        if k < 3:
            raise ValueError("intersection closing needs k >= 3")
        for i in range(1, k - 2):
            st.append(Stage(OP_FOR_ALL, i, DIR_OUT, out_var=i + 1, order=ORDER_AFTER,
                            window=WIN_SPAN, skip_eq=_skip(*range(i + 1))))
        st.append(Stage(OP_INTERSECT, k - 2, DIR_OUT, 0, DIR_IN, out_var=k - 1,
                        order=ORDER_AFTER, window=WIN_SPAN, skip_eq=_skip(*range(k - 1))))
    else:
        raise ValueError(closing)
    return Pattern(tuple(st), AGG_INSTANCES, delta, f"CYC{k}@{delta}")


def window_cycle(k: int, delta: int) -> Pattern:
    """Window k-cycle (Sec. 4's cycles with anticipatory edges): trigger
    N0 -> N1, then N_i.out -> N_{i+1} to a new node with every hop only after
    the trigger edge (the hops among themselves in any order), closed by an
    edge back into N0, all within delta."""
    if k < 2:
        raise ValueError("k >= 2")
    st: List[Stage] = [TRIGGER]
    for i in range(1, k - 1):
        st.append(Stage(OP_FOR_ALL, i, DIR_OUT, out_var=i + 1, order=ORDER_AFTER_TRIGGER,
                        window=WIN_SPAN, skip_eq=_skip(*range(i + 1))))
    st.append(Stage(OP_FOR_ALL, k - 1, DIR_OUT, out_var=0, order=ORDER_AFTER_TRIGGER,
                    window=WIN_SPAN))
    return Pattern(tuple(st), AGG_INSTANCES, delta, f"CYC{k}@{delta}" if k == 2
                   else f"CYCW{k}@{delta}")


def standard(delta: int, kmax: int = 5) -> List[Pattern]:
    """The ten per-window columns: DEG_OUT, DEG_IN, FAN_OUT, FAN_IN, GS, SG,
    CYC_2..CYC_kmax."""
    return ([deg_out(delta), deg_in(delta), fan_out(delta), fan_in(delta),
             gather_scatter(delta), scatter_gather(delta)]
            + [cycle(k, delta) for k in range(2, kmax + 1)])


def workload_patterns(name: str) -> List[Pattern]:
    """Column sets of the named workloads."""
    if name == "tiny-10k":
        return standard(DAY, 5)
    if name in ("hi-small", "hi-medium"):
        return standard(DAY, 5) + standard(WEEK, 5)
    if name == "hi-large":
        return ([fan_out(DAY), fan_in(DAY), gather_scatter(DAY), scatter_gather(DAY)]
                + [cycle(k, DAY) for k in range(3, 7)] + [fan_out(WEEK), fan_in(WEEK)])
    raise KeyError(name)
