"""Stage programs that no pattern family matches, for the generic
interpretation of stage programs: (op, a_var, a_dir, b_var, b_dir, out_var,
order, window, skip_eq) tuples, stage 0 the trigger.  Test data only (the
values are the library's stage vocabulary)."""
OP_TRIGGER, OP_FOR_ALL, OP_INTERSECT = 0, 1, 2
OUT, IN = 0, 1
NONE, AFTER, BEFORE, LEG, AFTER_TRIGGER = 0, 1, 2, 3, 4
TRAILING, SPAN = 0, 1
EDGES, DISTINCT, INSTANCES = 0, 1, 2

T = (OP_TRIGGER, 0, OUT, -1, 0, 1, NONE, TRAILING, 0)


def mask(*vs):
    m = 0
    for v in vs:
        m |= 1 << v
    return m


def F(a, d, out, order, window, skip=0):
    return (OP_FOR_ALL, a, d, -1, 0, out, order, window, skip)


def X(a, ad, b, bd, out, order, window, skip=0):
    return (OP_INTERSECT, a, ad, b, bd, out, order, window, skip)


NOVEL = {
    # a temporal 3-hop path N0 -> N1 -> N2 -> N3, every hop later
    "path3": ([T, F(1, OUT, 2, AFTER, SPAN, mask(0)), F(2, OUT, 3, AFTER, SPAN, mask(0, 1))],
              INSTANCES),
    # funds into N0 within the span, in either time order
    "gs_any_order": ([T, F(0, IN, 2, NONE, SPAN, mask(1))], INSTANCES),
    # a common counterparty of N0 and N1
    "common_out": ([T, X(0, OUT, 1, OUT, 2, NONE, SPAN, mask(0, 1))], INSTANCES),
    # how many later edges continue the trigger
    "continuations": ([T, F(1, OUT, 2, AFTER, SPAN)], EDGES),
    # distinct senders into the trigger's later receivers, trailing window
    "distinct_2hop": ([T, F(1, OUT, 2, AFTER_TRIGGER, SPAN, mask(0)),
                       F(2, IN, 3, NONE, TRAILING)], DISTINCT),
    # an intersection that closes back into N0, earlier than the hop before it
    "closing_intersect_before": ([T, F(1, OUT, 2, AFTER, SPAN, mask(0)),
                                  X(2, OUT, 0, IN, 3, BEFORE, SPAN, mask(0, 1, 2))], INSTANCES),
    # a last stage that closes onto N1 from an in-list
    "closing_in": ([T, F(0, IN, 2, BEFORE, SPAN, mask(1)), F(2, IN, 1, NONE, TRAILING)],
                   INSTANCES),
    # N0 -> x -> N1 with the first leg before the second
    "leg_triangle": ([T, X(0, OUT, 1, IN, 2, LEG, SPAN, mask(0, 1))], INSTANCES),
    # contradictory constraints (after the trigger, yet not after it): all zero
    "empty_trailing_after": ([T, X(0, IN, 1, IN, 2, AFTER_TRIGGER, TRAILING, mask(0, 1))],
                             EDGES),
    # pairs of N0's out-edges within the span (the trigger paired with itself
    # repeats an edge and is no instance)
    "fan_pairs": ([T, F(0, OUT, 2, NONE, SPAN)], INSTANCES),
    # the trigger alone
    "trigger_only": ([T], INSTANCES),
    # common senders of N0 and N1 inside the trailing window (an intersection
    # without order: the interpreter walks the shorter side)
    "common_in_trailing": ([T, X(0, IN, 1, IN, 2, NONE, TRAILING, mask(0, 1))], EDGES),
    # after a later hop N1 -> N2, the distinct accounts that pay both N1 and N2
    "hop_then_common_payer": ([T, F(1, OUT, 2, AFTER, SPAN, mask(0)),
                               X(1, IN, 2, IN, 3, NONE, SPAN, mask(0, 1, 2))], DISTINCT),
}

RANGE, RATIO = 1, 2


def amt(stage, flags, lo=0.0, hi=0.0, rlo=0.0, rhi=0.0):
    """A stage tuple with amount constraints (flags, range, ratio)."""
    return tuple(stage[:9]) + (flags, lo, hi, rlo, rhi)


# programs with amount constraints; graphs for them carry amounts
AMOUNT_PROGRAMS = {
    # funds passed on within the span, keeping 85-100% of the amount
    "fee_forward": ([T, amt(F(1, OUT, 2, AFTER, SPAN, mask(0)), RATIO, rlo=0.85, rhi=1.0)],
                    INSTANCES),
    # trailing out-degree, counted for large triggers only
    "large_trigger_degree": ([amt(T, RANGE, 150.0, 1e9), F(0, OUT, 2, NONE, TRAILING)], EDGES),
    # scatter-gather whose legs pass the funds on (80-100%) and whose second
    # scatter is 0.5-2x the first
    "sg_fee": ([T, amt(F(1, OUT, 2, AFTER, SPAN, mask(0)), RATIO, rlo=0.8, rhi=1.0),
                amt(X(0, OUT, 2, IN, 3, LEG, SPAN, mask(1)), RATIO, rlo=0.5, rhi=2.0)],
               INSTANCES),
    # 3-cycles in time order, every hop 90-100% of the hop before, amounts
    # between 50 and 250
    "cycle_ratio": ([T, amt(F(1, OUT, 2, AFTER, SPAN, mask(0, 1)), RATIO | RANGE, 50.0, 250.0,
                            0.9, 1.0),
                     amt(F(2, OUT, 0, AFTER, SPAN), RATIO | RANGE, 50.0, 250.0, 0.9, 1.0)],
                    INSTANCES),
    # distinct counterparties of an intersection whose edges both lie in a range
    "distinct_range": ([T, amt(X(0, OUT, 1, IN, 2, NONE, SPAN, mask(0, 1)), RANGE, 80.0, 120.0)],
                       DISTINCT),
}

# amounts drawn for the graphs of AMOUNT_PROGRAMS: ratio bounds fall on
# exact pairs (85/100, 90/100, 80/100)
AMOUNT_VALUES = (50.0, 80.0, 85.0, 90.0, 95.0, 100.0, 120.0, 150.0, 180.0, 200.0)
