"""Column translation between the library's pattern builders and the oracle's
column tuples (test helper: the oracle parses column names itself and the
product package knows nothing of the oracle)."""
from __future__ import annotations

from typing import List, Sequence

import oracle
from paper_2604_12241_b300 import patterns as P


def oracle_columns(patterns: Sequence[P.Pattern]) -> list:
    """The oracle's column tuples for a list of built-in patterns."""
    return oracle.columns_from_names([p.name for p in patterns])


def from_oracle_columns(cols) -> List[P.Pattern]:
    """Built-in patterns for oracle column tuples (inverse of oracle_columns)."""
    make = {"deg_out": P.deg_out, "deg_in": P.deg_in, "fan_out": P.fan_out, "fan_in": P.fan_in,
            "gs": P.gather_scatter, "sg": P.scatter_gather}
    out = []
    for c in cols:
        if c[0] == "cyc":
            out.append(P.cycle(int(c[1]), int(c[2])))
        elif c[0] == "cycw":
            out.append(P.window_cycle(int(c[1]), int(c[2])))
        else:
            out.append(make[c[0]](int(c[1])))
    return out
