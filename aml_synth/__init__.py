"""Seeded synthetic transaction graphs shaped like the IBM AML datasets.

This package holds input generators only: no pattern arithmetic lives here.
Both the CPU oracle's tests and the CUDA path's tests and benchmark draw their
inputs from it, so neither side depends on the other.
"""
from .gen import (  # noqa: F401
    Graph,
    Motif,
    WORKLOADS,
    capped_zipf_weights,
    generate,
    workload,
    tiny_random,
)
