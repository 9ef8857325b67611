"""bench.py reports a kernel's measured DRAM traffic only while the kernel
sources match the digest the traffic was captured with; the digest covers the
code, not its comments or layout."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_comments_and_layout_do_not_change_the_code():
    a = 'int f(int x) { return x + 1; }  // add one\n'
    b = '/* add\n one */ int  f(int x)\n{\n  return x + 1;\n}\n'
    assert bench.code_tokens(a) == bench.code_tokens(b)


def test_code_and_literals_do_change_it():
    base = bench.code_tokens('int f(int x) { return x + 1; }')
    assert bench.code_tokens('int f(int x) { return x + 2; }') != base
    s1 = bench.code_tokens('const char* s = "a // b"; // c')
    s2 = bench.code_tokens('const char* s = "a // x"; // c')
    assert s1 != s2 and '"a // b"' in s1
    assert bench.code_tokens("char c = '\\''; // q") == "char c = '\\'';"


def test_digest_is_stable_and_sixteen_hex_digits():
    d = bench.kernel_digest()
    assert d == bench.kernel_digest() and len(d) == 16
    int(d, 16)


def test_leg_pass_window_is_the_largest_window_with_leg_columns():
    from paper_2604_12241_b300 import patterns as P
    # hi-large: the 7-day window has FAN columns only; its legs run at 24h
    assert bench.leg_pass_window(P.workload_patterns("hi-large")) == P.DAY
    assert bench.leg_pass_window(P.workload_patterns("hi-small")) == P.WEEK
    assert bench.leg_pass_window([P.fan_out(P.DAY), P.fan_in(P.WEEK)]) == P.WEEK


def test_byte_models_are_finite_or_none():
    import math

    from paper_2604_12241_b300 import patterns as P
    pats = P.workload_patterns("hi-large")
    stats = {"legs": 1000, "front": {2: 10, 3: 20}}
    for k in ("k_assemble", "k_leg_emit", "k_sg_partition", "k_sg_bucket", "k_fan_reduce",
              "k_fan_scan", "k_cyc_level", "k_leg_count", "k_close_range", "k_unknown"):
        b = bench.algorithmic_bytes(k, 100, 90, pats, stats)
        assert b is None or (math.isfinite(b) and b > 0), k
    # hi-large: SG + CYC3..6 accumulators, one GS column, cycle columns
    assert bench.algorithmic_bytes("k_leg_count", 100, 90, pats, stats) == 100 * (48 + 40 + 4)
