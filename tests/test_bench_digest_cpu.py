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
