"""bench.py's roofline traffic comes from the committed ncu summary only while the kernel code
it was captured on is unchanged: the code hash ignores comments and blank lines but not code."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_hash_ignores_comments_only():
    src = "int f(int x) {\n    return x + 1;   // one more\n}\n"
    same = "// header\n/* block\n   comment */\nint f(int x) {\n\n    return x + 1;\n}\n"
    other = "int f(int x) {\n    return x + 2;   // one more\n}\n"
    assert bench.kernel_code(src) == bench.kernel_code(same)
    assert bench.kernel_code(src) != bench.kernel_code(other)


def test_committed_profile_matches_the_kernel_code():
    """The headline summary names the code it was captured on, and it is the current code,
    so the bench line carries measured DRAM traffic (not null)."""
    txt = open(bench.PROFILE).read()
    assert f"kernel_source_sha256_16: {bench.kernel_sha()}" in txt
    t = bench.profile_traffic(1_000_000)
    assert t is not None and 300e6 < t < 500e6   # 300-500 B/shot: the algorithmic 393 B/shot
