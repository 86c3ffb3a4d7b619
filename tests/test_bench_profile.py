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


def test_profile_traffic_only_for_the_captured_code():
    """The headline summary names the code it was captured on; its DRAM bytes are used
    exactly when that is the current code (else the bench line reports null traffic)."""
    import re
    txt = open(bench.PROFILE).read()
    sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]{16})", txt)
    per_shot = re.search(r"dram_bytes_per_shot:\s*([0-9.]+)", txt)
    assert sha and per_shot
    t = bench.profile_traffic(1_000_000)
    if sha.group(1) == bench.kernel_sha():
        assert t == float(per_shot.group(1)) * 1_000_000
        assert 300 < float(per_shot.group(1)) < 500   # the algorithmic 393 B/shot, no re-reads
    else:
        assert t is None
