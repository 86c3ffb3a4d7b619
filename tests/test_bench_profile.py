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


def _run_bench(args, env_extra=None):
    import json
    import subprocess
    env = {**os.environ, **(env_extra or {})}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host cores (no GPU) and prints
    one JSON line with the keys the contract names, on bench.py's metric and unit."""
    (line,) = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3", "--ref-sample", "300"])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["steps"] == 1 and line["warmup"] == 3 and line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and "300" in cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    assert _run_bench(["--impl", "reference", "--steps", "1", "--ref-sample", "50"], {"RANK": "1"}) == []
