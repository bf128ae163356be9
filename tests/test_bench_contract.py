"""The reference arm of bench.py (the oracle timed on the host cores, the
one place besides the CPU baseline where the bench runs the oracle) prints
the contract's JSON line: the GPU arm's metric and unit, impl = reference,
a cpu_baseline describing the run, and an e2e entry with no transfers."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    sys.path.insert(0, ROOT)
    import bench

    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "particle-steps/s"
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("config2")


def test_code_digest_ignores_comments_only():
    """The profile summary is tied to the kernel's code by a digest that
    ignores comments and blank lines but not code (string literals kept)."""
    sys.path.insert(0, ROOT)
    import bench

    a = 'int f(int x) {  // one\n  /* two\n lines */ return x + 1;\n}\nconst char* s = "// kept";\n'
    b = '// a header\nint f(int x) {\n\n  return x + 1;   \n}\nconst char* s = "// kept";\n'
    c = 'int f(int x) {\n  return x + 2;\n}\nconst char* s = "// kept";\n'
    d = 'int f(int x) {\n  return x + 1;\n}\nconst char* s = "// changed";\n'
    sa, sb = bench._strip_comments(a), bench._strip_comments(b)
    assert sa.replace(" ", "") == sb.replace(" ", "")
    assert bench._strip_comments(c) != sb and bench._strip_comments(d) != sb
    assert len(bench.code_digest(bench.PROFILE_SOURCES)) == 16
