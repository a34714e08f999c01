"""The bench's reference arm (the oracle timed on the host cores) prints the one
JSON line of the bench contract, with every key the contract names.  CPU only:
the reference arm never touches a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-sample", "150000"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["value"] > 0
    assert d["higher_is_better"] is True and d["config"]["workload"].startswith("scaled:")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["host"]["nproc"] >= 1 and cb["host"]["cpu_model"]
    e = d["e2e"]
    assert (e["value"], e["unit"], e["h2d_bytes_per_step"], e["d2h_bytes_per_step"]) == (d["value"], d["unit"], 0, 0)


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_captures_match_the_kernel_code():
    """The committed DRAM-traffic captures name the kernel sources they were taken on by a
    digest of the code: comment edits keep it, any code edit changes it (and the bench then
    reports no traffic rather than a stale one)."""
    import tempfile
    bench = _bench_module()
    for name in ("expand_kernel_scaled_traffic.json", "expand_kernel_mid_traffic.json"):
        with open(os.path.join(ROOT, "profiles", name)) as f:
            t = json.load(f)
        assert bench.kernel_code_digest(t["kernel_sources"]) == t["kernel_code_sha256"], name
    with tempfile.TemporaryDirectory(dir=ROOT) as d:
        rel = os.path.relpath(os.path.join(d, "k.cuh"), ROOT)
        path = os.path.join(ROOT, rel)
        with open(path, "w") as f:
            f.write("int a = 1;  // one\n\n// a note\nint b = 2;\n")
        base = bench.kernel_code_digest([rel])
        with open(path, "w") as f:
            f.write("int a = 1;  // another note\n// more\nint b = 2;\n\n")
        assert bench.kernel_code_digest([rel]) == base
        with open(path, "w") as f:
            f.write("int a = 1;\nint b = 3;\n")
        assert bench.kernel_code_digest([rel]) != base
