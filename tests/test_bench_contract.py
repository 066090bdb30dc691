"""bench.py's output contract where it needs no GPU: the reference arm (the
oracle timed on the host cores) prints one JSON line with the keys the
benchmark contract names; a rank other than 0 of a multi-rank launch prints
nothing and exits 0; the hash that validates the stored DRAM traffic of the
bulk kernel ignores comments."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=900)


def test_reference_arm_prints_one_contract_line():
    r = _reference({"RANK": "0", "WORLD_SIZE": "1"}, "--steps", "1", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["data"] == "synthetic" and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_other_ranks_exit_quietly():
    r = _reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--steps", "1", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_traffic_hash_ignores_comments():
    sys.path.insert(0, ROOT)
    import bench

    code = "int a; // one\n/* two\n   lines */ int b;\n\n   \nint c;  \n"
    assert bench._code_only(code) == "int a;\n int b;\nint c;"
    assert bench._code_only("x = 1;  // note") == bench._code_only("// header\nx = 1;")


def test_cpu_baseline_times_one_thread_and_every_host_core():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2210_06043_gb300 import workloads as wl

    caps = wl.sweep_capillaries()[:8]
    cb = bench.cpu_baseline(caps, 2e6)
    host = os.cpu_count()
    assert cb["kind"] == "oracle" and cb["host_cores"] == host and cb["cores"] == host
    assert cb["value"] > 0 and cb["one_thread"]["value"] > 0
    full = cb["small_capillary_full_run"]
    assert "2000 steps" in full["what"] and full["mlups"] > 0 and full["marker_updates_per_s"] > 0
