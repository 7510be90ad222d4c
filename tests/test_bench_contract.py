"""Host-side checks of bench.py: the reference arm's JSON line (the CPU oracle timed on the
host cores), its behaviour on ranks other than 0, the clock summary and the freshness of the
committed DRAM-traffic record.  No GPU is needed."""
import json
import os
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "3"],
                   {"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    r = _run_bench(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"],
                   {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_clock_summary():
    out = "\n".join([
        "1965, 2070, 1010.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2010, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # skipped
        "garbage",                                                                    # skipped
    ])
    c = bench.summarise_clocks(out)
    assert c["sm_mhz"] == 2010 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    c = bench.summarise_clocks("1500, 2070, 1, 0x8, Active, Not Active, Active, Not Active")
    assert c["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.summarise_clocks("")["sm_mhz"] is None


def test_traffic_is_dropped_when_the_kernel_source_changes(tmp_path, monkeypatch):
    """The roofline's `traffic` figure comes from a committed ncu record and is used only while
    the kernel source it was captured from is unchanged (same sha256); otherwise it is null."""
    import hashlib
    src = "paper_1309_5994_gb300/csrc/k_tc.cu"
    with open(os.path.join(ROOT, src), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    rec = {"kernels": {
        "same": {"bytes_per_launch": 123, "source": src, "sha256": sha},
        "changed": {"bytes_per_launch": 456, "source": src, "sha256": "0" * 64},
        "missing": {"bytes_per_launch": 789, "source": "no/such/file.cu", "sha256": sha}}}
    path = tmp_path / "traffic.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    assert bench.load_traffic() == {"same": 123, "changed": None, "missing": None}
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "absent.json"))
    assert bench.load_traffic() == {}
