"""The reference arm of bench.py (the oracle timed on the host cores) prints
the one-line JSON contract, and under a multi-rank launch only rank 0 does
any work. Runs on CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env, *args):
    env = dict(os.environ)
    env.update(extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_the_contract_line():
    r = _run({"RANK": "0"}, "--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["metric"] == "graph pairs/s at n=32768" and line["unit"] == "pairs/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3
    assert line["config"]["workload"] == "field_n32768_pair"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"}, "--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_warmup_below_three_is_refused():
    r = _run({}, "--warmup", "2")
    assert r.returncode != 0 and "--warmup must be >= 3" in r.stderr


def test_clock_sampler_parses_nvidia_smi(tmp_path, monkeypatch):
    """The clocks record of a bench line: median SM clock, maximum, and the
    throttle reasons seen active, from nvidia-smi's CSV (a stand-in script
    prints three samples here)."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '1965, 2070, 1200.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active'\n"
                    "echo '2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '2010, 2070, 1150.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    sys.path.insert(0, ROOT)
    try:
        import bench
        s = bench.ClockSampler(0)
        import time
        time.sleep(1.0)
        rec = s.stop()
    finally:
        sys.path.remove(ROOT)
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2010.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
