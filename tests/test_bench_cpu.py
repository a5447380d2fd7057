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
    import time
    t0 = time.perf_counter()
    r = _run({"RANK": "0"}, "--impl", "reference", "--steps", "1", "--warmup", "3")
    wall = time.perf_counter() - t0
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
    # ms_per_step is the wall time a step took: every step fits in the run
    assert (line["steps"] + line["warmup"]) * line["ms_per_step"] <= wall * 1e3
    # the whole-pair time the value stands for is an extrapolation, labelled so
    assert line["extrapolated_ms_per_pair"] > line["ms_per_step"] and "extrapolated" in line["value_basis"]
    full = cb["measured_full_pair_n1024"]
    assert full["seconds"] > 0 and abs(full["pairs_per_s"] * full["seconds"] - 1) < 1e-9


def test_phase_rooflines_arithmetic():
    """Each phase's fraction is its algorithmic work over its time, against
    the peak of the resource that binds it."""
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    n = 1000
    kc = {"square": dict(ms_per_step=2.0, launches=4, work=1e12),          # 4e12 flop in 2 ms
          "score": dict(ms_per_step=1.0, launches=1, work=123.0),          # work from n, not the library
          "project": dict(ms_per_step=0.5, launches=2, work=1e9),
          "apply": dict(ms_per_step=0.0, launches=0, work=0.0),            # absent phases are skipped
          "distance": dict(ms_per_step=4.0, launches=1, work=7.0)}
    pk = {"hbm_gbs": 5000.0, "bf16_tflops_sustained": 1000.0}
    out = bench.phase_rooflines(kc, n, pk, "measured", 100, 2000.0)
    assert set(out) == {"square", "score", "score_tensor", "project", "distance"}
    # the score phase also against the tensor flops the library counts for it
    assert out["score_tensor"]["bound"] == "tensor" and out["score_tensor"]["work_per_pair"] == 123.0
    assert abs(out["score_tensor"]["achieved"] - 123.0 / 1e-3 / 1e12) < 1e-15
    assert out["square"]["bound"] == "tensor" and abs(out["square"]["achieved"] - 2000.0) < 1e-9
    assert abs(out["square"]["frac"] - 2.0) < 1e-12
    assert out["score"]["work_per_pair"] == 8.0 * n * (n - 1)
    assert abs(out["score"]["achieved"] - 8.0 * n * (n - 1) / 1e-3 / 1e9) < 1e-6
    assert out["distance"]["work_per_pair"] == 16.0 * n * n
    alu = 100 * 128 * 2000e6 / 1e12
    assert out["project"]["bound"] == "alu" and abs(out["project"]["peak"] - alu) < 1e-12
    assert abs(out["project"]["achieved"] - 2e9 / 0.5e-3 / 1e12) < 1e-12


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
