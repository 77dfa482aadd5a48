"""Benchmark host logic on CPU.  The reference arm (`bench.py --impl reference`)
times the FP64 oracle on the host cores and prints one JSON line with the
metric, unit and config of the measured arm; under a multi-rank launch only
rank 0 prints.  The clock record parses the sampled nvidia-smi lines."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, *args):
    env = dict(os.environ, **(extra_env or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run(None, "--steps", "1", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"] == "lowp_n1e6_128L3"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--steps", "1", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_clock_summary_reports_median_clock_and_active_reasons():
    """The clock record beside each benchmark number: median SM clock under load,
    the maximum, and every throttle reason seen active (samples taken before the
    timed region are skipped)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    cs = bench.ClockSampler(0)
    cs.lines = ["1200, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # before the region
                "2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
                "2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                "2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "garbage line"]
    cs.skip = 1
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    cs.lines = ["1500, 2070, 1000.0, 0x8, Active, Not Active, Active, Not Active"]
    cs.skip = 0
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_serving_span_overlap_summary():
    """The serving overlap record: mean batches in flight over the busy time and the
    share of it with two or more batches in flight, from device-time spans."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod2", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    o = bench.span_overlap([(0.0, 10.0, 0, 2), (5.0, 12.0, 1, 3), (20.0, 25.0, 0, 1)])
    assert o["batches"] == 3 and o["waves_used"] == 2 and o["mean_batch_problems"] == 2.0
    assert abs(o["mean_in_flight"] - 22.0 / 17.0) < 1e-12
    assert abs(o["share_two_or_more"] - 5.0 / 17.0) < 1e-12
    assert bench.span_overlap([]) is None
