"""bench.py's reference arm (the oracle on the host cores) runs without a GPU
and prints one JSON line with the keys the measurement contract names."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = run_bench("--impl", "reference", "--workload", "ci4_64in", "--steps", "1", "--warmup", "0")
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "TCMAC/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_declines_the_packet_workload():
    d = run_bench("--impl", "reference", "--workload", "stream1024", "--steps", "1", "--warmup", "0")
    assert d["impl"] == "reference" and "unavailable" in d


def load_bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_the_timed_output_check_passes_the_oracle_and_flags_one_changed_entry():
    # bench.py compares the last timed step's output with the oracle; here the "output" is
    # the oracle's own result (must pass) and the same with one entry changed (must fail)
    import numpy as np

    import oracle
    from paper_1401_8288_gb300 import synth
    bench = load_bench()
    x = synth.uniform_ci4(64, 6, 20, seed=3)
    good = oracle.correlate(oracle.FMT_CI4, x).astype(np.int32)
    assert bench.oracle_check(good, x, "ci4", [0, 5], 50, seed=1)["exact"]
    for c, pair, comp in ((0, 7, 1), (3, 500, 0)):  # a checked channel; a channel only sampled
        bad = good.copy()
        bad[c, pair, comp] += 1
        r = bench.oracle_check(bad, x, "ci4", [0, 5], 2000, seed=1)
        assert not r["exact"], (c, pair, comp)
    # float input: within 1e-6 of sqrt(V_ii V_jj) passes, a 1e-5 relative error on one entry fails
    y = synth.gaussian_cf32(64, 3, 10, seed=4)
    fgood = oracle.correlate(oracle.FMT_CF32, y).astype(np.float32)
    r = bench.oracle_check(fgood, y, "cf32", [0, 2], 200, seed=2)
    assert r["exact"] and r["max_normalised_error"] < 1e-6
    fbad = fgood.copy()
    fbad[2, 11, 0] += 1e-5 * abs(float(fbad[2, 11, 0])) + 1e-3
    assert not bench.oracle_check(fbad, y, "cf32", [0, 2], 200, seed=2)["exact"]
