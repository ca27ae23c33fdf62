"""The reference arm of bench.py (the oracle on the host cores) prints the
contract's JSON line without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                         cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_line_keys():
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["unit"] == "terms/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"] == "step_T10000_S21"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["check"] == "generator truth"


def test_reference_large_is_unavailable():
    d = _run("--impl", "reference", "--workload", "large")
    assert d["impl"] == "reference" and "unavailable" in d


def test_both_arms_print_the_same_config():
    """The driver compares the two arms' `config` dicts: both come from one
    function, so they are equal for every workload and world size."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2505_24256_gb300 import workloads as W

    wl = W.step_workload(1002, 50, 5, 20, 21, name="step_T10000_S21")
    d = _run("--impl", "reference", "--steps", "1", "--warmup", "3")
    full = W.batched_step_1e4()
    assert d["config"] == bench.bench_config(full, 1)
    assert bench.bench_config(wl, 2)["parallelism"] == "replicas2"


def test_theoretical_ceiling_arithmetic():
    """mad.hi-issue ceilings: 152 SMs x 32 lanes x 2070 MHz over 4 (MAC) and 6 (chain step)."""
    sys.path.insert(0, ROOT)
    import bench
    mac, chain = bench.theoretical_rates(152, 2070.0)
    assert abs(mac - 152 * 32 * 2070e6 / 4) < 1 and abs(chain - 152 * 32 * 2070e6 / 6) < 1
    r = bench.solve_roofline(10_000, 21, 1.5e-3, {"mac_per_s": 2.0e12, "chain_per_s": 0.8e12, "sms": 152},
                             "no_such_workload")
    ops = 23 * 10_000 ** 2
    assert abs(r["achieved"] - ops / 1.5e-3 / 1e9) < 1e-6
    assert r["frac_theoretical"] < r["frac"] and r["traffic"] is None
