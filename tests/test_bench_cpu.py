"""bench.py host logic without a GPU: the clock-sample summary that decides whether a timed run saw
throttling, and the reference arm (the CPU oracle on a bounded sample), whose JSON line must
carry the keys of the bench contract."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def sample(sm, smax, hw="Not Active", hw_th="Not Active", sw_th="Not Active", pcap="Not Active"):
    return f"{sm}, {smax}, 900.5, 0x0000000000000000, {hw}, {hw_th}, {sw_th}, {pcap}\n"


def test_clock_summary_median_max_and_reasons():
    lines = [sample(2070, 2070), sample(1995, 2070, pcap="Active"), sample(2040, 2070),
             "garbage line\n", "[N/A], [N/A], [N/A], x, a, b, c, d\n"]
    out = bench.summarize_clocks(lines)
    assert out["sm_mhz"] == 2040 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_every_slowdown_kind():
    lines = [sample(1500, 2070, hw="Active"), sample(1500, 2070, hw_th="Active"), sample(1500, 2070, sw_th="Active")]
    assert bench.summarize_clocks(lines)["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    assert bench.summarize_clocks([])["reasons"] == ["no samples"]


def run_bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          timeout=600, env=e, cwd=ROOT)


def test_reference_arm_json_line():
    r = run_bench("--impl", "reference", "--workload", "random8x32", "--steps", "2", "--warmup", "1")
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 2 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "workload" in line["config"]


def test_reference_arm_other_ranks_exit_quietly():
    r = run_bench("--impl", "reference", "--workload", "random8x32", "--steps", "1", "--warmup", "0",
                  env={"RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_result_errors_of_the_small_workload():
    """The per-path error field: oracle blocks fed back as a snapshot give ~0; a planted error of
    1e-6 in one block of one path shows up as that path's error and only there."""
    import numpy as np

    import oracle
    import synthetic
    s = synthetic.random_device(3, 3, 8, 4)
    eps = 4
    perm = np.arange(4)
    refs = [oracle.solve_g(s, e, surface="eig") for e in range(eps)]
    keys = ("R_diag", "R_upper", "R_lower", "L_diag", "L_upper", "G_diag", "G_upper")
    snap = {k: np.stack([r[k] for r in refs]) for k in keys}
    bad = {k: v.copy() for k, v in snap.items()}
    blk = bad["R_upper"][2, 1]
    bad["R_upper"][2, 1] = blk + 1e-6 * np.linalg.norm(blk) / np.sqrt(blk.size)
    out = bench.result_errors(None, {"fp64": snap, "split_scope0": bad}, None, s, perm, 0, eps, tuple(range(s.nb)))
    assert out["fp64"] <= 1e-14
    assert 0.5e-6 <= out["split_scope0"] <= 2e-6
    assert out["tolerance"] == {"fp64": 1e-10, "split": 1e-8}
