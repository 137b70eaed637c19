"""bench.py's reference arm (the oracle on the host cores) on CPU: one JSON line with the
GPU arm's metric, unit and direction, the cpu_baseline and e2e objects, and nothing from
ranks other than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.strip()]


def test_reference_arm_prints_one_line():
    lines = _run({"RANK": "0"})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["metric"].startswith("32^4 SU(3) OR sweep") and d["dtype"] == "f64"
    assert d["config"]["workload"] and d["config"]["lattice"] == [32, 32, 32, 32]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    assert _run({"RANK": "1"}) == []


def test_timed_fix_launch_count():
    # The launch count the bench line reports for its timed gf_fix: 68 kernels for the
    # 20-step call, as ncu's launch list of that call counted them (launches 79-146 of the
    # run summarised under profiles/); 200 and 4000 steps as the bench lines reported.
    import bench
    assert bench.timed_fix_launches(20) == 68
    assert bench.timed_fix_launches(200) == 630
    assert bench.timed_fix_launches(4000) == 12504
    # short budgets: the graph that fits, at most two gated sweeps past the budget
    assert bench.timed_fix_launches(1) == 4 + 3 + 2
    assert bench.timed_fix_launches(3) == 4 + 3 * 4 + 2
