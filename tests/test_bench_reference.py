"""The benchmark's reference arm (the FP64 oracle on the host cores) prints
one JSON line with the benchmark's keys; run on the small tube workload, on
the CPU, as a subprocess the way the benchmark is launched."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "tube", "--steps", "20", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 20 and d["warmup"] == 3 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("rigid tube 24x24x64")
    assert d["vs_baseline"] is None and d["data"] == "synthetic"


def test_reference_arm_other_ranks_exit_without_work():
    # under torchrun with N > 1 only rank 0 runs the oracle and prints
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "tube", "--steps", "5", "--warmup", "3", "--gpus", "2"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_launch_count_follows_the_step_graphs():
    # lbm_step takes whole graphs of graph_steps steps, then single-step graphs;
    # a graph's first step (and a single step) issues launches_first_step
    # kernels, its later steps launches_per_step (the band velocities of the
    # next step issued beside the boundary kernels)
    sys.path.insert(0, ROOT)
    import bench
    from types import SimpleNamespace
    info = SimpleNamespace(graph_steps=64, launches_first_step=5, launches_per_step=6)
    assert bench.launches(info, 2000) == 31 * (5 + 63 * 6) + 16 * 5 == 11953
    assert bench.launches(info, 64) == 5 + 63 * 6
    assert bench.launches(info, 10) == 50
    assert bench.launches(SimpleNamespace(graph_steps=8, launches_first_step=5, launches_per_step=5), 203) == 1015
