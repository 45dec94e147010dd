"""The benchmark's host-side legs (CPU only): the oracle's standard Newton on
one core and spread over spawned single-threaded processes, and the
`--impl reference` JSON line, and the oracle's Algorithm 1 on a bounded
sample.  Small samples so that they take seconds."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_cpu_reference_one_and_several_processes():
    one = bench.cpu_reference("small", 4)
    assert one["n"] == 4 and one["procs"] == 1 and one["steps"] >= 4 and one["seconds"] > 0
    two = bench.cpu_reference("small", 4, procs=2)
    # two consecutive chunks: each chunk's first parameter starts cold, so the
    # split takes at least as many Newton steps as the warm-started sequence
    assert two["n"] == 4 and two["procs"] == 2 and two["steps"] >= one["steps"]


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "small", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    cores = bench.host_cores()
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["cores"] == cores
    assert d["config"]["sample_params"] == 2 * cores
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["higher_is_better"] is True and d["unit"] == "params/s"


@pytest.mark.parametrize("rank", ["1"])
def test_reference_arm_other_ranks_exit_without_work(rank):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="2", LOCAL_RANK=rank)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "small", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT, env=env)
    assert out.returncode == 0 and not [l for l in out.stdout.splitlines() if l.startswith("{")]


def test_cpu_algorithm1_reaches_the_target():
    # the first parameters of the 80 x 16 grid share nu_f (mu_s runs fastest): one narrow subset
    r = bench.cpu_algorithm1("medium", 4)
    assert r["n"] == 4 and r["max_relres"] <= 1e-6 and r["seconds"] > 0 and r["newton"] >= 1
