"""bench.py --impl reference: the oracle timed on the host cores prints one
JSON line in the benchmark's format (same metric, unit and workload as the
GPU arm, no host-device bytes), and under a multi-rank launch only rank 0
works and prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(env_extra):
    env = dict(os.environ, **env_extra)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--sample-pairs", "2"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    return p


def test_reference_line():
    sys.path.insert(0, ROOT)
    import bench
    p = run({"WORLD_SIZE": "1", "RANK": "0"})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [x for x in p.stdout.strip().splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] == d["cpu_baseline"]["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_reference_other_ranks_do_nothing():
    p = run({"WORLD_SIZE": "2", "RANK": "1"})
    assert p.returncode == 0
    assert not [x for x in p.stdout.splitlines() if x.startswith("{")]
