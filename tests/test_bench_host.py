"""Host-side contract of bench.py that needs no GPU: the reference arm (the
FP64 oracle on the host cores) prints one JSON line on rank 0 and nothing on
the other ranks of a multi-rank launch, which exit 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
        "blobs64", "--steps", "1", "--warmup", "3", "--ref-rows", "0.05"]


def _run(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return subprocess.run(ARGS, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_rank0_prints_contract_line():
    p = _run(0, 2)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "samples/s" and d["value"] > 0
    assert d["n_gpus"] == 2 and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"].startswith("blobs64")


def test_reference_arm_other_ranks_exit_quietly():
    p = _run(1, 2)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
