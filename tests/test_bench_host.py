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


def _ranks(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        mx = bench.reduce_over_ranks([1.0 + rank, 10.0 - rank, 0.5], "max", "cpu")
        sm = bench.reduce_over_ranks([float(100 * (rank + 1))], "sum", "cpu")
        out.put((rank, mx, sm))
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo_world2():
    """The bench's multi-rank reduction (max of times, sum of samples) on two
    CPU ranks over gloo."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_ranks, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm in got:
        assert mx == [2.0, 10.0, 0.5] and sm == [300.0]


def test_overlap_stats_sweep():
    """Device-interval bookkeeping of the serving section: a batch of one on
    stream 0 over [0, 1] s and a batch of two on stream 1 over [0.5, 2] s:
    busy 2 s, two or more requests in flight over [0.5, 2] (3/4), two
    batches at once over [0.5, 1] (1/4); failed requests (-1) are ignored."""
    sys.path.insert(0, ROOT)
    import bench
    r = [{"stream": 0, "t_gpu_start": 0.0, "t_gpu_end": 1.0, "batch_size": 1},
         {"stream": 1, "t_gpu_start": 0.5, "t_gpu_end": 2.0, "batch_size": 2},
         {"stream": 1, "t_gpu_start": 0.5, "t_gpu_end": 2.0, "batch_size": 2},
         {"stream": -1, "t_gpu_start": -1.0, "t_gpu_end": -1.0, "batch_size": 1}]
    s = bench.overlap_stats(r)
    assert s["batches"] == 2 and abs(s["busy_s"] - 2.0) < 1e-12
    assert abs(s["share_two_or_more_requests"] - 0.75) < 1e-12
    assert abs(s["share_two_or_more_batches"] - 0.25) < 1e-12
